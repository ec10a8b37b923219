"""Learned warm start for EPTV (not in the paper).

A small U-Net, trained on pairs that the plain method generates, predicts a warm-start image
f0 and a per-pixel edge-weight map w for a noisy sinogram y.  Plain EPTV then finishes the
solve from f0 (f^(0) = f0 instead of 0 in the outer loop of Sec. 2.2) and judges the result
by its own reported energy (Eq. 2); with k_w > 0 the first k_w outer iterations take their
edge weights from w (EPTV_WEIGHTS_PRIOR) instead of Eq. (5).

Network input (two channels, zero-padded to 16 so that every 3x3 conv runs on the tensor-core
kernel):
  channel 0  the back projection P^T y, times a scale fixed from the training set
  channel 1  the base image u_M = CGLS_M(0) (App. I, M = M_BASE iterations from zero),
             in units of F_SCALE
The network predicts the residual of the plain solution on that base:
  f0 = max(u_M + F_SCALE * o0, 0),   w = sigmoid(o1).
A 3-level U-Net sees about 45 pixels around each output; the blur of P^T (about 1/r) spans
the whole image, so the base image, which the projector/backprojector pair makes in well
under a millisecond, carries the global part and the network learns the local one.

Every step of the serving path runs in the library (eptv_backproject, eptv_cgls,
eptv_unet_pack_input, eptv_unet_conv3x3 / pooling / upsampling, eptv_unet_head); this module
allocates tensors and sequences the calls.  Training data are synthesised on the GPU with
torch (the same exact line integrals of the overwrite-painted ellipse phantom as the host
generator in inputs.py, Poisson noise from torch's generator), and their targets come from
the library's own plain EPTV (batched).

Network (BF16 activations, NHWC, FP32 master weights):
  enc1  conv 16->16 (2 real input channels), conv 16->16      full resolution -> skip 1
  enc2  pool, conv 16->32, conv 32->32                        1/2             -> skip 2
  mid   pool, conv 32->64, conv 64->64                        1/4
  dec2  up, [64 | skip 32] conv 96->32, conv 32->32
  dec1  up, [32 | skip 16] conv 48->16, conv 16->16
  head  1x1 16->2
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import List, Optional, Sequence

import numpy as np

from . import eptv as E
from . import inputs as I

F_SCALE = 0.02                      # 1/mm per unit of the network's image channels
N_IN = 2                            # real input channels
M_BASE = 10                         # CGLS iterations of the base image
CONVS = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64),
         (96, 32), (32, 32), (48, 16), (16, 16)]


class UNet:
    def __init__(self, seed: int = 0, device: str = "cuda", n_in: int = N_IN):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        rng = np.random.Generator(np.random.PCG64(seed))
        self.w, self.b = [], []
        for k, (ci, co) in enumerate(CONVS):
            real_ci = n_in if k == 0 else ci
            wk = np.zeros((co, 9, ci), dtype=np.float32)
            wk[:, :, :real_ci] = (rng.standard_normal((co, real_ci, 3, 3)) *
                                  math.sqrt(2.0 / (9 * real_ci))).transpose(0, 2, 3, 1).reshape(co, 9, real_ci)
            self.w.append(torch.tensor(wk).to(self.dev))
            self.b.append(torch.zeros(co, device=self.dev))
        self.hw = torch.tensor(rng.standard_normal((2, 16)) * math.sqrt(1.0 / 16),
                               dtype=torch.float32).to(self.dev)
        self.hb = torch.zeros(2, device=self.dev)
        self.params = [*self.w, *self.b, self.hw, self.hb]
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0
        self.bp_scale = 1.0          # channel-0 scale, set from the training set
        self.wf = [torch.empty(co, 9, ci, dtype=torch.bfloat16, device=self.dev) for ci, co in CONVS]
        self.wb = [torch.empty(ci, 9, co, dtype=torch.bfloat16, device=self.dev) for ci, co in CONVS]
        self.shape = None
        self.sync_weights()

    # -- parameters -----------------------------------------------------------------
    def set_from_oracle_layout(self, params):
        """Load weights given as [co][ci][3][3] / [co] lists (head last: [2][16], [2])."""
        torch = self.torch
        for k, (W, b) in enumerate(params[:len(CONVS)]):
            co, ci = W.shape[:2]
            wk = np.zeros((co, 9, CONVS[k][0]), dtype=np.float32)
            wk[:, :, :ci] = np.asarray(W).transpose(0, 2, 3, 1).reshape(co, 9, ci)
            self.w[k].copy_(torch.tensor(wk))
            self.b[k].copy_(torch.tensor(np.asarray(b, dtype=np.float32)))
        self.hw.copy_(torch.tensor(np.asarray(params[-1][0], dtype=np.float32)))
        self.hb.copy_(torch.tensor(np.asarray(params[-1][1], dtype=np.float32)))
        self.sync_weights()

    def state(self) -> dict:
        """Parameters and input scale as numpy arrays (for saving)."""
        out = {f"p{k}": p.detach().cpu().numpy() for k, p in enumerate(self.params)}
        out["bp_scale"] = np.array(self.bp_scale)
        return out

    def load_state(self, st: dict):
        torch = self.torch
        for k, p in enumerate(self.params):
            p.copy_(torch.tensor(st[f"p{k}"]))
        self.bp_scale = float(st["bp_scale"])
        self.sync_weights()

    def sync_weights(self):
        for k, (ci, co) in enumerate(CONVS):
            E.eptv_unet_weights_to_bf16(self.w[k], co, ci, self.wf[k], self.wb[k])

    # -- buffers --------------------------------------------------------------------
    def _alloc(self, n, H, W):
        if self.shape == (n, H, W):
            return
        if H % 4 or W % 4:
            raise ValueError("image sides must be multiples of 4 (two 2x2 poolings)")
        torch = self.torch
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        H2, W2, H4, W4 = H // 2, W // 2, H // 4, W // 4
        z = lambda h, w, c: torch.zeros(n, h, w, c, **bf)
        self.A = dict(inp=z(H, W, 16), a0=z(H, W, 16), cat1=z(H, W, 48), p1=z(H2, W2, 16),
                      a2=z(H2, W2, 32), cat2=z(H2, W2, 96), p2=z(H4, W4, 32), a4=z(H4, W4, 64),
                      bt=z(H4, W4, 64), a6=z(H2, W2, 32), d2=z(H2, W2, 32), a8=z(H, W, 16),
                      d1=z(H, W, 16))
        self.G = dict(dd1=z(H, W, 16), da8=z(H, W, 16), dcat1=z(H, W, 48), dd2=z(H2, W2, 32),
                      da6=z(H2, W2, 32), dcat2=z(H2, W2, 96), dbt=z(H4, W4, 64), da4=z(H4, W4, 64),
                      dp2=z(H4, W4, 32), da2=z(H2, W2, 32), dp1=z(H2, W2, 16), da0=z(H, W, 16))
        self.f0 = torch.empty(n, H, W, device=self.dev)
        self.wmap = torch.empty(n, H, W, device=self.dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.shape = (n, H, W)

    # -- forward / backward ---------------------------------------------------------
    def forward(self, bp, base, compose: bool = False, f_out=None, w_out=None):
        """bp, base: FP32 [n, H, W] (P^T y and the base image, 1/mm).  Packs the input and
        runs the network.  compose=False (training): f0 = o0, the residual in F_SCALE units.
        compose=True: f0 = max(base + F_SCALE o0, 0) in 1/mm.  Returns (f0, w), FP32
        [n, H, W] (or the given output buffers)."""
        n, H, W = bp.shape
        self._alloc(n, H, W)
        A, wf, b = self.A, self.wf, self.b
        E.eptv_unet_pack_input(bp.reshape(-1), self.bp_scale, base.reshape(-1), 1.0 / F_SCALE, A["inp"])
        conv = E.eptv_unet_conv3x3
        conv(A["inp"], 0, 16, wf[0], b[0], 16, A["a0"], 0, True)
        conv(A["a0"], 0, 16, wf[1], b[1], 16, A["cat1"], 32, True)       # e1 -> skip slot
        E.eptv_unet_maxpool2(A["cat1"], 32, 16, A["p1"], 0)
        conv(A["p1"], 0, 16, wf[2], b[2], 32, A["a2"], 0, True)
        conv(A["a2"], 0, 32, wf[3], b[3], 32, A["cat2"], 64, True)       # e2 -> skip slot
        E.eptv_unet_maxpool2(A["cat2"], 64, 32, A["p2"], 0)
        conv(A["p2"], 0, 32, wf[4], b[4], 64, A["a4"], 0, True)
        conv(A["a4"], 0, 64, wf[5], b[5], 64, A["bt"], 0, True)
        E.eptv_unet_upsample2(A["bt"], 0, 64, A["cat2"], 0)
        conv(A["cat2"], 0, 96, wf[6], b[6], 32, A["a6"], 0, True)
        conv(A["a6"], 0, 32, wf[7], b[7], 32, A["d2"], 0, True)
        E.eptv_unet_upsample2(A["d2"], 0, 32, A["cat1"], 0)
        conv(A["cat1"], 0, 48, wf[8], b[8], 16, A["a8"], 0, True)
        conv(A["a8"], 0, 16, wf[9], b[9], 16, A["d1"], 0, True)
        f0 = self.f0 if f_out is None else f_out
        w = self.wmap if w_out is None else w_out
        E.eptv_unet_head(A["d1"], self.hw, self.hb, f0=f0, w=w,
                         base=base.reshape(-1) if compose else None, f_scale=F_SCALE)
        return f0, w

    def backward(self, ft, wt):
        """Gradients of mean((o0 - ft)^2) + mean((w - wt)^2) for the last forward pass
        (ft: residual target in F_SCALE units); returns the loss (device scalar)."""
        A, G, wb = self.A, self.G, self.wb
        for g in self.grads:
            g.zero_()
        self.loss.zero_()
        nw = len(CONVS)
        dW, dB = self.grads[:nw], self.grads[nw:2 * nw]
        dhw, dhb = self.grads[2 * nw], self.grads[2 * nw + 1]
        E.eptv_unet_head(A["d1"], self.hw, self.hb, ft=ft, wt=wt, dx=G["dd1"], dhw=dhw, dhb=dhb,
                         loss=self.loss)
        conv, wg, rb = E.eptv_unet_conv3x3, E.eptv_unet_conv3x3_wgrad, E.eptv_unet_relu_bwd

        def layer(k, x, x_off, a, a_off, dy, dy_off, dx, dx_off):
            ci, co = CONVS[k]
            rb(a, a_off, dy, dy_off, dy, dy_off, co)                      # through the ReLU
            wg(x, x_off, ci, dy, dy_off, co, dW[k], dB[k])
            if dx is not None:
                conv(dy, dy_off, co, wb[k], None, ci, dx, dx_off, False)  # data gradient

        layer(9, A["a8"], 0, A["d1"], 0, G["dd1"], 0, G["da8"], 0)
        layer(8, A["cat1"], 0, A["a8"], 0, G["da8"], 0, G["dcat1"], 0)
        E.eptv_unet_upsample2_bwd(G["dcat1"], 0, 32, G["dd2"], 0)
        layer(7, A["a6"], 0, A["d2"], 0, G["dd2"], 0, G["da6"], 0)
        layer(6, A["cat2"], 0, A["a6"], 0, G["da6"], 0, G["dcat2"], 0)
        E.eptv_unet_upsample2_bwd(G["dcat2"], 0, 64, G["dbt"], 0)
        layer(5, A["a4"], 0, A["bt"], 0, G["dbt"], 0, G["da4"], 0)
        layer(4, A["p2"], 0, A["a4"], 0, G["da4"], 0, G["dp2"], 0)
        E.eptv_unet_maxpool2_bwd(A["cat2"], 64, 32, G["dp2"], 0, G["dcat2"], 64, True)
        layer(3, A["a2"], 0, A["cat2"], 64, G["dcat2"], 64, G["da2"], 0)
        layer(2, A["p1"], 0, A["a2"], 0, G["da2"], 0, G["dp1"], 0)
        E.eptv_unet_maxpool2_bwd(A["cat1"], 32, 16, G["dp1"], 0, G["dcat1"], 32, True)
        layer(1, A["a0"], 0, A["cat1"], 32, G["dcat1"], 32, G["da0"], 0)
        layer(0, A["inp"], 0, A["a0"], 0, G["da0"], 0, None, 0)
        return self.loss

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        for p, g, m, v in zip(self.params, self.grads, self.m, self.v):
            E.eptv_unet_adam(p, g, m, v, lr, beta1, beta2, eps, self.step_count)
        self.sync_weights()


# ------------------------------------------------------------------ serving

class WarmStart:
    """Warm start for sinograms of one geometry: P^T y, u_M = CGLS_M(0), the network,
    f0 = max(u_M + F_SCALE o0, 0) and w, written straight into the caller's buffers."""

    def __init__(self, net: UNet, geo: E.Geometry):
        import torch
        g = geo.g
        self.net, self.geo = net, geo
        self.bp = torch.empty(g.n_pix, device=net.dev)
        self.base = torch.empty(g.n_pix, device=net.dev)
        self.hw = (g.ny, g.nx)
        net._alloc(1, g.ny, g.nx)

    def __call__(self, y, f_out, w_out=None):
        ny, nx = self.hw
        E.eptv_backproject(self.geo, y, self.bp)
        self.base.zero_()
        E.eptv_cgls(self.geo, M_BASE, y, self.base)
        self.net.forward(self.bp.view(1, ny, nx), self.base.view(1, ny, nx), compose=True,
                         f_out=f_out, w_out=w_out)
        return f_out


def solve_learned(warm: WarmStart, p: I.EptvParams, y, f, w=None, k_w: int = 0):
    """Learned warm start, then plain EPTV (p.n_outer iterations) from it; with k_w > 0 the
    first k_w outer iterations use the network's edge weights (w: FP32 [n_pix] buffer)."""
    import torch
    if k_w > 0 and w is None:
        w = torch.empty_like(f)
    warm(y, f, w if k_w > 0 else None)
    if k_w > 0:
        q = dataclasses.replace(p, weights_mode=2, prior_iters=k_w)
        return E.eptv_reconstruct(warm.geo, q, y, f, wprior=w)
    return E.eptv_reconstruct(warm.geo, p, y, f)


# ------------------------------------------------------------------ training data

def c4_ellipses(seed: int, g: I.FanGeometry):
    """The ellipse set that inputs.make_c4 draws for this seed (same generator, same order)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = g.nx * g.dx / 2.0
    els = I.random_ellipses(rng, R, 29)
    for k in range(8):
        ang = 2 * np.pi * k / 8
        I.add_insert(els, 120.0 * math.cos(ang), 120.0 * math.sin(ang), 0.5 * (2.0 + 13.0 * k / 7.0),
                     rng.choice([-1.0, 1.0]) * rng.uniform(0.003, 0.01))
    return els


class RaySet:
    """The rays of a geometry on the device (FP64), for exact phantom line integrals."""

    def __init__(self, g: I.FanGeometry, device):
        import torch
        sx, sy, ux, uy = I.fan_rays(g)
        self.t = [torch.tensor(a, dtype=torch.float64, device=device) for a in (sx, sy, ux, uy)]


def line_integrals_gpu(ellipses: Sequence[I.Ellipse], rays: RaySet):
    """Exact line integrals of the overwrite-painted ellipse phantom (the definition of
    inputs.line_integrals): each ray's chords cut it into intervals; an interval carries the
    value of the last ellipse that covers its midpoint.  FP64 [n_rays]."""
    import torch
    sx, sy, ux, uy = rays.t
    Ne = len(ellipses)
    dev = sx.device
    el = torch.tensor([[e.cx, e.cy, e.a, e.b, e.phi, e.value] for e in ellipses], dtype=torch.float64,
                      device=dev)
    cx, cy, a, b, phi = (el[:, k][None, :] for k in range(5))
    c, s = torch.cos(phi), torch.sin(phi)
    qx, qy = sx[:, None] - cx, sy[:, None] - cy
    qu, qw = qx * c + qy * s, -qx * s + qy * c
    eu, ew = ux[:, None] * c + uy[:, None] * s, -ux[:, None] * s + uy[:, None] * c
    A = eu * eu / a ** 2 + ew * ew / b ** 2
    B = 2.0 * (qu * eu / a ** 2 + qw * ew / b ** 2)
    C = qu * qu / a ** 2 + qw * qw / b ** 2 - 1.0
    disc = B * B - 4.0 * A * C
    ok = disc > 0
    sq = torch.sqrt(torch.where(ok, disc, torch.zeros_like(disc)))
    nan = torch.full_like(disc, float("nan"))
    t1 = torch.where(ok, (-B - sq) / (2 * A), nan)
    t2 = torch.where(ok, (-B + sq) / (2 * A), nan)
    pts, _ = torch.sort(torch.cat([t1, t2], dim=1), dim=1)          # NaN sort last
    lo, hi = pts[:, :-1], pts[:, 1:]
    mid = 0.5 * (lo + hi)
    cov = (t1[:, None, :] < mid[:, :, None]) & (mid[:, :, None] < t2[:, None, :])
    idx = torch.arange(Ne, device=dev)[None, None, :]
    top = torch.where(cov, idx, torch.full_like(idx, -1)).amax(dim=2)
    vals = torch.cat([el[:, 5], torch.zeros(1, dtype=torch.float64, device=dev)])
    v = vals[torch.where(top >= 0, top, torch.full_like(top, Ne))]
    seg = torch.where(torch.isfinite(lo) & torch.isfinite(hi), hi - lo, torch.zeros_like(lo))
    return (torch.where(top >= 0, v, torch.zeros_like(v)) * seg).sum(dim=1)


def c4_sinogram_gpu(seed: int, g: I.FanGeometry, rays: RaySet, i0: float = 5e4, gen=None):
    """Noisy sinogram of the learned workload's phantom for this seed, on the device:
    Poisson counts ~ I0 exp(-p) (torch generator seeded with the seed), y = ln(I0 / max(c, 1))."""
    import torch
    p = line_integrals_gpu(c4_ellipses(seed, g), rays)
    if gen is None:
        gen = torch.Generator(device=p.device)
    gen.manual_seed(int(seed))
    counts = torch.poisson(i0 * torch.exp(-p), generator=gen)
    return torch.log(i0 / counts.clamp_min(1.0)).float().contiguous()


@dataclasses.dataclass
class PairSet:
    bp: object         # [N, H, W] P^T y
    base: object       # [N, H, W] u_M = CGLS_M(0), 1/mm
    res: object        # [N, H, W] (plain-EPTV image - base) / F_SCALE
    wt: object         # [N, H, W] per-pixel edge weights of the plain solve


def edge_weight_map(geo: E.Geometry, p: I.EptvParams, f_dev):
    """Per-pixel mean of the Eq. (5) weights of the four half-edges around each pixel, for a
    (P2) solve started at f: the weights the plain method settles on there."""
    import torch
    g = geo.g
    wts = torch.empty(2 * (g.nx + 1) * (g.ny + 1), device=f_dev.device)
    out = torch.empty_like(f_dev)
    E.eptv_tv_step(geo, p, f_dev, out, weights=wts)
    w3 = wts.reshape(2, g.ny + 1, g.nx + 1)
    wx = w3[0, :g.ny, :]              # x half-edges: [ny][nx+1]
    wy = w3[1, :, :g.nx]              # y half-edges: [ny+1][nx]
    return 0.25 * (wx[:, :-1] + wx[:, 1:] + wy[:-1, :] + wy[1:, :])


def make_pairs(seeds: Sequence[int], p: I.EptvParams, device="cuda", batch: int = 64,
               g: Optional[I.FanGeometry] = None, log=None) -> PairSet:
    """Training pairs of the learned workload (256^2 at 1.6 mm, 30 views x 888 bins,
    I0 = 5e4): GPU-synthesised noisy sinogram -> inputs (P^T y, CGLS_M(0)) and targets
    (plain EPTV after p.n_outer iterations, batched; its edge-weight map)."""
    import torch
    g = g or I.ge_geometry(256, 1.6, 30)
    n = len(seeds)
    rays = RaySet(g, device)
    shape = (n, g.ny, g.nx)
    BP, BASE, RES, WT = (torch.empty(shape, device=device) for _ in range(4))
    gen = torch.Generator(device=device)
    t0 = time.time()
    geos = [E.Geometry(g) for _ in range(min(batch, n))]
    E.eptv_autotune_batched(geos)
    for b0 in range(0, n, batch):
        ids = list(range(b0, min(n, b0 + batch)))
        ys, fs = [], []
        for j, i in enumerate(ids):
            y = c4_sinogram_gpu(seeds[i], g, rays, gen=gen)
            ys.append(y)
            fs.append(torch.zeros(g.n_pix, device=device))
            E.eptv_backproject(geos[j], y, BP[i].view(-1))
            BASE[i].zero_()
            E.eptv_cgls(geos[j], M_BASE, y, BASE[i].view(-1))
        E.eptv_reconstruct_batched(geos[:len(ids)], p, ys, fs, report=False)
        for j, i in enumerate(ids):
            RES[i] = (fs[j].view(g.ny, g.nx) - BASE[i]) / F_SCALE
            WT[i] = edge_weight_map(geos[j], p, fs[j])
        if log:
            log(f"pairs {ids[-1] + 1}/{n}  {time.time() - t0:.1f}s")
    return PairSet(BP, BASE, RES, WT)


def train(net: UNet, pairs: PairSet, epochs: int = 40, batch: int = 16, lr: float = 2e-3,
          lr_min: float = 1e-5, seed: int = 0, log=None) -> List[float]:
    """Adam with a cosine learning-rate schedule over shuffled mini-batches; returns the
    loss of every step (synchronises once at the end)."""
    import torch
    n = pairs.bp.shape[0]
    net.bp_scale = float(1.0 / pairs.bp.mean().clamp_min(1e-12).item())
    rng = np.random.Generator(np.random.PCG64(seed))
    steps = epochs * (n // batch)
    losses, k = [], 0
    for ep in range(epochs):
        order = rng.permutation(n)
        for b0 in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(order[b0:b0 + batch], device=pairs.bp.device)
            net.forward(pairs.bp[idx], pairs.base[idx])
            loss = net.backward(pairs.res[idx].contiguous(), pairs.wt[idx].contiguous())
            net.adam_step(lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * k / steps)))
            losses.append(loss.clone())
            k += 1
        if log:
            log(f"epoch {ep}: loss {float(losses[-1].item()):.5f}")
    return [float(l.item()) for l in losses]


# ------------------------------------------------------------------ judging by the energy

def first_reach(energies: Sequence[float], target: float, window: int = 5, rtol: float = 1e-3):
    """First k (1-based) whose mean reported energy over iterations k-window+1..k is within
    rtol of target (or below); None if there is none.  The reported energy (Eq. 2) swings
    from one outer iteration to the next, hence the window."""
    for k in range(window, len(energies) + 1):
        if sum(energies[k - window:k]) / window <= target * (1.0 + rtol):
            return k
    return None


def iterations_to_energy(geo: E.Geometry, p: I.EptvParams, y, f, target: float, sigma_ref: float,
                         n_max: int, wprior=None, k_w: int = 0):
    """Runs plain EPTV from the content of f one outer iteration at a time (the step size
    carried over), with E_report(f; sigma_ref) after each; returns (k, energies), k as in
    first_reach (None if n_max iterations do not reach the target)."""
    t_prev = p.t_init_eff
    es = []
    for k in range(1, n_max + 1):
        prior = k <= k_w
        q = dataclasses.replace(p, n_outer=1, t_init=t_prev, weights_mode=2 if prior else p.weights_mode,
                                prior_iters=1 if prior else 0)
        rep = E.eptv_reconstruct(geo, q, y, f, wprior=wprior if prior else None)
        t_prev = rep.t_prev
        es.append(E.eptv_report_energy(geo, p, sigma_ref, f, y))
        k_hit = first_reach(es, target)
        if k_hit is not None:
            return k_hit, es
    return None, es
