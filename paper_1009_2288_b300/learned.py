"""Learned warm start for EPTV (not in the paper): a small U-Net trained on pairs that the
plain method generates predicts, from the back projection of a noisy sinogram, a
warm-start image f0 and a per-pixel edge-weight map w.  Plain EPTV then finishes the
solve from f0, using w for its edge weights during the first iterations
(EPTV_WEIGHTS_PRIOR), and judges the result by its own energy (Eq. 2).

All arithmetic of the network runs in the library's kernels (eptv_unet_*); this module
only allocates tensors and sequences the layer calls.

Network (BF16 activations, NHWC, FP32 master weights):
  enc1  conv 1->16, conv 16->16            (full resolution; the input is zero-padded to
                                           16 channels so that every 3x3 conv runs on
                                           the tensor-core kernel)
  enc2  pool, conv 16->32, conv 32->32     (1/2)
  mid   pool, conv 32->64, conv 64->64     (1/4)
  dec2  up, [64 | skip 32] conv 96->32, conv 32->32
  dec1  up, [32 | skip 16] conv 48->16, conv 16->16
  head  1x1 16->2: f0 = o0 * F_SCALE, w = sigmoid(o1)
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import List, Optional

import numpy as np

from . import eptv as E
from . import inputs as I

F_SCALE = 0.02                      # 1/mm per unit of the network's image channel
CONVS = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64),
         (96, 32), (32, 32), (48, 16), (16, 16)]
REAL_CIN0 = 1                       # channels of the network input before padding


class UNet:
    def __init__(self, seed: int = 0, device: str = "cuda"):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        rng = np.random.Generator(np.random.PCG64(seed))
        self.w, self.b = [], []
        for k, (ci, co) in enumerate(CONVS):
            real_ci = REAL_CIN0 if k == 0 else ci
            wk = np.zeros((co, 9, ci), dtype=np.float32)
            wk[:, :, :real_ci] = (rng.standard_normal((co, real_ci, 3, 3)) *
                                  math.sqrt(2.0 / (9 * real_ci))).transpose(0, 2, 3, 1).reshape(co, 9, real_ci)
            self.w.append(torch.tensor(wk, device=self.dev))
            self.b.append(torch.zeros(co, device=self.dev))
        self.hw = torch.tensor(rng.standard_normal((2, 16)) * math.sqrt(1.0 / 16), dtype=torch.float32,
                               device=self.dev)
        self.hb = torch.zeros(2, device=self.dev)
        self.params = [*self.w, *self.b, self.hw, self.hb]
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0
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

    def sync_weights(self):
        for k, (ci, co) in enumerate(CONVS):
            E.eptv_unet_weights_to_bf16(self.w[k], co, ci, self.wf[k], self.wb[k])

    # -- buffers --------------------------------------------------------------------
    def _alloc(self, n, H, W):
        if self.shape == (n, H, W):
            return
        assert H % 4 == 0 and W % 4 == 0
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
    def forward(self, x):
        """x: [n, H, W] float32 (normalised input).  Returns (f0, w) views [n, H, W]."""
        n, H, W = x.shape
        self._alloc(n, H, W)
        A, wf, b = self.A, self.wf, self.b
        A["inp"][..., 0] = x.to(self.torch.bfloat16)          # channel 0; others stay 0
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
        E.eptv_unet_head(A["d1"], self.hw, self.hb, f0=self.f0, w=self.wmap)
        return self.f0, self.wmap

    def backward(self, ft, wt):
        """Gradients of mean((f0 - ft)^2) + mean((w - wt)^2) (ft in network units) for the
        last forward pass; returns the loss."""
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


# ------------------------------------------------------------------ data and targets

def rasterize_gpu(ellipses, g: I.FanGeometry, device, ss: int = 2):
    """Phantom on the GPU (training data only): ss x ss sub-pixel samples per pixel."""
    import torch
    x0, y0 = -g.nx * g.dx / 2.0, -g.ny * g.dy / 2.0
    off = (torch.arange(ss, device=device, dtype=torch.float64) + 0.5) / ss
    xs = x0 + (torch.arange(g.nx, device=device, dtype=torch.float64)[:, None] + off[None, :]).reshape(-1) * g.dx
    ys = y0 + (torch.arange(g.ny, device=device, dtype=torch.float64)[:, None] + off[None, :]).reshape(-1) * g.dy
    Y, X = torch.meshgrid(ys, xs, indexing="ij")
    img = torch.zeros_like(X)
    for el in ellipses:
        c, s = math.cos(el.phi), math.sin(el.phi)
        u = (X - el.cx) * c + (Y - el.cy) * s
        w = -(X - el.cx) * s + (Y - el.cy) * c
        img = torch.where((u / el.a) ** 2 + (w / el.b) ** 2 < 1.0, torch.full_like(img, el.value), img)
    return img.reshape(g.ny, ss, g.nx, ss).mean(dim=(1, 3)).float()


def c4_ellipses(seed: int, g: I.FanGeometry):
    """The ellipse set of the learned workload's phantom with this seed (see inputs.make_c4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = g.nx * g.dx / 2.0
    els = I.random_ellipses(rng, R, 29)
    for k in range(8):
        ang = 2 * np.pi * k / 8
        I.add_insert(els, 120.0 * math.cos(ang), 120.0 * math.sin(ang), 0.5 * (2.0 + 13.0 * k / 7.0),
                     rng.choice([-1.0, 1.0]) * rng.uniform(0.003, 0.01))
    return els


@dataclasses.dataclass
class PairSet:
    x: object          # [N, H, W] normalised back projections
    ft: object         # [N, H, W] plain-EPTV images / F_SCALE
    wt: object         # [N, H, W] per-pixel edge weights of the plain solve
    scale: object      # [N] input normalisation factors


def normalise_input(geo: E.Geometry, y_dev, out=None):
    """Back projection P^T y of a sinogram, divided by its mean (returns image, factor)."""
    import torch
    g = geo.g
    bp = out if out is not None else torch.empty(g.n_pix, device=y_dev.device)
    E.eptv_backproject(geo, y_dev, bp)
    s = bp.mean().clamp_min(1e-12)
    return (bp / s).reshape(g.ny, g.nx), s


def edge_weight_map(geo: E.Geometry, p: I.EptvParams, f_dev):
    """Per-pixel mean of the edge weights (Eq. 5) of a (P2) solve started at f: the
    weights the plain method settles on around each pixel."""
    import torch
    g = geo.g
    wts = torch.empty(2 * (g.nx + 1) * (g.ny + 1), device=f_dev.device)
    out = torch.empty_like(f_dev)
    E.eptv_tv_step(geo, p, f_dev, out, weights=wts)
    w3 = wts.reshape(2, g.ny + 1, g.nx + 1)
    wx = w3[0, :g.ny, :]              # x half-edges: [ny][nx+1]
    wy = w3[1, :, :g.nx]              # y half-edges: [ny+1][nx]
    return 0.25 * (wx[:, :-1] + wx[:, 1:] + wy[:-1, :] + wy[1:, :])


def make_pairs(seeds: List[int], p: I.EptvParams, device="cuda", batch: int = 64, log=print) -> PairSet:
    """Training pairs generated by the plain method: phantom (GPU raster), sinogram P f
    (library projector), Poisson noise, plain EPTV (batched) -> targets."""
    import torch
    g = I.ge_geometry(256, 1.6, 30)
    n = len(seeds)
    X = torch.empty(n, g.ny, g.nx, device=device)
    FT = torch.empty_like(X)
    WT = torch.empty_like(X)
    SC = torch.empty(n, device=device)
    gen = torch.Generator(device=device)
    t0 = time.time()
    geos = [E.Geometry(g) for _ in range(min(batch, n))]
    for b0 in range(0, n, batch):
        ids = list(range(b0, min(n, b0 + batch)))
        ys, fs = [], []
        for j, i in enumerate(ids):
            f = rasterize_gpu(c4_ellipses(seeds[i], g), g, device).reshape(-1).contiguous()
            pr = torch.empty(g.n_rays, device=device)
            E.eptv_project(geos[j], f, pr)
            gen.manual_seed(int(seeds[i]))
            counts = torch.poisson(5e4 * torch.exp(-pr.double()), generator=gen)
            y = torch.log(5e4 / counts.clamp_min(1.0)).float().contiguous()
            ys.append(y)
            fs.append(torch.zeros(g.n_pix, device=device))
            X[i], SC[i] = normalise_input(geos[j], y)
        E.eptv_reconstruct_batched(geos[:len(ids)], p, ys, fs, report=False)
        for j, i in enumerate(ids):
            FT[i] = fs[j].reshape(g.ny, g.nx) / F_SCALE
            WT[i] = edge_weight_map(geos[j], p, fs[j])
        log(f"pairs {ids[-1] + 1}/{n}  {time.time() - t0:.1f}s")
    return PairSet(X, FT, WT, SC)


def train(net: UNet, pairs: PairSet, epochs: int = 3, batch: int = 16, lr: float = 2e-3, seed: int = 0,
          log=print):
    import torch
    n = pairs.x.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    losses = []
    for ep in range(epochs):
        order = rng.permutation(n)
        for b0 in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(order[b0:b0 + batch], device=pairs.x.device)
            net.forward(pairs.x[idx])
            loss = net.backward(pairs.ft[idx].contiguous(), pairs.wt[idx].contiguous())
            net.adam_step(lr)
            losses.append(loss)
        log(f"epoch {ep}: loss {float(losses[-1].item()):.5f}")
    return [float(l.item()) for l in losses]


def warm_start(net: UNet, geo: E.Geometry, y_dev):
    """(f0 [1/mm], per-pixel weight prior) for one sinogram."""
    import torch
    x, _ = normalise_input(geo, y_dev)
    f0, w = net.forward(x[None])
    return (f0[0] * F_SCALE).reshape(-1).clone(), w[0].reshape(-1).clamp(1e-3, 1.0).clone()
