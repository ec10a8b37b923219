"""Cone-beam inputs on the device (the full-size scan has 23.6 M rays, too many for the host
generator): exact line integrals of the overwrite-painted ellipsoid phantom with torch, the
same definition as inputs.line_integrals3, Poisson noise from torch's generator.  Input
synthesis only; the reconstruction itself runs in the library (eptv3_* in eptv.py)."""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

from . import inputs as I


def rays_gpu(g: I.ConeGeometry, view: int, device):
    """Source and unit directions (FP64) of the rays of one view, ray order iv, iu."""
    import torch
    th = float(g.view_angles()[view])
    c, s = math.cos(th), math.sin(th)
    u = (torch.arange(g.nu, device=device, dtype=torch.float64) - (g.nu - 1) / 2.0 + g.u_off) * g.du
    w = (torch.arange(g.nv, device=device, dtype=torch.float64) - (g.nv - 1) / 2.0 + g.v_off) * g.dv
    W, U = torch.meshgrid(w, u, indexing="ij")
    dx = -g.sdd * c - U * s
    dy = -g.sdd * s + U * c
    dz = W
    n = torch.sqrt(dx * dx + dy * dy + dz * dz)
    return (g.sid * c, g.sid * s, 0.0), (dx / n).reshape(-1), (dy / n).reshape(-1), (dz / n).reshape(-1)


def line_integrals3_gpu(ellipsoids: Sequence[I.Ellipsoid], src, ux, uy, uz):
    """Exact integrals of the overwrite-painted phantom along rays from one source point
    (the definition of inputs.line_integrals3), FP64."""
    import torch
    dev = ux.device
    E = len(ellipsoids)
    el = torch.tensor([[e.cx, e.cy, e.cz, e.a, e.b, e.c, e.phi, e.value] for e in ellipsoids],
                      dtype=torch.float64, device=dev)
    cx, cy, cz, a, b, cc, phi = (el[:, k][None, :] for k in range(7))
    cs, sn = torch.cos(phi), torch.sin(phi)
    qx, qy, qz = src[0] - cx, src[1] - cy, src[2] - cz
    qu, qw = qx * cs + qy * sn, -qx * sn + qy * cs
    eu = ux[:, None] * cs + uy[:, None] * sn
    ew = -ux[:, None] * sn + uy[:, None] * cs
    ez = uz[:, None]
    A = eu * eu / a ** 2 + ew * ew / b ** 2 + ez * ez / cc ** 2
    B = 2.0 * (qu * eu / a ** 2 + qw * ew / b ** 2 + qz * ez / cc ** 2)
    C = qu * qu / a ** 2 + qw * qw / b ** 2 + qz * qz / cc ** 2 - 1.0
    disc = B * B - 4.0 * A * C
    ok = disc > 0
    sq = torch.sqrt(torch.where(ok, disc, torch.zeros_like(disc)))
    nan = torch.full_like(disc, float("nan"))
    t1 = torch.where(ok, (-B - sq) / (2 * A), nan)
    t2 = torch.where(ok, (-B + sq) / (2 * A), nan)
    pts, _ = torch.sort(torch.cat([t1, t2], dim=1), dim=1)
    lo, hi = pts[:, :-1], pts[:, 1:]
    mid = 0.5 * (lo + hi)
    cov = (t1[:, None, :] < mid[:, :, None]) & (mid[:, :, None] < t2[:, None, :])
    idx = torch.arange(E, device=dev)[None, None, :]
    top = torch.where(cov, idx, torch.full_like(idx, -1)).amax(dim=2)
    vals = torch.cat([el[:, 7], torch.zeros(1, dtype=torch.float64, device=dev)])
    v = vals[torch.where(top >= 0, top, torch.full_like(top, E))]
    seg = torch.where(torch.isfinite(lo) & torch.isfinite(hi), hi - lo, torch.zeros_like(lo))
    return (torch.where(top >= 0, v, torch.zeros_like(v)) * seg).sum(dim=1)


def c5_sinogram_gpu(seed: int, g: I.ConeGeometry, device, i0: float = 5e4):
    """Noisy projections [n_views * nv * nu] (FP32, device) of the cone-beam workload's
    phantom for this seed: exact line integrals, counts ~ Poisson(I0 exp(-p)),
    y = ln(I0 / max(counts, 1))."""
    import torch
    els, _ = I.c5_ellipsoids(seed, g)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.empty(g.n_rays, dtype=torch.float32, device=device)
    per = g.nu * g.nv
    for k in range(g.n_views):
        src, ux, uy, uz = rays_gpu(g, k, device)
        p = line_integrals3_gpu(els, src, ux, uy, uz)
        counts = torch.poisson(i0 * torch.exp(-p), generator=gen)
        out[k * per:(k + 1) * per] = torch.log(i0 / counts.clamp_min(1.0)).float()
    return out


def nnz_of(g: I.ConeGeometry) -> int:
    """Number of (ray, voxel) pairs with positive intersection length, counted per ray as
    1 + the interior planes crossed along x, y and z between entry and exit (FP64).  A ray
    that crosses two planes at one point is counted one cell too many, so this is an upper
    bound: 0.02-0.07 % above the exact count on the reduced scans of the workload."""
    th = g.view_angles()
    u = (np.arange(g.nu) - (g.nu - 1) / 2.0 + g.u_off) * g.du
    w = (np.arange(g.nv) - (g.nv - 1) / 2.0 + g.v_off) * g.dv
    W, U = np.meshgrid(w, u, indexing="ij")
    lo = np.array([-g.nx * g.dx / 2, -g.ny * g.dy / 2, -g.nz * g.dz / 2])
    pitch = np.array([g.dx, g.dy, g.dz])
    total = 0
    for k in range(g.n_views):
        c, s = math.cos(th[k]), math.sin(th[k])
        S = np.array([g.sid * c, g.sid * s, 0.0])
        d = np.stack([-g.sdd * c - U * s, -g.sdd * s + U * c, W], axis=-1).reshape(-1, 3)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (lo[None, :] - S[None, :]) / d
            tb = (-lo[None, :] - S[None, :]) / d
        tmin = np.nanmax(np.where(np.isfinite(ta), np.minimum(ta, tb), -np.inf), axis=1)
        tmax = np.nanmin(np.where(np.isfinite(ta), np.maximum(ta, tb), np.inf), axis=1)
        hit = tmax > tmin
        P0 = S[None, :] + tmin[:, None] * d
        P1 = S[None, :] + tmax[:, None] * d
        i0 = np.floor((np.minimum(P0, P1) - lo) / pitch + 1e-9)
        i1 = np.ceil((np.maximum(P0, P1) - lo) / pitch - 1e-9) - 1
        cells = 1 + np.sum(np.maximum(i1 - i0, 0), axis=1)
        total += int(np.sum(np.where(hit, cells, 0)))
    return total
