"""FP64 CPU oracle of EPTV for 3-D cone-beam CT (the extension of the paper's 2-D method).

TEST INFRASTRUCTURE ONLY.  Only the test suite and the benchmark's CPU baseline import
this module; it shares no code with the CUDA path.  The system matrix comes from the
plain-C 3-D Siddon tracer in siddon3d.c; everything else is numpy in float64.

The paper is 2-D.  The 3-D method is the same algorithm (Sec. 2.2: CGLS for (P1), GD with
Armijo for (P2), clamp) with the 2-D pieces extended as follows (readings, also listed in
the design notes):
  * P (Eq. 1): p_ij = length of ray i inside voxel j (Siddon in three dimensions);
  * half-faces instead of half-edges: between voxels a and b neighbouring along x (likewise
    y, z), with the volume 0 outside (App. II's zero boundary);
  * magnitude (A3 extended): T^2 = eps^2 + D^2 + 1/2 (c+^2 + c-^2) over each of the two
    transverse directions, D = f_b - f_a, c+ / c- = differences of the pair means m =
    (f_a + f_b) / 2 towards the next / from the previous row or slice;
  * weights (Eq. 5): w = exp(-(T / sigma)^2), sigma = k-th smallest T of the three face
    families of the (P2) input, k = ceil(q n);
  * variation (A2 extended, lagged): delta J / delta f = -sum over the three directions of
    the difference of q = w D / T across the voxel.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional

import numpy as np

from . import eptv_oracle as O2

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_siddon3d.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile siddon3d.c (plain C, float64, no fast-math) into a shared library."""
    src = os.path.join(_HERE, "siddon3d.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC",
                           "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        geo = [ctypes.c_int] * 3 + [ctypes.c_double] * 3
        for name in ("og3_project", "og3_backproject"):
            fn = getattr(_lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = geo + [ctypes.c_long] + [dp] * 8
        _lib.og3_ray_row.restype = ctypes.c_int
        _lib.og3_ray_row.argtypes = geo + [ctypes.c_double] * 6 + [ctypes.POINTER(ctypes.c_long), dp]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def rays3(g):
    """Source point and unit direction of each ray (float64), ray = (k nv + iv) nu + iu:
    source at sid (cos th, sin th, 0); detector pixel centre at source + sdd c + u e_u +
    w e_z with c = -(cos th, sin th, 0), e_u = (-sin th, cos th, 0), e_z = (0, 0, 1),
    u = (iu - (nu-1)/2 + u_off) du, w = (iv - (nv-1)/2 + v_off) dv."""
    n = g.n_rays
    out = [np.empty(n) for _ in range(6)]
    r = 0
    for th in g.view_angles():
        c, s = math.cos(th), math.sin(th)
        for iv in range(g.nv):
            w = (iv - (g.nv - 1) / 2.0 + g.v_off) * g.dv
            for iu in range(g.nu):
                u = (iu - (g.nu - 1) / 2.0 + g.u_off) * g.du
                d = np.array([-g.sdd * c - u * s, -g.sdd * s + u * c, w])
                d /= math.sqrt(float(d @ d))
                out[0][r], out[1][r], out[2][r] = g.sid * c, g.sid * s, 0.0
                out[3][r], out[4][r], out[5][r] = d
                r += 1
    return tuple(out)


def rays3_subset(g, idx):
    """{ray index: (source, unit direction)} for the given ray indices (FP64), the rays of
    rays3 without building all of them."""
    out = {}
    th = g.view_angles()
    per_view = g.nv * g.nu
    for i in np.asarray(idx, dtype=np.int64):
        k, rem = divmod(int(i), per_view)
        iv, iu = divmod(rem, g.nu)
        c, s = math.cos(th[k]), math.sin(th[k])
        u = (iu - (g.nu - 1) / 2.0 + g.u_off) * g.du
        w = (iv - (g.nv - 1) / 2.0 + g.v_off) * g.dv
        d = np.array([-g.sdd * c - u * s, -g.sdd * s + u * c, w])
        d /= math.sqrt(float(d @ d))
        out[int(i)] = (np.array([g.sid * c, g.sid * s, 0.0]), d)
    return out


def ray_row_of(g, s, u):
    """Nonzeros (voxel index, length) of the row of P of the ray s + t u."""
    cap = g.nx + g.ny + g.nz + 8
    vox = (ctypes.c_long * cap)()
    ln = np.empty(cap)
    c = _load().og3_ray_row(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, float(s[0]), float(s[1]), float(s[2]),
                            float(u[0]), float(u[1]), float(u[2]), vox, _dp(ln))
    assert c >= 0
    return np.array(vox[:c], dtype=np.int64), ln[:c].copy()


class Operator3:
    """P and P^T of a cone-beam geometry, float64."""

    def __init__(self, g):
        self.g = g
        self.r = rays3(g)

    def _geo(self):
        g = self.g
        return (g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)

    def project(self, f):
        g = self.g
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert f.size == g.n_vox
        y = np.empty(g.n_rays)
        rc = _load().og3_project(*self._geo(), g.n_rays, *[_dp(a) for a in self.r], _dp(f), _dp(y))
        assert rc == 0
        return y.reshape(g.n_views, g.nv, g.nu)

    def backproject(self, y):
        g = self.g
        y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        assert y.size == g.n_rays
        f = np.empty(g.n_vox)
        rc = _load().og3_backproject(*self._geo(), g.n_rays, *[_dp(a) for a in self.r], _dp(y), _dp(f))
        assert rc == 0
        return f.reshape(g.nz, g.ny, g.nx)

    def ray_row(self, i):
        g = self.g
        cap = g.nx + g.ny + g.nz + 8
        vox = (ctypes.c_long * cap)()
        ln = np.empty(cap)
        c = _load().og3_ray_row(*self._geo(), *[float(a[i]) for a in self.r], vox, _dp(ln))
        assert c >= 0
        return np.array(vox[:c], dtype=np.int64), ln[:c].copy()


# ------------------------------------------------------------------ 3-D EPTV

def half_faces(f, eps: float):
    """(D, T) of the x, y and z half-faces.  Shapes: x (nz, ny, nx+1) -- face e lies
    between voxel columns e-1 and e --, y (nz, ny+1, nx), z (nz+1, ny, nx); voxels outside
    the volume are 0."""
    f = np.asarray(f, dtype=np.float64)
    F = np.pad(f, 1)                                   # (nz+2, ny+2, nx+2)
    out = []
    for axis in (2, 1, 0):                             # x, y, z faces
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(None, -1)
        hi[axis] = slice(1, None)
        A, B = F[tuple(lo)], F[tuple(hi)]              # pairs along the face normal
        D = B - A
        M = 0.5 * (A + B)
        T2 = eps * eps + D * D
        for t in (0, 1, 2):                            # the two transverse axes
            if t == axis:
                continue
            up = [slice(1, -1)] * 3
            cen = [slice(1, -1)] * 3
            dn = [slice(1, -1)] * 3
            up[axis] = cen[axis] = dn[axis] = slice(None)
            up[t], dn[t] = slice(2, None), slice(None, -2)
            cp = M[tuple(up)] - M[tuple(cen)]
            cm = M[tuple(cen)] - M[tuple(dn)]
            inner = [slice(1, -1)] * 3
            inner[axis] = slice(None)
            T2[tuple(inner)] += 0.5 * cp * cp + 0.5 * cm * cm
        inner = [slice(1, -1)] * 3
        inner[axis] = slice(None)
        out.append((D[tuple(inner)], np.sqrt(T2[tuple(inner)])))
    return out                                         # [(Dx, Tx), (Dy, Ty), (Dz, Tz)]


def select_sigma(faces, q: float, floor: float = 1e-12) -> float:
    pool = np.sort(np.concatenate([T.ravel() for _, T in faces]))
    return max(float(pool[O2.sigma_rank(pool.size, q) - 1]), floor)


def weights(faces, sigma: float, mode: int):
    if mode == O2.ONE:
        return [np.ones_like(T) for _, T in faces]
    return [O2.edge_weights(T, sigma) for _, T in faces]


def tv_variation(faces, ws):
    """delta J / delta f: minus the divergence of q = w D / T (lagged, extended A2)."""
    (Dx, Tx), (Dy, Ty), (Dz, Tz) = faces
    wx, wy, wz = ws
    Qx, Qy, Qz = wx * Dx / Tx, wy * Dy / Ty, wz * Dz / Tz
    return -(Qx[:, :, 1:] - Qx[:, :, :-1]) - (Qy[:, 1:, :] - Qy[:, :-1, :]) - (Qz[1:] - Qz[:-1])


def tv_energy(faces, ws) -> float:
    return float(sum(np.sum(w * T) for (_, T), w in zip(faces, ws)))


def p2_gradient(f, v, lam, eps, sigma, mode=O2.EPTV):
    faces = half_faces(f, eps)
    ws = weights(faces, sigma, mode)
    g = lam * (f - v) + tv_variation(faces, ws)
    E = 0.5 * lam * float(np.sum((f - v) ** 2)) + tv_energy(faces, ws)
    return g, ws, E


def p2_energy_frozen(f, v, lam, eps, ws) -> float:
    return 0.5 * lam * float(np.sum((f - v) ** 2)) + tv_energy(half_faces(f, eps), ws)


def p2_solve(v, p, t_prev: float, mode: Optional[int] = None):
    """(P2) in 3-D: GD with Armijo backtracking, weights recomputed every GD iteration
    (the same rules as the 2-D oracle's p2_solve)."""
    mode = p.weights_mode if mode is None else mode
    st = O2.P2Stats()
    st.sigma = select_sigma(half_faces(v, p.eps), p.sigma_q, p.sigma_floor)
    f = np.array(v, dtype=np.float64)
    for _ in range(p.n_gd):
        g, ws, E0 = p2_gradient(f, v, p.lam, p.eps, st.sigma, mode)
        st.energies.append(E0)
        if p.step_rule == O2.FIXED:
            f = f - p.t_fixed * g
            st.steps.append(p.t_fixed)
            continue
        gg = float(np.sum(g * g))
        t0 = min(p.armijo_grow * t_prev, p.t_max_eff)
        accepted, t, tried = None, t0, []
        for m in range(p.max_trials):
            t = t0 * p.armijo_shrink ** m
            E1 = p2_energy_frozen(f - t * g, v, p.lam, p.eps, ws)
            tried.append((t, (E0 - E1) / (t * gg) if gg > 0 else math.inf))
            if E1 <= E0 - p.armijo_c * t * gg:
                accepted = t
                break
        st.trials.append(tried)
        if accepted is None:
            st.fails += 1
            st.steps.append(0.0)
            t_prev = t * p.armijo_shrink / p.armijo_grow
        else:
            f = f - accepted * g
            st.steps.append(accepted)
            t_prev = accepted
    st.t_prev = t_prev
    return f, st


def report_energy(op: Operator3, f, y, p, sigma_ref: float) -> float:
    """E(f) = mu/2 |P f - y|^2 + J(f; w(f; sigma_ref)) (Eq. 2 in 3-D)."""
    r = op.project(f) - np.asarray(y).reshape(op.g.n_views, op.g.nv, op.g.nu)
    faces = half_faces(f, p.eps)
    mode = p.weights_mode if p.weights_mode != O2.PRIOR else O2.EPTV
    return 0.5 * p.mu * float(np.sum(r * r)) + tv_energy(faces, weights(faces, sigma_ref, mode))


def reconstruct(op: Operator3, y, p, f0=None, log: Optional[O2.ReconLog] = None):
    """EPTV algorithm (Sec. 2.2) in 3-D: f^(0) = 0; CGLS_M from f^(k), (P2), clamp."""
    g = op.g
    f = np.zeros((g.nz, g.ny, g.nx)) if f0 is None else np.maximum(np.array(f0, dtype=np.float64), 0.0)
    y = np.asarray(y, dtype=np.float64).reshape(g.n_views, g.nv, g.nu)
    t_prev = p.t_init_eff
    for _ in range(p.n_outer):
        v = O2.cgls(op, y, f, p.cgls_iters)
        f, st = p2_solve(v, p, t_prev)
        t_prev = st.t_prev
        f = np.maximum(f, 0.0)
        if log is not None:
            log.sigmas.append(st.sigma)
            log.steps.append(st.steps)
            log.fails += st.fails
    if log is not None:
        log.t_prev = t_prev
    return f
