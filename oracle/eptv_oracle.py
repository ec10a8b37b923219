"""FP64 CPU oracle of the EPTV reconstruction (Tian et al., "GPU-based low dose CT
reconstruction via edge-preserving total variation regularization").

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
baseline import this module.  It shares no code with the CUDA path: the system matrix
comes from the plain-C Siddon tracer in siddon.c, everything else is numpy in float64,
written to be checked against the paper by eye.

Functions and the passages they follow (sharded.py evaluates the same P and P^T on every
host core, for timing):
  rays / project / backproject .... Eq. (1), Sec. 2.1 (p_ij = intersection length,
                                    Siddon), Sec. 3 (fan-beam arc detector); P^T is the
                                    exact transpose (Eq. A3 of App. III, adjoint identity)
  backproject_eq11 ................ Eq. (11), Sec. 2.3 and App. III: the paper's pixel-driven
                                    interpolating back projector (an approximation of P^T)
  relative_error / sobel_edges /
  edge_correlation / roi_snr ...... Eqs. (12), (13), (14), Sec. 3: image-quality metrics
  cgls ............................ App. I (CGLS for (P1), restarted at f^(k))
  half_edges ...................... Eq. (A3), App. II (half-point magnitudes)
  edge_weights .................... Eq. (5)
  select_sigma .................... Sec. 2.1, adaptive sigma from the gradient histogram
  tv_variation .................... Eq. (A2), App. II
  p2_gradient ..................... Eq. (9)
  p2_solve ........................ Sec. 2.2, (P2) by gradient descent + Armijo,
                                    weights recomputed every GD iteration
  reconstruct ..................... Sec. 2.2 EPTV algorithm (steps 1-3, f^(0) = 0)
  report_energy ................... Eq. (2)

Readings of points the paper leaves open (each also listed in the design notes):
  * differences are in pixel units (A2/A3 do not divide by the pixel size);
  * the magnitude is the isotropic one of A3, with eps^2 inside the square root;
  * "zero boundary condition" (App. II) = f is 0 outside the image, so the half-edges
    between the image and the outside are part of J;
  * Eq. (10) is read as -div(w grad f / |grad f|), discretised exactly as A2 (lagged
    diffusivity: no derivative through w or through the cross terms of A3);
  * sigma = k-th smallest of the pooled half-edge magnitudes of the (P2) input v,
    k = ceil(q n), held fixed during one (P2) solve;
  * (P2) starts at f = v; Armijo trial steps t0 * shrink^m, m < max_trials, with
    t0 = min(grow * t_prev, t_max); if none passes the step is 0 and the next GD
    iteration continues below the last trial; energy for the test = lambda/2 |f - v|^2
    + sum_e w_e T_e(f) with w frozen at the current GD iterate.
  * Eq. (11): beta* and l are taken at the pixel centre; y^theta(beta*) is the linear
    interpolation between the two bins around beta* (bins outside the detector read 0);
    the paper states the arc detector (uniform in beta); for a flat detector (uniform in
    t = tan beta) the same change of variables in (A7) gives the weight
    (du dv / dt) (1 + t*^2) / l.
  * Eq. (13): the "standard Sobel edge detector" is read as: 3x3 Sobel derivatives
    gx, gy at the interior pixels, an edge where gx^2 + gy^2 > s^2 mean(gx^2 + gy^2) over
    the interior (s = 2 by default), no thinning; border pixels are never edges.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_siddon.so")
_lib = None

EPTV, ONE, PRIOR = 0, 1, 2
ARMIJO, FIXED = 0, 1


def build(force: bool = False) -> str:
    """Compile siddon.c (plain C, float64, no fast-math) into a shared library."""
    src = os.path.join(_HERE, "siddon.c")
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
        for name in ("og_project", "og_backproject"):
            fn = getattr(_lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                           ctypes.c_long, dp, dp, dp, dp, dp, dp]
        _lib.og_ray_row.restype = ctypes.c_int
        _lib.og_ray_row.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_long), dp]
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------------- geometry (Sec. 3)

def rays(g):
    """Source point and unit direction of each ray of the fan-beam scan, ray = v*B + k.

    Source at sid (cos th_v, sin th_v); the central ray points at the isocentre; bin k
    sits at fan angle beta_k = (k - (B-1)/2 + o) dbeta (arc detector; flat detector:
    atan of that), measured from the central ray."""
    th = g.view_angles()
    out = [np.empty(g.n_rays) for _ in range(4)]
    for v in range(g.n_views):
        c, s = math.cos(th[v]), math.sin(th[v])
        for k in range(g.n_bins):
            kk = k - (g.n_bins - 1) / 2.0 + g.bin_offset
            beta = kk * g.dbeta if g.detector == 0 else math.atan(kk * g.dbeta)
            cb, sb = math.cos(beta), math.sin(beta)
            r = v * g.n_bins + k
            out[0][r] = g.sid * c
            out[1][r] = g.sid * s
            out[2][r] = -c * cb + s * sb          # rotate (-c, -s) by +beta
            out[3][r] = -c * sb - s * cb
    return tuple(out)


class Operator:
    """P and P^T of one geometry, float64 (Eq. 1)."""

    def __init__(self, g):
        self.g = g
        self.sx, self.sy, self.ux, self.uy = rays(g)

    def project(self, f: np.ndarray) -> np.ndarray:
        g = self.g
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.ny, g.nx)
        y = np.empty(g.n_rays)
        rc = _load().og_project(g.nx, g.ny, g.dx, g.dy, g.n_rays, _dp(self.sx), _dp(self.sy),
                                _dp(self.ux), _dp(self.uy), _dp(f), _dp(y))
        assert rc == 0
        return y.reshape(g.n_views, g.n_bins)

    def backproject(self, y: np.ndarray) -> np.ndarray:
        g = self.g
        y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        assert y.size == g.n_rays
        f = np.empty(g.ny * g.nx)
        rc = _load().og_backproject(g.nx, g.ny, g.dx, g.dy, g.n_rays, _dp(self.sx), _dp(self.sy),
                                    _dp(self.ux), _dp(self.uy), _dp(y), _dp(f))
        assert rc == 0
        return f.reshape(g.ny, g.nx)


def backproject_eq11(g, y: np.ndarray) -> np.ndarray:
    """Eq. (11): [P^T y](u, v) = (du dv / dbeta) sum_theta y^theta(beta*) / l(u, v), with
    beta* the fan angle of the line from the source through the pixel centre (measured
    from the central ray, positive counter-clockwise as in rays()), l its length from the
    source, y^theta(beta*) linearly interpolated between detector bins.  Flat detector:
    beta* -> t* = tan beta*, weight (du dv / dt) (1 + t*^2) / l (reading in the header)."""
    y = np.asarray(y, dtype=np.float64).reshape(g.n_views, g.n_bins)
    xc = (np.arange(g.nx) + 0.5) * g.dx - g.nx * g.dx / 2.0
    yc = (np.arange(g.ny) + 0.5) * g.dy - g.ny * g.dy / 2.0
    X, Y = np.meshgrid(xc, yc)                           # [ny][nx] pixel centres
    out = np.zeros((g.ny, g.nx))
    kc = (g.n_bins - 1) / 2.0 - g.bin_offset              # bin k sits at (k - kc) dbeta
    for v, th in enumerate(g.view_angles()):
        sx, sy = g.sid * math.cos(th), g.sid * math.sin(th)
        cx, cy = -math.cos(th), -math.sin(th)            # central ray direction
        wx, wy = X - sx, Y - sy
        cross = cx * wy - cy * wx                         # |w| sin(beta*)
        dot = cx * wx + cy * wy                           # |w| cos(beta*)
        l = np.hypot(wx, wy)
        if g.detector == 0:
            u = np.arctan2(cross, dot) / g.dbeta + kc
            weight = 1.0 / l
        else:
            t = cross / dot
            u = t / g.dbeta + kc
            weight = (1.0 + t * t) / l
        k0 = np.floor(u).astype(np.int64)
        frac = u - k0
        row = y[v]
        y0 = np.where((k0 >= 0) & (k0 < g.n_bins), row[np.clip(k0, 0, g.n_bins - 1)], 0.0)
        y1 = np.where((k0 + 1 >= 0) & (k0 + 1 < g.n_bins), row[np.clip(k0 + 1, 0, g.n_bins - 1)], 0.0)
        out += ((1.0 - frac) * y0 + frac * y1) * weight
    return out * (g.dx * g.dy / g.dbeta)


def project_rays(nx, ny, dx, dy, sx, sy, ux, uy, f):
    """P f for arbitrary rays (source point, unit direction)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (sx, sy, ux, uy)]
    f = np.ascontiguousarray(f, dtype=np.float64)
    y = np.empty(arrs[0].size)
    rc = _load().og_project(nx, ny, dx, dy, arrs[0].size, *[_dp(a) for a in arrs], _dp(f), _dp(y))
    assert rc == 0
    return y


def backproject_rays(nx, ny, dx, dy, sx, sy, ux, uy, y):
    """P^T y for arbitrary rays (source point, unit direction): the image [ny][nx]."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (sx, sy, ux, uy)]
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert y.size == arrs[0].size
    f = np.empty(ny * nx)
    rc = _load().og_backproject(nx, ny, dx, dy, arrs[0].size, *[_dp(a) for a in arrs], _dp(y), _dp(f))
    assert rc == 0
    return f


def ray_row(nx, ny, dx, dy, sx, sy, ux, uy):
    """Nonzeros (pixel index, length) of one ray's row of P."""
    cap = nx + ny + 4
    pix = (ctypes.c_long * cap)()
    ln = np.empty(cap)
    c = _load().og_ray_row(nx, ny, dx, dy, sx, sy, ux, uy, pix, _dp(ln))
    assert c >= 0
    return np.array(pix[:c], dtype=np.int64), ln[:c].copy()


# ------------------------------------------------------------------ CGLS (App. I)

def cgls(op: Operator, y: np.ndarray, u0: np.ndarray, M: int, log: Optional[list] = None):
    """M CGLS iterations for min |P u - y|^2 started at u0 (App. I); returns u^(M)."""
    u = np.array(u0, dtype=np.float64)
    r = y - op.project(u)
    s = op.backproject(r)
    gamma = float(np.sum(s * s))                 # |P^T r^(m)|^2
    for _ in range(M):
        q = op.project(s)                        # P s^(m)
        qq = float(np.sum(q * q))
        if qq == 0.0:
            break
        a = gamma / qq                           # step 1
        u = u + a * s                            # step 2
        r = r - a * q                            # step 3
        t = op.backproject(r)
        gamma_new = float(np.sum(t * t))
        b = gamma_new / gamma if gamma > 0 else 0.0   # step 4
        s = t + b * s                            # step 5
        gamma = gamma_new
        if log is not None:
            log.append(dict(a=a, b=b, rr=float(np.sum(r * r))))
    return u


# ------------------------------------------------------- EPTV stencil (App. II, Eq. A2-A3)

def half_edges(f: np.ndarray, eps: float):
    """Magnitudes |f_{i+1/2,j}| and |f_{i,j+1/2}| of Eq. (A3) at every half-edge.

    Returns (Dx, Tx, Dy, Ty).  Dx, Tx have shape (ny, nx+1): column e is the half-edge
    between pixel columns e-1 and e (pixels outside the image are 0).  Dy, Ty have
    shape (ny+1, nx) likewise for rows.  D is the primary difference f_{i+1} - f_i;
    T = sqrt(eps^2 + D^2 + 1/2 (fbar_{+} - fbar)^2 + 1/2 (fbar - fbar_{-})^2) with
    fbar the half-point averages of Eq. (A3)."""
    ny, nx = f.shape
    F = np.zeros((ny + 2, nx + 2))
    F[1:-1, 1:-1] = f
    # x half-edges
    L, R = F[:, :-1], F[:, 1:]                   # (ny+2, nx+1)
    Dx = (R - L)[1:-1]
    mx = 0.5 * (L + R)                           # f_{i+1/2, l}
    cu = mx[2:] - mx[1:-1]                       # f_{i+1/2,j+1} - f_{i+1/2,j}
    cd = mx[1:-1] - mx[:-2]                      # f_{i+1/2,j} - f_{i+1/2,j-1}
    Tx = np.sqrt(eps * eps + Dx * Dx + 0.5 * cu * cu + 0.5 * cd * cd)
    # y half-edges
    Bm, Tp = F[:-1, :], F[1:, :]                 # (ny+1, nx+2)
    Dy = (Tp - Bm)[:, 1:-1]
    my = 0.5 * (Bm + Tp)
    cr = my[:, 2:] - my[:, 1:-1]
    cl = my[:, 1:-1] - my[:, :-2]
    Ty = np.sqrt(eps * eps + Dy * Dy + 0.5 * cr * cr + 0.5 * cl * cl)
    return Dx, Tx, Dy, Ty


def edge_weights(T: np.ndarray, sigma: float) -> np.ndarray:
    """w = exp(-(T / sigma)^2), Eq. (5) with the A3 magnitude."""
    return np.exp(-(T * T) / (sigma * sigma))


def sigma_rank(n: int, q: float) -> int:
    """1-based rank k = ceil(q n), clamped to [1, n]."""
    return min(max(int(math.ceil(q * n)), 1), n)


def select_sigma(Tx, Ty, q: float, floor: float = 1e-12) -> float:
    """Adaptive sigma: the k-th smallest pooled half-edge magnitude, k = ceil(q n)."""
    pool = np.sort(np.concatenate([Tx.ravel(), Ty.ravel()]))
    return max(float(pool[sigma_rank(pool.size, q) - 1]), floor)


def tv_variation(Dx, Tx, wx, Dy, Ty, wy) -> np.ndarray:
    """delta J / delta f_{i,j} by the symmetric scheme of Eq. (A2)."""
    Qx = wx * Dx / Tx                            # w_{i+1/2,j} (f_{i+1,j} - f_{i,j}) / |.|
    Qy = wy * Dy / Ty
    return -(Qx[:, 1:] - Qx[:, :-1]) - (Qy[1:, :] - Qy[:-1, :])


def tv_energy(Tx, wx, Ty, wy) -> float:
    """J = sum over half-edges of w_e T_e (Eq. 4 discretised with the A3 magnitude)."""
    return float(np.sum(wx * Tx) + np.sum(wy * Ty))


@dataclasses.dataclass
class P2Stats:
    sigma: float = 0.0
    steps: list = dataclasses.field(default_factory=list)
    energies: list = dataclasses.field(default_factory=list)
    fails: int = 0
    t_prev: float = 0.0
    trials: list = dataclasses.field(default_factory=list)   # per GD iteration: [(t, rho)]


def _weights(mode, Tx, Ty, sigma, prior):
    if mode == ONE:
        return np.ones_like(Tx), np.ones_like(Ty)
    if mode == PRIOR:
        return prior
    return edge_weights(Tx, sigma), edge_weights(Ty, sigma)


def prior_edge_weights(w: np.ndarray):
    """Edge weights from a per-pixel map w: the mean of the two pixels beside each
    half-edge (a pixel outside the image takes the value of its neighbour inside)."""
    W = np.pad(w, 1, mode="edge")
    wx = 0.5 * (W[1:-1, :-1] + W[1:-1, 1:])
    wy = 0.5 * (W[:-1, 1:-1] + W[1:, 1:-1])
    return wx, wy


def p2_gradient(f, v, lam, eps, sigma, mode=EPTV, prior=None):
    """g = lambda (f - v) + delta J/delta f (Eq. 9 with Eq. A2); also returns the
    frozen weights and the energy lambda/2 |f-v|^2 + J at f."""
    Dx, Tx, Dy, Ty = half_edges(f, eps)
    wx, wy = _weights(mode, Tx, Ty, sigma, prior)
    g = lam * (f - v) + tv_variation(Dx, Tx, wx, Dy, Ty, wy)
    E = 0.5 * lam * float(np.sum((f - v) ** 2)) + tv_energy(Tx, wx, Ty, wy)
    return g, wx, wy, E


def p2_energy_frozen(f, v, lam, eps, wx, wy) -> float:
    """lambda/2 |f - v|^2 + sum_e w_e T_e(f) with given (frozen) weights."""
    _, Tx, _, Ty = half_edges(f, eps)
    return 0.5 * lam * float(np.sum((f - v) ** 2)) + tv_energy(Tx, wx, Ty, wy)


def p2_solve(v, p, t_prev: float, f_init=None, prior=None, mode=None):
    """(P2): min lambda/2 |f - v|^2 + |f|_EPTV by GD with Armijo backtracking (Sec. 2.2);
    the weights are recomputed from the current iterate at every GD iteration."""
    mode = p.weights_mode if mode is None else mode
    st = P2Stats()
    _, Tvx, _, Tvy = half_edges(v, p.eps)
    st.sigma = select_sigma(Tvx, Tvy, p.sigma_q, p.sigma_floor)
    f = np.array(v if f_init is None else f_init, dtype=np.float64)
    for _ in range(p.n_gd):
        g, wx, wy, E0 = p2_gradient(f, v, p.lam, p.eps, st.sigma, mode, prior)
        st.energies.append(E0)
        if p.step_rule == FIXED:
            t = p.t_fixed
            f = f - t * g
            st.steps.append(t)
            continue
        gg = float(np.sum(g * g))
        t0 = min(p.armijo_grow * t_prev, p.t_max_eff)
        accepted = None
        t = t0
        tried = []
        for m in range(p.max_trials):
            t = t0 * p.armijo_shrink ** m
            E1 = p2_energy_frozen(f - t * g, v, p.lam, p.eps, wx, wy)
            # rho = achieved decrease / (t |g|^2); Armijo accepts rho >= c
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


def report_energy(op: Operator, f, y, p, sigma_ref: float) -> float:
    """E(f) = mu/2 |P f - y|^2 + J(f; w(f; sigma_ref)), Eq. (2)."""
    r = op.project(f) - y
    Dx, Tx, Dy, Ty = half_edges(f, p.eps)
    wx, wy = _weights(p.weights_mode if p.weights_mode != PRIOR else EPTV, Tx, Ty, sigma_ref, None)
    return 0.5 * p.mu * float(np.sum(r * r)) + tv_energy(Tx, wx, Ty, wy)


@dataclasses.dataclass
class ReconLog:
    sigmas: list = dataclasses.field(default_factory=list)
    steps: list = dataclasses.field(default_factory=list)
    trials: list = dataclasses.field(default_factory=list)
    fails: int = 0
    energies: list = dataclasses.field(default_factory=list)
    t_prev: float = 0.0


def reconstruct(op: Operator, y, p, f0=None, prior_w=None, n_outer=None,
                sigma_ref: Optional[float] = None, log: Optional[ReconLog] = None):
    """EPTV algorithm (Sec. 2.2): f^(0) = 0 (or a warm start); per outer iteration
    (1) v = CGLS_M started at f^(k); (2) f = (P2) solution by GD + Armijo;
    (3) f = max(f, 0)."""
    g = op.g
    f = np.zeros((g.ny, g.nx)) if f0 is None else np.maximum(np.array(f0, dtype=np.float64), 0.0)
    y = np.asarray(y, dtype=np.float64).reshape(g.n_views, g.n_bins)
    n_outer = p.n_outer if n_outer is None else n_outer
    t_prev = p.t_init_eff
    prior = prior_edge_weights(prior_w) if prior_w is not None else None
    for k in range(n_outer):
        v = cgls(op, y, f, p.cgls_iters)
        if prior is not None and k < p.prior_iters:
            mode = PRIOR
        else:
            mode = EPTV if p.weights_mode == PRIOR else p.weights_mode
        f, st = p2_solve(v, p, t_prev, prior=prior, mode=mode)
        t_prev = st.t_prev
        f = np.maximum(f, 0.0)
        if log is not None:
            log.sigmas.append(st.sigma)
            log.steps.append(st.steps)
            log.trials.append(st.trials)
            log.fails += st.fails
            if sigma_ref is not None:
                log.energies.append(report_energy(op, f, y, p, sigma_ref))
    if log is not None:
        log.t_prev = t_prev
    return f


# ------------------------------------------------------------------ Sec. 3 metrics

def relative_error(f, f_true):
    """Eq. (12): e = |f - f*|^2 / |f*|^2 (squared norms, as printed)."""
    f = np.asarray(f, dtype=np.float64)
    t = np.asarray(f_true, dtype=np.float64)
    return float(np.sum((f - t) ** 2) / np.sum(t ** 2))


def sobel_gradient2(f):
    """gx^2 + gy^2 of the 3x3 Sobel derivatives at the interior pixels (0 on the border);
    x = column index, y = row index."""
    f = np.asarray(f, dtype=np.float64)
    ny, nx = f.shape
    g2 = np.zeros((ny, nx))
    if nx < 3 or ny < 3:
        return g2
    gx = ((f[:-2, 2:] + 2.0 * f[1:-1, 2:] + f[2:, 2:]) - (f[:-2, :-2] + 2.0 * f[1:-1, :-2] + f[2:, :-2]))
    gy = ((f[2:, :-2] + 2.0 * f[2:, 1:-1] + f[2:, 2:]) - (f[:-2, :-2] + 2.0 * f[:-2, 1:-1] + f[:-2, 2:]))
    g2[1:-1, 1:-1] = gx * gx + gy * gy
    return g2


def sobel_edges(f, scale: float = 2.0):
    """Binary edge map of Eq. (13) (reading in the header): interior pixels whose squared
    Sobel magnitude exceeds scale^2 times its mean over the interior."""
    g2 = sobel_gradient2(f)
    ny, nx = g2.shape
    if nx < 3 or ny < 3:
        return np.zeros((ny, nx), dtype=np.uint8)
    mean = float(np.mean(g2[1:-1, 1:-1]))
    return (g2 > scale * scale * mean).astype(np.uint8)


def edge_correlation(b, b_true):
    """Eq. (13): correlation coefficient of two binary edge maps over all pixels."""
    b = np.asarray(b, dtype=np.float64).ravel()
    t = np.asarray(b_true, dtype=np.float64).ravel()
    db, dt = b - b.mean(), t - t.mean()
    den = math.sqrt(float(np.sum(db * db)) * float(np.sum(dt * dt)))
    return float(np.sum(db * dt) / den) if den > 0 else float("nan")


def roi_snr(f, x0: int, y0: int, w: int, h: int):
    """Eq. (14): SNR = 10 log10(E(P)^2 / E([P - E(P)]^2)) over the ROI pixels P
    (columns x0 .. x0 + w - 1, rows y0 .. y0 + h - 1)."""
    P = np.asarray(f, dtype=np.float64)[y0:y0 + h, x0:x0 + w]
    m = float(np.mean(P))
    return 10.0 * math.log10(m * m / float(np.mean((P - m) ** 2)))
