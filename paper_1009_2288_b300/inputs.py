"""Seeded synthetic inputs for EPTV reconstruction: scan geometries, ellipse phantoms
and noisy fan-beam sinograms.

This module is the only code shared by the CUDA path, its tests and the FP64 oracle.
It holds no arithmetic of the reconstruction method itself (no projector, no adjoint,
no CGLS, no TV stencil): it describes scanners and draws data.

The paper's experiments use an NCAT digital phantom and physical chest / Catphan scans
(Sec. 3), none of which is available.  Seeded ellipse phantoms stand in for them, with
the paper's scanner geometry (Sec. 3: GE LightSpeed-like fan beam, 888-bin arc detector
of 1.0239 mm pitch, source-detector 949.075 mm, source-isocenter 541.0 mm, 512x512
image).  Sinograms are the exact line integrals of the analytic ellipses (not a
pixelised projection, to avoid the inverse crime), with Poisson counting noise and the
log transform of Eq. (1).

Conventions (shared by every implementation of the geometry in this repository):
  * image f is row-major [ny][nx], x fastest; pixel (i, j) covers
    x in [x0 + i*dx, x0 + (i+1)*dx], y in [y0 + j*dy, y0 + (j+1)*dy],
    x0 = -nx*dx/2, y0 = -ny*dy/2 (mm); values are attenuation in 1/mm;
  * sinogram is [n_views][n_bins], bins fastest;
  * view v: angle theta_v (angles[v], else 2*pi*v/n_views); source at
    sid*(cos theta, sin theta); central ray direction -(cos theta, sin theta);
  * bin k: k' = k - (n_bins-1)/2 + bin_offset; fan angle beta_k = k'*dbeta for the
    arc detector, atan(k'*dbeta) for the flat detector (dbeta = pitch/sdd);
    ray direction = central direction rotated by +beta_k.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

ARC = 0
FLAT = 1

# GE LightSpeed-like fan geometry (Sec. 3).
GE_SID = 541.0
GE_SDD = 949.075
GE_PITCH = 1.0239
GE_BINS = 888


@dataclasses.dataclass
class FanGeometry:
    """Parameter record of a 2-D fan-beam scan (no arithmetic of the method)."""
    nx: int
    ny: int
    dx: float
    dy: float
    n_views: int
    n_bins: int
    dbeta: float
    bin_offset: float = 0.25
    sid: float = 1000.0
    sdd: float = 1500.0
    detector: int = ARC
    angles: Optional[np.ndarray] = None

    @property
    def n_rays(self) -> int:
        return self.n_views * self.n_bins

    @property
    def n_pix(self) -> int:
        return self.nx * self.ny

    def view_angles(self) -> np.ndarray:
        if self.angles is not None:
            a = np.asarray(self.angles, dtype=np.float64)
            assert a.shape == (self.n_views,)
            return a
        return 2.0 * np.pi * np.arange(self.n_views, dtype=np.float64) / self.n_views


@dataclasses.dataclass
class Ellipse:
    cx: float
    cy: float
    a: float
    b: float
    phi: float
    value: float


@dataclasses.dataclass
class Case:
    """One synthetic reconstruction instance."""
    name: str
    geom: FanGeometry
    ellipses: List[Ellipse]
    i0: float
    n_outer: int
    seed: int
    f_true: Optional[np.ndarray] = None    # [ny][nx] float64, 4x4 supersampled
    p_clean: Optional[np.ndarray] = None   # [V][B] float64 exact line integrals
    y: Optional[np.ndarray] = None         # [V][B] float64 noisy log data


# ----------------------------------------------------------------------------- rays

def fan_rays(g: FanGeometry):
    """Source points and unit directions of every ray, float64, ray index v*B + k."""
    th = g.view_angles()
    kp = np.arange(g.n_bins, dtype=np.float64) - (g.n_bins - 1) / 2.0 + g.bin_offset
    beta = kp * g.dbeta if g.detector == ARC else np.arctan(kp * g.dbeta)
    cth, sth = np.cos(th)[:, None], np.sin(th)[:, None]
    cb, sb = np.cos(beta)[None, :], np.sin(beta)[None, :]
    sx = np.broadcast_to(g.sid * cth, (g.n_views, g.n_bins))
    sy = np.broadcast_to(g.sid * sth, (g.n_views, g.n_bins))
    ccx, ccy = -cth, -sth
    ux = ccx * cb - ccy * sb
    uy = ccx * sb + ccy * cb
    return (sx.reshape(-1).copy(), sy.reshape(-1).copy(),
            ux.reshape(-1).copy(), uy.reshape(-1).copy())


# ------------------------------------------------------------------------- phantoms

def _inside(el: Ellipse, x, y):
    c, s = math.cos(el.phi), math.sin(el.phi)
    u = (x - el.cx) * c + (y - el.cy) * s
    w = -(x - el.cx) * s + (y - el.cy) * c
    return (u / el.a) ** 2 + (w / el.b) ** 2 < 1.0


def paint(ellipses: Sequence[Ellipse], x, y):
    """Overwrite-painted phantom value at points (x, y): the last covering ellipse wins."""
    out = np.zeros(np.broadcast(x, y).shape, dtype=np.float64)
    for el in ellipses:
        out = np.where(_inside(el, x, y), el.value, out)
    return out


def rasterize(ellipses: Sequence[Ellipse], g: FanGeometry, ss: int = 4):
    """Ground-truth image: mean of ss x ss sub-pixel samples per pixel."""
    x0, y0 = -g.nx * g.dx / 2.0, -g.ny * g.dy / 2.0
    off = (np.arange(ss) + 0.5) / ss
    xs = x0 + (np.arange(g.nx)[:, None] + off[None, :]).reshape(-1) * g.dx
    ys = y0 + (np.arange(g.ny)[:, None] + off[None, :]).reshape(-1) * g.dy
    X, Y = np.meshgrid(xs, ys)
    img = paint(ellipses, X, Y)
    return img.reshape(g.ny, ss, g.nx, ss).mean(axis=(1, 3))


def line_integrals(ellipses: Sequence[Ellipse], sx, sy, ux, uy, chunk: int = 4096):
    """Exact integral of the overwrite-painted phantom along each ray (float64).

    Each ray's chords through the ellipses split it into intervals; on each interval the
    value is that of the last ellipse covering its midpoint."""
    n = sx.shape[0]
    E = len(ellipses)
    out = np.zeros(n, dtype=np.float64)
    vals = np.array([e.value for e in ellipses] + [0.0])
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        t1 = np.full((hi - lo, E), np.nan)
        t2 = np.full((hi - lo, E), np.nan)
        for k, el in enumerate(ellipses):
            c, s = math.cos(el.phi), math.sin(el.phi)
            qx, qy = sx[lo:hi] - el.cx, sy[lo:hi] - el.cy
            qu, qw = qx * c + qy * s, -qx * s + qy * c
            eu, ew = ux[lo:hi] * c + uy[lo:hi] * s, -ux[lo:hi] * s + uy[lo:hi] * c
            A = eu * eu / el.a ** 2 + ew * ew / el.b ** 2
            B = 2.0 * (qu * eu / el.a ** 2 + qw * ew / el.b ** 2)
            C = qu * qu / el.a ** 2 + qw * qw / el.b ** 2 - 1.0
            disc = B * B - 4.0 * A * C
            ok = disc > 0
            sq = np.sqrt(np.where(ok, disc, 0.0))
            t1[:, k] = np.where(ok, (-B - sq) / (2 * A), np.nan)
            t2[:, k] = np.where(ok, (-B + sq) / (2 * A), np.nan)
        pts = np.sort(np.concatenate([t1, t2], axis=1), axis=1)     # NaN sort last
        a, b = pts[:, :-1], pts[:, 1:]
        mid = 0.5 * (a + b)
        cov = (t1[:, None, :] < mid[:, :, None]) & (mid[:, :, None] < t2[:, None, :])
        idx = np.arange(E)[None, None, :]
        top = np.where(cov, idx, -1).max(axis=2)                   # last covering ellipse
        v = vals[np.where(top >= 0, top, E)]
        seg = np.where(np.isfinite(a) & np.isfinite(b), b - a, 0.0)
        out[lo:hi] = np.sum(np.where(top >= 0, v, 0.0) * seg, axis=1)
    return out


def random_ellipses(rng: np.random.Generator, R: float, n_random: int,
                    body_mu: float = 0.02):
    """Body ellipse plus n_random ellipses (centres in the 0.7R disc)."""
    els = [Ellipse(0.0, 0.0, rng.uniform(0.85, 0.95) * R, rng.uniform(0.85, 0.95) * R,
                   rng.uniform(0.0, np.pi), body_mu)]
    for _ in range(n_random):
        r = 0.7 * R * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2 * np.pi)
        els.append(Ellipse(r * math.cos(ang), r * math.sin(ang),
                           rng.uniform(0.03, 0.3) * R, rng.uniform(0.03, 0.3) * R,
                           rng.uniform(0.0, np.pi), rng.uniform(0.01, 0.03)))
    return els


def add_insert(els: List[Ellipse], cx, cy, radius, contrast):
    """Low-contrast disc: value = underlying value at its centre * (1 + contrast)."""
    under = float(paint(els, np.array(cx), np.array(cy)))
    els.append(Ellipse(cx, cy, radius, radius, 0.0, under * (1.0 + contrast)))


def noisy_sinogram(rng: np.random.Generator, p: np.ndarray, i0: float):
    """Poisson counts ~ I0*exp(-p); y = ln(I0 / max(counts, 1))."""
    counts = rng.poisson(i0 * np.exp(-p))
    return np.log(i0 / np.maximum(counts, 1)).astype(np.float64)


def _finish(case: Case, rng: np.random.Generator, with_truth: bool = True):
    g = case.geom
    sx, sy, ux, uy = fan_rays(g)
    case.p_clean = line_integrals(case.ellipses, sx, sy, ux, uy).reshape(g.n_views, g.n_bins)
    case.y = noisy_sinogram(rng, case.p_clean, case.i0)
    if with_truth:
        case.f_true = rasterize(case.ellipses, g)
    return case


# -------------------------------------------------------------------------- configs

def c1_geometry() -> FanGeometry:
    """128x128, 2 mm pixels, 30 views x 256 bins, SID 1000, SDD 1500 (arc).
    Bin pitch: the fan covers 1.02 x the image half-diagonal."""
    nx = 128
    rdiag = nx * 2.0 / 2.0 * math.sqrt(2.0)
    dbeta = 2.0 * math.asin(1.02 * rdiag / 1000.0) / 256
    return FanGeometry(nx, nx, 2.0, 2.0, 30, 256, dbeta, 0.25, 1000.0, 1500.0, ARC)


def ge_geometry(n: int, pixel: float, n_views: int, n_bins: int = GE_BINS,
                dbeta: Optional[float] = None) -> FanGeometry:
    if dbeta is None:
        dbeta = GE_PITCH / GE_SDD
    return FanGeometry(n, n, pixel, pixel, n_views, n_bins, dbeta, 0.25, GE_SID, GE_SDD, ARC)


def make_c1(seed: int = 1, with_truth: bool = True) -> Case:
    """Plain EPTV, 128^2: 10 ellipses incl. two +-0.5% inserts, I0 = 1e5, 50 iterations."""
    g = c1_geometry()
    rng = np.random.Generator(np.random.PCG64(seed))
    R = g.nx * g.dx / 2.0
    els = random_ellipses(rng, R, 7)
    for sgn in (+1.0, -1.0):
        r = 0.5 * R * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        add_insert(els, r * math.cos(ang), r * math.sin(ang),
                   rng.uniform(0.05, 0.1) * R, sgn * 0.005)
    return _finish(Case("eptv_128x128_30v_256b", g, els, 1e5, 50, seed), rng, with_truth)


def make_c2(seed: int = 2, with_truth: bool = True) -> Case:
    """Plain EPTV, 512^2 at 0.8 mm, 40 views x 888 bins (GE): 30 ellipses + ring of 8
    low-contrast discs (ring radius 120 mm, diameters 2-15 mm, contrast 0.3-1%),
    I0 = 5e4, 100 iterations."""
    g = ge_geometry(512, 0.8, 40)
    rng = np.random.Generator(np.random.PCG64(seed))
    R = g.nx * g.dx / 2.0
    els = random_ellipses(rng, R, 29)
    for k in range(8):
        ang = 2 * np.pi * k / 8
        add_insert(els, 120.0 * math.cos(ang), 120.0 * math.sin(ang),
                   0.5 * (2.0 + 13.0 * k / 7.0), rng.choice([-1.0, 1.0]) * rng.uniform(0.003, 0.01))
    return _finish(Case("eptv_512x512_40v_888b", g, els, 5e4, 100, seed), rng, with_truth)


def make_c3_slice(seed: int, with_truth: bool = True) -> Case:
    """One slice of the batched workload: N in {256, 384, 512} over a 409.6 mm FOV,
    20..60 views, 512..888 bins across the GE fan (0.958 rad), I0 log-uniform [1e4, 1e5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.choice([256, 384, 512]))
    v = int(rng.integers(20, 61))
    b = int(rng.integers(512, 889))
    g = ge_geometry(n, 409.6 / n, v, b, 0.958 / b)
    i0 = float(10.0 ** rng.uniform(4.0, 5.0))
    R = g.nx * g.dx / 2.0
    els = random_ellipses(rng, R, 19)
    for k in range(4):
        ang = 2 * np.pi * k / 4 + rng.uniform(0, 0.5)
        add_insert(els, 100.0 * math.cos(ang), 100.0 * math.sin(ang),
                   rng.uniform(2.0, 8.0), rng.choice([-1.0, 1.0]) * rng.uniform(0.003, 0.01))
    return _finish(Case(f"slice_{n}x{n}_{v}v_{b}b", g, els, i0, 50, seed), rng, with_truth)


def make_c3(n_slices: int = 64, first_seed: int = 100, with_truth: bool = False):
    return [make_c3_slice(first_seed + i, with_truth) for i in range(n_slices)]


def make_c4(seed: int, with_truth: bool = True) -> Case:
    """Learned warm-start workload: 256^2 at 1.6 mm, 30 views x 888 bins (GE), I0 = 5e4."""
    g = ge_geometry(256, 1.6, 30)
    rng = np.random.Generator(np.random.PCG64(seed))
    R = g.nx * g.dx / 2.0
    els = random_ellipses(rng, R, 29)
    for k in range(8):
        ang = 2 * np.pi * k / 8
        add_insert(els, 120.0 * math.cos(ang), 120.0 * math.sin(ang),
                   0.5 * (2.0 + 13.0 * k / 7.0), rng.choice([-1.0, 1.0]) * rng.uniform(0.003, 0.01))
    return _finish(Case("learned_256x256_30v_888b", g, els, 5e4, 50, seed), rng, with_truth)


def random_image(g: FanGeometry, seed: int, kind: str = "uniform") -> np.ndarray:
    """Seeded test image [ny][nx] float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "uniform":
        return rng.uniform(0.0, 0.03, size=(g.ny, g.nx))
    if kind == "normal":
        return rng.standard_normal(size=(g.ny, g.nx))
    raise ValueError(kind)


def random_sino(g: FanGeometry, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=(g.n_views, g.n_bins))


# ----------------------------------------------------------------------- parameters

@dataclasses.dataclass
class EptvParams:
    """Parameter record of one EPTV solve (read by the oracle and by the C-ABI binding).

    The paper fixes none of these numerically except the 90-95% sigma percentile
    (Sec. 2.1); the defaults are this implementation's choices."""
    n_outer: int = 50            # NI, outer iterations (Sec. 2.2)
    cgls_iters: int = 3          # M, CGLS iterations per (P1) (App. I)
    n_gd: int = 10               # GD iterations per (P2)
    lam: float = 2000.0          # lambda of (P2), Eq. (8)
    mu: float = 1.0              # mu of Eq. (2) (reported energy only)
    sigma_q: float = 0.9         # fraction of half-edges below sigma
    sigma_floor: float = 1e-12
    eps: float = 1e-5            # smoothing inside the A3 magnitude (1/mm)
    step_rule: int = 0           # 0 = Armijo, 1 = fixed step t_fixed
    t_fixed: float = 1e-4
    armijo_c: float = 1e-4
    armijo_shrink: float = 0.5
    armijo_grow: float = 2.0
    max_trials: int = 4
    t_max: float = 0.0           # <= 0: 1/lambda
    t_init: float = 0.0          # <= 0: 1/lambda
    weights_mode: int = 0        # 0 = EPTV (Eq. 5), 1 = plain TV (w = 1), 2 = learned prior
    prior_iters: int = 0         # outer iterations that use the prior weights

    @property
    def t_max_eff(self) -> float:
        return self.t_max if self.t_max > 0 else 1.0 / self.lam

    @property
    def t_init_eff(self) -> float:
        return self.t_init if self.t_init > 0 else 1.0 / self.lam


# ------------------------------------------------------------------ 3-D cone beam
#
# Conventions of the cone-beam geometry (3-D extension; the paper is 2-D only):
#   * volume f is [nz][ny][nx], x fastest; voxel (ix, iy, iz) covers
#     [x0 + ix dx, x0 + (ix+1) dx] x [y0 + iy dy, ...] x [z0 + iz dz, ...],
#     x0 = -nx dx / 2, y0 = -ny dy / 2, z0 = -nz dz / 2 (mm);
#   * projections are [n_views][nv][nu] (detector columns u fastest, rows v);
#   * view k: angle theta (angles[k], else 2 pi k / n_views); source at
#     sid (cos theta, sin theta, 0); central direction c = -(cos theta, sin theta, 0);
#     flat detector perpendicular to c at distance sdd from the source, with axes
#     e_u = (-sin theta, cos theta, 0) and e_z = (0, 0, 1);
#   * detector pixel (iu, iv) centre: source + sdd c + u e_u + w e_z with
#     u = (iu - (nu-1)/2 + u_off) du, w = (iv - (nv-1)/2 + v_off) dv;
#   * ray index (k nv + iv) nu + iu; the ray runs from the source to that centre.

@dataclasses.dataclass
class ConeGeometry:
    """Parameter record of a circular cone-beam scan with a flat detector."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    n_views: int
    nu: int
    nv: int
    du: float
    dv: float
    u_off: float = 0.25
    v_off: float = 0.0
    sid: float = 1000.0
    sdd: float = 1500.0
    angles: Optional[np.ndarray] = None

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_rays(self) -> int:
        return self.n_views * self.nu * self.nv

    def view_angles(self) -> np.ndarray:
        if self.angles is not None:
            a = np.asarray(self.angles, dtype=np.float64)
            assert a.shape == (self.n_views,)
            return a
        return 2.0 * np.pi * np.arange(self.n_views, dtype=np.float64) / self.n_views


def cone_rays(g: ConeGeometry):
    """Source points and unit directions of every ray, float64, ray index (k nv + iv) nu + iu."""
    th = g.view_angles()
    u = (np.arange(g.nu) - (g.nu - 1) / 2.0 + g.u_off) * g.du
    w = (np.arange(g.nv) - (g.nv - 1) / 2.0 + g.v_off) * g.dv
    c, s = np.cos(th)[:, None, None], np.sin(th)[:, None, None]
    U, W = u[None, None, :], w[None, :, None]
    sx, sy = g.sid * c, g.sid * s
    dx = -g.sdd * c - U * s
    dy = -g.sdd * s + U * c
    dz = np.broadcast_to(W, (g.n_views, g.nv, g.nu))
    n = np.sqrt(dx * dx + dy * dy + dz * dz)
    shape = (g.n_views, g.nv, g.nu)
    out = [np.broadcast_to(sx, shape), np.broadcast_to(sy, shape), np.zeros(shape),
           dx / n, dy / n, dz / n]
    return tuple(np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in out)


@dataclasses.dataclass
class Ellipsoid:
    cx: float
    cy: float
    cz: float
    a: float        # semi-axes (mm) along the rotated x', y' and z
    b: float
    c: float
    phi: float      # rotation about z (rad)
    value: float    # attenuation (1/mm), overwrites what was painted before


def _inside3(el: Ellipsoid, x, y, z):
    cs, sn = math.cos(el.phi), math.sin(el.phi)
    u = (x - el.cx) * cs + (y - el.cy) * sn
    w = -(x - el.cx) * sn + (y - el.cy) * cs
    return (u / el.a) ** 2 + (w / el.b) ** 2 + ((z - el.cz) / el.c) ** 2 < 1.0


def paint3(ellipsoids: Sequence[Ellipsoid], x, y, z):
    out = np.zeros(np.broadcast(x, y, z).shape, dtype=np.float64)
    for el in ellipsoids:
        out = np.where(_inside3(el, x, y, z), el.value, out)
    return out


def random_ellipsoids(rng: np.random.Generator, R: float, H: float, n_random: int, body_mu: float = 0.02):
    """Body ellipsoid (semi-axes 0.85-0.95 R in x, y; 0.85-0.95 H in z) plus n_random
    ellipsoids with centres in the 0.7 R cylinder of half-height 0.7 H."""
    els = [Ellipsoid(0.0, 0.0, 0.0, rng.uniform(0.85, 0.95) * R, rng.uniform(0.85, 0.95) * R,
                     rng.uniform(0.85, 0.95) * H, rng.uniform(0.0, np.pi), body_mu)]
    for _ in range(n_random):
        r = 0.7 * R * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2 * np.pi)
        els.append(Ellipsoid(r * math.cos(ang), r * math.sin(ang), rng.uniform(-0.7, 0.7) * H,
                             rng.uniform(0.03, 0.3) * R, rng.uniform(0.03, 0.3) * R,
                             rng.uniform(0.03, 0.3) * H, rng.uniform(0.0, np.pi), rng.uniform(0.01, 0.03)))
    return els


def add_sphere(els: List[Ellipsoid], cx, cy, cz, radius, contrast):
    """Low-contrast sphere: value = underlying value at its centre * (1 + contrast)."""
    under = float(paint3(els, np.array(cx), np.array(cy), np.array(cz)))
    els.append(Ellipsoid(cx, cy, cz, radius, radius, radius, 0.0, under * (1.0 + contrast)))


def line_integrals3(ellipsoids: Sequence[Ellipsoid], sx, sy, sz, ux, uy, uz, chunk: int = 8192):
    """Exact integral of the overwrite-painted ellipsoid phantom along each ray (float64):
    each ray's chords cut it into intervals; an interval carries the value of the last
    ellipsoid covering its midpoint."""
    n = sx.shape[0]
    E = len(ellipsoids)
    out = np.zeros(n, dtype=np.float64)
    vals = np.array([e.value for e in ellipsoids] + [0.0])
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        t1 = np.full((hi - lo, E), np.nan)
        t2 = np.full((hi - lo, E), np.nan)
        for k, el in enumerate(ellipsoids):
            cs, sn = math.cos(el.phi), math.sin(el.phi)
            qx, qy, qz = sx[lo:hi] - el.cx, sy[lo:hi] - el.cy, sz[lo:hi] - el.cz
            qu, qw = qx * cs + qy * sn, -qx * sn + qy * cs
            eu, ew = ux[lo:hi] * cs + uy[lo:hi] * sn, -ux[lo:hi] * sn + uy[lo:hi] * cs
            ez = uz[lo:hi]
            A = eu * eu / el.a ** 2 + ew * ew / el.b ** 2 + ez * ez / el.c ** 2
            B = 2.0 * (qu * eu / el.a ** 2 + qw * ew / el.b ** 2 + qz * ez / el.c ** 2)
            C = qu * qu / el.a ** 2 + qw * qw / el.b ** 2 + qz * qz / el.c ** 2 - 1.0
            disc = B * B - 4.0 * A * C
            ok = disc > 0
            sq = np.sqrt(np.where(ok, disc, 0.0))
            t1[:, k] = np.where(ok, (-B - sq) / (2 * A), np.nan)
            t2[:, k] = np.where(ok, (-B + sq) / (2 * A), np.nan)
        pts = np.sort(np.concatenate([t1, t2], axis=1), axis=1)
        a, b = pts[:, :-1], pts[:, 1:]
        mid = 0.5 * (a + b)
        cov = (t1[:, None, :] < mid[:, :, None]) & (mid[:, :, None] < t2[:, None, :])
        top = np.where(cov, np.arange(E)[None, None, :], -1).max(axis=2)
        v = vals[np.where(top >= 0, top, E)]
        seg = np.where(np.isfinite(a) & np.isfinite(b), b - a, 0.0)
        out[lo:hi] = np.sum(np.where(top >= 0, v, 0.0) * seg, axis=1)
    return out


def rasterize3(ellipsoids: Sequence[Ellipsoid], g: ConeGeometry, ss: int = 2):
    """Ground-truth volume: mean of ss^3 sub-voxel samples per voxel."""
    off = (np.arange(ss) + 0.5) / ss
    xs = -g.nx * g.dx / 2 + (np.arange(g.nx)[:, None] + off[None, :]).reshape(-1) * g.dx
    ys = -g.ny * g.dy / 2 + (np.arange(g.ny)[:, None] + off[None, :]).reshape(-1) * g.dy
    out = np.empty((g.nz, g.ny, g.nx))
    for iz in range(g.nz):
        zs = -g.nz * g.dz / 2 + (iz + off) * g.dz
        acc = np.zeros((g.ny * ss, g.nx * ss))
        Y, X = np.meshgrid(ys, xs, indexing="ij")
        for z in zs:
            acc += paint3(ellipsoids, X, Y, np.full_like(X, z))
        out[iz] = (acc / ss).reshape(g.ny, ss, g.nx, ss).mean(axis=(1, 3))
    return out


@dataclasses.dataclass
class ConeCase:
    name: str
    geom: ConeGeometry
    ellipsoids: List[Ellipsoid]
    i0: float
    n_outer: int
    seed: int
    y: Optional[np.ndarray] = None
    p_clean: Optional[np.ndarray] = None
    f_true: Optional[np.ndarray] = None


def c5_geometry(scale: int = 1) -> ConeGeometry:
    """256^3 at 1 mm, 120 views over 360 deg, flat 512 x 384 detector at 0.8 mm, SID 1000,
    SDD 1500; scale divides the grid and detector counts (and multiplies the pitches) for
    reduced test cases of the same scan."""
    return ConeGeometry(256 // scale, 256 // scale, 256 // scale, 1.0 * scale, 1.0 * scale, 1.0 * scale,
                        120 // scale if scale > 1 else 120, 512 // scale, 384 // scale, 0.8 * scale,
                        0.8 * scale)


def c5_ellipsoids(seed: int, g: ConeGeometry):
    """Ellipsoid phantom of the cone-beam workload: body + 19 ellipsoids + a ring of 6
    low-contrast spheres (radii 2-8 mm, contrast 0.5-1 %) in the mid plane."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = min(g.nx * g.dx, g.ny * g.dy) / 2.0
    H = g.nz * g.dz / 2.0
    els = random_ellipsoids(rng, R, H, 19)
    for k in range(6):
        ang = 2 * np.pi * k / 6
        add_sphere(els, 0.45 * R * math.cos(ang), 0.45 * R * math.sin(ang), 0.0,
                   2.0 + 6.0 * k / 5.0, rng.choice([-1.0, 1.0]) * rng.uniform(0.005, 0.01))
    return els, rng


def make_c5(seed: int = 5, scale: int = 1, with_truth: bool = True, with_sinogram: bool = True) -> ConeCase:
    """Cone-beam workload: the phantom of c5_ellipsoids, exact line integrals, Poisson
    noise I0 = 5e4, 50 iterations.  (The full-size sinogram has 23.6 M rays; the host
    line integrals are meant for the reduced scales.)"""
    g = c5_geometry(scale)
    els, rng = c5_ellipsoids(seed, g)
    case = ConeCase(f"cone_{g.nx}x{g.ny}x{g.nz}_{g.n_views}v_{g.nu}x{g.nv}", g, els, 5e4, 50, seed)
    if with_sinogram:
        case.p_clean = line_integrals3(els, *cone_rays(g)).reshape(g.n_views, g.nv, g.nu)
        case.y = noisy_sinogram(rng, case.p_clean, case.i0)
    if with_truth:
        case.f_true = rasterize3(els, g)
    return case
