"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(chord lengths, ramp magnitudes, corner values), brute force on tiny inputs (per-pixel
clipping, dense least squares), invariants (adjoint identity, CGLS monotonicity,
Armijo sufficient decrease) and library routines (partition for the order statistic).
"""
import math

import numpy as np
import pytest

from oracle import eptv_oracle as O
from paper_1009_2288_b300 import inputs as I


def _box_chord(nx, ny, dx, dy, sx, sy, ux, uy):
    """Length of the line s + t u (t >= 0) inside the image rectangle (slab clipping)."""
    lo = [-nx * dx / 2, -ny * dy / 2]
    hi = [nx * dx / 2, ny * dy / 2]
    t0, t1 = 0.0, math.inf
    for s, u, a, b in ((sx, ux, lo[0], hi[0]), (sy, uy, lo[1], hi[1])):
        if u == 0.0:
            if not (a < s < b):
                return 0.0
            continue
        ta, tb = (a - s) / u, (b - s) / u
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0)


def _pixel_clip(x0, x1, y0, y1, sx, sy, ux, uy):
    """Liang-Barsky clip of the line against one pixel rectangle."""
    t0, t1 = -math.inf, math.inf
    for s, u, a, b in ((sx, ux, x0, x1), (sy, uy, y0, y1)):
        if u == 0.0:
            if not (a <= s <= b):
                return 0.0
            continue
        ta, tb = (a - s) / u, (b - s) / u
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    t0 = max(t0, 0.0)
    return max(0.0, t1 - t0)


# ---------------------------------------------------------------- geometry (Sec. 3)

def test_geometry_sources_and_fan_angles():
    g = I.FanGeometry(32, 32, 1.0, 1.0, 7, 9, 0.01, 0.0, 541.0, 949.075, I.ARC)
    sx, sy, ux, uy = O.rays(g)
    assert np.allclose(np.hypot(sx, sy), 541.0, rtol=0, atol=1e-12)
    assert np.allclose(np.hypot(ux, uy), 1.0, atol=1e-15)
    for v in range(g.n_views):
        th = 2 * np.pi * v / g.n_views
        for k in range(g.n_bins):
            r = v * g.n_bins + k
            # angle between the ray and the central ray -(cos th, sin th), signed (+ = ccw)
            cx, cy = -math.cos(th), -math.sin(th)
            beta = math.atan2(cx * uy[r] - cy * ux[r], cx * ux[r] + cy * uy[r])
            assert beta == pytest.approx((k - 4) * 0.01, abs=1e-14)
    # central bin (offset 0, odd count) passes through the isocentre
    for v in range(g.n_views):
        r = v * g.n_bins + 4
        assert abs(sx[r] * uy[r] - sy[r] * ux[r]) < 1e-12


def test_geometry_flat_detector_and_offset():
    g = I.FanGeometry(16, 16, 1.0, 1.0, 3, 6, 0.002, 0.25, 1000.0, 1500.0, I.FLAT)
    sx, sy, ux, uy = O.rays(g)
    for k in range(6):
        cx, cy = -1.0, 0.0                       # view 0
        tanb = (cx * uy[k] - cy * ux[k]) / (cx * ux[k] + cy * uy[k])
        assert tanb == pytest.approx((k - 2.5 + 0.25) * 0.002, abs=1e-15)


def test_oracle_rays_agree_with_data_generator_rays():
    g = I.c1_geometry()
    a = O.rays(g)
    b = I.fan_rays(g)
    for u, w in zip(a, b):
        assert np.allclose(u, w, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- P (Eq. 1, Siddon)

@pytest.mark.parametrize("nx,ny,dx,dy", [(8, 8, 1.0, 1.0), (7, 5, 0.8, 1.3), (64, 48, 2.0, 2.0)])
def test_row_sum_is_chord_through_image(nx, ny, dx, dy):
    """sum_j p_ij = length of ray i inside the image square (closed form)."""
    rng = np.random.Generator(np.random.PCG64(5))
    ones = np.ones(nx * ny)
    for _ in range(200):
        ang = rng.uniform(0, 2 * np.pi)
        sx, sy = 3 * nx * dx * math.cos(ang), 3 * ny * dy * math.sin(ang)
        tgt = (rng.uniform(-0.6, 0.6) * nx * dx, rng.uniform(-0.6, 0.6) * ny * dy)
        ux, uy = tgt[0] - sx, tgt[1] - sy
        n = math.hypot(ux, uy)
        ux, uy = ux / n, uy / n
        got = O.project_rays(nx, ny, dx, dy, [sx], [sy], [ux], [uy], ones)[0]
        want = _box_chord(nx, ny, dx, dy, sx, sy, ux, uy)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_axis_aligned_rays_give_pixel_pitch():
    nx, ny, dx, dy = 6, 4, 0.7, 1.1
    x0, y0 = -nx * dx / 2, -ny * dy / 2
    for j in range(ny):   # horizontal rays through pixel-row centres
        pix, ln = O.ray_row(nx, ny, dx, dy, -100.0, y0 + (j + 0.5) * dy, 1.0, 0.0)
        assert sorted(pix.tolist()) == [j * nx + i for i in range(nx)]
        assert np.allclose(ln, dx, rtol=0, atol=1e-12)
    for i in range(nx):   # vertical rays, pointing down
        pix, ln = O.ray_row(nx, ny, dx, dy, x0 + (i + 0.5) * dx, 100.0, 0.0, -1.0)
        assert sorted(pix.tolist()) == [j * nx + i for j in range(ny)]
        assert np.allclose(ln, dy, rtol=0, atol=1e-12)


@pytest.mark.parametrize("nx,ny,dx,dy", [(4, 4, 1.0, 1.0), (5, 3, 0.8, 1.3)])
def test_brute_force_pixel_clipping(nx, ny, dx, dy):
    """Every p_ij equals the clip of ray i against pixel j alone."""
    rng = np.random.Generator(np.random.PCG64(11))
    x0, y0 = -nx * dx / 2, -ny * dy / 2
    for _ in range(300):
        ang = rng.uniform(0, 2 * np.pi)
        sx, sy = 10 * math.cos(ang), 10 * math.sin(ang)
        tx, ty = rng.uniform(x0, -x0), rng.uniform(y0, -y0)
        ux, uy = tx - sx, ty - sy
        n = math.hypot(ux, uy)
        ux, uy = ux / n, uy / n
        pix, ln = O.ray_row(nx, ny, dx, dy, sx, sy, ux, uy)
        dense = np.zeros(nx * ny)
        np.add.at(dense, pix, ln)
        want = np.array([_pixel_clip(x0 + i * dx, x0 + (i + 1) * dx, y0 + j * dy,
                                     y0 + (j + 1) * dy, sx, sy, ux, uy)
                         for j in range(ny) for i in range(nx)])
        assert np.allclose(dense, want, rtol=0, atol=1e-12)


def test_disk_projection_converges_to_chord():
    """P 1_disk -> 2 sqrt(R^2 - d^2) for a finely rasterised uniform disk."""
    R = 40.0
    n, d = 256, 0.5
    g = I.FanGeometry(n, n, d, d, 3, 64, 0.0016, 0.25, 500.0, 800.0, I.ARC)
    disk = I.rasterize([I.Ellipse(0, 0, R, R, 0.0, 1.0)], g, ss=8)
    y = O.Operator(g).project(disk).ravel()
    sx, sy, ux, uy = O.rays(g)
    dist = np.abs(sx * uy - sy * ux)
    want = 2 * np.sqrt(np.maximum(R * R - dist * dist, 0.0))
    inner = dist < 0.9 * R
    assert np.max(np.abs(y - want)[inner]) < 0.02 * 2 * R
    assert np.mean(np.abs(y - want)[inner]) < 0.002 * 2 * R


# ---------------------------------------------------------------- P^T (adjoint, Eq. A3)

def test_adjoint_identity_fp64():
    g = I.c1_geometry()
    op = O.Operator(g)
    for seed in range(3):
        x = I.random_image(g, 100 + seed, "normal")
        y = I.random_sino(g, 200 + seed)
        px = op.project(x)
        lhs, rhs = float(np.sum(px * y)), float(np.sum(x * op.backproject(y)))
        assert abs(lhs - rhs) / (np.linalg.norm(px) * np.linalg.norm(y)) < 1e-13


def test_backprojection_is_dense_transpose():
    g = I.FanGeometry(6, 5, 1.0, 1.2, 4, 7, 0.03, 0.25, 30.0, 60.0, I.ARC)
    op = O.Operator(g)
    P = np.stack([op.project(np.eye(30)[j].reshape(5, 6)).ravel() for j in range(30)], 1)
    PT = np.stack([op.backproject(np.eye(28)[i].reshape(4, 7)).ravel() for i in range(28)], 1)
    assert np.array_equal(PT, P.T)
    assert np.count_nonzero(P) > 20


# ---------------------------------------------------------------- CGLS (App. I)

def _tiny():
    g = I.FanGeometry(16, 16, 1.0, 1.0, 12, 32, 0.045, 0.25, 60.0, 100.0, I.ARC)
    return g, O.Operator(g)


def test_cgls_residual_non_increasing():
    g, op = _tiny()
    rng = np.random.Generator(np.random.PCG64(3))
    y = op.project(rng.uniform(0, 1, (16, 16))) + 0.01 * rng.standard_normal((12, 32))
    log = []
    O.cgls(op, y, np.zeros((16, 16)), 40, log)
    rr = [e["rr"] for e in log]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(rr, rr[1:]))


def test_cgls_first_step_is_exact_line_search():
    g, op = _tiny()
    rng = np.random.Generator(np.random.PCG64(4))
    P = np.stack([op.project(np.eye(256)[j].reshape(16, 16)).ravel() for j in range(256)], 1)
    y = rng.standard_normal(12 * 32)
    u0 = rng.uniform(0, 1, 256)
    r0 = y - P @ u0
    s0 = P.T @ r0
    q = P @ s0
    a_star = float(q @ r0) / float(q @ q)    # argmin_a |P (u0 + a s0) - y|
    u1 = O.cgls(op, y.reshape(12, 32), u0.reshape(16, 16), 1).ravel()
    assert np.allclose(u1, u0 + a_star * s0, rtol=1e-12, atol=1e-12)


def test_cgls_converges_to_min_norm_least_squares():
    g, op = _tiny()
    rng = np.random.Generator(np.random.PCG64(6))
    P = np.stack([op.project(np.eye(256)[j].reshape(16, 16)).ravel() for j in range(256)], 1)
    y = rng.standard_normal(12 * 32)
    u0 = rng.uniform(0, 1, 256)
    want = u0 + np.linalg.lstsq(P, y - P @ u0, rcond=None)[0]
    got = O.cgls(op, y.reshape(12, 32), u0.reshape(16, 16), 400).ravel()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-6


# ------------------------------------------------------ EPTV stencil (Eqs. A2, A3, 5, 9)

def test_half_edge_magnitude_on_ramp():
    """For f = a i + b j, interior T = sqrt(eps^2 + a^2 + b^2) (pins the 1/2 factors)."""
    a, b, eps = 0.3, -0.7, 1e-3
    j, i = np.mgrid[0:9, 0:11]
    f = a * i + b * j + 5.0
    Dx, Tx, Dy, Ty = O.half_edges(f, eps)
    want = math.sqrt(eps * eps + a * a + b * b)
    assert np.allclose(Tx[1:-1, 1:-1], want, rtol=1e-14)
    assert np.allclose(Ty[1:-1, 1:-1], want, rtol=1e-14)
    assert np.allclose(Dx[:, 1:-1], a) and np.allclose(Dy[1:-1, :], b)


def test_half_edge_magnitude_zero_boundary_corner():
    """A single pixel h at (0, 0), zero outside: hand-computed magnitudes."""
    h, eps = 2.0, 1e-3
    f = np.zeros((4, 5))
    f[0, 0] = h
    Dx, Tx, Dy, Ty = O.half_edges(f, eps)
    # x half-edge between the outside and pixel (0,0): D = h, cross terms +-h/2
    assert Dx[0, 0] == h
    assert Tx[0, 0] == pytest.approx(math.sqrt(eps ** 2 + h * h + 0.25 * h * h))
    # x half-edge between (0,0) and (1,0): D = -h, same cross terms
    assert Dx[0, 1] == -h
    assert Tx[0, 1] == pytest.approx(math.sqrt(eps ** 2 + 1.25 * h * h))
    # x half-edge between (0,1) and (1,1): D = 0, upper-neighbour average h/2 below it
    assert Tx[1, 1] == pytest.approx(math.sqrt(eps ** 2 + 0.5 * 0.25 * h * h))
    # far away: T = eps
    assert Tx[3, 4] == pytest.approx(eps) and Ty[3, 4] == pytest.approx(eps)


def _lagged_energy_terms(f, eps):
    """Primary differences and frozen cross-term sums C_e per half-edge, by loops."""
    ny, nx = f.shape

    def F(i, j):
        return f[j, i] if (0 <= i < nx and 0 <= j < ny) else 0.0
    ex, ey = [], []
    for j in range(ny):
        for e in range(nx + 1):            # between pixels e-1 and e
            i = e - 1
            m = [0.5 * (F(i, l) + F(i + 1, l)) for l in (j - 1, j, j + 1)]
            ex.append(((i, j), (i + 1, j), 0.5 * (m[2] - m[1]) ** 2 + 0.5 * (m[1] - m[0]) ** 2))
    for e in range(ny + 1):
        for i in range(nx):
            j = e - 1
            m = [0.5 * (F(l, j) + F(l, j + 1)) for l in (i - 1, i, i + 1)]
            ey.append(((i, j), (i, j + 1), 0.5 * (m[2] - m[1]) ** 2 + 0.5 * (m[1] - m[0]) ** 2))
    return ex, ey


def test_a2_equals_derivative_of_lagged_energy():
    """Eq. (A2) is the gradient of sum_e w_e sqrt(eps^2 + D_e(f)^2 + C_e) with w and the
    cross terms C_e frozen at f (lagged diffusivity), checked by central differences."""
    rng = np.random.Generator(np.random.PCG64(8))
    ny, nx, eps, lam = 5, 6, 1e-2, 3.0
    f = rng.uniform(0, 1, (ny, nx))
    v = rng.uniform(0, 1, (ny, nx))
    _, Tx, _, Ty = O.half_edges(f, eps)
    sigma = float(np.median(np.concatenate([Tx.ravel(), Ty.ravel()])))
    g, wx, wy, _ = O.p2_gradient(f, v, lam, eps, sigma)
    ex, ey = _lagged_energy_terms(f, eps)
    w = np.concatenate([wx.ravel(), wy.ravel()])

    def F(fp, i, j):
        return fp[j, i] if (0 <= i < nx and 0 <= j < ny) else 0.0

    def energy(fp):
        E = 0.5 * lam * float(np.sum((fp - v) ** 2))
        for k, (a, b, C) in enumerate(ex + ey):
            D = F(fp, *b) - F(fp, *a)
            E += w[k] * math.sqrt(eps * eps + D * D + C)
        return E

    h = 1e-6
    fd = np.zeros_like(f)
    for j in range(ny):
        for i in range(nx):
            fp, fm = f.copy(), f.copy()
            fp[j, i] += h
            fm[j, i] -= h
            fd[j, i] = (energy(fp) - energy(fm)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-7)
    # and the cross terms frozen at f reproduce the A3 magnitude itself
    T_loop = np.array([math.sqrt(eps ** 2 + (F(f, *b) - F(f, *a)) ** 2 + C) for a, b, C in ex + ey])
    assert np.allclose(T_loop, np.concatenate([Tx.ravel(), Ty.ravel()]), rtol=1e-14)


def test_constant_image_interior_gradient_is_fidelity_only():
    f = np.full((12, 12), 0.02)
    v = np.random.Generator(np.random.PCG64(1)).uniform(0, 0.03, (12, 12))
    g, _, _, _ = O.p2_gradient(f, v, 7.0, 1e-5, 1e-3)
    assert np.allclose(g[2:-2, 2:-2], 7.0 * (f - v)[2:-2, 2:-2], rtol=0, atol=1e-15)


def test_tv_special_case_step_is_textbook_sign_gradient():
    """w = 1, eps -> 0, step along x: delta J = -1 left of the jump, +1 right of it."""
    f = np.zeros((10, 12))
    f[:, 6:] = 1.0
    g, _, _, _ = O.p2_gradient(f, f, 1.0, 1e-12, 1.0, mode=O.ONE)
    assert np.allclose(g[3:7, 5], -1.0, atol=1e-9)
    assert np.allclose(g[3:7, 6], 1.0, atol=1e-9)
    assert np.allclose(g[3:7, 2:4], 0.0, atol=1e-9)


def test_weights_in_unit_interval_and_value_at_sigma():
    rng = np.random.Generator(np.random.PCG64(2))
    T = rng.uniform(1e-6, 1.0, 1000)
    w = O.edge_weights(T, 0.3)
    assert np.all(w > 0) and np.all(w <= 1)
    assert O.edge_weights(np.array([0.3]), 0.3)[0] == pytest.approx(math.exp(-1.0), rel=1e-15)


# ---------------------------------------------------------------- sigma (Sec. 2.1)

@pytest.mark.parametrize("q", [0.9, 0.95, 0.5, 0.0, 1.0])
def test_sigma_is_order_statistic(q):
    rng = np.random.Generator(np.random.PCG64(9))
    f = rng.uniform(0, 0.03, (17, 23))
    _, Tx, _, Ty = O.half_edges(f, 1e-5)
    pool = np.concatenate([Tx.ravel(), Ty.ravel()])
    n = pool.size
    k = min(max(math.ceil(q * n), 1), n)
    s = O.select_sigma(Tx, Ty, q)
    assert s == np.partition(pool, k - 1)[k - 1]
    assert np.count_nonzero(pool <= s) >= k and np.count_nonzero(pool < s) < k


# ---------------------------------------------------------------- (P2) GD + Armijo

def _armijo_case():
    """A 20 x 20 (P2) input with an edge (so that the weights vary) on which the default
    line search backtracks and then accepts, fails, hits the t_max cap and grows the step
    again after a short accepted one."""
    rng = np.random.Generator(np.random.PCG64(13))
    v = rng.uniform(0, 0.03, (20, 20))
    v[:, 10:] += 0.02
    return v, I.EptvParams(n_gd=12, max_trials=6)


def test_armijo_accepts_first_passing_trial_and_replays_to_the_result():
    """Sec. 2.2 solves (P2) by gradient descent with Armijo's inexact line search: the
    search tries t0, t0 s, t0 s^2, ... and takes the FIRST trial that decreases the
    frozen-weight energy by at least c t |g|^2.  Every accepted step passes, every longer
    trial before it fails (so a later, shorter passing trial is never taken), a failed
    search tried max_trials steps that all fail, and replaying the accepted steps from v
    reproduces the oracle's image."""
    v, p = _armijo_case()
    fo, st = O.p2_solve(v, p, p.t_init_eff)
    _, Tvx, _, Tvy = O.half_edges(v, p.eps)
    assert st.sigma == O.select_sigma(Tvx, Tvy, p.sigma_q)
    assert len(st.steps) == len(st.trials) == p.n_gd
    assert any(t > 0 and len(tr) > 1 for t, tr in zip(st.steps, st.trials))   # backtracked, then accepted
    assert any(t == 0 for t in st.steps)                                       # a failed search
    f = v.copy()
    for t, tried in zip(st.steps, st.trials):
        g, wx, wy, E0 = O.p2_gradient(f, v, p.lam, p.eps, st.sigma)
        gg = float(np.sum(g * g))

        def passes(tt):
            return O.p2_energy_frozen(f - tt * g, v, p.lam, p.eps, wx, wy) <= E0 - p.armijo_c * tt * gg
        ts = [tt for tt, _ in tried]
        for a, b in zip(ts, ts[1:]):                       # trials shrink by the factor s
            assert b == pytest.approx(a * p.armijo_shrink, rel=1e-15)
        if t > 0:
            assert ts[-1] == t and passes(t)
            assert not any(passes(tt) for tt in ts[:-1])
            f = f - t * g
        else:
            assert len(ts) == p.max_trials and not any(passes(tt) for tt in ts)
    assert np.array_equal(f, fo)


def test_armijo_first_trial_grows_from_the_previous_step():
    """The first trial of each search is min(grow t_prev, t_max) (the reading of the
    silent constants, grow = 2, t_max = 1/lambda): t_prev is the step accepted by the
    previous GD iteration (or the initial 1/lambda), and after a failed search the next
    search continues just below that search's last (shortest) trial."""
    v, p = _armijo_case()
    t_start = p.t_init_eff
    _, st = O.p2_solve(v, p, t_start)
    t_prev = t_start
    grew = capped = after_fail = 0
    for n, (t, tried) in enumerate(zip(st.steps, st.trials)):
        t0 = tried[0][0]
        assert t0 == pytest.approx(min(2.0 * t_prev, 1.0 / p.lam), rel=1e-15)
        if n > 0 and st.steps[n - 1] > 0:
            grew += t0 == pytest.approx(2.0 * st.steps[n - 1], rel=1e-15)
        capped += t0 == 1.0 / p.lam
        if n > 0 and st.steps[n - 1] == 0:
            assert t0 == pytest.approx(st.trials[n - 1][-1][0] * p.armijo_shrink, rel=1e-15)
            after_fail += 1
        t_prev = t if t > 0 else tried[-1][0] * p.armijo_shrink / 2.0
    assert st.t_prev == pytest.approx(t_prev, rel=1e-15)
    assert grew >= 1 and capped >= 1 and after_fail >= 1     # every branch of the rule is met


def test_plain_tv_p2_energy_monotone():
    rng = np.random.Generator(np.random.PCG64(13))
    v = rng.uniform(0, 0.03, (24, 24))
    p = I.EptvParams(n_gd=15, weights_mode=O.ONE)
    _, st = O.p2_solve(v, p, p.t_init_eff)
    E = st.energies
    assert all(b <= a for a, b in zip(E, E[1:]))
    assert E[-1] < E[0]


# ---------------------------------------------------------------- outer loop, Eq. (2)

def test_report_energy_of_zero_image_closed_form():
    g = I.FanGeometry(8, 6, 1.0, 1.0, 3, 5, 0.05, 0.25, 30.0, 50.0, I.ARC)
    op = O.Operator(g)
    y = I.random_sino(g, 3)
    p = I.EptvParams(mu=2.5, eps=1e-3)
    sigma = 4e-3
    n_edges = 6 * 9 + 7 * 8
    want = 0.5 * 2.5 * float(np.sum(y * y)) + n_edges * 1e-3 * math.exp(-(1e-3 / sigma) ** 2)
    assert O.report_energy(op, np.zeros((6, 8)), y, p, sigma) == pytest.approx(want, rel=1e-14)


def test_reconstruct_positive_and_better_than_zero(c1_case):
    op = O.Operator(c1_case.geom)
    p = I.EptvParams(n_outer=4)
    f = O.reconstruct(op, c1_case.y, p)
    assert np.all(f >= 0)
    e = np.sum((f - c1_case.f_true) ** 2) / np.sum(c1_case.f_true ** 2)
    assert e < 0.05


def _dense(op, g):
    n = g.ny * g.nx
    return np.stack([op.project(np.eye(n)[j].reshape(g.ny, g.nx)).ravel() for j in range(n)], 1)


def test_outer_iteration_restarts_cgls_at_the_current_image():
    """Sec. 2.2, step 1 with App. I: each outer iteration runs CGLS started at the current
    (clamped) image f^(k), not at 0.  With M = 1 the CGLS step is the exact line search
    along s = P^T (y - P f^(k)) (a closed form on the dense matrix); one fixed (P2) step
    is v - t dJ(v) (at f = v the fidelity part of Eq. 9 vanishes); step 3 clamps.  Two
    outer iterations from a non-zero warm start, composed by hand, equal the oracle's
    reconstruction; starting CGLS at 0 instead moves the result by a large margin."""
    g = I.FanGeometry(12, 10, 1.0, 1.0, 9, 24, 0.05, 0.25, 40.0, 70.0, I.ARC)
    op = O.Operator(g)
    P = _dense(op, g)
    rng = np.random.Generator(np.random.PCG64(31))
    truth = rng.uniform(0, 0.03, (g.ny, g.nx))
    y = (P @ truth.ravel()).reshape(g.n_views, g.n_bins) + 1e-3 * rng.standard_normal((g.n_views, g.n_bins))
    f0 = rng.uniform(-0.01, 0.05, (g.ny, g.nx))       # warm start, clamped on entry
    p = I.EptvParams(cgls_iters=1, n_gd=1, step_rule=O.FIXED, t_fixed=2e-4, lam=50.0)

    def by_hand(fk):
        r0 = y.ravel() - P @ fk.ravel()
        s0 = P.T @ r0
        q = P @ s0
        a = float(q @ r0) / float(q @ q)
        v = fk + (a * s0).reshape(fk.shape)
        _, Tx, _, Ty = O.half_edges(v, p.eps)
        sigma = O.select_sigma(Tx, Ty, p.sigma_q)
        dJ, _, _, _ = O.p2_gradient(v, v, p.lam, p.eps, sigma)
        return np.maximum(v - p.t_fixed * dJ, 0.0)

    f1 = by_hand(np.maximum(f0, 0.0))
    f2 = by_hand(f1)
    got = O.reconstruct(op, y, p, f0=f0, n_outer=2)
    assert np.allclose(got, f2, rtol=1e-10, atol=1e-14)
    # start-point sensitivity: the same composition with CGLS from 0 is far away
    r0 = y.ravel()
    s0 = P.T @ r0
    q = P @ s0
    v0 = ((float(q @ r0) / float(q @ q)) * s0).reshape(g.ny, g.nx)
    assert np.linalg.norm(v0 - f1) > 0.05 * np.linalg.norm(f1)


def test_outer_loop_carries_the_armijo_step_across_iterations():
    """Default solver (M = 3, Armijo): each outer iteration is CGLS_M from the clamped
    f^(k), then (P2) started at v with the previous (P2) solve's last step t_prev, then the
    clamp; the first (P2) starts from t_prev = 1/lambda."""
    g = I.FanGeometry(16, 16, 1.0, 1.0, 12, 32, 0.045, 0.25, 60.0, 100.0, I.ARC)
    op = O.Operator(g)
    rng = np.random.Generator(np.random.PCG64(32))
    truth = np.zeros((16, 16))
    truth[4:12, 3:9] = 0.02
    truth[6:10, 9:13] = 0.035
    y = op.project(truth) + 2e-3 * rng.standard_normal((12, 32))
    p = I.EptvParams(n_gd=6, lam=200.0)
    f = np.zeros((16, 16))
    t_prev = 1.0 / p.lam
    lens = []
    for _ in range(3):
        v = O.cgls(op, y, f, 3)
        f, st = O.p2_solve(v, p, t_prev)
        lens.append(st.trials[0][0][0])
        t_prev = st.t_prev
        f = np.maximum(f, 0.0)
    log = O.ReconLog()
    got = O.reconstruct(op, y, p, n_outer=3, log=log)
    assert np.array_equal(got, f)
    assert log.t_prev == t_prev
    assert [tr[0][0][0] for tr in log.trials] == lens


def test_prior_edge_weights_hand_example():
    w = np.array([[0.2, 0.6], [1.0, 0.4]])
    wx, wy = O.prior_edge_weights(w)
    assert np.allclose(wx, [[0.2, 0.4, 0.6], [1.0, 0.7, 0.4]])
    assert np.allclose(wy, [[0.2, 0.6], [0.6, 0.5], [1.0, 0.4]])


# ---------------------------------------------------------------- synthetic inputs

def test_analytic_disk_line_integrals():
    g = I.c1_geometry()
    sx, sy, ux, uy = I.fan_rays(g)
    p = I.line_integrals([I.Ellipse(10.0, -5.0, 30.0, 30.0, 0.3, 0.02)], sx, sy, ux, uy)
    d = np.abs((sx - 10.0) * uy - (sy + 5.0) * ux)
    want = 0.02 * 2 * np.sqrt(np.maximum(900.0 - d * d, 0.0))
    assert np.allclose(p, want, rtol=0, atol=1e-10)     # near-tangent rays amplify rounding


def test_overwrite_painting_along_ray():
    # disk 0.02 radius 50 with a concentric 0.03 disk radius 20 painted over it
    els = [I.Ellipse(0, 0, 50, 50, 0, 0.02), I.Ellipse(0, 0, 20, 20, 0, 0.03)]
    p = I.line_integrals(els, np.array([-200.0]), np.array([0.0]), np.array([1.0]), np.array([0.0]))
    assert p[0] == pytest.approx(0.02 * 60 + 0.03 * 40, rel=1e-14)


# ------------------------------------------------------------------ Eq. (11)

def _blobs(g):
    x0 = (np.arange(g.nx) + 0.5) * g.dx - g.nx * g.dx / 2
    y0 = (np.arange(g.ny) + 0.5) * g.dy - g.ny * g.dy / 2
    X, Y = np.meshgrid(x0, y0)
    R = min(g.nx * g.dx, g.ny * g.dy) / 2
    f = np.exp(-((X - 0.5 * R) ** 2 + (Y + 0.3 * R) ** 2) / (0.25 * R) ** 2)
    h = np.exp(-((X + 0.4 * R) ** 2 + (Y - 0.2 * R) ** 2) / (0.35 * R) ** 2)
    return f, h


@pytest.mark.parametrize("det", [I.ARC, I.FLAT])
def test_eq11_adjoint_identity_wide_fan(det):
    """App. III derives Eq. (11) as the adjoint of P: <P f, y> = <f, P^T y> (A3) up to the
    discretisation.  On a wide fan (short source distance, |tan beta| up to 0.65) with
    smooth f and y = P h the identity holds to 1e-4 with the exact Siddon P.  This pins
    the du dv / dbeta factor, the 1/l weight, the sign of beta* and, for the flat
    detector, the (1 + t^2) weight of the reading (without it the mismatch is 2.7e-3)."""
    if det == I.ARC:
        g = I.FanGeometry(64, 64, 1.0, 1.0, 180, 400, 2 * math.atan(0.65) / 400, 0.25, 100.0, 150.0, det)
    else:
        g = I.FanGeometry(64, 64, 1.0, 1.0, 180, 400, 1.3 / 400, 0.25, 100.0, 150.0, det)
    op = O.Operator(g)
    f, h = _blobs(g)
    ys = op.project(h)
    lhs = float(np.sum(op.project(f) * ys))
    rhs = float(np.sum(f * O.backproject_eq11(g, ys)))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_eq11_adjoint_within_the_papers_bound_on_noise():
    """The paper reports (App. III) that its operator satisfies (A3) within 1 %: random,
    non-smooth images and sinograms on the 128^2 fan-beam workload."""
    g = I.c1_geometry()
    op = O.Operator(g)
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(3):
        f = rng.uniform(0, 1, (g.ny, g.nx))
        ys = rng.uniform(0, 1, (g.n_views, g.n_bins))
        lhs = float(np.sum(op.project(f) * ys))
        rhs = float(np.sum(f * O.backproject_eq11(g, ys)))
        assert abs(lhs - rhs) <= 1e-2 * abs(lhs)


def test_eq11_interpolation_exact_for_linear_sinograms():
    """A sinogram linear in the bin index per view is reproduced exactly by the linear
    interpolation: Eq. (11) equals (du dv / dbeta) sum_v (a_v + b_v u_v*) / l_v at pixels
    whose u* stays inside the detector, with u* from the complex argument of the
    source-to-pixel vector relative to the central ray (an independent route)."""
    g = I.FanGeometry(24, 20, 2.0, 2.0, 7, 301, 0.0022, 0.25, 500.0, 800.0, I.ARC)
    rng = np.random.Generator(np.random.PCG64(12))
    a, b = rng.uniform(-1, 1, g.n_views), rng.uniform(-0.01, 0.01, g.n_views)
    ys = a[:, None] + b[:, None] * np.arange(g.n_bins)[None, :]
    got = O.backproject_eq11(g, ys)
    kc = (g.n_bins - 1) / 2.0 - g.bin_offset
    want = np.zeros((g.ny, g.nx))
    for iy in range(g.ny):
        for ix in range(g.nx):
            p = complex((ix + 0.5) * g.dx - g.nx * g.dx / 2, (iy + 0.5) * g.dy - g.ny * g.dy / 2)
            for v, th in enumerate(g.view_angles()):
                s = g.sid * complex(math.cos(th), math.sin(th))
                z = (p - s) / (-s)                     # relative to the central ray
                u = np.angle(z) / g.dbeta + kc
                assert 0.0 <= u <= g.n_bins - 1
                want[iy, ix] += (a[v] + b[v] * u) / abs(p - s)
    want *= g.dx * g.dy / g.dbeta
    assert np.allclose(got, want, rtol=1e-12, atol=0)


# ------------------------------------------------------------------ Eqs. (12) - (14)

def test_relative_error_closed_form():
    rng = np.random.Generator(np.random.PCG64(21))
    t = rng.uniform(0.5, 1.5, (9, 7))
    assert O.relative_error(1.1 * t, t) == pytest.approx(0.01, rel=1e-12)
    assert O.relative_error(t, t) == 0.0


def test_sobel_gradient_matches_scipy():
    """Interior Sobel derivatives against scipy.ndimage.sobel (the library routine)."""
    from scipy import ndimage
    rng = np.random.Generator(np.random.PCG64(22))
    f = rng.standard_normal((13, 17))
    gx = ndimage.sobel(f, axis=1, mode="constant")
    gy = ndimage.sobel(f, axis=0, mode="constant")
    want = (gx * gx + gy * gy)[1:-1, 1:-1]
    assert np.allclose(O.sobel_gradient2(f)[1:-1, 1:-1], want, rtol=1e-12, atol=1e-12)


def test_sobel_edges_of_a_step():
    """A vertical step of height h: gx = 4h on the two columns beside the step, 0
    elsewhere, so exactly those interior pixels are edges (mean = 8h^2 (ny-2)/((nx-2)(ny-2)))."""
    f = np.zeros((10, 12))
    f[:, 6:] = 3.0
    b = O.sobel_edges(f)
    want = np.zeros_like(b)
    want[1:-1, 5:7] = 1
    assert np.array_equal(b, want)
    assert O.sobel_edges(np.outer(np.ones(10), np.arange(12.0))).sum() == 0   # a ramp has no edges


def test_edge_correlation_against_numpy_corrcoef():
    rng = np.random.Generator(np.random.PCG64(23))
    b = (rng.uniform(size=(20, 30)) < 0.2).astype(np.uint8)
    t = (rng.uniform(size=(20, 30)) < 0.3).astype(np.uint8)
    assert O.edge_correlation(b, t) == pytest.approx(np.corrcoef(b.ravel(), t.ravel())[0, 1], rel=1e-12)
    assert O.edge_correlation(b, b) == pytest.approx(1.0, rel=1e-12)
    assert O.edge_correlation(b, 1 - b) == pytest.approx(-1.0, rel=1e-12)


def test_roi_snr_closed_form():
    """ROI = m + a * (checkerboard of +-1): mean m, variance a^2."""
    f = np.full((16, 16), 7.0)
    cb = np.indices((6, 8)).sum(axis=0) % 2 * 2.0 - 1.0
    f[3:9, 5:13] = 2.0 + 0.1 * cb
    assert O.roi_snr(f, 5, 3, 8, 6) == pytest.approx(10 * math.log10(4.0 / 0.01), rel=1e-12)
