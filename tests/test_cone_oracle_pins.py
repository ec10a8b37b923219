"""Pins of the 3-D cone-beam oracle against facts fixed by geometry and mathematics:
brute-force voxel clipping, the adjoint identity, the chord through the volume box, the
detector geometry, hand-computed magnitudes of the extended A3, the extended A2 as the
derivative of the lagged energy (central differences, magnitudes rebuilt with loops), the
textbook sign gradient of plain TV at a step, monotone (P2) energy and a reconstruction
that improves on zero."""
import math

import numpy as np
import pytest

from oracle import cone_oracle as C
from oracle import eptv_oracle as O
from paper_1009_2288_b300 import inputs as I

TINY = I.ConeGeometry(5, 4, 3, 1.0, 1.2, 0.9, 5, 7, 6, 1.3, 1.1, 0.25, 0.1, 20.0, 35.0)


def _clip(lo, hi, s, u):
    """Length of the line s + t u (t >= 0) inside the axis-aligned box [lo, hi]."""
    t0, t1 = 0.0, math.inf
    for a, b, sa, ua in zip(lo, hi, s, u):
        if ua == 0.0:
            if not (a < sa < b):
                return 0.0
            continue
        ta, tb = (a - sa) / ua, (b - sa) / ua
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0)


def test_brute_force_voxel_clipping():
    """Every entry of every ray of a small scan equals the clip of that ray against that
    voxel alone (an independent slab computation per voxel)."""
    g = TINY
    op = C.Operator3(g)
    x0, y0, z0 = -g.nx * g.dx / 2, -g.ny * g.dy / 2, -g.nz * g.dz / 2
    for i in range(0, g.n_rays, 3):
        vox, ln = op.ray_row(i)
        got = np.zeros(g.n_vox)
        np.add.at(got, vox, ln)
        s = [op.r[k][i] for k in range(3)]
        u = [op.r[k][i] for k in range(3, 6)]
        want = np.zeros(g.n_vox)
        for iz in range(g.nz):
            for iy in range(g.ny):
                for ix in range(g.nx):
                    lo = (x0 + ix * g.dx, y0 + iy * g.dy, z0 + iz * g.dz)
                    hi = (lo[0] + g.dx, lo[1] + g.dy, lo[2] + g.dz)
                    want[(iz * g.ny + iy) * g.nx + ix] = _clip(lo, hi, s, u)
        assert np.allclose(got, want, rtol=0, atol=1e-12), i


def test_chord_through_the_volume_box():
    g = I.c5_geometry(8)
    op = C.Operator3(g)
    y = op.project(np.ones((g.nz, g.ny, g.nx))).ravel()
    lo = (-g.nx * g.dx / 2, -g.ny * g.dy / 2, -g.nz * g.dz / 2)
    hi = tuple(-a for a in lo)
    for i in range(0, g.n_rays, 997):
        s = [op.r[k][i] for k in range(3)]
        u = [op.r[k][i] for k in range(3, 6)]
        assert y[i] == pytest.approx(_clip(lo, hi, s, u), rel=1e-12, abs=1e-12)


def test_adjoint_identity_fp64():
    g = I.c5_geometry(8)
    op = C.Operator3(g)
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.standard_normal((g.nz, g.ny, g.nx))
    y = rng.standard_normal((g.n_views, g.nv, g.nu))
    px = op.project(x)
    lhs, rhs = float(np.sum(px * y)), float(np.sum(x * op.backproject(y)))
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(px) * np.linalg.norm(y)


def test_rays_hit_the_detector_pixel_centres():
    """The ray of pixel (iu, iv) meets the detector plane (distance sdd from the source
    along the central direction) at u e_u + w e_z from the detector centre."""
    g = TINY
    sx, sy, sz, ux, uy, uz = C.rays3(g)
    for k, th in enumerate(g.view_angles()):
        c = np.array([-math.cos(th), -math.sin(th), 0.0])
        eu = np.array([-math.sin(th), math.cos(th), 0.0])
        for iv in range(g.nv):
            for iu in range(g.nu):
                i = (k * g.nv + iv) * g.nu + iu
                s = np.array([sx[i], sy[i], sz[i]])
                d = np.array([ux[i], uy[i], uz[i]])
                assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-14)
                hit = s + d * (g.sdd / float(d @ c)) - (s + g.sdd * c)
                assert float(hit @ eu) == pytest.approx((iu - (g.nu - 1) / 2 + g.u_off) * g.du, abs=1e-12)
                assert hit[2] == pytest.approx((iv - (g.nv - 1) / 2 + g.v_off) * g.dv, abs=1e-12)


def test_extended_a3_magnitude_by_hand():
    """f = a * j (linear along y): an interior x-face has D = 0 and pair means a j, so
    T^2 = eps^2 + 1/2 (a^2 + a^2) from the y direction and 0 from z; likewise a z-linear
    volume gives x-faces T^2 = eps^2 + a^2 from the z direction."""
    eps, a = 1e-3, 0.7
    f = a * np.broadcast_to(np.arange(6.0)[None, :, None], (5, 6, 7)).copy()
    (Dx, Tx), _, _ = C.half_faces(f, eps)
    assert np.allclose(Dx[1:-1, 1:-1, 2:-2], 0.0)
    assert np.allclose(Tx[1:-1, 1:-1, 2:-2], math.sqrt(eps * eps + a * a), rtol=1e-14)
    fz = a * np.broadcast_to(np.arange(5.0)[:, None, None], (5, 6, 7)).copy()
    (Dx, Tx), (Dy, Ty), _ = C.half_faces(fz, eps)
    assert np.allclose(Tx[1:-1, 1:-1, 2:-2], math.sqrt(eps * eps + a * a), rtol=1e-14)
    assert np.allclose(Ty[1:-1, 2:-2, 1:-1], math.sqrt(eps * eps + a * a), rtol=1e-14)


def test_plain_tv_step_gradient_textbook_sign():
    """w = 1, eps -> 0, a step along x: delta J = -1 on the low side, +1 on the high side,
    0 away from it (interior, where the transverse differences vanish)."""
    f = np.zeros((8, 8, 10))
    f[:, :, 5:] = 1.0
    g, _, _ = C.p2_gradient(f, f, 1.0, 1e-12, 1.0, mode=O.ONE)
    assert np.allclose(g[2:-2, 2:-2, 4], -1.0, atol=1e-9)
    assert np.allclose(g[2:-2, 2:-2, 5], 1.0, atol=1e-9)
    assert np.allclose(g[2:-2, 2:-2, 1:3], 0.0, atol=1e-9)


def test_constant_volume_interior_gradient_is_fidelity_only():
    f = np.full((8, 9, 10), 0.02)
    v = np.random.Generator(np.random.PCG64(4)).uniform(0, 0.03, f.shape)
    g, _, _ = C.p2_gradient(f, v, 7.0, 1e-5, 1e-3)
    assert np.allclose(g[2:-2, 2:-2, 2:-2], 7.0 * (f - v)[2:-2, 2:-2, 2:-2], rtol=0, atol=1e-15)


def test_p2_energy_monotone_and_reconstruction_improves():
    rng = np.random.Generator(np.random.PCG64(5))
    v = rng.uniform(0, 0.03, (6, 10, 10))
    p = I.EptvParams(n_gd=12, weights_mode=O.ONE)     # fixed weights: a true descent
    _, st = C.p2_solve(v, p, p.t_init_eff)
    assert all(b <= a for a, b in zip(st.energies, st.energies[1:]))
    c = I.make_c5(scale=16)
    op = C.Operator3(c.geom)
    f = C.reconstruct(op, c.y, I.EptvParams(n_outer=3))
    err = np.linalg.norm(f - c.f_true) / np.linalg.norm(c.f_true)
    assert err < 0.5 and np.all(f >= 0)


def _lagged_faces(f, eps):
    """Every half-face of f, written out with loops in the oracle's storage order: the two
    voxels (a, b) across it and its frozen cross term C = sum over the two transverse axes
    of 1/2 (c+^2 + c-^2), c+- the differences of the pair means towards the next / from
    the previous row or slice (voxels outside the volume are 0)."""
    nz, ny, nx = f.shape

    def F(i, j, k):
        return f[k, j, i] if (0 <= i < nx and 0 <= j < ny and 0 <= k < nz) else 0.0

    out = []
    for d, shape in ((0, (nz, ny, nx + 1)), (1, (nz, ny + 1, nx)), (2, (nz + 1, ny, nx))):
        for k in range(shape[0]):
            for j in range(shape[1]):
                for i in range(shape[2]):
                    b = (i, j, k)
                    a = tuple(c - (t == d) for t, c in enumerate(b))

                    def M(off):
                        pa = tuple(c + o for c, o in zip(a, off))
                        pb = tuple(c + o for c, o in zip(b, off))
                        return 0.5 * (F(*pa) + F(*pb))
                    Cx = 0.0
                    for t in range(3):
                        if t == d:
                            continue
                        e = tuple(int(s == t) for s in range(3))
                        m = [M(tuple(-x for x in e)), M((0, 0, 0)), M(e)]
                        Cx += 0.5 * (m[2] - m[1]) ** 2 + 0.5 * (m[1] - m[0]) ** 2
                    out.append((a, b, Cx))
    return out, F


def test_extended_a2_equals_derivative_of_lagged_energy():
    """The 3-D variation (A2 extended to faces) is the gradient of
    sum_e w_e sqrt(eps^2 + D_e(f)^2 + C_e) with w and the cross terms C_e frozen at f,
    checked by central differences; the loop-built magnitudes equal the oracle's T."""
    rng = np.random.Generator(np.random.PCG64(12))
    nz, ny, nx, eps, lam = 3, 4, 5, 1e-2, 2.5
    f = rng.uniform(0, 1, (nz, ny, nx))
    v = rng.uniform(0, 1, (nz, ny, nx))
    faces = C.half_faces(f, eps)
    sigma = float(np.median(np.concatenate([T.ravel() for _, T in faces])))
    g, ws, _ = C.p2_gradient(f, v, lam, eps, sigma)
    terms, F0 = _lagged_faces(f, eps)
    w = np.concatenate([x.ravel() for x in ws])
    assert len(terms) == w.size
    T_loop = np.array([math.sqrt(eps ** 2 + (F0(*b) - F0(*a)) ** 2 + Cx) for a, b, Cx in terms])
    assert np.allclose(T_loop, np.concatenate([T.ravel() for _, T in faces]), rtol=1e-14)

    def energy(fp):
        def Fp(i, j, k):
            return fp[k, j, i] if (0 <= i < nx and 0 <= j < ny and 0 <= k < nz) else 0.0
        E = 0.5 * lam * float(np.sum((fp - v) ** 2))
        for wk, (a, b, Cx) in zip(w, terms):
            D = Fp(*b) - Fp(*a)
            E += wk * math.sqrt(eps * eps + D * D + Cx)
        return E

    h = 1e-6
    fd = np.zeros_like(f)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                fp, fm = f.copy(), f.copy()
                fp[k, j, i] += h
                fm[k, j, i] -= h
                fd[k, j, i] = (energy(fp) - energy(fm)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-7)


def test_armijo_sufficient_decrease_and_first_passing_trial():
    """Every accepted (P2) step in 3-D decreases the frozen-weight energy by at least
    c t |g|^2, each longer trial before it did not, and replaying the accepted steps from v
    gives the oracle's result."""
    rng = np.random.Generator(np.random.PCG64(22))
    v = rng.uniform(0, 1.0, (4, 5, 6))
    v[:, :, 3:] += 0.02                                      # an edge, so that w varies
    p = I.EptvParams(n_gd=8, max_trials=8)
    fo, st = C.p2_solve(v, p, p.t_init_eff)
    assert st.sigma == C.select_sigma(C.half_faces(v, p.eps), p.sigma_q, p.sigma_floor)
    f = v.copy()
    assert len(st.steps) == p.n_gd
    assert any(t > 0 and len(tr) > 1 for t, tr in zip(st.steps, st.trials))   # backtracked, then accepted
    assert any(t == 0 for t in st.steps)                                       # and a failed search
    for t, tried in zip(st.steps, st.trials):
        g, ws, E0 = C.p2_gradient(f, v, p.lam, p.eps, st.sigma)
        gg = float(np.sum(g * g))
        longer = [tt for tt, _ in tried if tt > t] if t > 0 else [tt for tt, _ in tried]
        for tt in longer:
            assert C.p2_energy_frozen(f - tt * g, v, p.lam, p.eps, ws) > E0 - p.armijo_c * tt * gg
        if t > 0:
            assert C.p2_energy_frozen(f - t * g, v, p.lam, p.eps, ws) <= E0 - p.armijo_c * t * gg
            f = f - t * g
    assert np.array_equal(f, fo)


def test_outer_iteration_restarts_cgls_at_the_current_volume():
    """Sec. 2.2, step 1 with App. I in 3-D: each outer iteration runs CGLS started at the
    current (clamped) volume f^(k).  With M = 1 the CGLS step is the exact line search along
    s = P^T (y - P f^(k)) on the dense matrix of a small scan; one fixed (P2) step is
    v - t dJ(v); step 3 clamps.  Two outer iterations from a non-zero warm start, composed
    by hand, equal the oracle's reconstruction, and a CGLS started at 0 lands far away."""
    g = TINY
    op = C.Operator3(g)
    n = g.n_vox
    P = np.stack([op.project(np.eye(n)[j].reshape(g.nz, g.ny, g.nx)).ravel() for j in range(n)], 1)
    rng = np.random.Generator(np.random.PCG64(41))
    truth = rng.uniform(0, 0.03, (g.nz, g.ny, g.nx))
    y = P @ truth.ravel() + 1e-3 * rng.standard_normal(P.shape[0])
    f0 = rng.uniform(-0.01, 0.05, (g.nz, g.ny, g.nx))
    p = I.EptvParams(cgls_iters=1, n_gd=1, step_rule=O.FIXED, t_fixed=2e-4, lam=50.0, n_outer=2)

    def by_hand(fk):
        r0 = y - P @ fk.ravel()
        s0 = P.T @ r0
        q = P @ s0
        v = fk + (float(q @ r0) / float(q @ q) * s0).reshape(fk.shape)
        sigma = C.select_sigma(C.half_faces(v, p.eps), p.sigma_q, p.sigma_floor)
        dJ, _, _ = C.p2_gradient(v, v, p.lam, p.eps, sigma)
        return np.maximum(v - p.t_fixed * dJ, 0.0)

    f1 = by_hand(np.maximum(f0, 0.0))
    want = by_hand(f1)
    got = C.reconstruct(op, y, p, f0=f0)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-14)
    s0 = P.T @ y
    q = P @ s0
    v0 = (float(q @ y) / float(q @ q) * s0).reshape(f1.shape)
    assert np.linalg.norm(v0 - f1) > 0.05 * np.linalg.norm(f1)
