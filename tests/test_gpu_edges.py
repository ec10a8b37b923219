"""Edge cases of the 2-D path on the GPU against the FP64 oracle: degenerate inputs and
parameters (zero sinogram, no outer / CGLS / GD iterations, one view and one bin, a
one-pixel image), non-finite input, and the largest image the library accepts (8192^2),
where P is checked on sampled rays against the oracle's rows and P^T of single-ray
sinograms against the same rows (the exact transpose)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import eptv_oracle as O
from paper_1009_2288_b300 import eptv as E
from paper_1009_2288_b300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def t32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV).reshape(-1)


def np64(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def coord_bound(g):
    R = 0.5 * math.hypot(g.nx * g.dx, g.ny * g.dy)
    return 2.0 ** -24 * R / min(g.dx, g.dy)


@pytest.fixture(scope="module")
def c1():
    return I.make_c1(with_truth=False)


def test_zero_sinogram_gives_zero_image(c1):
    """y = 0: every CGLS step is guarded (|Ps|^2 = 0), every half-edge magnitude is eps, so
    sigma = eps, and the (P2) gradient vanishes -- the image stays exactly 0, as in the
    oracle."""
    g = c1.geom
    geo = E.Geometry(g)
    p = I.EptvParams(n_outer=3)
    log = O.ReconLog()
    want = O.reconstruct(O.Operator(g), np.zeros(g.n_rays), p, log=log)
    assert np.all(want == 0.0) and log.sigmas[-1] == pytest.approx(p.eps)
    f = torch.zeros(g.n_pix, device=DEV)
    rep = E.eptv_reconstruct(geo, p, torch.zeros(g.n_rays, device=DEV), f)
    assert torch.count_nonzero(f).item() == 0
    assert rep.sigma_last == pytest.approx(log.sigmas[-1], rel=1e-6)


def test_zero_outer_iterations_clamp_the_warm_start(c1):
    g = c1.geom
    geo = E.Geometry(g)
    f0 = I.random_image(g, 3, "uniform") - 0.5
    p = I.EptvParams(n_outer=0)
    want = O.reconstruct(O.Operator(g), c1.y, p, f0=f0)
    f = t32(f0)
    E.eptv_reconstruct(geo, p, t32(c1.y), f)
    got = np64(f).reshape(g.ny, g.nx)
    assert np.array_equal(got, np.maximum(f0.astype(np.float32), 0.0).astype(np.float64))
    assert np.array_equal(got > 0, want > 0)


@pytest.mark.parametrize("field", ["n_gd", "cgls_iters"])
def test_no_gd_or_no_cgls_iterations_match_oracle(c1, field):
    """n_gd = 0: each outer iteration is CGLS then the clamp; cgls_iters = 0: the (P2) solve
    runs on the previous iterate itself (from a warm start, so that something moves)."""
    g = c1.geom
    geo = E.Geometry(g)
    op = O.Operator(g)
    # a warm start of the kind the method produces (a clamped CGLS image): on white noise
    # a fixed step is as large as the pixel values and the iteration is chaotic
    f0 = np.maximum(O.cgls(op, c1.y.reshape(g.n_views, g.n_bins), np.zeros((g.ny, g.nx)), 3), 0.0)
    p = I.EptvParams(n_outer=3, step_rule=O.FIXED, t_fixed=2e-5, **{field: 0})
    want = O.reconstruct(op, c1.y, p, f0=f0)
    f = t32(f0)
    E.eptv_reconstruct(geo, p, t32(c1.y), f)
    got = np64(f).reshape(g.ny, g.nx)
    assert rel(got, f0) > 1e-3                                  # the iterations changed f
    assert rel(got, want) < 1e-4


def test_nan_in_sinogram_raises_nonfinite(c1):
    g = c1.geom
    geo = E.Geometry(g)
    y = t32(c1.y)
    y[g.n_bins // 2] = float("nan")          # the central ray of view 0 (crosses the image)
    f = torch.zeros(g.n_pix, device=DEV)
    with pytest.raises(E.EptvError) as ei:
        E.eptv_reconstruct(geo, I.EptvParams(n_outer=1), y, f)
    assert ei.value.code == -3
    # the handle stays usable: a clean sinogram reconstructs again
    E.eptv_reconstruct(geo, I.EptvParams(n_outer=1), t32(c1.y), f.zero_())
    assert torch.isfinite(f).all()


@pytest.mark.parametrize("nx,ny,nv,nb", [(5, 4, 1, 1), (6, 3, 1, 7), (1, 1, 3, 5), (33, 1, 2, 9)])
def test_degenerate_sizes_match_oracle(nx, ny, nv, nb):
    g = I.FanGeometry(nx, ny, 1.3, 0.9, nv, nb, 0.004, 0.25, 80.0, 130.0, I.ARC)
    geo = E.Geometry(g)
    op = O.Operator(g)
    f = I.random_image(g, 7, "uniform")
    y = torch.empty(g.n_rays, device=DEV)
    E.eptv_project(geo, t32(f), y)
    want = op.project(f)
    scale = max(np.abs(want).max(), 1e-3)
    assert np.max(np.abs(np64(y).reshape(want.shape) - want)) <= 1e-5 * scale
    ys = np.abs(I.random_sino(g, 8))
    b = torch.empty(g.n_pix, device=DEV)
    E.eptv_backproject(geo, t32(ys), b)
    wb = op.backproject(ys)
    assert np.linalg.norm(np64(b).reshape(ny, nx) - wb) <= 4 * coord_bound(g) * max(np.linalg.norm(wb), 1e-30)
    # and a short reconstruction (fixed steps: no Armijo branch to flip)
    p = I.EptvParams(n_outer=2, step_rule=O.FIXED, t_fixed=1e-4, lam=50.0)
    yw = op.project(f)
    wr = O.reconstruct(op, yw, p)
    fr = torch.zeros(g.n_pix, device=DEV)
    E.eptv_reconstruct(geo, p, t32(yw), fr)
    assert np.max(np.abs(np64(fr).reshape(ny, nx) - wr)) <= 1e-4 * max(np.abs(wr).max(), 1e-3)


def test_largest_image_sampled_rays_and_exact_transpose():
    """8192^2 at 0.05 mm (the benchmark's 409.6 mm field), 8 views x 1024 bins: P on
    sampled rays against the oracle's rows, P^T of single-ray sinograms equal to those
    rows entry by entry (within the FP32 crossing bound), and the adjoint identity."""
    n = 8192
    g = I.FanGeometry(n, n, 0.05, 0.05, 8, 1024, 1.0239 / 949.075 * 888 / 1024, 0.25, 541.0, 949.075, I.ARC)
    geo = E.Geometry(g)
    xs = (np.arange(n) + 0.5) * g.dx - 0.5 * n * g.dx
    X, Y = np.meshgrid(xs, xs)
    f = (0.02 * np.exp(-(X ** 2 + Y ** 2) / (2 * 120.0 ** 2)) + 0.005 * np.cos(X / 7.0) * np.sin(Y / 11.0)).astype(np.float32)
    del X, Y
    fd = torch.from_numpy(f.reshape(-1)).to(DEV)
    y = torch.empty(g.n_rays, device=DEV)
    E.eptv_project(geo, fd, y)
    sx, sy, ux, uy = O.rays(g)
    idx = np.arange(3, g.n_rays, 257)
    want = O.project_rays(n, n, g.dx, g.dy, sx[idx], sy[idx], ux[idx], uy[idx], f.astype(np.float64))
    got = np64(y)[idx]
    assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-3)) < 1e-5
    R = 0.5 * math.hypot(n * g.dx, n * g.dy)
    b = torch.empty(g.n_pix, device=DEV)
    ys = torch.zeros(g.n_rays, device=DEV)
    for i in idx[::6][:5]:
        pix, ln = O.ray_row(n, n, g.dx, g.dy, sx[i], sy[i], ux[i], uy[i])
        ys.zero_()
        ys[int(i)] = 1.0
        E.eptv_backproject(geo, ys, b)
        nzi = torch.nonzero(b).reshape(-1).cpu().numpy()
        bb = b[torch.as_tensor(np.union1d(nzi, pix), device=DEV)].double().cpu().numpy()
        dense = dict(zip(pix.tolist(), ln.tolist()))
        ref = np.array([dense.get(j, 0.0) for j in np.union1d(nzi, pix)])
        assert np.max(np.abs(bb - ref)) <= 16 * 2.0 ** -24 * R, i
    yr = torch.rand(g.n_rays, device=DEV, generator=torch.Generator(device=DEV).manual_seed(5))
    E.eptv_backproject(geo, yr, b)
    lhs = float(torch.dot(y.double(), yr.double()))
    rhs = float(torch.dot(fd.double(), b.double()))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_full_benchmark_workload_reaches_the_oracle_energy():
    """The benchmark's 512^2, 40 x 888, 100-iteration reconstruction, in the launch
    configuration the benchmark times (autotuned shapes): its final reported energy
    (Eq. 2, sigma_ref = the oracle's last sigma) and its error against the truth agree
    with the FP64 oracle's (tests/golden/c2_oracle_energy.json, written by
    make_oracle_energy.py from the oracle alone)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "c2_oracle_energy.json")))
    case = I.make_c2(with_truth=True)
    g = case.geom
    geo = E.Geometry(g)
    E.eptv_autotune(geo)
    p = I.EptvParams(n_outer=gold["n_outer"])
    assert p.max_trials == gold["params"]["max_trials"] and p.lam == gold["params"]["lam"]
    f = torch.zeros(g.n_pix, device=DEV)
    y = t32(case.y)
    rep = E.eptv_reconstruct(geo, p, y, f)
    assert rep.n_fail == gold["line_search_failures"]
    e = E.eptv_report_energy(geo, p, gold["sigma_ref"], f, y)
    assert e == pytest.approx(gold["e_report_final"], rel=1e-3)
    got = np64(f).reshape(g.ny, g.nx)
    err = float(((got - case.f_true) ** 2).sum() / (case.f_true ** 2).sum())   # Eq. 12, as stored
    assert err == pytest.approx(gold["rel_error_vs_truth"], rel=1e-2)
