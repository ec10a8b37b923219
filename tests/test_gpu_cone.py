"""3-D cone-beam path on the GPU against the FP64 oracle (oracle/cone_oracle.py): the
projector and its exact transpose, CGLS, the 3-D (P2) solve, whole reconstructions and
the reported energy on reduced scans of the cone-beam workload; at the full 256^3,
120-view, 512 x 384 size, sampled rays against the oracle's rows and single-ray back
projections (the exact transpose) against the same rows."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cone_oracle as C
from oracle import eptv_oracle as O
from paper_1009_2288_b300 import eptv as E
from paper_1009_2288_b300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

GEOMS = {
    "c5_16": I.c5_geometry(16),
    "c5_8": I.c5_geometry(8),
    "aniso": I.ConeGeometry(20, 17, 11, 1.3, 1.1, 1.7, 9, 30, 14, 1.9, 2.3, 0.3, -0.4, 120.0, 200.0),
    # source close to the volume, tall detector: the row band of a z slab spans many rows
    "tall": I.ConeGeometry(16, 16, 24, 1.0, 1.0, 1.0, 12, 40, 64, 0.9, 0.5, 0.25, 0.1, 30.0, 45.0),
    # irregular angles over a short scan, including views along the grid axes
    "angles": I.ConeGeometry(12, 10, 6, 1.0, 1.2, 0.9, 7, 24, 10, 1.1, 1.0, 0.25, 0.0, 60.0, 90.0,
                             angles=np.array([0.0, 0.3, 0.31, 1.2, np.pi / 2, 2.0, np.pi])),
    # a single slice, three detector rows
    "slice": I.ConeGeometry(9, 13, 1, 1.0, 1.0, 2.0, 5, 21, 3, 1.0, 1.5, 0.25, 0.0, 40.0, 70.0),
}


def t32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV).reshape(-1)


def np64(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def coord_bound(g):
    R = 0.5 * math.sqrt((g.nx * g.dx) ** 2 + (g.ny * g.dy) ** 2 + (g.nz * g.dz) ** 2)
    return 2.0 ** -24 * R / min(g.dx, g.dy, g.dz)


def blobs(g, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    z, y, x = np.meshgrid((np.arange(g.nz) + 0.5) * g.dz - g.nz * g.dz / 2,
                          (np.arange(g.ny) + 0.5) * g.dy - g.ny * g.dy / 2,
                          (np.arange(g.nx) + 0.5) * g.dx - g.nx * g.dx / 2, indexing="ij")
    R = 0.5 * min(g.nx * g.dx, g.ny * g.dy, g.nz * g.dz)
    f = np.zeros((g.nz, g.ny, g.nx))
    for _ in range(5):
        c = rng.uniform(-0.5, 0.5, 3) * R
        f += rng.uniform(0.005, 0.02) * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (0.3 * R) ** 2)
    return f


@pytest.mark.parametrize("name", list(GEOMS))
def test_project_and_backproject_match_oracle(name):
    g = GEOMS[name]
    geo = E.Geometry3(g)
    op = C.Operator3(g)
    f = blobs(g, 1)
    y = torch.empty(g.n_rays, device=DEV)
    E.eptv3_project(geo, t32(f), y)
    want = op.project(f).reshape(g.n_views, -1)
    got = np64(y).reshape(g.n_views, -1)
    per_view = np.linalg.norm(got - want, axis=1) / np.maximum(np.linalg.norm(want, axis=1), 1e-300)
    assert per_view.max() < 1e-5, name
    rng = np.random.Generator(np.random.PCG64(2))
    fr = rng.standard_normal((g.nz, g.ny, g.nx))
    E.eptv3_project(geo, t32(fr), y)
    err = np.linalg.norm(np64(y) - op.project(fr).ravel())
    assert err <= 4 * coord_bound(g) * np.linalg.norm(op.project(np.abs(fr))), name
    for ys in (rng.uniform(-1, 1, g.n_rays), rng.uniform(0, 1, g.n_rays)):
        b = torch.empty(g.n_vox, device=DEV)
        E.eptv3_backproject(geo, t32(ys), b)
        err = np.linalg.norm(np64(b) - op.backproject(ys).ravel())
        assert err <= 4 * coord_bound(g) * np.linalg.norm(op.backproject(np.abs(ys))), name


@pytest.mark.parametrize("name", list(GEOMS))
def test_adjoint_identity_fp32(name):
    g = GEOMS[name]
    geo = E.Geometry3(g)
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.standard_normal(g.n_vox)
    ys = rng.standard_normal(g.n_rays)
    px = torch.empty(g.n_rays, device=DEV)
    bt = torch.empty(g.n_vox, device=DEV)
    E.eptv3_project(geo, t32(x), px)
    E.eptv3_backproject(geo, t32(ys), bt)
    xf, yf = x.astype(np.float32).astype(np.float64), ys.astype(np.float32).astype(np.float64)
    lhs, rhs = float(np64(px) @ yf), float(xf @ np64(bt))
    assert abs(lhs - rhs) / (np.linalg.norm(np64(px)) * np.linalg.norm(yf)) < 1e-6


@pytest.mark.parametrize("seg", [2, 4, 8, 16])
def test_projector_launch_shapes_agree(seg):
    g = GEOMS["c5_8"]
    geo = E.Geometry3(g)
    f = t32(blobs(g, 4))
    y0 = torch.empty(g.n_rays, device=DEV)
    E.eptv3_project(geo, f, y0)
    E.eptv3_set_tuning(geo, seg)
    y1 = torch.empty_like(y0)
    E.eptv3_project(geo, f, y1)
    assert rel(np64(y1), np64(y0)) < 1e-6


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_backprojector_stacks_agree(name):
    """Two and four voxels per thread of the back projector sum the same terms in the same
    order for every voxel (slab heights that do not divide nz included)."""
    g = GEOMS[name]
    geo = E.Geometry3(g)
    ys = t32(np.random.Generator(np.random.PCG64(21)).standard_normal(g.n_rays))
    out = []
    for zp in (2, 4):
        E.eptv3_set_backprojector_stack(geo, zp)
        b = torch.full((g.n_vox,), float("nan"), device=DEV)
        E.eptv3_backproject(geo, ys, b)
        out.append(np64(b))
    assert np.isfinite(out[0]).all()
    assert np.array_equal(out[0], out[1])
    with pytest.raises(E.EptvError):
        E.eptv3_set_backprojector_stack(geo, 3)


@pytest.fixture(scope="module")
def c5():
    return I.make_c5(scale=8)


def test_cgls_matches_oracle(c5):
    g = c5.geom
    geo = E.Geometry3(g)
    op = C.Operator3(g)
    u0 = 0.5 * c5.f_true
    for M, tol in ((1, 2e-5), (3, 2e-5)):
        want = O.cgls(op, c5.y, u0, M)
        u = t32(u0).clone()
        E.eptv3_cgls(geo, M, t32(c5.y), u)
        assert rel(np64(u).reshape(want.shape), want) < tol, M


@pytest.mark.parametrize("rule", [O.FIXED, O.ARMIJO])
def test_tv_step_matches_oracle(c5, rule):
    g = c5.geom
    geo = E.Geometry3(g)
    op = C.Operator3(g)
    v = O.cgls(op, c5.y, np.zeros((g.nz, g.ny, g.nx)), 3)
    p = I.EptvParams(n_gd=5, step_rule=rule, t_fixed=2e-4)
    want, st = C.p2_solve(v, p, p.t_init_eff)
    want = np.maximum(want, 0.0)
    f = torch.empty(g.n_vox, device=DEV)
    stats, t_prev = E.eptv3_tv_step(geo, p, t32(v), f)
    assert stats.sigma == pytest.approx(st.sigma, rel=2e-3)
    assert rel(np64(f).reshape(want.shape), want) < 1e-4
    if rule == O.ARMIJO:
        assert t_prev == pytest.approx(st.t_prev, rel=1e-6)


@pytest.mark.parametrize("n_outer", [1, 3])
def test_reconstruct_and_energy_match_oracle(c5, n_outer):
    g = c5.geom
    geo = E.Geometry3(g)
    op = C.Operator3(g)
    p = I.EptvParams(n_outer=n_outer)
    log = O.ReconLog()
    want = C.reconstruct(op, c5.y, p, log=log)
    f = torch.zeros(g.n_vox, device=DEV)
    rep = E.eptv3_reconstruct(geo, p, t32(c5.y), f)
    assert rel(np64(f).reshape(want.shape), want) < 1e-4
    assert rep.sigma_last == pytest.approx(log.sigmas[-1], rel=2e-3)
    sig = log.sigmas[-1]
    e_gpu = E.eptv3_report_energy(geo, p, sig, f, t32(c5.y))
    e_orc = C.report_energy(op, np64(f).reshape(want.shape), c5.y, p, sig)
    assert e_gpu == pytest.approx(e_orc, rel=1e-5)


def test_full_size_sampled_rays_and_exact_transpose():
    """256^3, 120 views, 512 x 384: P f on sampled rays against the oracle's rows (1e-5),
    and P^T of a sinogram with a single ray equal to that ray's row (the exact transpose,
    entry by entry within the FP32 crossing bound)."""
    g = I.c5_geometry(1)
    geo = E.Geometry3(g)
    op_rays = C.rays3_subset(g, np.arange(0, g.n_rays, 49999))
    f = blobs(g, 5)
    y = torch.empty(g.n_rays, device=DEV)
    E.eptv3_project(geo, t32(f), y)
    got = np64(y)
    fr = f.ravel()
    for idx, (s, u) in op_rays.items():
        vox, ln = C.ray_row_of(g, s, u)
        want = float(ln @ fr[vox])
        assert abs(got[idx] - want) <= 1e-5 * max(abs(want), 1e-3), idx
    R = 0.5 * math.sqrt((g.nx * g.dx) ** 2 + (g.ny * g.dy) ** 2 + (g.nz * g.dz) ** 2)
    b = torch.empty(g.n_vox, device=DEV)
    ys = torch.zeros(g.n_rays, device=DEV)
    for idx in list(op_rays)[:6]:
        s, u = op_rays[idx]
        vox, ln = C.ray_row_of(g, s, u)
        ys.zero_()
        ys[idx] = 1.0
        E.eptv3_backproject(geo, ys, b)
        bb = np64(b)
        dense = np.zeros(g.n_vox)
        dense[vox] = ln
        nz = np.nonzero(bb)[0]
        tol = 16 * 2.0 ** -24 * R
        assert np.max(np.abs(bb[vox] - ln)) <= tol, idx
        assert np.max(np.abs(bb[nz] - dense[nz])) <= tol, idx


@pytest.mark.parametrize("rule", [O.FIXED, O.ARMIJO])
def test_tv_step_several_faces_per_thread(rule):
    """64^3 (798,720 faces, 262,144 voxels): the face and voxel kernels loop over several
    elements per thread on a grid of a few blocks per SM, so each thread's partial sums
    of the energy, the gradient products and the Armijo trials cover many terms."""
    g = I.c5_geometry(4)
    geo = E.Geometry3(g)
    rng = np.random.Generator(np.random.PCG64(11))
    v = blobs(g, 6) + 0.002 * rng.standard_normal((g.nz, g.ny, g.nx))
    p = I.EptvParams(n_gd=5, step_rule=rule, t_fixed=2e-4)
    want, st = C.p2_solve(v, p, p.t_init_eff)
    want = np.maximum(want, 0.0)
    f = torch.empty(g.n_vox, device=DEV)
    stats, t_prev = E.eptv3_tv_step(geo, p, t32(v), f)
    assert stats.sigma == pytest.approx(st.sigma, rel=2e-3)
    assert rel(np64(f).reshape(want.shape), want) < 1e-4
    if rule == O.ARMIJO:
        assert t_prev == pytest.approx(st.t_prev, rel=1e-6)


@pytest.mark.parametrize("change,msg", [
    (dict(sid=11.0), "half-diagonal"),                 # source inside the volume's circle
    (dict(sdd=25.0), "half-diagonal"),                 # detector before the source distance
    (dict(nv=400, dv=1.0), "too wide"),                # rays steeper than 45 deg in z
    (dict(n_views=70000), "65535 views"),
])
def test_create_rejects_geometries_outside_the_kernels_assumptions(change, msg):
    base = dict(nx=16, ny=16, nz=24, dx=1.0, dy=1.0, dz=1.0, n_views=12, nu=40, nv=64, du=0.9, dv=0.5,
                u_off=0.25, v_off=0.1, sid=30.0, sdd=45.0)
    base.update(change)
    with pytest.raises(E.EptvError) as ei:
        E.Geometry3(I.ConeGeometry(**base))
    assert ei.value.code == -1 and msg in str(ei.value)


@pytest.mark.parametrize("name", ["aniso", "tall", "slice"])
@pytest.mark.parametrize("rule", [O.FIXED, O.ARMIJO])
def test_tv_step_ragged_volumes(name, rule):
    """(P2) on volumes whose sides are not multiples of the kernels' work units: 20 x 17 x 11
    (a column segment of 11), 16 x 16 x 24 (a full 16-voxel segment and a short one above
    it) and 9 x 13 x 1 (a single plane: every face's z neighbours are outside), so the
    windows the threads carry up their columns start, stop and meet the volume's borders in
    every way, against the oracle."""
    g = GEOMS[name]
    rng = np.random.Generator(np.random.PCG64(12))
    v = blobs(g, 7) + 0.002 * rng.standard_normal((g.nz, g.ny, g.nx))
    p = I.EptvParams(n_gd=4, step_rule=rule, t_fixed=2e-4)
    want, st = C.p2_solve(v, p, p.t_init_eff)
    want = np.maximum(want, 0.0)
    geo = E.Geometry3(g)
    f = torch.empty(g.n_vox, device=DEV)
    stats, t_prev = E.eptv3_tv_step(geo, p, t32(v), f)
    assert stats.sigma == pytest.approx(st.sigma, rel=2e-3)
    assert rel(np64(f).reshape(want.shape), want) < 1e-4
    if rule == O.ARMIJO:
        assert t_prev == pytest.approx(st.t_prev, rel=1e-6)
