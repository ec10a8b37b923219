"""The stored-matrix operator (Sec. 2.3: P kept as a sparse matrix) against the FP64 oracle
and against the on-the-fly kernels: matrix entries element by element, the two stored
matrices as exact transposes, SpMV projections and back projections, CGLS and whole
reconstructions, batches."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import eptv_oracle as O
from paper_1009_2288_b300 import eptv as E
from paper_1009_2288_b300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

GEOMS = {
    "c1": I.c1_geometry(),
    "ge_ragged": I.ge_geometry(200, 1.7, 13, 301, 0.958 / 301),
    "flat_aniso": I.FanGeometry(45, 37, 1.1, 0.9, 11, 97, 0.0012, 0.25, 700.0, 1100.0, I.FLAT),
    "tiny": I.FanGeometry(3, 5, 2.0, 2.0, 4, 9, 0.02, 0.25, 60.0, 100.0, I.ARC),
}


def t32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


def np64(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def half_diag(g):
    return 0.5 * math.hypot(g.nx * g.dx, g.ny * g.dy)


def coord_bound(g):
    """FP32 crossing parameters of magnitude up to R: 2^-24 R / pitch relative."""
    return 2.0 ** -24 * half_diag(g) / min(g.dx, g.dy)


def stored(g):
    geo = E.Geometry(g)
    nnz = E.eptv_set_operator(geo, E.OPERATOR_STORED)
    return geo, nnz


def host_csr(geo, which):
    ptr, col, val = E.eptv_matrix(geo, which)
    return ptr.cpu().numpy().astype(np.int64), col.cpu().numpy().astype(np.int64), val.cpu().numpy()


@pytest.mark.parametrize("name", list(GEOMS))
def test_layout_padding_and_exact_transpose(name):
    """Rows padded to multiples of 4 with zero entries after the real ones, columns strictly
    increasing within each row, and P equal to (P^T)^T entry for entry (bit-exact)."""
    g = GEOMS[name]
    geo, nnz = stored(g)
    P = host_csr(geo, 0)
    PT = host_csr(geo, 1)
    assert nnz == P[0][-1] == len(P[1])
    coo = []
    for (ptr, col, val), nrows in ((P, g.n_rays), (PT, g.n_pix)):
        assert len(ptr) == nrows + 1 and ptr[0] == 0 and np.all(ptr % 4 == 0)
        rows = np.repeat(np.arange(nrows), np.diff(ptr))
        real = val != 0.0
        assert np.all(val >= 0.0)
        # padding only at the end of a row: real entries first, then < 4 zeros
        for r in range(0, nrows, max(1, nrows // 97)):
            v = val[ptr[r]:ptr[r + 1]]
            k = int(np.count_nonzero(v))
            assert np.all(v[:k] > 0) and not v[k:].any() and len(v) - k < 4
            c = col[ptr[r]:ptr[r] + k]
            assert np.all(np.diff(c) > 0)
        coo.append((rows[real], col[real], val[real]))
    (pr, pc, pv), (tr, tc, tv) = coo
    a = np.lexsort((pc, pr))
    b = np.lexsort((tr, tc))
    assert np.array_equal(pr[a], tc[b]) and np.array_equal(pc[a], tr[b])
    assert np.array_equal(pv[a].view(np.uint32), tv[b].view(np.uint32))


@pytest.mark.parametrize("name", ["c1", "ge_ragged", "flat_aniso"])
def test_entries_match_oracle_rows(name):
    """Every stored entry of sampled rays against the oracle's FP64 row of P (Siddon).
    A crossing parameter t = (X - p) / u is formed from FP32 coordinates of magnitude up to
    R, so it carries an absolute error of about 2^-24 R / |u| for the grid lines across
    the direction component u: the bound per ray is 8 x 2^-24 R (1/|u_x| + 1/|u_y|) (with
    |u| floored at 1e-3).  No oracle entry above that bound may be missing."""
    g = GEOMS[name]
    geo, _ = stored(g)
    ptr, col, val = host_csr(geo, 0)
    sx, sy, ux, uy = O.rays(g)
    for i in np.linspace(0, g.n_rays - 1, 61).astype(int):
        tol = 8 * 2.0 ** -24 * half_diag(g) * (1 / max(abs(ux[i]), 1e-3) + 1 / max(abs(uy[i]), 1e-3))
        pix, ln = O.ray_row(g.nx, g.ny, g.dx, g.dy, sx[i], sy[i], ux[i], uy[i])
        want = np.zeros(g.n_pix)
        want[pix] = ln
        got = np.zeros(g.n_pix)
        np.add.at(got, col[ptr[i]:ptr[i + 1]], val[ptr[i]:ptr[i + 1]])   # padding repeats a column
        bad = np.nonzero(np.abs(got - want) > tol)[0]
        assert len(bad) == 0, (name, i, [(int(j), got[j], want[j]) for j in bad[:6]])


@pytest.mark.parametrize("name", list(GEOMS))
def test_spmv_matches_oracle_and_on_the_fly(name):
    """Stored P f: 1e-5 per view (phantom-like images) against the oracle and 1e-6 against
    the on-the-fly projector (same p_ij, other summation order); stored P^T y within
    4 x coord_bound of P^T |y| against the oracle and 1e-6 against K2."""
    g = GEOMS[name]
    op = O.Operator(g)
    geo, _ = stored(g)
    fly = E.Geometry(g)
    phantom = I.rasterize(I.random_ellipses(np.random.Generator(np.random.PCG64(9)),
                                            0.5 * min(g.nx * g.dx, g.ny * g.dy), 6), g)
    for f in (phantom, I.random_image(g, 1, "uniform")):
        want = op.project(f)
        y = torch.empty(g.n_rays, device=DEV)
        E.eptv_project(geo, t32(f), y)
        got = np64(y).reshape(g.n_views, g.n_bins)
        num = np.linalg.norm(got - want, axis=1)
        assert np.max(num / np.maximum(np.linalg.norm(want, axis=1), 1e-300)) < 1e-5, name
        y2 = torch.empty_like(y)
        E.eptv_project(fly, t32(f), y2)
        assert rel(np64(y), np64(y2)) < 1e-6
    for ysin in (I.random_sino(g, 7), np.abs(I.random_sino(g, 8))):
        want = op.backproject(ysin)
        f = torch.empty(g.n_pix, device=DEV)
        E.eptv_backproject(geo, t32(ysin), f)
        err = np.linalg.norm(np64(f).reshape(g.ny, g.nx) - want)
        assert err <= 4 * coord_bound(g) * np.linalg.norm(op.backproject(np.abs(ysin))), name
        f2 = torch.empty_like(f)
        E.eptv_backproject(fly, t32(ysin), f2)
        assert rel(np64(f), np64(f2)) < 1e-6


def test_adjoint_identity_stored():
    g = GEOMS["c1"]
    geo, _ = stored(g)
    for seed in range(3):
        x = I.random_image(g, 30 + seed, "normal")
        ys = I.random_sino(g, 40 + seed)
        px = torch.empty(g.n_rays, device=DEV)
        bt = torch.empty(g.n_pix, device=DEV)
        E.eptv_project(geo, t32(x), px)
        E.eptv_backproject(geo, t32(ys), bt)
        xf = x.astype(np.float32).astype(np.float64).ravel()
        yf = ys.astype(np.float32).astype(np.float64).ravel()
        lhs, rhs = float(np64(px) @ yf), float(xf @ np64(bt))
        assert abs(lhs - rhs) / (np.linalg.norm(np64(px)) * np.linalg.norm(yf)) < 1e-6


def test_full_size_c2_spmv_sampled_views():
    """The 512^2, 40 x 888 workload: stored P f of the phantom on 5 sampled views against
    the oracle (1e-5 per view), stored entries = nonzeros of the oracle's rows."""
    c = I.make_c2(with_truth=True)
    g = c.geom
    geo, nnz = stored(g)
    op = O.Operator(g)
    y = torch.empty(g.n_rays, device=DEV)
    E.eptv_project(geo, t32(c.f_true), y)
    got = np64(y).reshape(g.n_views, g.n_bins)
    sx, sy, ux, uy = O.rays(g)
    for v in (0, 7, 19, 28, 39):
        want = np.empty(g.n_bins)
        for k in range(g.n_bins):
            i = v * g.n_bins + k
            pix, ln = O.ray_row(g.nx, g.ny, g.dx, g.dy, sx[i], sy[i], ux[i], uy[i])
            want[k] = float(ln @ c.f_true.ravel()[pix])
        assert np.linalg.norm(got[v] - want) / np.linalg.norm(want) < 1e-5, v
    ptr, col, val = host_csr(geo, 0)
    assert int(np.count_nonzero(val)) == pytest.approx(18_600_668, rel=1e-4)


def test_cgls_and_reconstruct_stored_match_oracle():
    c = I.make_c1()
    g = c.geom
    geo, _ = stored(g)
    op = O.Operator(g)
    u0 = 0.5 * c.f_true
    for M, tol in ((1, 2e-5), (3, 2e-5), (5, 2e-5)):
        want = O.cgls(op, c.y, u0, M)
        u = t32(u0).reshape(-1).clone()
        E.eptv_cgls(geo, M, t32(c.y).reshape(-1), u)
        assert rel(np64(u).reshape(g.ny, g.nx), want) < tol, M
    p = I.EptvParams(n_outer=3)
    want = O.reconstruct(op, c.y, p)
    f = torch.zeros(g.n_pix, device=DEV)
    rep = E.eptv_reconstruct(geo, p, t32(c.y).reshape(-1), f)
    assert rel(np64(f).reshape(g.ny, g.nx), want) < 1e-4
    assert rep.n_launches > 0
    sig = rep.sigma_last
    e_gpu = E.eptv_report_energy(geo, p, sig, f, t32(c.y).reshape(-1))
    e_orc = O.report_energy(op, np64(f).reshape(g.ny, g.nx), c.y, p, sig)
    assert e_gpu == pytest.approx(e_orc, rel=1e-5)


def test_stored_batch_equals_single_and_modes_must_agree():
    cases = [I.make_c3_slice(100 + i, with_truth=False) for i in range(3)]
    p = I.EptvParams(n_outer=4)
    geos = [E.Geometry(c.geom) for c in cases]
    for geo in geos:
        E.eptv_set_operator(geo, E.OPERATOR_STORED)
    ys = [t32(c.y).reshape(-1) for c in cases]
    fs = [torch.zeros(c.geom.n_pix, device=DEV) for c in cases]
    E.eptv_reconstruct_batched(geos, p, ys, fs)
    for c, geo, y, f in zip(cases, geos, ys, fs):
        f1 = torch.zeros(c.geom.n_pix, device=DEV)
        E.eptv_reconstruct(geo, p, y, f1)
        assert torch.equal(f, f1)
    E.eptv_set_operator(geos[1], E.OPERATOR_ON_THE_FLY)
    with pytest.raises(E.EptvError):
        E.eptv_reconstruct_batched(geos, p, ys, fs)
    E.eptv_set_operator(geos[1], E.OPERATOR_STORED)      # switching back reuses the matrices
    E.eptv_reconstruct_batched(geos, p, ys, fs)


def test_stored_pt_mode_mixes_the_operators_exactly():
    """EPTV_OPERATOR_STORED_PT: P on the fly (K1), P^T from the stored matrix.  The entries are
    the same canonical p_ij, so P^T agrees with the on-the-fly back projector to summation
    order, the adjoint identity holds, and reconstructions, batches and energies match the
    oracle as in the other modes."""
    c = I.make_c1()
    g = c.geom
    geo = E.Geometry(g)
    ref = E.Geometry(g)
    E.eptv_set_operator(geo, E.OPERATOR_STORED_PT)
    op = O.Operator(g)
    f = I.random_image(g, 3, "uniform")
    y1, y2 = torch.empty(g.n_rays, device=DEV), torch.empty(g.n_rays, device=DEV)
    E.eptv_project(geo, t32(f).reshape(-1), y1)
    E.eptv_project(ref, t32(f).reshape(-1), y2)
    assert torch.equal(y1, y2)                                   # the same K1
    ys = np.abs(I.random_sino(g, 4))
    b1, b2 = torch.empty(g.n_pix, device=DEV), torch.empty(g.n_pix, device=DEV)
    E.eptv_backproject(geo, t32(ys).reshape(-1), b1)
    E.eptv_backproject(ref, t32(ys).reshape(-1), b2)
    assert rel(np64(b1), np64(b2)) < 1e-6
    lhs = float(np64(y1) @ ys.astype(np.float32).astype(np.float64).ravel())
    rhs = float(f.astype(np.float32).astype(np.float64).ravel() @ np64(b1))
    assert abs(lhs - rhs) / abs(lhs) < 1e-6
    p = I.EptvParams(n_outer=3)
    want = O.reconstruct(op, c.y, p)
    fr = torch.zeros(g.n_pix, device=DEV)
    rep = E.eptv_reconstruct(geo, p, t32(c.y).reshape(-1), fr)
    assert rel(np64(fr).reshape(g.ny, g.nx), want) < 1e-4
    e_gpu = E.eptv_report_energy(geo, p, rep.sigma_last, fr, t32(c.y).reshape(-1))
    e_orc = O.report_energy(op, np64(fr).reshape(g.ny, g.nx), c.y, p, rep.sigma_last)
    assert e_gpu == pytest.approx(e_orc, rel=1e-5)
    cases = [I.make_c3_slice(200 + i, with_truth=False) for i in range(2)]
    geos = [E.Geometry(cc.geom) for cc in cases]
    for gg in geos:
        E.eptv_set_operator(gg, E.OPERATOR_STORED_PT)
    yb = [t32(cc.y).reshape(-1) for cc in cases]
    fb = [torch.zeros(cc.geom.n_pix, device=DEV) for cc in cases]
    E.eptv_reconstruct_batched(geos, p, yb, fb)
    for cc, gg, y, fv in zip(cases, geos, yb, fb):
        f1 = torch.zeros(cc.geom.n_pix, device=DEV)
        E.eptv_reconstruct(gg, p, y, f1)
        assert torch.equal(fv, f1)


def test_autotune_operator_keeps_the_faster_back_projector():
    """eptv_autotune_operator on the benchmark geometry: the kept mode is one of the two P^T
    forms, P^T then agrees with the on-the-fly kernel to summation order, a budget below
    the size bound keeps the kernel, and a handle in the fully stored mode is refused."""
    g = I.make_c2(with_truth=False).geom
    geo, ref = E.Geometry(g), E.Geometry(g)
    E.eptv_autotune(geo)
    mode = E.eptv_autotune_operator(geo, 4 << 30)
    assert mode in (E.OPERATOR_ON_THE_FLY, E.OPERATOR_STORED_PT)
    ys = t32(np.abs(I.random_sino(g, 8))).reshape(-1)
    b1, b2 = torch.empty(g.n_pix, device=DEV), torch.empty(g.n_pix, device=DEV)
    E.eptv_backproject(geo, ys, b1)
    E.eptv_backproject(ref, ys, b2)
    assert rel(np64(b1), np64(b2)) < 1e-6
    small = E.Geometry(g)
    assert E.eptv_autotune_operator(small, 1 << 20) == E.OPERATOR_ON_THE_FLY
    E.eptv_backproject(small, ys, b1)
    assert torch.equal(b1, b2)
    full = E.Geometry(I.c1_geometry())
    E.eptv_set_operator(full, E.OPERATOR_STORED)
    with pytest.raises(E.EptvError):
        E.eptv_autotune_operator(full, 4 << 30)
