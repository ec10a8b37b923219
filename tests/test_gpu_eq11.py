"""The paper's interpolating back projector (Eq. 11) on the GPU against the FP64 oracle:
the operator itself, CGLS and reconstructions that use it as P^T (operator mode EQ11),
and its adjoint mismatch against the exact Siddon P."""
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
    "wide_flat": I.FanGeometry(64, 64, 1.0, 1.0, 40, 400, 1.3 / 400, 0.25, 100.0, 150.0, I.FLAT),
}


class OpEq11(O.Operator):
    """The oracle's P with Eq. (11) as its back projector."""

    def backproject(self, y):
        return O.backproject_eq11(self.g, y)


def t32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


def np64(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("name", list(GEOMS))
def test_eq11_matches_oracle(name):
    """Smooth sinograms (projections of a phantom): 1e-5 relative L2.  Random sinograms:
    the fractional bin position u* is an FP32 number of magnitude up to n_bins, so the
    interpolation weight carries an absolute error of about 2^-24 n_bins, amplified by the
    jump between neighbouring bins: bound 8 x 2^-24 n_bins relative."""
    g = GEOMS[name]
    geo = E.Geometry(g)
    op = O.Operator(g)
    phantom = I.rasterize(I.random_ellipses(np.random.Generator(np.random.PCG64(9)),
                                            0.5 * min(g.nx * g.dx, g.ny * g.dy), 6), g)
    ys = op.project(phantom)
    f = torch.empty(g.n_pix, device=DEV)
    E.eptv_backproject_eq11(geo, t32(ys).reshape(-1), f)
    assert rel(np64(f).reshape(g.ny, g.nx), O.backproject_eq11(g, ys)) < 1e-5
    yr = I.random_sino(g, 7)
    E.eptv_backproject_eq11(geo, t32(yr).reshape(-1), f)
    assert rel(np64(f).reshape(g.ny, g.nx), O.backproject_eq11(g, yr)) < 8 * 2.0 ** -24 * g.n_bins


def test_operator_mode_eq11_in_cgls_and_reconstruct():
    c = I.make_c1()
    g = c.geom
    geo = E.Geometry(g)
    E.eptv_set_operator(geo, E.OPERATOR_EQ11)
    op = OpEq11(g)
    y = t32(c.y).reshape(-1)
    f = torch.empty(g.n_pix, device=DEV)
    E.eptv_backproject(geo, y, f)                       # the mode's P^T is Eq. (11)
    assert rel(np64(f).reshape(g.ny, g.nx), O.backproject_eq11(g, c.y)) < 1e-5
    u0 = 0.5 * c.f_true
    for M in (1, 3):
        want = O.cgls(op, c.y, u0, M)
        u = t32(u0).reshape(-1).clone()
        E.eptv_cgls(geo, M, y, u)
        assert rel(np64(u).reshape(g.ny, g.nx), want) < 2e-5, M
    p = I.EptvParams(n_outer=3)
    want = O.reconstruct(op, c.y, p)
    f.zero_()
    E.eptv_reconstruct(geo, p, y, f)
    assert rel(np64(f).reshape(g.ny, g.nx), want) < 1e-4
    E.eptv_set_operator(geo, E.OPERATOR_ON_THE_FLY)
    E.eptv_backproject(geo, y, f)
    assert rel(np64(f).reshape(g.ny, g.nx), O.Operator(g).backproject(c.y)) < 1e-5


def test_eq11_adjoint_mismatch_full_size():
    """On the 512^2, 40 x 888 workload: <P f, y> against <f, P^T y> with the GPU's exact P
    and Eq. (11), for the phantom and its sinogram: within the paper's 1 % (App. III)."""
    c = I.make_c2(with_truth=True)
    g = c.geom
    geo = E.Geometry(g)
    f = t32(c.f_true).reshape(-1)
    y = t32(c.y).reshape(-1)
    pf = torch.empty(g.n_rays, device=DEV)
    E.eptv_project(geo, f, pf)
    b = torch.empty(g.n_pix, device=DEV)
    E.eptv_backproject_eq11(geo, y, b)
    lhs = float((pf.double() * y.double()).sum())
    rhs = float((f.double() * b.double()).sum())
    assert abs(lhs - rhs) < 1e-2 * abs(lhs)
