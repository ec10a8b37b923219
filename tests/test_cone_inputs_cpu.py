"""The cone-beam benchmark's inputs, checked on the CPU: the torch synthesis of the
full-size sinogram (run on the device by the benchmark) against the host FP64 generator
on a reduced scan, and the nonzero count of the 3-D roofline against the oracle's exact
rows (an upper bound by construction)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cone_oracle as C
from paper_1009_2288_b300 import cone
from paper_1009_2288_b300 import inputs as I


def test_torch_line_integrals_equal_the_host_generator():
    g = I.c5_geometry(16)
    els, _ = I.c5_ellipsoids(5, g)
    sx, sy, sz, ux, uy, uz = I.cone_rays(g)
    want = I.line_integrals3(els, sx, sy, sz, ux, uy, uz).reshape(g.n_views, -1)
    for k in (0, g.n_views // 3, g.n_views - 1):
        src, tx, ty, tz = cone.rays_gpu(g, k, "cpu")
        got = cone.line_integrals3_gpu(els, src, tx, ty, tz).numpy()
        assert np.max(np.abs(got - want[k])) <= 1e-9 * max(np.abs(want[k]).max(), 1.0), k
    assert np.any(want > 0)


def test_noisy_sinogram_follows_the_poisson_model():
    g = I.c5_geometry(16)
    y = cone.c5_sinogram_gpu(5, g, "cpu").double().numpy()
    els, _ = I.c5_ellipsoids(5, g)
    p = I.line_integrals3(els, *I.cone_rays(g))
    assert y.shape == (g.n_rays,) and np.all(np.isfinite(y))
    # y = ln(I0 / counts), counts ~ Poisson(I0 e^-p): the error is a few percent of the
    # noise-free integral at I0 = 5e4 where the rays cross the phantom
    hit = p > 0.5
    assert np.median(np.abs(y[hit] - p[hit]) / p[hit]) < 0.05
    # rays that miss it: y = -ln(counts / I0) with counts ~ Poisson(I0), so y has mean ~0
    # and standard deviation ~1 / sqrt(I0)
    y0 = y[p == 0.0]
    sd = 1.0 / np.sqrt(5e4)
    assert y0.size > 500
    assert abs(y0.std() - sd) < 0.1 * sd
    assert abs(y0.mean()) < 5.0 * sd / np.sqrt(y0.size)


@pytest.mark.parametrize("name", ["c5_16", "aniso"])
def test_cone_nnz_count_bounds_the_oracle_rows(name):
    g = {"c5_16": I.c5_geometry(16),
         "aniso": I.ConeGeometry(20, 17, 11, 1.3, 1.1, 1.7, 9, 30, 14, 1.9, 2.3, 0.3, -0.4, 120.0, 200.0)}[name]
    op = C.Operator3(g)
    exact = sum(int(np.count_nonzero(op.ray_row(i)[1] > 0)) for i in range(g.n_rays))
    bound = cone.nnz_of(g)
    assert exact <= bound <= exact * 1.001
