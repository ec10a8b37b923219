"""Image-quality metrics of Sec. 3 (Eqs. 12-14) on the GPU against the FP64 oracle: edge
maps bit-exact (the decision is taken in FP64 on both sides; only a pixel whose Sobel
energy lies within 1e-12 of the threshold may differ), counts and correlation exact,
relative error and SNR to FP64 rounding."""
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


def check(g, f32, r32, roi, scale=2.0):
    geo = E.Geometry(g)
    f64 = f32.astype(np.float64)
    r64 = r32.astype(np.float64)
    ef = torch.zeros(g.n_pix, dtype=torch.uint8, device=DEV)
    er = torch.zeros(g.n_pix, dtype=torch.uint8, device=DEV)
    q = E.eptv_quality_metrics(geo, t32(f32), t32(r32), roi, scale, ef, er)
    for got, img in ((ef, f64), (er, r64)):
        want = O.sobel_edges(img, scale)
        g2 = O.sobel_gradient2(img)
        tau = scale * scale * float(np.mean(g2[1:-1, 1:-1]))
        got = got.cpu().numpy().reshape(g.ny, g.nx)
        differ = got != want
        assert np.all(np.abs(g2[differ] - tau) <= 1e-12 * tau)
    bf, br = O.sobel_edges(f64, scale), O.sobel_edges(r64, scale)
    assert q.edges == int(bf.sum()) and q.edges_ref == int(br.sum()) and q.edges_both == int((bf & br).sum())
    want_c = O.edge_correlation(bf, br)
    if math.isnan(want_c):                     # a constant edge map (e.g. no interior edges)
        assert math.isnan(q.ecc)
    else:
        assert q.ecc == pytest.approx(want_c, rel=1e-12, abs=1e-15)
    assert q.rel_error == pytest.approx(O.relative_error(f64, r64), rel=1e-12)
    assert q.snr_db == pytest.approx(O.roi_snr(f64, *roi), rel=1e-9)
    return q


def test_quality_of_a_reconstruction():
    c = I.make_c1()
    g = c.geom
    geo = E.Geometry(g)
    f = torch.zeros(g.n_pix, device=DEV)
    E.eptv_reconstruct(geo, I.EptvParams(n_outer=20), t32(c.y), f)
    q = check(g, f.cpu().numpy().reshape(g.ny, g.nx), c.f_true.astype(np.float32), (40, 50, 30, 20))
    assert 0.0 < q.rel_error < 0.1 and 0.2 < q.ecc <= 1.0


@pytest.mark.parametrize("shape", [(37, 45), (3, 3), (64, 96)])
def test_quality_random_images_ragged_tiles(shape):
    ny, nx = shape
    g = I.FanGeometry(nx, ny, 1.0, 1.0, 4, 16, 0.02, 0.25, 200.0, 300.0, I.ARC)
    rng = np.random.Generator(np.random.PCG64(nx * ny))
    f = rng.uniform(0.5, 1.5, (ny, nx)).astype(np.float32)
    r = (f + rng.normal(0, 0.05, (ny, nx))).astype(np.float32)
    check(g, f, r, (0, 0, nx, ny))


def test_quality_without_reference_and_bad_roi():
    g = I.c1_geometry()
    geo = E.Geometry(g)
    f = t32(np.ones((g.ny, g.nx)) + 0.01 * np.arange(g.n_pix).reshape(g.ny, g.nx) % 3)
    q = E.eptv_quality_metrics(geo, f, None, (0, 0, 8, 8))
    assert math.isnan(q.rel_error) and math.isnan(q.ecc) and q.edges_ref == 0
    with pytest.raises(E.EptvError):
        E.eptv_quality_metrics(geo, f, None, (120, 0, 16, 8))
