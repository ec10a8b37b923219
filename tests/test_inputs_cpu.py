"""The seeded input recipes the parity tests and the benchmark run on, checked on the
CPU against their stated parameters: the benchmark workload's geometry and noise model,
and the batched workload's per-slice draws (64 slices, seeds 100-163)."""
import math

import numpy as np

from paper_1009_2288_b300 import inputs as I


def test_benchmark_workload_geometry_and_noise():
    c = I.make_c2(with_truth=False)
    g = c.geom
    assert (g.nx, g.ny, g.n_views, g.n_bins) == (512, 512, 40, 888)
    assert math.isclose(g.dx, 0.8) and math.isclose(g.sid, 541.0) and math.isclose(g.sdd, 949.075)
    assert math.isclose(g.dbeta, 1.0239 / 949.075, rel_tol=1e-12)
    y = np.asarray(c.y).reshape(g.n_views, g.n_bins)
    assert np.all(np.isfinite(y))
    # rays that miss the body: y = -ln(counts / I0), counts ~ Poisson(5e4)
    edge = np.concatenate([y[:, :20].ravel(), y[:, -20:].ravel()])
    assert abs(edge.std() - 1.0 / math.sqrt(5e4)) < 0.15 / math.sqrt(5e4)


def test_batched_slices_follow_their_recipe():
    sizes, views, bins, i0s = set(), [], [], []
    for seed in range(100, 164, 7):
        c = I.make_c3_slice(seed, with_truth=False)
        g = c.geom
        assert g.nx == g.ny and g.nx in (256, 384, 512)
        assert math.isclose(g.nx * g.dx, 409.6, rel_tol=1e-12)
        assert 20 <= g.n_views <= 60 and 512 <= g.n_bins <= 888
        assert math.isclose(g.dbeta * g.n_bins, 0.958, rel_tol=1e-12)
        assert 1e4 <= c.i0 <= 1e5
        assert np.asarray(c.y).size == g.n_views * g.n_bins and np.all(np.isfinite(c.y))
        sizes.add(g.nx); views.append(g.n_views); bins.append(g.n_bins); i0s.append(c.i0)
    assert len(sizes) >= 2 and len(set(views)) > 3 and len(set(bins)) > 3
    # the same seed gives the same slice
    a, b = I.make_c3_slice(123, with_truth=False), I.make_c3_slice(123, with_truth=False)
    assert np.array_equal(np.asarray(a.y), np.asarray(b.y))
