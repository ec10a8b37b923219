"""The all-core evaluation of the oracle's P and P^T (oracle/sharded.py, used to time the
oracle on every host core) against the single-process oracle: P bit for bit, P^T to FP64
summation order, and a reconstruction with it equal to the oracle's to 1e-12."""
import numpy as np

from oracle import eptv_oracle as O
from oracle import sharded as SH
from paper_1009_2288_b300 import inputs as I


def test_sharded_operator_matches_the_oracle():
    g = I.ge_geometry(96, 2.0, 13, 301, 0.958 / 301)
    op = O.Operator(g)
    rng = np.random.Generator(np.random.PCG64(5))
    f = rng.uniform(0, 0.03, (g.ny, g.nx))
    y = rng.uniform(0, 1, (g.n_views, g.n_bins))
    with SH.ShardedOperator(g, n_workers=3) as sop:
        assert sop.n_workers == 3
        assert np.array_equal(sop.project(f), op.project(f))
        bt, bt1 = sop.backproject(y), op.backproject(y)
        assert np.allclose(bt, bt1, rtol=1e-13, atol=1e-13 * np.abs(bt1).max())
        p = I.EptvParams(n_outer=2)
        want = O.reconstruct(op, y, p)
        got = O.reconstruct(sop, y, p)
        assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
