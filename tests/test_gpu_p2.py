"""The persistent (P2) kernel (one cooperative launch per (P2) solve) against the
per-iteration kernels (one launch per GD iteration, then the clamp): both evaluate
Eqs. 5, 9, A2 and A3 with the same arithmetic, sum each 32 x 8 tile in the same order and
add the tiles exactly, so images, step logs and scalars must be bit-identical.  Covers
every region shape (1x1, 1x2, 1x4, 2x4 tiles), trial counts 1 / 4 / 8 (and 12, where both
use the per-iteration kernels), plain TV, prior weights, ragged image sizes, the (P2)
entry point with its edge-weight output, and the bounded barrier wait."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import eptv_oracle as O
from paper_1009_2288_b300 import eptv as E
from paper_1009_2288_b300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def t32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


def _recon(geo, g, y, p, mode, wprior=None):
    E.eptv_set_tv_kernel(geo, mode)
    f = torch.zeros(g.n_pix, device=DEV)
    rep = E.eptv_reconstruct(geo, p, y, f, wprior=wprior)
    steps, sigmas = E.eptv_get_log(geo)
    return f, rep, steps, sigmas


def _assert_same(geo, g, y, p, wprior=None):
    fa, ra, sa, ga = _recon(geo, g, y, p, E.TV_AUTO, wprior)
    fb, rb, sb, gb = _recon(geo, g, y, p, E.TV_PER_ITERATION, wprior)
    assert torch.equal(fa, fb)
    assert np.array_equal(sa, sb) and np.array_equal(ga, gb)
    assert (ra.n_fail, ra.t_prev, ra.sigma_last) == (rb.n_fail, rb.t_prev, rb.sigma_last)
    return ra, rb


GEOMS = {
    "c1_128": I.c1_geometry(),                                           # 4 x 16 tiles
    "ragged_200": I.ge_geometry(200, 1.7, 13, 301, 0.958 / 301),         # partial tiles both ways
    "learned_256": I.ge_geometry(256, 1.6, 30),
    "tiny_3x5": I.FanGeometry(3, 5, 2.0, 2.0, 4, 9, 0.02, 0.25, 60.0, 100.0, I.ARC),
    "wide_70x21": I.FanGeometry(70, 21, 1.0, 1.0, 9, 64, 0.012, 0.25, 200.0, 300.0, I.FLAT),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_persistent_equals_per_iteration_armijo(name):
    g = GEOMS[name]
    geo = E.Geometry(g)
    y = t32(I.random_sino(g, 5) * 0.05 + 0.5).reshape(-1)
    p = I.EptvParams(n_outer=3)
    ra, rb = _assert_same(geo, g, y, p)
    assert ra.n_launches < rb.n_launches          # one (P2) launch instead of 3 + n_gd + 1


@pytest.mark.parametrize("kw", [dict(step_rule=O.FIXED, t_fixed=2e-5), dict(max_trials=8),
                                dict(max_trials=12), dict(weights_mode=O.ONE),
                                dict(n_gd=1), dict(n_gd=3, max_trials=2)])
def test_persistent_equals_per_iteration_params(c1_case, kw):
    g = c1_case.geom
    geo = E.Geometry(g)
    p = I.EptvParams(n_outer=4, **kw)
    _assert_same(geo, g, t32(c1_case.y).reshape(-1), p)


def test_persistent_equals_per_iteration_prior_weights(c1_case):
    g = c1_case.geom
    geo = E.Geometry(g)
    rng = np.random.Generator(np.random.PCG64(3))
    w = t32(rng.uniform(0.05, 1.0, (g.ny, g.nx))).reshape(-1)
    p = I.EptvParams(n_outer=4, weights_mode=O.PRIOR, prior_iters=2)
    _assert_same(geo, g, t32(c1_case.y).reshape(-1), p, wprior=w)


def test_persistent_equals_per_iteration_benchmark_workload():
    """512^2 (2 x 4-tile regions, one block per SM), 40 x 888, in the benchmark's shapes."""
    c = I.make_c2(with_truth=False)
    g = c.geom
    geo = E.Geometry(g)
    E.eptv_autotune(geo)
    ra, rb = _assert_same(geo, g, t32(c.y).reshape(-1), I.EptvParams(n_outer=3))
    # per outer iteration: 3 sigma, n_gd GD and 1 clamp launches became the one persistent
    # launch, which also applies the CGLS's last u += a s as it loads v
    assert rb.n_launches - ra.n_launches == 3 * 14
    assert ra.n_launches == 3 * 12 + 6                # K1 x 4, K2 x 3, K3 x 4, K4p; 6 per call


def test_persistent_tv_step_with_weights(c1_case):
    """eptv_tv_step: f, the final edge weights, and every statistic."""
    g = c1_case.geom
    geo = E.Geometry(g)
    rng = np.random.Generator(np.random.PCG64(9))
    v = t32(np.clip(c1_case.f_true + 0.002 * rng.standard_normal(c1_case.f_true.shape), 0, None)).reshape(-1)
    p = I.EptvParams(n_gd=7)
    out = []
    for mode in (E.TV_AUTO, E.TV_PER_ITERATION):
        E.eptv_set_tv_kernel(geo, mode)
        f = torch.empty(g.n_pix, device=DEV)
        w = torch.full((2 * (g.ny + 1) * (g.nx + 1),), -1.0, device=DEV)
        st, t_prev = E.eptv_tv_step(geo, p, v, f, weights=w, t_prev=3e-4)
        out.append((f, w, st, t_prev))
    (fa, wa, sa, ta), (fb, wb, sb, tb) = out
    assert torch.equal(fa, fb) and torch.equal(wa, wb)
    assert ta == tb
    assert (sa.sigma, sa.energy_first, sa.energy_last, sa.n_accepted, sa.n_fail) == \
           (sb.sigma, sb.energy_first, sb.energy_last, sb.n_accepted, sb.n_fail)


def test_persistent_wait_runs_out_and_the_handle_recovers(c1_case):
    """The grid barrier waits for one phantom block that never arrives: every wait runs out
    after ~1 ms, the kernel stops, the call reports EPTV_ERR_TIMEOUT, the context stays
    usable, and with the hook removed the next solve equals the per-iteration result."""
    g = c1_case.geom
    geo = E.Geometry(g)
    y = t32(c1_case.y).reshape(-1)
    p = I.EptvParams(n_outer=2)
    E.eptv_debug_set_p2_wait(geo, 1, 2_000_000)
    f = torch.zeros(g.n_pix, device=DEV)
    with pytest.raises(E.EptvError) as ei:
        E.eptv_reconstruct(geo, p, y, f)
    assert ei.value.code == -4
    torch.cuda.synchronize()
    E.eptv_debug_set_p2_wait(geo, 0, 2_000_000_000)
    _assert_same(geo, g, y, p)


@pytest.mark.parametrize("mode", [E.TV_AUTO, E.TV_PER_ITERATION])
def test_nan_in_the_p2_input_raises_nonfinite(c1_case, mode):
    """A NaN pixel of v makes its half-edge magnitudes NaN: the sigma selection of either
    kernel flags it, the call reports EPTV_ERR_NONFINITE, and the handle stays usable."""
    g = c1_case.geom
    geo = E.Geometry(g)
    E.eptv_set_tv_kernel(geo, mode)
    v = t32(c1_case.f_true).reshape(-1).clone()
    v[g.nx * (g.ny // 2) + g.nx // 2] = float("nan")
    f = torch.empty(g.n_pix, device=DEV)
    with pytest.raises(E.EptvError) as ei:
        E.eptv_tv_step(geo, I.EptvParams(n_gd=3), v, f, t_prev=3e-4)
    assert ei.value.code == -3
    st, _ = E.eptv_tv_step(geo, I.EptvParams(n_gd=3), t32(c1_case.f_true).reshape(-1), f, t_prev=3e-4)
    assert torch.isfinite(f).all() and st.sigma > 0


def test_persistent_equals_per_iteration_over_many_launches(c1_case):
    """30 outer iterations: 30 cooperative launches in a row, each starting its barriers
    where the previous one left the counter and re-arming its accumulator sets and
    selection histograms itself, against the per-iteration kernels."""
    g = c1_case.geom
    geo = E.Geometry(g)
    _assert_same(geo, g, t32(c1_case.y).reshape(-1), I.EptvParams(n_outer=30))


def _accepted_indices(steps, p):
    """The accepted trial of every GD iteration (max_trials for a failed search) from the
    step log: t0 = min(grow t_prev, t_max), the accepted step t0 shrink^m."""
    t_prev, out = p.t_init_eff, []
    for s in np.asarray(steps, dtype=np.float64).reshape(-1):
        t0 = min(p.armijo_grow * t_prev, p.t_max_eff)
        if s == 0.0:
            out.append(p.max_trials)
            t_prev = t0 * p.armijo_shrink ** (p.max_trials - 1) * p.armijo_shrink / p.armijo_grow
        else:
            out.append(int(round(np.log(t0 / s) / np.log(1.0 / p.armijo_shrink))))
            t_prev = s
    return np.array(out)


@pytest.mark.parametrize("kw", [dict(armijo_grow=8.0), dict(armijo_grow=8.0, max_trials=8),
                                dict(armijo_c=0.9), dict(max_trials=3)])
def test_persistent_second_trial_evaluation(c1_case, kw):
    """The persistent kernel evaluates the first three Armijo trials before a GD
    iteration's barrier and the others behind one more barrier, only when none of the
    three passes.  A growth factor of 8 (or c = 0.9) makes that frequent, failed searches
    included; images, logs and scalars must still equal one evaluation of every trial, over
    6 launches whose barrier counts differ."""
    g = c1_case.geom
    geo = E.Geometry(g)
    p = I.EptvParams(n_outer=6, **kw)
    ra, _ = _assert_same(geo, g, t32(c1_case.y).reshape(-1), p)
    steps, _ = E.eptv_get_log(geo)
    idx = _accepted_indices(steps, p)
    assert np.all((idx >= 0) & (idx <= p.max_trials))
    assert ra.n_fail == int(np.sum(idx == p.max_trials))
    if p.max_trials > 3:
        assert np.any(idx >= 3)            # some iteration needed the second evaluation
