"""The learned warm start end to end: the GPU synthesis of training sinograms against the
host generator, and what the trained network gains over the method without it on held-out
phantoms of the learned workload (256^2, 30 views x 888 bins, I0 = 5e4), judged by the FP64
oracle's final reported energy (Eq. 2) stored in tests/golden."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1009_2288_b300 import eptv as E
from paper_1009_2288_b300 import inputs as I
from paper_1009_2288_b300 import learned as L

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_gpu_line_integrals_match_host_generator():
    g = I.ge_geometry(256, 1.6, 30)
    rays = L.RaySet(g, DEV)
    for s in (1, 5):
        want = I.make_c4(s, with_truth=False).p_clean.ravel()
        got = L.line_integrals_gpu(L.c4_ellipses(s, g), rays).cpu().numpy()
        assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()


@pytest.fixture(scope="module")
def trained():
    p = I.EptvParams(n_outer=50)
    pairs = L.make_pairs(list(range(20000, 20768)), p, device=DEV)
    net = L.UNet(seed=0, device=DEV)
    losses = L.train(net, pairs, epochs=30)
    return net, losses


def test_training_loss_decreases(trained):
    _, losses = trained
    assert np.mean(losses[-20:]) < 0.6 * np.mean(losses[:20])


@pytest.mark.parametrize("seed", [1, 2])
def test_warm_start_reaches_oracle_energy_in_fewer_iterations(trained, seed):
    """Plain EPTV from f = 0, the same solve from the network's base image alone (the method
    without the network), and from the learned warm start: iterations until the 5-iteration
    mean of E_report comes within 1e-3 of the oracle's final (last-5 mean) energy."""
    net, _ = trained
    gold = json.load(open(os.path.join(GOLD, f"c4_seed{seed}_oracle_energy.json")))
    target = float(np.mean(gold["e_report_per_iteration"][-5:]))
    sig = gold["sigma_ref"]
    g = I.ge_geometry(256, 1.6, 30)
    geo = E.Geometry(g)
    p = I.EptvParams(n_outer=50)
    y = torch.tensor(I.make_c4(seed, with_truth=False).y.astype(np.float32).ravel()).to(DEV)
    f = torch.zeros(g.n_pix, device=DEV)
    k_plain, _ = L.iterations_to_energy(geo, p, y, f, target, sig, 80)
    f.zero_()
    E.eptv_cgls(geo, L.M_BASE, y, f)
    f.clamp_(min=0.0)
    k_base, _ = L.iterations_to_energy(geo, p, y, f, target, sig, 80)
    warm = L.WarmStart(net, geo)
    warm(y, f)
    assert float(f.min()) >= 0.0
    k_learned, es = L.iterations_to_energy(geo, p, y, f, target, sig, 80)
    assert k_plain is not None and k_learned is not None, (k_plain, k_learned)
    assert k_learned <= 0.85 * k_plain, (k_learned, k_plain)
    assert k_base is None or k_learned < k_base, (k_learned, k_base)
