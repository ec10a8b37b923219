"""The benchmark's multi-rank path on the CPU: two processes joined over gloo on
127.0.0.1, as torchrun would start them (RANK / WORLD_SIZE / LOCAL_RANK / MASTER_* in the
environment).  Checks the rendezvous, the barrier, the whole-job rate (slowest rank's
time, all ranks' units), the per-rank slices of the replica run (no data-path
collective: each rank reconstructs its own seeded slice), and that the reference arm
runs on rank 0 only; also the CPU-baseline leg that times the oracle."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r, local = bench.dist_setup()
    import torch.distributed as dist
    try:
        assert dist.get_backend() == "gloo"
        bench.barrier(w)
        # rank r "took" 10 + 5 r ms for 100 units
        ms, value = bench.job_rate(10.0 + 5.0 * r, w, 100)
        seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(w)]
        dist.all_gather(seeds, torch.tensor([bench.replica_seed(r)]))
        res = {"rank": r, "world": w, "local": local, "ms": ms, "value": value,
               "seeds": [int(t.item()) for t in seeds]}
        with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
            json.dump(res, fh)
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_rate_and_slices(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == world and d["local"] == r
        assert d["ms"] == pytest.approx(15.0)                        # the slowest rank
        assert d["value"] == pytest.approx(world * 100 * 1e3 / 15.0)  # all ranks' units
        assert len(set(d["seeds"])) == world                          # one slice per rank


def test_single_process_rate_needs_no_process_group():
    import bench
    ms, value = bench.job_rate(20.0, 1, 100)
    assert ms == 20.0 and value == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(Args, 2, 1) is None
    assert capsys.readouterr().out == ""


def test_cpu_baseline_times_the_oracle_and_returns_its_image():
    """The bench's CPU leg times the oracle as it stands (on one core, and with its P and
    P^T on every host core) and hands its image on to the GPU-vs-oracle check (one outer
    iteration of the 128^2 workload here)."""
    import numpy as np
    import bench
    from oracle import eptv_oracle as O
    from paper_1009_2288_b300 import inputs as I
    case = I.make_c1(with_truth=False)
    cpu, f, op = bench.cpu_baseline(case, steps=1)
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0
    assert cpu["single_core"]["cores"] == 1 and cpu["single_core"]["value"] > 0 and cpu["cpu"]
    assert f.shape == (case.geom.ny, case.geom.nx) and np.all(f >= 0) and np.any(f > 0)
    assert np.array_equal(f, O.reconstruct(O.Operator(case.geom), case.y, I.EptvParams(n_outer=1)))
    assert isinstance(op, O.Operator)
