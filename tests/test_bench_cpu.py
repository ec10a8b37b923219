"""Host-side pieces of the benchmark that its numbers rest on, checked on the CPU: the
nonzero count behind the roofline's algorithmic bytes (against the FP64 oracle's rows of
P), and the JSON line of the reference arm (the oracle timed on the host cores, its P and
P^T sharded over them)."""
import io
import json
from contextlib import redirect_stdout

import numpy as np
import pytest

import bench
from oracle import eptv_oracle as O
from paper_1009_2288_b300 import inputs as I


@pytest.mark.parametrize("make", [
    lambda: I.FanGeometry(24, 17, 1.3, 0.9, 7, 41, 0.02, 0.25, 80.0, 130.0, I.ARC),
    lambda: I.ge_geometry(64, 6.4, 9, 96, 0.958 / 96),
])
def test_nnz_count_equals_the_oracle_rows(make):
    """nnz(P) from each ray's chord (closed form: 1 + interior planes crossed) equals the
    number of nonzero entries of the oracle's rows, ray by ray summed."""
    g = make()
    sx, sy, ux, uy = O.rays(g)
    want = 0
    for i in range(g.n_rays):
        pix, ln = O.ray_row(g.nx, g.ny, g.dx, g.dy, sx[i], sy[i], ux[i], uy[i])
        want += int(np.count_nonzero(ln > 0))
    assert bench.nnz_of(g) == want


def test_reference_arm_prints_the_contract_line():
    class Args:
        steps, warmup, gpus = 1, 0, 1
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(Args, 1, 0)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "iterations/s" and line["value"] > 0 and line["higher_is_better"]
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["cores"] <= cb["host_cores"]
    assert cb["cpu"] and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
