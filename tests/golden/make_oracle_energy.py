"""Writes the FP64 oracle's final reported energy (Eq. 2) for a synthetic workload.

Calls only the oracle and the seeded input generator.  The stored value is the target
of the time-to-oracle-energy measurement: E(f_oracle) after the workload's iterations,
with sigma_ref = the oracle's last sigma.

    python tests/golden/make_oracle_energy.py c2   # 512x512, 40 x 888, 100 iterations
    python tests/golden/make_oracle_energy.py c1   # 128x128, 30 x 256, 50 iterations
    python tests/golden/make_oracle_energy.py c4 1 # 256x256, 30 x 888, 50 iterations, seed 1
    python tests/golden/make_oracle_energy.py c3 100  # one slice of the batched workload
                                                      # (seed 100: 512^2; 101: 256^2; 102: 384^2)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import eptv_oracle as O                     # noqa: E402
from paper_1009_2288_b300 import inputs as I            # noqa: E402


def main(which: str, seed=None):
    if which == "c4":
        case = I.make_c4(int(seed), with_truth=True)
        which = f"c4_seed{int(seed)}"
    elif which == "c3":
        case = I.make_c3_slice(int(seed), with_truth=True)
        which = f"c3_seed{int(seed)}"
    else:
        case = {"c1": I.make_c1, "c2": I.make_c2}[which](with_truth=True)
    p = I.EptvParams(n_outer=case.n_outer)
    op = O.Operator(case.geom)
    log = O.ReconLog()
    t0 = time.time()
    f = O.reconstruct(op, case.y, p, log=log)
    dt = time.time() - t0
    sigma_ref = log.sigmas[-1]
    # energy trajectory of the oracle itself (for iterations-to-energy of the oracle)
    energies = []
    g = case.geom
    import numpy as np
    fk = np.zeros((g.ny, g.nx))
    t_prev = p.t_init_eff
    for k in range(case.n_outer):
        v = O.cgls(op, case.y, fk, p.cgls_iters)
        fk, st = O.p2_solve(v, p, t_prev)
        t_prev = st.t_prev
        fk = np.maximum(fk, 0.0)
        energies.append(O.report_energy(op, fk, case.y, p, sigma_ref))
    out = {
        "workload": case.name,
        "seed": case.seed,
        "n_outer": case.n_outer,
        "params": {k: getattr(p, k) for k in p.__dataclass_fields__},
        "sigma_ref": sigma_ref,
        "e_report_final": O.report_energy(op, f, case.y, p, sigma_ref),
        "e_report_per_iteration": energies,
        "rel_error_vs_truth": float(((f - case.f_true) ** 2).sum() / (case.f_true ** 2).sum()),
        "oracle_seconds": dt,
        "line_search_failures": log.fails,
    }
    path = os.path.join(HERE, f"{which}_oracle_energy.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, out["e_report_final"], f"{dt:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "c2", sys.argv[2] if len(sys.argv) > 2 else None)
