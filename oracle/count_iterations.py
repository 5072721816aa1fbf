"""Runs the oracle's FP64 CGNR to a 1e-10 true residual on the 24^3x64 twisted-mass
clover workload (c_sw 1.05, m 0.05, mu 0.01, gauge seed 102, Z2 source seed 202)
and writes the iteration count to tests/golden/oracle_cgnr_24x24x24x64.json.

The benchmark's CPU-baseline leg times a bounded number of oracle iterations and
scales them by this count to a time per solve. Test infrastructure only; calls
nothing but the oracle and the input generator. Takes about 15 minutes on 8 cores.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2201_09004_b300 import synth  # noqa: E402

DIMS = (24, 24, 24, 64)


def main():
    U = synth.thin_links(DIMS, 102).numpy()
    C = oracle.clover(DIMS, U, 1.05)
    b = synth.z2_source(DIMS, 202).numpy()
    W = oracle.Wilson(DIMS, U, 0.05, 0.01, clover=C)
    t = time.time()
    x, info = W.cgnr(b, tol=1e-10, maxiter=20000)
    out = {"workload": "wilson twisted-mass clover 24^3x64, c_sw=1.05, m=0.05, mu=0.01, gauge seed 102, "
                       "Z2 source seed 202, full lattice FP64 CGNR to true residual 1e-10",
           "iterations": info["iters"], "true_rel_residual": info["true_rel_residual"],
           "status": info["status"], "seconds": time.time() - t, "threads": os.cpu_count()}
    path = os.path.join(os.path.dirname(HERE), "tests", "golden", "oracle_cgnr_24x24x24x64.json")
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
