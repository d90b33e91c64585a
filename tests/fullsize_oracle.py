"""Whole FP64 oracle solves of the full-size configurations, for the GPU parity
tests of test_gpu_whole_solves.py (test infrastructure).

    python tests/fullsize_oracle.py OUT_DIR cfg4 cfg2 cfg3

Runs the oracle's value iteration (span test, tol 1e-4, OpenMP over the host
cores) on each named configuration in turn and writes OUT_DIR/<cfg>.npz holding
V, the policy, the stopping sweep and the solve's wall time; a failure writes
OUT_DIR/<cfg>.err.  Started in a subprocess by the test session so that the
host-core work overlaps the other GPU tests.
"""
import json
import os
import sys
import time
import traceback

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

TOL = 1e-4
MAX_ITERS = 5000
CONFIGS = {"cfg2": workloads.config2, "cfg3": workloads.config3, "cfg4": workloads.config4}


def main(out_dir, names):
    os.makedirs(out_dir, exist_ok=True)
    for name in names:
        try:
            inst = CONFIGS[name]()
            t0 = time.perf_counter()
            ref = oracle.Problem(inst).vi_solve(tol=TOL, max_iters=MAX_ITERS, stop_rule=0)
            dt = time.perf_counter() - t0
            tmp = os.path.join(out_dir, f"{name}.tmp.npz")
            np.savez(tmp, V=ref["V"], policy=ref["policy"], iters=ref["iters"], converged=ref["converged"],
                     seconds=dt, cores=os.cpu_count() or 1)
            os.replace(tmp, os.path.join(out_dir, f"{name}.npz"))
            print(json.dumps({"config": name, "iters": ref["iters"], "seconds": dt}), flush=True)
        except Exception:
            with open(os.path.join(out_dir, f"{name}.err"), "w") as f:
                f.write(traceback.format_exc())


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2:])
