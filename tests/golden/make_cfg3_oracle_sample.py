"""Writes cfg3_oracle_sample.json: the FP64 oracle's whole value-iteration solve of
the two-product configuration (2 x (m=3, L=1, Q=14), 50,625 states; span test,
tol 1e-4), kept at 2,048 seeded sampled states plus state 0 and the last state.
bench.py compares the GPU's solve of the same configuration, at the same sweep
count, with these values.  The file holds only what this script computes with the
oracle.

    python tests/golden/make_cfg3_oracle_sample.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads  # noqa: E402


def main():
    inst = workloads.config3()
    t0 = time.perf_counter()
    ref = oracle.Problem(inst).vi_solve(tol=1e-4, max_iters=5000, stop_rule=0)
    dt = time.perf_counter() - t0
    rng = np.random.default_rng(20231003)
    n = inst.n_states
    states = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 2048)]))
    out = {
        "what": "FP64 oracle value iteration of workloads.config3() (span test, tol 1e-4, V_0 = 0): values and "
                "first-argmax policy at sampled states after the oracle's stopping sweep",
        "workload": inst.name, "n_states": int(n), "iters": int(ref["iters"]), "tol": 1e-4,
        "max_abs_V": float(np.abs(ref["V"]).max()), "crit": float(ref["crit"]),
        "states": [int(s) for s in states], "V": [float(v) for v in ref["V"][states]],
        "policy": [int(a) for a in ref["policy"][states]], "oracle_seconds": dt,
    }
    with open(os.path.join(HERE, "cfg3_oracle_sample.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("iters", ref["iters"], "seconds %.0f" % dt)


if __name__ == "__main__":
    main()
