"""Whole solves of the full-size configurations against the FP64 oracle's whole
solves, every state compared, through the C ABI.

The oracle (plain FP64 value iteration on the host cores) runs each solve to its
own span test (tol 1e-4) in a subprocess started with the test session.  The GPU
then runs the same number of sweeps with the stopping test disabled, in the
kernels the benchmark times:
  - values: max_s |V_gpu(s) - V_oracle(s)| / max_s |V_oracle(s)| <= 1e-5, over all states;
  - policy: equal at every state except ties whose FP64 Q-gap (oracle Q-values
    from the oracle's V) is <= 1e-6 relative;
  - the GPU's own stopping test ends within two sweeps of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle, V_RTOL, compare_values, policy_mismatches  # noqa: E402

CASES = {"cfg4": workloads.config4, "cfg2": workloads.config2, "cfg3": workloads.config3}


def whole_solve_parity(name, fullsize_oracle):
    inst = CASES[name]()
    ref = fullsize_oracle(name)
    i_o = int(ref["iters"])
    assert bool(ref["converged"]) and i_o >= 2
    with Handle(inst) as H:
        V, pol, info = H.solve(0.0, i_o)
        assert info["iters"] == i_o
        v = H.v_abs(V, info)
        err = compare_values(v, ref["V"])
        assert err <= V_RTOL, f"{name}: value error {err:.3e} over {inst.n_states} states"
        pg = pol.cpu().numpy()
        diff = np.nonzero(pg != ref["policy"])[0]
        # every disagreement must be a tie of the oracle's Q-values
        bad = policy_mismatches(oracle.Problem(inst), ref["V"], pg[diff], diff) if len(diff) else []
        assert not bad, f"{name}: {len(bad)} non-tie policy differences, e.g. {bad[:3]}"
        V2, pol2, info2 = H.solve(1e-4, 5000)
        assert info2["status"] == vi.VI_OK and abs(info2["iters"] - i_o) <= 2, (info2["iters"], i_o)
        kernel = vi.vi_problem_kernel(H.h)
    print(f"\n{name}: {inst.n_states} states, {i_o} sweeps, max|dV|/max|V| = {err:.2e}, "
          f"{len(diff)} tie differences, kernel {kernel}, oracle {float(ref['seconds']):.0f} s on "
          f"{int(ref['cores'])} cores")


@pytest.mark.fullsize("cfg4")
def test_config4_whole_solve(fullsize_oracle):
    whole_solve_parity("cfg4", fullsize_oracle)


@pytest.mark.fullsize("cfg2")
def test_config2_whole_solve(fullsize_oracle):
    whole_solve_parity("cfg2", fullsize_oracle)


@pytest.mark.fullsize("cfg3")
def test_config3_whole_solve(fullsize_oracle):
    whole_solve_parity("cfg3", fullsize_oracle)
