"""FP64 policy evaluation inside a solve and the compensated FP32 sweeps, against
the FP64 oracle through the C ABI.

VI_FLAG_POLICY_EVAL evaluates the extracted policy in FP64 from the solve's
values until the sup-norm change is below 1e-9, and reports the gap
max_s |V_pe(s) - V(s)|.  The oracle's fixed-policy evaluation (pinned to the dense
solve (I - gamma P_pi) V = r_pi) of the same GPU policy from the same start gives
the reference gap (and its span, max - min of V_pe - V) and sweep count.
"""
import numpy as np
import pytest

import oracle
import workloads
from workloads import FIFO, LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle, solve_parity  # noqa: E402

PE_CASES = {
    "two_products_Q2_kahan": (lambda: workloads.config3(Q=2), "fp32_kahan"),
    "two_products_Q2_fp32": (lambda: workloads.config3(Q=2), "fp32"),
    "m4L2Q6_fifo": (lambda: workloads.single_product(4, 2, 6, (2.0, 1.0, 6.0, 3.0, 0.0),
                                                     workloads.poisson_pmf(3.0, 12), 0.95, FIFO), "fp32"),
    "m5L1Q5_lifo": (lambda: workloads.single_product(5, 1, 5, (3.0, 1.0, 5.0, 7.0, 0.0),
                                                     workloads.poisson_pmf(2.0, 9), 0.9, LIFO), "fp32"),
    "cfg1_fp64": (workloads.config1, "fp64"),
}


@pytest.mark.parametrize("name", sorted(PE_CASES))
def test_policy_eval_flag_matches_oracle(name):
    make, prec = PE_CASES[name]
    inst = make()
    with Handle(inst, precision=prec) as H:
        V, pol, info = H.solve(1e-4, 5000, flags=vi.VI_FLAG_POLICY_EVAL)
        assert info["status"] == vi.VI_OK
        v = H.v_abs(V, info)
        policy = pol.cpu().numpy()
    scale = max(abs(info["offset"]), 1.0)
    V_pe, it, ok = oracle.Problem(inst).policy_eval(policy, tol=1e-9 * scale, max_iters=100000, V0=v)
    assert ok
    gap_ref = float(np.abs(V_pe - v).max())
    span_ref = float((V_pe - v).max() - (V_pe - v).min())
    assert abs(info["pe_gap"] - gap_ref) <= 1e-8 * np.abs(V_pe).max(), (info["pe_gap"], gap_ref)
    assert abs(info["pe_span"] - span_ref) <= 1e-8 * np.abs(V_pe).max(), (info["pe_span"], span_ref)
    # the GPU reads the change back after every 8th sweep: it stops at the first
    # multiple of 8 at or past the oracle's stop sweep (that sweep itself may move by
    # one under summation-order rounding when its change is that close to the tolerance)
    at_8 = {8 * -(-(it + k) // 8) for k in (-1, 0, 1)}
    assert info["pe_iters"] in at_8, (info["pe_iters"], it)
    assert info["pe_delta"] < 1e-9 * scale


def test_kahan_routes():
    # lead time one on both products: the factorised two-product sweep, compensated
    with Handle(workloads.config3(Q=4), precision="fp32_kahan") as H:
        assert vi.vi_problem_kernel(H.h) == (vi.VI_KERNEL_GROUP, 0)
    # lead times 2: the pipeline form has no compensated sums, so Kahan runs the generic kernel
    b = workloads.scenario_b("P1")
    with Handle(b, precision="fp32_kahan") as H:
        assert vi.vi_problem_kernel(H.h)[0] == vi.VI_KERNEL_GENERIC
    with Handle(b, precision="fp32") as H:
        assert vi.vi_problem_kernel(H.h) == (vi.VI_KERNEL_GROUP, 0)


@pytest.mark.parametrize("Q", [3, 5])
def test_kahan_two_product_sweep_matches_oracle(Q):
    solve_parity(workloads.config3(Q=Q), "fp32_kahan")


def test_kahan_pipeline_two_products_generic_matches_oracle():
    c1 = (0.5, 0.1, 0.3, 0.2, 1.0)
    c2 = (0.5, 0.2, 0.1, 0.4, 1.0)
    prods = [workloads.Product(3, 2, 3, c1, workloads.poisson_pmf(1.5, 7)),
             workloads.Product(3, 2, 3, c2, workloads.poisson_pmf(2.0, 8))]
    inst = workloads.Instance("pipe2", prods, gamma=0.9, issuing=FIFO, subst_rate=0.5)
    solve_parity(inst, "fp32_kahan")
