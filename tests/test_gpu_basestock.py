"""Base-stock policy search by simulation (Methods, Scenario A heuristic,
A = [S - I]^+): every (S, rollout) return equals the oracle's rollout of the
same policy written out state by state, bit for bit, and the search picks the
same S."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from workloads import FIFO, LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle  # noqa: E402

C1 = (3.0, 1.0, 5.0, 7.0, 0.0)
C2 = (2.0, 1.5, 6.0, 4.0, 1.0)
CASES = [
    workloads.single_product(2, 1, 8, C1, workloads.poisson_pmf(4.0, 15), 0.9, FIFO),
    workloads.single_product(3, 2, 6, C2, workloads.poisson_pmf(3.0, 12), 0.95, LIFO),
    workloads.single_product(4, 1, 5, C1, workloads.negbin_pmf(2.5, 6.0, 14), 0.9, LIFO),
    workloads.single_product(3, 3, 7, C2, workloads.poisson_pmf(3.5, 16), 0.99, FIFO),
]


@pytest.mark.parametrize("inst", CASES, ids=[f"c{i}" for i in range(len(CASES))])
def test_basestock_returns_bit_exact(inst):
    p = inst.products[0]
    P = oracle.Problem(inst)
    n, H, W, seed = 300, 50, 10, 77
    s_lo, s_hi = 0, p.Q + 4   # past Q the order is capped
    with Handle(inst, precision="fp32") as Hh:
        ret = torch.empty((s_hi - s_lo + 1) * n, dtype=torch.float64, device="cuda")
        means, best = vi.vi_basestock_search(Hh.h, s_lo, s_hi, n, H, W, seed, ret)
        torch.cuda.synchronize()
        got = ret.cpu().numpy().reshape(s_hi - s_lo + 1, n)
        ref_means = []
        for i, S in enumerate(range(s_lo, s_hi + 1)):
            want = P.simulate(P.basestock_policy(S), n, H, seed, warmup=W)["returns"]
            np.testing.assert_array_equal(got[i], want)
            ref_means.append(sum(want) / n)      # rollout order, as the library sums
        np.testing.assert_array_equal(means, np.array(ref_means))
        assert best == s_lo + int(np.argmax(ref_means))


def test_basestock_matches_simulate_with_the_policy_array():
    """The search kernel and vi_simulate fed the materialised policy agree."""
    inst = CASES[1]
    P = oracle.Problem(inst)
    n, H, W, seed = 256, 40, 5, 3
    with Handle(inst, precision="fp32") as Hh:
        ret = torch.empty(n, dtype=torch.float64, device="cuda")
        vi.vi_basestock_search(Hh.h, 5, 5, n, H, W, seed, ret)
        pol = torch.tensor(P.basestock_policy(5), device="cuda")
        r2 = torch.empty(n, dtype=torch.float64, device="cuda")
        vi.vi_simulate(Hh.h, pol, n, H, W, seed, r2)
        torch.cuda.synchronize()
        assert torch.equal(ret, r2)


def test_basestock_config4_sampled():
    """The 19.5M-state LIFO instance: two order-up-to levels, bit-exact with the oracle."""
    inst = workloads.config4()
    P = oracle.Problem(inst)
    n, H, W, seed = 128, 60, 20, 4
    with Handle(inst, precision="fp32") as Hh:
        ret = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        vi.vi_basestock_search(Hh.h, 6, 7, n, H, W, seed, ret)
        got = ret.cpu().numpy().reshape(2, n)
        for i, S in enumerate((6, 7)):
            want = P.simulate(P.basestock_policy(S), n, H, seed, warmup=W)["returns"]
            np.testing.assert_array_equal(got[i], want)


def test_basestock_rejects_bad_arguments():
    two = workloads.config3(Q=2)
    with Handle(CASES[0], precision="fp32") as Hh:
        ret = torch.empty(10, dtype=torch.float64, device="cuda")
        with pytest.raises(vi.ViError):
            vi.vi_basestock_search(Hh.h, 3, 2, 5, 10, 0, 1, ret)
        with pytest.raises(vi.ViError):
            vi.vi_basestock_search(Hh.h, 0, 1, 0, 10, 0, 1, ret)
    with Handle(two) as Ht:
        with pytest.raises(vi.ViError):
            vi.vi_basestock_search(Ht.h, 0, 1, 5, 10, 0, 1, torch.empty(10, dtype=torch.float64, device="cuda"))
