"""The FIFO sweep by columns of rests (VI_KERNEL_FIFO_COL) against the FP64
oracle, through the C ABI.

The kernel computes the expectation of the column's first rest over the demand
and those of the column's other rests from the recurrence
C(x, r + 1, a) = C(x + 1, r, a) - P(D > x) (ref(r + 1, a) - ref(r, a)).

Values: max|V_gpu - V_oracle| / max|V_oracle| <= 1e-5 at the oracle's stopping
iteration; policies equal except ties whose FP64 Q-gap is <= 1e-6 relative; the
device stopping test within two sweeps of the oracle's.  The shapes cover every
pmf capacity (dmax up to 14, 30, 46 and 62), the smallest and largest radix
(Q+1 = 2 and 32), m = 2 (the arrival is the only stock slot of the rest), lead
times 2 to 4, a column count that leaves the last block of four columns ragged,
demand below the order cap (dmax < Q), zero demand, lead time one (the order
is the freshest stock slot and its own reward row enters each order's key:
m = 3..6, Q+1 up to 32, config 1's shape), and the 4.08M-state instance in the
launch configuration the benchmark times.
"""
import numpy as np
import pytest
import torch

import workloads
from workloads import FIFO, LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle, sampled_backup_parity, solve_parity  # noqa: E402

K = vi.VI_KERNEL_FIFO_COL

# (m, L, Q, Poisson mean, dmax, gamma); columns = (Q+1)^(m+L-4), four per block
SHAPES = [
    (3, 2, 6, 3.0, 12, 0.95),     # 7 columns: two blocks, the last with three
    (4, 2, 5, 4.0, 14, 0.9),      # dmax 14, the largest of the 16-entry capacity
    (3, 3, 4, 3.0, 20, 0.95),     # lead time 3
    (2, 2, 10, 5.0, 25, 0.9),     # m = 2: the arrival is the rest's only stock slot
    (2, 4, 3, 1.5, 9, 0.9),       # lead time 4
    (4, 2, 20, 8.0, 40, 0.99),    # config 2's radix and pmf capacity on 194,481 states
    (3, 2, 31, 10.0, 46, 0.9),    # Q+1 = 32, dmax 46
    (3, 2, 8, 6.0, 62, 0.9),      # dmax 62, the largest supported
    (3, 2, 12, 1.0, 4, 0.95),     # dmax < Q: the expectations vanish early
    (4, 2, 3, 2.0, 0, 0.9),       # deterministic zero demand
    (5, 2, 1, 0.7, 5, 0.9),       # Q+1 = 2, four stock slots
    (3, 1, 20, 5.0, 25, 0.99),    # lead time one: config 1's shape (one column)
    (4, 1, 6, 3.0, 14, 0.9),      # lead time one, 7 columns
    (5, 1, 4, 2.0, 30, 0.95),     # lead time one, 25 columns, dmax 30
    (3, 1, 31, 8.0, 46, 0.9),     # lead time one, Q+1 = 32
    (6, 1, 3, 1.5, 10, 0.9),      # lead time one, four rest slots
]


def _inst(m, L, Q, mu, dmax, gamma, seed=0):
    rng = np.random.default_rng(seed + 31 * m + 7 * L + Q)
    cost = tuple(float(c) for c in rng.uniform(1.0, 10.0, 4)) + (0.0,)
    return workloads.single_product(m, L, Q, cost, workloads.poisson_pmf(mu, dmax), gamma, FIFO)


@pytest.mark.parametrize("shape", SHAPES, ids=[f"m{s[0]}L{s[1]}Q{s[2]}D{s[4]}" for s in SHAPES])
def test_fifo_col_solve_matches_oracle(shape):
    inst = _inst(*shape)
    with Handle(inst, precision="fp32", kernel=K) as H:
        assert vi.vi_problem_kernel(H.h) == (K, 0)
    solve_parity(inst, "fp32", kernel=K)


def test_fifo_col_revenue_and_config2_costs():
    # config 2's demand and costs on 9,261 states (m = 3), with a revenue term
    p2 = workloads.config2().products[0]
    inst = workloads.single_product(3, 2, p2.Q, tuple(p2.cost[:4]) + (1.5,), p2.pmf, 0.99, FIFO)
    solve_parity(inst, "fp32", kernel=K)


def test_fifo_col_config2_full_size_sampled():
    # 4,084,101 states, the benchmark's workload and launch configuration
    sampled_backup_parity(workloads.config2(), 3, 400, 45, "fp32", kernel=K)


@pytest.mark.parametrize("L", [2, 1])
def test_fifo_col_matches_factorised_group_kernel(L):
    # the column recurrence and the direct sums over the demand agree after many sweeps
    inst = _inst(4 if L == 2 else 5, L, 9, 4.0, 20, 0.95, seed=3)
    with Handle(inst, precision="fp32", kernel=K) as A, Handle(inst, precision="fp32", kernel=vi.VI_KERNEL_GROUP) as B:
        Va, pa, ia = A.solve(0.0, 25)
        Vb, pb, ib = B.solve(0.0, 25)
        va, vb = A.v_abs(Va, ia), B.v_abs(Vb, ib)
        assert np.abs(va - vb).max() <= 1e-6 * np.abs(vb).max()
        assert abs(ia["dmax"] - ib["dmax"]) <= 1e-6 * np.abs(vb).max()


def test_fifo_col_extraction_and_host_loop():
    # the extraction sweep's policy and the host-driven loop give the graph loop's results
    inst = _inst(3, 3, 5, 2.5, 15, 0.95, seed=5)
    with Handle(inst, precision="fp32", kernel=K) as H:
        Vg, pg, ig = H.solve(1e-4, 5000)
        Vh, ph, ih = H.solve(1e-4, 5000, flags=vi.VI_FLAG_NO_GRAPH)
        assert ig["iters"] == ih["iters"]
        assert torch.equal(Vg, Vh) and torch.equal(pg, ph)


def test_fifo_col_rejected_where_unsupported():
    pmf = workloads.poisson_pmf(3, 12)
    bad = [workloads.single_product(3, 2, 32, (3, 1, 5, 7, 0), pmf, 0.9, FIFO),                        # Q+1 = 33
           workloads.single_product(3, 2, 6, (3, 1, 5, 7, 0), workloads.poisson_pmf(20, 63), 0.9, FIFO),  # dmax 63
           workloads.single_product(2, 1, 6, (3, 1, 5, 7, 0), pmf, 0.9, FIFO),                        # L = 1, m = 2
           workloads.single_product(4, 2, 6, (3, 1, 5, 7, 0), pmf, 0.9, LIFO),                        # LIFO
           workloads.single_product(1, 3, 6, (3, 1, 5, 7, 0), pmf, 0.9, FIFO)]                        # m = 1
    for inst in bad:
        with Handle(inst, precision="fp32") as H:
            with pytest.raises(vi.ViError):
                vi.vi_problem_set_option(H.h, vi.VI_OPT_KERNEL, K)
    inst = _inst(3, 2, 6, 3.0, 12, 0.9)
    for prec in ("fp64", "fp32_single", "fp32_kahan"):
        with Handle(inst, precision=prec) as H:
            with pytest.raises(vi.ViError):
                vi.vi_problem_set_option(H.h, vi.VI_OPT_KERNEL, K)
