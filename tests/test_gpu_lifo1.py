"""The persistent LIFO sweep for lead time one (VI_KERNEL_LIFO_L1) against the
FP64 oracle, through the C ABI.

Values: max|V_gpu - V_oracle| / max|V_oracle| <= 1e-5 at the oracle's stopping
iteration; policies equal except ties whose FP64 Q-gap is <= 1e-6 relative; the
device stopping test within two sweeps of the oracle's.  The shapes span several
128-rest tiles with a ragged last tile, both pmf capacities (dmax < 16 and
16..31), the smallest and largest radix (Q+1 = 2 and 16), a single rest (m = 2),
demand that stops inside the rest (dmax < units held) and, at full size (the
19.5M-state instance in the launch configuration the benchmark times and a
62.7M-state one of another radix), the columns of rests along X_{m-1} whose H
part follows from rest to rest.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from workloads import LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle, sampled_backup_parity, solve_parity  # noqa: E402

K = vi.VI_KERNEL_LIFO_L1

# (m, Q, Poisson mean, dmax, gamma): rests = (Q+1)^(m-2), tiles of 128 rests
SHAPES = [
    (5, 10, 4.0, 15, 0.95),    # 1331 rests: 11 tiles, last holds 51
    (5, 6, 3.0, 12, 0.9),      # 343 rests: 3 tiles, last holds 87
    (6, 4, 2.5, 9, 0.95),      # 625 rests, dmax below most rests' stock
    (4, 15, 7.0, 25, 0.9),     # Q+1 = 16, 32-entry pmf
    (5, 10, 8.0, 31, 0.95),    # 32-entry pmf at its limit
    (5, 5, 6.0, 20, 0.99),
    (10, 1, 1.2, 6, 0.9),      # Q+1 = 2, eight rest slots
    (2, 7, 3.0, 10, 0.9),      # m = 2: one rest, no rest slots
    (3, 12, 5.0, 14, 0.95),    # one rest slot
    (7, 3, 1.5, 0, 0.9),       # deterministic zero demand
]


def _inst(m, Q, mu, dmax, gamma, seed=0):
    rng = np.random.default_rng(seed + 17 * m + Q)
    cost = tuple(float(c) for c in rng.uniform(1.0, 10.0, 4)) + (0.0,)
    return workloads.single_product(m, 1, Q, cost, workloads.poisson_pmf(mu, dmax), gamma, LIFO)


@pytest.mark.parametrize("shape", SHAPES, ids=[f"m{s[0]}Q{s[1]}D{s[3]}" for s in SHAPES])
def test_lifo1_solve_matches_oracle(shape):
    inst = _inst(*shape)
    with Handle(inst, precision="fp32", kernel=K) as H:
        assert vi.vi_problem_kernel(H.h) == (K, 0)
    solve_parity(inst, "fp32", kernel=K)


def test_lifo1_config4_rescaled_costs():
    # the config-4 demand and costs on a 14,641-state instance (m = 5), with revenue
    p4 = workloads.config4().products[0]
    inst = workloads.single_product(5, 1, p4.Q, tuple(p4.cost[:4]) + (2.0,), p4.pmf, 0.95, LIFO)
    solve_parity(inst, "fp32", kernel=K)


def test_lifo1_config4_full_size_sampled():
    # 19,487,171 states, the benchmark's workload and launch configuration
    sampled_backup_parity(workloads.config4(), 3, 400, 44, "fp32", kernel=K)


def test_lifo1_columns_other_radix_sampled():
    # 13^7 = 62,748,517 states: enough column tiles (13^5 / 32) for every warp to walk whole
    # columns of rests along X_{m-1} (the H part carried from rest to rest) before the
    # leftover rests are dealt out one at a time; smaller instances compute every rest afresh
    inst = _inst(8, 12, 5.0, 15, 0.95, seed=8)
    assert inst.n_states == 13 ** 7
    sampled_backup_parity(inst, 3, 400, 46, "fp32", kernel=K)


def test_lifo1_matches_factorised_group_kernel():
    # the two factorised LIFO sweeps agree with each other after several sweeps
    inst = _inst(6, 5, 3.0, 14, 0.95, seed=3)
    with Handle(inst, precision="fp32", kernel=K) as A, Handle(inst, precision="fp32", kernel=vi.VI_KERNEL_GROUP) as B:
        Va, pa, ia = A.solve(0.0, 25)
        Vb, pb, ib = B.solve(0.0, 25)
        va, vb = A.v_abs(Va, ia), B.v_abs(Vb, ib)
        assert np.abs(va - vb).max() <= 1e-6 * np.abs(vb).max()
        assert abs(ia["dmax"] - ib["dmax"]) <= 1e-6 * np.abs(vb).max()


def test_lifo1_rejected_where_unsupported():
    bad = [workloads.single_product(4, 1, 16, (3, 1, 5, 7, 0), workloads.poisson_pmf(4, 15), 0.9, LIFO),  # Q+1 = 17
           workloads.single_product(4, 1, 6, (3, 1, 5, 7, 0), workloads.poisson_pmf(9, 32), 0.9, LIFO),   # dmax 32
           workloads.single_product(4, 2, 6, (3, 1, 5, 7, 0), workloads.poisson_pmf(3, 12), 0.9, LIFO),   # L = 2
           workloads.single_product(4, 1, 6, (3, 1, 5, 7, 0), workloads.poisson_pmf(3, 12), 0.9, 0)]      # FIFO
    for inst in bad:
        with Handle(inst, precision="fp32") as H:
            with pytest.raises(vi.ViError):
                vi.vi_problem_set_option(H.h, vi.VI_OPT_KERNEL, K)
    inst = _inst(5, 6, 3.0, 12, 0.9)
    for prec in ("fp64", "fp32_single", "fp32_kahan"):
        with Handle(inst, precision=prec) as H:
            with pytest.raises(vi.ViError):
                vi.vi_problem_set_option(H.h, vi.VI_OPT_KERNEL, K)


def test_lifo1_host_loop_matches_graph():
    inst = _inst(5, 10, 4.0, 15, 0.95, seed=9)
    with Handle(inst, precision="fp32", kernel=K) as H:
        Vg, pg, ig = H.solve(1e-4, 5000)
        Vh, ph, ih = H.solve(1e-4, 5000, flags=vi.VI_FLAG_NO_GRAPH)
        assert ig["iters"] == ih["iters"]
        assert torch.equal(Vg, Vh) and torch.equal(pg, ph)


def test_misaligned_value_buffers_rejected():
    # value buffers must sit on their element size; nothing is launched otherwise
    inst = _inst(5, 6, 3.0, 12, 0.9)
    with Handle(inst, precision="fp32", kernel=K) as H:
        n = H.sizes["n_states"]
        raw = torch.zeros(2 * n + 1, dtype=torch.float32, device="cuda")
        bad = raw[1:]                                  # 4 bytes past an 8-byte boundary
        good = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(vi.ViError):
            vi.vi_backup(H.h, bad, good, None)
        with pytest.raises(vi.ViError):
            vi.vi_backup(H.h, good, bad, None)
        with pytest.raises(vi.ViError):
            vi.vi_solve(H.h, 1e-4, 10, bad)
