"""The sweep kernels near the largest state counts the library accepts (|S| < 2^32),
against the FP64 oracle at sampled states, through the C ABI.

2,562,890,625 states (LIFO, L = 1, Q+1 = 15, past 2^31: every state index, tile
offset and gather address is above the signed 32-bit range somewhere) on the
persistent LIFO kernel, 1,801,088,541 states (FIFO, two pipeline slots) on
the factorised kernel and 2,494,357,888 states (FIFO, lead time 2) on the FIFO
column kernel.  The oracle needs V only at the next states of the sampled
states: those values are gathered on the device (vi_next_states gives their
indices) into a zero-filled host array whose other pages are never touched.
Checked: one backup's values (max relative error <= 1e-5), its first argmax up to
ties, and the sweep's change statistics against max / min of V_next - V_k
reduced on the device in slices.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from workloads import FIFO, LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle, V_RTOL, policy_mismatches  # noqa: E402


def _abs_at(V: torch.Tensor, idx: torch.Tensor) -> torch.Tensor:
    """V_abs = hi + lo of the float pairs at the given states (FP64)."""
    p = V.view(torch.float32).reshape(-1, 2)[idx]
    return p[:, 0].double() + p[:, 1].double()


def _sparse_values(H, V: torch.Tensor, states: np.ndarray) -> np.ndarray:
    """A host array of |S| zeros holding V_abs at every next state of `states`."""
    n = H.sizes["n_states"]
    per = H.sizes["n_actions"] * H.sizes["n_outcomes"]
    st = torch.as_tensor(states.astype(np.uint32).view(np.int32), device="cuda")
    out = torch.empty(len(states) * per, dtype=torch.int32, device="cuda")
    vi.vi_next_states(H.h, st, len(states), out)
    idx = out.to(torch.int64) & 0xFFFFFFFF        # uint32 indices held in int32
    vals = _abs_at(V, idx).cpu().numpy()
    host = np.zeros(n, dtype=np.float64)          # untouched pages stay unallocated
    host[idx.cpu().numpy()] = vals
    return host


def _max_size_backup(inst, kernel, k_sweeps, n_samples, seed):
    P = oracle.Problem(inst)
    with Handle(inst, precision="fp32", kernel=kernel) as H:
        n = H.sizes["n_states"]
        V, pol, info = H.solve(0.0, k_sweeps)
        del pol
        V_next = torch.empty_like(V)
        pol_next = torch.empty(n, dtype=torch.uint8, device="cuda")
        dmx, dmn = vi.vi_backup(H.h, V, V_next, pol_next)
        torch.cuda.synchronize()
        rng = np.random.default_rng(seed)
        edge = [0, n - 1, (1 << 31) - 1, 1 << 31, n // 2] if n > (1 << 31) else [0, n - 1, n // 2]
        states = np.unique(np.concatenate([edge, rng.integers(0, n, n_samples)])).astype(np.int64)
        v_k = _sparse_values(H, V, states)
        want, _ = P.backup_states(v_k, states)
        got = _abs_at(V_next, torch.as_tensor(states, device="cuda")).cpu().numpy()
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= V_RTOL, err
        bad = policy_mismatches(P, v_k, pol_next[torch.as_tensor(states, device="cuda")].cpu().numpy(), states)
        assert not bad, bad[:5]
        # change statistics over every state, reduced on the device in slices
        hi, lo = -np.inf, np.inf
        step = 1 << 28
        for s0 in range(0, n, step):
            a = V_next[s0:s0 + step].view(torch.float32).reshape(-1, 2)
            b = V[s0:s0 + step].view(torch.float32).reshape(-1, 2)
            d = (a[:, 0].double() - b[:, 0].double()) + (a[:, 1].double() - b[:, 1].double())
            hi, lo = max(hi, float(d.max())), min(lo, float(d.min()))
            del a, b, d
        scale = max(1.0, float(np.abs(want).max()))
        assert abs(dmx - hi) <= 1e-6 * scale and abs(dmn - lo) <= 1e-6 * scale, (dmx, hi, dmn, lo)
        kernel_run = vi.vi_problem_kernel(H.h)
        del V, V_next, pol_next
    torch.cuda.empty_cache()
    return kernel_run


def test_lifo_lead_time_one_past_2_31_states():
    inst = workloads.single_product(9, 1, 14, (3.0, 1.0, 5.0, 7.0, 0.0), workloads.poisson_pmf(4.0, 15), 0.95,
                                    LIFO)
    assert inst.n_states == 15 ** 8 > (1 << 31)
    k = _max_size_backup(inst, vi.VI_KERNEL_LIFO_L1, 2, 300, 61)
    assert k == (vi.VI_KERNEL_LIFO_L1, 0)


def test_fifo_pipeline_1_8e9_states():
    inst = workloads.single_product(6, 3, 20, (2.0, 1.0, 6.0, 3.0, 1.0), workloads.poisson_pmf(6.0, 20), 0.95,
                                    FIFO)
    assert inst.n_states == 21 ** 7
    k = _max_size_backup(inst, vi.VI_KERNEL_GROUP, 2, 300, 62)
    assert k[0] == vi.VI_KERNEL_GROUP


def test_fifo_column_past_2_31_states():
    # 22^7 = 2,494,357,888 states on the FIFO column kernel: column starts, state
    # indices and order offsets above the signed 32-bit range
    inst = workloads.single_product(7, 2, 21, (2.0, 1.0, 6.0, 3.0, 1.0), workloads.poisson_pmf(6.0, 20), 0.95,
                                    FIFO)
    assert inst.n_states == 22 ** 7 > (1 << 31)
    k = _max_size_backup(inst, vi.VI_KERNEL_FIFO_COL, 2, 300, 63)
    assert k == (vi.VI_KERNEL_FIFO_COL, 0)
