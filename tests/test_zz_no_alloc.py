"""vi_backup_noalloc: the sweep for callers that cannot allocate (inside an
allocator or memory pool that must not be re-entered, or with device memory
budgeted elsewhere).  Its output must equal vi_backup on a normally created
problem, and the FP64 oracle's backup at sampled states, within the parity
tolerance, on two calls in a row -- the second one checks that the shared
scratch left by the first call is reset -- and a call must leave the device's
free memory unchanged."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from workloads import FIFO, LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle, policy_mismatches, values_abs, V_RTOL  # noqa: E402


def reference_and_noalloc(inst, k_sweeps):
    p = inst.products[0]
    with Handle(inst, precision="fp32") as H:
        V, _, _ = H.solve(0.0, k_sweeps)                       # a non-trivial V_in
        n = H.sizes["n_states"]
        V_ref = torch.empty_like(V)
        pol_ref = torch.empty(n, dtype=torch.uint8, device="cuda")
        st_ref = vi.vi_backup(H.h, V, V_ref, pol_ref)
        V_na = torch.empty_like(V)
        pol_na = torch.empty(n, dtype=torch.uint8, device="cuda")
        st_na = vi.vi_backup_noalloc(p.m, p.L, p.Q, p.cost, p.pmf, inst.gamma, inst.issuing, V, V_na, pol_na)
        torch.cuda.synchronize()
        a = values_abs(V_ref, 0.0, "pair")
        b = values_abs(V_na, 0.0, "pair")
        scale = np.abs(a).max()
        assert np.abs(a - b).max() <= V_RTOL * scale
        assert abs(st_ref[0] - st_na[0]) <= V_RTOL * scale and abs(st_ref[1] - st_na[1]) <= V_RTOL * scale
        # against the oracle: one FP64 backup of the same V_in at sampled states, first
        # argmax up to ties of 1e-6 relative
        P = oracle.Problem(inst)
        v_in = values_abs(V, 0.0, "pair")
        rng = np.random.default_rng(inst.n_states)
        states = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 200)]))
        want, _ = P.backup_states(v_in, states)
        assert np.abs(b[states] - want).max() <= V_RTOL * np.abs(want).max()
        assert not policy_mismatches(P, v_in, pol_na.cpu().numpy()[states], states)
        assert not policy_mismatches(P, v_in, pol_ref.cpu().numpy()[states], states)
        # a further call allocates nothing on the device
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        vi.vi_backup_noalloc(p.m, p.L, p.Q, p.cost, p.pmf, inst.gamma, inst.issuing, V, V_na, pol_na)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_matches_backup_two_calls():
    # first call: FIFO with a pipeline; second call: a different LIFO instance on the same scratch
    reference_and_noalloc(workloads.config1(), 3)
    reference_and_noalloc(
        workloads.single_product(4, 2, 9, (2, 1, 4, 3, 0.5), workloads.poisson_pmf(3.5, 14), 0.95, LIFO), 4)


def test_noalloc_rejects_oversized_tables():
    pmf = workloads.poisson_pmf(4.0, 30)
    n = 256 ** 3                      # |S| of m = 4, L = 1, Q = 255: buffers of the full size
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    W = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(vi.ViError) as e:
        # (Q+1)((m-1)Q+1) pairs far beyond the fixed scratch (|S| = 256^3 fits, the tables do not)
        vi.vi_backup_noalloc(4, 1, 255, (1, 1, 1, 1, 0), pmf, 0.9, FIFO, V, W)
    assert e.value.status == vi.VI_EINVAL


def test_noalloc_refuses_short_buffers():
    # the wrapper checks sizes before the call: the C entry point cannot know |S|
    inst = workloads.config1()
    p = inst.products[0]
    n = inst.n_states
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    short = torch.zeros(n - 1, dtype=torch.float64, device="cuda")
    pol_short = torch.zeros(n - 1, dtype=torch.uint8, device="cuda")
    for args in ((short, V, None), (V, short, None), (V, torch.empty_like(V), pol_short)):
        with pytest.raises(vi.ViError) as e:
            vi.vi_backup_noalloc(p.m, p.L, p.Q, p.cost, p.pmf, inst.gamma, inst.issuing, *args)
        assert e.value.status == vi.VI_EINVAL
    with pytest.raises(vi.ViError):
        vi.vi_backup_noalloc(p.m, p.L, p.Q, p.cost[:4], p.pmf, inst.gamma, inst.issuing, V, torch.empty_like(V))


def test_noalloc_refused_while_capturing():
    # the tables go up from a host staging buffer that the next call overwrites, so a
    # captured call would replay another call's tables: a capturing stream is refused
    inst = workloads.config1()
    p = inst.products[0]
    n = inst.n_states
    V = torch.zeros(2 * n, dtype=torch.float32, device="cuda")
    W = torch.zeros_like(V)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    vi.lib()                     # the library is loaded before the capture starts
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        g.capture_begin()
        try:
            W.add_(1.0)          # the capture holds one node of its own
            with pytest.raises(vi.ViError) as e:
                vi.vi_backup_noalloc(p.m, p.L, p.Q, p.cost, p.pmf, inst.gamma, inst.issuing, V, W,
                                     stream=side)
            assert e.value.status == vi.VI_EINVAL
        finally:
            g.capture_end()
    g.replay()
    torch.cuda.synchronize()
    assert float(W[0]) == 1.0                    # the capture itself was left intact
    # outside the capture the same call runs
    vi.vi_backup_noalloc(p.m, p.L, p.Q, p.cost, p.pmf, inst.gamma, inst.issuing, V, W, stream=side)
    torch.cuda.synchronize()
