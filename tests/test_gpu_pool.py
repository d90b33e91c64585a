"""The library's cache of blocks released by destroyed handles: a handle built on
reused blocks (stale contents from another problem) solves exactly as one built
on fresh blocks, through the device API and the host-buffer API, and the cache
can be emptied."""
import numpy as np
import pytest
import torch

import workloads
from workloads import FIFO, LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import create  # noqa: E402


def _solve_host(inst):
    h = create(inst, "fp32")
    n = vi.vi_problem_sizes(h)["n_states"]
    V = np.empty(2 * n, np.float32)
    pol = np.empty(n, np.uint8)
    info = vi.vi_solve_host(h, 1e-4, 10_000, V, pol)
    vi.vi_problem_destroy(h)
    return V, pol, info["iters"]


def test_reused_blocks_give_identical_solves():
    a = workloads.Instance(name="pool_a", products=[workloads.Product(4, 2, 9, (3.0, 1.0, 5.0, 7.0, 0.0),
                                                                      workloads.poisson_pmf(4.0, 14))],
                           gamma=0.95, issuing=FIFO)
    b = workloads.Instance(name="pool_b", products=[workloads.Product(5, 1, 7, (2.0, 1.0, 6.0, 4.0, 0.0),
                                                                      workloads.poisson_pmf(3.0, 11))],
                           gamma=0.9, issuing=LIFO)
    vi.vi_release_cached_memory()
    assert vi.vi_cached_memory() == 0
    V1, p1, i1 = _solve_host(a)            # fresh blocks
    assert vi.vi_cached_memory() > 0       # kept after destroy
    _solve_host(b)                         # another problem writes into the reused blocks
    V2, p2, i2 = _solve_host(a)            # and a third solve reuses them again
    assert i1 == i2
    np.testing.assert_array_equal(V1, V2)
    np.testing.assert_array_equal(p1, p2)
    freed = vi.vi_release_cached_memory()
    assert freed > 0 and vi.vi_cached_memory() == 0


def _host_solve(inst, precision, pinned, max_iters, tol=1e-4):
    h = create(inst, precision)
    sz = vi.vi_problem_sizes(h)
    n = sz["n_states"]
    words = n * sz["value_bytes"] // 4
    if pinned:
        V = torch.empty(words, dtype=torch.float32).pin_memory().numpy()
        pol = torch.empty(n, dtype=torch.uint8).pin_memory().numpy()
    else:
        V = np.empty(words, np.float32)
        pol = np.empty(n, np.uint8)
    V[:] = np.nan
    pol[:] = 255
    info = vi.vi_solve_host(h, tol, max_iters, V, pol)
    vi.vi_problem_destroy(h)
    return V.copy(), pol.copy(), info["iters"]


HOST_CASES = [
    ("fifo_pipe", workloads.Instance(name="h1", products=[workloads.Product(4, 2, 9, (3.0, 1.0, 5.0, 7.0, 0.0),
                                                                          workloads.poisson_pmf(4.0, 14))],
                                     gamma=0.95, issuing=FIFO), "fp32"),
    ("lifo", workloads.Instance(name="h2", products=[workloads.Product(5, 1, 7, (2.0, 1.0, 6.0, 4.0, 0.0),
                                                                     workloads.poisson_pmf(3.0, 11))],
                                gamma=0.9, issuing=LIFO), "fp32"),
    ("fp64_generic", workloads.Instance(name="h3", products=[workloads.Product(3, 1, 6, (3.0, 1.0, 5.0, 7.0, 0.0),
                                                                             workloads.poisson_pmf(3.0, 10))],
                                        gamma=0.9, issuing=FIFO), "fp64"),
    ("two_products", workloads.config3(), "fp32_kahan"),
]


@pytest.mark.parametrize("case", HOST_CASES, ids=[c[0] for c in HOST_CASES])
@pytest.mark.parametrize("max_iters", [0, 5, 6, 10_000], ids=["extract_only", "odd", "even", "converge"])
def test_pinned_host_buffers_receive_the_same_result(case, max_iters):
    """Pinned host buffers are filled by the extraction sweep itself; pageable ones
    by copies after it: both must hold the same V and policy, whichever of the two
    device buffers the last sweep wrote."""
    _, inst, prec = case
    a = _host_solve(inst, prec, True, max_iters)
    b = _host_solve(inst, prec, False, max_iters)
    assert a[2] == b[2]
    np.testing.assert_array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    np.testing.assert_array_equal(a[1], b[1])
    vals = a[0].view(np.float64) if prec == "fp64" else a[0]   # NaN sentinels left if unwritten
    assert np.isfinite(vals).all() and (a[1] != 255).all()


def test_pinned_values_without_a_policy_and_mixed_buffers():
    """Pinned V with no policy buffer (the sweep writes V only), and pinned V with a
    pageable policy (copied after the sweep): the same V and policy as pageable."""
    inst = HOST_CASES[0][1]
    Vr, pr, ir = _host_solve(inst, "fp32", False, 10_000)
    h = create(inst, "fp32")
    n = vi.vi_problem_sizes(h)["n_states"]
    V = torch.empty(2 * n, dtype=torch.float32).pin_memory().numpy()
    V[:] = np.nan
    info = vi.vi_solve_host(h, 1e-4, 10_000, V, None)
    assert info["iters"] == ir
    np.testing.assert_array_equal(V.view(np.uint32), Vr.view(np.uint32))
    V[:] = np.nan
    pol = np.full(n, 255, np.uint8)
    vi.vi_solve_host(h, 1e-4, 10_000, V, pol)
    vi.vi_problem_destroy(h)
    np.testing.assert_array_equal(V.view(np.uint32), Vr.view(np.uint32))
    np.testing.assert_array_equal(pol, pr)


def test_pinned_host_buffers_periodic_problem():
    """Scenario C (FP64, periodic test): pinned and pageable host buffers agree."""
    inst = workloads.scenario_c(3, 1)

    def run(pinned):
        d, keep = vi.make_periodic_desc(inst.m, inst.Q, inst.pmf, inst.c0, inst.c1, inst.cost, inst.gamma,
                                        vi.VI_STOP_PERIODIC)
        h = vi.vi_problem_create_periodic(d)
        n = vi.vi_problem_sizes(h)["n_states"]
        if pinned:
            V = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
            pol = torch.empty(n, dtype=torch.uint8).pin_memory().numpy()
        else:
            V = np.empty(n, np.float64)
            pol = np.empty(n, np.uint8)
        V[:] = np.nan
        info = vi.vi_solve_host(h, 1e-4, 2000, V, pol)
        vi.vi_problem_destroy(h)
        return V.copy(), pol.copy(), info["iters"]

    a, b = run(True), run(False)
    assert a[2] == b[2]
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert np.isfinite(a[0]).all()


def test_pinned_host_buffers_warm_start():
    """A warm start through vi_solve_host: the host values are copied in before the
    solve and, on the pinned path, overwritten by the extraction sweep; pinned and
    pageable buffers give the same result."""
    inst = HOST_CASES[0][1]
    V0, _, _ = _host_solve(inst, "fp32", False, 4)          # four sweeps from zero

    def run(pinned):
        h = create(inst, "fp32")
        n = vi.vi_problem_sizes(h)["n_states"]
        if pinned:
            V = torch.empty(2 * n, dtype=torch.float32).pin_memory().numpy()
            pol = torch.empty(n, dtype=torch.uint8).pin_memory().numpy()
        else:
            V = np.empty(2 * n, np.float32)
            pol = np.empty(n, np.uint8)
        V[:] = V0
        info = vi.vi_solve_host(h, 1e-4, 10_000, V, pol, flags=vi.VI_FLAG_WARM_START)
        vi.vi_problem_destroy(h)
        return V.copy(), pol.copy(), info["iters"]

    a, b = run(True), run(False)
    assert a[2] == b[2] and a[2] > 0
    np.testing.assert_array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    np.testing.assert_array_equal(a[1], b[1])
    # and the warm start continues the cold solve: the same fixed point
    cold = _host_solve(inst, "fp32", False, 10_000)
    hi = lambda v: v.reshape(-1, 2).astype(np.float64).sum(1)
    assert np.abs(hi(a[0]) - hi(cold[0])).max() <= 1e-3
