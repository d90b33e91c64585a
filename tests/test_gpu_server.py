"""Continuous-batching solve server: every result equals the same instance solved
alone, admission respects the memory budget, and shutdown cancels pending work."""
import time

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle, compare_values, policy_mismatches, V_RTOL  # noqa: E402


def desc_of(inst):
    p = inst.products[0]
    return vi.make_desc([dict(m=p.m, L=p.L, Q=p.Q, cost=p.cost, pmf=p.pmf)], inst.gamma, inst.issuing)


def wait_all(srv, ids, n_states, timeout_s=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        for rid in ids:
            if rid in out:
                continue
            n = n_states[rid]
            V = np.empty(n, np.float64)
            pol = np.empty(n, np.uint8)
            done, info = vi.vi_server_poll(srv, rid, V, pol)
            if done:
                out[rid] = (V, pol, info)
        assert time.time() - t0 < timeout_s, "server did not finish"
        time.sleep(0.002)
    return out


def mix(n, seed, max_states=60_000):
    reqs = workloads.serving_mix(n, seed=seed, max_states=max_states)
    return [r.instance for r in reqs]


def _column_body(inst):
    """Whether the server runs the FIFO column body for this instance."""
    p = inst.products[0]
    return (inst.issuing == workloads.FIFO and ((p.L >= 2 and p.m >= 2) or (p.L == 1 and p.m >= 3))
            and p.Q + 1 <= 32 and p.dmax <= 46)


def test_results_equal_alone_and_in_the_mix():
    insts = mix(24, seed=11)
    srv = vi.vi_server_create(4 << 30, 16)
    try:
        keep, ids, sizes = [], [], {}
        for inst in insts:
            d, k = desc_of(inst)
            keep.append(k)
            rid = vi.vi_server_submit(srv, d, 1e-4, 5000)
            ids.append(rid)
            sizes[rid] = inst.n_states
        res = wait_all(srv, ids, sizes)
    finally:
        vi.vi_server_destroy(srv)
    # the mix holds instances of both bodies, and lead time one on the column body
    assert any(map(_column_body, insts)) and not all(map(_column_body, insts))
    assert any(_column_body(i) and i.products[0].L == 1 for i in insts)
    for inst, rid in zip(insts, ids):
        V, pol, info = res[rid]
        assert info["status"] == vi.VI_OK
        # the server runs the FIFO column body where it applies (pmf of at most 47
        # entries) and the factorised CUDA-core body otherwise (bit-identical across lane
        # widths); the standalone sweep with that body gives the same arithmetic
        col = _column_body(inst)
        kernel = vi.VI_KERNEL_FIFO_COL if col else vi.VI_KERNEL_GROUP
        with Handle(inst, precision="fp32", kernel=kernel) as H:
            Va, pola, ia = H.solve(1e-4, 5000)
            va = H.v_abs(Va, ia)
        assert info["iters"] == ia["iters"]
        # same kernel arithmetic alone and in the batch: identical values and policy
        np.testing.assert_array_equal(V, va)
        np.testing.assert_array_equal(pol, pola.cpu().numpy())


def test_server_result_matches_oracle():
    inst = mix(1, seed=3, max_states=5000)[0]
    ref = oracle.Problem(inst).vi_solve(tol=1e-4, max_iters=5000)
    srv = vi.vi_server_create(1 << 30, 4)
    try:
        d, k = desc_of(inst)
        rid = vi.vi_server_submit(srv, d, 0.0, ref["iters"])   # oracle's sweep count, stop test off
        V, pol, info = wait_all(srv, [rid], {rid: inst.n_states})[rid]
    finally:
        vi.vi_server_destroy(srv)
    assert info["iters"] == ref["iters"] and info["status"] == vi.VI_ENOTCONVERGED
    assert compare_values(V, ref["V"]) <= V_RTOL
    assert not policy_mismatches(oracle.Problem(inst), ref["V"], pol)


def test_admission_respects_budget():
    insts = mix(6, seed=5, max_states=30_000)
    biggest = max(i.n_states for i in insts)
    budget = biggest * 17 + (1 << 16) + (1 << 20)      # room for about one request at a time
    srv = vi.vi_server_create(budget, 8)
    try:
        ids, sizes, keep = [], {}, []
        for inst in insts:
            d, k = desc_of(inst)
            keep.append(k)
            rid = vi.vi_server_submit(srv, d, 1e-4, 5000)
            ids.append(rid)
            sizes[rid] = inst.n_states
        res = wait_all(srv, ids, sizes)
        assert all(r[2]["status"] == vi.VI_OK for r in res.values())
        # a request that can never fit is refused at once
        big = workloads.single_product(6, 1, 20, (1, 1, 1, 1, 0), workloads.poisson_pmf(3, 14), 0.9)
        d, k = desc_of(big)
        with pytest.raises(vi.ViError) as e:
            vi.vi_server_submit(srv, d, 1e-4, 100)
        assert e.value.status == vi.VI_EBUSY
    finally:
        vi.vi_server_destroy(srv)


def test_invalid_requests_and_shutdown_cancels():
    srv = vi.vi_server_create(1 << 30, 2)
    two = workloads.config3(Q=2)
    prods = [dict(m=p.m, L=p.L, Q=p.Q, cost=p.cost, pmf=p.pmf) for p in two.products]
    d2, k2 = vi.make_desc(prods, two.gamma, two.issuing, subst_rate=0.5)
    with pytest.raises(vi.ViError):
        vi.vi_server_submit(srv, d2, 1e-4, 10)
    inst = workloads.config2()
    d, k = desc_of(inst)
    rid = vi.vi_server_submit(srv, d, 0.0, 100000)     # never stops on its own
    t0 = time.time()
    vi.vi_server_destroy(srv)                          # cancels it
    assert time.time() - t0 < 60


def test_wait_reports_each_finished_request_once():
    rng = np.random.default_rng(8)
    insts = [workloads.random_small_instance(rng, max_states=3000) for _ in range(24)]
    insts = [i for i in insts if i.products[0].n_digits >= 1 and 2 <= i.products[0].Q + 1 <= 24]
    srv = vi.vi_server_create(1 << 30, 8)
    try:
        keep = [desc_of(i) for i in insts]
        ids = [vi.vi_server_submit(srv, d, 1e-4, 2000) for d, _ in keep]
        seen = []
        t0 = time.time()
        while len(seen) < len(ids):
            got = vi.vi_server_wait(srv, 20, max_ids=5)
            assert len(got) <= 5
            seen += got
            assert time.time() - t0 < 120.0, "server did not finish"
        assert sorted(seen) == sorted(ids)
        for rid, inst in zip(ids, insts):
            n = inst.n_states
            V, pol = np.empty(n, np.float64), np.empty(n, np.uint8)
            done, info = vi.vi_server_poll(srv, rid, V, pol)
            assert done and info["status"] == vi.VI_OK
        assert vi.vi_server_wait(srv, 0) == []
    finally:
        vi.vi_server_destroy(srv)


def test_submit_to_writes_the_callers_buffers():
    rng = np.random.default_rng(9)
    insts = [workloads.random_small_instance(rng, max_states=2000) for _ in range(16)]
    insts = [i for i in insts if i.products[0].n_digits >= 1 and 2 <= i.products[0].Q + 1 <= 24]
    srv = vi.vi_server_create(1 << 30, 8)
    try:
        keep = [desc_of(i) for i in insts]
        bufs = [(np.full(i.n_states, np.nan), np.full(i.n_states, 255, np.uint8)) for i in insts]
        ids_to = [vi.vi_server_submit_to(srv, d, 1e-4, 2000, *b) for (d, _), b in zip(keep, bufs)]
        ids = [vi.vi_server_submit(srv, d, 1e-4, 2000) for d, _ in keep]
        got = wait_all(srv, ids, {rid: i.n_states for rid, i in zip(ids, insts)})
        for rid, inst, (V, pol) in zip(ids_to, insts, bufs):
            t0 = time.time()
            while not vi.vi_server_poll(srv, rid)[0]:
                assert time.time() - t0 < 120.0
                time.sleep(0.002)
        for rid, (V, pol) in zip(ids, bufs):
            Vp, Pp, info = got[rid]
            np.testing.assert_array_equal(V, Vp)
            np.testing.assert_array_equal(pol, Pp)
    finally:
        vi.vi_server_destroy(srv)
