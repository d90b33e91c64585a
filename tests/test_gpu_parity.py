"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Values: max|V_gpu - V_oracle| / max|V_oracle| <= 1e-5 at the same iteration.
Policies: equal except ties whose FP64 Q-gap is <= 1e-6 relative.
Next-state indices: bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from workloads import FIFO, LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import (Handle, compare_values, policy_mismatches, values_abs, V_RTOL,  # noqa: E402
                         solve_parity, sampled_backup_parity)


def small_instances():
    out = []
    rng = np.random.default_rng(123)
    for i in range(24):
        out.append(workloads.random_small_instance(rng, max_states=600))
    # hand-picked shapes: m = 1 (single state / pure pipeline), Q = 0, dmax = 0, long pipelines
    out.append(workloads.single_product(1, 1, 6, (3, 1, 5, 7, 0), workloads.poisson_pmf(3, 10), 0.9, FIFO))
    out.append(workloads.single_product(1, 3, 4, (3, 1, 5, 7, 1), workloads.poisson_pmf(2, 8), 0.9, LIFO))
    out.append(workloads.single_product(3, 1, 0, (3, 1, 5, 7, 0), workloads.poisson_pmf(2, 5), 0.9, FIFO))
    out.append(workloads.single_product(3, 2, 4, (3, 1, 5, 7, 0), workloads.poisson_pmf(2, 0), 0.9, LIFO))
    out.append(workloads.single_product(2, 5, 3, (1, 1, 2, 1, 0), workloads.poisson_pmf(1.5, 9), 0.95, FIFO))
    out.append(workloads.single_product(6, 1, 2, (2, 1, 4, 3, 0), workloads.poisson_pmf(2.5, 12), 0.95, LIFO))
    out.append(workloads.single_product(4, 2, 5, (2, 1, 4, 3, 0), workloads.poisson_pmf(4.5, 30), 0.9, FIFO))
    return out


SMALL = small_instances()


def _ids(insts):
    return [f"{i}-m{x.products[0].m}L{x.products[0].L}Q{x.products[0].Q}{'L' if x.issuing else 'F'}"
            for i, x in enumerate(insts)]


# ---------------------------------------------------------------------------
# next-state indices, bit-exact
# ---------------------------------------------------------------------------

def check_next_states(inst, states):
    P = oracle.Problem(inst)
    with Handle(inst, precision="fp32") as H:
        st = torch.tensor(np.asarray(states, np.uint32).view(np.int32), device="cuda")
        A = H.sizes["n_actions"]
        if len(inst.products) == 1:
            D = inst.products[0].dmax + 1
            out = torch.empty(len(states) * A * D, dtype=torch.int32, device="cuda")
            vi.vi_next_states(H.h, st, len(states), out)
            got = out.cpu().numpy().view(np.uint32).reshape(len(states), A, D)
            for i, s in enumerate(states):
                for a in range(A):
                    for d in range(D):
                        assert got[i, a, d] == P.transition(int(s), a, d)["s_next"], (s, a, d)
        else:
            D1 = inst.products[0].dmax + 1
            ZL = inst.products[0].dmax + inst.products[1].dmax + 1
            out = torch.empty(len(states) * A * D1 * ZL, dtype=torch.int32, device="cuda")
            vi.vi_next_states(H.h, st, len(states), out)
            got = out.cpu().numpy().view(np.uint32).reshape(len(states), A, D1, ZL)
            D2 = inst.products[1].dmax
            for i, s in enumerate(states):
                for a in range(A):
                    for d1 in range(D1):
                        unmet = P.transition(int(s), a, d1, 0, 0)["unmet1"]
                        for d2 in range(D2 + 1):
                            for u in range(unmet + 1):
                                want = P.transition(int(s), a, d1, d2, u)["s_next"]
                                assert got[i, a, d1, d2 + u] == want, (s, a, d1, d2, u)


@pytest.mark.parametrize("inst", SMALL[:12], ids=_ids(SMALL[:12]))
def test_next_states_small_exhaustive(inst):
    check_next_states(inst, np.arange(inst.n_states))


@pytest.mark.parametrize("cfg", [1, 2, 4])
def test_next_states_configs_sampled(cfg):
    inst = workloads.CONFIGS[cfg]()
    rng = np.random.default_rng(cfg)
    states = np.unique(np.concatenate([[0, inst.n_states - 1], rng.integers(0, inst.n_states, 40)]))
    check_next_states(inst, states)


def test_next_states_two_products():
    inst = workloads.config3(Q=3)
    rng = np.random.default_rng(3)
    check_next_states(inst, np.unique(np.concatenate([[0, inst.n_states - 1],
                                                      rng.integers(0, inst.n_states, 12)])))


# ---------------------------------------------------------------------------
# full solves vs the oracle at the oracle's stopping iteration
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("inst", SMALL, ids=_ids(SMALL))
@pytest.mark.parametrize("precision", ["fp32", "fp32_kahan", "fp64", "fp32_single"])
def test_solve_small(inst, precision):
    solve_parity(inst, precision)


@pytest.mark.parametrize("inst", SMALL, ids=_ids(SMALL))
def test_solve_small_generic_kernel_fp32(inst):
    solve_parity(inst, "fp32", kernel=vi.VI_KERNEL_GENERIC)


def test_solve_config1_fp64_and_fp32():
    inst = workloads.config1()
    for prec in ("fp64", "fp32", "fp32_kahan", "fp32_single"):
        solve_parity(inst, prec)


def test_solve_supnorm_rule():
    inst = workloads.single_product(2, 2, 4, (3, 1, 5, 7, 0), workloads.poisson_pmf(2, 9), 0.8, LIFO)
    solve_parity(inst, "fp64", tol=1e-6, stop_rule=1)
    solve_parity(inst, "fp32", tol=1e-3, stop_rule=1)


@pytest.mark.parametrize("Q", [2, 4])
def test_solve_two_products(Q):
    inst = workloads.config3(Q=Q)
    for prec in ("fp32_kahan", "fp32", "fp64"):
        solve_parity(inst, prec)


@pytest.mark.parametrize("case", [dict(m=2, Q=2, m2=3, Q2=1, issuing=LIFO, rho=0.3),
                                  dict(m=3, Q=1, m2=2, Q2=3, issuing=FIFO, rho=0.8),
                                  dict(m=1, Q=3, m2=2, Q2=2, issuing=FIFO, rho=0.5)])
def test_solve_two_products_general_costs(case):
    c1 = (0.7, 0.3, 1.5, 0.9, 1.2)
    c2 = (0.4, 0.2, 0.8, 1.1, 1.6)
    prods = [workloads.Product(case["m"], 1, case["Q"], c1, workloads.poisson_pmf(1.3, 6)),
             workloads.Product(case["m2"], 1, case["Q2"], c2, workloads.poisson_pmf(1.8, 7))]
    inst = workloads.Instance("g2", prods, gamma=0.9, issuing=case["issuing"], subst_rate=case["rho"])
    for prec in ("fp64", "fp32_kahan"):
        solve_parity(inst, prec)


# ---------------------------------------------------------------------------
# full-size instances: one backup in the benchmark's launch configuration,
# compared on sampled states computed one by one by the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp32", "fp32_single"])
def test_config2_full_size_sampled(precision):
    sampled_backup_parity(workloads.config2(), 3, 300, 2, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp32_single"])
def test_config4_full_size_sampled(precision):
    sampled_backup_parity(workloads.config4(), 3, 300, 4, precision)


def test_config3_full_size_sampled():
    inst = workloads.config3()
    P = oracle.Problem(inst)
    with Handle(inst) as H:
        V, pol, info = H.solve(0.0, 2)
        n = H.sizes["n_states"]
        v_k = H.v_abs(V, info)
        V_next = torch.empty_like(V)
        vi.vi_backup(H.h, V, V_next, None)
        v_next = values_abs(V_next, inst.gamma * info["offset"], H.layout)
        states = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(5).integers(0, n, 24)]))
        want, _ = P.backup_states(v_k, states)
        err = np.abs(v_next[states] - want).max() / np.abs(want).max()
        assert err <= V_RTOL, err


# ---------------------------------------------------------------------------
# FP64 policy evaluation and rollouts
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("inst", [SMALL[3], SMALL[7], workloads.config3(Q=2)], ids=["a", "b", "two"])
def test_policy_eval_fp64(inst):
    P = oracle.Problem(inst)
    ref = P.vi_solve(tol=1e-4, max_iters=5000)
    pol = ref["policy"]
    Vpe_ref, _, _ = P.policy_eval(pol, tol=1e-12, max_iters=20000)
    with Handle(inst) as H:
        V = torch.zeros(inst.n_states, dtype=torch.float64, device="cuda")
        pol_t = torch.tensor(pol, device="cuda")
        r = vi.vi_policy_eval(H.h, pol_t, V, 1e-12, 20000)
        torch.cuda.synchronize()
        assert r["converged"]
        err = compare_values(V.cpu().numpy(), Vpe_ref)
        assert err < 1e-10, err


def rollout_parity(inst, policy, n, horizon, seed, warmup=0):
    P = oracle.Problem(inst)
    ref = P.simulate(policy, n, horizon, seed, warmup=warmup, with_traj=True)
    with Handle(inst) as H:
        pol_t = torch.tensor(policy, device="cuda")
        ret = torch.empty(n, dtype=torch.float64, device="cuda")
        kp = torch.empty(n * 3, dtype=torch.float64, device="cuda")
        tr = torch.empty(n * horizon, dtype=torch.int32, device="cuda")
        vi.vi_simulate(H.h, pol_t, n, horizon, warmup, seed, ret, kp, tr)
        torch.cuda.synchronize()
        assert (tr.cpu().numpy().reshape(n, horizon) == ref["traj"]).all()
        np.testing.assert_array_equal(ret.cpu().numpy(), ref["returns"])
        np.testing.assert_array_equal(kp.cpu().numpy().reshape(n, 3), ref["kpis"])


@pytest.mark.parametrize("inst", SMALL[:10] + [workloads.config1()], ids=_ids(SMALL[:10]) + ["cfg1"])
def test_rollouts_bit_exact(inst):
    pol = oracle.Problem(inst).vi_solve(tol=1e-4, max_iters=3000)["policy"]
    rollout_parity(inst, pol, 64, 50, seed=0xDEADBEEF12345, warmup=3)


@pytest.mark.parametrize("n, horizon, warmup", [(37, 29, 5), (1, 7, 0), (17, 9, 8), (5, 1, 0)])
def test_rollouts_ragged_counts_bit_exact(n, horizon, warmup):
    # rollout counts that leave part of the last warp's lane groups empty, and
    # horizons that end inside a group's block of periods
    inst = SMALL[7]
    pol = oracle.Problem(inst).vi_solve(tol=1e-4, max_iters=3000)["policy"]
    rollout_parity(inst, pol, n, horizon, seed=1234567, warmup=warmup)


def test_rollouts_ragged_two_products_bit_exact():
    inst = workloads.config3(Q=2)
    pol = oracle.Problem(inst).vi_solve(tol=1e-4, max_iters=3000)["policy"]
    rollout_parity(inst, pol, 13, 11, seed=99, warmup=2)


def test_rollouts_two_products_bit_exact():
    inst = workloads.config3(Q=3)
    pol = oracle.Problem(inst).vi_solve(tol=1e-4, max_iters=3000)["policy"]
    rollout_parity(inst, pol, 32, 40, seed=7)


def test_rollouts_config4_policy_bit_exact():
    inst = workloads.config4()
    with Handle(inst) as H:
        V, pol, info = H.solve(1e-4, 1000)
        policy = pol.cpu().numpy()
    rollout_parity(inst, policy, 256, 365, seed=workloads.CONFIG4_ROLLOUTS["seed"])


# ---------------------------------------------------------------------------
# edge cases and argument checks
# ---------------------------------------------------------------------------

def test_max_iters_zero_and_not_converged():
    inst = SMALL[5]
    with Handle(inst) as H:
        V, pol, info = H.solve(1e-4, 0)
        assert info["iters"] == 0 and info["status"] == vi.VI_ENOTCONVERGED
        assert (V == 0).all()
        V, pol, info = H.solve(0.0, 2)
        assert info["iters"] == 2 and info["status"] == vi.VI_ENOTCONVERGED


def test_warm_start_resume_is_bit_identical():
    inst = workloads.single_product(4, 2, 6, (2, 1, 4, 3, 0), workloads.poisson_pmf(3, 14), 0.95, FIFO)
    with Handle(inst) as H:
        V_a, _, ia = H.solve(0.0, 7)
        V_b, _, ib = H.solve(0.0, 4)
        V_c, _, ic = H.solve(0.0, 3, flags=vi.VI_FLAG_WARM_START, V=V_b, offset=ib["offset"])
        # compare absolute values (the single layout renormalises after a resume)
        va = H.v_abs(V_a, ia)
        vc = H.v_abs(V_c, ic)
        assert np.abs(va - vc).max() <= 1e-6 * np.abs(va).max()


def test_no_graph_loop_matches_graph():
    inst = SMALL[8]
    with Handle(inst) as H:
        V1, p1, i1 = H.solve(1e-4, 1000)
        V2, p2, i2 = H.solve(1e-4, 1000, flags=vi.VI_FLAG_NO_GRAPH)
        assert i1["iters"] == i2["iters"]
        assert torch.equal(V1, V2) and torch.equal(p1, p2)


def test_invalid_arguments():
    pmf = workloads.poisson_pmf(2, 5)
    with pytest.raises(vi.ViError):
        vi.vi_problem_create(0, 1, 3, (1, 1, 1, 1, 0), pmf, 0.9, 0)
    with pytest.raises(vi.ViError):
        vi.vi_problem_create(2, 1, 3, (1, -1, 1, 1, 0), pmf, 0.9, 0)
    with pytest.raises(vi.ViError):
        vi.vi_problem_create(2, 1, 3, (1, 1, 1, 1, 0), pmf * 0.5, 0.9, 0)
    with pytest.raises(vi.ViError):
        vi.vi_problem_create(2, 1, 3, (1, 1, 1, 1, 0), pmf, 1.5, 0)
    with pytest.raises(vi.ViError):
        vi.vi_problem_create(2, 1, 300, (1, 1, 1, 1, 0), pmf, 0.9, 0)
    with pytest.raises(vi.ViError):
        vi.vi_problem_create(12, 1, 20, (1, 1, 1, 1, 0), pmf, 0.9, 0)   # 21^11 states
    h = vi.vi_problem_create(2, 1, 3, (1, 1, 1, 1, 0), pmf, 0.9, 0)
    try:
        with pytest.raises(vi.ViError):
            vi.vi_solve(h, -1.0, 10, torch.zeros(8, device="cuda"))
        with pytest.raises(vi.ViError):
            vi.vi_solve(h, 1e-4, 10, None)
        # 4 states need 4 float pairs: a buffer of 4 floats is refused before any kernel runs
        with pytest.raises(ValueError):
            vi.vi_solve(h, 1e-4, 10, torch.zeros(4, device="cuda"))
        with pytest.raises(ValueError):
            vi.vi_solve(h, 1e-4, 10, torch.zeros(8, device="cuda"), torch.zeros(3, dtype=torch.uint8, device="cuda"))
        with pytest.raises(ValueError):
            vi.vi_backup(h, torch.zeros(8, device="cuda"), torch.zeros(6, device="cuda"))
        with pytest.raises(ValueError):
            vi.vi_solve_host(h, 1e-4, 10, np.zeros(7, np.float32), None)
        with pytest.raises(vi.ViError):
            vi.vi_problem_set_option(h, vi.VI_OPT_KERNEL, 99)
    finally:
        vi.vi_problem_destroy(h)


# ---------------------------------------------------------------------------
# lane widths of the factorised kernel: the demand sums keep their order, so
# every width gives bit-identical values and policies
# ---------------------------------------------------------------------------

WIDTH_CASES = [
    workloads.single_product(3, 2, 9, (2, 1, 4, 3, 0), workloads.poisson_pmf(3.0, 13), 0.95, FIFO),
    workloads.single_product(4, 1, 7, (2, 1, 4, 3, 0), workloads.poisson_pmf(2.5, 11), 0.95, LIFO),
    workloads.single_product(2, 3, 12, (3, 1, 5, 7, 1), workloads.poisson_pmf(5.0, 20), 0.9, FIFO),
    workloads.single_product(3, 1, 20, (3, 1, 5, 7, 0), workloads.poisson_pmf(5.0, 25), 0.99, LIFO),
]


@pytest.mark.parametrize("inst", WIDTH_CASES, ids=_ids(WIDTH_CASES))
@pytest.mark.parametrize("precision", ["fp32", "fp32_single"])
def test_group_widths_bit_identical(inst, precision):
    G = inst.products[0].Q + 1
    widths = [w for w in (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 16, 21, 24) if w <= G]
    ref = None
    for w in widths:
        with Handle(inst, precision=precision) as H:
            vi.vi_problem_set_option(H.h, vi.VI_OPT_GROUP_WIDTH, w)
            V, pol, info = H.solve(0.0, 12)
            got = (V.cpu().numpy().tobytes(), pol.cpu().numpy().tobytes(), info["offset"])
        if ref is None:
            ref = got
        else:
            assert got == ref, f"width {w} differs"
    # and the autotuned choice matches the oracle
    solve_parity(inst, precision)


def test_l2_read_probe():
    """The L2 read probe returns a plausible rate and rejects bad buffers."""
    import torch
    nbytes = 8 << 20
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
    ms = vi.vi_probe_l2_read(buf, nbytes, 16)
    gbs = nbytes * 16 / (ms * 1e-3) / 1e9
    assert 100.0 < gbs < 1e6
    assert torch.all(buf == 1.0)   # only read
    with pytest.raises(vi.ViError):
        vi.vi_probe_l2_read(buf, 15, 1)
    with pytest.raises(vi.ViError):
        vi.vi_probe_l2_read(buf, nbytes, 0)


def test_two_product_factorised_matches_generic():
    """The factorised two-product sweep (expectation tables of product 2 built
    per sweep) and the generic one agree after the same number of sweeps."""
    inst = workloads.config3(Q=4)
    with Handle(inst, precision="fp32") as F, Handle(inst, precision="fp32", kernel=vi.VI_KERNEL_GENERIC) as G:
        assert vi.vi_problem_kernel(F.h)[0] == vi.VI_KERNEL_GROUP
        assert vi.vi_problem_kernel(G.h)[0] == vi.VI_KERNEL_GENERIC
        Vf, pf, inf_ = F.solve(0.0, 8)
        Vg, pg, ing = G.solve(0.0, 8)
        err = compare_values(F.v_abs(Vf, inf_), G.v_abs(Vg, ing))
        assert err <= 1e-6, err
        assert (pf != pg).sum().item() <= 1e-3 * pf.numel()
