"""Scenario C (weekday-periodic demand, uncertain useful life on arrival) on the
CUDA path, in FP64.

* value iteration with the periodic stopping test against the FP64 oracle: the
  stopping iteration, values, policies, on instances spanning several blocks with
  a ragged tail (m = 2..4, exogenous and endogenous life on arrival), and on the
  paper's m = 3 settings;
* one backup at sampled states of the paper's instance against the oracle;
* rollouts bit-exact against the oracle (returns, KPIs, trajectories);
* the paper's results: the value-iteration policy's return (Table 6) and KPIs
  (Table 16), and the printed (s, S) policy's return (Tables 6, 15).
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")

HERE = os.path.dirname(os.path.abspath(__file__))
ROWS = [r for r in json.load(open(os.path.join(HERE, "golden", "scenario_c_tables.json")))["rows"] if r["m"] == 3]


class PHandle:
    def __init__(self, inst, stop_rule=vi.VI_STOP_PERIODIC):
        self.inst = inst
        self.desc, self._keep = vi.make_periodic_desc(inst.m, inst.Q, inst.pmf, inst.c0, inst.c1, inst.cost,
                                                      inst.gamma, stop_rule)
        self.h = vi.vi_problem_create_periodic(self.desc)
        self.sizes = vi.vi_problem_sizes(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        vi.vi_problem_destroy(self.h)

    def solve(self, tol, max_iters, flags=0):
        n = self.sizes["n_states"]
        V = torch.zeros(n, dtype=torch.float64, device="cuda")
        pol = torch.empty(n, dtype=torch.uint8, device="cuda")
        info = vi.vi_solve(self.h, tol, max_iters, V, pol, flags=flags)
        torch.cuda.synchronize()
        return V.cpu().numpy(), pol.cpu().numpy(), info


def sS_policy(inst, s_lo, S_up):
    G = inst.Q + 1
    per = inst.n_states // 7
    pol = np.zeros(inst.n_states, np.uint8)
    for st in range(inst.n_states):
        tau, x = divmod(st, per)
        stock = 0
        for _ in range(inst.m - 1):
            stock += x % G
            x //= G
        if stock <= s_lo[tau] and s_lo[tau] < S_up[tau]:
            pol[st] = max(S_up[tau] - stock, 0)
    return pol


def _policy_mismatches(P, V, pol, states):
    bad = []
    for s in states:
        q = P.qvalues(V, int(s))
        a = int(np.argmax(q))
        if a != int(pol[s]) and q[a] - q[int(pol[s])] > 1e-9 * abs(q[a]):
            bad.append((int(s), a, int(pol[s])))
    return bad


CASES = [
    # m, Q, dmax, c0, c1, gamma
    (2, 9, 10, (0.4,), (0.0,), 0.9),
    (3, 6, 8, (1.0, 0.5), (0.2, 0.3), 0.95),
    (3, 7, 9, (1.0, 0.5), (0.0, 0.0), 0.95),
    (4, 4, 7, (0.5, 1.0, 0.3), (-0.1, 0.1, 0.2), 0.9),
]


@pytest.mark.parametrize("case", CASES, ids=[f"m{c[0]}Q{c[1]}" for c in CASES])
@pytest.mark.parametrize("graph", [True, False], ids=["graph", "hostloop"])
def test_periodic_parity_with_oracle(case, graph):
    m, Q, dmax, c0, c1, gamma = case
    inst = w.periodic_instance(m, Q, dmax, c0, c1, (10.0, 1.0, 20.0, 5.0), gamma)
    P = oracle.PeriodicProblem(inst)
    ref = P.vi_solve(1e-4, 5000, stop_rule=2)
    with PHandle(inst) as H:
        assert H.sizes["n_states"] == inst.n_states
        V, pol, info = H.solve(1e-4, 5000, flags=0 if graph else vi.VI_FLAG_NO_GRAPH)
    assert info["status"] == vi.VI_OK
    assert abs(info["iters"] - ref["iters"]) <= 1
    if info["iters"] == ref["iters"]:
        assert np.abs(V - ref["V"]).max() <= 1e-10 * np.abs(ref["V"]).max()
        assert abs(info["dmax"] - ref["dmax"]) <= 1e-8 * abs(ref["dmax"])
    assert not _policy_mismatches(P, V, pol, range(inst.n_states))
    # fixed sweep count, both sides
    with PHandle(inst) as H:
        V2, _, info2 = H.solve(0.0, 11)
    ref2 = P.vi_solve(0.0, 11, stop_rule=2)
    assert info2["iters"] == 11
    assert np.abs(V2 - ref2["V"]).max() <= 1e-10 * np.abs(ref2["V"]).max()


@pytest.mark.parametrize("row", ROWS, ids=["m3e1", "m3e2"])
def test_paper_instance_parity(row):
    inst = w.scenario_c(3, row["exp"])
    P = oracle.PeriodicProblem(inst)
    ref = P.vi_solve(w.SCENARIO_C["eps"], 2000, stop_rule=2)
    with PHandle(inst) as H:
        assert H.sizes["n_states"] == row["n_states"] and H.sizes["n_actions"] == row["n_actions"]
        assert H.sizes["n_outcomes"] == row["n_outcomes"]
        V, pol, info = H.solve(w.SCENARIO_C["eps"], 2000)
        # one more sweep at sampled states against the oracle
        Vd = torch.tensor(V, device="cuda")
        Vo = torch.empty_like(Vd)
        po = torch.empty(len(V), dtype=torch.uint8, device="cuda")
        vi.vi_backup(H.h, Vd, Vo, po)
        vo, pn = Vo.cpu().numpy(), po.cpu().numpy()
    assert abs(info["iters"] - ref["iters"]) <= 1
    if info["iters"] == ref["iters"]:
        assert np.abs(V - ref["V"]).max() <= 1e-10 * np.abs(ref["V"]).max()
    rng = np.random.default_rng(4)
    states = np.unique(np.concatenate([[0, len(V) - 1], rng.choice(len(V), 60, replace=False)]))
    v_o, p_o = P.backup_states(V, states)
    assert np.abs(vo[states] - v_o).max() <= 1e-11 * np.abs(v_o).max()
    assert not _policy_mismatches(P, V, pn, states)


def test_rollouts_bit_exact():
    inst = w.scenario_c(3, 2)
    row = ROWS[1]
    pol = sS_policy(inst, row["s_best"], row["S_best"])
    n, H_, W = 256, 40, 9
    P = oracle.PeriodicProblem(inst)
    ref = P.simulate(pol, n, H_, seed=5, warmup=W, with_traj=True)
    with PHandle(inst) as H:
        pd = torch.tensor(pol, device="cuda")
        ret = torch.empty(n, dtype=torch.float64, device="cuda")
        kp = torch.empty(3 * n, dtype=torch.float64, device="cuda")
        tr = torch.empty(n * H_, dtype=torch.int32, device="cuda")
        vi.vi_simulate(H.h, pd, n, H_, W, 5, ret, kp, tr)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(tr.cpu().numpy().reshape(n, H_), ref["traj"])
    np.testing.assert_array_equal(ret.cpu().numpy(), ref["returns"])
    np.testing.assert_array_equal(kp.cpu().numpy().reshape(n, 3), ref["kpis"])


def test_periodic_rejections():
    inst = w.scenario_c(3, 1)
    with PHandle(inst) as H:
        V = torch.zeros(inst.n_states, dtype=torch.float64, device="cuda")
        pol = torch.zeros(inst.n_states, dtype=torch.uint8, device="cuda")
        ret = torch.empty(4, dtype=torch.float64, device="cuda")
        with pytest.raises(RuntimeError):
            vi.vi_simulate_ex(H.h, pol, 4, 3, 0, 1, ret, None,
                              torch.empty(24, dtype=torch.float64, device="cuda"))
        with pytest.raises(RuntimeError):
            vi.vi_solve(H.h, 1e-4, 10, V, pol, flags=vi.VI_FLAG_POLICY_EVAL)
        with pytest.raises(RuntimeError):
            vi.vi_problem_set_option(H.h, vi.VI_OPT_KERNEL, vi.VI_KERNEL_GROUP)
    bad = dict(m=3, Q=20, pmf=inst.pmf, c0=inst.c0, c1=inst.c1, cost=inst.cost, gamma=1.0)
    d, keep = vi.make_periodic_desc(**bad)
    with pytest.raises(RuntimeError):
        vi.vi_problem_create_periodic(d)


def _close(x, printed, n, floor):
    mean, sd = printed
    se = math.hypot(float(x.std(ddof=1)), sd) / math.sqrt(n)
    return abs(float(x.mean()) - mean) <= 4.0 * se + floor


@pytest.mark.parametrize("row", ROWS, ids=["m3e1", "m3e2"])
def test_scenario_c_matches_the_paper(row):
    """Value iteration to the periodic test, then 10,000 rollouts of 365 days
    after 100: Table 6's return and Table 16's KPIs for the value-iteration
    policy; the printed (s, S) policy (Table 15) scores Table 6's
    simulation-optimisation return on the same GPU rollouts."""
    inst = w.scenario_c(3, row["exp"])
    RO = w.SCENARIO_C_ROLLOUTS
    n = RO["n_rollouts"]
    with PHandle(inst) as H:
        V, pol, info = H.solve(w.SCENARIO_C["eps"], 2000)
        assert info["status"] == vi.VI_OK
        ret = torch.empty(n, dtype=torch.float64, device="cuda")
        kp = torch.empty(3 * n, dtype=torch.float64, device="cuda")
        vi.vi_simulate(H.h, torch.tensor(pol, device="cuda"), n, RO["horizon"], RO["warmup"], 2023, ret, kp)
        r, k = ret.cpu().numpy(), kp.cpu().numpy().reshape(n, 3)
        so = torch.empty(n, dtype=torch.float64, device="cuda")
        sp = torch.tensor(sS_policy(inst, row["s_best"], row["S_best"]), device="cuda")
        vi.vi_simulate(H.h, sp, n, RO["horizon"], RO["warmup"], 2023, so)
        rs = so.cpu().numpy()
    assert _close(r, (row["vi_return_mean"], row["vi_return_sd"]), n, 0.5), r.mean()
    assert abs(r.std(ddof=1) - row["vi_return_sd"]) <= 3.0
    for j, key in enumerate(("service_vi", "wastage_vi", "holding_vi")):
        assert _close(k[:, j], row[key], n, 0.05), (key, k[:, j].mean())
    assert _close(rs, (row["so_return_mean"], row["so_return_sd"]), n, 0.5), rs.mean()


def test_large_instance_sampled_backup():
    """The paper's m = 5 setting (1,361,367 states: the thread-per-state sweep;
    the m <= 4 cases above take the warp-per-state one): a backup from a value
    function three sweeps in, at sampled states, against the oracle."""
    inst = w.scenario_c(5, 2)
    P = oracle.PeriodicProblem(inst)
    with PHandle(inst) as H:
        V, _, info = H.solve(0.0, 3)
        Vd = torch.tensor(V, device="cuda")
        Vo = torch.empty_like(Vd)
        po = torch.empty(len(V), dtype=torch.uint8, device="cuda")
        vi.vi_backup(H.h, Vd, Vo, po)
        vo, pn = Vo.cpu().numpy(), po.cpu().numpy()
    rng = np.random.default_rng(12)
    states = np.unique(np.concatenate([[0, len(V) - 1], rng.choice(len(V), 14, replace=False)]))
    v_o, p_o = P.backup_states(V, states)
    assert np.abs(vo[states] - v_o).max() <= 1e-11 * np.abs(v_o).max()
    assert not _policy_mismatches(P, V, pn, states)
