"""Scenario C (weekday-periodic demand, uncertain useful life on arrival) in the
oracle, pinned to the paper and to brute force.

* the multinomial age-on-arrival law against brute-force enumeration of every
  sequence of unit draws, and its mean a p_k(a);
* one period against a hand-worked case and unit conservation;
* value iteration against exhaustive policy search with exact policy
  evaluation on a tiny periodic instance;
* the periodic stopping test: the policy is stable when it fires;
* state and outcome counts of Table 6;
* the paper's best (s, S) policies (Table 15) simulated on 10,000 rollouts:
  returns of Table 6 and KPIs of Table 16.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as w

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "scenario_c_tables.json")))


def sS_policy(inst, s_lo, S_up):
    """(s, S) by weekday: order [S^tau - I]^+ when I <= s^tau (and s^tau < S^tau),
    I = units in stock at the start of the day (Scenario C heuristic)."""
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


@pytest.mark.parametrize("m,exp", [(3, 1), (3, 2), (5, 2)])
def test_arrival_law_brute_force(m, exp):
    inst = w.scenario_c(m, exp)
    P = oracle.PeriodicProblem(inst)
    for a in (0, 1, 3, 5):
        p = P.arrival_params(a)
        assert abs(p.sum() - 1.0) < 1e-15
        # every sequence of a unit draws, each unit's age class independent
        brute = {}
        for seq in itertools.product(range(m), repeat=a):
            y = tuple(seq.count(k) for k in range(m))
            brute[y] = brute.get(y, 0.0) + float(np.prod([p[k] for k in seq]))
        profs = P.profiles(a)
        assert len(profs) == math.comb(a + m - 1, m - 1) == len(brute)
        for y in profs:
            assert abs(P.arrival_prob(a, y) - brute[tuple(int(v) for v in y)]) < 1e-14
        mean = sum(P.arrival_prob(a, y) * np.asarray(y, float) for y in profs)
        np.testing.assert_allclose(mean, a * p, rtol=0, atol=1e-13)


def test_one_period_by_hand():
    inst = w.scenario_c(3, 1)
    P = oracle.PeriodicProblem(inst)
    G = 21
    # Wednesday (tau 2), X_1 = 4 expiring today, X_2 = 19; order 5 arriving as
    # y = (1, 3, 1): Z_1 = 5, Z_2 = min(22, 20) = 20 (2 refused), Z_3 = 1; demand 8
    s = 2 * G * G + 4 + G * 19
    st = P.transition(s, 5, 8, [1, 3, 1])
    # oldest first: 5 from Z_1, 3 from Z_2 -> X'_1 = 17, X'_2 = 1; nothing wasted
    assert st["s_next"] == 3 * G * G + 17 + G * 1
    assert st["issued"] == 8 and st["wasted"] == 0 and st["held"] == 18
    assert st["accepted"] == 3 and st["refused"] == 2
    assert st["reward"] == -10.0 - 1.0 * 18
    # Sunday, demand 30 > stock: shortage, and the expiring units are all issued
    st = P.transition(6 * G * G + 2 + G * 1, 0, 20, [0, 0, 0])
    assert st["s_next"] == 0 and st["reward"] == -20.0 * 17 and st["held"] == 0


def test_unit_conservation():
    inst = w.scenario_c(3, 2)
    P = oracle.PeriodicProblem(inst)
    rng = np.random.default_rng(1)
    G, per = 21, 441
    for _ in range(300):
        s = int(rng.integers(P.n_states))
        a = int(rng.integers(21))
        d = int(rng.integers(21))
        profs = P.profiles(a)
        y = profs[int(rng.integers(len(profs)))]
        st = P.transition(s, a, d, y)
        x = s % per
        stock = x % G + x // G
        nx = st["s_next"] % per
        assert st["s_next"] // per == (s // per + 1) % 7
        assert st["accepted"] + st["refused"] == a
        assert stock + st["accepted"] == st["issued"] + st["held"]
        assert st["held"] == nx % G + nx // G + st["wasted"]


def test_value_iteration_equals_exhaustive_policy_search():
    inst = w.periodic_instance(2, 1, 3, (0.7,), (0.5,), (2.0, 1.0, 6.0, 3.0), 0.8,
                               pmf=np.tile([0.3, 0.4, 0.2, 0.1], (7, 1)))
    P = oracle.PeriodicProblem(inst)
    n = P.n_states                       # 7 x 2 states, 2 actions
    Pm = np.zeros((2, n, n))
    R = np.zeros((2, n))
    for s in range(n):
        tau = s // (n // 7)
        for a in range(2):
            for y in P.profiles(a):
                py = P.arrival_prob(a, y)
                for d in range(4):
                    st = P.transition(s, a, d, y)
                    pr = py * inst.pmf[tau, d]
                    Pm[a, s, st["s_next"]] += pr
                    R[a, s] += pr * st["reward"]
    best = None
    for bits in range(2 ** n):
        pol = [(bits >> s) & 1 for s in range(n)]
        Pp = np.array([Pm[pol[s], s] for s in range(n)])
        Rp = np.array([R[pol[s], s] for s in range(n)])
        V = np.linalg.solve(np.eye(n) - inst.gamma * Pp, Rp)
        best = V if best is None else np.maximum(best, V)
    res = P.vi_solve(1e-13, 5000, stop_rule=1)
    assert res["converged"]
    np.testing.assert_allclose(res["V"], best, rtol=0, atol=1e-9)


def test_periodic_test_fires_on_a_stable_policy():
    inst = w.periodic_instance(3, 6, 8, (1.0, 0.5), (0.2, 0.3), (10.0, 1.0, 20.0, 5.0), 0.95)
    P = oracle.PeriodicProblem(inst)
    res = P.vi_solve(1e-4, 10_000, stop_rule=2)
    assert res["converged"] and res["iters"] >= 7
    assert res["dmax"] - res["dmin"] <= 2e-4 * min(abs(res["dmax"]), abs(res["dmin"]))
    # the test's rationale: the weekly change is the same everywhere, so the
    # greedy policy no longer changes (300 more sweeps give the same policy)
    far = P.vi_solve(0.0, res["iters"] + 300, stop_rule=0)
    assert (res["policy"] == far["policy"]).all()


@pytest.mark.parametrize("row", GOLDEN["rows"], ids=[f"m{r['m']}e{r['exp']}" for r in GOLDEN["rows"]])
def test_scenario_c_sizes_match_table6(row):
    m = row["m"]
    inst = w.scenario_c(m, row["exp"])
    assert inst.n_states == row["n_states"]
    assert inst.n_actions == row["n_actions"]
    assert inst.n_outcomes == row["n_outcomes"]
    if m <= 5:
        P = oracle.PeriodicProblem(inst)
        assert P.n_states == row["n_states"]
        profiles = sum(len(P.profiles(a)) for a in range(inst.Q + 1))
        assert 21 * profiles == row["n_outcomes"]


@pytest.mark.parametrize("row", [r for r in GOLDEN["rows"] if r["m"] == 3], ids=["m3e1", "m3e2"])
def test_scenario_c_sS_policy_matches_the_paper(row):
    """The printed best (s, S) weekday parameters (Table 15), 10,000 rollouts of
    365 days after 100: Table 6's simulation-optimisation return and Table 16's
    KPIs (paper rounding plus 4 standard errors of two independent samples)."""
    inst = w.scenario_c(3, row["exp"])
    P = oracle.PeriodicProblem(inst)
    RO = w.SCENARIO_C_ROLLOUTS
    out = P.simulate(sS_policy(inst, row["s_best"], row["S_best"]), RO["n_rollouts"], RO["horizon"], seed=2023,
                     warmup=RO["warmup"])
    r, k = out["returns"], out["kpis"]
    n = len(r)
    assert abs(r.mean() - row["so_return_mean"]) <= 0.5 + 4 * row["so_return_sd"] * math.sqrt(2.0 / n)
    assert abs(r.std(ddof=1) - row["so_return_sd"]) <= 3.0
    for j, key in enumerate(("service_so", "wastage_so", "holding_so")):
        mean, sd = row[key]
        assert abs(k[:, j].mean() - mean) <= 0.05 + 4 * sd * math.sqrt(2.0 / n), (key, k[:, j].mean())
