"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only *generates inputs*: demand pmfs (truncated, tail mass folded
into the last support point), cost vectors drawn from a seeded generator, and
the request stream of the serving mix.  It holds none of the value-iteration
arithmetic, so both the CUDA path and the CPU oracle may take inputs from it
without sharing any of the method's code.

Demand distributions follow the paper's discretise-and-fold rule (Scenario A,
appendix "Scenario description": the mass above the truncation point is put
on D_max) applied to Poisson and negative-binomial demand.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np
from scipy import stats

FIFO, LIFO = 0, 1

# cost vector layout everywhere: (order c_o, holding c_h, shortage c_s, waste c_w, revenue c_r)
COST_FIELDS = ("order", "holding", "shortage", "waste", "revenue")


def folded_pmf(dist, dmax: int) -> np.ndarray:
    """pmf on {0..dmax}: P(D=d) for d < dmax and P(D >= dmax) on dmax."""
    d = np.arange(dmax, dtype=np.float64)
    p = np.empty(dmax + 1, dtype=np.float64)
    p[:dmax] = dist.pmf(d)
    p[dmax] = dist.sf(dmax - 1)  # P(D >= dmax)
    # renormalise the last few ulps so sum == 1 up to rounding of the sum itself
    p[dmax] += 1.0 - p.sum()
    if p[dmax] < 0.0:
        p[dmax] = 0.0
    return p


def poisson_pmf(mean: float, dmax: int) -> np.ndarray:
    return folded_pmf(stats.poisson(mean), dmax)


def negbin_pmf(mean: float, var: float, dmax: int) -> np.ndarray:
    """Negative binomial with the given mean and variance (var > mean):
    n = mean^2/(var-mean) successes, success probability p = mean/var."""
    n = mean * mean / (var - mean)
    p = mean / var
    return folded_pmf(stats.nbinom(n, p), dmax)


def gamma_discretised_pmf(mean: float, sd: float, dmax: int) -> np.ndarray:
    """Gamma demand rounded to the nearest integer (Scenario A appendix): P(D = d) =
    F(d + 1/2) - F(d - 1/2) for d < dmax and 1 - F(dmax - 1/2) on dmax, F = 0 below 0;
    shape (mean/sd)^2, scale sd^2/mean."""
    dist = stats.gamma(a=(mean / sd) ** 2, scale=sd * sd / mean)
    F = lambda x: np.where(x <= 0.0, 0.0, dist.cdf(np.maximum(x, 0.0)))
    d = np.arange(dmax, dtype=np.float64)
    p = np.empty(dmax + 1, dtype=np.float64)
    p[:dmax] = F(d + 0.5) - F(d - 0.5)
    p[dmax] = 1.0 - F(dmax - 0.5)
    return p


@dataclasses.dataclass
class Product:
    m: int                      # maximum useful life (periods)
    L: int                      # lead time (periods)
    Q: int                      # order cap, actions 0..Q, each age slot 0..Q
    cost: Sequence[float]       # (c_o, c_h, c_s, c_w, c_r)
    pmf: np.ndarray             # demand pmf on {0..dmax}

    @property
    def dmax(self) -> int:
        return len(self.pmf) - 1

    @property
    def n_digits(self) -> int:
        return (self.m - 1) + (self.L - 1)

    @property
    def n_states(self) -> int:
        return (self.Q + 1) ** self.n_digits


@dataclasses.dataclass
class Instance:
    """One value-iteration problem instance (one or two products)."""
    name: str
    products: List[Product]
    gamma: float
    issuing: int = FIFO
    subst_rate: float = 0.0      # share of product-1 shortfall willing to take product 2
    tol: float = 1e-4
    max_iters: int = 100_000
    precision: str = "fp32"      # "fp64" | "fp32" | "fp32_kahan"

    @property
    def n_states(self) -> int:
        n = 1
        for p in self.products:
            n *= p.n_states
        return n

    @property
    def n_actions(self) -> int:
        n = 1
        for p in self.products:
            n *= p.Q + 1
        return n

    @property
    def n_outcomes(self) -> int:
        n = 1
        for p in self.products:
            n *= p.dmax + 1
        return n

    @property
    def updates_per_sweep(self) -> int:
        """Nominal |S|*|A|*|Omega| (state-action-demand updates of one sweep)."""
        return self.n_states * self.n_actions * self.n_outcomes


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

PAPER_A_COSTS = (3.0, 1.0, 5.0, 7.0, 0.0)   # C_v=3, C_h=1, C_s=5, C_w=7 (Scenario A settings)


def single_product(m, L, Q, cost, pmf, gamma, issuing=FIFO, name="custom", **kw) -> Instance:
    return Instance(name=name, products=[Product(m, L, Q, tuple(float(c) for c in cost),
                                                 np.asarray(pmf, np.float64))],
                    gamma=gamma, issuing=issuing, **kw)


def config1() -> Instance:
    """m=3, L=1, Q=20 (441 states), Poisson(5) folded at 25, FIFO, costs (3,1,5,7), gamma .99."""
    return single_product(3, 1, 20, PAPER_A_COSTS, poisson_pmf(5.0, 25), 0.99, FIFO,
                          name="cfg1_m3L1Q20_fifo", precision="fp64")


def uniform_costs(rng: np.random.Generator) -> tuple:
    c = rng.uniform(1.0, 10.0, size=4)
    return (float(c[0]), float(c[1]), float(c[2]), float(c[3]), 0.0)


def config2(seed: int = 2) -> Instance:
    """m=5, L=2, Q=20 (21^5 = 4,084,101 states), NB(mean 8, var 20) folded at 40, FIFO,
    costs U[1,10] from a PCG64 stream seeded with `seed`, gamma .99, plain FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return single_product(5, 2, 20, uniform_costs(rng), negbin_pmf(8.0, 20.0, 40), 0.99, FIFO,
                          name="cfg2_m5L2Q20_nb_fifo", precision="fp32")


def config3(Q: int = 14) -> Instance:
    """Two substitutable products, each m=3, L=1, Q=14 (15^4 = 50,625 states, 225 joint
    actions), Poisson(4) and Poisson(6) folded at 20, half of product-1 shortfall accepts
    product 2, order cost 0.5 and revenue 1.0 per unit, gamma .99, FP32 with Kahan sums."""
    c = (0.5, 0.0, 0.0, 0.0, 1.0)
    p1 = Product(3, 1, Q, c, poisson_pmf(4.0, 20))
    p2 = Product(3, 1, Q, c, poisson_pmf(6.0, 20))
    return Instance(name=f"cfg3_2prod_m3L1Q{Q}_subst", products=[p1, p2], gamma=0.99,
                    issuing=FIFO, subst_rate=0.5, precision="fp32_kahan")


def config4() -> Instance:
    """m=8, L=1, Q=10 (11^7 = 19,487,171 states), Poisson(4) folded at 15, LIFO,
    costs (3,1,5,7), gamma .95, FP32."""
    return single_product(8, 1, 10, PAPER_A_COSTS, poisson_pmf(4.0, 15), 0.95, LIFO,
                          name="cfg4_m8L1Q10_lifo", precision="fp32")


CONFIG4_ROLLOUTS = dict(n_rollouts=4096, horizon=365, seed=4)


# The paper's Scenario A (de Moor et al. settings, Scenario A appendix): the state
# holds X_1..X_m (X_m arrived at the start of the day) and L-1 orders in transit,
# m + L - 1 digits in all.  X_m is available before the day's demand, exactly as
# the arrival slot P_1 of this library's state with lead time L + 1, and the
# reward has no revenue term.  Dmax 100, Amax 10, Cv 3, Ch 1, Cs 5, mean demand 4
# with coefficient of variation sigma/mu = 0.5, gamma 0.99, sup-norm test 1e-4.
SCENARIO_A = dict(dmax=100, q=10, c_v=3.0, c_h=1.0, c_s=5.0, mean=4.0, cv=0.5, gamma=0.99, eps=1e-4)
SCENARIO_A_ROLLOUTS = dict(n_rollouts=10_000, horizon=365, warmup=100)


def scenario_a(m: int, L: int, c_w: float, issuing: int) -> Instance:
    """Scenario A experiment (m, L, C_w, issuing) in this library's state convention."""
    a = SCENARIO_A
    pmf = gamma_discretised_pmf(a["mean"], a["cv"] * a["mean"], a["dmax"])
    return single_product(m, L + 1, a["q"], (a["c_v"], a["c_h"], a["c_s"], c_w, 0.0), pmf, a["gamma"], issuing,
                          name=f"scenA_m{m}L{L}Cw{int(c_w)}{'LIFO' if issuing else 'FIFO'}", precision="fp32")


# The paper's Scenario B (Hendrix et al. and Ortega et al. settings, Scenario B
# appendix): two perishable products with the same useful life m.  The paper's
# product B, half of whose unmet demand accepts product A, is product 1 here and
# product A is product 2; a joint action is a1 * (Amax_A + 1) + a2.  The paper's
# lead time L = 1 (an order arrives before the next day and sits in the state as
# X_m) is lead time 2 in this library's convention (the arrival slot P_1).
# Poisson demand, C_v = 0.5 and C_r = 1 per unit for both products, no holding,
# shortage or waste cost, rho = 0.5, gamma = 1, span test 1e-4.  Demand is
# folded at the smallest d with P(D > d) < 1e-12.
SCENARIO_B = dict(c_v=0.5, c_r=1.0, rho=0.5, gamma=1.0, eps=1e-4, tail=1e-12)
SCENARIO_B_ROLLOUTS = dict(n_rollouts=10_000, horizon=365, warmup=100)
# name: (m, mu_A, mu_B, Amax_A, Amax_B, fixed VI iterations or None); Table 4
# (Hendrix et al., run to convergence) and Table 5 (Ortega et al., 100 iterations)
SCENARIO_B_EXPERIMENTS = {
    "m2_exp1": (2, 5, 5, 10, 10, None),
    "m2_exp2": (2, 7, 3, 14, 6, None),
    "m3_exp1": (3, 5, 5, 15, 15, None),
    "m3_exp2": (3, 7, 3, 21, 9, None),
    "m3_exp3": (3, 5, 5, 13, 13, None),
    "m3_exp4": (3, 7, 3, 20, 4, None),
    "P1": (2, 5, 5, 10, 10, 100),
    "P2": (2, 5, 6, 10, 12, 100),
    "P3": (2, 6, 6, 12, 12, 100),
    "P4": (2, 7, 7, 13, 13, 100),
}


def poisson_dmax(mean: float, tail: float) -> int:
    """Smallest d with P(D > d) < tail for D ~ Poisson(mean)."""
    dist = stats.poisson(mean)
    d = 0
    while dist.sf(d) >= tail:
        d += 1
    return d


def scenario_b(name: str, precision: str = "fp32") -> Instance:
    """Scenario B experiment `name` in this library's convention (product 1 = paper's B)."""
    m, mu_a, mu_b, q_a, q_b, _ = SCENARIO_B_EXPERIMENTS[name]
    b = SCENARIO_B
    c = (b["c_v"], 0.0, 0.0, 0.0, b["c_r"])
    pB = Product(m, 2, q_b, c, poisson_pmf(mu_b, poisson_dmax(mu_b, b["tail"])))
    pA = Product(m, 2, q_a, c, poisson_pmf(mu_a, poisson_dmax(mu_a, b["tail"])))
    return Instance(name=f"scenB_{name}", products=[pB, pA], gamma=b["gamma"], issuing=FIFO,
                    subst_rate=b["rho"], tol=b["eps"], precision=precision)


# The paper's Scenario C (Mirjalili's platelet problem, Scenario C appendix):
# weekday-periodic negative binomial demand (Table 13: n^tau successes, mean
# delta^tau, p = n / (n + delta)) folded at D_max = 20; remaining useful life on
# arrival multinomial with log(p_k(a) / p_1(a)) = c0_k + c1_k a (Table 14);
# A_max = 20 for the order and for the stock of each age; C_f 10 per order
# placed, C_h 1, C_s 20, C_w 5 per unit, gamma 0.95, periodic test epsilon 1e-4
# (Table 12).
SCENARIO_C = dict(dmax=20, q=20, c_f=10.0, c_h=1.0, c_s=20.0, c_w=5.0, gamma=0.95, eps=1e-4)
SCENARIO_C_ROLLOUTS = dict(n_rollouts=10_000, horizon=365, warmup=100)
SCENARIO_C_DEMAND = ((3.5, 5.7), (11.0, 6.9), (7.2, 6.5), (11.1, 6.2), (5.9, 5.8), (5.5, 3.3), (2.2, 3.4))
# (m, experiment): (c0_2..c0_m, c1_2..c1_m); experiment 1 exogenous, 2 endogenous
SCENARIO_C_LIFE = {
    (3, 1): ((1.0, 0.5), (0.0, 0.0)),
    (3, 2): ((1.0, 0.5), (0.40, 0.80)),
    (5, 1): ((1.6, 2.6, 2.8, 1.6), (0.0, 0.0, 0.0, 0.0)),
    (5, 2): ((1.9, 3.1, 3.1, 2.5), (-0.03, -0.06, -0.03, -0.09)),
    (8, 1): ((0.8, 1.4, 1.9, 2.3, 1.7, 1.2, 0.8), (0.0,) * 7),
    (8, 2): ((0.8, 1.4, 1.9, 2.3, 1.7, 1.2, 0.8), (-0.03, -0.04, -0.05, -0.06, -0.07, -0.08, -0.09)),
}


@dataclasses.dataclass
class PeriodicInstance:
    """A Scenario C instance: weekday in the state, multinomial age on arrival."""
    name: str
    m: int
    Q: int                      # A_max
    pmf: np.ndarray             # 7 x (dmax+1), row tau = weekday demand pmf
    c0: Sequence[float]         # index k = 0..m (entries 0 and 1 unused, zero)
    c1: Sequence[float]
    cost: Sequence[float]       # (C_f, C_h, C_s, C_w)
    gamma: float
    tol: float = 1e-4

    @property
    def dmax(self) -> int:
        return self.pmf.shape[1] - 1

    @property
    def n_states(self) -> int:
        return 7 * (self.Q + 1) ** (self.m - 1)

    @property
    def n_actions(self) -> int:
        return self.Q + 1

    @property
    def n_outcomes(self) -> int:
        """The paper's |Omega|: demands x arrival age profiles y with sum y <= A_max."""
        from math import comb
        return (self.dmax + 1) * comb(self.Q + self.m, self.m)


def scenario_c_demand(dmax: int) -> np.ndarray:
    """Weekday demand pmfs (Eq. mirjalili:demand), folded at dmax."""
    rows = []
    for n, delta in SCENARIO_C_DEMAND:
        rows.append(folded_pmf(stats.nbinom(n, n / (n + delta)), dmax))
    return np.stack(rows)


def periodic_instance(m, Q, dmax, c0, c1, cost, gamma, name="periodic", pmf=None) -> PeriodicInstance:
    pmf = scenario_c_demand(dmax) if pmf is None else np.asarray(pmf, np.float64)
    return PeriodicInstance(name=name, m=m, Q=Q, pmf=pmf, c0=[0.0, 0.0] + list(c0), c1=[0.0, 0.0] + list(c1),
                            cost=tuple(cost), gamma=gamma)


def scenario_c(m: int, exp: int) -> PeriodicInstance:
    c = SCENARIO_C
    c0, c1 = SCENARIO_C_LIFE[(m, exp)]
    return periodic_instance(m, c["q"], c["dmax"], c0, c1, (c["c_f"], c["c_h"], c["c_s"], c["c_w"]), c["gamma"],
                             name=f"scenC_m{m}_exp{exp}")


@dataclasses.dataclass
class Request:
    arrival_s: float
    instance: Instance


def serving_mix(n_requests: int = 512, seed: int = 5, rate_per_s: float = 200.0,
                max_states: int = 21 ** 5) -> List[Request]:
    """Serving workload: independent single-product instances arriving as a Poisson stream.

    m ~ U{2..6}, L ~ U{1,2,3}, Q ~ U{8..20}, redrawn until (Q+1)^(m+L-2) <= max_states;
    demand Poisson(mu), mu ~ U[2,10], folded at floor(3 mu + 5); four costs U[1,10];
    gamma ~ U{0.9, 0.95, 0.99}; FIFO.  Exponential inter-arrival gaps of mean 1/rate.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n_requests):
        while True:
            m = int(rng.integers(2, 7))
            L = int(rng.integers(1, 4))
            Q = int(rng.integers(8, 21))
            if (Q + 1) ** (m + L - 2) <= max_states:
                break
        mu = float(rng.uniform(2.0, 10.0))
        dmax = int(np.floor(3.0 * mu + 5.0))
        cost = uniform_costs(rng)
        gamma = float(rng.choice([0.9, 0.95, 0.99]))
        t += float(rng.exponential(1.0 / rate_per_s))
        inst = single_product(m, L, Q, cost, poisson_pmf(mu, dmax), gamma, FIFO,
                              name=f"req{i}_m{m}L{L}Q{Q}", precision="fp32")
        out.append(Request(arrival_s=t, instance=inst))
    return out


def random_small_instance(rng: np.random.Generator, max_states: int = 400,
                          two_product: bool = False) -> Instance:
    """A random tiny instance (for exhaustive parity sweeps)."""
    if two_product:
        while True:
            Q1, Q2 = int(rng.integers(1, 4)), int(rng.integers(1, 4))
            m1, m2 = int(rng.integers(1, 4)), int(rng.integers(1, 4))
            n = (Q1 + 1) ** (m1 - 1) * (Q2 + 1) ** (m2 - 1)
            if n <= max_states:
                break
        mus = rng.uniform(0.5, 4.0, size=2)
        c1 = (float(rng.uniform(0, 2)), float(rng.uniform(0, 1)), float(rng.uniform(0, 3)),
              float(rng.uniform(0, 3)), float(rng.uniform(0, 3)))
        c2 = (float(rng.uniform(0, 2)), float(rng.uniform(0, 1)), float(rng.uniform(0, 3)),
              float(rng.uniform(0, 3)), float(rng.uniform(0, 3)))
        p1 = Product(m1, 1, Q1, c1, poisson_pmf(mus[0], int(rng.integers(1, 9))))
        p2 = Product(m2, 1, Q2, c2, poisson_pmf(mus[1], int(rng.integers(1, 9))))
        return Instance(name="rand2", products=[p1, p2], gamma=float(rng.uniform(0.5, 0.95)),
                        issuing=int(rng.integers(0, 2)), subst_rate=float(rng.uniform(0, 1)))
    while True:
        m = int(rng.integers(1, 5))
        L = int(rng.integers(1, 4))
        Q = int(rng.integers(0, 7))
        if (Q + 1) ** (m + L - 2) <= max_states:
            break
    mu = float(rng.uniform(0.3, 6.0))
    dmax = int(rng.integers(0, 14))
    cost = tuple(float(c) for c in rng.uniform(0.0, 10.0, size=5))
    return single_product(m, L, Q, cost, poisson_pmf(mu, dmax), float(rng.uniform(0.3, 0.99)),
                          int(rng.integers(0, 2)), name="rand1")


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4}
