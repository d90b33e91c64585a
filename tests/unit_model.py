"""An independent, unit-by-unit restatement of the inventory dynamics.

The oracle evaluates the paper's closed-form issuing equations (Eq. demoor:fifo
and Eq. demoor:lifo).  This module instead issues demand one unit at a time from
the oldest (FIFO) or freshest (LIFO) non-empty age slot, then expires what is
left in the oldest slot and ages the rest -- the verbal description of the
Scenario A / Scenario B dynamics.  Being a different formulation, it is used to
pin the oracle: brute-force policy enumeration, the gamma = 0 special case and
the invariants are computed from it.
"""
from __future__ import annotations

import itertools
import math
from typing import List, Tuple

import numpy as np


def decode(s: int, Q: int, K: int) -> List[int]:
    out = []
    for _ in range(K):
        out.append(s % (Q + 1))
        s //= Q + 1
    return out


def encode(digits, Q: int) -> int:
    s, w = 0, 1
    for x in digits:
        s += x * w
        w *= Q + 1
    return s


def product_period(m, L, Q, issuing, s, a, demand):
    """Returns (s_next, issued, wasted, carried, shortage, arrived, total)."""
    K = (m - 1) + (L - 1)
    dig = decode(s, Q, K)
    stock = dig[: m - 1]                 # remaining life 1..m-1
    pipe = dig[m - 1:]                   # P_1..P_{L-1}
    arrival = pipe[0] if L >= 2 else a
    slots = stock + [arrival]            # slots[0] oldest ... slots[m-1] freshest
    total = sum(slots)
    issued = 0
    left = demand
    while left > 0:
        order = range(m) if issuing == 0 else range(m - 1, -1, -1)
        took = False
        for j in order:
            if slots[j] > 0:
                slots[j] -= 1
                issued += 1
                left -= 1
                took = True
                break
        if not took:
            break
    shortage = demand - issued
    wasted = slots[0]                    # oldest slot expires at the end of the period
    new_stock = slots[1:]                # everything else loses one period of life
    carried = sum(new_stock)
    new_pipe = (pipe[1:] + [a]) if L >= 2 else []
    s_next = encode(new_stock + new_pipe, Q)
    return s_next, issued, wasted, carried, shortage, arrival, total


def outcomes(inst, s, a):
    """All (probability, s_next, reward) triples of one state-action pair."""
    prods = inst.products
    if len(prods) == 1:
        p = prods[0]
        c = p.cost
        for d, pd in enumerate(p.pmf):
            sn, iss, w, car, sh, arr, tot = product_period(p.m, p.L, p.Q, inst.issuing, s, a, d)
            r = -c[0] * a - c[1] * car - c[2] * sh - c[3] * w + c[4] * iss
            yield pd, sn, r
        return
    p1, p2 = prods
    S1 = p1.n_states
    s1, s2 = s % S1, s // S1
    a1, a2 = divmod(a, p2.Q + 1)
    rho = inst.subst_rate
    for d1, pd1 in enumerate(p1.pmf):
        sn1, iss1, w1, car1, sh1, _, _ = product_period(p1.m, p1.L, p1.Q, inst.issuing, s1, a1, d1)
        for d2, pd2 in enumerate(p2.pmf):
            for u in range(sh1 + 1):
                pb = math.comb(sh1, u) * rho ** u * (1 - rho) ** (sh1 - u)
                # product 2 first serves its own customers, then the u substitutes
                sn2, iss2, w2, car2, _, _, tot2 = product_period(p2.m, p2.L, p2.Q, inst.issuing,
                                                                s2, a2, d2 + u)
                own2 = min(d2, tot2)
                lost1 = sh1 - (iss2 - own2)
                lost2 = d2 - own2
                c1, c2 = p1.cost, p2.cost
                r = (-c1[0] * a1 - c1[1] * car1 - c1[2] * lost1 - c1[3] * w1 + c1[4] * iss1
                     - c2[0] * a2 - c2[1] * car2 - c2[2] * lost2 - c2[3] * w2 + c2[4] * iss2)
                yield pd1 * pd2 * pb, sn1 + S1 * sn2, r


def dense_model(inst) -> Tuple[np.ndarray, np.ndarray]:
    """P[a, s, s'] and expected one-step reward R[a, s]."""
    S, A = inst.n_states, inst.n_actions
    P = np.zeros((A, S, S))
    R = np.zeros((A, S))
    for s in range(S):
        for a in range(A):
            for pr, sn, r in outcomes(inst, s, a):
                P[a, s, sn] += pr
                R[a, s] += pr * r
    return P, R


def policy_values(P, R, gamma, policies: np.ndarray) -> np.ndarray:
    """Exact V^pi = (I - gamma P_pi)^{-1} r_pi for a batch of policies (n_pol x S)."""
    n, S = policies.shape
    idx = np.arange(S)
    Ppi = P[policies, idx[None, :], :]          # n x S x S
    Rpi = R[policies, idx[None, :]]             # n x S
    M = np.eye(S)[None] - gamma * Ppi
    return np.linalg.solve(M, Rpi[..., None])[..., 0]


def all_policies(S: int, A: int) -> np.ndarray:
    return np.array(list(itertools.product(range(A), repeat=S)), dtype=np.int64)
