"""ctypes wrapper around the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline / reference leg.  The product path (the CUDA library
and its Python binding) never imports this package, and this package never
imports the product.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = [os.path.join(HERE, "oracle.c"), os.path.join(HERE, "oracle_pc.c")]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, no fused multiply-add, OpenMP)."""
    newest = max(os.path.getmtime(p) for p in SOURCES + [os.path.join(HERE, "oracle.h")])
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", LIB_PATH] + SOURCES + ["-lm"]
    subprocess.check_call(cmd)
    return LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("n_products", C.c_int),
        ("m", C.c_int * 2), ("L", C.c_int * 2), ("Q", C.c_int * 2),
        ("cost", (C.c_double * 5) * 2),
        ("pmf", C.POINTER(C.c_double) * 2),
        ("dmax", C.c_int * 2),
        ("rho", C.c_double),
        ("gamma", C.c_double),
        ("issuing", C.c_int),
    ]


class _Step(C.Structure):
    _fields_ = [
        ("s_next", C.c_longlong), ("reward", C.c_double), ("demand", C.c_double),
        ("issued", C.c_double), ("wasted", C.c_double), ("carried", C.c_double),
        ("arrived", C.c_double), ("shortage", C.c_double), ("unmet1", C.c_int),
        ("demand_k", C.c_double * 2), ("issued_k", C.c_double * 2), ("wasted_k", C.c_double * 2),
        ("carried_k", C.c_double * 2), ("arrived_k", C.c_double * 2), ("sub_served", C.c_int),
    ]


class _Periodic(C.Structure):
    _fields_ = [
        ("m", C.c_int), ("Q", C.c_int), ("dmax", C.c_int),
        ("pmf", C.POINTER(C.c_double)),
        ("c0", C.c_double * 9), ("c1", C.c_double * 9),
        ("cost", C.c_double * 4),
        ("gamma", C.c_double),
    ]


class _PcStep(C.Structure):
    _fields_ = [
        ("s_next", C.c_longlong), ("reward", C.c_double), ("demand", C.c_double), ("issued", C.c_double),
        ("wasted", C.c_double), ("held", C.c_double), ("accepted", C.c_double), ("refused", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        P = C.POINTER(_Problem)
        dp = C.POINTER(C.c_double)
        L.orc_num_states.argtypes = [P]
        L.orc_num_states.restype = C.c_longlong
        L.orc_num_actions.argtypes = [P]
        L.orc_num_actions.restype = C.c_int
        L.orc_transition.argtypes = [P, C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.POINTER(_Step)]
        L.orc_qvalues.argtypes = [P, dp, C.c_longlong, dp]
        L.orc_vi_solve.argtypes = [P, C.c_double, C.c_int, C.c_int, dp, C.c_void_p,
                                   C.POINTER(C.c_int), dp, dp, dp, C.c_int]
        L.orc_backup_states.argtypes = [P, dp, C.c_void_p, C.c_longlong, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_int]
        L.orc_policy_eval.argtypes = [P, C.c_void_p, C.c_double, C.c_int, dp,
                                      C.POINTER(C.c_int), C.c_int]
        L.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_simulate.argtypes = [P, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_simulate_ex.argtypes = [P, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_basestock_policy.argtypes = [P, C.c_int, C.c_void_p]
        PP = C.POINTER(_Periodic)
        L.orc_pc_num_states.argtypes = [PP]
        L.orc_pc_num_states.restype = C.c_longlong
        L.orc_pc_arrival_params.argtypes = [PP, C.c_int, C.c_void_p]
        L.orc_pc_arrival_prob.argtypes = [PP, C.c_int, C.c_void_p]
        L.orc_pc_arrival_prob.restype = C.c_double
        L.orc_pc_next_profile.argtypes = [C.c_int, C.c_int, C.c_void_p]
        L.orc_pc_transition.argtypes = [PP, C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.POINTER(_PcStep)]
        L.orc_pc_qvalues.argtypes = [PP, dp, C.c_longlong, dp]
        L.orc_pc_backup_states.argtypes = [PP, dp, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p, C.c_int]
        L.orc_pc_vi_solve.argtypes = [PP, C.c_double, C.c_int, C.c_int, dp, C.c_void_p, C.POINTER(C.c_int), dp,
                                      dp, dp, C.c_int]
        L.orc_pc_simulate.argtypes = [PP, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_void_p,
                                      C.c_void_p, C.c_void_p]
        L.orc_issued_pmf.argtypes = [P, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p]
        L.orc_mbs_simulate.argtypes = [P, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.c_uint64, C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Problem:
    """An oracle view of a workloads.Instance (keeps its pmf arrays alive)."""

    def __init__(self, inst, gamma: Optional[float] = None):
        self.inst = inst
        st = _Problem()
        prods = inst.products
        st.n_products = len(prods)
        self._pmfs = []
        for k, p in enumerate(prods):
            st.m[k], st.L[k], st.Q[k] = p.m, p.L, p.Q
            for j in range(5):
                st.cost[k][j] = float(p.cost[j])
            arr = np.ascontiguousarray(p.pmf, dtype=np.float64)
            self._pmfs.append(arr)
            st.pmf[k] = arr.ctypes.data_as(C.POINTER(C.c_double))
            st.dmax[k] = len(arr) - 1
        st.rho = float(inst.subst_rate)
        st.gamma = float(inst.gamma if gamma is None else gamma)
        st.issuing = int(inst.issuing)
        self.st = st
        self.n_states = int(lib().orc_num_states(C.byref(st)))
        self.n_actions = int(lib().orc_num_actions(C.byref(st)))

    @property
    def ref(self):
        return C.byref(self.st)

    # -- model -------------------------------------------------------------
    def transition(self, s: int, a: int, d1: int, d2: int = 0, u: int = 0) -> dict:
        out = _Step()
        rc = lib().orc_transition(self.ref, s, a, d1, d2, u, C.byref(out))
        if rc != 0:
            raise ValueError("invalid outcome")
        res = {}
        for f, _ in _Step._fields_:
            v = getattr(out, f)
            res[f] = list(v) if f.endswith("_k") else v
        return res

    def issued_pmf(self, s: int, a: int) -> np.ndarray:
        """P(h1, h2 | s, a) from the Scenario B five-case formula; (T1+1) x (T2+1)."""
        T = np.zeros(2, np.int32)
        p1, p2 = self.inst.products
        buf = np.zeros((p1.m * p1.Q + 1) * (p2.m * p2.Q + 1), np.float64)
        if lib().orc_issued_pmf(self.ref, s, a, _ptr(buf), _ptr(T)) != 0:
            raise RuntimeError("orc_issued_pmf failed")
        n1, n2 = int(T[0]) + 1, int(T[1]) + 1
        return buf[: n1 * n2].reshape(n1, n2).copy()

    def qvalues(self, V: np.ndarray, s: int) -> np.ndarray:
        V = np.ascontiguousarray(V, np.float64)
        q = np.empty(self.n_actions, np.float64)
        lib().orc_qvalues(self.ref, V.ctypes.data_as(C.POINTER(C.c_double)), s,
                          q.ctypes.data_as(C.POINTER(C.c_double)))
        return q

    # -- algorithms ----------------------------------------------------------
    def vi_solve(self, tol: float, max_iters: int, stop_rule: int = 0, V0=None,
                 nthreads: int = 0) -> dict:
        V = np.zeros(self.n_states) if V0 is None else np.array(V0, np.float64, copy=True)
        pol = np.zeros(self.n_states, np.uint8)
        it = C.c_int(0)
        crit, dmx, dmn = C.c_double(0), C.c_double(0), C.c_double(0)
        rc = lib().orc_vi_solve(self.ref, tol, stop_rule, max_iters,
                                V.ctypes.data_as(C.POINTER(C.c_double)), _ptr(pol),
                                C.byref(it), C.byref(crit), C.byref(dmx), C.byref(dmn), nthreads)
        if rc not in (0, 3):
            raise RuntimeError(f"orc_vi_solve failed rc={rc}")
        return dict(V=V, policy=pol, iters=it.value, converged=(rc == 0), crit=crit.value,
                    dmax=dmx.value, dmin=dmn.value)

    def backup_states(self, V: np.ndarray, states, with_q: bool = False, nthreads: int = 0):
        V = np.ascontiguousarray(V, np.float64)
        states = np.ascontiguousarray(states, np.int64)
        n = len(states)
        v = np.empty(n, np.float64)
        pol = np.empty(n, np.int32)
        q = np.empty((n, self.n_actions), np.float64) if with_q else None
        rc = lib().orc_backup_states(self.ref, V.ctypes.data_as(C.POINTER(C.c_double)),
                                     _ptr(states), n, _ptr(v), _ptr(pol), _ptr(q), nthreads)
        if rc != 0:
            raise RuntimeError("orc_backup_states failed")
        return (v, pol, q) if with_q else (v, pol)

    def policy_eval(self, policy: np.ndarray, tol: float, max_iters: int, V0=None,
                    nthreads: int = 0):
        V = np.zeros(self.n_states) if V0 is None else np.array(V0, np.float64, copy=True)
        policy = np.ascontiguousarray(policy, np.uint8)
        it = C.c_int(0)
        rc = lib().orc_policy_eval(self.ref, _ptr(policy), tol, max_iters,
                                   V.ctypes.data_as(C.POINTER(C.c_double)), C.byref(it), nthreads)
        if rc not in (0, 3):
            raise RuntimeError("orc_policy_eval failed")
        return V, it.value, rc == 0

    def simulate(self, policy: np.ndarray, n_rollouts: int, horizon: int, seed: int,
                 warmup: int = 0, with_traj: bool = False):
        policy = np.ascontiguousarray(policy, np.uint8)
        ret = np.empty(n_rollouts, np.float64)
        kpis = np.empty((n_rollouts, 3), np.float64)
        kprod = np.empty((n_rollouts, 2, 3), np.float64)
        traj = np.empty((n_rollouts, horizon), np.int32) if with_traj else None
        dem = np.empty((n_rollouts, horizon), np.int32) if with_traj else None
        rc = lib().orc_simulate_ex(self.ref, _ptr(policy), n_rollouts, horizon, warmup,
                                   C.c_uint64(seed), _ptr(ret), _ptr(kpis), _ptr(kprod), _ptr(traj),
                                   _ptr(dem))
        if rc != 0:
            raise RuntimeError("orc_simulate failed")
        out = dict(returns=ret, kpis=kpis, kpis_prod=kprod)
        if with_traj:
            out["traj"] = traj
            out["demand"] = dem
        return out


    def mbs_simulate(self, S, mu, n_rollouts: int, horizon: int, seed: int, warmup: int = 0,
                     cap: bool = False) -> dict:
        """Modified base-stock rollouts: order [S_k - I_k + [X_1k - mu_k]^+]^+ per product."""
        Sv = np.ascontiguousarray(list(S) + [0] * (2 - len(S)), np.int32)
        mv = np.ascontiguousarray(list(mu) + [0] * (2 - len(mu)), np.int32)
        ret = np.empty(n_rollouts, np.float64)
        kprod = np.empty((n_rollouts, 2, 3), np.float64)
        rc = lib().orc_mbs_simulate(self.ref, _ptr(Sv), _ptr(mv), int(bool(cap)), n_rollouts, horizon,
                                    warmup, C.c_uint64(seed), _ptr(ret), _ptr(kprod))
        if rc != 0:
            raise RuntimeError("orc_mbs_simulate failed")
        return dict(returns=ret, kpis_prod=kprod)

    def basestock_policy(self, S: int) -> np.ndarray:
        """A = [S - I]^+ (I: stock on hand and in transit), capped at Q, for every state."""
        pol = np.empty(self.n_states, np.uint8)
        if lib().orc_basestock_policy(self.ref, int(S), _ptr(pol)) != 0:
            raise RuntimeError("orc_basestock_policy failed")
        return pol


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.empty(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


class PeriodicProblem:
    """An oracle view of a workloads.PeriodicInstance (Scenario C)."""

    def __init__(self, inst):
        self.inst = inst
        st = _Periodic()
        st.m, st.Q, st.dmax = inst.m, inst.Q, inst.dmax
        self._pmf = np.ascontiguousarray(inst.pmf, dtype=np.float64).reshape(7, inst.dmax + 1)
        st.pmf = self._pmf.ctypes.data_as(C.POINTER(C.c_double))
        for k in range(9):
            st.c0[k] = float(inst.c0[k]) if k < len(inst.c0) else 0.0
            st.c1[k] = float(inst.c1[k]) if k < len(inst.c1) else 0.0
        for j in range(4):
            st.cost[j] = float(inst.cost[j])
        st.gamma = float(inst.gamma)
        self.st = st
        self.n_states = int(lib().orc_pc_num_states(C.byref(st)))
        self.n_actions = inst.Q + 1

    @property
    def ref(self):
        return C.byref(self.st)

    def arrival_params(self, a: int) -> np.ndarray:
        p = np.zeros(9, np.float64)
        lib().orc_pc_arrival_params(self.ref, a, _ptr(p))
        return p[1:self.inst.m + 1].copy()

    def arrival_prob(self, a: int, y) -> float:
        v = np.zeros(9, np.int32)
        v[1:len(y) + 1] = y
        return float(lib().orc_pc_arrival_prob(self.ref, a, _ptr(v)))

    def profiles(self, a: int):
        """All y (y[0] = units with 1 day left ... y[m-1] fresh) with sum a, in the oracle's order."""
        m = self.inst.m
        y = np.zeros(9, np.int32)
        y[1] = a
        out = [y[1:m + 1].copy()]
        while lib().orc_pc_next_profile(m, a, _ptr(y)):
            out.append(y[1:m + 1].copy())
        return out

    def transition(self, s: int, a: int, d: int, y) -> dict:
        v = np.zeros(9, np.int32)
        v[1:len(y) + 1] = y
        out = _PcStep()
        if lib().orc_pc_transition(self.ref, s, a, d, _ptr(v), C.byref(out)) != 0:
            raise ValueError("invalid outcome")
        return {f: getattr(out, f) for f, _ in _PcStep._fields_}

    def qvalues(self, V: np.ndarray, s: int) -> np.ndarray:
        V = np.ascontiguousarray(V, np.float64)
        q = np.empty(self.n_actions, np.float64)
        lib().orc_pc_qvalues(self.ref, V.ctypes.data_as(C.POINTER(C.c_double)), s,
                             q.ctypes.data_as(C.POINTER(C.c_double)))
        return q

    def vi_solve(self, eps: float, max_iters: int, stop_rule: int = 2, V0=None, nthreads: int = 0) -> dict:
        V = np.zeros(self.n_states) if V0 is None else np.array(V0, np.float64, copy=True)
        pol = np.zeros(self.n_states, np.uint8)
        it = C.c_int(0)
        crit, dmx, dmn = C.c_double(0), C.c_double(0), C.c_double(0)
        rc = lib().orc_pc_vi_solve(self.ref, eps, stop_rule, max_iters, V.ctypes.data_as(C.POINTER(C.c_double)),
                                   _ptr(pol), C.byref(it), C.byref(crit), C.byref(dmx), C.byref(dmn), nthreads)
        if rc not in (0, 3):
            raise RuntimeError(f"orc_pc_vi_solve failed rc={rc}")
        return dict(V=V, policy=pol, iters=it.value, converged=(rc == 0), crit=crit.value, dmax=dmx.value,
                    dmin=dmn.value)

    def backup_states(self, V: np.ndarray, states, nthreads: int = 0):
        V = np.ascontiguousarray(V, np.float64)
        states = np.ascontiguousarray(states, np.int64)
        n = len(states)
        v = np.empty(n, np.float64)
        pol = np.empty(n, np.int32)
        if lib().orc_pc_backup_states(self.ref, V.ctypes.data_as(C.POINTER(C.c_double)), _ptr(states), n,
                                      _ptr(v), _ptr(pol), nthreads) != 0:
            raise RuntimeError("orc_pc_backup_states failed")
        return v, pol

    def simulate(self, policy: np.ndarray, n_rollouts: int, horizon: int, seed: int, warmup: int = 0,
                 with_traj: bool = False) -> dict:
        policy = np.ascontiguousarray(policy, np.uint8)
        ret = np.empty(n_rollouts, np.float64)
        kpis = np.empty((n_rollouts, 3), np.float64)
        traj = np.empty((n_rollouts, horizon), np.int32) if with_traj else None
        if lib().orc_pc_simulate(self.ref, _ptr(policy), n_rollouts, horizon, warmup, C.c_uint64(seed),
                                 _ptr(ret), _ptr(kpis), _ptr(traj)) != 0:
            raise RuntimeError("orc_pc_simulate failed")
        out = dict(returns=ret, kpis=kpis)
        if with_traj:
            out["traj"] = traj
        return out
