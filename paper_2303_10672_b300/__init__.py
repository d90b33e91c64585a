"""Python binding of libvi_b300.so (the C ABI in include/vi.h).

Argument marshalling only: every step of value iteration, policy evaluation and
simulation runs in the library's CUDA kernels.  Device buffers are passed as
torch tensors (or raw integer addresses), streams as torch.cuda.Stream (or raw
cudaStream_t integers).  If the shared library is missing or cannot be loaded
the import of the binding fails -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvi_b300.so")

VI_OK, VI_EINVAL, VI_ENOMEM, VI_ENOTCONVERGED, VI_ETIMEOUT, VI_EBUSY, VI_ECUDA, VI_ECANCELLED = range(8)
VI_FIFO, VI_LIFO = 0, 1
VI_STOP_SPAN, VI_STOP_SUPNORM, VI_STOP_PERIODIC = 0, 1, 2
VI_PREC_FP32, VI_PREC_FP32_KAHAN, VI_PREC_FP64, VI_PREC_FP32_SINGLE = 0, 1, 2, 3
VI_FLAG_WARM_START, VI_FLAG_NO_GRAPH, VI_FLAG_POLICY_EVAL = 1, 2, 4
VI_OPT_KERNEL, VI_OPT_PE_MAX_ITERS, VI_OPT_GROUP_WIDTH, VI_OPT_TEST_STALL = 1, 2, 3, 4
VI_KERNEL_AUTO, VI_KERNEL_GENERIC, VI_KERNEL_GROUP, VI_KERNEL_TENSOR, VI_KERNEL_LIFO_L1, VI_KERNEL_FIFO_COL = \
    0, 1, 2, 3, 4, 5

PRECISIONS = {"fp32": VI_PREC_FP32, "fp32_kahan": VI_PREC_FP32_KAHAN, "fp64": VI_PREC_FP64,
              "fp32_single": VI_PREC_FP32_SINGLE}


class ViError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {status_name(status)} ({message})")
        self.status = status


class vi_periodic_desc(C.Structure):
    _fields_ = [
        ("m", C.c_int), ("Q", C.c_int), ("dmax", C.c_int),
        ("pmf", C.POINTER(C.c_double)),
        ("c0", C.c_double * 9), ("c1", C.c_double * 9),
        ("cost", C.c_double * 4),
        ("gamma", C.c_double),
        ("stop_rule", C.c_int),
    ]


class vi_problem_desc(C.Structure):
    _fields_ = [
        ("n_products", C.c_int),
        ("m", C.c_int * 2), ("L", C.c_int * 2), ("Q", C.c_int * 2),
        ("cost", (C.c_double * 5) * 2),
        ("pmf", C.POINTER(C.c_double) * 2),
        ("dmax", C.c_int * 2),
        ("subst_rate", C.c_double),
        ("gamma", C.c_double),
        ("issuing", C.c_int),
        ("precision", C.c_int),
        ("stop_rule", C.c_int),
    ]


class vi_solve_info(C.Structure):
    _fields_ = [
        ("iters", C.c_int), ("status", C.c_int), ("crit", C.c_double),
        ("dmax", C.c_double), ("dmin", C.c_double), ("offset", C.c_double),
        ("wall_ms", C.c_double), ("updates_per_s", C.c_double),
        ("pe_iters", C.c_int), ("pe_delta", C.c_double), ("pe_gap", C.c_double),
        ("pe_span", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib() -> C.CDLL:
    """Load libvi_b300.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2303_10672_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp, u8p = C.c_void_p, C.c_void_p
    H = C.c_void_p
    sigs = {
        "vi_problem_create": ([C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.c_int, C.c_double, C.c_int, C.POINTER(H)], C.c_int),
        "vi_problem_create_desc": ([C.POINTER(vi_problem_desc), C.POINTER(H)], C.c_int),
        "vi_problem_destroy": ([H], C.c_int),
        "vi_release_cached_memory": ([C.POINTER(C.c_size_t)], C.c_int),
        "vi_cached_memory": ([C.POINTER(C.c_size_t)], C.c_int),
        "vi_problem_sizes": ([H, C.POINTER(C.c_uint64), C.POINTER(C.c_int), C.POINTER(C.c_int),
                              C.POINTER(C.c_int)], C.c_int),
        "vi_problem_set_option": ([H, C.c_int, C.c_int], C.c_int),
        "vi_solve": ([H, C.c_double, C.c_int, vp, u8p, vp, C.c_int, C.POINTER(vi_solve_info)], C.c_int),
        "vi_solve_host": ([H, C.c_double, C.c_int, vp, u8p, C.c_int, C.POINTER(vi_solve_info)], C.c_int),
        "vi_backup": ([H, vp, vp, u8p, vp, C.POINTER(C.c_double)], C.c_int),
        "vi_policy_eval": ([H, u8p, vp, C.c_double, C.c_int, vp, C.POINTER(C.c_int),
                            C.POINTER(C.c_double)], C.c_int),
        "vi_next_states": ([H, vp, C.c_int, vp, vp], C.c_int),
        "vi_simulate": ([H, u8p, C.c_int, C.c_int, C.c_int, C.c_uint64, vp, vp, vp, vp], C.c_int),
        "vi_problem_create_periodic": ([C.POINTER(vi_periodic_desc), C.POINTER(C.c_void_p)], C.c_int),
        "vi_simulate_ex": ([H, u8p, C.c_int, C.c_int, C.c_int, C.c_uint64, vp, vp, vp, vp, vp], C.c_int),
        "vi_mbs_search": ([H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int, C.c_int,
                           C.c_int, C.c_int, C.c_uint64, vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_int), vp],
                          C.c_int),
        "vi_server_create": ([C.c_size_t, C.c_int, vp, C.POINTER(C.c_void_p)], C.c_int),
        "vi_server_submit": ([C.c_void_p, C.POINTER(vi_problem_desc), C.c_double, C.c_int,
                              C.POINTER(C.c_uint64)], C.c_int),
        "vi_server_poll": ([C.c_void_p, C.c_uint64, C.POINTER(C.c_int), vp, vp, C.POINTER(vi_solve_info)],
                           C.c_int),
        "vi_server_destroy": ([C.c_void_p], C.c_int),
        "vi_server_wait": ([C.c_void_p, C.c_int, vp, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "vi_server_submit_to": ([C.c_void_p, C.POINTER(vi_problem_desc), C.c_double, C.c_int, vp, vp,
                                 C.POINTER(C.c_uint64)], C.c_int),
        "vi_backup_noalloc": ([C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.c_int, C.c_double, C.c_int, vp, vp, u8p, C.POINTER(C.c_double), vp], C.c_int),
        "vi_probe_l2_read": ([vp, C.c_size_t, C.c_int, vp, C.POINTER(C.c_float)], C.c_int),
        "vi_basestock_search": ([H, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, vp,
                                 C.POINTER(C.c_double), C.POINTER(C.c_int), vp], C.c_int),
        "vi_problem_kernel": ([H, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
        "vi_status_string": ([C.c_int], C.c_char_p),
        "vi_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def status_name(s: int) -> str:
    try:
        return lib().vi_status_string(s).decode()
    except Exception:  # pragma: no cover - only used while formatting an error
        return str(s)


def _check(status: int, where: str, allow=(VI_OK,)) -> int:
    if status not in allow:
        raise ViError(status, where, lib().vi_last_error().decode())
    return status


def _addr(x) -> Optional[int]:
    """Device/host address of a tensor, numpy array, integer or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _nbytes(x) -> Optional[int]:
    """Bytes a tensor or numpy array holds (None for raw addresses, which cannot be checked)."""
    if hasattr(x, "element_size") and hasattr(x, "numel"):
        return x.element_size() * x.numel()
    if isinstance(x, np.ndarray):
        return x.nbytes
    return None


def _check_sizes(h: int, where: str, values=(), policies=()) -> None:
    """The C ABI takes plain pointers: refuse a value buffer smaller than |S| values of
    the handle's layout, or a policy buffer smaller than |S| bytes, before any kernel
    writes past it."""
    n = C.c_uint64()
    vb = C.c_int()
    _check(lib().vi_problem_sizes(h, C.byref(n), None, None, C.byref(vb)), "vi_problem_sizes")
    for x in values:
        nb = _nbytes(x) if x is not None else None
        if nb is not None and nb < n.value * vb.value:
            raise ValueError(f"{where}: value buffer of {nb} bytes, the problem needs {n.value} x {vb.value}")
    for x in policies:
        nb = _nbytes(x) if x is not None else None
        if nb is not None and nb < n.value:
            raise ValueError(f"{where}: policy buffer of {nb} bytes, the problem needs {n.value}")


def _need(x, nbytes: int, where: str, what: str) -> None:
    """Refuse a buffer that holds fewer than `nbytes` (raw addresses are not checked)."""
    nb = _nbytes(x) if x is not None else None
    if nb is not None and nb < nbytes:
        raise ValueError(f"{where}: {what} buffer of {nb} bytes, the call needs {nbytes}")


def _stream(s) -> Optional[int]:
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---------------------------------------------------------------------------
# thin wrappers, same names as the C ABI
# ---------------------------------------------------------------------------

def vi_problem_create(m: int, L: int, Q: int, cost: Sequence[float], pmf: np.ndarray, gamma: float,
                      issuing: int) -> int:
    c = np.ascontiguousarray(cost, np.float64)
    p = np.ascontiguousarray(pmf, np.float64)
    h = C.c_void_p()
    _check(lib().vi_problem_create(m, L, Q, c.ctypes.data_as(C.POINTER(C.c_double)),
                                   p.ctypes.data_as(C.POINTER(C.c_double)), len(p) - 1, gamma, issuing,
                                   C.byref(h)), "vi_problem_create")
    return h.value


def make_desc(products: Sequence[dict], gamma: float, issuing: int = VI_FIFO, precision: int = VI_PREC_FP32,
              stop_rule: int = VI_STOP_SPAN, subst_rate: float = 0.0):
    """products: dicts with m, L, Q, cost (5), pmf (array).  Returns (desc, keepalive)."""
    d = vi_problem_desc()
    d.n_products = len(products)
    keep = []
    for k, p in enumerate(products):
        d.m[k], d.L[k], d.Q[k] = int(p["m"]), int(p["L"]), int(p["Q"])
        for j in range(5):
            d.cost[k][j] = float(p["cost"][j])
        arr = np.ascontiguousarray(p["pmf"], np.float64)
        keep.append(arr)
        d.pmf[k] = arr.ctypes.data_as(C.POINTER(C.c_double))
        d.dmax[k] = len(arr) - 1
    d.subst_rate = float(subst_rate)
    d.gamma = float(gamma)
    d.issuing = int(issuing)
    d.precision = int(precision)
    d.stop_rule = int(stop_rule)
    return d, keep


def make_periodic_desc(m: int, Q: int, pmf, c0, c1, cost, gamma: float, stop_rule: int = VI_STOP_PERIODIC):
    """Scenario C description: pmf 7 x (dmax+1) (row = weekday), c0 / c1 indexed by
    age class k (entries 2..m used), cost (C_f, C_h, C_s, C_w).  Returns (desc, keepalive)."""
    arr = np.ascontiguousarray(pmf, dtype=np.float64)
    d = vi_periodic_desc()
    d.m, d.Q, d.dmax = m, Q, arr.shape[1] - 1
    d.pmf = arr.ctypes.data_as(C.POINTER(C.c_double))
    for k in range(9):
        d.c0[k] = float(c0[k]) if k < len(c0) else 0.0
        d.c1[k] = float(c1[k]) if k < len(c1) else 0.0
    for j in range(4):
        d.cost[j] = float(cost[j])
    d.gamma = gamma
    d.stop_rule = stop_rule
    return d, arr


def vi_problem_create_periodic(desc: vi_periodic_desc) -> int:
    h = C.c_void_p()
    _check(lib().vi_problem_create_periodic(C.byref(desc), C.byref(h)), "vi_problem_create_periodic")
    return h.value


def vi_problem_create_desc(desc: vi_problem_desc) -> int:
    h = C.c_void_p()
    _check(lib().vi_problem_create_desc(C.byref(desc), C.byref(h)), "vi_problem_create_desc")
    return h.value


def vi_problem_destroy(h: int) -> None:
    _check(lib().vi_problem_destroy(h), "vi_problem_destroy")


def vi_release_cached_memory() -> int:
    """Free the device / pinned blocks and streams cached from destroyed handles; bytes freed."""
    n = C.c_size_t()
    _check(lib().vi_release_cached_memory(C.byref(n)), "vi_release_cached_memory")
    return n.value


def vi_cached_memory() -> int:
    """Bytes held in the library's cache of released blocks."""
    n = C.c_size_t()
    _check(lib().vi_cached_memory(C.byref(n)), "vi_cached_memory")
    return n.value


def vi_problem_sizes(h: int) -> dict:
    n = C.c_uint64()
    a, o, vb = C.c_int(), C.c_int(), C.c_int()
    _check(lib().vi_problem_sizes(h, C.byref(n), C.byref(a), C.byref(o), C.byref(vb)), "vi_problem_sizes")
    return dict(n_states=n.value, n_actions=a.value, n_outcomes=o.value, value_bytes=vb.value)


def vi_problem_set_option(h: int, option: int, value: int) -> None:
    _check(lib().vi_problem_set_option(h, option, value), "vi_problem_set_option")


def vi_solve(h: int, tol: float, max_iters: int, V, policy=None, stream=None, flags: int = 0,
             offset: float = 0.0) -> dict:
    _check_sizes(h, "vi_solve", (V,), (policy,))
    info = vi_solve_info()
    info.offset = offset
    st = lib().vi_solve(h, tol, max_iters, _addr(V), _addr(policy), _stream(stream), flags, C.byref(info))
    _check(st, "vi_solve", allow=(VI_OK, VI_ENOTCONVERGED))
    return info.as_dict()


def vi_solve_host(h: int, tol: float, max_iters: int, V_host: np.ndarray, policy_host: Optional[np.ndarray],
                  flags: int = 0, offset: float = 0.0) -> dict:
    _check_sizes(h, "vi_solve_host", (V_host,), (policy_host,))
    info = vi_solve_info()
    info.offset = offset
    st = lib().vi_solve_host(h, tol, max_iters, _addr(V_host), _addr(policy_host), flags, C.byref(info))
    _check(st, "vi_solve_host", allow=(VI_OK, VI_ENOTCONVERGED))
    return info.as_dict()


def vi_backup(h: int, V_in, V_out, policy=None, stream=None, stats: bool = True):
    _check_sizes(h, "vi_backup", (V_in, V_out), (policy,))
    ds = (C.c_double * 2)()
    _check(lib().vi_backup(h, _addr(V_in), _addr(V_out), _addr(policy), _stream(stream),
                           ds if stats else None), "vi_backup")
    return (ds[0], ds[1]) if stats else None


def _noalloc_buffer(x, nbytes: int, what: str, dtypes) -> None:
    """The allocation-free sweep has no handle to check sizes against: refuse a buffer
    that is not a contiguous CUDA tensor of a listed dtype holding nbytes."""
    if x is None:
        return
    if hasattr(x, "is_cuda"):
        if not x.is_cuda or not x.is_contiguous() or str(x.dtype) not in dtypes:
            raise ViError(VI_EINVAL, "vi_backup_noalloc", f"{what} must be a contiguous CUDA tensor of {dtypes}")
    nb = _nbytes(x)
    if nb is not None and nb < nbytes:
        raise ViError(VI_EINVAL, "vi_backup_noalloc", f"{what} buffer of {nb} bytes, the instance needs {nbytes}")


def vi_backup_noalloc(m: int, L: int, Q: int, cost: Sequence[float], pmf: np.ndarray, gamma: float, issuing: int,
                      V_in, V_out, policy=None, stream=None, stats: bool = True):
    """One sweep without any allocation (see vi.h); V_in / V_out in the float-pair layout."""
    if len(cost) != 5:
        raise ViError(VI_EINVAL, "vi_backup_noalloc", "cost needs 5 entries (c_o, c_h, c_s, c_w, c_r)")
    n_states = (Q + 1) ** ((m - 1) + (L - 1)) if m >= 1 and L >= 1 and Q >= 0 else 0
    _noalloc_buffer(V_in, 8 * n_states, "V_in", ("torch.float32", "torch.float64"))
    _noalloc_buffer(V_out, 8 * n_states, "V_out", ("torch.float32", "torch.float64"))
    _noalloc_buffer(policy, n_states, "policy", ("torch.uint8",))
    c = np.ascontiguousarray(cost, np.float64)
    p = np.ascontiguousarray(pmf, np.float64)
    ds = (C.c_double * 2)()
    _check(lib().vi_backup_noalloc(m, L, Q, c.ctypes.data_as(C.POINTER(C.c_double)),
                                   p.ctypes.data_as(C.POINTER(C.c_double)), len(p) - 1, gamma, issuing,
                                   _addr(V_in), _addr(V_out), _addr(policy), ds if stats else None,
                                   _stream(stream)), "vi_backup_noalloc")
    return (ds[0], ds[1]) if stats else None


def vi_policy_eval(h: int, policy, V, tol: float, max_iters: int, stream=None):
    _check_sizes(h, "vi_policy_eval", (), (policy,))
    _need(V, 8 * vi_problem_sizes(h)["n_states"], "vi_policy_eval", "FP64 value")
    it, dl = C.c_int(), C.c_double()
    st = lib().vi_policy_eval(h, _addr(policy), _addr(V), tol, max_iters, _stream(stream), C.byref(it),
                              C.byref(dl))
    _check(st, "vi_policy_eval", allow=(VI_OK, VI_ENOTCONVERGED))
    return dict(iters=it.value, delta=dl.value, converged=(st == VI_OK))


def vi_next_states(h: int, states, n: int, out, stream=None) -> None:
    _need(states, 4 * n, "vi_next_states", "state")
    _need(out, 4 * n, "vi_next_states", "output")
    _check(lib().vi_next_states(h, _addr(states), n, _addr(out), _stream(stream)), "vi_next_states")


def _check_rollout_bufs(h, where, policy, n, horizon, returns, kpis, kpis_prod, traj) -> None:
    _check_sizes(h, where, (), (policy,))
    _need(returns, 8 * n, where, "returns")
    _need(kpis, 24 * n, where, "KPI")
    _need(kpis_prod, 48 * n, where, "per-product KPI")
    _need(traj, 4 * n * horizon, where, "trajectory")


def vi_simulate(h: int, policy, n_rollouts: int, horizon: int, warmup: int, seed: int, returns, kpis=None,
                traj=None, stream=None) -> None:
    _check_rollout_bufs(h, "vi_simulate", policy, n_rollouts, horizon, returns, kpis, None, traj)
    _check(lib().vi_simulate(h, _addr(policy), n_rollouts, horizon, warmup, C.c_uint64(seed), _addr(returns),
                             _addr(kpis), _addr(traj), _stream(stream)), "vi_simulate")


def vi_simulate_ex(h: int, policy, n_rollouts: int, horizon: int, warmup: int, seed: int, returns, kpis=None,
                   kpis_prod=None, traj=None, stream=None) -> None:
    _check_rollout_bufs(h, "vi_simulate_ex", policy, n_rollouts, horizon, returns, kpis, kpis_prod, traj)
    _check(lib().vi_simulate_ex(h, _addr(policy), n_rollouts, horizon, warmup, C.c_uint64(seed), _addr(returns),
                                _addr(kpis), _addr(kpis_prod), _addr(traj), _stream(stream)), "vi_simulate_ex")


def vi_mbs_search(h: int, S_lo, S_hi, mu, cap: bool, n_rollouts: int, horizon: int, warmup: int, seed: int,
                  returns, kpis_prod=None, stream=None, means: bool = True):
    """Modified base-stock search over the (S_1, S_2) grid: per-pair mean returns
    (row-major, product 1 outer) and the best pair; per-rollout returns (and
    per-product KPIs if given) land in the device buffers.  means=False only
    launches (no synchronisation) and returns None."""
    lo = (C.c_int * 2)(*(list(S_lo) + [0] * (2 - len(S_lo))))
    hi = (C.c_int * 2)(*(list(S_hi) + [0] * (2 - len(S_hi))))
    mv = (C.c_int * 2)(*(list(mu) + [0] * (2 - len(mu))))
    n_pairs = (hi[0] - lo[0] + 1) * ((hi[1] - lo[1] + 1) if len(S_lo) == 2 else 1)
    _need(returns, 8 * max(n_pairs, 0) * n_rollouts, "vi_mbs_search", "returns")
    _need(kpis_prod, 48 * max(n_pairs, 0) * n_rollouts, "vi_mbs_search", "per-product KPI")
    if not means:
        _check(lib().vi_mbs_search(h, lo, hi, mv, int(bool(cap)), n_rollouts, horizon, warmup, C.c_uint64(seed),
                                   _addr(returns), _addr(kpis_prod), None, None, _stream(stream)), "vi_mbs_search")
        return None
    mr = (C.c_double * n_pairs)()
    best = (C.c_int * 2)()
    _check(lib().vi_mbs_search(h, lo, hi, mv, int(bool(cap)), n_rollouts, horizon, warmup, C.c_uint64(seed),
                               _addr(returns), _addr(kpis_prod), mr, best, _stream(stream)), "vi_mbs_search")
    return np.array(list(mr)), (best[0], best[1])


def vi_problem_kernel(h: int) -> tuple:
    """(kernel, lane width) of the sweep the handle runs; resolves the choice if needed."""
    k, w = C.c_int(), C.c_int()
    _check(lib().vi_problem_kernel(h, C.byref(k), C.byref(w)), "vi_problem_kernel")
    return k.value, w.value


def vi_basestock_search(h: int, s_lo: int, s_hi: int, n_rollouts: int, horizon: int, warmup: int, seed: int,
                        returns, stream=None):
    """Mean return per order-up-to level S in s_lo..s_hi and the best S; per-rollout
    returns land in the device buffer `returns` (row S - s_lo)."""
    n_S = s_hi - s_lo + 1
    _need(returns, 8 * max(n_S, 0) * n_rollouts, "vi_basestock_search", "returns")
    means = (C.c_double * n_S)()
    best = C.c_int()
    _check(lib().vi_basestock_search(h, s_lo, s_hi, n_rollouts, horizon, warmup, C.c_uint64(seed), _addr(returns),
                                     means, C.byref(best), _stream(stream)), "vi_basestock_search")
    return np.array(list(means)), best.value


def vi_probe_l2_read(buf, nbytes: int, reps: int, stream=None) -> float:
    """Duration in ms of `reps` L1-bypassing reads of an L2-resident device buffer."""
    ms = C.c_float()
    _check(lib().vi_probe_l2_read(_addr(buf), nbytes, reps, _stream(stream), C.byref(ms)), "vi_probe_l2_read")
    return ms.value


def vi_server_create(mem_budget_bytes: int, max_slots: int, stream=None) -> int:
    srv = C.c_void_p()
    _check(lib().vi_server_create(mem_budget_bytes, max_slots, _stream(stream), C.byref(srv)), "vi_server_create")
    return srv.value


def vi_server_submit(srv: int, desc: vi_problem_desc, tol: float, max_iters: int) -> int:
    rid = C.c_uint64()
    _check(lib().vi_server_submit(srv, C.byref(desc), tol, max_iters, C.byref(rid)), "vi_server_submit")
    return rid.value


def vi_server_poll(srv: int, request_id: int, V_host: Optional[np.ndarray] = None,
                   policy_host: Optional[np.ndarray] = None):
    """Returns (done, info); info["status"] is the request's status once done."""
    done = C.c_int()
    info = vi_solve_info()
    st = lib().vi_server_poll(srv, request_id, C.byref(done), _addr(V_host), _addr(policy_host), C.byref(info))
    if st not in (VI_OK, VI_ENOTCONVERGED, VI_ECANCELLED) or (not done.value and st != VI_OK):
        _check(st, "vi_server_poll")
    return bool(done.value), info.as_dict()


def vi_server_submit_to(srv: int, desc, tol: float, max_iters: int, V_host: np.ndarray,
                        policy_host: np.ndarray) -> int:
    """Submit with the result delivered into V_host / policy_host (keep them alive until done)."""
    rid = C.c_uint64()
    _check(lib().vi_server_submit_to(srv, C.byref(desc), tol, max_iters, _addr(V_host), _addr(policy_host),
                                     C.byref(rid)), "vi_server_submit_to")
    return rid.value


def vi_server_wait(srv: int, timeout_ms: int = 0, max_ids: int = 1024) -> list:
    """Ids of requests that finished since the last call (waits up to timeout_ms for one)."""
    buf = (C.c_uint64 * max_ids)()
    n = C.c_int()
    _check(lib().vi_server_wait(srv, timeout_ms, C.cast(buf, C.c_void_p), max_ids, C.byref(n)), "vi_server_wait")
    return list(buf[:n.value])


def vi_server_destroy(srv: int) -> None:
    _check(lib().vi_server_destroy(srv), "vi_server_destroy")
