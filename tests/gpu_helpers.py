"""Helpers shared by the GPU parity tests: marshal workloads.Instance into the
C ABI and run solves / backups through it."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2303_10672_b300 as vi

PREC = {"fp32": vi.VI_PREC_FP32, "fp32_kahan": vi.VI_PREC_FP32_KAHAN, "fp64": vi.VI_PREC_FP64,
        "fp32_single": vi.VI_PREC_FP32_SINGLE}
# storage layout of each precision: float pair, double, or single float + FP64 offset
LAYOUT = {"fp32": "pair", "fp32_kahan": "pair", "fp64": "double", "fp32_single": "single"}


def values_abs(V: torch.Tensor, offset: float, layout: str) -> np.ndarray:
    """Absolute values V_abs(s) in FP64 from a device value buffer."""
    if layout == "pair":
        p = V.view(torch.float32).reshape(-1, 2).double()
        return (p[:, 0] + p[:, 1]).cpu().numpy()
    if layout == "double":
        return V.view(torch.float64).cpu().numpy()
    return V.view(torch.float32).double().cpu().numpy() + offset

# tolerances stated by the benchmark spec: values max|dV|/max|V| <= 1e-5; policy ties within 1e-6 relative
V_RTOL = 1e-5
TIE_RTOL = 1e-6


def create(inst, precision=None, stop_rule=vi.VI_STOP_SPAN, kernel=vi.VI_KERNEL_AUTO):
    prods = [dict(m=p.m, L=p.L, Q=p.Q, cost=p.cost, pmf=p.pmf) for p in inst.products]
    prec = PREC[precision or inst.precision]
    desc, keep = vi.make_desc(prods, inst.gamma, inst.issuing, prec, stop_rule, inst.subst_rate)
    h = vi.vi_problem_create_desc(desc)
    if kernel != vi.VI_KERNEL_AUTO:
        vi.vi_problem_set_option(h, vi.VI_OPT_KERNEL, kernel)
    return h


class Handle:
    def __init__(self, inst, precision=None, stop_rule=vi.VI_STOP_SPAN, kernel=vi.VI_KERNEL_AUTO):
        self.inst = inst
        self.precision = precision or inst.precision
        self.h = create(inst, self.precision, stop_rule, kernel)
        self.sizes = vi.vi_problem_sizes(self.h)
        self.layout = LAYOUT[self.precision]
        # one 8-byte element per state holds a float pair or a double
        self.dtype = torch.float64 if self.sizes["value_bytes"] == 8 else torch.float32

    def close(self):
        if self.h:
            vi.vi_problem_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, tol, max_iters, flags=0, V=None, offset=0.0):
        n = self.sizes["n_states"]
        if V is None:
            V = torch.empty(n, dtype=self.dtype, device="cuda")
        pol = torch.empty(n, dtype=torch.uint8, device="cuda")
        info = vi.vi_solve(self.h, tol, max_iters, V, pol, flags=flags, offset=offset)
        torch.cuda.synchronize()
        return V, pol, info

    def v_abs(self, V, info) -> np.ndarray:
        return values_abs(V, info["offset"], self.layout)


def compare_values(v_gpu: np.ndarray, v_ref: np.ndarray) -> float:
    scale = max(np.abs(v_ref).max(), 1e-300)
    return float(np.abs(v_gpu - v_ref).max() / scale)


def policy_mismatches(P_oracle, V_ref: np.ndarray, pol_gpu: np.ndarray, states=None):
    """States where the GPU policy differs from the oracle's first argmax by more
    than a tie: Q(s, a_oracle) - Q(s, a_gpu) > TIE_RTOL |Q(s, a_oracle)| (FP64)."""
    if states is None:
        states = np.arange(len(pol_gpu))
    _, pol_o, q = P_oracle.backup_states(V_ref, states, with_q=True)
    bad = []
    for i, s in enumerate(states):
        ag = int(pol_gpu[i])
        ao = int(pol_o[i])
        if ag == ao:
            continue
        gap = q[i, ao] - q[i, ag]
        if gap > TIE_RTOL * abs(q[i, ao]):
            bad.append((int(s), ao, ag, float(gap)))
    return bad


# full solves vs the oracle at the oracle's stopping iteration
def solve_parity(inst, precision, kernel=vi.VI_KERNEL_AUTO, tol=1e-4, stop_rule=0):
    P = oracle.Problem(inst)
    ref = P.vi_solve(tol=tol, max_iters=5000, stop_rule=stop_rule)
    i_o = ref["iters"]
    with Handle(inst, precision=precision, stop_rule=stop_rule, kernel=kernel) as H:
        # same iteration count as the oracle, stop test disabled (tol = 0)
        V, pol, info = H.solve(0.0, i_o)
        assert info["iters"] == i_o
        v = H.v_abs(V, info)
        err = compare_values(v, ref["V"])
        assert err <= V_RTOL, f"value error {err:.3e}"
        bad = policy_mismatches(P, ref["V"], pol.cpu().numpy())
        assert not bad, bad[:5]
        # the device stopping test: same rule, own iteration count
        V2, pol2, info2 = H.solve(tol, 5000)
        assert info2["status"] == vi.VI_OK
        assert abs(info2["iters"] - i_o) <= 2, (info2["iters"], i_o)
    return err


# full-size instances: one backup in the benchmark's launch configuration, compared on
# sampled states computed one by one by the oracle
def sampled_backup_parity(inst, k_sweeps, n_samples, seed, precision="fp32", kernel=vi.VI_KERNEL_AUTO):
    P = oracle.Problem(inst)
    with Handle(inst, precision=precision, kernel=kernel) as H:
        V, pol, info = H.solve(0.0, k_sweeps)           # V_k (+ offset for the single layout)
        n = H.sizes["n_states"]
        V_next = torch.empty_like(V)
        pol_next = torch.empty(n, dtype=torch.uint8, device="cuda")
        dmx, dmn = vi.vi_backup(H.h, V, V_next, pol_next)
        torch.cuda.synchronize()
        b = info["offset"]
        v_k = H.v_abs(V, info)
        # single layout: V_next holds V_abs' - gamma b; pair / double: absolute
        v_next = values_abs(V_next, inst.gamma * b, H.layout)
        rng = np.random.default_rng(seed)
        states = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, n_samples)]))
        want, _ = P.backup_states(v_k, states)
        err = np.abs(v_next[states] - want).max() / np.abs(want).max()
        assert err <= V_RTOL, err
        bad = policy_mismatches(P, v_k, pol_next.cpu().numpy()[states], states)
        assert not bad, bad[:5]
        # the policy written by the extraction sweep of the solve is the argmax from V_k
        bad = policy_mismatches(P, v_k, pol.cpu().numpy()[states], states)
        assert not bad, bad[:5]
        # change statistics: max / min of V_next - V_k in the kernel's own value units
        dv = values_abs(V_next, 0.0, H.layout) - values_abs(V, 0.0, H.layout)
        scale = max(1.0, np.abs(v_k).max())
        assert abs(dmx - dv.max()) <= 1e-6 * scale and abs(dmn - dv.min()) <= 1e-6 * scale
