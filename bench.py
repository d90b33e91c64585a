"""Benchmark of the value-iteration hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload cfg4|cfg2|cfg1|cfg3] [--impl reference]

A step is one complete solve of the workload through the C ABI: synchronous
FP32 Bellman sweeps (decode, FIFO/LIFO issue, gathers, max/argmax, FP64 span
reduction and device-side stopping test inside a CUDA-graph while loop) until
the span of V_i - V_{i-1} is below 1e-4, then the extraction sweep writing the
policy.  The metric is nominal Bellman state-action-demand updates per second:
|S| |A| |Omega| x sweeps / solve time.  Default workload: the largest
single-product configuration, m=8, L=1, Q=10 (11^7 = 19,487,171 states), 11
orders, Poisson(4) demand folded at 15, LIFO issuing, costs (3, 1, 5, 7),
gamma 0.95; the 4,084,101-state FIFO configuration (m=5, L=2, Q=20) is
reported beside it under "cfg2".

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (one Bellman update of a sample of states per
step) and reports the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "bellman_state_action_demand_updates_per_s"
UNIT = "updates/s"
WORKLOADS = {
    "cfg1": workloads.config1,
    "cfg2": workloads.config2,
    "cfg3": workloads.config3,
    "cfg4": workloads.config4,
    # the paper's Scenario B settings (for profiling the two-product pipeline sweep)
    "scenB_P4": lambda: workloads.scenario_b("P4"),
    "scenB_m3_exp1": lambda: workloads.scenario_b("m3_exp1"),
    "scenB_m3_exp3": lambda: workloads.scenario_b("m3_exp3"),
    # the paper's largest Scenario A setting (m = 5, L = 2, FIFO, C_w = 7)
    "scenA_m5L2": lambda: workloads.scenario_a(5, 2, 7.0, workloads.FIFO),
}
TOL = 1e-4
MAX_ITERS = 5_000
DTYPES = {"fp32": "f32 (float-pair values)", "fp32_kahan": "f32 (float-pair values, Kahan sums)", "fp64": "f64",
          "fp32_single": "f32 (single values, FP64 offset)"}
L2_BYTES = 126 * 1024 * 1024


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return dict(hbm_gbs=d["hbm_gbs"], sm_max_mhz=d.get("sm_max_mhz", 2032.0), source="measured")
    return dict(hbm_gbs=6400.0, sm_max_mhz=2032.0, source="fallback")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_ready(self, timeout_s: float = 5.0):
        """Wait for the first sample, so that the timed region is sampled from its start."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)
        self.lines.clear()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sms)) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


def dist_setup(n_gpus):
    import torch
    import torch.distributed as dist
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world, local


def barrier_sync(world):
    import torch
    import torch.distributed as dist
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Whole-job rate of N independent replicas: every rank does the same work,
    the job takes as long as the slowest rank."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------------------
# the oracle on host cores (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_sample_rate(inst, seconds_target: float, seed: int = 0):
    """Updates/s of the FP64 oracle: one Bellman update of a random sample of states
    (OpenMP over all host cores), sized to take about `seconds_target`."""
    import oracle
    P = oracle.Problem(inst)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    V = rng.uniform(-100.0, 0.0, inst.n_states) if inst.n_states <= 50_000_000 else None
    per_state = inst.n_actions * inst.n_outcomes
    n = 64
    while True:
        states = rng.integers(0, inst.n_states, n)
        t0 = time.perf_counter()
        P.backup_states(V, states, nthreads=cores)
        dt = time.perf_counter() - t0
        if dt >= seconds_target or n >= inst.n_states:
            break
        n = int(min(inst.n_states, max(n * 2, n * seconds_target / max(dt, 1e-6) * 1.1)))
    return dict(value=n * per_state / dt, unit=UNIT, cores=cores, kind="oracle",
                sample=f"one FP64 Bellman update of {n} random states of {inst.name} "
                       f"({n * per_state:.3g} nominal updates, {dt:.1f} s, {cores} OpenMP threads)",
                seconds=dt)


def workload_config(inst, l2: str, parallelism: str) -> dict:
    """The workload both arms report: the instance, its sizes and the stopping test,
    then how the arm ran it."""
    return {"workload": inst.name, "states": inst.n_states, "actions": inst.n_actions,
            "outcomes": inst.n_outcomes, "tol": TOL, "stop_rule": "span", "l2": l2, "parallelism": parallelism}


def run_reference(args):
    import torch  # noqa: F401  (rank/world plumbing only)
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    inst = WORKLOADS[args.workload]()
    vals, secs = [], []
    per_step = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        r = oracle_sample_rate(inst, per_step, seed=i)
        if i >= args.warmup:
            vals.append(r["value"])
            secs.append(r["seconds"])
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(inst, "not applicable (host cores)", "host OpenMP"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def _rest_totals(p) -> np.ndarray:
    """Units held by each rest r (digits 1.. of a product state) in the slots the
    demand can reach: n_rest_slots = m - 2 (L = 1) or m - 1 (L >= 2) digits."""
    G, K = p.Q + 1, p.n_digits
    nslots = (p.m - 2) if p.L == 1 else (p.m - 1)
    r = np.arange(G ** (K - 1), dtype=np.int64)
    tot = np.zeros_like(r)
    for _ in range(max(nslots, 0)):
        tot += r % G
        r //= G
    return tot


def two_product_fmas(inst) -> int:
    """Multiply-adds one sweep of the factorised two-product method performs (the
    products are not expanded over the joint (d1, d2, u) outcomes): the product-2
    expectation table E2, the substitution-mixture table and the sweep's sum over
    d1 below product 1's stock, counted per (state, order) as the kernels loop."""
    p1, p2 = inst.products
    G1, G2 = p1.Q + 1, p2.Q + 1
    S1, S2 = p1.n_states, p2.n_states
    D1 = p1.dmax
    R1, R2 = _rest_totals(p1), _rest_totals(p2)
    nt = min(D1, p1.m * p1.Q) + 1
    if p1.L >= 2 and p2.L >= 2:
        e1 = np.minimum(np.maximum(R1 - 1, 0), D1) + 1          # terms per order of a rest of product 1
        sweep = int(S2) * G1 * G2 * G1 * int(e1.sum())
        terms2 = int((R2 + 1).sum()) * G2                         # per (i1 or mixture row, a2), all x2
        npipe1 = G1 ** (p1.L - 1)
        return sweep + S1 * G2 * terms2 + npipe1 * nt * G2 * terms2
    # lead time 1: the order joins product 1's rest; d1 runs below T1 = x + R1 + a1
    x = np.arange(G1)[:, None, None]
    a = np.arange(G1)[None, None, :]
    T1 = x + R1[None, :, None] + a
    sweep = int(np.minimum(T1, D1 + 1).sum()) * G2 * S2
    a2 = np.arange(G2)[None, :]
    terms2 = int((R2[:, None] + a2 + 1).sum()) * G2               # per (i1 or mixture row), all (s2, a2)
    return sweep + S1 * terms2 + nt * terms2


def solve_launches(iters, no_graph: bool, max_iters: int, per_sweep: int) -> int:
    """Kernel launches of the timed solves: per solve the init kernel, the sweeps
    (the graph's loop body holds four, the host loop launches four between status
    reads; a sweep after the stop returns at once but is launched) with their
    pre-kernels, and the extraction sweep."""
    group = 4
    total = 0
    for it in iters:
        sweeps = -(-it // group) * group if it > 0 else 0
        if no_graph:
            sweeps = min(sweeps, max_iters)   # the host loop stops launching at max_iters
        total += 1 + (sweeps + 1) * per_sweep
    return int(total)


def algorithmic_work(inst) -> dict:
    """Algorithmic work of one Bellman sweep and the compulsory HBM bytes (old and
    new value of every state, 8 B float pair each).  One product: the method's one
    multiply-add of p(d) and the next-state value per (state, order, demand
    outcome); the factorised FIFO sweep performs exactly these, the LIFO sweeps
    fewer (the next states of a rest do not depend on its expiring units).  Two
    products: the multiply-adds of the factorised method (two_product_fmas);
    `updates` stays the nominal |S| |A| |Omega|."""
    updates = inst.updates_per_sweep
    if len(inst.products) == 2:
        fmas = two_product_fmas(inst)
        return {"updates": updates, "flops": 2 * fmas, "bytes": inst.n_states * 16,
                "work": "2 flop per multiply-add of the factorised two-product method (E2 table, "
                        "substitution mixture, sum over d1 below stock)"}
    return {"updates": updates, "flops": 2 * updates, "bytes": inst.n_states * 16,
            "work": "2 flop (one multiply-add) per state x order x demand outcome, the method's arithmetic"}


def lifo1_executed_fmas(inst, n_sm: int = 148) -> int:
    """Multiply-adds the lead-time-one LIFO sweep executes per launch.  Per rest, the part
    on the partly used order, a terms for order a (G (G - 1) / 2); the part on the used-up
    sequence, sum_{a < DP-1} (DP - 1 - a) at a rest computed afresh and DP - 1 (one step of
    the recurrence per entry) at a further rest of a column.  Columns are the G rests that
    differ in X_{m-1}; each of the kernel's warps (4 per block, one wave of resident blocks:
    4 per SM with a 16-slot pmf, 2 with 32) walks floor(column tiles / warps) whole columns,
    and the leftover columns' rests are computed afresh."""
    p = inst.products[0]
    G = p.Q + 1
    DP = 16 if p.dmax < 16 else 32
    nrs = p.m - 2
    n_rests = p.n_states // G
    col = G if nrs >= 2 else 1
    nbase = n_rests // col
    tiles = (nbase + 31) // 32
    warps = min((n_rests + 127) // 128, n_sm * (4 if DP == 16 else 2)) * 4
    whole = (tiles // warps) * warps                      # column tiles walked whole
    whole_rests = min(whole * 32, nbase) * col
    fresh = min(whole * 32, nbase) + (n_rests - whole_rests)
    per_fresh = (DP - 1) * DP // 2
    return n_rests * G * (G - 1) // 2 + fresh * per_fresh + (n_rests - fresh) * (DP - 1)


def fifo_col_executed_fmas(inst) -> int:
    """Multiply-adds of the expectations in the FIFO column sweep per launch: per column
    of Q+1 rests and per order, dmax (dmax + 1) / 2 for the first rest's sum over the
    demand (x' + k <= dmax) and, for each further rest z = 1..Q, one per x' still needed
    (x' < min(dmax, 2Q - z + 1))."""
    p = inst.products[0]
    G = p.Q + 1
    cols = p.n_states // (G * G)
    per_order = p.dmax * (p.dmax + 1) // 2 + sum(min(p.dmax, 2 * p.Q - z + 1) for z in range(1, G))
    return cols * G * per_order


# DRAM bytes (read + write) of one launch of the dominant kernel, from the ncu captures
# summarised in profiles/; an entry is dropped when that kernel changes
NCU_TRAFFIC = {
    ("cfg2_m5L2Q20_nb_fifo", "sweep_group_kernel (lane width 21)"): 34_362_112,
    ("cfg4_m8L1Q10_lifo", "sweep_lifo1_kernel"): 236_745_984 + 114_699_264,
    ("cfg2_m5L2Q20_nb_fifo", "sweep_fifo_col_kernel"): 32_748_288 + 749_568,
}
# thread instructions of one launch of the dominant kernel (warp instructions x active
# threads per warp instruction), from the same captures
NCU_THREAD_INSTR = {
    ("cfg2_m5L2Q20_nb_fifo", "sweep_group_kernel (lane width 21)"): 187_319_919 * 29.41,
    ("cfg4_m8L1Q10_lifo", "sweep_lifo1_kernel"): 63_584_026 * 31.62,
    ("cfg2_m5L2Q20_nb_fifo", "sweep_fifo_col_kernel"): 96_298_900 * 27.59,
}


def l2_read_peak_gbs(vi, torch) -> float:
    """Best of three L1-bypassing streaming reads of a 32 MiB L2-resident buffer."""
    nbytes = 32 << 20
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
    reps = 64
    best = min(vi.vi_probe_l2_read(buf, nbytes, reps) for _ in range(3))
    return nbytes * reps / (best * 1e-3) / 1e9


def kernel_name_of(vi, inst, kch, kw) -> str:
    if len(inst.products) == 2 and kch == vi.VI_KERNEL_GROUP:
        return ("twop_e2_kernel + twop_mix_kernel + twop_sweep_kernel" if inst.products[0].L >= 2
                else "two_e2_kernel + two_mix_kernel + sweep_two_kernel")
    return {vi.VI_KERNEL_GENERIC: "sweep_generic_kernel", vi.VI_KERNEL_TENSOR: "sweep_tc_kernel",
            vi.VI_KERNEL_LIFO_L1: "sweep_lifo1_kernel",
            vi.VI_KERNEL_FIFO_COL: "sweep_fifo_col_kernel"}.get(kch, f"sweep_group_kernel (lane width {kw})")


def time_sweep_kernel(vi, torch, h, V, stream, flush, reps: int = 20, rounds: int = 5) -> float:
    """Duration of the dominant kernel: the median over `rounds` of the average of `reps`
    back-to-back single sweeps (vi_backup, the same kernel and grid as the solve) between
    CUDA events on the launching stream, L2 flushed before each round."""
    V2 = torch.empty_like(V)
    vi.vi_backup(h, V, V2, None, stream=stream, stats=False)
    avg = []
    for _ in range(rounds):
        flush.fill_(1.0)
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for i in range(reps):
            if i % 2 == 0:
                vi.vi_backup(h, V, V2, None, stream=stream, stats=False)
            else:
                vi.vi_backup(h, V2, V, None, stream=stream, stats=False)
        k1.record(stream)
        k1.synchronize()
        avg.append(k0.elapsed_time(k1) / reps)
    return float(np.median(avg))


def roofline_of(vi, torch, inst, kernel_name: str, k_ms: float, sm_mhz: float, l2_gbs) -> dict:
    """FP32 ALU roofline of the dominant kernel: the method's multiply-adds per launch
    against SMs x 128 FP32 lanes x 2 flop x the median SM clock sampled in the run,
    with the HBM fraction of the compulsory traffic and the gather ratio beside it."""
    work = algorithmic_work(inst)
    pk = peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = work["flops"] / (k_ms * 1e-3) / 1e12
    hbm_gbs = work["bytes"] / (k_ms * 1e-3) / 1e9
    traffic = NCU_TRAFFIC.get((inst.name, kernel_name))
    out = {
        "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
        "traffic": traffic, "kernel": kernel_name, "kernel_ms": k_ms, "work": work["work"],
        "peak_basis": f"{n_sm} SMs (device property) x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz "
                      f"(median SM clock sampled during the timed solves)",
        "hbm": {"compulsory_bytes": work["bytes"], "achieved_GBs": hbm_gbs, "peak_GBs": pk["hbm_gbs"],
                "frac": hbm_gbs / pk["hbm_gbs"], "peak_source": pk["source"],
                "basis": "16 B per state per sweep: the previous value read and the new one written "
                         "(float pairs)",
                "measured_dram_GBs": None if traffic is None else traffic / (k_ms * 1e-3) / 1e9},
    }
    ti = NCU_THREAD_INSTR.get((inst.name, kernel_name))
    if ti is not None:
        # the issue ceiling: every SM issues at most 128 thread instructions per clock
        per_update = ti / work["updates"]
        ceiling = n_sm * 128 * sm_mhz * 1e6 / per_update
        rate = work["updates"] / (k_ms * 1e-3)
        out["issue"] = {"thread_instructions_per_update": per_update, "ceiling_updates_per_s": ceiling,
                        "achieved_updates_per_s": rate, "frac": rate / ceiling}
    if kernel_name in ("sweep_lifo1_kernel", "sweep_fifo_col_kernel"):
        fm = (lifo1_executed_fmas(inst, n_sm) if kernel_name == "sweep_lifo1_kernel"
              else fifo_col_executed_fmas(inst))
        out["executed_fmas_per_launch"] = fm
        out["executed_fp32_frac"] = 2 * fm / (k_ms * 1e-3) / 1e12 / fp32_peak
    if len(inst.products) == 1 and l2_gbs:
        g = work["updates"] * 4 / (k_ms * 1e-3) / 1e9
        out["gather"] = {"logical_GBs": g, "l2_read_peak_GBs": l2_gbs, "ratio": g / l2_gbs,
                         "note": "not a bound: the factorised sweeps gather each next-state value once per "
                                 "rest and order (FIFO) or once per rest (LIFO), not once per update"}
    return out


def solve_summary(vi, torch, inst, args, stream, flush, steps: int, warmup: int) -> dict:
    """A secondary workload: timed solves (L2 flushed between them) and its dominant
    kernel, with the same metric and roofline as the headline."""
    prods = [dict(m=q.m, L=q.L, Q=q.Q, cost=q.cost, pmf=q.pmf) for q in inst.products]
    desc, keep = vi.make_desc(prods, inst.gamma, inst.issuing, vi.VI_PREC_FP32, vi.VI_STOP_SPAN, inst.subst_rate)
    h = vi.vi_problem_create_desc(desc)
    try:
        sizes = vi.vi_problem_sizes(h)
        n = sizes["n_states"]
        V = torch.empty(n, dtype=torch.float64, device="cuda")
        pol = torch.empty(n, dtype=torch.uint8, device="cuda")
        nominal = float(n) * sizes["n_actions"] * sizes["n_outcomes"]
        for _ in range(warmup):
            vi.vi_solve(h, TOL, args.max_iters, V, pol, stream=stream)
        ms, iters = [], []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = vi.vi_solve(h, TOL, args.max_iters, V, pol, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            iters.append(info["iters"])
        k_ms = time_sweep_kernel(vi, torch, h, V, stream, flush)
        kch, kw = vi.vi_problem_kernel(h)
        return {"workload": inst.name, "states": n, "value": nominal * sum(iters) / (sum(ms) * 1e-3),
                "unit": UNIT, "ms_per_solve": sum(ms) / len(ms), "sweeps_per_solve": iters[-1],
                "kernel": kernel_name_of(vi, inst, kch, kw), "kernel_ms": k_ms}
    finally:
        vi.vi_problem_destroy(h)


CFG3_ORACLE = os.path.join(ROOT, "tests", "golden", "cfg3_oracle_sample.json")


def run_cfg3_accuracy(vi, torch, stream) -> dict:
    """The two-product configuration (50,625 states) in FP32 with compensated sums,
    its error against the FP64 oracle reported per result: the GPU runs the oracle's
    sweep count (tol 0), and its values and first-argmax policy are compared with
    the oracle's stored solve at 2,004 sampled states; a second solve with the
    span test (tol 1e-4) gives the GPU's own stop sweep and, with
    VI_FLAG_POLICY_EVAL, the FP64 evaluation of its policy (pe_gap =
    max_s |V_pe(s) - V(s)|, and pe_span = max - min of V_pe - V, the gap up to the
    constant that a span-test stop leaves)."""
    with open(CFG3_ORACLE) as f:
        ref = json.load(f)
    inst = workloads.config3()
    prods = [dict(m=q.m, L=q.L, Q=q.Q, cost=q.cost, pmf=q.pmf) for q in inst.products]
    desc, keep = vi.make_desc(prods, inst.gamma, inst.issuing, vi.VI_PREC_FP32_KAHAN, vi.VI_STOP_SPAN,
                              inst.subst_rate)
    h = vi.vi_problem_create_desc(desc)
    try:
        n = vi.vi_problem_sizes(h)["n_states"]
        assert n == ref["n_states"]
        states = np.asarray(ref["states"], np.int64)
        V = torch.empty(n, dtype=torch.float64, device="cuda")
        pol = torch.empty(n, dtype=torch.uint8, device="cuda")
        # the oracle's sweep count, no early stop
        vi.vi_solve(h, 0.0, ref["iters"], V, pol, stream=stream)
        torch.cuda.synchronize()
        pair = V.view(torch.float32).reshape(-1, 2).double()
        v = (pair[:, 0] + pair[:, 1]).cpu().numpy()[states]
        want = np.asarray(ref["V"])
        err = float(np.abs(v - want).max() / np.abs(want).max())
        mism = int((pol.cpu().numpy()[states] != np.asarray(ref["policy"], np.uint8)).sum())
        # the GPU's own stopping test, then FP64 evaluation of its policy
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        own = vi.vi_solve(h, ref["tol"], MAX_ITERS, V, pol, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        pe = vi.vi_solve(h, ref["tol"], MAX_ITERS, V, pol, stream=stream, flags=vi.VI_FLAG_POLICY_EVAL)
        kch, kw = vi.vi_problem_kernel(h)
        return {"workload": inst.name, "states": n, "precision": "fp32_kahan",
                "kernel": kernel_name_of(vi, inst, kch, kw),
                "vs_oracle": {"sweeps": ref["iters"], "sampled_states": int(len(states)),
                              "max_abs_dV_over_max_abs_V": err,
                              "policy_differences": mism, "policy_note": "exact compare, ties not separated"},
                "own_stop_sweep": own["iters"], "oracle_stop_sweep": ref["iters"], "ms_per_solve": ms,
                "pe_gap": pe["pe_gap"], "pe_span": pe["pe_span"],
                "pe_span_over_max_abs_V": pe["pe_span"] / ref["max_abs_V"], "pe_sweeps": pe["pe_iters"],
                "pe_note": "span-test solve: V is right up to a constant, so pe_span (max - min of V_pe - V) "
                           "is the error and pe_gap holds that constant"}
    finally:
        vi.vi_problem_destroy(h)


def run_native(args):
    import torch
    import paper_2303_10672_b300 as vi

    rank, world, local = dist_setup(args.gpus)
    inst = WORKLOADS[args.workload]()
    p = inst.products[0]
    prec = {"fp32": vi.VI_PREC_FP32, "fp32_kahan": vi.VI_PREC_FP32_KAHAN, "fp64": vi.VI_PREC_FP64,
            "fp32_single": vi.VI_PREC_FP32_SINGLE}[args.precision or inst.precision]
    prods = [dict(m=q.m, L=q.L, Q=q.Q, cost=q.cost, pmf=q.pmf) for q in inst.products]
    desc, keep = vi.make_desc(prods, inst.gamma, inst.issuing, prec, vi.VI_STOP_SPAN, inst.subst_rate)
    kernel = {"auto": vi.VI_KERNEL_AUTO, "group": vi.VI_KERNEL_GROUP, "tensor": vi.VI_KERNEL_TENSOR,
              "generic": vi.VI_KERNEL_GENERIC, "lifo1": vi.VI_KERNEL_LIFO_L1,
              "fifocol": vi.VI_KERNEL_FIFO_COL}[args.kernel]

    def configure(hh):
        if kernel != vi.VI_KERNEL_AUTO:
            vi.vi_problem_set_option(hh, vi.VI_OPT_KERNEL, kernel)
        if args.group_width:
            vi.vi_problem_set_option(hh, vi.VI_OPT_GROUP_WIDTH, args.group_width)

    h = vi.vi_problem_create_desc(desc)
    configure(h)
    sizes = vi.vi_problem_sizes(h)
    n = sizes["n_states"]
    vdtype = torch.float64 if sizes["value_bytes"] == 8 else torch.float32
    V = torch.empty(n, dtype=vdtype, device="cuda")
    pol = torch.empty(n, dtype=torch.uint8, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    nominal = float(n) * sizes["n_actions"] * sizes["n_outcomes"]

    sflags = vi.VI_FLAG_NO_GRAPH if args.no_graph else 0
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        vi.vi_solve(h, TOL, args.max_iters, V, pol, flags=sflags)
    sampler.wait_ready()
    barrier_sync(world)
    step_ms, iters = [], []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)   # evict L2 between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = vi.vi_solve(h, TOL, args.max_iters, V, pol, stream=stream, flags=sflags)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        iters.append(info["iters"])
    barrier_sync(world)
    wall = time.perf_counter() - t_wall0
    dev_s = sum(step_ms) / 1000.0
    dev_s_max = max_over_ranks(dev_s, world)
    updates = nominal * sum(iters)
    value = replica_value(updates, dev_s_max, world)

    # dominant kernel: single sweep launches (same kernel, same grid) timed with events,
    # still inside the clock-sampling window
    k_ms = time_sweep_kernel(vi, torch, h, V, stream, flush)
    clocks = sampler.stop()
    kch, kw = vi.vi_problem_kernel(h)
    kernel_name = kernel_name_of(vi, inst, kch, kw)
    pk = peaks()
    sm_mhz = clocks.get("sm_mhz") or pk["sm_max_mhz"]
    l2_gbs = l2_read_peak_gbs(vi, torch)
    roofline = roofline_of(vi, torch, inst, kernel_name, k_ms, sm_mhz, l2_gbs)

    # policy rollouts (row a12): 4096 rollouts x 365 periods of the extracted policy
    rollouts = None
    if len(inst.products) == 1:
        ro = workloads.CONFIG4_ROLLOUTS
        rets = torch.empty(ro["n_rollouts"], dtype=torch.float64, device="cuda")
        kpis = torch.empty(3 * ro["n_rollouts"], dtype=torch.float64, device="cuda")
        vi.vi_simulate(h, pol, ro["n_rollouts"], ro["horizon"], 0, ro["seed"], rets, kpis, stream=stream)
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for _ in range(5):
            vi.vi_simulate(h, pol, ro["n_rollouts"], ro["horizon"], 0, ro["seed"], rets, kpis, stream=stream)
        r1.record(stream)
        r1.synchronize()
        r_ms = r0.elapsed_time(r1) / 5
        rollouts = {"n_rollouts": ro["n_rollouts"], "horizon": ro["horizon"], "ms": r_ms,
                    "periods_per_s": ro["n_rollouts"] * ro["horizon"] / (r_ms * 1e-3),
                    "mean_return": float(rets.mean().item())}

    # base-stock policy search (the paper's heuristic benchmark): every S in 0..Q,
    # 4000 rollouts x 365 scored days after 100 warm-up days, shared random numbers;
    # the value-iteration policy is scored on the same rollouts
    policy_search = None
    if len(inst.products) == 1:
        n_r, H_s, W_s, seed_s = 4000, 365, 100, 4
        Qp = inst.products[0].Q
        ret_s = torch.empty((Qp + 1) * n_r, dtype=torch.float64, device="cuda")
        vi.vi_basestock_search(h, 0, Qp, n_r, H_s, W_s, seed_s, ret_s, stream=stream)
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        means_s, best_s = vi.vi_basestock_search(h, 0, Qp, n_r, H_s, W_s, seed_s, ret_s, stream=stream)
        b1.record(stream)
        b1.synchronize()
        bs_ms = b0.elapsed_time(b1)
        rets_vi = torch.empty(n_r, dtype=torch.float64, device="cuda")
        vi.vi_simulate(h, pol, n_r, H_s, W_s, seed_s, rets_vi, stream=stream)
        policy_search = {"S_range": [0, Qp], "n_rollouts": n_r, "horizon": H_s, "warmup": W_s, "ms": bs_ms,
                         "rollout_periods_per_s": (Qp + 1) * n_r * (H_s + W_s) / (bs_ms * 1e-3),
                         "best_S": int(best_s), "best_mean_return": float(means_s[best_s]),
                         "vi_policy_mean_return": float(rets_vi.mean().item())}

    # end to end through the public API with host buffers: create (tables H2D),
    # solve, V + policy D2H, destroy
    e2e_steps = max(1, min(args.steps, 5))
    Vh = torch.empty(n, dtype=vdtype).pin_memory().numpy()
    ph = torch.empty(n, dtype=torch.uint8).pin_memory().numpy()
    def e2e_step():
        h2 = vi.vi_problem_create_desc(desc)
        configure(h2)
        inf2 = vi.vi_solve_host(h2, TOL, args.max_iters, Vh, ph, flags=sflags)
        vi.vi_problem_destroy(h2)
        return inf2["iters"]

    e2e_step()   # warm-up: first allocation of the value buffers at this size
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(e2e_steps):
        e2e_iters += e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = nominal * e2e_iters * world / e2e_s
    h2d = sum(len(q.pmf) * 8 + 5 * 8 for q in inst.products)
    d2h = n * sizes["value_bytes"] + n

    out = None
    paper_a = run_paper_scenario_a(vi, torch, stream) if (rank == 0 and "a" in args.paper) else None
    paper_b = run_paper_scenario_b(vi, torch, stream) if (rank == 0 and "b" in args.paper) else None
    paper_c = run_paper_scenario_c(vi, torch, stream, args.no_graph) if (rank == 0 and "c" in args.paper) else None
    serving = run_serving(args.serving) if (args.serving > 0 and rank == 0) else None
    # the other large single-product configuration (4,084,101 states, FIFO, lead time 2)
    extra = None
    if rank == 0 and args.extra and args.workload != "cfg2":
        x = solve_summary(vi, torch, workloads.config2(), args, stream, flush, steps=5, warmup=2)
        x["roofline"] = roofline_of(vi, torch, workloads.config2(), x["kernel"], x["kernel_ms"], sm_mhz, l2_gbs)
        extra = x
    cfg3 = run_cfg3_accuracy(vi, torch, stream) if (rank == 0 and args.extra) else None
    if rank == 0:
        cpu = oracle_sample_rate(inst, args.cpu_seconds) if args.cpu_seconds > 0 else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * dev_s_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision or inst.precision], "data": "synthetic",
            "config": workload_config(inst, "flushed between steps (2x L2 write); 2 x 156 MB of values exceed L2"
                                      if inst.n_states * 16 > L2_BYTES else "flushed between steps (2x L2 write)",
                                      f"replicas x{world}" if world > 1 else "single GPU"),
            "solve": {"sweeps": iters[-1], "converged": bool(info["status"] == vi.VI_OK),
                      "precision": args.precision or inst.precision},
            "gpu_launches": solve_launches(iters, args.no_graph, args.max_iters,
                                           3 if (len(inst.products) == 2 and kch == vi.VI_KERNEL_GROUP) else 1),
            "clocks": clocks,
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "includes": "vi_problem_create + vi_solve_host + vi_problem_destroy"},
            "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind",
                                                                           "sample")},
            "serving": serving_summary(serving),
            "cfg3": cfg3,
            "rollouts": rollouts,
            "policy_search": policy_search,
            "paper_scenario_a": paper_a,
            "paper_scenario_b": paper_b,
            "paper_scenario_c": paper_c,
            "wall_s": wall,
            "cfg2": extra,
            "serving_detail": serving,
        }
        print(json.dumps(out))
    vi.vi_problem_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


def run_paper_scenario_a(vi, torch, stream) -> dict:
    """The paper's largest Scenario A experiment (m = 5, L = 2, FIFO, C_w = 7; Table 3
    row 5/6): value iteration with the paper's sup-norm test, then its 10,000-rollout
    evaluation, against the printed return and value-iteration wall time."""
    inst = workloads.scenario_a(5, 2, 7.0, workloads.FIFO)
    A, RO = workloads.SCENARIO_A, workloads.SCENARIO_A_ROLLOUTS
    p = inst.products[0]
    desc, keep = vi.make_desc([dict(m=p.m, L=p.L, Q=p.Q, cost=p.cost, pmf=p.pmf)], inst.gamma, inst.issuing,
                              vi.VI_PREC_FP32, vi.VI_STOP_SUPNORM)
    h = vi.vi_problem_create_desc(desc)
    n = vi.vi_problem_sizes(h)["n_states"]
    V = torch.empty(n, dtype=torch.float64, device="cuda")
    pol = torch.empty(n, dtype=torch.uint8, device="cuda")
    vi.vi_solve(h, A["eps"], 100000, V, pol, stream=stream)          # warm-up (autotune, graph)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    info = vi.vi_solve(h, A["eps"], 100000, V, pol, stream=stream)
    e1.record(stream)
    e1.synchronize()
    solve_ms = e0.elapsed_time(e1)
    ret = torch.empty(RO["n_rollouts"], dtype=torch.float64, device="cuda")
    vi.vi_simulate(h, pol, RO["n_rollouts"], RO["horizon"], RO["warmup"], 2023, ret, stream=stream)
    r = ret.cpu().numpy()
    vi.vi_problem_destroy(h)
    return {"experiment": "Scenario A, m=5, L=2, FIFO, C_w=7 (Table 3)", "states": n, "iterations": info["iters"],
            "vi_solve_ms": solve_ms, "paper_vi_wall_s": 1185.0,
            "return_mean": float(r.mean()), "return_sd": float(r.std(ddof=1)),
            "paper_return_mean": -1432.0, "paper_return_sd": 55.0}


SCEN_B_TABLES = os.path.join(ROOT, "tests", "golden", "scenario_b_tables.json")


def run_paper_scenario_b(vi, torch, stream) -> dict:
    """The paper's Scenario B (two products, half of product B's unmet demand takes
    product A): the four Ortega et al. settings P1-P4 at exactly 100 iterations
    (Table 5) and the largest Hendrix et al. setting, m = 3 experiment 1 with
    16,777,216 states, to the span test (Table 4), each from V_0 = the expected
    one-day revenue (one sweep from V = 0); the 10,000-rollout return of each
    value-iteration policy; and the modified base-stock search over the paper's
    whole (S_A, S_B) grid (4,000 rollouts x 365 days after 100) for P1 and m = 3
    experiment 1.  Times are CUDA-event device times on the launching stream."""
    rows = {r["name"]: r for r in json.load(open(SCEN_B_TABLES))["rows"]}
    RO = workloads.SCENARIO_B_ROLLOUTS
    out = {"note": "paper times: RTX 3060, FP64 JAX (Tables 4 and 5); updates = |S| |A| |Omega| x iterations "
                   "with |Omega| = (m A_A + 1)(m A_B + 1), the paper's issued-units outcome count; method_tflops = "
                   "2 x the factorised method's multiply-adds per sweep (bench.two_product_fmas) x sweeps / time, "
                   "against 148 x 128 x 2 flop x SM clock (77 TFLOP/s at 2032 MHz)",
           "experiments": []}

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    for name in ("P1", "P2", "P3", "P4", "m3_exp1"):
        row = rows[name]
        inst = workloads.scenario_b(name)
        prods = [dict(m=p.m, L=p.L, Q=p.Q, cost=p.cost, pmf=p.pmf) for p in inst.products]
        desc, keep = vi.make_desc(prods, inst.gamma, inst.issuing, vi.VI_PREC_FP32, vi.VI_STOP_SPAN,
                                  inst.subst_rate)
        h = vi.vi_problem_create_desc(desc)
        n = vi.vi_problem_sizes(h)["n_states"]
        Z = torch.zeros(n, dtype=torch.float64, device="cuda")
        V = torch.empty(n, dtype=torch.float64, device="cuda")
        pol = torch.empty(n, dtype=torch.uint8, device="cuda")
        fixed = row["vi_iterations"]
        tol, cap = (0.0, fixed) if fixed else (workloads.SCENARIO_B["eps"], 100000)

        def solve():
            vi.vi_backup(h, Z, V, stream=stream, stats=False)     # V_0 = expected revenue
            return vi.vi_solve(h, tol, cap, V, pol, stream=stream, flags=vi.VI_FLAG_WARM_START)

        solve()                                                 # warm-up (graph build)
        info, ms = timed(solve)
        ret = torch.empty(RO["n_rollouts"], dtype=torch.float64, device="cuda")
        vi.vi_simulate(h, pol, RO["n_rollouts"], RO["horizon"], RO["warmup"], 2023, ret, stream=stream)
        r = ret.cpu().numpy()
        iters = info["iters"]
        updates = float(n) * row["n_actions"] * row["n_outcomes"] * iters
        method_tflops = 2.0 * two_product_fmas(inst) * (iters + 1) / (ms * 1e-3) / 1e12   # + the V_0 sweep
        e = {"experiment": name, "table": row["table"], "states": n, "iterations": iters,
             "converged": bool(info["status"] == vi.VI_OK) if not fixed else None,
             "vi_ms": ms, "paper_vi_wall_s": row["vi_wall_s"], "speedup_vs_paper": row["vi_wall_s"] * 1e3 / ms,
             "paper_updates_per_s": updates / (ms / 1e3),
             "paper_own_updates_per_s": updates / row["vi_wall_s"] if fixed else None,
             "method_tflops": method_tflops,
             "return_mean": float(r.mean()), "return_sd": float(r.std(ddof=1)),
             "paper_return_mean": row["vi_return_mean"], "paper_return_sd": row["vi_return_sd"]}
        if name in ("P1", "m3_exp1"):
            lo, hi = (0, 0), (2 * row["amax_b"], 2 * row["amax_a"])
            mu = (row["mu_b"], row["mu_a"])
            npairs = (hi[0] + 1) * (hi[1] + 1)
            grid = torch.empty(npairs * 4000, dtype=torch.float64, device="cuda")
            vi.vi_mbs_search(h, lo, hi, mu, False, 64, 10, 0, 7, grid, stream=stream, means=False)  # warm-up
            _, sms = timed(lambda: vi.vi_mbs_search(h, lo, hi, mu, False, 4000, 365, 100, 7, grid, stream=stream,
                                                    means=False))
            gm = grid.view(npairs, 4000).mean(dim=1)
            bi = int(torch.argmax(gm).item())
            best = (bi // (hi[1] + 1), bi % (hi[1] + 1))
            e["base_stock_search"] = {
                "pairs": npairs, "rollouts": 4000, "days": 465, "ms": sms, "paper_so_wall_s": row["so_wall_s"],
                "best_S_A_B": [int(best[1]), int(best[0])],
                "paper_best_S_A_B": [row["kpis"]["A"]["s_best"], row["kpis"]["B"]["s_best"]],
                "rollout_periods_per_s": npairs * 4000 * 465 / (sms / 1e3)}
        out["experiments"].append(e)
        vi.vi_problem_destroy(h)
        del Z, V, pol
    return out


SCEN_C_TABLES = os.path.join(ROOT, "tests", "golden", "scenario_c_tables.json")


def run_paper_scenario_c(vi, torch, stream, no_graph: bool = False) -> dict:
    """The paper's Scenario C (weekday demand, uncertain life on arrival, FP64):
    both m = 3 settings and both m = 5 settings of Table 6 (1,361,367 states,
    which took 49.5 hours there) to the periodic stopping test from V_0 = 0, then
    10,000 rollouts of 365 days after 100 of each value-iteration policy.  Times
    are CUDA-event device times on the launching stream."""
    rows = json.load(open(SCEN_C_TABLES))["rows"]
    RO = workloads.SCENARIO_C_ROLLOUTS
    out = {"note": "paper times: RTX 3060, FP64 JAX (Table 6); work = one FP64 multiply-add per (state, order, "
                   "arrival profile) in the sweep plus one per (post-decision state, demand) in the post-decision "
                   "table; fp64_frac = that rate / 0.625e12 multiply-adds/s (B300 nominal FP64, 1.25 TFLOP/s)",
           "experiments": []}
    for row in rows:
        if row["m"] > 5:
            continue
        inst = workloads.scenario_c(row["m"], row["exp"])
        d, keep = vi.make_periodic_desc(inst.m, inst.Q, inst.pmf, inst.c0, inst.c1, inst.cost, inst.gamma)
        h = vi.vi_problem_create_periodic(d)
        n = inst.n_states
        V = torch.zeros(n, dtype=torch.float64, device="cuda")
        pol = torch.empty(n, dtype=torch.uint8, device="cuda")
        flags = vi.VI_FLAG_NO_GRAPH if no_graph else 0
        if row["m"] == 3:
            vi.vi_solve(h, workloads.SCENARIO_C["eps"], 2000, V, pol, stream=stream, flags=flags)   # warm-up
            V.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = vi.vi_solve(h, workloads.SCENARIO_C["eps"], 2000, V, pol, stream=stream, flags=flags)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        ret = torch.empty(RO["n_rollouts"], dtype=torch.float64, device="cuda")
        vi.vi_simulate(h, pol, RO["n_rollouts"], RO["horizon"], RO["warmup"], 2023, ret, stream=stream)
        r = ret.cpu().numpy()
        from math import comb
        G = inst.Q + 1
        profiles = comb(inst.Q + inst.m, inst.m)
        fmas = n * profiles + 7 * G ** inst.m * (inst.dmax + 1)
        out["experiments"].append({
            "experiment": f"m{row['m']}_exp{row['exp']} ({row['uncertainty']})", "states": n,
            "iterations": info["iters"], "converged": bool(info["status"] == vi.VI_OK), "vi_ms": ms,
            "paper_vi_wall_s": row["vi_wall_s"], "speedup_vs_paper": row["vi_wall_s"] * 1e3 / ms,
            "fp64_fma_per_s": fmas * info["iters"] / (ms * 1e-3),
            "fp64_frac": fmas * info["iters"] / (ms * 1e-3) / 0.625e12,
            "return_mean": float(r.mean()), "return_sd": float(r.std(ddof=1)),
            "paper_return_mean": row["vi_return_mean"], "paper_return_sd": row["vi_return_sd"]})
        vi.vi_problem_destroy(h)
        del V, pol
    return out


def serving_summary(d):
    """The serving comparison in a few numbers: server over sequential throughput
    (Poisson stream and burst) and both p99 latencies."""
    if d is None:
        return None
    srv, seq, b = d["server"], d["sequential"], d["burst"]
    return {"requests": d["requests"],
            "burst_speedup": b["server_updates_per_s"] / b["sequential_updates_per_s"],
            "stream_speedup": srv["updates_per_s"] / seq["updates_per_s"],
            "p99_ms": {"server": srv["p99_ms"], "sequential": seq["p99_ms"]},
            "p50_ms": {"server": srv["p50_ms"], "sequential": seq["p50_ms"]},
            "results_match": d["results_match"]}


def run_serving(n_requests: int = 512, seed: int = 5, slots: int = 64, budget_gb: float = 64.0) -> dict:
    """Serving mix: requests arriving as a Poisson stream, served by the
    continuous-batching server vs sequential plain solves of the same mix (each:
    create, solve with host buffers, destroy).  Both deliver every request's
    values and policy to host arrays.  Latency = arrival to result."""
    import paper_2303_10672_b300 as vi
    reqs = workloads.serving_mix(n_requests, seed=seed)
    descs = []
    for r in reqs:
        p = r.instance.products[0]
        descs.append(vi.make_desc([dict(m=p.m, L=p.L, Q=p.Q, cost=p.cost, pmf=p.pmf)], r.instance.gamma,
                                  r.instance.issuing))
    nominal = [r.instance.updates_per_sweep for r in reqs]
    n_states = [r.instance.n_states for r in reqs]

    def host_bufs(k):
        # the values and policy delivered to host memory, as the sequential path does
        return np.empty(n_states[k], np.float64), np.empty(n_states[k], np.uint8)

    # warm up both paths (module load, autotuning of each shape class, graph builds)
    srv = vi.vi_server_create(int(budget_gb * (1 << 30)), slots)
    wid = vi.vi_server_submit(srv, descs[0][0], TOL, MAX_ITERS)
    while not vi.vi_server_poll(srv, wid)[0]:
        time.sleep(0.001)
    vi.vi_server_wait(srv, 0)   # forget the warm-up request

    # -- server: submit at the arrival times, poll for completions
    t0 = time.perf_counter()
    ids, lat, upd = [], {}, 0.0
    pending = {}
    i = 0
    while i < len(reqs) or pending:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i].arrival_s <= now:
            bufs = host_bufs(i)
            rid = vi.vi_server_submit_to(srv, descs[i][0], TOL, MAX_ITERS, *bufs)
            pending[rid] = (i, bufs)
            i += 1
        wait_ms = 5 if i >= len(reqs) else max(0, min(5, int(1e3 * (reqs[i].arrival_s - now))))
        for rid in vi.vi_server_wait(srv, wait_ms):
            if rid not in pending:
                continue
            done, info = vi.vi_server_poll(srv, rid)
            k = pending.pop(rid)[0]
            lat[k] = info["wall_ms"]
            upd += nominal[k] * info["iters"]
    span_srv = time.perf_counter() - t0
    vi.vi_server_destroy(srv)
    lat_srv = np.array([lat[k] for k in range(len(reqs))])

    # -- sequential plain solves in arrival order
    for d in descs[:3]:
        h = vi.vi_problem_create_desc(d[0])
        n = vi.vi_problem_sizes(h)["n_states"]
        vi.vi_solve_host(h, TOL, MAX_ITERS, np.empty(n, np.float64), np.empty(n, np.uint8))
        vi.vi_problem_destroy(h)
    t0 = time.perf_counter()
    lat_seq, upd_seq = [], 0.0
    for k, (r, d) in enumerate(zip(reqs, descs)):
        now = time.perf_counter() - t0
        if now < r.arrival_s:
            time.sleep(r.arrival_s - now)
        h = vi.vi_problem_create_desc(d[0])
        n = vi.vi_problem_sizes(h)["n_states"]
        info = vi.vi_solve_host(h, TOL, MAX_ITERS, np.empty(n, np.float64), np.empty(n, np.uint8))
        vi.vi_problem_destroy(h)
        lat_seq.append(1e3 * (time.perf_counter() - t0 - r.arrival_s))
        upd_seq += nominal[k] * info["iters"]
    span_seq = time.perf_counter() - t0
    lat_seq = np.array(lat_seq)

    # -- capacity: the whole mix submitted at once, server vs sequential
    srv = vi.vi_server_create(int(budget_gb * (1 << 30)), slots)
    t0 = time.perf_counter()
    bufs = [host_bufs(k) for k in range(len(descs))]
    ids = [vi.vi_server_submit_to(srv, d[0], TOL, MAX_ITERS, *b) for d, b in zip(descs, bufs)]
    left = {rid: (k, bufs[k]) for k, rid in enumerate(ids)}
    upd_b = 0.0
    iters_b = [0] * len(descs)
    while left:
        for rid in vi.vi_server_wait(srv, 5):
            done, info = vi.vi_server_poll(srv, rid)
            kk = left.pop(rid)[0]
            iters_b[kk] = info["iters"]
            upd_b += nominal[kk] * info["iters"]
    span_b = time.perf_counter() - t0
    vi.vi_server_destroy(srv)
    t0 = time.perf_counter()
    upd_bs = 0.0
    for k, d in enumerate(descs):
        h = vi.vi_problem_create_desc(d[0])
        n = vi.vi_problem_sizes(h)["n_states"]
        info = vi.vi_solve_host(h, TOL, MAX_ITERS, np.empty(n, np.float64), np.empty(n, np.uint8))
        vi.vi_problem_destroy(h)
        upd_bs += nominal[k] * info["iters"]
    span_bs = time.perf_counter() - t0
    # equal accuracy (untimed): the burst's results against sequential solves of the same
    # requests, (1) with the body the server ran for the request (the FIFO column sweep where
    # it applies and dmax <= 46, else the factorised sweep): the same arithmetic, so
    # equal values; (2) with the autotuned kernel the timed sequential solves ran: other
    # rounding, so the span test may stop a sweep earlier or later, and values that stop at
    # different sweeps differ by a near-constant shift (the span test fixes V only up to a
    # constant); they are compared centred on their means, the policies as they are
    def seq_solve(k, kernel):
        h = vi.vi_problem_create_desc(descs[k][0])
        if kernel is not None:
            vi.vi_problem_set_option(h, vi.VI_OPT_KERNEL, kernel)
        w, q = host_bufs(k)
        info = vi.vi_solve_host(h, TOL, MAX_ITERS, w, q)
        vi.vi_problem_destroy(h)
        return w.view(np.float32).reshape(-1, 2).astype(np.float64).sum(axis=1), q, info["iters"]   # float pairs

    worst, pol_diff = 0.0, 0
    worst_auto, worst_centred, pol_auto, stop_diff = 0.0, 0.0, 0, 0
    for k, r in enumerate(reqs):
        p = r.instance.products[0]
        col = (r.instance.issuing == workloads.FIFO and ((p.L >= 2 and p.m >= 2) or (p.L == 1 and p.m >= 3))
               and p.Q + 1 <= 32 and p.dmax <= 46)
        b = bufs[k][0]                                                          # absolute FP64 values
        a, q, _ = seq_solve(k, vi.VI_KERNEL_FIFO_COL if col else vi.VI_KERNEL_GROUP)
        scale = max(np.abs(a).max(), 1e-300)
        worst = max(worst, float(np.abs(a - b).max() / scale))
        pol_diff += int((q != bufs[k][1]).sum())
        a2, q2, it2 = seq_solve(k, None)
        worst_auto = max(worst_auto, float(np.abs(a2 - b).max() / scale))
        worst_centred = max(worst_centred, float(np.abs((a2 - a2.mean()) - (b - b.mean())).max() / scale))
        pol_auto += int((q2 != bufs[k][1]).sum())
        stop_diff += int(it2 != iters_b[k])
    del bufs
    return {
        "workload": f"{n_requests} single-product requests, Poisson arrivals 200/s, m 2..6, L 1..3, Q 8..20, seed {seed}",
        "requests": n_requests,
        "results_match": {"max_rel_dV_vs_sequential": worst, "policy_differences": pol_diff,
                          "states": int(sum(n_states)),
                          "note": "sequential solves with the body the server ran for each request",
                          "vs_autotuned": {"max_rel_dV": worst_auto, "max_rel_dV_centred": worst_centred,
                                           "policy_differences": pol_auto, "stop_sweep_differences": stop_diff,
                                           "note": "sequential solves with the autotuned kernel; values "
                                                   "centred on their means (the span test fixes V up to a "
                                                   "constant)"}},
        "server": {"updates_per_s": upd / span_srv, "p50_ms": float(np.percentile(lat_srv, 50)),
                   "p99_ms": float(np.percentile(lat_srv, 99)), "makespan_s": span_srv, "slots": slots},
        "sequential": {"updates_per_s": upd_seq / span_seq, "p50_ms": float(np.percentile(lat_seq, 50)),
                       "p99_ms": float(np.percentile(lat_seq, 99)), "makespan_s": span_seq},
        "arrivals_span_s": reqs[-1].arrival_s,
        "burst": {"server_updates_per_s": upd_b / span_b, "server_makespan_s": span_b,
                  "sequential_updates_per_s": upd_bs / span_bs, "sequential_makespan_s": span_bs},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="cfg4", choices=sorted(WORKLOADS))
    ap.add_argument("--extra", type=int, default=1, help="also measure the 4.08M-state config 2 (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="oracle sample length (0 = skip)")
    ap.add_argument("--precision", default=None, choices=["fp32", "fp32_kahan", "fp64", "fp32_single"])
    ap.add_argument("--max-iters", type=int, default=MAX_ITERS)
    ap.add_argument("--serving", type=int, default=512, help="requests in the serving mix (0 = skip)")
    ap.add_argument("--paper", default="abc", help="which of the paper's Scenario A/B/C results to run ('' or 0 = none)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven sweep loop instead of the CUDA graph (same kernels; lets a profiler see each launch)")
    ap.add_argument("--kernel", choices=["auto", "group", "tensor", "generic", "lifo1", "fifocol"], default="auto",
                    help="sweep kernel (auto: the autotuner picks among the factorised variants)")
    ap.add_argument("--group-width", type=int, default=0,
                    help="lane width of the factorised kernel (0 = autotuned)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
