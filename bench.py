#!/usr/bin/env python
"""Benchmark: time to a 1e-10 relative residual with GMRES-IR (FP32 inner GMRES(50)) against
FP64 GMRES(50) on one B300, plus the HBM roofline of the dominant cycle kernel.

Workload (N=1): 3D 7-point upwind convection-diffusion on a 100^3 grid (n = 1,000,000,
nnz = 6,940,000, int32 CSR, FP64 master values), three instances with Peclet 1 / 10 / 50
and seeded random wind, b = A*1 + 1e-3 N(0,1), x0 = 0.  One step solves the three
instances in turn; `value` is the mean device time per solve (seconds, lower is better).
Plan creation (workspace, FP32 copy of A, graph capture) is outside the timed region, as
the paper excludes the single-precision copy of A from its solve times (Section 5).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank solves the same workload on its own GPU (replicas: one
solve does not shard on this single-GPU design); the reported time is the max over ranks.
`--impl reference` times the CPU oracle on the host cores on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-10 rel. residual: GMRES-IR vs FP64 GMRES, 1 B300; % HBM peak"
PECLETS = (1.0, 10.0, 50.0)
M = 50
RTOL = 1e-10
WORKLOAD = ("3D 7-point convection-diffusion 100^3 (n=1,000,000, nnz=6,940,000), Pe 1/10/50 "
            "with seeded random wind, b=A*1+1e-3*N(0,1), x0=0; GMRES-IR FP32 inner GMRES(50) vs "
            "FP64 GMRES(50), outer rtol 1e-10; one step = the three instances solved in turn")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------ clocks ----
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------- byte model ----
def bytes_per_launch(kind: str, j: int, n: int, nnz: int, s_a: int, s_v: int, s_w: int) -> float:
    """Algorithmic DRAM bytes of one launch: Section 5.5's SpMV model with perfect reuse of
    the gathered vector, and every basis column read once per kernel."""
    if kind == "spmv":  # A, gathered source, new basis column, w, and j columns for the dots
        s_src = 8 if j == 0 else s_w
        return nnz * (s_a + 4) + 4 * (n + 1) + n * s_src + n * s_v + n * s_w + j * n * s_v
    if kind in ("u1", "u2"):  # V_j read once, w read, w' written
        return (j + 1) * n * s_v + 2 * n * s_w
    if kind == "xupd":
        return j * n * s_v + 16 * n
    if kind == "residual":  # FP64 A (SELL-32: values, columns, slice table), x, b read, r written
        return nnz * 12 + 8 * ((n + 31) // 32) + 24 * n
    return 0.0


def in_cycle(kernels: dict, cycle_ms: float) -> dict:
    """Each kernel class's share of an uninstrumented cycle: the cycle graph timed with events
    at its two ends only (cycle_ms), split by the classes' shares of the per-kernel event
    times.  The per-kernel events of the instrumented graph each add an event node between
    two kernels; here no event sits between kernels, so the time is the cycle as a solve
    runs it, launch gaps included (apportioned with the shares)."""
    out = {}
    for k, v in kernels.items():
        t = cycle_ms * v["share"]
        b = v["bytes_per_launch"] * v["launches"]
        out[k] = {"ms_total": t, "launches": v["launches"], "share": v["share"],
                  "achieved_gbs": (b / 1e9) / (t / 1e3) if t > 0 else None,
                  "bytes_per_launch": v["bytes_per_launch"]}
    return out


def roofline(ms: np.ndarray, n: int, nnz: int, prec: int):
    """ms: (m+1, 3) per-launch times (ms) of one profiled cycle -> per-kernel-class totals."""
    s_a = s_v = {0: 8, 1: 4, 2: 2, 3: 2}[prec]
    s_w = 8 if prec == 0 else 4
    m = ms.shape[0] - 1
    cls = {}
    for j in range(m):
        for c, name in enumerate(("spmv", "u1", "u2")):
            if ms[j, c] >= 0:
                t, b, k = cls.get(name, (0.0, 0.0, 0))
                cls[name] = (t + ms[j, c], b + bytes_per_launch(name, j, n, nnz, s_a, s_v, s_w),
                             k + 1)
    steps = sum(1 for j in range(m) if ms[j, 0] >= 0)
    for c, name in enumerate(("lsq", "xupd", "residual")):
        cls[name] = (ms[m, c], bytes_per_launch(name, steps, n, nnz, s_a, s_v, s_w), 1)
    total = sum(t for t, _, _ in cls.values())
    out = {k: {"ms_total": t, "launches": k_, "share": t / total,
               "achieved_gbs": (b / 1e9) / (t / 1e3) if t > 0 else None,
               "bytes_per_launch": b / k_}
           for k, (t, b, k_) in cls.items()}
    dom = max(out, key=lambda k: out[k]["ms_total"])
    return dom, out


KERNEL_CLASSES = {  # the paper's kernel classes (Section 5.2) in this fused design
    "spmv": "SpMV + v_j store + first-pass GEMV-T (dots), Givens of the previous step",
    "u1": "first-pass GEMV-N (update) + second-pass GEMV-T (dots)",
    "u2": "second-pass GEMV-N (update) + norm",
    "lsq": "least squares (FP64, both)",
    "xupd": "x += gamma V y",
    "residual": "FP64 residual r = b - A x",
}


def per_kernel_speedup(k_ir: dict, k_64: dict) -> dict:
    """Per-cycle device time of each kernel class in GMRES-IR (FP32 inner) and FP64 GMRES on
    the same instance, and their ratio (Section 5.2's per-kernel speed-up table)."""
    out = {}
    for name, what in KERNEL_CLASSES.items():
        a, b = k_ir.get(name), k_64.get(name)
        if a and b and a["ms_total"] > 0:
            out[name] = {"what": what, "ir_ms": round(a["ms_total"], 4),
                         "fp64_ms": round(b["ms_total"], 4),
                         "speedup": round(b["ms_total"] / a["ms_total"], 3)}
    t_ir = sum(v["ms_total"] for v in k_ir.values())
    t_64 = sum(v["ms_total"] for v in k_64.values())
    ortho = [c for c in ("u1", "u2") if c in k_ir and c in k_64]
    o_ir = sum(k_ir[c]["ms_total"] for c in ortho)
    o_64 = sum(k_64[c]["ms_total"] for c in ortho)
    out["ortho_updates"] = {"what": "u1 + u2", "ir_ms": round(o_ir, 4), "fp64_ms": round(o_64, 4),
                            "speedup": round(o_64 / o_ir, 3) if o_ir else None}
    out["total"] = {"what": "one 50-step cycle run as a captured graph", "ir_ms": round(t_ir, 4),
                    "fp64_ms": round(t_64, 4), "speedup": round(t_64 / t_ir, 3) if t_ir else None}
    return out


# ------------------------------------------------------ measured traffic ----
PROFILE_OF = {"spmv": "k_spmv_sell_3d100_fp32.md", "u1": "k_cgs_u1_3d100_fp32.md",
              "u2": "k_cgs_u2_3d100_fp32.md"}


KERNEL_SOURCES = ("common.cuh", "kernels.cuh")  # the step kernels' code


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2109_01232_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, alg_bytes_avg: float):
    """DRAM bytes per launch of `kernel` from its committed ncu summary (one captured launch,
    scaled to the cycle's average launch by the algorithmic bytes), or None when there is no
    summary or the kernel sources changed after the capture."""
    name = PROFILE_OF.get(kernel)
    path = os.path.join(ROOT, "profiles", name) if name else None
    if not path or not os.path.exists(path):
        return None
    fields = {}
    with open(path) as fh:
        for line in fh:
            k, sep, v = line.partition(":")
            if sep and k.strip() in ("traffic_bytes_per_launch", "alg_bytes_per_launch",
                                     "source_sha256_16"):
                fields[k.strip()] = v.strip()
    if fields.get("source_sha256_16") != kernel_source_hash():
        return None
    return float(fields["traffic_bytes_per_launch"]) * alg_bytes_avg / float(fields["alg_bytes_per_launch"])


# ------------------------------------------------------- batched workload ----
BATCH_M = 30


def batch_cycle_bytes(n: int, nnz: int, m: int) -> float:
    """Algorithmic bytes of one FP32 inner cycle of the batched solver on one system (the
    per-step byte model of the single-system kernels, summed over the m steps, plus the
    FP64 residual and the x update)."""
    steps = sum(nnz * 8 + 4 * (n + 1) + 3 * 4 * n + j * 4 * n      # A: SpMV, v_j, w, dots
                + (j + 1) * 4 * n + 2 * 4 * n                       # B: V once, w in/out
                + (j + 1) * 4 * n + 2 * 4 * n for j in range(m))    # C
    return steps + nnz * 12 + 4 * (n + 1) + 24 * n + m * 4 * n + 16 * n


def run_batched(g, torch, peak):
    """The batched workload: 512 independent 2D convection-diffusion systems solved by
    GMRES-IR (FP32 inner GMRES(30)) in one persistent launch, and by FP64 GMRES(30) per
    system in the same kernel form, on the same GPU."""
    import gen
    systems = gen.batched_systems()
    batch = g.DeviceBatch([p for p, _, _ in systems])
    b = torch.tensor(np.concatenate([bb for _, bb, _ in systems]), device="cuda")
    x = torch.zeros_like(b)
    t0 = time.perf_counter()
    plan = g.BatchPlan(batch, autotune=True, restart_m=BATCH_M, rtol=RTOL)
    tune_s = time.perf_counter() - t0
    info = plan.info()
    plan.solve(b, x)  # warm-up
    ms = []
    for _ in range(2):
        x.zero_()
        res = plan.solve(b, x)
        ms.append(res.t_solve_ms)
    plan.close()
    if not (res.status == g.OK).all():
        raise SystemExit("batched solve failed")
    xs = batch.split(x.cpu().numpy())
    err = max(float(np.abs(xi - xt).max() / np.abs(xt).max()) for xi, (_, _, xt) in zip(xs, systems))
    plan64 = g.BatchPlan(batch, autotune=False, restart_m=BATCH_M, rtol=RTOL, inner_prec="fp64")
    x.zero_()
    plan64.solve(b, x)
    x.zero_()
    r64 = plan64.solve(b, x)
    plan64.close()
    t = statistics.median(ms) / 1e3
    nbytes = sum(int(res.outer[i]) * batch_cycle_bytes(p.n, len(p.vals), BATCH_M)
                 for i, (p, _, _) in enumerate(systems))
    return {"workload": "512 2D convection-diffusion systems, sides U{32..256} (1,024-65,536 "
                        "rows, 12.8M in total), Pe U(0.1, 50), b = A x_true; GMRES-IR with FP32 "
                        "inner GMRES(30), rtol 1e-10, one persistent graph-captured launch",
            "solves_per_s": len(systems) / t, "ms_per_batch": t * 1e3,
            "fp64_gmres_ms_per_batch": r64.t_solve_ms,
            "speedup_vs_fp64": r64.t_solve_ms / (t * 1e3),
            "iters_mean": float(res.iters.mean()), "iters_max": int(res.iters.max()),
            "max_relres": float(res.rel_resid.max()), "max_x_err_vs_x_true": err,
            "autotuned": {"threads": info["threads"], "cluster": info["cluster"],
                          "ctas": info["ctas"], "seconds": tune_s},
            "hbm": {"alg_bytes": nbytes, "achieved_gbs": nbytes / t / 1e9,
                    "frac": nbytes / t / 1e9 / peak}}


# ---------------------------------------------------------- small case ----
def run_small_case(g, torch, reps: int = 20) -> dict:
    """The plain-method small case (2D 64 x 64, Pe 10, b = A x_true, x0 = 0, rtol 1e-10):
    FP64 GMRES(50) and GMRES-IR (FP32 inner GMRES(50), inner tolerance 1e-4) through a
    reused plan, median device time of `reps` solves after a warm-up.  Everything fits in
    L2, so this case is latency-bound: time and solves/s, no HBM fraction."""
    import gen
    p, b, x_true = gen.config_small_2d()
    A = g.DeviceCSR.from_problem(p)
    bt = torch.tensor(b, device="cuda")
    x = torch.zeros_like(bt)
    out = {"workload": "2D 5-point convection-diffusion 64x64 (n=4096), Pe 10, b = A x_true, "
                       "x0 = 0, rtol 1e-10; reused plan, median of %d solves" % reps}
    for name, kind, kw in (("fp64_gmres", "gmres", {}), ("gmres_ir", "ir", dict(inner_rtol=1e-4))):
        plan = g.Plan(A, kind, restart_m=M, rtol=RTOL, **kw)
        ts, r = [], None
        for _ in range(reps + 1):
            x.zero_()
            r = plan.solve(bt, x)
            ts.append(r.t_solve_ms)
        plan.close()
        err = float(np.linalg.norm(x.cpu().numpy() - x_true) / np.linalg.norm(x_true))
        t = statistics.median(ts[1:])
        out[name] = {"ms": t, "solves_per_s": 1e3 / t, "iters": r.iters, "status": r.status_name,
                     "relres": r.relres, "x_err_vs_x_true": err}
    out["speedup_ir_vs_fp64"] = out["fp64_gmres"]["ms"] / out["gmres_ir"]["ms"]
    return out


# ------------------------------------------------------------- multi-rank ----
def max_over_ranks(value: float, dist=None) -> float:
    """The largest `value` over the ranks of the default process group (replicas: every
    rank times the same workload, the job is as slow as its slowest rank)."""
    if dist is None:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------- our arm ----
def run_ours(args, rank, world, local_rank):
    import torch

    import gen
    import paper_2109_01232_b300 as g

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    insts = []
    for pe in PECLETS:
        p, b = gen.config_3d(pe)
        A = g.DeviceCSR.from_problem(p)
        insts.append(dict(pe=pe, p=p, b=b, A=A, bt=torch.tensor(b, device="cuda"),
                          x=torch.zeros(p.n, dtype=torch.float64, device="cuda")))
    kw = dict(restart_m=M, rtol=RTOL, max_iters=50000)
    for it in insts:
        it["ir"] = g.Plan(it["A"], "ir", inner_prec="fp32", **kw)
    stream = torch.cuda.current_stream()

    def step(kind="ir"):
        res = []
        for it in insts:
            it["x"].zero_()
            res.append(it[kind].solve(it["bt"], it["x"]))
        return res

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0.record(stream)
    results = []
    for k in range(args.steps):
        marks[k].record(stream)
        results.append(step())
    marks[-1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = [marks[k].elapsed_time(marks[k + 1]) for k in range(args.steps)]
    clocks = sampler.stop() if sampler else None
    if dist:
        dist.barrier()
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1), dist)
    per_solve_s = elapsed_ms / 1e3 / (args.steps * len(insts))
    for rs in results:
        for r in rs:
            if r.status != g.OK:
                raise SystemExit(f"solve failed: {r}")
    ir_iters = {f"pe{it['pe']:g}": r.iters for it, r in zip(insts, results[-1])}
    ir_relres = {f"pe{it['pe']:g}": r.relres for it, r in zip(insts, results[-1])}
    # per solve: the first residual, then per refinement step one cycle graph of 3 kernels per
    # Arnoldi step, the store of v_0 (low-precision cycles), the last Givens update, least
    # squares, x update and residual
    launches_per_step = sum(1 + r.outer * (3 * M + 5) for r in results[-1])

    # FP64 GMRES(50) on the same GPU (the comparison named by the metric).
    for it in insts:
        it["ir"].close()
        it["fp64"] = g.Plan(it["A"], "gmres", **kw)
    step("fp64")
    reps = 3

    def timed(kind):
        """Median over `reps` steps of the per-solve time (each step timed by events)."""
        ts, out = [], None
        for _ in range(reps):
            torch.cuda.synchronize()
            e0.record(stream)
            out = step(kind)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3 / len(insts))
        return statistics.median(ts), out

    fp64_s, last64 = timed("fp64")
    res64 = [last64]
    fp64_iters = {f"pe{it['pe']:g}": r.iters for it, r in zip(insts, res64[-1])}
    for it in insts:
        it["fp64"].close()

    # GMRES-IR with FP16 storage of A and V (FP32 accumulation), the metric's second inner
    # precision: time per solve, iterations and status of each instance.
    for it in insts:
        it["fp16"] = g.Plan(it["A"], "ir", inner_prec="fp16", **kw)
    step("fp16")
    fp16_s, last16 = timed("fp16")
    res16 = [last16]
    fp16 = dict(ir_s=fp16_s,
                iters={f"pe{it['pe']:g}": r.iters for it, r in zip(insts, res16[-1])},
                status={f"pe{it['pe']:g}": r.status_name for it, r in zip(insts, res16[-1])},
                relres={f"pe{it['pe']:g}": r.relres for it, r in zip(insts, res16[-1])})
    fp16["speedup_vs_fp64"] = fp64_s / fp16["ir_s"]
    for it in insts:
        it["fp16"].close()

    out = None
    if rank == 0:
        peak, peak_kind = load_peaks()
        # Per-kernel device times of one cycle (Pe 10 instance), CUDA events on this stream:
        # inside a captured graph of the cycle, as a solve runs it (event-record nodes between
        # the kernels; the roofline uses these), and kernel by kernel with a host
        # synchronisation after every step (reported beside them).
        it = insts[1]
        plan = g.Plan(it["A"], "ir", inner_prec="fp32", **kw)
        info = plan.info()
        x0 = torch.zeros_like(it["x"])
        plan.profile_cycle(it["bt"], x0, graph=True)  # warm
        ms = plan.profile_cycle(it["bt"], x0, graph=True)
        ms_1by1 = plan.profile_cycle(it["bt"], x0)
        cycles = [plan.time_cycle(it["bt"], x0) for _ in range(3)]
        plan.close()
        cycle_ms = statistics.median(c[0] for c in cycles)
        dom, kernels_ev = roofline(ms, info["n"], info["nnz"], 1)
        _, kernels_1by1 = roofline(ms_1by1, info["n"], info["nnz"], 1)
        kernels = in_cycle(kernels_ev, cycle_ms)
        kd = kernels[dom]
        # the same cycle in FP64 GMRES(50): per-kernel IR over FP64 (Section 5.2's table)
        plan = g.Plan(it["A"], "gmres", **kw)
        plan.profile_cycle(it["bt"], x0, graph=True)
        ms64 = plan.profile_cycle(it["bt"], x0, graph=True)
        cycle64_ms = statistics.median(plan.time_cycle(it["bt"], x0)[0] for _ in range(3))
        plan.close()
        _, kernels64 = roofline(ms64, info["n"], info["nnz"], 0)
        kernel_speedup = per_kernel_speedup(kernels, in_cycle(kernels64, cycle64_ms))
        # end to end through the host-pointer C ABI (copies in and out, plan creation)
        p = it["p"]
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        rp, ci, va, bh = pin(p.row_ptr), pin(p.col_idx), pin(p.vals), pin(it["b"])
        xh = torch.zeros(p.n, dtype=torch.float64).pin_memory()
        g.gmres_ir_solve_host(rp, ci, va, bh, xh, inner_prec="fp32", **kw)
        e2e = []
        for _ in range(2):
            xh.zero_()
            t0 = time.perf_counter()
            r = g.gmres_ir_solve_host(rp, ci, va, bh, xh, inner_prec="fp32", **kw)
            e2e.append(time.perf_counter() - t0)
            assert r.status == g.OK
        h2d = 4 * (p.n + 1) + 12 * p.nnz + 16 * p.n
        cpu = None if args.no_cpu_baseline else cpu_baseline(it["p"], it["b"])
        batched = None if args.no_batched else run_batched(g, torch, peak)
        small = run_small_case(g, torch)
        out = {
            "metric": METRIC, "value": per_solve_s, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": False,
            "ms_per_step_median": statistics.median(step_ms),
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": 1000000, "nnz": 6940000, "restart_m": M,
                       "inner": "fp32 storage and accumulation", "outer": "fp64",
                       "l2": "inputs larger than L2: FP64 + FP32 matrix 139 MB and a 204 MB "
                             "Krylov basis per solve; no explicit flush",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "fp64_gmres_s": fp64_s, "speedup_vs_fp64": fp64_s / per_solve_s,
            "fp16_storage_ir": {k: (round(v, 6) if isinstance(v, float) else v)
                                for k, v in fp16.items()},
            "iters": {"ir": ir_iters, "fp64": fp64_iters}, "relres": ir_relres,
            "roofline": {"bound": "hbm", "kernel": dom,
                         "achieved": kd["achieved_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": kd["achieved_gbs"] / peak, "peak_source": peak_kind,
                         "traffic": measured_traffic(dom, kd["bytes_per_launch"]),
                         "bytes_per_launch": kd["bytes_per_launch"],
                         "avg_launch_ms": kd["ms_total"] / kd["launches"],
                         "timing": "the kernel's share of one 50-step cycle (Pe 10 instance) "
                                   "run as a captured graph and timed by CUDA events at its two "
                                   "ends (median of 3); the share from a second capture with an "
                                   "event node before every kernel",
                         "event_bracketed": {
                             "achieved": kernels_ev[dom]["achieved_gbs"],
                             "frac": kernels_ev[dom]["achieved_gbs"] / peak,
                             "avg_launch_ms": kernels_ev[dom]["ms_total"] / kernels_ev[dom]["launches"],
                             "what": "the time between the event nodes around each launch "
                                     "(each adds a node between two kernels)"}},
            "cycle_ms": {"uninstrumented": cycle_ms,
                         "event_per_kernel": sum(v["ms_total"] for v in kernels_ev.values()),
                         "steps": cycles[0][1], "fp64_uninstrumented": cycle64_ms,
                         "fp64_event_per_kernel": sum(v["ms_total"] for v in kernels64.values())},
            "kernels": {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv)
                            for kk, vv in v.items()} for k, v in kernels.items()},
            "kernels_event_bracketed": {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv)
                                            for kk, vv in v.items()} for k, v in kernels_ev.items()},
            "kernels_one_by_one": {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv)
                                       for kk, vv in v.items()} for k, v in kernels_1by1.items()},
            "kernel_speedup_vs_fp64": kernel_speedup,
            "cpu_baseline": cpu,
            "batched": batched,
            "small_case": small,
            "e2e": {"value": statistics.median(e2e), "unit": "s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * p.n,
                    "what": "gmres_ir_solve_host on the Pe 10 instance from pinned host memory: "
                            "copies of A, b, x0 in, plan set-up, solve, x out"},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
    if dist:
        dist.destroy_process_group()
    return out


def _recorded(key: str):
    """The oracle's own solve of the 100^3 instance recorded by oracle/record_iterations.py
    (iterations, cycles, seconds), or None."""
    rec = os.path.join(ROOT, "oracle", "iterations_3d100.json")
    if os.path.exists(rec):
        d = json.load(open(rec)).get(key)
        if d and d.get("status") == 0:
            return d
    return None


def _time(fn) -> float:
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


def oracle_cycle_s(p, b, fp64: bool) -> float:
    """Seconds of ONE whole oracle cycle on the host: the FP64 residual of x0, one restart
    cycle of 50 Arnoldi steps (CGS2, Givens, least squares), the update and the new residual
    -- GMRES-IR with the FP32-emulated inner cycle, or FP64 GMRES(50).  Every cycle of a
    solve does the same work, so a solve takes (cycles) x this."""
    import oracle
    if fp64:
        return _time(lambda: oracle.gmres(p, b, m=M, rtol=RTOL, max_iters=M))
    return _time(lambda: oracle.gmres_ir(p, b, m=M, rtol=RTOL, inner="fp32", max_iters=M))


SMALL_CASE_CODE = """
import json, statistics, sys, time
sys.path.insert(0, {root!r})
import gen, oracle
p, b, _ = gen.config_small_2d()
runs = {{"fp64_gmres": lambda: oracle.gmres(p, b, m={m}, rtol={rtol}),
        "gmres_ir": lambda: oracle.gmres_ir(p, b, m={m}, rtol={rtol}, inner="fp32", inner_rtol=1e-4)}}
out = {{}}
for name, fn in runs.items():
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        info = fn()[1]
        ts.append(time.perf_counter() - t0)
    out[name] = {{"s_median_of_3": statistics.median(ts), "iters": int(info.iters)}}
print(json.dumps(out))
"""


def small_case_oracle(one_thread: bool = True) -> dict:
    """The plain-method small case (2D 64 x 64, Pe 10, b = A x_true): oracle FP64 GMRES(50)
    and GMRES-IR (FP32 inner GMRES(50), inner tolerance 1e-4) solved to 1e-10, median of 3
    full solves, in a child process with the default BLAS threads and in one with a single
    thread (OPENBLAS/OMP/MKL_NUM_THREADS=1)."""
    code = SMALL_CASE_CODE.format(root=ROOT, m=M, rtol=RTOL)
    res = {}
    for label, extra in (("all", {}), ("one", {"OPENBLAS_NUM_THREADS": "1", "OMP_NUM_THREADS": "1",
                                               "MKL_NUM_THREADS": "1"})):
        if label == "one" and not one_thread:
            continue
        env = dict(os.environ, **extra)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           check=True)
        res[label] = json.loads(r.stdout.strip().splitlines()[-1])
    out = res["all"]
    if "one" in res:
        for name in out:
            out[name]["s_1_thread"] = res["one"][name]["s_median_of_3"]
    return out


def cpu_baseline(p, b) -> dict:
    """The oracle on the GPU machine's host cores (a bounded sample of about 20-30 s).  The
    benchmark's Pe 10 instance: one whole GMRES-IR refinement step and one whole FP64
    GMRES(50) cycle, each timed and multiplied by the number of cycles the oracle's own
    full solve of that instance takes (oracle/iterations_3d100.json: 14 and the FP64
    count).  Plus the small 64 x 64 case solved in full (median of 3, all threads and one)."""
    rec_ir, rec_64 = _recorded("pe10"), _recorded("pe10_fp64")
    t_ir = oracle_cycle_s(p, b, fp64=False)
    t_64 = oracle_cycle_s(p, b, fp64=True)
    # cycle-equivalents of the oracle's own full solves (FP64's last cycle is partial)
    n_ir = int(rec_ir["iters"]) / M if rec_ir else 14.0
    n_64 = int(rec_64["iters"]) / M if rec_64 else None
    small = small_case_oracle()
    return {"value": t_ir * n_ir, "unit": "s", "cores": threads_used(), "kind": "oracle",
            "fp64_gmres_s": t_64 * n_64 if n_64 else None,
            "ir_cycle_s": t_ir, "fp64_cycle_s": t_64, "ir_cycles": n_ir, "fp64_cycles": n_64,
            "small_64x64": small,
            "sample": f"oracle.gmres_ir (numpy, FP32-emulated inner GMRES(50)) on the Pe 10 "
                      f"100^3 instance: one whole refinement step (residual, 50 Arnoldi steps, "
                      f"least squares, update, residual) took {t_ir:.2f} s, x {n_ir:g} cycles of "
                      f"the oracle's own full solve; FP64 GMRES(50): one cycle {t_64:.2f} s x "
                      f"{n_64:g} cycle-equivalents; 64x64 case: full solves.  The sparse products run on one "
                      f"thread (numpy), the dense basis products on `cores` BLAS threads"}


def threads_used() -> int:
    """BLAS threads of this process: threadpoolctl's count where it is installed, else the
    OPENBLAS/OMP thread variable, else every core (OpenBLAS's default)."""
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return os.cpu_count() or 1


# --------------------------------------------------------- reference arm ----
def run_reference(args, rank):
    """The reference arm: the CPU oracle on the host cores, on the benchmark's Pe 10 100^3
    instance.  Every step times one whole oracle GMRES-IR refinement step (FP64 residual, one
    FP32-emulated GMRES(50) cycle, update, residual); `value` is the mean step time x the
    number of refinement steps of the oracle's own full solve of that instance."""
    if rank != 0:
        return None
    import gen
    p, b = gen.config_3d(10.0)
    rec = _recorded("pe10")
    n_cyc = int(rec["outer"]) if rec else 14
    times = []
    for i in range(args.warmup + args.steps):
        t = oracle_cycle_s(p, b, fp64=False)
        if i >= args.warmup:
            times.append(t)
    value = statistics.mean(times) * n_cyc
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "s", "kind": "oracle",
                             "cores": threads_used(),
                             "sample": f"each step: one whole oracle GMRES-IR refinement step "
                                       f"(50 Arnoldi steps) on the Pe 10 instance; x {n_cyc} "
                                       f"steps of the oracle's own full solve"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def cpu_full(args) -> dict:
    """Complete oracle solves of the Pe 10 100^3 instance (GMRES-IR and FP64 GMRES(50) to
    1e-10), `--cpu-full-reps` each: several minutes per solve, so not part of the default
    run.  Checks the whole-cycle samples of the default run against whole solves."""
    import gen
    import oracle
    p, b = gen.config_3d(10.0)
    out = {"cores": threads_used(), "workload": "Pe 10 100^3 instance, x0 = 0, rtol 1e-10"}
    for name, fn in (("gmres_ir", lambda: oracle.gmres_ir(p, b, m=M, rtol=RTOL, inner="fp32")),
                     ("fp64_gmres", lambda: oracle.gmres(p, b, m=M, rtol=RTOL))):
        ts, info = [], None
        for _ in range(args.cpu_full_reps):
            t0 = time.perf_counter()
            _, info = fn()
            ts.append(time.perf_counter() - t0)
        out[name] = {"s": ts, "s_median": statistics.median(ts), "iters": int(info.iters),
                     "cycles": int(info.outer), "relres": float(info.relres),
                     "one_cycle_s": oracle_cycle_s(p, b, fp64=(name == "fp64_gmres"))}
    out["small_64x64"] = small_case_oracle()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-system batched workload")
    ap.add_argument("--cpu-full", action="store_true",
                    help="only time complete oracle solves on the host (minutes per solve)")
    ap.add_argument("--cpu-full-reps", type=int, default=1)
    args = ap.parse_args()
    if args.cpu_full:
        print(json.dumps(cpu_full(args)))
        return
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
