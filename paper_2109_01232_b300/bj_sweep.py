"""The block-Jacobi workloads (Section 5.8's "J k" rows): FP64 GMRES(50) against GMRES-IR
with an FP32 inner GMRES(50), both with the reverse Cuthill-McKee reordering and the
block-Jacobi right preconditioner of the row's block size, on this GPU.

The paper's matrices are SuiteSparse entries that are not available here; the workloads
are the synthetic stand-ins of gen.config_bj() (badly scaled, shuffled numbering).  For
each: the median of three solves (b = ones, x0 = 0, rtol 1e-10), iterations, explicit
relative residual in the caller's numbering, the speed-up of GMRES-IR, plan set-up time
(reordering, FP32 copy, block factorisation), and the device rate of M^{-1} v (a cast of v
into the working type and the block-Jacobi apply, timed with CUDA events over 50 calls;
bytes: v read and cast, the factors, the pivot order, v read again and z written).  Each
solve is capped at 20,000 iterations.

    python -m paper_2109_01232_b300.bj_sweep
    python -m paper_2109_01232_b300.bj_sweep --apply-only   # the ncu target: set-up of the
        # k = 42 FP32 plan, then five M^{-1} v calls (a cast kernel and k_bj_apply each)
"""
from __future__ import annotations

import os
import statistics
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def run(m: int = 50, rtol: float = 1e-10, max_iters: int = 20000, log=None):
    import torch

    import gen
    import paper_2109_01232_b300 as g
    rows = []
    for p, k in gen.config_bj():
        A = g.DeviceCSR.from_problem(p)
        bt = torch.ones(p.n, dtype=torch.float64, device="cuda")
        res = {}
        for name, kind, kw in (("FP64 GMRES", "gmres", {}), ("GMRES-IR FP32 inner", "ir",
                                                            dict(inner_prec="fp32"))):
            plan = g.Plan(A, kind, restart_m=m, rtol=rtol, max_iters=max_iters, bj_block=k,
                          bj_rcm=1, **kw)
            runs = []
            for _ in range(3):
                x = torch.zeros_like(bt)
                r = plan.solve(bt, x)
                runs.append((r, x))
            ms = statistics.median(r.t_solve_ms for r, _ in runs)
            r, x = runs[-1]
            Ax = torch.empty_like(bt)  # the residual in the caller's numbering
            g.spmv_fp64_noalloc(A, x, Ax)
            relres = float(torch.linalg.norm(bt - Ax) / torch.linalg.norm(bt))
            # M^{-1} v rate
            v = torch.tensor(np.random.default_rng(5).standard_normal(p.n), device="cuda")
            plan.bj_apply(v)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(50):
                plan.bj_apply(v)
            e1.record()
            torch.cuda.synchronize()
            apply_ms = e0.elapsed_time(e1) / 50
            wb = 8 if kind == "gmres" else 4
            nblocks = (p.n + k - 1) // k
            full, last = divmod(p.n, k)
            factor_vals = full * k * k + last * last
            bytes_ = p.n * 8 + p.n * wb + factor_vals * wb + p.n * 4 + 2 * p.n * wb
            res[name] = dict(status=r.status_name, iters=r.iters, ms=ms, relres=relres,
                             setup_ms=r.t_setup_ms, apply_ms=apply_ms,
                             apply_gbs=bytes_ / apply_ms / 1e6, nblocks=nblocks)
            if log:
                log(dict(matrix=p.name, solver=name, **res[name]))
            plan.close()
        rows.append((p, k, res))
    return rows


def table(rows) -> str:
    out = ["| matrix | n | nnz | k | solver | status | iterations | solve ms (median of 3) | "
           "explicit relres | set-up ms | M^-1 v: us / GB/s |",
           "|---|---:|---:|---:|---|---|---:|---:|---:|---:|---:|"]
    for p, k, res in rows:
        for name, r in res.items():
            out.append(f"| {p.name} | {p.n:,} | {len(p.vals):,} | {k} | {name} | {r['status']} | "
                       f"{r['iters']} | {r['ms']:.1f} | {r['relres']:.2e} | {r['setup_ms']:.0f} | "
                       f"{1e3 * r['apply_ms']:.1f} / {r['apply_gbs']:.0f} |")
        a, b = res["FP64 GMRES"], res["GMRES-IR FP32 inner"]
        out.append(f"| | | | | speed-up of GMRES-IR | | | {a['ms'] / b['ms']:.2f}x | | | |")
    return "\n".join(out)


def apply_only(calls: int = 5):
    import torch

    import gen
    import paper_2109_01232_b300 as g
    p, k = gen.config_bj()[0]
    plan = g.Plan(g.DeviceCSR.from_problem(p), "ir", restart_m=50, inner_prec="fp32",
                  bj_block=k, bj_rcm=1)
    v = torch.tensor(np.random.default_rng(5).standard_normal(p.n), device="cuda")
    for _ in range(calls):
        plan.bj_apply(v)
    torch.cuda.synchronize()
    full, last = divmod(p.n, k)
    print(f"{p.name}: n = {p.n}, k = {k}, factor values = {full * k * k + last * last}")
    plan.close()


if __name__ == "__main__":
    if "--apply-only" in sys.argv[1:]:
        apply_only()
    else:
        rows = run(log=lambda r: print(r, file=sys.stderr, flush=True))
        print(table(rows))
