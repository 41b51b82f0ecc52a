"""FP64 vs FP32 SpMV on Galeri-like stencils (Section 5.5's experiment on this GPU).

For each matrix: the plan's SELL-32 SpMV alone (gmres_plan_spmv_timed), 1000 calls on a
random vector after a warm-up, the minimum of three runs, in FP64 and in FP32; the speedup
beside the paper's perfect-x-reuse model 5w/(2w+1) (w = nonzeros per row), and the bytes
per second under that model's traffic (FP64: 20 bytes per nonzero, FP32: 8 per nonzero +
4 per row).

    python -m paper_2109_01232_b300.spmv_sweep
"""
from __future__ import annotations

import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

CASES = [("laplace_2d", 1500), ("laplace_2d", 2500), ("laplace_3d", 100), ("laplace_3d", 150),
         ("box_2d", 1500), ("star_3d", 120), ("uniflow_2d", 2500), ("bentpipe_2d", 1500)]


def build(kind: str, side: int):
    import gen
    if kind == "uniflow_2d":
        return gen.uniflow_2d(side)
    if kind == "bentpipe_2d":
        return gen.bentpipe_2d(side)
    return getattr(gen, kind)(side)


def run(reps: int = 1000, trials: int = 3):
    import torch

    import paper_2109_01232_b300 as g
    rows = []
    for kind, side in CASES:
        p = build(kind, side)
        A = g.DeviceCSR.from_problem(p)
        x64 = torch.tensor(np.random.default_rng(1).uniform(-1, 1, p.n), device="cuda")
        M = p.scipy()
        ref = M @ x64.cpu().numpy()
        t = {}
        for prec, kind_ in (("fp64", "gmres"), ("fp32", "ir")):
            plan = g.Plan(A, kind_, restart_m=2, inner_prec="fp32")
            x = x64 if prec == "fp64" else x64.float()
            y, _ = plan.spmv_timed(x, 1)
            err = np.abs(y.double().cpu().numpy() - ref).max() / np.abs(ref).max()
            assert err <= (1e-13 if prec == "fp64" else 1e-5), (p.name, prec, err)
            t[prec] = min(plan.spmv_timed(x, reps)[1] for _ in range(trials))
            plan.close()
        w = len(p.vals) / p.n
        nnz = len(p.vals)
        rows.append(dict(name=p.name, n=p.n, nnz=nnz, w=w, max_row=int(np.diff(p.row_ptr).max()),
                         ms64=t["fp64"], ms32=t["fp32"], speedup=t["fp64"] / t["fp32"],
                         model=5 * w / (2 * w + 1),
                         gbs64=20 * nnz / (t["fp64"] * 1e-3) / 1e9,
                         gbs32=(8 * nnz + 4 * p.n) / (t["fp32"] * 1e-3) / 1e9))
        del A
    return rows


def table(rows) -> str:
    out = ["| matrix | n | nnz | w | FP64 ms | FP32 ms | speedup | model 5w/(2w+1) | FP64 GB/s (model bytes) | FP32 GB/s (model bytes) |",
           "|---|---:|---:|---:|---:|---:|---:|---:|---:|---:|"]
    for r in rows:
        out.append(f"| {r['name']} | {r['n']:,} | {r['nnz']:,} | {r['w']:.2f} | {r['ms64']:.4f} | "
                   f"{r['ms32']:.4f} | {r['speedup']:.2f} | {r['model']:.2f} | {r['gbs64']:.0f} | {r['gbs32']:.0f} |")
    return "\n".join(out)


if __name__ == "__main__":
    print(table(run()))
