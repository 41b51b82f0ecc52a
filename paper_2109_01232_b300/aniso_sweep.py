"""The anisotropic 2D workload: inner precision x polynomial degree sweep (Section 5.4's
experiment on this GPU).

2000^2 anisotropic convection-diffusion (eps 1e-2, Pe 100, b = ones): GMRES-IR with FP32,
FP16-storage and BF16-storage inner GMRES(50) and a right GMRES-polynomial preconditioner of
degree 10, 25 and 40, and FP64 GMRES(50) with the same polynomials; each run's explicit
relative residual and its error against an FP64 reference solution (FP64 GMRES with the
degree-40 polynomial solved to 1e-11).  Each solve is capped at 20,000 iterations.

    python -m paper_2109_01232_b300.aniso_sweep [--side 2000]
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def run(side: int = 2000, m: int = 50, rtol: float = 1e-10, max_iters: int = 20000, log=None):
    import torch

    import gen
    import paper_2109_01232_b300 as g
    p, b = gen.config_aniso_2d(side=side)
    A = g.DeviceCSR.from_problem(p)
    bt = torch.tensor(b, device="cuda")
    xr = torch.zeros_like(bt)
    ref = g.gmres_solve(A, bt, xr, restart_m=m, rtol=1e-11, poly_degree=40, seed=7,
                        max_iters=max_iters)
    nref = float(torch.linalg.norm(xr))
    rows = [dict(solver="FP64 GMRES (reference, tol 1e-11)", degree=40, status=ref.status_name,
                 iters=ref.iters, ms=ref.t_solve_ms, relres=ref.relres, err=0.0)]
    if log:
        log(rows[-1])
    for d in (10, 25, 40):
        runs = [("FP64 GMRES", g.gmres_solve, {})] + [
            (f"GMRES-IR {pr.upper()} inner", g.gmres_ir_solve, dict(inner_prec=pr))
            for pr in ("fp32", "fp16", "bf16")]
        for name, fn, kw in runs:
            x = torch.zeros_like(bt)
            r = fn(A, bt, x, restart_m=m, rtol=rtol, poly_degree=d, seed=7, max_iters=max_iters, **kw)
            err = float(torch.linalg.norm(x - xr)) / nref
            rows.append(dict(solver=name, degree=d, status=r.status_name, iters=r.iters,
                             ms=r.t_solve_ms, relres=r.relres, err=err))
            if log:
                log(rows[-1])
    return p, rows


def table(p, rows) -> str:
    out = [f"Matrix {p.name}: n = {p.n:,}, nnz = {len(p.vals):,}; m = 50, rtol 1e-10, x0 = 0, b = ones.", "",
           "| solver | poly degree | status | iterations | solve ms | explicit relres | ||x - x_ref|| / ||x_ref|| |",
           "|---|---:|---|---:|---:|---:|---:|"]
    for r in rows:
        out.append(f"| {r['solver']} | {r['degree']} | {r['status']} | {r['iters']} | {r['ms']:.1f} | "
                   f"{r['relres']:.2e} | {r['err']:.2e} |")
    return "\n".join(out)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=2000)
    a = ap.parse_args()
    p, rows = run(a.side, log=lambda r: print(r, file=sys.stderr, flush=True))
    print(table(p, rows))
