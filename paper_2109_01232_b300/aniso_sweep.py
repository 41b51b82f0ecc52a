"""The anisotropic 2D workload: inner precision x polynomial degree sweep (Section 5.4's
experiment on this GPU).

2000^2 anisotropic convection-diffusion (eps 1e-2, Pe 100, b = ones): for polynomial
degrees 10, 25 and 40, the three configurations of Section 5.4 -- FP64 GMRES(50) with the
polynomial in FP64, FP64 GMRES(50) with the polynomial applied in FP32, GMRES-IR with an
FP32 inner cycle (polynomial in FP32) -- and GMRES-IR with FP16 and BF16 storage.  Each
run reports its explicit relative residual and its error against the exact solution that
the oracle's sparse direct solve wrote to oracle/aniso<side>_reference.npy (checked
against the SHA-256 in oracle/aniso<side>_reference.json; make it with
`python -m oracle.record_aniso_reference`).  Each solve is capped at 20,000 iterations.

    python -m paper_2109_01232_b300.aniso_sweep [--side 2000]
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def reference_solution(side: int) -> np.ndarray:
    """The exact solution recorded by the oracle's direct solve, verified by its hash."""
    import hashlib
    import json
    stem = os.path.join(ROOT, "oracle", f"aniso{side}_reference")
    if not (os.path.exists(stem + ".npy") and os.path.exists(stem + ".json")):
        raise SystemExit(f"{stem}.npy is missing: run `python -m oracle.record_aniso_reference "
                         f"--side {side}` first")
    x = np.load(stem + ".npy")
    if hashlib.sha256(x.tobytes()).hexdigest() != json.load(open(stem + ".json"))["sha256"]:
        raise SystemExit(f"{stem}.npy does not match its recorded hash")
    return x


def run(side: int = 2000, m: int = 50, rtol: float = 1e-10, max_iters: int = 20000, log=None,
        x_ref: np.ndarray | None = None):
    """x_ref: the exact solution (default: the recorded one for this side)."""
    import torch

    import gen
    import paper_2109_01232_b300 as g
    p, b = gen.config_aniso_2d(side=side)
    xr = torch.tensor(reference_solution(side) if x_ref is None else x_ref, device="cuda")
    nref = float(torch.linalg.norm(xr))
    A = g.DeviceCSR.from_problem(p)
    bt = torch.tensor(b, device="cuda")
    rows = []
    for d in (10, 25, 40):
        runs = [("FP64 GMRES, FP64 polynomial", g.gmres_solve, {}),
                ("FP64 GMRES, FP32 polynomial", g.gmres_solve, dict(poly_in_fp32=1))] + [
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
           "| solver | poly degree | status | iterations | solve ms | explicit relres | ||x - x*|| / ||x*|| (x*: oracle's exact solve) |",
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
