"""GMRES-FD switch-point sweep (Section 5.1's experiment on this GPU).

GMRES-FD runs FP32 GMRES(m) up to a restart and then FP64 GMRES(m) from that iterate
(Section 3.3).  For each problem this driver times, to the same 1e-10 relative residual
from x0 = 0 and b = ones:
  * FP64 GMRES(m) and GMRES-IR (FP32 inner GMRES(m)), one run each;
  * FP32 GMRES(m) alone with its per-iteration residual estimates, to find where single
    precision stops making progress (the last useful switch point);
  * GMRES-FD switching at restart multiples: a coarse grid from m up to a few cycles past
    that point, then every restart within two cycles of the best coarse point.
Device time of each solve (plan set-up excluded, as for the other solvers).

Problems: the paper's two, with seeded stand-ins for its Galeri matrices: a 7-point 3D
Laplacian on a 200^3 grid (8.0M rows) and a UniFlow2D-like 5-point convection-diffusion
(uniform diagonal wind, Peclet 100) on a 2500^2 grid (6.25M rows).

    python -m paper_2109_01232_b300.fd_sweep [--problem laplace3d|uniflow2d] [--side N]
        [--coarse 10] [--out profiles/fd_switch_sweep.md]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

DEFAULT_SIDE = {"laplace3d": 200, "uniflow2d": 2500}


def problem(kind: str, side: int):
    import gen
    if kind == "laplace3d":
        return gen.laplace_3d(side)
    if kind == "uniflow2d":
        return gen.uniflow_2d(side)
    raise ValueError(kind)


def stagnation_point(hist: np.ndarray, m: int, factor: float = 1.05) -> int:
    """Iteration (a restart multiple) after which the FP32 residual estimate never again
    drops below 1/factor of its value there: switching later cannot help."""
    if hist.size == 0:
        return m
    best_after = np.minimum.accumulate(hist[::-1])[::-1]  # min over iterations >= i
    for k in range(m, hist.size + 1, m):
        if best_after[k - 1] * factor >= hist[k - 1]:
            return k
    return (hist.size // m) * m


def run(kind: str, side: int, m: int = 50, rtol: float = 1e-10, coarse: int = 10,
        max_iters: int = 60000, log=print) -> dict:
    import torch

    import paper_2109_01232_b300 as g
    p = problem(kind, side)
    A = g.DeviceCSR.from_problem(p)
    b = torch.ones(p.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    kw = dict(restart_m=m, rtol=rtol, max_iters=max_iters)
    out = {"matrix": p.name, "n": p.n, "nnz": p.nnz, "m": m, "rtol": rtol}

    r = g.gmres_solve(A, b, x, **kw)
    out["fp64"] = dict(iters=r.iters, ms=r.t_solve_ms, relres=r.relres, status=r.status_name)
    log("fp64", out["fp64"])
    x.zero_()
    r = g.gmres_ir_solve(A, b, x, inner_prec="fp32", **kw)
    out["ir"] = dict(iters=r.iters, ms=r.t_solve_ms, relres=r.relres, status=r.status_name)
    log("ir", out["ir"])

    # FP32 GMRES alone: where does single precision stop making progress?
    cap = int(out["fp64"]["iters"]) + 10 * m
    plan = g.Plan(A, "fp32", restart_m=m, rtol=rtol, max_iters=cap, record_history=1)
    x.zero_()
    r32 = plan.solve(b, x)
    plan.close()
    hist = np.asarray(r32.history)
    stag = stagnation_point(hist, m)
    out["fp32"] = dict(iters=r32.iters, ms=r32.t_solve_ms, relres=r32.relres,
                       status=r32.status_name, min_estimate=float(hist.min()) if hist.size else None,
                       stagnation_iter=stag)
    log("fp32", out["fp32"])

    def fd(s: int) -> dict:
        x.zero_()
        a, bb = g.gmres_fd_solve(A, b, x, s, **kw)
        row = dict(switch=s, fp32_iters=a.iters, fp64_iters=bb.iters, iters=a.iters + bb.iters,
                   fp32_ms=a.t_solve_ms, fp64_ms=bb.t_solve_ms, ms=a.t_solve_ms + bb.t_solve_ms,
                   switch_relres=a.relres, relres=bb.relres, status=bb.status_name)
        log("fd", row)
        return row

    hi = max(m, min(stag + 4 * m, cap))
    grid = sorted({int(round(v / m)) * m for v in np.linspace(m, hi, coarse)})
    rows = {s: fd(s) for s in grid}
    best = min(rows.values(), key=lambda rr: rr["ms"])["switch"]
    for s in range(max(m, best - 2 * m), best + 3 * m, m):
        if s not in rows:
            rows[s] = fd(s)
    out["fd"] = [rows[s] for s in sorted(rows)]
    bestrow = min(out["fd"], key=lambda rr: rr["ms"])
    out["best_fd"] = bestrow
    return out


def table(res: dict) -> str:
    f64, ir, f32, best = res["fp64"], res["ir"], res["fp32"], res["best_fd"]
    lines = [f"### {res['matrix']}: n = {res['n']:,}, nnz = {res['nnz']:,}; GMRES({res['m']}), "
             f"rtol {res['rtol']:g}, x0 = 0, b = ones", "",
             f"* FP64 GMRES: {f64['iters']} iterations, {f64['ms']:.1f} ms ({f64['status']}, "
             f"relres {f64['relres']:.2e})",
             f"* GMRES-IR (FP32 inner): {ir['iters']} iterations, {ir['ms']:.1f} ms "
             f"({ir['status']}, relres {ir['relres']:.2e}) -- {f64['ms'] / ir['ms']:.2f}x FP64",
             f"* FP32 GMRES alone: smallest residual estimate {f32['min_estimate']:.2e}; no "
             f"further 5% progress after iteration {f32['stagnation_iter']}",
             f"* best GMRES-FD: switch at {best['switch']}, {best['iters']} iterations, "
             f"{best['ms']:.1f} ms -- {f64['ms'] / best['ms']:.2f}x FP64, "
             f"{ir['ms'] / best['ms']:.2f}x GMRES-IR", "",
             "| switch at | FP32 iters | FP64 iters | total iters | FP32 ms | FP64 ms | total ms | "
             "relres at switch | final relres | status |",
             "|---:|---:|---:|---:|---:|---:|---:|---:|---:|---|"]
    for rr in res["fd"]:
        lines.append(f"| {rr['switch']} | {rr['fp32_iters']} | {rr['fp64_iters']} | {rr['iters']} | "
                     f"{rr['fp32_ms']:.1f} | {rr['fp64_ms']:.1f} | {rr['ms']:.1f} | "
                     f"{rr['switch_relres']:.2e} | {rr['relres']:.2e} | {rr['status']} |")
    return "\n".join(lines)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--problem", choices=list(DEFAULT_SIDE), nargs="+", default=list(DEFAULT_SIDE))
    ap.add_argument("--side", type=int, default=0, help="grid side (default: the paper's)")
    ap.add_argument("--coarse", type=int, default=10)
    ap.add_argument("--json", default=None, help="also write the raw results here")
    a = ap.parse_args()
    results = []
    for kind in a.problem:
        res = run(kind, a.side or DEFAULT_SIDE[kind], coarse=a.coarse,
                  log=lambda *v: print(*v, file=sys.stderr, flush=True))
        results.append(res)
        print(table(res) + "\n", flush=True)
    if a.json:
        json.dump(results, open(a.json, "w"), indent=1)
