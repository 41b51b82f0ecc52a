"""Record the oracle's own iteration counts on the 100^3 convection-diffusion workload.

TEST INFRASTRUCTURE ONLY.  Runs oracle.gmres_ir (FP32 inner GMRES(50), outer tolerance
1e-10) and, with --fp64, oracle.gmres (FP64 GMRES(50), same tolerance) to convergence on
the seeded 100^3 instance(s) and writes oracle/iterations_3d100.json.  The CPU-baseline
legs of bench.py time whole oracle cycles and scale them to a time-to-solution with these
cycle counts.

    python -m oracle.record_iterations [--peclet 10] [--fp64] [--out oracle/iterations_3d100.json]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import gen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--peclet", type=float, nargs="+", default=[10.0])
    ap.add_argument("--fp64", action="store_true", help="FP64 GMRES(50) instead of GMRES-IR")
    ap.add_argument("--out", default=os.path.join(HERE, "iterations_3d100.json"))
    args = ap.parse_args()
    data = json.load(open(args.out)) if os.path.exists(args.out) else {}
    for pe in args.peclet:
        p, b = gen.config_3d(pe)
        t0 = time.time()
        if args.fp64:
            key, method = f"pe{pe:g}_fp64", "gmres fp64, m=50, rtol=1e-10"
            x, info = oracle.gmres(p, b, m=50, rtol=1e-10)
        else:
            key, method = f"pe{pe:g}", "gmres_ir fp32 inner, m=50, rtol=1e-10"
            x, info = oracle.gmres_ir(p, b, m=50, rtol=1e-10, inner="fp32")
        data[key] = dict(method=method, status=info.status, iters=info.iters, outer=info.outer,
                         relres=info.relres, seconds=time.time() - t0,
                         threads=os.environ.get("OPENBLAS_NUM_THREADS", "default"))
        json.dump(data, open(args.out, "w"), indent=1)
        print(key, data[key], flush=True)


if __name__ == "__main__":
    main()
