"""Record the oracle's own iteration counts on the 100^3 convection-diffusion workload.

TEST INFRASTRUCTURE ONLY.  Runs oracle.gmres_ir (FP32 inner GMRES(50), outer tolerance
1e-10) to convergence on the seeded 100^3 instance(s) and writes
oracle/iterations_3d100.json.  The CPU-baseline legs of bench.py time a bounded sample of
oracle iterations and scale it to a time-to-solution with these counts.

    python -m oracle.record_iterations [--peclet 10] [--out oracle/iterations_3d100.json]
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
    ap.add_argument("--out", default=os.path.join(HERE, "iterations_3d100.json"))
    args = ap.parse_args()
    data = json.load(open(args.out)) if os.path.exists(args.out) else {}
    for pe in args.peclet:
        p, b = gen.config_3d(pe)
        t0 = time.time()
        x, info = oracle.gmres_ir(p, b, m=50, rtol=1e-10, inner="fp32")
        data[f"pe{pe:g}"] = dict(method="gmres_ir fp32 inner, m=50, rtol=1e-10",
                                 status=info.status, iters=info.iters, outer=info.outer,
                                 relres=info.relres, seconds=time.time() - t0,
                                 threads=os.environ.get("OPENBLAS_NUM_THREADS", "default"))
        json.dump(data, open(args.out, "w"), indent=1)
        print(pe, data[f"pe{pe:g}"], flush=True)


if __name__ == "__main__":
    main()
