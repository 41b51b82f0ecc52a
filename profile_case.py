"""One restart cycle of the solver on the 3D convection-diffusion workload, kernel by kernel.

The profiling target for ncu (`-k regex:<kernel> -s <skip> -c <count>`): plan set-up, the
FP64 residual of x0 = 0 and one cycle of m Arnoldi steps launched one kernel at a time,
printing the per-launch device times measured with CUDA events.

    python profile_case.py [--side 100] [--prec fp32] [--m 50]
        [--cgs-kernel register|tma]
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    import torch

    import gen
    import paper_2109_01232_b300 as g

    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=100)
    ap.add_argument("--prec", default="fp32", choices=list(g.PREC))
    ap.add_argument("--m", type=int, default=50)
    ap.add_argument("--peclet", type=float, default=10.0)
    ap.add_argument("--cgs-kernel", default="register", choices=list(g.CGS_KERNEL))
    args = ap.parse_args()
    p, b = gen.config_3d(args.peclet, side=args.side)
    A = g.DeviceCSR.from_problem(p)
    kind = "gmres" if args.prec == "fp64" else "ir"
    plan = g.Plan(A, kind, restart_m=args.m, inner_prec=args.prec if kind == "ir" else "fp32",
                  cgs_kernel=args.cgs_kernel)
    bt = torch.tensor(b, device="cuda")
    x0 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    ms = plan.profile_cycle(bt, x0)
    torch.cuda.synchronize()
    run = ms[:-1, 0] >= 0
    print(f"n={p.n} nnz={p.nnz} prec={args.prec} m={args.m} plan={plan.info()}")
    print(f"spmv total {ms[:-1, 0][run].sum():.3f} ms, u1 {ms[:-1, 1][run].sum():.3f} ms, "
          f"u2 {ms[:-1, 2][run].sum():.3f} ms, lsq {ms[-1, 0]:.3f}, xupd {ms[-1, 1]:.3f}, "
          f"residual {ms[-1, 2]:.3f} ms")
    np.set_printoptions(precision=4, suppress=True, linewidth=150)
    print(ms)
    plan.close()


if __name__ == "__main__":
    main()
