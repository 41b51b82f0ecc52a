"""Record the exact solution of the anisotropic 2000^2 workload.

TEST INFRASTRUCTURE ONLY.  Solves the seeded 2D anisotropic convection-diffusion system
(2000 x 2000 grid, anisotropy 1e2, Peclet 100, b = ones) with the oracle's sparse direct
solve (oracle/direct.py), and writes
  oracle/aniso2000_reference.npy   x (FP64, 32 MB; not committed, rebuilt by this script)
  oracle/aniso2000_reference.json  its summary: residual, norms, SHA-256 of the array.
The anisotropic sweep measures each GPU solve's error against this x.

    python -m oracle.record_aniso_reference [--side 2000]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import time

import numpy as np

import gen
import oracle
from oracle.direct import direct_solve

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=2000)
    args = ap.parse_args()
    p, b = gen.config_aniso_2d(side=args.side)
    t0 = time.time()
    x = direct_solve(p, b)
    dt = time.time() - t0
    relres = float(np.linalg.norm(b - oracle.spmv(p, x)) / np.linalg.norm(b))
    stem = os.path.join(HERE, f"aniso{args.side}_reference")
    np.save(stem + ".npy", x)
    summary = dict(matrix=p.name, n=p.n, nnz=p.nnz, method="sparse LU (SuperLU, MMD on A+A^T)",
                   relres=relres, norm2=float(np.linalg.norm(x)),
                   norminf=float(np.abs(x).max()), sha256=hashlib.sha256(x.tobytes()).hexdigest(),
                   seconds=dt)
    json.dump(summary, open(stem + ".json", "w"), indent=1)
    print(summary, flush=True)


if __name__ == "__main__":
    main()
