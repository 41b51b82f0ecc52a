"""FP64 and FP32 arithmetic rates of this GPU, for the roofline of the FP64 GMRES baseline.

CGS2 in FP64 does 8 j n flop per Arnoldi step over 3 j n 8 bytes of basis reads (the fused
kernels read V three times): 1/3 flop per byte.  To run at the HBM copy bandwidth it needs
(copy GB/s) / 3 GFLOP/s of FP64.  This script measures the FP64 rate with a cuBLAS DGEMM
(8192^3, CUDA events, best of 5 after a warm-up; a library GEMM is the highest FP64 rate a
kernel can expect) and the FP32 SGEMM rate for comparison, and prints which bound applies.

    python fp64_rate.py
"""
from __future__ import annotations

import json
import os


def gemm_tflops(dtype, n: int = 8192, reps: int = 5) -> float:
    import torch
    a = torch.randn(n, n, dtype=dtype, device="cuda")
    b = torch.randn(n, n, dtype=dtype, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


def main():
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    f64 = gemm_tflops(torch.float64)
    f32 = gemm_tflops(torch.float32)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(root, "MEASURED_PEAKS.json")) as f:
            hbm = float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        hbm = 6400.0
    need = hbm / 3.0 / 1e3  # TFLOP/s of FP64 for CGS2 at the copy bandwidth
    out = dict(dgemm_tflops=round(f64, 3), sgemm_tflops_no_tf32=round(f32, 3), hbm_gbs=hbm,
               fp64_cgs2_needs_tflops=round(need, 3),
               fp64_cgs2_bound="fp64 alu" if f64 < need else "hbm",
               fp64_cgs2_max_frac_of_hbm=round(min(1.0, f64 / need), 3))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
