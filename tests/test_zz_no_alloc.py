"""The allocation-free FP64 SpMV (gmres_spmv_fp64_noalloc) against the plan-based SpMV.

Callers whose device memory is owned by another allocator, or that must not trigger the
implicit synchronisation of cudaMalloc, use the entry point that keeps its scratch in a
fixed device array.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2109_01232_b300 as lib
    lib.lib()
    return lib


def _plan_spmv(g, A, v):
    plan = g.Plan(A, "gmres", restart_m=2)
    y = plan.spmv(v)
    plan.close()
    return y


def test_noalloc_spmv_matches_plan_spmv_twice_in_a_row(g):
    import torch
    cases = [gen.conv_diff_3d(23, 10.0, (1.0, 0.5, -0.2)),   # n = 12,167: several tiles + tail
             gen.conv_diff_2d(81, 40.0, (0.3, 0.9))]          # n = 6,561, a second call
    for k, p in enumerate(cases):
        A = g.DeviceCSR.from_problem(p)
        v = torch.tensor(np.random.default_rng(k).uniform(-1, 1, p.n), device="cuda")
        y = torch.full((p.n,), np.nan, dtype=torch.float64, device="cuda")
        g.spmv_fp64_noalloc(A, v, y)
        ref = _plan_spmv(g, A, v)
        yn, rn = y.cpu().numpy(), ref.cpu().numpy()
        absA = np.abs(p.scipy()) @ np.abs(v.cpu().numpy())
        assert np.all(np.abs(yn - rn) <= 1e-13 * absA)  # the kernel tests' SpMV tolerance
        assert np.isfinite(yn).all()  # every row written (y started as NaN)


def test_noalloc_rejects_sizes_beyond_the_limit(g):
    c = g.csr_t(g.NOALLOC_MAX_N + 1, 1, 1, 1, 1)
    assert g.lib().gmres_spmv_fp64_noalloc(ctypes.byref(c), 1, 1, None) == g.ERR_TOO_LARGE
