"""The allocation-free FP64 SpMV (gmres_spmv_fp64_noalloc).

Callers whose device memory is owned by another allocator, or that must not trigger the
implicit synchronisation of cudaMalloc, use the entry point that keeps its scratch in a
fixed device array.  Its result is checked against the oracle's CSR product (row by row
against |A||v|, the SpMV tolerance of the kernel tests) and against the plan-based SpMV,
on two calls in a row.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle

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


def _check_rowwise(p, v, y, tol=1e-13):
    y_ref = oracle.spmv(p, v)
    absA = oracle.spmv(p, np.abs(v), np.abs(p.vals))  # (|A| |v|) per row
    assert np.all(np.abs(y - y_ref) <= tol * absA)


def test_noalloc_spmv_matches_oracle_twice_in_a_row(g):
    import torch
    cases = [gen.conv_diff_3d(23, 10.0, (1.0, 0.5, -0.2)),   # n = 12,167: several tiles + tail
             gen.conv_diff_2d(81, 40.0, (0.3, 0.9))]          # n = 6,561, a second call
    for k, p in enumerate(cases):
        A = g.DeviceCSR.from_problem(p)
        vh = np.random.default_rng(k).uniform(-1, 1, p.n)
        v = torch.tensor(vh, device="cuda")
        y = torch.full((p.n,), np.nan, dtype=torch.float64, device="cuda")
        g.spmv_fp64_noalloc(A, v, y)
        yn = y.cpu().numpy()
        assert np.isfinite(yn).all()  # every row written (y started as NaN)
        _check_rowwise(p, vh, yn)
        rn = _plan_spmv(g, A, v).cpu().numpy()
        absA = oracle.spmv(p, np.abs(vh), np.abs(p.vals))
        assert np.all(np.abs(yn - rn) <= 1e-13 * absA)


def test_noalloc_spmv_in_place(g):
    """y may be v itself: the entry point multiplies a staged copy of v."""
    import torch
    p = gen.conv_diff_2d(90, 5.0, (1.0, 0.0))
    A = g.DeviceCSR.from_problem(p)
    vh = np.random.default_rng(3).uniform(-1, 1, p.n)
    v = torch.tensor(vh, device="cuda")
    g.spmv_fp64_noalloc(A, v, v)
    _check_rowwise(p, vh, v.cpu().numpy())


def test_noalloc_rejects_a_malformed_csr_and_leaves_y_untouched(g):
    """The structure check runs on the device before the product; a column index out of
    range or a decreasing row pointer gives GMRES_ERR_INVALID and y keeps its contents."""
    import torch
    p = gen.conv_diff_2d(40, 5.0, (1.0, 0.0))
    v = torch.ones(p.n, dtype=torch.float64, device="cuda")
    bad_col = p.col_idx.copy()
    bad_col[17] = p.n  # one past the last column
    bad_rp = p.row_ptr.copy()
    bad_rp[5] = bad_rp[6] + 1  # row_ptr decreases between rows 5 and 6
    for rp, ci in ((p.row_ptr, bad_col), (bad_rp, p.col_idx)):
        A = g.DeviceCSR(rp, ci, p.vals, n=p.n)
        y = torch.full((p.n,), 7.0, dtype=torch.float64, device="cuda")
        with pytest.raises(g.GmresError) as e:
            g.spmv_fp64_noalloc(A, v, y)
        assert e.value.code == g.ERR_INVALID
        assert bool((y == 7.0).all())
    # a well-formed call right after works (the shared state starts clean every call)
    A = g.DeviceCSR.from_problem(p)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    g.spmv_fp64_noalloc(A, v, y)
    _check_rowwise(p, np.ones(p.n), y.cpu().numpy())


def test_noalloc_rejects_sizes_beyond_the_limit(g):
    c = g.csr_t(g.NOALLOC_MAX_N + 1, 1, 1, 1, 1)
    assert g.lib().gmres_spmv_fp64_noalloc(ctypes.byref(c), 1, 1, None) == g.ERR_TOO_LARGE
