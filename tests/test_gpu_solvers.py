"""Solver parity on the GPU: FP64 GMRES(m) and GMRES-IR through the C ABI against the CPU
oracle on the same seeded systems, plus the status/edge cases of the boundary."""
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


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def small():
    return gen.config_small_2d()  # 64 x 64, Pe 10, manufactured solution


def _dev(torch, *arrs):
    return [torch.tensor(a, dtype=torch.float64, device="cuda") for a in arrs]


def _relres(p, b, x):
    return np.linalg.norm(b - oracle.spmv(p, x)) / np.linalg.norm(b)


def test_fp64_gmres_small(g, torch, small):
    p, b, x_true = small
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    res = g.gmres_solve(A, bt, xt, restart_m=50, rtol=1e-10)
    x = xt.cpu().numpy()
    xo, io = oracle.gmres(p, b, m=50, rtol=1e-10)
    assert res.status == g.OK
    assert res.relres <= 1e-10 and _relres(p, b, x) <= 1.0001e-10
    assert abs(res.relres - _relres(p, b, x)) <= 1e-14
    assert abs(res.iters - io.iters) <= 50
    assert res.outer == io.outer or abs(res.outer - io.outer) <= 1


def test_ir_fp32_small_matches_oracle(g, torch, small):
    p, b, x_true = small
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    res = g.gmres_ir_solve(A, bt, xt, restart_m=50, rtol=1e-10, inner_prec="fp32")
    x = xt.cpu().numpy()
    xo, io = oracle.gmres_ir(p, b, m=50, rtol=1e-10, inner="fp32")
    assert res.status == g.OK and res.relres <= 1e-10
    assert _relres(p, b, x) <= 1.0001e-10
    assert res.iters % 50 == 0  # outer test only at a restart (Section 3.2)
    assert abs(res.iters - io.iters) <= 50
    x64, i64 = oracle.gmres(p, b, m=50, rtol=1e-10)
    assert i64.iters <= res.iters <= i64.iters + 100  # IR tracks FP64 GMRES (Section 5.2)


@pytest.mark.parametrize("kind,prec,rtol", [("gmres", "fp64", 1e-13), ("ir", "fp32", 1e-12)])
def test_solution_parity_to_1e8(g, torch, small, kind, prec, rtol):
    """x agrees with the oracle's FP64 solution to 1e-8 when both are solved to a residual
    that makes kappa * rtol < 1e-8 (kappa ~ 2e3 here)."""
    p, b, x_true = small
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    fn = g.gmres_solve if kind == "gmres" else g.gmres_ir_solve
    res = fn(A, bt, xt, restart_m=50, rtol=rtol, inner_prec=prec if prec != "fp64" else "fp32")
    assert res.status == g.OK
    xo, io = oracle.gmres(p, b, m=50, rtol=1e-13)
    x = xt.cpu().numpy()
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8
    assert np.linalg.norm(x - x_true) / np.linalg.norm(x_true) <= 1e-8


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_ir_half_storage(g, torch, prec):
    p, b, x_true = gen.config_small_2d(48)
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    res = g.gmres_ir_solve(A, bt, xt, restart_m=30, rtol=1e-10, inner_prec=prec)
    assert res.status == g.OK and res.relres <= 1e-10
    assert res.iters % 30 == 0
    assert _relres(p, b, xt.cpu().numpy()) <= 1.0001e-10
    _, io = oracle.gmres_ir(p, b, m=30, rtol=1e-10, inner=prec)
    assert abs(res.iters - io.iters) <= 2 * 30 + io.iters // 4


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_ir_half_storage_solution_matches_oracle(g, torch, prec):
    """GMRES-IR with FP16/BF16 storage reaches the FP64 solution: solved to 1e-12 on the
    48 x 48 system (kappa ~ 1e3, so kappa * 1e-12 < 1e-8), x agrees with the oracle's
    emulated GMRES-IR of the same storage precision, with the oracle's FP64 GMRES solved to
    1e-13 and with the manufactured solution, each to 1e-8 (Algorithm 2: the refinement
    recovers FP64 accuracy whatever the inner storage)."""
    p, b, x_true = gen.config_small_2d(48)
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    res = g.gmres_ir_solve(A, bt, xt, restart_m=30, rtol=1e-12, inner_prec=prec)
    assert res.status == g.OK and res.relres <= 1e-12
    x = xt.cpu().numpy()
    assert _relres(p, b, x) <= 1.0001e-12
    x_ir, i_ir = oracle.gmres_ir(p, b, m=30, rtol=1e-12, inner=prec)
    x_64, _ = oracle.gmres(p, b, m=30, rtol=1e-13)
    for ref in (x_ir, x_64, x_true):
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-8
    assert abs(res.iters - i_ir.iters) <= 2 * 30 + i_ir.iters // 4


def test_ir_inner_tolerance(g, torch, small):
    p, b, _ = small
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    res = g.gmres_ir_solve(A, bt, xt, restart_m=50, rtol=1e-10, inner_rtol=1e-2)
    assert res.status == g.OK and res.relres <= 1e-10
    assert res.iters < res.outer * 50


def test_plan_reuse_is_deterministic_and_matches_one_shot(g, torch, small):
    p, b, _ = small
    A = g.DeviceCSR.from_problem(p)
    plan = g.Plan(A, "ir", restart_m=40, rtol=1e-10)
    outs = []
    for _ in range(2):
        bt, xt = _dev(torch, b, np.zeros(p.n))
        r = plan.solve(bt, xt)
        assert r.status == g.OK
        outs.append((r.iters, xt.cpu().numpy()))
    assert outs[0][0] == outs[1][0]
    np.testing.assert_array_equal(outs[0][1], outs[1][1])  # bitwise reproducible
    bt, xt = _dev(torch, b, np.zeros(p.n))
    r = g.gmres_ir_solve(A, bt, xt, restart_m=40, rtol=1e-10)
    np.testing.assert_array_equal(xt.cpu().numpy(), outs[0][1])
    # a second right-hand side on the same plan
    b2 = oracle.spmv(p, np.ones(p.n))
    bt, xt = _dev(torch, b2, np.zeros(p.n))
    r2 = plan.solve(bt, xt)
    assert r2.status == g.OK and _relres(p, b2, xt.cpu().numpy()) <= 1.0001e-10
    plan.close()


def test_host_pointer_api(g, torch, small):
    p, b, _ = small
    x = np.zeros(p.n)
    r = g.gmres_ir_solve_host(p.row_ptr, p.col_idx, p.vals, b, x, restart_m=50)
    assert r.status == g.OK and _relres(p, b, x) <= 1.0001e-10
    x2 = np.zeros(p.n)
    r2 = g.gmres_solve_host(p.row_ptr, p.col_idx, p.vals, b, x2, restart_m=50)
    assert r2.status == g.OK and _relres(p, b, x2) <= 1.0001e-10


def test_history_records_every_step(g, torch, small):
    p, b, _ = small
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    r = g.gmres_solve(A, bt, xt, restart_m=50, record_history=1, max_iters=5000)
    assert len(r.history) == r.iters
    _, io = oracle.gmres(p, b, m=50)
    h = r.history[:50]
    assert np.all(np.diff(h) <= 1e-15)  # GMRES residual is monotone within a cycle
    np.testing.assert_allclose(h[:20], np.array(io.inner_hist[:20]), rtol=1e-8)


# ------------------------------------------------------------ edge cases ----

def test_zero_rhs_gives_zero(g, torch, small):
    p, _, _ = small
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, np.zeros(p.n), np.ones(p.n))
    r = g.gmres_ir_solve(A, bt, xt)
    assert r.status == g.OK and not xt.any().item()


def test_nonfinite_input(g, torch, small):
    p, b, _ = small
    A = g.DeviceCSR.from_problem(p)
    bb = b.copy()
    bb[17] = np.nan
    for fn in (g.gmres_solve, g.gmres_ir_solve):
        bt, xt = _dev(torch, bb, np.zeros(p.n))
        assert fn(A, bt, xt).status == g.NONFINITE
    vals = p.vals.copy()
    vals[5] = np.inf
    A2 = g.DeviceCSR(p.row_ptr, p.col_idx, vals, p.n)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    assert g.gmres_ir_solve(A2, bt, xt).status == g.NONFINITE


def test_iteration_cap(g, torch, small):
    p, b, _ = small
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    r = g.gmres_solve(A, bt, xt, restart_m=5, max_iters=7, rtol=1e-14)
    _, io = oracle.gmres(p, b, m=5, max_iters=7, rtol=1e-14)
    assert r.status == g.NOT_CONVERGED == io.status and r.iters == 7 == io.iters
    assert r.relres == pytest.approx(io.relres, rel=1e-9)


def test_refinement_step_cap(g, torch, small):
    """max_outer caps the cycles: GMRES-IR stops after that many refinement steps (and FP64
    GMRES after that many restarts) with NOT_CONVERGED and the oracle's iterate after the
    same number of steps."""
    p, b, _ = small
    A = g.DeviceCSR.from_problem(p)
    for fn, kind in ((g.gmres_ir_solve, "ir"), (g.gmres_solve, "gmres")):
        bt, xt = _dev(torch, b, np.zeros(p.n))
        r = fn(A, bt, xt, restart_m=10, max_outer=2, rtol=1e-12)
        assert r.status == g.NOT_CONVERGED and r.outer == 2 and r.iters == 20, (kind, r)
        if kind == "ir":
            _, io = oracle.gmres_ir(p, b, m=10, max_iters=20, rtol=1e-12, inner="fp32")
        else:
            _, io = oracle.gmres(p, b, m=10, max_iters=20, rtol=1e-12)
        assert io.iters == 20 and r.relres == pytest.approx(io.relres, rel=1e-3)
        assert _relres(p, b, xt.cpu().numpy()) == pytest.approx(r.relres, rel=1e-6)


def test_singular_breakdown_and_tiny_systems(g, torch):
    S = gen.Problem("diag10", 2, np.array([0, 1, 1], np.int32), np.array([0], np.int32),
                    np.array([1.0]))
    A = g.DeviceCSR.from_problem(S)
    bt, xt = _dev(torch, np.array([1.0, 1.0]), np.zeros(2))
    assert g.gmres_solve(A, bt, xt, restart_m=2).status == g.BREAKDOWN
    assert oracle.gmres(S, np.array([1.0, 1.0]), m=2)[1].status == oracle.BREAKDOWN
    one = gen.Problem("one", 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    A1 = g.DeviceCSR.from_problem(one)
    bt, xt = _dev(torch, np.array([6.0]), np.zeros(1))
    r = g.gmres_ir_solve(A1, bt, xt)  # each cycle ends by a lucky breakdown after one step
    assert r.status == g.OK and r.iters <= 3 and xt.item() == pytest.approx(2.0, rel=1e-12)
    r = g.gmres_solve(A1, bt, xt.zero_())
    assert r.status == g.OK and r.iters == 1 and xt.item() == pytest.approx(2.0, rel=1e-15)


def test_identity_and_k_distinct_eigenvalues(g, torch):
    d = np.repeat([1.0, 2.0, 5.0, 7.0, 11.0], 700)
    n = d.size
    D = gen.Problem("diag", n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    A = g.DeviceCSR.from_problem(D)
    b = np.random.default_rng(3).uniform(1, 2, n)
    bt, xt = _dev(torch, b, np.zeros(n))
    r = g.gmres_solve(A, bt, xt, restart_m=30, rtol=1e-12)
    assert r.status == g.OK and r.iters == 5
    np.testing.assert_allclose(xt.cpu().numpy(), b / d, rtol=1e-11)
    I = gen.Problem("eye", n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    bt, xt = _dev(torch, b, np.zeros(n))
    r = g.gmres_solve(g.DeviceCSR.from_problem(I), bt, xt)
    assert r.iters == 1 and np.allclose(xt.cpu().numpy(), b, rtol=1e-15)


def test_invalid_csr_rejected(g, torch, small):
    p, b, _ = small
    cols = p.col_idx.copy()
    cols[3] = p.n + 5
    A = g.DeviceCSR(p.row_ptr, cols, p.vals, p.n)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    with pytest.raises(g.GmresError) as e:
        g.gmres_ir_solve(A, bt, xt)
    assert e.value.code == g.ERR_INVALID


# ------------------------------------------------------- full-size case ----

@pytest.fixture(scope="module")
def cube():
    return gen.config_3d(10.0)  # 100^3, 1M unknowns, 6.94M nonzeros


def test_full_size_3d_ir_and_fp64(g, torch, cube):
    """The benchmark's workload and launch configuration: both solvers reach 1e-10; the
    explicit residual is recomputed by the oracle's SpMV; IR iterations are multiples of m."""
    p, b = cube
    A = g.DeviceCSR.from_problem(p)
    out = {}
    for kind in ("ir", "gmres"):
        plan = g.Plan(A, kind, restart_m=50, rtol=1e-10, inner_prec="fp32", max_iters=20000)
        bt, xt = _dev(torch, b, np.zeros(p.n))
        r = plan.solve(bt, xt)
        x = xt.cpu().numpy()
        assert r.status == g.OK, (kind, r)
        assert _relres(p, b, x) <= 1.0001e-10
        out[kind] = (r, x)
        plan.close()
    assert out["ir"][0].iters % 50 == 0
    assert out["ir"][0].iters <= out["gmres"][0].iters + 150
    xi, xg = out["ir"][1], out["gmres"][1]
    assert np.linalg.norm(xi - xg) / np.linalg.norm(xg) <= 1e-6
    # the oracle's own full solve of this instance (recorded by oracle/record_iterations.py):
    # the same number of refinement steps and of inner iterations, and the final explicit
    # residual to 1% (the two sum in different orders)
    import json
    import os
    rec = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                       "iterations_3d100.json")
    ref = json.load(open(rec))["pe10"]
    r = out["ir"][0]
    assert (r.iters, r.outer) == (ref["iters"], ref["outer"])
    assert r.relres == pytest.approx(ref["relres"], rel=1e-2)


def test_ir_gives_up_on_stalled_refinement():
    """The stall rule of the oracle (no 0.1% progress in IR_STALL_LIMIT refinement steps):
    GMRES(1) cannot reduce the residual of a 90-degree rotation."""
    import paper_2109_01232_b300 as g
    import torch
    from oracle.gmres import IR_STALL_LIMIT
    A = gen.Problem("rot", 2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32),
                    np.array([1.0, -1.0]))
    b = torch.tensor([1.0, 0.0], device="cuda", dtype=torch.float64)
    x = torch.zeros(2, device="cuda", dtype=torch.float64)
    r = g.gmres_ir_solve(g.DeviceCSR.from_problem(A), b, x, restart_m=1, rtol=1e-10)
    assert r.status == g.NOT_CONVERGED and r.outer == IR_STALL_LIMIT and r.iters == IR_STALL_LIMIT
    batch = g.DeviceBatch([A, A])
    bb = torch.tensor([1.0, 0.0, 0.0, 2.0], device="cuda", dtype=torch.float64)
    xb = torch.zeros_like(bb)
    res = g.BatchPlan(batch, autotune=False, restart_m=1).solve(bb, xb)
    assert list(res.status) == [g.NOT_CONVERGED] * 2 and list(res.outer) == [IR_STALL_LIMIT] * 2


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_resume_from_a_checkpoint_equals_one_solve(g, torch, prec):
    """The IR state is x alone: a solve stopped by the iteration cap at a cycle boundary and
    called again from its x (the remaining budget) takes the same steps as one solve, and
    ends at the same x (every refinement step starts from the FP64 residual of x)."""
    p = gen.conv_diff_3d(24, 10.0, (0.6, 0.8, 0.0))
    b = gen.rhs_ones(p)
    A = g.DeviceCSR.from_problem(p)
    bt, x1 = _dev(torch, b, np.zeros(p.n))
    one = g.gmres_ir_solve(A, bt, x1, restart_m=25, inner_prec=prec)
    assert one.status == g.OK and one.outer >= 3
    cut = 25 * (one.outer // 2)
    x2 = torch.zeros_like(x1)
    first = g.gmres_ir_solve(A, bt, x2, restart_m=25, inner_prec=prec, max_iters=cut)
    assert first.status == g.NOT_CONVERGED and first.iters == cut
    rest = g.gmres_ir_solve(A, bt, x2, restart_m=25, inner_prec=prec,
                            max_iters=100000 - cut)
    assert rest.status == g.OK
    assert first.iters + rest.iters == one.iters
    assert first.outer + rest.outer == one.outer
    np.testing.assert_allclose(x2.cpu().numpy(), x1.cpu().numpy(), rtol=0, atol=1e-14 * float(
        torch.abs(x1).max()))


@pytest.mark.parametrize("graph", [False, True])
def test_profile_cycle_times_every_kernel_of_one_cycle(g, torch, graph):
    """The per-kernel profile of one restart cycle (kernel by kernel, or inside a captured
    graph with event-record nodes): every kernel of the steps the cycle took has a positive
    time, the steps it did not reach are -1, and the cycle computes what a solve computes
    (the next profile of the same plan gives the same step count)."""
    p, b, _ = gen.config_small_2d(48)
    A = g.DeviceCSR.from_problem(p)
    bt, x0 = _dev(torch, b, np.zeros(p.n))
    for m, inner_rtol in ((20, 0.0), (40, 1e-2)):  # the second cycle ends early
        plan = g.Plan(A, "ir", restart_m=m, inner_rtol=inner_rtol)
        ms = plan.profile_cycle(bt, x0, graph=graph)
        assert ms.shape == (m + 1, 3)
        ran = ms[:-1, 0] >= 0
        k = int(ran.sum())
        assert k >= 1 and ran[:k].all() and not ran[k:].any()
        assert (ms[:k] > 0).all() and (ms[:-1][~ran] == -1).all() and (ms[-1] > 0).all()
        if inner_rtol == 0.0:
            assert k == m
        else:
            assert k < m
        ms2 = plan.profile_cycle(bt, x0, graph=graph)
        assert int((ms2[:-1, 0] >= 0).sum()) == k
        plan.close()


def test_time_cycle_matches_the_profiled_cycle(g, torch):
    """The uninstrumented cycle timer runs the same cycle as the per-kernel profile (same
    step count, the full m here and fewer with an inner tolerance) and, for a full cycle,
    takes less time than the sum of the per-kernel event intervals, whose event nodes sit
    between the kernels.  (A cycle that ends early still launches the remaining steps'
    kernels, which return at once: the uninstrumented time includes them, the profile
    reports -1 for them.)"""
    p, b, _ = gen.config_small_2d(48)
    A = g.DeviceCSR.from_problem(p)
    bt, x0 = _dev(torch, b, np.zeros(p.n))
    for m, inner_rtol in ((20, 0.0), (40, 1e-2)):
        plan = g.Plan(A, "ir", restart_m=m, inner_rtol=inner_rtol)
        ms = plan.profile_cycle(bt, x0, graph=True)
        k = int((ms[:-1, 0] >= 0).sum())
        t, steps = plan.time_cycle(bt, x0)
        assert steps == k and (k == m) == (inner_rtol == 0.0)
        assert t > 0.0
        if k == m:
            assert t < ms.sum()
        plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_ir_with_long_range_columns(g, torch, prec):
    """A matrix whose columns lie up to n - 1 away from the diagonal (the SELL copy's column
    entries span the whole index range): GMRES-IR solves it to 1e-10 and agrees with the
    oracle's FP64 GMRES."""
    n = 40000
    r = np.random.default_rng(10)
    cols = np.sort(np.concatenate([r.integers(0, n, (n, 5)), np.arange(n)[:, None]], axis=1), axis=1)
    vals = r.standard_normal((n, 6))
    vals[cols == np.arange(n)[:, None]] = 8.0
    p = gen.Problem("wide", n, np.arange(0, 6 * n + 1, 6, dtype=np.int32),
                    cols.ravel().astype(np.int32), vals.ravel())
    assert np.abs(cols - np.arange(n)[:, None]).max() > 32767
    b = np.ones(n)
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(n))
    res = g.gmres_ir_solve(A, bt, xt, restart_m=30, rtol=1e-10, inner_prec=prec)
    assert res.status == g.OK and res.relres <= 1e-10
    xo, _ = oracle.gmres(p, b, m=30, rtol=1e-12)
    x = xt.cpu().numpy()
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8
