"""Block-Jacobi preconditioner with reverse Cuthill-McKee reordering (Section 5.8) on the
GPU against the oracle: the plan's permutation, M^{-1} v block by block, and the
preconditioned FP64 GMRES and GMRES-IR solves."""
import numpy as np
import pytest

import gen
import oracle
from oracle import precond as pc

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


def _problem(which):
    # badly scaled, shuffled: the structure of the block-Jacobi workloads at test size
    if which == "box3d":  # n = 1728, 27 per row, SPD
        return gen.shuffled(gen.scaled(gen.box_3d(12), 1.0, 3), 3)
    return gen.shuffled(gen.scaled(gen.conv_diff_2d(37, 30.0, (0.6, 0.8)), 1.0, 4), 4)


# (inner working precision, tolerance on max|y - y_ref| / max|y_ref|)
PRECS = [("fp64", "gmres", 1e-12), ("fp32", "ir", 2e-5), ("bf16", "ir", 2e-5)]


@pytest.mark.parametrize("which", ["box3d", "convdiff"])
@pytest.mark.parametrize("k", [1, 5, 32, 42, 64])
@pytest.mark.parametrize("prec,kind,tol", PRECS)
def test_bj_apply_matches_oracle(g, torch, which, k, prec, kind, tol):
    p = _problem(which)
    A = g.DeviceCSR.from_problem(p)
    kw = dict(restart_m=10, bj_block=k, bj_rcm=1)
    if kind == "ir":
        kw["inner_prec"] = prec
    plan = g.Plan(A, kind, **kw)
    perm = plan.perm()
    np.testing.assert_array_equal(perm, pc.rcm(p.n, p.row_ptr, p.col_idx))
    B = pc.permute(p, perm)
    v = oracle.splitmix64_uniform(21 + k, p.n)
    y = plan.bj_apply(torch.tensor(v, device="cuda")).double().cpu().numpy()
    y_ref = pc.BlockJacobi(B, k).apply(v)
    assert np.abs(y - y_ref).max() <= tol * np.abs(y_ref).max()
    plan.close()


def test_bj_apply_without_reordering(g, torch):
    p = _problem("convdiff")
    plan = g.Plan(g.DeviceCSR.from_problem(p), "gmres", restart_m=10, bj_block=7)
    assert plan.perm() is None
    v = oracle.splitmix64_uniform(3, p.n)
    y = plan.bj_apply(torch.tensor(v, device="cuda")).cpu().numpy()
    y_ref = pc.BlockJacobi(p, 7).apply(v)
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    plan.close()


def test_singular_block_refused(g):
    # the first 2 x 2 block [[1, 1], [1, 1]] is singular
    rp = np.array([0, 3, 6, 8, 10], np.int32)
    ci = np.array([0, 1, 2, 0, 1, 3, 2, 3, 2, 3], np.int32)
    va = np.array([1, 1, 0.5, 1, 1, 0.5, 4, 1, 1, 4], np.float64)
    A = g.DeviceCSR(rp, ci, va)
    with pytest.raises(g.GmresError) as e:
        g.Plan(A, "gmres", restart_m=4, bj_block=2)
    assert e.value.code == g.ERR_INVALID
    g.Plan(A, "gmres", restart_m=4, bj_block=1).close()  # point Jacobi: diagonal 1, 1, 4, 4


def _orig_residual(p, x, b):
    return np.linalg.norm(b - oracle.spmv(p, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("which,k", [("box3d", 42), ("convdiff", 37)])
def test_bj_gmres_fp64_matches_oracle(g, torch, which, k):
    p = _problem(which)
    b = gen.rhs_ones(p)
    A = g.DeviceCSR.from_problem(p)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    res = g.gmres_solve(A, torch.tensor(b, device="cuda"), x, restart_m=30, bj_block=k, bj_rcm=1)
    assert res.status == g.OK and res.relres <= 1e-10
    assert _orig_residual(p, x.cpu().numpy(), b) <= 1e-10
    perm = pc.rcm(p.n, p.row_ptr, p.col_idx)
    B = pc.permute(p, perm)
    _, info = oracle.gmres(B, b[perm], m=30, rtol=1e-10, right_prec=pc.BlockJacobi(B, k).apply)
    assert info.status == oracle.OK
    assert abs(res.iters - info.iters) <= max(2, 0.03 * info.iters)
    # the unpreconditioned solve of the badly scaled matrix takes far more steps
    x.zero_()
    plain = g.gmres_solve(A, torch.tensor(b, device="cuda"), x, restart_m=30,
                          max_iters=4 * res.iters)
    assert plain.status == g.NOT_CONVERGED or plain.iters > 2 * res.iters


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_bj_gmres_ir_converges_like_oracle(g, torch, prec):
    p = _problem("box3d")
    b = np.ones(p.n)
    A = g.DeviceCSR.from_problem(p)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    res = g.gmres_ir_solve(A, torch.tensor(b, device="cuda"), x, restart_m=30, inner_prec=prec,
                           bj_block=42, bj_rcm=1)
    assert res.status == g.OK and res.relres <= 1e-10
    assert _orig_residual(p, x.cpu().numpy(), b) <= 1e-10
    perm = pc.rcm(p.n, p.row_ptr, p.col_idx)
    B = pc.permute(p, perm)
    _, info = oracle.gmres_ir(B, b[perm], m=30, rtol=1e-10, inner=prec,
                              right_prec=pc.BlockJacobi(B, 42).apply)
    assert info.status == oracle.OK
    assert abs(res.outer - info.outer) <= 1


def test_rcm_alone_keeps_the_answer(g, torch):
    # without a preconditioner: the well-scaled matrix (the scaled one needs one)
    p = gen.shuffled(gen.conv_diff_2d(37, 30.0, (0.6, 0.8)), 4)
    b = oracle.splitmix64_uniform(9, p.n)
    A = g.DeviceCSR.from_problem(p)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    res = g.gmres_ir_solve(A, torch.tensor(b, device="cuda"), x, restart_m=30, bj_rcm=1)
    assert res.status == g.OK
    xr = x.cpu().numpy()
    assert _orig_residual(p, xr, b) <= 1e-10
    x2 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    g.gmres_ir_solve(A, torch.tensor(b, device="cuda"), x2, restart_m=30)
    assert np.abs(xr - x2.cpu().numpy()).max() <= 1e-8 * np.abs(xr).max()


def test_bj_full_workload_sampled_blocks(g, torch):
    """The 216,000-row workload with k = 42 in the launch configuration of the sweep: the
    plan's permutation equals the host ordering, and sampled blocks of M^{-1} v (including
    the ragged last one) match dense FP64 solves of those blocks."""
    p, k = gen.config_bj()[0]
    A = g.DeviceCSR.from_problem(p)
    plan = g.Plan(A, "ir", restart_m=50, inner_prec="fp32", bj_block=k, bj_rcm=1)
    perm = plan.perm()
    np.testing.assert_array_equal(perm, g.rcm(p.row_ptr, p.col_idx))
    iperm = np.empty(p.n, np.int64)
    iperm[perm] = np.arange(p.n)
    v = oracle.splitmix64_uniform(5, p.n)
    y = plan.bj_apply(torch.tensor(v, device="cuda")).double().cpu().numpy()
    nb = (p.n + k - 1) // k
    for q in list(np.random.default_rng(1).choice(nb - 1, 40, replace=False)) + [nb - 1]:
        s, e = q * k, min(q * k + k, p.n)
        D = np.zeros((e - s, e - s))
        for i in range(s, e):
            o = perm[i]
            for t in range(p.row_ptr[o], p.row_ptr[o + 1]):
                j = iperm[p.col_idx[t]]
                if s <= j < e:
                    D[i - s, j - s] += p.vals[t]
        z = np.linalg.solve(D, v[s:e])
        assert np.abs(y[s:e] - z).max() <= 2e-5 * np.abs(z).max()
    plan.close()


@pytest.mark.parametrize("n,k", [(1, 1), (5, 42), (32, 32), (33, 33), (70, 64), (100, 7),
                                 (97, 32), (130, 33)])
def test_bj_apply_edge_sizes(g, torch, n, k):
    """One row; a single block smaller than k; k at the boundary of the two warp layouts
    (32: one block per warp in the packed form, 33: the two-rows-per-lane form); ragged
    tails."""
    import scipy.sparse as sp
    rng = np.random.default_rng(n * 100 + k)
    M = sp.random(n, n, density=min(1.0, 6.0 / n), random_state=n + k, format="csr")
    M = (M + sp.diags(np.abs(M).sum(axis=1).A.ravel() + 1.0 + rng.random(n))).tocsr()
    M.sort_indices()
    p = gen.Problem("edge", n, M.indptr.astype(np.int32), M.indices.astype(np.int32),
                    M.data.astype(np.float64))
    v = rng.standard_normal(n)
    for kind, tol in (("gmres", 1e-12), ("ir", 1e-5)):
        plan = g.Plan(g.DeviceCSR.from_problem(p), kind, restart_m=4, bj_block=k)
        y = plan.bj_apply(torch.tensor(v, device="cuda")).double().cpu().numpy()
        y_ref = pc.BlockJacobi(p, k).apply(v)
        assert np.abs(y - y_ref).max() <= tol * np.abs(y_ref).max()
        plan.close()
