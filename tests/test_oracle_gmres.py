"""Pins for the oracle's GMRES(m), GMRES-IR and GMRES-FD (CPU only).

Each property comes from linear algebra or from the paper, not from the oracle
itself: dense solves and least squares, the Arnoldi relation, GMRES optimality
and finite termination, and the paper's restart-only convergence test
(Section 3.2), which makes every GMRES-IR iteration count a multiple of m.
"""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from oracle.gmres import IR_STALL_LIMIT, _fp64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


class Dense:
    """CSR view of a dense matrix (explicit zeros dropped)."""

    def __init__(self, M):
        M = np.asarray(M, dtype=np.float64)
        self.n = M.shape[0]
        rows, cols = np.nonzero(M)
        self.row_ptr = np.zeros(self.n + 1, dtype=np.int32)
        np.add.at(self.row_ptr, rows + 1, 1)
        self.row_ptr = np.cumsum(self.row_ptr).astype(np.int32)
        self.col_idx = cols.astype(np.int32)
        self.vals = M[rows, cols]


def _op(A):
    return lambda v: oracle.spmv(A, v)


# ---------------------------------------------------------------- SpMV ----

def test_spmv_matches_dense_with_empty_rows():
    g = np.random.default_rng(0)
    M = g.standard_normal((37, 37)) * (g.uniform(size=(37, 37)) < 0.2)
    M[5, :] = 0.0  # empty row
    M[20, :] = 0.0
    A = Dense(M)
    x = g.standard_normal(37)
    np.testing.assert_allclose(oracle.spmv(A, x), M @ x, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(oracle.dense(A), M)


# ----------------------------------------------------------- generator ----

def _stencil_nnz(points, side, dim):
    if points == 9:  # 2D nine-point: interior 9, edges 6, corners 4
        return 9 * side * side - 12 * side + 4
    return points * side ** dim - 2 * dim * side ** (dim - 1)


def test_paper_matrix_sizes_follow_stencil_count():
    """The paper's printed n / nnz (Table 4) obey the Dirichlet stencil count that the
    generator's structure follows."""
    data = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    for m in data["matrices"]:
        assert m["n"] == m["side"] ** m["dim"]
        assert m["nnz"] == _stencil_nnz(m["points"], m["side"], m["dim"]), m["name"]


@pytest.mark.parametrize("side", [1, 2, 3, 7, 64])
def test_generator_2d_structure(side):
    p = gen.conv_diff_2d(side, 5.0, (0.6, 0.8))
    assert p.n == side * side
    assert p.nnz == _stencil_nnz(5, side, 2)
    M = oracle.dense(p)
    off = M - np.diag(np.diag(M))
    assert (off <= 0).all()  # M-matrix sign pattern
    assert (np.diag(M) >= -off.sum(axis=1) - 1e-12).all()  # weak diagonal dominance
    for i in range(p.n):  # sorted columns
        c = p.col_idx[p.row_ptr[i]:p.row_ptr[i + 1]]
        assert (np.diff(c) > 0).all()


@pytest.mark.parametrize("side", [1, 2, 5, 12])
def test_generator_3d_structure(side):
    p = gen.conv_diff_3d(side, 3.0, (1.0, 2.0, 2.0))
    assert p.nnz == _stencil_nnz(7, side, 3)
    M = oracle.dense(p)
    off = M - np.diag(np.diag(M))
    assert (off <= 0).all()


def test_generator_laplacian_is_the_textbook_stencil():
    p = gen.conv_diff_2d(4)  # Pe = 0: h^2 * (-Laplacian) = 5-point stencil 4, -1
    M = oracle.dense(p)
    T = 2 * np.eye(4) - np.eye(4, k=1) - np.eye(4, k=-1)
    np.testing.assert_allclose(M, np.kron(np.eye(4), T) + np.kron(T, np.eye(4)), atol=1e-15)
    assert p.meta["cell_peclet"] == 0.0


def test_generator_upwind_coefficients():
    h = 1.0 / 11
    p = gen.conv_diff_2d(10, 10.0, (1.0, 0.0))
    M = oracle.dense(p)
    i = 5 + 10 * 5
    assert M[i, i] == pytest.approx(4.0 + h * 10.0)
    assert M[i, i - 1] == pytest.approx(-1.0 - h * 10.0)  # upwind side
    assert M[i, i + 1] == pytest.approx(-1.0)
    assert M[i, i - 10] == pytest.approx(-1.0)


# ------------------------------------------------------------- Arnoldi ----

def test_arnoldi_relation_and_orthogonality_fp64():
    p = gen.conv_diff_2d(20, 20.0, (0.3, 1.0))
    A = oracle.dense(p)
    v0 = np.random.default_rng(1).standard_normal(p.n)
    V, H, k = oracle.arnoldi(_op(p), v0, 40)
    assert k == 40
    nA = np.linalg.norm(A, 2)
    assert np.linalg.norm(A @ V[:, :k] - V @ H, 2) / nA <= 1e-12
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V, 2) <= 1e-12
    np.testing.assert_allclose(V[:, 0], v0 / np.linalg.norm(v0), atol=1e-15)
    assert np.all(np.tril(H, -2) == 0)  # upper Hessenberg


def test_cgs2_projects_out_the_basis():
    g = np.random.default_rng(2)
    Q, _ = np.linalg.qr(g.standard_normal((300, 12)))
    w = g.standard_normal(300)
    h, w2 = oracle.cgs2(Q, w, _fp64(300))
    np.testing.assert_allclose(h, Q.T @ w, atol=1e-13)
    assert np.abs(Q.T @ w2).max() <= 1e-14 * np.linalg.norm(w)
    np.testing.assert_allclose(w2, w - Q @ (Q.T @ w), atol=1e-13)


def test_arnoldi_fp32_storage_loses_orthogonality_at_fp32_level():
    p = gen.conv_diff_2d(20, 20.0, (0.3, 1.0))
    A = oracle.dense(p)
    prec = oracle.Precision.for_inner("fp32", p)
    V, H, k = oracle.arnoldi(_op(p), np.ones(p.n), 30, prec)
    orth = np.linalg.norm(np.eye(k + 1) - V.T @ V, 2)
    assert 1e-9 < orth < 1e-5
    assert np.linalg.norm(A @ V[:, :k] - V @ H, 2) / np.linalg.norm(A, 2) < 1e-5


# ---------------------------------------------------- Givens / least sq ----

def test_givens_least_squares_matches_lstsq_and_explicit_residual():
    p = gen.conv_diff_2d(16, 30.0, (1.0, -0.5))
    A = oracle.dense(p)
    r = np.random.default_rng(4).standard_normal(p.n)
    cyc = oracle.gmres_cycle(_op(p), r, 25, -1.0, _fp64(p.n))
    e1 = np.zeros(cyc.k + 1)
    e1[0] = 1.0
    y_ref, *_ = np.linalg.lstsq(cyc.Hbar, e1, rcond=None)
    np.testing.assert_allclose(cyc.y, y_ref, rtol=1e-10, atol=1e-12)
    # implicit residual |g_{k+1}| equals the true residual of r - A (gamma V y)
    u = cyc.gamma * cyc.V[:, :cyc.k] @ cyc.y
    true = np.linalg.norm(r - A @ u) / cyc.gamma
    assert abs(cyc.hist[-1] - true) <= 1e-12
    # GMRES optimality: the residual never increases within a cycle
    assert all(b <= a * (1 + 1e-14) for a, b in zip(cyc.hist, cyc.hist[1:]))
    # rotations are orthogonal: c^2 + s^2 = 1
    c, s = oracle.givens(3.0, -4.0)
    assert (c, s) == (0.6, -0.8)
    assert oracle.givens(-2.0, 0.0) == (1.0, 0.0)


def test_back_substitute_matches_triangular_solve():
    g = np.random.default_rng(5)
    R = np.triu(g.standard_normal((9, 9))) + 5 * np.eye(9)
    b = g.standard_normal(9)
    np.testing.assert_allclose(oracle.back_substitute(R, b), np.linalg.solve(R, b), rtol=1e-12)


# ---------------------------------------------------------------- GMRES ----

def test_gmres_finite_termination_matches_dense_solve():
    g = np.random.default_rng(6)
    n = 40
    M = g.standard_normal((n, n)) + 8 * np.eye(n)
    A = Dense(M)
    b = g.standard_normal(n)
    x, info = oracle.gmres(A, b, m=n, rtol=1e-13)
    assert info.status == oracle.OK
    assert info.iters <= n
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-9, atol=1e-11)


def test_gmres_identity_one_iteration():
    A = Dense(np.eye(25))
    b = np.arange(1.0, 26.0)
    x, info = oracle.gmres(A, b, m=10)
    assert info.iters == 1
    np.testing.assert_allclose(x, b, rtol=1e-15)


def test_gmres_diagonal_with_k_distinct_eigenvalues():
    d = np.repeat([1.0, 2.0, 5.0, 7.0, 11.0], 8)
    A = Dense(np.diag(d))
    b = np.random.default_rng(7).uniform(1, 2, d.size)
    x, info = oracle.gmres(A, b, m=30, rtol=1e-12)
    assert info.iters == 5
    np.testing.assert_allclose(x, b / d, rtol=1e-11)


def test_gmres_manufactured_solution_small_2d():
    p, b, x_true = gen.config_small_2d(32)
    x, info = oracle.gmres(p, b, m=50, rtol=1e-10)
    assert info.status == oracle.OK and info.relres <= 1e-10
    r = b - oracle.spmv(p, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) == pytest.approx(info.relres)
    kappa = np.linalg.cond(oracle.dense(p))
    assert np.linalg.norm(x - x_true) / np.linalg.norm(x_true) <= kappa * 1e-10


def test_gmres_zero_rhs_nonfinite_singular_and_cap():
    p = gen.conv_diff_2d(8, 1.0)
    x, info = oracle.gmres(p, np.zeros(p.n), x0=np.ones(p.n))
    assert info.status == oracle.OK and not x.any()
    b = np.ones(p.n)
    b[3] = np.nan
    assert oracle.gmres(p, b)[1].status == oracle.NONFINITE
    assert oracle.gmres_ir(p, b)[1].status == oracle.NONFINITE
    _, info = oracle.gmres(p, np.ones(p.n), m=5, max_iters=7, rtol=1e-14)
    assert info.status == oracle.NOT_CONVERGED and info.iters == 7
    S = Dense(np.diag([1.0, 0.0]))
    _, info = oracle.gmres(S, np.array([1.0, 1.0]), m=2)
    assert info.status == oracle.BREAKDOWN


def test_gmres_restart_resume_equals_continuous():
    p, b, _ = gen.config_small_2d(24)
    x_all, info_all = oracle.gmres_ir(p, b, m=20, rtol=1e-10)
    x_half, info_half = oracle.gmres_ir(p, b, m=20, rtol=1e-10, max_iters=60)
    x_rest, info_rest = oracle.gmres_ir(p, b, x0=x_half, m=20, rtol=1e-10)
    assert info_half.iters + info_rest.iters == info_all.iters
    np.testing.assert_allclose(x_rest, x_all, rtol=0, atol=1e-12 * np.abs(x_all).max())


# ------------------------------------------------------------ GMRES-IR ----

def test_ir_iteration_counts_are_multiples_of_m_in_the_paper():
    d = json.load(open(os.path.join(GOLDEN, "paper_iteration_counts.json")))
    rs = d["restart_sweep_bentpipe"]
    assert all(it % m == 0 for it, m in zip(rs["ir_iters"], rs["m"]))
    assert not all(it % m == 0 for it, m in zip(rs["fp64_iters"], rs["m"]))
    assert all(it % d["table4"]["m"] == 0 for it in d["table4"]["ir_iters"])
    assert all(it % 50 == 0 for it in d["rhs_parabolic_fem"]["ir_iters"])
    assert d["switch_laplace3d200"]["ir_iters"] % 50 == 0


@pytest.mark.parametrize("m", [10, 25, 50])
def test_ir_fp32_reaches_fp64_accuracy_in_multiples_of_m(m):
    p, b, x_true = gen.config_small_2d(32)
    x, info = oracle.gmres_ir(p, b, m=m, rtol=1e-10, inner="fp32")
    assert info.status == oracle.OK and info.relres <= 1e-10
    assert info.iters % m == 0
    x64, info64 = oracle.gmres(p, b, m=m, rtol=1e-10)
    # Section 5.2: the IR convergence closely follows FP64 GMRES
    assert info64.iters <= info.iters <= info64.iters + 2 * m
    np.testing.assert_allclose(x, x64, rtol=0, atol=1e-6 * np.abs(x64).max())


def test_fp32_gmres_alone_stagnates_above_fp64_tolerance():
    """Section 5.2: single-precision GMRES alone floors far above 1e-10."""
    p, b, _ = gen.config_small_2d(32)
    _, info = oracle.gmres(p, b, m=50, rtol=1e-12, max_iters=1500, precision="fp32")
    assert info.status == oracle.NOT_CONVERGED
    assert 1e-9 < min(info.history) < 1e-4


@pytest.mark.parametrize("inner", ["fp16", "bf16"])
def test_ir_half_storage_converges(inner):
    p, b, _ = gen.config_small_2d(24)
    x, info = oracle.gmres_ir(p, b, m=30, rtol=1e-10, inner=inner)
    assert info.status == oracle.OK and info.relres <= 1e-10
    assert info.iters % 30 == 0


def test_ir_fp16_scaling_keeps_stored_basis_in_range():
    p, b, _ = gen.config_small_2d(24)
    prec = oracle.Precision.for_inner("fp16", p)
    # a power of two within a factor sqrt(2) of sqrt(n), so scaling adds no rounding
    k = int(np.log2(prec.s_v))
    assert prec.s_v == 2.0 ** k and np.sqrt(p.n / 2) < prec.s_v <= np.sqrt(2 * p.n)
    assert [oracle.vector_scale(n) for n in (1, 2, 7, 8, 1000, 2048, 8192, 10**6)] == \
        [1.0, 2.0, 2.0, 4.0, 32.0, 64.0, 128.0, 1024.0]
    assert prec.s_A == pytest.approx(np.abs(p.vals).max())
    v = np.ones(p.n) / np.sqrt(p.n)
    np.testing.assert_allclose(prec.store_vector(v), v, rtol=1e-3)
    assert np.abs(prec.matrix_values(p.vals)).max() == 1.0


def test_ir_inner_tolerance_stops_cycles_early():
    p, b, _ = gen.config_small_2d(32)
    _, info = oracle.gmres_ir(p, b, m=50, rtol=1e-10, inner="fp32", inner_rtol=1e-2)
    assert info.status == oracle.OK and info.relres <= 1e-10
    assert info.iters < info.outer * 50  # at least one cycle ended before m steps
    # each refinement step reduced the explicit residual by about the inner tolerance
    h = np.array(info.history)
    assert np.all(h[1:] / h[:-1] < 5e-2)


def test_ir_with_fp64_inner_equals_restarted_gmres():
    p, b, _ = gen.config_small_2d(20)
    x1, i1 = oracle.gmres_ir(p, b, m=15, rtol=1e-10, inner="fp64")
    x2, i2 = oracle.gmres(p, b, m=15, rtol=1e-10)
    assert i2.iters <= i1.iters <= i2.iters + 15
    np.testing.assert_allclose(x1, x2, atol=1e-8 * np.abs(x2).max())


# ------------------------------------------------------------ GMRES-FD ----

def test_fd_switch_at_zero_is_plain_fp64_gmres_and_converges_late():
    p, b, _ = gen.config_small_2d(24)
    x0, i32, i64 = oracle.gmres_fd(p, b, switch_iter=0, m=20)
    x, info = oracle.gmres(p, b, m=20)
    assert i32.iters == 0 and i64.iters == info.iters
    x1, i32b, i64b = oracle.gmres_fd(p, b, switch_iter=100, m=20)
    assert i32b.iters == 100 and i64b.relres <= 1e-10


def test_ir_stops_after_stalled_refinement():
    """GMRES(1) makes no progress on a 90-degree rotation (A r is orthogonal to r), so the
    refinement stalls and gives up after IR_STALL_LIMIT steps without 0.1% progress."""
    A = gen.Problem("rot", 2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32),
                    np.array([1.0, -1.0]))
    x, info = oracle.gmres_ir(A, np.array([1.0, 0.0]), m=1, rtol=1e-10)
    assert info.status == oracle.NOT_CONVERGED
    assert info.outer == IR_STALL_LIMIT and info.iters == info.outer
    assert info.relres == 1.0 and np.all(x == 0.0)
