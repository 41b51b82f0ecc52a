"""Pins of the RCM / block-Jacobi oracle against hand-derived orders, closed forms and
structural invariants (CPU)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

import gen
import oracle
from oracle import precond as pc


def _csr(M) -> gen.Problem:
    M = sp.csr_matrix(M)
    M.sort_indices()
    return gen.Problem("t", M.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32),
                       M.data.astype(np.float64))


def _shuffled(M, seed):
    q = np.random.default_rng(seed).permutation(M.shape[0])
    return sp.csr_matrix(M)[q][:, q]


def _grid(m):
    T = sp.diags([np.ones(m - 1), 4 * np.ones(m), np.ones(m - 1)], [-1, 0, 1])
    E = sp.diags([np.ones(m - 1), np.ones(m - 1)], [-1, 1])
    return (sp.kron(sp.eye(m), T) + sp.kron(E, sp.eye(m))).tocsr()


def test_rcm_star_by_hand():
    # centre 0 joined to leaves 1..4: ranks (deg, index) put leaf 1 first; the George-Liu
    # iteration from 1 picks leaf 2 (last level {2, 3, 4}, no deeper structure), the BFS
    # from 2 visits 2, 0, 1, 3, 4, reversed
    S = 4 * np.eye(5)
    S[0, 1:] = S[1:, 0] = 1
    A = _csr(S)
    assert pc.rcm(5, A.row_ptr, A.col_idx).tolist() == [4, 3, 1, 0, 2]


def test_rcm_path_gets_bandwidth_one():
    n = 50
    P = sp.diags([np.ones(n - 1), 2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1])
    A = _csr(_shuffled(P, 1))
    perm = pc.rcm(n, A.row_ptr, A.col_idx)
    assert sorted(perm.tolist()) == list(range(n))
    B = pc.permute(A, perm)
    assert pc.bandwidth(n, B.row_ptr, B.col_idx) == 1


@pytest.mark.parametrize("m", [7, 12, 20])
def test_rcm_grid_bandwidth_equals_side_and_library(m):
    A = _csr(_shuffled(_grid(m), 2))
    perm = pc.rcm(m * m, A.row_ptr, A.col_idx)
    B = pc.permute(A, perm)
    ours = pc.bandwidth(m * m, B.row_ptr, B.col_idx)
    M = sp.csr_matrix((A.vals, A.col_idx, A.row_ptr))
    q = reverse_cuthill_mckee(M, symmetric_mode=True)
    lib = sp.coo_matrix(M[q][:, q])
    assert ours == m == np.abs(lib.row - lib.col).max()


def test_rcm_components_are_contiguous_and_structure_symmetrised():
    # two paths (0-2-4, 1-3) and an isolated vertex 5; only the upper triangle is stored,
    # so the ordering must use A + A^T
    rows = [0, 2, 1]
    cols = [2, 4, 3]
    M = sp.csr_matrix((np.ones(3), (rows, cols)), shape=(6, 6)) + sp.eye(6)
    A = _csr(M)
    perm = pc.rcm(6, A.row_ptr, A.col_idx).tolist()
    assert sorted(perm) == list(range(6))
    pos = {v: i for i, v in enumerate(perm)}
    for comp in ({0, 2, 4}, {1, 3}, {5}):
        idx = sorted(pos[v] for v in comp)
        assert idx == list(range(idx[0], idx[0] + len(idx)))
    assert abs(pos[0] - pos[2]) == 1 and abs(pos[2] - pos[4]) == 1


def test_permute_is_similarity():
    rng = np.random.default_rng(3)
    M = sp.random(30, 30, density=0.15, random_state=4, format="csr") + 3 * sp.eye(30)
    A = _csr(M)
    perm = rng.permutation(30)
    B = pc.permute(A, perm)
    D, E = oracle.dense(A), oracle.dense(B)
    np.testing.assert_array_equal(E, D[np.ix_(perm, perm)])
    x = rng.standard_normal(30)
    # (P A P^T)(P x) = P (A x)
    np.testing.assert_allclose(oracle.spmv(B, x[perm]), (D @ x)[perm], rtol=1e-14, atol=1e-14)


def test_block_jacobi_point_is_diagonal_scaling():
    p = gen.conv_diff_2d(9, 20.0, (0.6, 0.8))
    v = np.random.default_rng(5).standard_normal(p.n)
    z = pc.BlockJacobi(p, 1).apply(v)
    np.testing.assert_allclose(z, v / np.diag(oracle.dense(p)), rtol=1e-15)


def test_block_jacobi_2x2_closed_form_and_ragged_tail():
    M = np.array([[4.0, 1.0, 0.5, 0.0, 0.0],
                  [2.0, 3.0, 0.0, 0.0, 0.0],
                  [0.0, 1.0, 5.0, -1.0, 0.0],
                  [0.0, 0.0, 2.0, 6.0, 1.0],
                  [0.0, 0.0, 0.0, 3.0, 7.0]])
    bj = pc.BlockJacobi(_csr(M), 2)
    assert [(s, e) for s, e, _ in bj.blocks] == [(0, 2), (2, 4), (4, 5)]
    v = np.array([1.0, -2.0, 3.0, 0.5, 7.0])
    z = bj.apply(v)
    # [[a, b], [c, d]]^{-1} = [[d, -b], [-c, a]] / (a d - b c)
    np.testing.assert_allclose(z[:2], np.array([3 * 1 - 1 * -2, -2 * 1 + 4 * -2]) / 10, rtol=1e-15)
    np.testing.assert_allclose(z[2:4], np.array([6 * 3 + 1 * 0.5, -2 * 3 + 5 * 0.5]) / 32, rtol=1e-15)
    assert z[4] == 1.0


def test_block_jacobi_of_a_block_diagonal_matrix_is_its_inverse():
    rng = np.random.default_rng(6)
    k, nb = 6, 5
    blocks = [rng.standard_normal((k, k)) + k * np.eye(k) for _ in range(nb)]
    A = _csr(sp.block_diag([sp.coo_matrix(B) for B in blocks]))
    bj = pc.BlockJacobi(A, k)
    v = rng.standard_normal(k * nb)
    np.testing.assert_allclose(bj.apply(oracle.spmv(A, v)), v, rtol=1e-12, atol=1e-12)
    # GMRES on A M^{-1} = I ends after one step with the exact answer
    b = rng.standard_normal(k * nb)
    x, info = oracle.gmres(A, b, m=10, rtol=1e-12, right_prec=bj.apply)
    assert info.status == oracle.OK and info.iters == 1
    np.testing.assert_allclose(oracle.spmv(A, x), b, rtol=1e-11, atol=1e-11)


def test_block_jacobi_lowers_gmres_iterations_and_ir_converges():
    p = gen.conv_diff_2d(24, 40.0, (0.6, 0.8))
    perm = pc.rcm(p.n, p.row_ptr, p.col_idx)
    B = pc.permute(p, perm)
    b = np.ones(p.n)
    _, plain = oracle.gmres(B, b, m=30, rtol=1e-10)
    # blocks of 24 rows (one grid line of the reordered stencil): a strong preconditioner
    # here (blocks of 1..8 rows barely change the iteration count of this problem)
    bj = pc.BlockJacobi(B, 24)
    x, pre = oracle.gmres(B, b, m=30, rtol=1e-10, right_prec=bj.apply)
    assert pre.status == oracle.OK and pre.iters < 0.6 * plain.iters
    xi, ir = oracle.gmres_ir(B, b, m=30, rtol=1e-10, inner="fp32", right_prec=bj.apply)
    assert ir.status == oracle.OK and ir.relres <= 1e-10
    # the IR answer, mapped back to the original numbering, solves the original system
    xo = np.empty(p.n)
    xo[perm] = xi
    assert np.linalg.norm(oracle.spmv(p, xo) - b) <= 1e-10 * np.linalg.norm(b)
