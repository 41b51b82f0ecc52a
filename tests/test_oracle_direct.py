"""Pins of the oracle's exact solve (oracle/direct.py) against dense linear algebra and
manufactured solutions."""
import numpy as np

import gen
import oracle
from oracle.direct import direct_solve


def test_matches_dense_solve_on_small_nonsymmetric_systems():
    for side, pe in ((9, 0.0), (12, 40.0), (7, 5.0)):
        p = gen.conv_diff_2d(side, pe, (0.6, -0.8))
        b = np.random.default_rng(side).standard_normal(p.n)
        x = direct_solve(p, b)
        xd = np.linalg.solve(oracle.dense(p), b)
        assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_manufactured_solution_on_a_3d_stencil():
    p = gen.conv_diff_3d(15, 20.0, (1.0, 0.3, -0.5))
    b, x_true = gen.rhs_manufactured(p, 77)
    x = direct_solve(p, b)
    assert np.linalg.norm(x - x_true) <= 1e-10 * np.linalg.norm(x_true)
    assert np.linalg.norm(b - oracle.spmv(p, x)) <= 1e-13 * np.linalg.norm(b)


def test_permutation_matrix_is_its_own_inverse_transpose():
    n = 50
    perm = np.random.default_rng(3).permutation(n)
    p = gen.Problem("perm", n, np.arange(n + 1, dtype=np.int32), perm.astype(np.int32),
                    np.ones(n))
    b = np.arange(n, dtype=np.float64)
    x = direct_solve(p, b)
    y = np.empty(n)
    y[perm] = b  # (P x)_i = x_{perm[i]} = b_i
    np.testing.assert_array_equal(x, y)
