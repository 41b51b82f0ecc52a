"""The seeded input generators: shapes and structure the workloads rely on (CPU)."""
import numpy as np
import scipy.sparse as sp

import gen


def _M(p):
    return sp.csr_matrix((p.vals, p.col_idx, p.row_ptr), shape=(p.n, p.n))


def test_box_3d_is_27_point_spd():
    p = gen.box_3d(5)
    M = _M(p)
    assert p.n == 125 and np.diff(p.row_ptr).max() == 27
    assert abs(M - M.T).max() == 0.0
    assert np.linalg.eigvalsh(M.toarray()).min() > 0.0


def test_shuffled_is_a_permutation_similarity():
    p = gen.conv_diff_2d(9, 20.0, (0.6, 0.8))
    q = gen.shuffled(p, 3)
    perm = np.random.default_rng(3).permutation(p.n)  # the documented relabelling
    np.testing.assert_array_equal(_M(q).toarray(), _M(p).toarray()[np.ix_(perm, perm)])
    assert np.all(np.diff(q.row_ptr) >= 0) and q.meta["shuffle_seed"] == 3
    for i in range(q.n):  # sorted columns in every row
        c = q.col_idx[q.row_ptr[i]:q.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_scaled_is_symmetric_diagonal_scaling():
    p = gen.box_3d(4)
    q = gen.scaled(p, 1.0, 7)
    d = np.exp(np.random.default_rng(7).standard_normal(p.n))
    np.testing.assert_allclose(_M(q).toarray(), np.diag(d) @ _M(p).toarray() @ np.diag(d),
                               rtol=1e-15)
    assert abs(_M(q) - _M(q).T).max() == 0.0


def test_config_bj_workloads():
    (a, ka), (b, kb) = gen.config_bj()
    assert (a.n, len(a.vals), ka) == (216000, 5639752, 42)
    assert (b.n, len(b.vals), kb) == (110592, 760320, 1)
    assert abs(_M(a) - _M(a).T).max() == 0.0          # SPD stand-in is symmetric
    assert abs(_M(b) - _M(b).T).max() > 0.0           # the other is not
