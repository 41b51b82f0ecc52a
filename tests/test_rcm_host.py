"""The library's host reverse Cuthill-McKee ordering (C ABI, no GPU) against the oracle's:
the same permutation, bit for bit, on shuffled stencils, unsymmetric and disconnected
structures; malformed structures are refused."""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
from oracle import precond as pc


@pytest.fixture(scope="module")
def g():
    import paper_2109_01232_b300 as lib
    lib.lib()
    return lib


def _shuffle(p, seed):
    q = np.random.default_rng(seed).permutation(p.n)
    M = sp.csr_matrix((p.vals, p.col_idx, p.row_ptr), shape=(p.n, p.n))[q][:, q]
    M.sort_indices()
    return M


CASES = {
    "conv_diff_2d": lambda: _shuffle(gen.conv_diff_2d(33, 20.0, (0.6, 0.8)), 1),
    "box_2d": lambda: _shuffle(gen.box_2d(21), 2),
    "star_3d": lambda: _shuffle(gen.star_3d(9), 3),
    "upper_triangle_only": lambda: sp.triu(_shuffle(gen.laplace_3d(8), 4)).tocsr(),
    "disconnected": lambda: sp.block_diag([_shuffle(gen.laplace_2d(7), 5), sp.eye(3),
                                           _shuffle(gen.laplace_2d(5), 6)]).tocsr(),
    "random_unsymmetric": lambda: (sp.random(400, 400, density=0.01, random_state=7)
                                   + sp.eye(400)).tocsr(),
}


@pytest.mark.parametrize("name", list(CASES))
def test_rcm_matches_oracle(g, name):
    M = CASES[name]()
    M.sort_indices()
    perm = g.rcm(M.indptr, M.indices)
    want = pc.rcm(M.shape[0], M.indptr, M.indices)
    np.testing.assert_array_equal(perm, want)
    assert sorted(perm.tolist()) == list(range(M.shape[0]))


def test_rcm_edge_cases(g):
    assert g.rcm(np.zeros(1, np.int32), np.zeros(0, np.int32)).size == 0
    np.testing.assert_array_equal(g.rcm([0, 1], [0]), [0])
    # diagonal only: every vertex is its own component, ranks by index, order reversed
    np.testing.assert_array_equal(g.rcm(np.arange(6), np.arange(5)), [4, 3, 2, 1, 0])


@pytest.mark.parametrize("rp,ci", [([1, 2], [0]), ([0, 2, 1], [0, 1]), ([0, 1], [3]),
                                   ([0, 1], [-1])])
def test_rcm_rejects_malformed(g, rp, ci):
    with pytest.raises(g.GmresError):
        g.rcm(rp, ci)


def test_rcm_full_block_jacobi_workload(g):
    """The 216,000-row shuffled 27-point workload: the same permutation as the oracle's,
    and a bandwidth far below the shuffled numbering's."""
    p, _ = gen.config_bj()[0]
    perm = g.rcm(p.row_ptr, p.col_idx)
    np.testing.assert_array_equal(perm, pc.rcm(p.n, p.row_ptr, p.col_idx))
    B = pc.permute(p, perm)
    assert pc.bandwidth(p.n, B.row_ptr, B.col_idx) < 0.06 * pc.bandwidth(p.n, p.row_ptr, p.col_idx)
