"""Pins for the oracle's GMRES-polynomial preconditioner (CPU only)."""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from oracle.gmres import _fp64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_op(M):
    return lambda v: M @ v


def test_splitmix64_reference_outputs():
    d = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    got = oracle.splitmix64_raw(d["seed"], len(d["outputs"]))
    assert [int(v) for v in got] == [int(s) for s in d["outputs"]]
    u = oracle.splitmix64_uniform(42, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01


def test_gmres_polynomial_identity():
    """A p(A) v0 is the GMRES(d+1) approximation of v0: ||v0 - A p(A) v0|| equals the
    implicit residual of d+1 GMRES steps started from v0."""
    p = gen.conv_diff_2d(24, 40.0, (0.8, 0.6))
    op = _op = (lambda v: oracle.spmv(p, v))
    for d in (1, 4, 12):
        v0 = oracle.splitmix64_uniform(3, p.n)
        th = oracle.poly_roots(op, p.n, d, v0=v0)
        assert len(th) == d + 1
        res = np.linalg.norm(v0 - op(oracle.poly_apply(op, th, v0))) / np.linalg.norm(v0)
        cyc = oracle.gmres_cycle(op, v0, d + 1, -1.0, _fp64(p.n))
        assert res == pytest.approx(cyc.hist[-1], rel=1e-8)


def test_polynomial_with_complex_roots_matches_dense_evaluation():
    g = np.random.default_rng(11)
    n = 12
    M = g.standard_normal((n, n)) + 6 * np.eye(n)
    th = oracle.poly_roots(_dense_op(M), n, 7, v0=g.standard_normal(n))
    assert np.any(th.imag != 0)  # exercises the conjugate-pair branch
    I = np.eye(n, dtype=complex)
    phi = I.copy()
    for t in th:
        phi = phi @ (I - M / t)
    P = ((I - phi) @ np.linalg.inv(M)).real
    v = g.standard_normal(n)
    np.testing.assert_allclose(oracle.poly_apply(_dense_op(M), th, v), P @ v, rtol=1e-8, atol=1e-10)


def test_full_arnoldi_harmonic_ritz_values_are_the_eigenvalues():
    g = np.random.default_rng(12)
    n = 6
    M = g.standard_normal((n, n)) + 3 * np.eye(n)
    V, H, k = oracle.arnoldi(_dense_op(M), g.standard_normal(n), n)
    th = np.sort_complex(oracle.harmonic_ritz(H[:k + 1, :k]))
    np.testing.assert_allclose(th, np.sort_complex(np.linalg.eigvals(M)), rtol=1e-8)


def test_polynomial_of_scaled_identity_is_the_inverse():
    v = np.arange(1.0, 6.0)
    np.testing.assert_allclose(oracle.poly_apply(lambda x: 4.0 * x, np.array([4.0 + 0j]), v),
                               v / 4.0)


def test_leja_order_properties():
    th = np.array([1.0, 3.0 + 2.0j, 3.0 - 2.0j, -0.5, 8.0, 2.0 + 0.1j, 2.0 - 0.1j])
    out = oracle.leja_order(th)
    assert out[0] == 8.0
    assert sorted(map(complex, out), key=lambda z: (z.real, z.imag)) == \
        sorted(map(complex, th), key=lambda z: (z.real, z.imag))
    for i, z in enumerate(out):
        if z.imag > 0:
            assert out[i + 1] == z.conjugate()
    # second point maximises the distance to the first
    assert out[1] == -0.5


def test_poly_preconditioned_solvers_converge():
    p, b, _ = gen.config_small_2d(32)
    op = lambda v: oracle.spmv(p, v)
    th = oracle.poly_roots(op, p.n, 10, seed=5)
    x, info = oracle.gmres(p, b, m=30, rtol=1e-10, poly_roots=th)
    x0, info0 = oracle.gmres(p, b, m=30, rtol=1e-10)
    assert info.status == oracle.OK and info.iters < info0.iters / 3
    x, info = oracle.gmres_ir(p, b, m=30, rtol=1e-10, poly_roots=th)
    assert info.status == oracle.OK and info.iters % 30 == 0
