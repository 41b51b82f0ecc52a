"""Pins of the selector oracle (features, MLP, gradient, Adam) against closed forms, finite
differences and hand-checked matrices."""
import math

import numpy as np
import pytest

import gen
from oracle import selector as sel


def _csr(dense):
    dense = np.asarray(dense, dtype=np.float64)
    n = dense.shape[0]
    rp, ci, va = [0], [], []
    for i in range(n):
        for j in range(n):
            if dense[i, j] != 0.0:
                ci.append(j)
                va.append(dense[i, j])
        rp.append(len(ci))
    return gen.Problem("t", n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va))


def test_features_identity():
    f = sel.features(_csr(np.eye(10)))
    want = [1, 1, 1, 1, 1, 1, 1, 0, 0.5, 0, 0, 0, 0, 0, 0, 0]
    np.testing.assert_allclose(f, want, atol=1e-15)


def test_features_tridiagonal_laplacian():
    T = 2 * np.eye(5) - np.eye(5, k=1) - np.eye(5, k=-1)
    f = sel.features(_csr(T))
    want = [math.log10(5), math.log10(13), 13 / 5, 3, (2 * 2 / 3 + 3 * 0.5) / 5, 0.5, 1.0,
            math.log10(4), math.log10(math.sqrt(28)), math.log10(2), math.log10(2), 0.0, 0.0,
            (-0.5 * 2 - 3) / 5, math.log10(1 + 8 / 13), math.log10(2)]
    np.testing.assert_allclose(f, want, rtol=1e-14, atol=1e-15)


def test_features_nonsymmetric_and_degenerate():
    f = sel.features(_csr([[1, 2], [0, 3]]))
    assert f[12] == 1.0                                    # a_21 absent: fully nonsymmetric
    assert f[13] == pytest.approx(1.0)                     # (2/1 + 0/3) / 2
    assert f[11] == pytest.approx(math.log10(3))
    assert f[4] == pytest.approx((1 / 3 + 1) / 2) and f[5] == pytest.approx(1 / 3)
    assert f[6] == 0.5
    assert sel.features(_csr([[1, 1], [-1, 1]]))[12] == 2.0   # antisymmetric off-diagonal
    z = sel.features(_csr([[0, 1], [1, 0]]))               # zero diagonal
    assert z[4] == 0.0 and z[10] == -30.0 and z[11] == 0.0 and z[13] == 0.0


def _rand_params(seed):
    return gen.mlp_init(seed).astype(np.float64)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((7, sel.N_FEATURES))
    y = rng.integers(0, sel.N_CLASSES, 7)
    p = _rand_params(11) + 0.05 * rng.standard_normal(sel.N_PARAMS)
    loss, g = sel.loss_grad(p, X, y)
    idx = rng.choice(sel.N_PARAMS, 300, replace=False)
    h = 1e-6
    fd = np.array([(sel.loss_grad(p + h * e, X, y)[0] - sel.loss_grad(p - h * e, X, y)[0]) / (2 * h)
                   for e in (np.eye(1, sel.N_PARAMS, k).ravel() for k in idx)])
    assert np.abs(fd - g[idx]).max() <= 1e-7 * max(1.0, np.abs(g).max())


def test_uniform_logits_and_softmax():
    p = _rand_params(5)
    W = sel.unpack(p)
    o = sel.N_FEATURES * sel.HIDDEN + sel.HIDDEN + sel.HIDDEN * sel.HIDDEN + sel.HIDDEN
    p[o:] = 0.0  # W3 = 0, b3 = 0
    X = np.random.default_rng(1).standard_normal((4, sel.N_FEATURES))
    probs, _ = sel.forward(p, X)
    np.testing.assert_allclose(probs, 1 / 32, rtol=1e-15)
    loss, _ = sel.loss_grad(p, X, np.array([0, 5, 31, 7]))
    assert loss == pytest.approx(math.log(32), rel=1e-15)
    p2 = _rand_params(5)
    p3 = p2.copy()
    p3[-sel.N_CLASSES:] += 3.0  # shifting every logit leaves the softmax unchanged
    np.testing.assert_allclose(sel.forward(p2, X)[0], sel.forward(p3, X)[0], rtol=1e-12)
    assert W[0].shape == (16, 64) and sel.N_PARAMS == 7328


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p, m, v = sel.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_training_separates_a_separable_problem():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((64, sel.N_FEATURES))
    y = (X[:, 0] > 0).astype(int) * 3 + (X[:, 1] > 0).astype(int)  # four classes
    _, losses = sel.train(_rand_params(2), X, y, 300, 1e-2)
    assert losses[-1] < 0.05 * losses[0]
    probs, _ = sel.forward(sel.train(_rand_params(2), X, y, 300, 1e-2)[0], X)
    assert (probs.argmax(axis=1) == y).all()
