"""Selector kernels against the oracle: features, MLP forward, loss gradient, Adam training,
and the parameter choice through the C ABI."""
import os

import numpy as np
import pytest

import gen
from oracle import selector as osel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2109_01232_b300 as lib
    lib.lib()
    return lib


def _irregular():
    rng = np.random.default_rng(4)
    n = 700
    lens = rng.integers(0, 9, n)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    ci = np.concatenate([np.sort(rng.choice(n, L, replace=False)) for L in lens]).astype(np.int32)
    va = rng.standard_normal(int(rp[-1]))
    return gen.Problem("irr", n, rp.astype(np.int32), ci, va)


MATS = {
    "2d": lambda: gen.conv_diff_2d(40, 30.0, (0.6, 0.8)),
    "3d_aniso": lambda: gen.build_selector_matrix(gen.selector_matrices(count=3, n_hi=3e4)[2]),
    "irregular": _irregular,
    "diag": lambda: gen.Problem("d", 5, np.arange(6, dtype=np.int32), np.arange(5, dtype=np.int32),
                                np.array([1.0, -2.0, 3.0, 4.0, 0.5])),
}


@pytest.mark.parametrize("which", list(MATS))
def test_features_match_oracle(g, which):
    p = MATS[which]()
    f = g.matrix_features(g.DeviceCSR.from_problem(p))
    fo = osel.features(p)
    np.testing.assert_allclose(f, fo.astype(np.float32), rtol=2e-6, atol=2e-6)


def _batch(seed, B):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, 16)).astype(np.float32)
    y = rng.integers(0, 32, B).astype(np.int32)
    p = (gen.mlp_init(seed) + 0.05 * rng.standard_normal(osel.N_PARAMS)).astype(np.float32)
    return p, X, y


def test_forward_and_gradient_match_oracle(g):
    p, X, y = _batch(1, 37)
    P = g.mlp_forward(p, X)
    Po, _ = osel.forward(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(P, Po, rtol=1e-5, atol=1e-7)
    loss, grad = g.mlp_loss_grad(p, X, y)
    lo, go = osel.loss_grad(p.astype(np.float64), X.astype(np.float64), y)
    assert loss == pytest.approx(lo, rel=1e-5)
    assert np.abs(grad - go).max() <= 1e-5 * np.abs(go).max()


def test_adam_training_matches_oracle(g):
    p, X, y = _batch(2, 24)
    pg, lg = g.mlp_train(p, X, y, 40, 1e-2)
    po, lo = osel.train(p.astype(np.float64), X.astype(np.float64), y, 40, 1e-2)
    # FP32 -log(p) near p = 1 carries ~1e-7 absolute error: relative plus absolute tolerance
    np.testing.assert_allclose(lg, lo, rtol=2e-4, atol=1e-6)
    assert np.abs(pg - po).max() <= 2e-3 * np.abs(po).max()
    assert lg[-1] < 0.5 * lg[0]


def test_select_params_default_and_model(g):
    p = MATS["2d"]()
    A = g.DeviceCSR.from_problem(p)
    q, cls, conf = g.Selector(None).choose(A, rtol=1e-9)
    assert (q.restart_m, q.poly_degree, q.inner_prec, q.inner_rtol, q.rtol, cls) == (50, 0, 1, 1e-4, 1e-9, -1)
    from paper_2109_01232_b300 import selector as ps
    model = dict(params=gen.mlp_init(9), feat_mean=np.zeros(16, np.float32),
                 feat_scale=np.full(16, 0.5, np.float32),
                 class_m=[ps.class_config(c)[0] for c in range(32)],
                 class_degree=[ps.class_config(c)[1] for c in range(32)],
                 class_prec=[g.PREC[ps.class_config(c)[2]] for c in range(32)],
                 class_inner_rtol=np.full(32, 1e-6), min_confidence=0.0, tol_index=np.full(32, 2))
    q, cls, conf = g.Selector(model).choose(A)
    c_ref, conf_ref = ps.predict(model, g.matrix_features(A)[None, :])
    assert cls == int(c_ref[0]) and conf == pytest.approx(float(conf_ref[0]), rel=1e-6)
    m, d, prec = ps.class_config(cls)
    assert (q.restart_m, q.poly_degree, q.inner_prec, q.inner_rtol) == (m, d, g.PREC[prec], 1e-6)
    model["min_confidence"] = 1.01  # never confident: the default
    q, cls, _ = g.Selector(model).choose(A)
    assert cls == -1 and q.restart_m == 50


@pytest.mark.skipif(not os.path.exists(os.path.join(os.path.dirname(__file__), "..",
                                                    "paper_2109_01232_b300", "selector_model.npz")),
                    reason="no trained selector model committed")
def test_trained_selector_gains_on_held_out(g):
    """The committed model, evaluated with the GPU forward kernel on the held-out matrices
    of the committed sweep: faster than the default (geometric mean) without losing solves,
    and the same choices as the oracle's forward pass."""
    from paper_2109_01232_b300 import selector as ps
    model, data = ps.load(ps.MODEL_PATH), ps.load(ps.SWEEP_PATH)
    te = model["held_out"]
    res = ps.evaluate(data, model, te)
    assert res["geomean_ratio"] < 1.0
    assert res["converged_selected"] >= res["converged_default"]
    X = (data["features"][te] - model["feat_mean"]) * model["feat_scale"]
    Po, _ = osel.forward(model["params"].astype(np.float64), X.astype(np.float64))
    assert np.array_equal(Po.argmax(axis=1), res["chosen"])


@pytest.mark.skipif(not os.path.exists(os.path.join(os.path.dirname(__file__), "..",
                                                    "paper_2109_01232_b300", "selector_model.npz")),
                    reason="no trained selector model committed")
def test_selector_choice_beats_default_on_fresh_solves(g):
    """Held-out matrices (up to 4e5 rows) solved again on the GPU, from b = ones, with the
    selector's choice (gmres_select_params on GPU-computed features) and with the fixed
    default: the chosen configurations are faster (geometric mean of the device times) and
    every solve the default converges on still converges."""
    from paper_2109_01232_b300 import selector as ps
    model, data = ps.load(ps.MODEL_PATH), ps.load(ps.SWEEP_PATH)
    idx = [int(k) for k in model["held_out"]
           if ps.descriptor(data, k)["side"] ** ps.descriptor(data, k)["dim"] <= 4e5][:16]
    assert len(idx) >= 10
    res = ps.live_evaluate(data, model, idx, reps=2)
    assert res["n"] == len(idx)
    assert res["lost_convergence"] == 0
    assert res["converged_selected"] >= res["converged_default"]
    assert res["geomean_ratio"] < 1.0, res
