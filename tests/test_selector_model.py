"""The committed selector model against the committed sweep, evaluated with the oracle's
forward pass on the CPU: on the held-out matrices the selected configurations beat the
fixed default (geometric-mean solve time) without losing a converged solve."""
import os

import numpy as np
import pytest

from oracle import selector as osel

HERE = os.path.join(os.path.dirname(__file__), "..", "paper_2109_01232_b300")
MODEL, SWEEP = os.path.join(HERE, "selector_model.npz"), os.path.join(HERE, "selector_sweep.npz")


@pytest.mark.skipif(not (os.path.exists(MODEL) and os.path.exists(SWEEP)),
                    reason="no trained selector model committed")
def test_selector_beats_default_on_held_out():
    with np.load(MODEL) as f:
        model = {k: f[k] for k in f.files}
    with np.load(SWEEP) as f:
        data = {k: f[k] for k in f.files}
    te = model["held_out"]
    assert len(te) >= 10 and not np.isin(te, np.setdiff1d(np.arange(len(data["default_ms"])), te)).any()
    X = (data["features"][te].astype(np.float64) - model["feat_mean"]) * model["feat_scale"]
    P, _ = osel.forward(model["params"].astype(np.float64), X)
    c = P.argmax(axis=1)
    T, T0 = data["times"][te], data["default_ms"][te]
    tol = model["tol_index"]
    chosen = np.array([T[k, c[k], tol[c[k]]] for k in range(len(te))])
    ok = np.isfinite(T0)
    ratio = np.where(np.isfinite(chosen[ok] / T0[ok]), chosen[ok] / T0[ok], 3.0)
    geomean = float(np.exp(np.mean(np.log(ratio))))
    assert geomean < 1.0
    assert np.isfinite(chosen).sum() >= ok.sum()
