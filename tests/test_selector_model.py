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


def test_corpus_split_holds_out_80_configured_matrices_and_their_siblings():
    """The held-out set of a sweep over the whole configured corpus: 80 of its 400 matrices by
    the seeded permutation; a matrix of the small corpus drawn from the same seed as a
    held-out one trains on neither side."""
    from paper_2109_01232_b300 import selector as ps
    rng = np.random.default_rng(0)
    n_small, n_conf = 128, 400
    di = np.concatenate([np.arange(n_small), rng.permutation(n_conf)])
    nh = np.concatenate([np.full(n_small, 2e5), np.full(n_conf, 4e6)])
    data = dict(desc_index=di, desc_n_hi=nh, desc_seed=4000 + di)
    tr, te = ps.corpus_split(data)
    assert len(te) == 80 and np.all(nh[te] == 4e6)
    held = np.random.Generator(np.random.PCG64(4999)).permutation(400)[:80]
    assert sorted(di[te].tolist()) == sorted(held.tolist())
    assert not np.intersect1d(tr, te).size
    siblings = np.flatnonzero((nh == 2e5) & np.isin(di, held))
    assert not np.intersect1d(tr, siblings).size
    assert len(tr) == n_small + n_conf - 80 - len(siblings)
    with pytest.raises(ValueError):  # part of the configured corpus missing
        ps.corpus_split(dict(desc_index=di[:-1], desc_n_hi=nh[:-1], desc_seed=4000 + di[:-1]))
