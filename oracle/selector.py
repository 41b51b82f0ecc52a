"""Oracle for the learned parameter selector (TEST INFRASTRUCTURE ONLY, like the rest of
`oracle/`): the 16 matrix features, the 16-64-64-32 MLP with softmax cross-entropy, its
gradient and Adam, all in plain numpy FP64.

The paper has no selector; the feature list, the network shape and the training rule are
the project's own definitions (the selector picks GMRES-IR's restart length, polynomial
degree, inner precision and inner tolerance from cheap matrix features).  Pins in
tests/test_oracle_selector.py: closed-form features of identity / diagonal / tridiagonal
/ hand-checked small matrices, the gradient against central finite differences, uniform
logits giving log(32), Adam's first step equal to -lr * sign(g).
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 16
HIDDEN = 64
N_CLASSES = 32
# flat parameter layout: W1[16][64], b1[64], W2[64][64], b2[64], W3[64][32], b3[32]
SHAPES = [(N_FEATURES, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, N_CLASSES),
          (N_CLASSES,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)
LOG_FLOOR = 1e-30


def _log10(x: float) -> float:
    return float(np.log10(max(x, LOG_FLOOR)))


def features(A) -> np.ndarray:
    """The 16 features of a CSR matrix (A.n, A.row_ptr, A.col_idx, A.vals), straight from
    their definitions, one row at a time.  With d_i the diagonal entry (0 if absent), s_i =
    sum_j |a_ij| and lg(x) = log10(max(x, 1e-30)):
      0 lg(n)             1 lg(nnz)                    2 nnz / n           3 max row length
      4 mean |d_i|/s_i     5 min |d_i|/s_i               6 share of rows with |d_i| >= s_i - |d_i|
      7 lg(max s_i)        8 lg(||A||_F)                 9 lg(max |a_ij|)   10 lg(mean |d_i|)
     11 lg(max |d_i|) - lg(min nonzero |d_i|)
     12 sum (a_ij - a_ji)^2 / sum (a_ij^2 + a_ji^2) over the off-diagonal pattern
     13 mean over rows with d_i != 0 of (sum_{j != i} a_ij) / d_i
     14 log10(1 + mean |i - j| over the nonzeros)   15 log10(1 + max |i - j|)"""
    n, rp, ci, av = int(A.n), A.row_ptr, A.col_idx, A.vals
    nnz = int(rp[n])
    ratio = np.zeros(n)
    dom = 0
    inf_norm = 0.0
    fro2 = 0.0
    amax = 0.0
    diag = np.zeros(n)
    rel_off = []
    dist_sum = 0.0
    dist_max = 0
    num = den = 0.0
    lens = np.diff(rp)
    for i in range(n):
        k0, k1 = int(rp[i]), int(rp[i + 1])
        s = d = so = 0.0
        for k in range(k0, k1):
            j, a = int(ci[k]), float(av[k])
            s += abs(a)
            fro2 += a * a
            amax = max(amax, abs(a))
            dist_sum += abs(i - j)
            dist_max = max(dist_max, abs(i - j))
            if j == i:
                d += a
            else:
                so += a
                # the transposed entry a_ji (0 if j's row does not hold column i)
                aji = 0.0
                for kk in range(int(rp[j]), int(rp[j + 1])):
                    if int(ci[kk]) == i:
                        aji += float(av[kk])
                num += (a - aji) ** 2
                den += a * a + aji * aji
        diag[i] = d
        ratio[i] = abs(d) / s if s > 0 else 0.0
        dom += abs(d) >= s - abs(d)
        inf_norm = max(inf_norm, s)
        if d != 0.0:
            rel_off.append(so / d)
    ad = np.abs(diag)
    nzd = ad[ad > 0]
    f = np.array([
        _log10(n),
        _log10(max(nnz, 1)),
        nnz / n,
        float(lens.max()) if n else 0.0,
        float(ratio.mean()),
        float(ratio.min()),
        dom / n,
        _log10(inf_norm),
        _log10(np.sqrt(fro2)),
        _log10(amax),
        _log10(float(ad.mean())),
        _log10(float(ad.max())) - _log10(float(nzd.min()) if len(nzd) else 0.0),
        num / den if den > 0 else 0.0,
        float(np.mean(rel_off)) if rel_off else 0.0,
        float(np.log10(1.0 + dist_sum / max(nnz, 1))),
        float(np.log10(1.0 + dist_max)),
    ])
    return f


def unpack(params: np.ndarray) -> list[np.ndarray]:
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(params[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def forward(params: np.ndarray, X: np.ndarray):
    """Class probabilities of the rows of X (B x 16) and the activations for backprop."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    h1 = np.maximum(X @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    z = h2 @ W3 + b3
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    p = e / e.sum(axis=1, keepdims=True)
    return p, (X, h1, h2)


def loss_grad(params: np.ndarray, X: np.ndarray, labels: np.ndarray):
    """Mean cross-entropy over the batch and its gradient (flat, same layout as params)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    p, (X, h1, h2) = forward(params, X)
    B = X.shape[0]
    loss = float(-np.mean(np.log(p[np.arange(B), labels])))
    dz = p.copy()
    dz[np.arange(B), labels] -= 1.0
    dz /= B
    dW3, db3 = h2.T @ dz, dz.sum(axis=0)
    dh2 = (dz @ W3.T) * (h2 > 0)
    dW2, db2 = h1.T @ dh2, dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (h1 > 0)
    dW1, db1 = X.T @ dh1, dh1.sum(axis=0)
    return loss, pack([dW1, db1, dW2, db2, dW3, db3])


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(params, grad, m, v, t: int, lr: float):
    """One Adam update (t counts from 1); returns new (params, m, v)."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1 - ADAM_B2) * grad * grad
    mh = m / (1 - ADAM_B1 ** t)
    vh = v / (1 - ADAM_B2 ** t)
    return params - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def train(params0, X, labels, epochs: int, lr: float):
    """Full-batch Adam on the cross-entropy; returns (params, losses per epoch)."""
    p = np.asarray(params0, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for t in range(1, epochs + 1):
        loss, g = loss_grad(p, X, labels)
        losses.append(loss)
        p, m, v = adam_step(p, g, m, v, t, lr)
    return p, np.array(losses)
