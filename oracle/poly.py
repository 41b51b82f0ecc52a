"""GMRES-polynomial preconditioner, oracle side.

TEST INFRASTRUCTURE ONLY (imported by tests/, smoke() and the CPU-baseline leg).

Section 3.4 of the paper applies a polynomial "based upon the GMRES polynomial"
as a right preconditioner, M^{-1} = p(A), and defers the construction to the
authors' earlier polynomial-preconditioning work.  Reading used here (the
published Loe-Morgan construction):

* Run d+1 Arnoldi steps (FP64, CGS2) from a start vector v0.
* The GMRES residual polynomial phi of degree d+1 has as roots the harmonic Ritz
  values theta_i: the eigenvalues of H + h_{k+1,k}^2 f e_k^T with H the square
  k x k Hessenberg matrix, f = H^{-T} e_k and k = d+1.
* p(z) = (1 - phi(z)) / z, phi(z) = prod_i (1 - z / theta_i), so that
  A p(A) v0 is the GMRES approximation of v0 after d+1 steps.
* The roots are put in modified Leja order (conjugate pairs adjacent, the one
  with positive imaginary part first) and p(A) v is applied in product form
  with real arithmetic, d matrix-vector products:
    real theta:           y += prod / theta;  prod -= A prod / theta
    pair a +- ib, |t|^2:  y += (2a/|t|^2) prod - (1/|t|^2) A prod
                          prod -= (2a/|t|^2) A prod - (1/|t|^2) A^2 prod
  (the prod update is skipped for the last root or pair).
  The power-basis form sum_k c_k A^k of Section 3.4 is the same polynomial but
  is not used for evaluation.

The start vector comes from SplitMix64 (Steele, Lea, Flood 2014), a
counter-based generator that the CUDA library implements independently from the
same published definition: element i is mix(seed + (i+1) * 0x9E3779B97F4A7C15)
mapped to [-1, 1) as (z >> 11) * 2^-52 - 1.
"""
from __future__ import annotations

import numpy as np

from .gmres import arnoldi

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_raw(seed: int, n: int) -> np.ndarray:
    """The first n 64-bit SplitMix64 outputs for state `seed` (uint64, wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n values in [-1, 1) from the SplitMix64 output sequence of `seed`."""
    z = splitmix64_raw(seed, n)
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -52 - 1.0


def harmonic_ritz(Hbar: np.ndarray) -> np.ndarray:
    """Harmonic Ritz values of a (k+1) x k Arnoldi Hessenberg matrix."""
    k = Hbar.shape[1]
    H = Hbar[:k, :k]
    e = np.zeros(k)
    e[-1] = 1.0
    f = np.linalg.solve(H.T, e)
    return np.linalg.eigvals(H + Hbar[k, k - 1] ** 2 * np.outer(f, e))


def leja_order(theta: np.ndarray) -> np.ndarray:
    """Modified Leja ordering: start from the largest modulus, then repeatedly take the point
    maximising the product of distances to the points already taken (sum of logs).  A complex
    point is taken with its conjugate right after it (positive imaginary part first)."""
    pts = [complex(t) for t in theta]
    remaining = [z for z in pts if z.imag >= 0.0]  # one representative per conjugate pair
    out: list[complex] = []

    def take(z):
        out.append(z)
        if z.imag > 0.0:
            out.append(z.conjugate())
        remaining.remove(z)

    if not remaining:
        return np.array([], dtype=complex)
    take(max(remaining, key=abs))
    while remaining:
        chosen = np.array(out)
        with np.errstate(divide="ignore"):
            scores = [np.sum(np.log(np.abs(z - chosen))) for z in remaining]
        take(remaining[int(np.argmax(scores))])
    return np.array(out, dtype=complex)


def poly_roots(opA, n: int, degree: int, seed: int = 0, v0: np.ndarray | None = None):
    """Leja-ordered roots of the GMRES residual polynomial of the given degree (d+1 roots;
    fewer after an Arnoldi breakdown).  opA(v) = A v in FP64."""
    if degree <= 0:
        return np.array([], dtype=complex)
    if v0 is None:
        v0 = splitmix64_uniform(seed, n)
    _, Hbar, k = arnoldi(opA, np.asarray(v0, dtype=np.float64), degree + 1)
    return leja_order(harmonic_ritz(Hbar[:k + 1, :k]))


def poly_apply(opA, roots: np.ndarray, v: np.ndarray, rw=None) -> np.ndarray:
    """y = p(A) v in product form (d matrix-vector products); rw rounds each vector result
    to the working precision (identity for FP64)."""
    rw = rw or (lambda t: np.asarray(t, dtype=np.float64))
    y = np.zeros_like(v, dtype=np.float64)
    prod = np.asarray(v, dtype=np.float64).copy()
    roots = np.asarray(roots, dtype=complex)
    nr = len(roots)
    i = 0
    while i < nr:
        th = roots[i]
        if th.imag == 0.0:
            t = th.real
            y = rw(y + prod / t)
            if i + 1 < nr:
                prod = rw(prod - opA(prod) / t)
            i += 1
        else:
            a, mod2 = th.real, abs(th) ** 2
            ap = opA(prod)
            y = rw(y + (2.0 * a / mod2) * prod - ap / mod2)
            if i + 2 < nr:
                prod = rw(prod - (2.0 * a / mod2) * ap + opA(ap) / mod2)
            i += 2
    return y
