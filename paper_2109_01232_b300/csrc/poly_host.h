// poly_host.h -- host part of the GMRES-polynomial set-up (Section 3.4):
// harmonic Ritz values of the (d+1)-step Arnoldi matrix and their Leja order.
//
// Harmonic Ritz values: eigenvalues of Hk + h_{k+1,k}^2 f e_k^T with f = Hk^{-T} e_k
// (Hk the square k x k Hessenberg block).  The rank-one term only changes the
// last column, so the matrix stays upper Hessenberg and its eigenvalues come from
// the implicit double-shift (Francis) QR iteration on a real Hessenberg matrix
// (Golub & Van Loan, Matrix Computations, Alg. 7.5.1/7.5.2), written here for
// eigenvalues only.  Complex eigenvalues come out as exact conjugate pairs of the
// trailing 2x2 blocks.
#pragma once

#include <cmath>
#include <complex>
#include <vector>

namespace gm {

// Solve the dense n x n system M z = rhs (row-major M), Gaussian elimination with
// partial pivoting.  Returns false for a singular matrix.
inline bool dense_solve(std::vector<double> M, std::vector<double>& z, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(M[i * n + k]) > std::fabs(M[piv * n + k])) piv = i;
    if (M[piv * n + k] == 0.0) return false;
    if (piv != k) {
      for (int c = 0; c < n; ++c) std::swap(M[k * n + c], M[piv * n + c]);
      std::swap(z[k], z[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = M[i * n + k] / M[k * n + k];
      if (f == 0.0) continue;
      for (int c = k; c < n; ++c) M[i * n + c] -= f * M[k * n + c];
      z[i] -= f * z[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = z[k];
    for (int c = k + 1; c < n; ++c) s -= M[k * n + c] * z[c];
    z[k] = s / M[k * n + k];
  }
  return true;
}

// Eigenvalues of the real upper Hessenberg matrix H (n x n, row-major, modified in
// place).  Returns false if the iteration does not converge.
inline bool hessenberg_eigenvalues(std::vector<double>& H, int n, std::vector<double>& wr,
                                   std::vector<double>& wi) {
  auto h = [&](int i, int j) -> double& { return H[(size_t)i * n + j]; };
  wr.assign(n, 0.0);
  wi.assign(n, 0.0);
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, its = 0;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      double s = std::fabs(h(l - 1, l - 1)) + std::fabs(h(l, l));
      if (s == 0.0) s = 1.0;
      if (std::fabs(h(l, l - 1)) <= eps * s) {
        h(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {  // 1x1 block
      wr[hi] = h(hi, hi);
      wi[hi] = 0.0;
      --hi;
      its = 0;
      continue;
    }
    if (l == hi - 1) {  // 2x2 block
      const double a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
      const double p = 0.5 * (a - d), mean = 0.5 * (a + d);
      const double disc = p * p + b * c;
      if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        // larger-magnitude root first, the other from the determinant (no cancellation)
        const double r1 = mean + (mean >= 0.0 ? sq : -sq);
        const double det = a * d - b * c;
        const double r2 = r1 != 0.0 ? det / r1 : mean - (mean >= 0.0 ? sq : -sq);
        wr[hi - 1] = r1;
        wr[hi] = r2;
        wi[hi - 1] = wi[hi] = 0.0;
      } else {
        const double im = std::sqrt(-disc);
        wr[hi - 1] = wr[hi] = mean;
        wi[hi - 1] = im;
        wi[hi] = -im;
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (++its > 60 * n) return false;
    // Shift polynomial from the trailing 2x2 block (exceptional shifts every 11 iterations).
    double s, t;
    if (its % 11 == 10) {
      const double w = std::fabs(h(hi, hi - 1)) + std::fabs(h(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    } else {
      s = h(hi - 1, hi - 1) + h(hi, hi);
      t = h(hi - 1, hi - 1) * h(hi, hi) - h(hi - 1, hi) * h(hi, hi - 1);
    }
    // First column of (H - s1 I)(H - s2 I) restricted to the active block.
    double x = h(l, l) * h(l, l) + h(l, l + 1) * h(l + 1, l) - s * h(l, l) + t;
    double y = h(l + 1, l) * (h(l, l) + h(l + 1, l + 1) - s);
    double z = h(l + 1, l) * h(l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      // Householder reflector P = I - 2 u u^T / (u^T u) with P [x y z]^T = [alpha 0 0]^T.
      const double nrm = std::sqrt(x * x + y * y + z * z);
      if (nrm != 0.0) {
        const double alpha = x >= 0.0 ? -nrm : nrm;
        const double u0 = x - alpha, u1 = y, u2 = z;
        const double beta = 2.0 / (u0 * u0 + u1 * u1 + u2 * u2);
        const int c0 = k > l ? k - 1 : l;
        for (int c = c0; c <= hi; ++c) {  // rows k..k+2 from the left
          const double d = beta * (u0 * h(k, c) + u1 * h(k + 1, c) + u2 * h(k + 2, c));
          h(k, c) -= d * u0;
          h(k + 1, c) -= d * u1;
          h(k + 2, c) -= d * u2;
        }
        const int r1 = std::min(k + 3, hi);
        for (int r = l; r <= r1; ++r) {  // columns k..k+2 from the right
          const double d = beta * (h(r, k) * u0 + h(r, k + 1) * u1 + h(r, k + 2) * u2);
          h(r, k) -= d * u0;
          h(r, k + 1) -= d * u1;
          h(r, k + 2) -= d * u2;
        }
      }
      x = h(k + 1, k);
      y = h(k + 2, k);
      if (k < hi - 2) z = h(k + 3, k);
    }
    // Final 2-vector reflector on rows/columns hi-1, hi.
    const double nrm = std::sqrt(x * x + y * y);
    if (nrm != 0.0) {
      const double alpha = x >= 0.0 ? -nrm : nrm;
      const double u0 = x - alpha, u1 = y;
      const double beta = 2.0 / (u0 * u0 + u1 * u1);
      for (int c = hi - 2; c <= hi; ++c) {
        const double d = beta * (u0 * h(hi - 1, c) + u1 * h(hi, c));
        h(hi - 1, c) -= d * u0;
        h(hi, c) -= d * u1;
      }
      for (int r = l; r <= hi; ++r) {
        const double d = beta * (h(r, hi - 1) * u0 + h(r, hi) * u1);
        h(r, hi - 1) -= d * u0;
        h(r, hi) -= d * u1;
      }
    }
  }
  return true;
}

// Harmonic Ritz values of a column-major (k+1) x k Hessenberg matrix Hb (ld = k+1).
inline bool harmonic_ritz_values(const double* Hb, int k, std::vector<double>& wr,
                                 std::vector<double>& wi) {
  std::vector<double> M((size_t)k * k);  // row-major Hk
  for (int i = 0; i < k; ++i)
    for (int c = 0; c < k; ++c) M[(size_t)i * k + c] = Hb[i + (size_t)c * (k + 1)];
  // f solves Hk^T f = e_k
  std::vector<double> Mt((size_t)k * k);
  for (int i = 0; i < k; ++i)
    for (int c = 0; c < k; ++c) Mt[(size_t)i * k + c] = M[(size_t)c * k + i];
  std::vector<double> f(k, 0.0);
  f[k - 1] = 1.0;
  if (!dense_solve(Mt, f, k)) return false;
  const double hl = Hb[k + (size_t)(k - 1) * (k + 1)];
  for (int i = 0; i < k; ++i) M[(size_t)i * k + (k - 1)] += hl * hl * f[i];
  return hessenberg_eigenvalues(M, k, wr, wi);
}

// Modified Leja order: largest modulus first, then the point maximising the sum of
// log distances to the points already chosen; a complex point (positive imaginary
// part) is followed by its conjugate.
inline void leja_order(std::vector<double>& wr, std::vector<double>& wi) {
  using C = std::complex<double>;
  std::vector<C> cand;
  for (size_t i = 0; i < wr.size(); ++i)
    if (wi[i] >= 0.0) cand.emplace_back(wr[i], wi[i]);
  std::vector<C> out;
  std::vector<bool> used(cand.size(), false);
  auto take = [&](size_t i) {
    used[i] = true;
    out.push_back(cand[i]);
    if (cand[i].imag() > 0.0) out.push_back(std::conj(cand[i]));
  };
  if (cand.empty()) {
    wr.clear();
    wi.clear();
    return;
  }
  size_t best = 0;
  for (size_t i = 1; i < cand.size(); ++i)
    if (std::abs(cand[i]) > std::abs(cand[best])) best = i;
  take(best);
  for (size_t step = 1; step < cand.size(); ++step) {
    double bscore = -INFINITY;
    size_t bi = cand.size();
    for (size_t i = 0; i < cand.size(); ++i) {
      if (used[i]) continue;
      double sc = 0.0;
      for (const C& c : out) sc += std::log(std::abs(cand[i] - c));
      if (bi == cand.size() || sc > bscore) {
        bscore = sc;
        bi = i;
      }
    }
    take(bi);
  }
  wr.resize(out.size());
  wi.resize(out.size());
  for (size_t i = 0; i < out.size(); ++i) {
    wr[i] = out[i].real();
    wi[i] = out[i].imag();
  }
}

}  // namespace gm
