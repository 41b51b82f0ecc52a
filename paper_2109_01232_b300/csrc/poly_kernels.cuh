// poly_kernels.cuh -- right preconditioning with the GMRES polynomial (Section 3.4):
// z = p(A) v in product form over the Leja-ordered roots theta_i of the GMRES residual
// polynomial phi(t) = prod_i (1 - t / theta_i), p(t) = (1 - phi(t)) / t.
//
//   real root theta:         y += prod / theta;          prod <- prod - (A prod) / theta
//   pair a +- ib, q = a^2+b^2: t = A prod;  y += (2a/q) prod - t/q;
//                            prod <- prod - (2a/q) t + (A t)/q
// (the prod update is skipped for the last root or pair).  Each matrix product is one
// SpMV kernel whose epilogue applies the vector updates row by row, so a degree-d
// polynomial costs d SpMV launches and no separate vector passes.  The matrix is the
// plan's SELL-32 copy in the inner storage precision; prod, t and y are in the working
// precision (FP32 for the FP32/FP16/BF16 inner cycles).
#pragma once

#include "kernels.cuh"

namespace gm {

enum { POLY_REAL = 0, POLY_PAIR_A = 1, POLY_PAIR_B = 2 };

__device__ __forceinline__ int poly_skip(const DevState* st, int in_cycle) {
  return read_flag(&st->stop) | (in_cycle ? read_flag(&st->cycle_done) : 0);
}

// First kernel of p(A) v_j inside an Arnoldi step.  For j > 0 it first applies the
// Givens update of step j-1 (every CTA computes it from the cluster's column sums, CTA 0
// stores it: see k_spmv_sell),
// which gives 1 / h_{j,j-1}; then V[:, j] = store(v_scale * sigma * src) (the
// normalisation of the previous step) and prod = v_j in the working type.
// PW: type of prod (the polynomial's working type; FP32 under an FP64 cycle when the
// polynomial is applied in single precision).
template <int P, class SrcT, class PW = typename Tr<P>::W>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT) k_poly_start(const SrcT* __restrict__ src, double v_scale,
                                                   int n, typename Tr<P>::S* V, long long ld,
                                                   int j, PW* __restrict__ prod,
                                                   StepParts<typename Tr<P>::W> parts,
                                                   DevState* st, Arrays arr) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  __shared__ double gsh[GIVENS_SH];
  __shared__ int s_skip;
  __shared__ W s_mine[2], s_nrm[2];
  double sigma;
  if (j > 0) {
    finalize_load(st, arr, j - 1, gsh);
    const W* pn = parts.p1_of(j - 1) + (long long)j * parts.g1;
    const auto col = [&](int c) {
      return c == 0 ? ColumnSrc<W>{parts.p3, parts.g2} : ColumnSrc<W>{pn, parts.g1};
    };
    if (!cluster_column_sums<W>(col, 2, s_mine, s_nrm, [&] { return poly_skip(st, 1); })) return;
    int done;
    finalize_compute(st, arr, j - 1, (double)s_nrm[0], (double)s_nrm[1], blockIdx.x == 0, gsh,
                     &done, &sigma);
    if (done) return;
  } else {
    if (threadIdx.x == 0) s_skip = poly_skip(st, 1);
    __syncthreads();
    if (s_skip) return;
    sigma = st->sigma;
  }
  const SrcT f = (SrcT)(v_scale * sigma);
  const W inv = (W)pow2_recip(v_scale);
  S* Vj = V + (long long)j * ld;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    const S v = to_s<S>(f * src[i]);
    Vj[i] = v;
    prod[i] = (PW)(to_w(v) * inv);
  }
}

// One matrix product of the product form with its vector updates (KIND above).
//   POLY_REAL:   t = A prod;  y = y0 + c1 prod;  out = prod - c1 t   (out == nullptr: skip)
//   POLY_PAIR_A: t = A prod;  y = y0 + c1 prod - c2 t;  out = t      (out == nullptr: skip)
//   POLY_PAIR_B: s = A tin;   out = prod - c1 tin + c2 s
// y0 = 0 when `first`, else the current y.  in_cycle: also skip once the cycle ended.
template <int P, int KIND>
__global__ void __launch_bounds__(NT, 2) k_poly_spmv(
    const int2* __restrict__ meta, const int* __restrict__ ci,
    const typename Tr<P>::S* __restrict__ av, int nslices,
    int n, double a_scale, const typename Tr<P>::W* __restrict__ prod,
    const typename Tr<P>::W* __restrict__ tin, typename Tr<P>::W* __restrict__ y,
    typename Tr<P>::W* __restrict__ out, double c1d, double c2d, int first, const DevState* st,
    int in_cycle) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int TR = SpmvSmem<P>::TR;
  constexpr int RPT = TR / NT;
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = poly_skip(st, in_cycle);
  __syncthreads();
  if (s_skip) return;
  const W as = (W)a_scale, c1 = (W)c1d, c2 = (W)c2d;
  const W* gsrc = KIND == POLY_PAIR_B ? tin : prod;
  auto xval = [&](int c) -> W { return gsrc[c]; };
  const bool ms = st->stream_matrix != 0;
  const int ntiles = (n + TR - 1) / TR;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * TR;
    W a[RPT];
    sell_rows<S, W, RPT>(meta, ci, av, nslices, r0, xval, a, ms);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int row = r0 + threadIdx.x + k * NT;
      if (row >= n) continue;
      const W ap = as * a[k];
      const W pv = prod[row];
      if (KIND == POLY_REAL) {
        y[row] = (first ? W(0) : y[row]) + c1 * pv;
        if (out) out[row] = pv - c1 * ap;
      } else if (KIND == POLY_PAIR_A) {
        y[row] = (first ? W(0) : y[row]) + c1 * pv - c2 * ap;
        if (out) out[row] = ap;
      } else {
        out[row] = pv - c1 * tin[row] + c2 * ap;
      }
    }
  }
}

// y = A x with the plan's SELL-32 copy alone (no dot products, no basis store): the SpMV
// of the fp64-vs-fp32 timing entry point (Section 5.5's experiment).
template <int P>
__global__ void __launch_bounds__(NT, 2) k_spmv_plain(const int2* __restrict__ meta, const int* __restrict__ ci,
                                                   const typename Tr<P>::S* __restrict__ av, int nslices,
                                                   int n, double a_scale,
                                                   const typename Tr<P>::W* __restrict__ x,
                                                   typename Tr<P>::W* __restrict__ y) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int TR = SpmvSmem<P>::TR;
  constexpr int RPT = TR / NT;
  const W as = (W)a_scale;
  auto xval = [&](int c) -> W { return x[c]; };
  const int ntiles = (n + TR - 1) / TR;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * TR;
    W a[RPT];
    sell_rows<S, W, RPT>(meta, ci, av, nslices, r0, xval, a);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int row = r0 + threadIdx.x + k * NT;
      if (row < n) y[row] = as * a[k];
    }
  }
}

// Last real root: y = y0 + c1 prod (no matrix product).
template <int P>
__global__ void __launch_bounds__(NT) k_poly_axpy(const typename Tr<P>::W* __restrict__ prod,
                                                  typename Tr<P>::W* __restrict__ y, int n,
                                                  double c1d, int first, const DevState* st,
                                                  int in_cycle) {
  using W = typename Tr<P>::W;
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = poly_skip(st, in_cycle);
  __syncthreads();
  if (s_skip) return;
  const W c1 = (W)c1d;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
    y[i] = (first ? W(0) : y[i]) + c1 * prod[i];
}

// Cycle end with a preconditioner: prod = (V y_ls) / v_scale in the working type
// (the correction before p(A) is applied).
template <int P, class UW = typename Tr<P>::W>
__global__ void __launch_bounds__(NT) k_vy(const typename Tr<P>::S* __restrict__ V, long long ld,
                                           double v_scale, const DevState* st,
                                           const double* __restrict__ y, UW* __restrict__ u) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* coef = reinterpret_cast<W*>(smem_raw);
  __shared__ int s_skip, s_kk;
  if (threadIdx.x == 0) {
    s_skip = read_flag(&st->stop);
    s_kk = st->k_used;
  }
  __syncthreads();
  if (s_skip) return;
  const int kk = s_kk;
  for (int c = threadIdx.x; c < kk; c += NT) coef[c] = (W)y[c];
  __syncthreads();
  const W inv = (W)pow2_recip(v_scale);
  const long long ngroups = ld / VEC;
  const long long g0 = cta_begin(ngroups, 32), g1 = cta_begin(ngroups, 32, 1);
  for (long long g = g0 + threadIdx.x; g < g1; g += NT) {
    const long long base = g * VEC;
    W acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = W(0);
    for (int c = 0; c < kk; ++c) {
      S v0[VEC];
      ldv(V + (long long)c * ld + base, v0);
      const W k0 = coef[c];
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] += k0 * to_w(v0[q]);
    }
#pragma unroll
    for (int q = 0; q < VEC; ++q) u[base + q] = (UW)(acc[q] * inv);
  }
}

// x += gamma * z (FP64 update of Algorithm 2 with the preconditioned correction z).
template <class ZW>
__global__ void __launch_bounds__(NT) k_xadd(const ZW* __restrict__ z, double* __restrict__ x, int n,
                                             const DevState* st) {
  __shared__ int s_skip;
  __shared__ double s_g;
  if (threadIdx.x == 0) {
    s_skip = read_flag(&st->stop);
    s_g = st->gamma;
  }
  __syncthreads();
  if (s_skip) return;
  const double g = s_g;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
    x[i] += g * (double)z[i];
}

// prod = (W) v for the stand-alone p(A) v entry point.
template <int P>
__global__ void k_load_work(const double* __restrict__ v, typename Tr<P>::W* __restrict__ out, int n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (typename Tr<P>::W)v[i];
}

}  // namespace gm
