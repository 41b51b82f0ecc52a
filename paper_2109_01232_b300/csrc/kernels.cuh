// kernels.cuh -- the GMRES(m) / GMRES-IR hot path for sm_103a.
//
// One Arnoldi step j (Algorithm 1 lines "w = A v_j" to "v_{j+1} = w / h_{j+1,j}",
// with the CGS2 orthogonalisation of Section 3.1) is three kernels:
//
//   k_spmv_arnoldi  v_j = store(sigma * src) for the tile's own rows (the
//                   normalisation of the previous step, done here so that no
//                   separate pass touches the vector), w = A v_j (CSR, FP32 or
//                   FP64 accumulation), then h1 = V_j^T w and ||w||^2 while w is
//                   still on chip (first CGS pass, transposed GEMV).
//   k_cgs_u1        w' = w - V_j h1 (first CGS pass, plain GEMV) and h2 = V_j^T w'
//                   (second pass, transposed GEMV) over the same rows.
//   k_cgs_u2        w'' = w' - V_j h2 (second pass, plain GEMV) and ||w''||^2; the
//                   last CTA to finish forms H[:, j] = h1 + h2, h_{j+1,j} = ||w''||,
//                   applies the Givens rotations in FP64 and sets the cycle flags.
//
// Cross-CTA sums are deterministic: each CTA writes its partial sums, and the
// last CTA to arrive (atomic ticket) adds them in a fixed order.  No kernel
// waits on another CTA, so nothing can spin.  Every kernel first reads the
// device flags and returns at once when the cycle or the solve has ended, which
// lets a captured graph of the whole cycle run without the host.
//
// Memory layout: V is column-major with leading dimension ld (a multiple of
// TILE_MAX, 16-byte aligned columns, zero padding rows); work vectors have the
// same length ld and zero padding, so vector loads never need a tail.
#pragma once

#include "common.cuh"

namespace gm {

__device__ __forceinline__ int read_flag(const int* p) { return *(volatile const int*)p; }

// ---------------------------------------------------------------------------
// CSR tile engine: computes sum_p a[p] * xval(col[p]) for the rows
// r0 + tid + k*NT (k < RPT) of one tile of TR rows.  The tile's nonzeros are
// streamed with coalesced loads in chunks of CAP entries; each product goes to
// shared memory and every thread then sums its rows' contiguous ranges.
// ---------------------------------------------------------------------------
template <class AT, class W, int TR, int CAP, class XF>
__device__ __forceinline__ void tile_spmv(const int* __restrict__ rp, const int* __restrict__ ci,
                                          const AT* __restrict__ av, int n, int r0,
                                          int* __restrict__ rp_s, W* __restrict__ prod_s,
                                          const XF& xval, W (&acc)[TR / NT]) {
  constexpr int RPT = TR / NT;
  const int tid = threadIdx.x;
  const int rows = min(TR, n - r0);
  for (int i = tid; i <= rows; i += NT) rp_s[i] = rp[r0 + i];
#pragma unroll
  for (int k = 0; k < RPT; ++k) acc[k] = W(0);
  __syncthreads();
  const int p0 = rp_s[0], p1 = rp_s[rows];
  for (int c0 = p0; c0 < p1; c0 += CAP) {
    const int c1 = min(c0 + CAP, p1);
    int e = c0 + tid;
    for (; e + 3 * NT < c1; e += 4 * NT) {
      const int ca = ci[e], cb = ci[e + NT], cc = ci[e + 2 * NT], cd = ci[e + 3 * NT];
      const AT aa = av[e], ab = av[e + NT], ac = av[e + 2 * NT], ad = av[e + 3 * NT];
      const W xa = xval(ca), xb = xval(cb), xc = xval(cc), xd = xval(cd);
      prod_s[e - c0] = to_w(aa) * xa;
      prod_s[e + NT - c0] = to_w(ab) * xb;
      prod_s[e + 2 * NT - c0] = to_w(ac) * xc;
      prod_s[e + 3 * NT - c0] = to_w(ad) * xd;
    }
    for (; e < c1; e += NT) prod_s[e - c0] = to_w(av[e]) * xval(ci[e]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int il = tid + k * NT;
      if (il < rows) {
        const int s = max(rp_s[il], c0) - c0, t = min(rp_s[il + 1], c1) - c0;
        W a = acc[k];
        for (int p = s; p < t; ++p) a += prod_s[p];
        acc[k] = a;
      }
    }
    __syncthreads();
  }
}

// Last-CTA detection for the deterministic two-level reductions.
__device__ __forceinline__ bool arrive_last(unsigned int* ticket, int* s_last) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!*s_last) return false;
  __threadfence();
  return true;
}

template <int P>
struct SpmvSmem {
  using W = typename Tr<P>::W;
  static constexpr int TR = NT * Tr<P>::VEC;
  static constexpr int CAP = TR * 8;
  static size_t bytes(int ncol) {
    return sizeof(W) * (size_t)(CAP + TR + NWARP * ncol) + sizeof(int) * (size_t)(TR + 1) + 16;
  }
};

// ---------------------------------------------------------------------------
// Step kernel 1: normalise + SpMV + first-pass dot products.
//   V[:, j] = store(v_scale * sigma * src)            (rows of this tile)
//   w = (a_scale / v_scale) * A_stored * V[:, j]      (= A v_j)
//   h1[c] = v_c . w  (c <= j),  wnorm = ||w||
// src is the FP64 residual (j = 0) or the previous step's w'' (working type).
// PLAIN: src is already the vector to multiply (p(A) v_j with a polynomial
// preconditioner, working type, unscaled): it is gathered as is and V[:, j], stored
// by the polynomial's first kernel, is not written.
// ---------------------------------------------------------------------------
template <int P, class SrcT, bool PLAIN = false>
__global__ void __launch_bounds__(NT) k_spmv_arnoldi(
    const int* __restrict__ rp, const int* __restrict__ ci, const typename Tr<P>::S* __restrict__ av,
    int n, long long ld, double row_scale_d, const SrcT* __restrict__ src, double v_scale,
    typename Tr<P>::S* V, int j, typename Tr<P>::W* __restrict__ wout,
    typename Tr<P>::W* __restrict__ part, DevState* st, double* __restrict__ h1) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VEC;
  constexpr int TR = SpmvSmem<P>::TR;
  constexpr int CAP = SpmvSmem<P>::CAP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* prod_s = reinterpret_cast<W*>(smem_raw);
  W* w_s = prod_s + CAP;
  W* acc = w_s + TR;
  const int ncol = j + 2;
  int* rp_s = reinterpret_cast<int*>(acc + NWARP * ncol);
  __shared__ int s_skip, s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_flag(&st->stop) | read_flag(&st->cycle_done);
  __syncthreads();
  if (s_skip) return;
  for (int i = tid; i < NWARP * ncol; i += NT) acc[i] = W(0);

  const SrcT f = (SrcT)(v_scale * st->sigma);
  const W row_scale = (W)row_scale_d;
  auto make = [&](SrcT x) -> S { return to_s<S>(f * x); };
  auto xval = [&](int c) -> W {
    if constexpr (PLAIN) return (W)src[c];
    else return to_w(make(src[c]));
  };
  S* Vj = V + (long long)j * ld;

  const int ntiles = (n + TR - 1) / TR;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * TR;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const int row = r0 + tid + k * NT;
      if (!PLAIN && row < n) Vj[row] = make(src[row]);
    }
    W a[VEC];
    tile_spmv<S, W, TR, CAP>(rp, ci, av, n, r0, rp_s, prod_s, xval, a);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const int il = tid + k * NT;
      const int row = r0 + il;
      const W wv = (row < n) ? row_scale * a[k] : W(0);
      w_s[il] = wv;
      if (row < n) wout[row] = wv;
    }
    __syncthreads();
    // First CGS pass, transposed GEMV: VEC consecutive rows per thread.
    const long long gb = (long long)r0 + tid * VEC;
    W wv[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) wv[q] = w_s[tid * VEC + q];
    W nrm = W(0);
#pragma unroll
    for (int q = 0; q < VEC; ++q) nrm += wv[q] * wv[q];
    int c = 0;
    for (; c + 4 <= j + 1; c += 4) {
      S v0[VEC], v1[VEC], v2[VEC], v3[VEC];
      ldv(V + (long long)c * ld + gb, v0);
      ldv(V + (long long)(c + 1) * ld + gb, v1);
      ldv(V + (long long)(c + 2) * ld + gb, v2);
      ldv(V + (long long)(c + 3) * ld + gb, v3);
      W d0 = 0, d1 = 0, d2 = 0, d3 = 0;
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        d0 += to_w(v0[q]) * wv[q];
        d1 += to_w(v1[q]) * wv[q];
        d2 += to_w(v2[q]) * wv[q];
        d3 += to_w(v3[q]) * wv[q];
      }
      d0 = warp_sum(d0); d1 = warp_sum(d1); d2 = warp_sum(d2); d3 = warp_sum(d3);
      if (lane == 0) {
        W* ac = acc + warp * ncol + c;
        ac[0] += d0; ac[1] += d1; ac[2] += d2; ac[3] += d3;
      }
    }
    for (; c <= j; ++c) {
      S v0[VEC];
      ldv(V + (long long)c * ld + gb, v0);
      W d0 = 0;
#pragma unroll
      for (int q = 0; q < VEC; ++q) d0 += to_w(v0[q]) * wv[q];
      d0 = warp_sum(d0);
      if (lane == 0) acc[warp * ncol + c] += d0;
    }
    nrm = warp_sum(nrm);
    if (lane == 0) acc[warp * ncol + j + 1] += nrm;
    __syncthreads();
  }
  const int G = gridDim.x;
  for (int c = tid; c < ncol; c += NT) {
    W s = W(0);
    for (int w = 0; w < NWARP; ++w) s += acc[w * ncol + c];
    part[(long long)c * G + blockIdx.x] = s;
  }
  if (!arrive_last(&st->ticket[0], &s_last)) return;
  for (int c = warp; c < ncol; c += NWARP) {
    W s = W(0);
    for (int b = lane; b < G; b += 32) s += __ldcg(&part[(long long)c * G + b]);
    s = warp_sum(s);
    if (lane == 0) {
      if (c <= j) h1[c] = (double)s / v_scale;
      else st->wnorm = sqrt((double)s);
    }
  }
  if (tid == 0) st->ticket[0] = 0;
}

// Store V[:, j] = store(v_scale * sigma * src) for all rows (the last basis vector of
// an Arnoldi run that is not followed by another SpMV).
template <int P, class SrcT>
__global__ void k_store_basis(const SrcT* __restrict__ src, double v_scale, int n,
                              typename Tr<P>::S* V, long long ld, int j, const DevState* st) {
  using S = typename Tr<P>::S;
  const SrcT f = (SrcT)(v_scale * st->sigma);
  S* Vj = V + (long long)j * ld;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    Vj[i] = to_s<S>(f * src[i]);
}

// ---------------------------------------------------------------------------
// Step kernel 2: w' = w - V_j h1 (first pass update) and h2 = V_j^T w'.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(NT) k_cgs_u1(const typename Tr<P>::S* __restrict__ V, long long ld,
                                               int j, double v_scale,
                                               const typename Tr<P>::W* __restrict__ win,
                                               typename Tr<P>::W* __restrict__ wout,
                                               typename Tr<P>::W* __restrict__ part, DevState* st,
                                               const double* __restrict__ h1,
                                               double* __restrict__ h2) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = j + 1;
  W* coef = reinterpret_cast<W*>(smem_raw);
  W* acc = coef + nc;
  __shared__ int s_skip, s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_flag(&st->stop) | read_flag(&st->cycle_done);
  __syncthreads();
  if (s_skip) return;
  for (int c = tid; c < nc; c += NT) coef[c] = (W)(h1[c] / v_scale);
  for (int i = tid; i < NWARP * nc; i += NT) acc[i] = W(0);
  __syncthreads();
  const long long ngroups = ld / VEC;
  for (long long g = (long long)blockIdx.x * NT + tid; g < ngroups; g += (long long)gridDim.x * NT) {
    const long long base = g * VEC;
    W wv[VEC];
    ldv(win + base, wv);
    int c = 0;
    for (; c + 4 <= nc; c += 4) {
      S v0[VEC], v1[VEC], v2[VEC], v3[VEC];
      ldv(V + (long long)c * ld + base, v0);
      ldv(V + (long long)(c + 1) * ld + base, v1);
      ldv(V + (long long)(c + 2) * ld + base, v2);
      ldv(V + (long long)(c + 3) * ld + base, v3);
      const W k0 = coef[c], k1 = coef[c + 1], k2 = coef[c + 2], k3 = coef[c + 3];
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        W t = wv[q];
        t -= k0 * to_w(v0[q]);
        t -= k1 * to_w(v1[q]);
        t -= k2 * to_w(v2[q]);
        t -= k3 * to_w(v3[q]);
        wv[q] = t;
      }
    }
    for (; c < nc; ++c) {
      S v0[VEC];
      ldv(V + (long long)c * ld + base, v0);
      const W k0 = coef[c];
#pragma unroll
      for (int q = 0; q < VEC; ++q) wv[q] -= k0 * to_w(v0[q]);
    }
    stv(wout + base, wv);
    c = 0;
    for (; c + 4 <= nc; c += 4) {
      S v0[VEC], v1[VEC], v2[VEC], v3[VEC];
      ldv(V + (long long)c * ld + base, v0);
      ldv(V + (long long)(c + 1) * ld + base, v1);
      ldv(V + (long long)(c + 2) * ld + base, v2);
      ldv(V + (long long)(c + 3) * ld + base, v3);
      W d0 = 0, d1 = 0, d2 = 0, d3 = 0;
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        d0 += to_w(v0[q]) * wv[q];
        d1 += to_w(v1[q]) * wv[q];
        d2 += to_w(v2[q]) * wv[q];
        d3 += to_w(v3[q]) * wv[q];
      }
      d0 = warp_sum(d0); d1 = warp_sum(d1); d2 = warp_sum(d2); d3 = warp_sum(d3);
      if (lane == 0) {
        W* ac = acc + warp * nc + c;
        ac[0] += d0; ac[1] += d1; ac[2] += d2; ac[3] += d3;
      }
    }
    for (; c < nc; ++c) {
      S v0[VEC];
      ldv(V + (long long)c * ld + base, v0);
      W d0 = 0;
#pragma unroll
      for (int q = 0; q < VEC; ++q) d0 += to_w(v0[q]) * wv[q];
      d0 = warp_sum(d0);
      if (lane == 0) acc[warp * nc + c] += d0;
    }
  }
  __syncthreads();
  const int G = gridDim.x;
  for (int c = tid; c < nc; c += NT) {
    W s = W(0);
    for (int w = 0; w < NWARP; ++w) s += acc[w * nc + c];
    part[(long long)c * G + blockIdx.x] = s;
  }
  if (!arrive_last(&st->ticket[1], &s_last)) return;
  for (int c = warp; c < nc; c += NWARP) {
    W s = W(0);
    for (int b = lane; b < G; b += 32) s += __ldcg(&part[(long long)c * G + b]);
    s = warp_sum(s);
    if (lane == 0) h2[c] = (double)s / v_scale;
  }
  if (tid == 0) st->ticket[1] = 0;
}

// Givens update of column j (Algorithm 1's least-squares problem solved
// incrementally, FP64, one thread).  Sets the cycle/solve flags.
__device__ void givens_step(DevState* st, const Arrays& a, int j, double hn) {
  const int m = st->m;
  const int ldh = m + 1;
  double* Hc = a.H + (long long)j * ldh;
  double* Rc = a.R + (long long)j * ldh;
  for (int i = 0; i <= j; ++i) Hc[i] = a.h1[i] + a.h2[i];
  Hc[j + 1] = hn;
  for (int i = 0; i <= j + 1; ++i) Rc[i] = Hc[i];
  for (int i = 0; i < j; ++i) {
    const double t = a.cs[i] * Rc[i] + a.sn[i] * Rc[i + 1];
    Rc[i + 1] = -a.sn[i] * Rc[i] + a.cs[i] * Rc[i + 1];
    Rc[i] = t;
  }
  const double x = Rc[j], y = hn;
  double c = 1.0, s = 0.0;
  if (y != 0.0) {
    const double rho = hypot(x, y);
    c = x / rho;
    s = y / rho;
  }
  Rc[j] = c * x + s * y;
  Rc[j + 1] = 0.0;
  a.cs[j] = c;
  a.sn[j] = s;
  a.g[j + 1] = -s * a.g[j];
  a.g[j] = c * a.g[j];
  st->k = j + 1;
  st->iters += 1;
  const double res = fabs(a.g[j + 1]);
  if (st->iters <= st->hist_cap)
    a.hist[st->iters - 1] = res * st->gamma / (st->bnorm > 0.0 ? st->bnorm : 1.0);
  if (!isfinite(hn) || !isfinite(res) || !isfinite(Rc[j])) {
    st->status = ST_NONFINITE;
    st->stop = 1;
    st->cycle_done = 1;
    return;
  }
  const int brk = hn <= 16.0 * st->u_work * st->wnorm;
  st->breakdown = brk;
  if (brk || res <= st->stop_rel || j + 1 >= m || st->iters >= st->max_iters) st->cycle_done = 1;
  st->sigma = brk ? 0.0 : 1.0 / hn;
}

// ---------------------------------------------------------------------------
// Step kernel 3: w'' = w' - V_j h2, ||w''||, then the Givens update.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(NT) k_cgs_u2(const typename Tr<P>::S* __restrict__ V, long long ld,
                                               int j, double v_scale,
                                               const typename Tr<P>::W* __restrict__ win,
                                               typename Tr<P>::W* __restrict__ wout,
                                               typename Tr<P>::W* __restrict__ part, DevState* st,
                                               Arrays arr) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = j + 1;
  W* coef = reinterpret_cast<W*>(smem_raw);
  __shared__ W accw[NWARP];
  __shared__ int s_skip, s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_flag(&st->stop) | read_flag(&st->cycle_done);
  __syncthreads();
  if (s_skip) return;
  for (int c = tid; c < nc; c += NT) coef[c] = (W)(arr.h2[c] / v_scale);
  __syncthreads();
  W nrm = W(0);
  const long long ngroups = ld / VEC;
  for (long long g = (long long)blockIdx.x * NT + tid; g < ngroups; g += (long long)gridDim.x * NT) {
    const long long base = g * VEC;
    W wv[VEC];
    ldv(win + base, wv);
    int c = 0;
    for (; c + 4 <= nc; c += 4) {
      S v0[VEC], v1[VEC], v2[VEC], v3[VEC];
      ldv(V + (long long)c * ld + base, v0);
      ldv(V + (long long)(c + 1) * ld + base, v1);
      ldv(V + (long long)(c + 2) * ld + base, v2);
      ldv(V + (long long)(c + 3) * ld + base, v3);
      const W k0 = coef[c], k1 = coef[c + 1], k2 = coef[c + 2], k3 = coef[c + 3];
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        W t = wv[q];
        t -= k0 * to_w(v0[q]);
        t -= k1 * to_w(v1[q]);
        t -= k2 * to_w(v2[q]);
        t -= k3 * to_w(v3[q]);
        wv[q] = t;
      }
    }
    for (; c < nc; ++c) {
      S v0[VEC];
      ldv(V + (long long)c * ld + base, v0);
      const W k0 = coef[c];
#pragma unroll
      for (int q = 0; q < VEC; ++q) wv[q] -= k0 * to_w(v0[q]);
    }
    stv(wout + base, wv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) nrm += wv[q] * wv[q];
  }
  nrm = warp_sum(nrm);
  if (lane == 0) accw[warp] = nrm;
  __syncthreads();
  const int G = gridDim.x;
  if (tid == 0) {
    W s = W(0);
    for (int w = 0; w < NWARP; ++w) s += accw[w];
    part[blockIdx.x] = s;
  }
  if (!arrive_last(&st->ticket[2], &s_last)) return;
  if (warp == 0) {
    W s = W(0);
    for (int b = lane; b < G; b += 32) s += __ldcg(&part[b]);
    s = warp_sum(s);
    if (lane == 0) {
      st->ticket[2] = 0;
      givens_step(st, arr, j, sqrt((double)s));
    }
  }
}

// ---------------------------------------------------------------------------
// End of a cycle: least squares R y = g by back substitution (one warp, FP64).
// A trailing diagonal entry below 16 u max|R| is dropped (singular factor).
// ---------------------------------------------------------------------------
__global__ void k_lsq(DevState* st, Arrays a) {
  __shared__ double gw[LSQ_MAX];
  __shared__ int s_kk;
  const int lane = threadIdx.x;
  if (read_flag(&st->stop)) return;
  const int k = st->k, ldh = st->m + 1;
  double rmax = 0.0;
  for (int c = lane; c < k; c += 32)
    for (int i = 0; i <= c; ++i) rmax = fmax(rmax, fabs(a.R[i + (long long)c * ldh]));
  rmax = warp_max(rmax);
  if (lane == 0) {
    int kk = k;
    while (kk > 0 && fabs(a.R[(kk - 1) + (long long)(kk - 1) * ldh]) <= 16.0 * st->u_work * rmax) --kk;
    s_kk = kk;
    st->k_used = kk;
    st->singular = kk < k;
  }
  __syncwarp();
  const int kk = s_kk;
  for (int i = lane; i < kk; i += 32) gw[i] = a.g[i];
  __syncwarp();
  for (int i = kk - 1; i >= 0; --i) {
    const double yi = gw[i] / a.R[i + (long long)i * ldh];
    __syncwarp();
    for (int l = lane; l < i; l += 32) gw[l] -= a.R[l + (long long)i * ldh] * yi;
    if (lane == 0) a.y[i] = yi;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// x += gamma * V y (the correction u = V y accumulates in the working precision,
// the update is FP64: Algorithm 2, "x_{i+1} = x_i + u_i [double]").
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(NT) k_xupd(const typename Tr<P>::S* __restrict__ V, long long ld,
                                             double v_scale, DevState* st,
                                             const double* __restrict__ y, double* __restrict__ x) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* coef = reinterpret_cast<W*>(smem_raw);
  __shared__ int s_skip, s_kk;
  __shared__ double s_fac;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_skip = read_flag(&st->stop);
    s_kk = st->k_used;
    s_fac = st->gamma / v_scale;
  }
  __syncthreads();
  if (s_skip) return;
  const int kk = s_kk;
  const double fac = s_fac;
  for (int c = tid; c < kk; c += NT) coef[c] = (W)y[c];
  __syncthreads();
  const long long ngroups = ld / VEC;
  for (long long g = (long long)blockIdx.x * NT + tid; g < ngroups; g += (long long)gridDim.x * NT) {
    const long long base = g * VEC;
    W u[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) u[q] = W(0);
    for (int c = 0; c < kk; ++c) {
      S v0[VEC];
      ldv(V + (long long)c * ld + base, v0);
      const W k0 = coef[c];
#pragma unroll
      for (int q = 0; q < VEC; ++q) u[q] += k0 * to_w(v0[q]);
    }
    double xv[VEC];
    ldv(x + base, xv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) xv[q] += fac * (double)u[q];
    stv(x + base, xv);
  }
}

// ---------------------------------------------------------------------------
// FP64 residual r = b - A x with the FP64 master matrix, ||r||, ||b||, and the
// restart decisions (Algorithm 1's explicit residual test / Algorithm 2
// "r_{i+1} = b - A x_{i+1} [double]").
// ---------------------------------------------------------------------------
constexpr int RES_TR = NT * 2;
constexpr int RES_CAP = RES_TR * 8;
inline size_t residual_smem() { return sizeof(double) * RES_CAP + sizeof(int) * (RES_TR + 1) + 16; }

__global__ void __launch_bounds__(NT) k_residual(const int* __restrict__ rp, const int* __restrict__ ci,
                                                 const double* __restrict__ av, int n,
                                                 const double* __restrict__ x,
                                                 const double* __restrict__ b, double* __restrict__ r,
                                                 double* __restrict__ part, DevState* st, Arrays arr,
                                                 int first) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* prod_s = reinterpret_cast<double*>(smem_raw);
  int* rp_s = reinterpret_cast<int*>(prod_s + RES_CAP);
  __shared__ double red_r[NWARP], red_b[NWARP];
  __shared__ int s_skip, s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_flag(&st->stop);
  __syncthreads();
  if (s_skip) return;
  auto xval = [&](int c) -> double { return x[c]; };
  double sr = 0.0, sb = 0.0;
  const int ntiles = (n + RES_TR - 1) / RES_TR;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * RES_TR;
    double a[RES_TR / NT];
    tile_spmv<double, double, RES_TR, RES_CAP>(rp, ci, av, n, r0, rp_s, prod_s, xval, a);
#pragma unroll
    for (int k = 0; k < RES_TR / NT; ++k) {
      const int row = r0 + tid + k * NT;
      if (row < n) {
        const double bv = b[row];
        const double rv = bv - a[k];
        r[row] = rv;
        sr += rv * rv;
        sb += bv * bv;
      }
    }
  }
  sr = warp_sum(sr);
  sb = warp_sum(sb);
  if (lane == 0) { red_r[warp] = sr; red_b[warp] = sb; }
  __syncthreads();
  const int G = gridDim.x;
  if (tid == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < NWARP; ++w) { a += red_r[w]; c += red_b[w]; }
    part[blockIdx.x] = a;
    part[G + blockIdx.x] = c;
  }
  if (!arrive_last(&st->ticket[3], &s_last)) return;
  if (warp == 0) {
    double a = 0.0, c = 0.0;
    for (int q = lane; q < G; q += 32) {
      a += __ldcg(&part[q]);
      c += __ldcg(&part[G + q]);
    }
    a = warp_sum(a);
    c = warp_sum(c);
    if (lane == 0) {
      st->ticket[3] = 0;
      const double gamma = sqrt(a);
      if (first) st->bnorm = sqrt(c);
      else st->outer += 1;
      const double bnorm = st->bnorm;
      st->gamma = gamma;
      st->relres = bnorm > 0.0 ? gamma / bnorm : 0.0;
      int stop = 1, status = ST_OK;
      if (!isfinite(gamma) || !isfinite(bnorm)) status = ST_NONFINITE;
      else if (bnorm == 0.0) { st->zero_rhs = 1; st->relres = 0.0; }
      else if (gamma <= st->rtol * bnorm) status = ST_OK;
      else if (st->singular) status = ST_BREAKDOWN;
      else if (st->iters >= st->max_iters) status = ST_NOT_CONVERGED;
      else stop = 0;
      st->status = status;
      if (!stop) {
        st->sigma = 1.0 / gamma;
        arr.g[0] = 1.0;
        st->k = 0;
        st->cycle_done = 0;
        st->breakdown = 0;
        st->stop_rel = st->mode == 0 ? st->rtol * bnorm / gamma
                                     : (st->inner_rtol > 0.0 ? st->inner_rtol : -1.0);
      }
      st->stop = stop;
    }
  }
}

// ---------------------------------------------------------------------------
// Set-up kernels.
// ---------------------------------------------------------------------------
__global__ void k_absmax(const double* __restrict__ v, long long nnz, unsigned long long* out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz;
       i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(v[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

template <class S>
__global__ void k_cast_vals(const double* __restrict__ v, S* __restrict__ out, long long nnz,
                            double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = to_s<S>(v[i] / scale);
}

// CSR structure check: row_ptr[0] = 0, row_ptr[n] = nnz, nondecreasing, 0 <= col < n.
__global__ void k_check_csr(const int* __restrict__ rp, const int* __restrict__ ci, int n, int nnz,
                            int* bad) {
  const long long tid0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (tid0 == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(bad, 1);
  for (long long i = tid0; i < n; i += stride)
    if (rp[i + 1] < rp[i]) atomicOr(bad, 2);
  for (long long e = tid0; e < nnz; e += stride) {
    const int c = ci[e];
    if (c < 0 || c >= n) atomicOr(bad, 4);
  }
}

// SplitMix64 (Steele, Lea, Flood 2014): out[i] = mix(seed + (i+1) * golden) mapped to [-1, 1).
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_splitmix64(double* out, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)(splitmix64_at(seed, (unsigned long long)i) >> 11) * 0x1p-52 - 1.0;
}

}  // namespace gm
