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

#include <cooperative_groups.h>
#include <type_traits>

#include "common.cuh"

namespace gm {

__device__ __forceinline__ int read_flag(const int* p) { return *(volatile const int*)p; }

// First unit of this CTA's (next == 0) or the next CTA's (next == 1) share when `units`
// work units are split into equal contiguous ranges, each a multiple of `align` units
// (the ranges of all CTAs differ by at most `align` units).  Every CTA of a grid gets
// about the same work, so no SM waits on a second wave.
__device__ __forceinline__ long long cta_begin(long long units, long long align, int next = 0) {
  const long long chunks = units / align;
  const long long b = blockIdx.x + next;
  const long long c = chunks * b / gridDim.x;
  return b >= gridDim.x ? units : c * align;
}

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
      prod_s[e - c0] = (W)to_w(aa) * xa;
      prod_s[e + NT - c0] = (W)to_w(ab) * xb;
      prod_s[e + 2 * NT - c0] = (W)to_w(ac) * xc;
      prod_s[e + 3 * NT - c0] = (W)to_w(ad) * xd;
    }
    for (; e < c1; e += NT) prod_s[e - c0] = (W)to_w(av[e]) * xval(ci[e]);
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

// ---------------------------------------------------------------------------
// SELL-32 engine (the inner copy of A built at plan set-up): rows are grouped in
// slices of 32 consecutive rows; slice s stores its entries column-major, entry e of
// row 32s + l at meta[s].x + 32 e + l, padded to the slice's longest row
// (meta[s].y) with zero values and an in-range column.  A warp owns whole slices, so
// every load of values and column indices is one coalesced 128-byte access and a row
// needs no shared memory or barrier.  Computes the rows r0 + tid + k*NT (k < RPT).
// ---------------------------------------------------------------------------
// acc[k] += sum over the entries e < mt[k].y of slice k's row `lane`: value * xval(column),
// in entry order.  EB entries of all R slices are loaded (indices and values) before any
// gather and the gathers before any product, so 2 R EB loads and then R EB gathers are in
// flight per lane; padding entries (value 0, a valid column) need no test.
// With 2-byte values (FP16/BF16 copies of A) the loop is software-pipelined: the indices
// and values of the next EB entries are loaded while the gathers of the current ones are
// in flight, so a round costs one dependent latency (gather) instead of two (index, then
// gather).  Measured on a B300 it shortens the FP16 SpMV by 9% and lengthens the FP32 one
// by 2% (its extra registers), so FP32/FP64 keep the plain loop.  Products and their order
// are the same either way.
// MS: the matrix is read once by this kernel; load it evict-first (ld.cs) so that it does not
// push other data out of L2.
template <int EB, class AT, int R, bool MS = false>
__device__ __forceinline__ void sell_load(const int2 (&mt)[R], int e0, const int* __restrict__ sc,
                                          const AT* __restrict__ sv, int lane, int (&ci)[EB][R],
                                          AT (&va)[EB][R]) {
#pragma unroll
  for (int eb = 0; eb < EB; ++eb) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const bool ok = e0 + eb < mt[k].y;
      const int idx = mt[k].x + (e0 + eb) * 32 + lane;
      if constexpr (MS) {
        ci[eb][k] = ok ? __ldcs(sc + idx) : -1;
        va[eb][k] = ok ? __ldcs(sv + idx) : AT(0);
      } else {
        ci[eb][k] = ok ? sc[idx] : -1;
        va[eb][k] = ok ? sv[idx] : AT(0);
      }
    }
  }
}

template <int EB, class AT, class W, int R, class XF>
__device__ __forceinline__ void sell_products(const int (&ci)[EB][R], const AT (&va)[EB][R],
                                              const W (&xv)[EB][R], W (&acc)[R]) {
#pragma unroll
  for (int eb = 0; eb < EB; ++eb) {
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (ci[eb][k] >= 0) acc[k] += (W)to_w(va[eb][k]) * xv[eb][k];
  }
}

template <int EB, class AT, class W, int R, class XF>
__device__ __forceinline__ void sell_gathers(const int (&ci)[EB][R], const XF& xval,
                                             W (&xv)[EB][R]) {
#pragma unroll
  for (int eb = 0; eb < EB; ++eb) {
#pragma unroll
    for (int k = 0; k < R; ++k) xv[eb][k] = ci[eb][k] >= 0 ? xval(ci[eb][k]) : W(0);
  }
}

template <int EB, bool MS, class AT, class W, int R, class XF>
__device__ __forceinline__ void sell_accumulate_ms(const int2 (&mt)[R], int maxw,
                                                   const int* __restrict__ sc,
                                                   const AT* __restrict__ sv, int lane,
                                                   const XF& xval, W (&acc)[R]) {
  if constexpr (sizeof(AT) == 2) {
    int ci[EB][R];
    AT va[EB][R];
    sell_load<EB, AT, R, MS>(mt, 0, sc, sv, lane, ci, va);
    for (int e0 = 0; e0 < maxw; e0 += EB) {
      W xv[EB][R];
      sell_gathers<EB, AT, W, R>(ci, xval, xv);
      int cn[EB][R];
      AT vn[EB][R];
      sell_load<EB, AT, R, MS>(mt, e0 + EB, sc, sv, lane, cn, vn);  // none past maxw
      sell_products<EB, AT, W, R, XF>(ci, va, xv, acc);
#pragma unroll
      for (int eb = 0; eb < EB; ++eb) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
          ci[eb][k] = cn[eb][k];
          va[eb][k] = vn[eb][k];
        }
      }
    }
  } else {
    for (int e0 = 0; e0 < maxw; e0 += EB) {
      int ci[EB][R];
      AT va[EB][R];
      sell_load<EB, AT, R, MS>(mt, e0, sc, sv, lane, ci, va);
      W xv[EB][R];
      sell_gathers<EB, AT, W, R>(ci, xval, xv);
      sell_products<EB, AT, W, R, XF>(ci, va, xv, acc);
    }
  }
}

// ms: load the matrix evict-first (see sell_load); chosen once per call.
template <int EB, class AT, class W, int R, class XF>
__device__ __forceinline__ void sell_accumulate(const int2 (&mt)[R], int maxw, const int* __restrict__ sc,
                                                const AT* __restrict__ sv, int lane, const XF& xval,
                                                W (&acc)[R], bool ms = false) {
  if (ms) sell_accumulate_ms<EB, true>(mt, maxw, sc, sv, lane, xval, acc);
  else sell_accumulate_ms<EB, false>(mt, maxw, sc, sv, lane, xval, acc);
}

template <class AT, class W, int RPT, class XF>
__device__ __forceinline__ void sell_rows(const int2* __restrict__ meta, const int* __restrict__ sc,
                                          const AT* __restrict__ sv, int nslices, int r0,
                                          const XF& xval, W (&acc)[RPT], bool ms = false) {
  const int lane = threadIdx.x & 31;
  const int s0 = (r0 >> 5) + (threadIdx.x >> 5);
  int2 mt[RPT];
  int maxw = 0;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int s = s0 + k * NWARP;
    mt[k] = s < nslices ? meta[s] : make_int2(0, 0);
    maxw = max(maxw, mt[k].y);
    acc[k] = W(0);
  }
  sell_accumulate<2>(mt, maxw, sc, sv, lane, xval, acc, ms);
}

// Sum of the G per-CTA partials p[0..G) by one warp, four independent load streams per
// lane (fixed order, so the result is reproducible).  Up to 320 partials (two CTAs per SM
// on 148 SMs give at most 296) all of a lane's loads are issued at once, one L2 round trip,
// and summed in the order of the general loop below (bitwise the same result).
template <class W>
__device__ __forceinline__ W warp_sum_partials(const W* __restrict__ p, int G) {
  const int lane = threadIdx.x & 31;
  W s0 = W(0), s1 = W(0), s2 = W(0), s3 = W(0);
  if (G <= 320) {
    W v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int b = lane + 32 * k;
      v[k] = k < 10 && b < G ? __ldcg(&p[b]) : W(0);
    }
    bool wide = true;  // still in the four-stream loop
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int b = lane + 128 * i;
      if (wide && b + 96 < G) {
        s0 += v[4 * i];
        s1 += v[4 * i + 1];
        s2 += v[4 * i + 2];
        s3 += v[4 * i + 3];
      } else {
        wide = false;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (b + 32 * q < G) s0 += v[4 * i + q];
      }
    }
    return warp_sum((s0 + s1) + (s2 + s3));
  }
  int b = lane;
  for (; b + 96 < G; b += 128) {
    s0 += __ldcg(&p[b]);
    s1 += __ldcg(&p[b + 32]);
    s2 += __ldcg(&p[b + 64]);
    s3 += __ldcg(&p[b + 96]);
  }
  for (; b < G; b += 32) s0 += __ldcg(&p[b]);
  return warp_sum((s0 + s1) + (s2 + s3));
}

// Reduces ncol columns of per-CTA partials part[c * G + b] with the CTA's first NW warps
// and calls out(c, sum) once per column (lane 0 of the warp that owns it).  Warp w owns
// columns w, w + NW, ...; each lane keeps four columns' loads in flight.  Fixed order.
template <int NW = NWARP, class W, class F>
__device__ __forceinline__ void block_reduce_columns(const W* __restrict__ part, int ncol, int G,
                                                     const F& out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = warp; c0 < ncol; c0 += 4 * NW) {
    W s[4] = {W(0), W(0), W(0), W(0)};
#pragma unroll 4
    for (int b = lane; b < G; b += 32) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + q * NW;
        if (c < ncol) s[q] += __ldcg(&part[(long long)c * G + b]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + q * NW;
      const W v = warp_sum(s[q]);
      if (c < ncol && lane == 0) out(c, v);
    }
  }
}

// w[q] -= sum_{b < B} coef[c0 + b] * V[c0 + b][base + q]: the B column vectors are loaded
// before any is used, so B 16-byte loads per thread are in flight.  EF: the last read of
// these columns in this kernel (L2 evict-first loads, see ldv_evict_first).
template <int B, bool EF, class S, class W, int VEC>
__device__ __forceinline__ void update_cols(const S* __restrict__ V, long long ld, long long base,
                                            int c0, const W* __restrict__ coef, W (&wv)[VEC]) {
  S v[B][VEC];
#pragma unroll
  for (int b = 0; b < B; ++b) ldv_sel<EF>(V + (long long)(c0 + b) * ld + base, v[b]);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const W k = coef[c0 + b];
#pragma unroll
    for (int q = 0; q < VEC; ++q) wv[q] -= k * to_w(v[b][q]);
  }
}

// d[b] = sum_q V[c0 + b][base + q] * w[q] for b < B (B loads in flight).
template <int B, bool EF, class S, class W, int VEC>
__device__ __forceinline__ void dot_cols(const S* __restrict__ V, long long ld, long long base, int c0,
                                         const W (&wv)[VEC], W (&d)[B]) {
  S v[B][VEC];
#pragma unroll
  for (int b = 0; b < B; ++b) ldv_sel<EF>(V + (long long)(c0 + b) * ld + base, v[b]);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    W t = W(0);
#pragma unroll
    for (int q = 0; q < VEC; ++q) t += to_w(v[b][q]) * wv[q];
    d[b] = t;
  }
}

// Warp totals of K = 2, 4 or 8 columns at once.  d[b] is this lane's term of column b;
// returns, in every lane, the warp total of column lane >> (5 - log2 K) (for K = 8: (lane >>
// 2) & 7).  Each of the first log2 K exchanges (xor 16, 8, 4) sends the half of the columns
// that the partner keeps, halving what a lane carries; plain butterfly steps finish (9
// shuffles instead of 8 x 5 for K = 8).  Every total is formed by the same additions, with
// the same operands, as warp_sum of that column (own value + partner's, partners xor 16, 8,
// 4, 2, 1), so the totals are bitwise warp_sum's.
template <int K, class W>
__device__ __forceinline__ W warp_sum_cols(const W (&d)[K]) {
  static_assert(K == 2 || K == 4 || K == 8, "2, 4 or 8 columns");
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  W h[K];
#pragma unroll
  for (int b = 0; b < K; ++b) h[b] = d[b];
  int o = 16;
#pragma unroll
  for (int half = K / 2; half >= 1; half >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;  // this lane keeps the upper half of its columns
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const W send = up ? h[i] : h[half + i];
      const W keep = up ? h[half + i] : h[i];
      h[i] = keep + __shfl_xor_sync(full, send, o);
    }
  }
  W v = h[0];
#pragma unroll
  for (; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
  return v;
}

// Dot products of w with the K columns V[c .. c+K) for this thread's rows, summed over the
// warp and added to acc: column c + b's total by one lane, always the same lane for a given
// K and b.  K loads per thread in flight.  EF: see update_cols.
template <int K, bool EF, class S, class W, int VEC>
__device__ __forceinline__ void dots_block(const S* __restrict__ V, long long ld, long long base,
                                           int c, const W (&wv)[VEC], W* acc) {
  const int lane = threadIdx.x & 31;
  W d[K];
  dot_cols<K, EF>(V, ld, base, c, wv, d);
  if constexpr (K == 1) {
    const W t = warp_sum(d[0]);
    if (lane == 0) acc[c] += t;
  } else {
    constexpr int SH = K == 2 ? 4 : K == 4 ? 3 : 2;  // lane >> SH: the column this lane holds
    const W t = warp_sum_cols<K>(d);
    if ((lane & ((1 << SH) - 1)) == 0) acc[c + (lane >> SH)] += t;
  }
}

// Dot products of w with the columns V[c0..nc) for this thread's rows, summed over the
// warp and added to acc[c]: blocks of 8 columns, then at most one block each of 4, 2 and 1
// (one round of loads per block instead of one per leftover column).  EF: see update_cols.
template <bool EF, class S, class W, int VEC>
__device__ __forceinline__ void dots_to_acc(const S* __restrict__ V, long long ld, long long base,
                                            int nc, const W (&wv)[VEC], W* acc, int c0 = 0) {
  int c = c0;
  for (; c + 8 <= nc; c += 8) dots_block<8, EF>(V, ld, base, c, wv, acc);
  if (nc - c >= 4) {
    dots_block<4, EF>(V, ld, base, c, wv, acc);
    c += 4;
  }
  if (nc - c >= 2) {
    dots_block<2, EF>(V, ld, base, c, wv, acc);
    c += 2;
  }
  if (c < nc) dots_block<1, EF>(V, ld, base, c, wv, acc);
}

// dots_to_acc over V[0..nc) with the columns taken newest first (the same value per
// column).  k_cgs_u1 calls it right after update_all has loaded the same columns in
// ascending order, so the newest lines, the likeliest to still be in L1, are read first:
// the leftover blocks (1, 2, 4 columns) from the top, then the blocks of 8 downwards.
template <class S, class W, int VEC>
__device__ __forceinline__ void dots_to_acc_desc(const S* __restrict__ V, long long ld,
                                                 long long base, int nc, const W (&wv)[VEC],
                                                 W* acc) {
  int c = nc;
  const int r = nc & 7;
  if (r & 1) {
    c -= 1;
    dots_block<1, false>(V, ld, base, c, wv, acc);
  }
  if (r & 2) {
    c -= 2;
    dots_block<2, false>(V, ld, base, c, wv, acc);
  }
  if (r & 4) {
    c -= 4;
    dots_block<4, false>(V, ld, base, c, wv, acc);
  }
  for (; c >= 8; c -= 8) dots_block<8, false>(V, ld, base, c - 8, wv, acc);
}

// w -= V[0..nc) coef for this thread's rows.  EF: see update_cols.
// Blocks of 8 columns, then at most one block each of 4, 2 and 1, in ascending order (every
// row's products are subtracted in column order whatever the blocking).
template <bool EF, class S, class W, int VEC>
__device__ __forceinline__ void update_all(const S* __restrict__ V, long long ld, long long base,
                                           int nc, const W* __restrict__ coef, W (&wv)[VEC]) {
  int c = 0;
  for (; c + 8 <= nc; c += 8) update_cols<8, EF>(V, ld, base, c, coef, wv);
  if (nc - c >= 4) {
    update_cols<4, EF>(V, ld, base, c, coef, wv);
    c += 4;
  }
  if (nc - c >= 2) {
    update_cols<2, EF>(V, ld, base, c, coef, wv);
    c += 2;
  }
  if (c < nc) update_cols<1, EF>(V, ld, base, c, coef, wv);
}

template <int P>
struct SpmvSmem {
  using W = typename Tr<P>::W;
  static constexpr int TR = NT * Tr<P>::RT;  // rows per CTA tile: RT rows per thread
  static constexpr int CAP = 4096;  // CSR engine: nonzeros staged per chunk
  // dynamic shared memory of k_spmv_arnoldi (CSR: staged products and row pointers)
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
// SPMV_ONLY (with PLAIN): w = A src and nothing else -- no dot products, no norm, no
// partial sums; V, part and h1 are not touched (the kernel still reads st->stop and
// returns at once when it is set).
// The matrix is CSR (rp, ci, av); plans use the SELL-32 form k_spmv_sell below.
// ---------------------------------------------------------------------------
template <int P, class SrcT, bool PLAIN = false, bool SPMV_ONLY = false>
__global__ void __launch_bounds__(NT) k_spmv_arnoldi(
    const int* __restrict__ rp, const int* __restrict__ ci, const typename Tr<P>::S* __restrict__ av,
    int n, long long ld, double row_scale_d, const SrcT* __restrict__ src, double v_scale,
    typename Tr<P>::S* V, int j, typename Tr<P>::W* __restrict__ wout,
    typename Tr<P>::W* __restrict__ part, DevState* st, double* __restrict__ h1) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::RT;  // rows per thread of the tile, also in its dot products
  constexpr int TR = SpmvSmem<P>::TR;
  constexpr int CAP = SpmvSmem<P>::CAP;
  static_assert(TR == NT * VEC, "the CSR tile's dot layout takes RT rows per thread");
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
      if constexpr (!SPMV_ONLY) w_s[il] = wv;
      if (row < n) wout[row] = wv;
    }
    __syncthreads();  // every thread has read rp_s before the next tile rewrites it
    if constexpr (SPMV_ONLY) continue;
    // First CGS pass, transposed GEMV: VEC consecutive rows per thread.
    const long long gb = (long long)r0 + tid * VEC;
    W wv[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) wv[q] = w_s[tid * VEC + q];
    W nrm = W(0);
#pragma unroll
    for (int q = 0; q < VEC; ++q) nrm += wv[q] * wv[q];
    dots_to_acc<false, S, W, VEC>(V, ld, gb, j + 1, wv, acc + warp * ncol);
    nrm = warp_sum(nrm);
    if (lane == 0) acc[warp * ncol + j + 1] += nrm;
    __syncthreads();
  }
  if constexpr (SPMV_ONLY) return;
  const int G = gridDim.x;
  for (int c = tid; c < ncol; c += NT) {
    W s = W(0);
    for (int w = 0; w < NWARP; ++w) s += acc[w * ncol + c];
    part[(long long)c * G + blockIdx.x] = s;
  }
  if (!arrive_last(&st->ticket[0], &s_last)) return;
  block_reduce_columns(part, ncol, G, [&](int c, W s) {
    if (c <= j) h1[c] = (double)s * pow2_recip(v_scale);
    else st->wnorm = sqrt((double)s);
  });
  if (tid == 0) st->ticket[0] = 0;
}

// ===========================================================================
// The Arnoldi step on the SELL-32 copy, with no serial tails.
//
// Each step kernel ends by writing one partial sum per CTA and column -- no fence, no
// ticket, no "last CTA".  The next kernel reduces those partials in its prologue: each
// cluster of CL CTAs splits the columns among its CTAs and shares the sums through
// distributed shared memory (cluster_column_sums), always in the same fixed order, so
// every CTA holds bitwise the same values:
//   k_spmv_sell(j)  prologue (j > 0): the Givens update of step j-1 from ||w''||
//                   (k_cgs_u2(j-1)'s partials) and ||A v_{j-1}|| (k_spmv_sell(j-1)'s);
//                   every CTA computes it and takes the same stop decision, CTA 0 stores
//                   it.  Body: v_j = store(sigma src), w = A v_j, partials of V_j^T w
//                   and ||w||^2.
//   k_cgs_u1(j)     prologue: h1 from the SpMV partials (CTA 0 stores h1).
//                   Body: w' = w - V_j h1, partials of V_j^T w'.
//   k_cgs_u2(j)     prologue: h2 (CTA 0 stores h2).  Body: w'' = w' - V_j h2, partials
//                   of ||w''||^2.
// k_finalize applies the update of the cycle's last step.  The SpMV partials are
// double-buffered by step parity (k_spmv_sell(j+1) reads step j's norm column while its
// CTAs write step j+1's partials).  The Givens update reads only data written by earlier
// launches (h1, h2, earlier rotations, |g_j|), so the redundant computations agree.
//
// Row order.  Each kernel of a step streams all j+1 basis columns, more than the L2 holds
// once j is large, and LRU keeps what a kernel touched last.  Consecutive step kernels
// therefore walk their CTA's rows in opposite directions (k_spmv_sell forward for even j,
// k_cgs_u1 the other way, k_cgs_u2 like k_spmv_sell), so each starts on the rows whose
// basis entries the previous kernel left in L2.  The SpMV streams the matrix evict-first
// (it is read once per step) and reads the old basis columns with half of them evict-first
// in FP64/FP32 and plainly in FP16/BF16 (Tr::V_EF), so the CGS kernels that follow find
// much of the basis in L2 while the gathered vector stays resident; measured on a B300,
// evict-first loads in the CGS kernels themselves cost more than they saved.
// ===========================================================================

// Partial-sum buffers of one Arnoldi step (working type, column-major: column c of a
// buffer with G CTAs is [c * G, c * G + G)).
template <class W>
struct StepParts {
  W* p1[2];    // k_spmv_sell(j) writes p1[j & 1]: j+2 columns (dots, ||w||^2), g1 CTAs
  W* p2;       // k_cgs_u1: j+1 columns, g2 CTAs
  W* p3;       // k_cgs_u2: 1 column, g2 CTAs
  int g1, g2;
  // p1[j & 1] without dynamic indexing (which would copy the parameter to local memory)
  __device__ __forceinline__ W* p1_of(int j) const { return (j & 1) ? p1[1] : p1[0]; }
};

// CTA sum of the per-warp accumulators acc_w[c] (warp w's at acc0 + w * stride) written
// as this CTA's partial of each column.
template <class W>
__device__ __forceinline__ void write_cta_partials(const W* acc0, int stride, int ncol, W* part) {
  const int G = gridDim.x;
  for (int c = threadIdx.x; c < ncol; c += NT) {
    W s = W(0);
    for (int w = 0; w < NWARP; ++w) s += acc0[(size_t)w * stride + c];
    part[(long long)c * G + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Column sums shared across a thread-block cluster.
//
// Every CTA of a step kernel needs the sums over the previous kernel's CTAs of a few
// columns of partials.  Summing every column in every CTA is slow on a B300 (6-17 us for
// 1-51 columns of ~300 partials, with all CTAs reading the same lines at once), so rank
// r of each cluster of CL CTAs sums only the columns c with c % CL == r (one warp per
// column, in the fixed order of warp_sum_partials), and the cluster exchanges the sums
// through distributed shared memory.  Every CTA ends with bitwise the same values.
//
// The CTAs of a cluster must reach the same cluster barriers, so the skip decision is
// made per cluster: a CTA whose own flag is clear still skips when another CTA of its
// cluster saw the flag set (which only happens when a CTA of the same launch has just
// ended the cycle or the solve, so the work would be discarded anyway).
// ---------------------------------------------------------------------------
constexpr int CL = 4;  // CTAs per cluster of the step kernels

template <class W>
struct ColumnSrc {    // column c of the partials: `count` values at `ptr`
  const W* ptr;
  int count;
};

// col(c) -> ColumnSrc<W>.  mine and out hold ncol values (shared memory).  skip_flag()
// is this CTA's skip flag, evaluated by thread 0 (its loads are in flight together with
// the partial sums' loads, which are made whether or not the CTA skips: their buffers
// always exist, and a skipping cluster discards the sums).  Returns false when the
// cluster skips; then out is not written.  Called by all threads of every CTA of the
// cluster.
template <class W, class ColF, class SkipF>
__device__ __forceinline__ bool cluster_column_sums(const ColF& col, int ncol, W* mine, W* out,
                                                    const SkipF& skip_flag) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int s_flag, s_any;
  int flag = 0;
  if (threadIdx.x == 0) flag = skip_flag();
  const int nw = blockDim.x >> 5;
  for (int c = rank + CL * warp; c < ncol; c += CL * nw) {
    const ColumnSrc<W> src = col(c);
    const W v = warp_sum_partials(src.ptr, src.count);
    if (lane == 0) mine[c] = v;
  }
  if (threadIdx.x == 0) s_flag = flag;
  cl.sync();
  if (warp == 0) {
    int f = lane < CL ? *cl.map_shared_rank(&s_flag, lane) : 0;
    f = __any_sync(0xffffffffu, f);
    if (lane == 0) s_any = f;
  }
  __syncthreads();
  const int any = s_any;
  if (!any)
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) out[c] = *cl.map_shared_rank(mine + c, c % CL);
  cl.sync();  // no CTA leaves while another may still read its shared memory
  return !any;
}

// Applies the rotations G_0 .. G_{js-1} (cs, sn) to the new Hessenberg column col[0..js]
// as an affine scan (see finalize_step): writes the rotated entries rot[0..js-1] and
// returns the rotated col[js] in every lane.  Called by all 32 lanes of one warp; col, cs,
// sn, rot in shared memory.
__device__ __forceinline__ double givens_scan(int js, const double* col, const double* cs,
                                              const double* sn, double* rot) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int seg = (js + 31) / 32;
  const int i0 = min(lane * seg, js), i1 = min(i0 + seg, js);
  // this lane's composite map x -> A x + B over rotations [i0, i1)
  double A = 1.0, B = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double ai = -sn[i], bi = cs[i] * col[i + 1];
    B = fma(ai, B, bi);
    A = ai * A;
  }
  // inclusive scan: lane l holds the composite of the segments of lanes 0..l
  for (int d = 1; d < 32; d <<= 1) {
    const double Ap = __shfl_up_sync(full, A, d), Bp = __shfl_up_sync(full, B, d);
    if (lane >= d) {
      B = fma(A, Bp, B);
      A = A * Ap;
    }
  }
  const double Ae = __shfl_up_sync(full, A, 1), Be = __shfl_up_sync(full, B, 1);
  double x = col[0];
  if (lane > 0) x = fma(Ae, x, Be);  // x entering this lane's segment
  for (int i = i0; i < i1; ++i) {
    const double h = col[i + 1];
    rot[i] = fma(cs[i], x, sn[i] * h);
    x = fma(-sn[i], x, cs[i] * h);
  }
  // x_js: lane 31's composite covers every rotation
  x = js > 0 ? fma(__shfl_sync(full, A, 31), col[0], __shfl_sync(full, B, 31)) : col[0];
  __syncwarp();
  return x;
}

// The new Givens rotation of a column whose rotated diagonal entry is x and whose
// subdiagonal is hn = sqrt(hn2), with wnorm = sqrt(wn2) for the breakdown test.  Called by
// all 32 lanes of a warp (every lane gets the results): the two square roots share one
// FP64 instruction (lanes 0 and 1), and c = x / rho, s = hn / rho and 1 / hn share one
// division (lanes 0, 1, 2) -- FP64 is slow on a B300, and these sit on every step's path.
// (c, s) = (1, 0) when hn == 0.
struct GivensRot {
  double c, s, rjj, hn, wnorm, inv_hn;
};
__device__ __forceinline__ GivensRot givens_rotation(double x, double hn2, double wn2) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const double sq = sqrt(lane == 0 ? hn2 : (lane == 1 ? wn2 : 1.0));
  GivensRot g;
  g.hn = __shfl_sync(full, sq, 0);
  g.wnorm = __shfl_sync(full, sq, 1);
  const double rho = hypot(x, g.hn);
  const double num = lane == 0 ? x : (lane == 1 ? g.hn : 1.0);
  const double den = lane <= 1 ? rho : g.hn;
  const double q = num / den;
  const double qc = __shfl_sync(full, q, 0), qs = __shfl_sync(full, q, 1);
  g.inv_hn = __shfl_sync(full, q, 2);
  g.c = g.hn != 0.0 ? qc : 1.0;
  g.s = g.hn != 0.0 ? qs : 0.0;
  g.rjj = g.c * x + g.s * g.hn;
  return g;
}

// Shared-memory doubles that finalize_step needs (for js < LSQ_MAX): the column, the old
// rotations and the rotated column (at most 4 LSQ_MAX), then GIVENS_SCAL scalars of the
// solver state at offset GIVENS_SCAL_AT.
constexpr int GIVENS_SCAL_AT = 4 * (LSQ_MAX + 2);
constexpr int GIVENS_SCAL = 6;
constexpr int GIVENS_SH = GIVENS_SCAL_AT + 8;

// Givens update of step js (Algorithm 1's least squares solved incrementally, FP64) with
// the stop decision.  Called by every thread of the CTA; `sh` holds GIVENS_SH doubles of
// shared memory.  Returns (through *done_out / *sigma_out, valid in all threads after the
// call) whether the cycle ends and 1 / h_{js+1,js}.  If `writer`, the CTA stores
// H[:, js], R[:, js], the rotation, |g_{js+1}|, the history and the flags.
// hn2 = ||w''||^2 and wn2 = ||A v_js||^2 are the column sums of the partials of
// k_cgs_u2(js) and of the norm column of k_spmv_sell(js) (the same values in every CTA).
//
// The previous rotations G_0 .. G_{js-1} act on the new column h as a chain: with x_0 =
// h_0, rotation i gives R_{i,js} = c_i x_i + s_i h_{i+1} and x_{i+1} = -s_i x_i + c_i h_{i+1},
// an affine recurrence in x.  FP64 instructions are slow on a B300 and a serial chain of
// 4 js of them costs about 0.2 us per rotation, so warp 0 evaluates it as a scan: each lane
// composes the affine maps of a segment of rotations, a shuffle scan gives every lane the
// x entering its segment, and the lanes replay their segments in parallel.
//
// The update is split so that a kernel can issue its global loads early:
// finalize_load (no barrier) gathers the column, the old rotations and the state scalars
// into `sh`; finalize_compute, after a CTA barrier, does the rest.  finalize_step is the
// two with the barrier between them.
__device__ __forceinline__ void finalize_load(const DevState* st, const Arrays& a, int js,
                                              double* sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* col = sh;                 // js + 2: the new column h (H[:, js] before rotation)
  double* cs = sh + (js + 2);       // js
  double* sn = cs + (js + 1);       // js
  if (warp == 2) {
    for (int i = lane; i <= js; i += 32) col[i] = a.h1[i] + a.h2[i];
  } else if (warp == 3) {
    for (int i = lane; i < js; i += 32) {
      cs[i] = a.cs[i];
      sn[i] = a.sn[i];
    }
  } else if (warp == 1 && lane == 0) {
    double* sc = sh + GIVENS_SCAL_AT;
    sc[0] = a.gabs[js];
    sc[1] = st->u_work;
    sc[2] = st->stop_rel;
    sc[3] = (double)(st->iters0 + js + 1);  // exact: step counts stay far below 2^53
    sc[4] = (double)st->max_iters;          // compared as doubles with sc[3]
    sc[5] = (double)st->m;
  }
}

__device__ void finalize_compute(DevState* st, const Arrays& a, int js, double hn2, double wn2,
                                 bool writer, double* sh, int* done_out, double* sigma_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* col = sh;
  const double* cs = sh + (js + 2);
  const double* sn = cs + (js + 1);
  double* rot = sh + (3 * js + 4);  // js: R[0..js, js]
  const double* sc = sh + GIVENS_SCAL_AT;
  const int m = (int)sc[5];
  const int ldh = m + 1;
  __shared__ int s_done;
  __shared__ double s_sigma;
  if (writer && warp == 2) {
    double* Hc = a.H + (long long)js * ldh;
    for (int i = lane; i <= js; i += 32) Hc[i] = col[i];
  }
  if (warp == 0) {
    const double x = givens_scan(js, col, cs, sn, rot);
    const GivensRot gr = givens_rotation(x, hn2, wn2);
    __syncwarp();
    if (writer) {
      double* Rc = a.R + (long long)js * ldh;
      for (int i = lane; i < js; i += 32) Rc[i] = rot[i];
    }
    if (lane == 0) {
      const double hn = gr.hn, wnorm = gr.wnorm, c = gr.c, s = gr.s, rjj = gr.rjj;
      const double res = sc[0] * fabs(s);
      const long long iters = (long long)sc[3];
      const bool bad = !isfinite(hn) || !isfinite(res) || !isfinite(rjj);
      const int brk = hn <= 16.0 * sc[1] * wnorm;
      const int done = bad || brk || res <= sc[2] || js + 1 >= m || sc[3] >= sc[4];
      s_done = done;
      s_sigma = brk ? 0.0 : gr.inv_hn;
      if (writer) {
        double* Hc = a.H + (long long)js * ldh;
        double* Rc = a.R + (long long)js * ldh;
        Hc[js + 1] = hn;
        Rc[js] = rjj;
        Rc[js + 1] = 0.0;
        a.cs[js] = c;
        a.sn[js] = s;
        a.gabs[js + 1] = res;
        st->k = js + 1;
        st->iters = iters;
        if (iters <= st->hist_cap)
          a.hist[iters - 1] = res * st->gamma / (st->bnorm > 0.0 ? st->bnorm : 1.0);
        st->breakdown = brk;
        if (bad) {
          st->status = ST_NONFINITE;
          st->stop = 1;
        }
        if (done) st->cycle_done = 1;
        st->sigma = s_sigma;
      }
    }
  }
  __syncthreads();
  *done_out = s_done;
  *sigma_out = s_sigma;
}

__device__ void finalize_step(DevState* st, const Arrays& a, int js, double hn2, double wn2,
                              bool writer, double* sh, int* done_out, double* sigma_out) {
  finalize_load(st, a, js, sh);
  __syncthreads();
  finalize_compute(st, a, js, hn2, wn2, writer, sh, done_out, sigma_out);
}

template <int P>
struct SellSmem {
  using W = typename Tr<P>::W;
  static constexpr int WT = 32 * Tr<P>::VT;
  static size_t bytes(int ncol) { return sizeof(W) * (size_t)NWARP * (WT + ncol) + 16; }
};

// Step kernel 1 (see above).  A warp owns "warp tiles" of WT = 32 VEC consecutive rows
// (VEC = Tr<P>::VT slices): it stores its rows of V[:, j], computes its rows of w = A v_j
// slice by slice, turns them from the slice layout (lane l holds rows 32q + l) into the
// vector layout (lane l holds rows VEC l .. VEC l + VEC-1) through a warp-private buffer, and
// accumulates the first-pass dot products over its rows.  There is no CTA barrier inside
// the loop, so warps at different phases overlap.  Each CTA owns an equal contiguous
// range of warp tiles (cta_begin).  PLAIN: src is p(A) v_j (working type, unscaled),
// gathered as is; V[:, j] was stored by the polynomial's first kernel.
template <int P, class SrcT, bool PLAIN>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, 2) k_spmv_sell(
    const int2* __restrict__ meta, const int* __restrict__ sc, const typename Tr<P>::S* __restrict__ sv,
    int nslices, int n, long long ld, double row_scale_d, const SrcT* __restrict__ src,
    double v_scale, typename Tr<P>::S* V, int j, typename Tr<P>::W* __restrict__ wout,
    StepParts<typename Tr<P>::W> parts, DevState* st, Arrays arr) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VT;
  constexpr int WT = SellSmem<P>::WT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double gsh[GIVENS_SH];
  const int ncol = j + 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  W* ws = reinterpret_cast<W*>(smem_raw) + (size_t)warp * (WT + ncol);
  W* acc = ws + WT;
  __shared__ int s_skip;
  __shared__ W s_mine[2], s_nrm[2];
  // the Givens update's global loads go out before the prologue's barriers
  if (!PLAIN && j > 0) finalize_load(st, arr, j - 1, gsh);
  const auto skip_flag = [&] { return read_flag(&st->stop) | read_flag(&st->cycle_done); };
  double sigma = 1.0;
  if (!PLAIN && j > 0) {  // with a polynomial, k_poly_start applied the update
    // ||w''|| of step j-1 (k_cgs_u2's partials) and ||A v_{j-1}|| (norm column of step j-1)
    const W* pn = parts.p1_of(j - 1) + (long long)j * parts.g1;
    const auto col = [&](int c) {
      return c == 0 ? ColumnSrc<W>{parts.p3, parts.g2} : ColumnSrc<W>{pn, parts.g1};
    };
    if (!cluster_column_sums<W>(col, 2, s_mine, s_nrm, skip_flag)) return;
    int done;
    finalize_compute(st, arr, j - 1, (double)s_nrm[0], (double)s_nrm[1], blockIdx.x == 0, gsh,
                     &done, &sigma);
    if (done) return;
  } else {
    if (tid == 0) s_skip = skip_flag();
    __syncthreads();
    if (s_skip) return;
    if (!PLAIN) sigma = st->sigma;
  }
  for (int c = lane; c < ncol; c += 32) acc[c] = W(0);
  __syncwarp();
  const bool ms = PLAIN ? st->stream_matrix != 0 : true;

  const SrcT f = (SrcT)(v_scale * sigma);
  const W row_scale = (W)row_scale_d;
  auto make = [&](SrcT x) -> S { return to_s<S>(f * x); };
  auto xval = [&](int c) -> W {
    if constexpr (PLAIN) return (W)src[c];
    else return to_w(make(src[c]));
  };
  S* Vj = V + (long long)j * ld;
  const int nwt = (n + WT - 1) / WT;
  const int t0 = (int)cta_begin(nwt, 1), t1 = (int)cta_begin(nwt, 1, 1);
  const bool rev = j & 1;  // traversal direction: see "Row order" above
  for (int k = warp; k < t1 - t0; k += NWARP) {
    const int wt = rev ? t1 - 1 - k : t0 + k;
    const int r0 = wt * WT;
    const int s0 = r0 >> 5;
    int2 mt[VEC];
    int maxw = 0;
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      mt[q] = s0 + q < nslices ? meta[s0 + q] : make_int2(0, 0);
      maxw = max(maxw, mt[q].y);
    }
    if constexpr (!PLAIN) {
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        const int row = r0 + 32 * q + lane;
        if (row < n) Vj[row] = make(src[row]);
      }
    }
    W a[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) a[q] = W(0);
    // The matrix is read once per step and evicted by the CGS kernels' streams anyway: loaded
    // evict-first, it leaves L2 to the basis the next kernels read.  After a preconditioner
    // (PLAIN) the plan decides (DevState::stream_matrix): a polynomial re-reads the matrix d
    // times per step, which pays only while it stays in L2.
    sell_accumulate<2>(mt, maxw, sc, sv, lane, xval, a, ms);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      const int row = r0 + 32 * q + lane;
      const W wv = row < n ? row_scale * a[q] : W(0);
      ws[32 * q + lane] = wv;
      if (row < n) wout[row] = wv;
    }
    __syncwarp();
    W wv[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) wv[q] = ws[VEC * lane + q];
    __syncwarp();
    W nrm = W(0);
#pragma unroll
    for (int q = 0; q < VEC; ++q) nrm += wv[q] * wv[q];
    // columns 0..j (half evict-first in FP64/FP32, see Tr::V_EF); column j, just stored by
    // the warp, goes into the last block with the old ones (one round of loads less than a
    // block of its own; its products and sums are the same)
    dots_to_acc<Tr<P>::V_EF, S, W, VEC>(V, ld, (long long)r0 + VEC * lane, j + 1, wv, acc);
    nrm = warp_sum(nrm);
    if (lane == 0) acc[j + 1] += nrm;
  }
  __syncthreads();
  write_cta_partials(reinterpret_cast<W*>(smem_raw) + WT, WT + ncol, ncol, parts.p1_of(j));
}

// Store V[:, j] = store(v_scale * sigma * src) for all rows (the last basis vector of
// an Arnoldi run that is not followed by another SpMV).
template <int P, class SrcT>
__global__ void k_store_basis(const SrcT* __restrict__ src, double v_scale, int n,
                              typename Tr<P>::S* V, long long ld, int j, const DevState* st,
                              int in_cycle = 0) {
  using S = typename Tr<P>::S;
  if (in_cycle && read_flag(&st->stop)) return;  // (the start of a cycle that is not run)
  const SrcT f = (SrcT)(v_scale * st->sigma);
  S* Vj = V + (long long)j * ld;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    Vj[i] = to_s<S>(f * src[i]);
}

// Prologue shared by the CGS kernels.  coef[c] holds on entry the column sum of the
// partials, i.e. the dot product with the stored (scaled) basis, so h[c] = coef[c] /
// v_scale is v_c . w; the update multiplies the stored basis, so its coefficient becomes
// h[c] / v_scale.  CTA 0 stores h in FP64.
template <class W>
__device__ __forceinline__ void coefs_from_sums(W* coef, int nc, double v_scale,
                                                double* __restrict__ h) {
  const bool writer = blockIdx.x == 0;
  const double r = pow2_recip(v_scale);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const double hc = (double)coef[c] * r;
    coef[c] = (W)(hc * r);
    if (writer) h[c] = hc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Step kernel 2: h1 (prologue), w' = w - V_j h1, partials of V_j^T w'.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, 2) k_cgs_u1(const typename Tr<P>::S* __restrict__ V, long long ld,
                                               int j, double v_scale,
                                               const typename Tr<P>::W* __restrict__ win,
                                               typename Tr<P>::W* __restrict__ wout,
                                               StepParts<typename Tr<P>::W> parts, DevState* st,
                                               double* __restrict__ h1) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = j + 1;
  W* coef = reinterpret_cast<W*>(smem_raw);
  W* acc = coef + nc;
  __shared__ W s_mine[LSQ_MAX + 2];
  const int tid = threadIdx.x, warp = tid >> 5;
  const W* pj = parts.p1_of(j);
  const int gp = parts.g1;
  const auto col = [&](int c) { return ColumnSrc<W>{pj + (long long)c * gp, gp}; };
  const auto skip_flag = [&] { return read_flag(&st->stop) | read_flag(&st->cycle_done); };
  if (!cluster_column_sums<W>(col, nc, s_mine, coef, skip_flag)) return;
  for (int i = tid; i < NWARP * nc; i += NT) acc[i] = W(0);
  coefs_from_sums(coef, nc, v_scale, h1);
  const long long ngroups = ld / VEC;
  const long long g0 = cta_begin(ngroups, 32), g1 = cta_begin(ngroups, 32, 1);
  const bool rev = !(j & 1);  // traversal direction: see "Row order" above
  for (long long i = tid; i < g1 - g0; i += NT) {
    const long long g = rev ? g1 - 1 - i : g0 + i;
    const long long base = g * VEC;
    W wv[VEC];
    ldv(win + base, wv);
    update_all<false, S, W, VEC>(V, ld, base, nc, coef, wv);
    stv(wout + base, wv);
    dots_to_acc_desc<S, W, VEC>(V, ld, base, nc, wv, acc + warp * nc);
  }
  __syncthreads();
  write_cta_partials(acc, nc, nc, parts.p2);
}

// ---------------------------------------------------------------------------
// Step kernel 3: h2 (prologue), w'' = w' - V_j h2, partials of ||w''||^2.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, 2) k_cgs_u2(const typename Tr<P>::S* __restrict__ V, long long ld,
                                               int j, double v_scale,
                                               const typename Tr<P>::W* __restrict__ win,
                                               typename Tr<P>::W* __restrict__ wout,
                                               StepParts<typename Tr<P>::W> parts, DevState* st,
                                               double* __restrict__ h2) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = j + 1;
  W* coef = reinterpret_cast<W*>(smem_raw);
  __shared__ W accw[NWARP];
  __shared__ W s_mine[LSQ_MAX + 2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const W* pj = parts.p2;
  const int gp = parts.g2;
  const auto col = [&](int c) { return ColumnSrc<W>{pj + (long long)c * gp, gp}; };
  const auto skip_flag = [&] { return read_flag(&st->stop) | read_flag(&st->cycle_done); };
  if (!cluster_column_sums<W>(col, nc, s_mine, coef, skip_flag)) return;
  coefs_from_sums(coef, nc, v_scale, h2);
  W nrm = W(0);
  const long long ngroups = ld / VEC;
  const long long g0 = cta_begin(ngroups, 32), g1 = cta_begin(ngroups, 32, 1);
  const bool rev = j & 1;  // traversal direction: see "Row order" above
  for (long long i = tid; i < g1 - g0; i += NT) {
    const long long g = rev ? g1 - 1 - i : g0 + i;
    const long long base = g * VEC;
    W wv[VEC];
    ldv(win + base, wv);
    update_all<false, S, W, VEC>(V, ld, base, nc, coef, wv);
    stv(wout + base, wv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) nrm += wv[q] * wv[q];
  }
  nrm = warp_sum(nrm);
  if (lane == 0) accw[warp] = nrm;
  __syncthreads();
  if (tid == 0) {
    W s = W(0);
    for (int w = 0; w < NWARP; ++w) s += accw[w];
    parts.p3[blockIdx.x] = s;
    if (blockIdx.x == 0) st->last_step = j;
  }
}

// Applies the pending Givens update of the cycle's last step (one CTA).
template <int P>
__global__ void __launch_bounds__(NT) k_finalize(StepParts<typename Tr<P>::W> parts, DevState* st,
                                                 Arrays arr) {
  __shared__ double gsh[GIVENS_SH];
  __shared__ int s_go, s_js;
  if (threadIdx.x == 0) {
    s_js = st->last_step;
    s_go = !read_flag(&st->stop) && s_js >= 0 && st->k == s_js;
  }
  __syncthreads();
  if (!s_go) return;
  using W = typename Tr<P>::W;
  __shared__ double s_n[2];
  const int warp = threadIdx.x >> 5;
  if (warp < 2) {
    const W v = warp == 0 ? warp_sum_partials(parts.p3, parts.g2)
                          : warp_sum_partials(parts.p1_of(s_js) + (long long)(s_js + 1) * parts.g1,
                                              parts.g1);
    if ((threadIdx.x & 31) == 0) s_n[warp] = (double)v;
  }
  __syncthreads();
  int done;
  double sigma;
  finalize_step(st, arr, s_js, s_n[0], s_n[1], true, gsh, &done, &sigma);
}

// ---------------------------------------------------------------------------
// End of a cycle: least squares R y = g by back substitution (FP64, one warp solves).
// g is rebuilt from the rotations (g_0 = 1).  A trailing diagonal entry below
// 16 u max|R| is dropped (singular factor).  R is staged in shared memory (packed upper
// triangle, column by column) when `packed` is set (m <= LSQ_PACKED_MAX).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_lsq(DevState* st, Arrays a, int packed) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Rs = reinterpret_cast<double*>(smem_raw);
  __shared__ double gw[LSQ_MAX + 1], cs_s[LSQ_MAX], sn_s[LSQ_MAX], rinv[LSQ_MAX];
  __shared__ double red[NWARP];
  __shared__ int s_kk, s_skip;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_flag(&st->stop);
  __syncthreads();
  if (s_skip) return;
  const int k = st->k, ldh = st->m + 1;
  auto rix = [](int i, int c) { return c * (c + 1) / 2 + i; };
  // All loads of R and of the rotations are issued by the whole block at once; the serial
  // parts below read shared memory only.
  // The divisions by the diagonal are done here, all at once: the substitution below
  // multiplies by these reciprocals, so its serial chain holds no FP64 division (slow to
  // issue on this part); y_i = g_i (1 / r_ii) carries one rounding more than g_i / r_ii.
  for (int i = tid; i < k; i += NT) {
    cs_s[i] = a.cs[i];
    sn_s[i] = a.sn[i];
    rinv[i] = 1.0 / a.R[i + (long long)i * ldh];
  }
  double rmax = 0.0;
  for (int c = warp; c < k; c += NWARP)
    for (int i = lane; i <= c; i += 32) {
      const double v = a.R[i + (long long)c * ldh];
      if (packed) Rs[rix(i, c)] = v;
      rmax = fmax(rmax, fabs(v));
    }
  rmax = warp_max(rmax);
  if (lane == 0) red[warp] = rmax;
  __syncthreads();
  if (tid == 0) {
    double g = 1.0;  // g_0 = 1 (unit least-squares right-hand side)
    for (int i = 0; i < k; ++i) {
      gw[i] = cs_s[i] * g;
      g = -sn_s[i] * g;
    }
    double mx = 0.0;
    for (int w = 0; w < NWARP; ++w) mx = fmax(mx, red[w]);
    int kk = k;
    auto diag = [&](int i) { return packed ? Rs[rix(i, i)] : a.R[i + (long long)i * ldh]; };
    while (kk > 0 && fabs(diag(kk - 1)) <= 16.0 * st->u_work * mx) --kk;
    s_kk = kk;
    st->k_used = kk;
    st->singular = kk < k;
  }
  __syncthreads();
  if (warp != 0) return;
  const int kk = s_kk;
  for (int i = kk - 1; i >= 0; --i) {
    const double yi = gw[i] * rinv[i];
    __syncwarp();
    for (int l = lane; l < i; l += 32)
      gw[l] -= (packed ? Rs[rix(l, i)] : a.R[l + (long long)i * ldh]) * yi;
    if (lane == 0) a.y[i] = yi;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// x += gamma * V y (the correction u = V y accumulates in the working precision,
// the update is FP64: Algorithm 2, "x_{i+1} = x_i + u_i [double]").
// ---------------------------------------------------------------------------
// F32: x kept in single precision (x = fl32(fl32(x) + fl32(gamma) u)), for GMRES-FD's first
// stage; otherwise x += gamma u in FP64.
template <int P, bool F32 = false>
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
    s_fac = st->gamma * pow2_recip(v_scale);
  }
  __syncthreads();
  if (s_skip) return;
  const int kk = s_kk;
  const double fac = s_fac;
  for (int c = tid; c < kk; c += NT) coef[c] = (W)y[c];
  __syncthreads();
  const long long ngroups = ld / VEC;
  const long long g0 = cta_begin(ngroups, 32), g1 = cta_begin(ngroups, 32, 1);
  for (long long g = g0 + tid; g < g1; g += NT) {
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
    for (int q = 0; q < VEC; ++q) {
      if constexpr (F32) xv[q] = (double)((float)xv[q] + (float)fac * (float)u[q]);
      else xv[q] += fac * (double)u[q];
    }
    stv(x + base, xv);
  }
}

// ---------------------------------------------------------------------------
// FP64 residual r = b - A x with the FP64 master matrix, ||r||, ||b||, and the
// restart decisions (Algorithm 1's explicit residual test / Algorithm 2
// "r_{i+1} = b - A x_{i+1} [double]").
// ---------------------------------------------------------------------------
constexpr int RES_TR = NT * 2;

// The matrix is the SELL-32 layout of the inner copy (same slices and columns) with FP64
// values: sv = A's values unscaled, in CSR order within each row, so every row's sum takes
// its entries in the order of the CSR input.  The SELL form keeps every load of the matrix
// coalesced and needs no shared-memory staging or barrier per tile.  The matrix is read once
// per call and is streamed evict-first.
// F32: the residual of GMRES run entirely in single precision (GMRES-FD's first stage,
// Section 3.3): b, A and x rounded to FP32 and the products and sums in FP32; the result
// is stored in the FP64 vector r and its norms accumulated in FP64.
template <bool F32>
__global__ void __launch_bounds__(NT, 2) k_residual(const int2* __restrict__ meta, const int* __restrict__ sc,
                                                    const double* __restrict__ sv, int nslices, int n,
                                                    const double* __restrict__ x,
                                                    const double* __restrict__ b, double* __restrict__ r,
                                                    double* __restrict__ part, DevState* st, Arrays arr,
                                                    int first) {
  using RW = typename std::conditional<F32, float, double>::type;
  constexpr int RPT = RES_TR / NT;
  __shared__ double red_r[NWARP], red_b[NWARP];
  __shared__ int s_skip, s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_flag(&st->stop);
  __syncthreads();
  if (s_skip) return;
  auto xval = [&](int c) -> RW { return (RW)x[c]; };
  double sr = 0.0, sb = 0.0;
  const int ntiles = (n + RES_TR - 1) / RES_TR;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * RES_TR;
    RW a[RPT];
    sell_rows<double, RW, RPT>(meta, sc, sv, nslices, r0, xval, a, true);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int row = r0 + tid + k * NT;
      if (row < n) {
        const RW bv = (RW)b[row];
        const RW rv = bv - a[k];
        r[row] = (double)rv;
        sr += (double)rv * (double)rv;
        sb += (double)bv * (double)bv;
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
      // GMRES-IR: progress of the refinement (explicit residual), for the stall test
      if (st->mode == 1) {
        const double rel = st->relres;
        if (first || rel < st->best_rel * (1.0 - 1e-3)) {
          st->best_rel = rel;
          st->stall = 0;
        } else {
          st->stall += 1;
        }
      }
      int stop = 1, status = ST_OK;
      if (!isfinite(gamma) || !isfinite(bnorm)) status = ST_NONFINITE;
      else if (bnorm == 0.0) { st->zero_rhs = 1; st->relres = 0.0; }
      else if (gamma <= st->rtol * bnorm) status = ST_OK;
      else if (st->singular) status = ST_BREAKDOWN;
      else if (st->iters >= st->max_iters) status = ST_NOT_CONVERGED;
      else if (st->mode == 1 && st->stall >= IR_STALL_LIMIT) status = ST_NOT_CONVERGED;
      else stop = 0;
      st->status = status;
      if (!stop) {
        st->sigma = 1.0 / gamma;
        arr.gabs[0] = 1.0;
        st->k = 0;
        st->last_step = -1;
        st->iters0 = st->iters;
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

// Fill the SELL-32 copy from CSR: one thread per (padded) row.  Values are divided by
// `scale` and rounded to the storage type; padding entries get value 0 and an in-range
// column (the row itself, or 0 past the last row).  sc == nullptr: values only (a second
// value array over columns already written).
template <class S>
__global__ void k_build_sell(const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ v, int n, const int2* __restrict__ meta,
                             int nslices, double scale, int* __restrict__ sc, S* __restrict__ sv) {
  const long long total = (long long)nslices * 32;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < total;
       r += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(r >> 5), l = (int)(r & 31);
    const int2 mt = meta[s];
    const int base = r < n ? rp[r] : 0;
    const int len = r < n ? rp[r + 1] - base : 0;
    const int pad_col = r < n ? (int)r : 0;
    for (int e = 0; e < mt.y; ++e) {
      const long long idx = (long long)mt.x + (long long)e * 32 + l;
      if (e < len) {
        if (sc) sc[idx] = ci[base + e];
        sv[idx] = to_s<S>(v[base + e] / scale);
      } else {
        if (sc) sc[idx] = pad_col;
        sv[idx] = to_s<S>(0.0);
      }
    }
  }
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
