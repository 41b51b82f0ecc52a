// bj_kernels.cuh -- block-Jacobi right preconditioner (Section 5.8: reverse Cuthill-McKee
// ordering, then block Jacobi with block size k; Section 3.4: a single-precision
// preconditioner inside GMRES-IR).  M = blockdiag(A[s:e, s:e]) over the contiguous blocks
// [s, e) = [q k, min((q + 1) k, n)) of the (reordered) matrix; the cycle multiplies by
// M^{-1} on the right, like the polynomial: w = A M^{-1} v_j, and x += gamma M^{-1} V y.
//
// Set-up factors every block once, in FP64, by LU with partial pivoting and stores the
// factors in the cycle's working type W; each application is a forward and a back
// substitution in W, one warp per block (or per 32 / k blocks when k <= 32).
#pragma once

#include "kernels.cuh"

namespace gm {

constexpr int BJ_MAX = 64;            // largest block size (GMRES_MAX_BJ_BLOCK)
constexpr int BJ_FACTOR_THREADS = 128;

// One CTA per diagonal block (grid-stride over the blocks).  The block is gathered from
// the FP64 CSR rows s..e-1 (entries outside the block's columns dropped, duplicates
// summed) into shared memory and factored P_q A_q = L U with partial pivoting (the pivot
// is the largest |a| of the column at or below the diagonal, the lowest row on ties).
// Output, block q at lu + q k^2, column-major with leading dimension k: L below the
// diagonal (unit diagonal implied), U above it, 1 / u_ii on it (rounded to W);
// rowp[s + i] = the block-local row of A_q that the pivoting moved to position i.  A zero
// pivot sets *bad (the block is singular; the plan is not created).
template <class W>
__global__ void __launch_bounds__(BJ_FACTOR_THREADS) k_bj_factor(
    const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ av, int n,
    int k, W* __restrict__ lu, int* __restrict__ rowp, int* bad) {
  __shared__ double a[BJ_MAX * BJ_MAX];  // row-major kb x kb
  __shared__ int prow[BJ_MAX];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblocks = (n + k - 1) / k;
  for (int q = blockIdx.x; q < nblocks; q += gridDim.x) {
    const int s = q * k;
    const int kb = min(k, n - s);
    for (int i = tid; i < kb * kb; i += blockDim.x) a[i] = 0.0;
    for (int i = tid; i < kb; i += blockDim.x) prow[i] = i;
    __syncthreads();
    for (int r = tid; r < kb; r += blockDim.x)  // one thread per row: duplicates add in order
      for (int p = rp[s + r]; p < rp[s + r + 1]; ++p) {
        const int c = ci[p] - s;
        if (c >= 0 && c < kb) a[r * kb + c] += av[p];
      }
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
      if (warp == 0) {  // pivot: largest |a_ic|, i >= c, lowest i on ties
        double best = -1.0;
        int bi = kb;
        for (int i = c + lane; i < kb; i += 32) {
          const double v = fabs(a[i * kb + c]);
          if (v > best) {
            best = v;
            bi = i;
          }
        }
        for (int d = 16; d > 0; d >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, best, d);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, d);
          if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
          }
        }
        if (lane == 0) {
          s_piv = bi < kb ? bi : c;  // no candidate (a NaN column): keep the row
          if (!(best > 0.0)) atomicOr(bad, 1);
        }
      }
      __syncthreads();
      const int pv = s_piv;
      if (pv != c) {
        for (int j = tid; j < kb; j += blockDim.x) {
          const double t = a[c * kb + j];
          a[c * kb + j] = a[pv * kb + j];
          a[pv * kb + j] = t;
        }
        if (tid == 0) {
          const int t = prow[c];
          prow[c] = prow[pv];
          prow[pv] = t;
        }
      }
      __syncthreads();
      const double d = a[c * kb + c];
      const double inv = d != 0.0 ? 1.0 / d : 0.0;
      for (int i = c + 1 + tid; i < kb; i += blockDim.x) a[i * kb + c] *= inv;
      __syncthreads();
      const int t = kb - c - 1;
      for (int e = tid; e < t * t; e += blockDim.x) {
        const int i = c + 1 + e / t, j = c + 1 + e % t;
        a[i * kb + j] -= a[i * kb + c] * a[c * kb + j];
      }
      __syncthreads();
    }
    W* out = lu + (size_t)q * k * k;
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      const int j = e / kb, i = e % kb;  // column j, row i
      const double v = a[i * kb + j];
      out[(size_t)j * k + i] = (W)(i == j ? (v != 0.0 ? 1.0 / v : 0.0) : v);
    }
    for (int i = tid; i < kb; i += blockDim.x) rowp[s + i] = prow[i];
    __syncthreads();
  }
}

// Shared-memory slot of one warp of k_bj_apply: its G = 32 / k blocks (k <= 32) or its
// one block (k > 32), k^2 values each.
__host__ __device__ constexpr int bj_slot(int k) { return k <= 32 ? (32 / k) * k * k : k * k; }
constexpr int BJ_APPLY_WARPS = 4;

// Copies cnt values of W from global to shared memory with one 4-byte cp.async per lane and
// word (no register round trip, every word in flight at once), then waits for them.
template <class W>
__device__ __forceinline__ void bj_stage(W* dst, const W* src, long long cnt) {
  const int lane = threadIdx.x & 31;
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  const long long words = cnt * (long long)(sizeof(W) / 4);
  for (long long t = lane; t < words; t += 32) {
    const unsigned da = (unsigned)__cvta_generic_to_shared(d + t);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(da), "l"(s + t) : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();
}

// z = M^{-1} v.  k <= 32: a warp takes G = 32 / k consecutive blocks, lane l row l % k of
// block l / k (lanes >= G k idle); 32 < k <= 64: a warp takes one block, lane l rows l and
// l + 32.  The warp first stages its blocks' factors in shared memory (the blocks are
// contiguous), so the 2k dependent steps of the substitutions read shared memory, not
// HBM.  y = rows of v in pivot order (rowp), forward substitution with the unit lower
// factor, back substitution with the upper factor (times the stored 1 / u_ii), column by
// column.  in_cycle: skip once the cycle (or the solve) has ended, like the cycle's other
// kernels.  Dynamic shared memory: BJ_APPLY_WARPS * bj_slot(k) values of W.
template <class W>
__global__ void __launch_bounds__(32 * BJ_APPLY_WARPS) k_bj_apply(
    const W* __restrict__ lu, const int* __restrict__ rowp, int n, int k,
    const W* __restrict__ v, W* __restrict__ z, const DevState* st, int in_cycle) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_skip;
  if (threadIdx.x == 0)
    s_skip = st ? (read_flag(&st->stop) | (in_cycle ? read_flag(&st->cycle_done) : 0)) : 0;
  __syncthreads();
  if (s_skip) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  W* sb = reinterpret_cast<W*>(smem_raw) + (size_t)(threadIdx.x >> 5) * bj_slot(k);
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int nblocks = (n + k - 1) / k;
  const long long kk = (long long)k * k;
  if (k <= 32) {
    const int G = 32 / k;
    const int g = lane / k, i = lane % k, base = g * k;
    for (long long w = warp0; w * G < nblocks; w += nwarps) {
      const long long q0 = w * G;
      const long long q = q0 + g;
      const bool active = g < G && q < nblocks;
      const long long s = q * k;
      const int kb = active ? (int)min((long long)k, n - s) : 0;
      const bool mine = i < kb;
      W y = mine ? v[s + rowp[s + i]] : W(0);
      __syncwarp();  // the previous iteration's reads of sb are done
      bj_stage(sb, lu + q0 * kk, min((long long)G, nblocks - q0) * kk);
      const W* B = sb + (active ? g : 0) * kk;
      for (int c = 0; c + 1 < k; ++c) {  // forward: rows below c
        const W yc = __shfl_sync(full, y, base + c);
        if (mine && i > c) y -= B[c * k + i] * yc;
      }
      for (int c = k - 1; c >= 0; --c) {  // back: rows above c
        const W yc = __shfl_sync(full, y, base + c);
        const W zc = c < kb ? yc * B[c * k + c] : W(0);
        if (mine && i == c) y = zc;
        if (mine && i < c && c < kb) y -= B[c * k + i] * zc;
      }
      if (mine) z[s + i] = y;
    }
  } else {
    for (long long q = warp0; q < nblocks; q += nwarps) {
      const long long s = q * k;
      const int kb = (int)min((long long)k, n - s);
      const int i0 = lane, i1 = lane + 32;
      W y0 = i0 < kb ? v[s + rowp[s + i0]] : W(0);
      W y1 = i1 < kb ? v[s + rowp[s + i1]] : W(0);
      __syncwarp();
      bj_stage(sb, lu + q * kk, kk);
      const W* B = sb;
      for (int c = 0; c + 1 < kb; ++c) {
        const W yc = __shfl_sync(full, c < 32 ? y0 : y1, c & 31);
        const W* col = B + c * k;
        if (i0 > c && i0 < kb) y0 -= col[i0] * yc;
        if (i1 > c && i1 < kb) y1 -= col[i1] * yc;
      }
      for (int c = kb - 1; c >= 0; --c) {
        const W* col = B + c * k;
        const W zc = __shfl_sync(full, c < 32 ? y0 : y1, c & 31) * col[c];
        if (i0 == c) y0 = zc;
        if (i1 == c) y1 = zc;
        if (i0 < c) y0 -= col[i0] * zc;
        if (i1 < c) y1 -= col[i1] * zc;
      }
      if (i0 < kb) z[s + i0] = y0;
      if (i1 < kb) z[s + i1] = y1;
    }
  }
}

// dst[i] = src[perm[i]] (into the reordered numbering).
__global__ void k_gather_perm(const double* __restrict__ src, const int* __restrict__ perm, int n,
                              double* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}

// dst[perm[i]] = src[i] (back to the caller's numbering).
__global__ void k_scatter_perm(const double* __restrict__ src, const int* __restrict__ perm, int n,
                               double* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[perm[i]] = src[i];
}

}  // namespace gm
