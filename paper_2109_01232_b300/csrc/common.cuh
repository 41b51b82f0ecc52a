// common.cuh -- precision traits, vector memory helpers, warp reductions and the
// device-resident solver state shared by the GMRES kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace gm {

constexpr int NT = 512;           // threads per CTA of the streaming kernels
constexpr int NWARP = NT / 32;
constexpr int LSQ_MAX = 512;      // largest restart length (GMRES_MAX_RESTART)
constexpr int LSQ_PACKED_MAX = 200;  // R staged in shared memory up to this m (160 KB)
constexpr int TILE_MAX = 4096;    // largest SpMV row tile; every buffer's leading dimension
                                  // is a multiple of it, so tiles never cross the padding

// Precision of the inner cycle: S = storage type of the Krylov basis and of the
// copy of A, W = working (accumulation) type, VEC = rows per thread of the CGS update
// kernels (one or two 16-byte vectors of S), VT = rows per lane in the SpMV kernel's dot
// products (its warp tile is VT slices of 32 rows: 128 rows in every precision; with
// 256-row tiles in FP16/BF16 a CTA had fewer tiles than warps on 10^6 rows), RT = rows per
// thread of the row-tiled SpMV kernels (CSR tile, polynomial, plain SpMV).
// FP64 takes 4 rows per thread (two 16-byte vectors) in the CGS and dot-product loops: its
// warp reductions then cost 9 FP64 additions per 8 columns and 128 rows instead of 64, and
// FP64 arithmetic, not bandwidth, bounds the FP64 cycle on this part.
template <int P> struct Tr;
// V_EF: the SpMV kernel reads the old basis columns with the half-evict-first L2 policy
// (FP64/FP32) or plainly (FP16/BF16: their basis is small enough that keeping all of it in
// L2 for the CGS kernels measured faster).
template <> struct Tr<0> { using S = double;        using W = double; static constexpr int VEC = 4, VT = 4, RT = 2; static constexpr bool V_EF = true; };
template <> struct Tr<1> { using S = float;         using W = float;  static constexpr int VEC = 4, VT = 4, RT = 4; static constexpr bool V_EF = true; };
template <> struct Tr<2> { using S = __half;        using W = float;  static constexpr int VEC = 8, VT = 4, RT = 4; static constexpr bool V_EF = false; };
template <> struct Tr<3> { using S = __nv_bfloat16; using W = float;  static constexpr int VEC = 8, VT = 4, RT = 4; static constexpr bool V_EF = false; };
// FP64 with two rows per thread in the step kernels, for plans too small to give every CTA
// of the four-row grid its rows (fewer rows per thread spread the FP64 work over more SMs);
// chosen at plan creation by the row count (solver.cu, fp64_kernel_set).  Not a storage
// precision of the API: a plan's precision stays GMRES_FP64.
constexpr int KP_FP64_NARROW = 4;
template <> struct Tr<KP_FP64_NARROW> { using S = double; using W = double; static constexpr int VEC = 2, VT = 2, RT = 2; static constexpr bool V_EF = true; };

// storage -> working type
// 1 / v for v an exact power of two in the normal range (the basis scale v_scale): the
// exponent is mirrored, so x * pow2_recip(v) == x / v exactly, without an FP64 division
// (slow to issue on this part).
__device__ __forceinline__ double pow2_recip(double v) {
  return __longlong_as_double(0x7FE0000000000000LL - __double_as_longlong(v));
}
__device__ __forceinline__ double to_w(double v) { return v; }
__device__ __forceinline__ float to_w(float v) { return v; }
__device__ __forceinline__ float to_w(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_w(__nv_bfloat16 v) { return __bfloat162float(v); }

// round to the storage type (round to nearest even)
template <class S> __device__ __forceinline__ S to_s(double v);
template <class S> __device__ __forceinline__ S to_s(float v);
template <> __device__ __forceinline__ double to_s<double>(double v) { return v; }
template <> __device__ __forceinline__ double to_s<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ float to_s<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ float to_s<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_s<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __half to_s<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_s<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_s<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// N consecutive elements through one or more 16-byte accesses, or one 8-byte access when
// the vector is 8 bytes (p aligned to the vector's size, at most 16).
template <class T, int N>
struct VecBits {
  static constexpr int BYTES = (int)(sizeof(T) * N);
  static_assert(BYTES % 16 == 0 || BYTES == 8, "vector must be 8 bytes or a multiple of 16");
  static constexpr bool WIDE = BYTES % 16 == 0;
  static constexpr int Q = WIDE ? BYTES / 16 : 1;
};
template <class T, int N>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T (&o)[N]) {
  using VB = VecBits<T, N>;
  if constexpr (VB::WIDE) {
    uint4 u[VB::Q];
#pragma unroll
    for (int q = 0; q < VB::Q; ++q) u[q] = reinterpret_cast<const uint4*>(p)[q];
    memcpy(o, u, sizeof(u));
  } else {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    memcpy(o, &u, sizeof(u));
  }
}
template <class T, int N>
__device__ __forceinline__ void stv(T* __restrict__ p, const T (&o)[N]) {
  using VB = VecBits<T, N>;
  if constexpr (VB::WIDE) {
    uint4 u[VB::Q];
    memcpy(u, o, sizeof(u));
#pragma unroll
    for (int q = 0; q < VB::Q; ++q) reinterpret_cast<uint4*>(p)[q] = u[q];
  } else {
    uint2 u;
    memcpy(&u, o, sizeof(u));
    *reinterpret_cast<uint2*>(p) = u;
  }
}
// Streaming load of data that is read once per kernel (evict-first in L1/L2).
template <class T, int N>
__device__ __forceinline__ void ldv_stream(const T* __restrict__ p, T (&o)[N]) {
  using VB = VecBits<T, N>;
  if constexpr (VB::WIDE) {
    uint4 u[VB::Q];
#pragma unroll
    for (int q = 0; q < VB::Q; ++q) u[q] = __ldcs(reinterpret_cast<const uint4*>(p) + q);
    memcpy(o, u, sizeof(u));
  } else {
    const uint2 u = __ldcs(reinterpret_cast<const uint2*>(p));
    memcpy(o, &u, sizeof(u));
  }
}

// L2 evict-first loads for data that the kernel reads for the last time before other
// data needs the cache (the basis V streams through L2 once per pass, and marking it
// keeps the matrix and the work vectors resident).  Only for memory that no thread
// writes during the kernel: the asm is not ordered against other memory operations.
// Half of the lines get the evict-first policy, the others keep the normal one: of the
// fractions measured in the SpMV's dot products on the 100^3 workload (FP32: 0, 0.25, 0.5,
// 0.75, 1), 0.5 gave the shortest solves -- the next kernel still finds part of the basis in
// L2 while the gathered vector stays resident.
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 0.5;" : "=l"(pol));
  return pol;
}
template <class T, int N>
__device__ __forceinline__ void ldv_evict_first(const T* __restrict__ p, T (&o)[N]) {
  using VB = VecBits<T, N>;
  const unsigned long long pol = l2_evict_first_policy();
  if constexpr (VB::WIDE) {
    uint4 u[VB::Q];
#pragma unroll
    for (int q = 0; q < VB::Q; ++q)
      asm("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
          : "=r"(u[q].x), "=r"(u[q].y), "=r"(u[q].z), "=r"(u[q].w)
          : "l"(reinterpret_cast<const uint4*>(p) + q), "l"(pol));
    memcpy(o, u, sizeof(u));
  } else {
    uint2 u;
    asm("ld.global.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
        : "=r"(u.x), "=r"(u.y)
        : "l"(reinterpret_cast<const uint2*>(p)), "l"(pol));
    memcpy(o, &u, sizeof(u));
  }
}
// ldv (EF = false) or ldv_evict_first (EF = true).
template <bool EF, class T, int N>
__device__ __forceinline__ void ldv_sel(const T* __restrict__ p, T (&o)[N]) {
  if constexpr (EF) ldv_evict_first(p, o);
  else ldv(p, o);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Status codes (mirrors gmres_status in include/gmres_ir.h).
enum { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_BREAKDOWN = 2, ST_NONFINITE = 3, ST_INVALID = 4,
       ST_TIMEOUT = 8 };

// Device-resident state of one solve.  The host writes it once before a solve and
// reads it once after; every decision in between is taken on the device.
struct DevState {
  int stop;          // 1: the solve is finished (status holds why)
  int cycle_done;    // 1: the current Arnoldi cycle has ended
  int status;
  int k;             // Arnoldi steps taken in the current cycle
  int k_used;        // columns used by the least-squares solve (after trimming)
  int singular;      // 1: the last least-squares factor was singular
  int breakdown;     // 1: the last cycle ended by a (lucky) breakdown
  int outer;         // cycles completed
  int m;             // restart length
  int mode;          // 0: FP64 GMRES (implicit test against rtol), 1: IR (inner_rtol)
  int zero_rhs;      // 1: ||b|| = 0, the answer is x = 0
  int hist_cap;      // capacity of the residual history
  long long iters;   // Arnoldi steps over the whole solve
  long long iters0;  // Arnoldi steps before the current cycle
  int last_step;     // last step whose second CGS kernel ran in this cycle (-1: none)
  long long max_iters;
  double rtol, inner_rtol;
  double bnorm, gamma, relres;
  double stop_rel;   // implicit-residual threshold of the current cycle, relative to gamma
  double sigma;      // 1 / norm of the next SpMV source vector
  double wnorm;      // ||A v_j|| of the current step (breakdown test)
  double u_work;     // unit roundoff of the working precision
  double best_rel;   // IR: smallest explicit relative residual so far
  int stall;         // IR: refinement steps since best_rel last dropped by 0.1%
  int stream_matrix; // 1: the preconditioned path's SpMVs load the copy of A evict-first
  unsigned int ticket[4];
};

// GMRES-IR stops as NOT_CONVERGED after this many refinement steps without progress (an
// inner precision too coarse for the problem makes the iteration stall or diverge).
constexpr int IR_STALL_LIMIT = 20;

// Small dense arrays of the cycle (FP64, device memory, one allocation).
struct Arrays {
  double* h1;    // m+2   first CGS pass coefficients (plus spare)
  double* h2;    // m+2   second CGS pass coefficients
  double* H;     // (m+1) x m, column-major, unrotated Hessenberg matrix
  double* R;     // (m+1) x m, column-major, after the Givens rotations
  double* cs;    // m
  double* sn;    // m
  double* gabs;  // m+1   |g_j| of the rotated right-hand side (|g_0| = 1 at a cycle start)
  double* y;     // m     least-squares solution
  double* hist;  // hist_cap relative residual estimates
};

}  // namespace gm
