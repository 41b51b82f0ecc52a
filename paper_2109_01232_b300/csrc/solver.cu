// solver.cu -- plans, CUDA-graph capture of one restart cycle, and the C ABI.
//
// A plan owns the workspace of one matrix: the Krylov basis V ((m+1) columns of
// ld values in the storage precision), three work vectors, the FP64 residual /
// iterate / right-hand-side buffers, the low-precision copy of A, the Hessenberg
// arrays and the device state.  One restart cycle of Algorithm 1 / Algorithm 2
// (m Arnoldi steps, least squares, x update, FP64 residual) is captured once as
// a CUDA graph; a solve launches that graph until the device state says stop.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gmres_ir.h"
#include "kernels.cuh"
#include "cgs_tma.cuh"
#include "poly_kernels.cuh"
#include "poly_host.h"
#include "bj_kernels.cuh"
#include "rcm_host.h"

namespace gm {

// The last CUDA failure seen by this thread (call site and runtime message), reported by
// gmres_last_error().
static thread_local char g_last_error[256] = "";

static int note_cuda(cudaError_t e, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "solver.cu:%d: %s: %s", line, cudaGetErrorName(e),
           cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA;
}
#define CK(x)                                                 \
  do {                                                        \
    cudaError_t e_ = (x);                                     \
    if (e_ != cudaSuccess) return ::gm::note_cuda(e_, __LINE__); \
  } while (0)
// Evaluates a CUDA call; on failure records it and yields the status code, else 0.
#define CUDA_STATUS(x) ([&]() -> int {                        \
    cudaError_t e_ = (x);                                     \
    return e_ == cudaSuccess ? 0 : ::gm::note_cuda(e_, __LINE__); \
  }())

static inline long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

struct PolyOp {
  int pair;       // 0: real root, 1: conjugate pair
  int last;       // last operation: the prod update is skipped
  double c1, c2;
};

struct Plan {
  int kind = 1;  // 0: FP64 GMRES, 1: GMRES-IR
  int prec = 1;  // storage precision of the cycle
  int kp = 1;    // kernel set (Tr index) of the cycle: prec, or KP_FP64_NARROW for small FP64 plans
  gmres_csr A{};
  int n = 0, m = 0;
  long long ld = 0;
  gmres_params p{};
  double a_scale = 1.0, v_scale = 1.0;
  // inner copy of A (SELL-32, storage precision)
  int2* sell_meta = nullptr;   // per slice: offset of its first entry, width
  int* sell_cols = nullptr;
  void* sell_vals = nullptr;
  int nslices = 0;
  long long sell_nnz = 0;      // stored entries including padding
  void* V = nullptr;
  void *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;
  double *r = nullptr, *xb = nullptr, *bb = nullptr;
  void* part = nullptr;  // per-CTA partial sums: residual, then the step buffers
  size_t part_step_off = 0;
  DevState* st = nullptr;
  DevState* h_st = nullptr;  // pinned
  double* arr_mem = nullptr;
  Arrays arr{};
  int hist_cap = 0;
  int sms = 148;
  int grid_spmv = 1, grid_vec = 1, grid_res = 1;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // polynomial preconditioner (right, p(A) in product form)
  std::vector<double> roots_re, roots_im;
  std::vector<PolyOp> poly;         // product-form program built from the roots
  void *pa = nullptr, *pb = nullptr, *pt = nullptr, *py = nullptr;  // working-type vectors
  bool poly32 = false;           // FP64 cycle, polynomial applied in FP32
  void* sell_vals32 = nullptr;   // FP32 values of the SELL copy (poly32)
  void* sell_vals64 = nullptr;   // FP64 values of the SELL copy (residual of non-FP64 plans)
  // block-Jacobi preconditioner (right) and the reverse Cuthill-McKee reordering
  int bj = 0;                    // block size k; 0 = none
  void* bj_lu = nullptr;         // factors of the diagonal blocks (working type, k*k per block)
  int* bj_rowp = nullptr;        // pivot order of each block's rows
  int grid_bj = 1;
  int* perm = nullptr;           // perm[new] = old (device); null without reordering
  int32_t* pA_rp = nullptr;      // the plan's reordered copy of A (device CSR)
  int32_t* pA_ci = nullptr;
  double* pA_v = nullptr;
  int grid_elem = 1;
  int stream_matrix = 0;         // DevState::stream_matrix (see plan_create)
  double t_setup_ms = 0.0;
};

// Product-form program of p(A) from Leja-ordered roots: a real root contributes one
// operation (c1 = 1/theta), a conjugate pair a +- ib one operation (c1 = 2a/q, c2 = 1/q,
// q = a^2 + b^2).
static std::vector<PolyOp> poly_program(const std::vector<double>& re, const std::vector<double>& im) {
  std::vector<PolyOp> ops;
  for (size_t i = 0; i < re.size();) {
    PolyOp op{};
    if (im[i] == 0.0) {
      op.pair = 0;
      op.c1 = 1.0 / re[i];
      i += 1;
    } else {
      const double q = re[i] * re[i] + im[i] * im[i];
      op.pair = 1;
      op.c1 = 2.0 * re[i] / q;
      op.c2 = 1.0 / q;
      i += 2;
    }
    ops.push_back(op);
  }
  if (!ops.empty()) ops.back().last = 1;
  return ops;
}

// ---------------------------------------------------------------------------
// Kernel launch sequences (templated on the storage precision).
// ---------------------------------------------------------------------------

// Partial-sum buffers of the Arnoldi step kernels (inside pl.part, after the residual's).
template <int P>
static StepParts<typename Tr<P>::W> step_parts(const Plan& pl) {
  using W = typename Tr<P>::W;
  StepParts<W> sp;
  W* base = reinterpret_cast<W*>(static_cast<unsigned char*>(pl.part) + pl.part_step_off);
  const size_t n1 = (size_t)(pl.m + 2) * pl.grid_spmv;
  sp.p1[0] = base;
  sp.p1[1] = base + n1;
  sp.p2 = base + 2 * n1;
  sp.p3 = sp.p2 + (size_t)(pl.m + 1) * pl.grid_vec;
  sp.g1 = pl.grid_spmv;
  sp.g2 = pl.grid_vec;
  return sp;
}

// y = p(A) prod0 (prod0 is pl.pa, overwritten; pl.pb / pl.pt are scratch).
template <int P>
static void launch_poly(Plan& pl, int in_cycle, cudaStream_t s) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  // P is the polynomial's precision: the plan's, or FP32 under an FP64 cycle (poly32)
  const void* vals = pl.poly32 && P == 1 ? pl.sell_vals32 : pl.sell_vals;
  W* cur = (W*)pl.pa;
  W* nxt = (W*)pl.pb;
  W* y = (W*)pl.py;
  W* t = (W*)pl.pt;
  int first = 1;
  for (const PolyOp& op : pl.poly) {
    if (!op.pair) {
      if (op.last) {
        k_poly_axpy<P><<<pl.grid_elem, NT, 0, s>>>(cur, y, pl.n, op.c1, first, pl.st, in_cycle);
      } else {
        k_poly_spmv<P, POLY_REAL><<<pl.grid_spmv, NT, 0, s>>>(
            pl.sell_meta, pl.sell_cols, (const S*)vals, pl.nslices, pl.n, pl.a_scale, cur,
            nullptr, y, nxt,
            op.c1, 0.0, first, pl.st, in_cycle);
        std::swap(cur, nxt);
      }
    } else {
      k_poly_spmv<P, POLY_PAIR_A><<<pl.grid_spmv, NT, 0, s>>>(
          pl.sell_meta, pl.sell_cols, (const S*)vals, pl.nslices, pl.n, pl.a_scale, cur,
          nullptr, y,
          op.last ? nullptr : t, op.c1, op.c2, first, pl.st, in_cycle);
      if (!op.last) {
        k_poly_spmv<P, POLY_PAIR_B><<<pl.grid_spmv, NT, 0, s>>>(
            pl.sell_meta, pl.sell_cols, (const S*)vals, pl.nslices, pl.n, pl.a_scale, cur,
            t, nullptr, nxt,
            op.c1, op.c2, 0, pl.st, in_cycle);
        std::swap(cur, nxt);
      }
    }
    first = 0;
  }
}

// Dynamic shared memory of k_bj_apply for the plan's block size.
template <class W>
static size_t bj_smem(const Plan& pl) {
  return sizeof(W) * (size_t)BJ_APPLY_WARPS * bj_slot(pl.bj);
}

// Kernel `which` (0: fused SpMV + first-pass dots -- with a polynomial preconditioner the
// whole w = A p(A) v_j chain --, 1: first CGS update + second-pass dots, 2: second CGS
// update + norm + Givens) of Arnoldi step j.
template <int P>
static void launch_step_kernel(Plan& pl, int j, int which, cudaStream_t s) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  S* V = (S*)pl.V;
  W* w1 = (W*)pl.w1;
  W* w2 = (W*)pl.w2;
  W* w3 = (W*)pl.w3;
  const StepParts<W> sp = step_parts<P>(pl);
  if (which == 0) {
    const size_t sm1 = SellSmem<P>::bytes(j + 2);
    if (pl.bj) {  // w = A M^{-1} v_j: store v_j, z = M^{-1} v_j, SpMV of z
      if (j == 0)
        k_poly_start<P, double><<<pl.grid_elem, NT, 0, s>>>(pl.r, pl.v_scale, pl.n, V, pl.ld, 0,
                                                           (W*)pl.pa, sp, pl.st, pl.arr);
      else
        k_poly_start<P, W><<<pl.grid_elem, NT, 0, s>>>(w3, pl.v_scale, pl.n, V, pl.ld, j,
                                                      (W*)pl.pa, sp, pl.st, pl.arr);
      k_bj_apply<W><<<pl.grid_bj, 32 * BJ_APPLY_WARPS, bj_smem<W>(pl), s>>>((const W*)pl.bj_lu, pl.bj_rowp, pl.n, pl.bj,
                                               (const W*)pl.pa, (W*)pl.py, pl.st, 1);
      k_spmv_sell<P, W, true><<<pl.grid_spmv, NT, sm1, s>>>(
          pl.sell_meta, pl.sell_cols, (const S*)pl.sell_vals, pl.nslices, pl.n, pl.ld, pl.a_scale,
          (const W*)pl.py, pl.v_scale, V, j, w1, sp, pl.st, pl.arr);
      return;
    }
    if (!pl.poly.empty() && pl.poly32) {  // FP64 cycle, polynomial in FP32
      if (j == 0)
        k_poly_start<P, double, float><<<pl.grid_elem, NT, 0, s>>>(pl.r, pl.v_scale, pl.n, V, pl.ld, 0,
                                                                  (float*)pl.pa, sp, pl.st, pl.arr);
      else
        k_poly_start<P, W, float><<<pl.grid_elem, NT, 0, s>>>(w3, pl.v_scale, pl.n, V, pl.ld, j,
                                                             (float*)pl.pa, sp, pl.st, pl.arr);
      launch_poly<1>(pl, 1, s);
      k_spmv_sell<P, float, true><<<pl.grid_spmv, NT, sm1, s>>>(
          pl.sell_meta, pl.sell_cols, (const S*)pl.sell_vals, pl.nslices, pl.n, pl.ld, pl.a_scale,
          (const float*)pl.py, pl.v_scale, V, j, w1, sp, pl.st, pl.arr);
      return;
    }
    if (!pl.poly.empty()) {
      if (j == 0)
        k_poly_start<P, double><<<pl.grid_elem, NT, 0, s>>>(pl.r, pl.v_scale, pl.n, V, pl.ld, 0,
                                                           (W*)pl.pa, sp, pl.st, pl.arr);
      else
        k_poly_start<P, W><<<pl.grid_elem, NT, 0, s>>>(w3, pl.v_scale, pl.n, V, pl.ld, j,
                                                      (W*)pl.pa, sp, pl.st, pl.arr);
      launch_poly<P>(pl, 1, s);
      k_spmv_sell<P, W, true><<<pl.grid_spmv, NT, sm1, s>>>(
          pl.sell_meta, pl.sell_cols, (const S*)pl.sell_vals, pl.nslices, pl.n, pl.ld, pl.a_scale,
          (const W*)pl.py, pl.v_scale, V, j, w1, sp, pl.st, pl.arr);
      return;
    }
    const double rs = pl.a_scale / pl.v_scale;
    if (j == 0 && P != GMRES_FP64) {
      // v_0 = store(v_scale sigma r) from the FP64 residual: formed once per row here (FP64
      // products issue slowly on this part), then the SpMV gathers the stored v_0 as a
      // preconditioned SpMV gathers its input (the same values as forming them per gather)
      k_store_basis<P, double><<<pl.grid_elem, NT, 0, s>>>(pl.r, pl.v_scale, pl.n, V, pl.ld, 0,
                                                          pl.st, 1);
      k_spmv_sell<P, S, true><<<pl.grid_spmv, NT, sm1, s>>>(
          pl.sell_meta, pl.sell_cols, (const S*)pl.sell_vals, pl.nslices, pl.n, pl.ld, rs,
          (const S*)V, pl.v_scale, V, 0, w1, sp, pl.st, pl.arr);
    } else if (j == 0)
      k_spmv_sell<P, double, false><<<pl.grid_spmv, NT, sm1, s>>>(
          pl.sell_meta, pl.sell_cols, (const S*)pl.sell_vals, pl.nslices, pl.n, pl.ld, rs, pl.r,
          pl.v_scale, V, 0, w1, sp, pl.st, pl.arr);
    else
      k_spmv_sell<P, W, false><<<pl.grid_spmv, NT, sm1, s>>>(
          pl.sell_meta, pl.sell_cols, (const S*)pl.sell_vals, pl.nslices, pl.n, pl.ld, rs, w3,
          pl.v_scale, V, j, w1, sp, pl.st, pl.arr);
  } else {
    // Both forms run on grid_vec CTAs, so the partial-sum layout does not depend on the form.
    const int nc = j + 1;
    const int ns = pl.p.cgs_kernel == GMRES_CGS_TMA ? TmaLayout<P>::stages(nc) : 0;
    const size_t tb = TmaLayout<P>::bytes(nc, ns);
    const TmaWait tw{pl.p.tma_wait_cycles > 0 ? pl.p.tma_wait_cycles : TMA_WAIT_CYCLES,
                     pl.p.tma_test_withhold != 0};
    if (which == 1) {
      if (ns && nc <= TMA_U1_MAX_COLS)
        k_cgs_u1_tma<P><<<pl.grid_vec, TMA_THREADS, tb, s>>>(V, pl.ld, j, pl.v_scale, w1, w2, sp,
                                                             pl.st, pl.arr.h1, ns, tw);
      else
        k_cgs_u1<P><<<pl.grid_vec, NT, sizeof(W) * (size_t)nc * (1 + NWARP), s>>>(
            V, pl.ld, j, pl.v_scale, w1, w2, sp, pl.st, pl.arr.h1);
    } else {
      if (ns)
        k_cgs_u2_tma<P><<<pl.grid_vec, TMA_THREADS, tb, s>>>(V, pl.ld, j, pl.v_scale, w2, w3, sp,
                                                             pl.st, pl.arr.h2, ns, tw);
      else
        k_cgs_u2<P><<<pl.grid_vec, NT, sizeof(W) * (size_t)nc, s>>>(V, pl.ld, j, pl.v_scale, w2,
                                                                    w3, sp, pl.st, pl.arr.h2);
    }
  }
}

template <int P>
static void launch_step(Plan& pl, int j, cudaStream_t s) {
  for (int which = 0; which < 3; ++which) launch_step_kernel<P>(pl, j, which, s);
}

static void launch_residual(Plan& pl, int first, cudaStream_t s) {
  const double* av = (const double*)(pl.prec == GMRES_FP64 ? pl.sell_vals : pl.sell_vals64);
  if (pl.kind == 2)  // single-precision GMRES: FP32 residual
    k_residual<true><<<pl.grid_res, NT, 0, s>>>(pl.sell_meta, pl.sell_cols, av, pl.nslices, pl.n,
                                                pl.xb, pl.bb, pl.r, (double*)pl.part, pl.st, pl.arr,
                                                first);
  else
    k_residual<false><<<pl.grid_res, NT, 0, s>>>(pl.sell_meta, pl.sell_cols, av, pl.nslices, pl.n,
                                                 pl.xb, pl.bb, pl.r, (double*)pl.part, pl.st, pl.arr,
                                                 first);
}

// Kernel `which` of the cycle's end (0: least squares, 1: x update -- x += gamma p(A) V y
// with a preconditioner --, 2: FP64 residual).
template <int P>
static void launch_tail_kernel(Plan& pl, int which, cudaStream_t s) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  if (which == 0) {
    k_finalize<P><<<1, NT, 0, s>>>(step_parts<P>(pl), pl.st, pl.arr);
    const int packed = pl.m <= LSQ_PACKED_MAX;
    k_lsq<<<1, NT, packed ? sizeof(double) * (size_t)pl.m * (pl.m + 1) / 2 : 0, s>>>(pl.st, pl.arr,
                                                                                   packed);
  } else if (which == 1) {
    if (pl.bj) {  // x += gamma M^{-1} (V y)
      k_vy<P><<<pl.grid_vec, NT, sizeof(W) * (size_t)pl.m, s>>>((const S*)pl.V, pl.ld, pl.v_scale,
                                                               pl.st, pl.arr.y, (W*)pl.pa);
      k_bj_apply<W><<<pl.grid_bj, 32 * BJ_APPLY_WARPS, bj_smem<W>(pl), s>>>((const W*)pl.bj_lu, pl.bj_rowp, pl.n, pl.bj,
                                               (const W*)pl.pa, (W*)pl.py, pl.st, 0);
      k_xadd<W><<<pl.grid_elem, NT, 0, s>>>((const W*)pl.py, pl.xb, pl.n, pl.st);
    } else if (!pl.poly.empty()) {
      if (pl.poly32) {
        k_vy<P, float><<<pl.grid_vec, NT, sizeof(W) * (size_t)pl.m, s>>>(
            (const S*)pl.V, pl.ld, pl.v_scale, pl.st, pl.arr.y, (float*)pl.pa);
        launch_poly<1>(pl, 0, s);
        k_xadd<float><<<pl.grid_elem, NT, 0, s>>>((const float*)pl.py, pl.xb, pl.n, pl.st);
      } else {
        k_vy<P><<<pl.grid_vec, NT, sizeof(W) * (size_t)pl.m, s>>>((const S*)pl.V, pl.ld, pl.v_scale,
                                                                 pl.st, pl.arr.y, (W*)pl.pa);
        launch_poly<P>(pl, 0, s);
        k_xadd<W><<<pl.grid_elem, NT, 0, s>>>((const W*)pl.py, pl.xb, pl.n, pl.st);
      }
    } else {
      if (pl.kind == 2)
        k_xupd<P, true><<<pl.grid_vec, NT, sizeof(W) * (size_t)pl.m, s>>>((const S*)pl.V, pl.ld,
                                                                         pl.v_scale, pl.st, pl.arr.y, pl.xb);
      else
        k_xupd<P><<<pl.grid_vec, NT, sizeof(W) * (size_t)pl.m, s>>>((const S*)pl.V, pl.ld,
                                                                   pl.v_scale, pl.st, pl.arr.y, pl.xb);
    }
  } else {
    launch_residual(pl, 0, s);
  }
}

template <int P>
static void launch_cycle_tail(Plan& pl, cudaStream_t s) {
  for (int which = 0; which < 3; ++which) launch_tail_kernel<P>(pl, which, s);
}

template <int P>
static void launch_cycle(Plan& pl, cudaStream_t s) {
  for (int j = 0; j < pl.m; ++j) launch_step<P>(pl, j, s);
  launch_cycle_tail<P>(pl, s);
}

// Grid of a cluster kernel: `want` CTAs rounded up to a multiple of CL, capped at the
// clusters that fit on the GPU at once.
template <class K>
static int cluster_grid(K* kernel, size_t smem, long long want, int* grid) {
  const long long want_cl = std::max(1LL, (want + CL - 1) / CL);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(want_cl * CL));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  int ncl = 0;
  CK(cudaOccupancyMaxActiveClusters(&ncl, kernel, &cfg));
  if (ncl < 1) return note_cuda(cudaErrorInvalidConfiguration, __LINE__);
  *grid = (int)(CL * std::min<long long>(want_cl, ncl));
  return GMRES_OK;
}

template <int P>
static int configure(Plan& pl) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  constexpr int VEC = Tr<P>::VEC;
  // The attributes are per kernel, shared by every plan: set them for the largest restart
  // length so that a plan with a smaller m never lowers them under another plan.
  const size_t sm_attr = SellSmem<P>::bytes(LSQ_MAX + 2);
  const size_t sm_max = SellSmem<P>::bytes(pl.m + 2);
  CK(cudaFuncSetAttribute(k_spmv_sell<P, double, false>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_attr));
  CK(cudaFuncSetAttribute(k_spmv_sell<P, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sm_attr));
  CK(cudaFuncSetAttribute(k_spmv_sell<P, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sm_attr));
  CK(cudaFuncSetAttribute(k_spmv_sell<P, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sm_attr));
  CK(cudaFuncSetAttribute(k_spmv_sell<P, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sm_attr));
  const size_t sm_u1 = sizeof(W) * (size_t)(pl.m + 1) * (1 + NWARP);
  CK(cudaFuncSetAttribute(k_cgs_u1<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)(sizeof(W) * (size_t)(LSQ_MAX + 1) * (1 + NWARP))));
  CK(cudaFuncSetAttribute(k_cgs_u1_tma<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)TMA_SMEM_BUDGET));
  CK(cudaFuncSetAttribute(k_cgs_u2_tma<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)TMA_SMEM_BUDGET));
  CK(cudaFuncSetAttribute(k_lsq, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)(sizeof(double) * LSQ_PACKED_MAX * (LSQ_PACKED_MAX + 1) / 2)));
  pl.grid_elem = pl.sms * 8;
  // At most two CTAs per SM, each with an equal contiguous share of the rows (the kernels
  // split the work with cta_begin): no second wave.  The step kernels run in clusters of
  // CL CTAs, so their grids are multiples of CL and hold no more clusters than the GPU
  // keeps resident at once (GPCs whose SM count is not a multiple of the cluster's leave a
  // few SMs out).
  const long long nwt = (pl.n + SellSmem<P>::WT - 1) / SellSmem<P>::WT;
  int e = cluster_grid(k_spmv_sell<P, W, false>, sm_max, std::min(nwt, 2LL * pl.sms), &pl.grid_spmv);
  if (e) return e;
  const long long nchunks = pl.ld / VEC / 32;  // 32-group chunks (one warp's worth)
  return cluster_grid(k_cgs_u1<P>, sm_u1, std::min(nchunks, 2LL * pl.sms), &pl.grid_vec);
}

static int configure_residual(Plan& pl) {
  int occ = 1;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_residual<false>, NT, 0));
  const long long ntiles = (pl.n + RES_TR - 1) / RES_TR;
  pl.grid_res = (int)std::max(1LL, std::min(ntiles, (long long)std::min(std::max(occ, 1), 2) * pl.sms));
  return GMRES_OK;
}

// Calls f with the Tr index kp (a plan's kernel set) as a compile-time constant.
template <class F>
static int dispatch(int kp, F&& f) {
  switch (kp) {
    case GMRES_FP64: return f(std::integral_constant<int, 0>{});
    case GMRES_FP32: return f(std::integral_constant<int, 1>{});
    case GMRES_FP16: return f(std::integral_constant<int, 2>{});
    case GMRES_BF16: return f(std::integral_constant<int, 3>{});
    case KP_FP64_NARROW: return f(std::integral_constant<int, KP_FP64_NARROW>{});
  }
  return GMRES_ERR_INVALID;
}

// Kernel set of an FP64 plan with n rows on `sms` SMs.  The four-row step kernels pay off
// once the FP64 work fills the GPU: below FP64_WIDE_ROWS_PER_SM rows per SM their grid
// leaves SMs idle or thin (each CTA owns whole 32-thread groups of rows), and the two-row
// kernels, on twice as many threads, finish a step sooner.
constexpr long long FP64_WIDE_ROWS_PER_SM = 1024;
static int fp64_kernel_set(long long n, int sms) {
  return n >= FP64_WIDE_ROWS_PER_SM * (long long)std::max(sms, 1) ? GMRES_FP64 : KP_FP64_NARROW;
}

static size_t storage_bytes(int prec) { return prec == 0 ? 8 : prec == 1 ? 4 : 2; }
static size_t work_bytes(int prec) { return prec == 0 ? 8 : 4; }

static void plan_free(Plan* pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  if (pl->ev0) cudaEventDestroy(pl->ev0);
  if (pl->ev1) cudaEventDestroy(pl->ev1);
  cudaFree(pl->sell_meta);
  cudaFree(pl->sell_cols);
  cudaFree(pl->sell_vals);
  cudaFree(pl->V);
  cudaFree(pl->w1);
  cudaFree(pl->w2);
  cudaFree(pl->w3);
  cudaFree(pl->r);
  cudaFree(pl->xb);
  cudaFree(pl->bb);
  cudaFree(pl->part);
  cudaFree(pl->pa);
  cudaFree(pl->sell_vals32);
  cudaFree(pl->sell_vals64);
  cudaFree(pl->pb);
  cudaFree(pl->pt);
  cudaFree(pl->py);
  cudaFree(pl->bj_lu);
  cudaFree(pl->bj_rowp);
  cudaFree(pl->perm);
  cudaFree(pl->pA_rp);
  cudaFree(pl->pA_ci);
  cudaFree(pl->pA_v);
  cudaFree(pl->st);
  cudaFree(pl->arr_mem);
  if (pl->h_st) cudaFreeHost(pl->h_st);
  delete pl;
}

static int validate_csr(const gmres_csr* A) {
  if (!A || A->n < 0 || A->nnz < 0) return GMRES_ERR_INVALID;
  if (A->n > 0 && (!A->row_ptr || !A->vals || (A->nnz > 0 && !A->col_idx))) return GMRES_ERR_INVALID;
  return GMRES_OK;
}

static int validate_params(const gmres_params* p) {
  if (!p) return GMRES_ERR_INVALID;
  if (p->restart_m < 1) return GMRES_ERR_INVALID;
  if (p->restart_m > GMRES_MAX_RESTART) return GMRES_ERR_TOO_LARGE;
  if (!(p->rtol >= 0.0) || !(p->inner_rtol >= 0.0) || p->max_iters < 0) return GMRES_ERR_INVALID;
  if (p->inner_prec < 0 || p->inner_prec > 3) return GMRES_ERR_INVALID;
  if (p->poly_degree < 0) return GMRES_ERR_INVALID;
  if (p->poly_degree > GMRES_MAX_POLY_DEGREE) return GMRES_ERR_TOO_LARGE;
  if (p->cgs_kernel != GMRES_CGS_REGISTER && p->cgs_kernel != GMRES_CGS_TMA) return GMRES_ERR_INVALID;
  if (p->bj_block < 0) return GMRES_ERR_INVALID;
  if (p->bj_block > GMRES_MAX_BJ_BLOCK) return GMRES_ERR_TOO_LARGE;
  if (p->bj_block > 0 && p->poly_degree > 0) return GMRES_ERR_INVALID;  // one preconditioner
  if (p->max_outer < 0) return GMRES_ERR_INVALID;
  if (p->tma_wait_cycles < 0) return GMRES_ERR_INVALID;
  return GMRES_OK;
}

// Reverse Cuthill-McKee reordering at plan creation (host, rcm_host.h): the plan keeps the
// reordered CSR P A P^T (columns ascending in each row, stable for equal columns) and the
// permutation, and solves (P A P^T)(P x) = P b.
static int rcm_reorder_impl(Plan& pl, const gmres_csr* A, cudaStream_t s) {
  const int n = A->n, nnz = A->nnz;
  std::vector<int32_t> rp((size_t)n + 1), ci((size_t)nnz), perm((size_t)n), iperm((size_t)n);
  std::vector<double> va((size_t)nnz);
  CK(cudaMemcpyAsync(rp.data(), A->row_ptr, 4 * rp.size(), cudaMemcpyDeviceToHost, s));
  if (nnz) {
    CK(cudaMemcpyAsync(ci.data(), A->col_idx, 4 * ci.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(va.data(), A->vals, 8 * va.size(), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  rcm_order(n, rp.data(), ci.data(), perm.data());
  for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
  std::vector<int32_t> prp((size_t)n + 1, 0), pci((size_t)nnz);
  std::vector<double> pva((size_t)nnz);
  std::vector<std::pair<int32_t, int32_t>> row;  // (new column, position in the old row)
  for (int i = 0; i < n; ++i) {
    const int o = perm[i];
    row.clear();
    for (int32_t q = rp[o]; q < rp[o + 1]; ++q) row.emplace_back(iperm[ci[q]], q - rp[o]);
    std::stable_sort(row.begin(), row.end(),
                     [](const std::pair<int32_t, int32_t>& a, const std::pair<int32_t, int32_t>& b) {
                       return a.first < b.first;
                     });
    prp[i + 1] = prp[i] + (int32_t)row.size();
    for (size_t t = 0; t < row.size(); ++t) {
      pci[prp[i] + t] = row[t].first;
      pva[prp[i] + t] = va[rp[o] + row[t].second];
    }
  }
  CK(cudaMalloc((void**)&pl.pA_rp, 4 * prp.size()));
  CK(cudaMalloc((void**)&pl.pA_ci, 4 * std::max<size_t>(pci.size(), 1)));
  CK(cudaMalloc((void**)&pl.pA_v, 8 * std::max<size_t>(pva.size(), 1)));
  CK(cudaMalloc((void**)&pl.perm, 4 * std::max<size_t>(perm.size(), 1)));
  CK(cudaMemcpyAsync(pl.pA_rp, prp.data(), 4 * prp.size(), cudaMemcpyHostToDevice, s));
  if (nnz) {
    CK(cudaMemcpyAsync(pl.pA_ci, pci.data(), 4 * pci.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pl.pA_v, pva.data(), 8 * pva.size(), cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(pl.perm, perm.data(), 4 * perm.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the host vectors go out of scope
  pl.A = gmres_csr{n, nnz, pl.pA_rp, pl.pA_ci, pl.pA_v};
  return GMRES_OK;
}

static int rcm_reorder(Plan& pl, const gmres_csr* A, cudaStream_t s) {
  try {
    return rcm_reorder_impl(pl, A, s);
  } catch (const std::bad_alloc&) {  // host arrays of the reordering
    cudaStreamSynchronize(s);
    return GMRES_ERR_OOM;
  }
}

// Device check of the CSR structure (once per plan).
static int check_csr_device(const gmres_csr* A, cudaStream_t s) {
  int* d_bad = nullptr;
  CK(cudaMallocAsync((void**)&d_bad, sizeof(int), s));
  CK(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
  k_check_csr<<<256, 256, 0, s>>>(A->row_ptr, A->col_idx, A->n, A->nnz, d_bad);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaFreeAsync(d_bad, s));
  CK(cudaStreamSynchronize(s));
  return bad ? GMRES_ERR_INVALID : GMRES_OK;
}

int plan_create(Plan** out, const gmres_csr* A, int kind, const gmres_params* p, cudaStream_t s) {
  *out = nullptr;
  if (int e = validate_csr(A)) return e;
  if (int e = validate_params(p)) return e;
  if (kind < 0 || kind > 2) return GMRES_ERR_INVALID;
  if (kind == 2 && (p->poly_degree != 0 || p->bj_block != 0 || p->bj_rcm != 0))
    return GMRES_ERR_INVALID;  // FP32 GMRES: no preconditioner, no reordering
  if (A->n == 0) return GMRES_ERR_INVALID;  // an empty system has no plan (solves return OK)
  Plan* pl = new (std::nothrow) Plan();
  if (!pl) return GMRES_ERR_OOM;
  auto fail = [&](int e) {
    cudaStreamSynchronize(s);
    plan_free(pl);
    return e;
  };
  pl->kind = kind;
  pl->prec = kind == 0 ? GMRES_FP64 : kind == 2 ? GMRES_FP32 : p->inner_prec;
  pl->A = *A;
  pl->n = A->n;
  pl->m = p->restart_m;
  pl->p = *p;
  pl->ld = round_up(std::max(A->n, 1), TILE_MAX);
  int dev = 0;
  if (int e_ = CUDA_STATUS(cudaGetDevice(&dev))) return fail(e_);
  cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, dev);
  pl->kp = pl->prec == GMRES_FP64 ? fp64_kernel_set(pl->n, pl->sms) : pl->prec;
  if (int e = check_csr_device(A, s)) return fail(e);
  if (p->bj_rcm) {  // from here on the plan works on its reordered copy, pl->A
    auto tr0 = std::chrono::steady_clock::now();
    if (int e = rcm_reorder(*pl, A, s)) return fail(e);
    pl->t_setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tr0).count();
  }
  A = &pl->A;

  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, s);
  const size_t sb = storage_bytes(pl->prec), wb = work_bytes(pl->prec);
  const long long ld = pl->ld, m = pl->m;
  auto alloc = [&](void** ptr, size_t bytes) -> int {
    if (int e_ = CUDA_STATUS(cudaMalloc(ptr, std::max<size_t>(bytes, 16)))) return e_;
    if (int e_ = CUDA_STATUS(cudaMemsetAsync(*ptr, 0, std::max<size_t>(bytes, 16), s))) return e_;
    return GMRES_OK;
  };
  int e = GMRES_OK;
  if ((e = alloc(&pl->V, sb * (size_t)ld * (m + 1)))) return fail(e);
  if ((e = alloc(&pl->w1, wb * (size_t)ld))) return fail(e);
  if ((e = alloc(&pl->w2, wb * (size_t)ld))) return fail(e);
  if ((e = alloc(&pl->w3, wb * (size_t)ld))) return fail(e);
  if ((e = alloc((void**)&pl->r, 8 * (size_t)ld))) return fail(e);
  if ((e = alloc((void**)&pl->xb, 8 * (size_t)ld))) return fail(e);
  if ((e = alloc((void**)&pl->bb, 8 * (size_t)ld))) return fail(e);
  if ((e = alloc((void**)&pl->st, sizeof(DevState)))) return fail(e);
  pl->hist_cap = p->record_history ? (int)std::min<int64_t>(std::max<int64_t>(p->max_iters, 1), 1 << 22) : 1;
  const size_t arr_n = 2 * (m + 2) + 2 * (m + 1) * m + 2 * m + (m + 1) + m + pl->hist_cap;
  if ((e = alloc((void**)&pl->arr_mem, 8 * arr_n))) return fail(e);
  double* q = pl->arr_mem;
  pl->arr.h1 = q; q += m + 2;
  pl->arr.h2 = q; q += m + 2;
  pl->arr.H = q; q += (m + 1) * m;
  pl->arr.R = q; q += (m + 1) * m;
  pl->arr.cs = q; q += m;
  pl->arr.sn = q; q += m;
  pl->arr.gabs = q; q += m + 1;
  pl->arr.y = q; q += m;
  pl->arr.hist = q;
  if (cudaMallocHost((void**)&pl->h_st, sizeof(DevState)) != cudaSuccess) return fail(GMRES_ERR_OOM);

  // Inner copy of A in SELL-32 (slices of 32 rows, column-major, padded to the slice's
  // longest row): values / s_A rounded to the storage type (FP64 plans keep FP64 values).
  if (pl->prec == GMRES_FP16 && A->nnz > 0) {
    unsigned long long* d_mx = nullptr;
    if (int e_ = CUDA_STATUS(cudaMalloc((void**)&d_mx, 8))) return fail(e_);
    cudaMemsetAsync(d_mx, 0, 8, s);
    k_absmax<<<pl->sms * 4, 256, 0, s>>>(A->vals, A->nnz, d_mx);
    unsigned long long bits = 0;
    cudaMemcpyAsync(&bits, d_mx, 8, cudaMemcpyDeviceToHost, s);
    if (int e_ = CUDA_STATUS(cudaStreamSynchronize(s))) { cudaFree(d_mx); return fail(e_); }
    cudaFree(d_mx);
    double mx;
    memcpy(&mx, &bits, 8);
    if (!std::isfinite(mx)) return fail(GMRES_NONFINITE);
    pl->a_scale = mx > 0.0 ? mx : 1.0;
    // basis scale: the largest power of two s with s^2 <= 2n, within a factor sqrt(2) of
    // sqrt(n) (unit vectors' entries held near 1); a power of two, so scaling adds no
    // rounding and the kernels divide by it exactly with a multiplication
    pl->v_scale = std::ldexp(1.0, (63 - __builtin_clzll(2ULL * (unsigned long long)std::max(pl->n, 1))) / 2);
  }
  {
    std::vector<int> hrp((size_t)pl->n + 1);
    if (int e_ = CUDA_STATUS(cudaMemcpyAsync(hrp.data(), A->row_ptr, sizeof(int) * hrp.size(),
                                             cudaMemcpyDeviceToHost, s)))
      return fail(e_);
    if (int e_ = CUDA_STATUS(cudaStreamSynchronize(s))) return fail(e_);
    pl->nslices = (pl->n + 31) / 32;
    std::vector<int2> meta(pl->nslices);
    long long off = 0;
    for (int sl = 0; sl < pl->nslices; ++sl) {
      int w = 0;
      for (int r = sl * 32; r < std::min(pl->n, sl * 32 + 32); ++r) w = std::max(w, hrp[r + 1] - hrp[r]);
      meta[sl] = make_int2((int)off, w);
      off += 32LL * w;
      if (off >= (1LL << 31)) return fail(GMRES_ERR_TOO_LARGE);
    }
    pl->sell_nnz = off;
    if ((e = alloc((void**)&pl->sell_meta, sizeof(int2) * meta.size()))) return fail(e);
    if ((e = alloc((void**)&pl->sell_cols, sizeof(int) * (size_t)std::max(off, 1LL)))) return fail(e);
    if ((e = alloc(&pl->sell_vals, sb * (size_t)std::max(off, 1LL)))) return fail(e);
    if (int e_ = CUDA_STATUS(cudaMemcpyAsync(pl->sell_meta, meta.data(), sizeof(int2) * meta.size(),
                                             cudaMemcpyHostToDevice, s)))
      return fail(e_);
    const int blocks = pl->sms * 8;
    const int* rp = A->row_ptr;
    const int* ci = A->col_idx;
    const double* va = A->vals;
    dispatch(pl->kp, [&](auto PP) {
      using S = typename Tr<decltype(PP)::value>::S;
      k_build_sell<S><<<blocks, 256, 0, s>>>(rp, ci, va, pl->n, pl->sell_meta, pl->nslices,
                                             pl->a_scale, pl->sell_cols, (S*)pl->sell_vals);
      return 0;
    });
    // The FP64 residual reads A in the same SELL layout with its FP64 values (an FP64
    // plan's copy already is that).
    if (pl->prec != GMRES_FP64) {
      if ((e = alloc(&pl->sell_vals64, 8 * (size_t)std::max(off, 1LL)))) return fail(e);
      k_build_sell<double><<<blocks, 256, 0, s>>>(rp, ci, va, pl->n, pl->sell_meta, pl->nslices, 1.0,
                                                  nullptr, (double*)pl->sell_vals64);
    }
    // the meta upload reads `meta` asynchronously: finish before it goes out of scope
    if (int e_ = CUDA_STATUS(cudaStreamSynchronize(s))) return fail(e_);
  }
  if ((e = dispatch(pl->kp, [&](auto P) { return configure<decltype(P)::value>(*pl); }))) return fail(e);
  if ((e = configure_residual(*pl))) return fail(e);
  pl->part_step_off = 8 * (size_t)(2 * pl->grid_res + 2);
  const size_t step_parts_n = 2 * (size_t)(m + 2) * pl->grid_spmv + (size_t)(m + 2) * pl->grid_vec;
  if ((e = alloc(&pl->part, pl->part_step_off + 8 * step_parts_n))) return fail(e);
  cudaEventRecord(t1, s);
  if (int e_ = CUDA_STATUS(cudaStreamSynchronize(s))) return fail(e_);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, t0, t1);
  pl->t_setup_ms += ms;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);

  // Polynomial preconditioner roots (set-up, FP64 Arnoldi on the GPU + host eigenvalues).
  if (p->poly_degree > 0) {
    std::vector<double> re(p->poly_degree + 1), im(p->poly_degree + 1);
    int nr = 0;
    auto tp0 = std::chrono::steady_clock::now();
    e = gmres_poly_roots(A, p->poly_degree, p->seed, nullptr, re.data(), im.data(), &nr, s);
    if (e) return fail(e);
    pl->roots_re.assign(re.begin(), re.begin() + nr);
    pl->roots_im.assign(im.begin(), im.begin() + nr);
    pl->poly = poly_program(pl->roots_re, pl->roots_im);
    pl->poly32 = p->poly_in_fp32 != 0 && pl->prec == GMRES_FP64;
    const size_t pwb = pl->poly32 ? 4 : wb;
    if (pl->poly32) {  // FP32 copy of the SELL values for the polynomial
      if ((e = alloc(&pl->sell_vals32, 4 * (size_t)std::max(pl->sell_nnz, 1LL)))) return fail(e);
      k_build_sell<float><<<pl->sms * 8, 256, 0, s>>>(A->row_ptr, A->col_idx, A->vals, pl->n,
                                                     pl->sell_meta, pl->nslices, 1.0, nullptr,
                                                     (float*)pl->sell_vals32);
      if (int e_ = CUDA_STATUS(cudaGetLastError())) return fail(e_);
    }
    if ((e = alloc(&pl->pa, pwb * (size_t)ld))) return fail(e);
    if ((e = alloc(&pl->pb, pwb * (size_t)ld))) return fail(e);
    if ((e = alloc(&pl->pt, pwb * (size_t)ld))) return fail(e);
    if ((e = alloc(&pl->py, pwb * (size_t)ld))) return fail(e);
    if (int e_ = CUDA_STATUS(cudaStreamSynchronize(s))) return fail(e_);
    pl->t_setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tp0).count();
  }

  // Block-Jacobi preconditioner: the diagonal blocks of A (the reordered copy when bj_rcm)
  // factored once, in FP64, factors kept in the working type.
  if (p->bj_block > 0) {
    pl->bj = p->bj_block;
    auto tb0 = std::chrono::steady_clock::now();
    const long long nblocks = (pl->n + pl->bj - 1) / pl->bj;
    if ((e = alloc(&pl->bj_lu, wb * (size_t)nblocks * pl->bj * pl->bj))) return fail(e);
    if ((e = alloc((void**)&pl->bj_rowp, sizeof(int) * (size_t)pl->n))) return fail(e);
    if ((e = alloc(&pl->pa, wb * (size_t)ld))) return fail(e);
    if ((e = alloc(&pl->py, wb * (size_t)ld))) return fail(e);
    int* d_bad = nullptr;
    if ((e = alloc((void**)&d_bad, sizeof(int)))) return fail(e);
    const int fgrid = (int)std::min<long long>(nblocks, (long long)pl->sms * 16);
    dispatch(pl->kp, [&](auto PP) {
      using W = typename Tr<decltype(PP)::value>::W;
      k_bj_factor<W><<<fgrid, BJ_FACTOR_THREADS, 0, s>>>(A->row_ptr, A->col_idx, A->vals, pl->n,
                                                         pl->bj, (W*)pl->bj_lu, pl->bj_rowp, d_bad);
      return 0;
    });
    int bad = 0;
    cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    const cudaError_t ce = cudaStreamSynchronize(s);
    cudaFree(d_bad);
    if (int e_ = CUDA_STATUS(ce)) return fail(e_);
    if (int e_ = CUDA_STATUS(cudaGetLastError())) return fail(e_);
    if (bad) return fail(GMRES_ERR_INVALID);  // a singular diagonal block
    const long long warps = pl->bj <= 32 ? (nblocks + 32 / pl->bj - 1) / (32 / pl->bj) : nblocks;
    pl->grid_bj = (int)std::max<long long>(
        1, std::min<long long>((warps + BJ_APPLY_WARPS - 1) / BJ_APPLY_WARPS, (long long)pl->sms * 32));
    if (int e_ = CUDA_STATUS(cudaFuncSetAttribute(k_bj_apply<float>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  BJ_APPLY_WARPS * bj_slot(BJ_MAX) * 4)))
      return fail(e_);
    if (int e_ = CUDA_STATUS(cudaFuncSetAttribute(k_bj_apply<double>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  BJ_APPLY_WARPS * bj_slot(BJ_MAX) * 8)))
      return fail(e_);
    pl->t_setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tb0).count();
  }

  // L2 policy of the SpMVs that gather a stored input (after a preconditioner, and the first
  // step of a plain low-precision cycle): block Jacobi and the plain cycle read the matrix once
  // per step, so it is streamed evict-first like the other steps'; the polynomial re-reads
  // it d times per step, which pays while the copy of A and the polynomial's vectors stay in
  // L2 (measured: 100^3, 56 MB FP32 copy, degree 10/25, streaming 17-28% slower; 2000^2,
  // 160 MB FP32 / 120 MB FP16 copy, degree 40, streaming 24% faster).
  {
    int dev = 0, l2 = 0;
    if (int e_ = CUDA_STATUS(cudaGetDevice(&dev))) return fail(e_);
    if (int e_ = CUDA_STATUS(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev))) return fail(e_);
    const double vals = pl->poly32 ? 4.0 : (double)storage_bytes(pl->prec);
    const double work = pl->poly32 ? 4.0 : (double)work_bytes(pl->prec);
    const double bytes = (double)pl->sell_nnz * (4.0 + vals) + 4.0 * work * (double)pl->n;
    pl->stream_matrix = pl->poly.empty() ? 1 : (bytes > 0.75 * (double)l2 ? 1 : 0);
  }

  // Capture one restart cycle as a CUDA graph.
  if (int e_ = CUDA_STATUS(cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking))) return fail(e_);
  if (int e_ = CUDA_STATUS(cudaEventCreate(&pl->ev0))) return fail(e_);
  if (int e_ = CUDA_STATUS(cudaEventCreate(&pl->ev1))) return fail(e_);
  if (int e_ = CUDA_STATUS(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal)))
    return fail(e_);
  dispatch(pl->kp, [&](auto P) {
    launch_cycle<decltype(P)::value>(*pl, pl->cap);
    return 0;
  });
  if (int e_ = CUDA_STATUS(cudaStreamEndCapture(pl->cap, &pl->graph))) return fail(e_);
  if (int e_ = CUDA_STATUS(cudaGraphInstantiate(&pl->exec, pl->graph, 0))) return fail(e_);
  *out = pl;
  return GMRES_OK;
}

static void init_state(Plan& pl, DevState& h) {
  memset(&h, 0, sizeof(h));
  h.m = pl.m;
  h.mode = pl.kind == 1 ? 1 : 0;  // GMRES (FP64 or FP32) ends a cycle at the tolerance
  h.max_iters = pl.p.max_iters;
  h.rtol = pl.p.rtol;
  h.inner_rtol = pl.p.inner_rtol;
  h.u_work = pl.prec == GMRES_FP64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
  h.hist_cap = pl.hist_cap;
  h.sigma = 1.0;
  h.stream_matrix = pl.stream_matrix;
}

// b and x0 into the plan's vectors (through the permutation when the plan is reordered).
static int load_rhs(Plan& pl, const double* b, const double* x0, cudaStream_t s) {
  const size_t nb = sizeof(double) * (size_t)pl.n;
  if (pl.perm) {
    k_gather_perm<<<pl.grid_elem, NT, 0, s>>>(b, pl.perm, pl.n, pl.bb);
    k_gather_perm<<<pl.grid_elem, NT, 0, s>>>(x0, pl.perm, pl.n, pl.xb);
    CK(cudaGetLastError());
  } else {
    CK(cudaMemcpyAsync(pl.bb, b, nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(pl.xb, x0, nb, cudaMemcpyDeviceToDevice, s));
  }
  return GMRES_OK;
}

int plan_solve(Plan& pl, const double* b, double* x, gmres_stats* stats, cudaStream_t s) {
  if (!b || !x) return GMRES_ERR_INVALID;
  const size_t nb = sizeof(double) * (size_t)pl.n;
  init_state(pl, *pl.h_st);
  CK(cudaMemcpyAsync(pl.st, pl.h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  if (int e = load_rhs(pl, b, x, s)) return e;
  CK(cudaEventRecord(pl.ev0, s));
  launch_residual(pl, 1, s);
  CK(cudaGetLastError());
  int* h_stop = &pl.h_st->stop;
  CK(cudaMemcpyAsync(h_stop, &pl.st->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // one cycle (= one refinement step of GMRES-IR, one restart of GMRES) per graph launch;
  // max_outer > 0 caps their number on the host
  long long max_cycles = pl.p.max_iters + 2;
  if (pl.p.max_outer > 0) max_cycles = std::min<long long>(max_cycles, pl.p.max_outer);
  for (long long c = 0; !*h_stop && c < max_cycles; ++c) {
    CK(cudaGraphLaunch(pl.exec, s));
    CK(cudaMemcpyAsync(h_stop, &pl.st->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaEventRecord(pl.ev1, s));
  CK(cudaMemcpyAsync(pl.h_st, pl.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const DevState& h = *pl.h_st;
  // a solve ended by the cycle cap has no decision from the device: not converged
  const int status = h.stop ? h.status : (int)ST_NOT_CONVERGED;
  if (h.zero_rhs) {
    CK(cudaMemsetAsync(x, 0, nb, s));
  } else if (pl.perm) {
    k_scatter_perm<<<pl.grid_elem, NT, 0, s>>>(pl.xb, pl.perm, pl.n, x);
    CK(cudaGetLastError());
  } else {
    CK(cudaMemcpyAsync(x, pl.xb, nb, cudaMemcpyDeviceToDevice, s));
  }
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pl.ev0, pl.ev1);
    stats->status = status;
    stats->iters = h.iters;
    stats->outer_iters = h.outer;
    stats->rel_resid = h.relres;
    stats->t_solve_ms = ms;
    stats->t_setup_ms = pl.t_setup_ms;
    stats->history_len = 0;
    if (stats->history && stats->history_cap > 0 && pl.p.record_history) {
      const long long cnt = std::min<long long>({(long long)h.iters, (long long)pl.hist_cap, stats->history_cap});
      if (cnt > 0)
        CK(cudaMemcpyAsync(stats->history, pl.arr.hist, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
      stats->history_len = cnt;
    }
  }
  CK(cudaStreamSynchronize(s));
  return status;
}

// ---------------------------------------------------------------------------
// Test entry points on a plan.
// ---------------------------------------------------------------------------
int plan_poly_apply(Plan& pl, const double* v, void* y, cudaStream_t s) {
  if (pl.poly.empty() || !v || !y) return GMRES_ERR_INVALID;
  init_state(pl, *pl.h_st);
  CK(cudaMemcpyAsync(pl.st, pl.h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  // the polynomial's precision: the plan's, or FP32 for an FP64 plan with poly_in_fp32
  int e = dispatch(pl.poly32 ? GMRES_FP32 : pl.kp, [&](auto PP) {
    constexpr int P = decltype(PP)::value;
    using W = typename Tr<P>::W;
    k_load_work<P><<<pl.grid_elem, NT, 0, s>>>(v, (W*)pl.pa, pl.n);
    launch_poly<P>(pl, 0, s);
    return (int)cudaMemcpyAsync(y, pl.py, sizeof(W) * (size_t)pl.n, cudaMemcpyDeviceToDevice, s);
  });
  if (e) return note_cuda((cudaError_t)e, __LINE__);
  CK(cudaStreamSynchronize(s));
  return GMRES_OK;
}

// y = M^{-1} v with the plan's block-Jacobi factors (v: n doubles, y: n values of the
// working type, both in the plan's numbering).  Asynchronous on s (two kernels).
int plan_bj_apply(Plan& pl, const double* v, void* y, cudaStream_t s) {
  if (!pl.bj || !v || !y) return GMRES_ERR_INVALID;
  int e = dispatch(pl.kp, [&](auto PP) {
    constexpr int P = decltype(PP)::value;
    using W = typename Tr<P>::W;
    k_load_work<P><<<pl.grid_elem, NT, 0, s>>>(v, (W*)pl.pa, pl.n);
    k_bj_apply<W><<<pl.grid_bj, 32 * BJ_APPLY_WARPS, bj_smem<W>(pl), s>>>((const W*)pl.bj_lu, pl.bj_rowp, pl.n, pl.bj,
                                             (const W*)pl.pa, (W*)y, nullptr, 0);
    return (int)cudaGetLastError();
  });
  if (e) return note_cuda((cudaError_t)e, __LINE__);
  return GMRES_OK;
}

int plan_spmv(Plan& pl, const double* v, void* y, cudaStream_t s) {
  init_state(pl, *pl.h_st);
  CK(cudaMemcpyAsync(pl.st, pl.h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  int e = dispatch(pl.kp, [&](auto PP) {
    constexpr int P = decltype(PP)::value;
    using S = typename Tr<P>::S;
    using W = typename Tr<P>::W;
    k_spmv_sell<P, double, false><<<pl.grid_spmv, NT, SellSmem<P>::bytes(2), s>>>(
        pl.sell_meta, pl.sell_cols, (const S*)pl.sell_vals, pl.nslices, pl.n, pl.ld,
        pl.a_scale / pl.v_scale, v,
        pl.v_scale, (S*)pl.V, 0, (W*)pl.w1, step_parts<P>(pl), pl.st, pl.arr);
    return (int)cudaMemcpyAsync(y, pl.w1, sizeof(W) * (size_t)pl.n, cudaMemcpyDeviceToDevice, s);
  });
  if (e) return note_cuda((cudaError_t)e, __LINE__);
  CK(cudaStreamSynchronize(s));
  return GMRES_OK;
}

int plan_arnoldi(Plan& pl, const double* v0, int steps, void* V_out, double* H_out, int* k_out,
                 cudaStream_t s) {
  if (steps < 1 || steps > pl.m || !v0 || !H_out || !k_out) return GMRES_ERR_INVALID;
  init_state(pl, *pl.h_st);
  pl.h_st->mode = 1;
  pl.h_st->rtol = 0.0;
  pl.h_st->inner_rtol = 0.0;
  pl.h_st->max_iters = 1LL << 62;
  const size_t nb = sizeof(double) * (size_t)pl.n;
  CK(cudaMemcpyAsync(pl.st, pl.h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(pl.bb, v0, nb, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(pl.xb, 0, nb, s));
  launch_residual(pl, 1, s);  // r = v0, sigma = 1/||v0||, |g_0| = 1
  int e = dispatch(pl.kp, [&](auto PP) {
    constexpr int P = decltype(PP)::value;
    using S = typename Tr<P>::S;
    using W = typename Tr<P>::W;
    for (int j = 0; j < steps; ++j) launch_step<P>(pl, j, s);
    k_finalize<P><<<1, NT, 0, s>>>(step_parts<P>(pl), pl.st, pl.arr);
    k_store_basis<P, W><<<pl.sms * 4, 256, 0, s>>>((const W*)pl.w3, pl.v_scale, pl.n, (S*)pl.V, pl.ld,
                                                   steps, pl.st);
    return (int)cudaGetLastError();
  });
  if (e) return note_cuda((cudaError_t)e, __LINE__);
  CK(cudaMemcpyAsync(pl.h_st, pl.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int k = pl.h_st->k;
  *k_out = k;
  const size_t sb = storage_bytes(pl.prec);
  if (V_out)
    CK(cudaMemcpy2DAsync(V_out, sb * pl.n, pl.V, sb * pl.ld, sb * pl.n, steps + 1, cudaMemcpyDeviceToDevice, s));
  std::vector<double> Hfull((size_t)(pl.m + 1) * pl.m);
  CK(cudaMemcpyAsync(Hfull.data(), pl.arr.H, sizeof(double) * Hfull.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int c = 0; c < steps; ++c)
    for (int i = 0; i <= steps; ++i)
      H_out[i + (size_t)c * (steps + 1)] = (c < k && i <= c + 1) ? Hfull[i + (size_t)c * (pl.m + 1)] : 0.0;
  if (pl.h_st->status == ST_TIMEOUT) return GMRES_ERR_DEVICE_TIMEOUT;
  return pl.h_st->status == ST_NONFINITE ? GMRES_NONFINITE : GMRES_OK;
}

// One restart cycle launched kernel by kernel (not through the graph), each launch
// bracketed by CUDA events on `s`.  ms_out[3j + {0,1,2}] = the three kernels of step j,
// ms_out[3m + {0,1,2}] = least squares / x update / residual; -1 for the steps that the
// cycle did not reach.  The host reads the cycle flag after every step.
int plan_profile_cycle(Plan& pl, const double* b, const double* x0, double* ms_out, cudaStream_t s) {
  const int m = pl.m, nslots = 3 * m + 3;
  init_state(pl, *pl.h_st);
  CK(cudaMemcpyAsync(pl.st, pl.h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  if (int e = load_rhs(pl, b, x0, s)) return e;
  launch_residual(pl, 1, s);
  std::vector<cudaEvent_t> ev(2 * (size_t)nslots, nullptr);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  std::vector<int> ran(nslots, 0);
  int* h_flag = &pl.h_st->cycle_done;
  int err = dispatch(pl.kp, [&](auto PP) -> int {
    constexpr int P = decltype(PP)::value;
    for (int j = 0; j < m; ++j) {
      for (int w = 0; w < 3; ++w) {
        const int sl = 3 * j + w;
        cudaEventRecord(ev[2 * sl], s);
        launch_step_kernel<P>(pl, j, w, s);
        cudaEventRecord(ev[2 * sl + 1], s);
        ran[sl] = 1;
      }
      cudaMemcpyAsync(h_flag, &pl.st->cycle_done, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (int e_ = CUDA_STATUS(cudaStreamSynchronize(s))) return e_;
      if (*h_flag) break;
    }
    for (int w = 0; w < 3; ++w) {
      const int sl = 3 * m + w;
      cudaEventRecord(ev[2 * sl], s);
      launch_tail_kernel<P>(pl, w, s);
      cudaEventRecord(ev[2 * sl + 1], s);
      ran[sl] = 1;
    }
    return cudaGetLastError() == cudaSuccess ? GMRES_OK : GMRES_ERR_CUDA;
  });
  if (err == GMRES_OK && cudaStreamSynchronize(s) != cudaSuccess) err = GMRES_ERR_CUDA;
  for (int i = 0; i < nslots; ++i) {
    float ms = -1.f;
    if (err == GMRES_OK && ran[i]) cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
    ms_out[i] = ran[i] ? (double)ms : -1.0;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return err;
}

// The same cycle as the plan's graph, captured with an event-record node before every
// kernel and after the last (cudaEventRecordExternal), and launched once: ms_out[i] is the
// time between the events around kernel i as it runs inside a graph, the way a solve runs
// it (layout as plan_profile_cycle; -1 for the steps the cycle did not reach, whose kernels
// returned at once).  Costs one graph instantiation per call.
// per_kernel == false: the same graph with only the first and the last event node, so no
// event sits between two kernels; ms_out[0] = the whole cycle (residual of the next cycle
// included), ms_out[1] = the Arnoldi steps it took.
int plan_profile_cycle_graph(Plan& pl, const double* b, const double* x0, double* ms_out,
                             cudaStream_t s, bool per_kernel = true) {
  const int m = pl.m, nslots = 3 * m + 3;
  init_state(pl, *pl.h_st);
  CK(cudaMemcpyAsync(pl.st, pl.h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  if (int e = load_rhs(pl, b, x0, s)) return e;
  launch_residual(pl, 1, s);
  CK(cudaStreamSynchronize(s));
  std::vector<cudaEvent_t> ev((size_t)nslots + 1, nullptr);
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int err = GMRES_OK;
  auto done = [&](int e) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    for (auto& x : ev)
      if (x) cudaEventDestroy(x);
    return e;
  };
  for (auto& x : ev)
    if ((err = CUDA_STATUS(cudaEventCreate(&x)))) return done(err);
  if ((err = CUDA_STATUS(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)))) return done(err);
  if ((err = CUDA_STATUS(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal))))
    return done(err);
  dispatch(pl.kp, [&](auto PP) -> int {
    constexpr int P = decltype(PP)::value;
    for (int j = 0; j < m; ++j)
      for (int w = 0; w < 3; ++w) {
        if (per_kernel || j + w == 0) cudaEventRecordWithFlags(ev[3 * j + w], cs, cudaEventRecordExternal);
        launch_step_kernel<P>(pl, j, w, cs);
      }
    for (int w = 0; w < 3; ++w) {
      if (per_kernel) cudaEventRecordWithFlags(ev[3 * m + w], cs, cudaEventRecordExternal);
      launch_tail_kernel<P>(pl, w, cs);
    }
    cudaEventRecordWithFlags(ev[nslots], cs, cudaEventRecordExternal);
    return 0;
  });
  if ((err = CUDA_STATUS(cudaStreamEndCapture(cs, &graph)))) return done(err);
  if ((err = CUDA_STATUS(cudaGraphInstantiate(&exec, graph, 0)))) return done(err);
  // upload the graph before the timed launch, so that its first launch does not include it
  if ((err = CUDA_STATUS(cudaGraphUpload(exec, s)))) return done(err);
  if ((err = CUDA_STATUS(cudaStreamSynchronize(s)))) return done(err);
  if ((err = CUDA_STATUS(cudaGraphLaunch(exec, s)))) return done(err);
  if ((err = CUDA_STATUS(cudaMemcpyAsync(pl.h_st, pl.st, sizeof(DevState), cudaMemcpyDeviceToHost, s))))
    return done(err);
  if ((err = CUDA_STATUS(cudaStreamSynchronize(s)))) return done(err);
  // Arnoldi steps the cycle took (the solve's step count starts at zero in init_state;
  // st->k is already reset for the next cycle by the residual kernel)
  const long long steps = pl.h_st->iters;
  if (!per_kernel) {
    float ms = -1.f;
    if ((err = CUDA_STATUS(cudaEventElapsedTime(&ms, ev[0], ev[nslots])))) return done(err);
    ms_out[0] = ms;
    ms_out[1] = (double)steps;
    return done(GMRES_OK);
  }
  for (int i = 0; i < nslots; ++i) {
    const bool ran = i >= 3 * m || i / 3 < steps;
    float ms = -1.f;
    if (ran && cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      ms = -1.f;
    }
    ms_out[i] = ran ? (double)ms : -1.0;
  }
  return done(GMRES_OK);
}

}  // namespace gm

using gm::Plan;

struct gmres_plan_s {
  Plan* pl;
};

extern "C" {

void gmres_default_params(gmres_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->restart_m = 50;
  p->rtol = 1e-10;
  p->inner_rtol = 0.0;
  p->max_iters = 100000;
  p->inner_prec = GMRES_FP32;
  p->poly_degree = 0;
  p->seed = 0;
  p->record_history = 0;
}

const char* gmres_last_error(void) { return gm::g_last_error; }

const char* gmres_status_string(int status) {
  switch (status) {
    case GMRES_OK: return "converged";
    case GMRES_NOT_CONVERGED: return "maximum iterations reached";
    case GMRES_BREAKDOWN: return "breakdown: singular least-squares factor";
    case GMRES_NONFINITE: return "non-finite value in the input or a reduction";
    case GMRES_ERR_INVALID: return "invalid argument";
    case GMRES_ERR_OOM: return "device allocation failed";
    case GMRES_ERR_CUDA: return "CUDA runtime error";
    case GMRES_ERR_TOO_LARGE: return "size exceeds a documented maximum";
    case GMRES_ERR_DEVICE_TIMEOUT: return "a device-side bounded wait expired";
  }
  return "unknown status";
}

int gmres_plan_create(gmres_plan* plan, const gmres_csr* A, int32_t kind, const gmres_params* p,
                      void* stream) {
  if (!plan) return GMRES_ERR_INVALID;
  *plan = nullptr;
  Plan* pl = nullptr;
  int e = gm::plan_create(&pl, A, kind, p, (cudaStream_t)stream);
  if (e) return e;
  auto* h = new (std::nothrow) gmres_plan_s{pl};
  if (!h) {
    gm::plan_free(pl);
    return GMRES_ERR_OOM;
  }
  *plan = h;
  return GMRES_OK;
}

int gmres_plan_set_tolerances(gmres_plan plan, double rtol, double inner_rtol, int64_t max_iters) {
  if (!plan || !(rtol >= 0.0) || !(inner_rtol >= 0.0) || max_iters < 0) return GMRES_ERR_INVALID;
  gm::Plan* pl = plan->pl;
  pl->p.rtol = rtol;
  pl->p.inner_rtol = inner_rtol;
  pl->p.max_iters = max_iters;
  return GMRES_OK;
}

int gmres_plan_spmv_timed(gmres_plan plan, const void* x, void* y, int32_t reps, float* ms_out,
                          void* stream) {
  if (!plan || !x || !y || reps < 1 || !ms_out) return GMRES_ERR_INVALID;
  gm::Plan& pl = *plan->pl;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = pl.grid_spmv;
  auto launch = [&](auto PP) {
    constexpr int P = decltype(PP)::value;
    using S = typename gm::Tr<P>::S;
    using W = typename gm::Tr<P>::W;
    gm::k_spmv_plain<P><<<grid, gm::NT, 0, s>>>(pl.sell_meta, pl.sell_cols, (const S*)pl.sell_vals,
                                                pl.nslices, pl.n, pl.a_scale, (const W*)x, (W*)y);
    return 0;
  };
  gm::dispatch(pl.kp, launch);  // warm-up
  CK(cudaGetLastError());
  CK(cudaEventRecord(pl.ev0, s));
  for (int r = 0; r < reps; ++r) gm::dispatch(pl.kp, launch);
  CK(cudaEventRecord(pl.ev1, s));
  CK(cudaGetLastError());
  CK(cudaEventSynchronize(pl.ev1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, pl.ev0, pl.ev1));
  *ms_out = ms / (float)reps;
  return GMRES_OK;
}

int gmres_plan_destroy(gmres_plan plan) {
  if (!plan) return GMRES_ERR_INVALID;
  cudaDeviceSynchronize();
  gm::plan_free(plan->pl);
  delete plan;
  return GMRES_OK;
}

int gmres_plan_solve(gmres_plan plan, const double* b, double* x, gmres_stats* stats, void* stream) {
  if (!plan) return GMRES_ERR_INVALID;
  return gm::plan_solve(*plan->pl, b, x, stats, (cudaStream_t)stream);
}

int gmres_plan_spmv(gmres_plan plan, const double* v, void* y, void* stream) {
  if (!plan || !v || !y) return GMRES_ERR_INVALID;
  return gm::plan_spmv(*plan->pl, v, y, (cudaStream_t)stream);
}

int gmres_plan_arnoldi(gmres_plan plan, const double* v0, int32_t steps, void* V_out, double* H_out,
                       int32_t* k_out, void* stream) {
  if (!plan) return GMRES_ERR_INVALID;
  return gm::plan_arnoldi(*plan->pl, v0, steps, V_out, H_out, k_out, (cudaStream_t)stream);
}

int gmres_plan_profile_cycle(gmres_plan plan, const double* b, const double* x0, double* ms_out,
                             void* stream) {
  if (!plan || !b || !x0 || !ms_out) return GMRES_ERR_INVALID;
  return gm::plan_profile_cycle(*plan->pl, b, x0, ms_out, (cudaStream_t)stream);
}

int gmres_plan_profile_cycle_graph(gmres_plan plan, const double* b, const double* x0,
                                   double* ms_out, void* stream) {
  if (!plan || !b || !x0 || !ms_out) return GMRES_ERR_INVALID;
  return gm::plan_profile_cycle_graph(*plan->pl, b, x0, ms_out, (cudaStream_t)stream);
}

int gmres_plan_time_cycle_graph(gmres_plan plan, const double* b, const double* x0,
                                double* ms_out, void* stream) {
  if (!plan || !b || !x0 || !ms_out) return GMRES_ERR_INVALID;
  return gm::plan_profile_cycle_graph(*plan->pl, b, x0, ms_out, (cudaStream_t)stream, false);
}

int gmres_plan_poly_apply(gmres_plan plan, const double* v, void* y, void* stream) {
  if (!plan) return GMRES_ERR_INVALID;
  return gm::plan_poly_apply(*plan->pl, v, y, (cudaStream_t)stream);
}

int gmres_plan_bj_apply(gmres_plan plan, const double* v, void* y, void* stream) {
  if (!plan) return GMRES_ERR_INVALID;
  return gm::plan_bj_apply(*plan->pl, v, y, (cudaStream_t)stream);
}

int gmres_plan_perm(gmres_plan plan, int32_t* perm, int32_t* reordered) {
  if (!plan || !reordered) return GMRES_ERR_INVALID;
  const Plan& pl = *plan->pl;
  *reordered = pl.perm != nullptr;
  if (pl.perm && perm) {
    CK(cudaMemcpy(perm, pl.perm, sizeof(int32_t) * (size_t)pl.n, cudaMemcpyDeviceToHost));
  }
  return GMRES_OK;
}

int gmres_rcm(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* perm) {
  if (n < 0 || (n > 0 && (!row_ptr || !col_idx || !perm))) return GMRES_ERR_INVALID;
  if (n == 0) return GMRES_OK;
  if (row_ptr[0] != 0) return GMRES_ERR_INVALID;
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return GMRES_ERR_INVALID;
  for (int32_t q = 0; q < row_ptr[n]; ++q)
    if (col_idx[q] < 0 || col_idx[q] >= n) return GMRES_ERR_INVALID;
  try {
    gm::rcm_order(n, row_ptr, col_idx, perm);
  } catch (const std::bad_alloc&) {
    return GMRES_ERR_OOM;
  }
  return GMRES_OK;
}

int gmres_plan_poly_roots(gmres_plan plan, double* roots_re, double* roots_im, int32_t* nroots) {
  if (!plan || !nroots) return GMRES_ERR_INVALID;
  const Plan& pl = *plan->pl;
  *nroots = (int32_t)pl.roots_re.size();
  for (size_t i = 0; i < pl.roots_re.size(); ++i) {
    if (roots_re) roots_re[i] = pl.roots_re[i];
    if (roots_im) roots_im[i] = pl.roots_im[i];
  }
  return GMRES_OK;
}

int gmres_plan_info(gmres_plan plan, int64_t* info_out) {
  if (!plan || !info_out) return GMRES_ERR_INVALID;
  const Plan& pl = *plan->pl;
  const int64_t v[8] = {pl.n, pl.A.nnz, pl.ld, pl.m, pl.prec, pl.grid_spmv, pl.grid_vec, pl.grid_res};
  for (int i = 0; i < 8; ++i) info_out[i] = v[i];
  return GMRES_OK;
}

static int solve_once(const gmres_csr* A, const double* b, double* x, const gmres_params* p, int kind,
                      gmres_stats* stats, void* stream) {
  if (int e = gm::validate_csr(A)) return e;
  if (int e = gm::validate_params(p)) return e;
  if (!b || !x) return GMRES_ERR_INVALID;
  if (A->n == 0) {
    if (stats) {  // an empty system is solved by the empty vector
      stats->status = GMRES_OK;
      stats->iters = 0;
      stats->outer_iters = 0;
      stats->rel_resid = 0.0;
      stats->t_solve_ms = stats->t_setup_ms = 0.0;
      stats->history_len = 0;
    }
    return GMRES_OK;
  }
  Plan* pl = nullptr;
  int e = gm::plan_create(&pl, A, kind, p, (cudaStream_t)stream);
  if (e) {
    if (stats) stats->status = e;
    return e;
  }
  e = gm::plan_solve(*pl, b, x, stats, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  gm::plan_free(pl);
  return e;
}

int gmres_solve(const gmres_csr* A, const double* b, double* x, const gmres_params* p,
                gmres_stats* stats, void* stream) {
  return solve_once(A, b, x, p, 0, stats, stream);
}

int gmres_ir_solve(const gmres_csr* A, const double* b, double* x, const gmres_params* p,
                   gmres_stats* stats, void* stream) {
  return solve_once(A, b, x, p, 1, stats, stream);
}

int gmres_fd_solve(const gmres_csr* A, const double* b, double* x, const gmres_params* p,
                   int64_t switch_iters, gmres_stats* stats_fp32, gmres_stats* stats_fp64,
                   void* stream) {
  if (int e = gm::validate_params(p)) return e;
  if (switch_iters < 0 || p->poly_degree != 0 || p->bj_block != 0 || p->bj_rcm != 0)
    return GMRES_ERR_INVALID;
  // the switch happens at a restart: round up to whole cycles of the FP32 stage
  const int64_t m = p->restart_m;
  gmres_params q = *p;
  q.max_iters = std::min<int64_t>(p->max_iters, (switch_iters + m - 1) / m * m);
  int e = GMRES_OK;
  int64_t used = 0;
  if (q.max_iters > 0) {
    e = solve_once(A, b, x, &q, 2, stats_fp32, stream);
    if (e != GMRES_OK && e != GMRES_NOT_CONVERGED && e != GMRES_BREAKDOWN) return e;
    if (stats_fp32) used = stats_fp32->iters;
    else used = q.max_iters;
  } else if (stats_fp32) {
    memset(stats_fp32, 0, sizeof(*stats_fp32));
  }
  q = *p;
  q.max_iters = std::max<int64_t>(0, p->max_iters - used);
  return solve_once(A, b, x, &q, 0, stats_fp64, stream);
}

static int solve_host(const gmres_csr* Ah, const double* b, double* x, const gmres_params* p, int kind,
                      gmres_stats* stats, void* stream) {
  if (int e = gm::validate_csr(Ah)) return e;
  if (!b || !x) return GMRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)Ah->n, nnz = (size_t)Ah->nnz;
  if (n == 0) return solve_once(Ah, b, x, p, kind, stats, stream);
  int32_t *rp = nullptr, *ci = nullptr;
  double *va = nullptr, *bd = nullptr, *xd = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    cudaFree(rp); cudaFree(ci); cudaFree(va); cudaFree(bd); cudaFree(xd);
  };
  if (cudaMalloc((void**)&rp, 4 * (n + 1)) != cudaSuccess || cudaMalloc((void**)&ci, 4 * std::max<size_t>(nnz, 1)) != cudaSuccess ||
      cudaMalloc((void**)&va, 8 * std::max<size_t>(nnz, 1)) != cudaSuccess || cudaMalloc((void**)&bd, 8 * n) != cudaSuccess ||
      cudaMalloc((void**)&xd, 8 * n) != cudaSuccess) {
    cleanup();
    return GMRES_ERR_OOM;
  }
  cudaMemcpyAsync(rp, Ah->row_ptr, 4 * (n + 1), cudaMemcpyHostToDevice, s);
  if (nnz) {
    cudaMemcpyAsync(ci, Ah->col_idx, 4 * nnz, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(va, Ah->vals, 8 * nnz, cudaMemcpyHostToDevice, s);
  }
  cudaMemcpyAsync(bd, b, 8 * n, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(xd, x, 8 * n, cudaMemcpyHostToDevice, s);
  gmres_csr Ad{Ah->n, Ah->nnz, rp, ci, va};
  int e = solve_once(&Ad, bd, xd, p, kind, stats, stream);
  if (e == GMRES_OK || e == GMRES_NOT_CONVERGED || e == GMRES_BREAKDOWN)
    cudaMemcpyAsync(x, xd, 8 * n, cudaMemcpyDeviceToHost, s);
  cleanup();
  return e;
}

int gmres_ir_solve_host(const gmres_csr* A, const double* b, double* x, const gmres_params* p,
                        gmres_stats* stats, void* stream) {
  return solve_host(A, b, x, p, 1, stats, stream);
}

int gmres_solve_host(const gmres_csr* A, const double* b, double* x, const gmres_params* p,
                     gmres_stats* stats, void* stream) {
  return solve_host(A, b, x, p, 0, stats, stream);
}

int gmres_poly_roots(const gmres_csr* A, int32_t degree, uint64_t seed, const double* v0,
                     double* roots_re, double* roots_im, int32_t* nroots, void* stream) {
  if (int e = gm::validate_csr(A)) return e;
  if (!roots_re || !roots_im || !nroots || degree < 1 || A->n < 1) return GMRES_ERR_INVALID;
  if (degree > GMRES_MAX_POLY_DEGREE) return GMRES_ERR_TOO_LARGE;
  cudaStream_t s = (cudaStream_t)stream;
  gmres_params p;
  gmres_default_params(&p);
  p.restart_m = degree + 1;
  Plan* pl = nullptr;
  int e = gm::plan_create(&pl, A, 0, &p, s);
  if (e) return e;
  double* vtmp = nullptr;
  const double* start = v0;
  if (!start) {
    if (cudaMalloc((void**)&vtmp, sizeof(double) * (size_t)A->n) != cudaSuccess) {
      gm::plan_free(pl);
      return GMRES_ERR_OOM;
    }
    gm::k_splitmix64<<<592, 256, 0, s>>>(vtmp, A->n, seed);
    start = vtmp;
  }
  const int steps = degree + 1;
  std::vector<double> H((size_t)(steps + 1) * steps);
  int k = 0;
  e = gm::plan_arnoldi(*pl, start, steps, nullptr, H.data(), &k, s);
  cudaStreamSynchronize(s);
  if (vtmp) cudaFree(vtmp);
  gm::plan_free(pl);
  if (e) return e;
  if (k < 1) return GMRES_BREAKDOWN;
  std::vector<double> Hk((size_t)(k + 1) * k);
  for (int c = 0; c < k; ++c)
    for (int i = 0; i <= k; ++i) Hk[i + (size_t)c * (k + 1)] = H[i + (size_t)c * (steps + 1)];
  std::vector<double> wr, wi;
  if (!gm::harmonic_ritz_values(Hk.data(), k, wr, wi)) return GMRES_BREAKDOWN;
  gm::leja_order(wr, wi);
  for (size_t i = 0; i < wr.size(); ++i) {
    roots_re[i] = wr[i];
    roots_im[i] = wi[i];
  }
  *nroots = (int32_t)wr.size();
  return GMRES_OK;
}

int gmres_splitmix64_fill(double* out, int64_t n, uint64_t seed, void* stream) {
  if (!out || n < 0) return GMRES_ERR_INVALID;
  if (n == 0) return GMRES_OK;
  gm::k_splitmix64<<<592, 256, 0, (cudaStream_t)stream>>>(out, n, seed);
  if (cudaGetLastError() != cudaSuccess) return GMRES_ERR_CUDA;
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? GMRES_OK : GMRES_ERR_CUDA;
}

}  // extern "C"

// ===========================================================================
// FP64 SpMV that allocates nothing.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by another
// allocator that reserved the GPU up front, latency-critical loops that cannot afford
// the implicit device synchronisation of cudaMalloc/cudaFree, and plug-ins that are not
// allowed to allocate at all.  gmres_spmv_fp64_noalloc runs the CSR SpMV kernel
// (k_spmv_arnoldi with only its product, no basis store or dot products) and keeps its
// scratch -- the device state whose stop flag the CSR check sets and the kernel reads,
// and a staging copy of v for calls whose y overlaps v -- in the file-scope array below.
// Every GPU that loads this library holds that array until the process exits.
// ===========================================================================
namespace gm {
namespace {

constexpr int kNoAllocGrid = 1184;  // CTAs per launch at most (8 per SM on 148 SMs)
constexpr long long kNoAllocRows =
    ((long long)GMRES_NOALLOC_MAX_N + TILE_MAX - 1) / TILE_MAX * TILE_MAX;

struct NoAllocHead {
  DevState st;  // st.stop: nonzero when the CSR check found a malformed structure
};
constexpr size_t kNoAllocHeadBytes = (sizeof(NoAllocHead) + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kNoAllocHeadBytes + sizeof(double) * (size_t)kNoAllocRows;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Clears the state (the stop flag above all), so a call never sees the last call's flags.
__global__ void k_noalloc_reset(DevState* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *st = DevState{};
    st->sigma = 1.0;
  }
}

__global__ void k_copy_f64(const double* __restrict__ src, double* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// Device address of the scratch array on the current device and its SM count.  Looked up
// on every call (cudaGetSymbolAddress, with the caller's device current), so a context
// that was destroyed and re-created (cudaDeviceReset) never leaves a stale address.
int noalloc_scratch(void** out, int* sms) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return GMRES_ERR_CUDA;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return GMRES_ERR_CUDA;
  }
  int count = 0;
  if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return GMRES_ERR_CUDA;
  }
  *out = p;
  *sms = count > 0 ? count : 1;
  return GMRES_OK;
}

}  // namespace
}  // namespace gm

extern "C" int gmres_spmv_fp64_noalloc(const gmres_csr* A, const double* v, double* y,
                                       void* stream) {
  if (!A || A->n < 0 || A->nnz < 0 || !v || !y) return GMRES_ERR_INVALID;
  if (A->n > GMRES_NOALLOC_MAX_N) return GMRES_ERR_TOO_LARGE;
  if (A->n == 0) return GMRES_OK;
  if (!A->row_ptr || !A->vals || (A->nnz > 0 && !A->col_idx)) return GMRES_ERR_INVALID;
  void* base = nullptr;
  int sms = 1;
  if (int e = gm::noalloc_scratch(&base, &sms)) return e;
  cudaStream_t s = (cudaStream_t)stream;
  auto* head = reinterpret_cast<gm::NoAllocHead*>(base);
  double* stage = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + gm::kNoAllocHeadBytes);
  const int n = A->n;
  gm::k_noalloc_reset<<<1, 1, 0, s>>>(&head->st);
  // a malformed structure sets st.stop, and the SpMV kernel then returns before any load
  gm::k_check_csr<<<256, 256, 0, s>>>(A->row_ptr, A->col_idx, n, A->nnz, &head->st.stop);
  const double* src = v;
  const uintptr_t vb = (uintptr_t)v, yb = (uintptr_t)y, bytes = sizeof(double) * (uintptr_t)n;
  if (vb < yb + bytes && yb < vb + bytes) {  // y overlaps v: multiply a staged copy of v
    const int cgrid = std::max(1, std::min((n + 255) / 256, sms * 8));
    gm::k_copy_f64<<<cgrid, 256, 0, s>>>(v, stage, n);
    src = stage;
  }
  constexpr int TR = gm::SpmvSmem<0>::TR;
  const int ntiles = (n + TR - 1) / TR;
  const int grid = std::max(1, std::min({ntiles, sms * 8, gm::kNoAllocGrid}));
  gm::k_spmv_arnoldi<0, double, true, true><<<grid, gm::NT, gm::SpmvSmem<0>::bytes(2), s>>>(
      A->row_ptr, A->col_idx, A->vals, n, gm::kNoAllocRows, 1.0, src, 1.0, nullptr, 0, y,
      nullptr, &head->st, nullptr);
  if (cudaGetLastError() != cudaSuccess) return GMRES_ERR_CUDA;
  int bad = 0;
  if (cudaMemcpyAsync(&bad, &head->st.stop, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return GMRES_ERR_CUDA;
  }
  return bad ? GMRES_ERR_INVALID : GMRES_OK;
}

// Batched GMRES-IR (many small systems, one persistent kernel).
#include "batched.cuh"

// Learned parameter selector (features, MLP inference and training kernels).
#include "selector.cuh"
