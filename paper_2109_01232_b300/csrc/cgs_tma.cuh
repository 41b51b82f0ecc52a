// cgs_tma.cuh -- the two CGS update kernels fed by TMA bulk copies (sm_103a).
//
// The basis V is streamed through shared memory.  One producer warp issues cp.async.bulk
// copies (global -> shared, completion counted on an mbarrier) of every basis column's
// chunk of a row block, plus the block of w, into a ring of stages; eight consumer warps
// compute from shared memory and hand each stage back through a second mbarrier.  A
// CTA's copies are in flight independently of its registers, so HBM sees many requests
// at once, and the second pass over V of the first update (the dot products with the
// updated vector) reads shared memory instead of L2.  The producer starts copying while
// the consumers are still reducing the previous kernel's partial sums.
//
//   k_cgs_u1_tma(j): w' = w - V_j h1 (thread per row), then partials of V_j^T w' (warp
//                    per column, lanes over rows, one register accumulator per column);
//   k_cgs_u2_tma(j): w'' = w' - V_j h2 and partials of ||w''||^2.
// Prologues and partial-sum outputs are those of k_cgs_u1 / k_cgs_u2 (kernels.cuh), and
// both run on the same grid, so either form can produce any step's partials.
//
// Every mbarrier wait is bounded (TmaWait::cycles SM clocks, TMA_WAIT_CYCLES by default,
// and an iteration cap).  If one expires the kernel records ST_TIMEOUT and stops the
// solve; the other warps stop waiting as soon as they see the error, the producer waits
// for the copies it issued (bounded by TMA_WAIT_CYCLES whatever the first bound), and the
// CTA returns without writing partial sums.  TmaWait::withhold (a test hook) makes the
// producer issue only its first row block's copies, so the consumers' wait for the second
// block can only end by the bound: the timeout path runs with no fault and no hang.
#pragma once

#include "kernels.cuh"

namespace gm {

constexpr int TMA_CW = 8;                    // consumer warps
constexpr int TMA_RB = TMA_CW * 32;          // rows per block: one consumer thread per row
constexpr int TMA_THREADS = TMA_RB + 32;     // + one producer warp
constexpr int TMA_MAX_STAGES = 32;
constexpr int TMA_U1_ACC = 8;                // u1: register accumulators per lane
constexpr int TMA_U1_MAX_COLS = TMA_U1_ACC * TMA_CW;
constexpr size_t TMA_SMEM_BUDGET = 108 * 1024;  // two CTAs per SM
constexpr long long TMA_WAIT_CYCLES = 1LL << 31;  // about a second at the B300's SM clocks
constexpr long long TMA_SPIN_LIMIT = 1LL << 28;

struct TmaWait {
  long long cycles;  // bound of the producer's and consumers' waits
  bool withhold;     // test hook: copies of the first row block only
};

// Shared-memory layout of both kernels for a step with nc basis columns.
template <int P>
struct TmaLayout {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  static constexpr size_t chunk = (size_t)TMA_RB * sizeof(S);   // one column of a block
  static constexpr size_t wchunk = (size_t)TMA_RB * sizeof(W);  // the block of w
  __host__ __device__ static size_t stage(int nc) { return (size_t)nc * chunk + wchunk; }
  // after the stages: the updated block of w (u1) and the coefficients
  __host__ __device__ static size_t extra(int nc) {
    return wchunk + ((sizeof(W) * (size_t)nc + 15) & ~(size_t)15);
  }
  // stages that fit the budget; 0 when fewer than two fit (use the register kernels)
  __host__ __device__ static int stages(int nc) {
    if (extra(nc) >= TMA_SMEM_BUDGET) return 0;
    const size_t s = (TMA_SMEM_BUDGET - extra(nc)) / stage(nc);
    return s < 2 ? 0 : (s > (size_t)TMA_MAX_STAGES ? TMA_MAX_STAGES : (int)s);
  }
  __host__ __device__ static size_t bytes(int nc, int ns) { return (size_t)ns * stage(nc) + extra(nc); }
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the completion of the phase of parity `parity`.  Gives up (false) when
// `cycles` SM clocks or the iteration limit have passed, or when *abort becomes non-zero
// (abort may be null).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          const int* abort, long long cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (long long i = 1; i < TMA_SPIN_LIMIT; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 0) {
      if (abort && *(volatile const int*)abort) return false;
      if (clock64() - t0 > cycles) return false;
    }
  }
  return false;
}
// cp.async.bulk global -> shared; both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Named barrier 1 among the consumer warps (the producer warp never takes part).
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(TMA_RB) : "memory");
}

struct TmaCtl {
  unsigned long long full[TMA_MAX_STAGES];   // stage filled (1 arrival + the copies' bytes)
  unsigned long long empty[TMA_MAX_STAGES];  // stage released (one arrival per consumer warp)
  int skip, err;
};

// Producer side of the ring over this CTA's row blocks [b0, b1) (the producer warp; lane 0
// issues).  Stage s of fill k holds the block's nc basis chunks and then its chunk of w.
// Returns after the copies it issued have landed (bounded wait).
template <int P>
__device__ __forceinline__ void tma_produce(const typename Tr<P>::S* __restrict__ V, long long ld,
                                            int nc, const typename Tr<P>::W* __restrict__ win,
                                            unsigned char* stages, int ns, TmaCtl& ctl,
                                            long long b0, long long b1, TmaWait tw) {
  using L = TmaLayout<P>;
  if ((threadIdx.x & 31) == 0) {
    const size_t stage_bytes = L::stage(nc);
    long long issued = 0;
    const long long nblk = tw.withhold ? (b1 - b0 < 1 ? b1 - b0 : 1) : b1 - b0;
    for (long long k = 0; k < nblk; ++k) {
      if (*(volatile int*)&ctl.err) break;
      const int s = (int)(k % ns);
      const unsigned it = (unsigned)(k / ns);
      if (k >= ns && !mbar_wait(&ctl.empty[s], (it - 1) & 1u, &ctl.err, tw.cycles)) {
        *(volatile int*)&ctl.err = 1;
        break;
      }
      unsigned char* st = stages + (size_t)s * stage_bytes;
      const long long row0 = (b0 + k) * TMA_RB;
      mbar_arrive_expect_tx(&ctl.full[s], (unsigned)stage_bytes);
      for (int c = 0; c < nc; ++c)
        bulk_g2s(st + (size_t)c * L::chunk, V + (long long)c * ld + row0, (unsigned)L::chunk,
                 &ctl.full[s]);
      bulk_g2s(st + (size_t)nc * L::chunk, win + row0, (unsigned)L::wchunk, &ctl.full[s]);
      issued = k + 1;
    }
    // the copies into the last stages must land before the CTA exits
    for (long long k = issued > ns ? issued - ns : 0; k < issued; ++k)
      mbar_wait(&ctl.full[k % ns], (unsigned)(k / ns) & 1u, nullptr, TMA_WAIT_CYCLES);
  }
  __syncwarp();
}

// Consumer side: waits for fill k of its stage.  Returns whether the stage may be used;
// false once any wait of the CTA has failed (the result is the same on all lanes).  Every
// consumer thread still runs the loop body for every block, so named barriers in it match.
__device__ __forceinline__ bool tma_acquire(TmaCtl& ctl, long long k, int ns, bool valid,
                                            long long cycles) {
  bool ok = valid && mbar_wait(&ctl.full[k % ns], (unsigned)(k / ns) & 1u, &ctl.err, cycles);
  ok = __all_sync(0xffffffffu, ok);
  if (!ok && valid && (threadIdx.x & 31) == 0) *(volatile int*)&ctl.err = 1;
  return ok;
}
// Consumer side: this warp is done with fill k of its stage.
__device__ __forceinline__ void tma_release(TmaCtl& ctl, long long k, int ns, bool valid) {
  __syncwarp();
  if (valid && (threadIdx.x & 31) == 0) mbar_arrive(&ctl.empty[k % ns]);
}

// Prologue: skip test and mbarrier set-up (thread 0), then the consumer warps reduce the
// partials into the update coefficients while the producer warp goes ahead.  Returns
// false when the kernel has nothing to do.
template <int P>
__device__ __forceinline__ bool tma_prologue(DevState* st, const typename Tr<P>::W* part, int nc,
                                             int G, double v_scale, typename Tr<P>::W* coef,
                                             double* h, TmaCtl& ctl, int ns) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    ctl.skip = read_flag(&st->stop) | read_flag(&st->cycle_done);
    ctl.err = 0;
    for (int s = 0; s < ns; ++s) {
      mbar_init(&ctl.full[s], 1);
      mbar_init(&ctl.empty[s], TMA_CW);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (ctl.skip) return false;
  if (tid < TMA_RB) {
    const bool writer = blockIdx.x == 0;
    block_reduce_columns<TMA_CW>(part, nc, G, [&](int c, typename Tr<P>::W v) {
      const double hc = (double)v * pow2_recip(v_scale);
      coef[c] = (typename Tr<P>::W)(hc * pow2_recip(v_scale));
      if (writer) h[c] = hc;
    });
    consumers_sync();
  }
  return true;
}

template <int P>
__global__ void __launch_bounds__(TMA_THREADS, 2) k_cgs_u1_tma(
    const typename Tr<P>::S* __restrict__ V, long long ld, int j, double v_scale,
    const typename Tr<P>::W* __restrict__ win, typename Tr<P>::W* __restrict__ wout,
    StepParts<typename Tr<P>::W> parts, DevState* st, double* __restrict__ h1, int ns,
    TmaWait tw) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  using L = TmaLayout<P>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TmaCtl ctl;
  const int nc = j + 1;
  unsigned char* stages = smem_raw;
  W* wsh = reinterpret_cast<W*>(smem_raw + (size_t)ns * L::stage(nc));
  W* coef = wsh + TMA_RB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (!tma_prologue<P>(st, parts.p1_of(j), nc, parts.g1, v_scale, coef, h1, ctl, ns)) return;
  const long long nb = ld / TMA_RB;
  const long long b0 = cta_begin(nb, 1), b1 = cta_begin(nb, 1, 1);
  W dot[TMA_U1_ACC];
#pragma unroll
  for (int q = 0; q < TMA_U1_ACC; ++q) dot[q] = W(0);
  if (warp == TMA_CW) {
    tma_produce<P>(V, ld, nc, win, stages, ns, ctl, b0, b1, tw);
  } else {
    bool valid = true;
    for (long long k = 0; k < b1 - b0; ++k) {
      valid = tma_acquire(ctl, k, ns, valid, tw.cycles);
      const unsigned char* stg = stages + (size_t)(k % ns) * L::stage(nc);
      const S* Vs = reinterpret_cast<const S*>(stg);
      consumers_sync();  // every warp is done with the previous block's wsh
      if (valid) {
        W w = reinterpret_cast<const W*>(stg + (size_t)nc * L::chunk)[tid];
        for (int c = 0; c < nc; ++c) w -= coef[c] * to_w(Vs[(size_t)c * TMA_RB + tid]);
        wout[(b0 + k) * TMA_RB + tid] = w;
        wsh[tid] = w;
      }
      consumers_sync();
      if (valid) {
        W wr[TMA_RB / 32];
#pragma unroll
        for (int i = 0; i < TMA_RB / 32; ++i) wr[i] = wsh[lane + 32 * i];
#pragma unroll
        for (int q = 0; q < TMA_U1_ACC; ++q) {
          const int c = warp + TMA_CW * q;
          if (c < nc) {
            const S* vc = Vs + (size_t)c * TMA_RB;
            W d = W(0);
#pragma unroll
            for (int i = 0; i < TMA_RB / 32; ++i) d += to_w(vc[lane + 32 * i]) * wr[i];
            dot[q] += d;
          }
        }
      }
      tma_release(ctl, k, ns, valid);
    }
  }
  __syncthreads();
  if (ctl.err) {
    if (tid == 0) {
      st->status = ST_TIMEOUT;
      st->stop = 1;
    }
    return;
  }
  if (tid < TMA_RB) {
    const int G = gridDim.x;
#pragma unroll
    for (int q = 0; q < TMA_U1_ACC; ++q) {
      const int c = warp + TMA_CW * q;
      const W d = warp_sum(dot[q]);
      if (c < nc && lane == 0) parts.p2[(long long)c * G + blockIdx.x] = d;
    }
  }
}

template <int P>
__global__ void __launch_bounds__(TMA_THREADS, 2) k_cgs_u2_tma(
    const typename Tr<P>::S* __restrict__ V, long long ld, int j, double v_scale,
    const typename Tr<P>::W* __restrict__ win, typename Tr<P>::W* __restrict__ wout,
    StepParts<typename Tr<P>::W> parts, DevState* st, double* __restrict__ h2, int ns,
    TmaWait tw) {
  using S = typename Tr<P>::S;
  using W = typename Tr<P>::W;
  using L = TmaLayout<P>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TmaCtl ctl;
  __shared__ W accw[TMA_CW];
  const int nc = j + 1;
  unsigned char* stages = smem_raw;
  W* coef = reinterpret_cast<W*>(smem_raw + (size_t)ns * L::stage(nc) + L::wchunk);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (!tma_prologue<P>(st, parts.p2, nc, parts.g2, v_scale, coef, h2, ctl, ns)) return;
  const long long nb = ld / TMA_RB;
  const long long b0 = cta_begin(nb, 1), b1 = cta_begin(nb, 1, 1);
  W nrm = W(0);
  if (warp == TMA_CW) {
    tma_produce<P>(V, ld, nc, win, stages, ns, ctl, b0, b1, tw);
  } else {
    bool valid = true;
    for (long long k = 0; k < b1 - b0; ++k) {
      valid = tma_acquire(ctl, k, ns, valid, tw.cycles);
      if (valid) {
        const unsigned char* stg = stages + (size_t)(k % ns) * L::stage(nc);
        const S* Vs = reinterpret_cast<const S*>(stg);
        W w = reinterpret_cast<const W*>(stg + (size_t)nc * L::chunk)[tid];
        for (int c = 0; c < nc; ++c) w -= coef[c] * to_w(Vs[(size_t)c * TMA_RB + tid]);
        wout[(b0 + k) * TMA_RB + tid] = w;
        nrm += w * w;
      }
      tma_release(ctl, k, ns, valid);
    }
  }
  if (tid < TMA_RB) {
    nrm = warp_sum(nrm);
    if (lane == 0) accw[warp] = nrm;
  }
  __syncthreads();
  if (ctl.err) {
    if (tid == 0) {
      st->status = ST_TIMEOUT;
      st->stop = 1;
    }
    return;
  }
  if (tid == 0) {
    W s = W(0);
    for (int w = 0; w < TMA_CW; ++w) s += accw[w];
    parts.p3[blockIdx.x] = s;
    if (blockIdx.x == 0) st->last_step = j;
  }
}

}  // namespace gm
