// kf_step_staged.cuh -- persistent single-step kernel with bulk-async staging
// (paper section 2: propagateToZ / propagateToR + KalmanUpdate per track).
//
// The direct kernel (kf_step.cu) loads each track's 36 input floats with
// scalar loads and then computes; a warp has nothing in flight while it
// computes, so HBM idles unless many other warps happen to be loading.  Here
// a persistent CTA splits the two jobs:
//
//   * one producer warp streams tiles of T = 256 tracks into shared memory
//     with cp.async.bulk (the Blackwell bulk-copy engine), S stages deep
//     (3 with two CTAs per SM, 2 with three), each completion tracked by an
//     mbarrier's transaction count;
//   * eight compute warps take a staged tile, read their track's inputs from
//     shared memory (bank-conflict-free for AoSoA), release the stage, and run
//     the step in registers, writing results straight to global memory.
//
// For AoSoA layouts a tile of an array is one contiguous run (T is a multiple
// of the block width W), so a stage is four bulk copies.  charge and the
// per-track surface are plain [n] arrays read directly (tiny, and a bulk copy
// of a ragged tail could run past their end).  Every mbarrier wait is
// bounded; on timeout the kernel records KF_DEVERR_TIMEOUT in a device error
// word and leaves its loop, so a broken pipeline cannot hang the GPU; the
// producer waits (bounded) for its last copies to land before it exits.
// Launches use programmatic dependent launch: the next kernel on the stream
// is scheduled while this one drains and waits for it on the GPU.
//
// The kernel template and its launch helpers live here; the instantiations
// are spread over kf_staged_{p2z,p2r}_{f32,f64}.cu so that they compile in
// parallel, and kf_step_staged.cu dispatches to them.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "kf_common.cuh"
#include "kf_device.cuh"
#include "kf_step.cuh"

namespace kf {

namespace staged {

constexpr int kComputeWarps = 8;
constexpr int kThreads = (kComputeWarps + 1) * 32;
constexpr int kT = kComputeWarps * 32;  // tracks per tile
constexpr int kStateB = kT * 6 * 4;
constexpr int kCovB = kT * 21 * 4;
constexpr int kHitB = kT * 3 * 4;
constexpr int kHcB = kT * 6 * 4;
constexpr int kStageB = kStateB + kCovB + kHitB + kHcB;
// Pipeline depth per CTA for a given number of resident CTAs per SM: the
// SM's shared memory holds six stages, as 3 stages x 2 CTAs or 2 x 3 (the
// latter with more compute warps per SM, at <= 72 registers a thread).
constexpr int stages_for(int ctas) { return ctas >= 3 ? 2 : 3; }
constexpr int smem_bytes(int ctas) { return stages_for(ctas) * (kStageB + 16); }
// Polls of a barrier before giving up (with back-off, several seconds).
constexpr uint32_t kMaxPolls = 1u << 24;

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  uint64_t state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(saddr(bar)), "r"(bytes)
               : "memory");
  (void)state;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  uint64_t state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];"
               : "=l"(state)
               : "r"(saddr(bar))
               : "memory");
  (void)state;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete, polling at most
// `limit` times (with back-off); false when it gives up.  A wait that runs
// out ORs KF_DEVERR_TIMEOUT into the library's device error word and, when
// the CTA has an abort flag, raises it; a wait given an abort flag also
// gives up (without a second error bit) as soon as another warp of the CTA
// has raised it, so one warp's timeout ends the whole CTA's pipeline in
// microseconds instead of every warp polling to its own limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err,
                                          uint32_t limit = kMaxPolls,
                                          volatile int *abort = nullptr) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort && *abort) return false;
    if (it > 32) __nanosleep(128);
  }
  if (err) atomicOr(err, (unsigned)KF_DEVERR_TIMEOUT);
  if (abort) *abort = 1;
  return false;
}

// Global -> shared bulk copy completing on `bar` (sizes and addresses are
// multiples of 16 bytes).
__device__ __forceinline__ void bulk_g2s(void *sdst, const void *gsrc, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(sdst)),
      "l"(gsrc), "r"(bytes), "r"(saddr(bar))
      : "memory");
}

// Prefetch [gsrc, gsrc + bytes) into L2 (16-byte aligned, multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void *gsrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}

// Tile schedule of the persistent grid (G CTAs).  Full tiles of kT tracks go
// round-robin (tile k of CTA b is global tile k G + b), so at any moment the
// grid works on one narrow window of the arrays.  What is left after the
// last complete round (fewer than G + 1 tiles' worth) is cut into G equal
// pieces of whole AoSoA blocks, at most kT tracks each, so that the final
// round keeps every CTA busy instead of a third of them.
struct Schedule {
  int64_t R;     // complete rounds of full tiles
  int64_t base;  // first track of the remainder
  int64_t per;   // tracks per remainder piece (multiple of W, <= kT)
  int64_t P;     // remainder pieces
  int64_t G;

  __device__ __forceinline__ int64_t tiles_of(int64_t b) const {
    return R + (b < P ? (P - 1 - b) / G + 1 : 0);
  }
  __device__ __forceinline__ void tile(int64_t k, int64_t b, int64_t n, int64_t *first,
                                       int64_t *m) const {
    if (k < R) {
      *first = (k * G + b) * kT;
      *m = kT;
    } else {
      *first = base + (b + (k - R) * G) * per;
      *m = (n - *first < per) ? n - *first : per;
    }
  }
};

template <int W>
__device__ __forceinline__ Schedule make_schedule(int64_t n, int64_t G) {
  Schedule s;
  s.G = G;
  s.R = (n / kT) / G;
  s.base = s.R * G * kT;
  const int64_t rem = n - s.base;
  if (rem == 0) {
    s.per = kT;
    s.P = 0;
  } else {
    const int64_t share = ((rem + G - 1) / G + W - 1) / W * W;
    s.per = share < kT ? share : kT;
    s.P = (rem + s.per - 1) / s.per;
  }
  return s;
}

// W is the AoSoA block width, or 0 for SoA: then every component of a tile
// is its own contiguous run [c][first, first + m) (n a multiple of 4, so runs
// start and end on 16-byte boundaries) and a stage holds one row of kT floats
// per component.
template <int KIND, int VARIANT, int W, int CTAS>
__global__ void __launch_bounds__(kThreads, CTAS)
    step_staged_kernel(const __grid_constant__ StepArgs a) {
  constexpr bool kSoa = W == 0;
  constexpr int SW = kSoa ? kT : W;  // shared-memory row length of a block
  constexpr int GR = kSoa ? 4 : W;   // tile boundaries are multiples of GR
  static_assert(kT % SW == 0, "tile must hold whole AoSoA blocks");
  constexpr int kStages = stages_for(CTAS);
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageB);
  uint64_t *empty = full + kStages;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const Schedule sch = make_schedule<GR>(a.n, gridDim.x);
  const int64_t ntiles = sch.tiles_of(blockIdx.x);
  // Raised when a warp of this CTA gives up a bounded wait: the compute
  // warps stop, and the producer stops issuing copies and drains the ones
  // in flight before the CTA exits.
  __shared__ int abort_flag;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kComputeWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  // Programmatic dependent launch: let the next kernel on the stream be
  // scheduled now (its CTAs take SMs as ours retire and set up their
  // barriers), and wait here until the previous kernel has completed and its
  // writes are visible -- nothing global is read or written before this
  // point.  Meanwhile the producer asks L2 for this CTA's first tiles, so
  // that a CTA that lands on an SM while the previous kernel drains starts
  // from L2 instead of HBM.  A prefetch only moves lines into L2, the point
  // where every SM's loads and stores meet, so it cannot return a value the
  // previous kernel has yet to write: the copies after the wait read
  // whatever is current.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (warp == kComputeWarps && lane == 0) {
    const int64_t npre = ntiles < kStages ? ntiles : kStages;
    for (int64_t k = 0; k < npre; ++k) {
      int64_t first, m;
      sch.tile(k, blockIdx.x, a.n, &first, &m);
      const uint32_t cols = (uint32_t)(((m + GR - 1) / GR) * GR);
      if constexpr (kSoa) {
        for (int c = 0; c < 6; ++c) bulk_prefetch_l2(a.state_in + c * a.n + first, cols * 4);
        for (int e = 0; e < 21; ++e) bulk_prefetch_l2(a.cov_in + e * a.n + first, cols * 4);
      } else {
        bulk_prefetch_l2(a.state_in + first * 6, cols * 6 * 4);
        bulk_prefetch_l2(a.cov_in + first * 21, cols * 21 * 4);
        bulk_prefetch_l2(a.hit + first * 3, cols * 3 * 4);
        bulk_prefetch_l2(a.hitcov + first * 6, cols * 6 * 4);
      }
    }
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");

  if (warp == kComputeWarps) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t k = 0; k < ntiles; ++k) {
        const int s = (int)(k % kStages);
        const uint32_t ph = (uint32_t)(k / kStages) & 1u;
        if (k >= kStages && !mbar_wait(&empty[s], ph ^ 1u, a.err, kMaxPolls, &abort_flag)) break;
        int64_t first, m;
        sch.tile(k, blockIdx.x, a.n, &first, &m);
        const uint32_t cols = (uint32_t)(((m + GR - 1) / GR) * GR);  // whole blocks
        unsigned char *st = smem + s * kStageB;
        if constexpr (kSoa) {
          // one copy per component row; p2z skips hit z and hit cov rows 3-5
          constexpr int nh = KIND == kP2r ? 3 : 2, nhc = KIND == kP2r ? 6 : 3;
          const uint32_t bytes = cols * 4;
          mbar_arrive_expect_tx(&full[s], bytes * (6 + 21 + nh + nhc));
          for (int c = 0; c < 6; ++c)
            bulk_g2s(st + c * kT * 4, a.state_in + c * a.n + first, bytes, &full[s]);
          for (int e = 0; e < 21; ++e)
            bulk_g2s(st + kStateB + e * kT * 4, a.cov_in + e * a.n + first, bytes, &full[s]);
          for (int c = 0; c < nh; ++c)
            bulk_g2s(st + kStateB + kCovB + c * kT * 4, a.hit + c * a.n + first, bytes, &full[s]);
          for (int c = 0; c < nhc; ++c)
            bulk_g2s(st + kStateB + kCovB + kHitB + c * kT * 4, a.hitcov + c * a.n + first, bytes,
                     &full[s]);
        } else if (KIND == kP2r) {
          mbar_arrive_expect_tx(&full[s], cols * (6 + 21 + 3 + 6) * 4);
          bulk_g2s(st, a.state_in + first * 6, cols * 6 * 4, &full[s]);
          bulk_g2s(st + kStateB, a.cov_in + first * 21, cols * 21 * 4, &full[s]);
          bulk_g2s(st + kStateB + kCovB, a.hit + first * 3, cols * 3 * 4, &full[s]);
          bulk_g2s(st + kStateB + kCovB + kHitB, a.hitcov + first * 6, cols * 6 * 4, &full[s]);
        } else {
          // p2z measures x, y only: per AoSoA block, copy hit rows x, y and
          // hit-covariance rows xx, xy, yy (237 instead of 253 B per track)
          const uint32_t nb = cols / W;
          mbar_arrive_expect_tx(&full[s], cols * (6 + 21 + 2 + 3) * 4);
          bulk_g2s(st, a.state_in + first * 6, cols * 6 * 4, &full[s]);
          bulk_g2s(st + kStateB, a.cov_in + first * 21, cols * 21 * 4, &full[s]);
          for (uint32_t b = 0; b < nb; ++b) {
            bulk_g2s(st + kStateB + kCovB + b * 3 * W * 4, a.hit + (first + b * W) * 3,
                     2 * W * 4, &full[s]);
            bulk_g2s(st + kStateB + kCovB + kHitB + b * 6 * W * 4, a.hitcov + (first + b * W) * 6,
                     3 * W * 4, &full[s]);
          }
        }
        issued = k + 1;
      }
      // No copy may still be writing this CTA's shared memory when it exits
      // (the compute warps have normally consumed them all already; after an
      // abort they have not, and these waits, at the full limit and deaf to
      // the abort flag, let the copies land).
      for (int64_t k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
        if (!mbar_wait(&full[k % kStages], (uint32_t)(k / kStages) & 1u, a.err)) break;
    }
    return;
  }

  // --------------------------------------------------------------- compute
  const int il = warp * 32 + lane;          // track within the tile
  const int blk = il / SW, r = il % SW;     // block and slot within the tile
  // charge and the per-track surface are plain [n] arrays, read directly;
  // each tile's values are requested one tile ahead so that their latency
  // hides behind the previous tile's step.
  auto fetch = [&](int64_t k, float &q, float &sf) {
    int64_t f, mm;
    sch.tile(k, blockIdx.x, a.n, &f, &mm);
    const bool lv = il < mm;
    q = lv ? (float)__ldg(a.charge + f + il) : 1.0f;
    sf = __ldg(a.surf + ((a.surf_per_track && lv) ? f + il : 0));
  };
  float qf_next = 1.0f, surf_next = 0.0f;
  if (ntiles > 0) fetch(0, qf_next, surf_next);
  for (int64_t k = 0; k < ntiles; ++k) {
    const int s = (int)(k % kStages);
    const uint32_t ph = (uint32_t)(k / kStages) & 1u;
    int64_t first, m;
    sch.tile(k, blockIdx.x, a.n, &first, &m);
    const int64_t i = first + il;
    const bool live = il < m;
    const float qf = qf_next, surf = surf_next;
    if (k + 1 < ntiles) fetch(k + 1, qf_next, surf_next);
    if (!mbar_wait(&full[s], ph, a.err, a.wait_polls, &abort_flag)) break;

    const float *sst = reinterpret_cast<const float *>(smem + s * kStageB);
    const float *scv = sst + kT * 6;
    const float *sht = scv + kT * 21;
    const float *shc = sht + kT * 3;
    float p[6], C[21];
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = sst[blk * 6 * SW + c * SW + r];
#pragma unroll
    for (int e = 0; e < 21; ++e) C[e] = scv[blk * 21 * SW + e * SW + r];
    const float hx = sht[blk * 3 * SW + r];
    const float hy = sht[blk * 3 * SW + SW + r];
    float hz = 0.0f, hc[6];
    if (KIND == kP2r) {
      hz = sht[blk * 3 * SW + 2 * SW + r];
#pragma unroll
      for (int c = 0; c < 6; ++c) hc[c] = shc[blk * 6 * SW + c * SW + r];
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) hc[c] = shc[blk * 6 * SW + c * SW + r];
      hc[3] = hc[4] = hc[5] = 0.0f;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // stage may be refilled
    if (!live) continue;

    unsigned st;
    if (KIND == kP2z)
      st = p2z_step<VARIANT>(p, C, qf, a.bz, surf, hx, hy, hc[0], hc[1], hc[2]);
    else
      st = p2r_step<VARIANT>(p, C, qf, a.bz, surf, hx, hy, hz, hc);
    if constexpr (VARIANT == kAdaptive) {
      if (st & kRedo) {  // ill-conditioned in FP32: left to the FP64 redo pass
        a.status[i] = (uint8_t)kRedo;
        continue;
      }
    }
    st |= finite_status(p, C);
    // element (c, i): i + c n (SoA) or block-major i / W, c, i % W (AoSoA)
    const int64_t b6 = kSoa ? i : (i / SW) * (6 * SW) + (i % SW);
    const int64_t b21 = kSoa ? i : (i / SW) * (21 * SW) + (i % SW);
    const int64_t s_out = kSoa ? a.n : SW;
#pragma unroll
    for (int c = 0; c < 6; ++c) __stcs(a.state_out + b6 + c * s_out, p[c]);
#pragma unroll
    for (int e = 0; e < 21; ++e) __stcs(a.cov_out + b21 + e * s_out, C[e]);
    if (a.status) a.status[i] = (uint8_t)st;
  }
}

template <int KIND, int VARIANT, int W, int CTAS>
int launch_w(const StepArgs &a, cudaStream_t s, int grid, int dev) {
  auto kern = step_staged_kernel<KIND, VARIANT, W, CTAS>;
  constexpr int smem = smem_bytes(CTAS);
  static std::atomic<bool> configured[64] = {};  // per instantiation and device
  if (dev < 0 || dev >= 64 || !configured[dev].load(std::memory_order_acquire)) {
    if (int rc = check_cuda(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
            "cudaFuncSetAttribute"))
      return rc;
    if (dev >= 0 && dev < 64) configured[dev].store(true, std::memory_order_release);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return check_cuda(cudaLaunchKernelEx(&cfg, kern, a), "staged step launch");
}

template <int KIND, int VARIANT, int CTAS>
int launch_c(const StepArgs &a, cudaStream_t s, int grid, int dev) {
  if (a.soa) return launch_w<KIND, VARIANT, 0, CTAS>(a, s, grid, dev);
  switch (a.lw) {
    case 4: return launch_w<KIND, VARIANT, 16, CTAS>(a, s, grid, dev);
    case 5: return launch_w<KIND, VARIANT, 32, CTAS>(a, s, grid, dev);
    case 6: return launch_w<KIND, VARIANT, 64, CTAS>(a, s, grid, dev);
    default: return launch_w<KIND, VARIANT, 128, CTAS>(a, s, grid, dev);
  }
}

// Three CTAs per SM exist for the FP32-arithmetic variants (the FP64 ones
// need more than 72 registers a thread); others take the two-CTA shape.
template <int KIND, int VARIANT>
int launch_v(const StepArgs &a, cudaStream_t s, int grid, int dev, int ctas) {
  if constexpr (VARIANT == kFP32 || VARIANT == kAdaptive || VARIANT == kJoseph) {
    if (ctas == 3) return launch_c<KIND, VARIANT, 3>(a, s, grid, dev);
  }
  return launch_c<KIND, VARIANT, 2>(a, s, grid, dev);
}

// Launch the staged kernel for one kind and one group of variants (each
// defined in its own translation unit).
int launch_staged_p2z_f32(int precision, const StepArgs &a, cudaStream_t s, int grid, int dev,
                          int ctas);
int launch_staged_p2z_f64(int precision, const StepArgs &a, cudaStream_t s, int grid, int dev,
                          int ctas);
int launch_staged_p2r_f32(int precision, const StepArgs &a, cudaStream_t s, int grid, int dev,
                          int ctas);
int launch_staged_p2r_f64(int precision, const StepArgs &a, cudaStream_t s, int grid, int dev,
                          int ctas);

}  // namespace staged
}  // namespace kf
