// kf_staged_compressed.cu -- the single step on the compressed covariance
// store (FP32 sigmas, FP16 correlations), staged like the FP32-store step:
// a persistent CTA whose producer warp streams AoSoA tiles of 256 tracks into
// shared memory with bulk asynchronous copies (state, sigma, rho, hit, hit
// covariance: five contiguous runs per tile) while eight compute warps
// decode, step, encode and store (the correlations in FP16 pairs:
// kf_compressed.cuh).  The one-thread-per-track kernel reads 193
// algorithmic bytes per p2r track through 2- and 4-byte loads; staging moves
// them at the bulk-copy rate.  Arithmetic and results are those of the
// one-thread-per-track kernel, bit for bit.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>

#include "kf_compressed.cuh"
#include "kf_step_staged.cuh"

namespace kf {
namespace staged {
// defined with the staged step kernel's dispatch (kf_step_staged.cu)
int sm_count(int dev, int *out);
int error_word(int dev, unsigned **out);
uint32_t device_wait_polls();
}  // namespace staged

namespace {

using staged::bulk_g2s;
using staged::kComputeWarps;
using staged::kT;
using staged::kThreads;
using staged::mbar_arrive;
using staged::mbar_arrive_expect_tx;
using staged::mbar_fence_init;
using staged::mbar_init;
using staged::mbar_wait;
using staged::Schedule;

constexpr int kStateB = kT * 6 * 4;
constexpr int kSigB = kT * 6 * 4;
constexpr int kRhoB = kT * 15 * 2;
constexpr int kHitB = kT * 3 * 4;
constexpr int kHcB = kT * 6 * 4;
constexpr int kStageB = kStateB + kSigB + kRhoB + kHitB + kHcB;  // 29,184 B
// Resident CTAs per SM: 3 of 2 stages each (24 compute warps per SM, at most
// 72 registers a thread), or 2 of 3 stages.
constexpr int kCompressedCtas = 3;
constexpr int stages_of(int ctas) { return ctas >= 3 ? 2 : 3; }
constexpr int smem_of(int ctas) { return stages_of(ctas) * (kStageB + 16); }

template <int KIND, int VARIANT, int W, int CTAS>
__global__ void __launch_bounds__(kThreads, CTAS)
    compressed_staged_kernel(const __grid_constant__ CompressedArgs a, unsigned *err,
                             uint32_t wait_polls) {
  static_assert(kT % W == 0, "tile must hold whole AoSoA blocks");
  static_assert(W % 2 == 0, "pairs of correlation rows per block");
  constexpr int kStages = stages_of(CTAS);
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageB);
  uint64_t *empty = full + kStages;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const Schedule sch = staged::make_schedule<W>(a.n, gridDim.x);
  const int64_t ntiles = sch.tiles_of(blockIdx.x);
  // raised when a warp of this CTA gives up a bounded wait (the pipeline
  // then stops and drains, as in the FP32-store kernel)
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
  // Programmatic dependent launch, with this CTA's first tiles requested
  // into L2 while the previous kernel drains (a prefetch cannot return data
  // that kernel has yet to write: the copies after the wait read L2's
  // current lines).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (warp == kComputeWarps && lane == 0) {
    const int64_t npre = ntiles < kStages ? ntiles : kStages;
    for (int64_t k = 0; k < npre; ++k) {
      int64_t first, m;
      sch.tile(k, blockIdx.x, a.n, &first, &m);
      const uint32_t cols = (uint32_t)(((m + W - 1) / W) * W);
      staged::bulk_prefetch_l2(a.state_in + first * 6, cols * 6 * 4);
      staged::bulk_prefetch_l2(a.sigma_in + first * 6, cols * 6 * 4);
      staged::bulk_prefetch_l2(a.rho_in + first * 15, cols * 15 * 2);
      staged::bulk_prefetch_l2(a.hit + first * 3, cols * 3 * 4);
      staged::bulk_prefetch_l2(a.hitcov + first * 6, cols * 6 * 4);
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
        if (k >= kStages && !mbar_wait(&empty[s], ph ^ 1u, err, staged::kMaxPolls, &abort_flag))
          break;
        int64_t first, m;
        sch.tile(k, blockIdx.x, a.n, &first, &m);
        const uint32_t cols = (uint32_t)(((m + W - 1) / W) * W);  // whole blocks
        unsigned char *st = smem + s * kStageB;
        mbar_arrive_expect_tx(&full[s], cols * (6 * 4 + 6 * 4 + 15 * 2 + 3 * 4 + 6 * 4));
        bulk_g2s(st, a.state_in + first * 6, cols * 6 * 4, &full[s]);
        bulk_g2s(st + kStateB, a.sigma_in + first * 6, cols * 6 * 4, &full[s]);
        bulk_g2s(st + kStateB + kSigB, a.rho_in + first * 15, cols * 15 * 2, &full[s]);
        bulk_g2s(st + kStateB + kSigB + kRhoB, a.hit + first * 3, cols * 3 * 4, &full[s]);
        bulk_g2s(st + kStateB + kSigB + kRhoB + kHitB, a.hitcov + first * 6, cols * 6 * 4,
                 &full[s]);
        issued = k + 1;
      }
      for (int64_t k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
        if (!mbar_wait(&full[k % kStages], (uint32_t)(k / kStages) & 1u, err)) break;
    }
    return;
  }

  // --------------------------------------------------------------- compute
  const int il = warp * 32 + lane;
  const int blk = il / W, r = il % W;
  // this thread's track within a tile of whole AoSoA blocks: its elements
  // sit at these offsets from the tile's start, in shared memory as in
  // global memory (the tile's first track, a multiple of W, times the
  // components per track)
  const int o6 = blk * 6 * W + r, o3 = blk * 3 * W + r;
  const RhoLoc orh{blk * (15 * W / 2) + r, W, blk * (15 * W) + 14 * W + r};
  // the next tile's first track and size, with its charge and per-track
  // surface requested one tile ahead so that their latency hides behind the
  // previous tile's step.  Nothing consumes the loaded values before that
  // step (a thread past the tile's end loads the last track's, unused), so
  // the warp does not wait for them here.
  int64_t first_next = 0;
  int m_next = 0;
  int8_t q_next = 1;
  float surf_next = 0.0f;
  auto fetch = [&](int64_t k) {
    int64_t mm;
    sch.tile(k, blockIdx.x, a.n, &first_next, &mm);
    m_next = (int)mm;
    const int64_t j = il < m_next ? first_next + il : a.n - 1;
    q_next = __ldg(a.charge + j);
    surf_next = __ldg(a.surf + (a.surf_per_track ? j : 0));
  };
  if (ntiles > 0) fetch(0);
  for (int64_t k = 0; k < ntiles; ++k) {
    const int s = (int)(k % kStages);
    const uint32_t ph = (uint32_t)(k / kStages) & 1u;
    const int64_t first = first_next;
    const bool live = il < m_next;
    const int8_t q = q_next;
    const float surf = surf_next;
    if (k + 1 < ntiles) fetch(k + 1);
    if (!mbar_wait(&full[s], ph, err, wait_polls, &abort_flag)) break;

    const unsigned char *st = smem + s * kStageB;
    const float *sst = reinterpret_cast<const float *>(st);
    const float *ssg = reinterpret_cast<const float *>(st + kStateB);
    const __half *srh = reinterpret_cast<const __half *>(st + kStateB + kSigB);
    const float *sht = reinterpret_cast<const float *>(st + kStateB + kSigB + kRhoB);
    const float *shc = reinterpret_cast<const float *>(st + kStateB + kSigB + kRhoB + kHitB);
    float p[6], sg[6], hc[6];
    Rho rh;
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = sst[o6 + c * W];
#pragma unroll
    for (int c = 0; c < 6; ++c) sg[c] = ssg[o6 + c * W];
    load_rho(srh, orh, rh);
    const float hx = sht[o3];
    const float hy = sht[o3 + W];
    const float hz = sht[o3 + 2 * W];
#pragma unroll
    for (int c = 0; c < 6; ++c) hc[c] = shc[o6 + c * W];
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // stage may be refilled
    if (!live) continue;
    const int64_t i = first + il;
    const float qf = (float)q;

    float C[21];
    decode_cov(sg, rh, C);
    unsigned stt;
    if (KIND == kP2z)
      stt = p2z_step<VARIANT>(p, C, qf, a.bz, surf, hx, hy, hc[0], hc[1], hc[2]);
    else
      stt = p2r_step<VARIANT>(p, C, qf, a.bz, surf, hx, hy, hz, hc);
    if constexpr (VARIANT == kAdaptive) {
      if (stt & kRedo) {  // left to the FP64 redo pass, inputs untouched
        a.status[i] = (uint8_t)kRedo;
        continue;
      }
    }
    stt |= finite_status(p, C);
    const int64_t b6 = first * 6 + o6;
    const RhoLoc lr{(first >> 1) * 15 + orh.word, W, first * 15 + orh.last};
    if (!(stt & kNoIntersect)) {
      encode_cov(C, sg, rh);
    } else {
      // a track that was not propagated gets its input sigma / rho back, bit
      // for bit: re-read from global memory (rare), so that the staged input
      // need not stay in registers across the step
#pragma unroll
      for (int c = 0; c < 6; ++c) sg[c] = a.sigma_in[b6 + c * W];
      load_rho(a.rho_in, lr, rh);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) __stcs(a.state_out + b6 + c * W, p[c]);
#pragma unroll
    for (int c = 0; c < 6; ++c) __stcs(a.sigma_out + b6 + c * W, sg[c]);
    store_rho(a.rho_out, lr, rh);
    if (a.status) a.status[i] = (uint8_t)stt;
  }
}

template <int KIND, int VARIANT, int W>
int launch_w(const CompressedArgs &a, cudaStream_t s, int grid, unsigned *err, int dev) {
  constexpr int kSmem = smem_of(kCompressedCtas);
  auto kern = compressed_staged_kernel<KIND, VARIANT, W, kCompressedCtas>;
  static std::atomic<bool> configured[64] = {};
  if (dev < 0 || dev >= 64 || !configured[dev].load(std::memory_order_acquire)) {
    if (int rc = check_cuda(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem),
            "cudaFuncSetAttribute"))
      return rc;
    if (dev >= 0 && dev < 64) configured[dev].store(true, std::memory_order_release);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return check_cuda(cudaLaunchKernelEx(&cfg, kern, a, err, staged::device_wait_polls()),
                    "compressed staged launch");
}

template <int KIND, int VARIANT>
int launch_v(const CompressedArgs &a, cudaStream_t s, int grid, unsigned *err, int dev) {
  switch (a.lw) {
    case 4: return launch_w<KIND, VARIANT, 16>(a, s, grid, err, dev);
    case 5: return launch_w<KIND, VARIANT, 32>(a, s, grid, err, dev);
    case 6: return launch_w<KIND, VARIANT, 64>(a, s, grid, err, dev);
    default: return launch_w<KIND, VARIANT, 128>(a, s, grid, err, dev);
  }
}

}  // namespace

int launch_compressed_staged(int kind, int precision, const CompressedArgs &a, cudaStream_t s) {
  if (a.n == 0) return KF_OK;
  if (a.soa) return set_error(KF_ERR_UNSUPPORTED, "the staged compressed step takes AoSoA");
  int dev = 0, sms = 0;
  if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
  if (int rc = staged::sm_count(dev, &sms)) return rc;
  unsigned *err = nullptr;
  if (int rc = staged::error_word(dev, &err)) return rc;
  const int64_t ntiles = (a.n + kT - 1) / kT;
  const int64_t slots = (int64_t)kCompressedCtas * sms;
  const int grid = (int)(ntiles < slots ? ntiles : slots);
  // the float-arithmetic variants (the FP64 ones stay one thread per track)
  if (kind == kP2z) {
    switch (precision) {
      case KF_FP32: return launch_v<kP2z, kFP32>(a, s, grid, err, dev);
      case KF_JOSEPH: return launch_v<kP2z, kJoseph>(a, s, grid, err, dev);
      case KF_ADAPTIVE: return launch_v<kP2z, kAdaptive>(a, s, grid, err, dev);
      default: return set_error(KF_ERR_UNSUPPORTED, "staged compressed: FP32 variants only");
    }
  }
  switch (precision) {
    case KF_FP32: return launch_v<kP2r, kFP32>(a, s, grid, err, dev);
    case KF_JOSEPH: return launch_v<kP2r, kJoseph>(a, s, grid, err, dev);
    case KF_ADAPTIVE: return launch_v<kP2r, kAdaptive>(a, s, grid, err, dev);
    default: return set_error(KF_ERR_UNSUPPORTED, "staged compressed: FP32 variants only");
  }
}

}  // namespace kf
