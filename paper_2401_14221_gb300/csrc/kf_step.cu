// kf_step.cu -- single-step kernels (p2z / p2r propagate + Kalman update)
// and their C-ABI entry points (paper section 2: propagateToZ /
// propagateToR followed by KalmanUpdate, one track per thread).
//
// One thread owns one track: it reads the 6 state floats, 21 covariance
// floats, charge, hit and hit covariance (coalesced across the warp in SoA
// and AoSoA alike), runs the whole step in registers and writes the 27
// result floats with streaming stores.  The work is HBM-bound: 237 B (p2z)
// or 253 B (p2r) of algorithmic traffic per track against ~400-600 FP32
// instructions.
#include <cuda_runtime.h>

#include <atomic>

#include "kf_common.cuh"
#include "kf_device.cuh"
#include "kf_step.cuh"

namespace kf {

namespace staged {
// defined with the staged step kernel's dispatch (kf_step_staged.cu)
int sm_count(int dev, int *out);
}  // namespace staged

// CTAs per SM of the grid-stride kernel for arrays in host memory.
constexpr int kHostGridPerSm = 1;

// Without a tuning entry every batch in device memory runs the
// one-thread-per-track kernel in 128-thread CTAs.  With every operation
// explicitly rounded it needs 76 registers (six CTAs, 24 warps per SM), and
// on GB300 (graphs of 16 launches, microseconds per launch, against the
// staged kernel's better shape) it led or tied at every size and layout
// tried: p2r AoSoA32 240,000 tracks 11.5 vs 12.3; 960,000 36.6 vs 37.3
// (0.977 of the measured HBM copy bandwidth); 1,920,000 70.2 vs 74.5;
// 3,840,000 137.5 vs 158.6 (1.04); AoSoA16/64/128 and SoA at 960,000
// likewise; p2z AoSoA32 960,000 34.9 vs 35.5.  Only at 480,000 p2r tracks
// was the staged kernel (3 CTAs/SM) ahead, 19.4 vs 19.9.  64-thread CTAs
// time the same; 256-thread CTAs are 3 % slower; holding it to 72 or 64
// registers for more warps gained nothing or spilled.  The autotuner still
// times both kernels.
constexpr int kDirectThreads = 128;

struct Loc {
  int64_t base;
  int64_t stride;
};

// Element (c, i) of a C-component array sits at base + c * stride.
template <int C>
__device__ __forceinline__ Loc locate(int64_t i, int64_t n, int32_t soa, int32_t lw) {
  if (soa) return {i, n};
  const int64_t W = int64_t(1) << lw;
  return {(i >> lw) * (C * W) + (i & (W - 1)), W};
}

// Track i of a step launch (i < a.n): load, step, store.
template <int KIND, int VARIANT>
__device__ __forceinline__ void step_track(const StepArgs &a, int64_t i) {
  const Loc l6 = locate<6>(i, a.n, a.soa, a.lw);
  const Loc l21 = locate<21>(i, a.n, a.soa, a.lw);
  const Loc l3 = locate<3>(i, a.n, a.soa, a.lw);

  float p[6], C[21];
#pragma unroll
  for (int c = 0; c < 6; ++c) p[c] = __ldg(a.state_in + l6.base + c * l6.stride);
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = __ldg(a.cov_in + l21.base + e * l21.stride);
  const float qf = (float)__ldg(a.charge + i);
  const float surf = __ldg(a.surf + (a.surf_per_track ? i : 0));

  unsigned st;
  if (KIND == kP2z) {
    const float hx = __ldg(a.hit + l3.base);
    const float hy = __ldg(a.hit + l3.base + l3.stride);
    const float vxx = __ldg(a.hitcov + l6.base);
    const float vxy = __ldg(a.hitcov + l6.base + l6.stride);
    const float vyy = __ldg(a.hitcov + l6.base + 2 * l6.stride);
    st = p2z_step<VARIANT>(p, C, qf, a.bz, surf, hx, hy, vxx, vxy, vyy);
  } else {
    const float hx = __ldg(a.hit + l3.base);
    const float hy = __ldg(a.hit + l3.base + l3.stride);
    const float hz = __ldg(a.hit + l3.base + 2 * l3.stride);
    float hc[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) hc[c] = __ldg(a.hitcov + l6.base + c * l6.stride);
    st = p2r_step<VARIANT>(p, C, qf, a.bz, surf, hx, hy, hz, hc);
  }
  if constexpr (VARIANT == kAdaptive) {
    if (st & kRedo) {  // ill-conditioned in FP32: left to the FP64 redo pass
      a.status[i] = (uint8_t)kRedo;
      return;
    }
  }
  st |= finite_status(p, C);

#pragma unroll
  for (int c = 0; c < 6; ++c) __stcs(a.state_out + l6.base + c * l6.stride, p[c]);
#pragma unroll
  for (int e = 0; e < 21; ++e) __stcs(a.cov_out + l21.base + e * l21.stride, C[e]);
  if (a.status) a.status[i] = (uint8_t)st;
}

// Ask L2 for the AoSoA blocks of a C-component array that hold tracks
// [i0, i1): one bulk prefetch of the whole blocks (contiguous, 16-byte
// aligned: the array is, and a block is C * W * 4 bytes with W >= 16).
template <int C>
__device__ __forceinline__ void prefetch_blocks(const float *arr, int64_t i0, int64_t i1,
                                                int32_t lw) {
  const int64_t b0 = i0 >> lw, b1 = (i1 - 1) >> lw;
  const int64_t W = int64_t(1) << lw;
  const uint32_t bytes = (uint32_t)((b1 - b0 + 1) * C * W * 4);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(arr + b0 * C * W), "r"(bytes)
               : "memory");
}

// One track per thread.  Launched as a programmatic dependent of the
// previous kernel on the stream: it lets the next one be scheduled at once
// and waits for the previous one to complete before it touches memory.
// Under AoSoA a CTA that lands on an SM while the previous kernel drains
// first asks L2 for its inputs -- one bulk prefetch per array of the CTA's
// whole blocks: the state and covariance, for p2r also the hit and hit
// covariance; p2z reads only the first rows of those (x, y and the 2x2
// covariance), so for p2z one prefetch per block of each covers just those
// rows -- so that its loads after the wait find them there instead of in
// HBM.  A prefetch only moves lines
// into L2, where every SM's loads and stores meet, so it cannot return a
// value the previous kernel has yet to write.  Measured on GB300, 960,000
// p2r tracks in graphs of 16 launches: AoSoA 36.6-37.2 -> 35.5 us per
// launch.  Under SoA the same would take one prefetch per component row of
// 512 bytes; that measured slower (37.9 -> 40.0 us) and is not done.
template <int KIND, int VARIANT>
__global__ void __launch_bounds__(256) step_kernel(const __grid_constant__ StepArgs a) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
  if (!a.soa) {
    const int64_t i1 = i0 + blockDim.x < a.n ? i0 + blockDim.x : a.n;
    if (threadIdx.x == 0) {
      prefetch_blocks<6>(a.state_in, i0, i1, a.lw);
      prefetch_blocks<21>(a.cov_in, i0, i1, a.lw);
      if (KIND == kP2r) {
        prefetch_blocks<3>(a.hit, i0, i1, a.lw);
        prefetch_blocks<6>(a.hitcov, i0, i1, a.lw);
      }
    }
    if (KIND == kP2z) {
      // p2z reads the hit's x, y rows and the covariance's xx, xy, yy rows:
      // the first 2 and 3 rows of each block, one prefetch each per block
      const int64_t W = int64_t(1) << a.lw, b0 = i0 >> a.lw, nb = ((i1 - 1) >> a.lw) - b0 + 1;
      if ((int64_t)threadIdx.x < nb) {
        const int64_t blk = b0 + threadIdx.x;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.hit + blk * 3 * W),
                     "r"((uint32_t)(2 * W * 4))
                     : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.hitcov + blk * 6 * W),
                     "r"((uint32_t)(3 * W * 4))
                     : "memory");
      }
    }
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t i = i0 + threadIdx.x;
  if (i < a.n) step_track<KIND, VARIANT>(a, i);
}

// The same as a persistent grid-stride loop, for arrays in host memory: a
// small grid whose warps are at different points of their tracks keeps both
// directions of the CPU-GPU link busy at once, where a grid of n / 256 CTAs
// reads in waves and then writes in waves.  Measured on GB300, 960,000 p2r
// tracks from page-locked memory: one track per thread 0.896 ms; grid-stride
// with 1, 2, 4 CTAs of 256 threads per SM 0.725, 0.758, 0.780 ms; half the
// SMs 0.739 ms; 128-thread CTAs 0.736 ms.
template <int KIND, int VARIANT>
__global__ void __launch_bounds__(256) step_kernel_strided(const __grid_constant__ StepArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
    step_track<KIND, VARIANT>(a, i);
}

// The redo pass of KF_ADAPTIVE: each block gathers the marked tracks of its
// span of kRedoSpan tracks (one 16-byte status load per 16 tracks), then its
// threads run the FP64 step on them, 32 marked tracks to a warp.
template <int KIND>
__global__ void __launch_bounds__(kRedoThreads) redo_pass_kernel(const __grid_constant__ StepArgs a) {
  __shared__ uint16_t list[kRedoSpan];
  __shared__ int count;
  // Launched as a programmatic dependent of the step kernel: wait here until
  // it has completed and its status marks are visible.  Before that, let the
  // next kernel on the stream be scheduled (a staged step then sets up and
  // prefetches while this pass runs; it waits for this grid to complete
  // before it reads or writes anything).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t span0 = (int64_t)blockIdx.x * kRedoSpan;
  const int cnt = gather_marked(a.status, span0, a.n, list, &count);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int64_t i = span0 + list[q];
    a.status[i] = (uint8_t)redo_track_fp64<KIND>(a, i);
  }
}

int launch_redo_pass(int kind, const StepArgs &a, cudaStream_t s) {
  if (a.n == 0) return KF_OK;
  const int64_t blocks = (a.n + kRedoSpan - 1) / kRedoSpan;
  if (blocks > 0x7fffffffLL) return set_error(KF_ERR_ARG, "n too large for one launch");
  const unsigned g = (unsigned)blocks;
  // programmatic dependent launch: scheduled while the step kernel drains
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g);
  cfg.blockDim = dim3(kRedoThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = kind == kP2z ? cudaLaunchKernelEx(&cfg, redo_pass_kernel<kP2z>, a)
                                     : cudaLaunchKernelEx(&cfg, redo_pass_kernel<kP2r>, a);
  return check_cuda(e, "adaptive redo pass launch");
}

template <int KIND>
static int launch_step(const kf_params *params, kf_layout layout, const float *state_in,
                       const float *cov_in, float *state_out, float *cov_out,
                       const int8_t *charge, const float *hit, const float *hit_cov,
                       const float *surf, int32_t surf_per_track, uint8_t *status,
                       void *stream) {
  clear_error();
  if (!params) return set_error(KF_ERR_ARG, "params is NULL");
  if (params->flags != 0) return set_error(KF_ERR_ARG, "params->flags must be 0");
  if (params->precision < KF_FP32 || params->precision > KF_DF_UPDATE)
    return set_error(KF_ERR_ARG, "unknown precision %d", params->precision);
  LayoutDesc d;
  if (int rc = check_layout(layout, &d)) return rc;
  if (d.n == 0) return KF_OK;
  if (!state_in || !cov_in || !state_out || !cov_out || !charge || !hit || !hit_cov || !surf)
    return set_error(KF_ERR_ARG, "a required pointer is NULL");
  if (!aligned16(state_in) || !aligned16(cov_in) || !aligned16(state_out) ||
      !aligned16(cov_out) || !aligned16(hit) || !aligned16(hit_cov))
    return set_error(KF_ERR_ARG, "float arrays must be 16-byte aligned");
  if (surf_per_track != 0 && surf_per_track != 1)
    return set_error(KF_ERR_ARG, "surf_per_track must be 0 or 1");
  bool plain_loads = false;  // some array in host or managed memory
  {
    const int64_t b6 = 4 * layout_floats(d, 6), b21 = 4 * layout_floats(d, 21);
    const void *ptrs[] = {state_in, cov_in, state_out, cov_out, charge, hit, hit_cov, surf};
    const int64_t bytes[] = {b6, b21, b6, b21, d.n, 4 * layout_floats(d, 3), b6,
                             surf_per_track ? 4 * d.n : 4};
    const char *names[] = {"state_in", "cov_in", "state_out", "cov_out",
                           "charge",   "hit",    "hit_cov",   "surf"};
    for (int k = 0; k < 8; ++k) {
      bool nd = false;
      if (int rc = check_device_range(ptrs[k], bytes[k], names[k], &nd)) return rc;
      plain_loads |= nd;
    }
    if (status) {
      bool nd = false;
      if (int rc = check_device_range(status, d.n, "status", &nd)) return rc;
      plain_loads |= nd;
    }
    if (!status && params->precision == KF_ADAPTIVE)
      return set_error(KF_ERR_ARG, "KF_ADAPTIVE needs a status array (its redo pass reads it)");
  }
  if (partial_overlap(state_in, 4 * layout_floats(d, 6), state_out, 4 * layout_floats(d, 6)) ||
      partial_overlap(cov_in, 4 * layout_floats(d, 21), cov_out, 4 * layout_floats(d, 21)))
    return set_error(KF_ERR_ARG, "input and output overlap without coinciding");

  StepArgs a{state_in, cov_in, state_out, cov_out, charge, hit, hit_cov, surf, status,
             d.n,      d.soa,  d.lw,      params->bz, surf_per_track};
  return launch_step_kernel(KIND, params->precision, a, static_cast<cudaStream_t>(stream),
                            plain_loads);
}

namespace {
std::atomic<int> g_step_mode{KF_STEP_AUTO};
std::atomic<int> g_staged_ctas{0};
}

int step_kernel_mode() { return g_step_mode.load(std::memory_order_relaxed); }

static int launch_step_main(int kind, int precision, const StepArgs &a, cudaStream_t s,
                            bool plain_loads);

int launch_step_kernel(int kind, int precision, const StepArgs &a, cudaStream_t s,
                       bool plain_loads) {
  if (a.n == 0) return KF_OK;
  if (precision == KF_ADAPTIVE && !a.status)
    return set_error(KF_ERR_ARG, "KF_ADAPTIVE needs a status array (its redo pass reads it)");
  if (int rc = launch_step_main(kind, precision, a, s, plain_loads)) return rc;
  return precision == KF_ADAPTIVE ? launch_redo_pass(kind, a, s) : KF_OK;
}

static int launch_step_main(int kind, int precision, const StepArgs &a, cudaStream_t s,
                            bool plain_loads) {
  // The staged kernel copies whole tiles of device memory with 16-byte-
  // aligned bulk copies: any AoSoA layout, SoA when n is a multiple of 4.
  const bool staged_ok = !plain_loads && (!a.soa || (a.n & 3) == 0);
  // the FP64 variants are bound by GB300's FP64 pipe, where the staged
  // kernel's decoupled loads help (960,000 p2r tracks: FP64 update 262 us
  // staged at 2 CTAs/SM against 300 us direct; all-FP64 1,044 against 1,092)
  const bool fp64 = precision == KF_FP64_UPDATE || precision == KF_FP64;
  LaunchConfig cfg{(fp64 && staged_ok) ? KF_STEP_STAGED : KF_STEP_DIRECT, kDirectThreads, 2};
  if (plain_loads) {
    // host or managed memory: the grid-stride kernel below
  } else if (const LaunchConfig *o = thread_override()) {
    cfg = *o;
  } else {
    const int mode = step_kernel_mode();
    if (mode == KF_STEP_DIRECT) {
      cfg.kernel = KF_STEP_DIRECT;
    } else if (mode == KF_STEP_STAGED) {
      cfg.kernel = KF_STEP_STAGED;
      const int c = g_staged_ctas.load(std::memory_order_relaxed);
      if (c > 0) cfg.ctas_per_sm = c;
    } else if (mode == KF_STEP_AUTO) {
      LaunchConfig t;
      if (tune_lookup(kOpStep, kind, precision, a.soa, a.lw, a.n, &t)) cfg = t;
    }
  }
  if (staged_ok && cfg.kernel == KF_STEP_STAGED)
    return launch_step_staged(kind, precision, a, s, cfg.ctas_per_sm);
  if (plain_loads) {
    int dev = 0, sms = 0;
    if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
    if (int rc = staged::sm_count(dev, &sms)) return rc;
    const int64_t want = (a.n + 255) / 256, cap = (int64_t)kHostGridPerSm * sms;
    const unsigned g = (unsigned)(want < cap ? want : cap);
    if (kind == kP2z) {
      switch (precision) {
        case KF_FP32: step_kernel_strided<kP2z, kFP32><<<g, 256, 0, s>>>(a); break;
        case KF_FP64_UPDATE: step_kernel_strided<kP2z, kFP64Update><<<g, 256, 0, s>>>(a); break;
        case KF_JOSEPH: step_kernel_strided<kP2z, kJoseph><<<g, 256, 0, s>>>(a); break;
        case KF_FP64: step_kernel_strided<kP2z, kFP64><<<g, 256, 0, s>>>(a); break;
        case KF_DF_UPDATE: step_kernel_strided<kP2z, kDFUpdate><<<g, 256, 0, s>>>(a); break;
        default: step_kernel_strided<kP2z, kAdaptive><<<g, 256, 0, s>>>(a); break;
      }
    } else {
      switch (precision) {
        case KF_FP32: step_kernel_strided<kP2r, kFP32><<<g, 256, 0, s>>>(a); break;
        case KF_FP64_UPDATE: step_kernel_strided<kP2r, kFP64Update><<<g, 256, 0, s>>>(a); break;
        case KF_JOSEPH: step_kernel_strided<kP2r, kJoseph><<<g, 256, 0, s>>>(a); break;
        case KF_FP64: step_kernel_strided<kP2r, kFP64><<<g, 256, 0, s>>>(a); break;
        case KF_DF_UPDATE: step_kernel_strided<kP2r, kDFUpdate><<<g, 256, 0, s>>>(a); break;
        default: step_kernel_strided<kP2r, kAdaptive><<<g, 256, 0, s>>>(a); break;
      }
    }
    return check_cuda(cudaGetLastError(), "host-resident step launch");
  }
  const int threads = (cfg.threads == 128 || cfg.threads == 64) ? cfg.threads : 256;
  const int64_t blocks = (a.n + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return set_error(KF_ERR_ARG, "n too large for one launch");
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)blocks);
  lc.blockDim = dim3((unsigned)threads);
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaError_t e;
  if (kind == kP2z) {
    switch (precision) {
      case KF_FP32: e = cudaLaunchKernelEx(&lc, step_kernel<kP2z, kFP32>, a); break;
      case KF_FP64_UPDATE: e = cudaLaunchKernelEx(&lc, step_kernel<kP2z, kFP64Update>, a); break;
      case KF_JOSEPH: e = cudaLaunchKernelEx(&lc, step_kernel<kP2z, kJoseph>, a); break;
      case KF_FP64: e = cudaLaunchKernelEx(&lc, step_kernel<kP2z, kFP64>, a); break;
      case KF_DF_UPDATE: e = cudaLaunchKernelEx(&lc, step_kernel<kP2z, kDFUpdate>, a); break;
      default: e = cudaLaunchKernelEx(&lc, step_kernel<kP2z, kAdaptive>, a); break;
    }
  } else {
    switch (precision) {
      case KF_FP32: e = cudaLaunchKernelEx(&lc, step_kernel<kP2r, kFP32>, a); break;
      case KF_FP64_UPDATE: e = cudaLaunchKernelEx(&lc, step_kernel<kP2r, kFP64Update>, a); break;
      case KF_JOSEPH: e = cudaLaunchKernelEx(&lc, step_kernel<kP2r, kJoseph>, a); break;
      case KF_FP64: e = cudaLaunchKernelEx(&lc, step_kernel<kP2r, kFP64>, a); break;
      case KF_DF_UPDATE: e = cudaLaunchKernelEx(&lc, step_kernel<kP2r, kDFUpdate>, a); break;
      default: e = cudaLaunchKernelEx(&lc, step_kernel<kP2r, kAdaptive>, a); break;
    }
  }
  return check_cuda(e, kind == kP2z ? "p2z step launch" : "p2r step launch");
}

}  // namespace kf

extern "C" int kf_p2z_propagate_update(const kf_params *params, kf_layout layout,
                                       const float *state_in, const float *cov_in,
                                       float *state_out, float *cov_out, const int8_t *charge,
                                       const float *hit, const float *hit_cov,
                                       const float *z_surf, int32_t surf_per_track,
                                       uint8_t *status, void *stream) {
  return kf::launch_step<kf::kP2z>(params, layout, state_in, cov_in, state_out, cov_out, charge,
                                   hit, hit_cov, z_surf, surf_per_track, status, stream);
}

extern "C" int kf_p2r_propagate_update(const kf_params *params, kf_layout layout,
                                       const float *state_in, const float *cov_in,
                                       float *state_out, float *cov_out, const int8_t *charge,
                                       const float *hit, const float *hit_cov,
                                       const float *r_surf, int32_t surf_per_track,
                                       uint8_t *status, void *stream) {
  return kf::launch_step<kf::kP2r>(params, layout, state_in, cov_in, state_out, cov_out, charge,
                                   hit, hit_cov, r_surf, surf_per_track, status, stream);
}

extern "C" int kf_set_step_kernel(int32_t mode) {
  kf::clear_error();
  if (mode != KF_STEP_AUTO && mode != KF_STEP_DIRECT && mode != KF_STEP_STAGED)
    return kf::set_error(KF_ERR_ARG, "unknown step kernel mode %d", mode);
  kf::g_step_mode.store(mode, std::memory_order_relaxed);
  return KF_OK;
}

extern "C" int kf_set_staged_ctas_per_sm(int32_t ctas) {
  kf::clear_error();
  if (ctas < 0 || ctas > 3) return kf::set_error(KF_ERR_ARG, "ctas_per_sm = %d is not 0..3", ctas);
  kf::g_staged_ctas.store(ctas, std::memory_order_relaxed);
  return KF_OK;
}
