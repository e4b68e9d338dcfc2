// kf_chain.cu -- fused multi-layer chain: each track runs propagate + update
// through L detector layers inside one kernel (paper section 2 and the
// per-track layer loop of Figs. 3-5: for each layer, propagateTo{R,Z} then
// KalmanUpdate).
//
// One thread owns one track for the whole chain: state, covariance and
// charge are loaded once, kept in registers across all layers, and written
// back once; only the per-layer hits stream in (the next layer's hit is
// loaded while the current layer computes).  Per track that is 109 B in,
// 36 B per layer and 108 B out, against 253 B per layer for L separate
// single-step launches that round-trip the state through HBM.  The layer
// kind is uniform across the grid, so the p2z / p2r branch never diverges.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "kf_common.cuh"
#include "kf_device.cuh"
#include "kf_step.cuh"
#include "kf_chain.cuh"

namespace kf {
namespace staged {
// SM count of a device (cached; kf_step_staged.cu)
int sm_count(int dev, int *out);
}  // namespace staged

struct ChainArgs {
  float *state;
  float *cov;
  const int8_t *charge;
  const float *hits;     // [L] arrays of 3 components in the layout
  const float *hitcovs;  // [L] arrays of 6 components in the layout
  uint8_t *status;
  int64_t n;
  int64_t hit_stride;  // floats between consecutive layers' hit arrays
  int64_t hc_stride;   // floats between consecutive layers' hit-cov arrays
  int32_t soa;
  int32_t lw;
  float bz;
  int32_t L;
  int32_t kinds[KF_MAX_LAYERS];
  float pos[KF_MAX_LAYERS];
};

namespace {

// Track i of the chain: load, run every layer, store.
template <int VARIANT>
__device__ __forceinline__ void chain_one(const ChainArgs &a, int64_t i) {
  const ChainLoc l6 = chain_locate<6>(i, a.n, a.soa, a.lw);
  const ChainLoc l21 = chain_locate<21>(i, a.n, a.soa, a.lw);
  const ChainLoc l3 = chain_locate<3>(i, a.n, a.soa, a.lw);

  float p[6], C[21];
#pragma unroll
  for (int c = 0; c < 6; ++c) p[c] = a.state[l6.base + c * l6.stride];
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = a.cov[l21.base + e * l21.stride];
  const float qf = (float)__ldg(a.charge + i);

  unsigned st;
  if constexpr (VARIANT == kAdaptive) {
    st = chain_track_marking(p, C, qf, a.bz, a.L, a.kinds, a.pos, a.hits, a.hit_stride, a.hitcovs,
                             a.hc_stride, l3, l6);
    if (st & kRedo) {  // left to chain_redo_kernel, inputs untouched
      a.status[i] = (uint8_t)kRedo;
      return;
    }
  } else if constexpr (VARIANT == kFP64) {
    st = chain_track_fp64(p, C, qf, a.bz, a.L, a.kinds, a.pos, a.hits, a.hit_stride, a.hitcovs,
                          a.hc_stride, l3, l6);
  } else {
    st = chain_track<VARIANT>(p, C, qf, a.bz, a.L, a.kinds, a.pos, a.hits, a.hit_stride,
                              a.hitcovs, a.hc_stride, l3, l6);
  }
  st |= finite_status(p, C);
#pragma unroll
  for (int c = 0; c < 6; ++c) a.state[l6.base + c * l6.stride] = p[c];
#pragma unroll
  for (int e = 0; e < 21; ++e) a.cov[l21.base + e * l21.stride] = C[e];
  if (a.status) a.status[i] = (uint8_t)st;
}

template <int VARIANT>
__global__ void __launch_bounds__(256) chain_kernel(const ChainArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) chain_one<VARIANT>(a, i);
}

// KF_ADAPTIVE's first pass, held to 80 registers so that three 256-thread
// CTAs fit an SM (unbounded it takes 96: two CTAs; measured on the 256-event
// chain workload, the adaptive chain 1.057 -> 0.949 ms, no spills).
__global__ void __launch_bounds__(256, 3) chain_mark_kernel(const ChainArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) chain_one<kAdaptive>(a, i);
}

// KF_ADAPTIVE's second pass for one marked track: the whole chain again
// from its (untouched) inputs, in double (chain_track_fp64).
__device__ __forceinline__ void chain_redo_track(const ChainArgs &a, int64_t i) {
  const ChainLoc l6 = chain_locate<6>(i, a.n, a.soa, a.lw);
  const ChainLoc l21 = chain_locate<21>(i, a.n, a.soa, a.lw);
  const ChainLoc l3 = chain_locate<3>(i, a.n, a.soa, a.lw);
  float p[6], C[21];
  for (int c = 0; c < 6; ++c) p[c] = a.state[l6.base + c * l6.stride];
  for (int e = 0; e < 21; ++e) C[e] = a.cov[l21.base + e * l21.stride];
  const float qf = (float)a.charge[i];
  unsigned st = chain_track_fp64(p, C, qf, a.bz, a.L, a.kinds, a.pos, a.hits, a.hit_stride,
                                 a.hitcovs, a.hc_stride, l3, l6);
  st |= finite_status(p, C);
  for (int c = 0; c < 6; ++c) a.state[l6.base + c * l6.stride] = p[c];
  for (int e = 0; e < 21; ++e) a.cov[l21.base + e * l21.stride] = C[e];
  a.status[i] = (uint8_t)st;
}

// The second pass over one list of the whole batch's marked tracks, 32 to
// a warp.  An FP64 warp instruction occupies the FP64 pipe as long with one
// lane active as with 32 (spreading a span's marks over two warps instead
// of one made the adaptive chain slower, 0.761 -> 0.795 ms), so full warps
// need about a quarter fewer FP64 warp instructions than one partly filled
// warp per span; one-warp blocks, four per SM, spread them over the SMs.
// chain_compact_kernel builds the list: each block gathers its span's marks
// and appends them (one atomic per block; the order of the list varies from
// run to run, the result of each track does not).
__global__ void __launch_bounds__(kRedoThreads) chain_compact_kernel(const uint8_t *status,
                                                                     int64_t n,
                                                                     uint32_t *count,
                                                                     uint32_t *list) {
  __shared__ uint16_t span_list[kRedoSpan];
  __shared__ int span_count;
  __shared__ uint32_t base;
  const int64_t span0 = (int64_t)blockIdx.x * kRedoSpan;
  const int cnt = gather_marked(status, span0, n, span_list, &span_count);
  if (cnt == 0) return;  // the same count in every thread of the block
  if (threadIdx.x == 0) base = atomicAdd(count, (uint32_t)cnt);
  __syncthreads();
  for (int q = threadIdx.x; q < cnt; q += blockDim.x)
    list[base + q] = (uint32_t)(span0 + span_list[q]);
}

constexpr int kRedoListBlocksPerSm = 4;

__global__ void __launch_bounds__(32) chain_redo_list_kernel(const ChainArgs a,
                                                             const uint32_t *count,
                                                             const uint32_t *list) {
  const int64_t total = *count;
  for (int64_t g = blockIdx.x; g * 32 < total; g += gridDim.x) {
    const int64_t q = g * 32 + threadIdx.x;
    if (q < total) chain_redo_track(a, list[q]);
  }
}

// KF_ADAPTIVE's second pass without a list (no scratch memory could be had,
// or more than 2^32 - 1 tracks): each block gathers the marked tracks of its
// span (gather_marked) and reruns them.
__global__ void __launch_bounds__(kRedoThreads) chain_redo_kernel(const ChainArgs a) {
  __shared__ uint16_t list[kRedoSpan];
  __shared__ int count;
  const int64_t span0 = (int64_t)blockIdx.x * kRedoSpan;
  const int cnt = gather_marked(a.status, span0, a.n, list, &count);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) chain_redo_track(a, span0 + list[q]);
}

// A stream-ordered memory pool per device for the second pass's list,
// created on first use and kept (with its memory: release threshold at the
// maximum) for the life of the process.  It is not created while the
// stream is being captured into a graph (creating a pool is not a
// capturable call); allocating from an existing pool is, and gives the
// graph an allocation node.
constexpr int kMaxPoolDevices = 64;
std::mutex g_redo_pool_mu;
cudaMemPool_t g_redo_pool[kMaxPoolDevices] = {};

bool redo_pool(int dev, bool may_create, cudaMemPool_t *out) {
  if (dev < 0 || dev >= kMaxPoolDevices) return false;
  std::lock_guard<std::mutex> lock(g_redo_pool_mu);
  if (!g_redo_pool[dev]) {
    if (!may_create) return false;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    uint64_t keep = UINT64_MAX;
    (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_redo_pool[dev] = pool;
  }
  *out = g_redo_pool[dev];
  return true;
}

std::atomic<int> g_chain_redo{KF_CHAIN_REDO_LIST};

// Launch the second pass on stream s: over a compacted list when its
// scratch can be allocated, else per span (the same results).
int launch_chain_redo(const ChainArgs &a, cudaStream_t s) {
  const unsigned spans = (unsigned)((a.n + kRedoSpan - 1) / kRedoSpan);
  int dev = 0, sms = 0;
  cudaMemPool_t pool = nullptr;
  void *buf = nullptr;
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(s, &capture) != cudaSuccess ||
                         capture != cudaStreamCaptureStatusNone;
  if (g_chain_redo.load(std::memory_order_relaxed) == KF_CHAIN_REDO_LIST &&
      a.n < (int64_t)UINT32_MAX && cudaGetDevice(&dev) == cudaSuccess &&
      staged::sm_count(dev, &sms) == KF_OK && redo_pool(dev, !capturing, &pool) &&
      cudaMallocFromPoolAsync(&buf, 4 * (size_t)(a.n + 1), pool, s) == cudaSuccess) {
    uint32_t *count = static_cast<uint32_t *>(buf), *list = count + 1;
    int rc = check_cuda(cudaMemsetAsync(count, 0, sizeof(uint32_t), s), "cudaMemsetAsync");
    if (rc == KF_OK) {
      chain_compact_kernel<<<spans, kRedoThreads, 0, s>>>(a.status, a.n, count, list);
      rc = check_cuda(cudaGetLastError(), "chain compaction launch");
    }
    if (rc == KF_OK) {
      chain_redo_list_kernel<<<(unsigned)(kRedoListBlocksPerSm * sms), 32, 0, s>>>(a, count,
                                                                                  list);
      rc = check_cuda(cudaGetLastError(), "chain redo pass launch");
    }
    const cudaError_t freed = cudaFreeAsync(buf, s);  // returned to the pool on every path
    return rc != KF_OK ? rc : check_cuda(freed, "cudaFreeAsync");
  }
  clear_error();
  (void)cudaGetLastError();  // a refused allocation is not the caller's error
  chain_redo_kernel<<<spans, kRedoThreads, 0, s>>>(a);
  return check_cuda(cudaGetLastError(), "chain redo pass launch");
}

}  // namespace
}  // namespace kf

extern "C" int kf_set_chain_redo(int32_t mode) {
  kf::clear_error();
  if (mode != KF_CHAIN_REDO_LIST && mode != KF_CHAIN_REDO_SPAN)
    return kf::set_error(KF_ERR_ARG, "chain redo mode %d is neither KF_CHAIN_REDO_LIST nor "
                         "KF_CHAIN_REDO_SPAN", mode);
  kf::g_chain_redo.store(mode, std::memory_order_relaxed);
  return KF_OK;
}

extern "C" int kf_kalman_chain(const kf_params *params, kf_layout layout, float *state,
                               float *cov, const int8_t *charge, const float *hits,
                               const float *hit_covs, const kf_layer *layers, int32_t L,
                               uint8_t *status, void *stream) {
  using namespace kf;
  clear_error();
  if (!params) return set_error(KF_ERR_ARG, "params is NULL");
  if (params->flags != 0) return set_error(KF_ERR_ARG, "params->flags must be 0");
  if (params->precision < KF_FP32 || params->precision > KF_DF_UPDATE)
    return set_error(KF_ERR_ARG, "unknown precision %d", params->precision);
  LayoutDesc d;
  if (int rc = check_layout(layout, &d)) return rc;
  if (L < 0 || L > KF_MAX_LAYERS)
    return set_error(KF_ERR_ARG, "L = %d not in [0, %d]", L, KF_MAX_LAYERS);
  if (d.n == 0 || L == 0) return KF_OK;
  if (!layers) return set_error(KF_ERR_ARG, "layers is NULL");
  ChainArgs a{};
  for (int l = 0; l < L; ++l) {
    if (layers[l].kind != KF_P2Z && layers[l].kind != KF_P2R)
      return set_error(KF_ERR_ARG, "layers[%d].kind = %d is neither KF_P2Z nor KF_P2R", l,
                       layers[l].kind);
    a.kinds[l] = layers[l].kind;
    a.pos[l] = layers[l].pos;
  }
  if (!aligned16(state) || !aligned16(cov) || !aligned16(hits) || !aligned16(hit_covs))
    return set_error(KF_ERR_ARG, "float arrays must be 16-byte aligned");
  const int64_t f3 = layout_floats(d, 3), f6 = layout_floats(d, 6), f21 = layout_floats(d, 21);
  if (int rc = check_device_range(state, 4 * f6, "state")) return rc;
  if (int rc = check_device_range(cov, 4 * f21, "cov")) return rc;
  if (int rc = check_device_range(charge, d.n, "charge")) return rc;
  if (int rc = check_device_range(hits, 4 * f3 * L, "hits")) return rc;
  if (int rc = check_device_range(hit_covs, 4 * f6 * L, "hit_covs")) return rc;
  if (status)
    if (int rc = check_device_range(status, d.n, "status")) return rc;
  if (!status && params->precision == KF_ADAPTIVE)
    return set_error(KF_ERR_ARG, "KF_ADAPTIVE needs a status array (its redo pass reads it)");

  a.state = state;
  a.cov = cov;
  a.charge = charge;
  a.hits = hits;
  a.hitcovs = hit_covs;
  a.status = status;
  a.n = d.n;
  a.hit_stride = f3;
  a.hc_stride = f6;
  a.soa = d.soa;
  a.lw = d.lw;
  a.bz = params->bz;
  a.L = L;
  LaunchConfig cfg{KF_STEP_DIRECT, 256, 0};
  if (const LaunchConfig *o = thread_override()) {
    cfg = *o;
  } else {
    LaunchConfig t;
    if (tune_lookup(kOpChain, 0, params->precision, d.soa, d.lw, d.n, &t)) cfg = t;
  }
  const int threads = (cfg.threads == 128 || cfg.threads == 64) ? cfg.threads : 256;
  const int64_t blocks = (d.n + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return set_error(KF_ERR_ARG, "n too large for one launch");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (params->precision) {
    case KF_FP32: chain_kernel<kFP32><<<(unsigned)blocks, threads, 0, s>>>(a); break;
    case KF_FP64_UPDATE: chain_kernel<kFP64Update><<<(unsigned)blocks, threads, 0, s>>>(a); break;
    case KF_JOSEPH: chain_kernel<kJoseph><<<(unsigned)blocks, threads, 0, s>>>(a); break;
    case KF_FP64: chain_kernel<kFP64><<<(unsigned)blocks, threads, 0, s>>>(a); break;
    case KF_DF_UPDATE: chain_kernel<kDFUpdate><<<(unsigned)blocks, threads, 0, s>>>(a); break;
    default: chain_mark_kernel<<<(unsigned)blocks, threads, 0, s>>>(a); break;
  }
  if (int rc = check_cuda(cudaGetLastError(), "chain launch")) return rc;
  if (params->precision != KF_ADAPTIVE) return KF_OK;
  return launch_chain_redo(a, s);
}
