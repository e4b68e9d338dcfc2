// kf_step.cuh -- arguments of the single-step kernel and its launcher,
// shared by the device-pointer and host-pointer entry points.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kf_device.cuh"

namespace kf {

// Device pointers and sizes for one single-step launch (already validated).
struct StepArgs {
  const float *state_in;
  const float *cov_in;
  float *state_out;
  float *cov_out;
  const int8_t *charge;
  const float *hit;
  const float *hitcov;
  const float *surf;
  uint8_t *status;  // may be NULL
  int64_t n;
  int32_t soa;  // 1: [C][n] arrays; 0: AoSoA blocks of 2^lw tracks
  int32_t lw;
  float bz;
  int32_t surf_per_track;
  unsigned *err = nullptr;  // device error word (set by the staged launcher)
  // Polls of a staged-pipeline barrier by a compute warp before it gives up
  // (set by the staged launcher from kf_set_device_wait_limit).
  uint32_t wait_polls = 0;
};

#ifdef __CUDACC__
// The kAdaptive redo of track i of a step launch: read its inputs from
// global memory, run the step in double, write its outputs there and return
// its status (finite check included).  Used by the redo pass, a kernel of its
// own, so that the FP32 kernel's registers never carry the FP64 step.  In
// place is safe: the FP32 kernel did not store this track's result.
template <int KIND>
__device__ __forceinline__ unsigned redo_track_fp64(const StepArgs &a, int64_t i) {
  int64_t b6, b21, b3, s;
  if (a.soa) {
    b6 = b21 = b3 = i;
    s = a.n;
  } else {
    const int64_t W = int64_t(1) << a.lw, blk = i >> a.lw, r = i & (W - 1);
    b6 = blk * 6 * W + r;
    b21 = blk * 21 * W + r;
    b3 = blk * 3 * W + r;
    s = W;
  }
  double p[6], C[21], hc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, cinc;
  bool shrink;
#pragma unroll
  for (int c = 0; c < 6; ++c) p[c] = a.state_in[b6 + c * s];
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = a.cov_in[b21 + e * s];
  constexpr int nhc = KIND == kP2z ? 3 : 6;
#pragma unroll
  for (int c = 0; c < nhc; ++c) hc[c] = a.hitcov[b6 + c * s];
  const double qf = a.charge[i];
  const double surf = a.surf[a.surf_per_track ? i : 0];
  const double hx = a.hit[b3], hy = a.hit[b3 + s];
  unsigned st;
  if (KIND == kP2z)
    st = p2z_step_t<double, kStandard>(p, C, qf, (double)a.bz, surf, hx, hy, hc[0], hc[1], hc[2],
                                       shrink);
  else
    st = p2r_step_t<double, kStandard>(p, C, qf, (double)a.bz, surf, hx, hy,
                                       (double)a.hit[b3 + 2 * s], hc, shrink, cinc);
  // exact when the track was not propagated (float -> double -> float)
  float pf[6], Cf[21];
#pragma unroll
  for (int c = 0; c < 6; ++c) pf[c] = (float)p[c];
#pragma unroll
  for (int e = 0; e < 21; ++e) Cf[e] = (float)C[e];
  st |= finite_status(pf, Cf);
#pragma unroll
  for (int c = 0; c < 6; ++c) __stcs(a.state_out + b6 + c * s, pf[c]);
#pragma unroll
  for (int e = 0; e < 21; ++e) __stcs(a.cov_out + b21 + e * s, Cf[e]);
  return st;
}

// Status bytes base .. base+15 of an [n] array as four little-endian words:
// one 16-byte load where the array is 16-byte aligned and the run is whole,
// byte loads otherwise (bytes at or past n read as 0).
__device__ __forceinline__ uint4 load_status16(const uint8_t *status, int64_t base, int64_t n) {
  if (base + 16 <= n && (reinterpret_cast<uintptr_t>(status) & 15u) == 0)
    return *reinterpret_cast<const uint4 *>(status + base);
  uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (base + j < n) w[j >> 2] |= (uint32_t)status[base + j] << (8 * (j & 3));
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Redo passes gather the marked tracks of a span of kRedoSpan tracks into a
// shared-memory list before running them, so that each warp runs up to 32
// marked tracks instead of one marked track among 31 idle lanes: GB300
// issues an FP64 warp instruction over many cycles whether or not its lanes
// are active.  The pass is latency-bound (one FP64 warp per scheduler
// issues on 8 % of cycles), so its time is one warp's chain as long as every
// marked track runs in the first round: a block has kRedoThreads threads
// (the double-precision step takes about 190 registers; five 64-thread
// blocks fit an SM, so the 478 spans of a 1.96 M-track chain are resident
// at once), and a span is small enough that its marks rarely exceed the
// block's threads (about 0.6 % of chain tracks are marked: 24 per span on
// average).  256-thread blocks (one per SM) and 8,192-track spans (48 marks
// on average, some spans over 64) each took a second round and about
// doubled the pass.
constexpr int kRedoSpan = 4096;
constexpr int kRedoThreads = 64;

// Fill list[0..count) with the offsets (from span0) of the tracks marked
// kRedo among [span0, min(span0 + kRedoSpan, n)); returns the count.  Every
// thread of the block (kRedoThreads of them) must call it.  Each thread
// scans kRedoSpan / (16 kRedoThreads) runs of 16 status bytes, striding by
// the block; all its loads are issued before any is examined, so a span
// with nothing marked costs one memory latency.
__device__ __forceinline__ int gather_marked(const uint8_t *status, int64_t span0, int64_t n,
                                             uint16_t *list, int *count) {
  constexpr int kRuns = kRedoSpan / (16 * kRedoThreads);
  static_assert(kRuns * 16 * kRedoThreads == kRedoSpan, "whole runs per thread");
  static_assert(kRedoSpan <= 65536, "span offsets are 16-bit");
  constexpr uint32_t kMarks = 0x01010101u * kRedo;  // the kRedo bit of each byte
  if (threadIdx.x == 0) *count = 0;
  uint4 v[kRuns];
#pragma unroll
  for (int r = 0; r < kRuns; ++r) {
    const int64_t base = span0 + (int64_t)(r * kRedoThreads + threadIdx.x) * 16;
    v[r] = base < n ? load_status16(status, base, n) : make_uint4(0u, 0u, 0u, 0u);
  }
  __syncthreads();  // count is 0
#pragma unroll
  for (int r = 0; r < kRuns; ++r) {
    const uint32_t w[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
    if (((w[0] | w[1] | w[2] | w[3]) & kMarks) == 0u) continue;
    const int off = (r * kRedoThreads + threadIdx.x) * 16;
    for (int j = 0; j < 16; ++j)
      if ((w[j >> 2] >> (8 * (j & 3))) & kRedo) list[atomicAdd(count, 1)] = (uint16_t)(off + j);
  }
  __syncthreads();
  return *count;
}

#endif

// How a step (or chain) launch is shaped.
struct LaunchConfig {
  int kernel;       // KF_STEP_DIRECT or KF_STEP_STAGED
  int threads;      // CTA size of the one-thread-per-track kernels
  int ctas_per_sm;  // persistent CTAs per SM of the staged kernel
};

// Launch the p2z (kind 0) or p2r (kind 1) step kernel for `a` on stream s
// with the given KF_* precision variant.  The shape comes from, in order:
// the autotuner's per-thread override while it measures, the process-wide
// kf_set_step_kernel mode, the tuning cache, the defaults.  plain_loads
// (arrays in host or managed memory) overrides all of them: the
// one-thread-per-track kernel, 256 threads per CTA.
int launch_step_kernel(int kind, int precision, const StepArgs &a, cudaStream_t s,
                       bool plain_loads = false);

// Second pass of KF_ADAPTIVE: redo in FP64 every track whose status the
// step kernel marked with kRedo (those tracks' outputs are not yet written).
int launch_redo_pass(int kind, const StepArgs &a, cudaStream_t s);

// The persistent bulk-async-staged kernel (AoSoA layouts only).
int launch_step_staged(int kind, int precision, const StepArgs &a, cudaStream_t s,
                       int ctas_per_sm);

// Process-wide choice between the kernels: KF_STEP_AUTO / _DIRECT / _STAGED.
int step_kernel_mode();

// ------------------------------------------------------------- tuning
enum TuneOp : int { kOpStep = 0, kOpChain = 1 };

// Shape forced on the calling thread's launches (the autotuner sets it
// while it measures candidates); nullptr when none.
const LaunchConfig *thread_override();
void set_thread_override(const LaunchConfig *cfg);

// Cached best shape for (current device, op, kind, precision, layout, n).
bool tune_lookup(int op, int kind, int precision, int soa, int lw, int64_t n, LaunchConfig *out);
void tune_store(int op, int kind, int precision, int soa, int lw, int64_t n,
                const LaunchConfig &cfg, float ms);

}  // namespace kf
