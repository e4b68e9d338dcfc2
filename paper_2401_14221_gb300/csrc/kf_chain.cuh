// kf_chain.cuh -- per-track body of the multi-layer chain (paper section 2
// and the layer loop of Figs. 3-5: propagateTo{Z,R} then KalmanUpdate for
// every layer), shared by the single-launch chain kernel and the serving
// loop's batched kernel.
#pragma once

#include <cstdint>

#include "kf_device.cuh"

namespace kf {

struct ChainLoc {
  int64_t base;
  int64_t stride;
};

// Element (c, i) of a C-component array sits at base + c * stride.
template <int C>
__device__ __forceinline__ ChainLoc chain_locate(int64_t i, int64_t n, int32_t soa, int32_t lw) {
  if (soa) return {i, n};
  const int64_t W = int64_t(1) << lw;
  return {(i >> lw) * (C * W) + (i & (W - 1)), W};
}

struct LayerHit {
  float hx, hy, hz, hc[6];
};

// Walks one track's hit and hit covariance through the layers: pointers to
// the track's element of the current layer, advanced by the per-layer strides
// (no index arithmetic per layer beyond two pointer increments).
struct HitCursor {
  const float *hp, *cp;
  int64_t s3, s6, hit_stride, hc_stride;

  __device__ __forceinline__ HitCursor(const float *hits, int64_t hit_stride_,
                                       const float *hitcovs, int64_t hc_stride_,
                                       const ChainLoc &l3, const ChainLoc &l6)
      : hp(hits + l3.base), cp(hitcovs + l6.base), s3(l3.stride), s6(l6.stride),
        hit_stride(hit_stride_), hc_stride(hc_stride_) {}

  __device__ __forceinline__ void load(LayerHit &h) const {
    h.hx = __ldg(hp);
    h.hy = __ldg(hp + s3);
    h.hz = __ldg(hp + 2 * s3);
#pragma unroll
    for (int c = 0; c < 6; ++c) h.hc[c] = __ldg(cp + c * s6);
  }
  // What a layer of the given kind measures: a plane only x, y and their
  // 2x2 covariance (the rest is set to 0 and not read).
  __device__ __forceinline__ void load(LayerHit &h, int kind) const {
    if (kind != kP2z) {
      load(h);
      return;
    }
    h.hx = __ldg(hp);
    h.hy = __ldg(hp + s3);
    h.hz = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) h.hc[c] = __ldg(cp + c * s6);
    h.hc[3] = h.hc[4] = h.hc[5] = 0.0f;
  }
  __device__ __forceinline__ void next_layer() {
    hp += hit_stride;
    cp += hc_stride;
  }
};

// Run one track (p, C in registers) through layers 0..L-1 in float
// arithmetic (kFP32, kJoseph, kFP64Update, kDFUpdate); the next layer's hit is loaded
// while the current layer computes.  Returns the OR of the per-layer status
// bits.
template <int VARIANT>
__device__ __forceinline__ unsigned chain_track(float (&p)[6], float (&C)[21], float qf, float bz,
                                                int L, const int32_t *kinds, const float *pos,
                                                const float *hits, int64_t hit_stride,
                                                const float *hitcovs, int64_t hc_stride,
                                                const ChainLoc &l3, const ChainLoc &l6) {
  static_assert(VARIANT == kFP32 || VARIANT == kJoseph || VARIANT == kFP64Update ||
                    VARIANT == kDFUpdate,
                "float-state chain variants only");
  unsigned st = 0;
  HitCursor cur(hits, hit_stride, hitcovs, hc_stride, l3, l6);
  LayerHit next;
  cur.load(next, kinds[0]);
  for (int l = 0; l < L; ++l) {
    const LayerHit h = next;
    if (l + 1 < L) {
      cur.next_layer();
      cur.load(next, kinds[l + 1]);
    }
    if (kinds[l] == kP2z)
      st |= p2z_step<VARIANT>(p, C, qf, bz, pos[l], h.hx, h.hy, h.hc[0], h.hc[1], h.hc[2]);
    else
      st |= p2r_step<VARIANT>(p, C, qf, bz, pos[l], h.hx, h.hy, h.hz, h.hc);
  }
  return st;
}

// The whole chain in double: the state and covariance are converted once,
// kept in double registers across all layers and converted back once.  No
// FP32 rounding happens between layers -- a crossing at grazing incidence
// amplifies any error in its input by 1/cos(incidence), which reached 250 on
// the outermost barrel layer for tracks that barely reach it.  Serves
// kFP64 and the redo pass of kAdaptive.
__device__ __forceinline__ unsigned chain_track_fp64(float (&pf)[6], float (&Cf)[21], float qf,
                                                     float bz, int L, const int32_t *kinds,
                                                     const float *pos, const float *hits,
                                                     int64_t hit_stride, const float *hitcovs,
                                                     int64_t hc_stride, const ChainLoc &l3,
                                                     const ChainLoc &l6) {
  double p[6], C[21];
  for (int c = 0; c < 6; ++c) p[c] = pf[c];
  for (int e = 0; e < 21; ++e) C[e] = Cf[e];
  unsigned st = 0;
  HitCursor cur(hits, hit_stride, hitcovs, hc_stride, l3, l6);
  for (int l = 0; l < L; ++l, cur.next_layer()) {
    LayerHit h;
    cur.load(h, kinds[l]);
    double hc[6], rcos;
    bool shrink;
    for (int c = 0; c < 6; ++c) hc[c] = h.hc[c];
    if (kinds[l] == kP2z)
      st |= p2z_step_t<double, kStandard>(p, C, (double)qf, (double)bz, (double)pos[l],
                                          (double)h.hx, (double)h.hy, hc[0], hc[1], hc[2],
                                          shrink);
    else
      st |= p2r_step_t<double, kStandard>(p, C, (double)qf, (double)bz, (double)pos[l],
                                          (double)h.hx, (double)h.hy, (double)h.hz, hc, shrink,
                                          rcos);
  }
  for (int c = 0; c < 6; ++c) pf[c] = (float)p[c];
  for (int e = 0; e < 21; ++e) Cf[e] = (float)C[e];
  return st;
}

// KF_ADAPTIVE's first pass: the chain in FP32 that gives up on the track at
// the first ill-conditioned layer and returns kRedo (p and C are then
// scratch; the caller stores nothing, so the track's inputs stay intact for
// the redo pass, which reruns the whole chain with chain_track_fp64).  Other
// tracks finish here at the FP32 cost, with no FP64 code in this kernel's
// register allocation.
__device__ __forceinline__ unsigned chain_track_marking(float (&p)[6], float (&C)[21], float qf,
                                                        float bz, int L, const int32_t *kinds,
                                                        const float *pos, const float *hits,
                                                        int64_t hit_stride, const float *hitcovs,
                                                        int64_t hc_stride, const ChainLoc &l3,
                                                        const ChainLoc &l6) {
  unsigned st = 0;
  HitCursor cur(hits, hit_stride, hitcovs, hc_stride, l3, l6);
  LayerHit next;
  cur.load(next, kinds[0]);
  for (int l = 0; l < L; ++l) {
    const LayerHit h = next;
    if (l + 1 < L) {
      cur.next_layer();
      cur.load(next, kinds[l + 1]);
    }
    const unsigned sl =
        kinds[l] == kP2z
            ? p2z_step<kAdaptive>(p, C, qf, bz, pos[l], h.hx, h.hy, h.hc[0], h.hc[1], h.hc[2])
            : p2r_step<kAdaptive>(p, C, qf, bz, pos[l], h.hx, h.hy, h.hz, h.hc);
    if (sl & kRedo) return kRedo;
    st |= sl;
  }
  return st;
}

}  // namespace kf
