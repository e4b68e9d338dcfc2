// kf_compressed.cuh -- the compressed covariance store shared by the
// one-thread-per-track and the staged compressed kernels: per track six FP32
// standard deviations sigma_i = sqrt(C_ii) and fifteen FP16 correlations
// rho_ij = C_ij / (sigma_i sigma_j), packed order 10, 20, 21, 30, ..., 54
// (rho_0 .. rho_14).
//
// The correlations are stored in pairs: per block of W tracks (an AoSoA
// block; SoA is one block of n tracks) seven rows of W 32-bit words, word r
// of row p holding track r's (rho_2p, rho_2p+1) with rho_2p in the low half,
// then one row of W FP16 values rho_14 -- 15 W halves per block, the size of
// fifteen FP16 rows.  A thread then moves its correlations with seven 32-bit
// and one 16-bit access instead of fifteen 16-bit ones, and converts and
// clamps them two at a time.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "kf_device.cuh"

namespace kf {

struct CompressedArgs {
  const float *state_in;
  const float *sigma_in;
  const __half *rho_in;
  float *state_out;
  float *sigma_out;
  __half *rho_out;
  const int8_t *charge;
  const float *hit;
  const float *hitcov;
  const float *surf;
  uint8_t *status;
  int64_t n;
  int32_t soa;
  int32_t lw;
  float bz;
  int32_t surf_per_track;
};

// Off-diagonal (row, column) of correlation k, packed order.
__device__ __forceinline__ constexpr int od_row(int k) {
  return k < 1 ? 1 : k < 3 ? 2 : k < 6 ? 3 : k < 10 ? 4 : 5;
}
__device__ __forceinline__ constexpr int od_col(int k) {
  return k - (od_row(k) * (od_row(k) - 1)) / 2;
}

// One track's correlations in registers: the seven pairs as stored and
// rho_14.
struct Rho {
  __half2 pr[7];
  __half last;
};

// Where track i's correlations sit in the rho array (see the layout above).
struct RhoLoc {
  int64_t word;    // 32-bit word of pair 0
  int64_t stride;  // words from one pair row to the next
  int64_t last;    // FP16 element of rho_14
};

__device__ __forceinline__ RhoLoc locate_rho(int64_t i, int64_t n, int32_t soa, int32_t lw) {
  if (soa) return {i, n, 14 * n + i};
  const int64_t W = int64_t(1) << lw, blk = i >> lw, r = i & (W - 1);
  return {blk * (15 * W / 2) + r, W, blk * (15 * W) + 14 * W + r};
}

__device__ __forceinline__ void load_rho(const __half *rho, const RhoLoc &l, Rho &rh) {
  const __half2 *w = reinterpret_cast<const __half2 *>(rho);
#pragma unroll
  for (int p = 0; p < 7; ++p) rh.pr[p] = w[l.word + p * l.stride];
  rh.last = rho[l.last];
}

// streaming stores, as the kernels' other outputs
__device__ __forceinline__ void store_rho(__half *rho, const RhoLoc &l, const Rho &rh) {
  __half2 *w = reinterpret_cast<__half2 *>(rho);
#pragma unroll
  for (int p = 0; p < 7; ++p) __stcs(w + l.word + p * l.stride, rh.pr[p]);
  __stcs(rho + l.last, rh.last);
}

// C_ii = sigma_i^2, C_ij = rho_ij sigma_i sigma_j (FP32).  Each product is
// rounded on its own (__fmul_rn): left as a plain multiply, the compiler may
// fuse it with an addition of the transport that follows into one FMA, and
// whether it does depends on the surrounding kernel, so the staged and the
// one-thread-per-track kernels would round differently.
__device__ __forceinline__ void decode_cov(const float (&sg)[6], const Rho &rh, float (&C)[21]) {
  float r[15];
#pragma unroll
  for (int p = 0; p < 7; ++p) {
    const float2 f = __half22float2(rh.pr[p]);
    r[2 * p] = f.x;
    r[2 * p + 1] = f.y;
  }
  r[14] = __half2float(rh.last);
#pragma unroll
  for (int c = 0; c < 6; ++c) C[tri(c, c)] = __fmul_rn(sg[c], sg[c]);
#pragma unroll
  for (int k = 0; k < 15; ++k)
    C[tri(od_row(k), od_col(k))] = __fmul_rn(__fmul_rn(r[k], sg[od_row(k)]), sg[od_col(k)]);
}

// sigma_i = sqrt(C_ii), rho_ij = C_ij / (sigma_i sigma_j) clamped to [-1, 1]
// and rounded to nearest (0 where a sigma is 0).  One reciprocal square root
// per variance gives both 1/sigma and sigma = C_ii / sigma (a few ulp, far
// below the 2^-12 of the FP16 correlations).  The pairs are rounded to FP16
// first and clamped there: +-1 are FP16 values, so rounding and clamping
// commute (a quotient above 1 rounds to 1 or above and is clamped to 1; a
// NaN quotient becomes -1 either way, min and max returning the non-NaN
// operand).
__device__ __forceinline__ void encode_cov(const float (&C)[21], float (&sg)[6], Rho &rh) {
  float inv[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const float v = fmaxf(C[tri(c, c)], 0.0f);
    inv[c] = v > 0.0f ? rsqrtf(v) : 0.0f;
    sg[c] = v * inv[c];
  }
  float r[15];
#pragma unroll
  for (int k = 0; k < 15; ++k)
    r[k] = C[tri(od_row(k), od_col(k))] * inv[od_row(k)] * inv[od_col(k)];
  const __half2 lo = __float2half2_rn(-1.0f), hi = __float2half2_rn(1.0f);
#pragma unroll
  for (int p = 0; p < 7; ++p)
    rh.pr[p] = __hmin2(__hmax2(__floats2half2_rn(r[2 * p], r[2 * p + 1]), lo), hi);
  rh.last = __float2half_rn(fminf(fmaxf(r[14], -1.0f), 1.0f));
}

// The staged (bulk-copy) compressed step for AoSoA layouts; KF_ERR_UNSUPPORTED
// for SoA (the caller then runs the one-thread-per-track kernel).
int launch_compressed_staged(int kind, int precision, const CompressedArgs &a, cudaStream_t s);

}  // namespace kf
