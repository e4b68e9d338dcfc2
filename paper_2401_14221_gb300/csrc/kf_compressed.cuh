// kf_compressed.cuh -- the compressed covariance store shared by the
// one-thread-per-track and the staged compressed kernels: per track six FP32
// standard deviations sigma_i = sqrt(C_ii) and fifteen FP16 correlations
// rho_ij = C_ij / (sigma_i sigma_j), packed order 10, 20, 21, 30, ..., 54.
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

// C_ii = sigma_i^2, C_ij = rho_ij sigma_i sigma_j (FP32).  Each product is
// rounded on its own (__fmul_rn): left as a plain multiply, the compiler may
// fuse it with an addition of the transport that follows into one FMA, and
// whether it does depends on the surrounding kernel, so the staged and the
// one-thread-per-track kernels would round differently.
__device__ __forceinline__ void decode_cov(const float (&sg)[6], const __half (&rh)[15],
                                           float (&C)[21]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) C[tri(c, c)] = __fmul_rn(sg[c], sg[c]);
#pragma unroll
  for (int k = 0; k < 15; ++k)
    C[tri(od_row(k), od_col(k))] =
        __fmul_rn(__fmul_rn(__half2float(rh[k]), sg[od_row(k)]), sg[od_col(k)]);
}

// sigma_i = sqrt(C_ii), rho_ij = C_ij / (sigma_i sigma_j) clamped to [-1, 1]
// and rounded to nearest (0 where a sigma is 0).  One reciprocal square root
// per variance gives both 1/sigma and sigma = C_ii / sigma (a few ulp, far
// below the 2^-12 of the FP16 correlations).
__device__ __forceinline__ void encode_cov(const float (&C)[21], float (&sg)[6],
                                           __half (&rh)[15]) {
  float inv[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const float v = fmaxf(C[tri(c, c)], 0.0f);
    inv[c] = v > 0.0f ? rsqrtf(v) : 0.0f;
    sg[c] = v * inv[c];
  }
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    const float r = C[tri(od_row(k), od_col(k))] * inv[od_row(k)] * inv[od_col(k)];
    rh[k] = __float2half_rn(fminf(fmaxf(r, -1.0f), 1.0f));
  }
}

// The staged (bulk-copy) compressed step for AoSoA layouts; KF_ERR_UNSUPPORTED
// for SoA (the caller then runs the one-thread-per-track kernel).
int launch_compressed_staged(int kind, int precision, const CompressedArgs &a, cudaStream_t s);

}  // namespace kf
