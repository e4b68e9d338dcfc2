// kf_step.cuh -- arguments of the single-step kernel and its launcher,
// shared by the device-pointer and host-pointer entry points.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

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
};

// Launch the p2z (kind 0) or p2r (kind 1) step kernel for `a` on stream s
// with the given KF_FP32 / KF_FP64_UPDATE / KF_JOSEPH variant.
int launch_step_kernel(int kind, int precision, const StepArgs &a, cudaStream_t s);

// The persistent bulk-async-staged kernel (AoSoA layouts only).
int launch_step_staged(int kind, int precision, const StepArgs &a, cudaStream_t s);

// Process-wide choice between the kernels: KF_STEP_AUTO / _DIRECT / _STAGED.
int step_kernel_mode();

}  // namespace kf
