// kf_host.cuh -- the direct path shared by the host-array entry points
// (kf_p2*_propagate_update_host and kf_propagate_update_host_noalloc).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kf_common.cuh"

namespace kf {

// The arrays of one host-array call, as the caller passed them.
struct HostArrays {
  const float *state_in, *cov_in;
  float *state_out, *cov_out;
  const int8_t *charge;
  const float *hit, *hit_cov, *surf;
  int32_t surf_per_track;
  uint8_t *status;  // may be NULL
};

// Process-wide KF_HOST_* mode (kf_set_host_path).
int host_path_mode();

// The direct path: when the mode allows it and every array can be read and
// written in place by a kernel on the current device (host_reach), launch
// the step on the caller's arrays themselves -- the one-thread-per-track
// kernel, whose loads and stores cross the CPU-GPU link -- on stream s and
// set *taken.  A KF_ADAPTIVE call without a status array keeps its redo marks
// in `scratch` (device memory of scratch_bytes >= n bytes); without one it is
// left to the copy path.  With KF_OK and *taken false the copy path serves
// the call (KF_HOST_AUTO only; under KF_HOST_DIRECT that case is
// KF_ERR_ARG).
int host_direct(int kind, const kf_params &params, const LayoutDesc &d, const HostArrays &h,
                uint8_t *scratch, int64_t scratch_bytes, cudaStream_t s, bool *taken);

}  // namespace kf
