// kf_common.cuh -- host-side helpers shared by the C-ABI entry points:
// per-thread error messages, argument checks and the layout descriptor.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "kf.h"

namespace kf {

// Record a message for kf_last_error_string() and return `code`.
int set_error(int code, const char *fmt, ...);
void clear_error();

// Map a CUDA error to KF_ERR_CUDA with its message (KF_OK if none).
int check_cuda(cudaError_t e, const char *what);

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Validated layout: element (c, i) of a C-component array sits at
// base(i) + c * stride with base/stride given by locate<C>() on the device.
struct LayoutDesc {
  int64_t n;
  int32_t soa;  // 1: [C][n]; 0: AoSoA blocks of 2^lw tracks
  int32_t lw;   // log2 of the AoSoA block width
};

// Validate a kf_layout; returns KF_OK and fills `out`, or KF_ERR_ARG.
int check_layout(const kf_layout &layout, LayoutDesc *out);

// Number of floats a C-component array occupies under the layout.
inline int64_t layout_floats(const LayoutDesc &d, int C) {
  if (d.soa) return (int64_t)C * d.n;
  const int64_t W = int64_t(1) << d.lw;
  return ((d.n + W - 1) / W) * W * C;
}

// KF_OK when [p, p + bytes) is memory a kernel may read or write: device
// or managed memory lying wholly inside one live allocation, or registered
// (pinned) host memory.  KF_ERR_ARG for NULL, pageable host memory, an
// address CUDA does not know, or a range running past the end of its
// allocation -- so that a wrong pointer or a short buffer is refused on the
// host instead of faulting the GPU.
int check_device_range(const void *p, int64_t bytes, const char *name);

// True when [a, a+na) and [b, b+nb) overlap but do not coincide.
inline bool partial_overlap(const void *a, int64_t na, const void *b, int64_t nb) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  if (a0 == b0) return false;
  return a0 < b0 + (uintptr_t)nb && b0 < a0 + (uintptr_t)na;
}

}  // namespace kf
