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
// or managed memory, or page-locked host memory whose device address is its
// host address, lying wholly inside one live allocation.  KF_ERR_ARG for
// NULL, pageable host memory, an address CUDA does not know, or a range
// running past the end of its allocation -- so that a wrong pointer or a
// short buffer is refused on the host instead of faulting the GPU.  When
// `not_device` is given it is set for page-locked host and managed memory:
// those arrays are read with plain loads by the one-thread-per-track
// kernels, never by the bulk copies of the staged kernels.
int check_device_range(const void *p, int64_t bytes, const char *name,
                       bool *not_device = nullptr);

// As check_device_range, but only device memory proper (cudaMalloc'd or
// from a device memory pool) is accepted: workspaces and arenas.
int check_device_memory(const void *p, int64_t bytes, const char *name);

// For the host-array entries: KF_OK with *direct set when a kernel on the
// current device can read and write [p, p + bytes) in place -- device,
// managed or page-locked memory as check_device_range accepts it, or, on a
// device that reaches pageable memory through the host page tables, host
// memory that is mapped over the whole range -- and `align` divides p;
// KF_OK with *direct cleared when only the copy path can serve it; KF_ERR_ARG
// for NULL or a range that is short or not mapped.
// `dev` is the device whose kernels would do the access (-1: the calling
// thread's current device).
int host_reach(const void *p, int64_t bytes, int align, const char *name, bool *direct,
               int dev = -1);

// True when [a, a+na) and [b, b+nb) overlap but do not coincide.
inline bool partial_overlap(const void *a, int64_t na, const void *b, int64_t nb) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  if (a0 == b0) return false;
  return a0 < b0 + (uintptr_t)nb && b0 < a0 + (uintptr_t)na;
}

}  // namespace kf
