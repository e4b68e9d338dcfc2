// kf_api.cu -- library-wide C-ABI functions and host helpers: version,
// per-thread error strings and layout validation.
#include <cerrno>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <atomic>

#include <cuda.h>  // driver API types and attribute names only; not linked
#include <sys/mman.h>
#include <unistd.h>

#include "kf_common.cuh"

namespace kf {

namespace {
thread_local char g_error[512] = "";
}

int set_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_error, sizeof(g_error), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_error[0] = '\0'; }

int check_cuda(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return KF_OK;
  return set_error(KF_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

namespace {
// Driver API functions fetched through the runtime, so the library does not
// link libcuda directly.
typedef CUresult (*MemRangeFn)(CUdeviceptr *base, size_t *size, CUdeviceptr ptr);
typedef CUresult (*PtrAttrFn)(void *data, CUpointer_attribute attribute, CUdeviceptr ptr);

void *driver_fn(const char *name) {
  void *f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    f = nullptr;
  }
  return f;
}

MemRangeFn mem_range_fn() {
  static MemRangeFn fn = reinterpret_cast<MemRangeFn>(driver_fn("cuMemGetAddressRange"));
  return fn;
}

PtrAttrFn ptr_attr_fn() {
  static PtrAttrFn fn = reinterpret_cast<PtrAttrFn>(driver_fn("cuPointerGetAttribute"));
  return fn;
}

int check_end(const char *name, uintptr_t ptr, int64_t bytes, uintptr_t base, size_t size) {
  if (bytes < 0 || ptr + (uint64_t)bytes > base + size)
    return set_error(KF_ERR_ARG, "%s: needs %lld bytes but its allocation ends %lld bytes later",
                     name, (long long)bytes, (long long)(base + size - ptr));
  return KF_OK;
}

// Whether kernels on device `dev` may dereference pageable host memory
// (the device walks the host page tables: address translation services on
// a CPU-GPU coherent link).  Asked once per device.
constexpr int kMaxDevices = 64;
std::atomic<int> g_pageable_access[kMaxDevices];  // 0 unknown, 1 no, 2 yes

bool pageable_access(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return false;
  int v = g_pageable_access[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    int a = 0, b = 0;
    const bool ok =
        cudaDeviceGetAttribute(&a, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&b, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) ==
            cudaSuccess;
    if (!ok) cudaGetLastError();
    v = (ok && a && b) ? 2 : 1;
    g_pageable_access[dev].store(v, std::memory_order_relaxed);
  }
  return v == 2;
}

// True when every page of [p, p + bytes) is mapped in this process
// (mincore fails with ENOMEM on a range that holds unmapped pages).
bool host_range_mapped(const void *p, int64_t bytes) {
  static const uintptr_t page = (uintptr_t)sysconf(_SC_PAGESIZE);
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t first = a & ~(page - 1);
  const uintptr_t len = a + (uintptr_t)(bytes > 0 ? bytes : 1) - first;
  thread_local std::vector<unsigned char> vec;
  vec.resize((len + page - 1) / page);
  return mincore(reinterpret_cast<void *>(first), len, vec.data()) == 0;
}
}  // namespace

int check_device_range(const void *p, int64_t bytes, const char *name, bool *not_device) {
  if (!p) return set_error(KF_ERR_ARG, "%s is NULL", name);
  cudaPointerAttributes attr;
  const cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // this query's error is not sticky; clear it
    return set_error(KF_ERR_ARG, "%s: not a CUDA-visible pointer (%s)", name,
                     cudaGetErrorString(e));
  }
  const uintptr_t ptr = reinterpret_cast<uintptr_t>(p);
  if (attr.type == cudaMemoryTypeHost && attr.devicePointer == nullptr) {
    // A host thread that has made no CUDA call yet has no context bound, and
    // page-locked memory then reports no device address: bind the thread's
    // current device and ask again.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess ||
        cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
      cudaGetLastError();
      return set_error(KF_ERR_ARG, "%s: page-locked memory not reachable from this thread's "
                       "device", name);
    }
  }
  if (attr.type == cudaMemoryTypeHost) {  // page-locked host memory
    if (attr.devicePointer != p)
      return set_error(KF_ERR_ARG, "%s: page-locked memory whose device address (%p) differs "
                       "from its host address (%p)", name, attr.devicePointer, p);
    PtrAttrFn fn = ptr_attr_fn();
    if (!fn) return set_error(KF_ERR_CUDA, "cuPointerGetAttribute is unavailable");
    CUdeviceptr base = 0;
    size_t size = 0;
    if (fn(&base, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)ptr) != CUDA_SUCCESS ||
        fn(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)ptr) != CUDA_SUCCESS)
      return set_error(KF_ERR_ARG, "%s: the extent of its page-locked allocation is unknown", name);
    if (int rc = check_end(name, ptr, bytes, (uintptr_t)base, size)) return rc;
    if (not_device) *not_device = true;
    return KF_OK;
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return set_error(KF_ERR_ARG, "%s: pageable host memory, not reachable from the GPU", name);
  MemRangeFn fn = mem_range_fn();
  if (!fn) return set_error(KF_ERR_CUDA, "cuMemGetAddressRange is unavailable");
  CUdeviceptr base = 0;
  size_t size = 0;
  if (fn(&base, &size, (CUdeviceptr)ptr) != CUDA_SUCCESS)
    return set_error(KF_ERR_ARG, "%s: address is not inside a device allocation", name);
  if (int rc = check_end(name, ptr, bytes, (uintptr_t)base, size)) return rc;
  if (not_device) *not_device = attr.type == cudaMemoryTypeManaged;
  return KF_OK;
}

int check_device_memory(const void *p, int64_t bytes, const char *name) {
  bool not_device = false;
  if (int rc = check_device_range(p, bytes, name, &not_device)) return rc;
  if (not_device) return set_error(KF_ERR_ARG, "%s must be device memory", name);
  return KF_OK;
}

int host_reach(const void *p, int64_t bytes, int align, const char *name, bool *direct,
               int dev) {
  *direct = false;
  if (!p) return set_error(KF_ERR_ARG, "%s is NULL", name);
  const bool aligned = (reinterpret_cast<uintptr_t>(p) % (uintptr_t)align) == 0;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    attr.type = cudaMemoryTypeUnregistered;
  }
  if (attr.type != cudaMemoryTypeUnregistered) {
    if (int rc = check_device_range(p, bytes, name)) return rc;
    *direct = aligned;
    return KF_OK;
  }
  if (!host_range_mapped(p, bytes))
    return set_error(KF_ERR_ARG, "%s: [%p, +%lld bytes) is not mapped host memory", name, p,
                     (long long)bytes);
  if (dev < 0)
    if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
  *direct = aligned && pageable_access(dev);
  return KF_OK;
}

int check_layout(const kf_layout &layout, LayoutDesc *out) {
  if (layout.n < 0) return set_error(KF_ERR_ARG, "layout.n = %lld < 0", (long long)layout.n);
  out->n = layout.n;
  if (layout.kind == KF_SOA) {
    out->soa = 1;
    out->lw = 0;
    return KF_OK;
  }
  if (layout.kind != KF_AOSOA)
    return set_error(KF_ERR_ARG, "layout.kind = %d is neither KF_SOA nor KF_AOSOA", layout.kind);
  out->soa = 0;
  switch (layout.width) {
    case 16: out->lw = 4; break;
    case 32: out->lw = 5; break;
    case 64: out->lw = 6; break;
    case 128: out->lw = 7; break;
    default:
      return set_error(KF_ERR_ARG, "AoSoA width %d not in {16, 32, 64, 128}", layout.width);
  }
  return KF_OK;
}

}  // namespace kf

extern "C" int kf_version(void) { return KF_VERSION; }

extern "C" const char *kf_last_error_string(void) { return kf::g_error; }
