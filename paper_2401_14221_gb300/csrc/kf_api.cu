// kf_api.cu -- library-wide C-ABI functions and host helpers: version,
// per-thread error strings and layout validation.
#include <cstdarg>
#include <cstdio>
#include <cstring>

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
// cuMemGetAddressRange (driver API) fetched through the runtime, so the
// library does not link libcuda directly.  CUdeviceptr is 64-bit.
typedef int (*MemRangeFn)(unsigned long long *base, size_t *size, unsigned long long ptr);

MemRangeFn mem_range_fn() {
  static MemRangeFn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<MemRangeFn>(f);
  }();
  return fn;
}
}  // namespace

int check_device_range(const void *p, int64_t bytes, const char *name) {
  if (!p) return set_error(KF_ERR_ARG, "%s is NULL", name);
  cudaPointerAttributes attr;
  const cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // this query's error is not sticky; clear it
    return set_error(KF_ERR_ARG, "%s: not a CUDA-visible pointer (%s)", name,
                     cudaGetErrorString(e));
  }
  if (attr.type == cudaMemoryTypeHost) return KF_OK;  // pinned host memory
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return set_error(KF_ERR_ARG, "%s: pageable host memory, not reachable from the GPU", name);
  MemRangeFn fn = mem_range_fn();
  if (!fn) return set_error(KF_ERR_CUDA, "cuMemGetAddressRange is unavailable");
  unsigned long long base = 0;
  size_t size = 0;
  const unsigned long long ptr = reinterpret_cast<uintptr_t>(p);
  if (fn(&base, &size, ptr) != 0)
    return set_error(KF_ERR_ARG, "%s: address is not inside a device allocation", name);
  if (bytes < 0 || ptr + (unsigned long long)bytes > base + size)
    return set_error(KF_ERR_ARG, "%s: needs %lld bytes but its allocation ends %lld bytes later",
                     name, (long long)bytes, (long long)(base + size - ptr));
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
