// kf_selftest.cu -- entry points that expose pieces of the device arithmetic
// to the tests (no paper counterpart).
#include <cuda_runtime.h>

#include "kf_common.cuh"
#include "kf_device.cuh"

namespace kf {
namespace {

__global__ void __launch_bounds__(256) sincos_kernel(const float *x, float *s, float *c,
                                                     int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Fp<float>::sincos_(x[i], s + i, c + i);
}

}  // namespace
}  // namespace kf

extern "C" int kf_selftest_sincos(const float *x, float *s, float *c, int64_t n, void *stream) {
  using namespace kf;
  clear_error();
  if (n < 0) return set_error(KF_ERR_ARG, "n < 0");
  if (n == 0) return KF_OK;
  if (n > (int64_t)0x7fffffff * 256) return set_error(KF_ERR_ARG, "n too large");
  if (int rc = check_device_range(x, 4 * n, "x")) return rc;
  if (int rc = check_device_range(s, 4 * n, "s")) return rc;
  if (int rc = check_device_range(c, 4 * n, "c")) return rc;
  sincos_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      x, s, c, n);
  return check_cuda(cudaGetLastError(), "sincos self-test launch");
}
