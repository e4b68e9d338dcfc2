// kf_step_staged.cu -- dispatch of the persistent staged step kernel
// (kf_step_staged.cuh) and the library's device error word.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "kf_step_staged.cuh"

namespace kf {

// Device error word: bounded waits that time out OR their KF_DEVERR_* bit
// into it (the kernels get its address).
__device__ unsigned int g_device_error = 0;

namespace staged {

std::mutex g_sm_mu;
int g_sm_count[64] = {};

// Polls of a pipeline barrier by a compute warp before it gives up
// (kf_set_device_wait_limit).
std::atomic<uint32_t> g_wait_polls{kMaxPolls};

uint32_t device_wait_polls() { return g_wait_polls.load(std::memory_order_relaxed); }

// Device address of g_device_error, looked up once per device.
std::atomic<unsigned *> g_err_addr[64] = {};

int error_word(int dev, unsigned **out) {
  if (dev >= 0 && dev < 64) {
    if (unsigned *p = g_err_addr[dev].load(std::memory_order_acquire)) {
      *out = p;
      return KF_OK;
    }
  }
  void *p = nullptr;
  if (int rc = check_cuda(cudaGetSymbolAddress(&p, g_device_error), "cudaGetSymbolAddress"))
    return rc;
  if (dev >= 0 && dev < 64)
    g_err_addr[dev].store(static_cast<unsigned *>(p), std::memory_order_release);
  *out = static_cast<unsigned *>(p);
  return KF_OK;
}

int sm_count(int dev, int *out) {
  std::lock_guard<std::mutex> lock(g_sm_mu);
  if (dev >= 0 && dev < 64 && g_sm_count[dev] > 0) {
    *out = g_sm_count[dev];
    return KF_OK;
  }
  int v = 0;
  if (int rc = check_cuda(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev),
                          "cudaDeviceGetAttribute"))
    return rc;
  if (dev >= 0 && dev < 64) g_sm_count[dev] = v;
  *out = v;
  return KF_OK;
}

}  // namespace staged

// Persistent staged launch for AoSoA layouts: one or two CTAs per SM,
// tiles scheduled as in Schedule.
int launch_step_staged(int kind, int precision, const StepArgs &a, cudaStream_t s,
                       int ctas_per_sm) {
  using namespace staged;
  if (a.n == 0) return KF_OK;
  if (a.soa && (a.n & 3))
    return set_error(KF_ERR_UNSUPPORTED, "the staged kernel takes SoA only for n a multiple of 4");
  int dev = 0, sms = 0;
  if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
  if (int rc = sm_count(dev, &sms)) return rc;
  const int64_t ntiles = (a.n + kT - 1) / kT;
  const int ctas = (ctas_per_sm == 1 || ctas_per_sm == 3) ? ctas_per_sm : 2;
  const bool three = ctas == 3 && (precision == KF_FP32 || precision == KF_ADAPTIVE ||
                                   precision == KF_JOSEPH);
  const int64_t slots = (int64_t)sms * (three ? 3 : (ctas == 1 ? 1 : 2));
  const int grid = (int)(ntiles < slots ? ntiles : slots);
  StepArgs b = a;
  if (int rc = error_word(dev, &b.err)) return rc;
  b.wait_polls = device_wait_polls();
  const bool f64 = precision == KF_FP64_UPDATE || precision == KF_FP64;
  if (kind == kP2z)
    return f64 ? launch_staged_p2z_f64(precision, b, s, grid, dev, ctas)
               : launch_staged_p2z_f32(precision, b, s, grid, dev, ctas);
  return f64 ? launch_staged_p2r_f64(precision, b, s, grid, dev, ctas)
             : launch_staged_p2r_f32(precision, b, s, grid, dev, ctas);
}

}  // namespace kf

extern "C" int kf_set_device_wait_limit(int64_t polls) {
  kf::clear_error();
  if (polls < -1 || polls > (int64_t)kf::staged::kMaxPolls)
    return kf::set_error(KF_ERR_ARG, "wait limit %lld is not -1 or 0..%u", (long long)polls,
                         kf::staged::kMaxPolls);
  kf::staged::g_wait_polls.store(polls < 0 ? kf::staged::kMaxPolls : (uint32_t)polls,
                                 std::memory_order_relaxed);
  return KF_OK;
}

extern "C" int kf_take_device_error(unsigned int *error_bits) {
  kf::clear_error();
  if (!error_bits) return kf::set_error(KF_ERR_ARG, "error_bits is NULL");
  unsigned int v = 0, zero = 0;
  if (int rc = kf::check_cuda(cudaMemcpyFromSymbol(&v, kf::g_device_error, sizeof(v)),
                              "read device error word"))
    return rc;
  if (int rc = kf::check_cuda(cudaMemcpyToSymbol(kf::g_device_error, &zero, sizeof(zero)),
                              "clear device error word"))
    return rc;
  *error_bits = v;
  return KF_OK;
}
