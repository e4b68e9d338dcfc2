// kf_host_noalloc.cu -- the host-array step for callers that cannot allocate
// device memory.
//
// Who needs it: a program that owns only host arrays and may not call
// cudaMalloc -- for example a plugin or a module inside a larger framework
// whose device allocator belongs to the host application, or a latency-
// critical loop where cudaMalloc's implicit device synchronisation is not
// acceptable.  kf_p2*_propagate_update_host needs a caller-provided device
// workspace; this variant instead stages the chunks through a fixed buffer
// that the library declares in device memory, so the call allocates nothing.
//
// Where every array is reachable in place from the GPU (page-locked memory,
// or pageable memory on a device that walks the host page tables) the
// shared direct path of the host-array calls serves the call instead, and
// nothing is staged.
//
// The staging buffer is a file-scope __device__ array: every GPU that loads
// the library holds it until the process exits.  Host code cannot use the
// array's name as a device address (it is a host-side stand-in), so its
// device address is looked up once per device with cudaGetSymbolAddress and
// the kernels are given that address.
#include <mutex>

#include <cuda_runtime.h>

#include "kf_common.cuh"
#include "kf_device.cuh"
#include "kf_host.cuh"
#include "kf_step.cuh"

namespace kf {
namespace {

constexpr int kNoallocMaxDevices = 64;

// Offsets of the staged arrays for KF_NOALLOC_MAX_CHUNK tracks.
struct StaticSlot {
  int64_t state_in, cov_in, hit, hitcov, state_out, cov_out, charge, status, surf, bytes;
};

constexpr StaticSlot static_slot() {
  StaticSlot s{};
  int64_t off = 0;
  const int64_t m = KF_NOALLOC_MAX_CHUNK;
  s.state_in = off; off += (4 * 6 * m + 255) & ~int64_t(255);
  s.cov_in = off; off += (4 * 21 * m + 255) & ~int64_t(255);
  s.hit = off; off += (4 * 3 * m + 255) & ~int64_t(255);
  s.hitcov = off; off += (4 * 6 * m + 255) & ~int64_t(255);
  s.state_out = off; off += (4 * 6 * m + 255) & ~int64_t(255);
  s.cov_out = off; off += (4 * 21 * m + 255) & ~int64_t(255);
  s.charge = off; off += (m + 255) & ~int64_t(255);
  s.status = off; off += (m + 255) & ~int64_t(255);
  s.surf = off; off += (4 * m + 255) & ~int64_t(255);
  s.bytes = off;
  return s;
}

constexpr StaticSlot kSlot = static_slot();
static_assert(kSlot.bytes == KF_NOALLOC_STAGING_BYTES,
              "KF_NOALLOC_STAGING_BYTES in kf.h must match the staged layout");

// The staging buffer.  Nothing in it needs to start at zero: every chunk's
// inputs are copied in before the kernel reads them and the kernel writes
// every output (and status) entry of the chunk before it is copied out.
static __device__ __align__(256) unsigned char g_noalloc_staging[KF_NOALLOC_STAGING_BYTES];

std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the staging buffer on the current device, looked up on
// the first call on that device (with that device current).
int staging_address(unsigned char **out) {
  int dev = 0;
  if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
  if (dev < 0 || dev >= kNoallocMaxDevices)
    return set_error(KF_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    if (int rc = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_staging),
                            "cudaGetSymbolAddress(staging buffer)"))
      return rc;
    g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return KF_OK;
}

// Copy tracks [c0, c0 + m) of a C-component host array (n tracks) to or
// from a staged array laid out for m tracks.
cudaError_t stage_copy(void *dst, const void *src, int C, const LayoutDesc &d, int64_t c0,
                       int64_t m, bool to_device, cudaStream_t s) {
  if (d.soa) {
    if (to_device)
      return cudaMemcpy2DAsync(dst, 4 * m, static_cast<const float *>(src) + c0, 4 * d.n, 4 * m,
                               C, cudaMemcpyDefault, s);
    return cudaMemcpy2DAsync(static_cast<float *>(dst) + c0, 4 * d.n, src, 4 * m, 4 * m, C,
                             cudaMemcpyDefault, s);
  }
  const int64_t W = int64_t(1) << d.lw;
  const int64_t blocks = (m + W - 1) / W;
  const int64_t first = (c0 / W) * C * W;
  const size_t bytes = 4 * blocks * C * W;
  if (to_device)
    return cudaMemcpyAsync(dst, static_cast<const float *>(src) + first, bytes, cudaMemcpyDefault,
                           s);
  return cudaMemcpyAsync(static_cast<float *>(dst) + first, src, bytes, cudaMemcpyDefault, s);
}

}  // namespace
}  // namespace kf

extern "C" int kf_propagate_update_host_noalloc(int32_t kind, const kf_params *params,
                                                kf_layout layout, const float *state_in,
                                                const float *cov_in, float *state_out,
                                                float *cov_out, const int8_t *charge,
                                                const float *hit, const float *hit_cov,
                                                const float *surf, int32_t surf_per_track,
                                                uint8_t *status, int64_t chunk_tracks,
                                                void *stream) {
  using namespace kf;
  clear_error();
  if (kind != KF_P2Z && kind != KF_P2R)
    return set_error(KF_ERR_ARG, "kind = %d is neither KF_P2Z nor KF_P2R", kind);
  if (!params) return set_error(KF_ERR_ARG, "params is NULL");
  if (params->flags != 0) return set_error(KF_ERR_ARG, "params->flags must be 0");
  if (params->precision < KF_FP32 || params->precision > KF_DF_UPDATE)
    return set_error(KF_ERR_ARG, "unknown precision %d", params->precision);
  LayoutDesc d;
  if (int rc = check_layout(layout, &d)) return rc;
  if (chunk_tracks < 0) return set_error(KF_ERR_ARG, "chunk_tracks < 0");
  if (chunk_tracks > KF_NOALLOC_MAX_CHUNK)
    return set_error(KF_ERR_ARG,
                     "chunk_tracks = %lld exceeds the static staging capacity of %d tracks",
                     (long long)chunk_tracks, KF_NOALLOC_MAX_CHUNK);
  if (d.n == 0) return KF_OK;
  if (!state_in || !cov_in || !state_out || !cov_out || !charge || !hit || !hit_cov || !surf)
    return set_error(KF_ERR_ARG, "a required pointer is NULL");
  if (surf_per_track != 0 && surf_per_track != 1)
    return set_error(KF_ERR_ARG, "surf_per_track must be 0 or 1");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    // arrays reachable in place: the kernel works on them, nothing is staged
    // (the staging buffer holds KF_ADAPTIVE's redo marks when status is NULL)
    const HostArrays h{state_in, cov_in, state_out, cov_out, charge,
                       hit,      hit_cov, surf,     surf_per_track, status};
    uint8_t *scratch = nullptr;
    if (!status && params->precision == KF_ADAPTIVE && d.n <= KF_NOALLOC_STAGING_BYTES) {
      unsigned char *staging = nullptr;
      if (int rc = staging_address(&staging)) return rc;
      scratch = staging;
    }
    bool taken = false;
    if (int rc = host_direct(kind, *params, d, h, scratch, KF_NOALLOC_STAGING_BYTES, s, &taken))
      return rc;
    if (taken) return KF_OK;
  }

  // Chunk c's outputs are copied back before chunk c + 1's inputs are copied
  // in: outputs that partially overlap the inputs would overwrite inputs not
  // yet read (in place, exactly coinciding, is safe).
  {
    const int64_t b6 = 4 * layout_floats(d, 6), b21 = 4 * layout_floats(d, 21);
    if (partial_overlap(state_in, b6, state_out, b6) || partial_overlap(cov_in, b21, cov_out, b21))
      return set_error(KF_ERR_ARG, "input and output overlap without coinciding");
  }

  // Chunk: the requested size (default: the capacity), a whole number of
  // AoSoA blocks, never more than the staged layout holds.
  const int64_t W = d.soa ? 1 : (int64_t(1) << d.lw);
  int64_t chunk = chunk_tracks > 0 ? chunk_tracks : KF_NOALLOC_MAX_CHUNK;
  chunk = (chunk / W) * W;
  if (chunk <= 0) return set_error(KF_ERR_ARG, "chunk_tracks smaller than the AoSoA width");

  unsigned char *base = nullptr;
  if (int rc = staging_address(&base)) return rc;
  float *d_st_in = reinterpret_cast<float *>(base + kSlot.state_in);
  float *d_cv_in = reinterpret_cast<float *>(base + kSlot.cov_in);
  float *d_hit = reinterpret_cast<float *>(base + kSlot.hit);
  float *d_hc = reinterpret_cast<float *>(base + kSlot.hitcov);
  float *d_st_out = reinterpret_cast<float *>(base + kSlot.state_out);
  float *d_cv_out = reinterpret_cast<float *>(base + kSlot.cov_out);
  int8_t *d_q = reinterpret_cast<int8_t *>(base + kSlot.charge);
  uint8_t *d_status = reinterpret_cast<uint8_t *>(base + kSlot.status);
  float *d_surf = reinterpret_cast<float *>(base + kSlot.surf);

  // Everything runs on the caller's stream, chunk after chunk through the one
  // staging area: stream order keeps a chunk's copies-in behind the previous
  // chunk's copies-out.
  for (int64_t c0 = 0; c0 < d.n; c0 += chunk) {
    const int64_t m = (d.n - c0 < chunk) ? d.n - c0 : chunk;
    LayoutDesc dc = d;
    dc.n = m;
    cudaError_t e = stage_copy(d_st_in, state_in, 6, d, c0, m, true, s);
    if (e == cudaSuccess) e = stage_copy(d_cv_in, cov_in, 21, d, c0, m, true, s);
    if (e == cudaSuccess) e = stage_copy(d_hit, hit, 3, d, c0, m, true, s);
    if (e == cudaSuccess) e = stage_copy(d_hc, hit_cov, 6, d, c0, m, true, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_q, charge + c0, m, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_surf, surf_per_track ? surf + c0 : surf, surf_per_track ? 4 * m : 4,
                          cudaMemcpyDefault, s);
    if (int rc = check_cuda(e, "host-to-device copy into the staging buffer")) return rc;
    StepArgs a{d_st_in, d_cv_in, d_st_out, d_cv_out, d_q, d_hit, d_hc, d_surf,
               (status || params->precision == KF_ADAPTIVE) ? d_status : nullptr, m, dc.soa, dc.lw, params->bz, surf_per_track};
    if (int rc = launch_step_kernel(kind, params->precision, a, s)) return rc;
    e = stage_copy(state_out, d_st_out, 6, d, c0, m, false, s);
    if (e == cudaSuccess) e = stage_copy(cov_out, d_cv_out, 21, d, c0, m, false, s);
    if (e == cudaSuccess && status)
      e = cudaMemcpyAsync(status + c0, d_status, m, cudaMemcpyDefault, s);
    if (int rc = check_cuda(e, "device-to-host copy from the staging buffer")) return rc;
  }
  return KF_OK;
}
