// kf_host.cu -- the single step on HOST arrays, with the host<->device
// transfers inside the call (the paper's p2z measurement includes the data
// transfers; section 4, Figure 6 shows them on one stream before and after
// the kernel).
//
// GB300 design, two paths.
//
// Direct: on a Grace-Blackwell node the GPU reaches host memory over the
// coherent CPU-GPU link, page-locked memory always and pageable memory too
// where the device walks the host page tables.  Then the step kernel itself
// reads the inputs from and writes the results to the caller's arrays: no
// copy engine, no staging buffer, and both link directions busy for the
// whole kernel (copy engines measured 211 GB/s in, 193 GB/s out and 315 GB/s
// both ways at once on GB300; one kernel reading 139 MB and writing 105 MB
// of page-locked memory moved 316-327 GB/s, pageable 271-278 GB/s).
//
// Copy: otherwise the batch is cut into chunks that alternate between two
// library-owned streams.  While chunk c runs its kernel and copies its
// results out, chunk c+1 is already copying in on the other stream, so
// both copy directions and the kernels overlap.  The device buffers for the
// two chunks in flight live in a caller-provided workspace.
#include <atomic>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "kf_common.cuh"
#include "kf_device.cuh"
#include "kf_host.cuh"
#include "kf_step.cuh"

namespace kf {
namespace {

constexpr int kMaxDevices = 64;
constexpr int64_t kDefaultChunk = 1 << 18;

struct HostPipe {
  cudaStream_t s[2];
  cudaEvent_t fork;
  cudaEvent_t join[2];
};

std::mutex g_pipe_mu;
HostPipe *g_pipes[kMaxDevices] = {};

// Two non-blocking streams and three events per device, created on first use
// and kept for the life of the process.
int get_pipe(HostPipe **out) {
  int dev = 0;
  if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
  if (dev < 0 || dev >= kMaxDevices) return set_error(KF_ERR_UNSUPPORTED, "device %d", dev);
  if (!g_pipes[dev]) {
    HostPipe *p = new HostPipe;
    for (int i = 0; i < 2; ++i) {
      if (int rc = check_cuda(cudaStreamCreateWithFlags(&p->s[i], cudaStreamNonBlocking),
                              "cudaStreamCreate"))
        return rc;
      if (int rc = check_cuda(cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming),
                              "cudaEventCreate"))
        return rc;
    }
    if (int rc = check_cuda(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming),
                            "cudaEventCreate"))
      return rc;
    g_pipes[dev] = p;
  }
  *out = g_pipes[dev];
  return KF_OK;
}

int64_t round256(int64_t x) { return (x + 255) & ~int64_t(255); }

// Device buffers of one pipeline slot holding `chunk` tracks.
struct Slot {
  int64_t state_in, cov_in, hit, hitcov, state_out, cov_out, charge, status, surf, bytes;
};

Slot slot_layout(int64_t chunk) {
  Slot s;
  int64_t off = 0;
  auto take = [&](int64_t b) {
    const int64_t o = off;
    off += round256(b);
    return o;
  };
  s.state_in = take(4 * 6 * chunk);
  s.cov_in = take(4 * 21 * chunk);
  s.hit = take(4 * 3 * chunk);
  s.hitcov = take(4 * 6 * chunk);
  s.state_out = take(4 * 6 * chunk);
  s.cov_out = take(4 * 21 * chunk);
  s.charge = take(chunk);
  s.status = take(chunk);
  s.surf = take(4 * chunk);
  s.bytes = off;
  return s;
}

int64_t effective_chunk(const LayoutDesc &d, int64_t chunk_tracks) {
  const int64_t W = d.soa ? 1 : (int64_t(1) << d.lw);
  int64_t c = chunk_tracks > 0 ? chunk_tracks : kDefaultChunk;
  c = ((c + W - 1) / W) * W;
  const int64_t n_pad = ((d.n + W - 1) / W) * W;
  return c < n_pad ? c : (n_pad > 0 ? n_pad : W);
}

// Copy tracks [c0, c0 + m) of a C-component array between the full host
// array (n tracks) and a chunk buffer laid out for m tracks.
cudaError_t copy_chunk(void *dst, const void *src, int C, const LayoutDesc &d, int64_t c0,
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

std::atomic<int> g_host_path{KF_HOST_AUTO};

}  // namespace

int host_path_mode() { return g_host_path.load(std::memory_order_relaxed); }

int host_direct(int kind, const kf_params &params, const LayoutDesc &d, const HostArrays &h,
                uint8_t *scratch, int64_t scratch_bytes, cudaStream_t s, bool *taken) {
  *taken = false;
  const int mode = host_path_mode();
  if (mode == KF_HOST_COPY) return KF_OK;
  const int64_t b6 = 4 * layout_floats(d, 6), b21 = 4 * layout_floats(d, 21);
  const void *ptrs[] = {h.state_in, h.cov_in, h.state_out, h.cov_out, h.charge,
                        h.hit,      h.hit_cov, h.surf,     h.status};
  const int64_t bytes[] = {b6, b21, b6, b21, d.n, 4 * layout_floats(d, 3), b6,
                           h.surf_per_track ? 4 * d.n : 4, d.n};
  const int align[] = {4, 4, 4, 4, 1, 4, 4, 4, 1};
  const char *names[] = {"state_in", "cov_in", "state_out", "cov_out", "charge",
                         "hit",      "hit_cov", "surf",     "status"};
  const int count = h.status ? 9 : 8;
  for (int k = 0; k < count; ++k) {
    bool direct = false;
    if (int rc = host_reach(ptrs[k], bytes[k], align[k], names[k], &direct)) return rc;
    if (!direct) {
      if (mode == KF_HOST_AUTO) return KF_OK;
      return set_error(KF_ERR_ARG,
                       "KF_HOST_DIRECT: %s is not reachable in place from this device "
                       "(pageable memory on a device without host page-table access, or "
                       "misaligned)",
                       names[k]);
    }
  }
  if (partial_overlap(h.state_in, b6, h.state_out, b6) ||
      partial_overlap(h.cov_in, b21, h.cov_out, b21))
    return set_error(KF_ERR_ARG, "input and output overlap without coinciding");
  uint8_t *status = h.status;
  if (!status && params.precision == KF_ADAPTIVE) {
    if (!scratch || scratch_bytes < d.n) {
      if (mode == KF_HOST_AUTO) return KF_OK;
      return set_error(KF_ERR_ARG,
                       "KF_HOST_DIRECT with KF_ADAPTIVE and no status array needs %lld bytes "
                       "of device scratch for the redo marks",
                       (long long)d.n);
    }
    status = scratch;
  }
  StepArgs a{h.state_in, h.cov_in, h.state_out, h.cov_out, h.charge, h.hit, h.hit_cov, h.surf,
             status,     d.n,      d.soa,       d.lw,      params.bz, h.surf_per_track};
  if (int rc = launch_step_kernel(kind, params.precision, a, s, /*plain_loads=*/true)) return rc;
  *taken = true;
  return KF_OK;
}

namespace {

int run_host(int kind, const kf_params *params, kf_layout layout, const float *state_in,
             const float *cov_in, float *state_out, float *cov_out, const int8_t *charge,
             const float *hit, const float *hit_cov, const float *surf, int32_t surf_per_track,
             uint8_t *status, void *workspace, int64_t workspace_bytes, int64_t chunk_tracks,
             void *stream) {
  clear_error();
  if (!params) return set_error(KF_ERR_ARG, "params is NULL");
  if (params->flags != 0) return set_error(KF_ERR_ARG, "params->flags must be 0");
  if (params->precision < KF_FP32 || params->precision > KF_DF_UPDATE)
    return set_error(KF_ERR_ARG, "unknown precision %d", params->precision);
  LayoutDesc d;
  if (int rc = check_layout(layout, &d)) return rc;
  if (d.n == 0) return KF_OK;
  if (!state_in || !cov_in || !state_out || !cov_out || !charge || !hit || !hit_cov || !surf)
    return set_error(KF_ERR_ARG, "a required pointer is NULL");
  if (surf_per_track != 0 && surf_per_track != 1)
    return set_error(KF_ERR_ARG, "surf_per_track must be 0 or 1");
  if (chunk_tracks < 0) return set_error(KF_ERR_ARG, "chunk_tracks < 0");
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  {
    const HostArrays h{state_in, cov_in, state_out, cov_out, charge,
                       hit,      hit_cov, surf,     surf_per_track, status};
    // KF_ADAPTIVE without a status array: the workspace holds the redo marks
    uint8_t *scratch = nullptr;
    if (!status && params->precision == KF_ADAPTIVE && workspace && workspace_bytes >= d.n) {
      if (check_device_memory(workspace, d.n, "workspace") == KF_OK)
        scratch = static_cast<uint8_t *>(workspace);
      clear_error();
    }
    bool taken = false;
    if (int rc = host_direct(kind, *params, d, h, scratch, workspace_bytes, caller, &taken))
      return rc;
    if (taken) return KF_OK;
  }
  // Chunks are copied back while later chunks are still to be copied in:
  // outputs that partially overlap the inputs would overwrite inputs not yet
  // read (in place, exactly coinciding, is safe).
  {
    const int64_t b6 = 4 * layout_floats(d, 6), b21 = 4 * layout_floats(d, 21);
    if (partial_overlap(state_in, b6, state_out, b6) || partial_overlap(cov_in, b21, cov_out, b21))
      return set_error(KF_ERR_ARG, "input and output overlap without coinciding");
  }
  const int64_t chunk = effective_chunk(d, chunk_tracks);
  const Slot sl = slot_layout(chunk);
  if (workspace_bytes < 2 * sl.bytes)
    return set_error(KF_ERR_ARG, "workspace holds %lld bytes, needs %lld",
                     (long long)workspace_bytes, (long long)(2 * sl.bytes));
  if (reinterpret_cast<uintptr_t>(workspace) & 255u)
    return set_error(KF_ERR_ARG, "workspace must be 256-byte aligned");
  if (int rc = check_device_memory(workspace, 2 * sl.bytes, "workspace")) return rc;

  std::lock_guard<std::mutex> lock(g_pipe_mu);
  HostPipe *pipe = nullptr;
  if (int rc = get_pipe(&pipe)) return rc;
  if (int rc = check_cuda(cudaEventRecord(pipe->fork, caller), "cudaEventRecord")) return rc;
  for (int i = 0; i < 2; ++i)
    if (int rc = check_cuda(cudaStreamWaitEvent(pipe->s[i], pipe->fork, 0), "cudaStreamWaitEvent"))
      return rc;

  char *ws = static_cast<char *>(workspace);
  int64_t c = 0;
  for (int64_t c0 = 0; c0 < d.n; c0 += chunk, ++c) {
    const int64_t m = (d.n - c0 < chunk) ? d.n - c0 : chunk;
    cudaStream_t s = pipe->s[c & 1];
    char *base = ws + (c & 1) * sl.bytes;
    float *d_st_in = reinterpret_cast<float *>(base + sl.state_in);
    float *d_cv_in = reinterpret_cast<float *>(base + sl.cov_in);
    float *d_hit = reinterpret_cast<float *>(base + sl.hit);
    float *d_hc = reinterpret_cast<float *>(base + sl.hitcov);
    float *d_st_out = reinterpret_cast<float *>(base + sl.state_out);
    float *d_cv_out = reinterpret_cast<float *>(base + sl.cov_out);
    int8_t *d_q = reinterpret_cast<int8_t *>(base + sl.charge);
    uint8_t *d_status = reinterpret_cast<uint8_t *>(base + sl.status);
    float *d_surf = reinterpret_cast<float *>(base + sl.surf);
    LayoutDesc dc = d;
    dc.n = m;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = copy_chunk(d_st_in, state_in, 6, d, c0, m, true, s);
    if (e == cudaSuccess) e = copy_chunk(d_cv_in, cov_in, 21, d, c0, m, true, s);
    if (e == cudaSuccess) e = copy_chunk(d_hit, hit, 3, d, c0, m, true, s);
    if (e == cudaSuccess) e = copy_chunk(d_hc, hit_cov, 6, d, c0, m, true, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_q, charge + c0, m, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_surf, surf_per_track ? surf + c0 : surf,
                          surf_per_track ? 4 * m : 4, cudaMemcpyDefault, s);
    if (int rc = check_cuda(e, "host-to-device copy")) return rc;
    StepArgs a{d_st_in, d_cv_in, d_st_out, d_cv_out, d_q,  d_hit, d_hc, d_surf,
               (status || params->precision == KF_ADAPTIVE) ? d_status : nullptr, m, dc.soa, dc.lw, params->bz, surf_per_track};
    if (int rc = launch_step_kernel(kind, params->precision, a, s)) return rc;
    e = copy_chunk(state_out, d_st_out, 6, d, c0, m, false, s);
    if (e == cudaSuccess) e = copy_chunk(cov_out, d_cv_out, 21, d, c0, m, false, s);
    if (e == cudaSuccess && status)
      e = cudaMemcpyAsync(status + c0, d_status, m, cudaMemcpyDefault, s);
    if (int rc = check_cuda(e, "device-to-host copy")) return rc;
  }
  for (int i = 0; i < 2; ++i) {
    if (int rc = check_cuda(cudaEventRecord(pipe->join[i], pipe->s[i]), "cudaEventRecord"))
      return rc;
    if (int rc = check_cuda(cudaStreamWaitEvent(caller, pipe->join[i], 0), "cudaStreamWaitEvent"))
      return rc;
  }
  return KF_OK;
}

}  // namespace
}  // namespace kf

extern "C" int64_t kf_host_workspace_bytes(kf_layout layout, int64_t chunk_tracks) {
  kf::LayoutDesc d;
  if (kf::check_layout(layout, &d) || chunk_tracks < 0) return -1;
  return 2 * kf::slot_layout(kf::effective_chunk(d, chunk_tracks)).bytes;
}

extern "C" int kf_p2z_propagate_update_host(const kf_params *params, kf_layout layout,
                                            const float *state_in, const float *cov_in,
                                            float *state_out, float *cov_out,
                                            const int8_t *charge, const float *hit,
                                            const float *hit_cov, const float *z_surf,
                                            int32_t surf_per_track, uint8_t *status,
                                            void *workspace, int64_t workspace_bytes,
                                            int64_t chunk_tracks, void *stream) {
  return kf::run_host(kf::kP2z, params, layout, state_in, cov_in, state_out, cov_out, charge, hit,
                      hit_cov, z_surf, surf_per_track, status, workspace, workspace_bytes,
                      chunk_tracks, stream);
}

extern "C" int kf_p2r_propagate_update_host(const kf_params *params, kf_layout layout,
                                            const float *state_in, const float *cov_in,
                                            float *state_out, float *cov_out,
                                            const int8_t *charge, const float *hit,
                                            const float *hit_cov, const float *r_surf,
                                            int32_t surf_per_track, uint8_t *status,
                                            void *workspace, int64_t workspace_bytes,
                                            int64_t chunk_tracks, void *stream) {
  return kf::run_host(kf::kP2r, params, layout, state_in, cov_in, state_out, cov_out, charge, hit,
                      hit_cov, r_surf, surf_per_track, status, workspace, workspace_bytes,
                      chunk_tracks, stream);
}

extern "C" int kf_set_host_path(int32_t mode) {
  kf::clear_error();
  if (mode != KF_HOST_AUTO && mode != KF_HOST_COPY && mode != KF_HOST_DIRECT)
    return kf::set_error(KF_ERR_ARG, "unknown host path mode %d", mode);
  kf::g_host_path.store(mode, std::memory_order_relaxed);
  return KF_OK;
}
