// kf_server.cu -- continuous-batching serving loop for the multi-layer chain.
//
// Events (a batch of tracks each, with a hit per layer) are submitted from
// host threads at any time.  A scheduler thread owned by the server
//
//   1. admits pending events while an event slot and space in the caller's
//      device arena are free, and copies each admitted event in on the
//      copy-in stream;
//   2. whenever no batch is computing, launches ONE batched chain kernel over
//      every admitted event whose copies have landed (up to 128 events), on
//      the compute stream -- events that arrived while the previous batch was
//      running join the next batch, so work from different requests overlaps
//      on the device;
//   3. when a batch finishes, copies each event's results out on the
//      copy-out stream while the next batch computes, and when those copies
//      land marks the event done, records its latency (submit to results in
//      host memory) and returns its slot and arena space.
//
// Direct events skip the copies: where the GPU reaches every array of an
// event in place (page-locked memory, or pageable memory on a device that
// walks the host page tables -- the host-array calls' direct path), the
// batch kernel reads the event's inputs from and writes its results to the
// caller's arrays over the CPU-GPU link.  Such an event is ready as soon as
// it is admitted and done as soon as its batch completes; the arena holds
// only its status marks.
//
// The track arithmetic is the chain kernel's (kf_chain.cuh), one thread per
// track, so an event's results do not depend on what else is in its batch.
// Streams, events and the thread are created when the server is created;
// per-event device memory comes from the caller's arena (first-fit free list),
// so submitting and serving allocate nothing.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <sys/prctl.h>

#include <cuda_runtime.h>

#include "kf_chain.cuh"
#include "kf_common.cuh"
#include "kf_device.cuh"
#include "kf_host.cuh"
#include "kf_step.cuh"

namespace kf {
namespace srv {

constexpr int kMaxBatch = 128;

// Tracks per block of the batch grid.  A batch is a few events of a few
// thousand tracks, and each track's 15 layers are a chain of dependent
// instructions: 64-thread blocks spread such a batch over four times as many
// SMs as 256-thread blocks would, so fewer warps share each scheduler.
constexpr int kBatchThreads = 64;

// How long after its last progress the scheduler keeps polling (in-flight
// GPU work, and new submissions) without sleeping, microseconds.
constexpr double kSpinUs = 200.0;

// One event of a batch.  Copied events: inputs and outputs are the same
// arena arrays (the chain runs in place).  Direct events: the caller's host
// arrays.
struct EventDesc {
  const float *state_in;
  const float *cov_in;
  float *state_out;
  float *cov_out;
  const int8_t *charge;
  const float *hits;
  const float *hitcovs;
  uint8_t *status;
  int64_t n;
  int64_t block_begin;  // first block of this event in the batch grid
};

struct BatchArgs {
  int32_t nev;
  int32_t L;
  float bz;
  int32_t pad;
  int32_t kinds[KF_MAX_LAYERS];
  float pos[KF_MAX_LAYERS];
  EventDesc ev[kMaxBatch];
};

// One grid over all tracks of a batch: block b belongs to the last event
// whose block_begin <= b (binary search, uniform within the block).  Each
// event's arrays are SoA [C][n_event].
template <int VARIANT>
__global__ void __launch_bounds__(256) batch_chain_kernel(const __grid_constant__ BatchArgs a) {
  int lo = 0, hi = a.nev - 1;
  const int64_t b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.ev[mid].block_begin <= b) lo = mid;
    else hi = mid - 1;
  }
  const EventDesc &e = a.ev[lo];
  const int64_t i = (b - e.block_begin) * blockDim.x + threadIdx.x;
  if (i >= e.n) return;
  const ChainLoc l6{i, e.n}, l21{i, e.n}, l3{i, e.n};
  float p[6], C[21];
#pragma unroll
  for (int c = 0; c < 6; ++c) p[c] = e.state_in[l6.base + c * l6.stride];
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = e.cov_in[l21.base + k * l21.stride];
  const float qf = (float)__ldg(e.charge + i);
  unsigned st;
  if constexpr (VARIANT == kAdaptive) {
    st = chain_track_marking(p, C, qf, a.bz, a.L, a.kinds, a.pos, e.hits, 3 * e.n, e.hitcovs,
                             6 * e.n, l3, l6);
    if (st & kRedo) {  // left to batch_redo_kernel, inputs untouched
      e.status[i] = (uint8_t)kRedo;
      return;
    }
  } else if constexpr (VARIANT == kFP64) {
    st = chain_track_fp64(p, C, qf, a.bz, a.L, a.kinds, a.pos, e.hits, 3 * e.n, e.hitcovs,
                          6 * e.n, l3, l6);
  } else {
    st = chain_track<VARIANT>(p, C, qf, a.bz, a.L, a.kinds, a.pos, e.hits, 3 * e.n, e.hitcovs,
                              6 * e.n, l3, l6);
  }
  st |= finite_status(p, C);
#pragma unroll
  for (int c = 0; c < 6; ++c) e.state_out[l6.base + c * l6.stride] = p[c];
#pragma unroll
  for (int k = 0; k < 21; ++k) e.cov_out[l21.base + k * l21.stride] = C[k];
  if (e.status) e.status[i] = (uint8_t)st;
}

// KF_ADAPTIVE's second pass over a batch.  Block r covers batch-grid blocks
// [64 r, 64 r + 64) (4,096 track slots, possibly of several events); it
// gathers the slots whose track is marked kRedo into shared memory, then its
// threads rerun those tracks' whole chain in double (chain_track_fp64), so
// that warps run full.  Every event has a status array (the caller's, for a
// direct event that gave one, else the arena's).
constexpr int kBatchRedoBlocks = 64;

__device__ __forceinline__ int batch_event_of(const BatchArgs &a, int64_t b) {
  int lo = 0, hi = a.nev - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.ev[mid].block_begin <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) batch_redo_kernel(const __grid_constant__ BatchArgs a,
                                                         int64_t nblocks) {
  __shared__ int16_t ev_of[kBatchRedoBlocks * kBatchThreads];
  __shared__ int32_t idx_of[kBatchRedoBlocks * kBatchThreads];
  __shared__ int count;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  for (int slot = threadIdx.x; slot < kBatchRedoBlocks * kBatchThreads; slot += blockDim.x) {
    const int64_t b = (int64_t)blockIdx.x * kBatchRedoBlocks + slot / kBatchThreads;
    if (b >= nblocks) break;
    const int ev = batch_event_of(a, b);
    const EventDesc &e = a.ev[ev];
    const int64_t i = (b - e.block_begin) * kBatchThreads + slot % kBatchThreads;
    if (i < e.n && (e.status[i] & kRedo)) {
      const int q = atomicAdd(&count, 1);
      ev_of[q] = (int16_t)ev;
      idx_of[q] = (int32_t)i;
    }
  }
  __syncthreads();
  const int cnt = count;
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const EventDesc &e = a.ev[ev_of[q]];
    const int64_t i = idx_of[q];
    const ChainLoc l6{i, e.n}, l21{i, e.n}, l3{i, e.n};
    float p[6], C[21];
    for (int c = 0; c < 6; ++c) p[c] = e.state_in[l6.base + c * l6.stride];
    for (int k = 0; k < 21; ++k) C[k] = e.cov_in[l21.base + k * l21.stride];
    const float qf = (float)e.charge[i];
    unsigned st = chain_track_fp64(p, C, qf, a.bz, a.L, a.kinds, a.pos, e.hits, 3 * e.n,
                                   e.hitcovs, 6 * e.n, l3, l6);
    st |= finite_status(p, C);
    for (int c = 0; c < 6; ++c) e.state_out[l6.base + c * l6.stride] = p[c];
    for (int k = 0; k < 21; ++k) e.cov_out[l21.base + k * l21.stride] = C[k];
    e.status[i] = (uint8_t)st;
  }
}

int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }

struct Layout {
  int64_t state, cov, charge, hits, hitcovs, status, bytes;
};

Layout event_layout(int64_t n, int L) {
  Layout l{};
  int64_t off = 0;
  l.state = off; off += align256(4 * 6 * n);
  l.cov = off; off += align256(4 * 21 * n);
  l.charge = off; off += align256(n);
  l.hits = off; off += align256(4 * 3 * n * L);
  l.hitcovs = off; off += align256(4 * 6 * n * L);
  l.status = off; off += align256(n);
  l.bytes = off;
  return l;
}

// A direct event's arena block: its status marks only.
Layout direct_layout(int64_t n) {
  Layout l{};
  l.state = l.cov = l.charge = l.hits = l.hitcovs = -1;
  l.status = 0;
  l.bytes = align256(n);
  return l;
}

enum class Phase { kPending, kCopying, kRunning, kReturning, kDone };

struct Request {
  uint64_t ticket;
  int64_t n;
  const float *state;
  const float *cov;
  const int8_t *charge;
  const float *hits;
  const float *hitcovs;
  float *state_out;
  float *cov_out;
  uint8_t *status_out;
  bool direct = false;  // the batch kernel works on the caller's arrays in place
  Phase phase = Phase::kPending;
  int64_t off = -1;  // arena offset
  Layout lay{};
  cudaEvent_t ev = nullptr;  // copies in / copies out landed
  // timing events around the copies in (then around the copies out) on the
  // GPU, for the device-side durations of the phases
  cudaEvent_t g0 = nullptr, g1 = nullptr;
  std::chrono::steady_clock::time_point t_submit, t_admit, t_issued, t_copied, t_launch,
      t_finished, t_done;
  float gpu_in_ms = 0.0f, gpu_compute_ms = 0.0f, gpu_out_ms = 0.0f;
  bool copied = false;  // copy-in seen complete (t_copied set)
};

// First-fit allocator over [0, size) with coalescing.
struct Arena {
  std::map<int64_t, int64_t> free_;  // offset -> size
  explicit Arena(int64_t size) { if (size > 0) free_[0] = size; }
  int64_t alloc(int64_t bytes) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const int64_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest > 0) free_[off + bytes] = rest;
        return off;
      }
    }
    return -1;
  }
  void release(int64_t off, int64_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace srv
}  // namespace kf

struct kf_server {
  kf_server_config cfg;
  char *arena_base = nullptr;
  kf::srv::Arena arena{0};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread thread;
  bool stop = false;
  bool paused = false;
  int error = KF_OK;
  char error_msg[256] = "";
  uint64_t next_ticket = 1;
  std::deque<kf::srv::Request *> pending;
  std::vector<kf::srv::Request *> copying, running, returning;
  std::unordered_map<uint64_t, kf::srv::Request *> by_ticket;
  std::vector<cudaEvent_t> event_pool;
  cudaStream_t s_in = nullptr, s_compute = nullptr, s_out = nullptr;
  cudaEvent_t batch_ev = nullptr;
  bool batch_in_flight = false;
  int in_flight = 0;  // admitted, not yet done
  // statistics
  std::vector<double> latencies_ms;
  // queue, ready, compute, out, copy-in (as the scheduler observes them),
  // then the device-side durations of the copies in, the batch kernel(s)
  // and the copies out, then the host time spent issuing the copies in
  std::vector<double> phase_ms[9];
  double sched_pass_max_ms = 0.0, sched_gap_max_ms = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timing_pool;
  cudaEvent_t batch_g0 = nullptr, batch_g1 = nullptr;
  int64_t tracks_done = 0, batches = 0, max_batch_events = 0;
};

namespace {

using kf::srv::Phase;
using kf::srv::Request;

void fail_locked(kf_server *s, cudaError_t e, const char *what) {
  if (s->error == KF_OK) {
    s->error = KF_ERR_CUDA;
    snprintf(s->error_msg, sizeof(s->error_msg), "%s: %s", what, cudaGetErrorString(e));
  }
}

// Copy an admitted request's inputs into its arena block (copy-in stream).
bool start_copy_in(kf_server *s, Request *r) {
  char *b = s->arena_base + r->off;
  const int64_t n = r->n, L = s->cfg.L;
  cudaError_t e = cudaEventRecord(r->g0, s->s_in);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b + r->lay.state, r->state, 4 * 6 * n, cudaMemcpyDefault, s->s_in);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b + r->lay.cov, r->cov, 4 * 21 * n, cudaMemcpyDefault, s->s_in);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b + r->lay.charge, r->charge, n, cudaMemcpyDefault, s->s_in);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b + r->lay.hits, r->hits, 4 * 3 * n * L, cudaMemcpyDefault, s->s_in);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b + r->lay.hitcovs, r->hitcovs, 4 * 6 * n * L, cudaMemcpyDefault, s->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(r->g1, s->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev, s->s_in);
  if (e != cudaSuccess) {
    fail_locked(s, e, "server copy in");
    return false;
  }
  return true;
}

bool start_copy_out(kf_server *s, Request *r) {
  char *b = s->arena_base + r->off;
  const int64_t n = r->n;
  cudaError_t e = cudaStreamWaitEvent(s->s_out, s->batch_ev, 0);
  if (e == cudaSuccess) e = cudaEventRecord(r->g0, s->s_out);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->state_out, b + r->lay.state, 4 * 6 * n, cudaMemcpyDefault, s->s_out);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->cov_out, b + r->lay.cov, 4 * 21 * n, cudaMemcpyDefault, s->s_out);
  if (e == cudaSuccess && r->status_out)
    e = cudaMemcpyAsync(r->status_out, b + r->lay.status, n, cudaMemcpyDefault, s->s_out);
  if (e == cudaSuccess) e = cudaEventRecord(r->g1, s->s_out);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev, s->s_out);
  if (e != cudaSuccess) {
    fail_locked(s, e, "server copy out");
    return false;
  }
  return true;
}

bool launch_batch(kf_server *s, std::vector<Request *> &batch) {
  using namespace kf;
  using namespace kf::srv;
  BatchArgs a{};
  a.nev = (int32_t)batch.size();
  a.L = s->cfg.L;
  a.bz = s->cfg.bz;
  for (int l = 0; l < s->cfg.L; ++l) {
    a.kinds[l] = s->cfg.layers[l].kind;
    a.pos[l] = s->cfg.layers[l].pos;
  }
  int64_t blocks = 0;
  for (size_t k = 0; k < batch.size(); ++k) {
    Request *r = batch[k];
    char *b = s->arena_base + r->off;
    EventDesc &e = a.ev[k];
    if (r->direct) {
      e.state_in = r->state;
      e.cov_in = r->cov;
      e.state_out = r->state_out;
      e.cov_out = r->cov_out;
      e.charge = r->charge;
      e.hits = r->hits;
      e.hitcovs = r->hitcovs;
      e.status = r->status_out ? r->status_out : reinterpret_cast<uint8_t *>(b + r->lay.status);
    } else {
      float *st = reinterpret_cast<float *>(b + r->lay.state);
      float *cv = reinterpret_cast<float *>(b + r->lay.cov);
      e.state_in = st;
      e.cov_in = cv;
      e.state_out = st;
      e.cov_out = cv;
      e.charge = reinterpret_cast<const int8_t *>(b + r->lay.charge);
      e.hits = reinterpret_cast<const float *>(b + r->lay.hits);
      e.hitcovs = reinterpret_cast<const float *>(b + r->lay.hitcovs);
      e.status = reinterpret_cast<uint8_t *>(b + r->lay.status);
    }
    e.n = r->n;
    e.block_begin = blocks;
    blocks += (r->n + kBatchThreads - 1) / kBatchThreads;
  }
  cudaError_t e = cudaSuccess;
  for (Request *r : batch) {
    e = cudaStreamWaitEvent(s->s_compute, r->ev, 0);
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->batch_g0, s->s_compute);
  if (e == cudaSuccess && blocks > 0) {
    const unsigned g = (unsigned)blocks;
    switch (s->cfg.precision) {
      case KF_FP32: batch_chain_kernel<kFP32><<<g, kBatchThreads, 0, s->s_compute>>>(a); break;
      case KF_FP64_UPDATE: batch_chain_kernel<kFP64Update><<<g, kBatchThreads, 0, s->s_compute>>>(a); break;
      case KF_JOSEPH: batch_chain_kernel<kJoseph><<<g, kBatchThreads, 0, s->s_compute>>>(a); break;
      case KF_FP64: batch_chain_kernel<kFP64><<<g, kBatchThreads, 0, s->s_compute>>>(a); break;
      case KF_DF_UPDATE: batch_chain_kernel<kDFUpdate><<<g, kBatchThreads, 0, s->s_compute>>>(a); break;
      default:
        batch_chain_kernel<kAdaptive><<<g, kBatchThreads, 0, s->s_compute>>>(a);
        e = cudaGetLastError();
        if (e == cudaSuccess)
          batch_redo_kernel<<<(g + kBatchRedoBlocks - 1) / kBatchRedoBlocks, 256, 0, s->s_compute>>>(
              a, (int64_t)g);
        break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->batch_g1, s->s_compute);
  if (e == cudaSuccess) e = cudaEventRecord(s->batch_ev, s->s_compute);
  if (e != cudaSuccess) {
    fail_locked(s, e, "server batch launch");
    return false;
  }
  s->batches += 1;
  s->max_batch_events = std::max<int64_t>(s->max_batch_events, (int64_t)batch.size());
  return true;
}

// The event's results are in host memory: record its latency, return its
// slot, event object and arena space, wake its waiters.
void finish_request(kf_server *s, Request *r) {
  r->t_done = std::chrono::steady_clock::now();
  r->phase = Phase::kDone;
  auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  s->latencies_ms.push_back(ms(r->t_submit, r->t_done));
  s->phase_ms[0].push_back(ms(r->t_submit, r->t_admit));
  s->phase_ms[1].push_back(ms(r->t_admit, r->t_launch));
  s->phase_ms[2].push_back(ms(r->t_launch, r->t_finished));
  s->phase_ms[3].push_back(ms(r->t_finished, r->t_done));
  s->phase_ms[4].push_back(ms(r->t_admit, r->t_copied));
  s->phase_ms[5].push_back(r->gpu_in_ms);
  s->phase_ms[6].push_back(r->gpu_compute_ms);
  s->phase_ms[7].push_back(r->gpu_out_ms);
  s->phase_ms[8].push_back(ms(r->t_admit, r->t_issued));
  s->tracks_done += r->n;
  s->arena.release(r->off, r->lay.bytes);
  s->event_pool.push_back(r->ev);
  s->timing_pool.emplace_back(r->g0, r->g1);
  r->ev = r->g0 = r->g1 = nullptr;
  s->in_flight -= 1;
  s->cv_done.notify_all();
}

// One pass of the scheduler; returns true if anything moved.
bool schedule_once(kf_server *s) {
  bool moved = false;
  // copies out that landed: the event is done
  for (size_t k = 0; k < s->returning.size();) {
    Request *r = s->returning[k];
    const cudaError_t q = cudaEventQuery(r->ev);
    if (q == cudaErrorNotReady) {
      ++k;
      continue;
    }
    if (q != cudaSuccess) fail_locked(s, q, "server copy-out completion");
    if (q == cudaSuccess) cudaEventElapsedTime(&r->gpu_out_ms, r->g0, r->g1);
    finish_request(s, r);
    s->returning.erase(s->returning.begin() + k);
    moved = true;
  }
  // the running batch finished: direct events are done (the kernel wrote
  // their results to host memory), the others are copied out
  if (s->batch_in_flight) {
    const cudaError_t q = cudaEventQuery(s->batch_ev);
    if (q != cudaErrorNotReady) {
      if (q != cudaSuccess) fail_locked(s, q, "server batch completion");
      const auto now = std::chrono::steady_clock::now();
      float gpu_ms = 0.0f;
      if (q == cudaSuccess) cudaEventElapsedTime(&gpu_ms, s->batch_g0, s->batch_g1);
      for (Request *r : s->running) {
        r->t_finished = now;
        r->gpu_compute_ms = gpu_ms;
        if (r->direct) {
          finish_request(s, r);
        } else if (start_copy_out(s, r)) {
          r->phase = Phase::kReturning;
          s->returning.push_back(r);
        }
      }
      s->running.clear();
      s->batch_in_flight = false;
      moved = true;
    }
  }
  if (s->paused || s->error != KF_OK) return moved;
  // admit while a slot, an event object and arena space are free
  while (!s->pending.empty() && s->in_flight < s->cfg.max_events_in_flight &&
         !s->event_pool.empty() && !s->timing_pool.empty()) {
    Request *r = s->pending.front();
    const int64_t off = s->arena.alloc(r->lay.bytes);
    if (off < 0) break;  // wait for space: first come, first served
    r->off = off;
    r->t_admit = std::chrono::steady_clock::now();
    r->ev = s->event_pool.back();
    s->event_pool.pop_back();
    r->g0 = s->timing_pool.back().first;
    r->g1 = s->timing_pool.back().second;
    s->timing_pool.pop_back();
    s->pending.pop_front();
    s->in_flight += 1;
    if (r->direct) {  // nothing to copy: ready for the next batch
      r->copied = true;
      r->t_issued = r->t_copied = r->t_admit;
    } else if (!start_copy_in(s, r)) {
      break;
    } else {
      r->t_issued = std::chrono::steady_clock::now();
    }
    r->phase = Phase::kCopying;
    s->copying.push_back(r);
    moved = true;
  }
  // note when copies land (the copy-in phase ends even while a batch runs)
  {
    const auto now = std::chrono::steady_clock::now();
    for (Request *r : s->copying) {
      if (!r->copied && cudaEventQuery(r->ev) == cudaSuccess) {
        r->copied = true;
        r->t_copied = now;
        cudaEventElapsedTime(&r->gpu_in_ms, r->g0, r->g1);
      }
    }
  }
  // launch everything whose copies have landed
  if (!s->batch_in_flight && !s->copying.empty()) {
    std::vector<Request *> batch;
    for (size_t k = 0; k < s->copying.size() && (int)batch.size() < kf::srv::kMaxBatch;) {
      Request *r = s->copying[k];
      if (r->copied) {
        batch.push_back(r);
        s->copying.erase(s->copying.begin() + k);
      } else {
        ++k;
      }
    }
    if (!batch.empty() && launch_batch(s, batch)) {
      const auto now = std::chrono::steady_clock::now();
      for (Request *r : batch) {
        r->phase = Phase::kRunning;
        r->t_launch = now;
      }
      s->running = batch;
      s->batch_in_flight = true;
      moved = true;
    }
  }
  return moved;
}

void scheduler_main(kf_server *s) {
  cudaSetDevice(s->cfg.device);
  // Linux stretches a thread's sleeps by its timer slack (50 us by default),
  // which would make every 10 us back-off below a 60 us one and delay the
  // moment a finished batch is noticed; 1 us keeps the back-off as asked.
  prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
  std::unique_lock<std::mutex> lock(s->mu);
  auto last = std::chrono::steady_clock::now();
  auto progress = last;  // when a pass last moved something
  while (!s->stop) {
    // the scheduler's own timing: how long a pass takes, and how long it
    // was away between passes while GPU work was in flight (the mutex, the
    // back-off sleep and the OS's scheduling of this thread)
    const auto t0 = std::chrono::steady_clock::now();
    const bool was_busy = s->batch_in_flight || !s->copying.empty() || !s->returning.empty();
    if (was_busy)
      s->sched_gap_max_ms =
          std::max(s->sched_gap_max_ms, std::chrono::duration<double, std::milli>(t0 - last).count());
    const bool moved = schedule_once(s);
    last = std::chrono::steady_clock::now();
    s->sched_pass_max_ms =
        std::max(s->sched_pass_max_ms, std::chrono::duration<double, std::milli>(last - t0).count());
    const bool busy = s->batch_in_flight || !s->copying.empty() || !s->returning.empty();
    if (moved) {
      progress = last;
      continue;
    }
    if (busy) {
      // GPU work in flight: poll its events again at once for the first
      // kSpinUs after the last progress (a batch of a few events takes tens
      // of microseconds), then every 10 us
      lock.unlock();
      if (std::chrono::duration<double, std::micro>(last - progress).count() < kf::srv::kSpinUs)
        std::this_thread::yield();
      else
        std::this_thread::sleep_for(std::chrono::microseconds(10));
      lock.lock();
    } else if (std::chrono::duration<double, std::micro>(last - progress).count() <
               kf::srv::kSpinUs) {
      // idle, but work arrived recently: look for the next submission at
      // once instead of waiting to be woken (a wake-up costs about 10 us)
      lock.unlock();
      std::this_thread::yield();
      lock.lock();
    } else {
      s->cv_work.wait_for(lock, std::chrono::milliseconds(5));
    }
  }
}

int server_error(kf_server *s) {
  return kf::set_error(s->error, "server: %s", s->error_msg);
}

}  // namespace

extern "C" int64_t kf_server_event_bytes(int64_t n, int32_t L) {
  if (n < 0 || L < 0 || L > KF_MAX_LAYERS) return -1;
  return kf::srv::event_layout(n, L).bytes;
}

extern "C" int kf_server_create(const kf_server_config *cfg, kf_server **out) {
  using namespace kf;
  clear_error();
  if (!cfg || !out) return set_error(KF_ERR_ARG, "cfg or out is NULL");
  *out = nullptr;
  if (cfg->L < 1 || cfg->L > KF_MAX_LAYERS)
    return set_error(KF_ERR_ARG, "L = %d not in [1, %d]", cfg->L, KF_MAX_LAYERS);
  for (int l = 0; l < cfg->L; ++l)
    if (cfg->layers[l].kind != KF_P2Z && cfg->layers[l].kind != KF_P2R)
      return set_error(KF_ERR_ARG, "layers[%d].kind = %d", l, cfg->layers[l].kind);
  if (cfg->precision < KF_FP32 || cfg->precision > KF_DF_UPDATE)
    return set_error(KF_ERR_ARG, "unknown precision %d", cfg->precision);
  if (cfg->max_events_in_flight < 1)
    return set_error(KF_ERR_ARG, "max_events_in_flight must be >= 1");
  if (reinterpret_cast<uintptr_t>(cfg->arena) & 255u)
    return set_error(KF_ERR_ARG, "arena must be 256-byte aligned");
  if (int rc = check_cuda(cudaSetDevice(cfg->device), "cudaSetDevice")) return rc;
  if (int rc = check_device_memory(cfg->arena, cfg->arena_bytes, "arena")) return rc;

  kf_server *s = new kf_server;
  s->cfg = *cfg;
  s->arena_base = static_cast<char *>(cfg->arena);
  s->arena = kf::srv::Arena(cfg->arena_bytes);
  cudaError_t e = cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_compute, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->batch_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&s->batch_g0);
  if (e == cudaSuccess) e = cudaEventCreate(&s->batch_g1);
  for (int k = 0; e == cudaSuccess && k < cfg->max_events_in_flight; ++k) {
    cudaEvent_t ev, g0 = nullptr, g1 = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) s->event_pool.push_back(ev);
    if (e == cudaSuccess) e = cudaEventCreate(&g0);
    if (e == cudaSuccess) e = cudaEventCreate(&g1);
    if (e == cudaSuccess) s->timing_pool.emplace_back(g0, g1);
    else {
      if (g0) cudaEventDestroy(g0);
      if (g1) cudaEventDestroy(g1);
    }
  }
  if (e != cudaSuccess) {
    kf_server_destroy(s);
    return check_cuda(e, "server create");
  }
  s->thread = std::thread(scheduler_main, s);
  *out = s;
  return KF_OK;
}

extern "C" int kf_server_submit(kf_server *s, int64_t n, const float *state, const float *cov,
                                const int8_t *charge, const float *hits, const float *hit_covs,
                                float *state_out, float *cov_out, uint8_t *status_out,
                                uint64_t *ticket) {
  using namespace kf;
  clear_error();
  if (!s || !ticket) return set_error(KF_ERR_ARG, "server or ticket is NULL");
  if (n < 1 || n > 0x7fffffffLL)
    return set_error(KF_ERR_ARG, "an event needs 1 <= n < 2^31 tracks");
  if (!state || !cov || !charge || !hits || !hit_covs || !state_out || !cov_out)
    return set_error(KF_ERR_ARG, "a required pointer is NULL");
  // Direct when the host-path mode allows it and the server's device reaches
  // every array in place (input and output may coincide, not overlap
  // otherwise); else copied through the arena.
  bool direct = false;
  if (host_path_mode() != KF_HOST_COPY) {
    const int64_t L = s->cfg.L;
    const void *ptrs[] = {state, cov, charge, hits, hit_covs, state_out, cov_out, status_out};
    const int64_t bytes[] = {4 * 6 * n, 4 * 21 * n, n, 4 * 3 * n * L, 4 * 6 * n * L,
                             4 * 6 * n, 4 * 21 * n, n};
    const int align[] = {4, 4, 1, 4, 4, 4, 4, 1};
    const char *names[] = {"state", "cov", "charge", "hits", "hit_covs",
                           "state_out", "cov_out", "status_out"};
    direct = true;
    for (int k = 0; k < 8 && direct; ++k) {
      if (!ptrs[k]) continue;  // status_out may be NULL
      bool reach = false;
      if (int rc = host_reach(ptrs[k], bytes[k], align[k], names[k], &reach, s->cfg.device))
        return rc;
      direct = reach;
    }
    if (partial_overlap(state, 4 * 6 * n, state_out, 4 * 6 * n) ||
        partial_overlap(cov, 4 * 21 * n, cov_out, 4 * 21 * n))
      direct = false;
    if (!direct && host_path_mode() == KF_HOST_DIRECT)
      return set_error(KF_ERR_ARG, "KF_HOST_DIRECT: an array of the event is not reachable in "
                                   "place from the server's device (or input and output "
                                   "overlap without coinciding)");
  }
  const kf::srv::Layout lay =
      direct ? kf::srv::direct_layout(n) : kf::srv::event_layout(n, s->cfg.L);
  if (lay.bytes > s->cfg.arena_bytes)
    return set_error(KF_ERR_ARG, "event of %lld tracks needs %lld arena bytes, the arena has %lld",
                     (long long)n, (long long)lay.bytes, (long long)s->cfg.arena_bytes);
  Request *r = new Request;
  r->direct = direct;
  r->n = n;
  r->state = state;
  r->cov = cov;
  r->charge = charge;
  r->hits = hits;
  r->hitcovs = hit_covs;
  r->state_out = state_out;
  r->cov_out = cov_out;
  r->status_out = status_out;
  r->lay = lay;
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->error != KF_OK) {
      delete r;
      return server_error(s);
    }
    r->ticket = s->next_ticket++;
    s->pending.push_back(r);
    s->by_ticket[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv_work.notify_one();
  return KF_OK;
}

extern "C" int kf_server_poll(kf_server *s, uint64_t ticket, int32_t *done) {
  using namespace kf;
  clear_error();
  if (!s || !done) return set_error(KF_ERR_ARG, "server or done is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return set_error(KF_ERR_ARG, "unknown ticket %llu",
                                                 (unsigned long long)ticket);
  *done = it->second->phase == Phase::kDone ? 1 : 0;
  if (s->error != KF_OK) return server_error(s);
  return KF_OK;
}

extern "C" int kf_server_wait(kf_server *s, uint64_t ticket, double timeout_s) {
  using namespace kf;
  clear_error();
  if (!s) return set_error(KF_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end())
    return set_error(KF_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  Request *r = it->second;
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
  while (r->phase != Phase::kDone && s->error == KF_OK) {
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout &&
        r->phase != Phase::kDone)
      return set_error(KF_ERR_TIMEOUT, "ticket %llu not done within %.3f s",
                       (unsigned long long)ticket, timeout_s);
  }
  if (r->phase != Phase::kDone) return server_error(s);
  s->by_ticket.erase(it);
  delete r;
  return KF_OK;
}

extern "C" int kf_server_pause(kf_server *s, int32_t paused) {
  using namespace kf;
  clear_error();
  if (!s) return set_error(KF_ERR_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->paused = paused != 0;
  }
  s->cv_work.notify_one();
  return KF_OK;
}

extern "C" int kf_server_get_stats(kf_server *s, kf_server_stats *out) {
  using namespace kf;
  clear_error();
  if (!s || !out) return set_error(KF_ERR_ARG, "server or out is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  std::vector<double> v = s->latencies_ms;
  std::sort(v.begin(), v.end());
  *out = kf_server_stats{};
  out->events_done = (int64_t)v.size();
  out->tracks_done = s->tracks_done;
  out->batches = s->batches;
  out->max_batch_events = s->max_batch_events;
  if (!v.empty()) {
    auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
  }
  double *dst[9][2] = {{&out->queue_p50_ms, &out->queue_p99_ms},
                       {&out->ready_p50_ms, &out->ready_p99_ms},
                       {&out->compute_p50_ms, &out->compute_p99_ms},
                       {&out->out_p50_ms, &out->out_p99_ms},
                       {&out->copyin_p50_ms, &out->copyin_p99_ms},
                       {&out->gpu_copyin_p50_ms, &out->gpu_copyin_p99_ms},
                       {&out->gpu_compute_p50_ms, &out->gpu_compute_p99_ms},
                       {&out->gpu_out_p50_ms, &out->gpu_out_p99_ms},
                       {&out->copyin_issue_p50_ms, &out->copyin_issue_p99_ms}};
  out->sched_pass_max_ms = s->sched_pass_max_ms;
  out->sched_gap_max_ms = s->sched_gap_max_ms;
  for (int k = 0; k < 9; ++k) {
    std::vector<double> w = s->phase_ms[k];
    if (w.empty()) continue;
    std::sort(w.begin(), w.end());
    *dst[k][0] = w[std::min(w.size() - 1, (size_t)(0.50 * (w.size() - 1) + 0.5))];
    *dst[k][1] = w[std::min(w.size() - 1, (size_t)(0.99 * (w.size() - 1) + 0.5))];
  }
  return KF_OK;
}

extern "C" int kf_server_reset_stats(kf_server *s) {
  using namespace kf;
  clear_error();
  if (!s) return set_error(KF_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  s->latencies_ms.clear();
  for (auto &w : s->phase_ms) w.clear();
  s->sched_pass_max_ms = s->sched_gap_max_ms = 0.0;
  s->tracks_done = s->batches = s->max_batch_events = 0;
  return KF_OK;
}

extern "C" int kf_server_destroy(kf_server *s) {
  using namespace kf;
  clear_error();
  if (!s) return KF_OK;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    s->paused = false;
  }
  s->cv_work.notify_one();
  // let admitted work finish (bounded), then stop the thread
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(30);
  for (;;) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if ((s->pending.empty() && s->in_flight == 0) || s->error != KF_OK ||
          std::chrono::steady_clock::now() > deadline)
        break;
    }
    std::this_thread::sleep_for(std::chrono::milliseconds(1));
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_one();
  if (s->thread.joinable()) s->thread.join();
  if (s->s_in) cudaStreamSynchronize(s->s_in);
  if (s->s_compute) cudaStreamSynchronize(s->s_compute);
  if (s->s_out) cudaStreamSynchronize(s->s_out);
  for (auto &kv : s->by_ticket) {
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    delete kv.second;
  }
  for (cudaEvent_t ev : s->event_pool) cudaEventDestroy(ev);
  for (auto &g : s->timing_pool) {
    cudaEventDestroy(g.first);
    cudaEventDestroy(g.second);
  }
  if (s->batch_g0) cudaEventDestroy(s->batch_g0);
  if (s->batch_g1) cudaEventDestroy(s->batch_g1);
  if (s->batch_ev) cudaEventDestroy(s->batch_ev);
  if (s->s_in) cudaStreamDestroy(s->s_in);
  if (s->s_compute) cudaStreamDestroy(s->s_compute);
  if (s->s_out) cudaStreamDestroy(s->s_out);
  delete s;
  return KF_OK;
}
