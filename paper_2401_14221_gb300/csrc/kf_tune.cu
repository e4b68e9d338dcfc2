// kf_tune.cu -- the autotuner: measure candidate launch shapes of the step
// and chain kernels on the caller's own arrays, keep the fastest in a cache
// keyed by (GPU model, operation, kind, precision, layout, n bucket), and
// let later launches in KF_STEP_AUTO mode use it.
//
// Candidates.  Single step: the one-thread-per-track kernel with 128 or 256
// threads per CTA, and (AoSoA layouts, or SoA with n a multiple of 4) the
// persistent staged kernel with one, two or three CTAs per SM.  Chain: 64,
// 128 or 256 threads per CTA.  n buckets are
// powers of two (floor(log2 n)), so one measurement serves batches of
// similar size.  The cache lives in host memory for the life of the process;
// kf_autotune_export / kf_autotune_import move it between processes as text.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include <algorithm>

#include <cuda_runtime.h>

#include "kf_common.cuh"
#include "kf_device.cuh"
#include "kf_step.cuh"

namespace kf {
namespace {

thread_local const LaunchConfig *t_override = nullptr;

struct Entry {
  LaunchConfig cfg;
  float ms;
};

using Key = std::tuple<std::string, int, int, int, int, int, int>;  // gpu, op, kind, prec, soa, lw, nb

std::mutex g_tune_mu;
std::map<Key, Entry> g_tune;

int n_bucket(int64_t n) {
  int b = 0;
  while (n > 1) {
    n >>= 1;
    ++b;
  }
  return b;
}

// "<device name>/sm<count>" of the current device, looked up once per device.
std::string gpu_name() {
  static std::mutex mu;
  static std::string names[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return "unknown";
  std::lock_guard<std::mutex> lock(mu);
  if (names[dev].empty()) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string name(prop.name);
    for (char &c : name)
      if (c == '|' || c == '\n') c = '_';
    names[dev] = name + "/sm" + std::to_string(prop.multiProcessorCount);
  }
  return names[dev];
}

// Time `reps` calls of fn() on stream s (after `warm` untimed ones).
template <class Fn>
int time_calls(Fn fn, cudaStream_t s, int warm, int reps, float *ms) {
  for (int i = 0; i < warm; ++i)
    if (int rc = fn()) return rc;
  cudaEvent_t a, b;
  if (int rc = check_cuda(cudaEventCreate(&a), "cudaEventCreate")) return rc;
  if (int rc = check_cuda(cudaEventCreate(&b), "cudaEventCreate")) {
    cudaEventDestroy(a);
    return rc;
  }
  int rc = check_cuda(cudaEventRecord(a, s), "cudaEventRecord");
  for (int i = 0; rc == KF_OK && i < reps; ++i) rc = fn();
  if (rc == KF_OK) rc = check_cuda(cudaEventRecord(b, s), "cudaEventRecord");
  if (rc == KF_OK) rc = check_cuda(cudaEventSynchronize(b), "cudaEventSynchronize");
  if (rc == KF_OK) rc = check_cuda(cudaEventElapsedTime(ms, a, b), "cudaEventElapsedTime");
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc == KF_OK) *ms /= (float)reps;
  return rc;
}

}  // namespace

const LaunchConfig *thread_override() { return t_override; }
void set_thread_override(const LaunchConfig *cfg) { t_override = cfg; }

bool tune_lookup(int op, int kind, int precision, int soa, int lw, int64_t n, LaunchConfig *out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (g_tune.empty()) return false;
  auto it = g_tune.find(Key(gpu_name(), op, kind, precision, soa, soa ? 0 : lw, n_bucket(n)));
  if (it == g_tune.end()) return false;
  *out = it->second.cfg;
  return true;
}

void tune_store(int op, int kind, int precision, int soa, int lw, int64_t n,
                const LaunchConfig &cfg, float ms) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[Key(gpu_name(), op, kind, precision, soa, soa ? 0 : lw, n_bucket(n))] = Entry{cfg, ms};
}

}  // namespace kf

extern "C" int kf_autotune_step(int32_t kind, const kf_params *params, kf_layout layout,
                                const float *state_in, const float *cov_in, float *state_out,
                                float *cov_out, const int8_t *charge, const float *hit,
                                const float *hit_cov, const float *surf, int32_t surf_per_track,
                                uint8_t *status, void *stream, kf_tuning *out) {
  using namespace kf;
  clear_error();
  if (kind != KF_P2Z && kind != KF_P2R)
    return set_error(KF_ERR_ARG, "kind = %d is neither KF_P2Z nor KF_P2R", kind);
  if (!params || !out) return set_error(KF_ERR_ARG, "params or out is NULL");
  LayoutDesc d;
  if (int rc = check_layout(layout, &d)) return rc;
  if (d.n == 0) return set_error(KF_ERR_ARG, "nothing to tune for n = 0");
  auto call = [&]() {
    return kind == KF_P2Z
               ? kf_p2z_propagate_update(params, layout, state_in, cov_in, state_out, cov_out,
                                         charge, hit, hit_cov, surf, surf_per_track, status,
                                         stream)
               : kf_p2r_propagate_update(params, layout, state_in, cov_in, state_out, cov_out,
                                         charge, hit, hit_cov, surf, surf_per_track, status,
                                         stream);
  };
  LaunchConfig cands[5] = {{KF_STEP_DIRECT, 128, 0},
                           {KF_STEP_DIRECT, 256, 0},
                           {KF_STEP_STAGED, 256, 1},
                           {KF_STEP_STAGED, 256, 2},
                           {KF_STEP_STAGED, 256, 3}};
  const int ncand = (d.soa && (d.n & 3)) ? 2 : 5;  // staged: AoSoA, or SoA with n % 4 == 0
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Candidates take turns over kRounds rounds (so that clock or memory
  // drift during tuning hits all of them alike); each keeps its median.
  constexpr int kRounds = 5;
  float ms_of[5][kRounds];
  for (int round = 0; round < kRounds; ++round) {
    for (int c = 0; c < ncand; ++c) {
      set_thread_override(&cands[c]);
      const int rc = time_calls(call, s, round == 0 ? 3 : 1, 10, &ms_of[c][round]);
      set_thread_override(nullptr);
      if (rc) return rc;
    }
  }
  int best = -1;
  float best_ms = 0.0f;
  for (int c = 0; c < ncand; ++c) {
    std::sort(ms_of[c], ms_of[c] + kRounds);
    const float med = ms_of[c][kRounds / 2];
    if (best < 0 || med < best_ms) {
      best = c;
      best_ms = med;
    }
  }
  tune_store(kOpStep, kind, params->precision, d.soa, d.lw, d.n, cands[best], best_ms);
  out->step_kernel = cands[best].kernel;
  out->threads = cands[best].threads;
  out->ctas_per_sm = cands[best].ctas_per_sm;
  out->ms = best_ms;
  return KF_OK;
}

extern "C" int kf_autotune_chain(const kf_params *params, kf_layout layout, float *state,
                                 float *cov, const int8_t *charge, const float *hits,
                                 const float *hit_covs, const kf_layer *layers, int32_t L,
                                 uint8_t *status, float *state_scratch, float *cov_scratch,
                                 void *stream, kf_tuning *out) {
  using namespace kf;
  clear_error();
  if (!params || !out) return set_error(KF_ERR_ARG, "params or out is NULL");
  LayoutDesc d;
  if (int rc = check_layout(layout, &d)) return rc;
  if (d.n == 0 || L <= 0) return set_error(KF_ERR_ARG, "nothing to tune");
  const int64_t b6 = 4 * layout_floats(d, 6), b21 = 4 * layout_floats(d, 21);
  if (int rc = check_device_memory(state_scratch, b6, "state_scratch")) return rc;
  if (int rc = check_device_memory(cov_scratch, b21, "cov_scratch")) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // keep the start state; restore it before every call and at the end
  if (int rc = check_cuda(cudaMemcpyAsync(state_scratch, state, b6, cudaMemcpyDeviceToDevice, s),
                          "save state"))
    return rc;
  if (int rc = check_cuda(cudaMemcpyAsync(cov_scratch, cov, b21, cudaMemcpyDeviceToDevice, s),
                          "save covariance"))
    return rc;
  auto restore = [&]() {
    if (int rc = check_cuda(cudaMemcpyAsync(state, state_scratch, b6, cudaMemcpyDeviceToDevice, s),
                            "restore state"))
      return rc;
    return check_cuda(cudaMemcpyAsync(cov, cov_scratch, b21, cudaMemcpyDeviceToDevice, s),
                      "restore covariance");
  };
  LaunchConfig cands[3] = {{KF_STEP_DIRECT, 64, 0}, {KF_STEP_DIRECT, 128, 0},
                           {KF_STEP_DIRECT, 256, 0}};
  cudaEvent_t a, b;
  if (int rc = check_cuda(cudaEventCreate(&a), "cudaEventCreate")) return rc;
  if (int rc = check_cuda(cudaEventCreate(&b), "cudaEventCreate")) {
    cudaEventDestroy(a);
    return rc;
  }
  int rc = KF_OK, best = -1;
  float best_ms = 0.0f;
  for (int c = 0; rc == KF_OK && c < 3; ++c) {
    set_thread_override(&cands[c]);
    float total = 0.0f;
    for (int rep = 0; rc == KF_OK && rep < 4; ++rep) {  // rep 0 warms up
      rc = restore();
      if (rc == KF_OK) rc = check_cuda(cudaEventRecord(a, s), "cudaEventRecord");
      if (rc == KF_OK)
        rc = kf_kalman_chain(params, layout, state, cov, charge, hits, hit_covs, layers, L,
                             status, stream);
      if (rc == KF_OK) rc = check_cuda(cudaEventRecord(b, s), "cudaEventRecord");
      if (rc == KF_OK) rc = check_cuda(cudaEventSynchronize(b), "cudaEventSynchronize");
      float ms = 0.0f;
      if (rc == KF_OK) rc = check_cuda(cudaEventElapsedTime(&ms, a, b), "cudaEventElapsedTime");
      if (rep > 0) total += ms;
    }
    set_thread_override(nullptr);
    if (rc == KF_OK && (best < 0 || total / 3.0f < best_ms)) {
      best = c;
      best_ms = total / 3.0f;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc == KF_OK) rc = restore();
  if (rc == KF_OK) rc = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (rc) return rc;
  tune_store(kOpChain, 0, params->precision, d.soa, d.lw, d.n, cands[best], best_ms);
  out->step_kernel = cands[best].kernel;
  out->threads = cands[best].threads;
  out->ctas_per_sm = cands[best].ctas_per_sm;
  out->ms = best_ms;
  return KF_OK;
}

extern "C" int kf_autotune_export(char *buf, int64_t cap, int64_t *len) {
  using namespace kf;
  clear_error();
  std::string text;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    char line[512];
    for (const auto &kv : g_tune) {
      const Key &k = kv.first;
      const Entry &e = kv.second;
      snprintf(line, sizeof(line), "%s|%d|%d|%d|%d|%d|%d|%d|%d|%d|%.6g\n",
               std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k),
               std::get<4>(k), std::get<5>(k), std::get<6>(k), e.cfg.kernel, e.cfg.threads,
               e.cfg.ctas_per_sm, e.ms);
      text += line;
    }
  }
  if (len) *len = (int64_t)text.size();
  if (!buf) return KF_OK;
  if (cap < (int64_t)text.size() + 1)
    return set_error(KF_ERR_ARG, "buffer of %lld bytes, need %lld", (long long)cap,
                     (long long)text.size() + 1);
  memcpy(buf, text.c_str(), text.size() + 1);
  return KF_OK;
}

extern "C" int kf_autotune_import(const char *text) {
  using namespace kf;
  clear_error();
  if (!text) return set_error(KF_ERR_ARG, "text is NULL");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const char *p = text;
  int lineno = 0;
  while (*p) {
    const char *e = strchr(p, '\n');
    std::string line = e ? std::string(p, e - p) : std::string(p);
    p = e ? e + 1 : p + line.size();
    ++lineno;
    if (line.empty()) continue;
    const size_t bar = line.find('|');
    if (bar == std::string::npos) return set_error(KF_ERR_ARG, "line %d: no GPU field", lineno);
    int op, kind, prec, soa, lw, nb, kern, thr, cps;
    float ms;
    if (sscanf(line.c_str() + bar + 1, "%d|%d|%d|%d|%d|%d|%d|%d|%d|%g", &op, &kind, &prec, &soa,
               &lw, &nb, &kern, &thr, &cps, &ms) != 10)
      return set_error(KF_ERR_ARG, "line %d: malformed entry", lineno);
    if ((op != kOpStep && op != kOpChain) || (kind != KF_P2Z && kind != KF_P2R) ||
        prec < KF_FP32 || prec > KF_DF_UPDATE || (soa != 0 && soa != 1) || lw < 0 || lw > 7 ||
        (kern != KF_STEP_DIRECT && kern != KF_STEP_STAGED) ||
        (thr != 64 && thr != 128 && thr != 256) || cps < 0 || cps > 3 || !(ms >= 0.0f))
      return set_error(KF_ERR_ARG, "line %d: value out of range", lineno);
    g_tune[Key(line.substr(0, bar), op, kind, prec, soa, lw, nb)] =
        Entry{LaunchConfig{kern, thr, cps}, ms};
  }
  return KF_OK;
}

extern "C" int kf_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(kf::g_tune_mu);
  kf::g_tune.clear();
  return KF_OK;
}
