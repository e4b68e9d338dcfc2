// kf_step_compressed.cu -- the single step on a compressed covariance store:
// per track six FP32 standard deviations sigma_i = sqrt(C_ii) and fifteen
// FP16 correlation coefficients rho_ij = C_ij / (sigma_i sigma_j)
// (off-diagonal entries in packed order 10, 20, 21, 30, ..., 54, stored in
// pairs: kf_compressed.cuh).
//
// The step is HBM-bound, so a smaller covariance store is a direct speed-up:
// 24 + 30 = 54 B instead of 84 B per covariance, 193 B instead of 253 B per
// p2r track (read 115, write 78).  FP16 keeps correlations to 2^-12 absolute
// (|rho| <= 1), i.e. every covariance element to ~2.4e-4 of its correlation
// scale sqrt(C_ii C_jj), inside the 1e-3 element bound.  Arithmetic is
// unchanged: the kernel decodes to FP32 registers, runs the same step and
// encodes the result (round to nearest).  A track that is not propagated
// (no intersection) gets its input sigma/rho back bit for bit.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "kf_common.cuh"
#include "kf_compressed.cuh"
#include "kf_device.cuh"
#include "kf_step.cuh"

namespace kf {
namespace {

struct Loc {
  int64_t base;
  int64_t stride;
};

template <int C>
__device__ __forceinline__ Loc locate(int64_t i, int64_t n, int32_t soa, int32_t lw) {
  if (soa) return {i, n};
  const int64_t W = int64_t(1) << lw;
  return {(i >> lw) * (C * W) + (i & (W - 1)), W};
}

// Load track i: state, and the covariance decoded from sigma / rho.
template <class T>
__device__ __forceinline__ void load_compressed(const CompressedArgs &a, const Loc &l6,
                                                const RhoLoc &lr, T (&p)[6], T (&C)[21]) {
  float sg[6], Cf[21];
  Rho rh;
#pragma unroll
  for (int c = 0; c < 6; ++c) p[c] = __ldg(a.state_in + l6.base + c * l6.stride);
#pragma unroll
  for (int c = 0; c < 6; ++c) sg[c] = __ldg(a.sigma_in + l6.base + c * l6.stride);
  load_rho(a.rho_in, lr, rh);
  decode_cov(sg, rh, Cf);
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = T(Cf[e]);
}

// Encode and store track i's result; a track that was not propagated gets
// its input sigma / rho back bit for bit.
__device__ __forceinline__ void store_compressed(const CompressedArgs &a, const Loc &l6,
                                                 const RhoLoc &lr, const float (&p)[6],
                                                 const float (&C)[21], unsigned st) {
  float sg[6];
  Rho rh;
  if (!(st & kNoIntersect)) {
    encode_cov(C, sg, rh);
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) sg[c] = __ldg(a.sigma_in + l6.base + c * l6.stride);
    load_rho(a.rho_in, lr, rh);
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) __stcs(a.state_out + l6.base + c * l6.stride, p[c]);
#pragma unroll
  for (int c = 0; c < 6; ++c) __stcs(a.sigma_out + l6.base + c * l6.stride, sg[c]);
  store_rho(a.rho_out, lr, rh);
}

template <int KIND, int VARIANT>
__global__ void __launch_bounds__(256)
    step_compressed_kernel(const __grid_constant__ CompressedArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const Loc l6 = locate<6>(i, a.n, a.soa, a.lw);
  const RhoLoc lr = locate_rho(i, a.n, a.soa, a.lw);
  const Loc l3 = locate<3>(i, a.n, a.soa, a.lw);

  float p[6], C[21];
  load_compressed(a, l6, lr, p, C);
  const float qf = (float)__ldg(a.charge + i);
  const float surf = __ldg(a.surf + (a.surf_per_track ? i : 0));

  unsigned st;
  if (KIND == kP2z) {
    const float hx = __ldg(a.hit + l3.base);
    const float hy = __ldg(a.hit + l3.base + l3.stride);
    const float vxx = __ldg(a.hitcov + l6.base);
    const float vxy = __ldg(a.hitcov + l6.base + l6.stride);
    const float vyy = __ldg(a.hitcov + l6.base + 2 * l6.stride);
    st = p2z_step<VARIANT>(p, C, qf, a.bz, surf, hx, hy, vxx, vxy, vyy);
  } else {
    const float hx = __ldg(a.hit + l3.base);
    const float hy = __ldg(a.hit + l3.base + l3.stride);
    const float hz = __ldg(a.hit + l3.base + 2 * l3.stride);
    float hc[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) hc[c] = __ldg(a.hitcov + l6.base + c * l6.stride);
    st = p2r_step<VARIANT>(p, C, qf, a.bz, surf, hx, hy, hz, hc);
  }
  if constexpr (VARIANT == kAdaptive) {
    if (st & kRedo) {  // ill-conditioned in FP32: left to the FP64 redo pass
      a.status[i] = (uint8_t)kRedo;
      return;
    }
  }
  st |= finite_status(p, C);
  store_compressed(a, l6, lr, p, C, st);
  if (a.status) a.status[i] = (uint8_t)st;
}

// KF_ADAPTIVE's second pass on the compressed store: tracks marked kRedo
// are decoded again from their (untouched) inputs and stepped in FP64.  Each
// block gathers the marked tracks of its span first, so warps run full.
template <int KIND>
__global__ void __launch_bounds__(kRedoThreads)
    redo_compressed_kernel(const __grid_constant__ CompressedArgs a) {
  __shared__ uint16_t list[kRedoSpan];
  __shared__ int count;
  // a programmatic dependent of the step kernel, as the FP32-store redo pass
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t span0 = (int64_t)blockIdx.x * kRedoSpan;
  const int cnt = gather_marked(a.status, span0, a.n, list, &count);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int64_t i = span0 + list[q];
    const Loc l6 = locate<6>(i, a.n, a.soa, a.lw);
    const RhoLoc lr = locate_rho(i, a.n, a.soa, a.lw);
    const Loc l3 = locate<3>(i, a.n, a.soa, a.lw);
    double p[6], C[21], hc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, cinc;
    bool shrink;
    load_compressed(a, l6, lr, p, C);
    constexpr int nhc = KIND == kP2z ? 3 : 6;
#pragma unroll
    for (int c = 0; c < nhc; ++c) hc[c] = a.hitcov[l6.base + c * l6.stride];
    const double qf = a.charge[i];
    const double surf = a.surf[a.surf_per_track ? i : 0];
    const double hx = a.hit[l3.base], hy = a.hit[l3.base + l3.stride];
    unsigned st;
    if (KIND == kP2z)
      st = p2z_step_t<double, kStandard>(p, C, qf, (double)a.bz, surf, hx, hy, hc[0], hc[1],
                                         hc[2], shrink);
    else
      st = p2r_step_t<double, kStandard>(p, C, qf, (double)a.bz, surf, hx, hy,
                                         (double)a.hit[l3.base + 2 * l3.stride], hc, shrink, cinc);
    float pf[6], Cf[21];
#pragma unroll
    for (int c = 0; c < 6; ++c) pf[c] = (float)p[c];
#pragma unroll
    for (int e = 0; e < 21; ++e) Cf[e] = (float)C[e];
    st |= finite_status(pf, Cf);
    store_compressed(a, l6, lr, pf, Cf, st);
    a.status[i] = (uint8_t)st;
  }
}

}  // namespace
}  // namespace kf

extern "C" int kf_propagate_update_compressed(
    int32_t kind, const kf_params *params, kf_layout layout, const float *state_in,
    const float *sigma_in, const uint16_t *rho_in, float *state_out, float *sigma_out,
    uint16_t *rho_out, const int8_t *charge, const float *hit, const float *hit_cov,
    const float *surf, int32_t surf_per_track, uint8_t *status, void *stream) {
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
  if (d.n == 0) return KF_OK;
  if (surf_per_track != 0 && surf_per_track != 1)
    return set_error(KF_ERR_ARG, "surf_per_track must be 0 or 1");
  const void *fptrs[] = {state_in, sigma_in, rho_in, state_out, sigma_out, rho_out, hit, hit_cov};
  for (const void *q : fptrs)
    if (!aligned16(q)) return set_error(KF_ERR_ARG, "arrays must be 16-byte aligned");
  const int64_t b6 = 4 * layout_floats(d, 6), b15 = 2 * layout_floats(d, 15);
  const void *ptrs[] = {state_in, sigma_in, rho_in, state_out, sigma_out,
                        rho_out,  charge,   hit,    hit_cov,   surf};
  const int64_t bytes[] = {b6,  b6,  b15, b6, b6, b15, d.n, 4 * layout_floats(d, 3), b6,
                           surf_per_track ? 4 * d.n : 4};
  const char *names[] = {"state_in", "sigma_in", "rho_in", "state_out", "sigma_out",
                         "rho_out",  "charge",   "hit",    "hit_cov",   "surf"};
  bool plain_loads = false;  // some array in host or managed memory
  for (int k = 0; k < 10; ++k) {
    bool nd = false;
    if (int rc = check_device_range(ptrs[k], bytes[k], names[k], &nd)) return rc;
    plain_loads |= nd;
  }
  if (status) {
    bool nd = false;
    if (int rc = check_device_range(status, d.n, "status", &nd)) return rc;
    plain_loads |= nd;
  }
  if (!status && params->precision == KF_ADAPTIVE)
    return set_error(KF_ERR_ARG, "KF_ADAPTIVE needs a status array (its redo pass reads it)");
  if (partial_overlap(state_in, b6, state_out, b6) || partial_overlap(sigma_in, b6, sigma_out, b6) ||
      partial_overlap(rho_in, b15, rho_out, b15))
    return set_error(KF_ERR_ARG, "input and output overlap without coinciding");

  CompressedArgs a{state_in, sigma_in, reinterpret_cast<const __half *>(rho_in),
                   state_out, sigma_out, reinterpret_cast<__half *>(rho_out),
                   charge, hit, hit_cov, surf, status, d.n, d.soa, d.lw, params->bz,
                   surf_per_track};
  const int threads = 128;  // as the FP32-store step kernel
  const int64_t blocks = (d.n + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return set_error(KF_ERR_ARG, "n too large for one launch");
  const unsigned g = (unsigned)blocks;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // AoSoA in device memory with a float-arithmetic variant: the staged
  // kernel (same results)
  const bool staged = !d.soa && !plain_loads && step_kernel_mode() != KF_STEP_DIRECT &&
                      (params->precision == KF_FP32 || params->precision == KF_JOSEPH ||
                       params->precision == KF_ADAPTIVE);
  if (staged) {
    if (int rc = launch_compressed_staged(kind, params->precision, a, s)) return rc;
  } else if (kind == KF_P2Z) {
    switch (params->precision) {
      case KF_FP32: step_compressed_kernel<kP2z, kFP32><<<g, threads, 0, s>>>(a); break;
      case KF_FP64_UPDATE: step_compressed_kernel<kP2z, kFP64Update><<<g, threads, 0, s>>>(a); break;
      case KF_JOSEPH: step_compressed_kernel<kP2z, kJoseph><<<g, threads, 0, s>>>(a); break;
      case KF_FP64: step_compressed_kernel<kP2z, kFP64><<<g, threads, 0, s>>>(a); break;
      case KF_DF_UPDATE: step_compressed_kernel<kP2z, kDFUpdate><<<g, threads, 0, s>>>(a); break;
      default: step_compressed_kernel<kP2z, kAdaptive><<<g, threads, 0, s>>>(a); break;
    }
  } else {
    switch (params->precision) {
      case KF_FP32: step_compressed_kernel<kP2r, kFP32><<<g, threads, 0, s>>>(a); break;
      case KF_FP64_UPDATE: step_compressed_kernel<kP2r, kFP64Update><<<g, threads, 0, s>>>(a); break;
      case KF_JOSEPH: step_compressed_kernel<kP2r, kJoseph><<<g, threads, 0, s>>>(a); break;
      case KF_FP64: step_compressed_kernel<kP2r, kFP64><<<g, threads, 0, s>>>(a); break;
      case KF_DF_UPDATE: step_compressed_kernel<kP2r, kDFUpdate><<<g, threads, 0, s>>>(a); break;
      default: step_compressed_kernel<kP2r, kAdaptive><<<g, threads, 0, s>>>(a); break;
    }
  }
  if (int rc = check_cuda(cudaGetLastError(), "compressed step launch")) return rc;
  if (params->precision != KF_ADAPTIVE) return KF_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((d.n + kRedoSpan - 1) / kRedoSpan));
  cfg.blockDim = dim3(kRedoThreads);  // a block gathers its span of kRedoSpan
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = kind == KF_P2Z ? cudaLaunchKernelEx(&cfg, redo_compressed_kernel<kP2z>, a)
                                       : cudaLaunchKernelEx(&cfg, redo_compressed_kernel<kP2r>, a);
  return check_cuda(e, "compressed redo pass launch");
}
