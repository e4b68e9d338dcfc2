// kf_device.cuh -- per-track device arithmetic of the Kalman step (sm_103a).
//
// Paper section 2: each track is propagated to a surface at fixed z
// (propagateToZ) or fixed r (propagateToR) and then Kalman-updated
// (KalmanUpdate).  The paper gives no formulas; this file implements the
// exact helix in a uniform field bz, its transport Jacobian and the linear
// Kalman update, in registers, one track per thread.  The arithmetic is
// written once for a scalar type T: T = float is the bulk path, T = double
// serves the FP64 variant and the FP64 redo of ill-conditioned tracks.
//
// Design notes (what differs from a textbook transcription):
//  * The helix uses the half-angle form (chord = 2 sin(h)/omega with
//    h = omega*s/2), so nothing cancels as omega -> 0 (high pT).
//  * The cylinder crossing (p2r) is solved in closed form through the
//    tangent of the half turning angle: |P0 + chord*u(phi+h)|^2 = R^2 is a
//    quadratic in tan(h) * 2/omega, whose stable root gives cos(h), sin(h)
//    and the chord with one sqrt and no trigonometry; atan2 recovers h.
//  * The Jacobian's zero/unit pattern is a compile-time mask, so
//    C' = J C J^T costs only the structurally non-zero products.
//  * p2r transports and updates the covariance in the surface frame, whose
//    radial row is exactly zero, and rotates back at the end.
//  * Columns of a measured component use the cancellation-free posterior
//    C' H^T S^-1 V H^-T instead of C' - K U^T.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kf {

constexpr unsigned kNoIntersect = 1u;
constexpr unsigned kSNotPD = 2u;
constexpr unsigned kBadK = 4u;
constexpr unsigned kNonFinite = 8u;

// Update variants (the KF_* precision values of the C ABI).
enum Variant : int { kFP32 = 0, kFP64Update = 1, kJoseph = 2, kFP64 = 3, kAdaptive = 4 };
// Step kinds.
enum Kind : int { kP2z = 0, kP2r = 1 };

// Tracks whose FP32 step is ill-conditioned get an FP64 redo under
// kAdaptive: a measured variance shrunk by more than kRedoShrink by the hit,
// or a cylinder crossed at an incidence cosine below kRedoGrazing.
constexpr float kRedoShrink = 1e4f;
constexpr float kRedoGrazing = 0.2f;

// Scalar-type traits: math functions and constants for float and double.
template <class T>
struct Fp;

template <>
struct Fp<float> {
  static constexpr float alpha = 0.299792458e-2f;  // GeV / (cm T), unit charge
  static constexpr float pi = 3.14159265358979f;
  static constexpr float two_pi_hi = 6.28318548202514648f;     // float(2 pi)
  static constexpr float two_pi_lo = -1.7484555314695172e-7f;  // 2 pi - float(2 pi)
  static constexpr float inv_two_pi = 0.15915494309189535f;
  static constexpr float dsinc_series = 0.25f;  // below: Taylor series for S'(h)
  static __device__ __forceinline__ void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
  static __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
  static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
  static __device__ __forceinline__ float rint_(float x) { return rintf(x); }
  // Quotients of well-scaled operands (|b| far below 2^126): the fast
  // reciprocal-based division, within 2 ulp, instead of the IEEE sequence.
  static __device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float rcp_(float b) { return __fdividef(1.0f, b); }
};

template <>
struct Fp<double> {
  static constexpr double alpha = 0.299792458e-2;
  static constexpr double pi = 3.141592653589793;
  static constexpr double two_pi_hi = 6.283185307179586;
  static constexpr double two_pi_lo = 2.4492935982947064e-16;
  static constexpr double inv_two_pi = 0.15915494309189535;
  static constexpr double dsinc_series = 0.05;
  static __device__ __forceinline__ void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
  static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
  static __device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
  static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
  static __device__ __forceinline__ double rint_(double x) { return rint(x); }
  static __device__ __forceinline__ double div_(double a, double b) { return a / b; }
  static __device__ __forceinline__ double rcp_(double b) { return 1.0 / b; }
};

// Packed lower-triangular index of a symmetric matrix element.
__host__ __device__ constexpr int tri(int i, int j) {
  return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

constexpr uint64_t bit(int i, int j) { return 1ull << (i * 6 + j); }

// Structural non-zeros (NZ) and unit entries (ONE) of the transport
// Jacobian, row = output component, column = input component, components
// ordered (x, y, z, k, phi, theta).
// p2z: z' is pinned to the plane (zero row); x', y', phi' depend on z and
// theta through the path length s = (zt - z) tan(theta).
constexpr uint64_t kP2zNZ =
    bit(0, 0) | bit(0, 2) | bit(0, 3) | bit(0, 4) | bit(0, 5) |
    bit(1, 1) | bit(1, 2) | bit(1, 3) | bit(1, 4) | bit(1, 5) |
    bit(3, 3) |
    bit(4, 2) | bit(4, 3) | bit(4, 4) | bit(4, 5) |
    bit(5, 5);
constexpr uint64_t kP2zOne = bit(0, 0) | bit(1, 1) | bit(3, 3) | bit(4, 4) | bit(5, 5);
// p2r in the surface frame at the crossing point, rows (t, r, z', k, phi', theta):
// t is the tangential and r the radial position coordinate.  The radial row
// n.J is identically zero (the crossing stays on the cylinder), so it is
// structurally zero here and C' has an exactly zero radial row and column.
constexpr uint64_t kP2rFrameNZ =
    bit(0, 0) | bit(0, 1) | bit(0, 3) | bit(0, 4) |
    bit(2, 0) | bit(2, 1) | bit(2, 2) | bit(2, 3) | bit(2, 4) | bit(2, 5) |
    bit(3, 3) |
    bit(4, 0) | bit(4, 1) | bit(4, 3) | bit(4, 4) |
    bit(5, 5);
constexpr uint64_t kP2rFrameOne = bit(2, 2) | bit(3, 3) | bit(5, 5);

// Azimuth wrapped to (-pi, pi]: subtract the nearest multiple of 2 pi in two
// parts (the rounded 2 pi and its remainder), so the wrap adds no error of
// its own beyond the final rounding.
template <class T>
__device__ __forceinline__ T wrap_phi(T a) {
  using F = Fp<T>;
  const T n = F::rint_(a * F::inv_two_pi);
  T w = F::fma_(-n, F::two_pi_hi, a);
  w = F::fma_(-n, F::two_pi_lo, w);
  if (w <= -F::pi) w += F::two_pi_hi;
  return w;
}

// S(h) = sin(h)/h given sin(h); S(0) = 1.
template <class T>
__device__ __forceinline__ T sinc_from(T h, T sh) {
  return Fp<T>::abs_(h) < T(1e-4) ? Fp<T>::fma_(-h * h, T(1) / T(6), T(1)) : Fp<T>::div_(sh, h);
}

// dS/dh = (cos(h) - S(h)) / h; the difference cancels for small |h|, where
// the Taylor series -h/3 + h^3/30 - h^5/840 + h^7/45360 is used instead.
template <class T>
__device__ __forceinline__ T dsinc_from(T h, T ch, T S) {
  using F = Fp<T>;
  if (F::abs_(h) < F::dsinc_series) {
    const T h2 = h * h;
    return h * F::fma_(h2, F::fma_(h2, F::fma_(h2, T(1) / T(45360), T(-1) / T(840)),
                                   T(1) / T(30)),
                       T(-1) / T(3));
  }
  return F::div_(ch - S, h);
}

// C' = J C J^T for packed symmetric C, with J's structure fixed by NZ/ONE.
// Loops unroll completely, so every mask test folds at compile time and
// only the structurally non-zero multiply-adds remain.
template <class T, uint64_t NZ, uint64_t ONE>
__device__ __forceinline__ void transport(const T (&J)[36], const T (&C)[21], T (&Co)[21]) {
  using F = Fp<T>;
  T M[6][6];  // M = J C
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      T acc = T(0);
      bool first = true;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if ((NZ >> (i * 6 + l)) & 1ull) {
          const T c = C[tri(l, j)];
          if ((ONE >> (i * 6 + l)) & 1ull)
            acc = first ? c : acc + c;
          else
            acc = first ? J[i * 6 + l] * c : F::fma_(J[i * 6 + l], c, acc);
          first = false;
        }
      }
      M[i][j] = acc;
    }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int m = 0; m <= i; ++m) {
      if (((NZ >> (i * 6)) & 0x3Full) == 0 || ((NZ >> (m * 6)) & 0x3Full) == 0) {
        Co[tri(i, m)] = T(0);  // a zero row of J gives a zero row of C'
        continue;
      }
      T acc = T(0);
      bool first = true;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if ((NZ >> (m * 6 + l)) & 1ull) {
          if ((ONE >> (m * 6 + l)) & 1ull)
            acc = first ? M[i][l] : acc + M[i][l];
          else
            acc = first ? M[i][l] * J[m * 6 + l] : F::fma_(M[i][l], J[m * 6 + l], acc);
          first = false;
        }
      }
      Co[tri(i, m)] = acc;
    }
  }
}

// ------------------------------------------------------------------- p2z
// Propagate to the plane z = zt.  Returns false (nothing written) when the
// track is parallel to the plane (|cos(theta)| <= 1e-4).
template <class T>
__device__ __forceinline__ bool propagate_to_z(const T (&in)[6], T qf, T bz, T zt, T (&out)[6],
                                               T (&J)[36]) {
  using F = Fp<T>;
  const T x = in[0], y = in[1], z = in[2], k = in[3], phi = in[4], th = in[5];
  T sp, cp, st, ct;
  F::sincos_(phi, &sp, &cp);
  F::sincos_(th, &st, &ct);
  if (!(F::abs_(ct) > T(1e-4))) return false;
  const T ict = F::rcp_(ct);
  const T tanth = st * ict;
  const T dz = zt - z;
  const T s = dz * tanth;                 // transverse path to the plane
  const T dwdk = -qf * F::alpha * bz;     // d omega / d k
  const T omega = dwdk * k;
  const T h = T(0.5) * omega * s;         // half turning angle
  T sh, ch;
  F::sincos_(h, &sh, &ch);
  const T S = sinc_from(h, sh);
  const T dS = dsinc_from(h, ch, S);
  const T L = s * S;                      // chord length
  const T cpm = cp * ch - sp * sh;        // cos(phi + h)
  const T spm = sp * ch + cp * sh;        // sin(phi + h)
  const T cp1 = cpm * ch - spm * sh;      // cos(phi + 2h)
  const T sp1 = spm * ch + cpm * sh;      // sin(phi + 2h)

  out[0] = F::fma_(L, cpm, x);
  out[1] = F::fma_(L, spm, y);
  out[2] = zt;
  out[3] = k;
  out[4] = wrap_phi(phi + T(2) * h);
  out[5] = th;

  // Partials at fixed s, then the path-length terms ds/dz = -tan(theta),
  // ds/dtheta = (zt - z) / cos^2(theta) along dp'/ds = (cos, sin, ., 0, omega, 0).
  const T hs2 = T(0.5) * s * s * dwdk;
  const T Xk = hs2 * (dS * cpm - S * spm);
  const T Yk = hs2 * (dS * spm + S * cpm);
  const T dsz = -tanth;
  const T dsth = dz * ict * ict;
#pragma unroll
  for (int e = 0; e < 36; ++e) J[e] = T(0);
  J[0 * 6 + 2] = cp1 * dsz;
  J[0 * 6 + 3] = Xk;
  J[0 * 6 + 4] = -L * spm;
  J[0 * 6 + 5] = cp1 * dsth;
  J[1 * 6 + 2] = sp1 * dsz;
  J[1 * 6 + 3] = Yk;
  J[1 * 6 + 4] = L * cpm;
  J[1 * 6 + 5] = sp1 * dsth;
  J[4 * 6 + 2] = omega * dsz;
  J[4 * 6 + 3] = s * dwdk;
  J[4 * 6 + 5] = omega * dsth;
  return true;
}

// ------------------------------------------------------------------- p2r
// Propagate to the first outward crossing of the cylinder r = R.  Returns
// false when the track starts on/outside the cylinder or never reaches it.
// rcos receives R times the cosine between the track direction and the
// surface normal at the crossing (the incidence test needs no division).
//
// With A = P0.t0, B = P0.n0 (t0 = (cos phi, sin phi), n0 = (-sin, cos)),
// d = R^2 - |P0|^2 and t = tan(h), the crossing condition becomes
//   (1 + omega B - d omega^2/4) tau^2 + 2 A tau - d = 0,  tau = 2 t / omega,
// whose first-crossing root is tau = d / (A + sqrt(A^2 + a2 d)).  Then
//   (cos h, sin h) = (2 (A + sqrt(.)), omega d) / norm,  chord = 2 d / norm.
template <class T>
__device__ __forceinline__ bool propagate_to_r(const T (&in)[6], T qf, T bz, T R, T (&out)[6],
                                               T (&J)[36], T &rcos) {
  using F = Fp<T>;
  const T x = in[0], y = in[1], z = in[2], k = in[3], phi = in[4], th = in[5];
  const T r0sq = F::fma_(x, x, y * y);
  const T d = F::fma_(R, R, -r0sq);
  if (!(d > T(0))) return false;
  T sp, cp, st, ct;
  F::sincos_(phi, &sp, &cp);
  F::sincos_(th, &st, &ct);
  const T dwdk = -qf * F::alpha * bz;
  const T omega = dwdk * k;
  const T A = F::fma_(x, cp, y * sp);
  const T B = F::fma_(y, cp, -x * sp);
  const T a2 = F::fma_(omega, B, F::fma_(T(-0.25) * d * omega, omega, T(1)));
  const T D = F::fma_(A, A, a2 * d);
  if (!(D >= T(0))) return false;
  const T den = A + F::sqrt_(D);
  const T yv = omega * d;
  const T xv = T(2) * den;
  const T inv = F::rsqrt_(F::fma_(xv, xv, yv * yv));
  const T ch = xv * inv;                  // cos(h)
  const T sh = yv * inv;                  // sin(h)
  const T h = F::atan2_(yv, xv);          // half turning angle
  const T L = T(2) * d * inv;             // chord
  const T s = F::abs_(omega) > T(1e-12) ? F::div_(T(2) * h, omega) : F::div_(d, den);
  const T ist = F::rcp_(st);
  const T cot = ct * ist;
  const T S = sinc_from(h, sh);
  const T dS = dsinc_from(h, ch, S);
  const T cpm = cp * ch - sp * sh;
  const T spm = sp * ch + cp * sh;
  const T cp1 = cpm * ch - spm * sh;
  const T sp1 = spm * ch + cpm * sh;

  const T x1 = F::fma_(L, cpm, x);
  const T y1 = F::fma_(L, spm, y);
  out[0] = x1;
  out[1] = y1;
  out[2] = F::fma_(s, cot, z);
  out[3] = k;
  out[4] = wrap_phi(phi + T(2) * h);
  out[5] = th;

  // Fixed-s partials.
  const T hs2 = T(0.5) * s * s * dwdk;
  const T Xk = hs2 * (dS * cpm - S * spm);
  const T Yk = hs2 * (dS * spm + S * cpm);
  const T Xphi = -L * spm;
  const T Yphi = L * cpm;
  // s(p) from g = x'^2 + y'^2 - R^2 = 0: ds/dp = -(x' dx'/dp + y' dy'/dp) / (x' cos + y' sin).
  const T gs = F::fma_(x1, cp1, y1 * sp1);
  rcos = gs;
  const T ig = -F::rcp_(gs);
  const T dsx = ig * x1;
  const T dsy = ig * y1;
  const T dsk = ig * F::fma_(x1, Xk, y1 * Yk);
  const T dsphi = ig * F::fma_(x1, Xphi, y1 * Yphi);
#pragma unroll
  for (int e = 0; e < 36; ++e) J[e] = T(0);
  J[0 * 6 + 0] = F::fma_(cp1, dsx, T(1));
  J[0 * 6 + 1] = cp1 * dsy;
  J[0 * 6 + 3] = F::fma_(cp1, dsk, Xk);
  J[0 * 6 + 4] = F::fma_(cp1, dsphi, Xphi);
  J[1 * 6 + 0] = sp1 * dsx;
  J[1 * 6 + 1] = F::fma_(sp1, dsy, T(1));
  J[1 * 6 + 3] = F::fma_(sp1, dsk, Yk);
  J[1 * 6 + 4] = F::fma_(sp1, dsphi, Yphi);
  J[2 * 6 + 0] = cot * dsx;
  J[2 * 6 + 1] = cot * dsy;
  J[2 * 6 + 3] = cot * dsk;
  J[2 * 6 + 4] = cot * dsphi;
  J[2 * 6 + 5] = -s * ist * ist;
  J[4 * 6 + 0] = omega * dsx;
  J[4 * 6 + 1] = omega * dsy;
  J[4 * 6 + 3] = F::fma_(omega, dsk, s * dwdk);
  J[4 * 6 + 4] = F::fma_(omega, dsphi, T(1));
  return true;
}

// ---------------------------------------------------------------- update
// Update forms below the variants: the standard form in T, the standard form
// with S^-1, K and C'' in double (from float inputs), the Joseph form.
enum UpdateForm : int { kStandard = 0, kStandardF64 = 1, kJosephForm = 2 };

// Two-row Kalman update in a frame where the measurement is
//   row 0: h0 * (component 0),   row 1: component M1,
// and component SKIP has a structurally zero row and column in C' (the
// surface normal: z for p2z, the radial coordinate for p2r in the surface
// frame), so its gain row is skipped and stays zero.  U = C' H^T (columns
// U0, U1), S = H U + V, r the residual.  Returns kSNotPD (state untouched)
// or 0.
//
// Except under the Joseph form, every element with a measured column uses
// C' - K U^T = C' H^T S^-1 V H^-T (because I - S^-1 (S - V) = S^-1 V): a
// precise hit shrinks the measured variances by orders of magnitude, and in
// the subtracted form those digits would cancel away.
template <class T, int FORM, int SKIP, int M1>
__device__ __forceinline__ unsigned kalman_update(T (&p)[6], T (&C)[21], const T (&U0)[6],
                                                  const T (&U1)[6], T S00, T S01, T S11, T h0,
                                                  T V00, T V01, T V11, T r0, T r1) {
  using F = Fp<T>;
  if constexpr (FORM == kStandardF64) {
    const double dS00 = S00, dS01 = S01, dS11 = S11;
    const double det = dS00 * dS11 - dS01 * dS01;
    if (!(dS00 > 0.0) || !(det > 0.0)) return kSNotPD;
    const double inv = 1.0 / det;
    const double Si00 = dS11 * inv, Si01 = -dS01 * inv, Si11 = dS00 * inv;
    double K0[6], K1[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i == SKIP) continue;
      K0[i] = (double)U0[i] * Si00 + (double)U1[i] * Si01;
      K1[i] = (double)U0[i] * Si01 + (double)U1[i] * Si11;
      p[i] = (T)((double)p[i] + K0[i] * (double)r0 + K1[i] * (double)r1);
    }
    const double G00 = Si00 * V00 + Si01 * V01, G01 = Si00 * V01 + Si01 * V11;
    const double G10 = Si01 * V00 + Si11 * V01, G11 = Si01 * V01 + Si11 * V11;
    const double ih0 = 1.0 / (double)h0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i == SKIP) continue;
#pragma unroll
      for (int m = 0; m <= i; ++m) {
        if (m == SKIP) continue;
        const bool im = (i == 0 || i == M1), mm = (m == 0 || m == M1);
        double v;
        if (mm || im) {
          const int r = mm ? i : m, c = mm ? m : i;  // row r, measured column c
          v = (c == 0) ? ((double)U0[r] * G00 + (double)U1[r] * G10) * ih0
                       : (double)U0[r] * G01 + (double)U1[r] * G11;
        } else {
          v = (double)C[tri(i, m)] - (K0[i] * (double)U0[m] + K1[i] * (double)U1[m]);
        }
        C[tri(i, m)] = (T)v;
      }
    }
    return 0u;
  } else {
    const T det = F::fma_(S00, S11, -S01 * S01);
    if (!(S00 > T(0)) || !(det > T(0))) return kSNotPD;
    const T inv = F::rcp_(det);
    const T Si00 = S11 * inv, Si01 = -S01 * inv, Si11 = S00 * inv;
    T K0[6], K1[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i == SKIP) {
        K0[i] = K1[i] = T(0);
        continue;
      }
      K0[i] = F::fma_(U0[i], Si00, U1[i] * Si01);
      K1[i] = F::fma_(U0[i], Si01, U1[i] * Si11);
      p[i] = F::fma_(K0[i], r0, F::fma_(K1[i], r1, p[i]));
    }
    if constexpr (FORM == kJosephForm) {
      // Product (Joseph) form: B = (I - K H) C' = C' - K U^T, then
      // C'' = B (I - K H)^T + K V K^T = B - (B H0^T) K0^T - (B H1^T) K1^T + K V K^T,
      // a sum of positive semi-definite terms for any gain K.
      T B[6][6];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j)
          B[i][j] = C[tri(i, j)] - F::fma_(K0[i], U0[j], K1[i] * U1[j]);
      T b0[6], b1[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        b0[i] = h0 * B[i][0];
        b1[i] = B[i][M1];
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i == SKIP) continue;
        const T kv0 = F::fma_(K0[i], V00, K1[i] * V01);
        const T kv1 = F::fma_(K0[i], V01, K1[i] * V11);
#pragma unroll
        for (int m = 0; m <= i; ++m) {
          if (m == SKIP) continue;
          T c = B[i][m];
          c = F::fma_(-b0[i], K0[m], c);
          c = F::fma_(-b1[i], K1[m], c);
          c = F::fma_(kv0, K0[m], c);
          c = F::fma_(kv1, K1[m], c);
          C[tri(i, m)] = c;
        }
      }
      return 0u;
    } else {
      const T G00 = F::fma_(Si00, V00, Si01 * V01), G01 = F::fma_(Si00, V01, Si01 * V11);
      const T G10 = F::fma_(Si01, V00, Si11 * V01), G11 = F::fma_(Si01, V01, Si11 * V11);
      const T ih0 = F::rcp_(h0);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i == SKIP) continue;
#pragma unroll
        for (int m = 0; m <= i; ++m) {
          if (m == SKIP) continue;
          const bool im = (i == 0 || i == M1), mm = (m == 0 || m == M1);
          if (mm || im) {
            const int r = mm ? i : m, c = mm ? m : i;  // row r, measured column c
            C[tri(i, m)] = (c == 0) ? F::fma_(U0[r], G00, U1[r] * G10) * ih0
                                    : F::fma_(U0[r], G01, U1[r] * G11);
          } else {
            C[tri(i, m)] = C[tri(i, m)] - F::fma_(K0[i], U0[m], K1[i] * U1[m]);
          }
        }
      }
      return 0u;
    }
  }
}

// ------------------------------------------------------------ full steps
// One p2z step in scalar type T.  p/C hold the input and receive the result.
// ill (named shrink) is set to 1 when the hit shrinks a measured variance by
// more than kRedoShrink (the update is ill-conditioned in FP32), else 0.
template <class T, int FORM>
__device__ __forceinline__ unsigned p2z_step_t(T (&p)[6], T (&C)[21], T qf, T bz, T zt, T hx,
                                               T hy, T vxx, T vxy, T vyy, T &shrink) {
  T pp[6], J[36], Cp[21];
  shrink = T(0);
  if (!propagate_to_z(p, qf, bz, zt, pp, J)) return kNoIntersect;
  transport<T, kP2zNZ, kP2zOne>(J, C, Cp);
  // H = [e_x; e_y]: U = columns x and y of C' (its z row and column are zero).
  T U0[6], U1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    U0[i] = Cp[tri(i, 0)];
    U1[i] = Cp[tri(i, 1)];
  }
  const T S00 = U0[0] + vxx, S01 = U0[1] + vxy, S11 = U1[1] + vyy;
  // ill-conditioned when the hit shrinks a measured variance by > kRedoShrink
  shrink = (S00 > T(kRedoShrink) * vxx || S11 > T(kRedoShrink) * vyy) ? T(1) : T(0);
  const unsigned st = kalman_update<T, FORM, 2, 1>(pp, Cp, U0, U1, S00, S01, S11, T(1), vxx, vxy,
                                                   vyy, hx - pp[0], hy - pp[1]);
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = pp[i];
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = Cp[e];
  if (!st) p[4] = wrap_phi(p[4]);
  return st | (p[3] > T(0) ? 0u : kBadK);
}

// One p2r step in scalar type T.  hc = packed 3x3 hit covariance.
//
// The covariance is transported and updated in the surface frame at the
// crossing point P' = R (cos a, sin a): position coordinates t (along
// (-sin a, cos a)) and r (along (cos a, sin a)).  The radial row of the
// Jacobian is identically zero, so C' has an exactly zero radial row and
// column there; rotating the updated covariance back gives
// C_xx = sin^2 a C_tt, C_xy = -sin a cos a C_tt, ..., which keeps full
// relative precision even where an axis is nearly radial.
template <class T, int FORM>
__device__ __forceinline__ unsigned p2r_step_t(T (&p)[6], T (&C)[21], T qf, T bz, T R, T hx,
                                               T hy, T hz, const T (&hc)[6], T &shrink,
                                               T &rcos) {
  using F = Fp<T>;
  T pp[6], J[36], Cp[21];
  shrink = T(0);
  rcos = R;
  if (!propagate_to_r(p, qf, bz, R, pp, J, rcos)) return kNoIntersect;
  const T ip = F::rsqrt_(F::fma_(pp[0], pp[0], pp[1] * pp[1]));
  const T ca = pp[0] * ip, sa = pp[1] * ip;  // direction of P'
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    J[0 * 6 + j] = F::fma_(-sa, J[0 * 6 + j], ca * J[1 * 6 + j]);  // t row
    J[1 * 6 + j] = T(0);                                          // r row: zero
  }
  transport<T, kP2rFrameNZ, kP2rFrameOne>(J, C, Cp);
  // Measurement direction at the hit, u = (-sin phi_h, cos phi_h), and z.
  // In the frame u acts on t with weight u.t = cos(phi_h - a) (the radial
  // column of C' is zero).
  const T ir = F::rsqrt_(F::fma_(hx, hx, hy * hy));
  const T ux = -hy * ir, uy = hx * ir;
  const T ut = F::fma_(-sa, ux, ca * uy);
  T U0[6], U1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    U0[i] = ut * Cp[tri(i, 0)];
    U1[i] = Cp[tri(i, 2)];
  }
  // V = P V_hit P^T with P = [[ux, uy, 0], [0, 0, 1]].
  const T V00 = F::fma_(ux * ux, hc[0], F::fma_(T(2) * ux * uy, hc[1], uy * uy * hc[2]));
  const T V01 = F::fma_(ux, hc[3], uy * hc[4]);
  const T V11 = hc[5];
  const T S00 = F::fma_(ut, U0[0], V00);
  const T S01 = U0[2] + V01;
  const T S11 = U1[2] + V11;
  shrink = (S00 > T(kRedoShrink) * V00 || S11 > T(kRedoShrink) * V11) ? T(1) : T(0);
  const T r0 = F::fma_(ux, hx - pp[0], uy * (hy - pp[1]));
  const T r1 = hz - pp[2];
  // frame state: the position offsets (t, r) start at 0 on P'
  T pf[6] = {T(0), T(0), pp[2], pp[3], pp[4], pp[5]};
  const unsigned st = kalman_update<T, FORM, 1, 2>(pf, Cp, U0, U1, S00, S01, S11, ut, V00, V01,
                                                   V11, r0, r1);
  p[0] = F::fma_(-sa, pf[0], pp[0]);
  p[1] = F::fma_(ca, pf[0], pp[1]);
#pragma unroll
  for (int i = 2; i < 6; ++i) p[i] = pf[i];
  // back to (x, y): only the t row/column carries position variance
  const T ctt = Cp[tri(0, 0)];
  C[tri(0, 0)] = sa * sa * ctt;
  C[tri(1, 0)] = -sa * ca * ctt;
  C[tri(1, 1)] = ca * ca * ctt;
#pragma unroll
  for (int j = 2; j < 6; ++j) {
    const T ctj = Cp[tri(j, 0)];
    C[tri(j, 0)] = -sa * ctj;
    C[tri(j, 1)] = ca * ctj;
#pragma unroll
    for (int m = 2; m <= j; ++m) C[tri(j, m)] = Cp[tri(j, m)];
  }
  if (!st) p[4] = wrap_phi(p[4]);
  return st | (p[3] > T(0) ? 0u : kBadK);
}

// Run a T = double step on float registers (convert in and out).  Kept out
// of line so that the float path's register allocation does not carry it.
template <int KIND>
__device__ __noinline__ unsigned step_in_double(float (&p)[6], float (&C)[21], float qf, float bz,
                                                float surf, float hx, float hy, float hz,
                                                const float (&hc)[6]) {
  double dp[6], dC[21], dhc[6], shrink, cinc;
#pragma unroll
  for (int i = 0; i < 6; ++i) dp[i] = p[i];
#pragma unroll
  for (int e = 0; e < 21; ++e) dC[e] = C[e];
#pragma unroll
  for (int i = 0; i < 6; ++i) dhc[i] = hc[i];
  unsigned st;
  if (KIND == kP2z)
    st = p2z_step_t<double, kStandard>(dp, dC, qf, bz, surf, hx, hy, dhc[0], dhc[1], dhc[2],
                                       shrink);
  else
    st = p2r_step_t<double, kStandard>(dp, dC, qf, bz, surf, hx, hy, hz, dhc, shrink, cinc);
  if (!(st & kNoIntersect)) {
#pragma unroll
    for (int i = 0; i < 6; ++i) p[i] = (float)dp[i];
#pragma unroll
    for (int e = 0; e < 21; ++e) C[e] = (float)dC[e];
  }
  return st;
}

// Status bit (internal, never stored) with which a kAdaptive step asks its
// kernel to redo the track in FP64 from the original inputs.
constexpr unsigned kRedo = 0x80u;

// The step of a variant on float registers.  kFP32 / kJoseph / kFP64Update
// run in float (with their update form); kFP64 runs every operation in
// double.  kAdaptive runs in float and, when the step is ill-conditioned (the
// hit shrinks a measured variance by more than kRedoShrink, or a cylinder is
// crossed at an incidence cosine below kRedoGrazing), returns kRedo: the
// caller then reloads the track's inputs and calls step_in_double -- FP64
// where the conditioning demands it, FP32 for everything else, and no
// register copies of the inputs on the common path.
template <int KIND, int VARIANT>
__device__ __forceinline__ unsigned step_variant(float (&p)[6], float (&C)[21], float qf,
                                                 float bz, float surf, float hx, float hy,
                                                 float hz, const float (&hc)[6]) {
  if constexpr (VARIANT == kFP64) {
    return step_in_double<KIND>(p, C, qf, bz, surf, hx, hy, hz, hc);
  } else {
    constexpr int FORM = VARIANT == kJoseph ? kJosephForm
                         : VARIANT == kFP64Update ? kStandardF64 : kStandard;
    float ill, rcos = surf;
    unsigned st;
    if (KIND == kP2z)
      st = p2z_step_t<float, FORM>(p, C, qf, bz, surf, hx, hy, hc[0], hc[1], hc[2], ill);
    else
      st = p2r_step_t<float, FORM>(p, C, qf, bz, surf, hx, hy, hz, hc, ill, rcos);
    if constexpr (VARIANT == kAdaptive) {
      if (!(st & kNoIntersect) && (ill != 0.0f || !(fabsf(rcos) >= kRedoGrazing * surf)))
        st |= kRedo;
    }
    return st;
  }
}

// Convenience entry points used by the kernels.  Under kAdaptive the
// returned status may carry kRedo (see step_variant).
template <int VARIANT>
__device__ __forceinline__ unsigned p2z_step(float (&p)[6], float (&C)[21], float qf, float bz,
                                             float zt, float hx, float hy, float vxx, float vxy,
                                             float vyy) {
  const float hc[6] = {vxx, vxy, vyy, 0.0f, 0.0f, 0.0f};
  return step_variant<kP2z, VARIANT>(p, C, qf, bz, zt, hx, hy, 0.0f, hc);
}

template <int VARIANT>
__device__ __forceinline__ unsigned p2r_step(float (&p)[6], float (&C)[21], float qf, float bz,
                                             float R, float hx, float hy, float hz,
                                             const float (&hc)[6]) {
  return step_variant<kP2r, VARIANT>(p, C, qf, bz, R, hx, hy, hz, hc);
}

// Non-finite check over the written result (any NaN/Inf poisons the sum;
// the values are far from overflow, so a finite sum means finite entries).
__device__ __forceinline__ unsigned finite_status(const float (&p)[6], const float (&C)[21]) {
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) acc += p[i];
#pragma unroll
  for (int e = 0; e < 21; ++e) acc += C[e];
  return isfinite(acc) ? 0u : kNonFinite;
}

}  // namespace kf
