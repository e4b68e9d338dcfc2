// kf_device.cuh -- per-track device arithmetic of the Kalman step (sm_103a).
//
// Paper section 2: each track is propagated to a surface at fixed z
// (propagateToZ) or fixed r (propagateToR) and then Kalman-updated
// (KalmanUpdate).  The paper gives no formulas; this file implements the
// exact helix in a uniform field bz, its transport Jacobian and the linear
// Kalman update, in registers, one track per thread.  The arithmetic is
// written once for a number type T (kf_num.cuh): float is the bulk path,
// double serves the FP64 variants and the FP64 redo of ill-conditioned
// tracks.  Every operation is explicitly rounded, so a track's result does
// not depend on which kernel computes it.
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
//  * Per-track decisions (surface not reached, S not positive definite, the
//    series branches near h = 0) are masks, on which the code branches.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kf_num.cuh"

namespace kf {

using namespace num;

constexpr unsigned kNoIntersect = 1u;
constexpr unsigned kSNotPD = 2u;
constexpr unsigned kBadK = 4u;
constexpr unsigned kNonFinite = 8u;

// Update variants (the KF_* precision values of the C ABI).
enum Variant : int {
  kFP32 = 0,
  kFP64Update = 1,
  kJoseph = 2,
  kFP64 = 3,
  kAdaptive = 4,
  kDFUpdate = 5
};
// Step kinds.
enum Kind : int { kP2z = 0, kP2r = 1 };

// Tracks whose FP32 step is ill-conditioned get an FP64 redo under
// kAdaptive: a measured variance shrunk by more than kRedoShrink by the hit,
// a cylinder crossed at an incidence cosine below kRedoGrazing, or an update
// that leaves 1/pT at or below zero (a hit far off the track, whose update
// the FP32 rounding no longer resolves).  With a threshold of 0.2 instead
// of 0.3, tracks crossing the outer barrel layers at cosines of 0.21-0.22
// missed the covariance bound by up to 27 % in the 15-layer chain.
constexpr float kRedoShrink = 1e4f;
constexpr float kRedoGrazing = 0.3f;

// Constants per lane precision.
template <class S>
struct Consts;

template <>
struct Consts<float> {
  static constexpr double alpha = 0.299792458e-2;  // GeV / (cm T), unit charge
  static constexpr double pi = 3.14159265358979;
  static constexpr double two_pi_hi = 6.28318548202514648;     // float(2 pi)
  static constexpr double two_pi_lo = -1.7484555314695172e-7;  // 2 pi - float(2 pi)
  static constexpr double inv_two_pi = 0.15915494309189535;
  static constexpr double dsinc_series = 0.25;  // below: Taylor series for S'(h)
};

template <>
struct Consts<double> {
  static constexpr double alpha = 0.299792458e-2;
  static constexpr double pi = 3.141592653589793;
  static constexpr double two_pi_hi = 6.283185307179586;
  static constexpr double two_pi_lo = 2.4492935982947064e-16;
  static constexpr double inv_two_pi = 0.15915494309189535;
  static constexpr double dsinc_series = 0.05;
};

template <class T>
using K_ = Consts<scalar_t<T>>;

// value = m ? a() : b(), computing only the side that is taken.
template <class T, class FA, class FB>
__device__ __forceinline__ T choose(mask_t<T> m, FA &&a, FB &&b) {
  return m ? a() : b();
}

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
  using K = K_<T>;
  const T n = rint_(mul_(a, cst<T>(K::inv_two_pi)));
  T w = fma_(n, cst<T>(-K::two_pi_hi), a);
  w = fma_(n, cst<T>(-K::two_pi_lo), w);
  return choose<T>(le_(w, cst<T>(-K::pi)), [&] { return add_(w, cst<T>(K::two_pi_hi)); },
                   [&] { return w; });
}

// S(h) = sin(h)/h given sin(h); S(0) = 1.
template <class T>
__device__ __forceinline__ T sinc_from(T h, T sh) {
  return choose<T>(
      lt_(abs_(h), cst<T>(1e-4)),
      [&] { return fma_(mul_(h, h), cst<T>(-1.0 / 6.0), cst<T>(1.0)); },
      [&] { return div_(sh, h); });
}

// dS/dh = (cos(h) - S(h)) / h; the difference cancels for small |h|, where
// the Taylor series -h/3 + h^3/30 - h^5/840 + h^7/45360 is used instead.
template <class T>
__device__ __forceinline__ T dsinc_from(T h, T ch, T S) {
  return choose<T>(
      lt_(abs_(h), cst<T>(K_<T>::dsinc_series)),
      [&] {
        const T h2 = mul_(h, h);
        return mul_(h, fma_(h2,
                            fma_(h2, fma_(h2, cst<T>(1.0 / 45360.0), cst<T>(-1.0 / 840.0)),
                                 cst<T>(1.0 / 30.0)),
                            cst<T>(-1.0 / 3.0)));
      },
      [&] { return div_(sub_(ch, S), h); });
}

// C' = J C J^T for packed symmetric C, with J's structure fixed by NZ/ONE.
// Loops unroll completely, so every mask test folds at compile time and
// only the structurally non-zero multiply-adds remain.  A sum over a row of
// J that has a unit entry starts from that entry's term, so it needs no
// product.
template <class T, uint64_t NZ, uint64_t ONE>
__device__ __forceinline__ void transport(const T (&J)[36], const T (&C)[21], T (&Co)[21]) {
  T M[6][6];  // M = J C
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      T acc = cst<T>(0.0);
      bool first = true;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if (((NZ & ONE) >> (i * 6 + l)) & 1ull) {
          const T c = C[tri(l, j)];
          acc = first ? c : add_(acc, c);
          first = false;
        }
      }
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if (((NZ & ~ONE) >> (i * 6 + l)) & 1ull) {
          const T c = C[tri(l, j)];
          acc = first ? mul_(J[i * 6 + l], c) : fma_(J[i * 6 + l], c, acc);
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
        Co[tri(i, m)] = cst<T>(0.0);  // a zero row of J gives a zero row of C'
        continue;
      }
      T acc = cst<T>(0.0);
      bool first = true;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if (((NZ & ONE) >> (m * 6 + l)) & 1ull) {
          acc = first ? M[i][l] : add_(acc, M[i][l]);
          first = false;
        }
      }
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if (((NZ & ~ONE) >> (m * 6 + l)) & 1ull) {
          acc = first ? mul_(M[i][l], J[m * 6 + l]) : fma_(M[i][l], J[m * 6 + l], acc);
          first = false;
        }
      }
      Co[tri(i, m)] = acc;
    }
  }
}

// cos(phi + h), sin(phi + h), cos(phi + 2h), sin(phi + 2h) from the sines and
// cosines of phi and h (nsh = -sin h).
template <class T>
__device__ __forceinline__ void rotate_angles(T sp, T cp, T sh, T ch, T &cpm, T &spm, T &cp1,
                                              T &sp1) {
  const T nsh = neg_(sh);
  cpm = fma_(sp, nsh, mul_(cp, ch));
  spm = fma_(cp, sh, mul_(sp, ch));
  cp1 = fma_(spm, nsh, mul_(cpm, ch));
  sp1 = fma_(cpm, sh, mul_(spm, ch));
}

// ------------------------------------------------------------------- p2z
// Propagate to the plane z = zt.  The mask is false where the track is
// parallel to the plane (|cos(theta)| <= 1e-4): out and J are then scratch.
template <class T>
__device__ __forceinline__ mask_t<T> propagate_to_z(const T (&in)[6], T qf, T bz, T zt,
                                                    T (&out)[6], T (&J)[36]) {
  using K = K_<T>;
  const T x = in[0], y = in[1], z = in[2], k = in[3], phi = in[4], th = in[5];
  T sp, cp, st, ct;
  sincos_(phi, &sp, &cp);
  sincos_(th, &st, &ct);
  const mask_t<T> ok = gt_(abs_(ct), cst<T>(1e-4));
  const T ict = rcp_(ct);
  const T tanth = mul_(st, ict);
  const T dz = sub_(zt, z);
  const T s = mul_(dz, tanth);                         // transverse path to the plane
  const T dwdk = mul_(mul_(qf, cst<T>(-K::alpha)), bz);  // d omega / d k
  const T omega = mul_(dwdk, k);
  const T h = mul_(mul_(cst<T>(0.5), omega), s);        // half turning angle
  T sh, ch;
  sincos_(h, &sh, &ch);
  const T S = sinc_from(h, sh);
  const T dS = dsinc_from(h, ch, S);
  const T L = mul_(s, S);  // chord length
  T cpm, spm, cp1, sp1;
  rotate_angles(sp, cp, sh, ch, cpm, spm, cp1, sp1);
  const T nspm = neg_(spm);

  out[0] = fma_(L, cpm, x);
  out[1] = fma_(L, spm, y);
  out[2] = zt;
  out[3] = k;
  out[4] = add_(phi, add_(h, h));  // wrapped once, after the update
  out[5] = th;

  // Partials at fixed s, then the path-length terms ds/dz = -tan(theta),
  // ds/dtheta = (zt - z) / cos^2(theta) along dp'/ds = (cos, sin, ., 0, omega, 0).
  const T hs2 = mul_(mul_(mul_(cst<T>(0.5), s), s), dwdk);
  const T Xk = mul_(hs2, fma_(dS, cpm, mul_(S, nspm)));
  const T Yk = mul_(hs2, fma_(dS, spm, mul_(S, cpm)));
  const T dsz = neg_(tanth);
  const T dsth = mul_(mul_(dz, ict), ict);
#pragma unroll
  for (int e = 0; e < 36; ++e) J[e] = cst<T>(0.0);
  J[0 * 6 + 2] = mul_(cp1, dsz);
  J[0 * 6 + 3] = Xk;
  J[0 * 6 + 4] = mul_(L, nspm);
  J[0 * 6 + 5] = mul_(cp1, dsth);
  J[1 * 6 + 2] = mul_(sp1, dsz);
  J[1 * 6 + 3] = Yk;
  J[1 * 6 + 4] = mul_(L, cpm);
  J[1 * 6 + 5] = mul_(sp1, dsth);
  J[4 * 6 + 2] = mul_(omega, dsz);
  J[4 * 6 + 3] = mul_(s, dwdk);
  J[4 * 6 + 5] = mul_(omega, dsth);
  return ok;
}

// ------------------------------------------------------------------- p2r
// Propagate to the first outward crossing of the cylinder r = R.  The mask
// is false where the track starts on/outside the cylinder or never reaches
// it (out, J and rcos are then scratch).  rcos receives R times the cosine
// between the track direction and the surface normal at the crossing (the
// incidence test needs no division).
//
// With A = P0.t0, B = P0.n0 (t0 = (cos phi, sin phi), n0 = (-sin, cos)),
// d = R^2 - |P0|^2 and t = tan(h), the crossing condition becomes
//   (1 + omega B - d omega^2/4) tau^2 + 2 A tau - d = 0,  tau = 2 t / omega,
// whose first-crossing root is tau = d / (A + sqrt(A^2 + a2 d)).  Then
//   (cos h, sin h) = (2 (A + sqrt(.)), omega d) / norm,  chord = 2 d / norm.
template <class T>
__device__ __forceinline__ mask_t<T> propagate_to_r(const T (&in)[6], T qf, T bz, T R,
                                                    T (&out)[6], T (&J)[36], T &rcos) {
  using K = K_<T>;
  const T x = in[0], y = in[1], z = in[2], k = in[3], phi = in[4], th = in[5];
  const T r0sq = fma_(x, x, mul_(y, y));
  const T d = fma_(R, R, neg_(r0sq));
  T sp, cp, st, ct;
  sincos_(phi, &sp, &cp);
  sincos_(th, &st, &ct);
  const T dwdk = mul_(mul_(qf, cst<T>(-K::alpha)), bz);
  const T omega = mul_(dwdk, k);
  const T A = fma_(x, cp, mul_(y, sp));
  const T B = fma_(y, cp, mul_(neg_(x), sp));
  const T a2 = fma_(omega, B, fma_(mul_(mul_(cst<T>(-0.25), d), omega), omega, cst<T>(1.0)));
  const T D = fma_(A, A, mul_(a2, d));
  // reached: starts strictly inside and the crossing is real
  const mask_t<T> ok = and_(gt_(d, cst<T>(0.0)), ge_(D, cst<T>(0.0)));
  const T den = add_(A, sqrt_(D));
  const T yv = mul_(omega, d);
  const T xv = add_(den, den);
  const T inv = rsqrt_(fma_(xv, xv, mul_(yv, yv)));
  const T ch = mul_(xv, inv);                 // cos(h)
  const T sh = mul_(yv, inv);                 // sin(h)
  const T h = atan2_(yv, xv);                 // half turning angle
  const T L = mul_(add_(d, d), inv);          // chord
  const T s = choose<T>(gt_(abs_(omega), cst<T>(1e-12)),
                        [&] { return div_(add_(h, h), omega); }, [&] { return div_(d, den); });
  const T ist = rcp_(st);
  const T cot = mul_(ct, ist);
  const T S = sinc_from(h, sh);
  const T dS = dsinc_from(h, ch, S);
  T cpm, spm, cp1, sp1;
  rotate_angles(sp, cp, sh, ch, cpm, spm, cp1, sp1);
  const T nspm = neg_(spm);

  const T x1 = fma_(L, cpm, x);
  const T y1 = fma_(L, spm, y);
  out[0] = x1;
  out[1] = y1;
  out[2] = fma_(s, cot, z);
  out[3] = k;
  out[4] = add_(phi, add_(h, h));  // wrapped once, after the update
  out[5] = th;

  // Fixed-s partials.
  const T hs2 = mul_(mul_(mul_(cst<T>(0.5), s), s), dwdk);
  const T Xk = mul_(hs2, fma_(dS, cpm, mul_(S, nspm)));
  const T Yk = mul_(hs2, fma_(dS, spm, mul_(S, cpm)));
  const T Xphi = mul_(L, nspm);
  const T Yphi = mul_(L, cpm);
  // s(p) from g = x'^2 + y'^2 - R^2 = 0: ds/dp = -(x' dx'/dp + y' dy'/dp) / (x' cos + y' sin).
  const T gs = fma_(x1, cp1, mul_(y1, sp1));
  rcos = gs;
  const T ig = neg_(rcp_(gs));
  const T dsx = mul_(ig, x1);
  const T dsy = mul_(ig, y1);
  const T dsk = mul_(ig, fma_(x1, Xk, mul_(y1, Yk)));
  const T dsphi = mul_(ig, fma_(x1, Xphi, mul_(y1, Yphi)));
  const T one = cst<T>(1.0);
#pragma unroll
  for (int e = 0; e < 36; ++e) J[e] = cst<T>(0.0);
  J[0 * 6 + 0] = fma_(cp1, dsx, one);
  J[0 * 6 + 1] = mul_(cp1, dsy);
  J[0 * 6 + 3] = fma_(cp1, dsk, Xk);
  J[0 * 6 + 4] = fma_(cp1, dsphi, Xphi);
  J[1 * 6 + 0] = mul_(sp1, dsx);
  J[1 * 6 + 1] = fma_(sp1, dsy, one);
  J[1 * 6 + 3] = fma_(sp1, dsk, Yk);
  J[1 * 6 + 4] = fma_(sp1, dsphi, Yphi);
  J[2 * 6 + 0] = mul_(cot, dsx);
  J[2 * 6 + 1] = mul_(cot, dsy);
  J[2 * 6 + 3] = mul_(cot, dsk);
  J[2 * 6 + 4] = mul_(cot, dsphi);
  J[2 * 6 + 5] = mul_(mul_(neg_(s), ist), ist);
  J[4 * 6 + 0] = mul_(omega, dsx);
  J[4 * 6 + 1] = mul_(omega, dsy);
  J[4 * 6 + 3] = fma_(omega, dsk, mul_(s, dwdk));
  J[4 * 6 + 4] = fma_(omega, dsphi, one);
  return ok;
}

// ---------------------------------------------------------------- update
// Update forms below the variants: the standard form in T, the standard form
// with S^-1, K and C'' in double (from float inputs), the Joseph form, the
// standard form with S^-1, K and C'' in double-float (from float inputs).
enum UpdateForm : int { kStandard = 0, kStandardF64 = 1, kJosephForm = 2, kStandardDF = 3 };

// Two-row Kalman update in a frame where the measurement is
//   row 0: h0 * (component 0),   row 1: component M1,
// and component SKIP has a structurally zero row and column in C' (the
// surface normal: z for p2z, the radial coordinate for p2r in the surface
// frame), so its gain row is skipped and stays zero.  U = C' H^T (columns
// U0, U1), S = H U + V, r the residual.  UNIT0: h0 is 1 (p2z), so nothing is
// divided by it.  Returns the mask of tracks whose S
// is not positive definite; those keep p and C untouched.
//
// Except under the Joseph form, every element with a measured column uses
// C' - K U^T = C' H^T S^-1 V H^-T (because I - S^-1 (S - V) = S^-1 V): a
// precise hit shrinks the measured variances by orders of magnitude, and in
// the subtracted form those digits would cancel away.
template <class T, int FORM, int SKIP, int M1, bool UNIT0>
__device__ __forceinline__ void kalman_update_body(T (&p)[6], T (&C)[21], const T (&U0)[6],
                                                   const T (&U1)[6], T S00, T S01, T S11, T h0,
                                                   T V00, T V01, T V11, T r0, T r1) {
  auto put = [&](T &dst, T v) { dst = v; };
  const T nS01 = neg_(S01);
  const T det = fma_(S00, S11, mul_(nS01, S01));
  const T inv = rcp_(det);
  const T Si00 = mul_(S11, inv), Si01 = mul_(nS01, inv), Si11 = mul_(S00, inv);
  T K0[6], K1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (i == SKIP) {
      K0[i] = K1[i] = cst<T>(0.0);
      continue;
    }
    K0[i] = fma_(U0[i], Si00, mul_(U1[i], Si01));
    K1[i] = fma_(U0[i], Si01, mul_(U1[i], Si11));
    put(p[i], fma_(K0[i], r0, fma_(K1[i], r1, p[i])));
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
        B[i][j] = sub_(C[tri(i, j)], fma_(K0[i], U0[j], mul_(K1[i], U1[j])));
    const T nh0 = neg_(h0);
    T nb0[6], nb1[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      nb0[i] = mul_(nh0, B[i][0]);
      nb1[i] = neg_(B[i][M1]);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i == SKIP) continue;
      const T kv0 = fma_(K0[i], V00, mul_(K1[i], V01));
      const T kv1 = fma_(K0[i], V01, mul_(K1[i], V11));
#pragma unroll
      for (int m = 0; m <= i; ++m) {
        if (m == SKIP) continue;
        T c = B[i][m];
        c = fma_(nb0[i], K0[m], c);
        c = fma_(nb1[i], K1[m], c);
        c = fma_(kv0, K0[m], c);
        c = fma_(kv1, K1[m], c);
        put(C[tri(i, m)], c);
      }
    }
  } else {
    const T G00 = fma_(Si00, V00, mul_(Si01, V01)), G01 = fma_(Si00, V01, mul_(Si01, V11));
    const T G10 = fma_(Si01, V00, mul_(Si11, V01)), G11 = fma_(Si01, V01, mul_(Si11, V11));
    const T ih0 = UNIT0 ? cst<T>(1.0) : rcp_(h0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i == SKIP) continue;
#pragma unroll
      for (int m = 0; m <= i; ++m) {
        if (m == SKIP) continue;
        const bool im = (i == 0 || i == M1), mm = (m == 0 || m == M1);
        if (mm || im) {
          const int r = mm ? i : m, c = mm ? m : i;  // row r, measured column c
          const T g0 = fma_(U0[r], G00, mul_(U1[r], G10));
          put(C[tri(i, m)], (c == 0) ? (UNIT0 ? g0 : mul_(g0, ih0))
                                     : fma_(U0[r], G01, mul_(U1[r], G11)));
        } else {  // C' - K0 U0^T - K1 U1^T, two fused steps
          put(C[tri(i, m)], fma_(neg_(K0[i]), U0[m], fma_(neg_(K1[i]), U1[m], C[tri(i, m)])));
        }
      }
    }
  }
}

// The standard form with S^-1, K and C'' in double from float inputs (the
// kFP64Update variant).
template <int SKIP, int M1, bool UNIT0>
__device__ __forceinline__ bool kalman_update_f64(float (&p)[6], float (&C)[21],
                                                  const float (&U0)[6], const float (&U1)[6],
                                                  float S00, float S01, float S11, float h0,
                                                  float V00, float V01, float V11, float r0,
                                                  float r1) {
  const double dS00 = S00, dS01 = S01, dS11 = S11;
  const double det = __fma_rn(dS00, dS11, __dmul_rn(-dS01, dS01));
  if (!(dS00 > 0.0) || !(det > 0.0)) return true;
  const double inv = __ddiv_rn(1.0, det);
  const double Si00 = __dmul_rn(dS11, inv), Si01 = __dmul_rn(-dS01, inv),
               Si11 = __dmul_rn(dS00, inv);
  double K0[6], K1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (i == SKIP) continue;
    K0[i] = __fma_rn((double)U0[i], Si00, __dmul_rn((double)U1[i], Si01));
    K1[i] = __fma_rn((double)U0[i], Si01, __dmul_rn((double)U1[i], Si11));
    p[i] = (float)__fma_rn(K0[i], (double)r0, __fma_rn(K1[i], (double)r1, (double)p[i]));
  }
  const double G00 = __fma_rn(Si00, V00, __dmul_rn(Si01, V01));
  const double G01 = __fma_rn(Si00, V01, __dmul_rn(Si01, V11));
  const double G10 = __fma_rn(Si01, V00, __dmul_rn(Si11, V01));
  const double G11 = __fma_rn(Si01, V01, __dmul_rn(Si11, V11));
  const double ih0 = UNIT0 ? 1.0 : __ddiv_rn(1.0, (double)h0);
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
        const double g0 = __fma_rn((double)U0[r], G00, __dmul_rn((double)U1[r], G10));
        v = (c == 0) ? (UNIT0 ? g0 : __dmul_rn(g0, ih0))
                     : __fma_rn((double)U0[r], G01, __dmul_rn((double)U1[r], G11));
      } else {  // C' - K0 U0^T - K1 U1^T, two fused steps
        v = __fma_rn(-K0[i], (double)U0[m], __fma_rn(-K1[i], (double)U1[m], (double)C[tri(i, m)]));
      }
      C[tri(i, m)] = (float)v;
    }
  }
  return false;
}

// The standard form with S^-1, K and C'' in double-float (kDFUpdate): the
// same algebra as kalman_update_f64, every quantity carried as an
// unevaluated pair of floats (kf_num.cuh) and rounded to float once at the
// end.  The float inputs enter exactly: S's determinant starts from exact
// two-float products, and each two-term sum of products (the gain, G, the
// posterior elements) is a compensated dot product of the double-word
// factors and the float inputs (dot2_df).
template <int SKIP, int M1, bool UNIT0>
__device__ __forceinline__ bool kalman_update_df(float (&p)[6], float (&C)[21],
                                                 const float (&U0)[6], const float (&U1)[6],
                                                 float S00, float S01, float S11, float h0,
                                                 float V00, float V01, float V11, float r0,
                                                 float r1) {
  const dfl det = add_dd(two_prod(S00, S11), neg_d(two_prod(S01, S01)));
  if (!(S00 > 0.0f) || !(det.hi > 0.0f)) return true;
  const dfl inv = rcp_d(det);
  const dfl Si00 = mul_df(inv, S11), Si01 = mul_df(inv, -S01), Si11 = mul_df(inv, S00);
  dfl K0[6], K1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (i == SKIP) continue;
    K0[i] = dot2_df(Si00, U0[i], Si01, U1[i]);
    K1[i] = dot2_df(Si01, U0[i], Si11, U1[i]);
    p[i] = to_float(add_df(dot2_df(K0[i], r0, K1[i], r1), p[i]));
  }
  const dfl G00 = dot2_df(Si00, V00, Si01, V01);
  const dfl G01 = dot2_df(Si00, V01, Si01, V11);
  const dfl G10 = dot2_df(Si01, V00, Si11, V01);
  const dfl G11 = dot2_df(Si01, V01, Si11, V11);
  const dfl ih0 = UNIT0 ? dfl{1.0f, 0.0f} : rcp_d(dfl{h0, 0.0f});
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (i == SKIP) continue;
#pragma unroll
    for (int m = 0; m <= i; ++m) {
      if (m == SKIP) continue;
      const bool im = (i == 0 || i == M1), mm = (m == 0 || m == M1);
      dfl v;
      if (mm || im) {
        const int r = mm ? i : m, c = mm ? m : i;  // row r, measured column c
        if (c == 0) {
          const dfl g0 = dot2_df(G00, U0[r], G10, U1[r]);
          v = UNIT0 ? g0 : mul_dd(g0, ih0);
        } else {
          v = dot2_df(G01, U0[r], G11, U1[r]);
        }
      } else {
        v = sub_dot2_df(C[tri(i, m)], K0[i], U0[m], K1[i], U1[m]);
      }
      C[tri(i, m)] = to_float(v);
    }
  }
  return false;
}

template <class T, int FORM, int SKIP, int M1, bool UNIT0>
__device__ __forceinline__ mask_t<T> kalman_update(T (&p)[6], T (&C)[21], const T (&U0)[6],
                                                   const T (&U1)[6], T S00, T S01, T S11, T h0,
                                                   T V00, T V01, T V11, T r0, T r1) {
  if constexpr (FORM == kStandardF64) {
    return kalman_update_f64<SKIP, M1, UNIT0>(p, C, U0, U1, S00, S01, S11, h0, V00, V01, V11, r0,
                                              r1);
  } else if constexpr (FORM == kStandardDF) {
    return kalman_update_df<SKIP, M1, UNIT0>(p, C, U0, U1, S00, S01, S11, h0, V00, V01, V11, r0,
                                             r1);
  } else {
    const T nS01 = neg_(S01);
    const T det = fma_(S00, S11, mul_(nS01, S01));
    const mask_t<T> bad = or_(not_(gt_(S00, cst<T>(0.0))), not_(gt_(det, cst<T>(0.0))));
    if (any_(bad)) return bad;
    kalman_update_body<T, FORM, SKIP, M1, UNIT0>(p, C, U0, U1, S00, S01, S11, h0, V00, V01, V11,
                                                 r0, r1);
    return bad;
  }
}

template <class T, int N>
__device__ __forceinline__ void copy_to(T (&dst)[N], const T (&src)[N]) {
#pragma unroll
  for (int e = 0; e < N; ++e) dst[e] = src[e];
}

// Status of a reached track after its update: kSNotPD where S was not
// positive definite, plus kBadK where the updated 1/pT is not positive.
template <class T>
__device__ __forceinline__ stat_t<T> step_status(mask_t<T> bad, T k) {
  return stat_if<T>(bad, kSNotPD) | stat_if<T>(not_(gt_(k, cst<T>(0.0))), kBadK);
}

// ------------------------------------------------------------ full steps
// One p2z step in number type T.  p/C hold the input and receive the result
// (untouched when the plane is not reached); shrink is set where the hit
// shrank a measured variance by more than kRedoShrink.
template <class T, int FORM>
__device__ __forceinline__ stat_t<T> p2z_step_t(T (&p)[6], T (&C)[21], T qf, T bz, T zt, T hx,
                                                T hy, T vxx, T vxy, T vyy, mask_t<T> &shrink) {
  T pp[6], J[36], Cp[21];
  shrink = mask_t<T>(false);
  if (!all_(propagate_to_z(p, qf, bz, zt, pp, J))) return kNoIntersect;
  transport<T, kP2zNZ, kP2zOne>(J, C, Cp);
  // H = [e_x; e_y]: U = columns x and y of C' (its z row and column are zero).
  T U0[6], U1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    U0[i] = Cp[tri(i, 0)];
    U1[i] = Cp[tri(i, 1)];
  }
  const T S00 = add_(U0[0], vxx), S01 = add_(U0[1], vxy), S11 = add_(U1[1], vyy);
  // ill-conditioned when the hit shrinks a measured variance by > kRedoShrink
  shrink = or_(gt_(S00, mul_(cst<T>(kRedoShrink), vxx)), gt_(S11, mul_(cst<T>(kRedoShrink), vyy)));
  const mask_t<T> bad = kalman_update<T, FORM, 2, 1, true>(pp, Cp, U0, U1, S00, S01, S11,
                                                     cst<T>(1.0), vxx, vxy, vyy,
                                                     sub_(hx, pp[0]), sub_(hy, pp[1]));
  pp[4] = wrap_phi(pp[4]);
  copy_to(p, pp);
  copy_to(C, Cp);
  return step_status<T>(bad, p[3]);
}

// One p2r step in number type T.  hc = packed 3x3 hit covariance.
//
// The covariance is transported and updated in the surface frame at the
// crossing point P' = R (cos a, sin a): position coordinates t (along
// (-sin a, cos a)) and r (along (cos a, sin a)).  The radial row of the
// Jacobian is identically zero, so C' has an exactly zero radial row and
// column there; rotating the updated covariance back gives
// C_xx = sin^2 a C_tt, C_xy = -sin a cos a C_tt, ..., which keeps full
// relative precision even where an axis is nearly radial.
template <class T, int FORM>
__device__ __forceinline__ stat_t<T> p2r_step_t(T (&p)[6], T (&C)[21], T qf, T bz, T R, T hx,
                                                T hy, T hz, const T (&hc)[6],
                                                mask_t<T> &shrink, T &rcos) {
  T pp[6], J[36], Cp[21];
  shrink = mask_t<T>(false);
  if (!all_(propagate_to_r(p, qf, bz, R, pp, J, rcos))) {
    rcos = R;
    return kNoIntersect;
  }
  const T ip = rsqrt_(fma_(pp[0], pp[0], mul_(pp[1], pp[1])));
  const T ca = mul_(pp[0], ip), sa = mul_(pp[1], ip);  // direction of P'
  const T nsa = neg_(sa);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    if (((kP2rFrameNZ >> j) & 1ull) == 0) continue;  // structurally zero in the t row
    J[0 * 6 + j] = fma_(nsa, J[0 * 6 + j], mul_(ca, J[1 * 6 + j]));  // t row
  }
  transport<T, kP2rFrameNZ, kP2rFrameOne>(J, C, Cp);
  // Measurement direction at the hit, u = (-sin phi_h, cos phi_h), and z.
  // In the frame u acts on t with weight u.t = cos(phi_h - a) (the radial
  // column of C' is zero).
  const T ir = rsqrt_(fma_(hx, hx, mul_(hy, hy)));
  const T ux = mul_(neg_(hy), ir), uy = mul_(hx, ir);
  const T ut = fma_(nsa, ux, mul_(ca, uy));
  T U0[6], U1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    U0[i] = mul_(ut, Cp[tri(i, 0)]);
    U1[i] = Cp[tri(i, 2)];
  }
  // V = P V_hit P^T with P = [[ux, uy, 0], [0, 0, 1]].
  const T V00 = fma_(mul_(ux, ux), hc[0],
                     fma_(mul_(mul_(cst<T>(2.0), ux), uy), hc[1], mul_(mul_(uy, uy), hc[2])));
  const T V01 = fma_(ux, hc[3], mul_(uy, hc[4]));
  const T V11 = hc[5];
  const T S00 = fma_(ut, U0[0], V00);
  const T S01 = add_(U0[2], V01);
  const T S11 = add_(U1[2], V11);
  shrink = or_(gt_(S00, mul_(cst<T>(kRedoShrink), V00)), gt_(S11, mul_(cst<T>(kRedoShrink), V11)));
  const T r0 = fma_(ux, sub_(hx, pp[0]), mul_(uy, sub_(hy, pp[1])));
  const T r1 = sub_(hz, pp[2]);
  // frame state: the position offsets (t, r) start at 0 on P'
  T pf[6] = {cst<T>(0.0), cst<T>(0.0), pp[2], pp[3], pp[4], pp[5]};
  const mask_t<T> bad = kalman_update<T, FORM, 1, 2, false>(pf, Cp, U0, U1, S00, S01, S11, ut,
                                                            V00, V01, V11, r0, r1);
  T pn[6], Cn[21];
  pn[0] = fma_(nsa, pf[0], pp[0]);
  pn[1] = fma_(ca, pf[0], pp[1]);
#pragma unroll
  for (int i = 2; i < 6; ++i) pn[i] = pf[i];
  // back to (x, y): only the t row/column carries position variance
  const T ctt = Cp[tri(0, 0)];
  Cn[tri(0, 0)] = mul_(mul_(sa, sa), ctt);
  Cn[tri(1, 0)] = mul_(mul_(nsa, ca), ctt);
  Cn[tri(1, 1)] = mul_(mul_(ca, ca), ctt);
#pragma unroll
  for (int j = 2; j < 6; ++j) {
    const T ctj = Cp[tri(j, 0)];
    Cn[tri(j, 0)] = mul_(nsa, ctj);
    Cn[tri(j, 1)] = mul_(ca, ctj);
#pragma unroll
    for (int m = 2; m <= j; ++m) Cn[tri(j, m)] = Cp[tri(j, m)];
  }
  pn[4] = wrap_phi(pn[4]);
  copy_to(p, pn);
  copy_to(C, Cn);
  return step_status<T>(bad, p[3]);
}

// Run a T = double step on float registers (convert in and out).  Kept out
// of line so that the float path's register allocation does not carry it.
template <int KIND>
__device__ __noinline__ unsigned step_in_double(float (&p)[6], float (&C)[21], float qf, float bz,
                                                float surf, float hx, float hy, float hz,
                                                const float (&hc)[6]) {
  double dp[6], dC[21], dhc[6], cinc;
  bool shrink;
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
// / kDFUpdate run in float (with their update form); kFP64 runs every
// operation in double.  kAdaptive runs in float and, when the step is ill-conditioned (the
// hit shrinks a measured variance by more than kRedoShrink, a cylinder is
// crossed at an incidence cosine below kRedoGrazing, or the updated 1/pT is
// not positive), sets kRedo: the caller
// then reloads the track's inputs and calls step_in_double -- FP64 where the
// conditioning demands it, FP32 for everything else, and no register copies
// of the inputs on the common path.
template <int KIND, int VARIANT, class T>
__device__ __forceinline__ stat_t<T> step_variant(T (&p)[6], T (&C)[21], T qf, T bz, T surf,
                                                  T hx, T hy, T hz, const T (&hc)[6]) {
  if constexpr (VARIANT == kFP64) {
    return step_in_double<KIND>(p, C, qf, bz, surf, hx, hy, hz, hc);
  } else {
    constexpr int FORM = VARIANT == kJoseph       ? kJosephForm
                         : VARIANT == kFP64Update ? kStandardF64
                         : VARIANT == kDFUpdate   ? kStandardDF
                                                  : kStandard;
    mask_t<T> ill;
    T rcos = surf;
    stat_t<T> st;
    if (KIND == kP2z)
      st = p2z_step_t<T, FORM>(p, C, qf, bz, surf, hx, hy, hc[0], hc[1], hc[2], ill);
    else
      st = p2r_step_t<T, FORM>(p, C, qf, bz, surf, hx, hy, hz, hc, ill, rcos);
    if constexpr (VARIANT == kAdaptive) {
      // reached, and ill-conditioned, crossed at grazing incidence or left
      // with 1/pT <= 0
      const mask_t<T> reached = not_(has_bit_(st, kNoIntersect));
      const mask_t<T> grazing =
          not_(ge_(abs_(rcos), mul_(cst<T>(kRedoGrazing), surf)));
      const mask_t<T> bad_k = has_bit_(st, kBadK);
      st = st | stat_if<T>(and_(reached, or_(or_(ill, grazing), bad_k)), kRedo);
    }
    return st;
  }
}

// Convenience entry points used by the kernels (one track per thread).
// Under kAdaptive the returned status may carry kRedo (see step_variant).
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
template <class T>
__device__ __forceinline__ stat_t<T> finite_status(const T (&p)[6], const T (&C)[21]) {
  T acc = cst<T>(0.0);
#pragma unroll
  for (int i = 0; i < 6; ++i) acc = add_(acc, p[i]);
#pragma unroll
  for (int e = 0; e < 21; ++e) acc = add_(acc, C[e]);
  return stat_if<T>(not_(finite_(acc)), kNonFinite);
}

}  // namespace kf
