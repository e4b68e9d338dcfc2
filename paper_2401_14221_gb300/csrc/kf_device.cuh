// kf_device.cuh -- per-track device arithmetic of the Kalman step (sm_103a).
//
// Paper section 2: each track is propagated to a surface at fixed z
// (propagateToZ) or fixed r (propagateToR) and then Kalman-updated
// (KalmanUpdate).  The paper gives no formulas; this file implements the
// exact helix in a uniform field bz, its transport Jacobian and the linear
// Kalman update, in FP32 registers, one track per thread.
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
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kf {

constexpr float kAlpha = 0.299792458e-2f;  // GeV / (cm T), unit charge
constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPiHi = 6.28318548202514648f;     // float(2 pi)
constexpr float kTwoPiLo = -1.7484555314695172e-7f;  // 2 pi - float(2 pi)
constexpr float kInvTwoPi = 0.15915494309189535f;

constexpr unsigned kNoIntersect = 1u;
constexpr unsigned kSNotPD = 2u;
constexpr unsigned kBadK = 4u;
constexpr unsigned kNonFinite = 8u;

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
// p2r: the path length depends on x, y, k, phi through the cylinder
// constraint, so x', y', phi' are dense in those; z' also in z and theta.
constexpr uint64_t kP2rNZ =
    bit(0, 0) | bit(0, 1) | bit(0, 3) | bit(0, 4) |
    bit(1, 0) | bit(1, 1) | bit(1, 3) | bit(1, 4) |
    bit(2, 0) | bit(2, 1) | bit(2, 2) | bit(2, 3) | bit(2, 4) | bit(2, 5) |
    bit(3, 3) |
    bit(4, 0) | bit(4, 1) | bit(4, 3) | bit(4, 4) |
    bit(5, 5);
constexpr uint64_t kP2rOne = bit(2, 2) | bit(3, 3) | bit(5, 5);
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
// parts (float(2 pi) and its remainder), so the wrap adds < 1e-13 error.
__device__ __forceinline__ float wrap_phi(float a) {
  const float n = rintf(a * kInvTwoPi);
  float w = fmaf(-n, kTwoPiHi, a);
  w = fmaf(-n, kTwoPiLo, w);
  if (w <= -kPi) w += kTwoPiHi;
  return w;
}

// S(h) = sin(h)/h given sin(h); S(0) = 1.
__device__ __forceinline__ float sinc_from(float h, float sh) {
  return fabsf(h) < 1e-4f ? fmaf(-h * h, 1.0f / 6.0f, 1.0f) : sh / h;
}

// dS/dh = (cos(h) - S(h)) / h; the difference cancels for small |h|, where
// the Taylor series -h/3 + h^3/30 - h^5/840 + h^7/45360 is used instead.
__device__ __forceinline__ float dsinc_from(float h, float ch, float S) {
  if (fabsf(h) < 0.25f) {
    const float h2 = h * h;
    return h * fmaf(h2, fmaf(h2, fmaf(h2, 1.0f / 45360.0f, -1.0f / 840.0f), 1.0f / 30.0f),
                    -1.0f / 3.0f);
  }
  return (ch - S) / h;
}

// C' = J C J^T for packed symmetric C, with J's structure fixed by NZ/ONE.
// Loops unroll completely, so every mask test folds at compile time and
// only the structurally non-zero multiply-adds remain.
template <uint64_t NZ, uint64_t ONE>
__device__ __forceinline__ void transport(const float (&J)[36], const float (&C)[21],
                                          float (&Co)[21]) {
  float T[6][6];  // T = J C
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float acc = 0.0f;
      bool first = true;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if ((NZ >> (i * 6 + l)) & 1ull) {
          const float c = C[tri(l, j)];
          if ((ONE >> (i * 6 + l)) & 1ull)
            acc = first ? c : acc + c;
          else
            acc = first ? J[i * 6 + l] * c : fmaf(J[i * 6 + l], c, acc);
          first = false;
        }
      }
      T[i][j] = acc;
    }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int m = 0; m <= i; ++m) {
      if (((NZ >> (i * 6)) & 0x3Full) == 0 || ((NZ >> (m * 6)) & 0x3Full) == 0) {
        Co[tri(i, m)] = 0.0f;  // a zero row of J gives a zero row of C'
        continue;
      }
      float acc = 0.0f;
      bool first = true;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if ((NZ >> (m * 6 + l)) & 1ull) {
          if ((ONE >> (m * 6 + l)) & 1ull)
            acc = first ? T[i][l] : acc + T[i][l];
          else
            acc = first ? T[i][l] * J[m * 6 + l] : fmaf(T[i][l], J[m * 6 + l], acc);
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
__device__ __forceinline__ bool propagate_to_z(const float (&in)[6], float qf, float bz,
                                               float zt, float (&out)[6], float (&J)[36]) {
  const float x = in[0], y = in[1], z = in[2], k = in[3], phi = in[4], th = in[5];
  float sp, cp, st, ct;
  sincosf(phi, &sp, &cp);
  sincosf(th, &st, &ct);
  if (!(fabsf(ct) > 1e-4f)) return false;
  const float tanth = st / ct;
  const float cot = ct / st;
  const float dz = zt - z;
  const float s = dz * tanth;                 // transverse path to the plane
  const float dwdk = -qf * kAlpha * bz;       // d omega / d k
  const float omega = dwdk * k;
  const float h = 0.5f * omega * s;           // half turning angle
  float sh, ch;
  sincosf(h, &sh, &ch);
  const float S = sinc_from(h, sh);
  const float dS = dsinc_from(h, ch, S);
  const float L = s * S;                      // chord length
  const float cpm = cp * ch - sp * sh;        // cos(phi + h)
  const float spm = sp * ch + cp * sh;        // sin(phi + h)
  const float cp1 = cpm * ch - spm * sh;      // cos(phi + 2h)
  const float sp1 = spm * ch + cpm * sh;      // sin(phi + 2h)

  out[0] = fmaf(L, cpm, x);
  out[1] = fmaf(L, spm, y);
  out[2] = zt;
  out[3] = k;
  out[4] = wrap_phi(phi + 2.0f * h);
  out[5] = th;

  // Partials at fixed s, then the path-length terms ds/dz = -tan(theta),
  // ds/dtheta = (zt - z) / cos^2(theta) along dp'/ds = (cos, sin, ., 0, omega, 0).
  const float hs2 = 0.5f * s * s * dwdk;
  const float Xk = hs2 * (dS * cpm - S * spm);
  const float Yk = hs2 * (dS * spm + S * cpm);
  const float dsz = -tanth;
  const float dsth = dz / (ct * ct);
#pragma unroll
  for (int e = 0; e < 36; ++e) J[e] = 0.0f;
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
  (void)cot;
  return true;
}

// ------------------------------------------------------------------- p2r
// Propagate to the first outward crossing of the cylinder r = R.  Returns
// false when the track starts on/outside the cylinder or never reaches it.
//
// With A = P0.t0, B = P0.n0 (t0 = (cos phi, sin phi), n0 = (-sin, cos)),
// d = R^2 - |P0|^2 and t = tan(h), the crossing condition becomes
//   (1 + omega B - d omega^2/4) tau^2 + 2 A tau - d = 0,  tau = 2 t / omega,
// whose first-crossing root is tau = d / (A + sqrt(A^2 + a2 d)).  Then
//   (cos h, sin h) = (2 (A + sqrt(.)), omega d) / norm,  chord = 2 d / norm.
__device__ __forceinline__ bool propagate_to_r(const float (&in)[6], float qf, float bz,
                                               float R, float (&out)[6], float (&J)[36]) {
  const float x = in[0], y = in[1], z = in[2], k = in[3], phi = in[4], th = in[5];
  const float r0sq = fmaf(x, x, y * y);
  const float d = fmaf(R, R, -r0sq);
  if (!(d > 0.0f)) return false;
  float sp, cp, st, ct;
  sincosf(phi, &sp, &cp);
  sincosf(th, &st, &ct);
  const float dwdk = -qf * kAlpha * bz;
  const float omega = dwdk * k;
  const float A = fmaf(x, cp, y * sp);
  const float B = fmaf(y, cp, -x * sp);
  const float a2 = fmaf(omega, B, fmaf(-0.25f * d * omega, omega, 1.0f));
  const float D = fmaf(A, A, a2 * d);
  if (!(D >= 0.0f)) return false;
  const float den = A + sqrtf(D);
  const float yv = omega * d;
  const float xv = 2.0f * den;
  const float inv = rsqrtf(fmaf(xv, xv, yv * yv));
  const float ch = xv * inv;                  // cos(h)
  const float sh = yv * inv;                  // sin(h)
  const float h = atan2f(yv, xv);             // half turning angle
  const float L = 2.0f * d * inv;             // chord
  const float s = fabsf(omega) > 1e-12f ? 2.0f * h / omega : d / den;
  const float cot = ct / st;
  const float S = sinc_from(h, sh);
  const float dS = dsinc_from(h, ch, S);
  const float cpm = cp * ch - sp * sh;
  const float spm = sp * ch + cp * sh;
  const float cp1 = cpm * ch - spm * sh;
  const float sp1 = spm * ch + cpm * sh;

  const float x1 = fmaf(L, cpm, x);
  const float y1 = fmaf(L, spm, y);
  out[0] = x1;
  out[1] = y1;
  out[2] = fmaf(s, cot, z);
  out[3] = k;
  out[4] = wrap_phi(phi + 2.0f * h);
  out[5] = th;

  // Fixed-s partials.
  const float hs2 = 0.5f * s * s * dwdk;
  const float Xk = hs2 * (dS * cpm - S * spm);
  const float Yk = hs2 * (dS * spm + S * cpm);
  const float Xphi = -L * spm;
  const float Yphi = L * cpm;
  // s(p) from g = x'^2 + y'^2 - R^2 = 0: ds/dp = -(x' dx'/dp + y' dy'/dp) / (x' cos + y' sin).
  const float ig = -1.0f / fmaf(x1, cp1, y1 * sp1);
  const float dsx = ig * x1;
  const float dsy = ig * y1;
  const float dsk = ig * fmaf(x1, Xk, y1 * Yk);
  const float dsphi = ig * fmaf(x1, Xphi, y1 * Yphi);
#pragma unroll
  for (int e = 0; e < 36; ++e) J[e] = 0.0f;
  J[0 * 6 + 0] = fmaf(cp1, dsx, 1.0f);
  J[0 * 6 + 1] = cp1 * dsy;
  J[0 * 6 + 3] = fmaf(cp1, dsk, Xk);
  J[0 * 6 + 4] = fmaf(cp1, dsphi, Xphi);
  J[1 * 6 + 0] = sp1 * dsx;
  J[1 * 6 + 1] = fmaf(sp1, dsy, 1.0f);
  J[1 * 6 + 3] = fmaf(sp1, dsk, Yk);
  J[1 * 6 + 4] = fmaf(sp1, dsphi, Yphi);
  J[2 * 6 + 0] = cot * dsx;
  J[2 * 6 + 1] = cot * dsy;
  J[2 * 6 + 3] = cot * dsk;
  J[2 * 6 + 4] = cot * dsphi;
  J[2 * 6 + 5] = -s / (st * st);
  J[4 * 6 + 0] = omega * dsx;
  J[4 * 6 + 1] = omega * dsy;
  J[4 * 6 + 3] = fmaf(omega, dsk, s * dwdk);
  J[4 * 6 + 4] = fmaf(omega, dsphi, 1.0f);
  return true;
}

// ---------------------------------------------------------------- update
// Update variants.
enum Variant : int { kFP32 = 0, kFP64Update = 1, kJoseph = 2 };
// Step kinds.
enum Kind : int { kP2z = 0, kP2r = 1 };

// Two-row Kalman update in a frame where the measurement is
//   row 0: h0 * (component 0),   row 1: component M1,
// and component SKIP has a structurally zero row and column in C' (the
// surface normal: z for p2z, the radial coordinate for p2r in the surface
// frame), so its gain row is skipped and stays zero.  U = C' H^T (columns
// U0, U1), S = H U + V, r the residual.  Returns kSNotPD (state untouched)
// or 0.
template <int VARIANT, int SKIP, int M1>
__device__ __forceinline__ unsigned kalman_update(float (&p)[6], float (&C)[21],
                                                  const float (&U0)[6], const float (&U1)[6],
                                                  float S00, float S01, float S11, float h0,
                                                  float V00, float V01, float V11, float r0,
                                                  float r1) {
  if constexpr (VARIANT == kFP64Update) {
    // S^-1, K and C'' = C' - K U^T in double precision.
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
      p[i] = (float)((double)p[i] + K0[i] * (double)r0 + K1[i] * (double)r1);
    }
    // G = S^-1 V; columns of a measured component use the cancellation-free
    // form (see the FP32 branch below).
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
        C[tri(i, m)] = (float)v;
      }
    }
    return 0u;
  } else {
    const float det = fmaf(S00, S11, -S01 * S01);
    if (!(S00 > 0.0f) || !(det > 0.0f)) return kSNotPD;
    const float inv = 1.0f / det;
    const float Si00 = S11 * inv, Si01 = -S01 * inv, Si11 = S00 * inv;
    float K0[6], K1[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i == SKIP) {
        K0[i] = K1[i] = 0.0f;
        continue;
      }
      K0[i] = fmaf(U0[i], Si00, U1[i] * Si01);
      K1[i] = fmaf(U0[i], Si01, U1[i] * Si11);
      p[i] = fmaf(K0[i], r0, fmaf(K1[i], r1, p[i]));
    }
    if constexpr (VARIANT == kJoseph) {
      // Product (Joseph) form: B = (I - K H) C' = C' - K U^T, then
      // C'' = B (I - K H)^T + K V K^T = B - (B H0^T) K0^T - (B H1^T) K1^T + K V K^T,
      // a sum of positive semi-definite terms for any gain K.
      float B[6][6];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j)
          B[i][j] = C[tri(i, j)] - fmaf(K0[i], U0[j], K1[i] * U1[j]);
      float b0[6], b1[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        b0[i] = h0 * B[i][0];
        b1[i] = B[i][M1];
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i == SKIP) continue;
        const float kv0 = fmaf(K0[i], V00, K1[i] * V01);
        const float kv1 = fmaf(K0[i], V01, K1[i] * V11);
#pragma unroll
        for (int m = 0; m <= i; ++m) {
          if (m == SKIP) continue;
          float c = B[i][m];
          c = fmaf(-b0[i], K0[m], c);
          c = fmaf(-b1[i], K1[m], c);
          c = fmaf(kv0, K0[m], c);
          c = fmaf(kv1, K1[m], c);
          C[tri(i, m)] = c;
        }
      }
      return 0u;
    } else {
      // Standard form C'' = C' - K U^T, except where a measured component
      // (0 or M1) is involved: there C' - K U^T = C' H^T S^-1 V H^-T exactly
      // (because I - S^-1 (S - V) = S^-1 V), with no subtraction.  A precise
      // hit shrinks the measured variances by orders of magnitude; in the
      // subtracted form those digits would cancel away.
      const float G00 = fmaf(Si00, V00, Si01 * V01), G01 = fmaf(Si00, V01, Si01 * V11);
      const float G10 = fmaf(Si01, V00, Si11 * V01), G11 = fmaf(Si01, V01, Si11 * V11);
      const float ih0 = 1.0f / h0;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i == SKIP) continue;
#pragma unroll
        for (int m = 0; m <= i; ++m) {
          if (m == SKIP) continue;
          const bool im = (i == 0 || i == M1), mm = (m == 0 || m == M1);
          if (mm || im) {
            const int r = mm ? i : m, c = mm ? m : i;  // row r, measured column c
            C[tri(i, m)] = (c == 0) ? fmaf(U0[r], G00, U1[r] * G10) * ih0
                                    : fmaf(U0[r], G01, U1[r] * G11);
          } else {
            C[tri(i, m)] = C[tri(i, m)] - fmaf(K0[i], U0[m], K1[i] * U1[m]);
          }
        }
      }
      return 0u;
    }
  }
}

// ------------------------------------------------------------ full steps
// One p2z step on registers.  p/C hold the input and receive the result.
template <int VARIANT>
__device__ __forceinline__ unsigned p2z_step(float (&p)[6], float (&C)[21], float qf, float bz,
                                             float zt, float hx, float hy, float vxx, float vxy,
                                             float vyy) {
  float pp[6], J[36], Cp[21];
  if (!propagate_to_z(p, qf, bz, zt, pp, J)) return kNoIntersect;
  transport<kP2zNZ, kP2zOne>(J, C, Cp);
  // H = [e_x; e_y]: U = columns x and y of C' (its z row and column are zero).
  float U0[6], U1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    U0[i] = Cp[tri(i, 0)];
    U1[i] = Cp[tri(i, 1)];
  }
  const float S00 = U0[0] + vxx, S01 = U0[1] + vxy, S11 = U1[1] + vyy;
  const unsigned st = kalman_update<VARIANT, 2, 1>(pp, Cp, U0, U1, S00, S01, S11, 1.0f, vxx,
                                                   vxy, vyy, hx - pp[0], hy - pp[1]);
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = pp[i];
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = Cp[e];
  if (!st) p[4] = wrap_phi(p[4]);
  return st | (p[3] > 0.0f ? 0u : kBadK);
}

// One p2r step on registers.  hc = packed 3x3 hit covariance.
//
// The covariance is transported and updated in the surface frame at the
// crossing point P' = R (cos a, sin a): position coordinates t (along
// (-sin a, cos a)) and r (along (cos a, sin a)).  The radial row of the
// Jacobian is identically zero, so C' has an exactly zero radial row and
// column there; rotating the updated covariance back gives
// C_xx = sin^2 a C_tt, C_xy = -sin a cos a C_tt, ..., which keeps full
// relative precision even where an axis is nearly radial (in Cartesian FP32,
// C_xx would be a difference of much larger terms).
template <int VARIANT>
__device__ __forceinline__ unsigned p2r_step(float (&p)[6], float (&C)[21], float qf, float bz,
                                             float R, float hx, float hy, float hz,
                                             const float (&hc)[6]) {
  float pp[6], J[36], Cp[21];
  if (!propagate_to_r(p, qf, bz, R, pp, J)) return kNoIntersect;
  const float ip = rsqrtf(fmaf(pp[0], pp[0], pp[1] * pp[1]));
  const float ca = pp[0] * ip, sa = pp[1] * ip;  // direction of P'
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    J[0 * 6 + j] = fmaf(-sa, J[0 * 6 + j], ca * J[1 * 6 + j]);  // t row
    J[1 * 6 + j] = 0.0f;                                      // r row: zero
  }
  transport<kP2rFrameNZ, kP2rFrameOne>(J, C, Cp);
  // Measurement direction at the hit, u = (-sin phi_h, cos phi_h), and z.
  // In the frame u acts on t with weight u.t = cos(phi_h - a) (the radial
  // column of C' is zero).
  const float ir = rsqrtf(fmaf(hx, hx, hy * hy));
  const float ux = -hy * ir, uy = hx * ir;
  const float ut = fmaf(-sa, ux, ca * uy);
  float U0[6], U1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    U0[i] = ut * Cp[tri(i, 0)];
    U1[i] = Cp[tri(i, 2)];
  }
  // V = P V_hit P^T with P = [[ux, uy, 0], [0, 0, 1]].
  const float V00 = fmaf(ux * ux, hc[0], fmaf(2.0f * ux * uy, hc[1], uy * uy * hc[2]));
  const float V01 = fmaf(ux, hc[3], uy * hc[4]);
  const float V11 = hc[5];
  const float S00 = fmaf(ut, U0[0], V00);
  const float S01 = U0[2] + V01;
  const float S11 = U1[2] + V11;
  const float r0 = fmaf(ux, hx - pp[0], uy * (hy - pp[1]));
  const float r1 = hz - pp[2];
  // frame state: the position offsets (t, r) start at 0 on P'
  float pf[6] = {0.0f, 0.0f, pp[2], pp[3], pp[4], pp[5]};
  const unsigned st = kalman_update<VARIANT, 1, 2>(pf, Cp, U0, U1, S00, S01, S11, ut, V00,
                                                   V01, V11, r0, r1);
  p[0] = fmaf(-sa, pf[0], pp[0]);
  p[1] = fmaf(ca, pf[0], pp[1]);
#pragma unroll
  for (int i = 2; i < 6; ++i) p[i] = pf[i];
  // back to (x, y): only the t row/column carries position variance
  const float ctt = Cp[tri(0, 0)];
  C[tri(0, 0)] = sa * sa * ctt;
  C[tri(1, 0)] = -sa * ca * ctt;
  C[tri(1, 1)] = ca * ca * ctt;
#pragma unroll
  for (int j = 2; j < 6; ++j) {
    const float ctj = Cp[tri(j, 0)];
    C[tri(j, 0)] = -sa * ctj;
    C[tri(j, 1)] = ca * ctj;
#pragma unroll
    for (int m = 2; m <= j; ++m) C[tri(j, m)] = Cp[tri(j, m)];
  }
  if (!st) p[4] = wrap_phi(p[4]);
  return st | (p[3] > 0.0f ? 0u : kBadK);
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
