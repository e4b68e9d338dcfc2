// kf_num.cuh -- the number types of the per-track arithmetic, with every
// rounding written out.
//
// The step is written once (kf_device.cuh) for a number type T: float (the
// FP32 bulk path) or double (the FP64 variants and redo passes).  Every
// operation is an explicit, individually rounded IEEE operation: a product
// and a sum are fused only where the source says fma_, never by the
// compiler.  So every kernel that runs the same source on the same inputs
// rounds the same way, bit for bit, whatever the surrounding kernel's
// register allocation and instruction scheduling -- which the tests rely on
// (the staged and one-thread-per-track kernels, the chain of one layer and
// the single step, the fused chain and its per-layer launches).
//
// Comparisons give masks (bool); sel_ picks; all_/any_ reduce a mask.  The
// mask vocabulary lets the step code state per-track decisions once, in a
// form a wider number type could also take.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kf {
namespace num {

// ================================================================== float
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float neg_(float a) { return -a; }
__device__ __forceinline__ float abs_(float a) { return fabsf(a); }
__device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
__device__ __forceinline__ float rsqrt_(float a) { return rsqrtf(a); }
__device__ __forceinline__ float rint_(float a) { return rintf(a); }
// Quotients of well-scaled operands (|b| far below 2^126): the fast
// reciprocal-based division, within 2 ulp, instead of the IEEE sequence.
__device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float rcp_(float b) { return __fdividef(1.0f, b); }
__device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }

__device__ __forceinline__ bool lt_(float a, float b) { return a < b; }
__device__ __forceinline__ bool le_(float a, float b) { return a <= b; }
__device__ __forceinline__ bool gt_(float a, float b) { return a > b; }
__device__ __forceinline__ bool ge_(float a, float b) { return a >= b; }
__device__ __forceinline__ float sel_(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ bool finite_(float a) { return isfinite(a); }

// ================================================================= double
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double neg_(double a) { return -a; }
__device__ __forceinline__ double abs_(double a) { return fabs(a); }
__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
__device__ __forceinline__ double rsqrt_(double a) { return rsqrt(a); }
__device__ __forceinline__ double rint_(double a) { return rint(a); }
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double rcp_(double b) { return __ddiv_rn(1.0, b); }
__device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ void sincos_(double x, double *s, double *c) { sincos(x, s, c); }

__device__ __forceinline__ bool lt_(double a, double b) { return a < b; }
__device__ __forceinline__ bool le_(double a, double b) { return a <= b; }
__device__ __forceinline__ bool gt_(double a, double b) { return a > b; }
__device__ __forceinline__ bool ge_(double a, double b) { return a >= b; }
__device__ __forceinline__ double sel_(bool m, double a, double b) { return m ? a : b; }
__device__ __forceinline__ bool finite_(double a) { return isfinite(a); }

// Masks and status words of the scalar types.
__device__ __forceinline__ bool all_(bool m) { return m; }
__device__ __forceinline__ bool any_(bool m) { return m; }
__device__ __forceinline__ bool not_(bool m) { return !m; }
__device__ __forceinline__ bool and_(bool a, bool b) { return a && b; }
__device__ __forceinline__ bool or_(bool a, bool b) { return a || b; }
__device__ __forceinline__ unsigned bits_(bool m, unsigned b) { return m ? b : 0u; }
__device__ __forceinline__ unsigned sel_(bool m, unsigned a, unsigned b) { return m ? a : b; }
__device__ __forceinline__ bool has_bit_(unsigned st, unsigned b) { return (st & b) != 0u; }

// ========================================================== double-float
// A double-float (double-word) number: the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2, about 48 significant bits, computed with
// FP32 instructions only (GB300 issues FP32 at 64 times its FP64 rate).  The
// operations are the error-free transformations and double-word algorithms
// of the literature, written from their published descriptions (u = 2^-24):
//   two_sum       Knuth, TAOCP vol. 2, 3rd ed., sec. 4.2.2 (Moller 1965):
//                 s + e = a + b exactly, 6 operations, any a, b
//   fast_two_sum  Dekker, Numer. Math. 18 (1971) 224: the same in 3
//                 operations when |a| >= |b| (or a = 0)
//   two_prod      the product's rounding error by one fused multiply-add:
//                 p + e = a b exactly
//   add_dd        Joldes, Muller, Popescu, ACM TOMS 44 (2017) art. 15,
//                 Algorithm 6 (accurate double-word + double-word), relative
//                 error <= 3u^2 / (1 - 4u)
//   add_df        ibid., Algorithm 4 (double-word + float), <= 2u^2
//   mul_df        ibid., Algorithm 9 (double-word x float with an FMA), <= 2u^2
//   mul_dd        ibid., Algorithm 12 (double-word x double-word with FMAs),
//                 <= 4u^2
//   rcp_d         one Newton-Raphson step x0 + x0 (1 - y x0) from the
//                 correctly rounded float reciprocal x0 of y's leading part
//   dot2_df       a x + b y as a compensated dot product (below)
// Every step is an explicitly rounded float operation, so no compiler
// contraction can break an error-free transformation.
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  return {s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dfl add_dd(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  const dfl t = two_sum(x.lo, y.lo);
  const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dfl add_df(dfl x, float y) {
  const dfl s = two_sum(x.hi, y);
  return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}
__device__ __forceinline__ dfl mul_df(dfl x, float y) {
  const dfl c = two_prod(x.hi, y);
  return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}
__device__ __forceinline__ dfl mul_dd(dfl x, dfl y) {
  const dfl c = two_prod(x.hi, y.hi);
  const float t0 = __fmul_rn(x.lo, y.lo);
  const float t1 = __fmaf_rn(x.hi, y.lo, t0);
  const float c2 = __fmaf_rn(x.lo, y.hi, t1);
  return fast_two_sum(c.hi, __fadd_rn(c.lo, c2));
}
__device__ __forceinline__ dfl neg_d(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl rcp_d(dfl y) {
  const float x0 = __frcp_rn(y.hi);
  const dfl p = mul_df(y, x0);                       // y x0 = 1 - e, p.hi within ulps of 1
  const float e = __fsub_rn(__fsub_rn(1.0f, p.hi), p.lo);  // 1 - p.hi is exact
  return fast_two_sum(x0, __fmul_rn(x0, e));
}
// The float nearest to hi + lo.
__device__ __forceinline__ float to_float(dfl x) { return __fadd_rn(x.hi, x.lo); }

// a x + b y for double-word a, b and floats x, y, as a compensated dot
// product (the structure of Algorithm Dot2 of Ogita, Rump and Oishi, SIAM
// J. Sci. Comput. 26 (2005) 1955): the leading products and their sum are
// error-free (two_prod, two_sum), every rounding error and the low words'
// products are gathered in one float, and fast_two_sum renormalises.  The
// error is of order u^2 (|a x| + |b y|): like the double-word sum of the two
// double-word products (mul_df, add_dd), at about half the instructions.
__device__ __forceinline__ dfl dot2_df(dfl a, float x, dfl b, float y) {
  const dfl p = two_prod(a.hi, x), q = two_prod(b.hi, y);
  const dfl s = two_sum(p.hi, q.hi);
  float t = __fadd_rn(p.lo, q.lo);
  t = __fmaf_rn(a.lo, x, t);
  t = __fmaf_rn(b.lo, y, t);
  return fast_two_sum(s.hi, __fadd_rn(t, s.lo));
}

// c - (a x + b y) the same way, with the float c taken into the error-free
// sum.
__device__ __forceinline__ dfl sub_dot2_df(float c, dfl a, float x, dfl b, float y) {
  const dfl p = two_prod(-a.hi, x), q = two_prod(-b.hi, y);
  const dfl s1 = two_sum(p.hi, q.hi);
  const dfl s2 = two_sum(s1.hi, c);
  float t = __fadd_rn(p.lo, q.lo);
  t = __fmaf_rn(-a.lo, x, t);
  t = __fmaf_rn(-b.lo, y, t);
  t = __fadd_rn(t, s1.lo);
  return fast_two_sum(s2.hi, __fadd_rn(t, s2.lo));
}

// =============================================================== traits
// mask_t / stat_t: a comparison's result and a status word of type T;
// scalar_t: T's precision; cst<T>(v): the constant v in T.
template <class T> struct Traits;
template <> struct Traits<float> {
  using mask = bool;
  using stat = unsigned;
  using scalar = float;
};
template <> struct Traits<double> {
  using mask = bool;
  using stat = unsigned;
  using scalar = double;
};
template <class T> using mask_t = typename Traits<T>::mask;
template <class T> using stat_t = typename Traits<T>::stat;
template <class T> using scalar_t = typename Traits<T>::scalar;

template <class T> __device__ __forceinline__ T cst(double v);
template <> __device__ __forceinline__ float cst<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double cst<double>(double v) { return v; }

// A status word with `b` set where m holds.
template <class T>
__device__ __forceinline__ stat_t<T> stat_if(mask_t<T> m, unsigned b) { return bits_(m, b); }

}  // namespace num
}  // namespace kf
