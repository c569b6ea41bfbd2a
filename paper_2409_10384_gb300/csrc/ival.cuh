// FP32 interval arithmetic with outward (directed) rounding.  An interval
// [lo, hi] encloses the exact real value of the expression it was computed
// from, for every input in the input intervals (Moore, Interval Analysis,
// 1966).  The FP32 pipe issues about 64 times the FP64 one on this part, so
// a decision that an FP32 enclosure settles costs next to nothing beside an
// FP64 evaluation.  A NaN endpoint (out-of-range input, inf - inf, 0 * inf)
// propagates through every operation here and fails every test, so such a
// value is left to the FP64 path.
#pragma once
#include <cuda_runtime.h>

namespace grmhd {

struct Iv {
  float lo, hi;
};

__device__ __forceinline__ Iv iv_pt(float a) { return {a, a}; }
__device__ __forceinline__ Iv iv_nan() { return {__int_as_float(0x7fc00000), __int_as_float(0x7fc00000)}; }

// NaN-propagating min / max (fminf / fmaxf would drop a NaN operand)
__device__ __forceinline__ float mn_p(float a, float b) { return (a != a || a < b) ? a : b; }
__device__ __forceinline__ float mx_p(float a, float b) { return (a != a || a > b) ? a : b; }

// The FP32 interval of a double, on the integer pipe: the magnitude truncated
// to 24 significant bits and the next float above it.  |x| < 2^-126 (zero and
// subnormals) gives [0, 2^-126] with x's sign; |x| >= 2^128, inf and NaN give
// a NaN interval.
__device__ __forceinline__ Iv iv_d(double x) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned s = h & 0x80000000u;
  const int e = (int)((h >> 20) & 0x7FFu);
  if (e >= 897 && e <= 1150) {   // 2^-126 <= |x| < 2^128
    const unsigned mag = ((unsigned)(e - 896) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29);
    const float a = __uint_as_float(s | mag), b = __uint_as_float(s | (mag + 1u));   // |a| <= |x| < |b|
    return s ? Iv{b, a} : Iv{a, b};
  }
  if (e < 897) return s ? Iv{-1.17549435e-38f, 0.0f} : Iv{0.0f, 1.17549435e-38f};
  return iv_nan();
}

__device__ __forceinline__ Iv iadd(Iv a, Iv b) { return {__fadd_rd(a.lo, b.lo), __fadd_ru(a.hi, b.hi)}; }
__device__ __forceinline__ Iv isub(Iv a, Iv b) { return {__fsub_rd(a.lo, b.hi), __fsub_ru(a.hi, b.lo)}; }
__device__ __forceinline__ Iv imul(Iv a, Iv b) {
  const float p = __fmul_rd(a.lo, b.lo), q = __fmul_rd(a.lo, b.hi), r = __fmul_rd(a.hi, b.lo),
              t = __fmul_rd(a.hi, b.hi);
  const float P = __fmul_ru(a.lo, b.lo), Q = __fmul_ru(a.lo, b.hi), R = __fmul_ru(a.hi, b.lo),
              T = __fmul_ru(a.hi, b.hi);
  return {mn_p(mn_p(p, q), mn_p(r, t)), mx_p(mx_p(P, Q), mx_p(R, T))};
}
// b >= 0 (b.lo >= 0): two products
__device__ __forceinline__ Iv imulp(Iv a, Iv b) {
  return {__fmul_rd(a.lo, a.lo >= 0.0f ? b.lo : b.hi), __fmul_ru(a.hi, a.hi >= 0.0f ? b.hi : b.lo)};
}
// c >= 0 a point
__device__ __forceinline__ Iv iscale(Iv a, float c) { return {__fmul_rd(a.lo, c), __fmul_ru(a.hi, c)}; }
__device__ __forceinline__ Iv isq(Iv a) {
  if (a.lo >= 0.0f) return {__fmul_rd(a.lo, a.lo), __fmul_ru(a.hi, a.hi)};
  if (a.hi <= 0.0f) return {__fmul_rd(a.hi, a.hi), __fmul_ru(a.lo, a.lo)};
  if (a.lo != a.lo || a.hi != a.hi) return iv_nan();
  return {0.0f, mx_p(__fmul_ru(a.lo, a.lo), __fmul_ru(a.hi, a.hi))};
}
// Reciprocal and reciprocal square root from the hardware's approximations
// (rcp.approx.ftz.f32, rsqrt.approx.ftz.f32) refined by one Newton step in
// FP32.  The step leaves e0^2 (reciprocal) or 1.5 e0^2 (reciprocal square
// root) of the approximation's relative error e0 and adds its own rounding,
// at most 1.5 units of 2^-24: with e0 < 2^-13 (the documented error is about
// 2^-23) the result is within 2^-23 of the exact value, and widening it
// outward by 2^-22 encloses it.  A subnormal argument
// gives inf or NaN (a bound that decides nothing), a result below 2^-126
// gives 0 (a valid lower bound).
__device__ __forceinline__ float rcp_nr32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.0f), r);   // r (2 - x r)
}
__device__ __forceinline__ float rsqrt_nr32(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  const float e = fmaf(-x * y, y, 1.0f);   // 1 - x y^2
  return fmaf(0.5f * y, e, y);             // y (1 + e/2)
}
constexpr float IV_DN = 0.99999976f;   // 1 - 2^-22
constexpr float IV_UP = 1.00000024f;   // 1 + 2^-22
// 1/b, b > 0 (otherwise NaN)
__device__ __forceinline__ Iv ircp(Iv b) {
  if (!(b.lo > 0.0f)) return iv_nan();
  return {__fmul_rd(rcp_nr32(b.hi), IV_DN), __fmul_ru(rcp_nr32(b.lo), IV_UP)};
}
// a / b, b > 0 (otherwise NaN)
__device__ __forceinline__ Iv idiv(Iv a, Iv b) { return imulp(a, ircp(b)); }
// 1/sqrt(a), a > 0 (otherwise NaN)
__device__ __forceinline__ Iv irsqrt(Iv a) {
  if (!(a.lo > 0.0f)) return iv_nan();
  return {__fmul_rd(rsqrt_nr32(a.hi), IV_DN), __fmul_ru(rsqrt_nr32(a.lo), IV_UP)};
}
__device__ __forceinline__ Iv imax(Iv a, Iv b) { return {mx_p(a.lo, b.lo), mx_p(a.hi, b.hi)}; }
__device__ __forceinline__ Iv imin(Iv a, Iv b) { return {mn_p(a.lo, b.lo), mn_p(a.hi, b.hi)}; }
// dot product of three intervals
__device__ __forceinline__ Iv idot3(const Iv* a, const Iv* b) {
  return iadd(iadd(imul(a[0], b[0]), imul(a[1], b[1])), imul(a[2], b[2]));
}
// v_i = g_ij u^j with g packed xx, xy, xz, yy, yz, zz
__device__ __forceinline__ void ilower3(const Iv* g, const Iv* u, Iv* o) {
  o[0] = iadd(iadd(imul(g[0], u[0]), imul(g[1], u[1])), imul(g[2], u[2]));
  o[1] = iadd(iadd(imul(g[1], u[0]), imul(g[3], u[1])), imul(g[4], u[2]));
  o[2] = iadd(iadd(imul(g[2], u[0]), imul(g[4], u[1])), imul(g[5], u[2]));
}
// the whole interval strictly below / above the whole of another
__device__ __forceinline__ bool ilt(Iv a, Iv b) { return a.hi < b.lo; }
__device__ __forceinline__ bool igt(Iv a, Iv b) { return a.lo > b.hi; }

}  // namespace grmhd
