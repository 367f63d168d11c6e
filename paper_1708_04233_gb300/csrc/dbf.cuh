// Double-float arithmetic (a real number as an unevaluated sum of two FP32
// values) for phases that FP32 alone cannot carry: GB300's FP64 units run far
// slower than its FP32 units, and phases of 10^4 .. 10^6 cycles need some 44
// bits before their reduction to [0, 1).
#pragma once

#include "internal.cuh"

namespace wsb {

// A real number as an unevaluated sum hi + lo of two FP32 values
// ("double-float"): the error-free transformations are Knuth's two-sum and
// the exact product through one fused multiply-add.  Products that feed
// them are rounded explicitly (__fmul_rn) so that no contraction into an FMA
// changes them.
struct Dbf {
  float hi, lo;
};
__device__ __forceinline__ Dbf two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// (c.hi + c.lo) x for a float x exact in FP32.
__device__ __forceinline__ Dbf dbf_mul_f(Dbf c, float x) {
  const float p = __fmul_rn(c.hi, x);
  return {p, __fmaf_rn(c.lo, x, __fmaf_rn(c.hi, x, -p))};
}
// (a.hi + a.lo)^2.
__device__ __forceinline__ Dbf dbf_sqr(Dbf a) {
  const float p = __fmul_rn(a.hi, a.hi);
  return {p, __fmaf_rn(2.0f * a.hi, a.lo, __fmaf_rn(a.hi, a.hi, -p))};
}

// A double as a double-float.
inline Dbf split(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}

// The spherical reference wave in double-float: source position (x, y) in
// pixels, a2 = (pitch / lambda)^2, c = (z / lambda)^2, sgn = sign of z.
struct RefDbf {
  Dbf x, y, a2, c;
  float sgn;
  int kind;
};

// A real a.hi + a.lo + b, renormalised.
__device__ __forceinline__ Dbf dbf_add_f(Dbf a, float b) {
  const Dbf s = two_sum(a.hi, b);
  return two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// frac(t) of the reference phase t = sqrt(a2 ((X - x)^2 + (Y - y)^2) + c)
// cycles at plane pixel (X, Y), |X|, |Y| < 2^24: t reaches 10^6 cycles for a
// source some 0.4 m away, so it is carried in double-float like the transfer
// function's phase.
__device__ __forceinline__ float ref_frac(const RefDbf& r, float X, float Y) {
  const Dbf ex = dbf_add_f(two_sum(X, -r.x.hi), -r.x.lo), ey = dbf_add_f(two_sum(Y, -r.y.hi), -r.y.lo);
  const Dbf px = dbf_sqr(ex), py = dbf_sqr(ey);
  const Dbf rho = two_sum(px.hi, py.hi);
  const float rl = __fadd_rn(rho.lo, __fadd_rn(px.lo, py.lo));
  const float p = __fmul_rn(r.a2.hi, rho.hi);
  const float pe = __fmaf_rn(r.a2.hi, rho.hi, -p) + (r.a2.hi * rl + r.a2.lo * rho.hi);
  const Dbf t0 = two_sum(p, r.c.hi);
  const Dbf tt = two_sum(t0.hi, __fadd_rn(t0.lo, __fadd_rn(pe, r.c.lo)));
  const float y = __fsqrt_rn(tt.hi);
  const float yy = __fmul_rn(y, y), ye = __fmaf_rn(y, y, -yy);
  const float corr = __fmul_rn(__fadd_rn(__fsub_rn(__fsub_rn(tt.hi, yy), ye), tt.lo), __fdividef(0.5f, y));
  float f = __fadd_rn(__fsub_rn(y, floorf(y)), corr);
  return f - floorf(f);
}

// The spherical reference of a frame in double-float.
inline RefDbf ref_dbf(const RefDev& r) {
  RefDbf d;
  d.kind = r.kind;
  d.sgn = r.sgn;
  d.x = split(r.x);
  d.y = split(r.y);
  d.a2 = split(r.a2);
  d.c = split(r.c);
  return d;
}

}  // namespace wsb
