// Float-float arithmetic (the unevaluated sum hi + lo of two FP32 values, ~2^-48 relative) and
// FP32 <-> FP64 conversions on the integer pipe, for the small R x R stages of the Gram-route QRs
// and the Gram partials of the mode update.
#pragma once
#include <cuda_runtime.h>

namespace cpqr {
namespace ffa {

constexpr unsigned FF_FULL = 0xffffffffu;

// ---- float-float numbers: the unevaluated sum hi + lo of two FP32 values (~2^-48 relative) ----
// GB300 issues one FP64 warp instruction per 64 cycles per SM sub-partition at a 64-cycle
// latency, FP32 one per cycle at 4 cycles, so the serial Cholesky runs in float-float.  The
// operations are the error-free transformations TwoSum (Knuth) and TwoProd by FMA, written with
// the _rn intrinsics so that the compiler neither contracts nor reorders them.
struct ffn {
  float hi, lo;
};
__device__ __forceinline__ ffn ff_make(float hi, float lo) {
  ffn r;
  r.hi = hi;
  r.lo = lo;
  return r;
}
__device__ __forceinline__ ffn ff_ld(const float2& v) { return ff_make(v.x, v.y); }
__device__ __forceinline__ float2 ff_st(ffn a) { return make_float2(a.hi, a.lo); }
// FP32 -> FP64, exact for zero and normal numbers (subnormal inputs, below 1.2e-38, read as
// zero), by moving the IEEE-754 fields on the integer pipe: exponent rebiased from 127 to 1023,
// mantissa widened.  (A conversion instruction would occupy the slow FP64 pipe.)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xffu;
  const unsigned int E = (e == 0u) ? 0u : ((e == 255u) ? 2047u : e + 896u);
  const unsigned long long m = (e == 0u) ? 0ull : (unsigned long long)(b & 0x7fffffu) << 29;
  return __longlong_as_double(
      (long long)(((unsigned long long)(b & 0x80000000u) << 32) | ((unsigned long long)E << 52) | m));
}
// FP64 -> FP32 rounded toward zero (below the FP32 normal range: zero; above: infinity, which
// fails the pivot test), by moving the fields.
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32);
  const unsigned int sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned int)e << 23) | (unsigned int)((b >> 29) & 0x7fffffull));
}
// x as hi + lo (both truncated: ~2^-48 relative; x - hi is exact in FP64), one FP64 subtraction
__device__ __forceinline__ ffn ff_from_bits(double x) {
  const float h = d2f_trunc(x);
  return ff_make(h, d2f_trunc(x - f2d_bits(h)));
}
// hi + lo in FP64 with one FP64 addition
__device__ __forceinline__ double ff_val(const float2& v) { return f2d_bits(v.x) + f2d_bits(v.y); }
__device__ __forceinline__ double ff_val(ffn a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }
__device__ __forceinline__ ffn ff_shfl(ffn a, int src) {
  return ff_make(__shfl_sync(FF_FULL, a.hi, src), __shfl_sync(FF_FULL, a.lo, src));
}
// a b
__device__ __forceinline__ ffn ff_mul(ffn a, ffn b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float h = __fadd_rn(p, e);
  return ff_make(h, __fsub_rn(e, __fsub_rn(h, p)));
}
// t - a b
__device__ __forceinline__ ffn ff_fms(ffn t, ffn a, ffn b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const float s = __fsub_rn(t.hi, p);  // TwoSum(t.hi, -p)
  const float bb = __fsub_rn(s, t.hi);
  float err = __fadd_rn(__fsub_rn(t.hi, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
  err = __fadd_rn(err, __fsub_rn(t.lo, pe));
  const float h = __fadd_rn(s, err);
  return ff_make(h, __fsub_rn(err, __fsub_rn(h, s)));
}
// a + b
__device__ __forceinline__ ffn ff_add(ffn a, ffn b) {
  const float s = __fadd_rn(a.hi, b.hi);  // TwoSum(a.hi, b.hi)
  const float bb = __fsub_rn(s, a.hi);
  float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  err = __fadd_rn(err, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, err);
  return ff_make(h, __fsub_rn(err, __fsub_rn(h, s)));
}
__device__ __forceinline__ ffn ff_neg(ffn a) { return ff_make(-a.hi, -a.lo); }
// 1 / d for a pivot d: rcp.approx.ftz.f32 (at most 1 ulp off) and one Newton-Raphson step
// y <- y + y (1 - d y) with the residual formed in float-float (error ~2^-46).  A pivot outside
// (1e-30, 1e30), or not a number, sets *bad and gives 0.  d is warp-uniform.
__device__ __forceinline__ ffn ff_recip(ffn d, int* bad) {
  if (!(d.hi > 1e-30f && d.hi < 1e30f)) {
    *bad = 1;
    return ff_make(0.0f, 0.0f);
  }
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d.hi));
  const float p = __fmul_rn(d.hi, y);
  float pe = __fmaf_rn(d.hi, y, -p);
  pe = __fmaf_rn(d.lo, y, pe);
  const float r = __fsub_rn(__fsub_rn(1.0f, p), pe);
  const float c = __fmul_rn(y, r);
  const float h = __fadd_rn(y, c);
  return ff_make(h, __fsub_rn(c, __fsub_rn(h, y)));
}

}  // namespace ffa
}  // namespace cpqr
