// Double-float arithmetic: a real number is the unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi) / 2), added with Knuth's two-sum and multiplied with an
// FMA-based two-product (Dekker), following the double-double formulas of Hida, Li and
// Bailey's QD library with float in place of double.  ~2^-48 relative precision on the
// FP32 pipes, which on this GPU run ~58x the FP64 rate at a fraction of its latency.
// Used by the eigen-solvers (null-space step) for their serial and reduction-heavy
// parts.  Operands must stay inside the FP32 range (the callers pre-scale by a power of
// two so that the largest entry is O(1)).
#pragma once

#include <cuda_runtime.h>

namespace hicu {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
  return {s, e};
}
__device__ __forceinline__ dfl df_fast(float a, float b) {  // requires |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  return {s, __fadd_rn(b, -__fadd_rn(s, -a))};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_fast(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_fast(p, e);
}
__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {  // double-float times float
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
  return df_fast(p, e);
}
__device__ __forceinline__ dfl df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl df_f(float x) { return {x, 0.f}; }

// approximate FP32 reciprocal (one MUFU instruction, relative error ~2^-22)
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// a / b: three quotient digits, each from an approximate reciprocal of b.hi and the exact
// remainder; every digit removes the reciprocal's ~2^-22 error from the previous remainder, so
// the quotient is accurate to the double-float precision
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float r = rcp_approx(b.hi);
  const float q1 = __fmul_rn(a.hi, r);
  dfl s = df_sub(a, df_mul_f(b, q1));
  const float q2 = __fmul_rn(s.hi, r);
  s = df_sub(s, df_mul_f(b, q2));
  const float q3 = __fmul_rn(s.hi, r);
  return df_add(df_fast(q1, q2), df_f(q3));
}

// 1 / b by Newton-Raphson from an approximate reciprocal: one FP32 Newton step brings r0 to
// within an ulp of 1 / b.hi, then with the residual e = 1 - b r0 (FMA-exact for the hi part,
// |e| ~ 2^-24) the series 1 / b = r0 (1 + e + e^2 + ...) truncated after e^2 gives the low
// word.  Relative error ~2^-46, about that of one df_mul; ~10 instructions against ~35 for
// df_div, and a dependency chain half as long (used on the serial recurrences).
__device__ __forceinline__ dfl df_rcp(dfl b) {
  float r0 = rcp_approx(b.hi);
  r0 = __fmaf_rn(r0, __fmaf_rn(-b.hi, r0, 1.f), r0);
  float e = __fmaf_rn(-b.hi, r0, 1.f);
  e = __fmaf_rn(-b.lo, r0, e);
  return df_fast(r0, __fmul_rn(r0, __fmaf_rn(e, e, e)));
}

// sqrt(a), a >= 0: one Newton correction of the FP32 root with the exact residual a - x^2
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float x = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(x, x);
  const float e = __fmaf_rn(x, x, -p);
  const dfl res = df_sub(a, df_fast(p, e));
  return df_fast(x, __fmul_rn(res.hi, rcp_approx(__fmul_rn(2.f, x))));  // the correction needs ~20 bits
}

__device__ __forceinline__ dfl df_shfl_xor(dfl a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ dfl df_warp_sum(dfl a) {
  for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
  return a;
}

// complex double-float
struct cdf {
  dfl re, im;
};
__device__ __forceinline__ cdf ld4(const float4* p) {
  const float4 v = *p;
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void st4(float4* p, cdf a) { *p = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ cdf c_conj(cdf a) { return {a.re, df_neg(a.im)}; }
__device__ __forceinline__ cdf c_add(cdf a, cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf c_sub(cdf a, cdf b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ cdf c_mul(cdf a, cdf b) {
  return {df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ cdf c_mulc(cdf a, cdf b) {  // conj(a) * b
  return {df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_sub(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ cdf c_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }

// Lazily normalised accumulation for long dot products: acc.hi takes each rounded product
// through an error-free two-sum, acc.lo collects the two-sum errors and the products' low-order
// terms; renormalising after every complex product (two real products per component) keeps the
// error at the double-float level (~2^-46 of the sum of |terms|), with ~50 instructions per
// complex multiply-add against ~72 for c_add(acc, c_mul(a, b)).
__device__ __forceinline__ void df_acc_mul(dfl& acc, dfl a, dfl b) {  // acc += a b
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.hi, -p)));
  const dfl s = df_two_sum(acc.hi, p);
  acc = {s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, e))};
}
__device__ __forceinline__ cdf c_renorm(cdf a) { return {df_fast(a.re.hi, a.re.lo), df_fast(a.im.hi, a.im.lo)}; }
__device__ __forceinline__ void c_acc_mul(cdf& acc, cdf a, cdf b) {  // acc += a b
  df_acc_mul(acc.re, a.re, b.re);
  df_acc_mul(acc.re, df_neg(a.im), b.im);
  df_acc_mul(acc.im, a.re, b.im);
  df_acc_mul(acc.im, a.im, b.re);
  acc = c_renorm(acc);
}
__device__ __forceinline__ void c_acc_mulc(cdf& acc, cdf a, cdf b) {  // acc += conj(a) b
  df_acc_mul(acc.re, a.re, b.re);
  df_acc_mul(acc.re, a.im, b.im);
  df_acc_mul(acc.im, a.re, b.im);
  df_acc_mul(acc.im, df_neg(a.im), b.re);
  acc = c_renorm(acc);
}
__device__ __forceinline__ cdf c_from(double2 z) { return {df_from(z.x), df_from(z.y)}; }
__device__ __forceinline__ double2 c_to(cdf a) { return make_double2(df_to(a.re), df_to(a.im)); }
__device__ __forceinline__ cdf c_warp_sum(cdf a) { return {df_warp_sum(a.re), df_warp_sum(a.im)}; }

}  // namespace hicu
