// dfloat.cuh -- double-float ("float pair") arithmetic for FP64-mode kernels.
//
// GB300 runs FP64 at 1/62 of the FP32 rate, so FP64-mode sums and products
// that do not need the FP64 exponent range are carried as unevaluated pairs
// hi + lo of floats (~48-bit significand):
//   * a double is split into hi + lo with integer bit operations only (no
//     FP64 instruction);
//   * a product is formed exactly (p = ah*bh, its rounding error by an FMA)
//     plus the cross terms ah*bl + al*bh;
//   * sums use the two-sum error-free transformation.
// Relative error per operation ~2^-47.  Range: the float exponent range
// (|x| in [2^-126, 2^127]); smaller magnitudes flush to zero.
#pragma once
#include <cuda_runtime.h>

namespace nusht {

__device__ __forceinline__ void split_q(double q, float& qh, float& ql) {
  const int hi = __double2hiint(q);
  const unsigned lo = (unsigned)__double2loint(q);
  const int eb = (hi >> 20) & 0x7ff;  // biased exponent
  const unsigned sign = (unsigned)hi & 0x80000000u;
  if (eb < 1023 - 126) {  // |q| < 2^-126 (or zero): negligible, flushed
    qh = 0.0f;
    ql = 0.0f;
    return;
  }
  // leading 24 significant bits, exactly representable as a float
  const unsigned mh = ((unsigned)(hi & 0xfffff) << 3) | (lo >> 29);
  qh = __uint_as_float(sign | ((unsigned)(eb - 1023 + 127) << 23) | mh);
  // remaining 29 bits r: value r * 2^(e - 52), rounded to 24 bits
  const float r = __uint2float_rn(lo & 0x1fffffffu);
  const int ef = eb - 1023 - 52 + 127;
  const float sc = ef >= 1 ? __uint_as_float((unsigned)ef << 23) : 0.0f;
  ql = __uint_as_float(__float_as_uint(__fmul_rn(r, sc)) | sign);
}

// (sh + sl) += (ah + al) * (qh + ql)
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float qh, float ql) {
  const float p = __fmul_rn(ah, qh);
  const float e = __fmaf_rn(ah, qh, -p);
  const float t = __fmaf_rn(ah, ql, __fmaf_rn(al, qh, e));
  const float s = __fadd_rn(sh, p);
  const float bp = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  const float l = __fadd_rn(sl, __fadd_rn(err, t));
  // renormalise (fast two-sum, |s| >= |l|): lo stays within half an ulp of
  // hi, so its rounding error per step is ~2^-48 of the sum and does not
  // grow with the number of accumulated terms
  sh = __fadd_rn(s, l);
  sl = __fsub_rn(l, __fsub_rn(sh, s));
}

// (ah + al) += (bh + bl)
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float bp = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bp)), __fsub_rn(bh, bp));
  const float l = __fadd_rn(__fadd_rn(al, bl), err);
  ah = __fadd_rn(s, l);  // renormalise, as in df_mac
  al = __fsub_rn(l, __fsub_rn(ah, s));
}

__device__ __forceinline__ double df_value(float h, float l) { return (double)h + (double)l; }

// float pair of a double: h = rn(v), l = rn(v - h)
__device__ __forceinline__ void df_of(double v, float& h, float& l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - (double)h);
}

// split of an arbitrary double (saturates to +-inf above the float range)
__device__ __forceinline__ void df_split(double v, float& h, float& l) {
  const int eb = (__double2hiint(v) >> 20) & 0x7ff;
  if (eb > 1023 + 127) {
    h = v > 0.0 ? __int_as_float(0x7f800000) : __int_as_float((int)0xff800000);
    l = 0.0f;
    return;
  }
  split_q(v, h, l);
}

// (h + l) = (ah + al) * (bh + bl), renormalised
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
  const float s = __fadd_rn(p, e);
  return make_float2(s, __fsub_rn(e, __fsub_rn(s, p)));
}

}  // namespace nusht
