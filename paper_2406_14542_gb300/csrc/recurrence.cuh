// recurrence.cuh -- device pieces of the scaled-exponent Legendre recurrence
// shared by the single-transform kernels (legendre.cu) and the batched ones
// (batch.cu).  See legendre.cu for the formulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nusht_internal.cuh"

namespace nusht {
namespace rec {

__device__ __forceinline__ int mbase_of(int L, int m) { return m * (2 * L + 1 - m) / 2; }

__device__ __forceinline__ double exp2i(int e) {
  // 2^e for -1022 <= e <= 1023, built from the exponent field
  return __hiloint2double((e + 1023) << 20, 0);
}

// v = mant * 2^k with mant in [0.5, 1); v must be a positive normal number
__device__ __forceinline__ void renorm(double& v, int& e) {
  int hi = __double2hiint(v);
  int lo = __double2loint(v);
  int k = ((hi >> 20) & 0x7ff) - 1022;
  hi = (hi & 0x800fffff) | (1022 << 20);
  v = __hiloint2double(hi, lo);
  e += k;
}

// s^m = mant * 2^ex (s in (0, 1]), by binary powering with integer exponents
__device__ __forceinline__ void pow_scaled(double s, int m, double& mant, int& ex) {
  double b = s;
  int be = 0;
  renorm(b, be);
  double r = 1.0;
  int re = 0;
  renorm(r, re);
  while (m) {
    if (m & 1) {
      r *= b;
      re += be;
      renorm(r, re);
    }
    m >>= 1;
    if (m) {
      b *= b;
      be *= 2;
      renorm(b, be);
    }
  }
  mant = r;
  ex = re;
}

// Float from a double known to lie in (-2^64, 2^64), by truncation of the
// mantissa with integer operations (keeps the conversion off the FP64 pipe);
// values below 2^-126 become 0.
__device__ __forceinline__ float to_f32(double q) {
  int hi = __double2hiint(q);
  unsigned lo = (unsigned)__double2loint(q);
  int e = ((hi >> 20) & 0x7ff) - 1023;
  unsigned mant = ((unsigned)(hi & 0xfffff) << 3) | (lo >> 29);
  unsigned bits = ((unsigned)hi & 0x80000000u) | ((unsigned)(e + 127) << 23) | mant;
  return (e < -126) ? 0.0f : __uint_as_float(bits);
}

template <typename T>
struct V2;
template <>
struct V2<double> {
  using t = double2;
};
template <>
struct V2<float> {
  using t = float2;
};

template <typename T>
__device__ __forceinline__ T conv(double q);
template <>
__device__ __forceinline__ double conv<double>(double q) {
  return q;
}
template <>
__device__ __forceinline__ float conv<float>(double q) {
  return to_f32(q);
}

// One recurrence chain (a ring pair).
struct Chain {
  double x, q1, q2;
  int E;      // > 0: scaled phase, value = q * 2^-E; 0: ordinary values
  bool valid;
};

template <class A>
__device__ __forceinline__ void chain_init(Chain& ch, const A& a, int m, int j) {
  ch.valid = (j >= 1 && j <= a.npairs);
  ch.q2 = 0.0;
  if (!ch.valid) {
    ch.x = 0.0;
    ch.q1 = 0.0;
    ch.E = 0;
    return;
  }
  ch.x = __ldg(a.ring_x + (j - 1));
  double s = __ldg(a.ring_s + (j - 1));
  double mant;
  int ex;
  pow_scaled(s, m, mant, ex);
  double q0 = __ldg(a.cm + m) * mant;
  if (ex >= LEG_TINY_EXP) {
    ch.q1 = q0 * exp2i(ex);
    ch.E = 0;
  } else {
    int E = LEG_STEP_EXP * ((LEG_TINY_EXP - ex + LEG_STEP_EXP - 1) / LEG_STEP_EXP);
    ch.q1 = q0 * exp2i(ex + E);
    ch.E = E;
  }
}

// v * 2^k through the exponent field (integer operations only); zero and
// subnormal inputs are returned unchanged.  Used for the power-of-two
// rescalings so that they never occupy the FP64 pipe (on sm_103a the FP64
// pipe is 1/64 of the FP32 rate, and warp-uniform branches around FP64
// multiplies are if-converted into predicated instructions that still issue).
__device__ __forceinline__ double scale_pow2(double v, int k) {
  int hi = __double2hiint(v);
  const int lo = __double2loint(v);
  hi = (hi & 0x7ff00000) ? hi + (k << 20) : hi;
  return __hiloint2double(hi, lo);
}

// Advance to degree l: optional segment rescale (q_{l-1}, q_{l-2}) *= 2^48,
// then q_l = x q_{l-1} - c q_{l-2}: two FP64 operations.  In the scaled phase
// the exponent check and the 2^-256 step are integer operations.
__device__ __forceinline__ void chain_step(Chain& ch, double c, bool do_rescale) {
  if (do_rescale) {
    ch.q1 = scale_pow2(ch.q1, LEG_SEG_BITS);
    ch.q2 = scale_pow2(ch.q2, LEG_SEG_BITS);
  }
  double t = c * ch.q2;
  double q = fma(ch.x, ch.q1, -t);
  ch.q2 = ch.q1;
  ch.q1 = q;
  if (ch.E != 0) {
    int expo = (__double2hiint(q) >> 20) & 0x7ff;
    if (expo >= 1023 - 44) {
      ch.q1 = scale_pow2(ch.q1, -LEG_STEP_EXP);
      ch.q2 = scale_pow2(ch.q2, -LEG_STEP_EXP);
      ch.E -= LEG_STEP_EXP;
    }
  }
}

}  // namespace rec
}  // namespace nusht
