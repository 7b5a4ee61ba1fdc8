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

// Advance to degree l: optional segment rescale (q_{l-1}, q_{l-2}) *= 2^shift
// (shift from the plan's table: its segment width, or 0), then
// q_l = x q_{l-1} - c q_{l-2}: two FP64 operations.  In the scaled phase the
// exponent check and the 2^-256 step are integer operations.
__device__ __forceinline__ void chain_step(Chain& ch, double c, int shift) {
  if (shift) {
    ch.q1 = scale_pow2(ch.q1, shift);
    ch.q2 = scale_pow2(ch.q2, shift);
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

// ---------------------------------------------------------------------------
// The same recurrence in double-float (opt-in, opts.fast_recurrence): x, q_l
// and c_l are float pairs hi + lo, one step is two exact float-pair products
// and a two-sum difference, renormalised (~20 FP32 operations, ~2^-47
// relative per step, against two FP64 operations on a pipe 62x slower).
// The float exponent range changes two things.  The plan's normalisation
// segments are LEG_SEG_BITS_DF = 24 bits wide (so q = Pbar / Ahat varies by at
// most 2^24 against Pbar inside a segment), and values below 2^-76 are
// carried as q * 2^E (E a multiple of 64): an ordinary value then stays above
// 2^-100 with a normal lo word, and a scaled one has |Pbar| < 2^-52.
// ---------------------------------------------------------------------------
constexpr int DF_TINY_EXP = -76;
constexpr int DF_STEP_EXP = 64;

struct DfChain {
  float2 x, q1, q2;
  int E;  // > 0: scaled phase, value = q * 2^-E; 0: ordinary values
  bool valid;
};

// float pair of a double (plan/initialisation only: FP64 conversions)
__device__ __forceinline__ float2 df2_of(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// v * 2^k, -126 <= k <= 127: one FP32 multiply by an exact power of two
// (correct for zero and subnormal inputs as well)
__device__ __forceinline__ float scale_pow2f(float v, int k) {
  return __fmul_rn(v, __uint_as_float((unsigned)(k + 127) << 23));
}

template <class A>
__device__ __forceinline__ void chain_init(DfChain& ch, const A& a, int m, int j) {
  ch.valid = (j >= 1 && j <= a.npairs);
  ch.q2 = make_float2(0.f, 0.f);
  if (!ch.valid) {
    ch.x = make_float2(0.f, 0.f);
    ch.q1 = make_float2(0.f, 0.f);
    ch.E = 0;
    return;
  }
  ch.x = df2_of(__ldg(a.ring_x + (j - 1)));
  const double s = __ldg(a.ring_s + (j - 1));
  double mant;
  int ex;
  pow_scaled(s, m, mant, ex);
  const double q0 = __ldg(a.cm + m) * mant;
  if (ex >= DF_TINY_EXP) {
    ch.q1 = df2_of(q0 * exp2i(ex));
    ch.E = 0;
  } else {
    const int E = DF_STEP_EXP * ((DF_TINY_EXP - ex + DF_STEP_EXP - 1) / DF_STEP_EXP);
    ch.q1 = df2_of(q0 * exp2i(ex + E));
    ch.E = E;
  }
}

__device__ __forceinline__ void chain_step(DfChain& ch, float2 c, int shift) {
  if (shift) {
    ch.q1 = make_float2(scale_pow2f(ch.q1.x, shift), scale_pow2f(ch.q1.y, shift));
    ch.q2 = make_float2(scale_pow2f(ch.q2.x, shift), scale_pow2f(ch.q2.y, shift));
  }
  // x q1 and c q2, each exact product plus cross terms
  const float p1 = __fmul_rn(ch.x.x, ch.q1.x);
  float e1 = __fmaf_rn(ch.x.x, ch.q1.x, -p1);
  e1 = __fmaf_rn(ch.x.x, ch.q1.y, __fmaf_rn(ch.x.y, ch.q1.x, e1));
  const float p2 = __fmul_rn(c.x, ch.q2.x);
  float e2 = __fmaf_rn(c.x, ch.q2.x, -p2);
  e2 = __fmaf_rn(c.x, ch.q2.y, __fmaf_rn(c.y, ch.q2.x, e2));
  // (p1 - p2) by two-sum, then the error terms, then renormalise
  const float sd = __fsub_rn(p1, p2);
  const float bp = __fsub_rn(sd, p1);
  const float err = __fadd_rn(__fsub_rn(p1, __fsub_rn(sd, bp)), __fsub_rn(-p2, bp));
  const float t = __fadd_rn(err, __fsub_rn(e1, e2));
  const float hi = __fadd_rn(sd, t);
  ch.q2 = ch.q1;
  ch.q1 = make_float2(hi, __fsub_rn(t, __fsub_rn(hi, sd)));
  if (ch.E != 0) {
    const int expo = (int)((__float_as_uint(ch.q1.x) >> 23) & 0xff);
    if (expo >= 127 + DF_TINY_EXP + DF_STEP_EXP) {
      ch.q1 = make_float2(scale_pow2f(ch.q1.x, -DF_STEP_EXP), scale_pow2f(ch.q1.y, -DF_STEP_EXP));
      ch.q2 = make_float2(scale_pow2f(ch.q2.x, -DF_STEP_EXP), scale_pow2f(ch.q2.y, -DF_STEP_EXP));
      ch.E -= DF_STEP_EXP;
    }
  }
}

// per-chain-type access: the step coefficient and the current value as a
// float pair or a single float
template <class A>
__device__ __forceinline__ double coef(const A& a, int i, const Chain&) {
  return __ldg(a.c + i);
}
template <class A>
__device__ __forceinline__ float2 coef(const A& a, int i, const DfChain&) {
  return __ldg(a.cdf + i);
}
__device__ __forceinline__ float qf(const Chain& ch) { return to_f32(ch.q1); }
__device__ __forceinline__ float qf(const DfChain& ch) { return ch.q1.x; }

}  // namespace rec
}  // namespace nusht
