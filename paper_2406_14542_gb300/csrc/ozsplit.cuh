// ozsplit.cuh -- the integer arithmetic of the split ("Ozaki") contraction of
// FP64 batched plans (batch.cu): a value x with |x| < 2^e becomes
//   F = round(x 2^(OZ_FB - e)) = sum_{i < OZ_NS} d_i 256^(OZ_NS - 1 - i),
// its balanced base-256 digits d_i (|d_i| <= 129), stored as the bf16 slices
// d_i 2^(-8 i); and a 64-bit fixed-point sum N becomes the double N 2^k.
// Everything here is integer and bit arithmetic (no FP64 instruction on the
// device), written for both the device and the host so that the CPU tests
// can check it directly.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#endif

namespace nusht {

constexpr int OZ_NS = 6;                    // slices per operand
constexpr int OZ_FB = 8 * (OZ_NS - 1) + 7;  // F = round(x 2^(OZ_FB - e)), |F| < 2^47

OZ_HD unsigned long long oz_bits_d(double v) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  std::memcpy(&b, &v, 8);
  return b;
#endif
}
OZ_HD double oz_double_of(unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double v;
  std::memcpy(&v, &b, 8);
  return v;
#endif
}
OZ_HD uint32_t oz_bits_f(float v) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(v);
#else
  uint32_t b;
  std::memcpy(&b, &v, 4);
  return b;
#endif
}
OZ_HD float oz_float_of(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float v;
  std::memcpy(&v, &b, 4);
  return v;
#endif
}
OZ_HD int oz_clz64(unsigned long long u) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)u);
#else
  return __builtin_clzll(u);
#endif
}

// balanced base-256 digits: F = sum_i d[i] 256^(OZ_NS - 1 - i), d[1..] in [-128, 127]
OZ_HD void oz_digits(long long F, int (&d)[OZ_NS]) {
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int i = OZ_NS - 1; i > 0; --i) {
    const long long r = ((F + 128) & 255) - 128;
    d[i] = (int)r;
    F = (F - r) >> 8;  // exact: F - r is a multiple of 256
  }
  d[0] = (int)F;
}

// bf16 bits of d 2^(-8 i): the float is exact and its low 16 bits are zero
OZ_HD uint32_t oz_bf16(int d, int i) { return oz_bits_f((float)d * oz_float_of((uint32_t)(127 - 8 * i) << 23)) >> 16; }

// round(v 2^k) as a 64-bit integer (|v 2^k| < 2^52); zero and subnormal v give 0
OZ_HD long long oz_fix_d(double v, int k) {
  const unsigned long long b = oz_bits_d(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return 0;
  const long long mant = (long long)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  const int sh = ex - 1075 + k;  // v = mant 2^(ex - 1075)
  long long r;
  if (sh >= 0)
    r = mant << (sh < 11 ? sh : 11);
  else if (sh <= -54)
    r = 0;
  else
    r = (mant + (1ll << (-sh - 1))) >> (-sh);
  return (b >> 63) ? -r : r;
}

// round(v 2^k) for a float (|v 2^k| < 2^62)
OZ_HD long long oz_fix_f(float v, int k) {
  const uint32_t b = oz_bits_f(v);
  const int ex = (int)((b >> 23) & 0xff);
  if (ex == 0) return 0;
  const long long mant = (long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = ex - 150 + k;  // v = mant 2^(ex - 150)
  long long r;
  if (sh >= 0)
    r = mant << (sh < 38 ? sh : 38);
  else if (sh <= -25)
    r = 0;
  else
    r = (mant + (1ll << (-sh - 1))) >> (-sh);
  return (b >> 31) ? -r : r;
}

// N 2^k as a double (round half away from zero to 53 bits); results below
// the normal range are 0
OZ_HD double oz_dbl(long long N, int k) {
  if (N == 0) return 0.0;
  const unsigned long long sgn = N < 0 ? (1ull << 63) : 0ull;
  const unsigned long long u = N < 0 ? (unsigned long long)(-N) : (unsigned long long)N;
  const int top = 63 - oz_clz64(u);  // index of the leading one
  int e2 = top + k;
  unsigned long long mnt;
  if (top > 52) {
    const int s = top - 52;
    mnt = (u + (1ull << (s - 1))) >> s;
    if (mnt >> 53) {
      mnt >>= 1;
      ++e2;
    }
  } else {
    mnt = u << (52 - top);
  }
  if (e2 < -1022) return 0.0;
  if (e2 > 1023) return oz_double_of(sgn | 0x7ff0000000000000ull);
  return oz_double_of(sgn | ((unsigned long long)(e2 + 1023) << 52) | (mnt & 0xfffffffffffffull));
}

// 2^k as a float (0 below the normal range, saturated above)
OZ_HD float oz_pow2f(int k) {
  k = k > 127 ? 127 : k;
  return k < -126 ? 0.f : oz_float_of((uint32_t)(k + 127) << 23);
}

// exponent e with |x| < 2^e of the double whose |bits| are b (0 for b = 0)
OZ_HD int oz_exp_of(unsigned long long b) { return b ? (int)(b >> 52) - 1022 : 0; }

}  // namespace nusht
