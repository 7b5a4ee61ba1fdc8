// dfft.cu -- double-float FFTs of FP64 plans: the theta transform (F in
// Eq. SHTfast, the 1D DFT of the doubled ring map along theta) and the 2D
// real transform of the NUFFT's fine grid (the uniform FFT step of the type 1
// and type 2 NUFFT), each line transformed in shared memory.
//
// GB300 issues FP64 at 1/62 of its FP32 rate, and cuFFT's FP64 transforms are
// bound by that pipe.  Here every complex value is an unevaluated pair of
// floats per component (re.hi, re.lo, im.hi, im.lo; ~2^-47 relative per
// operation, see dfloat.cuh), and the arithmetic runs on the FP32 pipe.
//
// One CTA owns one line of length N (N * 16 bytes of shared memory, N up to
// DFFT_NMAX).  The transform is an in-place mixed-radix decimation in
// frequency (radices 2, 3, 4, 5, 7): a pass of radix R over sub-blocks of
// length L combines the R values b*L + j + r*(L/R) and multiplies output q by
// W_L^(j q).  The result is left in digit-reversed order; `rev` maps an output
// index to its shared-memory position and the store reads through it.
//
// Fine grid (n1 x n2 real, rows of stride n2 + 2 doubles):
//   synthesis: dfft_cols_synth_k  (per order m <= mmax: deconvolve and
//              zero-pad the theta spectrum to n1, inverse DFT along theta,
//              store the column as row m of the order-major buffer T[m][j]);
//              dfft_rows_c2r_k (per pair of rows j, j+1: the two Hermitian
//              half spectra X_j[m], X_j+1[m] (m <= mmax) packed as
//              C = X_j + i X_j+1 over the full length, one inverse DFT,
//              x_j = Re, x_j+1 = Im).
//   adjoint:   dfft_rows_r2c_k (the two real rows as one complex sequence,
//              one forward DFT, spectra of each separated by the Hermitian
//              symmetry, m <= mmax kept); dfft_cols_adj_k (forward DFT along
//              theta per order, truncation to |k| <= lmax and deconvolution).
// The DFT sign and scale match cuFFT's (unnormalised; "forward" = e^-i).
#include <algorithm>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "nusht_internal.cuh"

namespace nusht {
namespace {

// threads per line: 1024 for lengths whose radices are 2, 3, 4 (54 to 62
// registers), 512 when a radix 5 or 7 pass is compiled in (up to 128)
constexpr int DFFT_T_WIDE = 1024, DFFT_T_ODD = 512;

// ---------------------------------------------------------------------------
// float-pair complex arithmetic (float4 = re.hi, re.lo, im.hi, im.lo)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 dd_add(float ah, float al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float bp = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bp)), __fsub_rn(bh, bp));
  const float l = __fadd_rn(__fadd_rn(al, bl), err);
  const float h = __fadd_rn(s, l);
  return make_float2(h, __fsub_rn(l, __fsub_rn(h, s)));
}

// x*y + u*v for float pairs, one renormalisation
__device__ __forceinline__ float2 dd_dot2(float xh, float xl, float yh, float yl, float uh, float ul, float vh,
                                          float vl) {
  const float p1 = __fmul_rn(xh, yh);
  const float e1 = __fmaf_rn(xh, yh, -p1);
  const float p2 = __fmul_rn(uh, vh);
  const float e2 = __fmaf_rn(uh, vh, -p2);
  const float s = __fadd_rn(p1, p2);
  const float bp = __fsub_rn(s, p1);
  const float err = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bp)), __fsub_rn(p2, bp));
  float t = __fadd_rn(e1, e2);
  t = __fmaf_rn(xh, yl, t);
  t = __fmaf_rn(xl, yh, t);
  t = __fmaf_rn(uh, vl, t);
  t = __fmaf_rn(ul, vh, t);
  const float l = __fadd_rn(t, err);
  const float h = __fadd_rn(s, l);
  return make_float2(h, __fsub_rn(l, __fsub_rn(h, s)));
}

__device__ __forceinline__ float4 c_add(float4 a, float4 b) {
  const float2 r = dd_add(a.x, a.y, b.x, b.y), i = dd_add(a.z, a.w, b.z, b.w);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ float4 c_sub(float4 a, float4 b) {
  const float2 r = dd_add(a.x, a.y, -b.x, -b.y), i = dd_add(a.z, a.w, -b.z, -b.w);
  return make_float4(r.x, r.y, i.x, i.y);
}
// a * (SG i)
template <int SG>
__device__ __forceinline__ float4 c_mul_i(float4 a) {
  return SG > 0 ? make_float4(-a.z, -a.w, a.x, a.y) : make_float4(a.z, a.w, -a.x, -a.y);
}
// a * (c + SG i s), w = (c.hi, c.lo, s.hi, s.lo)
template <int SG>
__device__ __forceinline__ float4 c_mul_tw(float4 a, float4 w) {
  const float sh = SG > 0 ? w.z : -w.z, sl = SG > 0 ? w.w : -w.w;
  const float2 re = dd_dot2(a.x, a.y, w.x, w.y, -a.z, -a.w, sh, sl);
  const float2 im = dd_dot2(a.x, a.y, sh, sl, a.z, a.w, w.x, w.y);
  return make_float4(re.x, re.y, im.x, im.y);
}
// a * (real pair c)
__device__ __forceinline__ float4 c_scale(float4 a, float2 c) {
  const float2 re = df_mul(make_float2(a.x, a.y), c), im = df_mul(make_float2(a.z, a.w), c);
  return make_float4(re.x, re.y, im.x, im.y);
}
// acc += a * (real pair c)
__device__ __forceinline__ void c_mac(float4& acc, float4 a, float2 c) {
  df_mac(acc.x, acc.y, a.x, a.y, c.x, c.y);
  df_mac(acc.z, acc.w, a.z, a.w, c.x, c.y);
}

// conversions with integer operations only (the FP64 pipe issues a warp's
// conversion or add once per 64 cycles per SM sub-partition)
// double -> float pair: leading 24 bits and the rounded rest; |v| below 2^-126
// flushes to zero, above the float range saturates
__device__ __forceinline__ void split_d(double v, float& h, float& l) {
  const int hi = __double2hiint(v);
  if (((hi >> 20) & 0x7ff) > 1023 + 127) {
    h = __int_as_float(hi < 0 ? (int)0xff800000 : 0x7f800000);
    l = 0.0f;
    return;
  }
  split_q(v, h, l);
}
// renormalised float pair (|l| <= ulp(h)) -> double, within 2^-52 relative:
// the two significands aligned and added as integers
__device__ __forceinline__ double pair_to_double(float h, float l) {
  const unsigned hb = __float_as_uint(h), lb = __float_as_uint(l);
  const int eh = (int)((hb >> 23) & 0xffu);
  if (eh == 0) return 0.0;
  long long mh = (long long)((hb & 0x7fffffu) | 0x800000u) << 29;  // unit 2^(eh - 127 - 52)
  int el = (int)((lb >> 23) & 0xffu);
  long long ml = (long long)(lb & 0x7fffffu);
  if (el != 0) {
    ml |= 0x800000;
  } else {
    el = 1;  // subnormal l
  }
  if (ml != 0) {
    const int sh = el - eh + 29;
    ml = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> -sh) : 0);
    mh = ((hb ^ lb) & 0x80000000u) ? mh - ml : mh + ml;
  }
  long long e = eh - 127 + 1023;
  if (mh >= (1LL << 53)) {
    mh >>= 1;
    ++e;
  } else if (mh < (1LL << 52)) {
    mh <<= 1;
    --e;
  }
  const unsigned long long bits = ((unsigned long long)(hb & 0x80000000u) << 32) | ((unsigned long long)e << 52) |
                                  ((unsigned long long)mh & ((1ULL << 52) - 1));
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ float4 c_of(double2 v) {
  float4 r;
  split_d(v.x, r.x, r.y);
  split_d(v.y, r.z, r.w);
  return r;
}
__device__ __forceinline__ double2 c_value(float4 c) {
  return make_double2(pair_to_double(c.x, c.y), pair_to_double(c.z, c.w));
}

// ---------------------------------------------------------------------------
// The float-pair line transform is written against a complex-type trait
// (CDF: the float-pair complex above).
// ---------------------------------------------------------------------------
struct CDF {
  using V = float4;
  static __device__ __forceinline__ V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ V add(V a, V b) { return c_add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return c_sub(a, b); }
  template <int SG>
  static __device__ __forceinline__ V mul_i(V a) {
    return c_mul_i<SG>(a);
  }
  template <int SG>
  static __device__ __forceinline__ V mul_tw(V a, float4 w) {
    return c_mul_tw<SG>(a, w);
  }
  // acc += a * (h + l), a real float pair
  static __device__ __forceinline__ void mac(V& acc, V a, float h, float l) { c_mac(acc, a, make_float2(h, l)); }
};


// Shared-memory position of value i of a float-pair line (16 bytes per
// value, 8 values per 128-byte bank row): i ^ ((i >> 3 ^ i >> 7 ^ i >> 11)
// mod 8), a permutation inside each aligned group of 8 values.  The strided
// butterfly accesses and the digit-reversed read of the output then spread
// over the banks (1.2 wavefronts per quarter warp against the ideal 1, where
// the plain layout takes 2.0, 8 for the reversed read alone).
__device__ __forceinline__ int dsw(int i) { return i ^ (((i >> 3) ^ (i >> 7) ^ (i >> 11)) & 7); }
// float4 slots of a line of n values
__host__ __device__ __forceinline__ int dline_words(int n) { return (n + 7) & ~7; }

// ---------------------------------------------------------------------------
// small DFTs of the butterflies (sign SG: +1 inverse, -1 forward)
// ---------------------------------------------------------------------------
template <int SG, class C>
__device__ __forceinline__ void dft4(typename C::V* v) {
  using V = typename C::V;
  const V t0 = C::add(v[0], v[2]), t1 = C::sub(v[0], v[2]);
  const V t2 = C::add(v[1], v[3]), t3 = C::template mul_i<SG>(C::sub(v[1], v[3]));
  v[0] = C::add(t0, t2);
  v[2] = C::sub(t0, t2);
  v[1] = C::add(t1, t3);
  v[3] = C::sub(t1, t3);
}

// odd R: X_q = v0 + sum_r cos(2 pi r q / R) (v_r + v_R-r) + SG i sin(...) (v_r - v_R-r);
// the constants are entries of the length-N twiddle table (R divides N)
template <int R, int SG, class C>
__device__ __forceinline__ void dft_odd(typename C::V* v, const float4* __restrict__ tw, int n_over_r) {
  using V = typename C::V;
  constexpr int H = R / 2;
  V t[H], u[H];
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    t[r - 1] = C::add(v[r], v[R - r]);
    u[r - 1] = C::sub(v[r], v[R - r]);
  }
  V out[R];
  out[0] = v[0];
#pragma unroll
  for (int r = 0; r < H; ++r) out[0] = C::add(out[0], t[r]);
#pragma unroll
  for (int q = 1; q <= H; ++q) {
    V a = v[0], b = C::zero();
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const float4 w = __ldg(tw + ((r * q) % R) * n_over_r);
      C::mac(a, t[r - 1], w.x, w.y);
      C::mac(b, u[r - 1], w.z, w.w);
    }
    const V ib = C::template mul_i<SG>(b);
    out[q] = C::add(a, ib);
    out[R - q] = C::sub(a, ib);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = out[r];
}

template <int R, int SG, class C>
__device__ __forceinline__ void dif_pass(typename C::V* X, const DfftLen& f, int L, int mul) {
  using V = typename C::V;
  const int S = L / R;
  const int nb = f.N / R;
  const bool pow2 = (S & (S - 1)) == 0;
  const int sh = pow2 ? __ffs(S) - 1 : 0;
  // the twiddles of the thread's next butterfly are fetched one butterfly
  // ahead (they come from L2: the table does not fit in L1 next to the line)
  float4 w[R - 1];
  {
    const int t = threadIdx.x < nb ? threadIdx.x : 0;
    const int j = t - (pow2 ? (t >> sh) : t / S) * S;
#pragma unroll
    for (int q = 1; q < R; ++q) w[q - 1] = __ldg(f.tw + mul * j * q);
  }
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    const int b = pow2 ? (t >> sh) : t / S;
    const int j = t - b * S;
    const int base = b * L + j;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = X[dsw(base + r * S)];
    float4 wn[R - 1];
    {
      const int tn = t + blockDim.x < nb ? t + blockDim.x : t;
      const int jn = tn - (pow2 ? (tn >> sh) : tn / S) * S;
#pragma unroll
      for (int q = 1; q < R; ++q) wn[q - 1] = __ldg(f.tw + mul * jn * q);
    }
    if constexpr (R == 2) {
      const V a = v[0];
      v[0] = C::add(a, v[1]);
      v[1] = C::sub(a, v[1]);
    } else if constexpr (R == 4) {
      dft4<SG, C>(v);
    } else {
      dft_odd<R, SG, C>(v, f.tw, f.N / R);
    }
    // output q times W_L^(j q) = W_N^(mul j q), mul = N / L
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = C::template mul_tw<SG>(v[q], w[q - 1]);
#pragma unroll
    for (int r = 0; r < R; ++r) X[dsw(base + r * S)] = v[r];
#pragma unroll
    for (int q = 0; q < R - 1; ++q) w[q] = wn[q];
  }
}

// all passes; natural-order input in X (value i at dsw(i)), output k at X[dsw(f.rev[k])]
template <int SG, int NT, class C = CDF>
__device__ void dif_line(typename C::V* X, const DfftLen& f) {
  int L = f.N;
  for (int s = 0; s < f.npass; ++s) {
    const int R = (int)((f.code >> (4 * s)) & 15u);
    const int mul = f.N / L;
    if (R == 4) {
      dif_pass<4, SG, C>(X, f, L, mul);
    } else if (R == 2) {
      dif_pass<2, SG, C>(X, f, L, mul);
    } else if (R == 3) {
      dif_pass<3, SG, C>(X, f, L, mul);
    } else if constexpr (NT == DFFT_T_ODD) {
      if (R == 5)
        dif_pass<5, SG, C>(X, f, L, mul);
      else
        dif_pass<7, SG, C>(X, f, L, mul);
    }
    __syncthreads();
    L /= R;
  }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// complex lines of length f.N (stride ld), in place allowed; input and
// output either double2 or float pairs (INP / OUTP), 16 bytes per value
template <int SG, bool INP, bool OUTP, int NT>
__global__ void __launch_bounds__(NT) dfft_lines_k(const void* in, void* out, int64_t ld, int nlines, DfftLen f) {
  extern __shared__ float4 X[];
  for (int line = blockIdx.x; line < nlines; line += gridDim.x) {
    const int64_t o = (int64_t)line * ld;
    for (int k = threadIdx.x; k < f.N; k += blockDim.x)
      X[dsw(k)] = INP ? static_cast<const float4*>(in)[o + k] : c_of(static_cast<const double2*>(in)[o + k]);
    __syncthreads();
    dif_line<SG, NT>(X, f);
    for (int k = threadIdx.x; k < f.N; k += blockDim.x) {
      const float4 c = X[dsw(__ldg(f.rev + k))];
      if (OUTP)
        static_cast<float4*>(out)[o + k] = c;
      else
        static_cast<double2*>(out)[o + k] = c_value(c);
    }
    __syncthreads();
  }
}

// synthesis, per order m: H[k1] = Ghat[m][k mod M] d1[k] d2[m] for |k| <= lmax
// (k1 = k mod n1), zero elsewhere; inverse DFT along theta; T[m][j]
template <bool INP, int NT>
__global__ void __launch_bounds__(NT) dfft_cols_synth_k(const void* __restrict__ Gh, float4* __restrict__ T,
                                                            int lmax, int M, const float2* __restrict__ d1,
                                                            const float2* __restrict__ d2, DfftLen f,
                                                            const unsigned char* __restrict__ rowmask) {
  extern __shared__ float4 X[];
  const int m = blockIdx.x, n1 = f.N;
  const float2 dm = d2[m];
  const int64_t o = (int64_t)m * M;
  for (int k1 = threadIdx.x; k1 < n1; k1 += blockDim.x) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    int k = k1;
    bool keep = true;
    if (k1 > lmax) {
      k = k1 - n1;
      keep = k >= -lmax;
    }
    if (keep) {
      const int64_t i = o + (k < 0 ? k + M : k);
      const float4 gv = INP ? static_cast<const float4*>(Gh)[i] : c_of(static_cast<const double2*>(Gh)[i]);
      v = c_scale(gv, df_mul(d1[k + lmax], dm));
    }
    X[dsw(k1)] = v;
  }
  __syncthreads();
  dif_line<1, NT>(X, f);
  // only the rows some point reaches (the others of T stay zero)
  float4* dst = T + (int64_t)m * n1;
  for (int j = threadIdx.x; j < n1; j += blockDim.x)
    if (__ldg(rowmask + j)) dst[j] = X[dsw(__ldg(f.rev + j))];
}

// synthesis, per row pair (j, j + 1): the real rows of the fine grid
template <int NT>
__global__ void __launch_bounds__(NT) dfft_rows_c2r_k(const float4* __restrict__ T, double* __restrict__ grid,
                                                          int64_t stride, int n1, int mmax, DfftLen f,
                                                          const int* __restrict__ rowpairs) {
  extern __shared__ float4 X[];
  const int n2 = f.N;
  const int j = 2 * __ldg(rowpairs + blockIdx.x);  // a row pair some point reaches
  const bool two = j + 1 < n1;
  for (int k = mmax + 1 + threadIdx.x; k < n2 - mmax; k += blockDim.x) X[dsw(k)] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int m = threadIdx.x; m <= mmax; m += blockDim.x) {
    const float4 a = T[(int64_t)m * n1 + j];
    const float4 b = two ? T[(int64_t)m * n1 + j + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (m == 0) {
      // the imaginary parts of the m = 0 entries do not enter a real transform
      X[dsw(0)] = make_float4(a.x, a.y, b.x, b.y);
    } else {
      // C[m] = a + i b, C[n2 - m] = conj(a) + i conj(b)
      const float2 r1 = dd_add(a.x, a.y, -b.z, -b.w), i1 = dd_add(a.z, a.w, b.x, b.y);
      const float2 r2 = dd_add(a.x, a.y, b.z, b.w), i2 = dd_add(b.x, b.y, -a.z, -a.w);
      X[dsw(m)] = make_float4(r1.x, r1.y, i1.x, i1.y);
      X[dsw(n2 - m)] = make_float4(r2.x, r2.y, i2.x, i2.y);
    }
  }
  __syncthreads();
  dif_line<1, NT>(X, f);
  double* r0 = grid + (int64_t)j * stride;
  for (int n = threadIdx.x; n < n2; n += blockDim.x) {
    const float4 c = X[dsw(__ldg(f.rev + n))];
    r0[n] = pair_to_double(c.x, c.y);
    if (two) r0[stride + n] = pair_to_double(c.z, c.w);
  }
}

// adjoint, per row pair: spectra m <= mmax of rows j, j + 1 into T[m][j], T[m][j + 1]
template <int NT>
__global__ void __launch_bounds__(NT) dfft_rows_r2c_k(const double* __restrict__ grid, float4* __restrict__ T,
                                                          int64_t stride, int n1, int mmax, DfftLen f,
                                                          const int* __restrict__ rowpairs) {
  extern __shared__ float4 X[];
  const int n2 = f.N;
  const int j = 2 * __ldg(rowpairs + blockIdx.x);  // a row pair some point reaches
  const bool two = j + 1 < n1;
  const double* r0 = grid + (int64_t)j * stride;
  for (int n = threadIdx.x; n < n2; n += blockDim.x) {
    float4 v;
    split_d(r0[n], v.x, v.y);
    if (two) {
      split_d(r0[stride + n], v.z, v.w);
    } else {
      v.z = v.w = 0.f;
    }
    X[dsw(n)] = v;
  }
  __syncthreads();
  dif_line<-1, NT>(X, f);
  for (int m = threadIdx.x; m <= mmax; m += blockDim.x) {
    const float4 cm = X[dsw(__ldg(f.rev + m))];
    const float4 cn = X[dsw(__ldg(f.rev + (m == 0 ? 0 : n2 - m)))];
    // X_j = (C[m] + conj C[n2-m]) / 2, X_j+1 = -i (C[m] - conj C[n2-m]) / 2
    const float2 ar = dd_add(cm.x, cm.y, cn.x, cn.y), ai = dd_add(cm.z, cm.w, -cn.z, -cn.w);
    const float2 br = dd_add(cm.z, cm.w, cn.z, cn.w), bi = dd_add(cn.x, cn.y, -cm.x, -cm.y);
    T[(int64_t)m * n1 + j] = make_float4(0.5f * ar.x, 0.5f * ar.y, 0.5f * ai.x, 0.5f * ai.y);
    if (two) T[(int64_t)m * n1 + j + 1] = make_float4(0.5f * br.x, 0.5f * br.y, 0.5f * bi.x, 0.5f * bi.y);
  }
}

// adjoint, per order m: forward DFT of T[m][.] along theta, then
// Ghat[m][kk] = H[k mod n1] d1[k] d2[m] for |k| <= lmax (k = kk or kk - M), else 0
template <bool OUTP, int NT>
__global__ void __launch_bounds__(NT) dfft_cols_adj_k(const float4* __restrict__ T, void* __restrict__ Gh,
                                                          int lmax, int M, const float2* __restrict__ d1,
                                                          const float2* __restrict__ d2, DfftLen f,
                                                          const unsigned char* __restrict__ rowmask) {
  extern __shared__ float4 X[];
  const int m = blockIdx.x, n1 = f.N;
  const float4* src = T + (int64_t)m * n1;
  // rows no point reaches hold zero spectra: not read
  for (int k = threadIdx.x; k < n1; k += blockDim.x)
    X[dsw(k)] = __ldg(rowmask + k) ? src[k] : make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  dif_line<-1, NT>(X, f);
  const float2 dm = d2[m];
  const int64_t o = (int64_t)m * M;
  for (int kk = threadIdx.x; kk < M; kk += blockDim.x) {
    const int k = kk <= M / 2 ? kk : kk - M;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k >= -lmax && k <= lmax) {
      const float4 c = X[dsw(__ldg(f.rev + (k < 0 ? k + n1 : k)))];
      v = c_scale(c, df_mul(d1[k + lmax], dm));
    }
    if (OUTP)
      static_cast<float4*>(Gh)[o + kk] = v;
    else
      static_cast<double2*>(Gh)[o + kk] = c_value(v);
  }
}

// ---------------------------------------------------------------------------
// FP32 fine-grid transforms of mixed plans, for one plan or every member of a
// batch in one launch per pass: CTA b finds its member (the last one whose
// first CTA is <= b) and the line it owns.
//
// The FP32 line transform is its own engine (the float-pair one above is
// bound by its arithmetic, this one by shared-memory traffic): the odd
// radices 3, 5, 7 first (so that every later pass has a power-of-two
// stride), then radix-8 passes (three levels of the 2-power part each), then
// one radix-4 or radix-2 pass; twiddles from a two-level table in shared
// memory, W^k = C[k / 64] F[k % 64] (64 + N / 64 + 1 entries, 1.5 KB at
// N = 8192), three table products per radix-8 butterfly and the other four
// twiddles as products of those.  Value i of the line sits at
// i ^ ((i >> 4 ^ i >> 8 ^ i >> 12) mod 16): a permutation inside each
// aligned group of 16 that keeps contiguous and power-of-two-strided
// accesses conflict-free and spreads the digit-reversed read of the output
// over the banks (2 to 2.7 wavefronts per half-warp instead of 8).  256
// threads per CTA (four per SM) up to 8192 values, 1024 beyond.
// ---------------------------------------------------------------------------
// threads per CTA: 256 (four CTAs per SM, each barrier waits on 8 warps)
// for lines up to 8192; 1024 for longer lines, whose shared memory leaves
// room for one CTA per SM
constexpr int SFFT_T_SHORT = 256, SFFT_T_LONG = 1024, SFFT_SHORT_MAX = 8192;

__host__ __device__ __forceinline__ int spad(int i) { return i ^ (((i >> 4) ^ (i >> 8) ^ (i >> 12)) & 15); }

__device__ __forceinline__ float2 cmulf(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
template <int SG>
__device__ __forceinline__ float2 cmulif(float2 a) {  // a * (SG i)
  return SG > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// e^(SG 2 pi i k / N) from the shared-memory table (fine 0..63, coarse after)
template <int SG>
__device__ __forceinline__ float2 stw(const float2* __restrict__ T, int k) {
  const float2 w = cmulf(T[64 + (k >> 6)], T[k & 63]);
  return SG > 0 ? w : make_float2(w.x, -w.y);
}

template <int SG>
__device__ __forceinline__ void bfly4(float2* v) {
  const float2 t0 = caddf(v[0], v[2]), t1 = csubf(v[0], v[2]);
  const float2 t2 = caddf(v[1], v[3]), t3 = cmulif<SG>(csubf(v[1], v[3]));
  v[0] = caddf(t0, t2);
  v[2] = csubf(t0, t2);
  v[1] = caddf(t1, t3);
  v[3] = csubf(t1, t3);
}

// X_q = sum_r v_r e^(SG 2 pi i r q / 8): two 4-point DFTs of v_r + v_r+4 (even q)
// and (v_r - v_r+4) e^(SG 2 pi i r / 8) (odd q)
template <int SG>
__device__ __forceinline__ void bfly8(float2* v) {
  constexpr float H = 0.70710678118654752f;
  float2 a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = caddf(v[r], v[r + 4]);
    b[r] = csubf(v[r], v[r + 4]);
  }
  const float sg = (float)SG;
  b[1] = make_float2(H * (b[1].x - sg * b[1].y), H * (b[1].y + sg * b[1].x));
  b[2] = cmulif<SG>(b[2]);
  b[3] = make_float2(H * (-b[3].x - sg * b[3].y), H * (-b[3].y + sg * b[3].x));
  bfly4<SG>(a);
  bfly4<SG>(b);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[2 * q] = a[q];
    v[2 * q + 1] = b[q];
  }
}

// odd R: X_q = v0 + sum_k cos(2 pi k q / R) (v_k + v_R-k) + SG i sin(...) (v_k - v_R-k),
// cs[k - 1] = (cos, sin)(2 pi k / R), k = 1..R/2
template <int R, int SG>
__device__ __forceinline__ void bfly_odd(float2* v, const float2* cs) {
  constexpr int Hh = R / 2;
  float2 t[Hh], u[Hh], out[R];
#pragma unroll
  for (int k = 1; k <= Hh; ++k) {
    t[k - 1] = caddf(v[k], v[R - k]);
    u[k - 1] = csubf(v[k], v[R - k]);
  }
  out[0] = v[0];
#pragma unroll
  for (int k = 0; k < Hh; ++k) out[0] = caddf(out[0], t[k]);
#pragma unroll
  for (int q = 1; q <= Hh; ++q) {
    float2 a = v[0], b = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 1; k <= Hh; ++k) {
      const int m = (k * q) % R;
      const float c = cs[(m <= Hh ? m : R - m) - 1].x;
      const float sn = m <= Hh ? cs[m - 1].y : -cs[R - m - 1].y;
      a = make_float2(fmaf(c, t[k - 1].x, a.x), fmaf(c, t[k - 1].y, a.y));
      b = make_float2(fmaf(sn, u[k - 1].x, b.x), fmaf(sn, u[k - 1].y, b.y));
    }
    const float2 ib = cmulif<SG>(b);
    out[q] = caddf(a, ib);
    out[R - q] = csubf(a, ib);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = out[r];
}

// one in-place decimation-in-frequency pass of radix R over sub-blocks of
// length L: butterfly (b, j) combines b L + j + r (L / R), output q times
// W_L^(j q) = W_N^(j q N / L)
template <int R, int SG>
__device__ __forceinline__ void spass(float2* X, const float2* __restrict__ T, int N, int L) {
  const int S = L / R, nb = N / R, mul = N / L;
  const bool pow2 = (S & (S - 1)) == 0;
  const int sh = __ffs(S) - 1;
  float2 cs[R / 2 > 0 ? R / 2 : 1];
  if constexpr (R == 3 || R == 5 || R == 7) {
#pragma unroll
    for (int k = 1; k <= R / 2; ++k) cs[k - 1] = stw<1>(T, k * (N / R));
  }
  for (int t = threadIdx.x; t < nb; t += (int)blockDim.x) {
    const int b = pow2 ? t >> sh : t / S;
    const int j = t - b * S;
    const int base = b * L + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = X[spad(base + r * S)];
    if constexpr (R == 2) {
      const float2 a = v[0];
      v[0] = caddf(a, v[1]);
      v[1] = csubf(a, v[1]);
    } else if constexpr (R == 4) {
      bfly4<SG>(v);
    } else if constexpr (R == 8) {
      bfly8<SG>(v);
    } else {
      bfly_odd<R, SG>(v, cs);
    }
    if (j != 0) {
      const int k = mul * j;
      const float2 w1 = stw<SG>(T, k);
      v[1] = cmulf(v[1], w1);
      if constexpr (R >= 3) {
        const float2 w2 = stw<SG>(T, 2 * k);
        v[2] = cmulf(v[2], w2);
        if constexpr (R >= 4) {
          const float2 w3 = cmulf(w1, w2);
          v[3] = cmulf(v[3], w3);
          if constexpr (R >= 5) {
            const float2 w4 = stw<SG>(T, 4 * k);
            v[4] = cmulf(v[4], w4);
            if constexpr (R >= 7) {
              v[5] = cmulf(v[5], cmulf(w1, w4));
              v[6] = cmulf(v[6], cmulf(w2, w4));
              if constexpr (R == 8) v[7] = cmulf(v[7], cmulf(w3, w4));
            }
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) X[spad(base + r * S)] = v[r];
  }
}

// the whole line: natural-order input in X (padded), output k at X[spad(rev[k])]
template <int SG>
__device__ void sline(float2* X, const float2* __restrict__ T, const DfftLen& f) {
  int L = f.N;
  for (int s = 0; s < f.npass; ++s) {
    const int R = (int)((f.code >> (4 * s)) & 15u);
    if (R == 8)
      spass<8, SG>(X, T, f.N, L);
    else if (R == 4)
      spass<4, SG>(X, T, f.N, L);
    else if (R == 2)
      spass<2, SG>(X, T, f.N, L);
    else if (R == 3)
      spass<3, SG>(X, T, f.N, L);
    else if (R == 5)
      spass<5, SG>(X, T, f.N, L);
    else
      spass<7, SG>(X, T, f.N, L);
    __syncthreads();
    L /= R;
  }
}

// shared memory of a CTA: the padded line, then the twiddle table
__host__ __device__ __forceinline__ int sline_words(int n) { return (n + 15) & ~15; }
__host__ __device__ __forceinline__ int stw_words(int n) { return 64 + n / 64 + 1; }

__device__ __forceinline__ float2* stw_load(float2* Xs, int maxn, const DfftLen& f) {
  float2* T = Xs + sline_words(maxn);
  const int nt = stw_words(f.N);
  for (int k = threadIdx.x; k < nt; k += (int)blockDim.x) T[k] = __ldg(f.tw2 + k);
  return T;
}

__device__ __forceinline__ int member_of(const SfftMember* __restrict__ mem, int nm, int b, bool rows) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((rows ? mem[mid].row0 : mem[mid].col0) <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// synthesis, per (member, order m): deconvolve and zero-pad the theta
// spectrum to n1, inverse DFT along theta, store T[m][.]
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) sfft_cols_synth_k(const SfftMember* __restrict__ mem, int nm, int maxn) {
  extern __shared__ float2 Xs[];
  const SfftMember& q = mem[member_of(mem, nm, blockIdx.x, false)];
  const float2* T = stw_load(Xs, maxn, q.f1);
  const int m = blockIdx.x - q.col0;
  const int n1 = q.n1, lmax = q.lmax, M = q.M;
  const float dm = q.d2[m];
  const float2* g = q.Gh + (int64_t)m * M;
  for (int k1 = threadIdx.x; k1 < n1; k1 += (int)blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    const int k = k1 > lmax ? k1 - n1 : k1;
    if (k >= -lmax) {
      const float2 gv = g[k < 0 ? k + M : k];
      const float d = q.d1[k + lmax] * dm;
      v = make_float2(gv.x * d, gv.y * d);
    }
    Xs[spad(k1)] = v;
  }
  __syncthreads();
  sline<1>(Xs, T, q.f1);
  // only the rows some point reaches (the others of T stay zero)
  float2* dst = q.T + (int64_t)m * n1;
  for (int j = threadIdx.x; j < n1; j += (int)blockDim.x)
    if (__ldg(q.rowmask + j)) dst[j] = Xs[spad(__ldg(q.f1.rev + j))];
}

// synthesis, per (member, row pair j, j + 1): the two Hermitian half spectra
// packed as C = X_j + i X_j+1, one inverse DFT, x_j = Re, x_j+1 = Im
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) sfft_rows_c2r_k(const SfftMember* __restrict__ mem, int nm, int maxn) {
  extern __shared__ float2 Xs[];
  const SfftMember& q = mem[member_of(mem, nm, blockIdx.x, true)];
  const float2* T = stw_load(Xs, maxn, q.f2);
  const int j = 2 * __ldg(q.rowpairs + (blockIdx.x - q.row0));  // a row pair some point reaches
  const int n1 = q.n1, n2 = q.n2, mmax = q.mmax;
  const bool two = j + 1 < n1;
  for (int k = mmax + 1 + threadIdx.x; k < n2 - mmax; k += (int)blockDim.x) Xs[spad(k)] = make_float2(0.f, 0.f);
  // the column pair of T: strided loads, four per thread in flight; with n1
  // even (the fine-grid sizes are) T[m][j], T[m][j+1] are one aligned 16-byte load
  const bool vec = (n1 & 1) == 0;
  for (int m0 = threadIdx.x; m0 <= mmax; m0 += 4 * (int)blockDim.x) {
    float2 a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int m = m0 + u * (int)blockDim.x;
      a[u] = b[u] = make_float2(0.f, 0.f);
      if (m <= mmax) {
        const float2* t = q.T + (int64_t)m * n1 + j;
        if (vec) {
          const float4 ab = __ldg(reinterpret_cast<const float4*>(t));
          a[u] = make_float2(ab.x, ab.y);
          b[u] = make_float2(ab.z, ab.w);
        } else {
          a[u] = __ldg(t);
          if (two) b[u] = __ldg(t + 1);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int m = m0 + u * (int)blockDim.x;
      if (m > mmax) break;
      if (m == 0) {
        Xs[spad(0)] = make_float2(a[u].x, b[u].x);  // a real transform takes only Re of m = 0
      } else {
        Xs[spad(m)] = make_float2(a[u].x - b[u].y, a[u].y + b[u].x);
        Xs[spad(n2 - m)] = make_float2(a[u].x + b[u].y, b[u].x - a[u].y);
      }
    }
  }
  __syncthreads();
  sline<1>(Xs, T, q.f2);
  float* r0 = q.grid + (int64_t)j * q.stride;
  for (int n = threadIdx.x; n < n2; n += (int)blockDim.x) {
    const float2 c = Xs[spad(__ldg(q.f2.rev + n))];
    r0[n] = c.x;
    if (two) r0[q.stride + n] = c.y;
  }
}

// adjoint, per (member, row pair): spectra m <= mmax of rows j, j + 1 into T
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) sfft_rows_r2c_k(const SfftMember* __restrict__ mem, int nm, int maxn) {
  extern __shared__ float2 Xs[];
  const SfftMember& q = mem[member_of(mem, nm, blockIdx.x, true)];
  const float2* T = stw_load(Xs, maxn, q.f2);
  const int j = 2 * __ldg(q.rowpairs + (blockIdx.x - q.row0));  // a row pair some point reaches
  const int n1 = q.n1, n2 = q.n2, mmax = q.mmax;
  const bool two = j + 1 < n1;
  const float* r0 = q.grid + (int64_t)j * q.stride;
  for (int n = threadIdx.x; n < n2; n += (int)blockDim.x) Xs[spad(n)] = make_float2(r0[n], two ? r0[q.stride + n] : 0.f);
  __syncthreads();
  sline<-1>(Xs, T, q.f2);
  for (int m = threadIdx.x; m <= mmax; m += (int)blockDim.x) {
    const float2 cm = Xs[spad(__ldg(q.f2.rev + m))];
    const float2 cn = Xs[spad(__ldg(q.f2.rev + (m == 0 ? 0 : n2 - m)))];
    // X_j = (C[m] + conj C[n2-m]) / 2, X_j+1 = -i (C[m] - conj C[n2-m]) / 2
    const float2 xa = make_float2(0.5f * (cm.x + cn.x), 0.5f * (cm.y - cn.y));
    const float2 xb = make_float2(0.5f * (cm.y + cn.y), 0.5f * (cn.x - cm.x));
    float2* t = q.T + (int64_t)m * n1 + j;
    if ((n1 & 1) == 0) {
      *reinterpret_cast<float4*>(t) = make_float4(xa.x, xa.y, xb.x, xb.y);  // aligned: n1 and j even
    } else {
      t[0] = xa;
      if (two) t[1] = xb;
    }
  }
}

// adjoint, per (member, order m): forward DFT of T[m][.] along theta, then
// Gh[m][kk] = H[k mod n1] d1[k] d2[m] for |k| <= lmax (k = kk or kk - M), else 0
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) sfft_cols_adj_k(const SfftMember* __restrict__ mem, int nm, int maxn) {
  extern __shared__ float2 Xs[];
  const SfftMember& q = mem[member_of(mem, nm, blockIdx.x, false)];
  const float2* T = stw_load(Xs, maxn, q.f1);
  const int m = blockIdx.x - q.col0;
  const int n1 = q.n1, lmax = q.lmax, M = q.M;
  const float2* src = q.T + (int64_t)m * n1;
  // rows no point reaches hold zero spectra: not read
  for (int k = threadIdx.x; k < n1; k += (int)blockDim.x) Xs[spad(k)] = __ldg(q.rowmask + k) ? src[k] : make_float2(0.f, 0.f);
  __syncthreads();
  sline<-1>(Xs, T, q.f1);
  const float dm = q.d2[m];
  float2* g = const_cast<float2*>(q.Gh) + (int64_t)m * M;
  for (int kk = threadIdx.x; kk < M; kk += (int)blockDim.x) {
    const int k = kk <= M / 2 ? kk : kk - M;
    float2 v = make_float2(0.f, 0.f);
    if (k >= -lmax && k <= lmax) {
      const float2 c = Xs[spad(__ldg(q.f1.rev + (k < 0 ? k + n1 : k)))];
      const float d = q.d1[k + lmax] * dm;
      v = make_float2(c.x * d, c.y * d);
    }
    g[kk] = v;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool factor(int n, DfftLen& f) {
  std::vector<int> r;
  for (int p : {7, 5, 3}) {
    while (n % p == 0) {
      r.push_back(p);
      n /= p;
    }
  }
  if (n % 2 == 0 && (n & (n - 1)) == 0) {
    int e = 0;
    while ((1 << e) < n) ++e;
    if (e % 2) r.push_back(2);
    for (int i = 0; i < e / 2; ++i) r.push_back(4);
    n = 1;
  }
  if (n != 1 || (int)r.size() > DFFT_MAXPASS) return false;
  f.npass = (int)r.size();
  f.code = 0;
  for (int i = 0; i < f.npass; ++i) f.code |= (unsigned long long)r[i] << (4 * i);
  return true;
}

// FP32 engine: the odd radices, then radix 8 while three factors of 2
// remain, then one 4 or 2
bool factor8(int n, DfftLen& f) {
  std::vector<int> r;
  for (int p : {7, 5, 3}) {
    while (n % p == 0) {
      r.push_back(p);
      n /= p;
    }
  }
  if ((n & (n - 1)) != 0) return false;
  int e = 0;
  while ((1 << e) < n) ++e;
  for (int i = 0; i < e / 3; ++i) r.push_back(8);
  if (e % 3 == 2) r.push_back(4);
  if (e % 3 == 1) r.push_back(2);
  if (r.empty() || (int)r.size() > DFFT_MAXPASS) return false;
  f.npass = (int)r.size();
  f.code = 0;
  for (int i = 0; i < f.npass; ++i) f.code |= (unsigned long long)r[i] << (4 * i);
  return true;
}

// digit-reversal table of a factorisation: output k = k_1 + R_1 (k_2 + R_2 (...))
// sits at sum_s k_s N / (R_1 ... R_s)
std::vector<int> rev_of(int N, const DfftLen& f) {
  std::vector<int> rev(N);
  for (int k = 0; k < N; ++k) {
    int kk = k, pos = 0, L = N;
    for (int s = 0; s < f.npass; ++s) {
      const int R = (int)((f.code >> (4 * s)) & 15u);
      const int d = kk % R;
      kk /= R;
      L /= R;
      pos += d * L;
    }
    rev[k] = pos;
  }
  return rev;
}

// FP32 line of length N: factorisation, digit reversal and the two-level
// twiddle table (F[k] = e^(2 pi i k / N), k < 64; C[c] = e^(2 pi i 64 c / N))
int make_len_s(int N, DfftLen& f, size_t* bytes) {
  f.N = N;
  if (!factor8(N, f)) return set_error(NUSHT_EUNSUPPORTED, "FP32 FFT: length has a prime factor above 7");
  const int nt = 64 + N / 64 + 1;
  std::vector<float2> tw(nt);
  for (int k = 0; k < nt; ++k) {
    const double a = 2.0 * M_PI * (double)(k < 64 ? k : 64 * (k - 64)) / (double)N;
    tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  const std::vector<int> rev = rev_of(N, f);
  NUSHT_TRY(dev_alloc((void**)&f.tw2, (size_t)nt * sizeof(float2), bytes));
  NUSHT_TRY(dev_alloc((void**)&f.rev, (size_t)N * sizeof(int), bytes));
  NUSHT_CUDA(cudaMemcpy(f.tw2, tw.data(), (size_t)nt * sizeof(float2), cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(f.rev, rev.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice));
  return NUSHT_OK;
}

int make_len(int N, DfftLen& f, size_t* bytes) {
  f.N = N;
  if (!factor(N, f)) return set_error(NUSHT_EUNSUPPORTED, "double-float FFT: length has a prime factor above 7");
  std::vector<float4> tw(N);
  for (int k = 0; k < N; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)N;
    const double c = std::cos(a), s = std::sin(a);
    const float ch = (float)c, sh = (float)s;
    tw[k] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
  }
  const std::vector<int> rev = rev_of(N, f);
  NUSHT_TRY(dev_alloc((void**)&f.tw, (size_t)N * sizeof(float4), bytes));
  NUSHT_TRY(dev_alloc((void**)&f.rev, (size_t)N * sizeof(int), bytes));
  NUSHT_CUDA(cudaMemcpy(f.tw, tw.data(), (size_t)N * sizeof(float4), cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(f.rev, rev.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice));
  return NUSHT_OK;
}

template <int NT>
int optin_all(int b) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_lines_k<-1, false, false, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_lines_k<-1, false, true, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_lines_k<1, false, false, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_lines_k<1, true, false, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_lines_k<-1, true, true, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_lines_k<1, true, true, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_cols_synth_k<false, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_cols_synth_k<true, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_rows_c2r_k<NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_rows_r2c_k<NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_cols_adj_k<false, NT>, a, b));
  NUSHT_CUDA(cudaFuncSetAttribute(dfft_cols_adj_k<true, NT>, a, b));
  return NUSHT_OK;
}

// whether every pass of f has radix 2, 3 or 4 (the 1024-thread kernels)
bool wide(const DfftLen& f) {
  for (int i = 0; i < f.npass; ++i) {
    const int R = (int)((f.code >> (4 * i)) & 15u);
    if (R == 5 || R == 7) return false;
  }
  return true;
}

int smem_optin() {
  static int done = 0;
  if (done) return NUSHT_OK;
  const int b = DFFT_NMAX * (int)sizeof(float4);
  NUSHT_TRY(optin_all<DFFT_T_WIDE>(b));
  NUSHT_TRY(optin_all<DFFT_T_ODD>(b));
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int bs = SFFT_SMEM_MAX;
  NUSHT_CUDA(cudaFuncSetAttribute(sfft_cols_synth_k<SFFT_T_SHORT>, a, bs));
  NUSHT_CUDA(cudaFuncSetAttribute(sfft_rows_c2r_k<SFFT_T_SHORT>, a, bs));
  NUSHT_CUDA(cudaFuncSetAttribute(sfft_rows_r2c_k<SFFT_T_SHORT>, a, bs));
  NUSHT_CUDA(cudaFuncSetAttribute(sfft_cols_adj_k<SFFT_T_SHORT>, a, bs));
  NUSHT_CUDA(cudaFuncSetAttribute(sfft_cols_synth_k<SFFT_T_LONG>, a, bs));
  NUSHT_CUDA(cudaFuncSetAttribute(sfft_rows_c2r_k<SFFT_T_LONG>, a, bs));
  NUSHT_CUDA(cudaFuncSetAttribute(sfft_rows_r2c_k<SFFT_T_LONG>, a, bs));
  NUSHT_CUDA(cudaFuncSetAttribute(sfft_cols_adj_k<SFFT_T_LONG>, a, bs));
  done = 1;
  return NUSHT_OK;
}

std::vector<float2> pairs_of(const std::vector<double>& v) {
  std::vector<float2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const float h = (float)v[i];
    o[i] = make_float2(h, (float)(v[i] - (double)h));
  }
  return o;
}

}  // namespace

bool dfft_fits(const nusht_sizes& z, bool theta, bool fine) {
  auto ok = [](int n) {
    DfftLen f;
    return n >= 2 && n <= DFFT_NMAX && factor(n, f);
  };
  if (theta && !ok(z.M)) return false;
  if (fine && (!ok(z.n1) || !ok(z.n2) || z.n2 % 2 || z.n1 <= 2 * z.lmax || 2 * z.mmax >= z.n2)) return false;
  return true;
}

int dfft_setup(nusht_plan_t p, bool theta, bool fine, const double* d1, const double* d2) {
  const nusht_sizes& z = p->sz;
  NUSHT_TRY(smem_optin());
  if (theta) {
    NUSHT_TRY(make_len(z.M, p->dft_theta, &p->bytes));
    p->dfft_theta = true;
  }
  if (fine) {
    NUSHT_TRY(make_len(z.n1, p->dft_n1, &p->bytes));
    NUSHT_TRY(make_len(z.n2, p->dft_n2, &p->bytes));
    NUSHT_TRY(dev_alloc(&p->tcols, (size_t)(z.mmax + 1) * z.n1 * sizeof(float4), &p->bytes));
    const std::vector<double> v1(d1, d1 + 2 * z.lmax + 1), v2(d2, d2 + z.mmax + 1);
    const std::vector<float2> f1 = pairs_of(v1), f2 = pairs_of(v2);
    NUSHT_TRY(dev_alloc((void**)&p->deconv1f, f1.size() * sizeof(float2), &p->bytes));
    NUSHT_TRY(dev_alloc((void**)&p->deconv2f, f2.size() * sizeof(float2), &p->bytes));
    NUSHT_CUDA(cudaMemcpy(p->deconv1f, f1.data(), f1.size() * sizeof(float2), cudaMemcpyHostToDevice));
    NUSHT_CUDA(cudaMemcpy(p->deconv2f, f2.data(), f2.size() * sizeof(float2), cudaMemcpyHostToDevice));
    p->dfft_fine = true;
  }
  return NUSHT_OK;
}

void dfft_free(nusht_plan_t p) {
  for (DfftLen* f : {&p->dft_theta, &p->dft_n1, &p->dft_n2}) {
    dev_free(f->tw);
    dev_free(f->tw2);
    dev_free(f->rev);
    f->tw = nullptr;
    f->tw2 = nullptr;
    f->rev = nullptr;
  }
  dev_free(p->tcols);
  dev_free(p->deconv1f);
  dev_free(p->deconv2f);
  dev_free(p->deconv1s);
  dev_free(p->deconv2s);
  dev_free(p->sfft_mem);
  p->tcols = nullptr;
  p->deconv1f = p->deconv2f = nullptr;
  p->deconv1s = p->deconv2s = nullptr;
  p->sfft_mem = nullptr;
  p->dfft_theta = p->dfft_fine = p->sfft_fine = false;
}

// With both the theta and the fine-grid transforms here, the theta spectrum
// passes between them as float pairs: synthesis writes Ghat as pairs for the
// column pass, the adjoint's column pass writes pairs for the inverse theta
// DFT; the ring map G and the adjoint's final Ghat stay double2.
int dfft_theta_exec(nusht_plan_t p, const void* src, void* dst, int sign, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const size_t sm = (size_t)dline_words(z.M) * sizeof(float4);
  const int nl = z.mmax + 1;
  const DfftLen& f = p->dft_theta;
  auto go = [&](auto kw, auto ko) {
    if (wide(f))
      kw<<<nl, DFFT_T_WIDE, sm, s>>>(src, dst, z.M, nl, f);
    else
      ko<<<nl, DFFT_T_ODD, sm, s>>>(src, dst, z.M, nl, f);
  };
  if (sign < 0) {
    if (p->dfft_fine)
      go(dfft_lines_k<-1, false, true, DFFT_T_WIDE>, dfft_lines_k<-1, false, true, DFFT_T_ODD>);
    else
      go(dfft_lines_k<-1, false, false, DFFT_T_WIDE>, dfft_lines_k<-1, false, false, DFFT_T_ODD>);
  } else {
    if (p->dfft_fine)
      go(dfft_lines_k<1, true, false, DFFT_T_WIDE>, dfft_lines_k<1, true, false, DFFT_T_ODD>);
    else
      go(dfft_lines_k<1, false, false, DFFT_T_WIDE>, dfft_lines_k<1, false, false, DFFT_T_ODD>);
  }
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int dfft_theta_pairs(nusht_plan_t p, const void* src, void* dst, int sign, cudaStream_t s) {
  if (!p->dfft_theta || !p->dfft_fine) return set_error(NUSHT_EUNSUPPORTED, "theta DFT on pairs needs both kernels");
  const nusht_sizes& z = p->sz;
  const size_t sm = (size_t)dline_words(z.M) * sizeof(float4);
  const int nl = z.mmax + 1;
  const DfftLen& f = p->dft_theta;
  auto go = [&](auto kw, auto ko) {
    if (wide(f))
      kw<<<nl, DFFT_T_WIDE, sm, s>>>(src, dst, z.M, nl, f);
    else
      ko<<<nl, DFFT_T_ODD, sm, s>>>(src, dst, z.M, nl, f);
  };
  if (sign < 0)
    go(dfft_lines_k<-1, true, true, DFFT_T_WIDE>, dfft_lines_k<-1, true, true, DFFT_T_ODD>);
  else
    go(dfft_lines_k<1, true, true, DFFT_T_WIDE>, dfft_lines_k<1, true, true, DFFT_T_ODD>);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int dfft_cols_synth(nusht_plan_t p, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const size_t sm = (size_t)dline_words(z.n1) * sizeof(float4);
  const DfftLen& f = p->dft_n1;
  auto go = [&](auto kw, auto ko) {
    if (wide(f))
      kw<<<z.mmax + 1, DFFT_T_WIDE, sm, s>>>(p->Ghat, (float4*)p->tcols, z.lmax, z.M, p->deconv1f, p->deconv2f, f,
                                             p->pts.rowmask);
    else
      ko<<<z.mmax + 1, DFFT_T_ODD, sm, s>>>(p->Ghat, (float4*)p->tcols, z.lmax, z.M, p->deconv1f, p->deconv2f, f,
                                            p->pts.rowmask);
  };
  if (p->dfft_theta)
    go(dfft_cols_synth_k<true, DFFT_T_WIDE>, dfft_cols_synth_k<true, DFFT_T_ODD>);
  else
    go(dfft_cols_synth_k<false, DFFT_T_WIDE>, dfft_cols_synth_k<false, DFFT_T_ODD>);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int dfft_rows_c2r(nusht_plan_t p, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const int64_t stride = 2 * (z.n2 / 2 + 1);
  const size_t sm = (size_t)dline_words(z.n2) * sizeof(float4);
  const DfftLen& f = p->dft_n2;
  const int np = p->pts.nrowpairs;  // only the row pairs some point reaches
  if (np == 0) return NUSHT_OK;
  if (wide(f))
    dfft_rows_c2r_k<DFFT_T_WIDE><<<np, DFFT_T_WIDE, sm, s>>>((const float4*)p->tcols, (double*)p->fine, stride, z.n1,
                                                            z.mmax, f, p->pts.rowpairs);
  else
    dfft_rows_c2r_k<DFFT_T_ODD><<<np, DFFT_T_ODD, sm, s>>>((const float4*)p->tcols, (double*)p->fine, stride, z.n1,
                                                          z.mmax, f, p->pts.rowpairs);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int dfft_rows_r2c(nusht_plan_t p, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const int64_t stride = 2 * (z.n2 / 2 + 1);
  const size_t sm = (size_t)dline_words(z.n2) * sizeof(float4);
  const DfftLen& f = p->dft_n2;
  const int np = p->pts.nrowpairs;  // rows no point reaches stay zero: their spectra in T are zero
  if (np == 0) return NUSHT_OK;
  if (wide(f))
    dfft_rows_r2c_k<DFFT_T_WIDE><<<np, DFFT_T_WIDE, sm, s>>>((const double*)p->fine, (float4*)p->tcols, stride,
                                                            z.n1, z.mmax, f, p->pts.rowpairs);
  else
    dfft_rows_r2c_k<DFFT_T_ODD><<<np, DFFT_T_ODD, sm, s>>>((const double*)p->fine, (float4*)p->tcols, stride, z.n1,
                                                          z.mmax, f, p->pts.rowpairs);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int dfft_cols_adjoint(nusht_plan_t p, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const size_t sm = (size_t)dline_words(z.n1) * sizeof(float4);
  const DfftLen& f = p->dft_n1;
  auto go = [&](auto kw, auto ko) {
    if (wide(f))
      kw<<<z.mmax + 1, DFFT_T_WIDE, sm, s>>>((const float4*)p->tcols, p->Ghat, z.lmax, z.M, p->deconv1f,
                                             p->deconv2f, f, p->pts.rowmask);
    else
      ko<<<z.mmax + 1, DFFT_T_ODD, sm, s>>>((const float4*)p->tcols, p->Ghat, z.lmax, z.M, p->deconv1f,
                                            p->deconv2f, f, p->pts.rowmask);
  };
  if (p->dfft_theta)
    go(dfft_cols_adj_k<true, DFFT_T_WIDE>, dfft_cols_adj_k<true, DFFT_T_ODD>);
  else
    go(dfft_cols_adj_k<false, DFFT_T_WIDE>, dfft_cols_adj_k<false, DFFT_T_ODD>);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

bool sfft_fits(const nusht_sizes& z) {
  auto ok = [](int n) {
    DfftLen f;
    return n >= 8 && n <= SFFT_NMAX && factor8(n, f) && sfft_smem(n) <= SFFT_SMEM_MAX;
  };
  return ok(z.n1) && ok(z.n2) && z.n2 % 2 == 0 && z.n1 > 2 * z.lmax && 2 * z.mmax < z.n2;
}

int sfft_setup(nusht_plan_t p, const double* d1, const double* d2) {
  const nusht_sizes& z = p->sz;
  NUSHT_TRY(smem_optin());
  NUSHT_TRY(make_len_s(z.n1, p->dft_n1, &p->bytes));
  NUSHT_TRY(make_len_s(z.n2, p->dft_n2, &p->bytes));
  NUSHT_TRY(dev_alloc(&p->tcols, (size_t)(z.mmax + 1) * z.n1 * sizeof(float2), &p->bytes));
  std::vector<float> f1(2 * z.lmax + 1), f2(z.mmax + 1);
  for (size_t i = 0; i < f1.size(); ++i) f1[i] = (float)d1[i];
  for (size_t i = 0; i < f2.size(); ++i) f2[i] = (float)d2[i];
  NUSHT_TRY(dev_alloc((void**)&p->deconv1s, f1.size() * sizeof(float), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&p->deconv2s, f2.size() * sizeof(float), &p->bytes));
  NUSHT_CUDA(cudaMemcpy(p->deconv1s, f1.data(), f1.size() * sizeof(float), cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(p->deconv2s, f2.data(), f2.size() * sizeof(float), cudaMemcpyHostToDevice));
  p->sfft_fine = true;
  SfftMember m;
  sfft_member(p, m);
  NUSHT_TRY(dev_alloc((void**)&p->sfft_mem, sizeof(SfftMember), &p->bytes));
  NUSHT_CUDA(cudaMemcpy(p->sfft_mem, &m, sizeof(SfftMember), cudaMemcpyHostToDevice));
  return NUSHT_OK;
}

void sfft_member(nusht_plan_t p, SfftMember& m) {
  const nusht_sizes& z = p->sz;
  m.Gh = static_cast<float2*>(p->Ghat);
  m.T = static_cast<float2*>(p->tcols);
  m.grid = static_cast<float*>(p->fine);
  m.d1 = p->deconv1s;
  m.d2 = p->deconv2s;
  m.stride = 2 * (z.n2 / 2 + 1);
  m.lmax = z.lmax;
  m.mmax = z.mmax;
  m.M = z.M;
  m.n1 = z.n1;
  m.n2 = z.n2;
  m.col0 = m.row0 = 0;
  m.f1 = p->dft_n1;
  m.f2 = p->dft_n2;
  m.rowpairs = p->pts.rowpairs;
  m.rowmask = p->pts.rowmask;
}

SfftLaunch sfft_launch_of(nusht_plan_t p) {
  SfftLaunch l;
  l.mem = p->sfft_mem;
  l.nm = 1;
  l.ncols = p->sz.mmax + 1;
  l.nrows = p->pts.nrowpairs;
  l.maxn1 = p->sz.n1;
  l.maxn2 = p->sz.n2;
  return l;
}

int sfft_smem(int n) { return (sline_words(n) + stw_words(n)) * (int)sizeof(float2); }

#define NUSHT_SFFT_LAUNCH(KERNEL, NCTA, NMAXLEN)                                                       \
  do {                                                                                                 \
    if ((NCTA) <= 0) return NUSHT_OK;                                                                  \
    if ((NMAXLEN) <= SFFT_SHORT_MAX)                                                                   \
      KERNEL<SFFT_T_SHORT><<<(NCTA), SFFT_T_SHORT, (size_t)sfft_smem(NMAXLEN), s>>>(l.mem, l.nm, (NMAXLEN)); \
    else                                                                                               \
      KERNEL<SFFT_T_LONG><<<(NCTA), SFFT_T_LONG, (size_t)sfft_smem(NMAXLEN), s>>>(l.mem, l.nm, (NMAXLEN));   \
    NUSHT_CUDA(cudaGetLastError());                                                                    \
    return NUSHT_OK;                                                                                   \
  } while (0)

int sfft_cols_synth(const SfftLaunch& l, cudaStream_t s) { NUSHT_SFFT_LAUNCH(sfft_cols_synth_k, l.ncols, l.maxn1); }
int sfft_rows_c2r(const SfftLaunch& l, cudaStream_t s) { NUSHT_SFFT_LAUNCH(sfft_rows_c2r_k, l.nrows, l.maxn2); }
int sfft_rows_r2c(const SfftLaunch& l, cudaStream_t s) { NUSHT_SFFT_LAUNCH(sfft_rows_r2c_k, l.nrows, l.maxn2); }
int sfft_cols_adjoint(const SfftLaunch& l, cudaStream_t s) { NUSHT_SFFT_LAUNCH(sfft_cols_adj_k, l.ncols, l.maxn1); }

}  // namespace nusht
