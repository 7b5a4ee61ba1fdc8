// legendre.cu -- the iso-latitude step S and its adjoint S^dagger (Sec. 2.2,
// Sec. 3) on Clenshaw-Curtis rings, with the doubling D fused into the
// synthesis store and the fold D^dagger fused into the adjoint load.
//
// Recurrence.  For a fixed order m the orthonormal functions obey
//   Pbar_l = alpha_l x Pbar_{l-1} - alpha_l b_l Pbar_{l-2},  x = cos(theta),
//   alpha_l^2 = (4l^2-1)/(l^2-m^2),  b_l^2 = ((l-1)^2-m^2)/(4(l-1)^2-1).
// Writing Pbar_l = Ahat_l q_l with Ahat_l = 2^-sigma_l prod_{k=m+1}^{l} alpha_k
// (a theta-independent table) turns it into
//   q_l = x q_{l-1} - c_l q_{l-2},  c_l = b_l / alpha_{l-1}
//       = (l-1-m)(l-1+m) / ((2l-3)(2l-1))            (a rational number),
// two FP64 operations per step instead of three; Ahat_l is folded into the
// coefficients once per call (atilde = a Ahat).  sigma_l grows by
// LEG_SEG_BITS whenever Ahat would leave [1, 2^48); those steps first scale
// (q_{l-1}, q_{l-2}) by 2^LEG_SEG_BITS (table dshift).  The start value is
// Pbar_mm = c_m sin^m(theta), with sin^m by binary powering and an integer
// exponent.  While the value is below 2^-300 it is carried with a separate
// exponent E (the scaled-exponent phase; checks are integer operations) and
// not accumulated; ring blocks of an order whose every ring stays below that
// threshold up to lmax are dropped from the work list at plan time.
//
// Parallel layout: one warp per work item (order m, block of 128 ring pairs),
// four ring pairs (theta_j, pi - theta_j) per lane that share the recurrence
// through Pbar_l(pi - theta) = (-1)^(l+m) Pbar_l(theta).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "nusht_internal.cuh"
#include "recurrence.cuh"
#include "dfloat.cuh"

namespace nusht {

namespace {

using namespace rec;
constexpr unsigned FULL = 0xffffffffu;

struct LegArgs {
  int lmax, mmax, M, npairs, bpm;
  const int* items;
  const double* c;
  const float2* cdf;
  const int8_t* dshift;
  const double* cm;
  const double* ring_x;
  const double* ring_s;
};

// the recurrence value in the contraction's type: float (mixed) or a float
// pair split off the double (FP64 chain) / taken as is (double-float chain)
template <typename T>
__device__ __forceinline__ T qconv(const Chain& ch) {
  return conv<T>(ch.q1);
}
template <typename T>
__device__ __forceinline__ T qconv(const DfChain& ch) {
  return (T)ch.q1.x;
}

__device__ __forceinline__ void item_of(const LegArgs& a, int it, int& m, int& blk) {
  int v = __ldg(a.items + it);
  m = v >> 16;
  blk = v & 0xffff;
}

// ---------------------------------------------------------------------------
// synthesis: G[m][*] (doubled, theta-contiguous) from atilde
// ---------------------------------------------------------------------------
template <typename T, class CH = Chain>
__global__ void __launch_bounds__(128) legendre_synth_k(LegArgs a, const typename V2<T>::t* __restrict__ at,
                                                        typename V2<T>::t* __restrict__ G, int nitems) {
  using T2 = typename V2<T>::t;
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  int m, blk;
  item_of(a, it, m, blk);
  const int L = a.lmax;
  const int mb = mbase_of(L, m);
  CH ch[LEG_K];
  T2 accE[LEG_K], accO[LEG_K];
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) {
    chain_init(ch[k], a, m, 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane);
    accE[k].x = accE[k].y = accO[k].x = accO[k].y = (T)0;
  }
  // l = m (even parity)
  {
    T2 av = at[mb + m];
#pragma unroll
    for (int k = 0; k < LEG_K; ++k)
      if (ch[k].E == 0) {
        T q = qconv<T>(ch[k]);
        accE[k].x = fma(av.x, q, accE[k].x);
        accE[k].y = fma(av.y, q, accE[k].y);
      }
  }
  // degrees in pairs (l - m odd, l - m even) so that the parity is static
  int l = m + 1;
  for (; l + 1 <= L; l += 2) {
    {
      const auto c = coef(a, mb + l, ch[0]);
      const int rs = __ldg(a.dshift + mb + l);
      const T2 av = at[mb + l];
#pragma unroll
      for (int k = 0; k < LEG_K; ++k) {
        chain_step(ch[k], c, rs);
        if (ch[k].E == 0) {
          T q = qconv<T>(ch[k]);
          accO[k].x = fma(av.x, q, accO[k].x);
          accO[k].y = fma(av.y, q, accO[k].y);
        }
      }
    }
    {
      const auto c = coef(a, mb + l + 1, ch[0]);
      const int rs = __ldg(a.dshift + mb + l + 1);
      const T2 av = at[mb + l + 1];
#pragma unroll
      for (int k = 0; k < LEG_K; ++k) {
        chain_step(ch[k], c, rs);
        if (ch[k].E == 0) {
          T q = qconv<T>(ch[k]);
          accE[k].x = fma(av.x, q, accE[k].x);
          accE[k].y = fma(av.y, q, accE[k].y);
        }
      }
    }
  }
  if (l <= L) {
    const auto c = coef(a, mb + l, ch[0]);
    const int rs = __ldg(a.dshift + mb + l);
    const T2 av = at[mb + l];
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) {
      chain_step(ch[k], c, rs);
      if (ch[k].E == 0) {
        T q = qconv<T>(ch[k]);
        accO[k].x = fma(av.x, q, accO[k].x);
        accO[k].y = fma(av.y, q, accO[k].y);
      }
    }
  }
  // F(theta_j) = E + O, F(pi - theta_j) = E - O, then the doubling
  // G(theta) = (-1)^m F(2 pi - theta) for theta in (pi, 2 pi)  (Fig. doubling)
  const int M = a.M;
  const T sg = (m & 1) ? (T)-1 : (T)1;
  T2* row = G + (size_t)m * M;
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) {
    if (!ch[k].valid) continue;
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane;
    const int js = M / 2 - jn;
    T2 fn, fs;
    fn.x = accE[k].x + accO[k].x;
    fn.y = accE[k].y + accO[k].y;
    fs.x = accE[k].x - accO[k].x;
    fs.y = accE[k].y - accO[k].y;
    row[jn] = fn;
    T2 t;
    t.x = sg * fn.x;
    t.y = sg * fn.y;
    row[M - jn] = t;
    if (js != jn) {
      row[js] = fs;
      t.x = sg * fs.x;
      t.y = sg * fs.y;
      row[M - js] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// adjoint: partial[blk][l,m] = sum over the block's rings of q_l(theta) S(theta)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ typename V2<T>::t shfl2(typename V2<T>::t v, int mask) {
  typename V2<T>::t r;
  r.x = __shfl_xor_sync(FULL, v.x, mask);
  r.y = __shfl_xor_sync(FULL, v.y, mask);
  return r;
}

template <typename T, class CH = Chain>
__global__ void __launch_bounds__(128) legendre_adj_k(LegArgs a, const typename V2<T>::t* __restrict__ Gt,
                                                      typename V2<T>::t* __restrict__ partial, int nitems,
                                                      int64_t nalm) {
  using T2 = typename V2<T>::t;
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  int m, blk;
  item_of(a, it, m, blk);
  const int L = a.lmax;
  const int M = a.M;
  const int mb = mbase_of(L, m);
  const T sg = (m & 1) ? (T)-1 : (T)1;
  const T2* row = Gt + (size_t)m * M;
  CH ch[LEG_K];
  T2 SE[LEG_K], SO[LEG_K];
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) {
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane;
    chain_init(ch[k], a, m, jn);
    T2 fn, fs;
    fn.x = fn.y = fs.x = fs.y = (T)0;
    if (ch[k].valid) {
      // D^dagger: F(theta_j) = G(theta_j) + (-1)^m G(2 pi - theta_j)
      const int js = M / 2 - jn;
      T2 g0 = row[jn], g1 = row[M - jn];
      fn.x = g0.x + sg * g1.x;
      fn.y = g0.y + sg * g1.y;
      if (js != jn) {
        T2 h0 = row[js], h1 = row[M - js];
        fs.x = h0.x + sg * h1.x;
        fs.y = h0.y + sg * h1.y;
      }
    }
    SE[k].x = fn.x + fs.x;
    SE[k].y = fn.y + fs.y;
    SO[k].x = fn.x - fs.x;
    SO[k].y = fn.y - fs.y;
  }
  T2* out = partial + (size_t)blk * nalm + mb;
  for (int base = m; base <= L; base += 8) {
    T2 v[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      v[s].x = v[s].y = (T)0;
      const int l = base + s;
      if (l <= L) {
        if (l > m) {
          const auto c = coef(a, mb + l, ch[0]);
          const int rs = __ldg(a.dshift + mb + l);
#pragma unroll
          for (int k = 0; k < LEG_K; ++k) chain_step(ch[k], c, rs);
        }
#pragma unroll
        for (int k = 0; k < LEG_K; ++k) {
          if (ch[k].E == 0) {
            T q = qconv<T>(ch[k]);
            const T2 S = (s & 1) ? SO[k] : SE[k];
            v[s].x = fma(q, S.x, v[s].x);
            v[s].y = fma(q, S.y, v[s].y);
          }
        }
      }
    }
    // reduce-scatter the 8 degrees over the 32 lanes (warp-level reduction)
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    T2 w4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T2 send = u16 ? v[i] : v[i + 4];
      T2 keep = u16 ? v[i + 4] : v[i];
      T2 r = shfl2<T>(send, 16);
      w4[i].x = keep.x + r.x;
      w4[i].y = keep.y + r.y;
    }
    T2 w2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      T2 send = u8 ? w4[i] : w4[i + 2];
      T2 keep = u8 ? w4[i + 2] : w4[i];
      T2 r = shfl2<T>(send, 8);
      w2[i].x = keep.x + r.x;
      w2[i].y = keep.y + r.y;
    }
    T2 z;
    {
      T2 send = u4 ? w2[0] : w2[1];
      T2 keep = u4 ? w2[1] : w2[0];
      T2 r = shfl2<T>(send, 4);
      z.x = keep.x + r.x;
      z.y = keep.y + r.y;
    }
    T2 r = shfl2<T>(z, 2);
    z.x += r.x;
    z.y += r.y;
    r = shfl2<T>(z, 1);
    z.x += r.x;
    z.y += r.y;
    const int l = base + ((lane >> 2) & 7);
    if ((lane & 3) == 0 && l <= L) out[l] = z;
  }
}

// Sum of the ring-block partials in a fixed order, times Ahat; the poles
// (theta = 0, pi) contribute to m = 0 only: Pbar_l0(0) = sqrt((2l+1)/4pi),
// Pbar_l0(pi) = (-1)^l sqrt((2l+1)/4pi).
// wpos multiplies the m > 0 entries: 1 for the adjoint, 2 for the gradient of
// a real loss with respect to the complex coefficients (nusht_adjoint_grad).
template <typename T>
__global__ void adj_reduce_k(const typename V2<T>::t* __restrict__ partial, int bpm, int64_t nalm,
                             const double* __restrict__ ahat, const double* __restrict__ pole_norm,
                             const typename V2<T>::t* __restrict__ Gt, int lmax, int M, double wpos,
                             typename V2<T>::t* out) {
  using T2 = typename V2<T>::t;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  double sx = 0.0, sy = 0.0;
  for (int b = 0; b < bpm; ++b) {
    T2 v = partial[(size_t)b * nalm + i];
    sx += (double)v.x;
    sy += (double)v.y;
  }
  const double ah = (i <= lmax) ? ahat[i] : ahat[i] * wpos;
  sx *= ah;
  sy *= ah;
  T2 r;
  if (i <= lmax) {  // m = 0 block: real
    const int l = (int)i;
    double np = (double)Gt[0].x, sp = (double)Gt[M / 2].x;
    sx += pole_norm[l] * (np + ((l & 1) ? -sp : sp));
    sy = 0.0;
  }
  r.x = (T)sx;
  r.y = (T)sy;
  out[i] = r;
}

// atilde_lm = a_lm Ahat_lm, with Im(a_l0) dropped
template <typename Tin, typename T>
__global__ void scale_alm_k(const Tin* __restrict__ alm, const double* __restrict__ ahat, int64_t nalm, int lmax,
                            typename V2<T>::t* __restrict__ at) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  double re = (double)alm[2 * i], im = (double)alm[2 * i + 1];
  if (i <= lmax) im = 0.0;
  const double ah = ahat[i];
  typename V2<T>::t r;
  r.x = (T)(re * ah);
  r.y = (T)(im * ah);
  at[i] = r;
}

// F_0 at the poles: G[0][0] and G[0][M/2] (all m > 0 pole entries stay 0)
template <typename Tin, typename T>
__global__ void poles_synth_k(const Tin* __restrict__ alm, const double* __restrict__ pole_norm, int lmax, int M,
                              typename V2<T>::t* G) {
  __shared__ double sn[256], ss[256];
  double n = 0.0, s = 0.0;
  for (int l = threadIdx.x; l <= lmax; l += blockDim.x) {
    double v = (double)alm[2 * l] * pole_norm[l];
    n += v;
    s += (l & 1) ? -v : v;
  }
  sn[threadIdx.x] = n;
  ss[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sn[threadIdx.x] += sn[threadIdx.x + h];
      ss[threadIdx.x] += ss[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    typename V2<T>::t a, b;
    a.x = (T)sn[0];
    a.y = (T)0;
    b.x = (T)ss[0];
    b.y = (T)0;
    G[0] = a;
    G[M / 2] = b;
  }
}

// ---------------------------------------------------------------------------
// FP64 mode with the contraction on the FP32 pipe.  The recurrence is the
// FP64 one above; only the sums  sum_l atilde_l q_l  (synthesis) and
// sum_rings q_l S (adjoint) are carried as unevaluated float pairs
// hi + lo ("double-float": ~48-bit significand):
//   * q (double) is split into qh + ql with integer bit operations;
//   * each product is formed exactly (p = ah*qh, its error by an FMA) plus
//     the cross terms ah*ql + al*qh;
//   * sums use the two-sum error-free transformation.
// Relative error per operation ~2^-48; the FP64 pipe then carries only the
// two recurrence operations per step.
// ---------------------------------------------------------------------------
// atilde as double-float complex: (hi_re, lo_re, hi_im, lo_im)
__global__ void scale_alm_df_k(const double* __restrict__ alm, const double* __restrict__ ahat, int64_t nalm, int lmax,
                               float4* __restrict__ at) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  double re = alm[2 * i], im = alm[2 * i + 1];
  if (i <= lmax) im = 0.0;
  const double ah = ahat[i];
  float4 r;
  df_of(re * ah, r.x, r.y);
  df_of(im * ah, r.z, r.w);
  at[i] = r;
}

// q as a float pair: split off the FP64 chain's double, or the double-float
// chain's own pair
__device__ __forceinline__ void qsplit(const Chain& ch, float& qh, float& ql) { split_q(ch.q1, qh, ql); }
__device__ __forceinline__ void qsplit(const DfChain& ch, float& qh, float& ql) {
  qh = ch.q1.x;
  ql = ch.q1.y;
}

template <class CH>
__device__ __forceinline__ void df_acc_step(float4& acc, const float4 av, const CH& ch) {
  float qh, ql;
  qsplit(ch, qh, ql);
  df_mac(acc.x, acc.y, av.x, av.y, qh, ql);
  df_mac(acc.z, acc.w, av.z, av.w, qh, ql);
}

template <class CH>
__global__ void __launch_bounds__(128) legendre_synth_df_k(LegArgs a, const float4* __restrict__ at,
                                                           double2* __restrict__ G, int nitems) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  int m, blk;
  item_of(a, it, m, blk);
  const int L = a.lmax;
  const int mb = mbase_of(L, m);
  CH ch[LEG_K];
  float4 accE[LEG_K], accO[LEG_K];
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) {
    chain_init(ch[k], a, m, 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane);
    accE[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    accO[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  {
    const float4 av = at[mb + m];
#pragma unroll
    for (int k = 0; k < LEG_K; ++k)
      if (ch[k].E == 0) df_acc_step(accE[k], av, ch[k]);
  }
  int l = m + 1;
  for (; l + 1 <= L; l += 2) {
    {
      const auto c = coef(a, mb + l, ch[0]);
      const int rs = __ldg(a.dshift + mb + l);
      const float4 av = at[mb + l];
#pragma unroll
      for (int k = 0; k < LEG_K; ++k) {
        chain_step(ch[k], c, rs);
        if (ch[k].E == 0) df_acc_step(accO[k], av, ch[k]);
      }
    }
    {
      const auto c = coef(a, mb + l + 1, ch[0]);
      const int rs = __ldg(a.dshift + mb + l + 1);
      const float4 av = at[mb + l + 1];
#pragma unroll
      for (int k = 0; k < LEG_K; ++k) {
        chain_step(ch[k], c, rs);
        if (ch[k].E == 0) df_acc_step(accE[k], av, ch[k]);
      }
    }
  }
  if (l <= L) {
    const auto c = coef(a, mb + l, ch[0]);
    const int rs = __ldg(a.dshift + mb + l);
    const float4 av = at[mb + l];
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) {
      chain_step(ch[k], c, rs);
      if (ch[k].E == 0) df_acc_step(accO[k], av, ch[k]);
    }
  }
  const int M = a.M;
  const double sg = (m & 1) ? -1.0 : 1.0;
  double2* row = G + (size_t)m * M;
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) {
    if (!ch[k].valid) continue;
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane;
    const int js = M / 2 - jn;
    const double er = df_value(accE[k].x, accE[k].y), ei = df_value(accE[k].z, accE[k].w);
    const double orr = df_value(accO[k].x, accO[k].y), oi = df_value(accO[k].z, accO[k].w);
    const double2 fn = make_double2(er + orr, ei + oi);
    const double2 fs = make_double2(er - orr, ei - oi);
    row[jn] = fn;
    row[M - jn] = make_double2(sg * fn.x, sg * fn.y);
    if (js != jn) {
      row[js] = fs;
      row[M - js] = make_double2(sg * fs.x, sg * fs.y);
    }
  }
}

__device__ __forceinline__ float4 shfl4(float4 v, int mask) {
  float4 r;
  r.x = __shfl_xor_sync(FULL, v.x, mask);
  r.y = __shfl_xor_sync(FULL, v.y, mask);
  r.z = __shfl_xor_sync(FULL, v.z, mask);
  r.w = __shfl_xor_sync(FULL, v.w, mask);
  return r;
}

__device__ __forceinline__ void df4_add(float4& a4, const float4 b4) {
  df_add(a4.x, a4.y, b4.x, b4.y);
  df_add(a4.z, a4.w, b4.z, b4.w);
}

// The adjoint's degree loop is rolled (two degrees, one of each parity, per
// iteration) so that its body stays small: the unrolled eight-degree body
// with register accumulators (and the shuffle reduce-scatter after it) ran
// 12 % slower, stalled on instruction fetch.  Each degree's sum over the
// lane's four chains goes to a shared-memory slot; every eight degrees the
// warp reduces the slots over its 32 lanes through the transpose: lane t sums
// one float pair (degree t / 4, re or im) over 16 lanes, and the two halves
// are combined with one shuffle.
template <class CH>
__global__ void __launch_bounds__(128, 5) legendre_adj_df_k(LegArgs a, const double2* __restrict__ Gt,
                                                         float4* __restrict__ partial, int nitems, int64_t nalm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int it = blockIdx.x * 4 + warp;
  if (it >= nitems) return;
  int m, blk;
  item_of(a, it, m, blk);
  const int L = a.lmax;
  const int M = a.M;
  const int mb = mbase_of(L, m);
  const double sg = (m & 1) ? -1.0 : 1.0;
  const double2* row = Gt + (size_t)m * M;
  CH ch[LEG_K];
  // folded spectrum per chain as double-float (hi_re, lo_re, hi_im, lo_im),
  // even / odd l - m, and the per-degree sums of each lane (rows padded to
  // 9 entries: conflict-free 16-byte stores)
  __shared__ float4 sS[2][LEG_K][128];
  __shared__ float4 red[4][32][9];
  float4* SE = &sS[0][0][threadIdx.x];
  float4* SO = &sS[1][0][threadIdx.x];
  float4(*rw)[9] = red[warp];
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) {
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane;
    chain_init(ch[k], a, m, jn);
    double2 fn = make_double2(0.0, 0.0), fs = make_double2(0.0, 0.0);
    if (ch[k].valid) {
      const int js = M / 2 - jn;
      const double2 g0 = row[jn], g1 = row[M - jn];
      fn = make_double2(g0.x + sg * g1.x, g0.y + sg * g1.y);
      if (js != jn) {
        const double2 h0 = row[js], h1 = row[M - js];
        fs = make_double2(h0.x + sg * h1.x, h0.y + sg * h1.y);
      }
    }
    float4 e4, o4;
    df_of(fn.x + fs.x, e4.x, e4.y);
    df_of(fn.y + fs.y, e4.z, e4.w);
    df_of(fn.x - fs.x, o4.x, o4.y);
    df_of(fn.y - fs.y, o4.z, o4.w);
    SE[k * 128] = e4;
    SO[k * 128] = o4;
  }
  float4* out = partial + (size_t)blk * nalm + mb;
  // one degree: advance the chains to l, sum q_l S over the lane's chains
  auto degree = [&](int l, const float4* S, float4* dst) {
    if (l > m) {
      const auto c = coef(a, mb + l, ch[0]);
      const int rs = __ldg(a.dshift + mb + l);
#pragma unroll
      for (int k = 0; k < LEG_K; ++k) chain_step(ch[k], c, rs);
    }
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) {
      if (ch[k].E == 0) {
        float qh, ql;
        qsplit(ch[k], qh, ql);
        const float4 Sv = S[k * 128];
        df_mac(acc.x, acc.y, Sv.x, Sv.y, qh, ql);
        df_mac(acc.z, acc.w, Sv.z, Sv.w, qh, ql);
      }
    }
    *dst = acc;
  };
  const int d = lane >> 2, cpt = (lane >> 1) & 1, half = lane & 1;
  for (int base = m; base <= L; base += 8) {
    const int nst = min(8, L - base + 1);
#pragma unroll 1
    for (int st = 0; st < nst; st += 2) {
      degree(base + st, SE, &rw[lane][st]);
      if (st + 1 < nst) degree(base + st + 1, SO, &rw[lane][st + 1]);
    }
    __syncwarp();
    float sh = 0.f, sl = 0.f;
    if (d < nst) {
#pragma unroll 4
      for (int i = 0; i < 16; ++i) {
        const float2 x = reinterpret_cast<const float2*>(&rw[half * 16 + i][d])[cpt];
        df_add(sh, sl, x.x, x.y);
      }
    }
    const float oh = __shfl_xor_sync(FULL, sh, 1), ol = __shfl_xor_sync(FULL, sl, 1);
    df_add(sh, sl, oh, ol);
    __syncwarp();  // the slots are rewritten by the next eight degrees
    // float pairs; adj_reduce_df_k sums the ring blocks and converts
    if (half == 0 && d < nst) reinterpret_cast<float2*>(out + base + d)[cpt] = make_float2(sh, sl);
  }
}

// c_lm = Ahat sum_blocks (hi + lo) in double, plus the poles (m = 0)
__global__ void adj_reduce_df_k(const float4* __restrict__ partial, int bpm, int64_t nalm,
                                const double* __restrict__ ahat, const double* __restrict__ pole_norm,
                                const double2* __restrict__ Gt, int lmax, int M, double wpos, double2* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  // the block partials summed as float pairs (FP32 pipe), in a fixed order,
  // then one conversion to double
  float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
  for (int b = 0; b < bpm; ++b) {
    const float4 v = partial[(size_t)b * nalm + i];
    df_add(xh, xl, v.x, v.y);
    df_add(yh, yl, v.z, v.w);
  }
  double sx = df_value(xh, xl), sy = df_value(yh, yl);
  const double ah = (i <= lmax) ? ahat[i] : ahat[i] * wpos;
  sx *= ah;
  sy *= ah;
  if (i <= lmax) {
    const int l = (int)i;
    const double np = Gt[0].x, sp = Gt[M / 2].x;
    sx += pole_norm[l] * (np + ((l & 1) ? -sp : sp));
    sy = 0.0;
  }
  out[i] = make_double2(sx, sy);
}

// ---------------------------------------------------------------------------
// Table mode (opts.legendre_table = 1).  The recurrence values at the rings
// do not depend on the coefficients, so the plan can run the FP64 recurrence
// once and keep them in HBM: per kept work item, [l - m][4 chains][32 lanes]
// of q as float (mixed) or as a float pair qh + ql (FP64 mode, ~2^-48).
// Each call then streams the table through the same contractions as above.
// ---------------------------------------------------------------------------
template <bool DF>
struct TabT;
template <>
struct TabT<false> {
  using v = float;
};
template <>
struct TabT<true> {
  using v = float2;
};

template <bool DF>
__global__ void __launch_bounds__(128) legendre_tab_build_k(LegArgs a, const int64_t* __restrict__ off,
                                                            typename TabT<DF>::v* __restrict__ tab, int nitems) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  int m, blk;
  item_of(a, it, m, blk);
  const int L = a.lmax;
  const int mb = mbase_of(L, m);
  Chain ch[LEG_K];
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) chain_init(ch[k], a, m, 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane);
  typename TabT<DF>::v* out = tab + off[it];
  for (int l = m; l <= L; ++l) {
    const bool step = l > m;
    const double c = step ? __ldg(a.c + mb + l) : 0.0;
    const int rs = step ? (int)__ldg(a.dshift + mb + l) : 0;
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) {
      if (step) chain_step(ch[k], c, rs);
      const bool use = ch[k].valid && ch[k].E == 0;
      typename TabT<DF>::v val;
      if constexpr (DF) {
        float qh = 0.f, ql = 0.f;
        if (use) split_q(ch[k].q1, qh, ql);
        val = make_float2(qh, ql);
      } else {
        val = use ? to_f32(ch[k].q1) : 0.f;
      }
      out[(size_t)(l - m) * LEG_PAIRS_PER_WARP + k * 32 + lane] = val;
    }
  }
}

// synthesis from the table; mixed: float2 atilde / float2 sums, FP64 mode:
// float4 double-float atilde and sums
template <bool DF>
__global__ void __launch_bounds__(128) legendre_synth_tab_k(LegArgs a, const int64_t* __restrict__ off,
                                                            const typename TabT<DF>::v* __restrict__ tab,
                                                            const void* __restrict__ atv, void* __restrict__ Gv,
                                                            int nitems) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  int m, blk;
  item_of(a, it, m, blk);
  const int L = a.lmax;
  const int mb = mbase_of(L, m);
  const typename TabT<DF>::v* tp = tab + off[it];
  float4 accE[LEG_K], accO[LEG_K];  // DF: (hi_re, lo_re, hi_im, lo_im); mixed: (re, im, -, -)
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) accE[k] = accO[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  // one degree into the sums of its parity (static: the loop runs in pairs)
  auto deg = [&](int l, float4* acc) {
    const typename TabT<DF>::v* row = tp + (size_t)(l - m) * LEG_PAIRS_PER_WARP + lane;
    if constexpr (DF) {
      const float4 av = reinterpret_cast<const float4*>(atv)[mb + l];
#pragma unroll
      for (int k = 0; k < LEG_K; ++k) {
        const float2 q = row[k * 32];
        df_mac(acc[k].x, acc[k].y, av.x, av.y, q.x, q.y);
        df_mac(acc[k].z, acc[k].w, av.z, av.w, q.x, q.y);
      }
    } else {
      const float2 av = reinterpret_cast<const float2*>(atv)[mb + l];
#pragma unroll
      for (int k = 0; k < LEG_K; ++k) {
        const float q = row[k * 32];
        acc[k].x = fmaf(av.x, q, acc[k].x);
        acc[k].y = fmaf(av.y, q, acc[k].y);
      }
    }
  };
  int l = m;
  for (; l + 1 <= L; l += 2) {
    deg(l, accE);
    deg(l + 1, accO);
  }
  if (l <= L) deg(l, accE);
  const int M = a.M;
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) {
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane;
    if (jn > a.npairs) continue;
    const int js = M / 2 - jn;
    double er, ei, orr, oi;
    if constexpr (DF) {
      er = df_value(accE[k].x, accE[k].y);
      ei = df_value(accE[k].z, accE[k].w);
      orr = df_value(accO[k].x, accO[k].y);
      oi = df_value(accO[k].z, accO[k].w);
    } else {
      er = accE[k].x;
      ei = accE[k].y;
      orr = accO[k].x;
      oi = accO[k].y;
    }
    const double sg = (m & 1) ? -1.0 : 1.0;
    if constexpr (DF) {
      double2* row = reinterpret_cast<double2*>(Gv) + (size_t)m * M;
      row[jn] = make_double2(er + orr, ei + oi);
      row[M - jn] = make_double2(sg * (er + orr), sg * (ei + oi));
      if (js != jn) {
        row[js] = make_double2(er - orr, ei - oi);
        row[M - js] = make_double2(sg * (er - orr), sg * (ei - oi));
      }
    } else {
      float2* row = reinterpret_cast<float2*>(Gv) + (size_t)m * M;
      row[jn] = make_float2((float)(er + orr), (float)(ei + oi));
      row[M - jn] = make_float2((float)(sg * (er + orr)), (float)(sg * (ei + oi)));
      if (js != jn) {
        row[js] = make_float2((float)(er - orr), (float)(ei - oi));
        row[M - js] = make_float2((float)(sg * (er - orr)), (float)(sg * (ei - oi)));
      }
    }
  }
}

// adjoint from the table (same reduce-scatter as legendre_adj_k)
template <bool DF>
__global__ void __launch_bounds__(128) legendre_adj_tab_k(LegArgs a, const int64_t* __restrict__ off,
                                                          const typename TabT<DF>::v* __restrict__ tab,
                                                          const void* __restrict__ Gtv, void* __restrict__ partv,
                                                          int nitems, int64_t nalm) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  int m, blk;
  item_of(a, it, m, blk);
  const int L = a.lmax;
  const int M = a.M;
  const int mb = mbase_of(L, m);
  const typename TabT<DF>::v* tp = tab + off[it];
  float4 SE[LEG_K], SO[LEG_K];  // DF: double-float pairs; mixed: (re, im, -, -)
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) {
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane;
    double2 fn = make_double2(0.0, 0.0), fs = make_double2(0.0, 0.0);
    if (jn <= a.npairs) {
      const int js = M / 2 - jn;
      const double sg = (m & 1) ? -1.0 : 1.0;
      if constexpr (DF) {
        const double2* row = reinterpret_cast<const double2*>(Gtv) + (size_t)m * M;
        const double2 g0 = row[jn], g1 = row[M - jn];
        fn = make_double2(g0.x + sg * g1.x, g0.y + sg * g1.y);
        if (js != jn) {
          const double2 h0 = row[js], h1 = row[M - js];
          fs = make_double2(h0.x + sg * h1.x, h0.y + sg * h1.y);
        }
      } else {
        const float2* row = reinterpret_cast<const float2*>(Gtv) + (size_t)m * M;
        const float2 g0 = row[jn], g1 = row[M - jn];
        fn = make_double2(g0.x + sg * g1.x, g0.y + sg * g1.y);
        if (js != jn) {
          const float2 h0 = row[js], h1 = row[M - js];
          fs = make_double2(h0.x + sg * h1.x, h0.y + sg * h1.y);
        }
      }
    }
    if constexpr (DF) {
      df_of(fn.x + fs.x, SE[k].x, SE[k].y);
      df_of(fn.y + fs.y, SE[k].z, SE[k].w);
      df_of(fn.x - fs.x, SO[k].x, SO[k].y);
      df_of(fn.y - fs.y, SO[k].z, SO[k].w);
    } else {
      SE[k] = make_float4((float)(fn.x + fs.x), (float)(fn.y + fs.y), 0.f, 0.f);
      SO[k] = make_float4((float)(fn.x - fs.x), (float)(fn.y - fs.y), 0.f, 0.f);
    }
  }
  for (int base = m; base <= L; base += 8) {
    float4 v[8];
#pragma unroll
    for (int st = 0; st < 8; ++st) {
      v[st] = make_float4(0.f, 0.f, 0.f, 0.f);
      const int l = base + st;
      if (l <= L) {
        const typename TabT<DF>::v* row = tp + (size_t)(l - m) * LEG_PAIRS_PER_WARP + lane;
#pragma unroll
        for (int k = 0; k < LEG_K; ++k) {
          const float4 S = (st & 1) ? SO[k] : SE[k];
          if constexpr (DF) {
            const float2 q = row[k * 32];
            df_mac(v[st].x, v[st].y, S.x, S.y, q.x, q.y);
            df_mac(v[st].z, v[st].w, S.z, S.w, q.x, q.y);
          } else {
            const float q = row[k * 32];
            v[st].x = fmaf(q, S.x, v[st].x);
            v[st].y = fmaf(q, S.y, v[st].y);
          }
        }
      }
    }
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    float4 w4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 send = u16 ? v[i] : v[i + 4];
      w4[i] = u16 ? v[i + 4] : v[i];
      const float4 r = shfl4(send, 16);
      if constexpr (DF) {
        df4_add(w4[i], r);
      } else {
        w4[i].x += r.x;
        w4[i].y += r.y;
      }
    }
    float4 w2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float4 send = u8 ? w4[i] : w4[i + 2];
      w2[i] = u8 ? w4[i + 2] : w4[i];
      const float4 r = shfl4(send, 8);
      if constexpr (DF) {
        df4_add(w2[i], r);
      } else {
        w2[i].x += r.x;
        w2[i].y += r.y;
      }
    }
    float4 z;
    {
      const float4 send = u4 ? w2[0] : w2[1];
      z = u4 ? w2[1] : w2[0];
      const float4 r = shfl4(send, 4);
      if constexpr (DF) {
        df4_add(z, r);
      } else {
        z.x += r.x;
        z.y += r.y;
      }
    }
#pragma unroll
    for (int msk = 2; msk >= 1; msk >>= 1) {
      const float4 r = shfl4(z, msk);
      if constexpr (DF) {
        df4_add(z, r);
      } else {
        z.x += r.x;
        z.y += r.y;
      }
    }
    const int l = base + ((lane >> 2) & 7);
    if ((lane & 3) == 0 && l <= L) {
      if constexpr (DF)
        reinterpret_cast<float4*>(partv)[(size_t)blk * nalm + mb + l] = z;
      else
        reinterpret_cast<float2*>(partv)[(size_t)blk * nalm + mb + l] = make_float2(z.x, z.y);
    }
  }
}

// Plan-time probe: does any ring of the item leave the scaled phase by lmax?
__global__ void __launch_bounds__(128) legendre_probe_k(LegArgs a, int ntotal, int* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= ntotal) return;
  const int m = it / a.bpm, blk = it % a.bpm;
  const int L = a.lmax;
  const int mb = mbase_of(L, m);
  Chain ch[LEG_K];
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) chain_init(ch[k], a, m, 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane);
  auto significant = [&]() {
    bool any = false;
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) any |= (ch[k].valid && ch[k].E == 0);
    return any;
  };
  bool sig = __any_sync(FULL, significant());
  for (int l = m + 1; l <= L && !sig; ++l) {
    const double c = __ldg(a.c + mb + l);
    const int rs = __ldg(a.dshift + mb + l);
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) chain_step(ch[k], c, rs);
    sig = __any_sync(FULL, significant());
  }
  if (lane == 0) flags[it] = sig ? 1 : 0;
}

// ---------------------------------------------------------------------------
// host: tables in double-double, then the probe and the work list
// ---------------------------------------------------------------------------
struct dd {
  double hi, lo;
};

inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
inline dd dd_norm(double hi, double lo) { return two_sum(hi, lo); }
inline dd dd_mul_d(dd a, double b) {
  double p = a.hi * b;
  double e = std::fma(a.hi, b, -p);
  e += a.lo * b;
  return dd_norm(p, e);
}
inline dd dd_div_d(dd a, double b) {
  double q1 = a.hi / b;
  dd p = dd_mul_d({q1, 0.0}, b);
  double r = ((a.hi - p.hi) - p.lo + a.lo) / b;
  return dd_norm(q1, r);
}
inline double dd_sqrt(dd a) {
  if (a.hi <= 0.0) return 0.0;
  double s = std::sqrt(a.hi);
  // one Newton step in double-double: s + (a - s^2) / (2 s)
  double p = s * s;
  double e = std::fma(s, s, -p);
  double r = ((a.hi - p) - e + a.lo) / (2.0 * s);
  return s + r;
}

}  // namespace

static LegArgs make_args(nusht_plan_t p) {
  LegArgs a;
  a.lmax = p->lmax;
  a.mmax = p->mmax;
  a.M = p->sz.M;
  a.npairs = p->leg.npairs;
  a.bpm = p->leg.blocks_per_m;
  a.items = p->leg.items;
  a.c = p->leg.c;
  a.cdf = p->leg.cdf;
  a.dshift = p->leg.dshift;
  a.cm = p->leg.cm;
  a.ring_x = p->leg.ring_x;
  a.ring_s = p->leg.ring_s;
  return a;
}

int legendre_build_tables(nusht_plan_t p, cudaStream_t s) {
  const int L = p->lmax, mmax = p->mmax, M = p->sz.M;
  const int64_t nalm = p->nalm;
  std::vector<double> c(nalm), ah(nalm);
  std::vector<int8_t> dsh(nalm, 0);
  // the double-float recurrence applies to the per-call kernels of mixed
  // plans and of FP64 plans with float-pair sums; it needs narrower segments
  const bool fastrec = p->opts.fast_recurrence && !(p->precision == NUSHT_FP64 && p->opts.fp64_contraction) &&
                       p->opts.legendre_table <= 0 && p->has_nufft;
  const int seg = fastrec ? LEG_SEG_BITS_DF : LEG_SEG_BITS;
  for (int m = 0; m <= mmax; ++m) {
    const int64_t mb = (int64_t)m * (2 * L + 1 - m) / 2;
    dd a2 = {1.0, 0.0};  // Ahat^2 (scaled)
    for (int l = m; l <= L; ++l) {
      if (l == m) {
        c[mb + l] = 0.0;
        ah[mb + l] = 1.0;
        continue;
      }
      const double dl = l, dm = m;
      // alpha_l^2 = (4 l^2 - 1) / (l^2 - m^2), exact integers
      a2 = dd_mul_d(a2, 4.0 * dl * dl - 1.0);
      a2 = dd_div_d(a2, dl * dl - dm * dm);
      int e2 = 0;
      std::frexp(a2.hi, &e2);
      if (e2 > 2 * seg) {  // Ahat >= 2^seg: next segment
        a2.hi = std::ldexp(a2.hi, -2 * seg);
        a2.lo = std::ldexp(a2.lo, -2 * seg);
        dsh[mb + l] = (int8_t)seg;
      }
      ah[mb + l] = dd_sqrt(a2);
      c[mb + l] = (l == m + 1) ? 0.0 : ((dl - 1.0 - dm) * (dl - 1.0 + dm)) / ((2.0 * dl - 3.0) * (2.0 * dl - 1.0));
    }
  }
  // c_m = Pbar_mm / sin^m(theta) = (-1)^m sqrt(prod_{i<=m} (2i+1)/(2i) / (4 pi))
  std::vector<double> cm(mmax + 1);
  {
    dd c2 = {1.0 / (4.0 * M_PI), 0.0};
    // 1/(4 pi) to double-double accuracy
    c2.lo = std::fma(-c2.hi, 4.0 * M_PI, 1.0) / (4.0 * M_PI);
    for (int m = 0; m <= mmax; ++m) {
      if (m > 0) {
        c2 = dd_mul_d(c2, 2.0 * m + 1.0);
        c2 = dd_div_d(c2, 2.0 * m);
      }
      double v = dd_sqrt(c2);
      cm[m] = (m & 1) ? -v : v;
    }
  }
  const int npairs = M / 4;
  std::vector<double> rx(npairs), rs(npairs), pn(L + 1);
  for (int j = 1; j <= npairs; ++j) {
    const double th = M_PI * (double)j / (double)(M / 2);
    rx[j - 1] = std::cos(th);
    rs[j - 1] = std::sin(th);
  }
  for (int l = 0; l <= L; ++l) pn[l] = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI));

  LegTables& t = p->leg;
  t.npairs = npairs;
  t.blocks_per_m = (npairs + LEG_PAIRS_PER_WARP - 1) / LEG_PAIRS_PER_WARP;
  NUSHT_TRY(dev_alloc((void**)&t.c, nalm * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.ahat, nalm * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.dshift, nalm, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.cm, (mmax + 1) * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.ring_x, npairs * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.ring_s, npairs * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.pole_norm, (L + 1) * 8, &p->bytes));
  NUSHT_CUDA(cudaMemcpyAsync(t.c, c.data(), nalm * 8, cudaMemcpyHostToDevice, s));
  if (fastrec) {
    std::vector<float2> cd(nalm);
    for (int64_t i = 0; i < nalm; ++i) {
      const float h = (float)c[i];
      cd[i] = make_float2(h, (float)(c[i] - (double)h));
    }
    NUSHT_TRY(dev_alloc((void**)&t.cdf, nalm * sizeof(float2), &p->bytes));
    NUSHT_CUDA(cudaMemcpyAsync(t.cdf, cd.data(), nalm * sizeof(float2), cudaMemcpyHostToDevice, s));
    NUSHT_CUDA(cudaStreamSynchronize(s));
  }
  NUSHT_CUDA(cudaMemcpyAsync(t.ahat, ah.data(), nalm * 8, cudaMemcpyHostToDevice, s));
  NUSHT_CUDA(cudaMemcpyAsync(t.dshift, dsh.data(), nalm, cudaMemcpyHostToDevice, s));
  NUSHT_CUDA(cudaMemcpyAsync(t.cm, cm.data(), (mmax + 1) * 8, cudaMemcpyHostToDevice, s));
  NUSHT_CUDA(cudaMemcpyAsync(t.ring_x, rx.data(), npairs * 8, cudaMemcpyHostToDevice, s));
  NUSHT_CUDA(cudaMemcpyAsync(t.ring_s, rs.data(), npairs * 8, cudaMemcpyHostToDevice, s));
  NUSHT_CUDA(cudaMemcpyAsync(t.pole_norm, pn.data(), (L + 1) * 8, cudaMemcpyHostToDevice, s));

  // probe every (order, ring block), keep the significant ones (m ascending:
  // the longest recurrences are issued first)
  const int ntotal = (mmax + 1) * t.blocks_per_m;
  t.nitems_total = ntotal;
  int* dflags = nullptr;
  NUSHT_TRY(dev_alloc((void**)&dflags, (size_t)ntotal * 4, nullptr));
  LegArgs a = make_args(p);
  a.items = nullptr;
  legendre_probe_k<<<(ntotal + 3) / 4, 128, 0, s>>>(a, ntotal, dflags);
  cudaError_t e = cudaGetLastError();
  std::vector<int> flags(ntotal);
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags.data(), dflags, (size_t)ntotal * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(dflags);
  if (e != cudaSuccess) return cuda_status(e, "legendre probe");
  std::vector<int> items;
  items.reserve(ntotal);
  for (int i = 0; i < ntotal; ++i)
    if (flags[i]) items.push_back(((i / t.blocks_per_m) << 16) | (i % t.blocks_per_m));
  t.nitems = (int)items.size();
  // triples (ring pair, l, m) processed per call: the roofline's unit of work
  int64_t tri = 0;
  for (int v : items) {
    const int m = v >> 16, blk = v & 0xffff;
    const int j0 = 1 + blk * LEG_PAIRS_PER_WARP;
    const int nvalid = std::max(0, std::min(LEG_PAIRS_PER_WARP, npairs - j0 + 1));
    tri += (int64_t)nvalid * (L - m + 1);
  }
  t.triples = tri;
  NUSHT_TRY(dev_alloc((void**)&t.items, std::max<size_t>(1, items.size()) * 4, &p->bytes));
  if (!items.empty())
    NUSHT_CUDA(cudaMemcpyAsync(t.items, items.data(), items.size() * 4, cudaMemcpyHostToDevice, s));
  // the work list is on the device now; the table kernel reads it.
  // Recurrence table when it fits in half the free memory: with
  // opts.legendre_table = 1, and by default for standalone mixed plans (the
  // per-call FP64 recurrence is then most of a mixed call; its table is a
  // float per triple, 59 GB at lmax 4095) unless the caller asked for the
  // double-float per-call recurrence.
  const bool want_tab = p->opts.legendre_table > 0 ||
                        (p->opts.legendre_table == 0 && p->precision == NUSHT_MIXED && p->has_nufft && !fastrec);
  if (want_tab && t.nitems > 0) {
    const bool df = p->precision == NUSHT_FP64;
    const size_t es = df ? sizeof(float2) : sizeof(float);
    std::vector<int64_t> off(items.size() + 1, 0);
    for (size_t k = 0; k < items.size(); ++k)
      off[k + 1] = off[k] + (int64_t)(L - (items[k] >> 16) + 1) * LEG_PAIRS_PER_WARP;
    const size_t need = (size_t)off.back() * es;
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    if (need < freeb / 2) {
      NUSHT_TRY(dev_alloc(&t.tab, need, &p->bytes));
      NUSHT_TRY(dev_alloc((void**)&t.tab_off, off.size() * 8, &p->bytes));
      NUSHT_CUDA(cudaMemcpyAsync(t.tab_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, s));
      LegArgs ta = make_args(p);
      if (df)
        legendre_tab_build_k<true><<<(t.nitems + 3) / 4, 128, 0, s>>>(ta, t.tab_off, (float2*)t.tab, t.nitems);
      else
        legendre_tab_build_k<false><<<(t.nitems + 3) / 4, 128, 0, s>>>(ta, t.tab_off, (float*)t.tab, t.nitems);
      NUSHT_CUDA(cudaGetLastError());
      t.tab_bytes = need;
    }
  }

  NUSHT_CUDA(cudaStreamSynchronize(s));
  return NUSHT_OK;
}

int legendre_synth(nusht_plan_t p, const void* d_alm, cudaStream_t s) {
  const int64_t nalm = p->nalm;
  const bool fastrec = p->leg.cdf != nullptr;  // opts.fast_recurrence (built when it applies)
  const int tb = 256;
  const int nb = (int)((nalm + tb - 1) / tb);
  LegArgs a = make_args(p);
  const int nitems = p->leg.nitems;
  if (p->leg.tab) {
    if (p->precision == NUSHT_FP64) {
      scale_alm_df_k<<<nb, tb, 0, s>>>((const double*)d_alm, p->leg.ahat, nalm, p->lmax, (float4*)p->atilde);
      if (nitems > 0)
        legendre_synth_tab_k<true><<<(nitems + 3) / 4, 128, 0, s>>>(a, p->leg.tab_off, (const float2*)p->leg.tab,
                                                                     p->atilde, p->G, nitems);
      poles_synth_k<double, double><<<1, 256, 0, s>>>((const double*)d_alm, p->leg.pole_norm, p->lmax, p->sz.M,
                                                      (double2*)p->G);
    } else {
      scale_alm_k<float, float><<<nb, tb, 0, s>>>((const float*)d_alm, p->leg.ahat, nalm, p->lmax,
                                                  (float2*)p->atilde);
      if (nitems > 0)
        legendre_synth_tab_k<false><<<(nitems + 3) / 4, 128, 0, s>>>(a, p->leg.tab_off, (const float*)p->leg.tab,
                                                                      p->atilde, p->G, nitems);
      poles_synth_k<float, float><<<1, 256, 0, s>>>((const float*)d_alm, p->leg.pole_norm, p->lmax, p->sz.M,
                                                    (float2*)p->G);
    }
  } else if (p->precision == NUSHT_FP64 && !p->opts.fp64_contraction) {
    scale_alm_df_k<<<nb, tb, 0, s>>>((const double*)d_alm, p->leg.ahat, nalm, p->lmax, (float4*)p->atilde);
    if (nitems > 0)
    {
      if (fastrec)
        legendre_synth_df_k<DfChain><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const float4*)p->atilde, (double2*)p->G,
                                                                      nitems);
      else
        legendre_synth_df_k<Chain><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const float4*)p->atilde, (double2*)p->G,
                                                                    nitems);
    }
    poles_synth_k<double, double><<<1, 256, 0, s>>>((const double*)d_alm, p->leg.pole_norm, p->lmax, p->sz.M,
                                                    (double2*)p->G);
  } else if (p->precision == NUSHT_FP64) {
    scale_alm_k<double, double><<<nb, tb, 0, s>>>((const double*)d_alm, p->leg.ahat, nalm, p->lmax,
                                                  (double2*)p->atilde);
    if (nitems > 0)
      legendre_synth_k<double><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const double2*)p->atilde, (double2*)p->G, nitems);
    poles_synth_k<double, double><<<1, 256, 0, s>>>((const double*)d_alm, p->leg.pole_norm, p->lmax, p->sz.M,
                                                    (double2*)p->G);
  } else {
    scale_alm_k<float, float><<<nb, tb, 0, s>>>((const float*)d_alm, p->leg.ahat, nalm, p->lmax, (float2*)p->atilde);
    if (nitems > 0)
    {
      if (fastrec)
        legendre_synth_k<float, DfChain><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const float2*)p->atilde,
                                                                          (float2*)p->G, nitems);
      else
        legendre_synth_k<float><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const float2*)p->atilde, (float2*)p->G, nitems);
    }
    poles_synth_k<float, float><<<1, 256, 0, s>>>((const float*)d_alm, p->leg.pole_norm, p->lmax, p->sz.M,
                                                  (float2*)p->G);
  }
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int legendre_adjoint(nusht_plan_t p, void* d_alm, cudaStream_t s, double wpos) {
  const int64_t nalm = p->nalm;
  const bool fastrec = p->leg.cdf != nullptr;
  LegArgs a = make_args(p);
  const int nitems = p->leg.nitems;
  const int tb = 256;
  const int nb = (int)((nalm + tb - 1) / tb);
  if (p->leg.tab) {
    if (p->precision == NUSHT_FP64) {
      if (nitems > 0)
        legendre_adj_tab_k<true><<<(nitems + 3) / 4, 128, 0, s>>>(a, p->leg.tab_off, (const float2*)p->leg.tab,
                                                                   p->Ghat, p->partial, nitems, nalm);
      adj_reduce_df_k<<<nb, tb, 0, s>>>((const float4*)p->partial, p->leg.blocks_per_m, nalm, p->leg.ahat,
                                        p->leg.pole_norm, (const double2*)p->Ghat, p->lmax, p->sz.M, wpos,
                                        (double2*)d_alm);
    } else {
      if (nitems > 0)
        legendre_adj_tab_k<false><<<(nitems + 3) / 4, 128, 0, s>>>(a, p->leg.tab_off, (const float*)p->leg.tab,
                                                                    p->Ghat, p->partial, nitems, nalm);
      adj_reduce_k<float><<<nb, tb, 0, s>>>((const float2*)p->partial, p->leg.blocks_per_m, nalm, p->leg.ahat,
                                            p->leg.pole_norm, (const float2*)p->Ghat, p->lmax, p->sz.M, wpos,
                                            (float2*)d_alm);
    }
  } else if (p->precision == NUSHT_FP64 && !p->opts.fp64_contraction) {
    if (nitems > 0)
    {
      if (fastrec)
        legendre_adj_df_k<DfChain><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const double2*)p->Ghat, (float4*)p->partial,
                                                                    nitems, nalm);
      else
        legendre_adj_df_k<Chain><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const double2*)p->Ghat, (float4*)p->partial,
                                                                  nitems, nalm);
    }
    adj_reduce_df_k<<<nb, tb, 0, s>>>((const float4*)p->partial, p->leg.blocks_per_m, nalm, p->leg.ahat,
                                      p->leg.pole_norm, (const double2*)p->Ghat, p->lmax, p->sz.M, wpos,
                                      (double2*)d_alm);
  } else if (p->precision == NUSHT_FP64) {
    if (nitems > 0)
      legendre_adj_k<double><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const double2*)p->Ghat, (double2*)p->partial, nitems,
                                                              nalm);
    adj_reduce_k<double><<<nb, tb, 0, s>>>((const double2*)p->partial, p->leg.blocks_per_m, nalm, p->leg.ahat,
                                           p->leg.pole_norm, (const double2*)p->Ghat, p->lmax, p->sz.M, wpos,
                                           (double2*)d_alm);
  } else {
    if (nitems > 0)
    {
      if (fastrec)
        legendre_adj_k<float, DfChain><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const float2*)p->Ghat,
                                                                        (float2*)p->partial, nitems, nalm);
      else
        legendre_adj_k<float><<<(nitems + 3) / 4, 128, 0, s>>>(a, (const float2*)p->Ghat, (float2*)p->partial,
                                                               nitems, nalm);
    }
    adj_reduce_k<float><<<nb, tb, 0, s>>>((const float2*)p->partial, p->leg.blocks_per_m, nalm, p->leg.ahat,
                                          p->leg.pole_norm, (const float2*)p->Ghat, p->lmax, p->sz.M, wpos,
                                          (float2*)d_alm);
  }
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

}  // namespace nusht

// ---------------------------------------------------------------------------
// Allocation-free, plan-free adjoint for small band limits.
//
// A variant of legendre_adj_k for callers that cannot allocate device memory:
// instead of rings it runs the recurrence at the caller's points directly
// (c_lm = sum_i f_i Pbar_lm(theta_i) e^{-i m phi_i}, no FFT and no NUFFT, so
// no plan and no plan-time allocation), computing the recurrence
// coefficients on the fly, and it keeps its per-warp partial sums in the
// file-scope device array below instead of plan-owned memory.
// ---------------------------------------------------------------------------
namespace nusht {
namespace {

constexpr int NA_LMAX = 255;   // largest lmax accepted
constexpr int NA_SLOTS = 16;   // partial-sum slots per coefficient at the largest size
constexpr int NA_NALM_MAX = (NA_LMAX + 1) * (NA_LMAX + 2) / 2;
constexpr int NA_CAP = NA_SLOTS * NA_NALM_MAX;  // complex entries of the array
constexpr int NA_CHUNK = 32 * LEG_K;            // points per warp pass
constexpr int NA_SLOTS_MAX = 4096;              // bound on the slots of small problems

// NA_CAP complex partial sums = 16 x 33024 x 16 B = 8.45 MB.  Every device
// that loads this library holds it until the process exits.
static __device__ __align__(256) double2 g_noalloc_partial[NA_CAP];

// One warp per (order m, slot); slot s takes the point chunks s, s + nslots,
// ... and writes its partial sums to partial[s][l, m] (nslots x nalm <= NA_CAP).
__global__ void __launch_bounds__(128) direct_adj_k(int L, int mmax, int64_t npts, const double* __restrict__ pts,
                                                    const double* __restrict__ f, double2* __restrict__ partial,
                                                    int nalm, int nslots) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= (mmax + 1) * nslots) return;
  const int m = it / nslots, slot = it % nslots;
  const int mb = mbase_of(L, m);
  // Pbar_mm / sin^m = (-1)^m sqrt(prod_{i<=m} (2i+1)/(2i) / (4 pi))
  double cmm = 0.28209479177387814;  // 1/sqrt(4 pi)
  for (int i = 1; i <= m; ++i) cmm *= sqrt((2.0 * i + 1.0) / (2.0 * i));
  if (m & 1) cmm = -cmm;
  double2* out = partial + (size_t)slot * nalm + mb;
  const int64_t chunk = NA_CHUNK;
  bool first = true;
  for (int64_t c0 = (int64_t)slot * chunk; first || c0 < npts; c0 += (int64_t)nslots * chunk) {
    Chain ch[LEG_K];
    double2 S[LEG_K];
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) {
      const int64_t i = c0 + k * 32 + lane;
      ch[k].q2 = 0.0;
      ch[k].valid = i < npts;
      ch[k].x = 0.0;
      ch[k].q1 = 0.0;
      ch[k].E = 0;
      S[k].x = S[k].y = 0.0;
      if (!ch[k].valid) continue;
      const double th = pts[2 * i], ph = pts[2 * i + 1];
      double s, c;
      sincos(th, &s, &c);
      ch[k].x = c;
      double q0 = cmm;
      int ex = 0;
      if (m > 0) {
        const double as = fabs(s);
        if (as == 0.0) {
          q0 = 0.0;
        } else {
          double mant;
          pow_scaled(as, m, mant, ex);
          q0 = cmm * mant * ((s < 0.0 && (m & 1)) ? -1.0 : 1.0);
        }
      }
      if (q0 == 0.0 || ex >= LEG_TINY_EXP) {
        ch[k].q1 = q0 * exp2i(ex < LEG_TINY_EXP ? 0 : ex);
      } else {
        const int E = LEG_STEP_EXP * ((LEG_TINY_EXP - ex + LEG_STEP_EXP - 1) / LEG_STEP_EXP);
        ch[k].q1 = q0 * exp2i(ex + E);
        ch[k].E = E;
      }
      double sp, cp;
      sincos((double)m * ph, &sp, &cp);
      S[k].x = f[i] * cp;
      S[k].y = -f[i] * sp;
    }
    for (int base = m; base <= L; base += 8) {
      double2 v[8];
#pragma unroll
      for (int st = 0; st < 8; ++st) {
        v[st].x = v[st].y = 0.0;
        const int l = base + st;
        if (l <= L) {
          if (l > m) {
            // Pbar_l = alpha_l (x Pbar_{l-1} - b_l Pbar_{l-2}), coefficients on the fly
            const double dl = l, dm = m;
            const double al = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
            const double bl = (l == m + 1) ? 0.0
                                           : sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) /
                                                  (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
#pragma unroll
            for (int k = 0; k < LEG_K; ++k) {
              const double q = al * fma(ch[k].x, ch[k].q1, -bl * ch[k].q2);
              ch[k].q2 = ch[k].q1;
              ch[k].q1 = q;
              if (ch[k].E != 0) {
                const int expo = (__double2hiint(q) >> 20) & 0x7ff;
                if (expo >= 1023 - 44) {
                  ch[k].q1 = scale_pow2(ch[k].q1, -LEG_STEP_EXP);
                  ch[k].q2 = scale_pow2(ch[k].q2, -LEG_STEP_EXP);
                  ch[k].E -= LEG_STEP_EXP;
                }
              }
            }
          }
#pragma unroll
          for (int k = 0; k < LEG_K; ++k)
            if (ch[k].E == 0) {
              v[st].x = fma(ch[k].q1, S[k].x, v[st].x);
              v[st].y = fma(ch[k].q1, S[k].y, v[st].y);
            }
        }
      }
      // same reduce-scatter over the lanes as legendre_adj_k
      const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
      double2 w4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        double2 send = u16 ? v[i] : v[i + 4];
        double2 keep = u16 ? v[i + 4] : v[i];
        double2 r = shfl2<double>(send, 16);
        w4[i].x = keep.x + r.x;
        w4[i].y = keep.y + r.y;
      }
      double2 w2[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        double2 send = u8 ? w4[i] : w4[i + 2];
        double2 keep = u8 ? w4[i + 2] : w4[i];
        double2 r = shfl2<double>(send, 8);
        w2[i].x = keep.x + r.x;
        w2[i].y = keep.y + r.y;
      }
      double2 z;
      {
        double2 send = u4 ? w2[0] : w2[1];
        double2 keep = u4 ? w2[1] : w2[0];
        double2 r = shfl2<double>(send, 4);
        z.x = keep.x + r.x;
        z.y = keep.y + r.y;
      }
      double2 r = shfl2<double>(z, 2);
      z.x += r.x;
      z.y += r.y;
      r = shfl2<double>(z, 1);
      z.x += r.x;
      z.y += r.y;
      const int l = base + ((lane >> 2) & 7);
      if ((lane & 3) == 0 && l <= L) {
        // the first chunk of a slot overwrites what an earlier call left there
        if (first) {
          out[l] = z;
        } else {
          double2 o = out[l];
          o.x += z.x;
          o.y += z.y;
          out[l] = o;
        }
      }
    }
    first = false;
  }
}

__global__ void direct_adj_reduce_k(const double2* __restrict__ partial, int nalm, int nslots, int lmax,
                                    double2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  double sx = 0.0, sy = 0.0;
  for (int s = 0; s < nslots; ++s) {
    const double2 v = partial[(size_t)s * nalm + i];
    sx += v.x;
    sy += v.y;
  }
  if (i <= lmax) sy = 0.0;  // m = 0: real
  out[i] = make_double2(sx, sy);
}

}  // namespace
}  // namespace nusht

extern "C" int nusht_adjoint_direct_noalloc(int lmax, int mmax, int64_t npts, const double* d_pts,
                                            const double* d_map, void* d_alm, nusht_stream_t stream) {
  using namespace nusht;
  if (lmax < 0 || lmax > NA_LMAX)
    return set_error(NUSHT_EINVAL, "nusht_adjoint_direct_noalloc: lmax must be in [0, 255] (static scratch limit)");
  if (mmax < 0 || mmax > lmax) return set_error(NUSHT_EINVAL, "nusht_adjoint_direct_noalloc: mmax must be in [0, lmax]");
  if (npts < 0) return set_error(NUSHT_EINVAL, "nusht_adjoint_direct_noalloc: npts < 0");
  if (!d_alm || (npts > 0 && (!d_pts || !d_map)))
    return set_error(NUSHT_EINVAL, "nusht_adjoint_direct_noalloc: null pointer");
  // The array's device address in the current device's context.  Host code
  // cannot use the symbol itself (it names a host-side shadow), so it is
  // looked up here on every call, with the caller's device current: a cached
  // address would go stale after cudaDeviceReset or under another context.
  // The lookup is cheap once the library's device code is loaded; the first
  // call on a device loads it.
  void* scratch = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_partial);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_partial)");
  const int nalm = (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) / 2;
  // slots: as many as the array holds for this nalm, no more than there are
  // point chunks (at least one, whose first pass writes the zeros of an
  // empty point set)
  const int64_t nchunks = (npts + NA_CHUNK - 1) / NA_CHUNK;
  const int nslots = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)NA_CAP / nalm, nchunks,
                                                                   (int64_t)NA_SLOTS_MAX}));
  cudaStream_t s = (cudaStream_t)stream;
  const int nwarps = (mmax + 1) * nslots;
  direct_adj_k<<<(nwarps + 3) / 4, 128, 0, s>>>(lmax, mmax, npts, d_pts, d_map, (double2*)scratch, nalm, nslots);
  direct_adj_reduce_k<<<(nalm + 255) / 256, 256, 0, s>>>((const double2*)scratch, nalm, nslots, lmax,
                                                          (double2*)d_alm);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}
