// spin.cu -- spin-weighted transforms (the spin-n generalisation named in the
// Conclusion, Sec. 5) through the same double Fourier sphere chain.
//
// For spin s >= 1 two real fields Q, U carry Q + i U = sum (G_lm + i C_lm) sY_lm
// with sY_lm = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi} and G, C
// real-field coefficients (stored for m >= 0).  With
//   lambda+ = sY_lm(theta, 0),  lambda- = (-s)Y_lm(theta, 0),
//   W = (lambda+ + (-1)^s lambda-) / 2,  X = (lambda+ - (-1)^s lambda-) / 2,
// the iso-latitude step gives for each order the two ring functions
//   F^Q_m = sum_l (G_lm W + i C_lm X),   F^U_m = sum_l (C_lm W - i G_lm X),
// and Q, U are real-field syntheses of F^Q, F^U (F_0 + 2 Re sum_{m>0} F_m e^{imphi}).
// The doubling D carries one more sign: a spin-s quantity changes sign
// (-1)^s with the local frame on the continuation through the pole, so
// G(2 pi - theta) = (-1)^(m+s) F(theta).
//
// Legendre part.  For each (order m, ring pair theta, pi - theta) two Wigner-d
// recurrences in l run in FP64 (pv = lambda+ ~ d^l_{m,-s}, nv = lambda- ~
// d^l_{m,s}):
//   v_l = A_l (x - b_l) v_{l-1} - C_l v_{l-2},  b_l = -/+ m s / (l (l-1)),
// three FP64 operations per step with the plan-time tables A_l, A_l m s /
// (l (l-1)) and C_l; started at l0 = max(m, s) from
// sqrt(C(2 l0, k)) cos^a(theta/2) sin^b(theta/2) with an integer exponent
// beside the mantissa (values below 2^-300 are carried scaled and not
// accumulated, as in legendre.cu).  Since d^l_{m,-s}(pi - theta) =
// (-1)^(l+m) d^l_{m,s}(theta), the two chains at theta give both rings: with
// p = (-1)^(l+m+s), pv(pi - theta) = p (-1)^s nv and nv(pi - theta) =
// p (-1)^s pv.  In terms of A+ = (G + iC) / 2 and A- = (-1)^s (G - iC) / 2,
//   north: F^Q = sum pv A+ + nv A-,   F^U = -i (sum pv A+ - nv A-),
//   south: F^Q = (-1)^s sum p (nv A+ + pv A-),  F^U = (-1)^s i sum p (pv A- - nv A+),
// four complex sums per ring pair, kept as float pairs on the FP32 pipe
// (the FP64 pipe carries only the six recurrence operations per degree).
// The adjoint is the transpose: with B+- = H^Q +- i H^U at each ring,
// U1 = (B+_n + p B-_s) / 2, U2 = (-1)^s (B-_n + p B+_s) / 2 and V1, V2 with
// -p, each degree adds G = pv U1 + nv U2 and C = i (nv V2 - pv V1) per ring
// pair; the lanes' float-pair sums go to shared-memory slots and every four
// degrees the warp reduces them through a transpose (lane t sums one float
// pair over 16 lanes, one shuffle joins the halves).  One ring pair per
// lane, four passes per warp over an item's 128 ring pairs; every (order,
// ring block) is processed; one partial row per (ring block, pass), summed in
// a fixed order.  A plan-time probe runs the two chains of every pass once
// and records the passes (32 ring pairs of an order) where some value rises
// above 2^-300; the others contribute nothing and are skipped (synthesis
// writes their rings as zeros).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "nusht_internal.cuh"
#include "recurrence.cuh"

namespace nusht {

namespace {

using namespace rec;
constexpr unsigned FULL = 0xffffffffu;

struct SpinArgs {
  int lmax, mmax, M, npairs, bpm, s;
  const double* A;    // per packed (l, m): A_l
  const double* Ab;   // A_l m s / (l (l - 1))
  const double* Cc;   // C_l
  const double* st_mant;  // per m and sign (2 m + 0: lambda+, 2 m + 1: lambda-): start mantissa
  const int* st_exp;      // start exponent (binary)
  const int* st_ab;       // per m and sign: powers a (cos) and b (sin) of theta / 2, packed a << 16 | b
  const unsigned char* keep;  // per item: passes to run (bit k: pass k); null = all
};

// one Wigner-d chain: value = q1 * 2^-E
struct SChain {
  double q1, q2;
  int E;
};

__device__ __forceinline__ void schain_init(SChain& c, double mant, int ex, int a, int b, double ch, double sh) {
  double ma, mb;
  int ea, eb;
  pow_scaled(ch, a, ma, ea);
  pow_scaled(sh, b, mb, eb);
  const double v = mant * ma * mb;  // mantissas in [0.25, 1) x [0.5, 1): no overflow or underflow
  const int e = ex + ea + eb;
  c.q2 = 0.0;
  if (v == 0.0) {
    c.q1 = 0.0;
    c.E = 0;
  } else if (e >= LEG_TINY_EXP) {
    c.q1 = v * exp2i(e);
    c.E = 0;
  } else {
    const int E = LEG_STEP_EXP * ((LEG_TINY_EXP - e + LEG_STEP_EXP - 1) / LEG_STEP_EXP);
    c.q1 = v * exp2i(e + E);
    c.E = E;
  }
}

__device__ __forceinline__ void schain_step(SChain& c, double t, double cc) {
  const double q = fma(t, c.q1, -cc * c.q2);
  c.q2 = c.q1;
  c.q1 = q;
  if (c.E != 0) {
    const int expo = (__double2hiint(q) >> 20) & 0x7ff;
    if (expo >= 1023 - 44) {
      c.q1 = scale_pow2(c.q1, -LEG_STEP_EXP);
      c.q2 = scale_pow2(c.q2, -LEG_STEP_EXP);
      c.E -= LEG_STEP_EXP;
    }
  }
}

__device__ __forceinline__ double sval(const SChain& c) { return c.E == 0 ? c.q1 : 0.0; }

struct Ring {
  double x, ch, sh;  // cos(theta), cos(theta / 2), sin(theta / 2)
};

__device__ __forceinline__ Ring ring_of(int j, int M) {
  Ring r;
  double sh, ch;
  sincospi((double)j / (double)M, &sh, &ch);  // theta / 2 = pi j / M
  r.ch = ch;
  r.sh = sh;
  r.x = ch * ch - sh * sh;
  return r;
}

// (G + iC) / 2 and (-1)^s (G - iC) / 2 per packed (l, m) as float pairs
// (hi re, lo re, hi im, lo im); Im of the m = 0 entries is ignored
__global__ void spin_scale_k(const double2* __restrict__ glm, const double2* __restrict__ clm, int64_t nalm, int L,
                             int s, float4* __restrict__ ap, float4* __restrict__ am) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  double2 g = glm[i], c = clm[i];
  if (i <= L) g.y = c.y = 0.0;
  const double hs = (s & 1) ? -0.5 : 0.5;
  float4 p, q;
  df_of(0.5 * (g.x - c.y), p.x, p.y);
  df_of(0.5 * (g.y + c.x), p.z, p.w);
  df_of(hs * (g.x + c.y), q.x, q.y);
  df_of(hs * (g.y - c.x), q.z, q.w);
  ap[i] = p;
  am[i] = q;
}

// acc += (float-pair complex a) * (float-pair real v)
__device__ __forceinline__ void cmac(float4& acc, const float4 a, float vh, float vl) {
  df_mac(acc.x, acc.y, a.x, a.y, vh, vl);
  df_mac(acc.z, acc.w, a.z, a.w, vh, vl);
}

__device__ __forceinline__ double2 cval(const float4 v) {
  return make_double2(df_value(v.x, v.y), df_value(v.z, v.w));
}

// plan time: which passes of each (order, ring block) ever hold a value above
// 2^-300 in either chain (the same chain steps as the transforms)
__global__ void __launch_bounds__(128) spin_probe_k(SpinArgs a, unsigned char* __restrict__ keep) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= (a.mmax + 1) * a.bpm) return;
  const int m = it / a.bpm, blk = it % a.bpm;
  const int L = a.lmax, s = a.s, M = a.M;
  const int l0 = m > s ? m : s;
  unsigned bits = 0;
  if (l0 <= L) {
    const int mb = mbase_of(L, m);
    const double mp = __ldg(a.st_mant + 2 * m), mn = __ldg(a.st_mant + 2 * m + 1);
    const int ep = __ldg(a.st_exp + 2 * m), en = __ldg(a.st_exp + 2 * m + 1);
    const int abp = __ldg(a.st_ab + 2 * m), abn = __ldg(a.st_ab + 2 * m + 1);
    for (int pass = 0; pass < 4; ++pass) {
      const int jn = 1 + blk * LEG_PAIRS_PER_WARP + pass * 32 + lane;
      const bool valid = jn <= a.npairs;
      const Ring rg = ring_of(valid ? jn : 1, M);
      SChain P, N;
      schain_init(P, mp, ep, abp >> 16, abp & 0xffff, rg.ch, rg.sh);
      schain_init(N, mn, en, abn >> 16, abn & 0xffff, rg.ch, rg.sh);
      // the pass is kept as soon as one lane's chain is ordinary (warp-uniform exit)
      bool live = valid && (P.E == 0 || N.E == 0);
      for (int l = l0 + 1; l <= L && !__any_sync(FULL, live); ++l) {
        const double A = __ldg(a.A + mb + l), Ab = __ldg(a.Ab + mb + l), C = __ldg(a.Cc + mb + l);
        schain_step(P, fma(A, rg.x, Ab), C);
        schain_step(N, fma(A, rg.x, -Ab), C);
        live = valid && (P.E == 0 || N.E == 0);
      }
      if (__any_sync(FULL, live)) bits |= 1u << pass;
    }
  }
  if (lane == 0) keep[it] = (unsigned char)bits;
}

// synthesis: the Q and U ring maps, doubled, [m][M] complex each
__global__ void __launch_bounds__(128) spin_synth_k(SpinArgs a, const float4* __restrict__ ap,
                                                    const float4* __restrict__ am, double2* __restrict__ GQ,
                                                    double2* __restrict__ GU) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= (a.mmax + 1) * a.bpm) return;
  const int m = it / a.bpm, blk = it % a.bpm;
  const int L = a.lmax, s = a.s, M = a.M;
  const int l0 = m > s ? m : s;
  if (l0 > L) return;
  const int mb = mbase_of(L, m);
  const double sgs = (s & 1) ? -1.0 : 1.0;               // (-1)^s
  const double sgd = ((m + s) & 1) ? -1.0 : 1.0;         // doubling sign (-1)^(m+s)
  const double mp = __ldg(a.st_mant + 2 * m), mn = __ldg(a.st_mant + 2 * m + 1);
  const int ep = __ldg(a.st_exp + 2 * m), en = __ldg(a.st_exp + 2 * m + 1);
  const int abp = __ldg(a.st_ab + 2 * m), abn = __ldg(a.st_ab + 2 * m + 1);
  double2* rq = GQ + (size_t)m * M;
  double2* ru = GU + (size_t)m * M;
  const unsigned kp = a.keep ? a.keep[it] : 15u;
  for (int pass = 0; pass < 4; ++pass) {
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + pass * 32 + lane;
    const bool valid = jn <= a.npairs;
    if (!(kp & (1u << pass))) {
      // every value of this pass stays below 2^-300: its rings are zero
      if (valid) {
        const double2 z = make_double2(0.0, 0.0);
        const int js = M / 2 - jn;
        rq[jn] = ru[jn] = rq[M - jn] = ru[M - jn] = z;
        rq[js] = ru[js] = rq[M - js] = ru[M - js] = z;
      }
      continue;
    }
    const Ring rg = ring_of(valid ? jn : 1, M);
    SChain P, N;
    schain_init(P, mp, ep, abp >> 16, abp & 0xffff, rg.ch, rg.sh);
    schain_init(N, mn, en, abn >> 16, abn & 0xffff, rg.ch, rg.sh);
    // north: PA = sum pv A+, NA = sum nv A-; south: D1 = sum p nv A+, D2 = sum p pv A-
    float4 PA = make_float4(0.f, 0.f, 0.f, 0.f), NA = PA, D1 = PA, D2 = PA;
    auto acc = [&](int l) {
      if (P.E != 0 && N.E != 0) return;
      float ph, pl, nh, nl;
      split_q(sval(P), ph, pl);
      split_q(sval(N), nh, nl);
      const float4 A = __ldg(ap + mb + l), B = __ldg(am + mb + l);
      cmac(PA, A, ph, pl);
      cmac(NA, B, nh, nl);
      const bool neg = ((l + m + s) & 1) != 0;
      cmac(D1, A, neg ? -nh : nh, neg ? -nl : nl);
      cmac(D2, B, neg ? -ph : ph, neg ? -pl : pl);
    };
    acc(l0);
    for (int l = l0 + 1; l <= L; ++l) {
      const double A = __ldg(a.A + mb + l), Ab = __ldg(a.Ab + mb + l), C = __ldg(a.Cc + mb + l);
      schain_step(P, fma(A, rg.x, Ab), C);   // lambda+: d^l_{m,-s}, b_l = -m s / (l (l-1))
      schain_step(N, fma(A, rg.x, -Ab), C);  // lambda-: d^l_{m,s}
      acc(l);
    }
    if (!valid) continue;
    const double2 pa = cval(PA), na = cval(NA), d1 = cval(D1), d2 = cval(D2);
    const double2 fqn = make_double2(pa.x + na.x, pa.y + na.y);
    const double2 fun = make_double2(pa.y - na.y, na.x - pa.x);              // -i (PA - NA)
    const double2 fqs = make_double2(sgs * (d1.x + d2.x), sgs * (d1.y + d2.y));
    const double2 fus = make_double2(sgs * (d1.y - d2.y), sgs * (d2.x - d1.x));  // (-1)^s i (D2 - D1)
    const int js = M / 2 - jn;
    rq[jn] = fqn;
    ru[jn] = fun;
    rq[M - jn] = make_double2(sgd * fqn.x, sgd * fqn.y);
    ru[M - jn] = make_double2(sgd * fun.x, sgd * fun.y);
    if (js != jn) {
      rq[js] = fqs;
      ru[js] = fus;
      rq[M - js] = make_double2(sgd * fqs.x, sgd * fqs.y);
      ru[M - js] = make_double2(sgd * fus.x, sgd * fus.y);
    }
  }
}

// the poles theta = 0, pi: only the order m = s is nonzero there, with
// W(0) = -X(0) = N_l / 2 and W(pi) = X(pi) = (-1)^(l+s) (-1)^s N_l / 2, N_l = sqrt((2l+1)/4pi);
// the pole entries of every other order are set to zero (the adjoint uses the
// same buffers for the theta spectra)
__global__ void spin_poles_k(int L, int mmax, int s, int M, const double2* __restrict__ glm,
                             const double2* __restrict__ clm, double2* __restrict__ GQ, double2* __restrict__ GU) {
  __shared__ double red[8][256];
  for (int m = threadIdx.x; m <= mmax; m += blockDim.x) {
    if (m == s) continue;
    GQ[(size_t)m * M] = GU[(size_t)m * M] = make_double2(0.0, 0.0);
    GQ[(size_t)m * M + M / 2] = GU[(size_t)m * M + M / 2] = make_double2(0.0, 0.0);
  }
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // Q(0), U(0), Q(pi), U(pi), re and im each
  if (s <= mmax) {
    const int mb = s * (2 * L + 1 - s) / 2;
    const double sgs = (s & 1) ? -1.0 : 1.0;
    for (int l = s + threadIdx.x; l <= L; l += blockDim.x) {
      const double nl = sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846));
      const double2 g = glm[mb + l], c = clm[mb + l];
      const double gi = s == 0 ? 0.0 : g.y, ci = s == 0 ? 0.0 : c.y;
      double W = 0.5 * nl, X = -0.5 * nl;
      v[0] += g.x * W - ci * X;
      v[1] += gi * W + c.x * X;
      v[2] += c.x * W + gi * X;
      v[3] += ci * W - g.x * X;
      W = X = 0.5 * nl * sgs * (((l + s) & 1) ? -1.0 : 1.0);
      v[4] += g.x * W - ci * X;
      v[5] += gi * W + c.x * X;
      v[6] += c.x * W + gi * X;
      v[7] += ci * W - g.x * X;
    }
  }
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int k = 0; k < 8; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0 && s <= mmax) {
    double2* rq = GQ + (size_t)s * M;
    double2* ru = GU + (size_t)s * M;
    rq[0] = make_double2(red[0][0], red[1][0]);
    ru[0] = make_double2(red[2][0], red[3][0]);
    rq[M / 2] = make_double2(red[4][0], red[5][0]);
    ru[M / 2] = make_double2(red[6][0], red[7][0]);
  }
}

// shared-memory slots of the adjoint: per warp, 4 degrees x 32 lanes x 8
// floats (G and C as float pairs); a lane's 8 floats start at a multiple of
// 12 floats (two conflict-free 16-byte stores per quarter warp) and the
// degrees 392 = 8 (mod 32) floats apart, so that the transpose read (lane t:
// degree t/4, float pair t mod 4 of one lane) hits distinct banks per half warp
constexpr int SPIN_SL = 12, SPIN_SD = 32 * SPIN_SL + 8;

// adjoint: from the theta spectra HQ, HU (inverse theta FFT done), fold with
// the spin sign, then per degree G += pv U1 + nv U2, C += i (nv V2 - pv V1)
// over the warp's ring pairs; partial rows [(blk * 4 + pass)][nalm] as float
// pairs, G in pg and C in pc
__global__ void __launch_bounds__(128) spin_adj_k(SpinArgs a, const double2* __restrict__ HQ,
                                                  const double2* __restrict__ HU, float4* __restrict__ pg,
                                                  float4* __restrict__ pc, int64_t nalm) {
  __shared__ __align__(16) float slots[4][4 * SPIN_SD];
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= (a.mmax + 1) * a.bpm) return;
  float* sl = slots[threadIdx.x >> 5];
  const int m = it / a.bpm, blk = it % a.bpm;
  const int L = a.lmax, s = a.s, M = a.M;
  const int l0 = m > s ? m : s;
  if (l0 > L) return;
  const int mb = mbase_of(L, m);
  const double hs = (s & 1) ? -0.5 : 0.5;  // (-1)^s / 2
  const double sgd = ((m + s) & 1) ? -1.0 : 1.0;
  const double mp = __ldg(a.st_mant + 2 * m), mn = __ldg(a.st_mant + 2 * m + 1);
  const int ep = __ldg(a.st_exp + 2 * m), en = __ldg(a.st_exp + 2 * m + 1);
  const int abp = __ldg(a.st_ab + 2 * m), abn = __ldg(a.st_ab + 2 * m + 1);
  const double2* hq = HQ + (size_t)m * M;
  const double2* hu = HU + (size_t)m * M;
  // transpose-read role of this lane: float pair k = t mod 16 (degree k / 4,
  // component k mod 4: G re, G im, C re, C im) summed over lanes 16 h .. 16 h + 15
  const int tk = lane & 15, th = lane >> 4, td = tk >> 2, tc = tk & 3;
  const unsigned kp = a.keep ? a.keep[it] : 15u;
  for (int pass = 0; pass < 4; ++pass) {
    // a skipped pass adds nothing: its partial rows keep the zeros of the plan
    if (!(kp & (1u << pass))) continue;
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + pass * 32 + lane;
    const bool valid = jn <= a.npairs;
    const Ring rg = ring_of(valid ? jn : 1, M);
    // D^dagger with the spin sign: F(theta) = H(theta) + (-1)^(m+s) H(2 pi - theta)
    double2 qn = make_double2(0, 0), qs = qn, un = qn, us = qn;
    if (valid) {
      const int js = M / 2 - jn;
      qn = make_double2(hq[jn].x + sgd * hq[M - jn].x, hq[jn].y + sgd * hq[M - jn].y);
      un = make_double2(hu[jn].x + sgd * hu[M - jn].x, hu[jn].y + sgd * hu[M - jn].y);
      if (js != jn) {
        qs = make_double2(hq[js].x + sgd * hq[M - js].x, hq[js].y + sgd * hq[M - js].y);
        us = make_double2(hu[js].x + sgd * hu[M - js].x, hu[js].y + sgd * hu[M - js].y);
      }
    }
    // B+ = H^Q + i H^U, B- = H^Q - i H^U at each ring; U1 +- = (B+_n +- B-_s) / 2,
    // U2 +- = (-1)^s (B-_n +- B+_s) / 2 as float pairs
    const double2 bpn = make_double2(qn.x - un.y, qn.y + un.x), bmn = make_double2(qn.x + un.y, qn.y - un.x);
    const double2 bps = make_double2(qs.x - us.y, qs.y + us.x), bms = make_double2(qs.x + us.y, qs.y - us.x);
    float4 u1p, u1m, u2p, u2m;
    df_split(0.5 * (bpn.x + bms.x), u1p.x, u1p.y);
    df_split(0.5 * (bpn.y + bms.y), u1p.z, u1p.w);
    df_split(0.5 * (bpn.x - bms.x), u1m.x, u1m.y);
    df_split(0.5 * (bpn.y - bms.y), u1m.z, u1m.w);
    df_split(hs * (bmn.x + bps.x), u2p.x, u2p.y);
    df_split(hs * (bmn.y + bps.y), u2p.z, u2p.w);
    df_split(hs * (bmn.x - bps.x), u2m.x, u2m.y);
    df_split(hs * (bmn.y - bps.y), u2m.z, u2m.w);
    SChain P, N;
    schain_init(P, mp, ep, abp >> 16, abp & 0xffff, rg.ch, rg.sh);
    schain_init(N, mn, en, abn >> 16, abn & 0xffff, rg.ch, rg.sh);
    float4* og = pg + (size_t)(blk * 4 + pass) * nalm + mb;
    float4* oc = pc + (size_t)(blk * 4 + pass) * nalm + mb;
    for (int l = l0; l <= L; ++l) {
      if (l > l0) {
        const double A = __ldg(a.A + mb + l), Ab = __ldg(a.Ab + mb + l), C = __ldg(a.Cc + mb + l);
        schain_step(P, fma(A, rg.x, Ab), C);
        schain_step(N, fma(A, rg.x, -Ab), C);
      }
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f), w = g;
      if (P.E == 0 || N.E == 0) {
        float ph, pl, nh, nl;
        split_q(sval(P), ph, pl);
        split_q(sval(N), nh, nl);
        const bool even = ((l + m + s) & 1) == 0;
        const float4 x1 = even ? u1p : u1m, x2 = even ? u2p : u2m;  // G: p = (-1)^(l+m+s)
        const float4 y1 = even ? u1m : u1p, y2 = even ? u2m : u2p;  // C: -p
        cmac(g, x1, ph, pl);
        cmac(g, x2, nh, nl);
        cmac(w, y2, nh, nl);
        cmac(w, y1, -ph, -pl);
      }
      // C = i w = (-w.im, w.re)
      const int slot = (l - l0) & 3;
      float4* dst = reinterpret_cast<float4*>(sl + slot * SPIN_SD + lane * SPIN_SL);
      dst[0] = g;
      dst[1] = make_float4(-w.z, -w.w, w.x, w.y);
      if (slot == 3 || l == L) {
        __syncwarp();
        const float* src = sl + td * SPIN_SD + (16 * th) * SPIN_SL + 2 * tc;
        float sh = 0.f, slo = 0.f;
#pragma unroll 4
        for (int i = 0; i < 16; ++i) {
          const float2 v = *reinterpret_cast<const float2*>(src + i * SPIN_SL);
          df_add(sh, slo, v.x, v.y);
        }
        const float oh = __shfl_xor_sync(FULL, sh, 16), ol = __shfl_xor_sync(FULL, slo, 16);
        df_add(sh, slo, oh, ol);
        const int deg = l - slot + td;
        if (th == 0 && deg <= l) {
          float4* row = tc < 2 ? og : oc;
          reinterpret_cast<float2*>(row + deg)[tc & 1] = make_float2(sh, slo);
        }
        __syncwarp();
      }
    }
  }
}

// c_lm = sum over the partial rows in a fixed order (float pairs), plus the
// poles (order s); entries with l < s are 0, Im of the m = 0 entries is 0
__global__ void spin_adj_reduce_k(const float4* __restrict__ pg, const float4* __restrict__ pc, int nrows,
                                  int64_t nalm, int L, int mmax, int s, int M, const double2* __restrict__ HQ,
                                  const double2* __restrict__ HU, double2* __restrict__ og, double2* __restrict__ oc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  // (l, m) of packed index i: order m holds l = m..L at m (2L + 1 - m) / 2 + l,
  // so m is the largest order whose first entry m (2L + 1 - m) / 2 + m is <= i
  int lo = 0, hi = mmax;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int64_t)mid * (2 * L + 1 - mid) / 2 + mid <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int m = lo;
  const int l = (int)(i - (int64_t)m * (2 * L + 1 - m) / 2);
  double g0 = 0, g1 = 0, c0 = 0, c1 = 0;
  if (l >= s) {
    float4 sg = make_float4(0.f, 0.f, 0.f, 0.f), sc = sg;
    for (int r = 0; r < nrows; ++r) {
      const float4 a = pg[(size_t)r * nalm + i], b = pc[(size_t)r * nalm + i];
      df_add(sg.x, sg.y, a.x, a.y);
      df_add(sg.z, sg.w, a.z, a.w);
      df_add(sc.x, sc.y, b.x, b.y);
      df_add(sc.z, sc.w, b.z, b.w);
    }
    g0 = df_value(sg.x, sg.y);
    g1 = df_value(sg.z, sg.w);
    c0 = df_value(sc.x, sc.y);
    c1 = df_value(sc.z, sc.w);
    if (m == s) {
      // poles: F^Q, F^U at theta = 0 (index 0) and theta = pi (index M / 2),
      // each taken once (no fold partner)
      const double nl = sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846));
      const double sgs = (s & 1) ? -1.0 : 1.0;
      const double2 q0 = HQ[(size_t)m * M], u0 = HU[(size_t)m * M];
      const double2 qp = HQ[(size_t)m * M + M / 2], up = HU[(size_t)m * M + M / 2];
      double W = 0.5 * nl, X = -0.5 * nl;
      g0 += W * q0.x - X * u0.y;
      g1 += W * q0.y + X * u0.x;
      c0 += W * u0.x + X * q0.y;
      c1 += W * u0.y - X * q0.x;
      W = X = 0.5 * nl * sgs * (((l + s) & 1) ? -1.0 : 1.0);
      g0 += W * qp.x - X * up.y;
      g1 += W * qp.y + X * up.x;
      c0 += W * up.x + X * qp.y;
      c1 += W * up.y - X * qp.x;
    }
  }
  if (m == 0) g1 = c1 = 0.0;
  og[i] = make_double2(g0, g1);
  oc[i] = make_double2(c0, c1);
}

// value = p * 2^e
struct XN {
  double p;
  int e;
};
XN xn(double p, int e) {
  XN r{0.0, 0};
  if (p == 0.0) return r;
  int k;
  r.p = std::frexp(p, &k);
  r.e = e + k;
  return r;
}

SpinArgs spin_args(nusht_plan_t p) {
  SpinArgs a;
  a.lmax = p->lmax;
  a.mmax = p->mmax;
  a.M = p->sz.M;
  a.npairs = p->leg.npairs;
  a.bpm = p->leg.blocks_per_m;
  a.s = p->opts.spin;
  a.A = p->spin.A;
  a.Ab = p->spin.Ab;
  a.Cc = p->spin.C;
  a.st_mant = p->spin.st_mant;
  a.st_exp = p->spin.st_exp;
  a.st_ab = p->spin.st_ab;
  a.keep = p->spin.keep;
  return a;
}

}  // namespace

// plan time: recurrence tables, start values, ring maps and partial rows
int spin_setup(nusht_plan_t p, cudaStream_t s) {
  const int L = p->lmax, mmax = p->mmax, sp = p->opts.spin;
  const int64_t nalm = p->nalm;
  std::vector<double> A(nalm, 0.0), Ab(nalm, 0.0), C(nalm, 0.0);
  std::vector<double> mant(2 * (mmax + 1), 0.0);
  std::vector<int> ex(2 * (mmax + 1), 0), ab(2 * (mmax + 1), 0);
  const double sgs = (sp & 1) ? -1.0 : 1.0;
  for (int m = 0; m <= mmax; ++m) {
    const int64_t mb = (int64_t)m * (2 * L + 1 - m) / 2;
    const int l0 = std::max(m, sp);
    const double dm = m, ds = sp;
    for (int l = l0 + 1; l <= L; ++l) {
      const double dl = l;
      const double den = std::sqrt((dl * dl - dm * dm) * (dl * dl - ds * ds));
      A[mb + l] = std::sqrt((2.0 * dl + 1.0) * (2.0 * dl - 1.0)) * dl / den;
      Ab[mb + l] = A[mb + l] * dm * ds / (dl * (dl - 1.0));
      const double dl1 = dl - 1.0;
      C[mb + l] = std::sqrt((2.0 * dl + 1.0) / (2.0 * dl - 3.0)) * dl *
                  std::sqrt((dl1 * dl1 - dm * dm) * (dl1 * dl1 - ds * ds)) / (dl1 * den);
    }
    // start values at l0: (-1)^s sqrt((2 l0 + 1)/(4 pi)) d^l0_{m, mp} for mp = -s (lambda+), +s (lambda-)
    for (int sign = 0; sign < 2; ++sign) {
      const int mpv = sign == 0 ? -sp : sp;
      int k, a, b;
      bool neg;
      if (m >= sp) {  // d^l0_{l0, mp} = (-1)^(l0 - mp) sqrt(C(2 l0, l0 + mp)) c^(l0 + mp) s^(l0 - mp)
        k = l0 + mpv;
        a = l0 + mpv;
        b = l0 - mpv;
        neg = ((l0 - mpv) & 1) != 0;
      } else if (mpv > 0) {  // d^l0_{m, l0} = sqrt(C(2 l0, l0 + m)) c^(l0 + m) s^(l0 - m)
        k = l0 + m;
        a = l0 + m;
        b = l0 - m;
        neg = false;
      } else {  // d^l0_{m, -l0} = (-1)^(l0 + m) sqrt(C(2 l0, l0 - m)) c^(l0 - m) s^(l0 + m)
        k = l0 - m;
        a = l0 - m;
        b = l0 + m;
        neg = ((l0 + m) & 1) != 0;
      }
      XN r = xn(1.0, 0);
      for (int i = 1; i <= k; ++i) r = xn(r.p * ((double)(2 * l0 - k + i) / (double)i), r.e);
      if (r.e & 1) {
        r.p *= 2.0;
        r.e -= 1;
      }
      r = xn(std::sqrt(r.p) * std::sqrt((2.0 * l0 + 1.0) / (4.0 * M_PI)) * sgs * (neg ? -1.0 : 1.0), r.e / 2);
      mant[2 * m + sign] = r.p;
      ex[2 * m + sign] = r.e;
      ab[2 * m + sign] = (a << 16) | b;
    }
  }
  SpinTables& t = p->spin;
  NUSHT_TRY(dev_alloc((void**)&t.A, nalm * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.Ab, nalm * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.C, nalm * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.st_mant, mant.size() * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.st_exp, ex.size() * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.st_ab, ab.size() * 4, &p->bytes));
  NUSHT_CUDA(cudaMemcpy(t.A, A.data(), nalm * 8, cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(t.Ab, Ab.data(), nalm * 8, cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(t.C, C.data(), nalm * 8, cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(t.st_mant, mant.data(), mant.size() * 8, cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(t.st_exp, ex.data(), ex.size() * 4, cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(t.st_ab, ab.data(), ab.size() * 4, cudaMemcpyHostToDevice));
  const size_t gbytes = (size_t)(mmax + 1) * p->sz.M * sizeof(double2);
  NUSHT_TRY(dev_alloc((void**)&t.GQ, gbytes, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.GU, gbytes, &p->bytes));
  NUSHT_CUDA(cudaMemsetAsync(t.GQ, 0, gbytes, s));
  NUSHT_CUDA(cudaMemsetAsync(t.GU, 0, gbytes, s));
  NUSHT_TRY(dev_alloc((void**)&t.ap, nalm * sizeof(float4), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.am, nalm * sizeof(float4), &p->bytes));
  t.nrows = 4 * p->leg.blocks_per_m;
  const size_t pbytes = (size_t)t.nrows * nalm * sizeof(float4);
  NUSHT_TRY(dev_alloc((void**)&t.pg, pbytes, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.pc, pbytes, &p->bytes));
  NUSHT_CUDA(cudaMemsetAsync(t.pg, 0, pbytes, s));
  NUSHT_CUDA(cudaMemsetAsync(t.pc, 0, pbytes, s));
  // the passes that carry a value above 2^-300 (the probe runs with keep unset)
  const int nitems = (mmax + 1) * p->leg.blocks_per_m;
  unsigned char* keep = nullptr;
  NUSHT_TRY(dev_alloc((void**)&keep, (size_t)nitems, &p->bytes));
  spin_probe_k<<<(nitems + 3) / 4, 128, 0, s>>>(spin_args(p), keep);
  NUSHT_CUDA(cudaGetLastError());
  t.keep = keep;
  NUSHT_CUDA(cudaStreamSynchronize(s));
  return NUSHT_OK;
}

void spin_free(nusht_plan_t p) {
  SpinTables& t = p->spin;
  for (void* q : {(void*)t.A, (void*)t.Ab, (void*)t.C, (void*)t.st_mant, (void*)t.st_exp, (void*)t.st_ab,
                  (void*)t.GQ, (void*)t.GU, (void*)t.ap, (void*)t.am, (void*)t.pg, (void*)t.pc, (void*)t.keep})
    dev_free(q);
  t = SpinTables();
}

int spin_legendre_synth(nusht_plan_t p, const void* glm, const void* clm, cudaStream_t s) {
  const SpinArgs a = spin_args(p);
  const int nitems = (p->mmax + 1) * p->leg.blocks_per_m;
  spin_scale_k<<<(int)((p->nalm + 255) / 256), 256, 0, s>>>((const double2*)glm, (const double2*)clm, p->nalm,
                                                             p->lmax, p->opts.spin, p->spin.ap, p->spin.am);
  spin_synth_k<<<(nitems + 3) / 4, 128, 0, s>>>(a, p->spin.ap, p->spin.am, p->spin.GQ, p->spin.GU);
  spin_poles_k<<<1, 256, 0, s>>>(p->lmax, p->mmax, p->opts.spin, p->sz.M, (const double2*)glm, (const double2*)clm,
                                 p->spin.GQ, p->spin.GU);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int spin_legendre_adjoint(nusht_plan_t p, void* glm, void* clm, cudaStream_t s) {
  const SpinArgs a = spin_args(p);
  const int nitems = (p->mmax + 1) * p->leg.blocks_per_m;
  spin_adj_k<<<(nitems + 3) / 4, 128, 0, s>>>(a, p->spin.GQ, p->spin.GU, p->spin.pg, p->spin.pc, p->nalm);
  spin_adj_reduce_k<<<(int)((p->nalm + 255) / 256), 256, 0, s>>>(p->spin.pg, p->spin.pc, p->spin.nrows, p->nalm,
                                                                 p->lmax, p->mmax, p->opts.spin, p->sz.M,
                                                                 p->spin.GQ, p->spin.GU, (double2*)glm,
                                                                 (double2*)clm);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

}  // namespace nusht
