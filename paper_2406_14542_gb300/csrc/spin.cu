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
// recurrences in l run in FP64 (sqrt((2l+1)/4pi) d^l_{m,-s} and d^l_{m,s}):
//   v_l = A_l (x - b_l) v_{l-1} - C_l v_{l-2},  b_l = -/+ m s / (l (l-1)),
// three FP64 operations per step with the plan-time tables A_l, A_l m s /
// (l (l-1)) and C_l; started at l0 = max(m, s) from
// sqrt(C(2 l0, k)) cos^a(theta/2) sin^b(theta/2) with an integer exponent
// beside the mantissa (values below 2^-300 are carried scaled and not
// accumulated, as in legendre.cu).  Since d^l_{m,-s}(pi - theta) =
// (-1)^(l+m) d^l_{m,s}(theta), the two chains at theta give both rings: W
// changes by (-1)^(l+m+s) and X by -(-1)^(l+m+s) at pi - theta.  One ring
// pair per lane, four passes per warp over an item's 128 ring pairs; every
// (order, ring block) is processed (the spin-0 polar-skip list does not
// apply to spin functions).  The adjoint reduces each degree's products over
// the warp's lanes and writes one partial row per (ring block, pass).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

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

// synthesis: the Q and U ring maps, doubled, [m][M] complex each
__global__ void __launch_bounds__(128) spin_synth_k(SpinArgs a, const double2* __restrict__ glm,
                                                    const double2* __restrict__ clm, double2* __restrict__ GQ,
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
  for (int pass = 0; pass < 4; ++pass) {
    const int jn = 1 + blk * LEG_PAIRS_PER_WARP + pass * 32 + lane;
    const bool valid = jn <= a.npairs;
    const Ring rg = ring_of(valid ? jn : 1, M);
    SChain P, N;
    schain_init(P, mp, ep, abp >> 16, abp & 0xffff, rg.ch, rg.sh);
    schain_init(N, mn, en, abn >> 16, abn & 0xffff, rg.ch, rg.sh);
    // sums by the parity p = (-1)^(l+m+s): Q (W part, X part), U (W part, X part)
    double2 qw[2] = {{0, 0}, {0, 0}}, qx[2] = {{0, 0}, {0, 0}}, uw[2] = {{0, 0}, {0, 0}}, ux[2] = {{0, 0}, {0, 0}};
    auto acc = [&](int l, int par) {
      const double pv = sval(P), nv = sval(N);
      const double W = 0.5 * (pv + sgs * nv), X = 0.5 * (pv - sgs * nv);
      const double2 g = __ldg(glm + mb + l), c = __ldg(clm + mb + l);
      const double gi = m == 0 ? 0.0 : g.y, ci = m == 0 ? 0.0 : c.y;
      // G W + i C X  and  C W - i G X
      qw[par].x = fma(g.x, W, qw[par].x);
      qw[par].y = fma(gi, W, qw[par].y);
      qx[par].x = fma(-ci, X, qx[par].x);
      qx[par].y = fma(c.x, X, qx[par].y);
      uw[par].x = fma(c.x, W, uw[par].x);
      uw[par].y = fma(ci, W, uw[par].y);
      ux[par].x = fma(gi, X, ux[par].x);
      ux[par].y = fma(-g.x, X, ux[par].y);
    };
    acc(l0, (l0 + m + s) & 1);
    for (int l = l0 + 1; l <= L; ++l) {
      const double A = __ldg(a.A + mb + l), Ab = __ldg(a.Ab + mb + l), C = __ldg(a.Cc + mb + l);
      schain_step(P, fma(A, rg.x, Ab), C);   // lambda+: d^l_{m,-s}, b_l = -m s / (l (l-1))
      schain_step(N, fma(A, rg.x, -Ab), C);  // lambda-: d^l_{m,s}
      acc(l, (l + m + s) & 1);
    }
    if (!valid) continue;
    // north: all four sums; south: W parts times p, X parts times -p
    const int js = M / 2 - jn;
    const double2 fqn = make_double2(qw[0].x + qw[1].x + qx[0].x + qx[1].x, qw[0].y + qw[1].y + qx[0].y + qx[1].y);
    const double2 fun = make_double2(uw[0].x + uw[1].x + ux[0].x + ux[1].x, uw[0].y + uw[1].y + ux[0].y + ux[1].y);
    const double2 fqs = make_double2(qw[0].x - qw[1].x - qx[0].x + qx[1].x, qw[0].y - qw[1].y - qx[0].y + qx[1].y);
    const double2 fus = make_double2(uw[0].x - uw[1].x - ux[0].x + ux[1].x, uw[0].y - uw[1].y - ux[0].y + ux[1].y);
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// adjoint: from the theta spectra HQ, HU (inverse theta FFT done), fold with
// the spin sign, then per degree G += W S^Q + i X D^U, C += W S^U - i X D^Q
// over the warp's ring pairs; partial rows [(blk * 4 + pass)][nalm], G then C
__global__ void __launch_bounds__(128) spin_adj_k(SpinArgs a, const double2* __restrict__ HQ,
                                                  const double2* __restrict__ HU, double2* __restrict__ pg,
                                                  double2* __restrict__ pc, int64_t nalm) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= (a.mmax + 1) * a.bpm) return;
  const int m = it / a.bpm, blk = it % a.bpm;
  const int L = a.lmax, s = a.s, M = a.M;
  const int l0 = m > s ? m : s;
  if (l0 > L) return;
  const int mb = mbase_of(L, m);
  const double sgs = (s & 1) ? -1.0 : 1.0;
  const double sgd = ((m + s) & 1) ? -1.0 : 1.0;
  const double mp = __ldg(a.st_mant + 2 * m), mn = __ldg(a.st_mant + 2 * m + 1);
  const int ep = __ldg(a.st_exp + 2 * m), en = __ldg(a.st_exp + 2 * m + 1);
  const int abp = __ldg(a.st_ab + 2 * m), abn = __ldg(a.st_ab + 2 * m + 1);
  const double2* hq = HQ + (size_t)m * M;
  const double2* hu = HU + (size_t)m * M;
  for (int pass = 0; pass < 4; ++pass) {
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
    // parity p = +1 / -1: W multiplies north + p south, X multiplies north - p south
    const double2 sq[2] = {make_double2(qn.x + qs.x, qn.y + qs.y), make_double2(qn.x - qs.x, qn.y - qs.y)};
    const double2 dq[2] = {make_double2(qn.x - qs.x, qn.y - qs.y), make_double2(qn.x + qs.x, qn.y + qs.y)};
    const double2 su[2] = {make_double2(un.x + us.x, un.y + us.y), make_double2(un.x - us.x, un.y - us.y)};
    const double2 du[2] = {make_double2(un.x - us.x, un.y - us.y), make_double2(un.x + us.x, un.y + us.y)};
    SChain P, N;
    schain_init(P, mp, ep, abp >> 16, abp & 0xffff, rg.ch, rg.sh);
    schain_init(N, mn, en, abn >> 16, abn & 0xffff, rg.ch, rg.sh);
    double2* og = pg + (size_t)(blk * 4 + pass) * nalm + mb;
    double2* oc = pc + (size_t)(blk * 4 + pass) * nalm + mb;
    for (int l = l0; l <= L; ++l) {
      if (l > l0) {
        const double A = __ldg(a.A + mb + l), Ab = __ldg(a.Ab + mb + l), C = __ldg(a.Cc + mb + l);
        schain_step(P, fma(A, rg.x, Ab), C);
        schain_step(N, fma(A, rg.x, -Ab), C);
      }
      const int par = (l + m + s) & 1;
      const double pv = sval(P), nv = sval(N);
      const double W = 0.5 * (pv + sgs * nv), X = 0.5 * (pv - sgs * nv);
      // G: W S^Q + i X D^U;  C: W S^U - i X D^Q
      double gr = W * sq[par].x - X * du[par].y, gi = W * sq[par].y + X * du[par].x;
      double cr = W * su[par].x + X * dq[par].y, ci = W * su[par].y - X * dq[par].x;
      gr = warp_sum(gr);
      gi = warp_sum(gi);
      cr = warp_sum(cr);
      ci = warp_sum(ci);
      if (lane == 0) {
        og[l] = make_double2(gr, gi);
        oc[l] = make_double2(cr, ci);
      }
    }
  }
}

// c_lm = sum over the partial rows in a fixed order, plus the poles (order s);
// entries with l < s are 0, Im of the m = 0 entries is 0
__global__ void spin_adj_reduce_k(const double2* __restrict__ pg, const double2* __restrict__ pc, int nrows,
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
    for (int r = 0; r < nrows; ++r) {
      const double2 a = pg[(size_t)r * nalm + i], b = pc[(size_t)r * nalm + i];
      g0 += a.x;
      g1 += a.y;
      c0 += b.x;
      c1 += b.y;
    }
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
  t.nrows = 4 * p->leg.blocks_per_m;
  const size_t pbytes = (size_t)t.nrows * nalm * sizeof(double2);
  NUSHT_TRY(dev_alloc((void**)&t.pg, pbytes, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&t.pc, pbytes, &p->bytes));
  NUSHT_CUDA(cudaMemsetAsync(t.pg, 0, pbytes, s));
  NUSHT_CUDA(cudaMemsetAsync(t.pc, 0, pbytes, s));
  NUSHT_CUDA(cudaStreamSynchronize(s));
  return NUSHT_OK;
}

void spin_free(nusht_plan_t p) {
  SpinTables& t = p->spin;
  for (void* q : {(void*)t.A, (void*)t.Ab, (void*)t.C, (void*)t.st_mant, (void*)t.st_exp, (void*)t.st_ab,
                  (void*)t.GQ, (void*)t.GU, (void*)t.pg, (void*)t.pc})
    dev_free(q);
  t = SpinTables();
}

int spin_legendre_synth(nusht_plan_t p, const void* glm, const void* clm, cudaStream_t s) {
  const SpinArgs a = spin_args(p);
  const int nitems = (p->mmax + 1) * p->leg.blocks_per_m;
  spin_synth_k<<<(nitems + 3) / 4, 128, 0, s>>>(a, (const double2*)glm, (const double2*)clm, p->spin.GQ,
                                                p->spin.GU);
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
