// batch.cu -- many transforms of uneven lmax and point counts in one plan
// (mixed precision: FP64 recurrence, FP32 contraction / FFT / NUFFT; FP64:
// the contraction split into bf16 slices on the tensor cores, the members'
// FFTs and NUFFT in double-float, see the split-contraction section below).
//
// Members are grouped into buckets of up to 64 transforms that share one
// Clenshaw-Curtis ring set (the one of the bucket's largest lmax: more rings
// than a member needs keep its DFS coefficients exact, Sec. 2.2).  Within a
// bucket the FP64 recurrence is run once per (ring pair, l, m) and contracted
// with every member's coefficients at once, i.e. per order m a dense product
//   synthesis: F[ring][member] = sum_l P[ring][l] A[l][member]
//   adjoint:   C[l][member]    = sum_rings P[ring][l] S[ring][member]
// tiled through shared memory (CUDA-core FP32 FMA, FP32 accumulation).
// Each member keeps its own NUFFT state (points, fine grid, 2D FFTs) and its
// theta spectrum lives in a slice of the bucket's buffer, so the theta FFT is
// one batched cuFFT call per bucket.  The grouping minimises a cost model of
// the recurrence (per triple of the bucket's largest lmax) plus the
// contraction (per triple and member column).
//
// The whole stage sequence of one direction is captured once into a CUDA
// graph (re-captured when the caller's buffers change) and replayed.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "nusht_internal.cuh"
#include "recurrence.cuh"
#include "dfloat.cuh"
#include "ozsplit.cuh"

struct nusht_batch_s;

namespace nusht {
namespace {

using namespace rec;

constexpr int BK_MAXB = 64;          // members per bucket
constexpr int BK_COLS = 2 * BK_MAXB; // (re, im) columns of the contraction
constexpr int BS_PAIRS = 64;         // synthesis: ring pairs per block
constexpr int BS_LC = 16;            // synthesis: degrees per chunk
constexpr int BA_TILE = 256;         // adjoint: ring pairs per recurrence tile (one per thread)
constexpr int BA_LC = 32;            // adjoint: degrees per chunk
constexpr int BA_SUB = 32;           // adjoint: ring pairs per staged S tile

struct BucketArgs {
  int lmax, M, npairs, B;
  const double* c;
  const int8_t* dshift;
  const double* cm;
  const double* ring_x;
  const double* ring_s;
  const int* memberL;
};

__device__ __forceinline__ int idx_lm(int L, int l, int m) { return m * (2 * L + 1 - m) / 2 + l; }

// atb[(l,m)][slot] = a_slot(l, m) * Ahat(l, m) (zero where the member has no such (l, m))
__global__ void bucket_scale_k(int L, int B, const int* __restrict__ memberL, const float2* const* __restrict__ alm,
                               const double* __restrict__ ahat, float2* __restrict__ atb) {
  const int m = blockIdx.y;
  const int slot = threadIdx.x & (BK_MAXB - 1);
  const int l = m + blockIdx.x * 4 + (threadIdx.x >> 6);
  if (l > L) return;
  const int i = idx_lm(L, l, m);
  float2 v = make_float2(0.f, 0.f);
  if (slot < B) {
    const int Lb = memberL[slot];
    if (l <= Lb && m <= Lb) {  // single precision suffices for complex64 coefficients
      const float2 a = alm[slot][idx_lm(Lb, l, m)];
      const float ah = (float)ahat[i];
      v.x = a.x * ah;
      v.y = m == 0 ? 0.f : a.y * ah;
    }
  }
  atb[(size_t)i * BK_MAXB + slot] = v;
}

// synthesis: block = (order m, 64 ring pairs); 64 owner threads run the FP64
// recurrence chunk by chunk into shared memory, all 256 threads contract
// (64 pairs x 16 degrees) x (16 degrees x 128 columns) with even/odd degree
// parities kept apart (north = E + O, south = E - O).
__global__ void __launch_bounds__(256) bucket_synth_k(BucketArgs a, const int* __restrict__ items, int nitems,
                                                      const float2* __restrict__ atb, float2* __restrict__ G) {
  __shared__ __align__(16) float Ps[BS_LC][BS_PAIRS];
  __shared__ __align__(16) float As[BS_LC][BK_COLS];
  const int it = blockIdx.x;
  if (it >= nitems) return;
  const int v = items[it];
  const int m = v >> 16, tile = v & 0xffff;
  const int L = a.lmax;
  const int mb = idx_lm(L, 0, m);  // packed base of order m
  const int t = threadIdx.x;
  Chain ch;
  ch.valid = false;
  ch.E = 0;
  ch.q1 = ch.q2 = ch.x = 0.0;
  if (t < BS_PAIRS) chain_init(ch, a, m, 1 + tile * BS_PAIRS + t);
  const int pg = t >> 4, cg = t & 15;
  float accE[4][8], accO[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) accE[r][c] = accO[r][c] = 0.f;
  for (int l0 = m; l0 <= L; l0 += BS_LC) {
    if (t < BS_PAIRS) {
#pragma unroll
      for (int j = 0; j < BS_LC; ++j) {
        const int l = l0 + j;
        float q = 0.f;
        if (l <= L) {
          if (l > m) chain_step(ch, __ldg(a.c + mb + l), (int)__ldg(a.dshift + mb + l));
          if (ch.valid && ch.E == 0) q = to_f32(ch.q1);
        }
        Ps[j][t] = q;
      }
    }
    for (int e = t; e < BS_LC * BK_COLS / 4; e += 256) {
      const int r = e >> 5, c4 = e & 31;
      const int l = l0 + r;
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
      if (l <= L) val = reinterpret_cast<const float4*>(atb + (size_t)(mb + l) * BK_MAXB)[c4];
      reinterpret_cast<float4*>(&As[r][0])[c4] = val;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < BS_LC; ++j) {
      const float4 p = *reinterpret_cast<const float4*>(&Ps[j][pg * 4]);
      const float4 a0 = *reinterpret_cast<const float4*>(&As[j][cg * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[j][cg * 8 + 4]);
      const float pr[4] = {p.x, p.y, p.z, p.w};
      const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (j & 1)
            accO[r][c] = fmaf(pr[r], ar[c], accO[r][c]);
          else
            accE[r][c] = fmaf(pr[r], ar[c], accE[r][c]);
        }
    }
    __syncthreads();
  }
  const int M = a.M;
  const float sg = (m & 1) ? -1.f : 1.f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int jn = 1 + tile * BS_PAIRS + pg * 4 + r;
    if (jn > a.npairs) continue;
    const int js = M / 2 - jn;
#pragma unroll
    for (int ss = 0; ss < 4; ++ss) {
      const int slot = cg * 4 + ss;
      if (slot >= a.B || m > a.memberL[slot]) continue;
      const float2 fn = make_float2(accE[r][2 * ss] + accO[r][2 * ss], accE[r][2 * ss + 1] + accO[r][2 * ss + 1]);
      const float2 fs = make_float2(accE[r][2 * ss] - accO[r][2 * ss], accE[r][2 * ss + 1] - accO[r][2 * ss + 1]);
      float2* row = G + ((size_t)slot * (L + 1) + m) * M;
      row[jn] = fn;
      row[M - jn] = make_float2(sg * fn.x, sg * fn.y);
      if (js != jn) {
        row[js] = fs;
        row[M - js] = make_float2(sg * fs.x, sg * fs.y);
      }
    }
  }
}

// F_0 at the poles for every member (m > 0 pole entries stay 0)
__global__ void bucket_poles_k(int L, int M, const int* __restrict__ memberL, const float2* const* __restrict__ alm,
                               const double* __restrict__ pole_norm, float2* __restrict__ G) {
  __shared__ double sn[256], ss[256];
  const int slot = blockIdx.x;
  const int Lb = memberL[slot];
  double n = 0.0, s = 0.0;
  for (int l = threadIdx.x; l <= Lb; l += blockDim.x) {
    const double v = (double)alm[slot][l].x * pole_norm[l];
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
    float2* row = G + (size_t)slot * (L + 1) * M;
    row[0] = make_float2((float)sn[0], 0.f);
    row[M / 2] = make_float2((float)ss[0], 0.f);
  }
}

// adjoint, first step for the tensor-core path: the same fold, written as
// the contraction's B tiles BA[m][table tile][group of 8 ring pairs]: rows =
// 128 columns (member, re/im), k = the group's 8 ring pairs, E then O, each
// split into TF32 hi and lo.  Block = (32 ring pairs, order m).
__global__ void __launch_bounds__(256) bucket_fold_ba_k(int L, int M, int npairs, int B, int ntiles,
                                                        const int* __restrict__ memberL,
                                                        const float2* __restrict__ Gt,
                                                        unsigned char* __restrict__ BA);

// adjoint, first step: D^dagger fold into S[m][pair][E|O][slot (re, im)].
// Block = (32 ring pairs, order m); each warp reads one member's spectrum
// row for the 32 pairs contiguously (4 coalesced runs), the block transposes
// through shared memory and writes 32 contiguous S rows.
constexpr int FOLD_PAIRS = 32;
__global__ void __launch_bounds__(256) bucket_fold_k(int L, int M, int npairs, int B,
                                                     const int* __restrict__ memberL, const float2* __restrict__ Gt,
                                                     float* __restrict__ S) {
  __shared__ float2 sE[FOLD_PAIRS][BK_MAXB + 1], sO[FOLD_PAIRS][BK_MAXB + 1];
  const int p0 = blockIdx.x * FOLD_PAIRS, m = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = p0 + lane;
  const float sg = (m & 1) ? -1.f : 1.f;
  for (int slot = warp; slot < BK_MAXB; slot += 8) {
    float2 se = make_float2(0.f, 0.f), so = make_float2(0.f, 0.f);
    if (slot < B && m <= memberL[slot] && p < npairs) {
      const int jn = p + 1, js = M / 2 - jn;
      const float2* row = Gt + ((size_t)slot * (L + 1) + m) * M;
      const float2 g0 = row[jn], g1 = row[M - jn];
      const float2 fn = make_float2(g0.x + sg * g1.x, g0.y + sg * g1.y);
      float2 fs = make_float2(0.f, 0.f);
      if (js != jn) {
        const float2 h0 = row[js], h1 = row[M - js];
        fs = make_float2(h0.x + sg * h1.x, h0.y + sg * h1.y);
      }
      se = make_float2(fn.x + fs.x, fn.y + fs.y);
      so = make_float2(fn.x - fs.x, fn.y - fs.y);
    }
    sE[lane][slot] = se;
    sO[lane][slot] = so;
  }
  __syncthreads();
  // 32 rows of 2 x 64 float2
  for (int e = threadIdx.x; e < FOLD_PAIRS * 2 * BK_MAXB; e += 256) {
    const int r = e / (2 * BK_MAXB), c = e % (2 * BK_MAXB);
    if (p0 + r >= npairs) continue;
    float2* out = reinterpret_cast<float2*>(S + ((size_t)m * npairs + p0 + r) * 2 * BK_COLS);
    out[c] = c < BK_MAXB ? sE[r][c] : sO[r][c - BK_MAXB];
  }
}

// adjoint: block = order m with all its ring pairs; each thread owns NT
// chains (pairs t, t+256, ...) kept in registers across degree chunks; per
// chunk of 32 degrees the recurrence tile P[32][256] goes to shared memory
// and C[32 degrees][128 columns] += P S is accumulated over the pairs with S
// staged 32 pairs at a time.  The block owns its outputs: no atomics.
template <int NT>
__global__ void __launch_bounds__(256) bucket_adj_k(BucketArgs a, const int* __restrict__ mlist, int nm,
                                                    const float* __restrict__ S, float* __restrict__ cacc) {
  extern __shared__ __align__(16) float smem[];
  float* Ps = smem;                    // [BA_LC][BA_TILE]
  float* Ss = smem + BA_LC * BA_TILE;  // [BA_SUB][2 * BK_COLS]
  if ((int)blockIdx.x >= nm) return;
  const int m = mlist[blockIdx.x];
  const int L = a.lmax;
  const int mb = idx_lm(L, 0, m);  // packed base of order m
  const int t = threadIdx.x;
  const int npairs = a.npairs;
  Chain ch[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    ch[k].valid = false;
    ch[k].E = 0;
    ch[k].q1 = ch[k].q2 = ch[k].x = 0.0;
    if (k * BA_TILE < npairs) chain_init(ch[k], a, m, 1 + k * BA_TILE + t);
  }
  const int jj = t >> 4, cg = t & 15;  // rows 2jj (even) and 2jj+1 (odd), columns cg*8..cg*8+7
  for (int l0 = m; l0 <= L; l0 += BA_LC) {
    float acc0[8], acc1[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc0[c] = acc1[c] = 0.f;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      if (k * BA_TILE >= npairs) continue;
#pragma unroll 4
      for (int j = 0; j < BA_LC; ++j) {
        const int l = l0 + j;
        float q = 0.f;
        if (l <= L) {
          if (l > m) chain_step(ch[k], __ldg(a.c + mb + l), (int)__ldg(a.dshift + mb + l));
          if (ch[k].valid && ch[k].E == 0) q = to_f32(ch[k].q1);
        }
        Ps[j * BA_TILE + t] = q;
      }
      __syncthreads();
      for (int sub = 0; sub < BA_TILE / BA_SUB; ++sub) {
        const int pb = k * BA_TILE + sub * BA_SUB;
        if (pb >= npairs) break;
        // stage S[m][pb .. pb+31][256 floats]
        const float4* src = reinterpret_cast<const float4*>(S + ((size_t)m * npairs + pb) * 2 * BK_COLS);
        for (int e = t; e < BA_SUB * 2 * BK_COLS / 4; e += 256) {
          const int r = e / (2 * BK_COLS / 4);
          float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
          if (pb + r < npairs) val = src[e];
          reinterpret_cast<float4*>(Ss)[e] = val;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < BA_SUB; ++r) {
          const float pe = Ps[(2 * jj) * BA_TILE + sub * BA_SUB + r];
          const float po = Ps[(2 * jj + 1) * BA_TILE + sub * BA_SUB + r];
          const float* srow = Ss + r * 2 * BK_COLS;
          const float4 e0 = *reinterpret_cast<const float4*>(srow + cg * 8);
          const float4 e1 = *reinterpret_cast<const float4*>(srow + cg * 8 + 4);
          const float4 o0 = *reinterpret_cast<const float4*>(srow + BK_COLS + cg * 8);
          const float4 o1 = *reinterpret_cast<const float4*>(srow + BK_COLS + cg * 8 + 4);
          acc0[0] = fmaf(pe, e0.x, acc0[0]);
          acc0[1] = fmaf(pe, e0.y, acc0[1]);
          acc0[2] = fmaf(pe, e0.z, acc0[2]);
          acc0[3] = fmaf(pe, e0.w, acc0[3]);
          acc0[4] = fmaf(pe, e1.x, acc0[4]);
          acc0[5] = fmaf(pe, e1.y, acc0[5]);
          acc0[6] = fmaf(pe, e1.z, acc0[6]);
          acc0[7] = fmaf(pe, e1.w, acc0[7]);
          acc1[0] = fmaf(po, o0.x, acc1[0]);
          acc1[1] = fmaf(po, o0.y, acc1[1]);
          acc1[2] = fmaf(po, o0.z, acc1[2]);
          acc1[3] = fmaf(po, o0.w, acc1[3]);
          acc1[4] = fmaf(po, o1.x, acc1[4]);
          acc1[5] = fmaf(po, o1.y, acc1[5]);
          acc1[6] = fmaf(po, o1.z, acc1[6]);
          acc1[7] = fmaf(po, o1.w, acc1[7]);
        }
        __syncthreads();
      }
    }
    const int le = l0 + 2 * jj, lo = le + 1;
    if (le <= L) {
      float4* dst = reinterpret_cast<float4*>(cacc + (size_t)(mb + le) * BK_COLS + cg * 8);
      dst[0] = make_float4(acc0[0], acc0[1], acc0[2], acc0[3]);
      dst[1] = make_float4(acc0[4], acc0[5], acc0[6], acc0[7]);
    }
    if (lo <= L) {
      float4* dst = reinterpret_cast<float4*>(cacc + (size_t)(mb + lo) * BK_COLS + cg * 8);
      dst[0] = make_float4(acc1[0], acc1[1], acc1[2], acc1[3]);
      dst[1] = make_float4(acc1[4], acc1[5], acc1[6], acc1[7]);
    }
  }
}

// ---------------------------------------------------------------------------
// Table path.  The recurrence values depend only on the bucket's rings, not
// on the coefficients or the points, so the plan runs the FP64 recurrence
// once and keeps q = Pbar / Ahat (as float, 0 in the scaled phase) in HBM:
// P[item][l - m][64 pairs] for every kept (order, 64-pair tile).  Each call
// is then a pure FP32 contraction streaming that table (synthesis) or its
// transpose (adjoint); the double-buffered tiles arrive by cp.async.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) bucket_ptab_k(BucketArgs a, const int* __restrict__ items,
                                                     const int64_t* __restrict__ offs, int nitems,
                                                     float* __restrict__ P) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  const int v = items[it];
  const int m = v >> 16, tile = v & 0xffff;
  const int L = a.lmax;
  const int mb = idx_lm(L, 0, m);
  Chain ch[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) chain_init(ch[k], a, m, 1 + tile * BS_PAIRS + k * 32 + lane);
  float* out = P + offs[it];
  for (int l = m; l <= L; ++l) {
    const bool step = l > m;
    const double c = step ? __ldg(a.c + mb + l) : 0.0;
    const int rs = step ? (int)__ldg(a.dshift + mb + l) : 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (step) chain_step(ch[k], c, rs);
      out[(size_t)(l - m) * BS_PAIRS + k * 32 + lane] = (ch[k].valid && ch[k].E == 0) ? to_f32(ch[k].q1) : 0.f;
    }
  }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? 16 : 0;  // 0 source bytes: the 16 destination bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// synthesis from the table: block = kept item (m, 64 pairs)
__global__ void __launch_bounds__(256) bucket_synth_tab_k(BucketArgs a, const int* __restrict__ items,
                                                          const int64_t* __restrict__ offs, int nitems,
                                                          const float* __restrict__ P, const float2* __restrict__ atb,
                                                          float2* __restrict__ G) {
  __shared__ __align__(16) float Ps[2][BS_LC][BS_PAIRS];
  __shared__ __align__(16) float As[2][BS_LC][BK_COLS];
  const int it = blockIdx.x;
  if (it >= nitems) return;
  const int v = items[it];
  const int m = v >> 16, tile = v & 0xffff;
  const int L = a.lmax;
  const int mb = idx_lm(L, 0, m);
  const int t = threadIdx.x;
  const float* Pi = P + offs[it];
  const int nrow = L - m + 1;
  const int nchunk = (nrow + BS_LC - 1) / BS_LC;
  auto load = [&](int ck, int buf) {
    // P rows: 16 x 64 floats = 256 x 16 B; A rows: 16 x 128 floats = 512 x 16 B
    {
      const int r = t >> 4, c4 = t & 15;
      const int row = ck * BS_LC + r;
      const bool ok = row < nrow;
      cp_async16(&Ps[buf][r][c4 * 4], Pi + (size_t)(ok ? row : 0) * BS_PAIRS + c4 * 4, ok);
    }
    for (int e = t; e < BS_LC * BK_COLS / 4; e += 256) {
      const int r = e >> 5, c4 = e & 31;
      const int row = ck * BS_LC + r;
      const bool ok = row < nrow;
      cp_async16(&As[buf][r][c4 * 4],
                 reinterpret_cast<const float*>(atb + (size_t)(mb + m + (ok ? row : 0)) * BK_MAXB) + c4 * 4, ok);
    }
    cp_async_commit();
  };
  // thread tile: 8 pairs (warp-uniform, so P reads broadcast) x 4 columns
  const int pg = t >> 5, cg = t & 31;
  float accE[8][4], accO[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) accE[r][c] = accO[r][c] = 0.f;
  load(0, 0);
  for (int ck = 0; ck < nchunk; ++ck) {
    const int buf = ck & 1;
    if (ck + 1 < nchunk) {
      load(ck + 1, buf ^ 1);
      cp_async_wait1();
    } else {
      cp_async_wait0();
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < BS_LC; ++j) {
      const float4 p0 = *reinterpret_cast<const float4*>(&Ps[buf][j][pg * 8]);
      const float4 p1 = *reinterpret_cast<const float4*>(&Ps[buf][j][pg * 8 + 4]);
      const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][j][cg * 4]);
      const float pr[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
      const float ar[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (j & 1)
            accO[r][c] = fmaf(pr[r], ar[c], accO[r][c]);
          else
            accE[r][c] = fmaf(pr[r], ar[c], accE[r][c]);
        }
    }
    __syncthreads();
  }
  const int M = a.M;
  const float sg = (m & 1) ? -1.f : 1.f;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int jn = 1 + tile * BS_PAIRS + pg * 8 + r;
    if (jn > a.npairs) continue;
    const int js = M / 2 - jn;
#pragma unroll
    for (int ss = 0; ss < 2; ++ss) {
      const int slot = cg * 2 + ss;
      if (slot >= a.B || m > a.memberL[slot]) continue;
      const float2 fn = make_float2(accE[r][2 * ss] + accO[r][2 * ss], accE[r][2 * ss + 1] + accO[r][2 * ss + 1]);
      const float2 fs = make_float2(accE[r][2 * ss] - accO[r][2 * ss], accE[r][2 * ss + 1] - accO[r][2 * ss + 1]);
      float2* row = G + ((size_t)slot * (L + 1) + m) * M;
      row[jn] = fn;
      row[M - jn] = make_float2(sg * fn.x, sg * fn.y);
      if (js != jn) {
        row[js] = fs;
        row[M - js] = make_float2(sg * fs.x, sg * fs.y);
      }
    }
  }
}

// adjoint from the table: block = (order m, 128 degrees); loops over the
// order's kept tiles (items[mfirst[m] .. mfirst[m+1]) ), staging P
// transposed (Pt[pair][degree]) and S[64 pairs][E|O x 128]; thread tile =
// 16 consecutive degrees (warp-uniform) x 4 columns; the block owns its
// 128 x 128 outputs
constexpr int AT_LC = 128;
constexpr int AT_PAD = AT_LC + 4;  // Pt row stride (floats), 16-byte aligned rows
__global__ void __launch_bounds__(256) bucket_adj_tab_k(BucketArgs a, const int* __restrict__ items,
                                                        const int64_t* __restrict__ offs,
                                                        const int* __restrict__ mfirst, const int2* __restrict__ work,
                                                        int nwork, const float* __restrict__ P,
                                                        const float* __restrict__ S, float* __restrict__ cacc) {
  extern __shared__ __align__(16) float smem[];
  float* Pt = smem;                       // [64 pairs][AT_PAD]
  float* Ss = smem + BS_PAIRS * AT_PAD;   // [64 pairs][2 * BK_COLS]
  if ((int)blockIdx.x >= nwork) return;
  const int2 wk = work[blockIdx.x];
  const int m = wk.x, l0 = wk.y;  // degrees l0 .. l0 + 127
  const int L = a.lmax;
  const int mb = idx_lm(L, 0, m);
  const int t = threadIdx.x;
  const int jr = t >> 5, cg = t & 31;  // degrees jr*16 .. +15, columns cg*4 .. +3
  float acc[16][4];
#pragma unroll
  for (int i = 0; i < 16; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
  const int i0 = mfirst[m], i1 = mfirst[m + 1];
  const int nrow = L - m + 1;
  for (int it = i0; it < i1; ++it) {
    const int tile = items[it] & 0xffff;
    const float* Pi = P + offs[it];
    const float* Sp = S + ((size_t)m * a.npairs + (size_t)tile * BS_PAIRS) * 2 * BK_COLS;
    for (int e = t; e < BS_PAIRS * 2 * BK_COLS / 4; e += 256) {
      const int pr = e >> 6;
      const bool ok = tile * BS_PAIRS + pr < a.npairs;
      cp_async16(Ss + e * 4, Sp + (ok ? e * 4 : 0), ok);
    }
    cp_async_commit();
    // P rows (l0 - m) .. +127, transposed into Pt[pair][row]
    {
      const int pair = t & 63;
#pragma unroll 4
      for (int r = t >> 6; r < AT_LC; r += 4) {
        const int row = l0 - m + r;
        Pt[pair * AT_PAD + r] = row < nrow ? Pi[(size_t)row * BS_PAIRS + pair] : 0.f;
      }
    }
    cp_async_wait0();
    __syncthreads();
#pragma unroll 4
    for (int pr = 0; pr < BS_PAIRS; ++pr) {
      const float* prow = Pt + pr * AT_PAD + jr * 16;
      const float4 q0 = *reinterpret_cast<const float4*>(prow);
      const float4 q1 = *reinterpret_cast<const float4*>(prow + 4);
      const float4 q2 = *reinterpret_cast<const float4*>(prow + 8);
      const float4 q3 = *reinterpret_cast<const float4*>(prow + 12);
      const float q[16] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                           q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
      const float* srow = Ss + pr * 2 * BK_COLS;
      const float4 se = *reinterpret_cast<const float4*>(srow + cg * 4);
      const float4 so = *reinterpret_cast<const float4*>(srow + BK_COLS + cg * 4);
      const float e4[4] = {se.x, se.y, se.z, se.w};
      const float o4[4] = {so.x, so.y, so.z, so.w};
#pragma unroll
      for (int i = 0; i < 16; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(q[i], (i & 1) ? o4[c] : e4[c], acc[i][c]);
    }
    __syncthreads();
  }
  // degree l0 + jr*16 + i has parity i & 1 (l0 - m is a multiple of 128)
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int l = l0 + jr * 16 + i;
    if (l <= L)
      *reinterpret_cast<float4*>(cacc + (size_t)(mb + l) * BK_COLS + cg * 4) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core contractions (tcgen05.mma kind::tf32, accumulators in tensor
// memory).  Both directions are D[128 x 128] += A[128 x 8] B[128 x 8]^T per
// MMA into two accumulators: D_E collects the even l - m terms and D_O the
// odd ones, so no MMA multiplies zeros.
//   synthesis: rows = 128 ring pairs, K = 8 degrees of one parity,
//              B columns = the bucket's (member, re/im) coefficients;
//   adjoint:   rows = 128 degrees of one parity, K = 8 ring pairs,
//              B columns = the folded spectrum S_E or S_O.
// Precision.  Each FP32 operand is split into x = hi + lo, hi = x rounded to
// TF32 (cvt.rna), lo = x - hi exactly (|lo| <= 2^-11 |x|); D accumulates
// hi*hi + hi*lo + lo*hi, so a product keeps about 22 significant bits with
// an unbiased error.  The tensor core's own accumulation adds with reduced,
// truncating alignment, an error that grows with the number of MMAs folded
// into one accumulator; so the chunks are taken in groups of tcg (2, 4 or 8:
// the bucket's degree chunks per partial accumulation, picked by the
// autotuner with opts.tune, else 4), each group
// into one of two partial accumulator sets (TMEM columns 0..255 and
// 256..511, alternating), and every finished group is added in FP32 with
// round-to-nearest into per-thread registers while the tensor core runs the
// next group.
// Data flow.  A chunk (one K step of both parities) is 8 operand tiles of
// 4 KB in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per
// core matrix; K-adjacent core matrices 128 B apart, 8-row groups 256 B
// apart): A_E hi, A_E lo, A_O hi, A_O lo, then the same for B.  Operands are
// split and laid out before the contraction, so that the contraction moves
// them only with the bulk copy engine: the A tiles at plan time from the
// recurrence table (one copy in synthesis order, one in adjoint order), the
// B tiles per call by the kernels that produce the coefficients (scaling by
// Ahat) and the folded spectrum.  Warp roles: one thread issues two 16 KB
// cp.async.bulk copies per chunk into a ring of T6_NBUF buffers (mbarrier
// transaction counts), one thread waits for them and issues the six MMAs,
// committing to the buffer's "empty" barrier and, at the end of a group, to
// the group's barrier; 16 warps fold each finished group (64 accumulator
// columns of 32 TMEM lanes per warp) and arrive on the set's "free" barrier
// that the MMA thread waits for before refilling it.  One block per SM (512
// TMEM columns).  Every wait is bounded (one second of device time); a block
// that gives up flags the others, waits (bounded) for its copies in flight,
// sets *status and still frees its tensor memory.  test_giveup = 1 (a test
// hook, NUSHT_TEST_TC_GIVEUP=1 at plan time) gives the MMA thread's first
// wait for data a limit of zero polls, so that it runs out before any MMA is
// issued and the give-up path runs.
// ---------------------------------------------------------------------------
constexpr int TC_TILE = 128 * 8 * 4;              // one 128 x 8 fp32 operand tile
constexpr int TC_CHUNK = 8 * TC_TILE;             // AEh AEl AOh AOl BEh BEl BOh BOl
constexpr int TC_G = 4;                           // default chunks per partial accumulation
constexpr uint32_t TC_COLS = 512;                 // two partial sets of D_E, D_O
// instruction descriptor: D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9,
// 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}

// shared-memory matrix descriptor: start >> 4, leading byte offset (next core
// matrix along K) 128 B, stride byte offset (next 8-row group) 256 B,
// descriptor version 1 at bit 46, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Bounded wait for the phase `parity` of an mbarrier: gives up (false) after
// TC_WAIT_NS of device time or max_polls polls, or, when `stop` is given, as
// soon as *stop is set (another role of the block gave up).  Waits that drain
// asynchronous work before the block exits pass no `stop`.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* stop = nullptr,
                                          int max_polls = 1 << 30) {
  const unsigned long long t0 = gtimer();
  for (int it = 0; it < max_polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && (gtimer() - t0 > TC_WAIT_NS || (stop && *stop))) return false;
  }
  return false;
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
      : "memory");
}

// 16 consecutive columns of this warp's 32 TMEM lanes (no wait)
__device__ __forceinline__ void tc_ld16(uint32_t addr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr)
      : "memory");
}

// one operand row (8 values) of one tile pair (hi at `tile`, lo at tile + 1)
__device__ __forceinline__ void tc_store(unsigned char* buf, int tile, int row, const float (&v)[8]) {
  const int base = (row >> 3) * 256 + (row & 7) * 16;
  float h[8], l[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t hb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v[k]));
    h[k] = __uint_as_float(hb);
    l[k] = v[k] - h[k];
  }
  unsigned char* ph = buf + tile * TC_TILE + base;
  unsigned char* pl = ph + TC_TILE;
  *reinterpret_cast<float4*>(ph) = make_float4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<float4*>(ph + 128) = make_float4(h[4], h[5], h[6], h[7]);
  *reinterpret_cast<float4*>(pl) = make_float4(l[0], l[1], l[2], l[3]);
  *reinterpret_cast<float4*>(pl + 128) = make_float4(l[4], l[5], l[6], l[7]);
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
}

constexpr int T6_NBUF = 6;
constexpr int T6_FOLD_WARPS = 16;
constexpr int T6_THREADS = 32 * (T6_FOLD_WARPS + 2);
constexpr int T6_HALF = TC_CHUNK / 2;  // A or B half of a chunk (16 KB)
constexpr int T6_SMEM = T6_NBUF * TC_CHUNK + 256;
static_assert(128 * 129 * 4 <= T6_NBUF * TC_CHUNK, "epilogue exchange fits the chunk buffers");

struct T6Bars {
  uint64_t full[T6_NBUF], empty[T6_NBUF], gdone[2], gfree[2];
  uint32_t tslot;
  int abort;
};

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// bulk copy global -> shared of `bytes` (multiple of 16, both ends 16-byte
// aligned), completing on the barrier's transaction count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}

// Contraction of one block.  Synthesis (ADJ = false): block = (order m, 128
// ring pairs), chunks = 16 degrees, A = PA + aoff[block], B = BS + bsoff[m].
// Adjoint: block = (order m, 256 degrees from r0), chunks = (kept table tile,
// group of 8 ring pairs), A = PT + aoff[block], B = BA[m][tile][group].
template <bool ADJ>
__global__ void __launch_bounds__(T6_THREADS, 1) bucket_tc_k(BucketArgs a, int nblk, const int* __restrict__ titems,
                                                             const int2* __restrict__ work,
                                                             const int64_t* __restrict__ aoff,
                                                             const int64_t* __restrict__ bsoff,
                                                             const int* __restrict__ items,
                                                             const int* __restrict__ mfirst, int ntiles,
                                                             const unsigned char* __restrict__ Atab,
                                                             const unsigned char* __restrict__ Bbuf,
                                                             float2* __restrict__ G, float* __restrict__ cacc,
                                                             int* __restrict__ status, int test_giveup, int tcg) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  T6Bars* bars = reinterpret_cast<T6Bars*>(tc_smem + T6_NBUF * TC_CHUNK);
  if ((int)blockIdx.x >= nblk || *(volatile int*)status) return;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int L = a.lmax;
  int m, nchunk, u = 0, r0 = 0, i0 = 0;
  if (!ADJ) {
    const int v = titems[blockIdx.x];
    m = v >> 16;
    u = v & 0xffff;
    nchunk = (L - m + 1 + 15) / 16;
  } else {
    const int2 wk = work[blockIdx.x];
    m = wk.x;
    r0 = wk.y;
    i0 = mfirst[m];
    nchunk = (mfirst[m + 1] - i0) * (BS_PAIRS / 8);
  }
  const unsigned char* Asrc = Atab + aoff[blockIdx.x];
  volatile int* abort = &bars->abort;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tslot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int k = 0; k < T6_NBUF; ++k) {
      mbar_init(&bars->full[k], 1);
      mbar_init(&bars->empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&bars->gdone[k], 1);
      mbar_init(&bars->gfree[k], T6_FOLD_WARPS);
    }
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = bars->tslot;
  const int ngroups = (nchunk + tcg - 1) / tcg;
  float acc[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) acc[j] = 0.f;
  if (warp == T6_FOLD_WARPS) {
    if (lane == 0) {  // producer
      int issued = 0;
      for (int c = 0; c < nchunk && !*abort; ++c) {
        const int s = c % T6_NBUF;
        if (c >= T6_NBUF && !mbar_wait(smem_u32(&bars->empty[s]), (uint32_t)((c / T6_NBUF - 1) & 1), abort)) {
          *abort = 1;
          break;
        }
        unsigned char* dst = tc_smem + s * TC_CHUNK;
        const unsigned char* bsrc;
        if (ADJ) {
          const int tile = items[i0 + (c >> 3)] & 0xffff;
          bsrc = Bbuf + ((size_t)(m * ntiles + tile) * 8 + (c & 7)) * T6_HALF;
        } else {
          bsrc = Bbuf + bsoff[m] + (size_t)c * T6_HALF;
        }
        mbar_expect_tx(&bars->full[s], TC_CHUNK);
        bulk_g2s(dst, Asrc + (size_t)c * T6_HALF, T6_HALF, &bars->full[s]);
        bulk_g2s(dst + T6_HALF, bsrc, T6_HALF, &bars->full[s]);
        issued = c + 1;
      }
      if (*abort)  // wait (bounded) for the copies still in flight
        for (int c = issued > T6_NBUF ? issued - T6_NBUF : 0; c < issued; ++c)
          mbar_wait(smem_u32(&bars->full[c % T6_NBUF]), (uint32_t)((c / T6_NBUF) & 1));
    }
  } else if (warp == T6_FOLD_WARPS + 1) {
    if (lane == 0) {  // MMA issuer
      int last = -1;
      for (int c = 0; c < nchunk && !*abort; ++c) {
        const int s = c % T6_NBUF;
        if (!mbar_wait(smem_u32(&bars->full[s]), (uint32_t)((c / T6_NBUF) & 1), abort,
                       (test_giveup && c == 0) ? 0 : (1 << 30))) {
          *abort = 1;
          break;
        }
        const int g = c / tcg, set = g & 1;
        if (c % tcg == 0 && g >= 2 &&
            !mbar_wait(smem_u32(&bars->gfree[set]), (uint32_t)(((g - 2) >> 1) & 1), abort)) {
          *abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sb = smem_u32(tc_smem + s * TC_CHUNK);
        const uint32_t dE = tmem + (uint32_t)(set * 256), dO = dE + 128;
        const uint32_t acc_on = (c % tcg) != 0 ? 1u : 0u;
        tc_mma(dE, tc_desc(sb + 0 * TC_TILE), tc_desc(sb + 4 * TC_TILE), acc_on);
        tc_mma(dE, tc_desc(sb + 0 * TC_TILE), tc_desc(sb + 5 * TC_TILE), 1u);
        tc_mma(dE, tc_desc(sb + 1 * TC_TILE), tc_desc(sb + 4 * TC_TILE), 1u);
        tc_mma(dO, tc_desc(sb + 2 * TC_TILE), tc_desc(sb + 6 * TC_TILE), acc_on);
        tc_mma(dO, tc_desc(sb + 2 * TC_TILE), tc_desc(sb + 7 * TC_TILE), 1u);
        tc_mma(dO, tc_desc(sb + 3 * TC_TILE), tc_desc(sb + 6 * TC_TILE), 1u);
        tc_commit(&bars->empty[s]);
        if (c % tcg == tcg - 1 || c == nchunk - 1) tc_commit(&bars->gdone[set]);
        last = c;
      }
      // after a give-up, MMAs already issued still write tensor memory: wait
      // (bounded) for the commit that covers them before the block frees it
      if (*abort && last >= 0)
        mbar_wait(smem_u32(&bars->empty[last % T6_NBUF]), (uint32_t)((last / T6_NBUF) & 1));
    }
  } else {  // fold warps: lanes 32 (warp % 4) .., columns 64 (warp / 4) .. of a partial set
    const uint32_t tview = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 64);
    for (int g = 0; g < ngroups; ++g) {
      const int set = g & 1;
      const bool okw = mbar_wait(smem_u32(&bars->gdone[set]), (uint32_t)((g >> 1) & 1), abort);
      if (!__all_sync(0xffffffffu, okw)) {
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 16) {
        uint32_t r[16];
        tc_ld16(tview + (uint32_t)(set * 256 + c0), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(r[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->gfree[set]);
    }
  }
  __syncthreads();
  const bool ok = !*abort && nchunk > 0;
  if (warp < T6_FOLD_WARPS && ok) {
    const int lrow = (warp & 3) * 32 + lane;  // TMEM lane: ring pair (synthesis) / degree pair (adjoint)
    const int cb = warp >> 2;                 // column block of 64: 0, 1 = E; 2, 3 = O
    const int mb = idx_lm(L, 0, m);
    if (!ADJ) {
      // warps with O sums hand them over through shared memory (row stride
      // 129: conflict-free); the E warps form north = E + O, south = E - O
      float* xs = reinterpret_cast<float*>(tc_smem);
      if (cb >= 2)
#pragma unroll
        for (int j = 0; j < 64; ++j) xs[lrow * 129 + (cb - 2) * 64 + j] = acc[j];
      asm volatile("bar.sync 1, %0;" ::"n"(32 * T6_FOLD_WARPS) : "memory");
      if (cb < 2) {
        const int M = a.M;
        const float sg = (m & 1) ? -1.f : 1.f;
        const int jn = 1 + u * 128 + lrow;
        const int js = M / 2 - jn;
        if (jn <= a.npairs) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {  // static acc[] indices
            const int slot = cb * 32 + q;
            if (slot >= a.B || m > a.memberL[slot]) continue;
            const float oe = xs[lrow * 129 + 2 * slot], oi = xs[lrow * 129 + 2 * slot + 1];
            float2* rowp = G + ((size_t)slot * (L + 1) + m) * M;
            const float ee = acc[2 * q], ei = acc[2 * q + 1];
            const float2 fn = make_float2(ee + oe, ei + oi);
            rowp[jn] = fn;
            rowp[M - jn] = make_float2(sg * fn.x, sg * fn.y);
            if (js != jn) {
              const float2 fs = make_float2(ee - oe, ei - oi);
              rowp[js] = fs;
              rowp[M - js] = make_float2(sg * fs.x, sg * fs.y);
            }
          }
        }
      }
    } else {
      const int l = m + r0 + 2 * lrow + (cb >> 1);
      if (l <= L) {
        float* dst = cacc + (size_t)(mb + l) * BK_COLS + (cb & 1) * 64;
#pragma unroll
        for (int j = 0; j < 64; j += 4)
          *reinterpret_cast<float4*>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
      }
    }
  }
  if (!ok && nchunk > 0 && t == 0) atomicExch(status, 1);
  tc_teardown(tmem);
}

// Plan time: A tiles of the synthesis (rows = 128 ring pairs of tiles 2u,
// 2u + 1; k = 8 degrees of one parity per chunk of 16) from the table P.
__global__ void __launch_bounds__(256) tc_build_pa_k(const float* __restrict__ P, const int* __restrict__ titems,
                                                     const longlong2* __restrict__ toffs,
                                                     const int64_t* __restrict__ aoff, int L,
                                                     unsigned char* __restrict__ PA) {
  const int it = blockIdx.y, c = blockIdx.x;
  const int m = titems[it] >> 16;
  const int nrow = L - m + 1;
  if (16 * c >= nrow) return;
  const int row0 = threadIdx.x & 127, par = threadIdx.x >> 7;
  const longlong2 of = toffs[it];
  const long long off = row0 < 64 ? of.x : of.y;
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int r = 16 * c + 2 * k + par;
    v[k] = (off >= 0 && r < nrow) ? P[off + (size_t)r * BS_PAIRS + (row0 & 63)] : 0.f;
  }
  unsigned char* dst = PA + aoff[it] + (size_t)c * T6_HALF;
  tc_store(dst, 2 * par, row0, v);
}

// Plan time: A tiles of the adjoint (rows = 128 degrees of one parity from
// r0; k = 8 ring pairs of a kept tile per chunk) from the table P.
__global__ void __launch_bounds__(256) tc_build_pt_k(const float* __restrict__ P, const int* __restrict__ items,
                                                     const int64_t* __restrict__ offs,
                                                     const int* __restrict__ mfirst, const int2* __restrict__ work,
                                                     const int64_t* __restrict__ aoff, int L,
                                                     unsigned char* __restrict__ PT) {
  const int w = blockIdx.y, c = blockIdx.x;
  const int2 wk = work[w];
  const int m = wk.x, r0 = wk.y;
  const int i0 = mfirst[m], i1 = mfirst[m + 1];
  if (c >= (i1 - i0) * (BS_PAIRS / 8)) return;
  const int it = i0 + (c >> 3), j = c & 7;
  const int nrow = L - m + 1;
  const int row0 = threadIdx.x & 127, par = threadIdx.x >> 7;
  const int r = r0 + 2 * row0 + par;
  float v[8];
  if (r < nrow) {
    const float* src = P + offs[it] + (size_t)r * BS_PAIRS + 8 * j;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = src[k];
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 0.f;
  }
  unsigned char* dst = PT + aoff[w] + (size_t)c * T6_HALF;
  tc_store(dst, 2 * par, row0, v);
}

// Per call, synthesis: B tiles (rows = 128 columns (member, re/im), k = 8
// degrees of one parity per chunk) of atilde = a Ahat, straight from the
// members' coefficients.
__global__ void __launch_bounds__(256) tc_scale_bs_k(int L, int B, const int* __restrict__ memberL,
                                                     const float2* const* __restrict__ alm,
                                                     const double* __restrict__ ahat,
                                                     const int64_t* __restrict__ bsoff,
                                                     unsigned char* __restrict__ BS) {
  const int m = blockIdx.y, c = blockIdx.x;
  const int nrow = L - m + 1;
  if (16 * c >= nrow) return;
  const int n = threadIdx.x & 127, par = threadIdx.x >> 7;
  const int slot = n >> 1;
  const int Lb = slot < B ? memberL[slot] : -1;
  const float2* am = slot < B ? alm[slot] : nullptr;
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int l = m + 16 * c + 2 * k + par;
    float x = 0.f;
    if (l <= L && l <= Lb && m <= Lb) {
      const float2 av = am[idx_lm(Lb, l, m)];
      const float ah = (float)ahat[idx_lm(L, l, m)];
      x = (n & 1) ? (m == 0 ? 0.f : av.y * ah) : av.x * ah;
    }
    v[k] = x;
  }
  unsigned char* dst = BS + bsoff[m] + (size_t)c * T6_HALF;
  tc_store(dst, 2 * par, n, v);
}

__global__ void __launch_bounds__(256) bucket_fold_ba_k(int L, int M, int npairs, int B, int ntiles,
                                                        const int* __restrict__ memberL,
                                                        const float2* __restrict__ Gt,
                                                        unsigned char* __restrict__ BA) {
  __shared__ float2 sE[FOLD_PAIRS][BK_MAXB + 1], sO[FOLD_PAIRS][BK_MAXB + 1];
  const int p0 = blockIdx.x * FOLD_PAIRS, m = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = p0 + lane;
  const float sg = (m & 1) ? -1.f : 1.f;
  for (int slot = warp; slot < BK_MAXB; slot += 8) {
    float2 se = make_float2(0.f, 0.f), so = make_float2(0.f, 0.f);
    if (slot < B && m <= memberL[slot] && p < npairs) {
      const int jn = p + 1, js = M / 2 - jn;
      const float2* row = Gt + ((size_t)slot * (L + 1) + m) * M;
      const float2 g0 = row[jn], g1 = row[M - jn];
      const float2 fn = make_float2(g0.x + sg * g1.x, g0.y + sg * g1.y);
      float2 fs = make_float2(0.f, 0.f);
      if (js != jn) {
        const float2 h0 = row[js], h1 = row[M - js];
        fs = make_float2(h0.x + sg * h1.x, h0.y + sg * h1.y);
      }
      se = make_float2(fn.x + fs.x, fn.y + fs.y);
      so = make_float2(fn.x - fs.x, fn.y - fs.y);
    }
    sE[lane][slot] = se;
    sO[lane][slot] = so;
  }
  __syncthreads();
  // 4 groups of 8 ring pairs; thread = (column n, parity)
  const int n = threadIdx.x & 127, par = threadIdx.x >> 7;
  const int slot = n >> 1;
#pragma unroll
  for (int g = 0; g < FOLD_PAIRS / 8; ++g) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float2 x = par ? sO[8 * g + k][slot] : sE[8 * g + k][slot];
      v[k] = (n & 1) ? x.y : x.x;
    }
    const int pg = p0 + 8 * g;  // first ring pair of the group (multiple of 8)
    const int tile = pg / BS_PAIRS, j = (pg % BS_PAIRS) / 8;
    unsigned char* dst = BA + ((size_t)(m * ntiles + tile) * 8 + j) * T6_HALF;
    tc_store(dst, 2 * par, n, v);  // tiles 0..3 of the chunk's B half
  }
}

// member outputs: c_slot(l, m) = Ahat * C + poles (m = 0)
__global__ void bucket_final_k(int L, int M, int B, const int* __restrict__ memberL, const float* __restrict__ cacc,
                               const double* __restrict__ ahat, const double* __restrict__ pole_norm,
                               const float2* __restrict__ Gt, float2* const* __restrict__ out) {
  const int m = blockIdx.y;
  const int slot = threadIdx.x & (BK_MAXB - 1);
  const int l = m + blockIdx.x * 4 + (threadIdx.x >> 6);
  if (l > L || slot >= B) return;
  const int Lb = memberL[slot];
  if (l > Lb || m > Lb) return;
  const int i = idx_lm(L, l, m);
  const float2 v = reinterpret_cast<const float2*>(cacc + (size_t)i * BK_COLS)[slot];
  const float ah = (float)ahat[i];
  float re = v.x * ah, im = v.y * ah;
  if (m == 0) {
    const float2* row = Gt + (size_t)slot * (L + 1) * M;
    const float pn = (float)pole_norm[l];
    re += pn * (row[0].x + ((l & 1) ? -row[M / 2].x : row[M / 2].x));
    im = 0.f;
  }
  out[slot][idx_lm(Lb, l, m)] = make_float2(re, im);
}

// ---------------------------------------------------------------------------
// FP64 batched plans: the split ("Ozaki") contraction on the tensor cores.
//
// The products per order m are those above, but every operand is an exact
// sum of six bf16 slices under one power of two:
//   x = 2^(e - 47) F,  F = round(x 2^(47 - e)) = sum_{i<6} d_i 256^(5 - i),
// with |x| < 2^e and d_i the balanced base-256 digits of F (|d_i| <= 129), so
// the representation error is at most 2^(e - 48).  Slice i is stored as
// d_i 2^(-8 i) (at most 8 significant bits: exact in bf16), and then every
// slice product d_i d_j 2^(-8 (i + j)) is exact in the tensor core's FP32
// product.  The recurrence values Pbar_l^m(theta) are split at plan time
// with one exponent per order (their largest magnitude over the bucket's
// rings and degrees); the coefficients (synthesis) and the folded spectrum
// (adjoint) are split per call with one exponent per (order, member column).
// Synthesis: the 21 slice products with i + j <= 5 go to four accumulators
// per parity, one per level i + j (the last one takes levels 3 to 5):
//   D0 = sum d_0 d_0            integers below 2^14: exact while the sum stays
//                               below 2^24 (1024 full-magnitude terms);
//   D1 = sum over i + j = 1     multiples of 2^-8 below 2^6: exact while below
//                               2^16 (random-sign sums of 1024 terms stay
//                               near 2^11);
//   D2 = sum over i + j = 2     multiples of 2^-16 below 2^-2: exact while
//                               below 2^8;
//   D3 = sum over 3 <= i+j <= 5 rounded FP32 sums, ~2^-8 of D2.
// The tensor core's FP32 accumulation aligns with truncation, so a rounded
// accumulator's error grows with the number of MMAs folded into it; with one
// accumulator for every level from 2 on, that error reached 2^-33 of the
// result at 100 degrees.  With the exact levels apart, the dropped products
// (i + j >= 6), the representation errors and D3's truncation stay near
// 2^-46 of the product of the two operands' scales.  Six slices rather than
// five: the exponent is shared by a whole order, and at low orders the
// largest |Pbar| (near the poles) is 16 times the rms, so five slices (40
// bits) left the bulk of the values with ~36 bits and orders 0 and 1 of the
// adjoint at 1-3e-10 at lmax 2043.  D0 + D1 + D2 + D3 times 2^(eA + eB - 14)
// has the accuracy class of the FP64 recurrence path.
// The rounded level still matters when the leading digits are small: its
// magnitude comes from the full-range lower digits (|d| ~ 128), and its
// truncation bias grows with the MMAs folded into it.  With one exponent per
// order, the rings away from a low order's polar peak have leading digits
// ~16 times below full range, and the adjoint (K = every kept ring pair,
// 960 MMAs into the rounded level) lost 6e-11 to 1.6e-10 at orders 0-10.  So
// the synthesis table takes one exponent per kept item (128 ring pairs: K
// runs over degrees inside one item), and an adjoint block takes a single
// parity: its six levels then each get an accumulator of their own (6 x 64
// TMEM columns), all exact (level s: multiples of 2^-8s below 2^(14 - 8s),
// random-sign sums far from 2^(24 - 8s)), and the split adds ~1e-12 against
// standalone FP64 plans at every order.
//
// Block shapes: M = 128 rows, N = 64 columns (32 members, re / im), K = 16.
//   synthesis: rows = the 128 ring pairs of a kept work item, K = 16 degrees
//              of one parity (a chunk = 32 degrees);
//   adjoint:   rows = 128 degrees of one parity (256 degrees per block),
//              K = 16 ring pairs (8 chunks per kept work item).
// A chunk is 12 A tiles (2 parities x 6 slices, 128 x 16 bf16 = 4 KB each)
// and 12 B tiles (64 x 16 bf16 = 2 KB each) in the no-swizzle K-major
// core-matrix layout of the TF32 kernel above (with 16-bit elements a core
// matrix is 8 rows x 8 values), moved by two cp.async.bulk copies into a
// ring of three 72 KB buffers; one thread issues the 42 MMAs of a chunk.
// The eight accumulators (E, O) x (D0 .. D3) take all 512 TMEM columns.  An
// adjoint block moves half chunks (one parity, 36 KB) through six buffers.  The
// synthesis epilogue forms north = E + O and south = E - O as float pairs
// (the theta FFT of FP64 members reads float pairs); the adjoint's builds
// each coefficient's double from a 64-bit fixed-point sum with integer
// operations, so the FP64 pipe (1/64 of the FP32 rate on GB300) stays idle.
// ---------------------------------------------------------------------------
constexpr int OZ_ATILE = 128 * 16 * 2;          // 128 rows x 16 bf16
constexpr int OZ_BTILE = 64 * 16 * 2;           // 64 rows x 16 bf16
constexpr int OZ_A = 2 * OZ_NS * OZ_ATILE;      // A half of a chunk (48 KB)
constexpr int OZ_B = 2 * OZ_NS * OZ_BTILE;      // B half of a chunk (24 KB)
constexpr int OZ_CHUNK = OZ_A + OZ_B;           // synthesis chunk: both parities
constexpr int OZ_NBUF = 3;
constexpr int OZ_CHUNK_P = OZ_CHUNK / 2;        // adjoint chunk: one parity
constexpr int OZ_NBUF_P = 6;
constexpr int OZ_THREADS = 32 * 6;              // producer, MMA issuer, 4 epilogue warps
constexpr int OZ_SMEM = OZ_NBUF * OZ_CHUNK + 256;
constexpr int OZ_COLS = 128;                    // columns of eB per order (64 members, re / im)
constexpr int OZ_LV = 4;                        // accumulator levels per parity
// instruction descriptor: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9,
// 10-12 = 1), both K-major, N = 64 (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24)
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
static_assert(OZ_SMEM <= 227 * 1024, "three chunk buffers fit in shared memory");
static_assert(OZ_NBUF_P * OZ_CHUNK_P == OZ_NBUF * OZ_CHUNK, "both directions use the same buffer space");

// byte offset of element (row, k) in a K-major tile of 16 bf16 per row
__device__ __forceinline__ int oz_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned long long oz_warp_max(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Plan time, pass 1: the largest |Pbar| of every order over the bucket's
// rings and degrees, and of every kept work item (order m, 128 ring pairs),
// as the bits of a non-negative double (which order like unsigned integers).
// One warp per item.
__global__ void __launch_bounds__(128) oz_amax_k(BucketArgs a, const int* __restrict__ items, int nitems,
                                                 const double* __restrict__ ahat,
                                                 unsigned long long* __restrict__ amax,
                                                 unsigned long long* __restrict__ amax_item) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  const int v = items[it];
  const int m = v >> 16, blk = v & 0xffff;
  const int L = a.lmax;
  const int mb = idx_lm(L, 0, m);
  Chain ch[LEG_K];
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) chain_init(ch[k], a, m, 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane);
  unsigned long long mx = 0;
  for (int l = m; l <= L; ++l) {
    const bool step = l > m;
    const double c = step ? __ldg(a.c + mb + l) : 0.0;
    const int rs = step ? (int)__ldg(a.dshift + mb + l) : 0;
    const double ah = __ldg(ahat + mb + l);
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) {
      if (step) chain_step(ch[k], c, rs);
      if (ch[k].valid && ch[k].E == 0) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(ch[k].q1 * ah) & 0x7fffffffffffffffull;
        mx = b > mx ? b : mx;
      }
    }
  }
  mx = oz_warp_max(mx);
  if (lane == 0) {
    amax_item[it] = mx;
    if (mx) atomicMax(amax + m, mx);
  }
}

// Plan time, pass 2: the slices of Pbar = q Ahat into the synthesis table
// (per item, under the item's exponent eAi: [chunk of 32 degrees][parity]
// [slice] tiles, rows = ring pairs, k = degree / 2 within the chunk) and the
// adjoint table (per order, under the order's exponent eA, since an adjoint
// block sums over all the order's items:
// [block of 256 degrees][item, 16-pair group][parity][slice] tiles, rows =
// degree / 2 within the block, k = ring pair within the group).  The tables
// are zero-filled beforehand; zero values are not written.
__global__ void __launch_bounds__(128) oz_build_k(BucketArgs a, const int* __restrict__ items, int nitems,
                                                  const int* __restrict__ mfirst, const double* __restrict__ ahat,
                                                  const int* __restrict__ eA, const int* __restrict__ eAi,
                                                  const int64_t* __restrict__ soff,
                                                  const int64_t* __restrict__ tbase, unsigned char* __restrict__ AS,
                                                  unsigned char* __restrict__ AT) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= nitems) return;
  const int v = items[it];
  const int m = v >> 16, blk = v & 0xffff;
  const int L = a.lmax;
  const int mb = idx_lm(L, 0, m);
  const int j = it - mfirst[m], nim = mfirst[m + 1] - mfirst[m];
  const int sh = OZ_FB - eA[m], shi = OZ_FB - eAi[it];
  unsigned char* sbase = AS + soff[it];
  unsigned char* tb = AT + tbase[m];
  Chain ch[LEG_K];
#pragma unroll
  for (int k = 0; k < LEG_K; ++k) chain_init(ch[k], a, m, 1 + blk * LEG_PAIRS_PER_WARP + k * 32 + lane);
  for (int l = m; l <= L; ++l) {
    const bool step = l > m;
    const double c = step ? __ldg(a.c + mb + l) : 0.0;
    const int rs = step ? (int)__ldg(a.dshift + mb + l) : 0;
    const double ah = __ldg(ahat + mb + l);
    const int r = l - m, par = r & 1;
    unsigned char* ps = sbase + (size_t)(r >> 5) * OZ_A + par * OZ_NS * OZ_ATILE;
    const int ks = (r & 31) >> 1;
    unsigned char* pt = tb + (size_t)(r >> 8) * 8 * nim * OZ_A + par * OZ_NS * OZ_ATILE;
    const int arow = (r & 255) >> 1;
#pragma unroll
    for (int k = 0; k < LEG_K; ++k) {
      if (step) chain_step(ch[k], c, rs);
      if (!(ch[k].valid && ch[k].E == 0)) continue;
      const double pv = ch[k].q1 * ah;
      const int row = k * 32 + lane;  // ring pair within the item
      const long long Fs = oz_fix_d(pv, shi), Ft = oz_fix_d(pv, sh);
      int d[OZ_NS];
      if (Fs != 0) {
        oz_digits(Fs, d);
        unsigned char* qs = ps + oz_off(row, ks);
#pragma unroll
        for (int i = 0; i < OZ_NS; ++i)
          *reinterpret_cast<unsigned short*>(qs + i * OZ_ATILE) = (unsigned short)oz_bf16(d[i], i);
      }
      if (Ft != 0) {
        oz_digits(Ft, d);
        unsigned char* qt = pt + (size_t)(8 * j + (row >> 4)) * OZ_A + oz_off(arow, row & 15);
#pragma unroll
        for (int i = 0; i < OZ_NS; ++i)
          *reinterpret_cast<unsigned short*>(qt + i * OZ_ATILE) = (unsigned short)oz_bf16(d[i], i);
      }
    }
  }
}

// pack the 8 values of one 16-byte tile row piece (slice i of 8 consecutive k)
__device__ __forceinline__ void oz_put(uint32_t (&w)[OZ_NS][4], int kk, const int (&d)[OZ_NS]) {
#pragma unroll
  for (int i = 0; i < OZ_NS; ++i) {
    const uint32_t b = oz_bf16(d[i], i);
    w[i][kk >> 1] = (kk & 1) ? (w[i][kk >> 1] | (b << 16)) : b;
  }
}

__device__ __forceinline__ void oz_store(unsigned char* dst, const uint32_t (&w)[OZ_NS][4]) {
#pragma unroll
  for (int i = 0; i < OZ_NS; ++i)
    *reinterpret_cast<uint4*>(dst + i * OZ_BTILE) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}

// Per call, synthesis: the members' coefficients of order m (one block per
// order with kept items) as B slices [chunk of 32 degrees][column group]
// [parity][slice] (rows = the group's 64 columns, k = degree / 2 in the
// chunk), with eB[m][col] such that |a| < 2^eB over the order's degrees.
// Coefficients past a member's lmax, and slots without a member, are zero;
// m = 0 coefficients are real.
__global__ void __launch_bounds__(256) oz_bs_k(int L, int B, int ncg, const int* __restrict__ memberL,
                                               const double2* const* __restrict__ alm,
                                               const int* __restrict__ mfirst, const int64_t* __restrict__ boff,
                                               int* __restrict__ eB, unsigned char* __restrict__ Bt) {
  const int m = blockIdx.x;
  if (mfirst[m + 1] == mfirst[m]) return;
  __shared__ double2 sa[32][65];  // [degree in the chunk][member slot]
  __shared__ int se[OZ_COLS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int slot = warp; slot < BK_MAXB; slot += 8) {
    unsigned long long mr = 0, mi = 0;
    const int Ls = slot < B ? memberL[slot] : -1;
    if (m <= Ls) {
      const double2* src = alm[slot] + idx_lm(Ls, 0, m);
      for (int l = m + lane; l <= Ls; l += 32) {
        const double2 v = src[l];
        const unsigned long long br = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffull;
        const unsigned long long bi = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffull;
        mr = br > mr ? br : mr;
        if (m > 0) mi = bi > mi ? bi : mi;
      }
    }
    mr = oz_warp_max(mr);
    mi = oz_warp_max(mi);
    if (lane == 0) {
      se[2 * slot] = oz_exp_of(mr);
      se[2 * slot + 1] = oz_exp_of(mi);
      eB[(size_t)m * OZ_COLS + 2 * slot] = oz_exp_of(mr);
      eB[(size_t)m * OZ_COLS + 2 * slot + 1] = oz_exp_of(mi);
    }
  }
  __syncthreads();
  const int nch = (L - m + 1 + 31) >> 5;
  const int row = t & 63, kh = (t >> 6) & 1, par = t >> 7;
  for (int c = 0; c < nch; ++c) {
    for (int idx = t; idx < 32 * BK_MAXB; idx += 256) {
      const int slot = idx >> 5, li = idx & 31;
      const int l = m + 32 * c + li;
      double2 v = make_double2(0.0, 0.0);
      const int Ls = slot < B ? memberL[slot] : -1;
      if (m <= Ls && l <= Ls) {
        v = alm[slot][idx_lm(Ls, l, m)];
        if (m == 0) v.y = 0.0;
      }
      sa[li][slot] = v;
    }
    __syncthreads();
    for (int cg = 0; cg < ncg; ++cg) {
      const int col = cg * 64 + row, slot = col >> 1;
      const int sh = OZ_FB - se[col];
      uint32_t w[OZ_NS][4];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int li = 2 * (kh * 8 + kk) + par;
        const double x = (col & 1) ? sa[li][slot].y : sa[li][slot].x;
        int d[OZ_NS];
        oz_digits(oz_fix_d(x, sh), d);
        oz_put(w, kk, d);
      }
      oz_store(Bt + boff[m] + ((size_t)c * ncg + cg) * OZ_B + (size_t)par * OZ_NS * OZ_BTILE + (row >> 3) * 256 +
                   kh * 128 + (row & 7) * 16,
               w);
    }
    __syncthreads();
  }
}

// the DFS fold of one ring pair of a member's theta-grid row (float pairs
// hi_re, lo_re, hi_im, lo_im) in 2^k fixed point: e = S_E, o = S_O (re, im)
__device__ __forceinline__ long long oz_fixp(float h, float l, int k) { return oz_fix_f(h, k) + oz_fix_f(l, k); }

// Per call, adjoint: the members' folded spectrum of order m,
//   fn = G[j] + (-1)^m G[M - j],  fs = G[M/2 - j] + (-1)^m G[M/2 + j]  (0 at the equator pair),
//   S_E = fn + fs,  S_O = fn - fs,
// as B slices [item][16-pair group][column group][parity][slice] (rows = the
// group's 64 columns, k = ring pair in the group), with eB[m][col] such that
// |S| < 2^eB over the order's kept ring pairs (from the high words: a value
// may reach the digit 129, which bf16 holds exactly).
__global__ void __launch_bounds__(256) oz_fold_k(int L, int M, int npairs, int B, int ncg,
                                                 const int* __restrict__ memberL, const float4* const* __restrict__ gh,
                                                 const int* __restrict__ items, const int* __restrict__ mfirst,
                                                 const int64_t* __restrict__ boff, int* __restrict__ eB,
                                                 unsigned char* __restrict__ Bt) {
  const int m = blockIdx.x;
  const int i0 = mfirst[m], nim = mfirst[m + 1] - i0;
  if (nim == 0) return;
  __shared__ long long sF[2][16][OZ_COLS + 1];  // [parity][ring pair in the group][column]
  __shared__ int se[OZ_COLS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const float sg = (m & 1) ? -1.f : 1.f;
  for (int slot = warp; slot < BK_MAXB; slot += 8) {
    float mr = 0.f, mi = 0.f;
    const int Ls = slot < B ? memberL[slot] : -1;
    if (m <= Ls) {
      const float4* row = gh[slot] + (size_t)m * M;
      for (int q = lane; q < nim * 128; q += 32) {
        const int jn = 1 + (items[i0 + (q >> 7)] & 0xffff) * 128 + (q & 127);
        if (jn > npairs) continue;
        const int js = M / 2 - jn;
        const float4 g0 = row[jn], g1 = row[M - jn];
        float nr = g0.x + sg * g1.x, ni = g0.z + sg * g1.z, sr = 0.f, si = 0.f;
        if (js != jn) {
          const float4 h0 = row[js], h1 = row[M - js];
          sr = h0.x + sg * h1.x;
          si = h0.z + sg * h1.z;
        }
        mr = fmaxf(mr, fmaxf(fabsf(nr + sr), fabsf(nr - sr)));
        mi = fmaxf(mi, fmaxf(fabsf(ni + si), fabsf(ni - si)));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
      mi = fmaxf(mi, __shfl_xor_sync(0xffffffffu, mi, o));
    }
    if (lane == 0) {
      const int er = mr > 0.f ? ilogbf(mr) + 1 : 0, ei = mi > 0.f ? ilogbf(mi) + 1 : 0;
      se[2 * slot] = er;
      se[2 * slot + 1] = ei;
      eB[(size_t)m * OZ_COLS + 2 * slot] = er;
      eB[(size_t)m * OZ_COLS + 2 * slot + 1] = ei;
    }
  }
  __syncthreads();
  const int row = t & 63, kh = (t >> 6) & 1, par = t >> 7;
  for (int tt = 0; tt < 8 * nim; ++tt) {
    const int blk = items[i0 + (tt >> 3)] & 0xffff;
    for (int idx = t; idx < 16 * BK_MAXB; idx += 256) {
      const int slot = idx >> 4, kk = idx & 15;
      const int jn = 1 + blk * 128 + (tt & 7) * 16 + kk;
      long long er = 0, ei = 0, orr = 0, oi = 0;
      const int Ls = slot < B ? memberL[slot] : -1;
      if (m <= Ls && jn <= npairs) {
        const int kr = OZ_FB - se[2 * slot], ki = OZ_FB - se[2 * slot + 1];
        const float4* rw = gh[slot] + (size_t)m * M;
        const int js = M / 2 - jn;
        const float4 g0 = rw[jn], g1 = rw[M - jn];
        long long nr = oz_fixp(g0.x, g0.y, kr), ni = oz_fixp(g0.z, g0.w, ki);
        long long ur = oz_fixp(g1.x, g1.y, kr), ui = oz_fixp(g1.z, g1.w, ki);
        if (m & 1) {
          ur = -ur;
          ui = -ui;
        }
        nr += ur;
        ni += ui;
        long long sr = 0, si = 0;
        if (js != jn) {
          const float4 h0 = rw[js], h1 = rw[M - js];
          sr = oz_fixp(h0.x, h0.y, kr);
          si = oz_fixp(h0.z, h0.w, ki);
          long long vr = oz_fixp(h1.x, h1.y, kr), vi = oz_fixp(h1.z, h1.w, ki);
          if (m & 1) {
            vr = -vr;
            vi = -vi;
          }
          sr += vr;
          si += vi;
        }
        er = nr + sr;
        ei = ni + si;
        orr = nr - sr;
        oi = ni - si;
      }
      sF[0][kk][2 * slot] = er;
      sF[0][kk][2 * slot + 1] = ei;
      sF[1][kk][2 * slot] = orr;
      sF[1][kk][2 * slot + 1] = oi;
    }
    __syncthreads();
    for (int cg = 0; cg < ncg; ++cg) {
      const int col = cg * 64 + row;
      uint32_t w[OZ_NS][4];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        int d[OZ_NS];
        oz_digits(sF[par][kh * 8 + kk][col], d);
        oz_put(w, kk, d);
      }
      oz_store(Bt + boff[m] + ((size_t)tt * ncg + cg) * OZ_B + (size_t)par * OZ_NS * OZ_BTILE + (row >> 3) * 256 +
                   kh * 128 + (row & 7) * 16,
               w);
    }
    __syncthreads();
  }
}

// synthesis: F_0 at the poles of every member, G[0][0] and G[0][M/2], as float
// pairs (every other pole entry stays 0)
__global__ void __launch_bounds__(256) oz_poles_k(int M, const int* __restrict__ memberL,
                                                  const double2* const* __restrict__ alm,
                                                  const double* __restrict__ pole_norm, float4* const* __restrict__ gp) {
  const int slot = blockIdx.x;
  const int Ls = memberL[slot];
  __shared__ double sn[256], ss[256];
  double n = 0.0, s = 0.0;
  for (int l = threadIdx.x; l <= Ls; l += blockDim.x) {
    const double v = alm[slot][l].x * pole_norm[l];
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
    float h0, l0, h1, l1;
    df_of(sn[0], h0, l0);
    df_of(ss[0], h1, l1);
    gp[slot][0] = make_float4(h0, l0, 0.f, 0.f);
    gp[slot][M / 2] = make_float4(h1, l1, 0.f, 0.f);
  }
}

// the poles' part of an m = 0 adjoint coefficient
__device__ __forceinline__ double oz_pole_term(const float4* g, int M, const double* pole_norm, int l) {
  const float4 n = g[0], s = g[M / 2];
  const double np = (double)n.x + (double)n.y, sp = (double)s.x + (double)s.y;
  return pole_norm[l] * (np + ((l & 1) ? -sp : sp));
}

// adjoint: the coefficients of orders without kept items (0, plus the poles at m = 0)
__global__ void __launch_bounds__(128) oz_zero_k(int M, const int* __restrict__ memberL,
                                                 const int* __restrict__ mfirst, const float4* const* __restrict__ gh,
                                                 const double* __restrict__ pole_norm, double2* const* __restrict__ out) {
  const int m = blockIdx.x, slot = blockIdx.y;
  if (mfirst[m + 1] > mfirst[m]) return;
  const int Ls = memberL[slot];
  if (m > Ls) return;
  double2* o = out[slot] + idx_lm(Ls, 0, m);
  for (int l = m + threadIdx.x; l <= Ls; l += blockDim.x)
    o[l] = make_double2(m == 0 ? oz_pole_term(gh[slot], M, pole_norm, l) : 0.0, 0.0);
}

struct OzArgs {
  int L, M, npairs, B, ncg;
  const int* memberL;
  const int* items;          // kept work items (m << 16 | block of 128 ring pairs), by order
  const int* mfirst;         // items of order m: [mfirst[m], mfirst[m + 1])
  const int2* work;          // synthesis: (item, column group); adjoint: (m, block << 8 | column group)
  const unsigned char* A;    // split recurrence table (synthesis or adjoint order)
  const int64_t* aoff;       // synthesis: per item; adjoint: per order
  const unsigned char* Bt;   // split coefficients / folded spectrum
  const int64_t* boff;       // per order
  const int* eA;             // adjoint: per order
  const int* eAi;            // synthesis: per kept item
  const int* eB;             // [order][128 columns]
  float4* const* gout;       // synthesis: members' ring sums (float pairs)
  const float4* const* gh;   // adjoint: members' theta spectra (the poles)
  double2* const* aout;      // adjoint: members' coefficients
  const double* pole_norm;
};

struct OzBars {
  uint64_t full[OZ_NBUF_P], empty[OZ_NBUF_P], done;
  uint32_t tslot;
  int abort;
};

__device__ __forceinline__ void oz_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(OZ_IDESC), "r"(acc)
      : "memory");
}

// One block: synthesis (ADJ = false) = (kept item, column group), chunks of
// 32 degrees (both parities: 12 + 12 tiles, three 72 KB buffers, accumulators
// (E, O) x (D0 .. D3)); adjoint = (order m, 256 degrees, column group,
// parity), chunks of 16 ring pairs over the order's kept items (one parity:
// 6 + 6 tiles, six 36 KB buffers, one accumulator per level i + j = 0 .. 5,
// every one exact at these magnitudes, so the adjoint carries no truncated
// accumulation at all).  Warp 0 lane 0 copies the chunks,
// warp 1 lane 0 issues the MMAs, warps 2-5 (TMEM lanes 32 (warp % 4) ..) run
// the epilogue once the last MMA has completed.  Every wait is bounded (one
// second); a block that gives up flags the others, waits (bounded) for its
// copies and MMAs in flight, sets *status and still frees its tensor memory.
template <bool ADJ>
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_tc_k(OzArgs z, int nblk, int* __restrict__ status,
                                                        int test_giveup) {
  constexpr int NB = ADJ ? OZ_NBUF_P : OZ_NBUF;
  constexpr int CH = ADJ ? OZ_CHUNK_P : OZ_CHUNK;
  constexpr int CA = CH * 2 / 3;  // A part of a chunk
  constexpr int CB = CH - CA;     // B part
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  OzBars* bars = reinterpret_cast<OzBars*>(oz_smem + NB * CH);
  if ((int)blockIdx.x >= nblk || *(volatile int*)status) return;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int2 wk = z.work[blockIdx.x];
  int m, cg, nchunk, blk = 0, q = 0, par = 0;
  const unsigned char* Abase;
  if (!ADJ) {
    const int v = z.items[wk.x];
    m = v >> 16;
    blk = v & 0xffff;
    cg = wk.y;
    nchunk = (z.L - m + 1 + 31) >> 5;
    Abase = z.A + z.aoff[wk.x];
  } else {
    m = wk.x;
    q = wk.y >> 8;
    par = (wk.y >> 4) & 1;
    cg = wk.y & 15;
    nchunk = 8 * (z.mfirst[m + 1] - z.mfirst[m]);
    Abase = z.A + z.aoff[m] + (size_t)q * nchunk * OZ_A + (size_t)par * OZ_NS * OZ_ATILE;
  }
  const unsigned char* Bbase = z.Bt + z.boff[m] + (size_t)cg * OZ_B + (size_t)par * OZ_NS * OZ_BTILE;
  const size_t bstride = (size_t)z.ncg * OZ_B;
  volatile int* abort = &bars->abort;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tslot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int k = 0; k < NB; ++k) {
      mbar_init(&bars->full[k], 1);
      mbar_init(&bars->empty[k], 1);
    }
    mbar_init(&bars->done, 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = bars->tslot;
  if (warp == 0) {
    if (lane == 0) {  // producer
      int issued = 0;
      for (int c = 0; c < nchunk && !*abort; ++c) {
        const int s = c % NB;
        if (c >= NB && !mbar_wait(smem_u32(&bars->empty[s]), (uint32_t)((c / NB - 1) & 1), abort)) {
          *abort = 1;
          break;
        }
        unsigned char* dst = oz_smem + s * CH;
        mbar_expect_tx(&bars->full[s], CH);
        bulk_g2s(dst, Abase + (size_t)c * OZ_A, CA, &bars->full[s]);
        bulk_g2s(dst + CA, Bbase + (size_t)c * bstride, CB, &bars->full[s]);
        issued = c + 1;
      }
      if (*abort)  // wait (bounded) for the copies still in flight
        for (int c = issued > NB ? issued - NB : 0; c < issued; ++c)
          mbar_wait(smem_u32(&bars->full[c % NB]), (uint32_t)((c / NB) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int last = -1;
      for (int c = 0; c < nchunk && !*abort; ++c) {
        const int s = c % NB;
        if (!mbar_wait(smem_u32(&bars->full[s]), (uint32_t)((c / NB) & 1), abort,
                       (test_giveup && c == 0) ? 0 : (1 << 30))) {
          *abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sb = smem_u32(oz_smem + s * CH);
        if constexpr (ADJ) {
          // one parity, one accumulator per level: the first product into
          // level j of chunk 0 is (0, j)
#pragma unroll
          for (int i = 0; i < OZ_NS; ++i)
#pragma unroll
            for (int j = 0; j < OZ_NS - i; ++j)
              oz_mma(tmem + (uint32_t)((i + j) * 64), tc_desc(sb + i * OZ_ATILE), tc_desc(sb + CA + j * OZ_BTILE),
                     (c > 0 || i > 0) ? 1u : 0u);
        } else {
#pragma unroll
          for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int i = 0; i < OZ_NS; ++i)
#pragma unroll
              for (int j = 0; j < OZ_NS - i; ++j) {
                const int lv = i + j < OZ_LV - 1 ? i + j : OZ_LV - 1;
                // the first products into D0 .. D3 of chunk 0 are (0,0) .. (0,3)
                const uint32_t acc = (c > 0 || i > 0 || j > OZ_LV - 1) ? 1u : 0u;
                oz_mma(tmem + (uint32_t)((p * OZ_LV + lv) * 64), tc_desc(sb + (p * OZ_NS + i) * OZ_ATILE),
                       tc_desc(sb + CA + (p * OZ_NS + j) * OZ_BTILE), acc);
              }
        }
        tc_commit(&bars->empty[s]);
        last = c;
      }
      if (!*abort) {
        tc_commit(&bars->done);
      } else if (last >= 0) {
        // MMAs already issued still write tensor memory: wait (bounded) for
        // the commit that covers them before the block frees it
        mbar_wait(smem_u32(&bars->empty[last % NB]), (uint32_t)((last / NB) & 1));
      }
    }
  } else {  // epilogue: TMEM lanes 32 (warp % 4) .. + 31 = rows
    const bool okw = mbar_wait(smem_u32(&bars->done), 0u, abort);
    if (!__all_sync(0xffffffffu, okw)) {
      *abort = 1;
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int q4 = warp & 3;
      const int r = q4 * 32 + lane;
      const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
      const int M = z.M;
      const int ea = ADJ ? z.eA[m] : z.eAi[wk.x];
      const int* eb = z.eB + (size_t)m * OZ_COLS + cg * 64;
      const int jn = 1 + blk * 128 + r, js = M / 2 - jn;
      constexpr int NACC = ADJ ? OZ_NS : 2 * OZ_LV;  // accumulators in use
      for (int cc = 0; cc < 4; ++cc) {
        uint32_t v[NACC][16];
#pragma unroll
        for (int a8 = 0; a8 < NACC; ++a8) tc_ld16(tl + (uint32_t)(a8 * 64 + cc * 16), v[a8]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int mm = 0; mm < 8; ++mm) {
          const int slot = cg * 32 + cc * 8 + mm;
          const int Ls = slot < z.B ? z.memberL[slot] : -1;
          if (m > Ls) continue;
          const int c0 = 2 * mm;  // re column (im: c0 + 1) within the 16 loaded
          if constexpr (!ADJ) {
            if (jn > z.npairs) continue;
            float o[2][2][2];  // [re, im][north, south][hi, lo]
#pragma unroll
            for (int ri = 0; ri < 2; ++ri) {
              float eh = __uint_as_float(v[0][c0 + ri]), el = 0.f;
              float oh = __uint_as_float(v[OZ_LV][c0 + ri]), ol = 0.f;
#pragma unroll
              for (int k = 1; k < OZ_LV; ++k) {
                df_add(eh, el, __uint_as_float(v[k][c0 + ri]), 0.f);
                df_add(oh, ol, __uint_as_float(v[OZ_LV + k][c0 + ri]), 0.f);
              }
              float nh = eh, nl = el, sh = eh, sl = el;
              df_add(nh, nl, oh, ol);
              df_add(sh, sl, -oh, -ol);
              const float sc = oz_pow2f(ea + eb[cc * 16 + c0 + ri] - 14);
              o[ri][0][0] = nh * sc;
              o[ri][0][1] = nl * sc;
              o[ri][1][0] = sh * sc;
              o[ri][1][1] = sl * sc;
            }
            const float sg = (m & 1) ? -1.f : 1.f;
            float4* row = z.gout[slot] + (size_t)m * M;
            const float4 fn = make_float4(o[0][0][0], o[0][0][1], o[1][0][0], o[1][0][1]);
            row[jn] = fn;
            row[M - jn] = make_float4(sg * fn.x, sg * fn.y, sg * fn.z, sg * fn.w);
            if (js != jn) {
              const float4 fs = make_float4(o[0][1][0], o[0][1][1], o[1][1][0], o[1][1][1]);
              row[js] = fs;
              row[M - js] = make_float4(sg * fs.x, sg * fs.y, sg * fs.z, sg * fs.w);
            }
          } else {
            double2* dst = z.aout[slot] + idx_lm(Ls, 0, m);
            const int l = m + 256 * q + 2 * r + par;
            if (l > Ls) continue;
            double x[2];
#pragma unroll
            for (int ri = 0; ri < 2; ++ri) {
              // 2^-36 fixed point: D0 < 2^25 stays below 2^61
              long long N = 0;
#pragma unroll
              for (int k = 0; k < NACC; ++k) N += oz_fix_f(__uint_as_float(v[k][c0 + ri]), 36);
              x[ri] = oz_dbl(N, ea + eb[cc * 16 + c0 + ri] - 14 - 36);
            }
            if (m == 0) {
              x[0] += oz_pole_term(z.gh[slot], M, z.pole_norm, l);
              x[1] = 0.0;
            }
            dst[l] = make_double2(x[0], x[1]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (*abort && t == 0) atomicExch(status, 1);
  tc_teardown(tmem);
}

struct Bucket {
  int L = 0, M = 0, B = 0, npairs = 0, nt = 1;
  std::vector<int> members;
  nusht_plan_t leg = nullptr;
  int* items = nullptr;
  int nitems = 0;
  int* mlist = nullptr;
  int nm = 0;
  int* memberL = nullptr;
  float2* atb = nullptr;
  float2* G = nullptr;
  float2* Ghat = nullptr;
  float* S = nullptr;
  float* cacc = nullptr;
  const float2** alm_ptrs = nullptr;  // device [BK_MAXB]
  float2** out_ptrs = nullptr;        // device [BK_MAXB]
  // table path
  bool table = false;
  float* P = nullptr;                 // recurrence table, [item][l - m][64]
  int64_t* offs = nullptr;            // item offsets into P
  int* mfirst = nullptr;              // items of order m: [mfirst[m], mfirst[m+1])
  int2* work = nullptr;               // adjoint blocks (m, first degree)
  int nwork = 0;
  size_t table_bytes = 0;
  // tensor-core path (table only): synthesis blocks of 128 ring pairs and
  // adjoint blocks of 256 degrees
  bool tc = false;
  int* tc_items = nullptr;            // (m << 16) | u, table tiles 2u and 2u + 1
  longlong2* tc_offs = nullptr;       // their offsets into P (-1: not kept)
  int ntc = 0;
  int2* tc_work = nullptr;            // (m, first row l - m)
  int ntc_work = 0;
  int ntiles = 0;                     // 64-pair table tiles per order
  int maxch = 0, maxch_adj = 0;       // chunks per block, at most
  unsigned char* PA = nullptr;        // synthesis A tiles, per block, chunk after chunk
  unsigned char* PT = nullptr;        // adjoint A tiles, per block
  unsigned char* BS = nullptr;        // synthesis B tiles, per order (per call)
  unsigned char* BA = nullptr;        // adjoint B tiles [m][tile][group] (per call)
  int tcg_s = TC_G, tcg_a = TC_G;     // degree chunks per partial accumulation (synthesis, adjoint)
  int64_t* pa_off = nullptr;          // byte offsets of the blocks / orders
  int64_t* pt_off = nullptr;
  int64_t* bs_off = nullptr;
  cufftHandle theta = 0;
  bool have_theta = false;
  // FP64 plans: the split contraction (items / mfirst above hold the FP64
  // probe's kept work items of 128 ring pairs)
  bool oz = false;
  int ncg = 1;                        // column groups of 32 members
  int2* oz_ws = nullptr;              // synthesis blocks (item, column group)
  int2* oz_wa = nullptr;              // adjoint blocks (m, block << 8 | column group)
  int noz_s = 0, noz_a = 0;
  unsigned char* OZS = nullptr;       // split table, synthesis order (per item)
  unsigned char* OZT = nullptr;       // split table, adjoint order (per order)
  int64_t* ozs_off = nullptr;         // per item
  int64_t* ozt_base = nullptr;        // per order
  unsigned char* OBS = nullptr;       // per call: split coefficients
  unsigned char* OBA = nullptr;       // per call: split folded spectrum
  int64_t* obs_off = nullptr;         // per order
  int64_t* oba_off = nullptr;         // per order
  int* eA = nullptr;                  // per order
  int* eAi = nullptr;                 // per kept item
  int* eBs = nullptr;                 // [order][128]
  int* eBa = nullptr;
  float4* Gp = nullptr;               // members' ring sums (float pairs), [slot][(L_k + 1) M]
  float4** gout = nullptr;            // device [BK_MAXB]
  float4** gh = nullptr;              // device [BK_MAXB]: members' theta spectra
  std::vector<float4*> gout_h;        // host copy of gout
  size_t oz_bytes = 0;
};

int64_t tri_count(int L, int M) { return (int64_t)(M / 4) * (int64_t)(L + 1) * (L + 2) / 2; }

}  // namespace
}  // namespace nusht

struct nusht_batch_s {
  int device = 0, nbatch = 0, precision = NUSHT_MIXED;
  double eps = 0;
  nusht_opts opts{};
  std::vector<int> L;
  std::vector<int64_t> npts;
  std::vector<nusht_plan_t> sub;
  std::vector<nusht::Bucket> buckets;
  std::vector<int> bucket_of, slot_of;
  size_t bytes = 0;
  cudaStream_t cap = nullptr;
  // members' NUFFT stages run on NSIDE streams forked from the capture
  // stream (graph branches), so that small members' kernels overlap
  static constexpr int NSIDE = 4;
  cudaStream_t side[NSIDE] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[NSIDE] = {};
  // members' NUFFT stages as one launch per stage for all members (mixed
  // precision, FP32 fine-grid FFT kernels, atomics): the member tables, in
  // table order (grouped by kernel width), and a per-call table of the
  // members' map pointers in the same order
  bool fused = false;
  bool fused_sfft = false;             // fine-grid FFTs by the FP32 line kernels (else cuFFT per member)
  std::vector<nusht::NufftBatch> nbw;  // one per kernel width
  nusht::NufftBatch nball;             // every member (grid zero fill)
  nusht::SfftLaunch sl;
  nusht::NufftMember* d_nmem = nullptr;
  nusht::SfftMember* d_smem = nullptr;
  float** d_maps = nullptr;
  std::vector<int> table_of;           // member -> position in the tables
  int* status = nullptr;  // device flag: a bounded wait in a tensor-core kernel gave up
  int test_giveup = 0;    // test hook (NUSHT_TEST_TC_GIVEUP=1): the first data wait runs out
  cudaGraphExec_t gs = nullptr, ga = nullptr;
  std::vector<const void*> gs_in;
  std::vector<void*> gs_out;
  std::vector<const void*> ga_in;
  std::vector<void*> ga_out;
};

namespace nusht {
namespace {

void bucket_free(Bucket& b) {
  if (b.leg) plan_destroy(b.leg);
  dev_free(b.items);
  dev_free(b.mlist);
  dev_free(b.memberL);
  dev_free(b.atb);
  dev_free(b.G);
  dev_free(b.Ghat);
  dev_free(b.S);
  dev_free(b.cacc);
  dev_free(b.alm_ptrs);
  dev_free(b.out_ptrs);
  dev_free(b.P);
  dev_free(b.offs);
  dev_free(b.mfirst);
  dev_free(b.work);
  dev_free(b.tc_items);
  dev_free(b.tc_offs);
  dev_free(b.tc_work);
  dev_free(b.PA);
  dev_free(b.PT);
  dev_free(b.BS);
  dev_free(b.BA);
  dev_free(b.pa_off);
  dev_free(b.pt_off);
  dev_free(b.bs_off);
  dev_free(b.oz_ws);
  dev_free(b.oz_wa);
  dev_free(b.OZS);
  dev_free(b.OZT);
  dev_free(b.ozs_off);
  dev_free(b.ozt_base);
  dev_free(b.OBS);
  dev_free(b.OBA);
  dev_free(b.obs_off);
  dev_free(b.oba_off);
  dev_free(b.eA);
  dev_free(b.eAi);
  dev_free(b.eBs);
  dev_free(b.eBa);
  dev_free(b.Gp);
  dev_free(b.gout);
  dev_free(b.gh);
  if (b.have_theta) cufftDestroy(b.theta);
  b = Bucket();
}

void batch_free(nusht_batch_t p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  if (p->gs) cudaGraphExecDestroy(p->gs);
  if (p->ga) cudaGraphExecDestroy(p->ga);
  for (auto* s : p->sub)
    if (s) plan_destroy(s);
  for (auto& b : p->buckets) bucket_free(b);
  dev_free(p->status);
  dev_free(p->d_nmem);
  dev_free(p->d_smem);
  dev_free(p->d_maps);
  for (int k = 0; k < nusht_batch_s::NSIDE; ++k) {
    if (p->side[k]) cudaStreamDestroy(p->side[k]);
    if (p->ev_join[k]) cudaEventDestroy(p->ev_join[k]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->cap) cudaStreamDestroy(p->cap);
  cudaSetDevice(cur);
  delete p;
}

// Grouping of the members (sorted by lmax) into contiguous buckets of at most
// 64 that minimises  sum over buckets of T(L_max) (c_rec + 128 c_col) + c_fix,
// T = (ring pairs) x (l, m) triples of the bucket's lmax.  The constants are
// per-triple costs of the FP64 recurrence and of the 128-column FP32
// contraction on GB300 and a per-bucket overhead (launches, theta FFT).
std::vector<std::vector<int>> group_members(const std::vector<int>& L, double c_rec, double c_col, double c_fix) {
  const int n = (int)L.size();
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return L[x] < L[y]; });
  std::vector<double> best(n + 1, 1e300);
  std::vector<int> cut(n + 1, 0);
  best[0] = 0.0;
  for (int j = 1; j <= n; ++j) {
    for (int i = std::max(0, j - BK_MAXB); i < j; ++i) {
      nusht_sizes z;
      const int Lb = L[order[j - 1]];
      if (choose_sizes(Lb, Lb, 1e-5, NUSHT_MIXED, nullptr, &z) != NUSHT_OK) continue;
      const double cost = best[i] + (double)tri_count(Lb, z.M) * (c_rec + BK_COLS * c_col) + c_fix;
      if (cost < best[j]) {
        best[j] = cost;
        cut[j] = i;
      }
    }
  }
  std::vector<std::vector<int>> groups;
  for (int j = n; j > 0; j = cut[j]) {
    std::vector<int> g(order.begin() + cut[j], order.begin() + j);
    groups.push_back(g);
  }
  std::reverse(groups.begin(), groups.end());
  return groups;
}

BucketArgs bucket_args(const Bucket& b) {
  BucketArgs a;
  a.lmax = b.L;
  a.M = b.M;
  a.npairs = b.npairs;
  a.B = b.B;
  a.c = b.leg->leg.c;
  a.dshift = b.leg->leg.dshift;
  a.cm = b.leg->leg.cm;
  a.ring_x = b.leg->leg.ring_x;
  a.ring_s = b.leg->leg.ring_s;
  a.memberL = b.memberL;
  return a;
}

// Autotuner of the tensor-core contraction's schedule: the degree chunks per
// partial accumulation (2, 4 or 8 chunks of 16 degrees into one TMEM partial
// set before the fold into registers) for each direction, timed on the
// bucket's own tables with zero operands (opts.tune = 1) and cached under the
// device, the bucket lmax and member count; opts.tune = 2 takes the cached
// choice.  Larger groups fold less often; smaller ones bound the tensor
// core's truncating accumulation to fewer MMAs (eps_eff 1.2e-6 at 4 chunks,
// lmax 2043).
int tune_tc(nusht_batch_t p, Bucket& b, cudaStream_t s) {
  std::string key = "C:" + tune_device(p->device) + ":L" + std::to_string(b.L) + ":B" + std::to_string(b.B);
  if (p->opts.tune == 2) {
    const int v = tune_cache_get(key);
    const int vs = v / 10, va = v % 10;
    if ((vs == 2 || vs == 4 || vs == 8) && (va == 2 || va == 4 || va == 8)) {
      b.tcg_s = vs;
      b.tcg_a = va;
    }
    return NUSHT_OK;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return set_error(NUSHT_ECUDA, "tuning events");
  }
  const BucketArgs a = bucket_args(b);
  int st = NUSHT_OK;
  for (int dir = 0; dir < 2 && st == NUSHT_OK; ++dir) {
    float best = 1e30f;
    int bestg = TC_G;
    for (int g : {2, 4, 8}) {
      auto launch = [&]() {
        if (dir == 0 && b.ntc > 0)
          bucket_tc_k<false><<<b.ntc, T6_THREADS, T6_SMEM, s>>>(a, b.ntc, b.tc_items, nullptr, b.pa_off, b.bs_off,
                                                                nullptr, nullptr, b.ntiles, b.PA, b.BS, b.G, nullptr,
                                                                p->status, 0, g);
        if (dir == 1 && b.ntc_work > 0)
          bucket_tc_k<true><<<b.ntc_work, T6_THREADS, T6_SMEM, s>>>(a, b.ntc_work, nullptr, b.tc_work, b.pt_off,
                                                                    nullptr, b.items, b.mfirst, b.ntiles, b.PT, b.BA,
                                                                    nullptr, b.cacc, p->status, 0, g);
      };
      launch();  // warm-up
      cudaEventRecord(e0, s);
      launch();
      launch();
      cudaEventRecord(e1, s);
      float ms = 0.f;
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        st = cuda_status(e, "tensor-core schedule tuning");
        break;
      }
      if (ms < best) {
        best = ms;
        bestg = g;
      }
    }
    if (dir == 0)
      b.tcg_s = bestg;
    else
      b.tcg_a = bestg;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NUSHT_OK) return st;
  tune_cache_put(key, b.tcg_s * 10 + b.tcg_a);
  return NUSHT_OK;
}

int bucket_build(nusht_batch_t p, Bucket& b, cudaStream_t s) {
  const int L = b.L;
  nusht_sizes z;
  NUSHT_TRY(choose_sizes(L, L, p->eps, NUSHT_MIXED, &p->opts, &z));
  b.M = z.M;
  b.npairs = b.M / 4;
  b.nt = 1;
  while (b.nt * BA_TILE < b.npairs) b.nt *= 2;
  if (b.nt > 8) return set_error(NUSHT_EUNSUPPORTED, "batched transforms support lmax <= 4095");
  PlanRole role;
  role.nufft = false;
  role.legendre = true;
  NUSHT_TRY(plan_create(&b.leg, L, L, 0, nullptr, p->eps, NUSHT_MIXED, &p->opts, s, role));
  // 64-pair synthesis tiles from the 128-pair work items kept by the probe
  std::vector<int> items(b.leg->leg.nitems);
  NUSHT_CUDA(cudaMemcpy(items.data(), b.leg->leg.items, items.size() * 4, cudaMemcpyDeviceToHost));
  std::vector<int> tiles, ms;
  for (int v : items) {
    const int m = v >> 16, blk = v & 0xffff;
    for (int h = 0; h < 2; ++h) {
      const int tile = 2 * blk + h;
      if (1 + tile * BS_PAIRS <= b.npairs) tiles.push_back((m << 16) | tile);
    }
    if (ms.empty() || ms.back() != m) ms.push_back(m);
  }
  b.nitems = (int)tiles.size();
  b.nm = (int)ms.size();
  NUSHT_TRY(dev_alloc((void**)&b.items, std::max<size_t>(1, tiles.size()) * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.mlist, std::max<size_t>(1, ms.size()) * 4, &p->bytes));
  if (!tiles.empty()) NUSHT_CUDA(cudaMemcpy(b.items, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice));
  if (!ms.empty()) NUSHT_CUDA(cudaMemcpy(b.mlist, ms.data(), ms.size() * 4, cudaMemcpyHostToDevice));
  std::vector<int> ml(BK_MAXB, -1);
  for (int k = 0; k < b.B; ++k) ml[k] = p->L[b.members[k]];
  NUSHT_TRY(dev_alloc((void**)&b.memberL, BK_MAXB * 4, &p->bytes));
  NUSHT_CUDA(cudaMemcpy(b.memberL, ml.data(), BK_MAXB * 4, cudaMemcpyHostToDevice));
  const int64_t nalm = b.leg->nalm;
  const size_t gbytes = (size_t)b.B * (L + 1) * b.M * sizeof(float2);
  NUSHT_TRY(dev_alloc((void**)&b.atb, (size_t)nalm * BK_MAXB * sizeof(float2), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.G, gbytes, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.Ghat, gbytes, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.S, (size_t)(L + 1) * b.npairs * 2 * BK_COLS * sizeof(float), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.cacc, (size_t)nalm * BK_COLS * sizeof(float), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.alm_ptrs, BK_MAXB * sizeof(void*), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.out_ptrs, BK_MAXB * sizeof(void*), &p->bytes));
  NUSHT_CUDA(cudaMemsetAsync(b.G, 0, gbytes, s));
  NUSHT_CUDA(cudaMemsetAsync(b.Ghat, 0, gbytes, s));
  NUSHT_CUDA(cudaMemsetAsync(b.cacc, 0, (size_t)nalm * BK_COLS * sizeof(float), s));
  // recurrence table when it fits (the on-the-fly kernels otherwise)
  {
    std::vector<int64_t> off(tiles.size() + 1, 0);
    for (size_t k = 0; k < tiles.size(); ++k) off[k + 1] = off[k] + (int64_t)(L - (tiles[k] >> 16) + 1) * BS_PAIRS;
    const size_t need = (size_t)off.back() * sizeof(float);
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    if (p->opts.legendre_table >= 0 && need > 0 && need < freeb / 2) {
      b.table = true;
      b.table_bytes = need;
      NUSHT_TRY(dev_alloc((void**)&b.P, need, &p->bytes));
      NUSHT_TRY(dev_alloc((void**)&b.offs, off.size() * 8, &p->bytes));
      NUSHT_CUDA(cudaMemcpy(b.offs, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
      std::vector<int> mf(L + 2, 0);
      for (size_t k = 0; k < tiles.size(); ++k) mf[(tiles[k] >> 16) + 1]++;
      for (int m = 0; m <= L; ++m) mf[m + 1] += mf[m];
      NUSHT_TRY(dev_alloc((void**)&b.mfirst, mf.size() * 4, &p->bytes));
      NUSHT_CUDA(cudaMemcpy(b.mfirst, mf.data(), mf.size() * 4, cudaMemcpyHostToDevice));
      std::vector<int2> wk;
      for (int m = 0; m <= L; ++m)
        if (mf[m + 1] > mf[m])
          for (int l0 = m; l0 <= L; l0 += AT_LC) wk.push_back(make_int2(m, l0));
      b.nwork = (int)wk.size();
      NUSHT_TRY(dev_alloc((void**)&b.work, std::max<size_t>(1, wk.size()) * sizeof(int2), &p->bytes));
      if (!wk.empty())
        NUSHT_CUDA(cudaMemcpy(b.work, wk.data(), wk.size() * sizeof(int2), cudaMemcpyHostToDevice));
      const BucketArgs a = bucket_args(b);
      if (b.nitems > 0) bucket_ptab_k<<<(b.nitems + 3) / 4, 128, 0, s>>>(a, b.items, b.offs, b.nitems, b.P);
      NUSHT_CUDA(cudaGetLastError());
      if (p->opts.tensor_cores >= 0) {
        // pairs of 64-pair tiles (2u, 2u + 1) of one order; tiles[] is
        // ordered by m, then tile
        std::vector<int> ti;
        std::vector<longlong2> to;
        for (size_t k = 0; k < tiles.size(); ++k) {
          const int m = tiles[k] >> 16, tile = tiles[k] & 0xffff;
          const int key = (m << 16) | (tile >> 1);
          if (ti.empty() || ti.back() != key) {
            ti.push_back(key);
            longlong2 z2;
            z2.x = -1;
            z2.y = -1;
            to.push_back(z2);
          }
          if (tile & 1)
            to.back().y = off[k];
          else
            to.back().x = off[k];
        }
        std::vector<int2> tw;
        for (int m = 0; m <= L; ++m)
          if (mf[m + 1] > mf[m])
            for (int r0 = 0; r0 <= L - m; r0 += 256) tw.push_back(make_int2(m, r0));
        b.ntc = (int)ti.size();
        b.ntc_work = (int)tw.size();
        NUSHT_TRY(dev_alloc((void**)&b.tc_items, std::max<size_t>(1, ti.size()) * 4, &p->bytes));
        NUSHT_TRY(dev_alloc((void**)&b.tc_offs, std::max<size_t>(1, to.size()) * sizeof(longlong2), &p->bytes));
        NUSHT_TRY(dev_alloc((void**)&b.tc_work, std::max<size_t>(1, tw.size()) * sizeof(int2), &p->bytes));
        if (!ti.empty()) {
          NUSHT_CUDA(cudaMemcpy(b.tc_items, ti.data(), ti.size() * 4, cudaMemcpyHostToDevice));
          NUSHT_CUDA(cudaMemcpy(b.tc_offs, to.data(), to.size() * sizeof(longlong2), cudaMemcpyHostToDevice));
        }
        if (!tw.empty())
          NUSHT_CUDA(cudaMemcpy(b.tc_work, tw.data(), tw.size() * sizeof(int2), cudaMemcpyHostToDevice));
        // pre-split operand tiles: sizes, then the tables when they fit
        b.ntiles = (b.npairs + BS_PAIRS - 1) / BS_PAIRS;
        b.maxch = (L + 1 + 15) / 16;
        std::vector<int64_t> pao(ti.size()), pto(tw.size()), bso(L + 1);
        int64_t pab = 0, ptb = 0, bsb = 0;
        for (size_t k = 0; k < ti.size(); ++k) {
          pao[k] = pab;
          pab += (int64_t)((L - (ti[k] >> 16) + 1 + 15) / 16) * T6_HALF;
        }
        b.maxch_adj = 0;
        for (size_t k = 0; k < tw.size(); ++k) {
          pto[k] = ptb;
          const int ch = (mf[tw[k].x + 1] - mf[tw[k].x]) * (BS_PAIRS / 8);
          b.maxch_adj = std::max(b.maxch_adj, ch);
          ptb += (int64_t)ch * T6_HALF;
        }
        for (int m = 0; m <= L; ++m) {
          bso[m] = bsb;
          bsb += (int64_t)((L - m + 1 + 15) / 16) * T6_HALF;
        }
        const int64_t bab = (int64_t)(L + 1) * b.ntiles * 8 * T6_HALF;
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        if (pab + ptb + bsb + bab > 0 && (size_t)(pab + ptb + bsb + bab) < fr / 2) {
          NUSHT_TRY(dev_alloc((void**)&b.PA, std::max<int64_t>(16, pab), &p->bytes));
          NUSHT_TRY(dev_alloc((void**)&b.PT, std::max<int64_t>(16, ptb), &p->bytes));
          NUSHT_TRY(dev_alloc((void**)&b.BS, std::max<int64_t>(16, bsb), &p->bytes));
          NUSHT_TRY(dev_alloc((void**)&b.BA, std::max<int64_t>(16, bab), &p->bytes));
          NUSHT_TRY(dev_alloc((void**)&b.pa_off, std::max<size_t>(1, pao.size()) * 8, &p->bytes));
          NUSHT_TRY(dev_alloc((void**)&b.pt_off, std::max<size_t>(1, pto.size()) * 8, &p->bytes));
          NUSHT_TRY(dev_alloc((void**)&b.bs_off, bso.size() * 8, &p->bytes));
          if (!pao.empty()) NUSHT_CUDA(cudaMemcpy(b.pa_off, pao.data(), pao.size() * 8, cudaMemcpyHostToDevice));
          if (!pto.empty()) NUSHT_CUDA(cudaMemcpy(b.pt_off, pto.data(), pto.size() * 8, cudaMemcpyHostToDevice));
          NUSHT_CUDA(cudaMemcpy(b.bs_off, bso.data(), bso.size() * 8, cudaMemcpyHostToDevice));
          NUSHT_CUDA(cudaMemsetAsync(b.BA, 0, bab, s));  // tiles of pairs past npairs stay zero
          if (b.ntc > 0)
            tc_build_pa_k<<<dim3(b.maxch, b.ntc), 256, 0, s>>>(b.P, b.tc_items, b.tc_offs, b.pa_off, L, b.PA);
          if (b.ntc_work > 0 && b.maxch_adj > 0)
            tc_build_pt_k<<<dim3(b.maxch_adj, b.ntc_work), 256, 0, s>>>(b.P, b.items, b.offs, b.mfirst, b.tc_work,
                                                                      b.pt_off, L, b.PT);
          NUSHT_CUDA(cudaGetLastError());
          NUSHT_CUDA(cudaStreamSynchronize(s));
          b.tc = true;
          if (p->opts.tune == 1 || p->opts.tune == 2) {
            NUSHT_CUDA(cudaMemsetAsync(b.BS, 0, std::max<int64_t>(16, bsb), s));
            NUSHT_TRY(tune_tc(p, b, s));
          }
          // the CUDA-core operands are not needed on this path
          dev_free(b.P);
          b.P = nullptr;
          dev_free(b.atb);
          b.atb = nullptr;
          dev_free(b.S);
          b.S = nullptr;
        }
      }
    }
  }
  NUSHT_CUFFT(cufftCreate(&b.theta));
  b.have_theta = true;
  int M = b.M;
  size_t ws = 0;
  NUSHT_CUFFT(cufftMakePlanMany(b.theta, 1, &M, nullptr, 1, M, nullptr, 1, M, CUFFT_C2C, b.B * (L + 1), &ws));
  NUSHT_CUDA(cudaStreamSynchronize(s));
  return NUSHT_OK;
}

// FP64 bucket: the FP64 probe's kept work items, both split tables, the
// per-call operand buffers and the members' ring-sum buffers.
int bucket_build_oz(nusht_batch_t p, Bucket& b, cudaStream_t s) {
  const int L = b.L;
  nusht_sizes z;
  NUSHT_TRY(choose_sizes(L, L, p->eps, NUSHT_FP64, &p->opts, &z));
  b.M = z.M;
  b.npairs = b.M / 4;
  PlanRole role;
  role.nufft = false;
  role.legendre = true;
  nusht_opts lo = p->opts;  // the FP64 chain's tables (no table mode, no double-float chain)
  lo.legendre_table = -1;
  lo.fast_recurrence = 0;
  lo.spin = 0;
  NUSHT_TRY(plan_create(&b.leg, L, L, 0, nullptr, p->eps, NUSHT_FP64, &lo, s, role));
  std::vector<int> items(b.leg->leg.nitems);
  if (!items.empty())
    NUSHT_CUDA(cudaMemcpy(items.data(), b.leg->leg.items, items.size() * 4, cudaMemcpyDeviceToHost));
  std::sort(items.begin(), items.end());  // by order, then ring block
  b.nitems = (int)items.size();
  std::vector<int> mf(L + 2, 0);
  for (int v : items) mf[(v >> 16) + 1]++;
  for (int m = 0; m <= L; ++m) mf[m + 1] += mf[m];
  b.ncg = (b.B + 31) / 32;
  std::vector<int64_t> soff(items.size()), tb(L + 1, 0), bso(L + 1, 0), bao(L + 1, 0);
  int64_t sa = 0, ta = 0, bs = 0, ba = 0;
  std::vector<int2> ws, wa;
  for (size_t it = 0; it < items.size(); ++it) {
    const int m = items[it] >> 16;
    soff[it] = sa;
    sa += (int64_t)((L - m + 1 + 31) / 32) * OZ_A;
    for (int cg = 0; cg < b.ncg; ++cg) ws.push_back(make_int2((int)it, cg));
  }
  for (int m = 0; m <= L; ++m) {
    const int nim = mf[m + 1] - mf[m];
    tb[m] = ta;
    bso[m] = bs;
    bao[m] = ba;
    if (nim == 0) continue;
    const int nq = (L - m + 1 + 255) / 256;
    ta += (int64_t)nq * 8 * nim * OZ_A;
    bs += (int64_t)((L - m + 1 + 31) / 32) * b.ncg * OZ_B;
    ba += (int64_t)8 * nim * b.ncg * OZ_B;
    for (int q = 0; q < nq; ++q)
      for (int cg = 0; cg < b.ncg; ++cg)
        for (int par = 0; par < 2; ++par) wa.push_back(make_int2(m, (q << 8) | (par << 4) | cg));
  }
  b.noz_s = (int)ws.size();
  b.noz_a = (int)wa.size();
  int64_t gsz = 0;
  b.gout_h.assign(BK_MAXB, nullptr);
  std::vector<int64_t> goff(b.B);
  for (int k = 0; k < b.B; ++k) {
    goff[k] = gsz;
    gsz += (int64_t)(p->L[b.members[k]] + 1) * b.M;
  }
  const size_t need = (size_t)(sa + ta + bs + ba) + (size_t)gsz * sizeof(float4);
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  if (need >= freeb / 2)
    return set_error(NUSHT_ENOMEM, "FP64 batched plan: the split recurrence tables do not fit in device memory");
  b.oz_bytes = need;
  NUSHT_TRY(dev_alloc((void**)&b.items, std::max<size_t>(1, items.size()) * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.mfirst, mf.size() * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.oz_ws, std::max<size_t>(1, ws.size()) * sizeof(int2), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.oz_wa, std::max<size_t>(1, wa.size()) * sizeof(int2), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.ozs_off, std::max<size_t>(1, soff.size()) * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.ozt_base, tb.size() * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.obs_off, bso.size() * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.oba_off, bao.size() * 8, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.OZS, std::max<int64_t>(16, sa), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.OZT, std::max<int64_t>(16, ta), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.OBS, std::max<int64_t>(16, bs), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.OBA, std::max<int64_t>(16, ba), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.eA, (size_t)(L + 1) * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.eAi, std::max<size_t>(1, items.size()) * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.eBs, (size_t)(L + 1) * OZ_COLS * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.eBa, (size_t)(L + 1) * OZ_COLS * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.Gp, std::max<int64_t>(1, gsz) * sizeof(float4), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.gout, BK_MAXB * sizeof(void*), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.gh, BK_MAXB * sizeof(void*), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.memberL, BK_MAXB * 4, &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.alm_ptrs, BK_MAXB * sizeof(void*), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&b.out_ptrs, BK_MAXB * sizeof(void*), &p->bytes));
  if (!items.empty()) {
    NUSHT_CUDA(cudaMemcpy(b.items, items.data(), items.size() * 4, cudaMemcpyHostToDevice));
    NUSHT_CUDA(cudaMemcpy(b.ozs_off, soff.data(), soff.size() * 8, cudaMemcpyHostToDevice));
  }
  NUSHT_CUDA(cudaMemcpy(b.mfirst, mf.data(), mf.size() * 4, cudaMemcpyHostToDevice));
  if (!ws.empty()) NUSHT_CUDA(cudaMemcpy(b.oz_ws, ws.data(), ws.size() * sizeof(int2), cudaMemcpyHostToDevice));
  if (!wa.empty()) NUSHT_CUDA(cudaMemcpy(b.oz_wa, wa.data(), wa.size() * sizeof(int2), cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(b.ozt_base, tb.data(), tb.size() * 8, cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(b.obs_off, bso.data(), bso.size() * 8, cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(b.oba_off, bao.data(), bao.size() * 8, cudaMemcpyHostToDevice));
  std::vector<int> ml(BK_MAXB, -1);
  for (int k = 0; k < b.B; ++k) {
    ml[k] = p->L[b.members[k]];
    b.gout_h[k] = b.Gp + goff[k];
  }
  NUSHT_CUDA(cudaMemcpy(b.memberL, ml.data(), BK_MAXB * 4, cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemcpy(b.gout, b.gout_h.data(), BK_MAXB * sizeof(void*), cudaMemcpyHostToDevice));
  NUSHT_CUDA(cudaMemsetAsync(b.OZS, 0, std::max<int64_t>(16, sa), s));
  NUSHT_CUDA(cudaMemsetAsync(b.OZT, 0, std::max<int64_t>(16, ta), s));
  NUSHT_CUDA(cudaMemsetAsync(b.Gp, 0, std::max<int64_t>(1, gsz) * sizeof(float4), s));
  // exponents of the recurrence values per order, then the tables
  unsigned long long* amax = nullptr;
  NUSHT_TRY(dev_alloc((void**)&amax, (size_t)(L + 1 + std::max(1, b.nitems)) * 8, nullptr));
  unsigned long long* amax_item = amax + L + 1;
  int st = NUSHT_OK;
  do {
    const BucketArgs a = bucket_args(b);
    cudaError_t e = cudaMemsetAsync(amax, 0, (size_t)(L + 1) * 8, s);
    if (e == cudaSuccess && b.nitems > 0) {
      oz_amax_k<<<(b.nitems + 3) / 4, 128, 0, s>>>(a, b.items, b.nitems, b.leg->leg.ahat, amax, amax_item);
      e = cudaGetLastError();
    }
    std::vector<unsigned long long> hm(L + 1 + std::max(1, b.nitems), 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hm.data(), amax, hm.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_status(e, "split table exponents");
      break;
    }
    std::vector<int> ea(L + 1), eai(std::max(1, b.nitems), 0);
    for (int m = 0; m <= L; ++m) ea[m] = hm[m] ? (int)(hm[m] >> 52) - 1022 : 0;
    for (int it = 0; it < b.nitems; ++it) {
      const unsigned long long v = hm[L + 1 + it];
      eai[it] = v ? (int)(v >> 52) - 1022 : 0;
    }
    e = cudaMemcpy(b.eA, ea.data(), (size_t)(L + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b.eAi, eai.data(), eai.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b.nitems > 0) {
      oz_build_k<<<(b.nitems + 3) / 4, 128, 0, s>>>(a, b.items, b.nitems, b.mfirst, b.leg->leg.ahat, b.eA, b.eAi,
                                                    b.ozs_off, b.ozt_base, b.OZS, b.OZT);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "split table build");
  } while (false);
  dev_free(amax);
  NUSHT_TRY(st);
  b.oz = true;
  return NUSHT_OK;
}

OzArgs oz_args(const Bucket& b, bool adj) {
  OzArgs z;
  z.L = b.L;
  z.M = b.M;
  z.npairs = b.npairs;
  z.B = b.B;
  z.ncg = b.ncg;
  z.memberL = b.memberL;
  z.items = b.items;
  z.mfirst = b.mfirst;
  z.work = adj ? b.oz_wa : b.oz_ws;
  z.A = adj ? b.OZT : b.OZS;
  z.aoff = adj ? b.ozt_base : b.ozs_off;
  z.Bt = adj ? b.OBA : b.OBS;
  z.boff = adj ? b.oba_off : b.obs_off;
  z.eA = b.eA;
  z.eAi = b.eAi;
  z.eB = adj ? b.eBa : b.eBs;
  z.gout = b.gout;
  z.gh = b.gh;
  z.aout = reinterpret_cast<double2* const*>(b.out_ptrs);
  z.pole_norm = b.leg->leg.pole_norm;
  return z;
}


int launch_adj(const Bucket& b, cudaStream_t s) {
  const BucketArgs a = bucket_args(b);
  const size_t sm = (size_t)(BA_LC * BA_TILE + BA_SUB * 2 * BK_COLS) * sizeof(float);
  switch (b.nt) {
    case 1:
      bucket_adj_k<1><<<b.nm, 256, sm, s>>>(a, b.mlist, b.nm, b.S, b.cacc);
      break;
    case 2:
      bucket_adj_k<2><<<b.nm, 256, sm, s>>>(a, b.mlist, b.nm, b.S, b.cacc);
      break;
    case 4:
      bucket_adj_k<4><<<b.nm, 256, sm, s>>>(a, b.mlist, b.nm, b.S, b.cacc);
      break;
    default:
      bucket_adj_k<8><<<b.nm, 256, sm, s>>>(a, b.mlist, b.nm, b.S, b.cacc);
      break;
  }
  return NUSHT_OK;
}

int set_adj_smem() {
  const int sm = (BA_LC * BA_TILE + BA_SUB * 2 * BK_COLS) * (int)sizeof(float);
  NUSHT_CUDA(cudaFuncSetAttribute(bucket_adj_k<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  NUSHT_CUDA(cudaFuncSetAttribute(bucket_adj_k<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  NUSHT_CUDA(cudaFuncSetAttribute(bucket_adj_k<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  NUSHT_CUDA(cudaFuncSetAttribute(bucket_adj_k<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  const int smt = (BS_PAIRS * AT_PAD + BS_PAIRS * 2 * BK_COLS) * (int)sizeof(float);
  NUSHT_CUDA(cudaFuncSetAttribute(bucket_adj_tab_k, cudaFuncAttributeMaxDynamicSharedMemorySize, smt));
  NUSHT_CUDA(cudaFuncSetAttribute(bucket_tc_k<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, T6_SMEM));
  NUSHT_CUDA(cudaFuncSetAttribute(bucket_tc_k<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, T6_SMEM));
  NUSHT_CUDA(cudaFuncSetAttribute(oz_tc_k<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  NUSHT_CUDA(cudaFuncSetAttribute(oz_tc_k<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  return NUSHT_OK;
}

// fork the side streams off `s` / join them back (inside a capture these
// become graph branches)
int fork(nusht_batch_t p, cudaStream_t s) {
  NUSHT_CUDA(cudaEventRecord(p->ev_fork, s));
  for (int k = 0; k < nusht_batch_s::NSIDE; ++k) NUSHT_CUDA(cudaStreamWaitEvent(p->side[k], p->ev_fork, 0));
  return NUSHT_OK;
}

int join(nusht_batch_t p, cudaStream_t s) {
  for (int k = 0; k < nusht_batch_s::NSIDE; ++k) {
    NUSHT_CUDA(cudaEventRecord(p->ev_join[k], p->side[k]));
    NUSHT_CUDA(cudaStreamWaitEvent(s, p->ev_join[k], 0));
  }
  return NUSHT_OK;
}

int enqueue_synth(nusht_batch_t p, void* const* d_map, cudaStream_t s) {
  for (auto& b : p->buckets) {
    const BucketArgs a = bucket_args(b);
    dim3 g((b.L + 1 + 3) / 4, b.L + 1);
    if (b.tc) {
      tc_scale_bs_k<<<dim3(b.maxch, b.L + 1), 256, 0, s>>>(b.L, b.B, b.memberL, b.alm_ptrs, b.leg->leg.ahat,
                                                           b.bs_off, b.BS);
      if (b.ntc > 0)
        bucket_tc_k<false><<<b.ntc, T6_THREADS, T6_SMEM, s>>>(a, b.ntc, b.tc_items, nullptr, b.pa_off, b.bs_off,
                                                              nullptr, nullptr, b.ntiles, b.PA, b.BS, b.G, nullptr,
                                                              p->status, p->test_giveup, b.tcg_s);
    } else {
      bucket_scale_k<<<g, 256, 0, s>>>(b.L, b.B, b.memberL, b.alm_ptrs, b.leg->leg.ahat, b.atb);
    }
    if (b.tc) {
    } else if (b.nitems > 0 && b.table)
      bucket_synth_tab_k<<<b.nitems, 256, 0, s>>>(a, b.items, b.offs, b.nitems, b.P, b.atb, b.G);
    else if (b.nitems > 0)
      bucket_synth_k<<<b.nitems, 256, 0, s>>>(a, b.items, b.nitems, b.atb, b.G);
    bucket_poles_k<<<b.B, 256, 0, s>>>(b.L, b.M, b.memberL, b.alm_ptrs, b.leg->leg.pole_norm, b.G);
    NUSHT_CUDA(cudaGetLastError());
    NUSHT_CUFFT(cufftSetStream(b.theta, s));
    NUSHT_CUFFT(cufftExecC2C(b.theta, (cufftComplex*)b.G, (cufftComplex*)b.Ghat, CUFFT_FORWARD));
  }
  if (p->fused) {
    // every member at once: deconvolution and zero padding (fused into the
    // column pass with the FP32 line kernels), the fine-grid FFT,
    // interpolation; members' cuFFT calls on the forked streams
    if (p->fused_sfft) {
      NUSHT_TRY(sfft_cols_synth(p->sl, s));
      NUSHT_TRY(sfft_rows_c2r(p->sl, s));
    } else {
      NUSHT_TRY(deconv_pad_many(p->nball, s));
      NUSHT_TRY(fork(p, s));
      for (int i = 0; i < p->nbatch; ++i) NUSHT_TRY(fine_fft_c2r(p->sub[i], p->side[i % nusht_batch_s::NSIDE]));
      NUSHT_TRY(join(p, s));
    }
    for (const NufftBatch& g : p->nbw) NUSHT_TRY(interp_many(g, p->d_maps + g.map_base, s));
    return NUSHT_OK;
  }
  NUSHT_TRY(fork(p, s));
  for (int i = 0; i < p->nbatch; ++i) {
    nusht_plan_t q = p->sub[i];
    cudaStream_t ms = p->side[i % nusht_batch_s::NSIDE];
    NUSHT_TRY(deconv_pad(q, ms));
    NUSHT_TRY(fine_fft_c2r(q, ms));
    NUSHT_TRY(interp(q, d_map[i], ms));
  }
  NUSHT_TRY(join(p, s));
  return NUSHT_OK;
}

int enqueue_adjoint(nusht_batch_t p, const void* const* d_map, cudaStream_t s) {
  if (p->fused) {
    // every member at once: zero the grids, spread, row pass, column pass + truncation
    NUSHT_TRY(zero_grids_many(p->nball, s));
    for (const NufftBatch& g : p->nbw)
      NUSHT_TRY(spread_many(g, const_cast<const float* const*>(p->d_maps) + g.map_base, s));
    if (p->fused_sfft) {
      NUSHT_TRY(sfft_rows_r2c(p->sl, s));
      NUSHT_TRY(sfft_cols_adjoint(p->sl, s));
    } else {
      NUSHT_TRY(fork(p, s));
      for (int i = 0; i < p->nbatch; ++i) NUSHT_TRY(fine_fft_r2c(p->sub[i], p->side[i % nusht_batch_s::NSIDE]));
      NUSHT_TRY(join(p, s));
      NUSHT_TRY(deconv_trunc_many(p->nball, s));
    }
  } else {
    NUSHT_TRY(fork(p, s));
    for (int i = 0; i < p->nbatch; ++i) {
      nusht_plan_t q = p->sub[i];
      cudaStream_t ms = p->side[i % nusht_batch_s::NSIDE];
      NUSHT_TRY(spread(q, d_map[i], ms));
      NUSHT_TRY(fine_fft_r2c(q, ms));
      NUSHT_TRY(deconv_trunc(q, ms));
    }
    NUSHT_TRY(join(p, s));
  }
  for (auto& b : p->buckets) {
    NUSHT_CUFFT(cufftSetStream(b.theta, s));
    NUSHT_CUFFT(cufftExecC2C(b.theta, (cufftComplex*)b.Ghat, (cufftComplex*)b.Ghat, CUFFT_INVERSE));
    if (b.tc) {
      dim3 gf(b.ntiles * BS_PAIRS / FOLD_PAIRS, b.L + 1);
      bucket_fold_ba_k<<<gf, 256, 0, s>>>(b.L, b.M, b.npairs, b.B, b.ntiles, b.memberL, b.Ghat, b.BA);
      if (b.ntc_work > 0)
        bucket_tc_k<true><<<b.ntc_work, T6_THREADS, T6_SMEM, s>>>(bucket_args(b), b.ntc_work, nullptr, b.tc_work,
                                                                  b.pt_off, nullptr, b.items, b.mfirst, b.ntiles,
                                                                  b.PT, b.BA, nullptr, b.cacc, p->status,
                                                                  p->test_giveup, b.tcg_a);
    } else {
      dim3 gf((b.npairs + FOLD_PAIRS - 1) / FOLD_PAIRS, b.L + 1);
      bucket_fold_k<<<gf, 256, 0, s>>>(b.L, b.M, b.npairs, b.B, b.memberL, b.Ghat, b.S);
    }
    if (b.tc) {
    } else if (b.table) {
      const size_t sm = (size_t)(BS_PAIRS * AT_PAD + BS_PAIRS * 2 * BK_COLS) * sizeof(float);
      if (b.nwork > 0)
        bucket_adj_tab_k<<<b.nwork, 256, sm, s>>>(bucket_args(b), b.items, b.offs, b.mfirst, b.work, b.nwork, b.P,
                                                  b.S, b.cacc);
    } else {
      NUSHT_TRY(launch_adj(b, s));
    }
    dim3 g((b.L + 1 + 3) / 4, b.L + 1);
    bucket_final_k<<<g, 256, 0, s>>>(b.L, b.M, b.B, b.memberL, b.cacc, b.leg->leg.ahat, b.leg->leg.pole_norm,
                                     b.Ghat, b.out_ptrs);
    NUSHT_CUDA(cudaGetLastError());
  }
  return NUSHT_OK;
}

// FP64 batched synthesis: per bucket the split coefficients, the tensor-core
// contraction into the members' ring sums and their poles; then every
// member's theta FFT (float pairs in and out), deconvolution, fine-grid FFT
// and interpolation on the forked streams.
int enqueue_synth_oz(nusht_batch_t p, void* const* d_map, cudaStream_t s) {
  for (auto& b : p->buckets) {
    oz_bs_k<<<b.L + 1, 256, 0, s>>>(b.L, b.B, b.ncg, b.memberL, reinterpret_cast<const double2* const*>(b.alm_ptrs),
                                    b.mfirst, b.obs_off, b.eBs, b.OBS);
    if (b.noz_s > 0)
      oz_tc_k<false><<<b.noz_s, OZ_THREADS, OZ_SMEM, s>>>(oz_args(b, false), b.noz_s, p->status, p->test_giveup);
    oz_poles_k<<<b.B, 256, 0, s>>>(b.M, b.memberL, reinterpret_cast<const double2* const*>(b.alm_ptrs),
                                   b.leg->leg.pole_norm, b.gout);
    NUSHT_CUDA(cudaGetLastError());
  }
  NUSHT_TRY(fork(p, s));
  for (int i = 0; i < p->nbatch; ++i) {
    nusht_plan_t q = p->sub[i];
    cudaStream_t ms = p->side[i % nusht_batch_s::NSIDE];
    const Bucket& b = p->buckets[p->bucket_of[i]];
    NUSHT_TRY(dfft_theta_pairs(q, b.gout_h[p->slot_of[i]], q->Ghat, -1, ms));
    NUSHT_TRY(deconv_pad(q, ms));
    NUSHT_TRY(fine_fft_c2r(q, ms));
    NUSHT_TRY(interp(q, d_map[i], ms));
  }
  NUSHT_TRY(join(p, s));
  return NUSHT_OK;
}

// FP64 batched adjoint: every member's spreading, fine-grid FFT, truncation
// and inverse theta FFT (float pairs) on the forked streams; then per bucket
// the folded split spectrum and the tensor-core contraction into the
// members' coefficients.
int enqueue_adjoint_oz(nusht_batch_t p, const void* const* d_map, cudaStream_t s) {
  NUSHT_TRY(fork(p, s));
  for (int i = 0; i < p->nbatch; ++i) {
    nusht_plan_t q = p->sub[i];
    cudaStream_t ms = p->side[i % nusht_batch_s::NSIDE];
    NUSHT_TRY(spread(q, d_map[i], ms));
    NUSHT_TRY(fine_fft_r2c(q, ms));
    NUSHT_TRY(deconv_trunc(q, ms));
    NUSHT_TRY(dfft_theta_pairs(q, q->Ghat, q->Ghat, 1, ms));
  }
  NUSHT_TRY(join(p, s));
  for (auto& b : p->buckets) {
    oz_fold_k<<<b.L + 1, 256, 0, s>>>(b.L, b.M, b.npairs, b.B, b.ncg, b.memberL, b.gh, b.items, b.mfirst, b.oba_off,
                                      b.eBa, b.OBA);
    oz_zero_k<<<dim3(b.L + 1, b.B), 128, 0, s>>>(b.M, b.memberL, b.mfirst, b.gh, b.leg->leg.pole_norm,
                                                 reinterpret_cast<double2* const*>(b.out_ptrs));
    if (b.noz_a > 0)
      oz_tc_k<true><<<b.noz_a, OZ_THREADS, OZ_SMEM, s>>>(oz_args(b, true), b.noz_a, p->status, p->test_giveup);
    NUSHT_CUDA(cudaGetLastError());
  }
  return NUSHT_OK;
}

// Member tables of the fused NUFFT stages (plan time): zero fill, spreading,
// interpolation and the deconvolution run as one launch each for every
// member; the fine-grid FFTs are the FP32 line kernels' two passes (one
// launch each) when every member uses them, else each member's cuFFT 2D
// plan.  They apply with the atomic spreading (not opts.deterministic);
// otherwise each member runs its own stages.
int build_fused(nusht_batch_t p) {
  p->fused = p->fused_sfft = false;
  if (p->opts.deterministic) return NUSHT_OK;
  int nsfft = 0;
  for (auto* q : p->sub) {
    if (q->pts.off == nullptr || q->dfft_fine) return NUSHT_OK;
    nsfft += q->sfft_fine ? 1 : 0;
  }
  if (nsfft != 0 && nsfft != p->nbatch) return NUSHT_OK;
  p->fused_sfft = nsfft == p->nbatch;
  std::vector<int> order(p->nbatch);
  for (int i = 0; i < p->nbatch; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p->sub[a]->sz.w < p->sub[b]->sz.w; });
  std::vector<NufftMember> nm(p->nbatch);
  std::vector<SfftMember> sm(p->nbatch);
  p->table_of.assign(p->nbatch, 0);
  p->nbw.clear();
  SfftLaunch& sl = p->sl;
  sl = SfftLaunch();
  int blk = 0, sub = 0, zero = 0, cols = 0, rows = 0, pad = 0, trunc = 0;
  for (int t = 0; t < p->nbatch; ++t) {
    const int i = order[t];
    nusht_plan_t q = p->sub[i];
    const nusht_sizes& z = q->sz;
    p->table_of[i] = t;
    if (p->nbw.empty() || p->nbw.back().w != z.w) {
      NufftBatch g;
      g.w = z.w;
      g.nm = t;  // first table position, turned into the count below
      p->nbw.push_back(g);
    }
    NufftBatch& g = p->nbw.back();
    NufftMember& a = nm[t];
    a.grid = static_cast<float*>(q->fine);
    a.cell = q->pts.cell;
    a.off = q->pts.off;
    a.perm = q->pts.perm;
    a.sub = q->pts.sub;
    a.stride = 2 * (z.n2 / 2 + 1);
    a.npts = q->pts.npts;
    a.n1 = z.n1;
    a.n2 = z.n2;
    a.nbins2 = q->pts.nbins2;
    a.bin = q->pts.bin > 0 ? q->pts.bin : 32;
    a.spread_rows = q->pts.spread_rows;
    a.beta = (float)z.beta;
    a.Gh = static_cast<float2*>(q->Ghat);
    a.d1 = q->deconv1;
    a.d2 = q->deconv2;
    a.lmax = z.lmax;
    a.mmax = z.mmax;
    a.M = z.M;
    a.blk0 = blk;
    a.sub0 = sub;
    a.zero0 = zero;
    a.pad0 = pad;
    a.trunc0 = trunc;
    pad += ((z.n2 / 2 + 1 + 31) / 32) * ((z.n1 + 31) / 32);
    trunc += ((z.M + 31) / 32) * ((z.mmax + 1 + 31) / 32);
    blk += (int)((q->pts.npts + 127) / 128);
    sub += q->pts.nsub;
    zero += (int)((z.n1 * a.stride + ZERO_CHUNK - 1) / ZERO_CHUNK);
    g.bin = std::max(g.bin, a.bin);
    if (p->fused_sfft) {
      SfftMember& f = sm[t];
      sfft_member(q, f);
      f.col0 = cols;
      f.row0 = rows;
      cols += z.mmax + 1;
      rows += q->pts.nrowpairs;  // the row pairs the member's points reach
      sl.maxn1 = std::max(sl.maxn1, z.n1);
      sl.maxn2 = std::max(sl.maxn2, z.n2);
    }
  }
  NUSHT_TRY(dev_alloc((void**)&p->d_nmem, nm.size() * sizeof(NufftMember), &p->bytes));
  if (p->fused_sfft) NUSHT_TRY(dev_alloc((void**)&p->d_smem, sm.size() * sizeof(SfftMember), &p->bytes));
  NUSHT_TRY(dev_alloc((void**)&p->d_maps, p->nbatch * sizeof(float*), &p->bytes));
  NUSHT_CUDA(cudaMemcpy(p->d_nmem, nm.data(), nm.size() * sizeof(NufftMember), cudaMemcpyHostToDevice));
  if (p->fused_sfft)
    NUSHT_CUDA(cudaMemcpy(p->d_smem, sm.data(), sm.size() * sizeof(SfftMember), cudaMemcpyHostToDevice));
  // each width group: its slice of the member table; block counts relative to
  // the group's first member (the kernels subtract blk0 / sub0 of members of
  // the same table, so a group's launch starts at its first member's offsets)
  for (size_t k = 0; k < p->nbw.size(); ++k) {
    NufftBatch& g = p->nbw[k];
    const int t0 = g.nm, t1 = k + 1 < p->nbw.size() ? p->nbw[k + 1].nm : p->nbatch;
    g.mem = p->d_nmem + t0;
    g.nm = t1 - t0;
    g.nblk = (t1 < p->nbatch ? nm[t1].blk0 : blk) - nm[t0].blk0;
    g.nsub = (t1 < p->nbatch ? nm[t1].sub0 : sub) - nm[t0].sub0;
    g.nzero = 0;
    g.blk_base = nm[t0].blk0;
    g.sub_base = nm[t0].sub0;
    g.map_base = t0;
  }
  p->nball.mem = p->d_nmem;
  p->nball.nm = p->nbatch;
  p->nball.nzero = zero;
  p->nball.npad = pad;
  p->nball.ntrunc = trunc;
  sl.mem = p->d_smem;
  sl.nm = p->nbatch;
  sl.ncols = cols;
  sl.nrows = rows;
  p->fused = true;
  return NUSHT_OK;
}

// pointer tables of every bucket (plan-owned device arrays, written before a
// capture; the captured kernels read them)
int set_tables(nusht_batch_t p, const void* const* in, void* const* out, bool synth) {
  if (p->fused) {
    std::vector<float*> maps(p->nbatch);
    for (int i = 0; i < p->nbatch; ++i)
      maps[p->table_of[i]] = static_cast<float*>(synth ? out[i] : const_cast<void*>(in[i]));
    NUSHT_CUDA(cudaMemcpy(p->d_maps, maps.data(), p->nbatch * sizeof(float*), cudaMemcpyHostToDevice));
  }
  for (auto& b : p->buckets) {
    std::vector<const void*> vin(BK_MAXB, nullptr);
    std::vector<void*> vout(BK_MAXB, nullptr);
    for (int k = 0; k < b.B; ++k) {
      if (synth)
        vin[k] = in[b.members[k]];
      else
        vout[k] = out[b.members[k]];
    }
    if (synth)
      NUSHT_CUDA(cudaMemcpy(b.alm_ptrs, vin.data(), BK_MAXB * sizeof(void*), cudaMemcpyHostToDevice));
    else
      NUSHT_CUDA(cudaMemcpy(b.out_ptrs, vout.data(), BK_MAXB * sizeof(void*), cudaMemcpyHostToDevice));
  }
  return NUSHT_OK;
}

}  // namespace
}  // namespace nusht

using namespace nusht;

extern "C" {

int nusht_plan_many(nusht_batch_t* out, int nbatch, const int* lmax, const int64_t* npts, const double* const* d_pts,
                    double eps, int precision, const nusht_opts* opts, nusht_stream_t stream) {
  if (!out) return set_error(NUSHT_EINVAL, "out is NULL");
  *out = nullptr;
  if (nbatch < 1 || nbatch > 4096) return set_error(NUSHT_EINVAL, "nbatch must be in [1, 4096]");
  if (!lmax || !npts || !d_pts) return set_error(NUSHT_EINVAL, "null array argument");
  if (precision != NUSHT_MIXED && precision != NUSHT_FP64)
    return set_error(NUSHT_EUNSUPPORTED, "batched transforms run in NUSHT_MIXED or NUSHT_FP64 precision");
  for (int i = 0; i < nbatch; ++i) {
    nusht_sizes z;
    NUSHT_TRY(choose_sizes(lmax[i], lmax[i], eps, precision, opts, &z));
    if (lmax[i] > 4095) return set_error(NUSHT_EUNSUPPORTED, "batched transforms support lmax <= 4095");
    if (npts[i] < 0 || npts[i] > 0x7fffffffLL) return set_error(NUSHT_EINVAL, "npts must be in [0, 2^31)");
    if (npts[i] > 0 && !d_pts[i]) return set_error(NUSHT_EINVAL, "null point array");
  }
  nusht_batch_t p = new (std::nothrow) nusht_batch_s();
  if (!p) return set_error(NUSHT_ENOMEM, "host allocation failed");
  cudaStream_t s = (cudaStream_t)stream;
  int st = NUSHT_OK;
  do {
    {
      cudaError_t e = cudaGetDevice(&p->device);
      if (e != cudaSuccess) {
        st = cuda_status(e, "cudaGetDevice");
        break;
      }
    }
    p->nbatch = nbatch;
    p->precision = precision;
    p->eps = eps;
    if (opts) p->opts = *opts;
    p->L.assign(lmax, lmax + nbatch);
    p->npts.assign(npts, npts + nbatch);
    {
      const char* tg = std::getenv("NUSHT_TEST_TC_GIVEUP");
      p->test_giveup = (tg && std::atoi(tg) == 1) ? 1 : 0;
    }
    if ((st = set_adj_smem()) != NUSHT_OK) break;
    if ((st = dev_alloc((void**)&p->status, sizeof(int), &p->bytes)) != NUSHT_OK) break;
    {
      cudaError_t e = cudaMemsetAsync(p->status, 0, sizeof(int), s);
      if (e != cudaSuccess) {
        st = cuda_status(e, "cudaMemsetAsync");
        break;
      }
    }
    // per-triple costs on GB300: FP64 recurrence (2 FP64 instructions at
    // ~70 % of 0.6e12/s), one FP32 FMA per column at ~50 % of 37e12/s, and a
    // fixed cost per bucket
    const auto groups = group_members(p->L, 4.6e-12, 5.4e-14, 2e-4);
    p->bucket_of.assign(nbatch, -1);
    p->slot_of.assign(nbatch, -1);
    p->buckets.resize(groups.size());
    for (size_t g = 0; g < groups.size() && st == NUSHT_OK; ++g) {
      Bucket& b = p->buckets[g];
      b.members = groups[g];
      b.B = (int)b.members.size();
      for (int k = 0; k < b.B; ++k) {
        b.L = std::max(b.L, p->L[b.members[k]]);
        p->bucket_of[b.members[k]] = (int)g;
        p->slot_of[b.members[k]] = k;
      }
      st = (precision == NUSHT_FP64) ? bucket_build_oz(p, b, s) : bucket_build(p, b, s);
    }
    if (st != NUSHT_OK) break;
    p->sub.assign(nbatch, nullptr);
    // members' fine-grid FFTs: by default this library's FP32 line kernels
    // (two launches per direction for the whole batch); -1 keeps cuFFT
    nusht_opts sub_opts = p->opts;
    if (sub_opts.fft_kernels == 0) sub_opts.fft_kernels = 1;
    for (int i = 0; i < nbatch && st == NUSHT_OK; ++i) {
      const Bucket& b = p->buckets[p->bucket_of[i]];
      PlanRole role;
      role.legendre = false;
      role.nufft = true;
      role.M_override = b.M;
      if (precision == NUSHT_FP64)
        role.theta = true;  // own theta FFT and theta spectrum, float pairs
      else
        role.ghat_external = b.Ghat + (size_t)p->slot_of[i] * (b.L + 1) * b.M;
      st = plan_create(&p->sub[i], p->L[i], p->L[i], p->npts[i], d_pts[i], eps, precision, &sub_opts, s, role);
      if (st == NUSHT_OK) p->bytes += p->sub[i]->bytes;
      if (st == NUSHT_OK && precision == NUSHT_FP64 && !(p->sub[i]->dfft_theta && p->sub[i]->dfft_fine))
        st = set_error(NUSHT_EUNSUPPORTED, "FP64 batched plans need the double-float FFT kernels (fft_kernels >= 0)");
    }
    if (st != NUSHT_OK) break;
    if (precision == NUSHT_FP64) {
      for (auto& b : p->buckets) {
        std::vector<const void*> gh(BK_MAXB, nullptr);
        for (int k = 0; k < b.B; ++k) gh[k] = p->sub[b.members[k]]->Ghat;
        cudaError_t e = cudaMemcpy(b.gh, gh.data(), BK_MAXB * sizeof(void*), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
          st = cuda_status(e, "member table upload");
          break;
        }
      }
      if (st != NUSHT_OK) break;
    }
    if ((st = build_fused(p)) != NUSHT_OK) break;
    {
      cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
      for (int k = 0; k < nusht_batch_s::NSIDE && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&p->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[k], cudaEventDisableTiming);
      }
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
      if (e != cudaSuccess) st = cuda_status(e, "stream / event creation");
    }
  } while (false);
  if (st != NUSHT_OK) {
    cudaStreamSynchronize(s);
    batch_free(p);
    return st;
  }
  *out = p;
  return NUSHT_OK;
}

static int run_many(nusht_batch_t p, const void* const* in, void* const* out, nusht_stream_t stream, bool synth) {
  if (!p) return set_error(NUSHT_EINVAL, "batch plan is NULL");
  if (!in || !out) return set_error(NUSHT_EINVAL, "null pointer array");
  // a member without points may pass NULL for its map (input of the
  // adjoint, output of the synthesis)
  for (int i = 0; i < p->nbatch; ++i) {
    const bool has_pts = p->npts[i] > 0;
    const bool bad = synth ? (!in[i] || (!out[i] && has_pts)) : ((!in[i] && has_pts) || !out[i]);
    if (bad) return set_error(NUSHT_EINVAL, "null member buffer");
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<const void*> vin(in, in + p->nbatch);
  std::vector<void*> vout(out, out + p->nbatch);
  cudaGraphExec_t& ex = synth ? p->gs : p->ga;
  std::vector<const void*>& kin = synth ? p->gs_in : p->ga_in;
  std::vector<void*>& kout = synth ? p->gs_out : p->ga_out;
  if (!ex || kin != vin || kout != vout) {
    if (ex) {
      NUSHT_CUDA(cudaStreamSynchronize(s));
      cudaGraphExecDestroy(ex);
      ex = nullptr;
    }
    NUSHT_TRY(set_tables(p, in, out, synth));
    cudaGraph_t g = nullptr;
    NUSHT_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    int st;
    if (p->precision == NUSHT_FP64)
      st = synth ? enqueue_synth_oz(p, out, p->cap) : enqueue_adjoint_oz(p, in, p->cap);
    else
      st = synth ? enqueue_synth(p, out, p->cap) : enqueue_adjoint(p, in, p->cap);
    cudaError_t e = cudaStreamEndCapture(p->cap, &g);
    if (st != NUSHT_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ex = nullptr;
      return cuda_status(e, "cudaGraphInstantiate");
    }
    kin = vin;
    kout = vout;
  }
  NUSHT_CUDA(cudaGraphLaunch(ex, s));
  return NUSHT_OK;
}

int nusht_synth_many(nusht_batch_t p, const void* const* d_alm, void* const* d_map, nusht_stream_t stream) {
  return run_many(p, d_alm, d_map, stream, true);
}

int nusht_adjoint_many(nusht_batch_t p, const void* const* d_map, void* const* d_alm, nusht_stream_t stream) {
  return run_many(p, d_map, d_alm, stream, false);
}

int nusht_destroy_many(nusht_batch_t p) {
  batch_free(p);
  return NUSHT_OK;
}

int nusht_batch_status(nusht_batch_t p, nusht_stream_t stream) {
  if (!p) return set_error(NUSHT_EINVAL, "batch plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  NUSHT_CUDA(cudaStreamSynchronize(s));
  int flag = 0;
  NUSHT_CUDA(cudaMemcpy(&flag, p->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    NUSHT_CUDA(cudaMemset(p->status, 0, sizeof(int)));
    return set_error(NUSHT_ETIMEOUT, "a tensor-core contraction block gave up waiting for its MMAs");
  }
  return NUSHT_OK;
}

int nusht_batch_schedule(nusht_batch_t p, int bucket, int* chunks_synth, int* chunks_adjoint) {
  if (!p || bucket < 0 || bucket >= (int)p->buckets.size()) return set_error(NUSHT_EINVAL, "bad bucket");
  const nusht::Bucket& b = p->buckets[bucket];
  if (chunks_synth) *chunks_synth = b.tc ? b.tcg_s : 0;
  if (chunks_adjoint) *chunks_adjoint = b.tc ? b.tcg_a : 0;
  return NUSHT_OK;
}

int nusht_batch_path(nusht_batch_t p, int bucket) {
  if (!p || bucket < 0 || bucket >= (int)p->buckets.size()) return -1;
  const nusht::Bucket& b = p->buckets[bucket];
  return b.oz ? 3 : (b.tc ? 2 : (b.table ? 1 : 0));
}

int nusht_batch_info(nusht_batch_t p, int* nbuckets, int* bucket_of, int* bucket_lmax, int64_t* bytes_device) {
  if (!p) return set_error(NUSHT_EINVAL, "batch plan is NULL");
  if (nbuckets) *nbuckets = (int)p->buckets.size();
  if (bucket_of)
    for (int i = 0; i < p->nbatch; ++i) bucket_of[i] = p->bucket_of[i];
  if (bucket_lmax)
    for (size_t g = 0; g < p->buckets.size(); ++g) bucket_lmax[g] = p->buckets[g].L;
  if (bytes_device) *bytes_device = (int64_t)p->bytes;
  return NUSHT_OK;
}

}  // extern "C"
