// nufft.cu -- the type 2 / type 1 NUFFT steps N and N^dagger (Sec. 2.2,
// Sec. 3) on the doubled torus, with the exponential-of-semicircle kernel
// psi(z) = exp(beta (sqrt(1 - z^2) - 1)), |z| <= 1, of width w fine-grid cells:
//   * point set-up: fold (theta, phi) onto [0, 2 pi)^2, first tap and
//     fractional offset in double, bin sort (tiles of bin x bin cells, bin chosen
//     by the plan: 16 for FP64 plans with w <= 17 and float-pair arithmetic,
//     32 otherwise, or by the autotuner),
//     FP64 kernel values per point;
//   * deconv_pad / deconv_trunc: divide by the kernel's Fourier transform,
//     zero-pad / truncate between the theta spectrum [m][k] and the fine
//     spectrum [k][m] (a tiled transpose through shared memory);
//   * interp: f_i = sum_{a,b} psi1_a psi2_b u[i1 + a, i2 + b]  (type 2);
//   * spread: u[i1 + a, i2 + b] += f_i psi1_a psi2_b  (type 1), accumulated
//     in a shared-memory tile per bin and flushed once with atomics.
// Spreading and interpolation read the same kernel values, so the fast
// adjoint is the exact transpose of the fast synthesis.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "nusht_internal.cuh"
#include "dfloat.cuh"

namespace nusht {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SUBMAX = 256;   // points per spreading subproblem
// FP32 spreading: the subproblem's points staged in shared memory after the
// tile (float4 per point, one padding slot after every 8, so that lanes that
// read every Lr-th point hit distinct banks)
constexpr int SP_SLOTS = SUBMAX + SUBMAX / 8;
__device__ __forceinline__ int sp_idx(int k) { return k + (k >> 3); }
inline size_t spread_f_smem(int tw) { return (size_t)((tw * tw + 3) & ~3) * 4 + (size_t)SP_SLOTS * 16; }
constexpr int WMAX = ES_WMAX;
constexpr int NRMAX = (WMAX * WMAX + 31) / 32;  // rounds of 32 cells for a w x w footprint

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

__device__ __forceinline__ double es_psi(double z, double beta) {
  double r = 1.0 - z * z;
  return r > 0.0 ? exp(beta * (sqrt(r) - 1.0)) : 0.0;
}
// exp(beta (sqrt(1 - z^2) - 1)) as 2^(beta log2(e) (sqrt(1 - z^2) - 1)): exp2f
// is the shorter of the two on the GPU; spreading and interpolation share it,
// so the FP32 adjoint stays the exact transpose
__device__ __forceinline__ float es_psif(float z, float beta) {
  float r = 1.0f - z * z;
  return r > 0.0f ? exp2f((beta * 1.44269504088896341f) * (sqrtf(r) - 1.0f)) : 0.0f;
}
// d psi / dz
__device__ __forceinline__ double es_dpsi(double z, double beta) {
  double r = 1.0 - z * z;
  if (!(r > 0.0)) return 0.0;
  double sr = sqrt(r);
  return exp(beta * (sr - 1.0)) * beta * (-z) / sr;
}
__device__ __forceinline__ float es_dpsif(float z, float beta) {
  float r = 1.0f - z * z;
  if (!(r > 0.0f)) return 0.0f;
  float sr = sqrtf(r);
  return expf(beta * (sr - 1.0f)) * beta * (-z) / sr;
}

// fold a coordinate onto [0, 2 pi) and split it into the first kernel tap
// (wrapped to [0, n)) and the offset t - i0 in (w/2 - 1, w/2]
__device__ __forceinline__ void tap(double x, int n, int w, int& i0w, double& off) {
  const double twopi = 6.283185307179586476925286766559;
  double xr = x - twopi * floor(x * (1.0 / twopi));
  if (xr >= twopi || xr < 0.0) xr = 0.0;
  double t = xr * ((double)n / twopi);
  double i0 = ceil(t - 0.5 * w);
  off = t - i0;
  int i = (int)i0;
  if (i < 0) i += n;
  if (i >= n) i -= n;
  i0w = i;
}

// sort key of a point: its bin (row-major over the bins), then its first tap
// row-major inside the bin, key = bin * binsz^2 + (i1 mod binsz) binsz + i2 mod binsz
__global__ void prep_k(const double* __restrict__ pts, int64_t npts, int n1, int n2, int w, int nb2, int binsz,
                       int64_t* __restrict__ key) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  int i1, i2;
  double o1, o2;
  tap(pts[2 * i], n1, w, i1, o1);
  tap(pts[2 * i + 1], n2, w, i2, o2);
  const int b1 = i1 / binsz, b2 = i2 / binsz;
  const int64_t bin = (int64_t)b1 * nb2 + b2;
  key[i] = bin * binsz * binsz + (int64_t)(i1 - b1 * binsz) * binsz + (i2 - b2 * binsz);
}

// sorted point s <- caller's point perm[s]: first taps, and kernel values
// (FP64: psi[s][0..w) along theta then psi[s][w..2w) along phi) or the
// offsets (MIXED, kernel evaluated on the fly in float)
__global__ void gather_k(const double* __restrict__ pts, const int* __restrict__ perm, int64_t npts, int n1, int n2,
                         int w, double beta, int* __restrict__ cell, double* __restrict__ psi,
                         float2* __restrict__ psid, float* __restrict__ offf, double* __restrict__ xy) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= npts) return;
  const int i = perm[s];
  int i1, i2;
  double o1, o2;
  const double th = pts[2 * (int64_t)i], ph = pts[2 * (int64_t)i + 1];
  xy[2 * s] = th;
  xy[2 * s + 1] = ph;
  tap(th, n1, w, i1, o1);
  tap(ph, n2, w, i2, o2);
  cell[2 * s] = i1;
  cell[2 * s + 1] = i2;
  const double sc = 2.0 / w;
  if (psi) {
    double* ps = psi + s * 2 * w;
    for (int a = 0; a < w; ++a) ps[a] = es_psi((o1 - a) * sc, beta);
    for (int b = 0; b < w; ++b) ps[w + b] = es_psi((o2 - b) * sc, beta);
  }
  if (psid) {
    float2* ps = psid + s * 2 * w;
    for (int a = 0; a < w; ++a) {
      const double v = es_psi((o1 - a) * sc, beta);
      const float h = __double2float_rn(v);
      ps[a] = make_float2(h, __double2float_rn(v - (double)h));
    }
    for (int b = 0; b < w; ++b) {
      const double v = es_psi((o2 - b) * sc, beta);
      const float h = __double2float_rn(v);
      ps[w + b] = make_float2(h, __double2float_rn(v - (double)h));
    }
  }
  if (offf) {
    offf[2 * s] = (float)o1;
    offf[2 * s + 1] = (float)o2;
  }
}

// ---------------------------------------------------------------------------
// deconvolution with transpose
// ---------------------------------------------------------------------------
// fine spectrum H[k1][m] (n1 x n2h) from the theta spectrum Ghat[m][kk] (M)
template <typename T>
__device__ __forceinline__ void deconv_pad_tile(const typename V2<T>::t* __restrict__ Gh,
                                                typename V2<T>::t* __restrict__ H, int lmax, int mmax, int M, int n1,
                                                int n2h, const double* __restrict__ d1,
                                                const double* __restrict__ d2, int bx, int by) {
  using T2 = typename V2<T>::t;
  __shared__ T2 tile[32][33];
  const int k0 = by * 32, m0 = bx * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  // is this row tile entirely in the zero band lmax < k1 < n1 - lmax?
  const bool zero_rows = (k0 > lmax) && (k0 + 31 < n1 - lmax);
  const bool zero_cols = m0 > mmax;
  if (!zero_rows && !zero_cols) {
    // load Ghat[m0 + r][kk(k0 + tx)] for r = ty, ty + 8, ...
    const int k1 = k0 + tx;
    int k = 0;
    bool kv = false;
    if (k1 < n1) {
      if (k1 <= lmax) {
        k = k1;
        kv = true;
      } else if (k1 >= n1 - lmax) {
        k = k1 - n1;
        kv = true;
      }
    }
    const int kk = kv ? (k < 0 ? k + M : k) : 0;
    const double f1 = kv ? d1[k + lmax] : 0.0;
    for (int r = ty; r < 32; r += 8) {
      const int m = m0 + r;
      T2 v;
      v.x = v.y = (T)0;
      if (kv && m <= mmax) {
        T2 g = Gh[(size_t)m * M + kk];
        const double f = f1 * d2[m];
        v.x = (T)(g.x * f);
        v.y = (T)(g.y * f);
      }
      tile[r][tx] = v;
    }
    __syncthreads();
  }
  for (int r = ty; r < 32; r += 8) {
    const int k1 = k0 + r, m = m0 + tx;
    if (k1 >= n1 || m >= n2h) continue;
    T2 v;
    if (zero_rows || zero_cols) {
      v.x = v.y = (T)0;
    } else {
      v = tile[tx][r];
    }
    H[(size_t)k1 * n2h + m] = v;
  }
}

// theta spectrum Gt[m][kk] from the fine spectrum H[k1][m] (after the r2c FFT)
template <typename T>
__device__ __forceinline__ void deconv_trunc_tile(const typename V2<T>::t* __restrict__ H,
                                                  typename V2<T>::t* __restrict__ Gt, int lmax, int mmax, int M,
                                                  int n1, int n2h, const double* __restrict__ d1,
                                                  const double* __restrict__ d2, int bx, int by) {
  using T2 = typename V2<T>::t;
  __shared__ T2 tile[32][33];
  const int kk0 = bx * 32, m0 = by * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  // load H[k1(kk0 + r)][m0 + tx]
  for (int r = ty; r < 32; r += 8) {
    const int kk = kk0 + r, m = m0 + tx;
    T2 v;
    v.x = v.y = (T)0;
    if (kk < M && m <= mmax) {
      const int k = (kk <= M / 2) ? kk : kk - M;
      if (k >= -lmax && k <= lmax) {
        const int k1 = k < 0 ? k + n1 : k;
        T2 h = H[(size_t)k1 * n2h + m];
        const double f = d1[k + lmax] * d2[m];
        v.x = (T)(h.x * f);
        v.y = (T)(h.y * f);
      }
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int m = m0 + r, kk = kk0 + tx;
    if (m <= mmax && kk < M) Gt[(size_t)m * M + kk] = tile[tx][r];
  }
}

template <typename T>
__global__ void deconv_pad_k(const typename V2<T>::t* __restrict__ Gh, typename V2<T>::t* __restrict__ H, int lmax,
                             int mmax, int M, int n1, int n2h, const double* __restrict__ d1,
                             const double* __restrict__ d2) {
  deconv_pad_tile<T>(Gh, H, lmax, mmax, M, n1, n2h, d1, d2, blockIdx.x, blockIdx.y);
}

template <typename T>
__global__ void deconv_trunc_k(const typename V2<T>::t* __restrict__ H, typename V2<T>::t* __restrict__ Gt, int lmax,
                               int mmax, int M, int n1, int n2h, const double* __restrict__ d1,
                               const double* __restrict__ d2) {
  deconv_trunc_tile<T>(H, Gt, lmax, mmax, M, n1, n2h, d1, d2, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// CMB lensing pointing (App. C): the point (theta, phi) moved along the
// geodesic that starts in the direction of the potential's gradient, by its
// length (Eq. pointing), with alpha_theta = dPhi/dtheta and
// alpha_phi = dPhi/dphi / sin(theta) (Eq. spin1deriv).  Evaluated in the
// frame turned by phi about the z axis, where n = (sin t, 0, cos t),
// e_theta = (cos t, 0, -sin t), e_phi = (0, 1, 0).  Writes theta' in [0, pi]
// and phi' in [0, 2 pi).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void deflect(double th, double ph, double gth, double gph, double* __restrict__ o) {
  double st, ct;
  sincos(th, &st, &ct);
  const double at = gth, ap = st != 0.0 ? gph / st : 0.0;
  const double a = sqrt(at * at + ap * ap);
  double sa, ca;
  sincos(a, &sa, &ca);
  const double sinc = a > 0.0 ? sa / a : 1.0;
  const double x = ca * st + sinc * at * ct;
  const double y = sinc * ap;
  const double z = ca * ct - sinc * at * st;
  const double twopi = 6.283185307179586476925286766559;
  double pp = ph + atan2(y, x);
  pp -= twopi * floor(pp * (1.0 / twopi));
  if (pp >= twopi || pp < 0.0) pp = 0.0;
  o[0] = atan2(sqrt(x * x + y * y), z);
  o[1] = pp;
}

// ---------------------------------------------------------------------------
// interpolation (type 2): one thread per sorted point; with GRAD the
// derivatives of the kernel give d/dtheta and d/dphi, written out, or with
// ptg turned into the deflected position (pointing), or with gpts multiplied
// by the cotangent cot (the position gradient of a loss, interleaved)
// ---------------------------------------------------------------------------
template <typename T, bool GRAD>
__global__ void __launch_bounds__(128) interp_k(const T* __restrict__ grid, int64_t stride, int n1, int n2, int w,
                                                float betaf, double beta, const int* __restrict__ cell,
                                                const double* __restrict__ psi, const float* __restrict__ offf,
                                                const double* __restrict__ xy, const int* __restrict__ perm,
                                                int64_t npts, T* __restrict__ out, T* __restrict__ dth,
                                                T* __restrict__ dph, double* __restrict__ ptg,
                                                const T* __restrict__ cot, double* __restrict__ gpts) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= npts) return;
  const int i1 = cell[2 * s], i2 = cell[2 * s + 1];
  T p1[WMAX], p2[WMAX], q1[WMAX], q2[WMAX];
  if (GRAD) {
    // kernel values and derivatives on the fly (not the hot path)
    int j1, j2;
    double o1, o2;
    tap(xy[2 * s], n1, w, j1, o1);
    tap(xy[2 * s + 1], n2, w, j2, o2);
    const double sc = 2.0 / w;
#pragma unroll
    for (int a = 0; a < WMAX; ++a) {
      if (a < w) {
        if (sizeof(T) == 8) {
          p1[a] = (T)es_psi((o1 - a) * sc, beta);
          p2[a] = (T)es_psi((o2 - a) * sc, beta);
          q1[a] = (T)es_dpsi((o1 - a) * sc, beta);
          q2[a] = (T)es_dpsi((o2 - a) * sc, beta);
        } else {
          const float scf = 2.0f / w;
          p1[a] = (T)es_psif(((float)o1 - a) * scf, betaf);
          p2[a] = (T)es_psif(((float)o2 - a) * scf, betaf);
          q1[a] = (T)es_dpsif(((float)o1 - a) * scf, betaf);
          q2[a] = (T)es_dpsif(((float)o2 - a) * scf, betaf);
        }
      }
    }
  } else if (psi) {
    const double* ps = psi + s * 2 * w;
#pragma unroll
    for (int a = 0; a < WMAX; ++a)
      if (a < w) {
        p1[a] = (T)ps[a];
        p2[a] = (T)ps[w + a];
      }
  } else {
    const float o1 = offf[2 * s], o2 = offf[2 * s + 1];
    const float scf = 2.0f / w;
#pragma unroll
    for (int a = 0; a < WMAX; ++a)
      if (a < w) {
        p1[a] = (T)es_psif((o1 - a) * scf, betaf);
        p2[a] = (T)es_psif((o2 - a) * scf, betaf);
      }
  }
  const bool wrap2 = i2 + w > n2;
  T acc = 0, g1 = 0, g2 = 0;
#pragma unroll
  for (int a = 0; a < WMAX; ++a) {
    if (a < w) {
      int r = i1 + a;
      if (r >= n1) r -= n1;
      const T* row = grid + (int64_t)r * stride;
      T in = 0, ind = 0;
      if (!wrap2) {
#pragma unroll
        for (int b = 0; b < WMAX; ++b)
          if (b < w) {
            const T u = row[i2 + b];
            in = fma(p2[b], u, in);
            if (GRAD) ind = fma(q2[b], u, ind);
          }
      } else {
#pragma unroll
        for (int b = 0; b < WMAX; ++b)
          if (b < w) {
            int c = i2 + b;
            if (c >= n2) c -= n2;
            const T u = row[c];
            in = fma(p2[b], u, in);
            if (GRAD) ind = fma(q2[b], u, ind);
          }
      }
      acc = fma(p1[a], in, acc);
      if (GRAD) {
        g1 = fma(q1[a], in, g1);
        g2 = fma(p1[a], ind, g2);
      }
    }
  }
  const int i = perm[s];
  if (!GRAD) {
    out[i] = acc;
  } else {
    // d/dx psi((x - x_j)/alpha) = psi'(z) / alpha, alpha = w pi / n
    const T a1 = (T)((double)n1 / (w * 3.14159265358979323846));
    const T a2 = (T)((double)n2 / (w * 3.14159265358979323846));
    if (ptg) {
      deflect(xy[2 * s], xy[2 * s + 1], (double)(g1 * a1), (double)(g2 * a2), ptg + 2 * (int64_t)i);
      return;
    }
    if (gpts) {
      const double c = (double)cot[i];
      gpts[2 * (int64_t)i] = c * (double)(g1 * a1);
      gpts[2 * (int64_t)i + 1] = c * (double)(g2 * a2);
      return;
    }
    if (dth) dth[i] = g1 * a1;
    if (dph) dph[i] = g2 * a2;
  }
}

// ---------------------------------------------------------------------------
// spreading (type 1): one warp per subproblem, one point at a time, the
// w x w cells of a point spread over the lanes (no two lanes share a cell),
// accumulated in a shared-memory tile with halo, flushed once with atomics
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(32) spread_k(T* __restrict__ grid, int64_t stride, int n1, int n2, int w, int nb2,
                                               int binsz, float betaf, const int* __restrict__ sub,
                                               const int* __restrict__ cell,
                                               const double* __restrict__ psi, const float* __restrict__ offf,
                                               const int* __restrict__ perm, const T* __restrict__ f,
                                               T* __restrict__ scratch) {
  extern __shared__ unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  const int lane = threadIdx.x;
  const int tw = binsz + w - 1;
  const int bin = sub[3 * blockIdx.x], start = sub[3 * blockIdx.x + 1], cnt = sub[3 * blockIdx.x + 2];
  const int r0 = (bin / nb2) * binsz, c0 = (bin % nb2) * binsz;
  for (int t = lane; t < tw * tw; t += 32) tile[t] = (T)0;
  __syncwarp();
  // this lane's cells of a point: (a, b) for idx = lane + 32 t < w^2
  const int nc = w * w;
  int ca[NRMAX], cb[NRMAX];
#pragma unroll
  for (int t = 0; t < NRMAX; ++t) {
    int idx = lane + 32 * t;
    ca[t] = idx < nc ? idx / w : 0;
    cb[t] = idx < nc ? idx % w : 0;
  }
  const float scf = 2.0f / w;
  for (int q = 0; q < cnt; ++q) {
    const int64_t s = (int64_t)start + q;
    const int lr = cell[2 * s] - r0, lc = cell[2 * s + 1] - c0;
    const T fv = f[perm[s]];
    // lane a < w: f psi1_a (k1) and psi2_a (k2)
    T k1 = 0, k2 = 0;
    if (lane < w) {
      if (psi) {
        k1 = (T)psi[s * 2 * w + lane];
        k2 = (T)psi[s * 2 * w + w + lane];
      } else {
        k1 = (T)es_psif((offf[2 * s] - lane) * scf, betaf);
        k2 = (T)es_psif((offf[2 * s + 1] - lane) * scf, betaf);
      }
      k1 *= fv;
    }
#pragma unroll
    for (int t = 0; t < NRMAX; ++t) {
      if (32 * t < nc) {
        const T va = __shfl_sync(FULL, k1, ca[t]);
        const T vb = __shfl_sync(FULL, k2, cb[t]);
        if (lane + 32 * t < nc) {
          T* cellp = tile + (lr + ca[t]) * tw + (lc + cb[t]);
          *cellp = fma(va, vb, *cellp);
        }
      }
    }
    __syncwarp();
  }
  __syncwarp();
  if (scratch) {  // deterministic: the whole tile to this subproblem's slot
    T* dst = scratch + (size_t)blockIdx.x * tw * tw;
    for (int t = lane; t < tw * tw; t += 32) dst[t] = tile[t];
    return;
  }
  for (int t = lane; t < tw * tw; t += 32) {
    const T v = tile[t];
    if (v != (T)0) {
      int r = r0 + t / tw, c = c0 + t % tw;
      while (r >= n1) r -= n1;
      while (c >= n2) c -= n2;
      atomicAdd(grid + (int64_t)r * stride + c, v);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 mode in double-float (FP32 pipe).  Both kernels work per spreading
// subproblem (a bin of binsz x binsz first taps, up to SUBMAX points) with the
// bin's fine-grid tile (bin + halo, wrapped) in shared memory as float pairs:
//   interpolation: the tile is loaded with coalesced row reads, each double
//     split once on the way in (integer operations); one thread per point
//     then reads its w x w taps from shared memory;
//   spreading: one warp per subproblem, the w x w cells of a point spread over
//     the lanes (no two lanes share a cell); the subproblem's taps and values
//     are staged in shared memory first and each point's kernel values are
//     fetched one point ahead; the tile is flushed as doubles with FP64
//     atomics, so the r2c FFT input stays FP64.
// Products are exact float-pair products, sums two-sum accumulations.
// ---------------------------------------------------------------------------
constexpr int IDF_THREADS = 128;

template <int W>
__global__ void __launch_bounds__(IDF_THREADS) interp_df_k(const double* __restrict__ grid, int64_t stride, int n1,
                                                           int n2, int nb2, int binsz, const int* __restrict__ sub,
                                                           const int* __restrict__ cell,
                                                           const float2* __restrict__ psi,
                                                           const int* __restrict__ perm, double* __restrict__ out) {
  extern __shared__ unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);
  const int tw = binsz + W - 1;
  const int bin = sub[3 * blockIdx.x], start = sub[3 * blockIdx.x + 1], cnt = sub[3 * blockIdx.x + 2];
  const int r0 = (bin / nb2) * binsz, c0 = (bin % nb2) * binsz;
  for (int e = threadIdx.x; e < tw * tw; e += IDF_THREADS) {
    const int r = e / tw, c = e - r * tw;
    const int gr = (r0 + r) % n1, gc = (c0 + c) % n2;  // the halo may wrap more than once on tiny grids
    float h, l;
    df_split(grid[(int64_t)gr * stride + gc], h, l);
    tile[e] = make_float2(h, l);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < cnt; q += IDF_THREADS) {
    const int64_t s = (int64_t)start + q;
    const int lr = cell[2 * s] - r0, lc = cell[2 * s + 1] - c0;
    const float2* ps = psi + s * 2 * W;
    float2 p2[W];
#pragma unroll
    for (int b = 0; b < W; ++b) p2[b] = ps[W + b];
    float ah = 0.f, al = 0.f;
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
      const float2* trow = tile + (lr + a) * tw + lc;
      float ih = 0.f, il = 0.f;
#pragma unroll
      for (int b = 0; b < W; ++b) {
        const float2 u = trow[b];
        df_mac(ih, il, p2[b].x, p2[b].y, u.x, u.y);
      }
      const float2 p1 = ps[a];
      df_mac(ah, al, p1.x, p1.y, ih, il);
    }
    out[perm[s]] = df_value(ah, al);
  }
}

// d psi / dz over psi for the ES kernel, -beta z / sqrt(1 - z^2), as a float
// pair at z = (o - a) 2 / W (o: the point's offset from its first tap);
// 0 where 1 - z^2 <= 0 (psi is 0 there)
template <int W>
__device__ __forceinline__ float2 es_dfac(float oh, float ol, int a, float2 beta) {
  // 2 / W as a float pair (folded at compile time)
  constexpr double cw = 2.0 / W;
  constexpr float cwh = (float)cw;
  constexpr float cwl = (float)(cw - (double)cwh);
  // o - a (a is an exact small integer), then z = (o - a) 2 / W
  float dh = 0.f, dl = 0.f;
  df_add(dh, dl, oh, ol);
  df_add(dh, dl, (float)-a, 0.f);
  const float2 z = df_mul(make_float2(dh, dl), make_float2(cwh, cwl));
  // r = 1 - z^2
  const float2 zz = df_mul(z, z);
  float rh = 1.0f, rl = 0.0f;
  df_add(rh, rl, -zz.x, -zz.y);
  if (!(rh > 0.0f)) return make_float2(0.0f, 0.0f);
  // s = sqrt(r): one Newton correction of the float root
  const float s0 = sqrtf(rh);
  const float e = __fadd_rn(__fmaf_rn(-s0, s0, rh), rl);
  float sh = s0, sl = __fdiv_rn(e, 2.0f * s0);
  {
    const float t = __fadd_rn(sh, sl);
    sl = __fsub_rn(sl, __fsub_rn(t, sh));
    sh = t;
  }
  // -beta z / s
  const float2 n = df_mul(beta, z);
  const float g0 = __fdiv_rn(n.x, sh);
  const float pr = __fmul_rn(g0, sh);
  const float pe = __fmaf_rn(g0, sh, -pr);
  const float rm = __fadd_rn(__fsub_rn(__fsub_rn(n.x, pr), pe), __fsub_rn(n.y, __fmul_rn(g0, sl)));
  const float g1 = __fdiv_rn(rm, sh);
  const float gh = __fadd_rn(g0, g1);
  return make_float2(-gh, -__fsub_rn(g1, __fsub_rn(gh, g0)));
}

// FP64-mode gradient interpolation on the double-float tile (the tile and
// the kernel values as in interp_df_k):
//   d f / d theta = (n1 / (W pi)) sum_a psi1'_a sum_b psi2_b u_ab,
//   d f / d phi   = (n2 / (W pi)) sum_a psi1_a sum_b psi2'_b u_ab,
// psi' = psi * es_dfac.  Writes the derivatives, or with ptg the deflected
// position (pointing, App. C), or with gpts the derivatives times the
// cotangent cot (interleaved, the position gradient of a loss).
template <int W>
__global__ void __launch_bounds__(IDF_THREADS) interp_grad_df_k(const double* __restrict__ grid, int64_t stride,
                                                                int n1, int n2, int nb2, int binsz,
                                                                const int* __restrict__ sub,
                                                                const int* __restrict__ cell,
                                                                const float2* __restrict__ psi,
                                                                const double* __restrict__ xy,
                                                                const int* __restrict__ perm, float2 beta,
                                                                double* __restrict__ dth, double* __restrict__ dph,
                                                                double* __restrict__ ptg,
                                                                const double* __restrict__ cot,
                                                                double* __restrict__ gpts) {
  extern __shared__ unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);
  const int tw = binsz + W - 1;
  const int bin = sub[3 * blockIdx.x], start = sub[3 * blockIdx.x + 1], cnt = sub[3 * blockIdx.x + 2];
  const int r0 = (bin / nb2) * binsz, c0 = (bin % nb2) * binsz;
  for (int e = threadIdx.x; e < tw * tw; e += IDF_THREADS) {
    const int r = e / tw, c = e - r * tw;
    const int gr = (r0 + r) % n1, gc = (c0 + c) % n2;
    float h, l;
    df_split(grid[(int64_t)gr * stride + gc], h, l);
    tile[e] = make_float2(h, l);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < cnt; q += IDF_THREADS) {
    const int64_t s = (int64_t)start + q;
    const int lr = cell[2 * s] - r0, lc = cell[2 * s + 1] - c0;
    const float2* ps = psi + s * 2 * W;
    int j1, j2;
    double o1, o2;
    tap(xy[2 * s], n1, W, j1, o1);
    tap(xy[2 * s + 1], n2, W, j2, o2);
    float o1h, o1l, o2h, o2l;
    df_split(o1, o1h, o1l);
    df_split(o2, o2h, o2l);
    float2 p2[W], q2[W];
#pragma unroll
    for (int b = 0; b < W; ++b) {
      p2[b] = ps[W + b];
      q2[b] = df_mul(p2[b], es_dfac<W>(o2h, o2l, b, beta));
    }
    float th = 0.f, tl = 0.f, fh = 0.f, fl = 0.f;
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
      const float2* trow = tile + (lr + a) * tw + lc;
      float ih = 0.f, il = 0.f, jh = 0.f, jl = 0.f;
#pragma unroll
      for (int b = 0; b < W; ++b) {
        const float2 u = trow[b];
        df_mac(ih, il, p2[b].x, p2[b].y, u.x, u.y);
        df_mac(jh, jl, q2[b].x, q2[b].y, u.x, u.y);
      }
      const float2 p1 = ps[a];
      const float2 q1 = df_mul(p1, es_dfac<W>(o1h, o1l, a, beta));
      df_mac(th, tl, q1.x, q1.y, ih, il);
      df_mac(fh, fl, p1.x, p1.y, jh, jl);
    }
    const double gth = df_value(th, tl) * ((double)n1 / (W * 3.14159265358979323846));
    const double gph = df_value(fh, fl) * ((double)n2 / (W * 3.14159265358979323846));
    const int i = perm[s];
    if (ptg) {
      deflect(xy[2 * s], xy[2 * s + 1], gth, gph, ptg + 2 * (int64_t)i);
    } else if (gpts) {
      const double c = cot[i];
      gpts[2 * (int64_t)i] = c * gth;
      gpts[2 * (int64_t)i + 1] = c * gph;
    } else {
      if (dth) dth[i] = gth;
      if (dph) dph[i] = gph;
    }
  }
}

// padded row stride of the double-float spreading tile: the least ts >= tw
// with ts = W (mod 16)
__host__ __device__ __forceinline__ int spread_df_stride(int tw, int W) { return tw + (((W - tw) % 16) + 16) % 16; }

template <int W>
__global__ void __launch_bounds__(32) spread_df_k(double* __restrict__ grid, int64_t stride, int n1, int n2, int nb2,
                                                  int binsz, const int* __restrict__ sub,
                                                  const int* __restrict__ cell, const float2* __restrict__ psi,
                                                  const int* __restrict__ perm, const double* __restrict__ f,
                                                  float2* __restrict__ scratch) {
  constexpr int NC = W * W;
  constexpr int NR = (NC + 31) / 32;  // rounds of 32 cells per point
  extern __shared__ unsigned char smem_raw[];
  const int tw = binsz + W - 1;
  // tile rows padded to a stride ts = W (mod 16): the W x W cells of a point,
  // taken in lane order, then sit on consecutive banks (conflict-free 64-bit
  // read and write, as if the patch were stored packed)
  const int ts = spread_df_stride(tw, W);
  float2* tile = reinterpret_cast<float2*>(smem_raw);
  int2* sp_cell = reinterpret_cast<int2*>(tile + tw * ts);    // [SUBMAX] local first taps
  float2* sp_f = reinterpret_cast<float2*>(sp_cell + SUBMAX);  // [SUBMAX] values as float pairs
  const int lane = threadIdx.x;
  const int bin = sub[3 * blockIdx.x], start = sub[3 * blockIdx.x + 1], cnt = sub[3 * blockIdx.x + 2];
  const int r0 = (bin / nb2) * binsz, c0 = (bin % nb2) * binsz;
  for (int t = lane; t < tw * ts; t += 32) tile[t] = make_float2(0.f, 0.f);
  for (int q = lane; q < cnt; q += 32) {
    const int64_t s = (int64_t)start + q;
    sp_cell[q] = make_int2(cell[2 * s] - r0, cell[2 * s + 1] - c0);
    float2 fv;
    df_split(f[perm[s]], fv.x, fv.y);
    sp_f[q] = fv;
  }
  __syncwarp();
  // this lane's cells of a point: (ca, cb) = divmod(lane + 32 t, W); offset in the tile
  int ca[NR], cb[NR], co[NR];
#pragma unroll
  for (int t = 0; t < NR; ++t) {
    const int idx = lane + 32 * t;
    ca[t] = idx < NC ? idx / W : 0;
    cb[t] = idx < NC ? idx % W : 0;
    co[t] = ca[t] * ts + cb[t];
  }
  // lane a < W holds psi1_a (k1, times f) and psi2_a (k2) of the current point
  float2 n1v = make_float2(0.f, 0.f), n2v = n1v;
  if (cnt > 0 && lane < W) {
    n1v = psi[(int64_t)start * 2 * W + lane];
    n2v = psi[(int64_t)start * 2 * W + W + lane];
  }
  for (int q = 0; q < cnt; ++q) {
    float2 k1 = n1v;
    const float2 k2 = n2v;
    if (q + 1 < cnt && lane < W) {
      n1v = psi[((int64_t)start + q + 1) * 2 * W + lane];
      n2v = psi[((int64_t)start + q + 1) * 2 * W + W + lane];
    }
    const int2 lrc = sp_cell[q];
    if (lane < W) k1 = df_mul(k1, sp_f[q]);
    float2* base = tile + lrc.x * ts + lrc.y;
    // a point's cells are distinct: read them all, update, write them all
    float2 c[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t)
      if (lane + 32 * t < NC) c[t] = base[co[t]];
#pragma unroll
    for (int t = 0; t < NR; ++t) {
      float2 va, vb;
      va.x = __shfl_sync(FULL, k1.x, ca[t]);
      va.y = __shfl_sync(FULL, k1.y, ca[t]);
      vb.x = __shfl_sync(FULL, k2.x, cb[t]);
      vb.y = __shfl_sync(FULL, k2.y, cb[t]);
      if (lane + 32 * t < NC) df_mac(c[t].x, c[t].y, va.x, va.y, vb.x, vb.y);
    }
#pragma unroll
    for (int t = 0; t < NR; ++t)
      if (lane + 32 * t < NC) base[co[t]] = c[t];
    __syncwarp();
  }
  __syncwarp();
  if (scratch) {  // deterministic: the whole tile (packed, tw x tw) to this subproblem's slot
    float2* dst = scratch + (size_t)blockIdx.x * tw * tw;
    for (int t = lane; t < tw * tw; t += 32) dst[t] = tile[(t / tw) * ts + t % tw];
    return;
  }
  for (int t = lane; t < tw * tw; t += 32) {
    const int tr = t / tw, tc = t - tr * tw;
    const float2 v = tile[tr * ts + tc];
    if (v.x != 0.f) {
      int r = r0 + tr, c = c0 + tc;
      while (r >= n1) r -= n1;
      while (c >= n2) c -= n2;
      atomicAdd(grid + (int64_t)r * stride + c, df_value(v.x, v.y));
    }
  }
}

// launch f<W> for the runtime width w (2 <= w <= WMAX)
#define NUSHT_W_DISPATCH(w, F, ...) \
  switch (w) {                      \
    case 2: F<2>(__VA_ARGS__); break;   \
    case 3: F<3>(__VA_ARGS__); break;   \
    case 4: F<4>(__VA_ARGS__); break;   \
    case 5: F<5>(__VA_ARGS__); break;   \
    case 6: F<6>(__VA_ARGS__); break;   \
    case 7: F<7>(__VA_ARGS__); break;   \
    case 8: F<8>(__VA_ARGS__); break;   \
    case 9: F<9>(__VA_ARGS__); break;   \
    case 10: F<10>(__VA_ARGS__); break; \
    case 11: F<11>(__VA_ARGS__); break; \
    case 12: F<12>(__VA_ARGS__); break; \
    case 13: F<13>(__VA_ARGS__); break; \
    case 14: F<14>(__VA_ARGS__); break; \
    case 15: F<15>(__VA_ARGS__); break; \
    case 16: F<16>(__VA_ARGS__); break; \
    case 17: F<17>(__VA_ARGS__); break; \
    case 18: F<18>(__VA_ARGS__); break; \
    case 19: F<19>(__VA_ARGS__); break; \
    default: F<20>(__VA_ARGS__); break; \
  }

template <int W>
void launch_interp_df(int nsub, size_t sm, cudaStream_t s, const double* grid, int64_t stride, int n1, int n2,
                      int nb2, int binsz, const int* sub, const int* cell, const float2* psi, const int* perm,
                      double* out) {
  interp_df_k<W><<<nsub, IDF_THREADS, sm, s>>>(grid, stride, n1, n2, nb2, binsz, sub, cell, psi, perm, out);
}

template <int W>
void launch_interp_grad_df(int nsub, size_t sm, cudaStream_t s, const double* grid, int64_t stride, int n1, int n2,
                           int nb2, int binsz, const int* sub, const int* cell, const float2* psi, const double* xy,
                           const int* perm, float2 beta, double* dth, double* dph, double* ptg, const double* cot,
                           double* gpts) {
  interp_grad_df_k<W><<<nsub, IDF_THREADS, sm, s>>>(grid, stride, n1, n2, nb2, binsz, sub, cell, psi, xy, perm, beta,
                                                    dth, dph, ptg, cot, gpts);
}

template <int W>
void launch_spread_df(int nsub, size_t sm, cudaStream_t s, double* grid, int64_t stride, int n1, int n2, int nb2,
                      int binsz, const int* sub, const int* cell, const float2* psi, const int* perm,
                      const double* f, float2* scratch) {
  spread_df_k<W><<<nsub, 32, sm, s>>>(grid, stride, n1, n2, nb2, binsz, sub, cell, psi, perm, f, scratch);
}

__device__ __forceinline__ double tile_value(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double tile_value(double v) { return v; }
__device__ __forceinline__ float tile_value(float v) { return v; }

// Deterministic type 1: grid cell (r, c) = the sum, in a fixed order, of the
// tile entries of every subproblem whose tile covers it.  A tile of bin
// (R', C') covers rows r0' .. r0' + bin + w - 2 (mod n1); with w - 1 <= bin
// these lie in the bins R - 2, R - 1, R (R - 2 only when a partial last bin
// lets footprints of the bin before it wrap into bin 0); all bins are taken
// when there are at most four per dimension, where tiles can wrap around the
// whole grid; likewise columns.  Bins whose tile misses the cell add nothing.
template <typename T, typename A, typename S>
__global__ void grid_gather_k(T* __restrict__ grid, int64_t stride, int n1, int n2, int binsz, int tw, int nb1,
                              int nb2, const int* __restrict__ binsub, const S* __restrict__ tiles) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n1 * n2) return;
  const int r = (int)(e / n2), c = (int)(e - (int64_t)r * n2);
  const int R = r / binsz, C = c / binsz;
  int rb[4], cb[4];
  int nr = 0, nc = 0;
  if (nb1 <= 4) {
    for (int b = 0; b < nb1; ++b) rb[nr++] = b;
  } else {
    rb[nr++] = (R + nb1 - 2) % nb1;
    rb[nr++] = (R + nb1 - 1) % nb1;
    rb[nr++] = R;
  }
  if (nb2 <= 4) {
    for (int b = 0; b < nb2; ++b) cb[nc++] = b;
  } else {
    cb[nc++] = (C + nb2 - 2) % nb2;
    cb[nc++] = (C + nb2 - 1) % nb2;
    cb[nc++] = C;
  }
  A acc = 0;
  auto val = [](const S& v) -> A { return tile_value(v); };
  for (int i = 0; i < nr; ++i) {
    const int r0 = rb[i] * binsz;
    for (int tr = ((r - r0) % n1 + n1) % n1; tr < tw; tr += n1) {
      for (int j = 0; j < nc; ++j) {
        const int c0 = cb[j] * binsz;
        const int bin = rb[i] * nb2 + cb[j];
        for (int tc = ((c - c0) % n2 + n2) % n2; tc < tw; tc += n2) {
          for (int k = binsub[bin]; k < binsub[bin + 1]; ++k) {
            acc += val(tiles[(size_t)k * tw * tw + tr * tw + tc]);
          }
        }
      }
    }
  }
  grid[(int64_t)r * stride + c] = (T)acc;
}

template <int W>
void optin_df(int* st) {
  const int mx = 84 * 84 * 8;
  const int mxs = 84 * spread_df_stride(84, W) * 8;
  if (cudaFuncSetAttribute(spread_df_k<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, mxs + SUBMAX * 16) !=
          cudaSuccess ||
      cudaFuncSetAttribute(interp_df_k<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
      cudaFuncSetAttribute(interp_grad_df_k<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess)
    *st = 1;
}

// one point into the FP32 spreading tile: w x w native shared-memory float atomics
template <int W>
__device__ __forceinline__ void spread_point_f(float* tile, int tw, int lr, int lc, float o1, float o2, float fv,
                                               float beta) {
  const float scf = 2.0f / W;
  float p1[W], p2[W];
#pragma unroll
  for (int a = 0; a < W; ++a) {
    p1[a] = fv * es_psif((o1 - a) * scf, beta);
    p2[a] = es_psif((o2 - a) * scf, beta);
  }
#pragma unroll
  for (int a = 0; a < W; ++a) {
    float* trow = tile + (lr + a) * tw + lc;
#pragma unroll
    for (int b = 0; b < W; ++b) atomicAdd(trow + b, p1[a] * p2[b]);
  }
}

// Spreading in float (mixed mode): one thread per point of the subproblem,
// kernel values evaluated on the fly from the FP32 offsets, w x w native
// shared-memory float atomics into the bin's tile, one atomic flush.
// Points are in cell order inside their bin.  rows = 0: consecutive points on
// consecutive lanes (regular point sets, e.g. ring grids, whose neighbours sit
// in distinct cells).  rows = 1 (scattered sets where neighbours often share a
// cell): the subproblem's points are staged in shared memory with coalesced
// loads, lane l of every warp takes the run l Lr .. l Lr + Lr - 1 and the
// warps interleave inside it, so a warp's lanes sit about a tile row apart
// and their atomics rarely share an address.
template <int W>
__global__ void __launch_bounds__(128) spread_pt_k(float* __restrict__ grid, int64_t stride, int n1, int n2, int nb2,
                                                   int binsz, float betaf, const int* __restrict__ sub,
                                                   const int* __restrict__ cell, const float* __restrict__ offf,
                                                   const int* __restrict__ perm, const float* __restrict__ f,
                                                   int rows) {
  extern __shared__ unsigned char smem_raw[];
  float* tile = reinterpret_cast<float*>(smem_raw);
  const int tw = binsz + W - 1;
  const int bin = sub[3 * blockIdx.x], start = sub[3 * blockIdx.x + 1], cnt = sub[3 * blockIdx.x + 2];
  const int r0 = (bin / nb2) * binsz, c0 = (bin % nb2) * binsz;
  for (int t = threadIdx.x; t < tw * tw; t += blockDim.x) tile[t] = 0.f;
  if (rows) {
    float4* sp = reinterpret_cast<float4*>(tile + ((tw * tw + 3) & ~3));
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      const int64_t s = (int64_t)start + k;
      const int lr = cell[2 * s] - r0, lc = cell[2 * s + 1] - c0;
      sp[sp_idx(k)] = make_float4(__int_as_float((lr << 16) | lc), offf[2 * s], offf[2 * s + 1], f[perm[s]]);
    }
    __syncthreads();
    const int Lr = (cnt + 31) >> 5, nwarp = (int)blockDim.x >> 5;
    for (int j = (int)threadIdx.x >> 5; j < Lr; j += nwarp) {
      const int q = ((int)threadIdx.x & 31) * Lr + j;
      if (q >= cnt) continue;
      const float4 pv = sp[sp_idx(q)];
      const int pk = __float_as_int(pv.x);
      spread_point_f<W>(tile, tw, pk >> 16, pk & 0xffff, pv.y, pv.z, pv.w, betaf);
    }
  } else {
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      const int64_t s = (int64_t)start + q;
      spread_point_f<W>(tile, tw, cell[2 * s] - r0, cell[2 * s + 1] - c0, offf[2 * s], offf[2 * s + 1],
                        f[perm[s]], betaf);
    }
  }
  __syncthreads();
  // tile row of t from a float reciprocal: (t + 1/2) / tw is at least
  // 1 / (2 tw) from an integer, far above the rounding for t < tw^2 < 2^13
  const float itw = 1.0f / (float)tw;
  for (int t = threadIdx.x; t < tw * tw; t += blockDim.x) {
    const float v = tile[t];
    if (v != 0.f) {
      const int tr = __float2int_rz(((float)t + 0.5f) * itw);
      int r = r0 + tr, c = c0 + (t - tr * tw);
      while (r >= n1) r -= n1;
      while (c >= n2) c -= n2;
      atomicAdd(grid + (int64_t)r * stride + c, v);
    }
  }
}

// interpolation in float (mixed mode): one thread per point, kernel values
// evaluated on the fly from the FP32 offsets
template <int W>
__global__ void __launch_bounds__(128) interp_f_k(const float* __restrict__ grid, int64_t stride, int n1, int n2,
                                                  float betaf, const int* __restrict__ cell,
                                                  const float* __restrict__ offf, const int* __restrict__ perm,
                                                  int64_t npts, float* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= npts) return;
  const int i1 = cell[2 * s], i2 = cell[2 * s + 1];
  const float o1 = offf[2 * s], o2 = offf[2 * s + 1];
  const float scf = 2.0f / W;
  float p1[W], p2[W];
#pragma unroll
  for (int a = 0; a < W; ++a) {
    p1[a] = es_psif((o1 - a) * scf, betaf);
    p2[a] = es_psif((o2 - a) * scf, betaf);
  }
  const bool wrap2 = i2 + W > n2;
  float acc = 0.f;
#pragma unroll
  for (int a = 0; a < W; ++a) {
    int r = i1 + a;
    if (r >= n1) r -= n1;
    const float* row = grid + (int64_t)r * stride;
    float in = 0.f;
#pragma unroll
    for (int b = 0; b < W; ++b) {
      int c = i2 + b;
      if (wrap2 && c >= n2) c -= n2;
      in = fmaf(p2[b], row[c], in);
    }
    acc = fmaf(p1[a], in, acc);
  }
  out[perm[s]] = acc;
}

template <int W>
void launch_spread_f(int nsub, size_t sm, cudaStream_t s, float* grid, int64_t stride, int n1, int n2, int nb2,
                     int binsz, float betaf, const int* sub, const int* cell, const float* offf, const int* perm,
                     const float* f, int rows) {
  spread_pt_k<W><<<nsub, 128, sm, s>>>(grid, stride, n1, n2, nb2, binsz, betaf, sub, cell, offf, perm, f, rows);
}

template <int W>
void launch_interp_f(int nb, cudaStream_t s, const float* grid, int64_t stride, int n1, int n2, float betaf,
                     const int* cell, const float* offf, const int* perm, int64_t npts, float* out) {
  interp_f_k<W><<<nb, 128, 0, s>>>(grid, stride, n1, n2, betaf, cell, offf, perm, npts, out);
}

// ---------------------------------------------------------------------------
// The same mixed-precision kernels for every member of a batch in one launch:
// a block finds its member by its first-block offset (binary search over the
// member table) and then works as spread_pt_k / interp_f_k do on that
// member's grid and points.
// ---------------------------------------------------------------------------
enum { MEMBER_BLK, MEMBER_SUB, MEMBER_ZERO, MEMBER_PAD, MEMBER_TRUNC };
template <int KEY>
__device__ __forceinline__ int nufft_member_of(const NufftMember* __restrict__ mem, int nm, int b) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int f = KEY == MEMBER_BLK     ? mem[mid].blk0
                  : KEY == MEMBER_SUB   ? mem[mid].sub0
                  : KEY == MEMBER_ZERO  ? mem[mid].zero0
                  : KEY == MEMBER_PAD   ? mem[mid].pad0
                                        : mem[mid].trunc0;
    if (f <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) zero_grids_k(const NufftMember* __restrict__ mem, int nm) {
  const NufftMember& q = mem[nufft_member_of<MEMBER_ZERO>(mem, nm, blockIdx.x)];
  const int64_t n = (int64_t)q.n1 * q.stride;
  const int64_t i0 = (int64_t)(blockIdx.x - q.zero0) * ZERO_CHUNK;
  const int64_t i1 = i0 + ZERO_CHUNK < n ? i0 + ZERO_CHUNK : n;
  // the grid starts 256-byte aligned and i0 is a multiple of 4: 16-byte stores,
  // the last partial vector element by element
  float4* g4 = reinterpret_cast<float4*>(q.grid);
  for (int64_t i = i0 + 4 * threadIdx.x; i < i1; i += 4 * blockDim.x) {
    if (i + 4 <= i1)
      g4[i >> 2] = make_float4(0.f, 0.f, 0.f, 0.f);
    else
      for (int64_t k = i; k < i1; ++k) q.grid[k] = 0.f;
  }
}

// blocks b = blockIdx.x + base of the table slice `mem` (base: sub0 / blk0 of
// its first member); maps[i] belongs to mem[i]
template <int W>
__global__ void __launch_bounds__(128) spread_many_k(const NufftMember* __restrict__ mem, int nm, int base,
                                                     const float* const* __restrict__ maps) {
  extern __shared__ unsigned char smem_raw[];
  float* tile = reinterpret_cast<float*>(smem_raw);
  const int b = blockIdx.x + base;
  const int i = nufft_member_of<MEMBER_SUB>(mem, nm, b);
  const NufftMember& q = mem[i];
  const int* sb = q.sub + 3 * (b - q.sub0);
  const int binsz = q.bin, tw = binsz + W - 1;
  const int bin = sb[0], start = sb[1], cnt = sb[2];
  const int r0 = (bin / q.nbins2) * binsz, c0 = (bin % q.nbins2) * binsz;
  const float* f = maps[i];
  for (int t = threadIdx.x; t < tw * tw; t += blockDim.x) tile[t] = 0.f;
  // the two lane mappings of spread_pt_k, by the member's spread_rows
  if (q.spread_rows) {
    float4* sp = reinterpret_cast<float4*>(tile + ((tw * tw + 3) & ~3));
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      const int64_t s = (int64_t)start + k;
      const int lr = q.cell[2 * s] - r0, lc = q.cell[2 * s + 1] - c0;
      sp[sp_idx(k)] = make_float4(__int_as_float((lr << 16) | lc), q.off[2 * s], q.off[2 * s + 1], f[q.perm[s]]);
    }
    __syncthreads();
    const int Lr = (cnt + 31) >> 5, nwarp = (int)blockDim.x >> 5;
    for (int j = (int)threadIdx.x >> 5; j < Lr; j += nwarp) {
      const int k = ((int)threadIdx.x & 31) * Lr + j;
      if (k >= cnt) continue;
      const float4 pv = sp[sp_idx(k)];
      const int pk = __float_as_int(pv.x);
      spread_point_f<W>(tile, tw, pk >> 16, pk & 0xffff, pv.y, pv.z, pv.w, q.beta);
    }
  } else {
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      const int64_t s = (int64_t)start + k;
      spread_point_f<W>(tile, tw, q.cell[2 * s] - r0, q.cell[2 * s + 1] - c0, q.off[2 * s], q.off[2 * s + 1],
                        f[q.perm[s]], q.beta);
    }
  }
  __syncthreads();
  const float itw = 1.0f / (float)tw;  // exact row of t, as in spread_pt_k
  for (int t = threadIdx.x; t < tw * tw; t += blockDim.x) {
    const float v = tile[t];
    if (v != 0.f) {
      const int tr = __float2int_rz(((float)t + 0.5f) * itw);
      int r = r0 + tr, c = c0 + (t - tr * tw);
      while (r >= q.n1) r -= q.n1;
      while (c >= q.n2) c -= q.n2;
      atomicAdd(q.grid + (int64_t)r * q.stride + c, v);
    }
  }
}

template <int W>
__global__ void __launch_bounds__(128) interp_many_k(const NufftMember* __restrict__ mem, int nm, int base,
                                                     float* const* __restrict__ maps) {
  const int b = blockIdx.x + base;
  const int i = nufft_member_of<MEMBER_BLK>(mem, nm, b);
  const NufftMember& q = mem[i];
  const int64_t s = (int64_t)(b - q.blk0) * 128 + threadIdx.x;
  if (s >= q.npts) return;
  const int i1 = q.cell[2 * s], i2 = q.cell[2 * s + 1];
  const float o1 = q.off[2 * s], o2 = q.off[2 * s + 1];
  const float scf = 2.0f / W;
  float p1[W], p2[W];
#pragma unroll
  for (int a = 0; a < W; ++a) {
    p1[a] = es_psif((o1 - a) * scf, q.beta);
    p2[a] = es_psif((o2 - a) * scf, q.beta);
  }
  const int n1 = q.n1, n2 = q.n2;
  const bool wrap2 = i2 + W > n2;
  float acc = 0.f;
#pragma unroll
  for (int a = 0; a < W; ++a) {
    int r = i1 + a;
    if (r >= n1) r -= n1;
    const float* row = q.grid + (int64_t)r * q.stride;
    float in = 0.f;
#pragma unroll
    for (int b = 0; b < W; ++b) {
      int c = i2 + b;
      if (wrap2 && c >= n2) c -= n2;
      in = fmaf(p2[b], row[c], in);
    }
    acc = fmaf(p1[a], in, acc);
  }
  maps[i][q.perm[s]] = acc;
}

// deconv_pad_k / deconv_trunc_k of every member: the member's 2D tile grid
// flattened, tiles in the same order
__global__ void deconv_pad_many_k(const NufftMember* __restrict__ mem, int nm) {
  const NufftMember& q = mem[nufft_member_of<MEMBER_PAD>(mem, nm, blockIdx.x)];
  const int n2h = q.n2 / 2 + 1, gx = (n2h + 31) / 32;
  const int t = blockIdx.x - q.pad0;
  deconv_pad_tile<float>(q.Gh, reinterpret_cast<float2*>(q.grid), q.lmax, q.mmax, q.M, q.n1, n2h, q.d1, q.d2,
                         t % gx, t / gx);
}
__global__ void deconv_trunc_many_k(const NufftMember* __restrict__ mem, int nm) {
  const NufftMember& q = mem[nufft_member_of<MEMBER_TRUNC>(mem, nm, blockIdx.x)];
  const int gx = (q.M + 31) / 32;
  const int t = blockIdx.x - q.trunc0;
  deconv_trunc_tile<float>(reinterpret_cast<const float2*>(q.grid), q.Gh, q.lmax, q.mmax, q.M, q.n1, q.n2 / 2 + 1,
                           q.d1, q.d2, t % gx, t / gx);
}

template <int W>
void launch_spread_many(const NufftBatch& nb, size_t sm, cudaStream_t s, const float* const* maps) {
  spread_many_k<W><<<nb.nsub, 128, sm, s>>>(nb.mem, nb.nm, nb.sub_base, maps);
}
template <int W>
void launch_interp_many(const NufftBatch& nb, cudaStream_t s, float* const* maps) {
  interp_many_k<W><<<nb.nblk, 128, 0, s>>>(nb.mem, nb.nm, nb.blk_base, maps);
}

template <int W>
void optin_f(int* st) {
  if (cudaFuncSetAttribute(spread_pt_k<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 84 * 84 * 8) != cudaSuccess ||
      cudaFuncSetAttribute(spread_many_k<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 84 * 84 * 8) != cudaSuccess)
    *st = 1;
}

}  // namespace

int spread_smem_optin() {
  // bins of up to 64 cells with w <= 20: (64 + 19)^2 x 8 B = 55.1 KB of tile
  const int mx = 84 * 84 * 8;
  NUSHT_CUDA(cudaFuncSetAttribute(spread_k<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  NUSHT_CUDA(cudaFuncSetAttribute(spread_k<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));

  int bad = 0;
  for (int w = 2; w <= WMAX; ++w) {
    NUSHT_W_DISPATCH(w, optin_df, &bad);
    NUSHT_W_DISPATCH(w, optin_f, &bad);
  }
  if (bad) return set_error(NUSHT_ECUDA, "shared-memory opt-in for the double-float NUFFT kernels");
  return NUSHT_OK;
}

void free_points(nusht_plan_t p) {
  PointData& d = p->pts;
  dev_free(d.perm);
  dev_free(d.cell);
  dev_free(d.psi);
  dev_free(d.xy);
  dev_free(d.off);
  dev_free(d.sub);
  dev_free(d.tiles);
  dev_free(d.binsub);
  dev_free(d.rowmask);
  dev_free(d.rowpairs);
  d = PointData();
}

// FP64 plans run interpolation and spreading in double-float unless the
// caller asked for FP64 instructions (opts.fp64_contraction)
static bool nufft_df(nusht_plan_t p) { return p->precision == NUSHT_FP64 && !p->opts.fp64_contraction; }

// Stable LSD radix sort of (key, index) pairs by key on the host, 16-bit
// digits, `passes` of them, each pass split over the host threads: every
// thread counts the digits of its slice, the offsets are laid out digit by
// digit and, inside a digit, slice by slice (which keeps the sort stable), and
// every thread scatters its slice.
static void radix_sort_pairs(std::vector<int64_t>& keys, std::vector<int>& idx, int passes) {
  const int64_t n = (int64_t)keys.size();
  constexpr int D = 1 << 16;
  int nt = (int)std::min(16u, std::max(1u, std::thread::hardware_concurrency()));
  if (n < (1 << 20)) nt = 1;
  std::vector<int64_t> k2(n);
  std::vector<int> i2(n);
  std::vector<int64_t> hist((size_t)nt * D);
  auto parallel = [&](auto&& body) {
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(body, t);
    body(0);
    for (auto& x : th) x.join();
  };
  for (int ps = 0; ps < passes; ++ps) {
    const int sh = 16 * ps;
    parallel([&](int t) {
      int64_t* h = hist.data() + (size_t)t * D;
      std::fill(h, h + D, 0);
      const int64_t a = n * t / nt, b = n * (t + 1) / nt;
      for (int64_t i = a; i < b; ++i) h[(keys[i] >> sh) & 0xffff]++;
    });
    int64_t run = 0;
    for (int d = 0; d < D; ++d)
      for (int t = 0; t < nt; ++t) {
        const int64_t c = hist[(size_t)t * D + d];
        hist[(size_t)t * D + d] = run;
        run += c;
      }
    parallel([&](int t) {
      int64_t* h = hist.data() + (size_t)t * D;
      const int64_t a = n * t / nt, b = n * (t + 1) / nt;
      for (int64_t i = a; i < b; ++i) {
        const int64_t o = h[(keys[i] >> sh) & 0xffff]++;
        k2[o] = keys[i];
        i2[o] = idx[i];
      }
    });
    keys.swap(k2);
    idx.swap(i2);
  }
}

// The fine-grid rows that some point's taps reach (first tap row i1 and the
// w - 1 rows after it, cyclically): the row FFT passes of this library's FFT
// kernels transform only their row pairs, and the column pass stores T only
// at those rows.  T's other entries are zeroed here and never written, so the
// adjoint's column pass reads zeros there (the spectra of rows that
// spreading leaves zero).  A superset is safe (an extra row is transformed
// for nothing), so per bin the first tap rows from its first to its last
// point (in cell order) are taken.  keys: the sorted point keys, off: the
// bins' point offsets (null: no points).
static int set_touched_rows(nusht_plan_t p, const std::vector<int64_t>* keys, const std::vector<int64_t>* off,
                            int nb2, int binsz, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  PointData& d = p->pts;
  const int n1 = z.n1;
  std::vector<unsigned char> first(n1, 0), mask(n1, 0);
  if (keys) {
    const int64_t cpb = (int64_t)binsz * binsz;
    const int nbins = (int)off->size() - 1;
    for (int b = 0; b < nbins; ++b) {
      const int64_t a0 = (*off)[b], a1 = (*off)[b + 1];
      if (a0 == a1) continue;
      const int base = (b / nb2) * binsz;
      const int rlo = (int)(((*keys)[a0] % cpb) / binsz), rhi = (int)(((*keys)[a1 - 1] % cpb) / binsz);
      for (int r = rlo; r <= rhi; ++r) first[base + r] = 1;
    }
  }
  for (int r = 0; r < n1; ++r)
    if (first[r])
      for (int a = 0; a < z.w; ++a) mask[(r + a) % n1] = 1;
  std::vector<int> pairs;
  for (int j = 0; j < n1; j += 2)
    if (mask[j] || (j + 1 < n1 && mask[j + 1])) pairs.push_back(j / 2);
  if (!d.rowmask) {
    NUSHT_TRY(dev_alloc((void**)&d.rowmask, (size_t)n1, &p->bytes));
    NUSHT_TRY(dev_alloc((void**)&d.rowpairs, (size_t)(n1 + 1) / 2 * sizeof(int), &p->bytes));
  }
  NUSHT_CUDA(cudaMemcpyAsync(d.rowmask, mask.data(), (size_t)n1, cudaMemcpyHostToDevice, s));
  if (!pairs.empty())
    NUSHT_CUDA(cudaMemcpyAsync(d.rowpairs, pairs.data(), pairs.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  d.nrowpairs = (int)pairs.size();
  if (p->tcols) {
    const size_t es = p->dfft_fine ? sizeof(float4) : sizeof(float2);
    NUSHT_CUDA(cudaMemsetAsync(p->tcols, 0, (size_t)(z.mmax + 1) * n1 * es, s));
  }
  if (p->sfft_mem) {
    // the plan's FP32 FFT member entry carries the row list and mask
    SfftMember m;
    sfft_member(p, m);
    NUSHT_CUDA(cudaMemcpyAsync(p->sfft_mem, &m, sizeof(SfftMember), cudaMemcpyHostToDevice, s));
  }
  NUSHT_CUDA(cudaStreamSynchronize(s));
  return NUSHT_OK;
}

int setpts_impl(nusht_plan_t p, int64_t npts, const double* d_pts, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  PointData& d = p->pts;
  // the deterministic gather takes the tiles of the bins R and R - 1 per
  // dimension, which needs w - 1 <= bin
  if (p->opts.deterministic && d.bin > 0 && d.bin < z.w) d.bin = 32;
  const int binsz = d.bin > 0 ? d.bin : 32;
  const int nb1 = (z.n1 + binsz - 1) / binsz, nb2 = (z.n2 + binsz - 1) / binsz;
  const bool dbl = p->precision == NUSHT_FP64;
  if (npts > d.cap) {
    size_t before = p->bytes;
    dev_free(d.perm);
    dev_free(d.cell);
    dev_free(d.psi);
    dev_free(d.off);
    dev_free(d.xy);
    d.perm = nullptr;
    d.cell = nullptr;
    d.psi = nullptr;
    d.off = nullptr;
    d.xy = nullptr;
    p->bytes = before - std::min(before, d.bytes);
    d.bytes = 0;
    NUSHT_TRY(dev_alloc((void**)&d.perm, (size_t)npts * 4, &d.bytes));
    NUSHT_TRY(dev_alloc((void**)&d.cell, (size_t)npts * 8, &d.bytes));
    NUSHT_TRY(dev_alloc((void**)&d.xy, (size_t)npts * 16, &d.bytes));
    if (dbl)
      NUSHT_TRY(dev_alloc((void**)&d.psi, (size_t)npts * 2 * z.w * 8, &d.bytes));
    else
      NUSHT_TRY(dev_alloc((void**)&d.off, (size_t)npts * 8, &d.bytes));
    p->bytes += d.bytes;
    d.cap = npts;
  }
  d.npts = npts;
  d.nbins1 = nb1;
  d.nbins2 = nb2;
  dev_free(d.sub);
  d.sub = nullptr;
  d.nsub = 0;
  if (npts == 0) return set_touched_rows(p, nullptr, nullptr, nb2, binsz, s);
  // sort keys on the device (bin, then the first tap row-major inside the
  // bin), LSD radix sort on the host: stable, so the order, and with it every
  // summation order, is deterministic.  Points of a bin in cell order make a
  // warp's lanes touch neighbouring cells of the tile and of the fine grid
  // (for scattered inputs such as uniform random points the input order is
  // random inside a bin).
  int64_t* dkey = nullptr;
  NUSHT_TRY(dev_alloc((void**)&dkey, (size_t)npts * 8, nullptr));
  const int tb = 256;
  const int nblk = (int)((npts + tb - 1) / tb);
  prep_k<<<nblk, tb, 0, s>>>(d_pts, npts, z.n1, z.n2, z.w, nb2, binsz, dkey);
  std::vector<int64_t> keys(npts);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(keys.data(), dkey, (size_t)npts * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(dkey);
  if (e != cudaSuccess) return cuda_status(e, "point binning");
  const int nbins = nb1 * nb2;
  const int64_t cells_per_bin = (int64_t)binsz * binsz;
  std::vector<int> perm(npts);
  {
    // 16-bit digits, as many passes as the largest key needs
    const int64_t kmax = (int64_t)nbins * cells_per_bin;
    int passes = 0;
    while (passes < 4 && (kmax >> (16 * passes)) > 0) ++passes;
    for (int64_t i = 0; i < npts; ++i) perm[i] = (int)i;
    radix_sort_pairs(keys, perm, passes);
  }
  // keys are now sorted: bin offsets, and how often a point shares its first
  // tap with the one before it (ring grids: almost never; uniform random
  // points at the fine grid's density: a large fraction), which picks the
  // lane mapping of the FP32 spreading kernels
  std::vector<int64_t> off(nbins + 1, 0);
  int64_t same = 0;
  for (int64_t i = 0; i < npts; ++i) {
    off[keys[i] / cells_per_bin + 1]++;
    same += i > 0 && keys[i] == keys[i - 1];
  }
  d.spread_rows = same * 20 > npts ? 1 : 0;  // more than 5 % of the points
  for (int b = 0; b < nbins; ++b) off[b + 1] += off[b];
  NUSHT_TRY(set_touched_rows(p, &keys, &off, nb2, binsz, s));
  std::vector<int> sub;
  for (int b = 0; b < nbins; ++b)
    for (int64_t st = off[b]; st < off[b + 1]; st += SUBMAX) {
      sub.push_back(b);
      sub.push_back((int)st);
      sub.push_back((int)std::min<int64_t>(SUBMAX, off[b + 1] - st));
    }
  d.nsub = (int)(sub.size() / 3);
  NUSHT_TRY(dev_alloc((void**)&d.sub, std::max<size_t>(1, sub.size()) * 4, &p->bytes));
  if (p->opts.deterministic) {
    std::vector<int> bs(nbins + 1, 0);
    for (size_t k = 0; k < sub.size() / 3; ++k) bs[sub[3 * k] + 1]++;
    for (int b = 0; b < nbins; ++b) bs[b + 1] += bs[b];
    dev_free(d.binsub);
    d.binsub = nullptr;
    NUSHT_TRY(dev_alloc((void**)&d.binsub, bs.size() * 4, &p->bytes));
    NUSHT_CUDA(cudaMemcpyAsync(d.binsub, bs.data(), bs.size() * 4, cudaMemcpyHostToDevice, s));
    const int tw = binsz + z.w - 1;
    const size_t need = std::max<size_t>(1, (size_t)d.nsub) * tw * tw * (dbl ? 8 : 4);
    if (need > d.tiles_cap) {
      dev_free(d.tiles);
      d.tiles = nullptr;
      d.tiles_cap = 0;
      NUSHT_TRY(dev_alloc(&d.tiles, need, &p->bytes));
      d.tiles_cap = need;
    }
  }
  NUSHT_CUDA(cudaMemcpyAsync(d.perm, perm.data(), (size_t)npts * 4, cudaMemcpyHostToDevice, s));
  if (!sub.empty()) NUSHT_CUDA(cudaMemcpyAsync(d.sub, sub.data(), sub.size() * 4, cudaMemcpyHostToDevice, s));
  const bool dfm = nufft_df(p);
  gather_k<<<nblk, tb, 0, s>>>(d_pts, d.perm, npts, z.n1, z.n2, z.w, z.beta, d.cell,
                               dbl && !dfm ? d.psi : nullptr, dfm ? reinterpret_cast<float2*>(d.psi) : nullptr,
                               dbl ? nullptr : d.off, d.xy);
  NUSHT_CUDA(cudaGetLastError());
  NUSHT_CUDA(cudaStreamSynchronize(s));
  return NUSHT_OK;
}

int deconv_pad(nusht_plan_t p, cudaStream_t s) {
  // double-float FFT plans: deconvolution and zero-padding happen in the load
  // of the column pass, which this stage then runs
  if (p->dfft_fine) return dfft_cols_synth(p, s);
  if (p->sfft_fine) return sfft_cols_synth(sfft_launch_of(p), s);
  const nusht_sizes& z = p->sz;
  const int n2h = z.n2 / 2 + 1;
  dim3 blk(32, 8), grd((n2h + 31) / 32, (z.n1 + 31) / 32);
  if (p->precision == NUSHT_FP64)
    deconv_pad_k<double><<<grd, blk, 0, s>>>((const double2*)p->Ghat, (double2*)p->fine, z.lmax, z.mmax, z.M, z.n1,
                                             n2h, p->deconv1, p->deconv2);
  else
    deconv_pad_k<float><<<grd, blk, 0, s>>>((const float2*)p->Ghat, (float2*)p->fine, z.lmax, z.mmax, z.M, z.n1, n2h,
                                            p->deconv1, p->deconv2);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int deconv_trunc(nusht_plan_t p, cudaStream_t s) {
  // double-float FFT plans: the column pass, with truncation and
  // deconvolution in its store
  if (p->dfft_fine) return dfft_cols_adjoint(p, s);
  if (p->sfft_fine) return sfft_cols_adjoint(sfft_launch_of(p), s);
  const nusht_sizes& z = p->sz;
  const int n2h = z.n2 / 2 + 1;
  dim3 blk(32, 8), grd((z.M + 31) / 32, (z.mmax + 1 + 31) / 32);
  if (p->precision == NUSHT_FP64)
    deconv_trunc_k<double><<<grd, blk, 0, s>>>((const double2*)p->fine, (double2*)p->Ghat, z.lmax, z.mmax, z.M, z.n1,
                                               n2h, p->deconv1, p->deconv2);
  else
    deconv_trunc_k<float><<<grd, blk, 0, s>>>((const float2*)p->fine, (float2*)p->Ghat, z.lmax, z.mmax, z.M, z.n1, n2h,
                                              p->deconv1, p->deconv2);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int interp(nusht_plan_t p, void* d_map, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const int64_t n = p->pts.npts;
  if (n == 0) return NUSHT_OK;
  const int64_t stride = 2 * (z.n2 / 2 + 1);
  const int tb = 128;
  const int nb = (int)((n + tb - 1) / tb);
  if (nufft_df(p)) {
    if (p->pts.nsub == 0) return NUSHT_OK;
    const int binsz = p->pts.bin > 0 ? p->pts.bin : 32;
    const int tw = binsz + z.w - 1;
    NUSHT_W_DISPATCH(z.w, launch_interp_df, p->pts.nsub, (size_t)tw * tw * 8, s, (const double*)p->fine, stride,
                     z.n1, z.n2, p->pts.nbins2, binsz, p->pts.sub, p->pts.cell,
                     reinterpret_cast<const float2*>(p->pts.psi), p->pts.perm, (double*)d_map);
  } else if (p->precision == NUSHT_FP64)
    interp_k<double, false><<<nb, tb, 0, s>>>((const double*)p->fine, stride, z.n1, z.n2, z.w, (float)z.beta, z.beta,
                                              p->pts.cell, p->pts.psi, nullptr, nullptr, p->pts.perm, n,
                                              (double*)d_map, nullptr, nullptr, nullptr, nullptr, nullptr);
  else
    NUSHT_W_DISPATCH(z.w, launch_interp_f, nb, s, (const float*)p->fine, stride, z.n1, z.n2, (float)z.beta,
                     p->pts.cell, p->pts.off, p->pts.perm, n, (float*)d_map);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

// FP64 plans with the double-float NUFFT: derivatives (or the pointing) from
// the bin tiles and the plan's kernel-value table
static int interp_grad_df(nusht_plan_t p, double* d_dth, double* d_dph, double* d_ptg, const double* cot,
                          double* gpts, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const int64_t stride = 2 * (z.n2 / 2 + 1);
  const int binsz = p->pts.bin > 0 ? p->pts.bin : 32;
  const int tw = binsz + z.w - 1;
  const float bh = (float)z.beta;
  const float2 beta = make_float2(bh, (float)(z.beta - (double)bh));
  NUSHT_W_DISPATCH(z.w, launch_interp_grad_df, p->pts.nsub, (size_t)tw * tw * 8, s, (const double*)p->fine, stride,
                   z.n1, z.n2, p->pts.nbins2, binsz, p->pts.sub, p->pts.cell,
                   reinterpret_cast<const float2*>(p->pts.psi), p->pts.xy, p->pts.perm, beta, d_dth, d_dph, d_ptg,
                   cot, gpts);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int interp_grad(nusht_plan_t p, void* d_dth, void* d_dph, const void* cot, double* gpts, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const int64_t n = p->pts.npts;
  if (n == 0) return NUSHT_OK;
  if (nufft_df(p) && p->pts.nsub > 0)
    return interp_grad_df(p, (double*)d_dth, (double*)d_dph, nullptr, (const double*)cot, gpts, s);
  const int64_t stride = 2 * (z.n2 / 2 + 1);
  const int tb = 128;
  const int nb = (int)((n + tb - 1) / tb);
  if (p->precision == NUSHT_FP64)
    interp_k<double, true><<<nb, tb, 0, s>>>((const double*)p->fine, stride, z.n1, z.n2, z.w, (float)z.beta, z.beta,
                                             p->pts.cell, nullptr, nullptr, p->pts.xy, p->pts.perm, n, nullptr,
                                             (double*)d_dth, (double*)d_dph, nullptr, (const double*)cot, gpts);
  else
    interp_k<float, true><<<nb, tb, 0, s>>>((const float*)p->fine, stride, z.n1, z.n2, z.w, (float)z.beta, z.beta,
                                            p->pts.cell, nullptr, nullptr, p->pts.xy, p->pts.perm, n, nullptr,
                                            (float*)d_dth, (float*)d_dph, nullptr, (const float*)cot, gpts);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int interp_pointing(nusht_plan_t p, double* d_ptg, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const int64_t n = p->pts.npts;
  if (n == 0) return NUSHT_OK;
  if (nufft_df(p) && p->pts.nsub > 0) return interp_grad_df(p, nullptr, nullptr, d_ptg, nullptr, nullptr, s);
  const int64_t stride = 2 * (z.n2 / 2 + 1);
  const int tb = 128;
  const int nb = (int)((n + tb - 1) / tb);
  if (p->precision == NUSHT_FP64)
    interp_k<double, true><<<nb, tb, 0, s>>>((const double*)p->fine, stride, z.n1, z.n2, z.w, (float)z.beta, z.beta,
                                             p->pts.cell, nullptr, nullptr, p->pts.xy, p->pts.perm, n, nullptr,
                                             nullptr, nullptr, d_ptg, nullptr, nullptr);
  else
    interp_k<float, true><<<nb, tb, 0, s>>>((const float*)p->fine, stride, z.n1, z.n2, z.w, (float)z.beta, z.beta,
                                            p->pts.cell, nullptr, nullptr, p->pts.xy, p->pts.perm, n, nullptr,
                                            nullptr, nullptr, d_ptg, nullptr, nullptr);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int spread(nusht_plan_t p, const void* d_map, cudaStream_t s) {
  const nusht_sizes& z = p->sz;
  const int64_t stride = 2 * (z.n2 / 2 + 1);
  const size_t es = p->precision == NUSHT_FP64 ? 8 : 4;
  const bool det = p->opts.deterministic != 0 && p->pts.tiles != nullptr;
  if (p->pts.nsub == 0 || !det) NUSHT_CUDA(cudaMemsetAsync(p->fine, 0, (size_t)z.n1 * stride * es, s));
  if (p->pts.nsub == 0) return NUSHT_OK;
  const int binsz = p->pts.bin > 0 ? p->pts.bin : 32;
  const int tw = binsz + z.w - 1;
  // FP32 spreading kernels stage the subproblem's points after the tile
  const size_t sm = p->precision == NUSHT_FP64 ? (size_t)tw * tw * es : spread_f_smem(tw);
  if (nufft_df(p)) {
    const size_t smd = (size_t)tw * spread_df_stride(tw, z.w) * 8 + (size_t)SUBMAX * 16;
    NUSHT_W_DISPATCH(z.w, launch_spread_df, p->pts.nsub, smd, s, (double*)p->fine, stride, z.n1,
                     z.n2, p->pts.nbins2, binsz, p->pts.sub, p->pts.cell,
                     reinterpret_cast<const float2*>(p->pts.psi), p->pts.perm, (const double*)d_map,
                     det ? (float2*)p->pts.tiles : nullptr);
  } else if (p->precision == NUSHT_FP64) {
    spread_k<double><<<p->pts.nsub, 32, sm, s>>>((double*)p->fine, stride, z.n1, z.n2, z.w, p->pts.nbins2, binsz,
                                                 (float)z.beta, p->pts.sub, p->pts.cell, p->pts.psi, nullptr,
                                                 p->pts.perm, (const double*)d_map,
                                                 det ? (double*)p->pts.tiles : nullptr);
  } else if (det) {
    // one warp per subproblem, points in order, lanes own distinct cells: no
    // atomics, so the tile is reproducible
    spread_k<float><<<p->pts.nsub, 32, sm, s>>>((float*)p->fine, stride, z.n1, z.n2, z.w, p->pts.nbins2, binsz,
                                                (float)z.beta, p->pts.sub, p->pts.cell, nullptr, p->pts.off,
                                                p->pts.perm, (const float*)d_map, (float*)p->pts.tiles);
  } else {
    NUSHT_W_DISPATCH(z.w, launch_spread_f, p->pts.nsub, sm, s, (float*)p->fine, stride, z.n1, z.n2, p->pts.nbins2,
                     binsz, (float)z.beta, p->pts.sub, p->pts.cell, p->pts.off, p->pts.perm, (const float*)d_map,
                     p->pts.spread_rows);
  }
  NUSHT_CUDA(cudaGetLastError());
  if (det) {
    const int64_t ncell = (int64_t)z.n1 * z.n2;
    const unsigned nb = (unsigned)((ncell + 255) / 256);
    const int nb1 = p->pts.nbins1, nb2 = p->pts.nbins2;
    if (nufft_df(p))
      grid_gather_k<double, double, float2><<<nb, 256, 0, s>>>((double*)p->fine, stride, z.n1, z.n2, binsz, tw, nb1,
                                                              nb2, p->pts.binsub, (const float2*)p->pts.tiles);
    else if (p->precision == NUSHT_FP64)
      grid_gather_k<double, double, double><<<nb, 256, 0, s>>>((double*)p->fine, stride, z.n1, z.n2, binsz, tw, nb1,
                                                              nb2, p->pts.binsub, (const double*)p->pts.tiles);
    else
      grid_gather_k<float, float, float><<<nb, 256, 0, s>>>((float*)p->fine, stride, z.n1, z.n2, binsz, tw, nb1, nb2,
                                                           p->pts.binsub, (const float*)p->pts.tiles);
    NUSHT_CUDA(cudaGetLastError());
  }
  return NUSHT_OK;
}

int zero_grids_many(const NufftBatch& nb, cudaStream_t s) {
  if (nb.nzero <= 0) return NUSHT_OK;
  zero_grids_k<<<nb.nzero, 256, 0, s>>>(nb.mem, nb.nm);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int spread_many(const NufftBatch& nb, const float* const* maps, cudaStream_t s) {
  if (nb.nsub <= 0) return NUSHT_OK;
  const int tw = nb.bin + nb.w - 1;
  NUSHT_W_DISPATCH(nb.w, launch_spread_many, nb, spread_f_smem(tw), s, maps);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int interp_many(const NufftBatch& nb, float* const* maps, cudaStream_t s) {
  if (nb.nblk <= 0) return NUSHT_OK;
  NUSHT_W_DISPATCH(nb.w, launch_interp_many, nb, s, maps);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int deconv_pad_many(const NufftBatch& nb, cudaStream_t s) {
  if (nb.npad <= 0) return NUSHT_OK;
  deconv_pad_many_k<<<nb.npad, dim3(32, 8), 0, s>>>(nb.mem, nb.nm);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

int deconv_trunc_many(const NufftBatch& nb, cudaStream_t s) {
  if (nb.ntrunc <= 0) return NUSHT_OK;
  deconv_trunc_many_k<<<nb.ntrunc, dim3(32, 8), 0, s>>>(nb.mem, nb.nm);
  NUSHT_CUDA(cudaGetLastError());
  return NUSHT_OK;
}

}  // namespace nusht
