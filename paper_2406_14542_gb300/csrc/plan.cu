// plan.cu -- host side of the library: argument checks, size choice, ES
// kernel parameters and Fourier factors, plan life cycle and the execute
// entry points that chain the device stages (Eq. SHTfast / adjointSHTfast).
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "nusht_internal.cuh"

namespace nusht {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  if (code != NUSHT_OK) g_last_error = msg;
  return code;
}

int cuda_status(cudaError_t e, const char* what) {
  (void)cudaGetLastError();  // clear sticky-free errors so the next call starts clean
  int code = (e == cudaErrorMemoryAllocation) ? NUSHT_ENOMEM
             : (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver || e == cudaErrorNoKernelImageForDevice)
                 ? NUSHT_EDEVICE
                 : NUSHT_ECUDA;
  return set_error(code, std::string(what) + ": " + cudaGetErrorString(e));
}

int cufft_status(cufftResult r, const char* what) {
  int code = (r == CUFFT_ALLOC_FAILED) ? NUSHT_ENOMEM : NUSHT_ECUDA;
  return set_error(code, std::string(what) + ": cuFFT error " + std::to_string((int)r));
}

// Allocation fault injection for tests: NUSHT_FAIL_ALLOC_AFTER=n makes the
// (n+1)-th device allocation of a plan fail as if the device were full.
static long g_fail_after = -1;
static long g_alloc_count = 0;

int dev_alloc(void** p, size_t bytes, size_t* counter) {
  *p = nullptr;
  if (bytes == 0) return NUSHT_OK;
  if (g_fail_after >= 0 && g_alloc_count++ >= g_fail_after)
    return set_error(NUSHT_ENOMEM, "injected allocation failure (NUSHT_FAIL_ALLOC_AFTER)");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_status(e, "cudaMalloc");
  }
  if (counter) *counter += bytes;
  return NUSHT_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

// ---------------------------------------------------------------------------
// Sizes (Sec. 2.2 and App. B)
// ---------------------------------------------------------------------------
static bool smooth(int64_t n, int maxprime) {
  for (int pr = 2; pr <= maxprime && n > 1; ++pr)
    while (n % pr == 0) n /= pr;
  return n == 1;
}

int64_t good_size(int64_t nmin, int multiple, int maxprime) {
  if (nmin < 1) nmin = 1;
  int64_t n = ((nmin + multiple - 1) / multiple) * multiple;
  while (!smooth(n, maxprime)) n += multiple;
  return n;
}

// Exponential-of-semicircle kernel parameters (Barnett, Magland and
// af Klinteberg, SIAM J. Sci. Comput. 2019, the kernel of cuFINUFFT that the
// paper's N and N^dagger use, Sec. 3): width w from the tolerance and the
// up-sampling factor, shape beta proportional to w.
int es_width(double eps, double sigma) {
  if (std::fabs(sigma - 2.0) < 1e-12) return (int)std::ceil(std::log10(1.0 / eps)) + 1;
  return (int)std::ceil(std::log(1.0 / eps) / (M_PI * std::sqrt(1.0 - 1.0 / sigma)));
}

static void es_params(double eps, double sigma, int w_override, int* w, double* beta) {
  int ww = es_width(eps, sigma);
  if (w_override > 0) ww = w_override;
  ww = std::max(2, std::min(ES_WMAX, ww));
  double b;
  if (std::fabs(sigma - 2.0) < 1e-12) {
    b = 2.30 * ww;
  } else {
    b = 0.97 * M_PI * ww * (1.0 - 0.5 / sigma);
  }
  *w = ww;
  *beta = b;
}

int choose_sizes(int lmax, int mmax, double eps, int precision, const nusht_opts* o, nusht_sizes* out) {
  if (!out) return set_error(NUSHT_EINVAL, "sizes output is NULL");
  if (lmax < 0 || lmax > 16383) return set_error(NUSHT_EINVAL, "lmax must be in [0, 16383]");
  if (mmax < 0 || mmax > lmax) return set_error(NUSHT_EINVAL, "mmax must be in [0, lmax]");
  if (!(eps >= 1e-14 && eps <= 1e-1)) return set_error(NUSHT_EINVAL, "eps must be in [1e-14, 1e-1]");
  if (precision != NUSHT_FP64 && precision != NUSHT_MIXED)
    return set_error(NUSHT_EINVAL, "precision must be NUSHT_FP64 or NUSHT_MIXED");
  if (precision == NUSHT_MIXED && eps < 1e-6)
    return set_error(NUSHT_EUNSUPPORTED, "NUSHT_MIXED supports eps >= 1e-6 only (single-precision grid)");
  nusht_opts opt{};
  if (o) opt = *o;
  // default up-sampling: FP64 grids are FFT-bound (the FP64 2D FFT costs more
  // than the wider kernel sigma = 1.5 needs); FP32 grids are not
  double sigma = opt.sigma > 0.0 ? opt.sigma : (precision == NUSHT_FP64 ? 1.5 : 2.0);
  if (!(sigma >= 1.2 && sigma <= 4.0)) return set_error(NUSHT_EINVAL, "sigma must be in [1.2, 4]");
  if (opt.kernel_width < 0 || opt.kernel_width > ES_WMAX)
    return set_error(NUSHT_EINVAL, "kernel_width must be in [0, 20]");
  std::memset(out, 0, sizeof(*out));
  out->lmax = lmax;
  out->mmax = mmax;
  // doubled theta length: M >= 2 lmax + 2 (so that N_r = M/2 + 1 >= lmax + 2
  // rings resolve every order, see the reading of App. B), multiple of 4 so
  // that ring pairs (theta, pi - theta) tile [0, pi] with the equator as a ring.
  out->M = (int)good_size(2 * (int64_t)lmax + 2, 4, 7);
  out->nrings = out->M / 2 + 1;
  // the NUFFT carries the whole approximation error of the method (S, D and
  // F are exact up to rounding), so it gets a tenth of the requested eps
  int w;
  double beta;
  es_params(0.1 * eps, sigma, opt.kernel_width, &w, &beta);
  out->w = w;
  out->beta = beta;
  out->sigma = sigma;
  int64_t nmin = (int64_t)std::ceil(sigma * (2.0 * lmax + 1.0));
  nmin = std::max<int64_t>(nmin, 2 * (int64_t)w);
  int64_t n = good_size(nmin, 2, 7);
  if (n > (1 << 17)) return set_error(NUSHT_EINVAL, "fine grid too large");
  out->n1 = (int)n;
  out->n2 = (int)n;
  out->precision = precision;
  return NUSHT_OK;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
  x.assign(n, 0.0);
  wt.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1, pn1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pn1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    double ww = 2.0 / ((1.0 - z * z) * dp * dp);
    wt[i] = ww;
    wt[n - 1 - i] = ww;
  }
}

// psihat(k) = int_{-alpha}^{alpha} psi(y / alpha) cos(k y) dy, alpha = w pi / n,
// evaluated with z = sin(t): 2 alpha int_0^{pi/2} e^{beta (cos t - 1)} cos(k alpha sin t) cos t dt.
void kernel_ft(int w, double beta, int n, int nk, double* out) {
  const int q = 256;
  std::vector<double> x, wt;
  gauss_legendre(q, x, wt);
  const double alpha = w * M_PI / n;
  std::vector<double> t(q), f(q), st(q);
  for (int i = 0; i < q; ++i) {
    t[i] = 0.25 * M_PI * (x[i] + 1.0);  // [0, pi/2]
    f[i] = 0.25 * M_PI * wt[i] * std::exp(beta * (std::cos(t[i]) - 1.0)) * std::cos(t[i]);
    st[i] = std::sin(t[i]);
  }
  for (int k = 0; k < nk; ++k) {
    double s = 0.0;
    for (int i = 0; i < q; ++i) s += f[i] * std::cos(k * alpha * st[i]);
    out[k] = 2.0 * alpha * s;
  }
}

}  // namespace nusht

using namespace nusht;

// ---------------------------------------------------------------------------
// plan life cycle
// ---------------------------------------------------------------------------
static void plan_free(nusht_plan_t p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  free_points(p);
  spin_free(p);
  dev_free(p->leg.c);
  dev_free(p->leg.cdf);
  dev_free(p->leg.ahat);
  dev_free(p->leg.dshift);
  dev_free(p->leg.cm);
  dev_free(p->leg.ring_x);
  dev_free(p->leg.ring_s);
  dev_free(p->leg.pole_norm);
  dev_free(p->leg.items);
  dev_free(p->leg.tab);
  dev_free(p->leg.tab_off);
  dev_free(p->deconv1);
  dev_free(p->deconv2);
  dev_free(p->atilde);
  dev_free(p->G);
  if (p->ghat_owned) dev_free(p->Ghat);
  dev_free(p->fine);
  dev_free(p->partial);
  dfft_free(p);
  if (p->have_theta) cufftDestroy(p->fft_theta);
  if (p->have_cols) cufftDestroy(p->fft_cols);
  if (p->have_c2r) cufftDestroy(p->fft_c2r);
  if (p->have_r2c) cufftDestroy(p->fft_r2c);
  for (auto* e : {&p->ev_synth, &p->ev_adj})
    if (e->ready)
      for (auto& ev : e->ev) cudaEventDestroy(ev);
  cudaSetDevice(cur);
  delete p;
}

static int make_ffts(nusht_plan_t p, const double* d1, const double* d2) {
  const nusht_sizes& z = p->sz;
  const bool dbl = p->precision == NUSHT_FP64;
  int M = z.M;
  size_t ws = 0;
  // FP64: double-float kernels for every length that fits in shared memory
  const bool own = dbl && p->opts.fft_kernels >= 0;
  const bool want_theta = p->has_legendre || p->theta_member;
  const bool own_theta = own && want_theta && dfft_fits(z, true, false);
  const bool own_fine = own && p->has_nufft && dfft_fits(z, false, true);
  if (own_theta || own_fine) NUSHT_TRY(dfft_setup(p, own_theta, own_fine, d1, d2));
  if (want_theta && !own_theta) {
    NUSHT_CUFFT(cufftCreate(&p->fft_theta));
    p->have_theta = true;
    NUSHT_CUFFT(cufftMakePlanMany(p->fft_theta, 1, &M, nullptr, 1, M, nullptr, 1, M, dbl ? CUFFT_Z2Z : CUFFT_C2C,
                                  z.mmax + 1, &ws));
  }
  if (!p->has_nufft || own_fine) return NUSHT_OK;
  if (!dbl && p->opts.fft_kernels >= 0 && sfft_fits(z)) {
    // FP32, opt-in: this library's line kernels, deconvolution fused into the
    // column pass (cuFFT's 2D plans measured 3-4x faster: the default)
    NUSHT_TRY(sfft_setup(p, d1, d2));
    return NUSHT_OK;
  }
  if (!dbl) {  // FP32: cuFFT's own 2D plans measured faster than the split below
    NUSHT_CUFFT(cufftCreate(&p->fft_c2r));
    p->have_c2r = true;
    NUSHT_CUFFT(cufftMakePlan2d(p->fft_c2r, z.n1, z.n2, CUFFT_C2R, &ws));
    NUSHT_CUFFT(cufftCreate(&p->fft_r2c));
    p->have_r2c = true;
    NUSHT_CUFFT(cufftMakePlan2d(p->fft_r2c, z.n1, z.n2, CUFFT_R2C, &ws));
    return NUSHT_OK;
  }
  // FP64: the 2D real FFT as two batched 1D passes, the first restricted to
  // the columns m <= mmax that deconvolution fills (zero columns stay zero);
  // at lmax 4095, sigma 1.5 this is 18.8 ms per direction against 22.5 ms
  int n1 = z.n1, n2 = z.n2, n2h = z.n2 / 2 + 1, n2r = 2 * n2h;
  NUSHT_CUFFT(cufftCreate(&p->fft_cols));
  p->have_cols = true;
  NUSHT_CUFFT(cufftMakePlanMany(p->fft_cols, 1, &n1, &n1, n2h, 1, &n1, n2h, 1, dbl ? CUFFT_Z2Z : CUFFT_C2C,
                                z.mmax + 1, &ws));
  NUSHT_CUFFT(cufftCreate(&p->fft_c2r));
  p->have_c2r = true;
  NUSHT_CUFFT(cufftMakePlanMany(p->fft_c2r, 1, &n2, &n2h, 1, n2h, &n2r, 1, n2r, dbl ? CUFFT_Z2D : CUFFT_C2R, n1, &ws));
  NUSHT_CUFFT(cufftCreate(&p->fft_r2c));
  p->have_r2c = true;
  NUSHT_CUFFT(cufftMakePlanMany(p->fft_r2c, 1, &n2, &n2r, 1, n2r, &n2h, 1, n2h, dbl ? CUFFT_D2Z : CUFFT_R2C, n1, &ws));
  return NUSHT_OK;
}

// theta DFT of the doubled ring map, [mmax + 1][M] complex: sign -1 forward
// (synthesis), +1 inverse (adjoint); src == dst allowed
static int theta_fft(nusht_plan_t p, const void* src, void* dst, int sign, cudaStream_t s) {
  if (p->dfft_theta) return dfft_theta_exec(p, src, dst, sign, s);
  const int dir = sign < 0 ? CUFFT_FORWARD : CUFFT_INVERSE;
  NUSHT_CUFFT(cufftSetStream(p->fft_theta, s));
  if (p->precision == NUSHT_FP64)
    NUSHT_CUFFT(cufftExecZ2Z(p->fft_theta, (cufftDoubleComplex*)src, (cufftDoubleComplex*)dst, dir));
  else
    NUSHT_CUFFT(cufftExecC2C(p->fft_theta, (cufftComplex*)src, (cufftComplex*)dst, dir));
  return NUSHT_OK;
}

int nusht::fine_fft_c2r(nusht_plan_t p, cudaStream_t s) {
  if (p->dfft_fine) return dfft_rows_c2r(p, s);
  if (p->sfft_fine) return sfft_rows_c2r(sfft_launch_of(p), s);
  NUSHT_CUFFT(cufftSetStream(p->fft_c2r, s));
  if (!p->have_cols) {
    NUSHT_CUFFT(cufftExecC2R(p->fft_c2r, (cufftComplex*)p->fine, (cufftReal*)p->fine));
    return NUSHT_OK;
  }
  NUSHT_CUFFT(cufftSetStream(p->fft_cols, s));
  if (p->precision == NUSHT_FP64) {
    NUSHT_CUFFT(cufftExecZ2Z(p->fft_cols, (cufftDoubleComplex*)p->fine, (cufftDoubleComplex*)p->fine, CUFFT_INVERSE));
    NUSHT_CUFFT(cufftExecZ2D(p->fft_c2r, (cufftDoubleComplex*)p->fine, (cufftDoubleReal*)p->fine));
  } else {
    NUSHT_CUFFT(cufftExecC2C(p->fft_cols, (cufftComplex*)p->fine, (cufftComplex*)p->fine, CUFFT_INVERSE));
    NUSHT_CUFFT(cufftExecC2R(p->fft_c2r, (cufftComplex*)p->fine, (cufftReal*)p->fine));
  }
  return NUSHT_OK;
}

int nusht::fine_fft_r2c(nusht_plan_t p, cudaStream_t s) {
  if (p->dfft_fine) return dfft_rows_r2c(p, s);
  if (p->sfft_fine) return sfft_rows_r2c(sfft_launch_of(p), s);
  NUSHT_CUFFT(cufftSetStream(p->fft_r2c, s));
  if (!p->have_cols) {
    NUSHT_CUFFT(cufftExecR2C(p->fft_r2c, (cufftReal*)p->fine, (cufftComplex*)p->fine));
    return NUSHT_OK;
  }
  NUSHT_CUFFT(cufftSetStream(p->fft_cols, s));
  if (p->precision == NUSHT_FP64) {
    NUSHT_CUFFT(cufftExecD2Z(p->fft_r2c, (cufftDoubleReal*)p->fine, (cufftDoubleComplex*)p->fine));
    NUSHT_CUFFT(cufftExecZ2Z(p->fft_cols, (cufftDoubleComplex*)p->fine, (cufftDoubleComplex*)p->fine, CUFFT_FORWARD));
  } else {
    NUSHT_CUFFT(cufftExecR2C(p->fft_r2c, (cufftReal*)p->fine, (cufftComplex*)p->fine));
    NUSHT_CUFFT(cufftExecC2C(p->fft_cols, (cufftComplex*)p->fine, (cufftComplex*)p->fine, CUFFT_FORWARD));
  }
  return NUSHT_OK;
}

static int check_device(int* dev) {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    (void)cudaGetLastError();
    return set_error(NUSHT_EDEVICE, "no CUDA device available");
  }
  NUSHT_CUDA(cudaGetDevice(dev));
  cudaDeviceProp prop;
  NUSHT_CUDA(cudaGetDeviceProperties(&prop, *dev));
  if (!(prop.major == 10 && prop.minor == 3))
    return set_error(NUSHT_EDEVICE, std::string("library is built for sm_103a (GB300); device is ") + prop.name);
  return NUSHT_OK;
}

static int plan_body(nusht_plan_t p, int64_t npts, const double* d_pts, cudaStream_t s, const PlanRole& role) {
  const nusht_sizes& z = p->sz;
  const size_t cplx = (p->precision == NUSHT_FP64) ? 16 : 8;
  const size_t gbytes = (size_t)(z.mmax + 1) * z.M * cplx;
  if (!role.nufft) {
    // bucket tables only: recurrence coefficients and the polar-skip work list
    NUSHT_TRY(legendre_build_tables(p, s));
    p->sz.nitems = p->leg.nitems;
    p->sz.nitems_total = p->leg.nitems_total;
    p->sz.leg_triples = p->leg.triples;
    return NUSHT_OK;
  }
  // Fourier factors of the ES kernel (deconvolution, Sec. 3 on the NUFFT):
  // d1[k] = h1 / (M psihat1(k)) folds the 1/M of the theta DFT, d2[m] = h2 / psihat2(m).
  std::vector<double> d1(2 * z.lmax + 1), d2(z.mmax + 1);
  {
    std::vector<double> f1(z.lmax + 1), f2(z.mmax + 1);
    kernel_ft(z.w, z.beta, z.n1, z.lmax + 1, f1.data());
    kernel_ft(z.w, z.beta, z.n2, z.mmax + 1, f2.data());
    const double h1 = 2.0 * M_PI / z.n1, h2 = 2.0 * M_PI / z.n2;
    for (int k = -z.lmax; k <= z.lmax; ++k) d1[k + z.lmax] = h1 / ((double)z.M * f1[std::abs(k)]);
    for (int m = 0; m <= z.mmax; ++m) d2[m] = h2 / f2[m];
    NUSHT_TRY(dev_alloc((void**)&p->deconv1, d1.size() * 8, &p->bytes));
    NUSHT_TRY(dev_alloc((void**)&p->deconv2, d2.size() * 8, &p->bytes));
    NUSHT_CUDA(cudaMemcpyAsync(p->deconv1, d1.data(), d1.size() * 8, cudaMemcpyHostToDevice, s));
    NUSHT_CUDA(cudaMemcpyAsync(p->deconv2, d2.data(), d2.size() * 8, cudaMemcpyHostToDevice, s));
    NUSHT_CUDA(cudaStreamSynchronize(s));
  }
  if (role.legendre) {
    NUSHT_TRY(dev_alloc(&p->atilde, (size_t)p->nalm * cplx, &p->bytes));
    NUSHT_TRY(dev_alloc(&p->G, gbytes, &p->bytes));
    NUSHT_CUDA(cudaMemsetAsync(p->G, 0, gbytes, s));
  }
  if (role.ghat_external) {
    p->Ghat = role.ghat_external;
    p->ghat_owned = false;
  } else {
    NUSHT_TRY(dev_alloc(&p->Ghat, gbytes, &p->bytes));
  }
  NUSHT_TRY(dev_alloc(&p->fine, (size_t)z.n1 * (z.n2 / 2 + 1) * cplx, &p->bytes));
  if (role.legendre) {
    NUSHT_TRY(legendre_build_tables(p, s));
    NUSHT_TRY(dev_alloc(&p->partial, (size_t)p->leg.blocks_per_m * p->nalm * cplx, &p->bytes));
    NUSHT_CUDA(cudaMemsetAsync(p->partial, 0, (size_t)p->leg.blocks_per_m * p->nalm * cplx, s));
    if (p->opts.spin > 0) NUSHT_TRY(spin_setup(p, s));
  }
  NUSHT_TRY(make_ffts(p, d1.data(), d2.data()));
  NUSHT_TRY(spread_smem_optin());
  if (role.bin > 0) {
    p->pts.bin = role.bin;
    NUSHT_TRY(setpts_impl(p, npts, d_pts, s));
  } else {
    NUSHT_TRY(tune_points(p, npts, d_pts, s));
  }
  NUSHT_CUDA(cudaStreamSynchronize(s));
  p->sz.nitems = p->leg.nitems;
  p->sz.nitems_total = p->leg.nitems_total;
  p->sz.leg_triples = p->leg.triples;
  p->sz.npts = p->pts.npts;
  return NUSHT_OK;
}

extern "C" {

int nusht_plan(nusht_plan_t* out, int lmax, int mmax, int64_t npts, const double* d_pts, double eps, int precision,
               const nusht_opts* opts, nusht_stream_t stream) {
  nusht_opts o{};
  if (opts) o = *opts;
  nusht::PlanRole role;
  if (out && o.sigma == 0.0 && (o.tune == 1 || o.tune == 2) && npts > 0 && d_pts) {
    double sg = 0.0;
    int bin = 0;
    NUSHT_TRY(nusht::tune_sigma(lmax, mmax, npts, d_pts, eps, precision, &o, (cudaStream_t)stream, &sg, &bin));
    if (sg > 0.0) {
      o.sigma = sg;
      role.bin = bin;
    }
  }
  return nusht::plan_create(out, lmax, mmax, npts, d_pts, eps, precision, &o, (cudaStream_t)stream, role);
}

}  // extern "C"

int nusht::plan_create(nusht_plan_t* out, int lmax, int mmax, int64_t npts, const double* d_pts, double eps,
                       int precision, const nusht_opts* opts, cudaStream_t stream, const PlanRole& role) {
  if (!out) return set_error(NUSHT_EINVAL, "out is NULL");
  *out = nullptr;
  nusht_sizes z;
  NUSHT_TRY(choose_sizes(lmax, mmax, eps, precision, opts, &z));
  if (role.M_override) {
    if (role.M_override < z.M || role.M_override % 4) return set_error(NUSHT_EINVAL, "bad theta length override");
    z.M = role.M_override;
    z.nrings = z.M / 2 + 1;
  }
  if (npts < 0 || npts > 0x7fffffffLL) return set_error(NUSHT_EINVAL, "npts must be in [0, 2^31)");
  if (npts > 0 && !d_pts) return set_error(NUSHT_EINVAL, "d_pts is NULL");
  if (opts && (opts->spin < 0 || opts->spin > lmax)) return set_error(NUSHT_EINVAL, "spin must be in [0, lmax]");
  if (opts && opts->spin > 0 && (precision != NUSHT_FP64 || !role.legendre || !role.nufft))
    return set_error(NUSHT_EUNSUPPORTED, "spin transforms need a standalone NUSHT_FP64 plan");
  int dev = 0;
  NUSHT_TRY(check_device(&dev));
  const char* fa = std::getenv("NUSHT_FAIL_ALLOC_AFTER");
  g_fail_after = fa ? std::atol(fa) : -1;
  g_alloc_count = 0;
  nusht_plan_t p = new (std::nothrow) nusht_plan_s();
  if (!p) return set_error(NUSHT_ENOMEM, "host allocation failed");
  p->device = dev;
  p->lmax = lmax;
  p->mmax = mmax;
  p->precision = precision;
  p->eps = eps;
  p->sz = z;
  if (opts) p->opts = *opts;
  p->nalm = (int64_t)(mmax + 1) * (lmax + 1) - (int64_t)mmax * (mmax + 1) / 2;
  p->has_legendre = role.legendre;
  p->has_nufft = role.nufft;
  p->theta_member = role.theta;
  cudaStream_t s = stream;
  int st = plan_body(p, npts, d_pts, s, role);
  g_fail_after = -1;
  if (st != NUSHT_OK) {
    cudaStreamSynchronize(s);
    plan_free(p);
    return st;
  }
  p->sz.bytes_device = (int64_t)p->bytes;
  *out = p;
  return NUSHT_OK;
}

void nusht::plan_destroy(nusht_plan_t p) { plan_free(p); }

extern "C" {

int nusht_setpts(nusht_plan_t p, int64_t npts, const double* d_pts, nusht_stream_t stream) {
  if (!p) return set_error(NUSHT_EINVAL, "plan is NULL");
  if (npts < 0 || npts > 0x7fffffffLL) return set_error(NUSHT_EINVAL, "npts must be in [0, 2^31)");
  if (npts > 0 && !d_pts) return set_error(NUSHT_EINVAL, "d_pts is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  NUSHT_TRY(setpts_impl(p, npts, d_pts, s));
  NUSHT_CUDA(cudaStreamSynchronize(s));
  p->sz.npts = p->pts.npts;
  p->sz.bytes_device = (int64_t)p->bytes;
  return NUSHT_OK;
}

static int ev_init(nusht::StageEvents& e) {
  if (e.ready) return NUSHT_OK;
  for (auto& ev : e.ev) NUSHT_CUDA(cudaEventCreate(&ev));
  e.ready = true;
  return NUSHT_OK;
}

#define STAGE(evs, i)                                               \
  do {                                                              \
    if (prof) NUSHT_CUDA(cudaEventRecord((evs).ev[i], s));          \
  } while (0)

int nusht_synth(nusht_plan_t p, const void* d_alm, void* d_map, nusht_stream_t stream) {
  if (!p) return set_error(NUSHT_EINVAL, "plan is NULL");
  if (!d_alm || (!d_map && p->pts.npts > 0)) return set_error(NUSHT_EINVAL, "null alm or map pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const bool prof = p->opts.profile != 0;
  if (prof) NUSHT_TRY(ev_init(p->ev_synth));
  p->last_stream = s;
  STAGE(p->ev_synth, 0);
  // S with D fused into its store: Legendre sums on the rings, written doubled
  NUSHT_TRY(legendre_synth(p, d_alm, s));
  STAGE(p->ev_synth, 1);
  // F along theta (the phi transforms of S and F cancel, Sec. 3)
  NUSHT_TRY(theta_fft(p, p->G, p->Ghat, -1, s));
  STAGE(p->ev_synth, 2);
  // N: deconvolve and zero-pad onto the fine spectrum, FFT to the fine grid, interpolate
  NUSHT_TRY(deconv_pad(p, s));
  STAGE(p->ev_synth, 3);
  NUSHT_TRY(fine_fft_c2r(p, s));
  STAGE(p->ev_synth, 4);
  NUSHT_TRY(interp(p, d_map, s));
  STAGE(p->ev_synth, 5);
  return NUSHT_OK;
}

}  // extern "C"

// N^dagger, F^dagger, D^dagger, S^dagger; the m > 0 coefficients are scaled
// by wpos (1: the adjoint, 2: the gradient convention of nusht_adjoint_grad)
static int adjoint_chain(nusht_plan_t p, const void* d_map, void* d_alm, cudaStream_t s, double wpos) {
  if (!p) return set_error(NUSHT_EINVAL, "plan is NULL");
  if (!d_alm || (!d_map && p->pts.npts > 0)) return set_error(NUSHT_EINVAL, "null alm or map pointer");
  const bool prof = p->opts.profile != 0;
  if (prof) NUSHT_TRY(ev_init(p->ev_adj));
  p->last_stream = s;
  STAGE(p->ev_adj, 0);
  // N^dagger: spread onto the fine grid
  NUSHT_TRY(spread(p, d_map, s));
  STAGE(p->ev_adj, 1);
  NUSHT_TRY(fine_fft_r2c(p, s));
  STAGE(p->ev_adj, 2);
  // truncate to |k| <= lmax, m <= mmax and deconvolve
  NUSHT_TRY(deconv_trunc(p, s));
  STAGE(p->ev_adj, 3);
  // F^dagger along theta
  NUSHT_TRY(theta_fft(p, p->Ghat, p->Ghat, 1, s));
  STAGE(p->ev_adj, 4);
  // D^dagger fused into S^dagger's load: fold, then adjoint Legendre sums
  NUSHT_TRY(legendre_adjoint(p, d_alm, s, wpos));
  STAGE(p->ev_adj, 5);
  return NUSHT_OK;
}

extern "C" {

int nusht_adjoint(nusht_plan_t p, const void* d_map, void* d_alm, nusht_stream_t stream) {
  return adjoint_chain(p, d_map, d_alm, (cudaStream_t)stream, 1.0);
}

int nusht_adjoint_grad(nusht_plan_t p, const void* d_cot, void* d_galm, nusht_stream_t stream) {
  return adjoint_chain(p, d_cot, d_galm, (cudaStream_t)stream, 2.0);
}

int nusht_synth_grad(nusht_plan_t p, const void* d_alm, void* d_dtheta, void* d_dphi, nusht_stream_t stream) {
  if (!p) return set_error(NUSHT_EINVAL, "plan is NULL");
  if (!d_alm) return set_error(NUSHT_EINVAL, "null alm pointer");
  if (!d_dtheta && !d_dphi) return NUSHT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  NUSHT_TRY(legendre_synth(p, d_alm, s));
  NUSHT_TRY(theta_fft(p, p->G, p->Ghat, -1, s));
  NUSHT_TRY(deconv_pad(p, s));
  NUSHT_TRY(fine_fft_c2r(p, s));
  NUSHT_TRY(interp_grad(p, d_dtheta, d_dphi, nullptr, nullptr, s));
  return NUSHT_OK;
}

int nusht_synth_grad_pts(nusht_plan_t p, const void* d_alm, const void* d_cot, double* d_gpts,
                         nusht_stream_t stream) {
  if (!p) return set_error(NUSHT_EINVAL, "plan is NULL");
  if (!d_alm || (p->pts.npts > 0 && (!d_cot || !d_gpts))) return set_error(NUSHT_EINVAL, "null pointer");
  if (!p->has_legendre || !p->has_nufft) return set_error(NUSHT_EUNSUPPORTED, "needs a standalone plan");
  cudaStream_t s = (cudaStream_t)stream;
  NUSHT_TRY(legendre_synth(p, d_alm, s));
  NUSHT_TRY(theta_fft(p, p->G, p->Ghat, -1, s));
  NUSHT_TRY(deconv_pad(p, s));
  NUSHT_TRY(fine_fft_c2r(p, s));
  NUSHT_TRY(interp_grad(p, nullptr, nullptr, d_cot, d_gpts, s));
  return NUSHT_OK;
}

int nusht_synth_spin(nusht_plan_t p, const void* d_glm, const void* d_clm, void* d_q, void* d_u,
                     nusht_stream_t stream) {
  if (!p) return set_error(NUSHT_EINVAL, "plan is NULL");
  if (p->opts.spin <= 0 || !p->spin.A) return set_error(NUSHT_EUNSUPPORTED, "plan made without opts.spin");
  if (!d_glm || !d_clm || (p->pts.npts > 0 && (!d_q || !d_u))) return set_error(NUSHT_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  // S for both fields at once (the Wigner-d recurrences are shared), then
  // F and N for each
  NUSHT_TRY(spin_legendre_synth(p, d_glm, d_clm, s));
  for (int k = 0; k < 2; ++k) {
    NUSHT_TRY(theta_fft(p, k ? p->spin.GU : p->spin.GQ, p->Ghat, -1, s));
    NUSHT_TRY(deconv_pad(p, s));
    NUSHT_TRY(fine_fft_c2r(p, s));
    NUSHT_TRY(interp(p, k ? d_u : d_q, s));
  }
  return NUSHT_OK;
}

int nusht_adjoint_spin(nusht_plan_t p, const void* d_q, const void* d_u, void* d_glm, void* d_clm,
                       nusht_stream_t stream) {
  if (!p) return set_error(NUSHT_EINVAL, "plan is NULL");
  if (p->opts.spin <= 0 || !p->spin.A) return set_error(NUSHT_EUNSUPPORTED, "plan made without opts.spin");
  if (!d_glm || !d_clm || (p->pts.npts > 0 && (!d_q || !d_u))) return set_error(NUSHT_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  // N^dagger and F^dagger for each field into its theta-spectrum buffer, then
  // D^dagger and S^dagger for both
  for (int k = 0; k < 2; ++k) {
    NUSHT_TRY(spread(p, k ? d_u : d_q, s));
    NUSHT_TRY(fine_fft_r2c(p, s));
    NUSHT_TRY(deconv_trunc(p, s));
    NUSHT_TRY(theta_fft(p, p->Ghat, k ? p->spin.GU : p->spin.GQ, 1, s));
  }
  NUSHT_TRY(spin_legendre_adjoint(p, d_glm, d_clm, s));
  return NUSHT_OK;
}

int nusht_pointing(nusht_plan_t p, const void* d_philm, double* d_ptg, nusht_stream_t stream) {
  if (!p) return set_error(NUSHT_EINVAL, "plan is NULL");
  if (!d_philm || (!d_ptg && p->pts.npts > 0)) return set_error(NUSHT_EINVAL, "null potential or pointing pointer");
  if (!p->has_legendre || !p->has_nufft) return set_error(NUSHT_EUNSUPPORTED, "pointing needs a standalone plan");
  cudaStream_t s = (cudaStream_t)stream;
  // the potential's synthesis up to the fine grid, then the derivative-of-kernel
  // interpolation with the deflection applied per point
  NUSHT_TRY(legendre_synth(p, d_philm, s));
  NUSHT_TRY(theta_fft(p, p->G, p->Ghat, -1, s));
  NUSHT_TRY(deconv_pad(p, s));
  NUSHT_TRY(fine_fft_c2r(p, s));
  NUSHT_TRY(interp_pointing(p, d_ptg, s));
  return NUSHT_OK;
}

int nusht_destroy(nusht_plan_t p) {
  plan_free(p);
  return NUSHT_OK;
}

int nusht_info(nusht_plan_t p, nusht_sizes* out) {
  if (!p || !out) return set_error(NUSHT_EINVAL, "null argument");
  *out = p->sz;
  out->bytes_device = (int64_t)p->bytes;
  return NUSHT_OK;
}

int nusht_plan_bin(nusht_plan_t p, int* bin) {
  if (!p || !bin) return set_error(NUSHT_EINVAL, "null argument");
  *bin = p->pts.bin;
  return NUSHT_OK;
}

int nusht_plan_sizes(int lmax, int mmax, double eps, int precision, const nusht_opts* opts, nusht_sizes* out) {
  return choose_sizes(lmax, mmax, eps, precision, opts, out);
}

int nusht_kernel_ft(int w, double beta, int n, int nk, double* out) {
  if (w < 2 || w > ES_WMAX || !(beta > 0) || n < 2 * w || nk < 0 || (nk > 0 && !out))
    return set_error(NUSHT_EINVAL, "bad kernel_ft arguments");
  kernel_ft(w, beta, n, nk, out);
  return NUSHT_OK;
}

int64_t nusht_good_size(int64_t nmin, int multiple, int maxprime) {
  if (multiple < 1 || maxprime < 2) return -1;
  return good_size(nmin, multiple, maxprime);
}

int nusht_stage_times(nusht_plan_t p, double* out) {
  if (!p || !out) return set_error(NUSHT_EINVAL, "null argument");
  for (int i = 0; i < 12; ++i) out[i] = 0.0;
  if (p->ev_synth.ready) NUSHT_CUDA(cudaEventSynchronize(p->ev_synth.ev[5]));
  if (p->ev_adj.ready) NUSHT_CUDA(cudaEventSynchronize(p->ev_adj.ev[5]));
  cudaError_t err = cudaSuccess;
  auto span = [&err](cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      err = e;
      return 0.0;
    }
    return (double)ms;
  };
  if (p->ev_synth.ready) {
    for (int i = 0; i < 5; ++i) out[i] = span(p->ev_synth.ev[i], p->ev_synth.ev[i + 1]);
    out[5] = span(p->ev_synth.ev[0], p->ev_synth.ev[5]);
  }
  if (p->ev_adj.ready) {
    for (int i = 0; i < 5; ++i) out[6 + i] = span(p->ev_adj.ev[i], p->ev_adj.ev[i + 1]);
    out[11] = span(p->ev_adj.ev[0], p->ev_adj.ev[5]);
  }
  if (err != cudaSuccess) return cuda_status(err, "cudaEventElapsedTime");
  return NUSHT_OK;
}

const char* nusht_strerror(int code) {
  switch (code) {
    case NUSHT_OK: return "NUSHT_OK";
    case NUSHT_EINVAL: return "NUSHT_EINVAL: invalid argument";
    case NUSHT_ENOMEM: return "NUSHT_ENOMEM: allocation failed";
    case NUSHT_ECUDA: return "NUSHT_ECUDA: CUDA or cuFFT error";
    case NUSHT_EUNSUPPORTED: return "NUSHT_EUNSUPPORTED: unsupported combination";
    case NUSHT_ETIMEOUT: return "NUSHT_ETIMEOUT: device wait timed out";
    case NUSHT_EDEVICE: return "NUSHT_EDEVICE: no usable device";
    default: return "unknown nusht status";
  }
}

const char* nusht_last_error(void) { return g_last_error.c_str(); }

const char* nusht_version(void) { return "nusht-gb300 0.1 (sm_103a)"; }

}  // extern "C"
