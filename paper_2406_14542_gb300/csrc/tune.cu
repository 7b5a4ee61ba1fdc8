// tune.cu -- plan-time autotuner of the NUFFT: up-sampling factor sigma and
// spreading / interpolation bin size.
//
// sigma (opts.sigma = 0 with opts.tune = 1): for each sigma in {2, 1.5, 1.25}
// whose accuracy formula width fits the kernel's limit of 20, a NUFFT-only
// trial plan (its own bin search included) times the sigma-dependent stages
// of one synthesis + adjoint: deconvolution/padding, the 2D FFTs,
// interpolation and spreading.  The fastest sigma is cached under the device,
// precision, lmax, mmax, eps decade and point-count power of two;
// opts.tune = 2 reuses the cached sigma.
//
// opts.tune = 0: bin edge 16 cells for FP64 plans with kernel width <= 17 and
// float-pair arithmetic (fp64_contraction = 0), 32 cells otherwise.
// opts.tune = 1 (search): the plan sorts
// its points for each candidate bin edge (16, 32, 64 cells), times one
// spreading + interpolation pass with CUDA events on the plan's own data, keeps
// the fastest and records it in a cache file.  opts.tune = 2 (cached): the
// cached choice for the same key when present, else the untuned default.  Key: device name,
// precision, lmax, kernel width, fine grid and the point count's power of two.
// Cache: $NUSHT_TUNE_CACHE, else $HOME/.cache/nusht_tune.txt, one
// "key bin" line per entry (the last entry of a key wins).
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>

#include "nusht_internal.cuh"

namespace nusht {

namespace {

std::string cache_path() {
  if (const char* e = std::getenv("NUSHT_TUNE_CACHE")) return e;
  const char* h = std::getenv("HOME");
  std::string d = std::string(h ? h : "/tmp") + "/.cache";
  mkdir(d.c_str(), 0755);
  return d + "/nusht_tune.txt";
}

std::string device_name(int dev);

std::string tune_key(nusht_plan_t p, int64_t npts) {
  std::ostringstream k;
  k << device_name(p->device) << ":p" << p->precision << ":L" << p->lmax << ":w" << p->sz.w << ":n" << p->sz.n1 << "x" << p->sz.n2
    << ":N" << (npts > 0 ? (int)std::floor(std::log2((double)npts)) : 0);
  return k.str();
}

int cache_lookup(const std::string& key) {
  std::ifstream f(cache_path());
  std::string k;
  int v = 0, found = 0;
  while (f >> k >> v)
    if (k == key) found = v;
  return found;
}

void cache_store(const std::string& key, int bin) {
  std::ofstream f(cache_path(), std::ios::app);
  if (f) f << key << " " << bin << "\n";
}

std::string device_name(int dev) {
  cudaDeviceProp prop;
  std::string d = "gpu";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) d = prop.name;
  for (auto& c : d)
    if (c == ' ') c = '_';
  return d;
}

// one synthesis + adjoint pass of the sigma-dependent stages of a NUFFT-only plan
int nufft_roundtrip(nusht_plan_t q, void* map, cudaStream_t s) {
  NUSHT_TRY(deconv_pad(q, s));
  NUSHT_TRY(fine_fft_c2r(q, s));
  NUSHT_TRY(interp(q, map, s));
  NUSHT_TRY(spread(q, map, s));
  NUSHT_TRY(fine_fft_r2c(q, s));
  NUSHT_TRY(deconv_trunc(q, s));
  return NUSHT_OK;
}

}  // namespace

int tune_sigma(int lmax, int mmax, int64_t npts, const double* d_pts, double eps, int precision,
               const nusht_opts* o, cudaStream_t s, double* sigma_out, int* bin_out) {
  *sigma_out = 0.0;
  *bin_out = 0;
  int dev = 0;
  NUSHT_CUDA(cudaGetDevice(&dev));
  std::ostringstream k;
  k << "S:" << device_name(dev) << ":p" << precision << ":L" << lmax << ":m" << mmax << ":e"
    << (int)std::lround(std::log10(eps)) << ":N" << (int)std::floor(std::log2((double)npts));
  const std::string key = k.str();
  if (o->tune == 2) {
    const int v = cache_lookup(key);
    if (v >= 120 && v <= 400) *sigma_out = v / 100.0;
    return NUSHT_OK;
  }
  const double cand[3] = {2.0, 1.5, 1.25};
  const size_t es = precision == NUSHT_FP64 ? 8 : 4;
  void* map = nullptr;
  NUSHT_TRY(dev_alloc(&map, (size_t)npts * es, nullptr));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = NUSHT_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = set_error(NUSHT_ECUDA, "event");
  if (st == NUSHT_OK && cudaMemsetAsync(map, 0, (size_t)npts * es, s) != cudaSuccess)
    st = set_error(NUSHT_ECUDA, "memset");
  double best_s = 0.0;
  int best_bin = 0;
  float best_ms = 1e30f;
  for (int c = 0; c < 3 && st == NUSHT_OK; ++c) {
    if (es_width(0.1 * eps, cand[c]) > ES_WMAX) continue;  // accuracy not reachable within the width limit
    // FP32 rounding amplified by the large deconvolution factors of sigma =
    // 1.25 measured eps_eff 2.2e-6 at eps = 1e-6 (lmax 1023): not offered there
    if (precision == NUSHT_MIXED && cand[c] < 1.4 && eps < 1e-5) continue;
    nusht_opts oc = *o;
    oc.sigma = cand[c];
    oc.tune = 1;
    PlanRole r;
    r.legendre = false;
    nusht_plan_t q = nullptr;
    if ((st = plan_create(&q, lmax, mmax, npts, d_pts, eps, precision, &oc, s, r)) != NUSHT_OK) break;
    const size_t gbytes = (size_t)(q->sz.mmax + 1) * q->sz.M * (precision == NUSHT_FP64 ? 16 : 8);
    if (cudaMemsetAsync(q->Ghat, 0, gbytes, s) != cudaSuccess) st = set_error(NUSHT_ECUDA, "memset");
    if (st == NUSHT_OK) st = nufft_roundtrip(q, map, s);  // warm-up
    if (st == NUSHT_OK) {
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 2 && st == NUSHT_OK; ++rep) st = nufft_roundtrip(q, map, s);
      cudaEventRecord(e1, s);
    }
    float ms = 0.f;
    if (st == NUSHT_OK) {
      if (cudaEventSynchronize(e1) != cudaSuccess)
        st = set_error(NUSHT_ECUDA, "tuning timer");
      else
        cudaEventElapsedTime(&ms, e0, e1);
    }
    if (st == NUSHT_OK && ms < best_ms) {
      best_ms = ms;
      best_s = cand[c];
      best_bin = q->pts.bin;
    }
    cudaStreamSynchronize(s);
    plan_destroy(q);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  dev_free(map);
  if (st != NUSHT_OK) return st;
  if (best_s > 0.0) {
    cache_store(key, (int)std::lround(best_s * 100.0));
    *sigma_out = best_s;
    *bin_out = best_bin;
  }
  return NUSHT_OK;
}

int tune_cache_get(const std::string& key) { return cache_lookup(key); }
void tune_cache_put(const std::string& key, int value) { cache_store(key, value); }
std::string tune_device(int dev) { return device_name(dev); }

int tune_points(nusht_plan_t p, int64_t npts, const double* d_pts, cudaStream_t s) {
  const int mode = p->opts.tune;
  // untuned bin edge (plans whose caller fixed no bin come here once, at
  // creation): 16 cells for the double-float FP64 NUFFT (one warp per bin, so
  // smaller tiles keep more warps per SM: spreading 12.8 -> 9.4 ms at lmax
  // 4095, interpolation 5.22 -> 5.31 ms), 32 otherwise; 16 needs w - 1 <= 16
  // for the deterministic gather
  p->pts.bin = (p->precision == NUSHT_FP64 && !p->opts.fp64_contraction && p->sz.w <= 17) ? 16 : 32;
  if (mode == 0 || npts == 0) return setpts_impl(p, npts, d_pts, s);
  const std::string key = tune_key(p, npts);
  if (mode == 2) {
    const int b = cache_lookup(key);
    if (b == 16 || b == 32 || b == 64) p->pts.bin = b;
    return setpts_impl(p, npts, d_pts, s);
  }
  // search: time spreading + interpolation for each candidate
  const size_t es = p->precision == NUSHT_FP64 ? 8 : 4;
  void* map = nullptr;
  NUSHT_TRY(dev_alloc(&map, (size_t)npts * es, nullptr));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = NUSHT_OK;
  int best = 32;
  float best_ms = 1e30f;
  const int cand[3] = {16, 32, 64};
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = set_error(NUSHT_ECUDA, "event");
  if (st == NUSHT_OK && cudaMemsetAsync(map, 0x3f, (size_t)npts * es, s) != cudaSuccess)
    st = set_error(NUSHT_ECUDA, "memset");
  for (int c = 0; c < 3 && st == NUSHT_OK; ++c) {
    p->pts.bin = cand[c];
    if ((st = setpts_impl(p, npts, d_pts, s)) != NUSHT_OK) break;
    if ((st = spread(p, map, s)) != NUSHT_OK) break;  // warm-up
    if ((st = interp(p, map, s)) != NUSHT_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2 && st == NUSHT_OK; ++r) {
      if ((st = spread(p, map, s)) != NUSHT_OK) break;
      st = interp(p, map, s);
    }
    cudaEventRecord(e1, s);
    if (st != NUSHT_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = set_error(NUSHT_ECUDA, "tuning timer");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = cand[c];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  dev_free(map);
  if (st != NUSHT_OK) return st;
  cache_store(key, best);
  p->pts.bin = best;
  return setpts_impl(p, npts, d_pts, s);
}

}  // namespace nusht
