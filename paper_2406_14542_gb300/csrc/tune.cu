// tune.cu -- plan-time autotuner of the spreading / interpolation bin size.
//
// opts.tune = 0: bin edge 32 cells.  opts.tune = 1 (search): the plan sorts
// its points for each candidate bin edge (16, 32, 64 cells), times one
// spreading + interpolation pass with CUDA events on the plan's own data, keeps
// the fastest and records it in a cache file.  opts.tune = 2 (cached): the
// cached choice for the same key when present, else 32.  Key: device name,
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

std::string tune_key(nusht_plan_t p, int64_t npts) {
  cudaDeviceProp prop;
  std::string dev = "gpu";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) dev = prop.name;
  for (auto& c : dev)
    if (c == ' ') c = '_';
  std::ostringstream k;
  k << dev << ":p" << p->precision << ":L" << p->lmax << ":w" << p->sz.w << ":n" << p->sz.n1 << "x" << p->sz.n2
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

}  // namespace

int tune_points(nusht_plan_t p, int64_t npts, const double* d_pts, cudaStream_t s) {
  const int mode = p->opts.tune;
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
