// nusht_internal.cuh -- plan layout and shared declarations of the CUDA
// library (not part of the public ABI; see include/nusht.h for that).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nusht.h"

namespace nusht {

// ---------------------------------------------------------------------------
// Error plumbing: every host entry point returns a status and records a
// thread-local message.
// ---------------------------------------------------------------------------
int set_error(int code, const std::string& msg);
int cuda_status(cudaError_t e, const char* what);
int cufft_status(cufftResult r, const char* what);

#define NUSHT_CUDA(call)                                                  \
  do {                                                                    \
    cudaError_t _e = (call);                                              \
    if (_e != cudaSuccess) return ::nusht::cuda_status(_e, #call);        \
  } while (0)
#define NUSHT_CUFFT(call)                                                 \
  do {                                                                    \
    cufftResult _r = (call);                                              \
    if (_r != CUFFT_SUCCESS) return ::nusht::cufft_status(_r, #call);     \
  } while (0)
#define NUSHT_TRY(call)                                                   \
  do {                                                                    \
    int _s = (call);                                                      \
    if (_s != NUSHT_OK) return _s;                                        \
  } while (0)

// Device allocation through one place so that tests can inject failures.
int dev_alloc(void** p, size_t bytes, size_t* counter);
void dev_free(void* p);

// ---------------------------------------------------------------------------
// Legendre work decomposition.
// Ring pairs (theta_j, pi - theta_j) for j = 1..M/4 (the poles are handled
// apart).  One warp owns RINGS_PER_WARP = 32*K consecutive pairs of one
// order m: a "work item".
// ---------------------------------------------------------------------------
constexpr int LEG_K = 4;                 // ring pairs per lane
constexpr int LEG_PAIRS_PER_WARP = 32 * LEG_K;
constexpr int LEG_SEG_BITS = 48;         // rescaled normalisation kept in [1, 2^(48+8))
constexpr int LEG_SEG_BITS_DF = 24;      // the same with the double-float recurrence

// Start exponent threshold of the scaled phase: values below 2^-300 (relative
// to the rescaled normalisation) are not accumulated (Sec. 3: on-the-fly
// recurrence with scaled exponents so that high-l values do not underflow).
constexpr int LEG_TINY_EXP = -300;
constexpr int LEG_STEP_EXP = 256;        // scaled-phase exponent step

struct LegTables {
  // per (l, m) packed m-major, nalm entries
  double* c = nullptr;        // c_lm = (l-1-m)(l-1+m)/((2l-3)(2l-1)) (0 for l = m, m+1)
  float2* cdf = nullptr;      // c_lm as a float pair (opts.fast_recurrence only)
  double* ahat = nullptr;     // rescaled normalisation Ahat_lm (>= 1)
  int8_t* dshift = nullptr;   // rescale exponent applied before step l (0 = none)
  // per m
  double* cm = nullptr;       // Pbar_mm / sin^m(theta) = signed c_m
  // per ring pair j = 1..M/4 (index j-1)
  double* ring_x = nullptr;   // cos(theta_j)
  double* ring_s = nullptr;   // sin(theta_j)
  double* pole_norm = nullptr; // sqrt((2l+1)/(4 pi)), l = 0..lmax
  int* items = nullptr;       // work list: (m << 16) | block
  int nitems = 0;
  int nitems_total = 0;
  int64_t triples = 0;        // (ring pair, l, m) triples of the kept items
  void* tab = nullptr;        // recurrence table (table mode): float or float2 per triple
  int64_t* tab_off = nullptr; // per-item offsets into tab
  size_t tab_bytes = 0;
  int blocks_per_m = 0;       // ring blocks per order
  int npairs = 0;             // M/4
};

struct PointData {
  int64_t npts = 0;
  int64_t cap = 0;
  int* perm = nullptr;        // sorted index -> caller index
  int* cell = nullptr;        // sorted: first tap (i1, i2) interleaved, wrapped to [0, n)
  double* psi = nullptr;      // FP64: kernel values [npts][2w] (w along theta, then w along phi);
                              // as float pairs (hi, lo) when the NUFFT runs in double-float
  double* xy = nullptr;       // sorted coordinates (theta, phi), for the position gradient
  float* off = nullptr;       // MIXED: fractional offsets (t - i) per dim, [2][npts]
  // subproblems for spreading: (bin index, first sorted point, count)
  int* sub = nullptr;
  int nsub = 0;
  int nbins1 = 0, nbins2 = 0;
  int bin = 32;               // bin edge in fine-grid cells (spreading tile = bin + w - 1)
  int spread_rows = 0;        // FP32 spreading: 1 = lanes a tile row apart (scattered points, many
                              // sharing a cell), 0 = consecutive points on consecutive lanes
  // fine-grid rows some point's taps reach (the others are neither read by
  // interpolation nor written by spreading): a flag per row and the list of
  // row pairs (j / 2 for the pair j, j + 1) the row FFT passes transform
  unsigned char* rowmask = nullptr;
  int* rowpairs = nullptr;
  int nrowpairs = 0;
  size_t bytes = 0;           // device bytes held for points (part of the plan's total)
  // opts.deterministic: every subproblem's tile is written here ([nsub][tile]),
  // then summed per grid cell in a fixed order (no atomics)
  void* tiles = nullptr;
  size_t tiles_cap = 0;
  int* binsub = nullptr;      // subproblems of bin b: [binsub[b], binsub[b + 1])
};

// One transform length of the double-float FFT kernels (dfft.cu): radices
// of the in-place decimation-in-frequency passes, the twiddle table
// W_N^k = (cos hi, cos lo, sin hi, sin lo) and the shared-memory position of
// each output index after the passes.
constexpr int DFFT_NMAX = 14336;  // longest line: N float-pair complex values in shared memory
constexpr int DFFT_MAXPASS = 16;
struct DfftLen {
  int N = 0, npass = 0;
  unsigned long long code = 0;  // radix of pass s in bits [4s, 4s + 4)
  float4* tw = nullptr;         // float-pair twiddles e^(2 pi i k / N), k < N (double-float engine)
  float2* tw2 = nullptr;        // FP32 engine: e^(2 pi i k / N) for k < 64, then for k = 64 c
  int* rev = nullptr;
};

// One transform of the FP32 fine-grid FFT kernels (dfft.cu) of mixed plans;
// a single plan has one, a batch one per member, so that each pass is one
// launch for all members.  The order-major spectrum T sits between the
// column pass (along theta, per order) and the row pass (along phi, per
// pair of real rows).
constexpr int SFFT_NMAX = 2 * DFFT_NMAX;  // longest line: float complex values in shared memory
struct SfftMember {
  float2* Gh = nullptr;        // theta spectrum [mmax + 1][M] (synthesis input, adjoint output)
  float2* T = nullptr;         // [mmax + 1][n1]
  float* grid = nullptr;       // fine grid, n1 rows of `stride` floats
  const float* d1 = nullptr;   // theta deconvolution factors, k = -lmax..lmax (1/M included)
  const float* d2 = nullptr;   // phi deconvolution factors, m = 0..mmax
  int64_t stride = 0;
  int lmax = 0, mmax = 0, M = 0, n1 = 0, n2 = 0;
  int col0 = 0, row0 = 0;      // first CTA of this member in the column / row launches
  DfftLen f1, f2;              // line tables of n1 and n2
  const int* rowpairs = nullptr;           // row pairs (j / 2) some point reaches: the row launches
  const unsigned char* rowmask = nullptr;  // per row: stored by the column pass
};

// One transform of the mixed-precision NUFFT kernels that serve every member
// of a batch in one launch (nufft.cu): the member's fine grid and sorted
// points.  Interpolation blocks of 128 threads never straddle two members
// (each member's points start at a multiple of 128 in the launch), spreading
// blocks are the members' subproblems one after another.
struct NufftMember {
  float* grid = nullptr;       // n1 rows of `stride` floats
  const int* cell = nullptr;   // sorted points: first tap (i1, i2)
  const float* off = nullptr;  // sorted points: fractional offsets
  const int* perm = nullptr;   // sorted index -> caller index
  const int* sub = nullptr;    // spreading subproblems (bin, first point, count)
  int64_t stride = 0;
  int64_t npts = 0;
  int n1 = 0, n2 = 0, nbins2 = 0, bin = 0;
  int spread_rows = 0;         // as PointData::spread_rows
  int blk0 = 0;                // first interpolation block
  int sub0 = 0;                // first spreading block
  int zero0 = 0;               // first block of the grid zero fill
  float beta = 0.f;
  // deconvolution between the theta spectrum and the fine spectrum (the
  // grid buffer seen as n1 x (n2/2 + 1) complex), 32 x 32 tiles
  float2* Gh = nullptr;        // theta spectrum [mmax + 1][M]
  const double* d1 = nullptr;  // k = -lmax..lmax
  const double* d2 = nullptr;  // m = 0..mmax
  int lmax = 0, mmax = 0, M = 0;
  int pad0 = 0;                // first block of the padding launch
  int trunc0 = 0;              // first block of the truncation launch
};
struct NufftBatch {
  const NufftMember* mem = nullptr;  // device table (a slice of the batch's table)
  int nm = 0, w = 0;
  int nblk = 0, nsub = 0, nzero = 0; // blocks of the three launches
  int blk_base = 0, sub_base = 0;    // blk0 / sub0 of the slice's first member
  int npad = 0, ntrunc = 0;          // blocks of the deconvolution launches
  int map_base = 0;                  // position of the slice in the batch's tables
  int bin = 32;                      // largest bin edge (spreading tile size)
};

// Spin-weighted transforms (spin.cu): Wigner-d recurrence tables of the
// plan's spin s (opts.spin), per packed (l, m), start values per order, the
// two ring maps (Q and U; theta spectra in the adjoint) and the partial rows
// of the adjoint
struct SpinTables {
  double* A = nullptr;        // sqrt((2l+1)(2l-1)) l / sqrt((l^2-m^2)(l^2-s^2))
  double* Ab = nullptr;       // A m s / (l (l-1))
  double* C = nullptr;        // the l-2 coefficient
  double* st_mant = nullptr;  // start value at max(m, s) per (m, sign): mantissa ...
  int* st_exp = nullptr;      // ... binary exponent ...
  int* st_ab = nullptr;       // ... and powers of cos and sin of theta / 2 (a << 16 | b)
  double2* GQ = nullptr;      // [mmax + 1][M]
  double2* GU = nullptr;
  float4* ap = nullptr;       // per call: (G + iC) / 2 and (-1)^s (G - iC) / 2 as float pairs
  float4* am = nullptr;
  float4* pg = nullptr;       // [nrows][nalm] float-pair partial sums of G and C
  float4* pc = nullptr;
  unsigned char* keep = nullptr;  // per (order, ring block): bit k = pass k has a value above 2^-300
  int nrows = 0;
};

struct StageEvents {
  cudaEvent_t ev[8] = {};
  bool ready = false;
};

}  // namespace nusht

struct nusht_plan_s {
  int device = 0;
  int lmax = 0, mmax = 0, precision = NUSHT_FP64;
  double eps = 0.0;
  nusht_sizes sz{};
  nusht_opts opts{};
  int64_t nalm = 0;

  nusht::LegTables leg;
  nusht::PointData pts;

  // kernel Fourier factors: d1[k + lmax] (k = -lmax..lmax), d2[m] (m = 0..mmax)
  double* deconv1 = nullptr;
  double* deconv2 = nullptr;

  // work buffers
  void* atilde = nullptr;     // per-call rescaled coefficients (complex, nalm)
  void* G = nullptr;          // doubled ring map [mmax+1][M] complex
  void* Ghat = nullptr;       // theta spectrum [mmax+1][M] complex
  void* fine = nullptr;       // fine spectrum / grid, n1 x (n2/2+1) complex == n1 x (n2+2) real
  void* partial = nullptr;    // adjoint Legendre partial sums [blocks_per_m][nalm] complex

  cufftHandle fft_theta = 0;  // batched 1D, length M, batch mmax+1
  // fine-grid FFT, in place on [n1][n2/2 + 1] complex = [n1][n2 + 2] real.
  // FP64: along the first dimension only the columns m <= mmax (the others
  // are zero), then the real transform along every row; FP32: 2D plans.
  cufftHandle fft_cols = 0;   // FP64: C2C along n1, columns 0..mmax (stride n2/2 + 1)
  cufftHandle fft_c2r = 0;    // FP64: rows complex-to-real along n2; FP32: 2D
  cufftHandle fft_r2c = 0;    // FP64: rows real-to-complex along n2; FP32: 2D
  bool have_theta = false, have_c2r = false, have_r2c = false, have_cols = false;

  // FP64 plans: the theta and fine-grid FFTs as double-float kernels (dfft.cu)
  // instead of cuFFT's FP64 transforms; tcols holds the fine spectrum order
  // by order, [mmax + 1][n1] float-pair complex, between the column and row passes
  bool dfft_theta = false, dfft_fine = false;
  nusht::DfftLen dft_theta, dft_n1, dft_n2;
  void* tcols = nullptr;
  float2* deconv1f = nullptr;  // deconv1 / deconv2 as float pairs
  float2* deconv2f = nullptr;

  // mixed plans: the fine-grid FFT as this library's FP32 line kernels
  // (dfft.cu) with the deconvolution and padding / truncation fused into the
  // column pass; tcols holds [mmax + 1][n1] float complex between the passes
  bool sfft_fine = false;
  float* deconv1s = nullptr;   // deconv1 / deconv2 as float
  float* deconv2s = nullptr;
  nusht::SfftMember* sfft_mem = nullptr;  // device copy of this plan's member entry

  size_t bytes = 0;

  nusht::SpinTables spin;     // opts.spin > 0 (FP64 plans)

  // role inside a batch (see nusht::PlanRole); a standalone plan has all parts
  bool has_legendre = true, has_nufft = true, ghat_owned = true;
  bool theta_member = false;  // PlanRole::theta

  // profiling
  nusht::StageEvents ev_synth, ev_adj;
  cudaStream_t last_stream = nullptr;
};

namespace nusht {

// What a plan builds.  A standalone plan has everything.  Inside a batch,
// member plans carry only the NUFFT part (points, fine grid, deconvolution
// factors, 2D FFTs) and read/write their theta spectrum in a slice of their
// bucket's buffer; a bucket owns one Legendre-only plan for the tables.
struct PlanRole {
  int M_override = 0;         // theta length shared by a bucket (0 = own choice)
  bool legendre = true;
  bool nufft = true;
  void* ghat_external = nullptr;
  int bin = 0;                // spreading bin edge chosen by the caller (0: opts.tune decides)
  bool theta = false;         // a NUFFT-only member that runs its own theta FFT on float pairs
};
int plan_create(nusht_plan_t* out, int lmax, int mmax, int64_t npts, const double* d_pts, double eps, int precision,
                const nusht_opts* opts, cudaStream_t s, const PlanRole& role);
void plan_destroy(nusht_plan_t p);

// sizes / host math (plan.cu)
int choose_sizes(int lmax, int mmax, double eps, int precision, const nusht_opts* o, nusht_sizes* out);
void kernel_ft(int w, double beta, int n, int nk, double* out);

// point set-up (nufft.cu)
int setpts_impl(nusht_plan_t p, int64_t npts, const double* d_pts, cudaStream_t s);
void free_points(nusht_plan_t p);

// Legendre (legendre.cu)
int legendre_build_tables(nusht_plan_t p, cudaStream_t s);
int legendre_synth(nusht_plan_t p, const void* d_alm, cudaStream_t s);
// wpos: factor of the m > 0 coefficients (1: the adjoint; 2: the gradient of a
// real loss with respect to complex a_lm)
int legendre_adjoint(nusht_plan_t p, void* d_alm, cudaStream_t s, double wpos = 1.0);

// NUFFT steps (nufft.cu)
int deconv_pad(nusht_plan_t p, cudaStream_t s);
int deconv_trunc(nusht_plan_t p, cudaStream_t s);
int interp(nusht_plan_t p, void* d_map, cudaStream_t s);
// d/dtheta and d/dphi at the points (either output may be NULL), or with
// gpts = (cot_i d/dtheta, cot_i d/dphi) interleaved
int interp_grad(nusht_plan_t p, void* d_dth, void* d_dph, const void* cot, double* gpts, cudaStream_t s);
int interp_pointing(nusht_plan_t p, double* d_ptg, cudaStream_t s);
int spread(nusht_plan_t p, const void* d_map, cudaStream_t s);
int spread_smem_optin();
// every member of a NufftBatch (mixed precision, atomics): zero the fine
// grids, spread the maps (caller order, maps[i] of member i), interpolate
int zero_grids_many(const NufftBatch& nb, cudaStream_t s);
int spread_many(const NufftBatch& nb, const float* const* maps, cudaStream_t s);
int interp_many(const NufftBatch& nb, float* const* maps, cudaStream_t s);
// deconvolution + zero padding (theta spectrum -> fine spectrum) and
// truncation + deconvolution (fine spectrum -> theta spectrum) of every member
int deconv_pad_many(const NufftBatch& nb, cudaStream_t s);
int deconv_trunc_many(const NufftBatch& nb, cudaStream_t s);
constexpr int ZERO_CHUNK = 1 << 14;  // floats zeroed per block

// spin-weighted transforms (spin.cu)
int spin_setup(nusht_plan_t p, cudaStream_t s);
void spin_free(nusht_plan_t p);
int spin_legendre_synth(nusht_plan_t p, const void* glm, const void* clm, cudaStream_t s);
int spin_legendre_adjoint(nusht_plan_t p, void* glm, void* clm, cudaStream_t s);

// autotuner (tune.cu)
int tune_points(nusht_plan_t p, int64_t npts, const double* d_pts, cudaStream_t s);
// the tuner's cache (one "key value" line per entry, the last one wins) and
// the device name used in its keys
int tune_cache_get(const std::string& key);
void tune_cache_put(const std::string& key, int value);
std::string tune_device(int dev);
// fine spectrum -> fine grid (inverse, both dimensions) and back (forward)
int fine_fft_c2r(nusht_plan_t p, cudaStream_t s);
int fine_fft_r2c(nusht_plan_t p, cudaStream_t s);
// double-float FFTs (dfft.cu): whether every length fits, set-up, execution
bool dfft_fits(const nusht_sizes& z, bool theta, bool fine);
int dfft_setup(nusht_plan_t p, bool theta, bool fine, const double* d1, const double* d2);
void dfft_free(nusht_plan_t p);
int dfft_theta_exec(nusht_plan_t p, const void* src, void* dst, int sign, cudaStream_t s);
// the theta DFT with float-pair input and output in both directions (members
// of FP64 batched plans; needs dfft_theta and dfft_fine)
int dfft_theta_pairs(nusht_plan_t p, const void* src, void* dst, int sign, cudaStream_t s);
int dfft_cols_synth(nusht_plan_t p, cudaStream_t s);
int dfft_rows_c2r(nusht_plan_t p, cudaStream_t s);
int dfft_rows_r2c(nusht_plan_t p, cudaStream_t s);
int dfft_cols_adjoint(nusht_plan_t p, cudaStream_t s);
// FP32 fine-grid FFTs of mixed plans (dfft.cu): whether every length fits,
// set-up (line tables, T, float deconvolution factors, the plan's member
// entry), a member entry from a plan's buffers (col0 / row0 left 0), and the
// passes for a device table of nm members with ncols / nrows CTAs in all
bool sfft_fits(const nusht_sizes& z);
int sfft_setup(nusht_plan_t p, const double* d1, const double* d2);
void sfft_member(nusht_plan_t p, SfftMember& m);
struct SfftLaunch {
  const SfftMember* mem = nullptr;  // device table
  int nm = 0, ncols = 0, nrows = 0;
  int maxn1 = 0, maxn2 = 0;         // longest lines (shared memory per CTA)
};
// shared memory of an FP32 line kernel CTA for lines up to n values (padded
// line + twiddle table), and its ceiling (the sm_103 per-CTA maximum)
int sfft_smem(int n);
constexpr int SFFT_SMEM_MAX = 227 * 1024;
int sfft_cols_synth(const SfftLaunch& l, cudaStream_t s);
int sfft_rows_c2r(const SfftLaunch& l, cudaStream_t s);
int sfft_rows_r2c(const SfftLaunch& l, cudaStream_t s);
int sfft_cols_adjoint(const SfftLaunch& l, cudaStream_t s);
SfftLaunch sfft_launch_of(nusht_plan_t p);
// largest ES kernel width the spreading / interpolation kernels support
constexpr int ES_WMAX = 20;
// ES kernel width the accuracy formula asks for at NUFFT tolerance eps and
// up-sampling sigma (before the [2, ES_WMAX] clamp)
int es_width(double eps, double sigma);
// opts.tune 1/2 with opts.sigma = 0: the up-sampling factor (and the bin edge
// found with it) from timing, or from the cache; *sigma_out = 0 if none
int tune_sigma(int lmax, int mmax, int64_t npts, const double* d_pts, double eps, int precision,
               const nusht_opts* o, cudaStream_t s, double* sigma_out, int* bin_out);

}  // namespace nusht
