/*
 * nusht.h -- C ABI of the GB300 (sm_103a) nonuniform spin-0 spherical
 * harmonic transform library (method of cuNUSHT, arXiv 2406.14542).
 *
 * Transforms (Sec. 2.1):
 *   type 2, "synthesis" (Eq. SHTbase):
 *       f_i = sum_{l<=lmax} sum_{|m|<=min(l,mmax)} a_lm Y_l^m(theta_i, phi_i)
 *   type 1, "adjoint" (Eq. adjointSHTbase), the exact adjoint of type 2:
 *       c_lm = sum_i f_i conj(Y_l^m(theta_i, phi_i))
 * with Y_l^m = P_l^m(theta) e^{i m phi} (Eq. Ylm) and the orthonormal
 * P_l^m = d^l_{m0}(theta) sqrt((2l+1)/(4 pi)) of the footnote of Sec. 2.2,
 * Condon-Shortley phase included (Y_1^1 = -sqrt(3/(8 pi)) sin(theta) e^{i phi}).
 *
 * Real fields.  Coefficients are stored for m >= 0 only; negative orders are
 * implied by a_{l,-m} = (-1)^m conj(a_lm), so maps are real.  Im(a_l0) is
 * ignored by synthesis and the adjoint returns Im(c_l0) = 0.  The adjoint is
 * the adjoint under <c, a> = sum_l Re(conj(c_l0) a_l0)
 *                           + 2 sum_{l, m>0} Re(conj(c_lm) a_lm).
 *
 * Coefficient layout ("m-major"): a_lm lives at index m (2 lmax + 1 - m)/2 + l
 * for 0 <= m <= mmax, m <= l <= lmax; nalm = (mmax+1)(lmax+1) - mmax(mmax+1)/2
 * complex numbers, interleaved (re, im).  Points: npts pairs (theta, phi) of
 * doubles, interleaved, any finite reals (theta and phi are taken modulo 2 pi
 * on the doubled torus of Fig. doubling, which names the same sphere point).
 *
 * Method (Sec. 2.2, Eq. SHTfast / adjointSHTfast): Y = N F D S.  S evaluates
 * the Legendre sums on Clenshaw-Curtis rings, D doubles theta to [0, 2 pi),
 * F is a uniform FFT (here a 1D theta FFT, the phi FFTs of S and F cancel,
 * Sec. 3), N is a type 2 NUFFT with the exponential-of-semicircle kernel.
 *
 * Precision modes (what each stage computes in; Sec. 4 reads accuracy as the
 * relative l2 error eps_eff against the exact sum):
 *   NUSHT_FP64   coefficients complex128, maps double.  In double (FP64
 *                instructions): the P_lm recurrence and its rescaling, the
 *                DFS doubling and fold, the coordinate reduction (cell index
 *                and offset), the kernel values and the deconvolution factors
 *                (both computed at plan time).  In double-float (unevaluated
 *                float pairs hi + lo on the FP32 pipe, ~2^-47 relative per
 *                operation, float exponent range) by default: the Legendre
 *                contraction (sum_l a_lm P_lm and its adjoint), the theta FFT
 *                and the fine-grid 2D FFT (lengths up to 14336; longer ones use
 *                cuFFT in double), spreading and interpolation; the kernel
 *                values are stored as float pairs.  opts.fp64_contraction = 1
 *                and opts.fft_kernels = -1 together select FP64 instructions
 *                for every stage.  Measured eps_eff at lmax 4095 is ~6e-12
 *                either way, against the 1e-10 target.
 *   NUSHT_MIXED  coefficients complex64, maps float.  The Legendre recurrence,
 *                its rescaling and the DFS fold in double (by default the
 *                recurrence runs once at plan time, see opts.legendre_table);
 *                the Legendre contraction, the FFTs and spreading /
 *                interpolation in float.  Point coordinates stay double in
 *                both modes (the cell index and offset are reduced in double,
 *                Sec. 4 on single-precision pointing).
 *
 * Memory and streams.  Every d_* pointer is DEVICE memory owned by the caller
 * and must stay valid for the duration of the call's stream work.  A plan owns
 * all of its workspace, allocated in nusht_plan; the execute calls
 * (nusht_synth, nusht_adjoint, nusht_synth_grad, nusht_adjoint_grad,
 * nusht_synth_grad_pts, nusht_pointing) allocate nothing, copy
 * nothing to or from the host and do not synchronise: they enqueue kernels and
 * cuFFT work on `stream` (NULL = the legacy default stream) and return.  A plan
 * may be used by one stream at a time.  Plans are bound to the device that was
 * current when they were created.
 *
 * Errors.  Every call returns NUSHT_OK (0) or a code below; nusht_strerror
 * names it and nusht_last_error returns the message of the calling thread's
 * most recent failure.  Invalid arguments are rejected before any GPU work.
 */
#ifndef NUSHT_H
#define NUSHT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NUSHT_API __attribute__((visibility("default")))
#else
#define NUSHT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* CUDA stream handle (identical to cudaStream_t). */
typedef struct CUstream_st* nusht_stream_t;

/* Opaque plan: sizes, recurrence tables, sorted points, fine-grid and cuFFT
 * workspaces for one (lmax, mmax, point set, eps, precision). */
typedef struct nusht_plan_s* nusht_plan_t;

enum {
  NUSHT_OK = 0,
  NUSHT_EINVAL = 1,      /* bad argument: sizes, null pointers, eps range */
  NUSHT_ENOMEM = 2,      /* device or host allocation failed */
  NUSHT_ECUDA = 3,       /* CUDA runtime or cuFFT error */
  NUSHT_EUNSUPPORTED = 4, /* valid but unsupported combination */
  NUSHT_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
  NUSHT_EDEVICE = 6      /* no usable CUDA device / wrong architecture */
};

enum { NUSHT_FP64 = 0, NUSHT_MIXED = 1 };

/* Options; a zeroed struct (or NULL) selects the defaults. */
typedef struct {
  double sigma;      /* fine-grid up-sampling factor in [1.2, 4]; 0 = default: 1.5 for
                        NUSHT_FP64 (the FP64 2D FFT dominates), 2.0 for NUSHT_MIXED; with
                        tune = 1 nusht_plan times sigma in {2, 1.5, 1.25} instead (each one
                        whose kernel width for eps fits the limit of 20) and caches the
                        winner, tune = 2 takes the cached one */
  int kernel_width;  /* ES kernel width w override in [2, 20]; 0 = from eps and sigma */
  int profile;       /* 1 = record per-stage CUDA-event times (nusht_stage_times) */
  int deterministic; /* 1 = bit-reproducible adjoint: each spreading subproblem writes its
                        tile (bin + halo) to a plan-owned scratch buffer and every fine-grid
                        cell sums the tiles covering it in a fixed order, instead of adding
                        halos with atomics (FP64 at lmax 4095: 4.0 GB of scratch).  0 = atomics
                        (rounding-level order effects).  Synthesis is always reproducible. */
  int tune;          /* NUFFT autotuner: 0 = off (bin edge 16 cells for FP64 plans with kernel
                        width <= 17 and fp64_contraction = 0, else 32); 1 = search at plan
                        time on the plan's own points (bin edge 16/32/64 and, when sigma = 0,
                        the up-sampling factor), caching the winners; 2 = the cached choices
                        for this device/size when present */
  int fp64_contraction; /* FP64 mode only: 1 = Legendre sums with FP64 instructions;
                           0 (default) = FP64 recurrence, sums as float pairs on the FP32
                           pipe (~2^-48 relative per operation; a_lm magnitudes below 1e20) */
  int legendre_table; /* where the FP64 recurrence runs.  0 = the plan type's default:
                         once at plan time for NUSHT_MIXED plans (nusht_plan, unless
                         fast_recurrence = 1, and nusht_plan_many), every call for
                         NUSHT_FP64 plans; 1 = once at plan time; -1 = every call.  At plan
                         time the values are kept in device memory (a float per (ring pair,
                         l, m) in mixed mode, a float pair in FP64 mode: 59 / 118 GB at lmax
                         4095) when they fit in half the free memory, else the recurrence
                         runs every call */
  int tensor_cores;   /* batched plans whose recurrence table fits: 0 (default) = the
                         contraction on the tensor cores (tcgen05.mma, TF32 operands split
                         into hi + lo, three products per term, FP32 accumulation;
                         ~2^-21 relative per product); -1 = FP32 FMA on the CUDA cores */
  int fast_recurrence; /* 1 = run the P_lm recurrence of single-transform per-call plans in
                          double-float on the FP32 pipe (x, q_l, c_l as float pairs, ~2^-47
                          relative per step instead of FP64's 2^-53; about 2.5x faster Legendre
                          stages on GB300).  Opt-in: the default recurrence is FP64.  Ignored
                          with fp64_contraction = 1 and in recurrence-table mode. */
  int fft_kernels;    /* FP64 plans: 0 (default) = the theta FFT and the fine-grid 2D real FFT
                         run as this library's double-float kernels (one line per CTA in
                         shared memory, ~2^-47 relative per operation) when every length is
                         at most 14336; longer lengths use cuFFT's FP64 transforms;
                         -1 = cuFFT's FP64 transforms always.  Mixed plans: 1 = this
                         library's FP32 line kernels for the fine grid (one line per CTA,
                         deconvolution fused into the column pass; lengths whose line and
                         twiddle table fit in 227 KB of shared memory, about 28,500),
                         -1 = cuFFT FP32 (2D plans, separate deconvolution); 0 (default) =
                         the FP32 line kernels where the lengths fit, else cuFFT.  The line
                         kernels transform only the row pairs some point's taps reach, and
                         in a batch every member's column and row passes are one launch
                         each. */
  int spin;           /* spin weight s >= 1 of nusht_synth_spin / nusht_adjoint_spin (NUSHT_FP64
                         plans; the plan then holds the Wigner-d recurrence tables and two more
                         ring maps); 0 = none */
  int reserved;
} nusht_opts;

/* Sizes a plan uses; filled by nusht_plan_sizes (no GPU needed) and nusht_info. */
typedef struct {
  int lmax, mmax;
  int nrings;        /* Clenshaw-Curtis rings on [0, pi], = M/2 + 1 (>= lmax + 2) */
  int M;             /* doubled theta length (multiple of 4, >= 2 lmax + 2) */
  int n1, n2;        /* fine grid (theta, phi) of the NUFFT */
  int w;             /* ES kernel width in fine-grid cells */
  double beta;       /* ES kernel shape parameter */
  double sigma;      /* up-sampling factor used */
  int precision;
  int nitems;        /* Legendre work items (order, ring block) kept after the polar skip */
  int nitems_total;  /* Legendre work items before the polar skip */
  int64_t npts;
  int64_t bytes_device; /* device memory held by the plan */
  int64_t leg_triples;  /* (ring pair, l, m) triples the Legendre kernels run per call */
} nusht_sizes;

/*
 * nusht_plan -- create a plan (Sec. 3: plans are made once and reused; the
 * NUFFT point set-up is the costly step and happens here, not in execute).
 *   out        receives the plan handle (set to NULL on failure)
 *   lmax       band limit, 0 <= lmax <= 16383
 *   mmax       order limit, 0 <= mmax <= lmax
 *   npts       number of points, >= 0 (< 2^31)
 *   d_pts      device double[2*npts] (theta, phi) pairs; may be NULL if npts == 0
 *   eps        requested relative accuracy, 1e-14 <= eps <= 1e-1
 *              (NUSHT_MIXED requires eps >= 1e-6: NUSHT_EUNSUPPORTED otherwise)
 *   precision  NUSHT_FP64 or NUSHT_MIXED
 *   opts       options or NULL
 *   stream     stream for the set-up kernels; the call synchronises it before
 *              returning (planning is not asynchronous)
 */
NUSHT_API int nusht_plan(nusht_plan_t* out, int lmax, int mmax, int64_t npts, const double* d_pts, double eps,
               int precision, const nusht_opts* opts, nusht_stream_t stream);

/*
 * nusht_setpts -- replace the point set of a plan (re-sort, recompute kernel
 * tables).  npts may differ from the plan's; buffers are reallocated only if
 * it grows beyond the capacity reserved so far.  Synchronises `stream`.
 */
NUSHT_API int nusht_setpts(nusht_plan_t p, int64_t npts, const double* d_pts, nusht_stream_t stream);

/*
 * nusht_synth -- type 2 (Eq. SHTbase, through Eq. SHTfast).
 *   d_alm  device complex (FP64: double[2*nalm]; MIXED: float[2*nalm]), packed m-major
 *   d_map  device FP64: double[npts] / MIXED: float[npts], in the caller's point order
 * Asynchronous on `stream`; allocates nothing.
 */
NUSHT_API int nusht_synth(nusht_plan_t p, const void* d_alm, void* d_map, nusht_stream_t stream);

/*
 * nusht_adjoint -- type 1 (Eq. adjointSHTbase, through Eq. adjointSHTfast).
 *   d_map  device FP64: double[npts] / MIXED: float[npts], caller's point order
 *   d_alm  device complex, overwritten with c_lm (all nalm entries)
 * Asynchronous on `stream`; allocates nothing.
 */
NUSHT_API int nusht_adjoint(nusht_plan_t p, const void* d_map, void* d_alm, nusht_stream_t stream);

/*
 * nusht_synth_grad -- gradient of the synthesised map with respect to the
 * point coordinates: d_dtheta[i] = d f_i / d theta_i, d_dphi[i] = d f_i / d phi_i,
 * evaluated by interpolating with the derivative of the ES kernel on the same
 * fine grid (Sec. 2.2: the torus function is differentiable term by term).
 * Either output pointer may be NULL.  Asynchronous; allocates nothing.
 */
NUSHT_API int nusht_synth_grad(nusht_plan_t p, const void* d_alm, void* d_dtheta, void* d_dphi, nusht_stream_t stream);

/*
 * nusht_adjoint_grad -- gradient of a real loss L(f) with respect to the
 * complex coefficients, given the cotangent g_i = dL/df_i of the synthesised
 * map f = Y a (Eq. SHTbase; the backward pass of a differentiable transform).
 * Because type 1 is the adjoint of type 2 (Sec. 2.1), the gradient is the
 * adjoint applied to g, with the m > 0 entries doubled (each stands for
 * a_{l,m} and a_{l,-m} = (-1)^m conj(a_lm) of the real field):
 *     d_galm[l, m] = w_m (Y^dagger g)_lm,  w_0 = 1, w_{m>0} = 2,
 * in the convention dL/dRe(a) + i dL/dIm(a) (Im of the m = 0 entries is 0).
 *   d_cot   device FP64: double[npts] / MIXED: float[npts], caller's order
 *   d_galm  device complex, nalm entries, overwritten
 * Asynchronous; allocates nothing.
 */
NUSHT_API int nusht_adjoint_grad(nusht_plan_t p, const void* d_cot, void* d_galm, nusht_stream_t stream);

/*
 * nusht_synth_grad_pts -- gradient of a real loss L(f) with respect to the
 * point coordinates, given the cotangent g_i = dL/df_i of f = Y a: since
 * f_i depends only on point i,
 *     d_gpts[2 i] = g_i d f_i / d theta_i,  d_gpts[2 i + 1] = g_i d f_i / d phi_i,
 * with the derivatives from the derivative-of-kernel interpolation of
 * nusht_synth_grad (the same layout as the points, (theta, phi) pairs).
 *   d_alm   device complex coefficients (the plan's precision)
 *   d_cot   device FP64: double[npts] / MIXED: float[npts], caller's order
 *   d_gpts  device double[2 * npts], overwritten
 * Plans made by nusht_plan only (NUSHT_EUNSUPPORTED otherwise).
 * Asynchronous; allocates nothing; overwrites the plan's work buffers.
 */
NUSHT_API int nusht_synth_grad_pts(nusht_plan_t p, const void* d_alm, const void* d_cot, double* d_gpts,
                                   nusht_stream_t stream);

/*
 * nusht_pointing -- CMB lensing pointing (App. C): the deflected position of
 * every point of the plan for the lensing potential Phi.
 *   d_philm  the potential's coefficients in the plan's a_lm layout and
 *            precision (packed m-major, complex128 for NUSHT_FP64, complex64
 *            for NUSHT_MIXED; real field, Im(Phi_l0) ignored)
 *   d_ptg    device double[2 * npts], caller's point order:
 *            d_ptg[2i] = theta'_i in [0, pi], d_ptg[2i + 1] = phi'_i in [0, 2 pi)
 * The gradient alpha_theta + i alpha_phi = (d/dtheta + (i / sin theta) d/dphi) Phi
 * (Eq. spin1deriv) is interpolated at each point with the derivative of the ES
 * kernel (as in nusht_synth_grad), and the point is moved along the geodesic
 * that starts in that direction by the angle alpha = |alpha|:
 * n' = cos(alpha) n + sin(alpha)/alpha (alpha_theta e_theta + alpha_phi e_phi)
 * (Eq. pointing), in double.  A point with sin(theta) = 0 takes alpha_phi = 0.
 * Plans made by nusht_plan only (NUSHT_EUNSUPPORTED otherwise).
 * Asynchronous; allocates nothing; overwrites the plan's work buffers.
 */
NUSHT_API int nusht_pointing(nusht_plan_t p, const void* d_philm, double* d_ptg, nusht_stream_t stream);

/*
 * nusht_synth_spin -- spin-weighted synthesis (the spin-n generalisation of
 * the Conclusion, Sec. 5) of two real fields at the plan's points:
 *     Q + i U = sum_{l >= s} sum_{|m| <= l} (G_lm + i C_lm) sY_lm,
 *     sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi},
 * for the plan's spin s = opts.spin >= 1, with d^l the Wigner small-d matrix
 * (1Y_lm = eth Y_lm / sqrt(l (l+1)), eth = -(d/dtheta + (i/sin theta) d/dphi)).
 * G and C are real-field coefficients (G_{l,-m} = (-1)^m conj(G_lm), same for
 * C) in the packed m-major layout; entries with l < s and Im of the m = 0
 * entries are ignored.  The same chain as nusht_synth (Eq. SHTfast) with a
 * Wigner-d recurrence for S and the spin sign (-1)^s in the doubling.
 * Precision: the two Wigner-d recurrences (d^l_{m,-s}, d^l_{m,s}) in FP64
 * with scaled exponents, the sums over l in double-float (as the spin-0
 * Legendre contraction), the rest as in nusht_synth; measured eps_eff 7e-12
 * at lmax 4095 against the 1e-10 target.
 *   d_glm, d_clm  device complex128[nalm]
 *   d_q, d_u      device double[npts], caller's point order
 * NUSHT_FP64 plans made with opts.spin >= 1 (NUSHT_EUNSUPPORTED otherwise).
 * Asynchronous; allocates nothing.
 */
NUSHT_API int nusht_synth_spin(nusht_plan_t p, const void* d_glm, const void* d_clm, void* d_q, void* d_u,
                               nusht_stream_t stream);

/*
 * nusht_adjoint_spin -- the adjoint (type 1) of nusht_synth_spin under
 * <(G, C), (G', C')> = sum over both of the real-field inner product:
 *     G_lm = sum_i (q_i W_lm + i u_i X_lm) e^{-i m phi_i},
 *     C_lm = sum_i (u_i W_lm - i q_i X_lm) e^{-i m phi_i},
 * W = (sY_lm + (-1)^s (-s)Y_lm) / 2, X = (sY_lm - (-1)^s (-s)Y_lm) / 2 at phi = 0.
 *   d_q, d_u      device double[npts]
 *   d_glm, d_clm  device complex128[nalm], overwritten (entries with l < s
 *                 and Im of the m = 0 entries are 0)
 * Asynchronous; allocates nothing.
 */
NUSHT_API int nusht_adjoint_spin(nusht_plan_t p, const void* d_q, const void* d_u, void* d_glm, void* d_clm,
                                 nusht_stream_t stream);

/*
 * nusht_adjoint_direct_noalloc -- type 1 transform (the adjoint, same result
 * as nusht_adjoint) for small problems, WITHOUT a plan and without
 * allocating any memory.  The paper has no counterpart to this call.
 *
 * Who it is for: callers that must not call cudaMalloc at all, for example
 * code whose device memory is entirely owned by another allocator (a
 * framework's caching pool that reserves the GPU up front, so a raw
 * cudaMalloc would fail or fragment it), or latency-critical loops where the
 * implicit device synchronisation and unbounded latency of cudaMalloc and
 * cudaFree are not acceptable.  nusht_plan allocates, so such callers cannot
 * use the planned path.  This call evaluates
 *     c_lm = sum_i f_i Pbar_lm(theta_i) e^{-i m phi_i}
 * by direct summation on the GPU (O(lmax^2 npts) work, exact to rounding;
 * no FFT or NUFFT), computing the recurrence coefficients on the fly.
 *
 *   lmax, mmax  0 <= mmax <= lmax <= 255; larger lmax is rejected with
 *               NUSHT_EINVAL ("static scratch limit")
 *   npts        >= 0
 *   d_pts       device double[2*npts] (theta, phi), any finite reals
 *   d_map       device double[npts] values f_i
 *   d_alm       device complex128[nalm] output, m-major as for nusht_adjoint
 *               (all entries overwritten; Im(c_l0) = 0)
 *
 * Scratch: partial sums live in one file-scope device array of
 * 16 x 33024 complex doubles (8.45 MB) that every GPU which loads the library
 * keeps until the process exits.  All calls share it, so calls whose GPU work
 * overlaps (different streams, or different host threads, on one device)
 * race on it and give wrong results; serialise them.  Each call overwrites
 * the part it reads, so nothing needs clearing between calls.  The number of
 * partial-sum slots per coefficient is the array's capacity over nalm,
 * capped by the number of 128-point chunks (and by 4096).
 * Set-up: every call looks up that array's device address
 * (cudaGetSymbolAddress) with the calling thread's current device; the first
 * call on a device also loads the library's device code there, so make that
 * first call before any stream capture begins.  Asynchronous on `stream`;
 * no host memory is touched.  Only NUSHT_FP64 (double) inputs are supported.
 */
NUSHT_API int nusht_adjoint_direct_noalloc(int lmax, int mmax, int64_t npts, const double* d_pts, const double* d_map,
                                           void* d_alm, nusht_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched transforms: many independent transforms of uneven lmax and point
 * count in one plan (NUSHT_MIXED or NUSHT_FP64; each lmax <= 4095).  Members are
 * grouped into buckets of up to 64 that share one Clenshaw-Curtis ring set,
 * so one FP64 recurrence per (ring pair, l, m) serves every member of a
 * bucket (Sec. 3: the recurrence is the O(lmax^3) part); the contraction
 * over l (synthesis) or rings (adjoint) runs for all members at once, on the
 * tensor cores (Sec. 4's mixed-precision split: TF32 hi/lo operands, FP32
 * accumulation) or in FP32 on the CUDA cores (opts.tensor_cores).  NUSHT_FP64
 * plans split both operands of the contraction into six bf16 slices under
 * one power of two (the recurrence values per 128-ring-pair block or per
 * order, the coefficients or folded spectrum per order and member) and run
 * the 21 leading slice products on the tensor cores, every level but the
 * synthesis's last summed exactly in FP32 (~46 significant bits against
 * the largest terms; eps down to 1e-10, the same per-order errors as
 * standalone FP64 plans); their members run the double-float FFT and NUFFT
 * kernels of FP64 plans.
 * The grouping minimises a cost model of recurrence and contraction
 * work.  Each direction's whole stage sequence is captured once into a CUDA
 * graph and replayed; it is re-captured when the buffer pointers change.
 * ------------------------------------------------------------------------ */
typedef struct nusht_batch_s* nusht_batch_t;

/*
 * nusht_plan_many -- plan nbatch transforms.
 *   lmax[b]   band limit of member b (mmax = lmax), 0 <= lmax[b] <= 4095
 *   npts[b]   its number of points; d_pts[b] its device (theta, phi) pairs
 *   eps       accuracy, >= 1e-6 for NUSHT_MIXED, >= 1e-10 for NUSHT_FP64
 *   precision NUSHT_MIXED or NUSHT_FP64 (NUSHT_ENOMEM when the FP64 split
 *             tables, ~24 bytes per kept (ring pair, l, m), do not fit in
 *             half the free device memory: on a 288 GB GB300 a bucket up to
 *             lmax ~3000).  For NUSHT_FP64 the contraction
 *             is always the split one (opts.legendre_table and
 *             opts.tensor_cores do not apply) and opts.fft_kernels must be
 *             >= 0 (NUSHT_EUNSUPPORTED otherwise: the members pass float
 *             pairs between the double-float FFT kernels)
 * The host arrays lmax, npts, d_pts are read during the call only.
 * Synchronises `stream`.
 */
NUSHT_API int nusht_plan_many(nusht_batch_t* out, int nbatch, const int* lmax, const int64_t* npts,
                              const double* const* d_pts, double eps, int precision, const nusht_opts* opts,
                              nusht_stream_t stream);

/*
 * nusht_synth_many / nusht_adjoint_many -- all members at once.
 *   d_alm[b]  device coefficients of member b (its own m-major layout):
 *             complex64 (NUSHT_MIXED) or complex128 (NUSHT_FP64)
 *   d_map[b]  device float[npts[b]] (NUSHT_MIXED) or double[npts[b]]
 *             (NUSHT_FP64) values in member b's point order
 * The pointer arrays are host arrays read during the call.  The first call
 * with a given set of buffers captures a CUDA graph (this synchronises the
 * stream and writes the plan's device pointer tables); later calls with the
 * same buffers only launch it on `stream`.
 */
NUSHT_API int nusht_synth_many(nusht_batch_t p, const void* const* d_alm, void* const* d_map, nusht_stream_t stream);
NUSHT_API int nusht_adjoint_many(nusht_batch_t p, const void* const* d_map, void* const* d_alm,
                                 nusht_stream_t stream);

/* nusht_destroy_many -- free a batch plan (NULL-safe). */
NUSHT_API int nusht_destroy_many(nusht_batch_t p);

/*
 * nusht_batch_info -- grouping chosen by the planner: number of buckets,
 * bucket index of each member (bucket_of[nbatch]), band limit of each
 * bucket (bucket_lmax[nbuckets]) and device bytes; any output may be NULL.
 */
NUSHT_API int nusht_batch_info(nusht_batch_t p, int* nbuckets, int* bucket_of, int* bucket_lmax,
                               int64_t* bytes_device);

/*
 * nusht_batch_status -- synchronises `stream`, then reports whether a
 * tensor-core contraction block of an earlier call gave up a bounded wait
 * (one second of device time per wait) and skipped its MMAs:
 * NUSHT_ETIMEOUT (that call's outputs are invalid; the flag is cleared),
 * else NUSHT_OK.  No counterpart in the paper: a guard of this library.
 */
NUSHT_API int nusht_batch_status(nusht_batch_t p, nusht_stream_t stream);

/*
 * nusht_batch_path -- the contraction path of bucket `bucket`: 2 = tensor
 * cores from the recurrence table, 1 = CUDA-core FP32 from the table,
 * 0 = CUDA-core FP32 with the recurrence run every call, 3 = FP64 split
 * bf16 contraction on the tensor cores; -1 for a bad
 * argument.
 */
NUSHT_API int nusht_batch_path(nusht_batch_t p, int bucket);

/*
 * nusht_batch_schedule -- the tensor-core contraction schedule of bucket
 * `bucket`: how many 16-degree chunks are accumulated into one tensor-memory
 * partial set before they are folded into the FP32 register sums, for the
 * synthesis and the adjoint (2, 4 or 8; 4 unless opts.tune chose, 0 for a
 * bucket not on the tensor-core path).  Either output may be NULL.
 * No counterpart in the paper: the schedule of this library's kernel.
 */
NUSHT_API int nusht_batch_schedule(nusht_batch_t p, int bucket, int* chunks_synth, int* chunks_adjoint);

/* nusht_destroy -- free the plan and its device memory (NULL-safe). */
NUSHT_API int nusht_destroy(nusht_plan_t p);

/* nusht_info -- sizes of an existing plan. */
NUSHT_API int nusht_info(nusht_plan_t p, nusht_sizes* out);

/* nusht_plan_bin -- spreading/interpolation bin edge (fine-grid cells) the plan
 * uses: without the autotuner 16 for FP64 plans with kernel width <= 17 and
 * fp64_contraction = 0, else 32; with opts.tune the autotuner's choice. */
NUSHT_API int nusht_plan_bin(nusht_plan_t p, int* bin);

/*
 * nusht_plan_sizes -- the sizes nusht_plan would choose, computed on the host
 * only (no CUDA call): theta length, fine grid, ES kernel width and shape.
 * nitems* and bytes_device are left 0.
 */
NUSHT_API int nusht_plan_sizes(int lmax, int mmax, double eps, int precision, const nusht_opts* opts, nusht_sizes* out);

/*
 * nusht_kernel_ft -- host-side Fourier transform of the ES kernel used for
 * deconvolution: out[k] = integral over |y| <= alpha of psi(y/alpha) cos(k y) dy,
 * alpha = w pi / n, psi(z) = exp(beta (sqrt(1 - z^2) - 1)), for k = 0..nk-1.
 * Exposed for tests of the planner; no CUDA call.
 */
NUSHT_API int nusht_kernel_ft(int w, double beta, int n, int nk, double* out);

/*
 * nusht_good_size -- smallest n >= nmin that is a multiple of `multiple` and
 * whose prime factors are all <= maxprime (App. B "good numbers").  Host only.
 */
NUSHT_API int64_t nusht_good_size(int64_t nmin, int multiple, int maxprime);

/*
 * nusht_stage_times -- per-stage device times (ms) of the last synth and
 * adjoint calls made with opts.profile = 1: out[0..5] synth
 * (legendre, theta_fft, deconv_pad, grid_fft, interp, total),
 * out[6..11] adjoint (spread, grid_fft, deconv_trunc, theta_fft, legendre, total).
 * Synchronises the plan's last stream.
 */
NUSHT_API int nusht_stage_times(nusht_plan_t p, double* out12);

/* nusht_strerror -- static name of a status code. */
NUSHT_API const char* nusht_strerror(int code);

/* nusht_last_error -- message of this thread's most recent failure ("" if none). */
NUSHT_API const char* nusht_last_error(void);

/* nusht_version -- library version string. */
NUSHT_API const char* nusht_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NUSHT_H */
