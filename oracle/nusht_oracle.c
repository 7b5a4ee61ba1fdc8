/*
 * nusht_oracle.c -- CPU oracle for the nonuniform spin-0 spherical harmonic
 * transform (cuNUSHT, arXiv 2406.14542).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, direct-summation
 * definition of the transform.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may build, load or call it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (Sec. 2.1):
 *   Y_l^m(theta, phi) = P_l^m(theta) e^{i m phi}                        (Eq. Ylm)
 *   P_l^m(theta)      = d^l_{m0}(theta) sqrt((2l+1)/(4 pi))   (footnote of Sec. 2.2)
 *     i.e. the orthonormal associated Legendre function including the
 *     Condon-Shortley phase (-1)^m, so Y_1^1 = -sqrt(3/(8 pi)) sin(theta) e^{i phi}.
 *   type 2:  f_i    = sum_{l<=L} sum_{|m|<=l} c_lm Y_l^m(theta_i, phi_i)  (Eq. SHTbase)
 *   type 1:  c_lm   = sum_i f_i  conj(Y_l^m(theta_i, phi_i))       (Eq. adjointSHTbase)
 *
 * Real-field storage: only m >= 0 is stored; c_{l,-m} = (-1)^m conj(c_lm), so
 *   f_i = sum_l [ Re(c_l0) Pbar_l0 + 2 Re sum_{1<=m<=min(l,mmax)} c_lm Pbar_lm e^{i m phi} ]
 * and the adjoint of that real-linear map under
 *   <c, a> = sum_l Re(conj(c_l0) a_l0) + 2 sum_{l, m>0} Re(conj(c_lm) a_lm)
 * is exactly c_lm = sum_i f_i Pbar_lm(theta_i) e^{-i m phi_i} (Sec. 2.1: type 1 is
 * the adjoint Y^dagger = (Y^t)^*, not the inverse).
 *
 * Packed layout ("m-major"): index(l, m) = m (2L + 1 - m) / 2 + l, 0 <= m <= mmax,
 * m <= l <= L; complex numbers as interleaved (re, im) doubles.
 *
 * Pbar_lm is computed by the textbook normalised three-term recurrence in
 * double precision:
 *   Pbar_00 = 1/sqrt(4 pi)
 *   Pbar_mm = -sqrt((2m+1)/(2m)) sin(theta) Pbar_{m-1,m-1}
 *   Pbar_{m+1,m} = sqrt(2m+3) cos(theta) Pbar_mm
 *   Pbar_lm = a_lm (cos(theta) Pbar_{l-1,m} - b_lm Pbar_{l-2,m}),
 *     a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
 * The product cos(theta) * P is formed as P - u P with u = 2 sin^2(theta/2)
 * when cos(theta) >= 0, and as v P - P with v = 2 cos^2(theta/2) otherwise
 * (the same number in exact arithmetic).  Near the poles cos(theta) rounded
 * to double loses the information that distinguishes theta, and the textbook
 * form then evaluates P_l at a shifted angle (relative error ~ l^2 ulp); u and
 * v keep full relative precision there.
 * Underflow of sin^m(theta) at large m is handled by carrying a separate
 * integer binary exponent beside each mantissa (value = p * 2^e), renormalised
 * with frexp/ldexp; values are formed with ldexp only when accumulated.
 * e^{i m phi} is evaluated directly as cos(m phi), sin(m phi) for every m.
 * theta and phi may be any finite reals: sin(theta) keeps its sign, which is
 * the analytic continuation of Pbar_lm and names the same point on the sphere.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* index of (l, m) in the packed m-major layout */
static int64_t lm_index(int L, int l, int m) {
  return (int64_t)m * (2 * L + 1 - m) / 2 + l;
}

int64_t oracle_nalm(int L, int mmax) {
  return (int64_t)(mmax + 1) * (L + 1) - (int64_t)mmax * (mmax + 1) / 2;
}

/* A number value = p * 2^e, the exponent kept outside the double. */
typedef struct {
  double p;
  int e;
} xnum;

static xnum xnorm(double p, int e) {
  xnum r;
  if (p == 0.0) {
    r.p = 0.0;
    r.e = 0;
    return r;
  }
  int k;
  r.p = frexp(p, &k);
  r.e = e + k;
  return r;
}

/*
 * Pbar_mm for one theta, advancing from Pbar_{m-1,m-1}: the caller keeps the
 * running value across m = 0, 1, 2, ...
 */
static xnum pmm_next(xnum prev, int m, double s) {
  if (m == 0) return xnorm(1.0 / sqrt(4.0 * M_PI), 0);
  return xnorm(-sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * prev.p, prev.e);
}

/*
 * Column of Pbar_lm(theta) for l = m..L into out[0..L-m], starting from
 * Pbar_mm = pmm.  The pair (Pbar_{l-1,m}, Pbar_{l-2,m}) shares one exponent e.
 * While e < 0 both mantissas are renormalised after every step (never beyond
 * e = 0); with e >= 0 the values are ordinary doubles bounded by
 * sqrt((2l+1)/(4 pi)) and need no scaling.
 */
static void plm_column(int L, int m, const double* tc, xnum pmm, double* out) {
  /* tc = {north, u_or_v}: north != 0 means cos(theta) = 1 - u, else -(1 - v) */
  const int north = tc[0] != 0.0;
  const double w = tc[1];
  double p1 = pmm.p, p2 = 0.0;
  int e = pmm.e;
  if (e > 0) { /* |Pbar_mm| <= O(1): fold the exponent into the mantissa */
    p1 = ldexp(p1, e);
    e = 0;
  }
  out[0] = ldexp(p1, e);
  for (int l = m + 1; l <= L; ++l) {
    double xp1 = north ? (p1 - w * p1) : (w * p1 - p1); /* cos(theta) * p1 */
    double p;
    if (l == m + 1) {
      p = sqrt(2.0 * m + 3.0) * xp1;
    } else {
      double dl = (double)l, dm = (double)m;
      double a = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
      double b = sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) / (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
      p = a * (xp1 - b * p2);
    }
    p2 = p1;
    p1 = p;
    if (e < 0 && p1 != 0.0) {
      int k;
      frexp(p1, &k);
      int shift = k;
      if (e + shift > 0) shift = -e;
      p1 = ldexp(p1, -shift);
      p2 = ldexp(p2, -shift);
      e += shift;
    }
    out[l - m] = ldexp(p1, e);
  }
}

/* cos(theta) in the form used by plm_column: {north flag, u or v} */
static void theta_cos(double theta, double* tc) {
  double c = cos(theta);
  if (c >= 0.0) {
    double h = sin(0.5 * theta);
    tc[0] = 1.0;
    tc[1] = 2.0 * h * h; /* u = 1 - cos(theta) */
  } else {
    double h = cos(0.5 * theta);
    tc[0] = 0.0;
    tc[1] = 2.0 * h * h; /* v = 1 + cos(theta) */
  }
}

/*
 * All Pbar_lm(theta) for 0 <= m <= mmax, m <= l <= L, in packed layout
 * (real values, one per (l,m)).  Used by the pins (closed forms, addition
 * theorem, quadrature orthogonality, library comparisons).
 */
void oracle_plm_all(int L, int mmax, double theta, double* out) {
  double tc[2], s = sin(theta);
  theta_cos(theta, tc);
  xnum pmm = {0.0, 0};
  for (int m = 0; m <= mmax; ++m) {
    pmm = pmm_next(pmm, m, s);
    plm_column(L, m, tc, pmm, out + lm_index(L, m, m));
  }
}

/*
 * Type 2 (Eq. SHTbase), real field: f[i] for npts points pts = (theta, phi)
 * interleaved.  alm: packed complex (re, im), Im(a_l0) ignored.
 */
void oracle_synth(int L, int mmax, const double* alm, int64_t npts, const double* pts, double* f) {
#pragma omp parallel
  {
    double* col = (double*)malloc(sizeof(double) * (size_t)(L + 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < npts; ++i) {
      double th = pts[2 * i], ph = pts[2 * i + 1];
      double tc[2], s = sin(th);
      theta_cos(th, tc);
      xnum pmm = {0.0, 0};
      double acc = 0.0;
      for (int m = 0; m <= mmax; ++m) {
        pmm = pmm_next(pmm, m, s);
        plm_column(L, m, tc, pmm, col);
        double sr = 0.0, si = 0.0;
        for (int l = m; l <= L; ++l) {
          const double* a = alm + 2 * lm_index(L, l, m);
          sr += a[0] * col[l - m];
          si += a[1] * col[l - m];
        }
        if (m == 0) {
          acc += sr;
        } else {
          double c = cos((double)m * ph), sn = sin((double)m * ph);
          acc += 2.0 * (sr * c - si * sn);
        }
      }
      f[i] = acc;
    }
    free(col);
  }
}

/*
 * Ring sums of the Legendre step: for each m <= mmax and each theta_j,
 * F[m][j] = sum_{l=m}^{L} a_lm Pbar_lm(theta_j), complex (re, im) with
 * Im(a_l0) ignored.  This is the definition of what the iso-latitude step S
 * produces before any phi transform (Sec. 2.2 and Sec. 3 on the phi-FFT that
 * S and F share).  out has (mmax+1) * nth complex entries, theta fastest.
 */
void oracle_ring_sums(int L, int mmax, const double* alm, int nth, const double* thetas, double* out) {
#pragma omp parallel
  {
    double* col = (double*)malloc(sizeof(double) * (size_t)(L + 1));
#pragma omp for schedule(dynamic, 4)
    for (int j = 0; j < nth; ++j) {
      double tc[2], s = sin(thetas[j]);
      theta_cos(thetas[j], tc);
      xnum pmm = {0.0, 0};
      for (int m = 0; m <= mmax; ++m) {
        pmm = pmm_next(pmm, m, s);
        plm_column(L, m, tc, pmm, col);
        double sr = 0.0, si = 0.0;
        for (int l = m; l <= L; ++l) {
          const double* a = alm + 2 * lm_index(L, l, m);
          sr += a[0] * col[l - m];
          if (m > 0) si += a[1] * col[l - m];
        }
        out[2 * ((int64_t)m * nth + j)] = sr;
        out[2 * ((int64_t)m * nth + j) + 1] = si;
      }
    }
    free(col);
  }
}

/*
 * Type 1 (Eq. adjointSHTbase) restricted to a list of orders: for each m in
 * mlist[0..nm-1] and every l in [m, L], c_lm = sum_i f_i Pbar_lm(theta_i)
 * e^{-i m phi_i}.  out: packed complex array of the full size; entries of
 * orders not in mlist are left untouched.  Pass all orders for the full
 * adjoint.  Summation: per thread partial sums over a static block of points,
 * then added in thread order.
 */
void oracle_adjoint_m(int L, int mmax, int64_t npts, const double* pts, const double* f, int nm, const int* mlist,
                      double* out) {
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  /* per-thread accumulators over the requested orders only */
  int64_t span = 0;
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nm + 1));
  for (int q = 0; q < nm; ++q) {
    off[q] = span;
    span += (L - mlist[q] + 1);
  }
  off[nm] = span;
  double* part = (double*)calloc((size_t)nthreads * (size_t)span * 2, sizeof(double));
#pragma omp parallel num_threads(nthreads)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double* acc = part + (size_t)t * (size_t)span * 2;
    double* col = (double*)malloc(sizeof(double) * (size_t)(L + 1));
#pragma omp for schedule(static)
    for (int64_t i = 0; i < npts; ++i) {
      double th = pts[2 * i], ph = pts[2 * i + 1];
      double tc[2], s = sin(th);
      theta_cos(th, tc);
      xnum pmm = {0.0, 0};
      /* Pbar_mm is advanced through every m up to the largest requested;
         mlist must be strictly increasing */
      int q = 0;
      for (int m = 0; m <= mmax && q < nm; ++m) {
        pmm = pmm_next(pmm, m, s);
        if (m != mlist[q]) continue;
        plm_column(L, m, tc, pmm, col);
        double c = cos((double)m * ph), sn = sin((double)m * ph);
        double fr = f[i] * c, fi = -f[i] * sn;
        double* a = acc + 2 * off[q];
        for (int l = m; l <= L; ++l) {
          a[2 * (l - m)] += fr * col[l - m];
          a[2 * (l - m) + 1] += fi * col[l - m];
        }
        ++q;
      }
    }
    free(col);
  }
  for (int q = 0; q < nm; ++q) {
    int m = mlist[q];
    for (int l = m; l <= L; ++l) {
      double sr = 0.0, si = 0.0;
      for (int t = 0; t < nthreads; ++t) {
        sr += part[((size_t)t * span + off[q] + (l - m)) * 2];
        si += part[((size_t)t * span + off[q] + (l - m)) * 2 + 1];
      }
      out[2 * lm_index(L, l, m)] = sr;
      out[2 * lm_index(L, l, m) + 1] = si;
    }
  }
  free(part);
  free(off);
}

/*
 * Analytic gradient of the real-field type 2 sum with respect to the point
 * coordinates: dtheta[i] = d f_i / d theta_i, dphi[i] = d f_i / d phi_i.
 *   d/dphi brings i m:   d f/d phi = sum_l 2 Re sum_{m>0} i m c_lm Pbar_lm e^{i m phi}
 *   d/dtheta uses the ladder relation (orthonormal, Condon-Shortley phase)
 *     dPbar_lm/dtheta = ( sqrt((l-m)(l+m+1)) Pbar_{l,m+1}
 *                       - sqrt((l+m)(l-m+1)) Pbar_{l,m-1} ) / 2,
 *   with Pbar_{l,-1} = -Pbar_{l,1} and Pbar_{l,m} = 0 for m > l.  This form
 *   has no 1/sin(theta) and is finite at the poles.
 * Columns m-1, m, m+1 are computed for every m (order mmax+1 is used for the
 * derivative of order mmax, so columns run to min(mmax+1, L)).
 */
void oracle_synth_grad(int L, int mmax, const double* alm, int64_t npts, const double* pts, double* dtheta,
                       double* dphi) {
#pragma omp parallel
  {
    double* cm = (double*)malloc(sizeof(double) * (size_t)(L + 2));
    double* cp = (double*)malloc(sizeof(double) * (size_t)(L + 2));
    double* cn = (double*)malloc(sizeof(double) * (size_t)(L + 2));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < npts; ++i) {
      double th = pts[2 * i], ph = pts[2 * i + 1];
      double tc[2], s = sin(th);
      theta_cos(th, tc);
      /* cm: column m-1 (indexed by l directly), cp: column m, cn: column m+1 */
      xnum pmm = {0.0, 0};
      pmm = pmm_next(pmm, 0, s);
      for (int l = 0; l <= L + 1; ++l) cm[l] = cp[l] = cn[l] = 0.0;
      plm_column(L, 0, tc, pmm, cp); /* cp[l] = Pbar_l0, l = 0..L */
      xnum pnext = pmm_next(pmm, 1, s);
      if (L >= 1) {
        plm_column(L, 1, tc, pnext, cn + 1); /* cn[l] = Pbar_l1 */
      }
      double gth = 0.0, gph = 0.0;
      for (int m = 0; m <= mmax; ++m) {
        /* column m-1: for m = 0 it is -Pbar_{l,1} */
        double sr = 0.0, si = 0.0, dr = 0.0, di = 0.0;
        for (int l = m; l <= L; ++l) {
          double lo = (m == 0) ? -cn[l] : cm[l];
          double hi = (m + 1 <= l) ? cn[l] : 0.0;
          double dl = (double)l, dm = (double)m;
          double dP = 0.5 * (sqrt((dl - dm) * (dl + dm + 1.0)) * hi - sqrt((dl + dm) * (dl - dm + 1.0)) * lo);
          const double* a = alm + 2 * lm_index(L, l, m);
          double ai = (m == 0) ? 0.0 : a[1];
          sr += a[0] * cp[l];
          si += ai * cp[l];
          dr += a[0] * dP;
          di += ai * dP;
        }
        if (m == 0) {
          gth += dr;
        } else {
          double c = cos((double)m * ph), sn = sin((double)m * ph);
          gth += 2.0 * (dr * c - di * sn);
          /* d/dphi Re[(sr + i si)(c + i sn)] = m Re[i (sr + i si)(c + i sn)] = -m (sr sn + si c) */
          gph += -2.0 * (double)m * (sr * sn + si * c);
        }
        /* shift columns: m-1 <- m, m <- m+1, m+1 <- m+2 */
        double* tmp = cm;
        cm = cp;
        cp = cn;
        cn = tmp;
        for (int l = 0; l <= L + 1; ++l) cn[l] = 0.0;
        if (m + 2 <= L) {
          pnext = pmm_next(pnext, m + 2, s);
          plm_column(L, m + 2, tc, pnext, cn + (m + 2));
        }
      }
      dtheta[i] = gth;
      dphi[i] = gph;
    }
    free(cm);
    free(cp);
    free(cn);
  }
}

/*
 * CMB lensing pointing (App. C): the deflected position of each point.
 *   alpha_theta + i alpha_phi = (d/dtheta + (i / sin theta) d/dphi) Phi    (Eq. spin1deriv)
 *   n' = cos(alpha) n + (sin(alpha) / alpha) (alpha_theta e_theta + alpha_phi e_phi),
 *   alpha = sqrt(alpha_theta^2 + alpha_phi^2)                             (Eq. pointing)
 * with n = (sin t cos p, sin t sin p, cos t), e_theta = (cos t cos p, cos t sin p,
 * -sin t), e_phi = (-sin p, cos p, 0).  The derivatives of the potential Phi
 * (real field, packed coefficients philm) are the analytic ones of
 * oracle_synth_grad.  At a point with sin(theta) = 0 alpha_phi is taken as 0.
 * Output: out[2i] = theta' in [0, pi], out[2i + 1] = phi' in [0, 2 pi).
 */
void oracle_pointing(int L, int mmax, const double* philm, int64_t npts, const double* pts, double* out) {
  double* dth = (double*)malloc(sizeof(double) * (size_t)(npts > 0 ? npts : 1));
  double* dph = (double*)malloc(sizeof(double) * (size_t)(npts > 0 ? npts : 1));
  oracle_synth_grad(L, mmax, philm, npts, pts, dth, dph);
  const double twopi = 2.0 * M_PI;
  for (int64_t i = 0; i < npts; ++i) {
    const double t = pts[2 * i], ph = pts[2 * i + 1];
    const double st = sin(t), ct = cos(t), sp = sin(ph), cp = cos(ph);
    const double n[3] = {st * cp, st * sp, ct};
    const double et[3] = {ct * cp, ct * sp, -st};
    const double ep[3] = {-sp, cp, 0.0};
    const double at = dth[i];
    const double ap = (st != 0.0) ? dph[i] / st : 0.0;
    const double a = sqrt(at * at + ap * ap);
    const double sinc = (a > 0.0) ? sin(a) / a : 1.0;
    const double ca = cos(a);
    double q[3];
    for (int k = 0; k < 3; ++k) q[k] = ca * n[k] + sinc * (at * et[k] + ap * ep[k]);
    const double tp = atan2(sqrt(q[0] * q[0] + q[1] * q[1]), q[2]);
    double pp = atan2(q[1], q[0]);
    if (pp < 0.0) pp += twopi;
    if (pp >= twopi) pp -= twopi;
    out[2 * i] = tp;
    out[2 * i + 1] = pp;
  }
  free(dth);
  free(dph);
}

/*
 * Spin-weighted harmonics (the spin-n generalisation named in the Conclusion,
 * Sec. 5; the paper gives no formulas, so these are the standard ones).  For spin s >= 0 and m >= 0 (negative orders follow from the
 * reality conditions below):
 *   sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi},
 * with d^l the Wigner small-d matrix.  For s = 0 this is Y_lm of the spin-0
 * transform (Condon-Shortley phase), and 1Y_lm = (eth Y_lm) / sqrt(l(l+1))
 * with eth = -(d/dtheta + (i / sin theta) d/dphi) on spin 0.
 * lambda^(+s)_lm(theta) = sY_lm(theta, 0) uses d^l_{m,-s};
 * lambda^(-s)_lm(theta) = (-s)Y_lm(theta, 0) uses d^l_{m,s}.
 *
 * d^l_{m,mp} for fixed (m, mp) from the three-term recurrence in l
 *   (l-1) sqrt(l^2-m^2) sqrt(l^2-mp^2) d^l
 *     = (2l-1) (l(l-1) cos(theta) - m mp) d^{l-1}
 *       - l sqrt((l-1)^2-m^2) sqrt((l-1)^2-mp^2) d^{l-2},
 * started at l0 = max(|m|, |mp|) from the closed forms
 *   d^l_{l,mp}  = (-1)^{l-mp} sqrt(C(2l, l+mp)) cos^{l+mp}(theta/2) sin^{l-mp}(theta/2),
 *   d^l_{m,l}   = sqrt(C(2l, l+m)) cos^{l+m}(theta/2) sin^{l-m}(theta/2),
 *   d^l_{m,-l}  = (-1)^{l+m} sqrt(C(2l, l-m)) cos^{l-m}(theta/2) sin^{l+m}(theta/2).
 * The start value and the pair (d^{l-1}, d^{l-2}) carry a separate binary
 * exponent, as for the spin-0 columns.  The values are normalised by
 * sqrt((2l+1)/(4 pi)) and multiplied by (-1)^s.
 */
/* value = p * 2^e of sqrt(C(2l, k)) cos^a(theta/2) sin^b(theta/2) */
static xnum spin_start(int l, int k, int a, int b, double ch, double sh) {
  xnum r = xnorm(1.0, 0);
  /* C(2l, k) = prod_{i=1}^{k} (2l - k + i) / i, accumulated with exponents */
  for (int i = 1; i <= k; ++i) r = xnorm(r.p * ((double)(2 * l - k + i) / (double)i), r.e);
  /* square root of p * 2^e: make e even first */
  if (r.e & 1) {
    r.p *= 2.0;
    r.e -= 1;
  }
  r = xnorm(sqrt(r.p), r.e / 2);
  for (int i = 0; i < a; ++i) r = xnorm(r.p * ch, r.e);
  for (int i = 0; i < b; ++i) r = xnorm(r.p * sh, r.e);
  return r;
}

/* sqrt((2l+1)/(4 pi)) d^l_{m,mp}(theta) for l = l0..L into out[l - l0] (l0 = max(m, |mp|), m >= 0) */
static void spin_column(int L, int m, int mp, double theta, double* out) {
  const int amp = mp < 0 ? -mp : mp;
  const int l0 = m > amp ? m : amp;
  if (l0 > L) return;
  const double ch = cos(0.5 * theta), sh = sin(0.5 * theta);
  xnum st;
  if (m >= amp) { /* d^{l0}_{l0, mp} */
    st = spin_start(l0, l0 + mp, l0 + mp, l0 - mp, ch, sh);
    if ((l0 - mp) & 1) st.p = -st.p;
  } else if (mp > 0) { /* d^{l0}_{m, l0} */
    st = spin_start(l0, l0 + m, l0 + m, l0 - m, ch, sh);
  } else { /* d^{l0}_{m, -l0} */
    st = spin_start(l0, l0 - m, l0 - m, l0 + m, ch, sh);
    if ((l0 + m) & 1) st.p = -st.p;
  }
  /* cos(theta) as 1 - 2 sin^2(theta/2) or 2 cos^2(theta/2) - 1 (as for spin 0) */
  double tc[2];
  theta_cos(theta, tc);
  const int north = tc[0] != 0.0;
  const double w = tc[1];
  double p1 = st.p, p2 = 0.0;
  int e = st.e;
  if (e > 0) {
    p1 = ldexp(p1, e);
    e = 0;
  }
  const double dm = (double)m, dmp = (double)mp;
  out[0] = ldexp(p1, e) * sqrt((2.0 * l0 + 1.0) / (4.0 * M_PI));
  for (int l = l0 + 1; l <= L; ++l) {
    const double dl = (double)l;
    const double xp1 = north ? (p1 - w * p1) : (w * p1 - p1); /* cos(theta) p1 */
    double p;
    if (l0 == 0 && l == 1) { /* m = mp = 0: the recurrence degenerates; d^1_00 = cos(theta) */
      p = xp1;
    } else {
      const double den = (dl - 1.0) * sqrt((dl * dl - dm * dm) * (dl * dl - dmp * dmp));
      p = (2.0 * dl - 1.0) * (dl * (dl - 1.0) * xp1 - dm * dmp * p1);
      if (l - 2 >= l0)
        p -= dl * sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) * ((dl - 1.0) * (dl - 1.0) - dmp * dmp)) * p2;
      p /= den;
    }
    p2 = p1;
    p1 = p;
    if (e < 0 && p1 != 0.0) {
      int k;
      frexp(p1, &k);
      int shift = k;
      if (e + shift > 0) shift = -e;
      p1 = ldexp(p1, -shift);
      p2 = ldexp(p2, -shift);
      e += shift;
    }
    out[l - l0] = ldexp(p1, e) * sqrt((2.0 * dl + 1.0) / (4.0 * M_PI));
  }
}

/*
 * lambda^(+s)_lm and lambda^(-s)_lm at theta for 0 <= m <= mmax, max(m, s) <= l <= L,
 * in the packed layout (entries with l < s are 0).
 */
void oracle_spin_lambda(int L, int mmax, int s, double theta, double* lp, double* lm) {
  const double sg = (s & 1) ? -1.0 : 1.0;
  double* col = (double*)malloc(sizeof(double) * (size_t)(L + 1));
  for (int m = 0; m <= mmax; ++m) {
    const int l0 = m > s ? m : s;
    for (int l = m; l <= L; ++l) lp[lm_index(L, l, m)] = lm[lm_index(L, l, m)] = 0.0;
    if (l0 > L) continue;
    spin_column(L, m, -s, theta, col);
    for (int l = l0; l <= L; ++l) lp[lm_index(L, l, m)] = sg * col[l - l0];
    spin_column(L, m, s, theta, col);
    for (int l = l0; l <= L; ++l) lm[lm_index(L, l, m)] = sg * col[l - l0];
  }
  free(col);
}

/*
 * Spin-s synthesis of two real fields:
 *   Q + i U = sum_{l >= s} sum_{|m| <= l} (G_lm + i C_lm) sY_lm,
 * G and C real-field coefficients (G_{l,-m} = (-1)^m conj(G_lm), same for C),
 * stored for m >= 0 in the packed layout (entries with l < s ignored,
 * Im of the m = 0 entries ignored).  With W = (lambda^(+s) + (-1)^s lambda^(-s)) / 2
 * and X = (lambda^(+s) - (-1)^s lambda^(-s)) / 2 this is
 *   Q = sum_l [ F_0 + 2 Re sum_{m>0} F_m e^{i m phi} ],  F_m = sum_l (G_lm W_lm + i C_lm X_lm),
 *   U = the same with F_m = sum_l (C_lm W_lm - i G_lm X_lm).
 */
void oracle_spin_synth(int L, int mmax, int s, const double* glm, const double* clm, int64_t npts,
                       const double* pts, double* q, double* u) {
  const double sg = (s & 1) ? -1.0 : 1.0;
#pragma omp parallel
  {
    double* cp = (double*)malloc(sizeof(double) * (size_t)(L + 1));
    double* cn = (double*)malloc(sizeof(double) * (size_t)(L + 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < npts; ++i) {
      const double th = pts[2 * i], ph = pts[2 * i + 1];
      double aq = 0.0, au = 0.0;
      for (int m = 0; m <= mmax; ++m) {
        const int l0 = m > s ? m : s;
        if (l0 > L) break;
        spin_column(L, m, -s, th, cp);
        spin_column(L, m, s, th, cn);
        double qr = 0.0, qi = 0.0, ur = 0.0, ui = 0.0;
        for (int l = l0; l <= L; ++l) {
          const double lpv = sg * cp[l - l0], lmv = sg * cn[l - l0];
          const double W = 0.5 * (lpv + sg * lmv), X = 0.5 * (lpv - sg * lmv);
          const double* g = glm + 2 * lm_index(L, l, m);
          const double* c = clm + 2 * lm_index(L, l, m);
          const double gi = (m == 0) ? 0.0 : g[1], ci = (m == 0) ? 0.0 : c[1];
          /* G W + i C X */
          qr += g[0] * W - ci * X;
          qi += gi * W + c[0] * X;
          /* C W - i G X */
          ur += c[0] * W + gi * X;
          ui += ci * W - g[0] * X;
        }
        if (m == 0) {
          aq += qr;
          au += ur;
        } else {
          const double cs = cos((double)m * ph), sn = sin((double)m * ph);
          aq += 2.0 * (qr * cs - qi * sn);
          au += 2.0 * (ur * cs - ui * sn);
        }
      }
      q[i] = aq;
      u[i] = au;
    }
    free(cp);
    free(cn);
  }
}

/*
 * Spin-s adjoint (type 1): the transpose of oracle_spin_synth under the
 * real inner product sum_l Re(.)_l0 + 2 sum_{l, m>0} Re(conj(.) .) applied to
 * both G and C:
 *   G_lm = sum_i (q_i W_lm + i u_i X_lm) e^{-i m phi_i},
 *   C_lm = sum_i (u_i W_lm - i q_i X_lm) e^{-i m phi_i},
 * for the orders in mlist (strictly increasing); entries with l < s are 0.
 */
void oracle_spin_adjoint_m(int L, int mmax, int s, int64_t npts, const double* pts, const double* q,
                           const double* u, int nm, const int* mlist, double* outg, double* outc) {
  const double sg = (s & 1) ? -1.0 : 1.0;
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  int64_t span = 0;
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nm + 1));
  for (int k = 0; k < nm; ++k) {
    off[k] = span;
    span += (L - mlist[k] + 1);
  }
  off[nm] = span;
  /* per thread: G (re, im), C (re, im) per entry */
  double* part = (double*)calloc((size_t)nthreads * (size_t)span * 4, sizeof(double));
#pragma omp parallel num_threads(nthreads)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double* acc = part + (size_t)t * (size_t)span * 4;
    double* cp = (double*)malloc(sizeof(double) * (size_t)(L + 1));
    double* cn = (double*)malloc(sizeof(double) * (size_t)(L + 1));
#pragma omp for schedule(static)
    for (int64_t i = 0; i < npts; ++i) {
      const double th = pts[2 * i], ph = pts[2 * i + 1];
      for (int k = 0; k < nm; ++k) {
        const int m = mlist[k];
        const int l0 = m > s ? m : s;
        if (l0 > L) continue;
        spin_column(L, m, -s, th, cp);
        spin_column(L, m, s, th, cn);
        const double cs = cos((double)m * ph), sn = -sin((double)m * ph); /* e^{-i m phi} */
        for (int l = l0; l <= L; ++l) {
          const double lpv = sg * cp[l - l0], lmv = sg * cn[l - l0];
          const double W = 0.5 * (lpv + sg * lmv), X = 0.5 * (lpv - sg * lmv);
          /* (q W + i u X)(cs + i sn) and (u W - i q X)(cs + i sn) */
          const double gr = q[i] * W, gi = u[i] * X;
          const double cr = u[i] * W, ci = -q[i] * X;
          double* a = acc + 4 * (off[k] + (l - m));
          a[0] += gr * cs - gi * sn;
          a[1] += gr * sn + gi * cs;
          a[2] += cr * cs - ci * sn;
          a[3] += cr * sn + ci * cs;
        }
      }
    }
    free(cp);
    free(cn);
  }
  for (int k = 0; k < nm; ++k) {
    const int m = mlist[k];
    for (int l = m; l <= L; ++l) {
      double v[4] = {0.0, 0.0, 0.0, 0.0};
      for (int t = 0; t < nthreads; ++t)
        for (int c = 0; c < 4; ++c) v[c] += part[((size_t)t * span + off[k] + (l - m)) * 4 + c];
      if (m == 0) v[1] = v[3] = 0.0;
      outg[2 * lm_index(L, l, m)] = v[0];
      outg[2 * lm_index(L, l, m) + 1] = v[1];
      outc[2 * lm_index(L, l, m)] = v[2];
      outc[2 * lm_index(L, l, m) + 1] = v[3];
    }
  }
  free(part);
  free(off);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
