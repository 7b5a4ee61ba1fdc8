"""Seeded synthetic inputs for the nuSHT workloads (shared by the tests, the
oracle legs and bench.py).

This module holds input generation only: random coefficients, point clouds,
Gauss-Legendre ring grids and a lensing-style deflection of those grids.  It
shares no code with the oracle or the CUDA library and neither of them
imports it; both take their inputs from here.  The one piece of spherical
harmonic arithmetic in it, ``phi_gradient_rings``, only places the deflected
grid points (the gradient of the synthetic lensing potential on the grid's
rings, a plain numpy recurrence); parity of the transform is checked on
whatever points it produces.

Workloads (Sec. 4, benchmark set-up; sizes and distributions as named in the
build's configuration list):

* ``uniform63``   lmax = mmax = 63, 20,000 points uniform on the sphere
  (theta = arccos U[-1, 1], phi ~ U[0, 2 pi)), unit-variance complex Gaussian
  a_lm (a_l0 real), seed 0.
* ``gl1023``      lmax = 1023, 1024 x 2047 Gauss-Legendre ring grid deflected
  by a 2.5 arcmin rms gradient field; a_lm with C_l ~ (l+1)^-2.
* ``gl4095``      lmax = 4095, 4096 x 8191 deflected ring grid (33,550,336
  points); a_lm with C_l ~ (l+1)^-2.
* ``gl2047``      lmax = 2047, 2048 x 4095 deflected ring grid (8,386,560 points).
* ``batch64``     64 transforms, lmax_b ~ U{256..2047}, N_b = 2 lmax_b^2
  uniform points each.

The paper's CMB simulations (Sec. 4, Fig. benchmark_setup) are not available;
the deflection here stands in for them.  It is the gradient of a Gaussian
random lensing potential Phi (``phi_lensing``: C_l ~ [l(l+1)]^-1 (1+l/60)^-3,
2 <= l <= min(512, lmax), scaled to 2.5 arcmin rms deflection), evaluated on
the grid's rings, applied with the lensing pointing relation of Appendix C:
n' = cos(a) n + sin(a)/a (a_theta e_theta + a_phi e_phi).
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

ARCMIN = np.pi / (180.0 * 60.0)


def nalm(lmax: int, mmax: int | None = None) -> int:
    mmax = lmax if mmax is None else mmax
    return (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) // 2


def alm_gaussian(lmax: int, seed: int, mmax: int | None = None, spectrum: str | None = None,
                 dtype=np.complex128) -> np.ndarray:
    """Packed m-major a_lm: Re, Im ~ N(0, 1/2) (E|a|^2 = 1), a_l0 ~ N(0, 1) real.

    ``spectrum='inv_l1_sq'`` scales every a_lm by 1/(l+1), i.e. C_l = (l+1)^-2.
    """
    mmax = lmax if mmax is None else mmax
    rng = np.random.default_rng(seed)
    n = nalm(lmax, mmax)
    re = rng.standard_normal(n) * np.sqrt(0.5)
    im = rng.standard_normal(n) * np.sqrt(0.5)
    a = re + 1j * im
    a[: lmax + 1] = rng.standard_normal(lmax + 1)  # m = 0 block: real, unit variance
    if spectrum == "inv_l1_sq":
        ells = np.concatenate([np.arange(m, lmax + 1) for m in range(mmax + 1)])
        a = a / (ells + 1.0)
    elif spectrum is not None:
        raise ValueError("unknown spectrum %r" % spectrum)
    return a.astype(dtype)


def phi_lensing(lmax: int, seed: int, rms_arcmin: float = 2.5, dtype=np.complex128) -> np.ndarray:
    """Packed m-major coefficients of a synthetic lensing potential Phi:
    Gaussian with C_l proportional to [l(l+1)]^-1 (1 + l/60)^-3 for l >= 2
    (zero for l < 2), scaled so that the rms deflection |grad Phi| over the
    sphere is rms_arcmin: sum_l (2l+1) l(l+1) C_l / (4 pi) = rms^2.  The
    stand-in for the paper's CMB lensing simulations (Sec. 4, App. C)."""
    ls = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros(lmax + 1)
    hi = ls >= 2
    cl[hi] = 1.0 / (ls[hi] * (ls[hi] + 1.0)) / (1.0 + ls[hi] / 60.0) ** 3
    var = np.sum((2.0 * ls + 1.0) * ls * (ls + 1.0) * cl) / (4.0 * np.pi)
    rms = rms_arcmin * np.pi / (180.0 * 60.0)
    if var > 0:
        cl *= rms**2 / var
    a = alm_gaussian(lmax, seed)
    ells = np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])
    return (a * np.sqrt(cl[ells])).astype(dtype)


def points_uniform(n: int, seed: int) -> np.ndarray:
    """n points uniform on the sphere: theta = arccos U[-1,1], phi ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    th = np.arccos(rng.uniform(-1.0, 1.0, n))
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    return np.ascontiguousarray(np.stack([th, ph], axis=1))


def gl_ring_grid(nrings: int, nphi: int) -> np.ndarray:
    """Gauss-Legendre ring grid: theta_r = arccos(x_r) for the nrings GL nodes,
    phi_k = 2 pi k / nphi; ring-major (theta, phi) pairs."""
    from scipy.special import roots_legendre

    x, _ = roots_legendre(nrings)
    th = np.arccos(x[::-1])  # north to south
    ph = 2.0 * np.pi * np.arange(nphi) / nphi
    out = np.empty((nrings * nphi, 2), dtype=np.float64)
    out[:, 0] = np.repeat(th, nphi)
    out[:, 1] = np.tile(ph, nrings)
    return out


def phi_gradient_rings(philm: np.ndarray, lphi: int, thetas: np.ndarray, nphi: int):
    """Gradient of the real field Phi = sum_lm philm_lm Y_lm (packed m-major,
    band limit lphi) on iso-latitude rings: returns (a_theta, a_phi), each of
    shape (len(thetas), nphi), with a_theta = dPhi/dtheta and
    a_phi = (1/sin theta) dPhi/dphi at phi_k = 2 pi k / nphi (the spin-1
    gradient of App. C, Eq. spin1deriv).  Input generation only: the
    orthonormal functions come from the textbook three-term recurrence in
    numpy, vectorised over the rings, their theta derivative from
    sin(theta) dP_lm = l cos(theta) P_lm - sqrt((2l+1)(l^2-m^2)/(2l-1)) P_{l-1,m},
    and the sum over m from a real inverse FFT per ring.  The rings must not
    touch the poles (Gauss-Legendre nodes never do)."""
    th = np.asarray(thetas, dtype=np.float64)
    x, s = np.cos(th), np.sin(th)
    nr = th.size
    A = np.zeros((nr, lphi + 1), dtype=np.complex128)  # sum_l phi_lm dP_lm/dtheta
    B = np.zeros((nr, lphi + 1), dtype=np.complex128)  # sum_l phi_lm P_lm
    pmm = np.full(nr, 1.0 / np.sqrt(4.0 * np.pi))
    base = 0
    with np.errstate(under="ignore"):
        for m in range(lphi + 1):
            if m > 0:
                pmm = -np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
            col = philm[base:base + lphi + 1 - m]
            base += lphi + 1 - m
            p2 = np.zeros(nr)
            p1 = pmm
            for l in range(m, lphi + 1):
                if l == m + 1:
                    p = np.sqrt(2.0 * m + 3.0) * x * p1
                elif l > m + 1:
                    a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                    b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                    p = a * (x * p1 - b * p2)
                else:
                    p = p1
                if l > m:
                    p2, p1 = p1, p
                    dp = (l * x * p1 - np.sqrt((2.0 * l + 1.0) * (l * l - m * m) / (2.0 * l - 1.0)) * p2) / s
                else:
                    dp = (l * x * p1) / s
                c = col[l - m]
                A[:, m] += c * dp
                B[:, m] += c * p1
    A[:, 0] = A[:, 0].real
    # real field: g(phi) = c_0 + 2 Re sum_{m>0} c_m e^{i m phi} = nphi * irfft(c)
    C = np.zeros((nr, nphi // 2 + 1), dtype=np.complex128)
    C[:, : lphi + 1] = A
    a_th = nphi * np.fft.irfft(C, n=nphi, axis=1)
    C[:] = 0.0
    C[:, : lphi + 1] = B * (1j * np.arange(lphi + 1))[None, :] / s[:, None]
    a_ph = nphi * np.fft.irfft(C, n=nphi, axis=1)
    return a_th, a_ph


def pointing_shift(th: np.ndarray, ph: np.ndarray, a_th: np.ndarray, a_ph: np.ndarray):
    """Move each point along the great circle that starts in the direction
    a_th e_theta + a_phi e_phi by the angle |a| (App. C, Eq. pointing):
    n' = cos|a| n + sin|a|/|a| (a_th e_theta + a_phi e_phi); returns
    (theta', phi') with theta' in [0, pi], phi' in [0, 2 pi)."""
    a = np.sqrt(a_th**2 + a_ph**2)
    sinc = np.where(a > 0, np.sin(a) / np.where(a > 0, a, 1.0), 1.0)
    ca = np.cos(a)
    st, ct = np.sin(th), np.cos(th)
    sp, cp = np.sin(ph), np.cos(ph)
    x = ca * st * cp + sinc * (a_th * ct * cp - a_ph * sp)
    y = ca * st * sp + sinc * (a_th * ct * sp + a_ph * cp)
    z = ca * ct + sinc * (-a_th * st)
    return np.arctan2(np.sqrt(x * x + y * y), z), np.mod(np.arctan2(y, x), 2.0 * np.pi)


LPHI_MAX = 512  # band limit of the synthetic lensing potential


def deflect_gl_grid(lmax: int, rms_arcmin: float, seed: int, chunk: int = 1 << 18) -> np.ndarray:
    """(lmax+1) x (2 lmax+1) Gauss-Legendre ring grid deflected by the
    gradient of a Gaussian lensing potential (``phi_lensing`` with band limit
    min(512, lmax), rms deflection ``rms_arcmin``), with the pointing
    relation of Appendix C."""
    nr, nphi = lmax + 1, 2 * lmax + 1
    pts = gl_ring_grid(nr, nphi)
    lphi = min(LPHI_MAX, lmax)
    phi = phi_lensing(lphi, seed, rms_arcmin)
    a_th, a_ph = phi_gradient_rings(phi, lphi, pts[::nphi, 0], nphi)
    a_th = a_th.reshape(-1)
    a_ph = a_ph.reshape(-1)
    out = np.empty_like(pts)

    def one(s0):
        sl = slice(s0, s0 + chunk)
        out[sl, 0], out[sl, 1] = pointing_shift(pts[sl, 0], pts[sl, 1], a_th[sl], a_ph[sl])

    # numpy ufuncs release the GIL, so chunks run in parallel threads; every
    # chunk is a pure function of its own points, so the result is the same
    # for any thread count.
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(one, range(0, pts.shape[0], chunk)))
    return out


def _cache_dir() -> str:
    d = os.environ.get("NUSHT_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "nusht_workloads"))
    os.makedirs(d, exist_ok=True)
    return d


def _cached(key: str, make):
    path = os.path.join(_cache_dir(), hashlib.sha1(key.encode()).hexdigest()[:16] + ".npy")
    if os.path.exists(path):
        try:
            return np.load(path)
        except Exception:
            pass
    arr = make()
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "wb") as fh:
        np.save(fh, arr)
    os.replace(tmp, path)
    return arr


def deflected_gl_grid(lmax: int, seed: int = 1, rms_arcmin: float = 2.5, cache: bool = True) -> np.ndarray:
    """(lmax+1) x (2 lmax+1) Gauss-Legendre ring grid deflected by ``rms_arcmin``."""
    def make():
        return deflect_gl_grid(lmax, rms_arcmin, seed)

    if not cache:
        return make()
    return _cached("glgrid-v2-%d-%d-%r" % (lmax, seed, rms_arcmin), make)


def subset(n: int, k: int, seed: int = 12345) -> np.ndarray:
    """Sorted seeded sample of k of n indices without replacement (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(n, k), replace=False))


WORKLOADS = {
    "uniform63": dict(lmax=63, npts=20000),
    "gl1023": dict(lmax=1023, npts=1024 * 2047),
    "gl2047": dict(lmax=2047, npts=2048 * 4095),
    "gl4095": dict(lmax=4095, npts=4096 * 8191),
}


def workload(name: str, dtype=np.complex128):
    """(lmax, alm, pts) of a named single-transform workload."""
    if name == "uniform63":
        return 63, alm_gaussian(63, seed=0, dtype=dtype), points_uniform(20000, seed=0)
    if name in ("gl1023", "gl2047", "gl4095"):
        lmax = int(name[2:])
        return lmax, alm_gaussian(lmax, seed=0, spectrum="inv_l1_sq", dtype=dtype), deflected_gl_grid(lmax)
    raise KeyError(name)


def batch64(seed: int = 0, nbatch: int = 64, lmin: int = 256, lmax: int = 2047):
    """lmax_b ~ U{lmin..lmax}; each transform has 2 lmax_b^2 uniform points."""
    rng = np.random.default_rng(seed)
    ls = rng.integers(lmin, lmax + 1, size=nbatch)
    out = []
    for b, lb in enumerate(ls):
        lb = int(lb)
        out.append((lb, alm_gaussian(lb, seed=1000 + b, dtype=np.complex64),
                    points_uniform(2 * lb * lb, seed=2000 + b)))
    return out
