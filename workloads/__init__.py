"""Seeded synthetic inputs for the nuSHT workloads (shared by the tests, the
oracle legs and bench.py).

This module holds input generation only: random coefficients, point clouds,
Gauss-Legendre ring grids and a lensing-style deflection of those grids.  It
contains none of the transform's arithmetic (no Legendre functions, no FFTs,
no spreading kernels), so that the oracle and the CUDA library can both take
their inputs from here without sharing any of the method.

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
the deflection here stands in for them.  It is the tangential gradient of a
random potential Phi(n) = sum_q A_q cos(k_q . n + phase_q) (a sum of random 3D
plane waves restricted to the unit sphere, |k_q| ~ U[kmin, kmax]), rescaled
so that the rms deflection over a fixed sample of grid points is exactly the
requested value, and applied with the lensing pointing relation of Appendix C:
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


class _Waves:
    """Random plane waves of the deflection potential."""

    def __init__(self, seed: int, nwaves: int, kmin: float, kmax: float):
        rng = np.random.default_rng(seed)
        d = rng.standard_normal((nwaves, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        kmag = rng.uniform(kmin, kmax, nwaves)
        self.k = d * kmag[:, None]
        self.amp = rng.standard_normal(nwaves) / kmag  # equal power per wave in the gradient
        self.phase = rng.uniform(0.0, 2.0 * np.pi, nwaves)

    def gradient(self, th: np.ndarray, ph: np.ndarray):
        """(a_theta, a_phi): 3D gradient of Phi projected on e_theta, e_phi."""
        st, ct = np.sin(th), np.cos(th)
        sp, cp = np.sin(ph), np.cos(ph)
        nx, ny, nz = st * cp, st * sp, ct
        gx = np.zeros_like(th)
        gy = np.zeros_like(th)
        gz = np.zeros_like(th)
        for q in range(self.k.shape[0]):
            kx, ky, kz = self.k[q]
            s = -self.amp[q] * np.sin(kx * nx + ky * ny + kz * nz + self.phase[q])
            gx += s * kx
            gy += s * ky
            gz += s * kz
        a_th = gx * ct * cp + gy * ct * sp - gz * st
        a_ph = -gx * sp + gy * cp
        return a_th, a_ph


def deflect(pts: np.ndarray, rms_arcmin: float, seed: int, nwaves: int = 24, kmin: float = 20.0,
            kmax: float = 400.0, chunk: int = 1 << 18) -> np.ndarray:
    """Displace points by the gradient deflection of a random potential with the
    pointing relation of Appendix C; the rms deflection is ``rms_arcmin``."""
    waves = _Waves(seed, nwaves, kmin, kmax)
    n = pts.shape[0]
    # scale: rms |a| over a fixed sample of the input points
    rng = np.random.default_rng(seed + 7919)
    sel = rng.choice(n, size=min(n, 20000), replace=False)
    a_th, a_ph = waves.gradient(pts[sel, 0], pts[sel, 1])
    scale = rms_arcmin * ARCMIN / np.sqrt(np.mean(a_th**2 + a_ph**2))
    out = np.empty_like(pts)

    def one(s0):
        th = pts[s0:s0 + chunk, 0]
        ph = pts[s0:s0 + chunk, 1]
        a_th, a_ph = waves.gradient(th, ph)
        a_th *= scale
        a_ph *= scale
        a = np.sqrt(a_th**2 + a_ph**2)
        sinc = np.where(a > 0, np.sin(a) / np.where(a > 0, a, 1.0), 1.0)
        ca = np.cos(a)
        st, ct = np.sin(th), np.cos(th)
        sp, cp = np.sin(ph), np.cos(ph)
        # n' = cos(a) n + sin(a)/a (a_th e_th + a_ph e_ph)
        x = ca * st * cp + sinc * (a_th * ct * cp - a_ph * sp)
        y = ca * st * sp + sinc * (a_th * ct * sp + a_ph * cp)
        z = ca * ct + sinc * (-a_th * st)
        out[s0:s0 + chunk, 0] = np.arctan2(np.sqrt(x * x + y * y), z)
        out[s0:s0 + chunk, 1] = np.mod(np.arctan2(y, x), 2.0 * np.pi)

    # numpy ufuncs release the GIL, so chunks run in parallel threads; every
    # chunk is a pure function of its own points, so the result is the same
    # for any thread count.
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(one, range(0, n, chunk)))
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
        return deflect(gl_ring_grid(lmax + 1, 2 * lmax + 1), rms_arcmin, seed)

    if not cache:
        return make()
    return _cached("glgrid-v1-%d-%d-%r" % (lmax, seed, rms_arcmin), make)


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
