"""CPU oracle for the nonuniform spin-0 spherical harmonic transform.

TEST INFRASTRUCTURE ONLY: the plain direct-summation definition of the type 2
transform (Sec. 2.1, Eq. SHTbase) and of its adjoint, type 1 (Eq.
adjointSHTbase), in double precision.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline``/``--impl reference`` legs
of ``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

The arithmetic lives in ``nusht_oracle.c`` (plain C + OpenMP, compiled with
gcc on first use into ``oracle/_build``); this module only marshals numpy
arrays.  Conventions (orthonormal Y_lm with Condon-Shortley phase, real-field
packed m-major storage) are stated in the C file's header.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, the addition theorem, Gauss-Legendre orthogonality,
scipy/mpmath, the reality symmetry, rotation invariance and the dot test; the
spin-weighted functions by ``tests/test_oracle_spin_pins.py`` (mpmath Wigner-d
sums, the spin-0 harmonics and the analytic spin-0 gradient, the spin
addition theorem, Gauss-Legendre orthogonality, the dot test).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nusht_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libnusht_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, IEEE semantics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i64 = ctypes.c_int64
        lib.oracle_nalm.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.oracle_nalm.restype = i64
        lib.oracle_plm_all.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        lib.oracle_synth.argtypes = [ctypes.c_int, ctypes.c_int, dp, i64, dp, dp]
        lib.oracle_ring_sums.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp]
        lib.oracle_adjoint_m.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, dp, ctypes.c_int, ip, dp]
        lib.oracle_synth_grad.argtypes = [ctypes.c_int, ctypes.c_int, dp, i64, dp, dp, dp]
        lib.oracle_pointing.argtypes = [ctypes.c_int, ctypes.c_int, dp, i64, dp, dp]
        lib.oracle_spin_lambda.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        lib.oracle_spin_synth.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, i64, dp, dp, dp]
        lib.oracle_spin_adjoint_m.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, dp, dp, dp, ctypes.c_int,
                                              ip, dp, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def nalm(lmax: int, mmax: int | None = None) -> int:
    """Number of packed coefficients for band limit lmax and order limit mmax."""
    mmax = lmax if mmax is None else mmax
    return (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) // 2


def lm_index(lmax: int, l, m):
    """Packed m-major index m(2L+1-m)/2 + l."""
    return m * (2 * lmax + 1 - m) // 2 + l


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def plm_all(lmax: int, theta: float, mmax: int | None = None) -> np.ndarray:
    """Orthonormal Pbar_lm(theta) (Condon-Shortley phase) for all packed (l, m)."""
    mmax = lmax if mmax is None else mmax
    out = np.zeros(nalm(lmax, mmax), dtype=np.float64)
    _load().oracle_plm_all(lmax, mmax, float(theta), _dp(out))
    return out


def _alm_pairs(alm: np.ndarray, lmax: int, mmax: int) -> np.ndarray:
    a = np.ascontiguousarray(alm, dtype=np.complex128)
    if a.shape != (nalm(lmax, mmax),):
        raise ValueError("alm has shape %s, expected (%d,)" % (a.shape, nalm(lmax, mmax)))
    return a.view(np.float64)


def _pts(pts: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(pts, dtype=np.float64)
    if p.ndim != 2 or p.shape[1] != 2:
        raise ValueError("pts must have shape (N, 2) = (theta, phi)")
    return p


def synth(alm: np.ndarray, pts: np.ndarray, lmax: int, mmax: int | None = None) -> np.ndarray:
    """Type 2 nuSHT by direct summation (Eq. SHTbase), real field; returns f[N]."""
    mmax = lmax if mmax is None else mmax
    a = _alm_pairs(alm, lmax, mmax)
    p = _pts(pts)
    out = np.empty(p.shape[0], dtype=np.float64)
    _load().oracle_synth(lmax, mmax, _dp(a), p.shape[0], _dp(p), _dp(out))
    return out


def ring_sums(alm: np.ndarray, thetas: np.ndarray, lmax: int, mmax: int | None = None) -> np.ndarray:
    """F[m, j] = sum_l a_lm Pbar_lm(theta_j), complex, shape (mmax+1, len(thetas))."""
    mmax = lmax if mmax is None else mmax
    a = _alm_pairs(alm, lmax, mmax)
    th = np.ascontiguousarray(thetas, dtype=np.float64)
    out = np.empty((mmax + 1, th.shape[0]), dtype=np.complex128)
    _load().oracle_ring_sums(lmax, mmax, _dp(a), th.shape[0], _dp(th), _dp(out.view(np.float64)))
    return out


def adjoint(f: np.ndarray, pts: np.ndarray, lmax: int, mmax: int | None = None, mlist=None) -> np.ndarray:
    """Type 1 nuSHT by direct summation (Eq. adjointSHTbase): c_lm = sum_i f_i conj(Y_lm).

    With ``mlist`` only those orders are computed (all l for each); the other
    packed entries are returned as NaN so that they cannot be mistaken for data.
    """
    mmax = lmax if mmax is None else mmax
    p = _pts(pts)
    fv = np.ascontiguousarray(f, dtype=np.float64)
    if fv.shape != (p.shape[0],):
        raise ValueError("f must have one value per point")
    if mlist is None:
        ms = np.arange(mmax + 1, dtype=np.int32)
        out = np.zeros(nalm(lmax, mmax), dtype=np.complex128)
    else:
        ms = np.unique(np.asarray(mlist, dtype=np.int32))
        if ms.size and (ms[0] < 0 or ms[-1] > mmax):
            raise ValueError("orders out of range")
        out = np.full(nalm(lmax, mmax), np.nan + 0j, dtype=np.complex128)
    ms = np.ascontiguousarray(ms)
    _load().oracle_adjoint_m(lmax, mmax, p.shape[0], _dp(p), _dp(fv), int(ms.size),
                             ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out.view(np.float64)))
    return out


def synth_grad(alm: np.ndarray, pts: np.ndarray, lmax: int, mmax: int | None = None):
    """Analytic (d f_i/d theta_i, d f_i/d phi_i) of the real-field type 2 sum."""
    mmax = lmax if mmax is None else mmax
    a = _alm_pairs(alm, lmax, mmax)
    p = _pts(pts)
    dth = np.empty(p.shape[0], dtype=np.float64)
    dph = np.empty(p.shape[0], dtype=np.float64)
    _load().oracle_synth_grad(lmax, mmax, _dp(a), p.shape[0], _dp(p), _dp(dth), _dp(dph))
    return dth, dph


def pointing(philm: np.ndarray, pts: np.ndarray, lmax: int, mmax: int | None = None) -> np.ndarray:
    """CMB lensing pointing (App. C, Eq. pointing and Eq. spin1deriv): the
    deflected (theta', phi') of every point for the lensing potential philm
    (packed real-field coefficients); shape (npts, 2), theta' in [0, pi],
    phi' in [0, 2 pi)."""
    mmax = lmax if mmax is None else mmax
    a = _alm_pairs(philm, lmax, mmax)
    p = _pts(pts)
    out = np.empty((p.shape[0], 2), dtype=np.float64)
    _load().oracle_pointing(lmax, mmax, _dp(a), p.shape[0], _dp(p), _dp(out))
    return out


def spin_lambda(lmax: int, spin: int, theta: float, mmax: int | None = None):
    """(lambda^(+s), lambda^(-s)): sY_lm(theta, 0) and (-s)Y_lm(theta, 0) for all
    packed (l, m), m >= 0 (entries with l < s are 0).  sY_lm =
    (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi}; spin 0 gives Pbar_lm."""
    mmax = lmax if mmax is None else mmax
    lp = np.zeros(nalm(lmax, mmax), dtype=np.float64)
    lm = np.zeros(nalm(lmax, mmax), dtype=np.float64)
    _load().oracle_spin_lambda(lmax, mmax, int(spin), float(theta), _dp(lp), _dp(lm))
    return lp, lm


def spin_synth(glm: np.ndarray, clm: np.ndarray, pts: np.ndarray, lmax: int, spin: int, mmax: int | None = None):
    """Spin-s synthesis of two real fields, Q + i U = sum (G_lm + i C_lm) sY_lm
    (G, C real-field coefficients in the packed layout); returns (Q, U)."""
    mmax = lmax if mmax is None else mmax
    g = _alm_pairs(glm, lmax, mmax)
    c = _alm_pairs(clm, lmax, mmax)
    p = _pts(pts)
    q = np.empty(p.shape[0], dtype=np.float64)
    u = np.empty(p.shape[0], dtype=np.float64)
    _load().oracle_spin_synth(lmax, mmax, int(spin), _dp(g), _dp(c), p.shape[0], _dp(p), _dp(q), _dp(u))
    return q, u


def spin_adjoint(q: np.ndarray, u: np.ndarray, pts: np.ndarray, lmax: int, spin: int, mmax: int | None = None,
                 mlist=None):
    """Spin-s adjoint (type 1): the transpose of spin_synth; returns (G, C).
    With ``mlist`` only those orders are computed (others NaN)."""
    mmax = lmax if mmax is None else mmax
    p = _pts(pts)
    qv = np.ascontiguousarray(q, dtype=np.float64)
    uv = np.ascontiguousarray(u, dtype=np.float64)
    if qv.shape != (p.shape[0],) or uv.shape != (p.shape[0],):
        raise ValueError("q and u must have one value per point")
    if mlist is None:
        ms = np.arange(mmax + 1, dtype=np.int32)
        g = np.zeros(nalm(lmax, mmax), dtype=np.complex128)
    else:
        ms = np.unique(np.asarray(mlist, dtype=np.int32))
        g = np.full(nalm(lmax, mmax), np.nan + 0j, dtype=np.complex128)
    c = g.copy()
    ms = np.ascontiguousarray(ms)
    _load().oracle_spin_adjoint_m(lmax, mmax, int(spin), p.shape[0], _dp(p), _dp(qv), _dp(uv), int(ms.size),
                                  ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(g.view(np.float64)),
                                  _dp(c.view(np.float64)))
    return g, c


def alm_dot(c: np.ndarray, a: np.ndarray, lmax: int, mmax: int | None = None) -> float:
    """Real inner product under which type 1 is the adjoint of real-field type 2:
    sum_l Re(conj(c_l0) a_l0) + 2 sum_{l, m>0} Re(conj(c_lm) a_lm)."""
    mmax = lmax if mmax is None else mmax
    w = np.full(nalm(lmax, mmax), 2.0)
    w[: lmax + 1] = 1.0  # m = 0 block comes first in the m-major layout
    return float(np.sum(w * (np.conj(c) * a).real))


def eps_eff(f_true: np.ndarray, f_est: np.ndarray) -> float:
    """Effective accuracy (Sec. 4): ||f_true - f_est||_2 / ||f_true||_2 (moduli for complex)."""
    num = np.sqrt(np.sum(np.abs(np.asarray(f_true) - np.asarray(f_est)) ** 2))
    den = np.sqrt(np.sum(np.abs(np.asarray(f_true)) ** 2))
    return float(num / den)
