"""Python binding of the GB300 nuSHT library (include/nusht.h).

Argument marshalling only: every step of the transform runs in the CUDA
library ``_lib/libnusht.so`` (built by ``paper_2406_14542_gb300.build``).
There is no CPU fallback; if the library is missing or the device is not a
GB300 (sm_103a) the calls raise.  PyTorch provides device memory and streams.

    import torch, paper_2406_14542_gb300 as nu
    plan = nu.Plan(lmax, pts_cuda_f64_Nx2, eps=1e-10, precision="fp64")
    f = plan.synth(alm_cuda_complex128)          # type 2 (Eq. SHTbase)
    c = plan.adjoint(f)                          # type 1 (Eq. adjointSHTbase)
    f = nu.nusht(alm, pts, plan)                 # differentiable in alm and pts
    ptg = grid_plan.pointing(phi_lm)             # CMB lensing pointing (App. C):
                                                 # (theta', phi') per point, (N, 2)
    batch = nu.BatchPlan(lmaxs, pts_list, eps=1e-5)   # many transforms of uneven lmax
    maps = batch.synth(alm_list)                 # one CUDA graph per direction
    batch64 = nu.BatchPlan(lmaxs, pts_list, eps=1e-10, precision="fp64")
                                                 # the same in FP64: complex128 / float64,
                                                 # bf16-sliced tensor-core contraction

Options (keyword arguments of Plan): sigma, kernel_width, tune (autotuner),
deterministic (bit-reproducible adjoint), legendre_table (plan-time
recurrence in HBM), fast_recurrence (double-float recurrence, opt-in),
fp64_contraction, fft_kernels (-1: cuFFT FP64 instead of the double-float
FFT kernels), profile (per-stage times, Plan.stage_times()), spin (spin-weighted
transforms Plan.synth_spin / adjoint_spin, FP64).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libnusht.so")

NUSHT_OK, NUSHT_EINVAL, NUSHT_ENOMEM, NUSHT_ECUDA, NUSHT_EUNSUPPORTED, NUSHT_ETIMEOUT, NUSHT_EDEVICE = range(7)
FP64, MIXED = 0, 1

EXPORTS = ("nusht_plan", "nusht_setpts", "nusht_synth", "nusht_adjoint", "nusht_synth_grad", "nusht_destroy",
           "nusht_info", "nusht_plan_sizes", "nusht_kernel_ft", "nusht_good_size", "nusht_stage_times",
           "nusht_strerror", "nusht_last_error", "nusht_version", "nusht_adjoint_direct_noalloc",
           "nusht_plan_many", "nusht_synth_many", "nusht_adjoint_many", "nusht_destroy_many", "nusht_batch_info",
           "nusht_plan_bin", "nusht_batch_status", "nusht_batch_path", "nusht_pointing", "nusht_adjoint_grad",
           "nusht_synth_grad_pts", "nusht_batch_schedule", "nusht_synth_spin", "nusht_adjoint_spin")


class NushtError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed: %s (%s)" % (where, msg, _name(code)))
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("kernel_width", ctypes.c_int), ("profile", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("tune", ctypes.c_int), ("fp64_contraction", ctypes.c_int),
                ("legendre_table", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("fast_recurrence", ctypes.c_int), ("fft_kernels", ctypes.c_int),
                ("spin", ctypes.c_int), ("reserved", ctypes.c_int)]


class Sizes(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_int), ("mmax", ctypes.c_int), ("nrings", ctypes.c_int), ("M", ctypes.c_int),
                ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("w", ctypes.c_int), ("beta", ctypes.c_double),
                ("sigma", ctypes.c_double), ("precision", ctypes.c_int), ("nitems", ctypes.c_int),
                ("nitems_total", ctypes.c_int), ("npts", ctypes.c_int64), ("bytes_device", ctypes.c_int64),
                ("leg_triples", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError("nuSHT CUDA library not built: %s (run python -m paper_2406_14542_gb300.build)" % p)
        lib = ctypes.CDLL(p)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.nusht_plan.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, i64, vp, ctypes.c_double,
                                   ctypes.c_int, ctypes.POINTER(Opts), vp]
        lib.nusht_setpts.argtypes = [vp, i64, vp, vp]
        lib.nusht_synth.argtypes = [vp, vp, vp, vp]
        lib.nusht_adjoint.argtypes = [vp, vp, vp, vp]
        lib.nusht_synth_grad.argtypes = [vp, vp, vp, vp, vp]
        lib.nusht_pointing.argtypes = [vp, vp, vp, vp]
        lib.nusht_adjoint_grad.argtypes = [vp, vp, vp, vp]
        lib.nusht_synth_spin.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.nusht_adjoint_spin.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.nusht_synth_grad_pts.argtypes = [vp, vp, vp, vp, vp]
        lib.nusht_destroy.argtypes = [vp]
        lib.nusht_info.argtypes = [vp, ctypes.POINTER(Sizes)]
        lib.nusht_plan_sizes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(Opts), ctypes.POINTER(Sizes)]
        lib.nusht_kernel_ft.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
        lib.nusht_good_size.argtypes = [i64, ctypes.c_int, ctypes.c_int]
        lib.nusht_good_size.restype = i64
        lib.nusht_stage_times.argtypes = [vp, dp]
        lib.nusht_adjoint_direct_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, vp]
        lib.nusht_plan_many.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(Opts), vp]
        lib.nusht_synth_many.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        lib.nusht_adjoint_many.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        lib.nusht_destroy_many.argtypes = [vp]
        lib.nusht_plan_bin.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.nusht_batch_status.argtypes = [vp, vp]
        lib.nusht_batch_path.argtypes = [vp, ctypes.c_int]
        lib.nusht_batch_schedule.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int)]
        lib.nusht_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64)]
        lib.nusht_strerror.argtypes = [ctypes.c_int]
        lib.nusht_strerror.restype = ctypes.c_char_p
        lib.nusht_last_error.restype = ctypes.c_char_p
        lib.nusht_version.restype = ctypes.c_char_p
        for name in ("nusht_plan", "nusht_setpts", "nusht_synth", "nusht_adjoint", "nusht_synth_grad",
                     "nusht_destroy", "nusht_info", "nusht_plan_sizes", "nusht_kernel_ft", "nusht_stage_times",
                     "nusht_adjoint_direct_noalloc", "nusht_plan_many", "nusht_synth_many",
                     "nusht_adjoint_many", "nusht_destroy_many", "nusht_batch_info", "nusht_plan_bin",
                     "nusht_batch_status", "nusht_batch_path", "nusht_pointing", "nusht_adjoint_grad",
                     "nusht_synth_grad_pts", "nusht_batch_schedule", "nusht_synth_spin",
                     "nusht_adjoint_spin"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _name(code: int) -> str:
    try:
        return load().nusht_strerror(code).decode()
    except Exception:
        return "status %d" % code


def _check(code: int, where: str):
    if code != NUSHT_OK:
        raise NushtError(code, where, load().nusht_last_error().decode())


def _opts(sigma=0.0, kernel_width=0, profile=False, fp64_contraction=False, legendre_table=0, tune=0,
          tensor_cores=0, deterministic=False, fast_recurrence=False, fft_kernels=0, spin=0) -> Opts:
    o = Opts()
    o.spin = int(spin)
    o.fft_kernels = int(fft_kernels)
    o.fast_recurrence = 1 if fast_recurrence else 0
    o.deterministic = 1 if deterministic else 0
    o.tensor_cores = int(tensor_cores)
    o.tune = int(tune)
    o.legendre_table = int(legendre_table)
    o.sigma = float(sigma)
    o.kernel_width = int(kernel_width)
    o.profile = 1 if profile else 0
    o.fp64_contraction = 1 if fp64_contraction else 0
    return o


def _prec(precision) -> int:
    if precision in (FP64, "fp64", "double"):
        return FP64
    if precision in (MIXED, "mixed"):
        return MIXED
    raise ValueError("precision must be 'fp64' or 'mixed'")


def nalm(lmax: int, mmax: int | None = None) -> int:
    mmax = lmax if mmax is None else mmax
    return (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) // 2


def plan_sizes(lmax: int, eps: float, precision="fp64", mmax: int | None = None, sigma=0.0, kernel_width=0) -> dict:
    """Sizes a plan would use (host-only computation, no GPU)."""
    mmax = lmax if mmax is None else mmax
    z = Sizes()
    o = _opts(sigma, kernel_width)
    _check(load().nusht_plan_sizes(lmax, mmax, eps, _prec(precision), ctypes.byref(o), ctypes.byref(z)),
           "nusht_plan_sizes")
    return z.as_dict()


def kernel_ft(w: int, beta: float, n: int, nk: int):
    """Fourier transform of the ES kernel as the planner computes it (host only)."""
    import numpy as np

    out = np.zeros(nk, dtype=np.float64)
    _check(load().nusht_kernel_ft(w, beta, n, nk, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "nusht_kernel_ft")
    return out


def good_size(nmin: int, multiple: int = 1, maxprime: int = 7) -> int:
    return int(load().nusht_good_size(int(nmin), int(multiple), int(maxprime)))


def version() -> str:
    return load().nusht_version().decode()


def _msign(lmax: int, mmax: int, like):
    """(-1)^m for every packed (l, m) entry (m-major, the m = 0 block first),
    as a real array of the kind of ``like`` (numpy array or torch tensor)."""
    import numpy as np

    s = np.concatenate([np.full(lmax + 1 - m, -1.0 if m & 1 else 1.0) for m in range(mmax + 1)])
    try:
        import torch

        if isinstance(like, torch.Tensor):
            return torch.as_tensor(s, device=like.device, dtype=like.real.dtype)
    except ImportError:
        pass
    return s


def complex_split(alm_pos, alm_neg, lmax: int, mmax: int | None = None):
    """A complex field F = sum_{l, |m| <= l} a_lm Y_lm as two real fields,
    F = R + i I (Sec. 2.1 treats real fields; a complex one is two of them).

    ``alm_pos`` holds a_{l,m} and ``alm_neg`` holds a_{l,-m}, both in the packed
    m-major layout of m >= 0 (the m = 0 entries of ``alm_neg`` are ignored).
    Returns the real-field coefficients (r, i) in that layout:
    r_lm = (a_lm + (-1)^m conj(a_{l,-m})) / 2,  i_lm = (a_lm - (-1)^m conj(a_{l,-m})) / (2i)
    (so r_l0 = Re a_l0, i_l0 = Im a_l0).  Works on numpy arrays and torch tensors."""
    mmax = lmax if mmax is None else mmax
    s = _msign(lmax, mmax, alm_pos)
    neg = alm_neg.copy() if hasattr(alm_neg, "copy") and not hasattr(alm_neg, "clone") else alm_neg.clone()
    neg[: lmax + 1] = alm_pos[: lmax + 1]
    t = s * neg.conj()
    return (alm_pos + t) / 2, (alm_pos - t) / 2j


def complex_merge_adjoint(cu, cv, lmax: int, mmax: int | None = None):
    """Adjoint of a complex map F = u + i v from the real-field adjoints
    cu = Y^H u and cv = Y^H v (m >= 0):  c_{l,m} = cu + i cv and
    c_{l,-m} = (-1)^m (conj(cu) + i conj(cv)).  Returns (c_pos, c_neg) in the
    packed layout of ``complex_split``."""
    mmax = lmax if mmax is None else mmax
    s = _msign(lmax, mmax, cu)
    return cu + 1j * cv, s * (cu.conj() + 1j * cv.conj())


def _stream_ptr(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(int(s.cuda_stream))


class Plan:
    """A planned transform for one band limit, point set, accuracy and precision.

    ``pts``: CUDA float64 tensor of shape (N, 2) holding (theta, phi).
    ``precision``: 'fp64' (complex128 a_lm, float64 maps) or 'mixed'
    (complex64 a_lm, float32 maps; recurrence and fold stay FP64).
    """

    def __init__(self, lmax: int, pts, eps: float = 1e-10, precision="fp64", mmax: int | None = None,
                 sigma: float = 0.0, kernel_width: int = 0, profile: bool = False, fp64_contraction: bool = False,
                 legendre_table: int = 0, tune: int = 0, deterministic: bool = False,
                 fast_recurrence: bool = False, fft_kernels: int = 0, spin: int = 0, stream=None):
        import torch

        self.lib = load()
        self.lmax = int(lmax)
        self.mmax = self.lmax if mmax is None else int(mmax)
        self.precision = _prec(precision)
        self.eps = float(eps)
        self.cdtype = torch.complex128 if self.precision == FP64 else torch.complex64
        self.rdtype = torch.float64 if self.precision == FP64 else torch.float32
        pts = self._check_pts(pts)
        self.npts = int(pts.shape[0])
        self.device = pts.device
        h = ctypes.c_void_p()
        o = _opts(sigma, kernel_width, profile, fp64_contraction, legendre_table, tune,
                  deterministic=deterministic, fast_recurrence=fast_recurrence, fft_kernels=fft_kernels, spin=spin)
        self.spin = int(spin)
        _check(self.lib.nusht_plan(ctypes.byref(h), self.lmax, self.mmax, self.npts,
                                   ctypes.c_void_p(pts.data_ptr() if self.npts else 0), self.eps, self.precision,
                                   ctypes.byref(o), _stream_ptr(stream)), "nusht_plan")
        self._h = h

    @staticmethod
    def _check_pts(pts):
        import torch

        if not (isinstance(pts, torch.Tensor) and pts.is_cuda and pts.dtype == torch.float64 and pts.dim() == 2
                and pts.shape[1] == 2):
            raise ValueError("pts must be a CUDA float64 tensor of shape (N, 2)")
        return pts.contiguous()

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h

    @property
    def nalm(self) -> int:
        return nalm(self.lmax, self.mmax)

    def bin_size(self) -> int:
        """Spreading/interpolation bin edge the plan uses (autotuned when tune=1/2)."""
        v = ctypes.c_int()
        _check(self.lib.nusht_plan_bin(self.handle, ctypes.byref(v)), "nusht_plan_bin")
        return v.value

    def info(self) -> dict:
        z = Sizes()
        _check(self.lib.nusht_info(self.handle, ctypes.byref(z)), "nusht_info")
        return z.as_dict()

    def setpts(self, pts, stream=None):
        pts = self._check_pts(pts)
        _check(self.lib.nusht_setpts(self.handle, int(pts.shape[0]), ctypes.c_void_p(pts.data_ptr()),
                                     _stream_ptr(stream)), "nusht_setpts")
        self.npts = int(pts.shape[0])

    def _alm(self, alm):
        import torch

        if not (isinstance(alm, torch.Tensor) and alm.is_cuda and alm.dtype == self.cdtype
                and alm.shape == (self.nalm,)):
            raise ValueError("alm must be a CUDA %s tensor of shape (%d,)" % (self.cdtype, self.nalm))
        return alm.contiguous()

    def _map(self, m):
        import torch

        if not (isinstance(m, torch.Tensor) and m.is_cuda and m.dtype == self.rdtype and m.shape == (self.npts,)):
            raise ValueError("map must be a CUDA %s tensor of shape (%d,)" % (self.rdtype, self.npts))
        return m.contiguous()

    def synth(self, alm, out=None, stream=None):
        """Type 2 nuSHT: values at the plan's points (caller's order)."""
        import torch

        alm = self._alm(alm)
        if out is None:
            out = torch.empty(self.npts, dtype=self.rdtype, device=self.device)
        out = self._map(out)
        _check(self.lib.nusht_synth(self.handle, ctypes.c_void_p(alm.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    _stream_ptr(stream)), "nusht_synth")
        return out

    def adjoint(self, m, out=None, stream=None):
        """Type 1 nuSHT (adjoint): c_lm = sum_i f_i conj(Y_lm(theta_i, phi_i))."""
        import torch

        m = self._map(m)
        if out is None:
            out = torch.empty(self.nalm, dtype=self.cdtype, device=self.device)
        out = self._alm(out)
        _check(self.lib.nusht_adjoint(self.handle, ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      _stream_ptr(stream)), "nusht_adjoint")
        return out

    def synth_complex(self, alm_pos, alm_neg, stream=None):
        """Complex field F = sum_{l,|m|<=l} a_lm Y_lm at the points (two real
        transforms, see ``complex_split``); returns a complex tensor."""
        r, i = complex_split(alm_pos, alm_neg, self.lmax, self.mmax)
        fr = self.synth(r.to(self.cdtype).contiguous(), stream=stream)
        fi = self.synth(i.to(self.cdtype).contiguous(), stream=stream)
        return fr + 1j * fi

    def adjoint_complex(self, fmap, stream=None):
        """Adjoint for a complex map: (c_pos, c_neg) with c_{l,+-m} =
        sum_j F_j conj(Y_{l,+-m}(x_j)) (see ``complex_merge_adjoint``)."""
        cu = self.adjoint(fmap.real.to(self.rdtype).contiguous(), stream=stream)
        cv = self.adjoint(fmap.imag.to(self.rdtype).contiguous(), stream=stream)
        return complex_merge_adjoint(cu, cv, self.lmax, self.mmax)

    def synth_grad(self, alm, stream=None):
        """(d f_i / d theta_i, d f_i / d phi_i) by derivative-of-kernel interpolation."""
        import torch

        alm = self._alm(alm)
        dth = torch.empty(self.npts, dtype=self.rdtype, device=self.device)
        dph = torch.empty(self.npts, dtype=self.rdtype, device=self.device)
        _check(self.lib.nusht_synth_grad(self.handle, ctypes.c_void_p(alm.data_ptr()),
                                         ctypes.c_void_p(dth.data_ptr()), ctypes.c_void_p(dph.data_ptr()),
                                         _stream_ptr(stream)), "nusht_synth_grad")
        return dth, dph

    def adjoint_grad(self, g, out=None, stream=None):
        """Gradient of a real loss in a_lm from the cotangent g = dL/df of the
        synthesised map (nusht_adjoint_grad: the adjoint with the m > 0
        entries doubled, torch's dL/dRe + i dL/dIm convention)."""
        import torch

        g = self._map(g)
        if out is None:
            out = torch.empty(self.nalm, dtype=self.cdtype, device=self.device)
        out = self._alm(out)
        _check(self.lib.nusht_adjoint_grad(self.handle, ctypes.c_void_p(g.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
               "nusht_adjoint_grad")
        return out

    def synth_grad_pts(self, alm, g, out=None, stream=None):
        """Gradient of a real loss in the point coordinates from the cotangent
        g = dL/df (nusht_synth_grad_pts): float64 (npts, 2) tensor of
        (g_i df_i/dtheta_i, g_i df_i/dphi_i)."""
        import torch

        alm = self._alm(alm)
        g = self._map(g)
        gp = out if out is not None else torch.empty((self.npts, 2), dtype=torch.float64, device=self.device)
        if gp.dtype != torch.float64 or tuple(gp.shape) != (self.npts, 2) or not gp.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of shape (npts, 2)")
        _check(self.lib.nusht_synth_grad_pts(self.handle, ctypes.c_void_p(alm.data_ptr()),
                                             ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(gp.data_ptr()),
                                             _stream_ptr(stream)), "nusht_synth_grad_pts")
        return gp

    def synth_spin(self, glm, clm, stream=None):
        """Spin-s synthesis (plan made with spin=s >= 1, FP64): Q + iU =
        sum (G_lm + i C_lm) sY_lm at the points; returns (Q, U) float64."""
        import torch

        glm, clm = self._alm(glm), self._alm(clm)
        q = torch.empty(self.npts, dtype=torch.float64, device=self.device)
        u = torch.empty(self.npts, dtype=torch.float64, device=self.device)
        _check(self.lib.nusht_synth_spin(self.handle, ctypes.c_void_p(glm.data_ptr()), ctypes.c_void_p(clm.data_ptr()),
                                         ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                         _stream_ptr(stream)), "nusht_synth_spin")
        return q, u

    def adjoint_spin(self, q, u, stream=None):
        """Adjoint of synth_spin: (G, C) complex128 coefficients."""
        import torch

        q, u = self._map(q), self._map(u)
        g = torch.empty(self.nalm, dtype=torch.complex128, device=self.device)
        c = torch.empty(self.nalm, dtype=torch.complex128, device=self.device)
        _check(self.lib.nusht_adjoint_spin(self.handle, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                           ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                           _stream_ptr(stream)), "nusht_adjoint_spin")
        return g, c

    def pointing(self, philm, out=None, stream=None):
        """CMB lensing pointing (App. C): the deflected (theta', phi') of every
        point for the lensing potential ``philm`` (the plan's a_lm layout and
        precision); float64 tensor of shape (npts, 2), theta' in [0, pi],
        phi' in [0, 2 pi), in the order of the plan's points."""
        import torch

        philm = self._alm(philm)
        ptg = out if out is not None else torch.empty((self.npts, 2), dtype=torch.float64, device=self.device)
        if ptg.dtype != torch.float64 or tuple(ptg.shape) != (self.npts, 2) or not ptg.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of shape (npts, 2)")
        _check(self.lib.nusht_pointing(self.handle, ctypes.c_void_p(philm.data_ptr()),
                                       ctypes.c_void_p(ptg.data_ptr()), _stream_ptr(stream)), "nusht_pointing")
        return ptg

    def stage_times(self) -> dict:
        import numpy as np

        out = np.zeros(12, dtype=np.float64)
        _check(self.lib.nusht_stage_times(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "nusht_stage_times")
        names = ["legendre", "theta_fft", "deconv_pad", "grid_fft", "interp", "total"]
        anames = ["spread", "grid_fft", "deconv_trunc", "theta_fft", "legendre", "total"]
        return {"synth": dict(zip(names, out[:6].tolist())), "adjoint": dict(zip(anames, out[6:].tolist()))}

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.lib.nusht_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchPlan:
    """Many transforms of uneven lmax and point count in one plan.
    ``precision="mixed"``: complex64 a_lm, float32 maps; ``"fp64"``:
    complex128 a_lm, float64 maps, the Legendre contraction split into bf16
    slices on the tensor cores.  ``pts_list[b]`` is a CUDA float64 (N_b, 2)
    tensor; each lmax <= 4095."""

    def __init__(self, lmaxs, pts_list, eps: float = 1e-5, sigma: float = 0.0, legendre_table: int = 0,
                 tune: int = 0, tensor_cores: int = 0, deterministic: bool = False, fft_kernels: int = 0,
                 stream=None, precision="mixed"):
        import torch

        self.lib = load()
        self.precision = _prec(precision)
        self._cdt = torch.complex128 if self.precision == FP64 else torch.complex64
        self._rdt = torch.float64 if self.precision == FP64 else torch.float32
        self.lmaxs = [int(l) for l in lmaxs]
        n = len(self.lmaxs)
        if len(pts_list) != n:
            raise ValueError("one point array per transform")
        self.pts = [Plan._check_pts(p) for p in pts_list]
        self.npts = [int(p.shape[0]) for p in self.pts]
        self.device = self.pts[0].device
        larr = (ctypes.c_int * n)(*self.lmaxs)
        narr = (ctypes.c_int64 * n)(*self.npts)
        parr = (ctypes.c_void_p * n)(*[p.data_ptr() if p.numel() else 0 for p in self.pts])
        o = _opts(sigma, legendre_table=legendre_table, tune=tune, tensor_cores=tensor_cores,
                  deterministic=deterministic, fft_kernels=fft_kernels)
        h = ctypes.c_void_p()
        _check(self.lib.nusht_plan_many(ctypes.byref(h), n, larr, narr, parr, float(eps), self.precision,
                                        ctypes.byref(o), _stream_ptr(stream)), "nusht_plan_many")
        self._h = h
        self.n = n

    def info(self) -> dict:
        nb = ctypes.c_int()
        of = (ctypes.c_int * self.n)()
        bl = (ctypes.c_int * self.n)()
        by = ctypes.c_int64()
        _check(self.lib.nusht_batch_info(self._h, ctypes.byref(nb), of, bl, ctypes.byref(by)), "nusht_batch_info")
        sched = []
        for g in range(nb.value):
            cs, ca = ctypes.c_int(), ctypes.c_int()
            _check(self.lib.nusht_batch_schedule(self._h, g, ctypes.byref(cs), ctypes.byref(ca)),
                   "nusht_batch_schedule")
            sched.append((cs.value, ca.value))
        return {"nbuckets": nb.value, "bucket_of": list(of), "bucket_lmax": list(bl)[: nb.value],
                "bytes_device": by.value,
                "paths": [self.lib.nusht_batch_path(self._h, g) for g in range(nb.value)],
                "schedule": sched}

    def status(self, stream=None):
        """Synchronise and raise if a tensor-core block of an earlier call gave
        up a bounded wait (its outputs are then invalid)."""
        _check(self.lib.nusht_batch_status(self._h, _stream_ptr(stream)), "nusht_batch_status")

    def synth(self, alms, outs=None, stream=None):
        import torch

        if outs is None:
            outs = [torch.empty(n, dtype=self._rdt, device=self.device) for n in self.npts]
        for a, l in zip(alms, self.lmaxs):
            if not (a.is_cuda and a.dtype == self._cdt and a.shape == (nalm(l),) and a.is_contiguous()):
                raise ValueError("alm must be contiguous CUDA %s of length nalm(lmax)" % self._cdt)
        ia = (ctypes.c_void_p * self.n)(*[a.data_ptr() for a in alms])
        oa = (ctypes.c_void_p * self.n)(*[o.data_ptr() for o in outs])
        _check(self.lib.nusht_synth_many(self._h, ia, oa, _stream_ptr(stream)), "nusht_synth_many")
        return outs

    def adjoint(self, maps, outs=None, stream=None):
        import torch

        if outs is None:
            outs = [torch.empty(nalm(l), dtype=self._cdt, device=self.device) for l in self.lmaxs]
        for m, n in zip(maps, self.npts):
            if not (m.is_cuda and m.dtype == self._rdt and m.shape == (n,) and m.is_contiguous()):
                raise ValueError("maps must be contiguous CUDA %s of length npts" % self._rdt)
        ia = (ctypes.c_void_p * self.n)(*[m.data_ptr() for m in maps])
        oa = (ctypes.c_void_p * self.n)(*[o.data_ptr() for o in outs])
        _check(self.lib.nusht_adjoint_many(self._h, ia, oa, _stream_ptr(stream)), "nusht_adjoint_many")
        return outs

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.lib.nusht_destroy_many(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    import torch

    class NuSHT(torch.autograd.Function):
        """f = Y a (type 2) with gradients in a_lm (through the adjoint, type 1)
        and in the point coordinates (derivative-of-kernel interpolation).

        For a real loss, torch's complex gradient is dL/dRe(a) + i dL/dIm(a)
        = w_m (Y^dagger g)_lm with w_0 = 1, w_{m>0} = 2 (the real-field map
        counts each m > 0 twice, once through a_{l,-m}); the library applies
        that weight (nusht_adjoint_grad) and the cotangent product of the
        position gradient (nusht_synth_grad_pts), so backward only calls them.
        """

        @staticmethod
        def forward(ctx, alm, pts, plan):
            ctx.plan = plan
            ctx.save_for_backward(alm)
            return plan.synth(alm.detach())

        @staticmethod
        def backward(ctx, g):
            plan = ctx.plan
            (alm,) = ctx.saved_tensors
            g = g.contiguous().to(plan.rdtype)
            ga = gp = None
            if ctx.needs_input_grad[0]:
                ga = plan.adjoint_grad(g)
            if ctx.needs_input_grad[1]:
                gp = plan.synth_grad_pts(alm.detach(), g)
            return ga, gp, None

    return NuSHT


_NuSHT = None


def nusht(alm, pts, plan: Plan):
    """Differentiable type 2 nuSHT at ``plan``'s points; ``pts`` must hold the
    same coordinates the plan was made with (it carries their gradient)."""
    global _NuSHT
    if _NuSHT is None:
        _NuSHT = _autograd()
    return _NuSHT.apply(alm, pts, plan)
