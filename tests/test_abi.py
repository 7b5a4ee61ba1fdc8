"""Host-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and its planner math (sizes, ES kernel Fourier transform,
good FFT sizes) matches independent computations.  No GPU needed."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nu():
    import paper_2406_14542_gb300 as nu
    from paper_2406_14542_gb300 import build

    build.build()
    nu.load()
    return nu


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "nusht.h")).read()
    return sorted(set(re.findall(r"NUSHT_API\s+[\w\s\*]+?\b(nusht_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(nu):
    syms = header_symbols()
    assert len(syms) >= 14
    lib = nu.load()
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(nu.EXPORTS)


def test_strerror_and_version(nu):
    lib = nu.load()
    for code in range(7):
        assert lib.nusht_strerror(code).decode().startswith("NUSHT_")
    assert "sm_103a" in nu.version()


def test_appendix_b_good_numbers(nu):
    """The paper's list of N_r (App. B): multiples of 4 up to 10000 with
    N_r - 1 11-smooth; underlined ones have largest prime factor 11."""
    rows = [l for l in open(os.path.join(ROOT, "tests", "golden", "appendix_b_good_numbers.txt"))
            if not l.startswith("#")]
    toks = " ".join(rows).split()
    listed = [int(t.rstrip("*")) for t in toks]
    under = {int(t.rstrip("*")) for t in toks if t.endswith("*")}
    ours = [n for n in range(4, 10001, 4) if nu.good_size(n - 1, 1, 11) == n - 1]
    assert ours == listed
    seven = {n for n in ours if nu.good_size(n - 1, 1, 7) == n - 1}
    assert set(ours) - seven == under


def test_good_size_small(nu):
    assert nu.good_size(1, 1, 7) == 1
    assert nu.good_size(8191, 1, 7) == 8192
    assert nu.good_size(8190, 4, 7) == 8192
    assert nu.good_size(10239, 2, 7) == 10240
    assert nu.good_size(11, 1, 7) == 12


@pytest.mark.parametrize("w,beta,n", [(12, 27.6, 64), (7, 16.1, 256), (11, 25.3, 16384), (16, 36.8, 40)])
def test_kernel_ft_against_quadrature(nu, w, beta, n):
    """psihat(k) = int_{|y|<=alpha} exp(beta(sqrt(1-(y/alpha)^2)-1)) cos(k y) dy, alpha = w pi / n."""
    from scipy.integrate import quad

    alpha = w * math.pi / n
    ks = [0, 1, 3, n // 8, n // 4 - 1]
    got = nu.kernel_ft(w, beta, n, max(ks) + 1)
    for k in ks:
        f = lambda y: math.exp(beta * (math.sqrt(max(0.0, 1 - (y / alpha) ** 2)) - 1)) * math.cos(k * y)
        ref, _ = quad(f, -alpha, alpha, limit=400, epsabs=1e-15 * alpha, epsrel=1e-13)
        assert abs(got[k] - ref) <= 1e-12 * abs(got[0]), (k, got[k], ref)


def test_plan_sizes(nu):
    z = nu.plan_sizes(4095, 1e-10, "fp64")  # default sigma 1.5 in FP64
    assert z["M"] == 8192 and z["nrings"] == 4097
    assert z["sigma"] == 1.5 and z["n1"] == z["n2"] == 12288
    assert 13 <= z["w"] <= 15
    z = nu.plan_sizes(4095, 1e-10, "fp64", sigma=2.0)
    assert z["n1"] == z["n2"] == 16384 and 10 <= z["w"] <= 13
    z = nu.plan_sizes(4095, 1e-5, "mixed")  # default sigma 2 in mixed precision
    assert z["sigma"] == 2.0 and z["n1"] == 16384 and z["w"] == 7
    z = nu.plan_sizes(63, 1e-10)
    assert z["M"] % 4 == 0 and z["M"] >= 128 and z["n1"] >= 1.5 * 127
    z = nu.plan_sizes(0, 1e-5, "mixed")
    assert z["M"] == 4 and z["n1"] >= 2 * z["w"]
    z = nu.plan_sizes(1023, 1e-5, "mixed", sigma=1.25)
    assert z["n1"] >= 1.25 * 2047 and z["sigma"] == 1.25


@pytest.mark.parametrize("args,code", [
    ((-1, 1e-10, "fp64"), 1), ((10, 0.5, "fp64"), 1), ((10, 1e-16, "fp64"), 1),
    ((10, 1e-8, "mixed"), 4), ((20000, 1e-10, "fp64"), 1),
])
def test_plan_sizes_rejects(nu, args, code):
    with pytest.raises(nu.NushtError) as e:
        nu.plan_sizes(*args)
    assert e.value.code == code


def test_mmax_validation(nu):
    with pytest.raises(nu.NushtError) as e:
        nu.plan_sizes(10, 1e-10, mmax=11)
    assert e.value.code == nu.NUSHT_EINVAL


def test_plan_without_gpu_reports_device_error(nu):
    """On a machine without a CUDA device the planner fails cleanly (no fallback)."""
    import ctypes
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = nu.load()
    h = ctypes.c_void_p()
    rc = lib.nusht_plan(ctypes.byref(h), 8, 8, 0, None, 1e-8, 0, None, None)
    assert rc == nu.NUSHT_EDEVICE and not h.value
    # argument errors come first, before any device query
    rc = lib.nusht_plan(ctypes.byref(h), 8, 9, 0, None, 1e-8, 0, None, None)
    assert rc == nu.NUSHT_EINVAL
    assert lib.nusht_destroy(None) == 0


def test_execute_calls_reject_null_plan(nu):
    """Every execute entry point rejects a NULL plan with NUSHT_EINVAL before
    any GPU work (host-side validation; no device needed)."""
    lib = nu.load()
    assert lib.nusht_synth(None, None, None, None) == nu.NUSHT_EINVAL
    assert lib.nusht_adjoint(None, None, None, None) == nu.NUSHT_EINVAL
    assert lib.nusht_synth_grad(None, None, None, None, None) == nu.NUSHT_EINVAL
    assert lib.nusht_pointing(None, None, None, None) == nu.NUSHT_EINVAL
    assert b"NULL" in lib.nusht_last_error()
