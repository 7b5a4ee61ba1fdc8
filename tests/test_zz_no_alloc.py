"""The allocation-free entry point nusht_adjoint_direct_noalloc, called
through the C ABI, against the planned adjoint nusht_adjoint and against the
oracle's direct sum.

It serves callers that cannot call cudaMalloc (their device memory belongs
to another allocator, or allocation latency is not acceptable): it takes
only caller-owned inputs and outputs and keeps its partial sums in a static
device array shared by every call.  Two calls in a row with different inputs
must both agree with the planned path: the second call must not see the
first call's partial sums, also when it uses a smaller layout (other lmax
and mmax) or fewer point chunks than the array has slots, and an empty point
set must give zeros.

The file name sorts last so that pytest collects it after every other test
file: if it fails, a run that stops at the first failure (-x) has already run
all other tests.  Its tests do not depend on that order; each passes in a
fresh process too.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # FP64 tolerance of the parity tests (relative l2, Sec. 4)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14542_gb300 import build

    build.build()
    import paper_2406_14542_gb300 as nu

    return torch, nu


def noalloc_adjoint(torch, nu, lmax, mmax, pts, f, out):
    lib = nu.load()
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    rc = lib.nusht_adjoint_direct_noalloc(lmax, mmax, int(pts.shape[0]), ctypes.c_void_p(pts.data_ptr()),
                                          ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)
    return rc


def rel(torch, a, b):
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


@pytest.mark.parametrize("lmax,mmax,npts", [(63, 63, 20000), (255, 200, 5000)])
def test_noalloc_matches_planned_adjoint_twice(env, lmax, mmax, npts):
    torch, nu = env
    pts = W.points_uniform(npts, seed=lmax)
    dpts = torch.from_numpy(pts).cuda()
    plan = nu.Plan(lmax, dpts, eps=1e-10, precision="fp64", mmax=mmax)
    out = torch.empty(plan.nalm, dtype=torch.complex128, device="cuda")
    for call in range(2):
        y = np.random.default_rng(100 + call).standard_normal(npts)
        f = torch.from_numpy(y).cuda()
        ref = plan.adjoint(f).clone()
        rc = noalloc_adjoint(torch, nu, lmax, mmax, dpts, f, out)
        assert rc == 0, nu.load().nusht_last_error().decode()
        torch.cuda.synchronize()
        err = rel(torch, out, ref)
        assert err <= TOL, (call, err)
        assert torch.all(out[: lmax + 1].imag == 0)
        if lmax <= 63:  # the direct sum itself, O(lmax^2 npts)
            orc = torch.from_numpy(oracle.adjoint(y, pts, lmax, mmax)).cuda()
            assert rel(torch, out, orc) <= TOL
    plan.close()


def test_noalloc_smaller_layout_after_a_large_call(env):
    """A large call fills every slot of the array; a following call with a
    different (lmax, mmax) and fewer points than one chunk per slot, then an
    empty point set, must not pick up anything the earlier calls left."""
    torch, nu = env
    big = W.points_uniform(20000, seed=1)
    fb = torch.from_numpy(np.random.default_rng(1).standard_normal(20000)).cuda()
    outb = torch.empty(nu.nalm(255), dtype=torch.complex128, device="cuda")
    assert noalloc_adjoint(torch, nu, 255, 255, torch.from_numpy(big).cuda(), fb, outb) == 0
    small = W.points_uniform(100, seed=2)
    ys = np.random.default_rng(2).standard_normal(100)
    outs = torch.empty(nu.nalm(40, 30), dtype=torch.complex128, device="cuda")
    assert noalloc_adjoint(torch, nu, 40, 30, torch.from_numpy(small).cuda(), torch.from_numpy(ys).cuda(), outs) == 0
    torch.cuda.synchronize()
    ref = torch.from_numpy(oracle.adjoint(ys, small, 40, 30)).cuda()
    assert rel(torch, outs, ref) <= TOL
    plan = nu.Plan(40, torch.from_numpy(small).cuda(), eps=1e-10, precision="fp64", mmax=30)
    assert rel(torch, outs, plan.adjoint(torch.from_numpy(ys).cuda())) <= TOL
    plan.close()
    empty = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    fe = torch.empty(0, dtype=torch.float64, device="cuda")
    oute = torch.full((nu.nalm(40, 30),), 7.0 + 7.0j, dtype=torch.complex128, device="cuda")
    assert noalloc_adjoint(torch, nu, 40, 30, empty, fe, oute) == 0
    torch.cuda.synchronize()
    assert torch.all(oute == 0)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, nu = env
    pts = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    f = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(nu.nalm(256), dtype=torch.complex128, device="cuda")
    rc = noalloc_adjoint(torch, nu, 256, 256, pts, f, out)
    assert rc == nu.NUSHT_EINVAL
    assert "255" in nu.load().nusht_last_error().decode()
