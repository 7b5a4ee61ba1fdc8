"""The allocation-free entry point nusht_adjoint_direct_noalloc, called
through the C ABI, against the planned adjoint nusht_adjoint.

It serves callers that cannot call cudaMalloc (their device memory belongs
to another allocator, or allocation latency is not acceptable): it takes
only caller-owned inputs and outputs and keeps its partial sums in a static
device array.  Two calls in a row with different inputs must both agree with
the planned path (the second call must not see the first call's partial
sums).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.parametrize("lmax,mmax,npts", [(63, 63, 20000), (255, 200, 5000)])
def test_noalloc_matches_planned_adjoint_twice(env, lmax, mmax, npts):
    torch, nu = env
    pts = W.points_uniform(npts, seed=lmax)
    dpts = torch.from_numpy(pts).cuda()
    plan = nu.Plan(lmax, dpts, eps=1e-10, precision="fp64", mmax=mmax)
    out = torch.empty(plan.nalm, dtype=torch.complex128, device="cuda")
    for call in range(2):
        f = torch.from_numpy(np.random.default_rng(100 + call).standard_normal(npts)).cuda()
        ref = plan.adjoint(f).clone()
        rc = noalloc_adjoint(torch, nu, lmax, mmax, dpts, f, out)
        assert rc == 0, nu.load().nusht_last_error().decode()
        torch.cuda.synchronize()
        err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        assert err <= TOL, (call, err)
        assert torch.all(out[: lmax + 1].imag == 0)
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, nu = env
    pts = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    f = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(nu.nalm(256), dtype=torch.complex128, device="cuda")
    rc = noalloc_adjoint(torch, nu, 256, 256, pts, f, out)
    assert rc == nu.NUSHT_EINVAL
    assert "255" in nu.load().nusht_last_error().decode()
