"""Failure handling on the GPU without a GPU fault: allocation failures are
injected on the host (NUSHT_FAIL_ALLOC_AFTER=k makes the (k+1)-th device
allocation of a plan report NUSHT_ENOMEM, as a full device would).  For every
k the plan call must return NUSHT_ENOMEM with a NULL handle, give back every
byte it had allocated, and leave the library usable: a plan made afterwards
without the injection is correct against the oracle.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14542_gb300 import build

    build.build()
    import paper_2406_14542_gb300 as nu

    return torch, nu


def raw_plan(torch, nu, L, dpts, eps, prec):
    lib = nu.load()
    h = ctypes.c_void_p()
    o = nu.Opts()
    rc = lib.nusht_plan(ctypes.byref(h), L, L, int(dpts.shape[0]), ctypes.c_void_p(dpts.data_ptr()), eps, prec,
                        ctypes.byref(o), ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    return rc, h


@pytest.mark.parametrize("prec,eps", [(0, 1e-10), (1, 1e-5)])
def test_injected_allocation_failures(env, prec, eps):
    torch, nu = env
    lib = nu.load()
    L, a, pts = W.workload("uniform63")
    dpts = torch.from_numpy(pts).cuda()
    # warm-up: module loading and cuFFT initialisation are not leaks
    rc, h = raw_plan(torch, nu, L, dpts, eps, prec)
    assert rc == 0
    lib.nusht_destroy(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for k in range(0, 64, 3):
        os.environ["NUSHT_FAIL_ALLOC_AFTER"] = str(k)
        try:
            rc, h = raw_plan(torch, nu, L, dpts, eps, prec)
        finally:
            del os.environ["NUSHT_FAIL_ALLOC_AFTER"]
        if rc == 0:  # k is beyond the plan's allocation count
            lib.nusht_destroy(h)
            break
        failed += 1
        assert rc == nu.NUSHT_ENOMEM, (k, rc, lib.nusht_last_error().decode())
        assert h.value is None
        assert "injected" in lib.nusht_last_error().decode()
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        assert abs(free - free0) <= (4 << 20), (k, free0 - free)
    assert failed >= 5
    # the library is still usable and correct
    cd = torch.complex128 if prec == 0 else torch.complex64
    plan = nu.Plan(L, dpts, eps=eps, precision=prec)
    f = plan.synth(torch.from_numpy(a).to(cd).cuda()).double().cpu().numpy()
    plan.close()
    assert oracle.eps_eff(oracle.synth(a, pts, L), f) <= (1e-10 if prec == 0 else 1e-5)


@pytest.mark.parametrize("precision,eps,path", [("mixed", 1e-5, 2), ("fp64", 1e-10, 3)])
def test_tensor_core_wait_runs_out_and_reports_timeout(env, precision, eps, path):
    """The tensor-core contractions' bounded waits (the TF32 split of mixed
    plans and the bf16 split of FP64 plans).  With the test hook
    NUSHT_TEST_TC_GIVEUP=1 at plan time the MMA thread's first wait for data
    has a limit of zero polls, so it runs out before any MMA is issued; the
    block's other roles stop waiting, the copies already issued are waited
    for, tensor memory is freed, and the plan's status word reports it:
    nusht_batch_status returns NUSHT_ETIMEOUT for the synthesis and for the
    adjoint, then NUSHT_OK once cleared.  A batch planned afterwards without
    the hook is correct against the oracle (the context stays usable)."""
    torch, nu = env
    ls = [40, 63, 100]
    cdt = np.complex128 if precision == "fp64" else np.complex64
    rdt = torch.float64 if precision == "fp64" else torch.float32
    alms = [W.alm_gaussian(l, seed=i, dtype=cdt) for i, l in enumerate(ls)]
    pts = [W.points_uniform(2 * l * l, seed=10 + i) for i, l in enumerate(ls)]
    dpts = [torch.from_numpy(p).cuda() for p in pts]
    dalm = [torch.from_numpy(a).cuda() for a in alms]
    os.environ["NUSHT_TEST_TC_GIVEUP"] = "1"
    try:
        bp = nu.BatchPlan(ls, dpts, eps=eps, precision=precision)
    finally:
        del os.environ["NUSHT_TEST_TC_GIVEUP"]
    assert set(bp.info()["paths"]) == {path}
    bp.synth(dalm)
    with pytest.raises(nu.NushtError) as ex:
        bp.status()
    assert ex.value.code == nu.NUSHT_ETIMEOUT
    bp.status()  # cleared
    bp.adjoint([torch.ones(p.shape[0], dtype=rdt, device="cuda") for p in pts])
    with pytest.raises(nu.NushtError) as ex:
        bp.status()
    assert ex.value.code == nu.NUSHT_ETIMEOUT
    bp.close()
    good = nu.BatchPlan(ls, dpts, eps=eps, precision=precision)
    outs = good.synth(dalm)
    good.status()
    for l, a, p, f in zip(ls, alms, pts, outs):
        sel = W.subset(p.shape[0], 2000, seed=l)
        ref = oracle.synth(a.astype(np.complex128), p[sel], l)
        assert oracle.eps_eff(ref, f.double().cpu().numpy()[sel]) <= eps
    good.close()
