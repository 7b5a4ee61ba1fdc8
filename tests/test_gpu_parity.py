"""GPU parity: the CUDA path (through the C ABI) against the direct-sum oracle
on the same seeded inputs.

Tolerances (relative l2 error eps_eff of Sec. 4): 1e-10 in FP64 mode, 1e-5 in
mixed mode (the targets of the requested accuracies); the adjoint dot test
<y, S a> = <S^H y, a> holds to 1e-12 in FP64 because spreading and
interpolation use the same kernel values (exact transposes), whatever eps.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14542_gb300 import build

    build.build()
    import paper_2406_14542_gb300 as nu

    return torch, nu


def dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def run_synth(torch, nu, L, alm, pts, prec, eps=None, mmax=None, **kw):
    eps = eps if eps is not None else TOL[prec]
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    plan = nu.Plan(L, dev(torch, pts), eps=eps, precision=prec, mmax=mmax, **kw)
    f = plan.synth(dev(torch, alm, cd))
    torch.cuda.synchronize()
    return plan, f.double().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_synth_uniform63(env, prec):
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    _, f = run_synth(torch, nu, L, a, pts, prec)
    ref = oracle.synth(a, pts, L)
    e = oracle.eps_eff(ref, f)
    assert e <= TOL[prec], e


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_uniform63(env, prec):
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    y = np.random.default_rng(7).standard_normal(pts.shape[0])
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    rd = torch.float64 if prec == "fp64" else torch.float32
    plan = nu.Plan(L, dev(torch, pts), eps=TOL[prec], precision=prec)
    c = plan.adjoint(dev(torch, y, rd)).cpu().numpy().astype(np.complex128)
    ref = oracle.adjoint(y, pts, L)
    e = oracle.eps_eff(ref, c)
    assert e <= TOL[prec], e
    assert np.all(c[: L + 1].imag == 0)


@pytest.mark.parametrize("eps", [1e-10, 1e-6, 1e-3])
def test_dot_product_fp64_any_eps(env, eps):
    """Exact adjointness of the fast path (independent of the NUFFT tolerance)."""
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    y = np.random.default_rng(8).standard_normal(pts.shape[0])
    plan, f = run_synth(torch, nu, L, a, pts, "fp64", eps=eps)
    c = plan.adjoint(dev(torch, y)).cpu().numpy()
    lhs = float(np.dot(y, f))
    rhs = oracle.alm_dot(c, a, L)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("L,mmax,npts", [(0, 0, 100), (1, 1, 37), (2, 1, 500), (5, 5, 1), (100, 60, 12345),
                                         (129, 129, 3001), (300, 17, 2000)])
def test_small_and_ragged_fp64(env, L, mmax, npts):
    torch, nu = env
    a = W.alm_gaussian(L, seed=L + 1, mmax=mmax)
    pts = W.points_uniform(npts, seed=npts)
    _, f = run_synth(torch, nu, L, a, pts, "fp64", mmax=mmax)
    ref = oracle.synth(a, pts, L, mmax)
    assert oracle.eps_eff(ref, f) <= 1e-10
    y = np.random.default_rng(1).standard_normal(npts)
    plan = nu.Plan(L, dev(torch, pts), eps=1e-10, mmax=mmax)
    c = plan.adjoint(dev(torch, y)).cpu().numpy()
    cref = oracle.adjoint(y, pts, L, mmax)
    assert oracle.eps_eff(cref, c) <= 1e-10


def test_poles_and_any_real_coordinates(env):
    """Points on the poles, theta outside [0, pi], negative and large phi."""
    torch, nu = env
    L = 40
    a = W.alm_gaussian(L, seed=3)
    rng = np.random.default_rng(4)
    th = np.concatenate([[0.0, math.pi, 0.0, math.pi, 1e-9, math.pi - 1e-9],
                         rng.uniform(-7.0, 13.0, 300)])
    ph = np.concatenate([[0.0, 0.0, 2.0, -1.0, 0.3, 6.2], rng.uniform(-20.0, 20.0, 300)])
    pts = np.stack([th, ph], 1)
    _, f = run_synth(torch, nu, L, a, pts, "fp64")
    ref = oracle.synth(a, pts, L)
    assert oracle.eps_eff(ref, f) <= 1e-10
    assert np.max(np.abs(f - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_empty_point_set(env):
    torch, nu = env
    L = 10
    plan = nu.Plan(L, torch.zeros((0, 2), dtype=torch.float64, device="cuda"), eps=1e-8)
    a = dev(torch, W.alm_gaussian(L, seed=1))
    f = plan.synth(a)
    assert f.numel() == 0
    c = plan.adjoint(torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(c).item() == 0


def test_repeated_calls_are_identical(env):
    """Synthesis is bit-reproducible (no atomics); the adjoint's halo flush adds
    tiles with atomics, so two calls agree to rounding only: the FP64 fine-grid
    FFT splits each grid value into a float pair (~2^-48 relative), so an
    order-of-summation difference in the last bits of a cell shows up at that
    level, not at 2^-53."""
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    plan = nu.Plan(L, dev(torch, pts), eps=1e-10)
    ad = dev(torch, a)
    f1 = plan.synth(ad).clone()
    f2 = plan.synth(ad).clone()
    assert torch.equal(f1, f2)
    c1 = plan.adjoint(f1).clone()
    c2 = plan.adjoint(f1).clone()
    assert (torch.linalg.norm(c1 - c2) / torch.linalg.norm(c1)).item() <= 1e-13


def test_setpts_replaces_points(env):
    torch, nu = env
    L = 30
    a = W.alm_gaussian(L, seed=2)
    p1 = W.points_uniform(1000, seed=1)
    p2 = W.points_uniform(3000, seed=2)
    plan = nu.Plan(L, dev(torch, p1), eps=1e-10)
    plan.setpts(dev(torch, p2))
    f = plan.synth(dev(torch, a)).cpu().numpy()
    assert oracle.eps_eff(oracle.synth(a, p2, L), f) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_setpts_changes_the_rows_reached(env, prec):
    """The row passes of the fine-grid FFT transform only the rows the points'
    taps reach, a set fixed by setpts (with T zeroed elsewhere).  A plan
    re-pointed from a narrow theta band to another band, then to uniform
    points half of which are given as their doubled-torus twins
    (2 pi - theta, phi + pi) (rows in the other half of the grid), matches
    the oracle after every change, synthesis and adjoint."""
    torch, nu = env
    L = 60
    rng = np.random.default_rng(5)

    def band(lo, hi, n):
        return np.stack([rng.uniform(lo, hi, n), rng.uniform(0.0, 2 * np.pi, n)], 1)

    a = W.alm_gaussian(L, seed=3)
    p1, p2 = band(0.2, 0.5, 4000), band(2.0, 2.8, 5000)
    p3 = W.points_uniform(6000, seed=4)
    twin = p3.copy()
    half = rng.random(p3.shape[0]) < 0.5
    twin[half, 0] = 2 * np.pi - p3[half, 0]
    twin[half, 1] = p3[half, 1] + np.pi
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    rd = torch.float64 if prec == "fp64" else torch.float32
    plan = nu.Plan(L, dev(torch, p1), eps=TOL[prec], precision=prec)
    ad = dev(torch, a, cd)
    for k, (given, ref_pts) in enumerate(((p1, p1), (p2, p2), (twin, p3))):
        if k > 0:
            plan.setpts(dev(torch, given))
        f = plan.synth(ad).double().cpu().numpy()
        assert oracle.eps_eff(oracle.synth(a, ref_pts, L), f) <= TOL[prec], k
        y = rng.standard_normal(given.shape[0]).astype(np.float32).astype(np.float64)
        c = plan.adjoint(dev(torch, y, rd)).cpu().numpy().astype(np.complex128)
        assert oracle.eps_eff(oracle.adjoint(y, ref_pts, L), c) <= TOL[prec], k
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gl1023_subset(env, prec):
    """lmax = 1023 on the 1024 x 2047 deflected GL grid; 10^4-point oracle subset."""
    torch, nu = env
    L, a, pts = W.workload("gl1023")
    _, f = run_synth(torch, nu, L, a, pts, prec)
    sel = W.subset(pts.shape[0], 10000)
    ref = oracle.synth(a, pts[sel], L)
    e = oracle.eps_eff(ref, f[sel])
    assert e <= TOL[prec], e


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gl1023_adjoint_msubset(env, prec):
    torch, nu = env
    L, _, pts = W.workload("gl1023")
    y = np.random.default_rng(9).standard_normal(pts.shape[0])
    rd = torch.float64 if prec == "fp64" else torch.float32
    plan = nu.Plan(L, dev(torch, pts), eps=TOL[prec], precision=prec)
    c = plan.adjoint(dev(torch, y, rd)).cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(10)
    ms = sorted({0, 1, *rng.integers(2, L + 1, 4).tolist()})
    ref = oracle.adjoint(y, pts, L, mlist=ms)
    idx = np.concatenate([np.arange(oracle.lm_index(L, m, m), oracle.lm_index(L, L, m) + 1) for m in ms])
    e = oracle.eps_eff(ref[idx], c[idx])
    assert e <= TOL[prec], e


def test_gl1023_dot_product_full(env):
    torch, nu = env
    L, a, pts = W.workload("gl1023")
    y = np.random.default_rng(11).standard_normal(pts.shape[0])
    plan, f = run_synth(torch, nu, L, a, pts, "fp64")
    c = plan.adjoint(dev(torch, y)).cpu().numpy()
    lhs = float(np.dot(y, f))
    rhs = oracle.alm_dot(c, a, L)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_legendre_table_mode(env, prec):
    """Recurrence once at plan time (table mode): same parity, synthesis and
    adjoint, and the same results as the per-call recurrence to rounding."""
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    rd = torch.float64 if prec == "fp64" else torch.float32
    dp = dev(torch, pts)
    pt = nu.Plan(L, dp, eps=TOL[prec], precision=prec, legendre_table=1)
    pr = nu.Plan(L, dp, eps=TOL[prec], precision=prec)
    ad = dev(torch, a, cd)
    f = pt.synth(ad).double().cpu().numpy()
    assert oracle.eps_eff(oracle.synth(a, pts, L), f) <= TOL[prec]
    assert oracle.eps_eff(pr.synth(ad).double().cpu().numpy(), f) <= (1e-13 if prec == "fp64" else 1e-6)
    y = np.random.default_rng(3).standard_normal(pts.shape[0])
    c = pt.adjoint(dev(torch, y, rd)).cpu().numpy().astype(np.complex128)
    assert oracle.eps_eff(oracle.adjoint(y, pts, L), c) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_legendre_table_mode_gl1023(env, prec):
    torch, nu = env
    L, a, pts = W.workload("gl1023")
    _, f = run_synth(torch, nu, L, a, pts, prec, legendre_table=1)
    sel = W.subset(pts.shape[0], 5000)
    assert oracle.eps_eff(oracle.synth(a, pts[sel], L), f[sel]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autotuned_sigma_and_bin_size(env, tmp_path, monkeypatch, prec):
    """tune=1 times the up-sampling factor and the bin size on the plan's own
    points and caches the winners; tune=2 reuses them; parity holds whichever
    are chosen."""
    torch, nu = env
    monkeypatch.setenv("NUSHT_TUNE_CACHE", str(tmp_path / "tune.txt"))
    L, a, pts = W.workload("uniform63")
    dp = dev(torch, pts)
    eps = 1e-10 if prec == "fp64" else 1e-5
    cd = np.complex128 if prec == "fp64" else np.complex64
    p1 = nu.Plan(L, dp, eps=eps, precision=prec, tune=1)
    b, sg = p1.bin_size(), p1.info()["sigma"]
    assert b in (16, 32, 64) and sg in (1.25, 1.5, 2.0)
    if prec == "fp64":
        assert sg != 1.25  # its kernel width for 1e-11 exceeds the limit
    lines = (tmp_path / "tune.txt").read_text().split("\n")
    assert any(l.startswith("S:") and l.endswith(" %d" % round(100 * sg)) for l in lines)
    f = p1.synth(dev(torch, a.astype(cd))).cpu().numpy().astype(np.float64)
    assert oracle.eps_eff(oracle.synth(a, pts, L), f) <= TOL[prec]
    y = np.random.default_rng(4).standard_normal(pts.shape[0])
    if prec == "mixed":
        y = y.astype(np.float32)
    c = p1.adjoint(dev(torch, y)).cpu().numpy().astype(np.complex128)
    assert oracle.eps_eff(oracle.adjoint(y.astype(np.float64), pts, L), c) <= TOL[prec]
    p2 = nu.Plan(L, dp, eps=eps, precision=prec, tune=2)
    assert p2.bin_size() == b and p2.info()["sigma"] == sg


@pytest.mark.parametrize("sigma", [1.5, 2.0])
def test_fp64_instruction_path_gl1023(env, sigma):
    """fp64_contraction=1: Legendre sums, interpolation and spreading with FP64
    instructions (the default runs them as float pairs on the FP32 pipe).
    Both paths against the oracle on a seeded subset, and against each other
    on every point and coefficient."""
    torch, nu = env
    L, a, pts = W.workload("gl1023")
    sel = W.subset(pts.shape[0], 3000, seed=11)
    ref = oracle.synth(a, pts[sel], L)
    dp = dev(torch, pts)
    y = dev(torch, np.random.default_rng(12).standard_normal(pts.shape[0]))
    out = {}
    for fc in (True, False):
        plan = nu.Plan(L, dp, eps=1e-10, sigma=sigma, fp64_contraction=fc)
        f = plan.synth(dev(torch, a)).cpu().numpy()
        assert oracle.eps_eff(ref, f[sel]) <= 1e-10, fc
        out[fc] = (f, plan.adjoint(y).cpu().numpy())
    (f1, c1), (f0, c0) = out[True], out[False]
    assert np.linalg.norm(f1 - f0) <= 1e-12 * np.linalg.norm(f1)
    assert np.linalg.norm(c1 - c0) <= 1e-12 * np.linalg.norm(c1)


def test_fp64_large_dynamic_range(env):
    """Float-pair arithmetic keeps FP64-class relative accuracy for coefficients
    and maps scaled by 1e15 and 1e-15 (the float exponent range is not hit)."""
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    y = np.random.default_rng(13).standard_normal(pts.shape[0])
    plan = nu.Plan(L, dev(torch, pts), eps=1e-10)
    for sc in (1e15, 1e-15):
        f = plan.synth(dev(torch, a * sc)).cpu().numpy()
        assert oracle.eps_eff(oracle.synth(a * sc, pts, L), f) <= 1e-10, sc
        c = plan.adjoint(dev(torch, y * sc)).cpu().numpy()
        assert oracle.eps_eff(oracle.adjoint(y * sc, pts, L), c) <= 1e-10, sc


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_execute_calls_capture_into_cuda_graph(env, prec):
    """nusht_synth / nusht_adjoint are stream-ordered, allocate nothing and do
    not synchronise, so they can be captured into a CUDA graph; replaying it
    gives the eager results."""
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    rd = torch.float64 if prec == "fp64" else torch.float32
    plan = nu.Plan(L, dev(torch, pts), eps=TOL[prec], precision=prec)
    ad = dev(torch, a, cd)
    y = dev(torch, np.random.default_rng(9).standard_normal(pts.shape[0]), rd)
    f = torch.empty(pts.shape[0], dtype=rd, device="cuda")
    c = torch.empty(plan.nalm, dtype=cd, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.synth(ad, out=f)
        plan.adjoint(y, out=c)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    f_eager, c_eager = f.clone(), c.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.synth(ad, out=f)
        plan.adjoint(y, out=c)
    f.zero_()
    c.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(f, f_eager)
    rel = (torch.linalg.norm(c - c_eager) / torch.linalg.norm(c_eager)).item()
    # the adjoint's spreading adds with atomics: equal to rounding in the plan's precision
    assert rel <= (1e-12 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec,sigma,kw,fc", [("fp64", 1.25, 0, False), ("fp64", 1.25, 0, True),
                                              ("fp64", 2.0, 17, False), ("mixed", 2.0, 20, False)])
def test_kernel_widths_above_16(env, prec, sigma, kw, fc):
    """Widths 17..20 (sigma = 1.25 at eps 1e-10 needs w = 19): synthesis and
    adjoint against the oracle, and the dot test, on every spreading and
    interpolation path (double-float, FP64 instructions, float)."""
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    rd = torch.float64 if prec == "fp64" else torch.float32
    plan = nu.Plan(L, dev(torch, pts), eps=TOL[prec], precision=prec, sigma=sigma, kernel_width=kw,
                   fp64_contraction=fc)
    assert plan.info()["w"] >= 17
    f = plan.synth(dev(torch, a, cd)).double().cpu().numpy()
    assert oracle.eps_eff(oracle.synth(a, pts, L), f) <= TOL[prec]
    y = np.random.default_rng(14).standard_normal(pts.shape[0])
    if prec == "mixed":
        y = y.astype(np.float32).astype(np.float64)
    c = plan.adjoint(dev(torch, y, rd)).cpu().numpy().astype(np.complex128)
    assert oracle.eps_eff(oracle.adjoint(y, pts, L), c) <= TOL[prec]
    lhs = float(np.dot(y, f))
    rhs = oracle.alm_dot(c, a, L)
    # at sigma = 1.25 the deconvolution factors 1 / psihat near the band edge
    # are large and amplify rounding in both directions alike: 1e-11 there
    dtol = 1e-5 if prec == "mixed" else (1e-11 if sigma < 1.4 else 1e-12)
    assert abs(lhs - rhs) <= dtol * abs(lhs)


@pytest.mark.parametrize("prec,fc,n", [("fp64", False, 20000), ("fp64", True, 20000), ("mixed", False, 20000),
                                       ("fp64", False, 3001)])
def test_deterministic_adjoint(env, prec, fc, n):
    """opts.deterministic: the adjoint is bit-reproducible (tiles summed per
    grid cell in a fixed order, no atomics) and agrees with the oracle and
    with the atomic path to rounding; includes a grid whose last bin is
    partial (lmax 129 -> n = 392 at sigma 1.5)."""
    torch, nu = env
    L = 63 if n == 20000 else 129
    a = W.alm_gaussian(L, seed=1)
    pts = W.points_uniform(n, seed=n + 1)
    rd = torch.float64 if prec == "fp64" else torch.float32
    y = np.random.default_rng(15).standard_normal(n)
    if prec == "mixed":
        y = y.astype(np.float32).astype(np.float64)
    dy = dev(torch, y, rd)
    pd = nu.Plan(L, dev(torch, pts), eps=TOL[prec], precision=prec, fp64_contraction=fc, deterministic=True)
    c1 = pd.adjoint(dy).clone()
    c2 = pd.adjoint(dy).clone()
    assert torch.equal(c1, c2)
    got = c1.cpu().numpy().astype(np.complex128)
    assert oracle.eps_eff(oracle.adjoint(y, pts, L), got) <= TOL[prec]
    pa = nu.Plan(L, dev(torch, pts), eps=TOL[prec], precision=prec, fp64_contraction=fc)
    ca = pa.adjoint(dy).cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ca) <= (1e-12 if prec == "fp64" else 1e-5) * np.linalg.norm(ca)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fast_recurrence(env, prec):
    """opts.fast_recurrence: the P_lm recurrence in double-float on the FP32
    pipe.  Synthesis on a seeded subset and the adjoint on an order subset
    against the oracle at the plan's tolerance (lmax 1023 on the deflected
    grid, where orders run into the scaled-exponent phase), the dot test, and
    agreement with the FP64 recurrence."""
    torch, nu = env
    L, a, pts = W.workload("gl1023")
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    rd = torch.float64 if prec == "fp64" else torch.float32
    dp = dev(torch, pts)
    plan = nu.Plan(L, dp, eps=TOL[prec], precision=prec, fast_recurrence=True)
    ref_plan = nu.Plan(L, dp, eps=TOL[prec], precision=prec)
    ad = dev(torch, a, cd)
    f = plan.synth(ad).double().cpu().numpy()
    sel = W.subset(pts.shape[0], 3000, seed=16)
    assert oracle.eps_eff(oracle.synth(a, pts[sel], L), f[sel]) <= TOL[prec]
    f0 = ref_plan.synth(ad).double().cpu().numpy()
    assert np.linalg.norm(f - f0) <= (1e-11 if prec == "fp64" else 3e-6) * np.linalg.norm(f0)
    y = np.random.default_rng(17).standard_normal(pts.shape[0])
    if prec == "mixed":
        y = y.astype(np.float32).astype(np.float64)
    c = plan.adjoint(dev(torch, y, rd)).cpu().numpy().astype(np.complex128)
    ms = [0, 1, 300, 700, 1023]
    ref = oracle.adjoint(y, pts, L, mlist=ms)
    idx = np.concatenate([np.arange(oracle.lm_index(L, m, m), oracle.lm_index(L, L, m) + 1) for m in ms])
    assert oracle.eps_eff(ref[idx], c[idx]) <= TOL[prec]
    if prec == "fp64":
        lhs = float(np.dot(y, f))
        rhs = oracle.alm_dot(c, a, L)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("L,npts", [(0, 50), (1, 200), (5, 999), (100, 20000), (200, 30001), (1023, 200000)])
def test_fp64_fft_kernels(env, L, npts):
    """opts.fft_kernels: the double-float theta and fine-grid FFT kernels
    (default in FP64) against cuFFT's FP64 transforms (fft_kernels = -1), on
    lengths with every radix (L = 5: n = 28 = 4 * 7; L = 100: M = 216,
    n = 320; L = 200: M = 420 = 4 * 3 * 5 * 7, n = 630 = 2 * 9 * 5 * 7),
    plus the oracle on a seeded subset and the adjoint dot test."""
    torch, nu = env
    pts = W.points_uniform(npts, seed=31 + L)
    a = W.alm_gaussian(L, seed=32 + L)
    dp = dev(torch, pts)
    own = nu.Plan(L, dp, eps=1e-10, precision="fp64")
    cuf = nu.Plan(L, dp, eps=1e-10, precision="fp64", fft_kernels=-1)
    ad = dev(torch, a, torch.complex128)
    f = own.synth(ad).cpu().numpy()
    f0 = cuf.synth(ad).cpu().numpy()
    assert np.linalg.norm(f - f0) <= 1e-12 * np.linalg.norm(f0)
    y = np.random.default_rng(33 + L).standard_normal(npts)
    yd = dev(torch, y)
    c = own.adjoint(yd).cpu().numpy()
    c0 = cuf.adjoint(yd).cpu().numpy()
    assert np.linalg.norm(c - c0) <= 1e-12 * np.linalg.norm(c0)
    sel = W.subset(npts, min(npts, 400), seed=34)
    assert oracle.eps_eff(oracle.synth(a, pts[sel], L), f[sel]) <= TOL["fp64"]
    if L <= 200:
        assert oracle.eps_eff(oracle.adjoint(y, pts, L), c) <= TOL["fp64"]
    lhs = float(np.dot(y, f))
    rhs = oracle.alm_dot(c, a, L)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300)


def test_fp64_fft_kernels_theta_only(env):
    """A fine grid longer than a shared-memory line (sigma = 4 at lmax 2047:
    n = 16384 > 14336) takes cuFFT FP64 for the 2D transform while the theta
    DFT (M = 4096) stays on the double-float kernel, which then hands the
    theta spectrum over as double2: against cuFFT throughout and the oracle."""
    torch, nu = env
    L = 2047
    pts = W.points_uniform(100000, seed=61)
    a = W.alm_gaussian(L, seed=62, spectrum="inv_l1_sq")
    dp = dev(torch, pts)
    own = nu.Plan(L, dp, eps=1e-10, precision="fp64", sigma=4.0)
    assert own.info()["n1"] > 14336
    cuf = nu.Plan(L, dp, eps=1e-10, precision="fp64", sigma=4.0, fft_kernels=-1)
    ad = dev(torch, a, torch.complex128)
    f = own.synth(ad).cpu().numpy()
    f0 = cuf.synth(ad).cpu().numpy()
    assert np.linalg.norm(f - f0) <= 1e-12 * np.linalg.norm(f0)
    y = np.random.default_rng(63).standard_normal(pts.shape[0])
    yd = dev(torch, y)
    c = own.adjoint(yd).cpu().numpy()
    c0 = cuf.adjoint(yd).cpu().numpy()
    assert np.linalg.norm(c - c0) <= 1e-12 * np.linalg.norm(c0)
    sel = W.subset(pts.shape[0], 200, seed=64)
    assert oracle.eps_eff(oracle.synth(a, pts[sel], L), f[sel]) <= TOL["fp64"]


@pytest.mark.parametrize("L,npts,sigma", [(5, 3000, 0.0), (100, 20000, 0.0), (200, 40000, 1.5), (1023, 200000, 0.0)])
def test_fp32_fft_kernels(env, L, npts, sigma):
    """Mixed plans: this library's FP32 fine-grid FFT kernels (fft_kernels =
    1, the default where the lengths fit; deconvolution fused into the column
    pass; only the row pairs the points reach) against cuFFT's 2D FP32
    transforms and the separate deconvolution kernels (fft_kernels = -1), on
    lengths with every radix (n = 24 = 8 * 3, 420 = 4 * 3 * 5 * 7,
    630 = 2 * 9 * 5 * 7 at sigma 1.5, 4096), the oracle on a seeded subset,
    and the dot test (relative to |y| |f|, float rounding)."""
    torch, nu = env
    pts = W.points_uniform(npts, seed=71 + L)
    a = W.alm_gaussian(L, seed=72 + L)
    dp = dev(torch, pts)
    own = nu.Plan(L, dp, eps=1e-5, precision="mixed", sigma=sigma, fft_kernels=1)
    cuf = nu.Plan(L, dp, eps=1e-5, precision="mixed", sigma=sigma, fft_kernels=-1)
    assert own.info()["n1"] == cuf.info()["n1"]
    ad = dev(torch, a, torch.complex64)
    f = own.synth(ad).double().cpu().numpy()
    f0 = cuf.synth(ad).double().cpu().numpy()
    assert np.linalg.norm(f - f0) <= 2e-6 * np.linalg.norm(f0)
    y = np.random.default_rng(73 + L).standard_normal(npts).astype(np.float32)
    yd = dev(torch, y)
    c = own.adjoint(yd).cpu().numpy().astype(np.complex128)
    c0 = cuf.adjoint(yd).cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(c - c0) <= 2e-6 * np.linalg.norm(c0)
    sel = W.subset(npts, min(npts, 400), seed=74)
    assert oracle.eps_eff(oracle.synth(a, pts[sel], L), f[sel]) <= TOL["mixed"]
    if L <= 200:
        assert oracle.eps_eff(oracle.adjoint(y.astype(np.float64), pts, L), c) <= TOL["mixed"]
    lhs = float(np.dot(y.astype(np.float64), f))
    rhs = oracle.alm_dot(c, a.astype(np.complex64).astype(np.complex128), L)
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(y) * np.linalg.norm(f)
