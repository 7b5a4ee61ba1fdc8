"""Batched transforms (many uneven lmax and point counts in one plan, mixed
precision) against the oracle, member by member, at the mixed tolerance
eps_eff <= 1e-5; plus graph re-capture when the buffers change and the
adjoint dot test."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14542_gb300 import build

    build.build()
    import paper_2406_14542_gb300 as nu

    return torch, nu


def make_batch(torch, nu, ls, seed=0, table=0, tc=0):
    alms = [W.alm_gaussian(l, seed=seed + 10 * i, dtype=np.complex64) for i, l in enumerate(ls)]
    pts = [W.points_uniform(max(1, 2 * l * l), seed=seed + 10 * i + 1) for i, l in enumerate(ls)]
    bp = nu.BatchPlan(ls, [torch.from_numpy(p).cuda() for p in pts], eps=1e-5, legendre_table=table,
                      tensor_cores=tc)
    return bp, alms, pts


# contraction paths: 2 = tensor cores (table), 1 = CUDA-core FP32 (table),
# 0 = CUDA-core FP32 with the recurrence on every call
PATHS = [(0, 0, 2), (0, -1, 1), (-1, 0, 0)]


@pytest.mark.parametrize("table,tc,path", PATHS)
def test_batch_small_against_oracle(env, table, tc, path):
    """Every Legendre contraction path against the oracle."""
    torch, nu = env
    ls = [0, 3, 16, 40, 63, 100, 130, 7]
    bp, alms, pts = make_batch(torch, nu, ls, table=table, tc=tc)
    info = bp.info()
    assert info["nbuckets"] >= 1 and max(info["bucket_lmax"]) == max(ls)
    assert info["paths"] == [path] * info["nbuckets"]
    outs = bp.synth([torch.from_numpy(a).cuda() for a in alms])
    torch.cuda.synchronize()
    for l, a, p, f in zip(ls, alms, pts, outs):
        sel = W.subset(p.shape[0], 3000, seed=l)
        ref = oracle.synth(a.astype(np.complex128), p[sel], l)
        assert oracle.eps_eff(ref, f.double().cpu().numpy()[sel]) <= TOL, l
    ys = [np.random.default_rng(i).standard_normal(p.shape[0]) for i, p in enumerate(pts)]
    cs = bp.adjoint([torch.from_numpy(y).float().cuda() for y in ys])
    bp.status()
    for l, p, y, c in zip(ls, pts, ys, cs):
        ref = oracle.adjoint(y.astype(np.float32).astype(np.float64), p, l)
        assert oracle.eps_eff(ref, c.cpu().numpy().astype(np.complex128)) <= TOL, l


def test_batch_recapture_and_dot(env):
    """New buffers force a new graph; results and the dot test hold."""
    torch, nu = env
    ls = [20, 31, 47]
    bp, alms, pts = make_batch(torch, nu, ls, seed=5)
    ad = [torch.from_numpy(a).cuda() for a in alms]
    f1 = [x.clone() for x in bp.synth(ad)]
    f2 = bp.synth(ad)  # fresh output buffers -> re-capture
    for x, y in zip(f1, f2):
        assert torch.equal(x, y)
    gen = torch.Generator(device="cuda").manual_seed(6)
    ys = [torch.randn(p.shape[0], device="cuda", generator=gen) for p in pts]
    cs = bp.adjoint(ys)
    for l, a, f, y, c in zip(ls, alms, f1, ys, cs):
        lhs = float(torch.dot(y.double(), f.double()))
        rhs = oracle.alm_dot(c.cpu().numpy().astype(np.complex128), a.astype(np.complex128), l)
        # rounding in either side is bounded by ~eps |y| |f|; <y, f> itself
        # can cancel to |y| |f| / sqrt(N), so the bound is not relative to it
        assert abs(lhs - rhs) <= 1e-6 * float(torch.linalg.norm(y.double()) * torch.linalg.norm(f.double()))


@pytest.mark.parametrize("tc,path", [(0, 2), (-1, 1)])
def test_batch64_members_against_oracle(env, tc, path):
    """64 transforms, lmax ~ U{64..511}, N_b = 2 lmax_b^2 uniform points: the
    batch structure of the 64-transform workload at a size the oracle can
    check (several 128-pair synthesis blocks and 256-degree adjoint blocks
    per order, polar-skipped tiles); members sampled across buckets."""
    torch, nu = env
    rng = np.random.default_rng(0)
    ls = [int(x) for x in rng.integers(64, 512, 64)]
    bp, alms, pts = make_batch(torch, nu, ls, seed=100, tc=tc)
    info = bp.info()
    assert set(info["paths"]) == {path}
    outs = bp.synth([torch.from_numpy(a).cuda() for a in alms])
    torch.cuda.synchronize()
    order = np.argsort(ls)
    check = sorted({int(order[0]), int(order[len(ls) // 2]), int(order[-1])} |
                   {int(np.argmax(np.array(info["bucket_of"]) == b)) for b in range(info["nbuckets"])})
    for i in check:
        sel = W.subset(pts[i].shape[0], 1500, seed=i)
        ref = oracle.synth(alms[i].astype(np.complex128), pts[i][sel], ls[i])
        assert oracle.eps_eff(ref, outs[i].double().cpu().numpy()[sel]) <= TOL, (i, ls[i])
    gen = torch.Generator(device="cuda").manual_seed(7)
    ys = [torch.randn(p.shape[0], device="cuda", generator=gen) for p in pts]
    cs = bp.adjoint(ys)
    bp.status()
    for i in check[:3]:
        l = ls[i]
        ms = [0, 1, l // 2, l]
        ref = oracle.adjoint(ys[i].double().cpu().numpy(), pts[i], l, mlist=ms)
        idx = np.concatenate([np.arange(oracle.lm_index(l, m, m), oracle.lm_index(l, l, m) + 1) for m in ms])
        got = cs[i].cpu().numpy().astype(np.complex128)
        assert oracle.eps_eff(ref[idx], got[idx]) <= TOL, (i, l)


def test_batch_tuned_schedule(env, tmp_path, monkeypatch):
    """opts.tune = 1 times the tensor-core contraction with 2, 4 and 8 degree
    chunks per partial accumulation for each direction (and the members'
    bin sizes), caches the choice, and tune = 2 takes it from the cache; the
    tuned batch stays within the mixed tolerance against the oracle."""
    torch, nu = env
    monkeypatch.setenv("NUSHT_TUNE_CACHE", str(tmp_path / "tune.txt"))
    ls = [40, 100, 130, 200]
    alms = [W.alm_gaussian(l, seed=80 + i, dtype=np.complex64) for i, l in enumerate(ls)]
    pts = [W.points_uniform(2 * l * l, seed=90 + i) for i, l in enumerate(ls)]
    dp = [torch.from_numpy(p).cuda() for p in pts]
    bp = nu.BatchPlan(ls, dp, eps=1e-5, tune=1)
    info = bp.info()
    assert set(info["paths"]) == {2}
    for cs, ca in info["schedule"]:
        assert cs in (2, 4, 8) and ca in (2, 4, 8)
    outs = bp.synth([torch.from_numpy(a).cuda() for a in alms])
    ys = [np.random.default_rng(95 + i).standard_normal(p.shape[0]).astype(np.float32) for i, p in enumerate(pts)]
    cs_ = bp.adjoint([torch.from_numpy(y).cuda() for y in ys])
    bp.status()
    for l, a, p, f, y, c in zip(ls, alms, pts, outs, ys, cs_):
        sel = W.subset(p.shape[0], 2000, seed=l)
        assert oracle.eps_eff(oracle.synth(a.astype(np.complex128), p[sel], l), f.double().cpu().numpy()[sel]) <= TOL
        ref = oracle.adjoint(y.astype(np.float64), p, l)
        assert oracle.eps_eff(ref, c.cpu().numpy().astype(np.complex128)) <= TOL
    assert any(line.startswith("C:") for line in (tmp_path / "tune.txt").read_text().splitlines())
    bp.close()
    again = nu.BatchPlan(ls, dp, eps=1e-5, tune=2)
    assert again.info()["schedule"] == info["schedule"]
    again.close()


def test_batch_fp32_fft_kernels(env):
    """The batch default (fft_kernels = 0): every member's fine-grid FFT by
    this library's FP32 line kernels, two launches per direction for the
    whole batch (radix 8, 4, 2 and odd 3 / 5 / 7 lengths among the members),
    against cuFFT per member (fft_kernels = -1) and the oracle."""
    torch, nu = env
    ls = [3, 16, 40, 63, 100, 130, 7, 211]
    alms = [W.alm_gaussian(l, seed=300 + 10 * i, dtype=np.complex64) for i, l in enumerate(ls)]
    pts = [W.points_uniform(2 * l * l, seed=301 + 10 * i) for i, l in enumerate(ls)]
    dpts = [torch.from_numpy(p).cuda() for p in pts]
    own = nu.BatchPlan(ls, dpts, eps=1e-5)
    cuf = nu.BatchPlan(ls, dpts, eps=1e-5, fft_kernels=-1)
    da = [torch.from_numpy(a).cuda() for a in alms]
    fo, fc = own.synth(da), cuf.synth(da)
    rng = np.random.default_rng(302)
    ys = [torch.from_numpy(rng.standard_normal(p.shape[0]).astype(np.float32)).cuda() for p in pts]
    co, cc = own.adjoint(ys), cuf.adjoint(ys)
    own.status()
    for l, a, p, f1, f0, c1, c0, y in zip(ls, alms, pts, fo, fc, co, cc, ys):
        f1, f0 = f1.double().cpu().numpy(), f0.double().cpu().numpy()
        c1 = c1.cpu().numpy().astype(np.complex128)
        c0 = c0.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(f1 - f0) <= 2e-6 * np.linalg.norm(f0), l
        assert np.linalg.norm(c1 - c0) <= 2e-6 * np.linalg.norm(c0), l
        sel = W.subset(p.shape[0], 2000, seed=l)
        assert oracle.eps_eff(oracle.synth(a.astype(np.complex128), p[sel], l), f1[sel]) <= TOL, l
        ref = oracle.adjoint(y.double().cpu().numpy(), p, l)
        assert oracle.eps_eff(ref, c1) <= TOL, l
    own.close()
    cuf.close()


def test_batch_empty_member(env):
    """Mixed precision: a member without points (NULL map pointers) beside
    others; its adjoint is zero and the others match the oracle."""
    torch, nu = env
    ls = [50, 30, 70]
    npts = [3000, 0, 3000]
    alms = [W.alm_gaussian(l, seed=80 + i, dtype=np.complex64) for i, l in enumerate(ls)]
    pts = [W.points_uniform(max(n, 1), seed=90 + i)[:n] for i, n in enumerate(npts)]
    bp = nu.BatchPlan(ls, [torch.from_numpy(p).cuda() for p in pts], eps=1e-5)
    outs = bp.synth([torch.from_numpy(a).cuda() for a in alms])
    ys = [torch.from_numpy(np.random.default_rng(95 + i).standard_normal(n).astype(np.float32)).cuda()
          for i, n in enumerate(npts)]
    cs = bp.adjoint(ys)
    torch.cuda.synchronize()
    bp.status()
    assert outs[1].numel() == 0
    assert float(cs[1].abs().max()) == 0.0
    for i in (0, 2):
        ref = oracle.synth(alms[i].astype(np.complex128), pts[i], ls[i])
        assert oracle.eps_eff(ref, outs[i].double().cpu().numpy()) <= TOL
        cref = oracle.adjoint(ys[i].double().cpu().numpy(), pts[i], ls[i])
        assert oracle.eps_eff(cref, cs[i].cpu().numpy().astype(np.complex128)) <= TOL
