"""FP64 batched transforms (uneven lmax and point counts in one plan, the
Legendre contraction split into bf16 slices on the tensor cores) against the
oracle, member by member, at the FP64 tolerance eps_eff <= 1e-10; both
column groups of a bucket (more than 32 members); points at the poles; the
adjoint dot test and repeatability."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14542_gb300 import build

    build.build()
    import paper_2406_14542_gb300 as nu

    return torch, nu


def make_batch(torch, nu, ls, seed=0, npts=None):
    alms = [W.alm_gaussian(l, seed=seed + 10 * i) for i, l in enumerate(ls)]
    pts = [W.points_uniform(npts or max(1, 2 * l * l), seed=seed + 10 * i + 1) for i, l in enumerate(ls)]
    bp = nu.BatchPlan(ls, [torch.from_numpy(p).cuda() for p in pts], eps=1e-10, precision="fp64")
    return bp, alms, pts


def check_members(torch, bp, ls, alms, pts, which, nsub=2000):
    outs = bp.synth([torch.from_numpy(a).cuda() for a in alms])
    torch.cuda.synchronize()
    bp.status()
    ys = [np.random.default_rng(100 + i).standard_normal(p.shape[0]) for i, p in enumerate(pts)]
    cs = bp.adjoint([torch.from_numpy(y).cuda() for y in ys])
    torch.cuda.synchronize()
    bp.status()
    worst = 0.0
    for i in which:
        l, a, p, f = ls[i], alms[i], pts[i], outs[i]
        sel = W.subset(p.shape[0], nsub, seed=l + i)
        ref = oracle.synth(a, p[sel], l)
        got = f.cpu().numpy()[sel]
        e = oracle.eps_eff(ref, got)
        worst = max(worst, e)
        assert e <= TOL, ("synthesis", i, l, e)
        assert np.max(np.abs(got - ref)) <= 10 * TOL * np.max(np.abs(ref)), ("synthesis max", i, l)
        cref = oracle.adjoint(ys[i], p, l)
        e = oracle.eps_eff(cref, cs[i].cpu().numpy())
        worst = max(worst, e)
        assert e <= TOL, ("adjoint", i, l, e)
    print("eps_eff worst", worst)
    return outs, cs


def test_batch_fp64_small_against_oracle(env):
    """Uneven members (lmax 0 .. 130) in one or more buckets: every member."""
    torch, nu = env
    ls = [0, 3, 16, 40, 63, 100, 130, 7]
    bp, alms, pts = make_batch(torch, nu, ls)
    info = bp.info()
    assert info["paths"] == [3] * info["nbuckets"]
    check_members(torch, bp, ls, alms, pts, range(len(ls)))


def test_batch_fp64_two_column_groups(env):
    """40 members of one bucket: members 0-31 and 32-39 use the two column groups."""
    torch, nu = env
    rng = np.random.default_rng(3)
    ls = [int(v) for v in rng.integers(60, 97, 40)]
    ls[0] = 96
    bp, alms, pts = make_batch(torch, nu, ls, seed=11, npts=3000)
    info = bp.info()
    assert info["nbuckets"] == 1 and info["paths"] == [3]
    check_members(torch, bp, ls, alms, pts, [0, 1, 17, 31, 32, 38, 39])


def test_batch_fp64_polar_points(env):
    """Every point within 0.05 rad of a pole: the pole rings and the high
    orders' small values near the poles."""
    torch, nu = env
    ls = [255, 200]
    rng = np.random.default_rng(5)
    pts = []
    for k, l in enumerate(ls):
        n = 4000
        th = np.concatenate([rng.uniform(0, 0.05, n // 2), np.pi - rng.uniform(0, 0.05, n - n // 2)])
        ph = rng.uniform(0, 2 * np.pi, n)
        pts.append(np.stack([th, ph], axis=1))
    alms = [W.alm_gaussian(l, seed=40 + k) for k, l in enumerate(ls)]
    bp = nu.BatchPlan(ls, [torch.from_numpy(p).cuda() for p in pts], eps=1e-10, precision="fp64")
    check_members(torch, bp, ls, alms, pts, [0, 1])


def test_batch_fp64_dot_and_repeat(env):
    """<y, S a> = <S^T y, a> to FP64 rounding; a second synthesis is
    bit-identical; a second adjoint agrees to 1e-11 of the largest
    coefficient: the spreading adds with atomics in an arbitrary order, and a
    last-bit change of the folded spectrum can move a slice digit by one unit
    (2^-39 of its column's scale).  With deterministic spreading the adjoint
    is bit-identical too."""
    torch, nu = env
    ls = [31, 64, 47]
    bp, alms, pts = make_batch(torch, nu, ls, seed=21)
    ad = [torch.from_numpy(a).cuda() for a in alms]
    f1 = [x.clone() for x in bp.synth(ad)]
    f2 = bp.synth(ad)
    for x, y in zip(f1, f2):
        assert torch.equal(x, y)
    gen = torch.Generator(device="cuda").manual_seed(6)
    ys = [torch.randn(p.shape[0], device="cuda", dtype=torch.float64, generator=gen) for p in pts]
    cs = bp.adjoint(ys)
    cs2 = bp.adjoint(ys, outs=[torch.empty_like(c) for c in cs])
    for c, c2 in zip(cs, cs2):
        assert float((c - c2).abs().max()) <= 1e-11 * float(c.abs().max())
    for l, a, f, y, c in zip(ls, alms, f1, ys, cs):
        lhs = float(torch.dot(y, f))
        rhs = oracle.alm_dot(c.cpu().numpy(), a, l)
        scale = float(torch.linalg.norm(y)) * float(torch.linalg.norm(f))
        assert abs(lhs - rhs) <= 1e-10 * scale, (l, lhs, rhs)


def test_batch_fp64_mid_size(env):
    """64 members, lmax U{64..511}: the largest member, and members from each
    bucket, against the oracle on point subsets."""
    torch, nu = env
    rng = np.random.default_rng(7)
    ls = [int(v) for v in rng.integers(64, 512, 64)]
    ls[5] = 511
    bp, alms, pts = make_batch(torch, nu, ls, seed=31, npts=8000)
    info = bp.info()
    assert set(info["paths"]) == {3}
    which = [5]
    for g in range(info["nbuckets"]):
        which.append([i for i in range(len(ls)) if info["bucket_of"][i] == g][0])
    check_members(torch, bp, ls, alms, pts, sorted(set(which)), nsub=1000)


def test_batch_fp64_deterministic_adjoint(env):
    """opts.deterministic: the adjoint of an FP64 batched plan is bit-identical
    from call to call and still meets the tolerance."""
    torch, nu = env
    ls = [40, 90]
    pts = [W.points_uniform(4000, seed=60 + k) for k in range(2)]
    bp = nu.BatchPlan(ls, [torch.from_numpy(p).cuda() for p in pts], eps=1e-10, precision="fp64",
                      deterministic=True)
    ys = [torch.from_numpy(np.random.default_rng(61 + k).standard_normal(4000)).cuda() for k in range(2)]
    c1 = [c.clone() for c in bp.adjoint(ys)]
    c2 = bp.adjoint(ys, outs=[torch.empty_like(c) for c in c1])
    bp.status()
    for l, p, y, a, b in zip(ls, pts, ys, c1, c2):
        assert torch.equal(a, b)
        assert oracle.eps_eff(oracle.adjoint(y.cpu().numpy(), p, l), a.cpu().numpy()) <= TOL


def test_batch_fp64_empty_member(env):
    """A member without points sits in the batch with the others: its
    synthesis writes nothing, its adjoint gives zeros, and the other members
    still match the oracle."""
    torch, nu = env
    ls = [50, 30, 70]
    npts = [3000, 0, 3000]
    alms = [W.alm_gaussian(l, seed=80 + i) for i, l in enumerate(ls)]
    pts = [W.points_uniform(max(n, 1), seed=90 + i)[:n] for i, n in enumerate(npts)]
    bp = nu.BatchPlan(ls, [torch.from_numpy(p).cuda() for p in pts], eps=1e-10, precision="fp64")
    outs = bp.synth([torch.from_numpy(a).cuda() for a in alms])
    ys = [torch.from_numpy(np.random.default_rng(95 + i).standard_normal(n)).cuda() for i, n in enumerate(npts)]
    cs = bp.adjoint(ys)
    torch.cuda.synchronize()
    bp.status()
    assert outs[1].numel() == 0
    assert float(cs[1].abs().max()) == 0.0
    for i in (0, 2):
        assert oracle.eps_eff(oracle.synth(alms[i], pts[i], ls[i]), outs[i].cpu().numpy()) <= TOL
        assert oracle.eps_eff(oracle.adjoint(ys[i].cpu().numpy(), pts[i], ls[i]), cs[i].cpu().numpy()) <= TOL
