"""Differentiable nuSHT: gradients in a_lm (through the adjoint) and in the
point coordinates (derivative-of-kernel interpolation on the same fine grid),
against central finite differences and the oracle's analytic dY.

Loss (the differentiable workload): L = sum_i w_i f_i^2 with seeded w_i ~ U[0, 1).
Tolerances: analytic position gradient vs oracle 1e-8 (FP64); central
differences with h = 1e-6 agree to ~1e-6 (truncation h^2 f'''/6 relative to
f' grows like lmax^2 h^2).
"""
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 1e-4)])
def test_synth_grad_against_oracle(env, prec, tol):
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    plan = nu.Plan(L, torch.from_numpy(pts).cuda(), eps=1e-10 if prec == "fp64" else 1e-5, precision=prec)
    dth, dph = plan.synth_grad(torch.from_numpy(a).to(cd).cuda())
    rth, rph = oracle.synth_grad(a, pts, L)
    assert rel(dth.double().cpu().numpy(), rth) <= tol
    assert rel(dph.double().cpu().numpy(), rph) <= tol


def test_autograd_alm_matches_adjoint_and_fd(env):
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    w = torch.from_numpy(np.random.default_rng(1).uniform(0, 1, pts.shape[0])).cuda()
    dpts = torch.from_numpy(pts).cuda()
    plan = nu.Plan(L, dpts, eps=1e-10)
    alm = torch.from_numpy(a).cuda().requires_grad_(True)
    f = nu.nusht(alm, dpts, plan)
    loss = (w * f * f).sum()
    loss.backward()
    g = alm.grad.detach()
    # analytic: w_m * adjoint(2 w f), w_0 = 1, w_{m>0} = 2 (torch's dL/dRe + i dL/dIm)
    c = plan.adjoint((2 * w * f).detach()).clone()
    c[L + 1:] *= 2
    assert (torch.linalg.norm(g - c) / torch.linalg.norm(c)).item() <= 1e-12
    # central differences along a random complex direction
    d = torch.from_numpy(W.alm_gaussian(L, seed=99)).cuda()
    d[: L + 1] += 1j * torch.from_numpy(np.random.default_rng(98).standard_normal(L + 1)).cuda()
    h = 1e-6

    def lossat(x):
        fx = plan.synth(x)
        return (w * fx * fx).sum().item()

    fd = (lossat(alm.detach() + h * d) - lossat(alm.detach() - h * d)) / (2 * h)
    an = torch.sum((torch.conj(g) * d).real).item()
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_autograd_pts_matches_fd(env):
    torch, nu = env
    L = 63
    a = W.alm_gaussian(L, seed=0)
    pts = W.points_uniform(5000, seed=3)
    w = torch.from_numpy(np.random.default_rng(1).uniform(0, 1, pts.shape[0])).cuda()
    dpts = torch.from_numpy(pts).cuda().requires_grad_(True)
    plan = nu.Plan(L, dpts.detach(), eps=1e-10)
    alm = torch.from_numpy(a).cuda()
    f = nu.nusht(alm, dpts, plan)
    (w * f * f).sum().backward()
    g = dpts.grad.detach()
    # per-point central differences (f_i depends on point i only)
    h = 1e-6
    for k in range(2):
        e = torch.zeros_like(dpts.detach())
        e[:, k] = h
        plan.setpts(dpts.detach() + e)
        fp = plan.synth(alm)
        plan.setpts(dpts.detach() - e)
        fm = plan.synth(alm)
        fd = w * (fp * fp - fm * fm) / (2 * h)
        assert (torch.linalg.norm(g[:, k] - fd) / torch.linalg.norm(fd)).item() <= 1e-6


def test_differentiable_gl2047(env):
    """lmax = 2047 on the 2048 x 4095 deflected GL grid (8.4M points):
    d L / d(theta, phi) against per-point central differences (step 1e-6) on
    all points and against the oracle's analytic derivatives on a seeded
    subset; d L / d a_lm against a directional central difference."""
    torch, nu = env
    L, a, pts = W.workload("gl2047")
    n = pts.shape[0]
    w = torch.from_numpy(np.random.default_rng(1).uniform(0, 1, n)).cuda()
    dpts = torch.from_numpy(pts).cuda().requires_grad_(True)
    plan = nu.Plan(L, dpts.detach(), eps=1e-10)
    alm = torch.from_numpy(a).cuda().requires_grad_(True)
    f = nu.nusht(alm, dpts, plan)
    (w * f * f).sum().backward()
    gp = dpts.grad.detach()
    ga = alm.grad.detach()
    fdet = f.detach()
    # oracle analytic derivative on a subset
    sel = W.subset(n, 2000, seed=5)
    rth, rph = oracle.synth_grad(a, pts[sel], L)
    gw = (2 * w * fdet).cpu().numpy()[sel]
    assert rel(gp[:, 0].cpu().numpy()[sel], gw * rth) <= 1e-8
    assert rel(gp[:, 1].cpu().numpy()[sel], gw * rph) <= 1e-8
    # per-point central differences on all points
    h = 1e-6
    for k in range(2):
        e = torch.zeros_like(dpts.detach())
        e[:, k] = h
        plan.setpts(dpts.detach() + e)
        fp = plan.synth(alm.detach())
        plan.setpts(dpts.detach() - e)
        fm = plan.synth(alm.detach())
        fd = w * (fp * fp - fm * fm) / (2 * h)
        assert (torch.linalg.norm(gp[:, k] - fd) / torch.linalg.norm(fd)).item() <= 5e-6
    plan.setpts(dpts.detach())
    d = torch.from_numpy(W.alm_gaussian(L, seed=98)).cuda()
    hh = 1e-6

    def lossat(x):
        fx = plan.synth(x)
        return (w * fx * fx).sum().item()

    fd = (lossat(alm.detach() + hh * d) - lossat(alm.detach() - hh * d)) / (2 * hh)
    an = torch.sum((torch.conj(ga) * d).real).item()
    assert abs(fd - an) <= 1e-6 * abs(an)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_gradient_entry_points(env, prec, tol):
    """nusht_adjoint_grad = the adjoint with the m > 0 entries doubled, and
    nusht_synth_grad_pts = the cotangent times nusht_synth_grad, through the
    C ABI (the autograd backward calls only these two)."""
    torch, nu = env
    L, a, pts = W.workload("uniform63")
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    rd = torch.float64 if prec == "fp64" else torch.float32
    plan = nu.Plan(L, torch.from_numpy(pts).cuda(), eps=1e-10 if prec == "fp64" else 1e-5, precision=prec,
                   deterministic=True)
    g = torch.from_numpy(np.random.default_rng(4).standard_normal(pts.shape[0])).to(rd).cuda()
    ga = plan.adjoint_grad(g).cpu().numpy().astype(np.complex128)
    c = plan.adjoint(g).cpu().numpy().astype(np.complex128)
    c[L + 1:] *= 2.0
    assert rel(ga, c) <= tol
    assert np.all(ga[: L + 1].imag == 0)
    alm = torch.from_numpy(a).to(cd).cuda()
    gp = plan.synth_grad_pts(alm, g).cpu().numpy()
    dth, dph = plan.synth_grad(alm)
    gd = g.double().cpu().numpy()
    assert rel(gp[:, 0], gd * dth.double().cpu().numpy()) <= tol
    assert rel(gp[:, 1], gd * dph.double().cpu().numpy()) <= tol
    # against the oracle: w_m (Y^dagger g) and g * analytic derivative
    ref = oracle.adjoint(gd, pts, L)
    ref[L + 1:] *= 2.0
    assert rel(ga, ref) <= (1e-10 if prec == "fp64" else 1e-5)
    rth, rph = oracle.synth_grad(a, pts, L)
    assert rel(gp[:, 0], gd * rth) <= (1e-8 if prec == "fp64" else 1e-4)
    assert rel(gp[:, 1], gd * rph) <= (1e-8 if prec == "fp64" else 1e-4)
    plan.close()
