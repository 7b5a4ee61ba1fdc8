"""GPU parity of the CMB lensing pointing routine (App. C, Eq. pointing and
Eq. spin1deriv) against the oracle's pointing on the same seeded inputs.

The deflected unit vectors are compared: || n'_gpu - n'_oracle ||_2 over the
point set, relative to the deflection || n'_oracle - n ||_2.  Its error is
that of the interpolated gradient (derivative-of-kernel interpolation at the
plan's eps), with the relative l2 bounds of nusht_synth_grad's tests: 1e-8 in
FP64, 1e-4 in mixed mode.  (Per point, azimuths near the poles are
ill-conditioned: a position error e moves phi' by ~e / sin(theta').)
"""
import math

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


def unit(p):
    th, ph = p[:, 0], p[:, 1]
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)


def chord_error(got, ref, pts):
    """|| n'_got - n'_ref ||_2 / || n'_ref - n ||_2 over the point set"""
    return float(np.linalg.norm(unit(got) - unit(ref)) / np.linalg.norm(unit(ref) - unit(pts)))


@pytest.mark.parametrize("prec,eps,tol,fc", [("fp64", 1e-10, 1e-8, False), ("fp64", 1e-10, 1e-8, True),
                                             ("mixed", 1e-5, 1e-4, False)])
def test_pointing_against_oracle(env, prec, eps, tol, fc):
    """fc: fp64_contraction = 1, the FP64-instruction derivative interpolation
    (kernel values evaluated on the fly) instead of the double-float one."""
    torch, nu = env
    L = 63
    pts = W.points_uniform(20000, seed=41)
    phi = W.phi_lensing(L, seed=42)
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    plan = nu.Plan(L, torch.from_numpy(pts).cuda(), eps=eps, precision=prec, fp64_contraction=fc)
    got = plan.pointing(torch.from_numpy(phi).to(cd).cuda()).cpu().numpy()
    ref = oracle.pointing(phi, pts, L)
    assert np.all((got[:, 0] >= 0) & (got[:, 0] <= math.pi))
    assert np.all((got[:, 1] >= 0) & (got[:, 1] < 2 * math.pi))
    assert chord_error(got, ref, pts) <= tol


def test_pointing_gl_grid_subset(env):
    """The paper's use: the undeflected Gauss-Legendre ring grid at lmax 1023
    (2,096,128 points) and a lensing potential of 2.5 arcmin rms deflection;
    a seeded subset against the oracle."""
    torch, nu = env
    L = 1023
    pts = W.gl_ring_grid(L + 1, 2 * L + 1)
    phi = W.phi_lensing(L, seed=43)
    plan = nu.Plan(L, torch.from_numpy(pts).cuda(), eps=1e-10, precision="fp64")
    got = plan.pointing(torch.from_numpy(phi).cuda()).cpu().numpy()
    sel = W.subset(pts.shape[0], 2000, seed=44)
    ref = oracle.pointing(phi, pts[sel], L)
    assert chord_error(got[sel], ref, pts[sel]) <= 1e-8


def test_pointing_y10_closed_form(env):
    """Phi = a10 Y_10: a pure meridional shift theta' = theta - a10 sqrt(3/4pi) sin(theta)."""
    torch, nu = env
    L = 8
    a10 = 1e-3
    phi = np.zeros(nu.nalm(L), dtype=np.complex128)
    phi[oracle.lm_index(L, 1, 0)] = a10
    pts = W.points_uniform(5000, seed=45)
    plan = nu.Plan(L, torch.from_numpy(pts).cuda(), eps=1e-10, precision="fp64")
    got = plan.pointing(torch.from_numpy(phi).cuda()).cpu().numpy()
    shift = a10 * math.sqrt(3.0 / (4.0 * math.pi)) * np.sin(pts[:, 0])
    np.testing.assert_allclose(got[:, 0], pts[:, 0] - shift, rtol=0, atol=1e-8 * np.max(shift))
    ref = np.stack([pts[:, 0] - shift, pts[:, 1]], 1)
    assert np.max(np.linalg.norm(unit(got) - unit(ref), axis=1)) <= 1e-8 * np.max(shift)


def test_pointing_empty_point_set(env):
    torch, nu = env
    plan = nu.Plan(16, torch.zeros((0, 2), dtype=torch.float64, device="cuda"), eps=1e-10)
    out = plan.pointing(torch.zeros(nu.nalm(16), dtype=torch.complex128, device="cuda"))
    assert tuple(out.shape) == (0, 2)
