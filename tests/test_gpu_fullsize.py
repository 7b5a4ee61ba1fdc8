"""Parity at the benchmark's full size, in the configuration bench.py times:
lmax = mmax = 4095 on the 4096 x 8191 deflected Gauss-Legendre grid
(33,550,336 points), default plan options.

* synthesis on a seeded sample of points against the oracle's direct sum
  (eps_eff <= 1e-10 in FP64, <= 1e-5 in mixed mode);
* the adjoint through the full-size dot test <y, S a> = <S^H y, a>, since a
  full-N oracle adjoint is O(L^2 N) = 5.6e14 operations.  For random y the
  inner product is only ~ |y| |S a| / sqrt(N) (sqrt(N) = 5.8e3), so the
  bound is taken relative to |y| |S a|: 1e-13 in FP64 (spreading and
  interpolation use the same kernel values; only rounding differs),
  1e-6 in mixed mode (float rounding).
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

    L, a, pts = W.workload("gl4095")
    return torch, nu, L, a, pts


@pytest.mark.parametrize("prec,eps,tol,dot_tol", [("fp64", 1e-10, 1e-10, 1e-13), ("mixed", 1e-5, 1e-5, 1e-6)])
def test_gl4095_synthesis_sample_and_dot(env, prec, eps, tol, dot_tol):
    torch, nu, L, a, pts = env
    n = pts.shape[0]
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    rd = torch.float64 if prec == "fp64" else torch.float32
    plan = nu.Plan(L, torch.from_numpy(pts).cuda(), eps=eps, precision=prec)
    ad = torch.from_numpy(a).to(cd).cuda()
    f = plan.synth(ad).double().cpu().numpy()
    sel = W.subset(n, 256, seed=51)
    assert oracle.eps_eff(oracle.synth(a, pts[sel], L), f[sel]) <= tol
    y = np.random.default_rng(52).standard_normal(n)
    if prec == "mixed":
        y = y.astype(np.float32).astype(np.float64)
    c = plan.adjoint(torch.from_numpy(y).to(rd).cuda()).cpu().numpy().astype(np.complex128)
    a_used = a.astype(np.complex64).astype(np.complex128) if prec == "mixed" else a
    lhs = float(np.dot(y, f))
    rhs = oracle.alm_dot(c, a_used, L)
    assert abs(lhs - rhs) <= dot_tol * np.linalg.norm(y) * np.linalg.norm(f)
    plan.close()
