"""Pins of the oracle's spin-weighted harmonics and spin transforms (CPU).

sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi}
(the spin-n generalisation named in the Conclusion, Sec. 5).  The oracle
computes d^l by a recurrence in l from a closed-form start; these tests pin it
to things computed another way:

* spin 0 equals the oracle's spin-0 Pbar_lm (itself pinned elsewhere);
* Wigner's explicit sum for d^l_{m m'} in mpmath at 40 digits (small l);
* spin 1 equals the spin-raising / lowering operators applied to Y_lm,
  1Y = eth Y / sqrt(l(l+1)), -1Y = -ethbar Y / sqrt(l(l+1)), with the
  derivatives from the oracle's analytic spin-0 gradient (a separate code
  path: the ladder relation for dPbar/dtheta);
* the spin-1 synthesis equals -(d/dtheta + (i/sin theta) d/dphi) applied to
  two scalar potentials (G and C parts);
* closed forms 1Y_10, 2Y_20, 2Y_22;
* the spin addition theorem sum_m |sY_lm|^2 = (2l+1)/(4 pi) up to l = 2047,
  near the poles too (normalisation and underflow handling);
* Gauss-Legendre orthogonality of the lambda^(s)_lm over l for fixed (m, s);
* the adjoint dot test and order-subset consistency of the spin adjoint.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

mpmath = pytest.importorskip("mpmath")


def wigner_d_mp(l, mp_, m, beta):
    """d^l_{mp_, m}(beta) from Wigner's explicit sum (40 digits)."""
    mpmath.mp.dps = 40
    b = mpmath.mpf(beta) / 2
    c, s = mpmath.cos(b), mpmath.sin(b)
    f = mpmath.factorial
    pre = mpmath.sqrt(f(l + mp_) * f(l - mp_) * f(l + m) * f(l - m))
    tot = mpmath.mpf(0)
    for k in range(0, 2 * l + 1):
        a1, a2, a3, a4 = l + m - k, k, mp_ - m + k, l - mp_ - k
        if min(a1, a2, a3, a4) < 0:
            continue
        tot += (-1) ** (mp_ - m + k) / (f(a1) * f(a2) * f(a3) * f(a4)) * c ** (2 * l + m - mp_ - 2 * k) * \
            s ** (mp_ - m + 2 * k)
    return pre * tot


def lam_mp(l, m, s, theta):
    return (-1) ** s * mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi)) * wigner_d_mp(l, m, -s, theta)


@pytest.mark.parametrize("theta", [0.013, 0.7, 1.5707963, 2.9])
def test_spin0_is_the_scalar_harmonic(theta):
    # two different recurrences (the Wigner-d one and the spin-0 one): they
    # agree to the rounding of l steps
    lp, lm = oracle.spin_lambda(60, 0, theta)
    ref = oracle.plm_all(60, theta)
    assert np.abs(lp - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(lm - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("s", [1, 2, 3])
def test_against_wigner_explicit_sum(s):
    L = 14
    for theta in (0.31, 1.2, 2.71):
        lp, lm = oracle.spin_lambda(L, s, theta)
        for m in range(L + 1):
            for l in range(max(m, s), L + 1):
                i = oracle.lm_index(L, l, m)
                assert abs(lp[i] - float(lam_mp(l, m, s, theta))) <= 1e-13, (s, l, m, theta)
                assert abs(lm[i] - float(lam_mp(l, m, -s, theta))) <= 1e-13, (s, l, m, theta)
            for l in range(m, min(s, L + 1)):
                assert lp[oracle.lm_index(L, l, m)] == 0.0


def test_closed_forms():
    for theta in (0.2, 1.0, 2.5):
        st, ct = math.sin(theta), math.cos(theta)
        lp1, _ = oracle.spin_lambda(2, 1, theta)
        assert abs(lp1[oracle.lm_index(2, 1, 0)] - math.sqrt(3 / (8 * math.pi)) * st) <= 1e-15
        assert abs(lp1[oracle.lm_index(2, 1, 1)] + math.sqrt(3 / (16 * math.pi)) * (1 - ct)) <= 1e-15
        lp2, _ = oracle.spin_lambda(2, 2, theta)
        assert abs(lp2[oracle.lm_index(2, 2, 0)] - math.sqrt(15 / (32 * math.pi)) * st * st) <= 1e-15
        assert abs(lp2[oracle.lm_index(2, 2, 2)] - math.sqrt(5 / (64 * math.pi)) * (1 - ct) ** 2) <= 1e-15


def test_spin1_is_eth_of_the_scalar_harmonic():
    """1Y_lm = -(dPbar/dtheta - m Pbar / sin) / sqrt(l(l+1)),
    -1Y_lm = (dPbar/dtheta + m Pbar / sin) / sqrt(l(l+1)) (at phi = 0)."""
    L = 40
    for theta in (0.05, 0.9, 2.2):
        lp, lm = oracle.spin_lambda(L, 1, theta)
        P = oracle.plm_all(L, theta)
        pts = np.array([[theta, 0.0]])
        for (l, m) in [(1, 0), (1, 1), (5, 2), (17, 17), (40, 3), (33, 20)]:
            a = np.zeros(oracle.nalm(L), dtype=np.complex128)
            a[oracle.lm_index(L, l, m)] = 1.0
            dth, _ = oracle.synth_grad(a, pts, L)
            dP = dth[0] / (1.0 if m == 0 else 2.0)  # f = w_m Re(Pbar e^{i m phi}) at phi = 0
            Pv = P[oracle.lm_index(L, l, m)]
            ref_p = -(dP - m * Pv / math.sin(theta)) / math.sqrt(l * (l + 1))
            ref_m = (dP + m * Pv / math.sin(theta)) / math.sqrt(l * (l + 1))
            i = oracle.lm_index(L, l, m)
            scale = math.sqrt((2 * l + 1) / (4 * math.pi))
            assert abs(lp[i] - ref_p) <= 1e-12 * scale, (l, m, theta)
            assert abs(lm[i] - ref_m) <= 1e-12 * scale, (l, m, theta)


def test_spin1_synthesis_is_the_gradient_of_two_potentials():
    """Q + iU = sum (G + iC) 1Y = eth(phi + i psi), phi_lm = G_lm / sqrt(l(l+1)),
    psi_lm = C_lm / sqrt(l(l+1)): Q = -d_theta phi + d_phi psi / sin,
    U = -d_phi phi / sin - d_theta psi."""
    L = 30
    pts = W.points_uniform(300, seed=4)
    g = W.alm_gaussian(L, seed=5)
    c = W.alm_gaussian(L, seed=6)
    ells = np.concatenate([np.arange(m, L + 1) for m in range(L + 1)]).astype(float)
    fac = np.where(ells > 0, 1.0 / np.sqrt(np.maximum(ells * (ells + 1), 1.0)), 0.0)
    q, u = oracle.spin_synth(g, c, pts, L, 1)
    pth, pph = oracle.synth_grad(g * fac, pts, L)
    sth, sph = oracle.synth_grad(c * fac, pts, L)
    st = np.sin(pts[:, 0])
    rq = -pth + sph / st
    ru = -pph / st - sth
    assert np.abs(q - rq).max() <= 1e-12 * np.abs(rq).max()
    assert np.abs(u - ru).max() <= 1e-12 * np.abs(ru).max()


@pytest.mark.parametrize("s", [1, 2, 5])
def test_spin_addition_theorem(s):
    L = 2047
    for theta in (1e-3, 0.3, 1.1, 2.0, math.pi - 2e-3):
        lp, lm = oracle.spin_lambda(L, s, theta)
        tot = np.zeros(L + 1)
        for m in range(L + 1):
            a, b = oracle.lm_index(L, m, m), oracle.lm_index(L, L, m) + 1
            ls = np.arange(m, L + 1)
            np.add.at(tot, ls, lp[a:b] ** 2 + (lm[a:b] ** 2 if m > 0 else 0.0))
        ls = np.arange(s, L + 1)
        ref = (2 * ls + 1) / (4 * math.pi)
        assert np.abs(tot[s:] / ref - 1).max() <= 1e-11, (s, theta)


@pytest.mark.parametrize("s,m", [(1, 0), (2, 1), (2, 7), (3, 12)])
def test_spin_orthogonality(s, m):
    L = 40
    n = L + 2
    x, wq = np.polynomial.legendre.leggauss(n)
    th = np.arccos(x)
    l0 = max(m, s)
    rows = []
    for t in th:
        lp, _ = oracle.spin_lambda(L, s, t)
        rows.append(lp[oracle.lm_index(L, l0, m): oracle.lm_index(L, L, m) + 1])
    A = np.array(rows)  # [node][l - l0]
    G = 2 * math.pi * (A * wq[:, None]).T @ A
    assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-12


@pytest.mark.parametrize("s", [1, 2])
def test_spin_adjoint_dot_test_and_orders(s):
    L = 24
    pts = W.points_uniform(500, seed=8)
    g = W.alm_gaussian(L, seed=9)
    c = W.alm_gaussian(L, seed=10)
    q, u = oracle.spin_synth(g, c, pts, L, s)
    rng = np.random.default_rng(11)
    yq, yu = rng.standard_normal(500), rng.standard_normal(500)
    ag, ac = oracle.spin_adjoint(yq, yu, pts, L, s)
    lhs = float(np.dot(yq, q) + np.dot(yu, u))
    rhs = oracle.alm_dot(ag, g, L) + oracle.alm_dot(ac, c, L)
    assert abs(lhs - rhs) <= 1e-12 * (np.linalg.norm(yq) * np.linalg.norm(q) + np.linalg.norm(yu) * np.linalg.norm(u))
    sg, sc = oracle.spin_adjoint(yq, yu, pts, L, s, mlist=[0, 3, L])
    for m in (0, 3, L):
        a, b = oracle.lm_index(L, m, m), oracle.lm_index(L, L, m) + 1
        assert np.allclose(sg[a:b], ag[a:b], rtol=0, atol=1e-12)
        assert np.allclose(sc[a:b], ac[a:b], rtol=0, atol=1e-12)
    # entries with l < s are zero; m = 0 entries are real
    for m in range(0, s):
        for l in range(m, s):
            assert ag[oracle.lm_index(L, l, m)] == 0 and ac[oracle.lm_index(L, l, m)] == 0
    assert np.all(ag[: L + 1].imag == 0) and np.all(ac[: L + 1].imag == 0)
