"""Pins of the CPU oracle to facts outside itself (closed forms, identities,
independent libraries, brute force).  None of these re-types the oracle's own
recurrence: each compares it against something the paper or the mathematics
fixes, chosen so that a dropped term, a wrong sign or phase, a wrong
normalisation or a lost underflow range fails at least one of them.

Definitions pinned: Eq. Ylm with the footnote of Sec. 2.2 (orthonormal P_l^m =
d^l_{m0} sqrt((2l+1)/4pi), Condon-Shortley phase), Eq. SHTbase (type 2),
Eq. adjointSHTbase (type 1 = adjoint), the DFS relation g(theta, phi) =
f(2pi - theta, phi + pi) of Fig. doubling.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

FOURPI = 4.0 * math.pi


def ylm_scipy(l, m, th, ph):
    from scipy.special import sph_harm_y

    return sph_harm_y(l, m, th, ph)


def test_closed_forms_low_degree():
    """Y_00, Y_10, Y_11, Y_2m, Y_33 from their textbook closed forms (CS phase)."""
    for th in [0.0, 0.1, 0.7, 1.3, math.pi / 2, 2.2, 3.0, math.pi]:
        p = oracle.plm_all(3, th)
        i = lambda l, m: oracle.lm_index(3, l, m)
        c, s = math.cos(th), math.sin(th)
        ref = {
            (0, 0): 1.0 / math.sqrt(FOURPI),
            (1, 0): math.sqrt(3.0 / FOURPI) * c,
            (1, 1): -math.sqrt(3.0 / (8.0 * math.pi)) * s,
            (2, 0): math.sqrt(5.0 / (16.0 * math.pi)) * (3.0 * c * c - 1.0),
            (2, 1): -math.sqrt(15.0 / (8.0 * math.pi)) * s * c,
            (2, 2): 0.25 * math.sqrt(15.0 / (2.0 * math.pi)) * s * s,
            (3, 3): -0.125 * math.sqrt(35.0 / math.pi) * s**3,
        }
        for (l, m), v in ref.items():
            assert abs(p[i(l, m)] - v) < 2e-16 * 8, (th, l, m, p[i(l, m)], v)


def test_pole_values():
    """At theta=0: Pbar_l0 = sqrt((2l+1)/4pi), Pbar_lm = 0 (m>0); at pi: (-1)^l."""
    L = 4095
    p0 = oracle.plm_all(L, 0.0)
    pp = oracle.plm_all(L, math.pi)
    ell = np.arange(L + 1)
    ref = np.sqrt((2 * ell + 1) / FOURPI)
    # the double-precision three-term recurrence loses about one ulp per step
    # at x = 1 (rounding excites the second, linearly growing solution), so
    # the bound is ~l * 2^-52 relative, 1e-11 at l = 4095
    np.testing.assert_allclose(p0[: L + 1], ref, rtol=1e-11, atol=0)
    np.testing.assert_array_equal(p0[L + 1:], 0.0)
    # sin(pi) is 1.2e-16, not 0: m>0 terms are tiny rather than exactly zero
    np.testing.assert_allclose(pp[: L + 1], ref * (-1.0) ** ell, rtol=1e-11, atol=0)
    assert np.max(np.abs(pp[L + 1:])) < 1e-10


def _pbar_equator_log(l, m):
    """log|Pbar_lm(pi/2)| for l+m even, from P_l^m(0) = (-1)^((l+m)/2) (l+m-1)!!/(l-m)!!."""
    k = (l + m) // 2
    lg = math.lgamma
    log_norm = 0.5 * math.log((2 * l + 1) / FOURPI) + 0.5 * (lg(l - m + 1) - lg(l + m + 1))
    log_odd_df = k * math.log(2.0) + lg(k + 0.5) - 0.5 * math.log(math.pi)  # (2k-1)!!
    log_even_df = ((l - m) // 2) * math.log(2.0) + lg((l - m) // 2 + 1)  # (l-m)!!
    return log_norm + log_odd_df - log_even_df, (-1) ** k


def test_equator_closed_form():
    L = 4095
    p = oracle.plm_all(L, math.pi / 2)
    rng = np.random.default_rng(5)
    for _ in range(400):
        m = int(rng.integers(0, L + 1))
        l = int(rng.integers(m, L + 1))
        v = p[oracle.lm_index(L, l, m)]
        if (l + m) % 2:
            assert abs(v) < 1e-12
        else:
            lv, sg = _pbar_equator_log(l, m)
            ref = sg * math.exp(lv)
            # lgamma differences of large arguments limit this check to ~1e-10
            assert abs(v - ref) <= 1e-9 * abs(ref), (l, m, v, ref)


def test_near_pole_mpmath():
    """Pbar_l0 and Pbar_l1 near the pole against mpmath at 40 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    L = 4095
    for th in [1e-6, 3e-4, 0.01]:
        p = oracle.plm_all(L, th)
        for l in [1, 17, 1000, 4095]:
            for m in [0, 1]:
                if m > l:
                    continue
                ref = mp.sqrt(mp.mpf(2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m)) * \
                    mp.legenp(l, m, mp.cos(mp.mpf(th)))
                ref = float(ref)  # mpmath's legenp includes the Condon-Shortley phase
                v = p[oracle.lm_index(L, l, m)]
                assert abs(v - ref) <= 1e-10 * abs(ref), (th, l, m, v, ref)


def test_equator_mpmath_exact():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    L = 600
    p = oracle.plm_all(L, math.pi / 2)
    for l, m in [(0, 0), (2, 0), (7, 3), (100, 50), (600, 0), (600, 600), (599, 301), (444, 2)]:
        ref = mp.sqrt(mp.mpf(2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m)) * \
            mp.legenp(l, m, 0)
        assert abs(p[oracle.lm_index(L, l, m)] - float(ref)) <= 1e-13 * max(1.0, abs(float(ref))), (l, m)


def test_parity_about_equator():
    """Pbar_lm(pi - theta) = (-1)^(l+m) Pbar_lm(theta)."""
    L = 300
    rng = np.random.default_rng(11)
    for th in rng.uniform(0.0, math.pi / 2, 5):
        a = oracle.plm_all(L, th)
        b = oracle.plm_all(L, math.pi - th)
        ls = np.concatenate([np.arange(m, L + 1) for m in range(L + 1)])
        ms = np.concatenate([np.full(L + 1 - m, m) for m in range(L + 1)])
        np.testing.assert_allclose(b, a * (-1.0) ** (ls + ms), rtol=0, atol=1e-12)


@pytest.mark.parametrize("th", [1e-6, 1e-2, 0.3, 1.1, math.pi / 2, 2.9, math.pi - 1e-4])
def test_addition_theorem(th):
    """sum_m |Y_lm|^2 over -l..l = (2l+1)/(4pi) for every l <= 4095.  At theta = 0.3
    the orders 583 < m < 1200 start below the double range (sin^m < 1e-308)
    and carry real weight, so a lost exponent range fails here."""
    L = 4095
    p = oracle.plm_all(L, th)
    s = np.zeros(L + 1)
    for m in range(L + 1):
        col = p[oracle.lm_index(L, m, m): oracle.lm_index(L, L, m) + 1]
        s[m:] += (1.0 if m == 0 else 2.0) * col * col
    ell = np.arange(L + 1)
    # Away from the poles the double recurrence keeps ~1e-14; as |cos(theta)| -> 1
    # its rounding grows with l (1.4e-11 relative on Pbar_l0 at l = 4095,
    # theta = 1e-6, against mpmath), so the bound there is looser.
    rtol = 5e-13 if abs(math.sin(th)) > 0.2 else 1e-10
    np.testing.assert_allclose(s, (2 * ell + 1) / FOURPI, rtol=rtol, atol=0)


def test_gauss_legendre_orthogonality():
    """2 pi sum_j w_j Pbar_lm Pbar_l'm = delta_ll' for l + l' <= 2n - 1."""
    n = 48
    L = n - 1
    x, w = np.polynomial.legendre.leggauss(n)
    P = np.stack([oracle.plm_all(L, math.acos(xi)) for xi in x])  # (n, nalm)
    for m in range(L + 1):
        sl = slice(oracle.lm_index(L, m, m), oracle.lm_index(L, L, m) + 1)
        G = 2.0 * math.pi * (P[:, sl].T * w) @ P[:, sl]
        np.testing.assert_allclose(G, np.eye(L + 1 - m), atol=3e-13)


def test_against_scipy_sph_harm():
    L = 60
    rng = np.random.default_rng(2)
    th = np.arccos(rng.uniform(-1, 1, 200))
    ph = rng.uniform(0, 2 * math.pi, 200)
    for t, f in zip(th[:40], ph[:40]):
        p = oracle.plm_all(L, t)
        for m in range(0, L + 1, 7):
            ls = np.arange(m, L + 1)
            ours = p[oracle.lm_index(L, m, m): oracle.lm_index(L, L, m) + 1] * np.exp(1j * m * f)
            ref = ylm_scipy(ls, m, t, f)
            np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12)


def test_synth_equals_full_complex_sum():
    """Real-field packed synthesis equals sum over -l..l with c_{l,-m} = (-1)^m conj(c_lm),
    built from scipy's Y_lm (reality symmetry; imaginary part vanishes)."""
    L = 12
    a = W.alm_gaussian(L, seed=3)
    pts = W.points_uniform(100, seed=4)
    full = np.zeros(100, dtype=np.complex128)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            c = a[oracle.lm_index(L, l, m)] if m >= 0 else (-1) ** m * np.conj(a[oracle.lm_index(L, l, -m)])
            full += c * ylm_scipy(l, m, pts[:, 0], pts[:, 1])
    assert np.max(np.abs(full.imag)) < 1e-12 * np.max(np.abs(full.real))
    np.testing.assert_allclose(oracle.synth(a, pts, L), full.real, rtol=0, atol=1e-12)


def test_synth_mpmath_bruteforce():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    L = 5
    a = W.alm_gaussian(L, seed=9)
    pts = W.points_uniform(12, seed=10)
    ours = oracle.synth(a, pts, L)
    for i in range(12):
        th, ph = pts[i]
        acc = mp.mpf(0)
        for l in range(L + 1):
            for m in range(-l, l + 1):
                c = a[oracle.lm_index(L, l, abs(m))]
                c = mp.mpc(c.real, c.imag) if m >= 0 else (-1) ** m * mp.conj(mp.mpc(c.real, c.imag))
                if m == 0:
                    c = mp.mpc(c.real, 0)
                acc += (c * mp.spherharm(l, m, th, ph)).real
        assert abs(ours[i] - float(acc)) < 1e-14 * max(1.0, abs(float(acc)))


def test_adjoint_bruteforce_scipy():
    """c_lm = sum_i f_i conj(Y_lm(theta_i, phi_i)) written with scipy's Y_lm."""
    L = 8
    pts = W.points_uniform(60, seed=12)
    f = np.random.default_rng(13).standard_normal(60)
    c = oracle.adjoint(f, pts, L)
    for l in range(L + 1):
        for m in range(l + 1):
            ref = np.sum(f * np.conj(ylm_scipy(l, m, pts[:, 0], pts[:, 1])))
            assert abs(c[oracle.lm_index(L, l, m)] - ref) < 1e-13 * max(1.0, abs(ref))


@pytest.mark.parametrize("L,mmax", [(40, 40), (40, 25), (1, 1), (0, 0)])
def test_dot_product(L, mmax):
    """<y, S a> = <S^H y, a> (type 1 is the adjoint of type 2, Sec. 2.1)."""
    a = W.alm_gaussian(L, seed=21, mmax=mmax)
    a[: L + 1] += 1j * np.random.default_rng(5).standard_normal(L + 1)  # Im(a_l0) is ignored
    pts = W.points_uniform(5000, seed=22)
    y = np.random.default_rng(23).standard_normal(5000)
    lhs = float(np.dot(y, oracle.synth(a, pts, L, mmax)))
    rhs = oracle.alm_dot(oracle.adjoint(y, pts, L, mmax), a, L, mmax)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300) + 1e-300
    c = oracle.adjoint(y, pts, L, mmax)
    assert np.all(c[: L + 1].imag == 0.0)


def test_adjoint_subset_matches_full():
    L = 30
    pts = W.points_uniform(800, seed=31)
    f = np.random.default_rng(32).standard_normal(800)
    full = oracle.adjoint(f, pts, L)
    sub = oracle.adjoint(f, pts, L, mlist=[0, 3, 17, 30])
    for m in [0, 3, 17, 30]:
        sl = slice(oracle.lm_index(L, m, m), oracle.lm_index(L, L, m) + 1)
        np.testing.assert_allclose(sub[sl], full[sl], rtol=0, atol=1e-12)
    assert np.isnan(sub[oracle.lm_index(L, 5, 1)])


def test_rotation_invariance():
    """a_lm e^{i m alpha} evaluated at phi equals a_lm evaluated at phi + alpha."""
    L = 25
    a = W.alm_gaussian(L, seed=41)
    pts = W.points_uniform(300, seed=42)
    alpha = 0.7311
    ms = np.concatenate([np.full(L + 1 - m, m) for m in range(L + 1)])
    rot = a * np.exp(1j * ms * alpha)
    shifted = pts.copy()
    shifted[:, 1] += alpha
    np.testing.assert_allclose(oracle.synth(rot, pts, L), oracle.synth(a, shifted, L), rtol=0, atol=1e-12)


def test_dfs_continuation():
    """Any real (theta, phi) names a point on the sphere: f(-t, p) = f(t, p + pi),
    f(2pi - t, p) = f(t, p + pi) (the doubling relation of Fig. doubling) and f is
    2pi-periodic in theta."""
    L = 20
    a = W.alm_gaussian(L, seed=51)
    pts = W.points_uniform(200, seed=52)
    base = oracle.synth(a, pts, L)
    flip = pts.copy()
    flip[:, 1] += math.pi
    f_flip = oracle.synth(a, flip, L)
    for alt in [np.stack([-pts[:, 0], pts[:, 1]], 1), np.stack([2 * math.pi - pts[:, 0], pts[:, 1]], 1)]:
        np.testing.assert_allclose(oracle.synth(a, alt, L), f_flip, rtol=0, atol=1e-11)
    per = pts.copy()
    per[:, 0] += 2 * math.pi
    np.testing.assert_allclose(oracle.synth(a, per, L), base, rtol=0, atol=1e-11)


def test_ring_sums_match_synth():
    L = 30
    a = W.alm_gaussian(L, seed=61)
    th = np.linspace(0, math.pi, 17)
    F = oracle.ring_sums(a, th, L)
    ph = 1.234
    ms = np.arange(L + 1)
    f_ring = F[0].real + 2.0 * np.sum((F[1:] * np.exp(1j * ms[1:, None] * ph)).real, axis=0)
    pts = np.stack([th, np.full_like(th, ph)], 1)
    np.testing.assert_allclose(f_ring, oracle.synth(a, pts, L), rtol=0, atol=1e-12)


def test_gradient_central_differences():
    L = 20
    a = W.alm_gaussian(L, seed=71)
    pts = W.points_uniform(60, seed=72)
    # include the poles, where the ladder form must stay finite
    pts = np.concatenate([pts, [[0.0, 0.4], [math.pi, 2.0]]])
    dth, dph = oracle.synth_grad(a, pts, L)
    h = 1e-6
    for k, d in [(0, dth), (1, dph)]:
        e = np.zeros(2)
        e[k] = h
        fd = (oracle.synth(a, pts + e, L) - oracle.synth(a, pts - e, L)) / (2 * h)
        scale = np.sqrt(np.mean(fd**2))
        np.testing.assert_allclose(d, fd, rtol=0, atol=2e-7 * scale)


def test_gradient_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    L = 4
    a = W.alm_gaussian(L, seed=81)
    pts = W.points_uniform(5, seed=82)
    dth, dph = oracle.synth_grad(a, pts, L)

    def f(th, ph):
        acc = mp.mpf(0)
        for l in range(L + 1):
            for m in range(-l, l + 1):
                c = a[oracle.lm_index(L, l, abs(m))]
                c = mp.mpc(c.real, c.imag) if m >= 0 else (-1) ** m * mp.conj(mp.mpc(c.real, c.imag))
                if m == 0:
                    c = mp.mpc(c.real, 0)
                acc += (c * mp.spherharm(l, m, th, ph)).real
        return acc

    for i in range(5):
        th, ph = mp.mpf(pts[i, 0]), mp.mpf(pts[i, 1])
        gth = mp.diff(lambda t: f(t, ph), th)
        gph = mp.diff(lambda p: f(th, p), ph)
        assert abs(dth[i] - float(gth)) < 1e-12 * max(1.0, abs(float(gth)))
        assert abs(dph[i] - float(gph)) < 1e-12 * max(1.0, abs(float(gph)))


def test_eps_eff_definition():
    """eps_eff (Sec. 4) is the relative l2 error."""
    t = np.array([3.0, 4.0])
    assert oracle.eps_eff(t, t) == 0.0
    assert abs(oracle.eps_eff(t, np.array([3.0, 3.0])) - 0.2) < 1e-15


# --- CMB lensing pointing (App. C, Eq. pointing and Eq. spin1deriv) -------


def _unit(th, ph):
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)


def test_pointing_y10_is_a_meridional_shift():
    """Phi = a10 Y_10 = a10 sqrt(3/4pi) cos(theta): the gradient points along
    e_theta only, so every point moves along its meridian by
    alpha_theta = -a10 sqrt(3/4pi) sin(theta): theta' = theta + alpha_theta, phi' = phi."""
    L = 3
    a10 = 2e-3
    phi = np.zeros(oracle.nalm(L), dtype=np.complex128)
    phi[oracle.lm_index(L, 1, 0)] = a10
    pts = W.points_uniform(200, seed=91)
    pts = np.concatenate([pts, [[1e-3, 0.5], [math.pi - 1e-3, 4.0], [math.pi / 2, 6.2]]])
    out = oracle.pointing(phi, pts, L)
    th_ref = pts[:, 0] - a10 * math.sqrt(3.0 / FOURPI) * np.sin(pts[:, 0])
    np.testing.assert_allclose(out[:, 0], th_ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[:, 1], np.mod(pts[:, 1], 2 * math.pi), rtol=0, atol=1e-14)


def test_pointing_zero_potential_is_identity():
    L = 5
    pts = W.points_uniform(50, seed=92)
    pts[:, 1] += 7.0  # any real phi: the output is reduced to [0, 2 pi)
    out = oracle.pointing(np.zeros(oracle.nalm(L), dtype=np.complex128), pts, L)
    np.testing.assert_allclose(out[:, 0], pts[:, 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[:, 1], np.mod(pts[:, 1], 2 * math.pi), rtol=0, atol=1e-14)


def test_pointing_moves_along_the_geodesic_of_the_gradient():
    """n' lies at angular distance alpha = |grad Phi| from n, in the direction
    of alpha_theta e_theta + alpha_phi e_phi (the geodesic the gradient starts)."""
    L = 12
    phi = W.alm_gaussian(L, seed=93) * 3e-3
    pts = W.points_uniform(300, seed=94)
    out = oracle.pointing(phi, pts, L)
    dth, dph = oracle.synth_grad(phi, pts, L)
    th, ph = pts[:, 0], pts[:, 1]
    at, ap = dth, dph / np.sin(th)
    alpha = np.hypot(at, ap)
    n, n2 = _unit(th, ph), _unit(out[:, 0], out[:, 1])
    dist = np.arctan2(np.linalg.norm(np.cross(n, n2), axis=1), np.sum(n * n2, axis=1))
    np.testing.assert_allclose(dist, alpha, rtol=1e-12, atol=1e-16)
    et = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], -1)
    ep = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], -1)
    d = (at[:, None] * et + ap[:, None] * ep) / alpha[:, None]
    t = n2 - np.sum(n * n2, axis=1)[:, None] * n
    t /= np.linalg.norm(t, axis=1)[:, None]
    np.testing.assert_allclose(t, d, rtol=0, atol=1e-9)


def test_pointing_rotation_equivariance():
    """Rotating the potential about the z axis by phi0 (c_lm -> c_lm e^{-i m phi0})
    rotates the deflected positions by the same angle."""
    L = 10
    phi = W.alm_gaussian(L, seed=95) * 2e-3
    ms = np.concatenate([np.full(L + 1 - m, m) for m in range(L + 1)])
    phi0 = 0.7
    rot = phi * np.exp(-1j * ms * phi0)
    pts = W.points_uniform(100, seed=96)
    out = oracle.pointing(phi, pts, L)
    out_r = oracle.pointing(rot, pts + np.array([0.0, phi0]), L)
    np.testing.assert_allclose(out_r[:, 0], out[:, 0], rtol=0, atol=1e-14)
    dphi = np.mod(out_r[:, 1] - out[:, 1] - phi0 + math.pi, 2 * math.pi) - math.pi
    np.testing.assert_allclose(dphi, 0.0, rtol=0, atol=1e-13)
