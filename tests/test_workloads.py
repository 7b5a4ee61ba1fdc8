"""The seeded input recipes (CPU): the synthetic lensing potential's
deflection has the rms it is scaled to, and the generators are reproducible."""
import numpy as np

import oracle
import workloads as W


def test_lensing_potential_rms_deflection():
    """sum_l (2l+1) l(l+1) C_l / 4pi = rms^2: the sampled |grad Phi| (the
    oracle's analytic gradient at uniform points) matches 2.5 arcmin within
    the sampling scatter."""
    L = 191
    phi = W.phi_lensing(L, seed=5)
    pts = W.points_uniform(4000, seed=6)
    dth, dph = oracle.synth_grad(phi, pts, L)
    alpha = np.hypot(dth, dph / np.sin(pts[:, 0]))
    rms = np.sqrt(np.mean(alpha**2)) * 180 * 60 / np.pi
    assert abs(rms - 2.5) < 0.1, rms
    # l < 2 carries no power
    assert np.all(phi[[oracle.lm_index(L, 0, 0), oracle.lm_index(L, 1, 0), oracle.lm_index(L, 1, 1)]] == 0)


def test_generators_are_seeded():
    a1, a2 = W.phi_lensing(31, seed=3), W.phi_lensing(31, seed=3)
    assert np.array_equal(a1, a2)
    assert not np.array_equal(a1, W.phi_lensing(31, seed=4))
    assert np.array_equal(W.points_uniform(10, seed=1), W.points_uniform(10, seed=1))


def test_ring_gradient_of_the_potential_matches_the_oracle():
    """The deflection's gradient on rings (numpy recurrence + inverse FFT in
    phi) against the oracle's analytic gradient at the same points."""
    L = 40
    phi = W.phi_lensing(L, seed=5)
    th = np.array([0.05, 0.3, 1.1, 2.0, 2.9, np.pi - 0.02])
    nphi = 81
    a_th, a_ph = W.phi_gradient_rings(phi, L, th, nphi)
    ph = 2 * np.pi * np.arange(nphi) / nphi
    pts = np.stack([np.repeat(th, nphi), np.tile(ph, th.size)], 1)
    dth, dph = oracle.synth_grad(phi, pts, L)
    assert np.abs(a_th.ravel() - dth).max() <= 1e-12 * np.abs(dth).max()
    assert np.abs(a_ph.ravel() - dph / np.sin(pts[:, 0])).max() <= 1e-12 * np.abs(dph / np.sin(pts[:, 0])).max()


def test_deflected_grid_rms():
    """The deflected lmax 255 grid moves its points by 2.5 arcmin rms."""
    L = 255
    g = W.gl_ring_grid(L + 1, 2 * L + 1)
    p = W.deflected_gl_grid(L, cache=False)

    def unit(q):
        return np.stack([np.sin(q[:, 0]) * np.cos(q[:, 1]), np.sin(q[:, 0]) * np.sin(q[:, 1]), np.cos(q[:, 0])], 1)

    d = np.arccos(np.clip(np.sum(unit(g) * unit(p), 1), -1.0, 1.0))
    rms = np.sqrt(np.mean(d**2)) * 180 * 60 / np.pi
    assert 1.5 < rms < 3.5, rms
