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
