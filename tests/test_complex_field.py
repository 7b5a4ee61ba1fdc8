"""Complex fields through the real-field transforms (the reading of a
complex map as two real transforms): the split / merge identities of
``complex_split`` and ``complex_merge_adjoint`` checked against scipy's
complex spherical harmonics, with the oracle as the real-field transform
(CPU), and the GPU plan end to end (GPU)."""
import numpy as np
import pytest

import oracle
import workloads as W
import paper_2406_14542_gb300 as nu

sph = pytest.importorskip("scipy.special")


def _fields(L, seed):
    rng = np.random.default_rng(seed)
    n = nu.nalm(L)
    pos = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    neg = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return pos, neg


def _lm(L):
    return [(l, m) for m in range(L + 1) for l in range(m, L + 1)]


def _ref_synth(pos, neg, pts, L):
    th, ph = pts[:, 0], pts[:, 1]
    f = np.zeros(pts.shape[0], dtype=np.complex128)
    for k, (l, m) in enumerate(_lm(L)):
        f += pos[k] * sph.sph_harm_y(l, m, th, ph)
        if m > 0:
            f += neg[k] * sph.sph_harm_y(l, -m, th, ph)
    return f


def _ref_adjoint(F, pts, L):
    th, ph = pts[:, 0], pts[:, 1]
    cp = np.zeros(nu.nalm(L), dtype=np.complex128)
    cn = np.zeros(nu.nalm(L), dtype=np.complex128)
    for k, (l, m) in enumerate(_lm(L)):
        cp[k] = np.sum(F * np.conj(sph.sph_harm_y(l, m, th, ph)))
        cn[k] = np.sum(F * np.conj(sph.sph_harm_y(l, -m, th, ph)))
    return cp, cn


def test_split_and_merge_against_scipy():
    L = 12
    pts = W.points_uniform(300, seed=21)
    pos, neg = _fields(L, 3)
    r, i = nu.complex_split(pos, neg, L)
    assert np.all(np.abs(r[: L + 1].imag) == 0) and np.all(np.abs(i[: L + 1].imag) == 0)
    f = oracle.synth(r, pts, L) + 1j * oracle.synth(i, pts, L)
    ref = _ref_synth(pos, neg, pts, L)
    assert np.linalg.norm(f - ref) <= 1e-12 * np.linalg.norm(ref)
    F = np.random.default_rng(5).standard_normal(300) + 1j * np.random.default_rng(6).standard_normal(300)
    cp, cn = nu.complex_merge_adjoint(oracle.adjoint(F.real.copy(), pts, L), oracle.adjoint(F.imag.copy(), pts, L), L)
    rp, rn = _ref_adjoint(F, pts, L)
    assert np.linalg.norm(cp - rp) <= 1e-12 * np.linalg.norm(rp)
    mpos = np.array([m for (l, m) in _lm(L)]) > 0
    assert np.linalg.norm((cn - rn)[mpos]) <= 1e-12 * np.linalg.norm(rn[mpos])


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_complex_field_gpu(prec, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14542_gb300 import build

    build.build()
    L = 20
    pts = W.points_uniform(2000, seed=22)
    pos, neg = _fields(L, 4)
    plan = nu.Plan(L, torch.from_numpy(pts).cuda(), eps=tol, precision=prec)
    cd = plan.cdtype
    f = plan.synth_complex(torch.from_numpy(pos).to(cd).cuda(), torch.from_numpy(neg).to(cd).cuda())
    ref = _ref_synth(pos, neg, pts, L)
    got = f.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    F = np.random.default_rng(7).standard_normal(2000) + 1j * np.random.default_rng(8).standard_normal(2000)
    cp, cn = plan.adjoint_complex(torch.from_numpy(F).to(cd).cuda())
    rp, rn = _ref_adjoint(F.astype(np.complex64).astype(np.complex128) if prec == "mixed" else F, pts, L)
    mpos = np.array([m for (l, m) in _lm(L)]) > 0
    assert np.linalg.norm(cp.cpu().numpy() - rp) <= tol * np.linalg.norm(rp)
    assert np.linalg.norm((cn.cpu().numpy() - rn)[mpos]) <= tol * np.linalg.norm(rn[mpos])
