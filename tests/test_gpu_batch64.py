"""The batched transform at the size bench.py times: 64 members,
lmax_b ~ U{256..2047} (seed 0), N_b = 2 lmax_b^2 uniform points
(211,888,640 points in all), default plan options, in both precisions:
mixed (complex64 coefficients, float32 maps, eps = 1e-5, TF32-split
tensor-core contraction from the plan-time recurrence table) and FP64 (the
same values as complex128 and float64, eps = 1e-10, bf16-sliced tensor-core
contraction).

Five members, at five ranks of the sorted lmax (smallest to largest), are
checked against the oracle's direct sums stored by tests/golden/make_refs.py
(oracle/ only): synthesis at 10^4 seeded points (eps_eff and the per-point
maximum, each <= the precision's tolerance), and the adjoint for every
degree of the orders {0, 1} and one seeded random order (eps_eff per order
<= the tolerance).  The stored references take the float32-rounded map and
the complex64 coefficients as exact inputs, so they serve both precisions.  The checked
members must cover every bucket the planner formed.  The errors are printed.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
REFS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch64_oracle_refs.npz")


@pytest.mark.parametrize("precision,TOL", [("mixed", 1e-5), ("fp64", 1e-10)])
def test_batch64_full_config_against_stored_oracle(precision, TOL):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14542_gb300 import build

    build.build()
    import paper_2406_14542_gb300 as nu

    refs = dict(np.load(REFS))
    members = W.batch64()
    ls = [m[0] for m in members]
    check = [int(i) for i in refs["members"]]
    dpts = [torch.from_numpy(m[2]).cuda() for m in members]
    bp = nu.BatchPlan(ls, dpts, eps=TOL, precision=precision)
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    rdt = torch.float64 if precision == "fp64" else torch.float32
    info = bp.info()
    assert {info["bucket_of"][i] for i in check} == set(range(info["nbuckets"])), info["bucket_of"]
    fo = bp.synth([torch.from_numpy(m[1]).to(cdt).cuda() for m in members])
    ys = []
    for i, m in enumerate(members):
        y = np.random.default_rng(3000 + i).standard_normal(m[2].shape[0]).astype(np.float32)
        ys.append(torch.from_numpy(y).to(rdt).cuda())
    co = bp.adjoint(ys)
    bp.status()
    torch.cuda.synchronize()
    report = {}
    for i in check:
        L = ls[i]
        idx, fref = refs["member%d_synth_idx" % i], refs["member%d_synth_ref" % i]
        f = fo[i].double().cpu().numpy()[idx]
        e_syn = oracle.eps_eff(fref, f)
        e_max = float(np.max(np.abs(f - fref)) / np.max(np.abs(fref)))
        c = co[i].cpu().numpy().astype(np.complex128)
        e_ord = {}
        pos = 0
        for m in refs["member%d_adj_orders" % i].tolist():
            k = L + 1 - m
            s = oracle.lm_index(L, m, m)
            e_ord[m] = oracle.eps_eff(refs["member%d_adj_ref" % i][pos:pos + k], c[s:s + k])
            pos += k
        report[i] = (L, e_syn, e_max, e_ord)
    print("\nbatch64 %s (%d buckets, lmax %s): %s" % (precision, info["nbuckets"], info["bucket_lmax"],
                                                  {i: "lmax %d synth %.3g max %.3g adjoint %s"
                                                   % (r[0], r[1], r[2], {m: "%.3g" % e for m, e in r[3].items()})
                                                   for i, r in report.items()}))
    bp.close()
    for i, (L, e_syn, e_max, e_ord) in report.items():
        assert e_syn <= TOL and e_max <= TOL, (i, L, e_syn, e_max)
        assert all(e <= TOL for e in e_ord.values()), (i, L, e_ord)
