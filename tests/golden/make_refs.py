"""Writes the stored oracle values that the full-size GPU parity tests compare
against (tests/test_gpu_fullsize.py, tests/test_gpu_batch64.py).

Every number written here comes from ``oracle/`` (the direct FP64 sums of
Eq. SHTbase and Eq. adjointSHTbase) on the seeded inputs of ``workloads/``;
nothing is taken from the CUDA library.  The sums are O(lmax^2) per point
(synthesis) and O(N (lmax - m)) per order (adjoint), minutes to an hour on a
few host cores, which is why they are stored instead of recomputed in every
GPU test run.

    python tests/golden/make_refs.py            # both files
    python tests/golden/make_refs.py gl4095     # one of them

Files (numpy .npz, float64 / complex128):

* gl4095_oracle_refs.npz -- the 4096 x 8191 deflected GL grid, lmax 4095:
    synth_idx, synth_pts   10^4 seeded points (PCG64 seed 12345) and their
                           exact coordinates (the GPU test puts these into
                           the regenerated point set: numpy's transcendental
                           functions and FFT differ in the last bits between
                           host platforms, and at lmax 4095 a coordinate
                           change delta moves f by ~lmax delta relative);
    synth_ref              the type 2 values at those points;
    adj_y, adj_orders,     a map that is N(0, 1) (seed 52, rounded to float32)
    adj_ref                on the sampled points and zero on every other
                           point, and its type 1 coefficients c_lm,
                           l = m..4095, for the orders {0, 1} and 4 seeded
                           random orders in [2, 4095], concatenated order by
                           order (a sum over the sampled points only).
* batch64_oracle_refs.npz -- the 64-member batch (lmax_b ~ U{256..2047},
  N_b = 2 lmax_b^2, seed 0): for members at five ranks of the sorted lmax
  (smallest, 25 %, median, 75 %, largest), member<i>_synth_idx / _synth_ref
  (10^4 points), member<i>_adj_orders / _adj_ref (orders {0, 1} and one
  seeded random order, map y ~ N(0, 1) rounded to float32, seed 3000 + i).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

NSYNTH = 10000


def f32_gauss(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n).astype(np.float32).astype(np.float64)


def adj_orders(lmax: int, nrand: int, seed: int) -> np.ndarray:
    rnd = np.random.default_rng(seed).choice(np.arange(2, lmax + 1), size=nrand, replace=False)
    return np.concatenate([[0, 1], np.sort(rnd)]).astype(np.int32)


def order_block(c: np.ndarray, lmax: int, orders) -> np.ndarray:
    return np.concatenate([c[oracle.lm_index(lmax, m, m): oracle.lm_index(lmax, m, m) + lmax + 1 - m]
                           for m in orders])


def make_gl4095(path: str):
    L, a, pts = W.workload("gl4095")
    n = pts.shape[0]
    idx = W.subset(n, NSYNTH, seed=12345)
    sp = np.ascontiguousarray(pts[idx])
    t0 = time.time()
    f = oracle.synth(a, sp, L)
    print("gl4095 synthesis on %d points: %.0f s" % (idx.size, time.time() - t0), flush=True)
    y = f32_gauss(idx.size, 52)
    orders = adj_orders(L, 4, 53)
    t0 = time.time()
    c = oracle.adjoint(y, sp, L, mlist=orders)
    print("gl4095 adjoint (map on the sampled points), orders %s: %.0f s" % (orders.tolist(), time.time() - t0),
          flush=True)
    np.savez(path, synth_idx=idx, synth_pts=sp, synth_ref=f, adj_y=y, adj_orders=orders,
             adj_ref=order_block(c, L, orders))


def batch64_members(lmaxs) -> list[int]:
    order = np.argsort(np.asarray(lmaxs), kind="stable")
    nb = len(lmaxs)
    return [int(order[r]) for r in (0, nb // 4, nb // 2, (3 * nb) // 4, nb - 1)]


def make_batch64(path: str):
    members = W.batch64()
    ls = [m[0] for m in members]
    out = {}
    for i in batch64_members(ls):
        L, a, pts = members[i]
        a = a.astype(np.complex128)
        n = pts.shape[0]
        t0 = time.time()
        idx = W.subset(n, NSYNTH, seed=12345)
        out["member%d_synth_idx" % i] = idx
        out["member%d_synth_ref" % i] = oracle.synth(a, pts[idx], L)
        y = f32_gauss(n, 3000 + i)
        orders = adj_orders(L, 1, 4000 + i)
        c = oracle.adjoint(y, pts, L, mlist=orders)
        out["member%d_adj_orders" % i] = orders
        out["member%d_adj_ref" % i] = order_block(c, L, orders)
        print("batch64 member %d (lmax %d, %d points): %.0f s" % (i, L, n, time.time() - t0), flush=True)
    np.savez(path, members=np.array(sorted(int(k[6:].split("_")[0]) for k in out if k.endswith("synth_ref"))),
             **out)


if __name__ == "__main__":
    which = sys.argv[1:] or ["gl4095", "batch64"]
    if "batch64" in which:
        make_batch64(os.path.join(HERE, "batch64_oracle_refs.npz"))
    if "gl4095" in which:
        make_gl4095(os.path.join(HERE, "gl4095_oracle_refs.npz"))
