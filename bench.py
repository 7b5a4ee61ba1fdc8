"""Benchmark: nonuniform SHT synthesis + adjoint at lmax = 4095 on the
4096 x 8191 deflected Gauss-Legendre grid (33,550,336 points).

One step = one type 2 transform (synthesis) plus one type 1 transform
(adjoint) with inputs resident on the GPU.  The headline is the FP64 path at
eps = 1e-10; the mixed path (FP64 recurrence, FP32 contraction / FFT / NUFFT)
at eps = 1e-5 is measured in the same run and reported beside it.  Prints one
JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 (under torchrun) every rank runs the same workload on its
own GPU (replicas: a single transform does not shard without an exchange
step); value = max-over-ranks time per step / N.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "nuSHT synth+adjoint ms at ℓmax 4095, 33.5M pts; FP64 1e-10 vs mixed 1e-5"
WORKLOAD = "gl4095"
LMAX = 4095
EPS = {"fp64": 1e-10, "mixed": 1e-5}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 pipe peak: 152 SMs x 2 FP64 FMA lanes per clock x 2 flops x 2.07 GHz
# (the recipe's nominal 1.25 TFLOP/s; 1.19 measured with an FMA probe)
FP64_PEAK_TFLOPS = 1.25


def legendre_fp64_work(triples: int) -> float:
    """FP64 work of one Legendre pass: 3 flops (one multiply, one FMA: the
    rescaled three-term recurrence) per (ring pair, l, m) triple the kernel
    runs.  The multiply occupies a full FMA slot, so the attainable peak for
    this 1:1 mix is 3/4 of the FMA peak."""
    return 3.0 * triples


class Clocks:
    """nvidia-smi sampler run during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(ngpus: int):
    import torch

    if ngpus > 1 or int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist

        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return dist, dist.get_rank(), dist.get_world_size(), local
    return None, 0, 1, 0


def barrier(dist):
    import torch

    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


def max_over_ranks(dist, x: float) -> float:
    import torch

    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(torch, fn, steps: int, warmup: int, dist):
    for _ in range(warmup):
        fn()
    barrier(dist)
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    barrier(dist)
    return e0.elapsed_time(e1) / steps


def step_spread(torch, fn, reps: int = 20):
    """Median and standard deviation of single-step device times (CUDA events
    around each step, after the timed run has warmed everything up)."""
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), float(np.std(ts))


def stage_breakdown(torch, plan, ad, y, reps: int = 3):
    """Per-stage device times from the library's own stream events."""
    acc = None
    for _ in range(reps):
        plan.synth(ad)
        plan.adjoint(y)
        st = plan.stage_times()
        if acc is None:
            acc = {k: {kk: [vv] for kk, vv in v.items()} for k, v in st.items()}
        else:
            for k, v in st.items():
                for kk, vv in v.items():
                    acc[k][kk].append(vv)
    return {k: {kk: float(np.mean(vv)) for kk, vv in v.items()} for k, v in acc.items()}


def cpu_oracle_step(a, pts, L, nsample: int, seed: int = 3):
    """Oracle synthesis + adjoint (all orders) on a seeded sample of points;
    returns (seconds, threads, sample indices)."""
    import oracle

    sel = W.subset(pts.shape[0], nsample, seed=seed)
    y = np.random.default_rng(seed).standard_normal(sel.size)
    t0 = time.perf_counter()
    oracle.synth(a, pts[sel], L)
    oracle.adjoint(y, pts[sel], L)
    return time.perf_counter() - t0, oracle.num_threads(), sel


def run_reference(args):
    """The oracle (direct O(lmax^2 N) sums, C + OpenMP on the host cores) on a
    bounded sample of the same workload, scaled to one full step."""
    dist, rank, world, _ = (None, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0)
    if rank != 0:
        return
    L, a, pts = W.workload(WORKLOAD)
    nsample = int(os.environ.get("NUSHT_REF_SAMPLE", "200"))
    times = []
    for k in range(args.warmup + args.steps):
        sec, threads, sel = cpu_oracle_step(a, pts, L, nsample, seed=100 + k)
        if k >= args.warmup:
            times.append(sec)
    scale = pts.shape[0] / float(nsample)
    ms = 1e3 * float(np.mean(times)) * scale
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "extrapolated": True,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "deflected GL grid 4096x8191 (33,550,336 pts), lmax=mmax=4095, "
                                   "C_l=(l+1)^-2, 2.5 arcmin rms deflection"},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": threads, "kind": "oracle", "extrapolated": True,
                             "sample": "%d seeded points per step (synthesis + full adjoint), scaled by N/%d "
                                       "(the direct sum is exactly linear in N)" % (nsample, nsample)},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-transform batched measurement")
    ap.add_argument("--no-table", action="store_true",
                    help="skip the FP64 recurrence-table run and the mixed per-call-recurrence run")
    ap.add_argument("--no-strict", action="store_true",
                    help="skip the all-FP64-instruction run (fp64_contraction=1, fft_kernels=-1)")
    ap.add_argument("--sweep", action="store_true",
                    help="accuracy / speed sweep over eps x sigma on the lmax 1023 deflected grid (one JSON line)")
    ap.add_argument("--no-fast", action="store_true",
                    help="skip the opt-in double-float recurrence (fast_recurrence=1) runs")
    ap.add_argument("--no-pointing", action="store_true", help="skip the lensing pointing measurement")
    ap.add_argument("--no-autograd", action="store_true", help="skip the differentiable-transform measurement")
    ap.add_argument("--no-spin", action="store_true", help="skip the spin-2 transform measurement")
    ap.add_argument("--sweep-workload", default="gl1023", choices=["gl1023", "gl2047", "gl4095"],
                    help="workload of --sweep")
    ap.add_argument("--only-batch", action="store_true", help="run only the 64-transform batched measurement")
    ap.add_argument("--batch-precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of --only-batch")
    ap.add_argument("--no-batch-fp64", action="store_true",
                    help="skip the 64-transform batched measurement in FP64 (eps 1e-10)")
    ap.add_argument("--no-sequential", action="store_true",
                    help="with --only-batch: skip the one-by-one comparison")
    ap.add_argument("--batch-n", type=int, default=64, help="transforms in the batched workload")
    ap.add_argument("--batch-lmax", type=int, default=2047, help="largest lmax of the batched workload")
    ap.add_argument("--workload", default=WORKLOAD, choices=["gl1023", "gl2047", "gl4095"],
                    help="smaller deflected-grid cases for profiling; the benchmark is gl4095")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    import paper_2406_14542_gb300 as nu

    dist, rank, world, local = dist_setup(args.gpus)
    if args.sweep:
        if rank == 0:
            print(json.dumps({"sweep": run_sweep(torch, nu, args)}), flush=True)
        return
    if args.only_batch:
        b = run_batch64(torch, nu, args, dist, rank, sequential=not args.no_sequential,
                        precision=args.batch_precision)
        if rank == 0:
            print(json.dumps({"batch64" if args.batch_precision == "mixed" else "batch64_fp64": b}), flush=True)
        return
    L, a, pts = W.workload(args.workload)
    npts = pts.shape[0]
    peaks, peak_src = load_peaks()
    dpts = torch.from_numpy(pts).cuda()
    results = {}
    y_host = np.random.default_rng(5).standard_normal(npts)
    # (key, precision, plan options); "mixed" is the mixed default, which
    # runs the FP64 recurrence once at plan time (recurrence table)
    runs = [("fp64", "fp64", {})] + ([] if args.no_mixed else [("mixed", "mixed", {})])
    if not args.no_strict:
        runs += [("fp64_strict", "fp64", {"fp64_contraction": True, "fft_kernels": -1})]
    if not args.no_table:
        runs += [("fp64_table", "fp64", {"legendre_table": 1})]
        runs += [] if args.no_mixed else [("mixed_percall", "mixed", {"legendre_table": -1})]
    if not args.no_fast:
        runs += [("fp64_fast_recurrence", "fp64", {"fast_recurrence": True})]
        runs += [] if args.no_mixed else [("mixed_fast_recurrence", "mixed", {"fast_recurrence": True})]
    sel_par = W.subset(npts, 300, seed=17)
    f_ref_par = None
    for key, prec, popts in runs:
        cd = torch.complex128 if prec == "fp64" else torch.complex64
        rd = torch.float64 if prec == "fp64" else torch.float32
        t0 = time.perf_counter()
        plan = nu.Plan(L, dpts, eps=EPS[prec], precision=prec, profile=True, **popts)
        torch.cuda.synchronize()
        t_plan = time.perf_counter() - t0
        ad = torch.from_numpy(a).to(cd).cuda()
        y = torch.from_numpy(y_host).to(rd).cuda()
        fmap = torch.empty(npts, dtype=rd, device="cuda")
        calm = torch.empty(plan.nalm, dtype=cd, device="cuda")

        def step():
            plan.synth(ad, out=fmap)
            plan.adjoint(y, out=calm)

        with Clocks(local) as clk:
            ms = time_steps(torch, step, args.steps, args.warmup, dist)
        ms = max_over_ranks(dist, ms)
        med, std = step_spread(torch, step, 20 if key == "fp64" else 5)
        stages = stage_breakdown(torch, plan, ad, y)
        # parity on a seeded subset against the oracle (rank 0)
        par = None
        if rank == 0:
            import oracle

            if f_ref_par is None:
                f_ref_par = oracle.synth(a, pts[sel_par], L)
            f = plan.synth(ad).double().cpu().numpy()
            par = oracle.eps_eff(f_ref_par, f[sel_par])
        results[key] = {"ms": ms, "plan_s": t_plan, "stages": stages, "clocks": clk.summary(), "eps_eff": par,
                        "info": plan.info(), "median": med, "std": std}
        if key == "fp64":
            # end to end through the public API with host buffers (pinned):
            # every step uploads its a_lm and map and downloads its map and
            # coefficients.  A copy stream overlaps the uploads and downloads
            # with compute (y's upload with the synthesis, the map's download
            # with the adjoint, the next a_lm's upload with this adjoint);
            # device and host buffers alternate between two slots.
            nb = 2
            a_pin = [torch.from_numpy(a).pin_memory() for _ in range(nb)]
            y_pin = [torch.from_numpy(y_host).pin_memory() for _ in range(nb)]
            f_pin = [torch.empty(npts, dtype=torch.float64).pin_memory() for _ in range(nb)]
            c_pin = [torch.empty(plan.nalm, dtype=torch.complex128).pin_memory() for _ in range(nb)]
            a_dev = [torch.empty_like(ad) for _ in range(nb)]
            y_dev = [torch.empty_like(y) for _ in range(nb)]
            f_dev = [torch.empty_like(fmap) for _ in range(nb)]
            c_dev = [torch.empty_like(calm) for _ in range(nb)]
            hs, ds = torch.cuda.Stream(), torch.cuda.Stream()  # uploads, downloads
            comp = torch.cuda.current_stream()
            ev = {k: [torch.cuda.Event() for _ in range(nb)] for k in ("a", "y", "f", "c", "fd", "cd")}
            it = [0]

            def e2e_step():
                b = it[0] % nb
                it[0] += 1
                with torch.cuda.stream(hs):
                    hs.wait_event(ev["c"][b])  # slot b's inputs are free once its last adjoint ran
                    a_dev[b].copy_(a_pin[b], non_blocking=True)
                    ev["a"][b].record(hs)
                    y_dev[b].copy_(y_pin[b], non_blocking=True)
                    ev["y"][b].record(hs)
                comp.wait_event(ev["a"][b])
                comp.wait_event(ev["fd"][b])  # slot b's map has been downloaded
                plan.synth(a_dev[b], out=f_dev[b])
                ev["f"][b].record(comp)
                with torch.cuda.stream(ds):
                    ds.wait_event(ev["f"][b])
                    f_pin[b].copy_(f_dev[b], non_blocking=True)
                    ev["fd"][b].record(ds)
                comp.wait_event(ev["y"][b])
                comp.wait_event(ev["cd"][b])
                plan.adjoint(y_dev[b], out=c_dev[b])
                ev["c"][b].record(comp)
                with torch.cuda.stream(ds):
                    ds.wait_event(ev["c"][b])
                    c_pin[b].copy_(c_dev[b], non_blocking=True)
                    ev["cd"][b].record(ds)

            def drain():  # the timed region ends when the last downloads have landed
                comp.wait_stream(ds)
                comp.wait_stream(hs)

            for b in range(nb):  # events start recorded, so the first waits pass
                for k in ev:
                    ev[k][b].record(comp)
            e2e_step()
            drain()
            barrier(dist)
            t0e = torch.cuda.Event(enable_timing=True)
            t1e = torch.cuda.Event(enable_timing=True)
            t0e.record(comp)
            for _ in range(args.steps):
                e2e_step()
            drain()
            t1e.record(comp)
            barrier(dist)
            e2e_ms = max_over_ranks(dist, t0e.elapsed_time(t1e) / args.steps)
            h2d = a_pin[0].numel() * 16 + y_pin[0].numel() * 8
            d2h = f_pin[0].numel() * 8 + c_pin[0].numel() * 16
            results["e2e"] = {"value": e2e_ms / world, "unit": "ms", "h2d_bytes_per_step": h2d,
                              "d2h_bytes_per_step": d2h,
                              "how": "public API; pinned host buffers; every step's uploads and downloads inside "
                                     "the timed region, overlapped with compute on upload / download streams"}
        plan.close()
        del ad, y, fmap, calm
        torch.cuda.empty_cache()

    pointing = None if args.no_pointing else run_pointing(torch, nu, args, dist, L)
    spin = None if args.no_spin else run_spin(torch, nu, args, dist, rank, L, pts)
    autograd = None if args.no_autograd or args.workload != WORKLOAD else run_autograd(torch, nu, args, dist)

    batch = batch_fp64 = None
    if not args.no_batch and args.workload == WORKLOAD:
        batch = run_batch64(torch, nu, args, dist, rank)
        if not args.no_batch_fp64:
            batch_fp64 = run_batch64(torch, nu, args, dist, rank, precision="fp64")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    fp = results["fp64"]
    M = fp["info"]["M"]
    flops = legendre_fp64_work(fp["info"]["leg_triples"])
    peak = FP64_PEAK_TFLOPS * 0.75
    traffic = {}
    prof = os.path.join(ROOT, "profiles", "legendre_traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as fh:
                tj = json.load(fh)
            if tj.get("kernel_hash") == _kernel_hash():
                traffic = tj.get("bytes_per_launch", {})
        except Exception:
            traffic = {}
    # both Legendre kernels against the FP64 pipe; the top-level entry is the
    # slower (dominant) one.  Stage times are the library's CUDA events on the
    # launching stream (the adjoint stage includes the 0.3 ms partial-sum
    # reduction kernel).
    leg = {}
    for kname, direction in (("legendre_synth_df_k", "synth"), ("legendre_adj_df_k", "adjoint")):
        t_leg = fp["stages"][direction]["legendre"] * 1e-3
        ach = flops / t_leg / 1e12
        leg[kname] = {"ms": t_leg * 1e3, "achieved": ach, "frac": ach / peak, "traffic": traffic.get(kname)}
    dom = max(leg, key=lambda k: leg[k]["ms"])
    roofline = {"bound": "alu", "achieved": leg[dom]["achieved"], "peak": peak, "unit": "TFLOP/s",
                "frac": leg[dom]["frac"], "traffic": leg[dom]["traffic"],
                "kernel": dom + ": FP64 recurrence (1 DMUL + 1 DFMA = 3 flops per triple) on the FP64 pipe; "
                                "peak = 152 SMs x 2 FP64 FMA lanes/clk x 2.07 GHz x 3 flops / 2 slots (nominal; "
                                "no FP64 figure in the measured peaks)",
                "flops_per_launch": flops, "triples_per_launch": fp["info"]["leg_triples"],
                "per_kernel": leg}
    cpu = None
    if not args.no_cpu:
        nsample = int(os.environ.get("NUSHT_CPU_SAMPLE", "200"))
        sec, threads, _ = cpu_oracle_step(a, pts, L, nsample)
        cpu = {"value": 1e3 * sec * npts / nsample, "unit": "ms", "cores": threads, "kind": "oracle",
               "extrapolated": True,
               "sample": "%d seeded points (synthesis + adjoint over all orders), scaled by N/%d; "
                         "the direct sum is exactly linear in N" % (nsample, nsample)}
    # synthesis: scale_alm_df, legendre_synth_df, poles_synth, theta DFT, column pass, row pass, interp_df;
    # adjoint: spread_df, row pass, column pass, theta DFT, legendre_adj_df, adj_reduce_df
    launches_per_step = 13
    line = {
        "metric": METRIC, "value": fp["ms"] / world, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": fp["ms"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 recurrence; double-float (float pairs, ~2^-47 per op) contraction, FFTs, NUFFT",
        "data": "synthetic",
        "config": {"workload": "deflected GL grid %dx%d (%d pts), lmax=mmax=%d, "
                               "C_l=(l+1)^-2 Gaussian a_lm, 2.5 arcmin rms deflection" % (L + 1, 2 * L + 1, npts, L),
                   "eps": 1e-10, "precision": "NUSHT_FP64 (default options)", "sigma": fp["info"]["sigma"],
                   "w": fp["info"]["w"],
                   "fine_grid": [fp["info"]["n1"], fp["info"]["n2"]], "M": M,
                   "l2": "inputs larger than L2 (%d^2 fine grid, %d points)" % (fp["info"]["n1"], npts),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "synth_ms": fp["stages"]["synth"]["total"], "adjoint_ms": fp["stages"]["adjoint"]["total"],
        "stages_ms": fp["stages"], "eps_eff": fp["eps_eff"], "plan_s": fp["plan_s"],
        "step_ms_median": fp["median"], "step_ms_std": fp["std"],
        "roofline": roofline, "e2e": results.get("e2e"),
        "gpu_launches": launches_per_step * args.steps,
        "clocks": fp["clocks"], "peak_source": peak_src,
    }
    if "mixed" in results:
        mx = results["mixed"]
        line["mixed"] = {"ms_per_step": mx["ms"], "step_ms_median": mx["median"], "step_ms_std": mx["std"],
                         "eps": 1e-5, "eps_eff": mx["eps_eff"], "plan_s": mx["plan_s"],
                         "plan_GB": mx["info"]["bytes_device"] / 1e9,
                         "synth_ms": mx["stages"]["synth"]["total"], "adjoint_ms": mx["stages"]["adjoint"]["total"],
                         "stages_ms": mx["stages"], "w": mx["info"]["w"], "sigma": mx["info"]["sigma"],
                         "dtype": "f64 recurrence (once, at plan time: the mixed default) / f32 contraction, FFT, "
                                  "NUFFT", "clocks": mx["clocks"],
                         "nufft_roofline": mixed_nufft_roofline(mx, npts, peaks["hbm_gbs"])}
    if "fp64_strict" in results:
        r = results["fp64_strict"]
        line["fp64_strict"] = {"ms_per_step": r["ms"], "eps_eff": r["eps_eff"],
                               "synth_ms": r["stages"]["synth"]["total"],
                               "adjoint_ms": r["stages"]["adjoint"]["total"], "stages_ms": r["stages"],
                               "dtype": "f64 instructions in every stage",
                               "what": "opts.fp64_contraction=1, opts.fft_kernels=-1: Legendre sums, spreading and "
                                       "interpolation with FP64 instructions, cuFFT FP64 transforms"}
    for key in ("fp64_table", "mixed_percall"):
        if key in results:
            r = results[key]
            line[key] = {"ms_per_step": r["ms"], "eps_eff": r["eps_eff"], "plan_s": r["plan_s"],
                         "synth_ms": r["stages"]["synth"]["total"], "adjoint_ms": r["stages"]["adjoint"]["total"],
                         "legendre_ms": [r["stages"]["synth"]["legendre"], r["stages"]["adjoint"]["legendre"]],
                         "plan_GB": r["info"]["bytes_device"] / 1e9,
                         "what": ("opts.legendre_table=1: the FP64 recurrence runs once at plan time and its "
                                  "values stay in HBM; each call streams them") if key == "fp64_table" else
                                 ("opts.legendre_table=-1: the FP64 recurrence runs in every call")}
    for key in ("fp64_fast_recurrence", "mixed_fast_recurrence"):
        if key in results:
            r = results[key]
            line[key] = {"ms_per_step": r["ms"], "eps_eff": r["eps_eff"],
                         "synth_ms": r["stages"]["synth"]["total"], "adjoint_ms": r["stages"]["adjoint"]["total"],
                         "legendre_ms": [r["stages"]["synth"]["legendre"], r["stages"]["adjoint"]["legendre"]],
                         "what": "opts.fast_recurrence=1 (opt-in): the P_lm recurrence in double-float on the FP32 "
                                 "pipe instead of FP64"}
    if pointing is not None:
        line["pointing"] = pointing
    if autograd is not None:
        line["autograd"] = autograd
    if spin is not None:
        line["spin2"] = spin
    if batch is not None:
        line["batch64"] = batch
    if batch_fp64 is not None:
        line["batch64_fp64"] = batch_fp64
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def mixed_nufft_roofline(r, npts: int, hbm_gbs: float) -> dict:
    """HBM roofline of the mixed-mode interpolation (interp_f_k) and
    spreading (spread_pt_k) stages.  Algorithmic bytes per launch: the part
    of the doubled float fine grid that points with theta in [0, pi] touch,
    (n1 / 2 + w) rows x (n2 + 2) x 4 B (read when interpolating,
    read-modify-written when spreading), + 24 B per point (sorted first taps
    8 B, offsets 8 B, permutation 4 B, the value 4 B); divided by the stage's
    CUDA-event time.  A one-pass ncu capture of the full-size launches
    measures the same bytes in DRAM (no re-reads)."""
    z = r["info"]
    grid = (z["n1"] // 2 + z["w"]) * (z["n2"] + 2) * 4
    out = {"peak_gbs": hbm_gbs}
    for kname, direction, stage, ngrid in (("interp_f_k", "synth", "interp", 1),
                                           ("spread_pt_k", "adjoint", "spread", 2)):
        nbytes = ngrid * grid + 24 * npts
        ms = r["stages"][direction][stage]
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[kname] = {"ms": ms, "bytes_per_launch": nbytes, "achieved_gbs": gbs, "frac": gbs / hbm_gbs}
    return out


def run_pointing(torch, nu, args, dist, L):
    """CMB lensing pointing (App. C) on the undeflected Gauss-Legendre grid of
    the workload's lmax, for a synthetic potential of 2.5 arcmin rms
    deflection: milliseconds per call (synthesis of the potential to the fine
    grid, derivative-of-kernel interpolation and the deflection per point),
    FP64 at eps 1e-10."""
    pts = W.gl_ring_grid(L + 1, 2 * L + 1)
    phi = W.phi_lensing(L, seed=7)
    dpts = torch.from_numpy(pts).cuda()
    plan = nu.Plan(L, dpts, eps=EPS["fp64"], precision="fp64")
    ph = torch.from_numpy(phi).cuda()
    out = torch.empty((pts.shape[0], 2), dtype=torch.float64, device="cuda")

    def step():
        plan.pointing(ph, out=out)

    ms = max_over_ranks(dist, time_steps(torch, step, args.steps, args.warmup, dist))
    # angle between each sampled point and its deflected position
    sub = pts[::997]
    o = out[::997].cpu().numpy()

    def unit(p):
        return np.stack([np.sin(p[:, 0]) * np.cos(p[:, 1]), np.sin(p[:, 0]) * np.sin(p[:, 1]), np.cos(p[:, 0])], 1)

    moved = np.arccos(np.clip(np.sum(unit(sub) * unit(o), 1), -1.0, 1.0))
    plan.close()
    del dpts, ph, out
    torch.cuda.empty_cache()
    return {"ms": ms, "lmax": L, "npts": int(pts.shape[0]),
            "workload": "undeflected GL grid %dx%d, lensing potential C_l ~ [l(l+1)]^-1 (1+l/60)^-3, "
                        "2.5 arcmin rms deflection (seed 7)" % (L + 1, 2 * L + 1),
            "rms_deflection_arcmin": float(np.sqrt(np.mean(moved**2)) * 180 * 60 / np.pi)}


def run_spin(torch, nu, args, dist, rank, L, pts):
    """Spin-2 synthesis + adjoint (Q + iU = sum (G + iC) 2Y_lm and its
    transpose; the spin-n generalisation of the Conclusion, Sec. 5) on the
    workload's points, FP64 at eps 1e-10: ms per step, and eps_eff of (Q, U)
    against the oracle's direct sum on a seeded sample of points."""
    npts = pts.shape[0]
    g = W.alm_gaussian(L, seed=41, spectrum="inv_l1_sq")
    c = W.alm_gaussian(L, seed=42, spectrum="inv_l1_sq")
    dpts = torch.from_numpy(pts).cuda()
    t0 = time.perf_counter()
    plan = nu.Plan(L, dpts, eps=EPS["fp64"], precision="fp64", spin=2)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    dg, dc = torch.from_numpy(g).cuda(), torch.from_numpy(c).cuda()
    rng = np.random.default_rng(43)
    yq = torch.from_numpy(rng.standard_normal(npts)).cuda()
    yu = torch.from_numpy(rng.standard_normal(npts)).cuda()

    def step():
        plan.synth_spin(dg, dc)
        plan.adjoint_spin(yq, yu)

    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms = max_over_ranks(dist, time_steps(torch, step, args.steps, args.warmup, dist))
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    q, u = plan.synth_spin(dg, dc)
    e[1].record()
    plan.adjoint_spin(yq, yu)
    e[2].record()
    torch.cuda.synchronize()
    par = None
    if rank == 0:
        import oracle

        sel = W.subset(npts, 200, seed=44)
        rq, ru = oracle.spin_synth(g, c, pts[sel], L, 2)
        got = np.concatenate([q.cpu().numpy()[sel], u.cpu().numpy()[sel]])
        par = oracle.eps_eff(np.concatenate([rq, ru]), got)
    nbytes = plan.info()["bytes_device"]
    plan.close()
    del dpts, dg, dc, yq, yu, q, u
    torch.cuda.empty_cache()
    return {"ms_per_step": ms, "synth_ms": e[0].elapsed_time(e[1]), "adjoint_ms": e[1].elapsed_time(e[2]),
            "eps_eff": par, "eps_eff_sample": 200, "plan_s": t_plan, "plan_GB": nbytes / 1e9, "spin": 2,
            "what": "FP64 Wigner-d recurrences (both +-s chains per ring pair), float-pair sums on the FP32 pipe, "
                    "passes whose values stay below 2^-300 skipped; theta FFT, fine-grid FFT and NUFFT once per "
                    "field (Q, U)", "clocks": clk.summary()}


def run_autograd(torch, nu, args, dist):
    """The differentiable transform (autograd) on the lmax 2047 deflected GL
    grid (8,386,560 points), FP64 at eps 1e-10: one forward synthesis and the
    backward pass of L = sum_i w_i f_i^2 (the adjoint for dL/da_lm, the
    derivative-of-kernel interpolation for dL/d(theta, phi)), ms per step."""
    L, a, pts = W.workload("gl2047")
    n = pts.shape[0]
    w = torch.from_numpy(np.random.default_rng(1).uniform(0, 1, n)).cuda()
    dpts = torch.from_numpy(pts).cuda()
    plan = nu.Plan(L, dpts, eps=EPS["fp64"], precision="fp64")
    ad = torch.from_numpy(a).cuda()

    def step():
        alm = ad.detach().requires_grad_(True)
        dp = dpts.detach().requires_grad_(True)
        f = nu.nusht(alm, dp, plan)
        (w * f * f).sum().backward()

    ms = max_over_ranks(dist, time_steps(torch, step, args.steps, args.warmup, dist))
    plan.close()
    del dpts, ad, w
    torch.cuda.empty_cache()
    return {"ms": ms, "lmax": L, "npts": int(n), "precision": "fp64", "eps": EPS["fp64"],
            "workload": "deflected GL grid 2048x4095, L = sum_i w_i f_i^2, w_i ~ U[0, 1) (seed 1)",
            "what": "forward synthesis + backward (grad a_lm and grad (theta, phi))"}


def run_sweep(torch, nu, args):
    """eps in {1e-2, 1e-6, 1e-10} x sigma in {1.25, 1.5, 2} (FP64; mixed for
    eps >= 1e-6) on a deflected GL grid (--sweep-workload, lmax 1023 by
    default): eps_eff against the oracle on a seeded subset (3000 points, 600
    at lmax 4095), milliseconds per synthesis + adjoint and the per-stage
    split, as the paper's accuracy/operator breakdown does."""
    import oracle

    L, a, pts = W.workload(args.sweep_workload)
    npts = pts.shape[0]
    dpts = torch.from_numpy(pts).cuda()
    sel = W.subset(npts, 3000 if L <= 2047 else 600, seed=18)
    f_ref = oracle.synth(a, pts[sel], L)
    y_host = np.random.default_rng(6).standard_normal(npts)
    out = []
    for prec in ("fp64", "mixed"):
        cd = torch.complex128 if prec == "fp64" else torch.complex64
        rd = torch.float64 if prec == "fp64" else torch.float32
        ad = torch.from_numpy(a).to(cd).cuda()
        y = torch.from_numpy(y_host).to(rd).cuda()
        for eps in (1e-2, 1e-6, 1e-10):
            if prec == "mixed" and eps < 1e-6:
                continue
            for sigma in (1.25, 1.5, 2.0):
                try:
                    plan = nu.Plan(L, dpts, eps=eps, precision=prec, sigma=sigma, profile=True)
                except Exception as e:  # width beyond the kernel limit
                    out.append({"precision": prec, "eps": eps, "sigma": sigma, "unavailable": str(e)})
                    continue

                def step():
                    plan.synth(ad)
                    plan.adjoint(y)

                ms = time_steps(torch, step, 3, 2, None)
                f = plan.synth(ad).double().cpu().numpy()
                st = stage_breakdown(torch, plan, ad, y)
                info = plan.info()
                out.append({"precision": prec, "eps": eps, "sigma": sigma, "w": info["w"],
                            "fine_grid": info["n1"], "eps_eff": oracle.eps_eff(f_ref, f[sel]), "ms_per_step": ms,
                            "stages_ms": st})
                plan.close()
                torch.cuda.empty_cache()
    return {"workload": "deflected GL grid %dx%d (%d pts), lmax=mmax=%d" % (L + 1, 2 * L + 1, npts, L),
            "oracle_sample": int(sel.size), "runs": out}


def run_batch64(torch, nu, args, dist, rank, sequential=True, precision="mixed"):
    """64 independent transforms, lmax_b ~ U{256..2047}, N_b = 2 lmax_b^2 uniform
    points: one batched plan (shared-ring buckets, graph replay) against the
    same transforms run one by one through standalone plans of the same
    precision.  "mixed": complex64 a_lm, float32 maps, eps 1e-5 (TF32-split
    tensor-core contraction); "fp64": the same coefficients as complex128,
    float64 maps, eps 1e-10 (bf16-sliced tensor-core contraction)."""
    fp64 = precision == "fp64"
    eps = 1e-10 if fp64 else 1e-5
    cdt = torch.complex128 if fp64 else torch.complex64
    rdt = torch.float64 if fp64 else torch.float32
    members = W.batch64(nbatch=args.batch_n, lmax=args.batch_lmax)
    ls = [m[0] for m in members]
    dpts = [torch.from_numpy(m[2]).cuda() for m in members]
    alms = [torch.from_numpy(m[1]).to(cdt).cuda() for m in members]
    ys = [torch.randn(d.shape[0], dtype=rdt, device="cuda") for d in dpts]
    t0 = time.perf_counter()
    bp = nu.BatchPlan(ls, dpts, eps=eps, precision=precision)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    fo = [torch.empty(d.shape[0], dtype=rdt, device="cuda") for d in dpts]
    co = [torch.empty(nu.nalm(l), dtype=cdt, device="cuda") for l in ls]

    def step():
        bp.synth(alms, fo)
        bp.adjoint(ys, co)

    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms = max_over_ranks(dist, time_steps(torch, step, args.steps, args.warmup, dist))
    info = bp.info()
    # parity on sampled members (largest, smallest, median lmax)
    par = None
    if rank == 0:
        import oracle

        order = np.argsort(ls)
        errs = []
        for i in [int(order[-1]), int(order[0]), int(order[len(ls) // 2])]:
            sel = W.subset(dpts[i].shape[0], 200, seed=i)
            ref = oracle.synth(members[i][1].astype(np.complex128), members[i][2][sel], ls[i])
            errs.append(oracle.eps_eff(ref, fo[i].double().cpu().numpy()[sel]))
        par = max(errs)
    bp.close()
    torch.cuda.synchronize()
    # the same transforms one by one (standalone plans, same eps / precision)
    seq = 0.0
    for i in range(len(ls) if sequential else 0):
        pl = nu.Plan(ls[i], dpts[i], eps=eps, precision=precision)
        f = torch.empty_like(fo[i])
        c = torch.empty_like(co[i])

        def one():
            pl.synth(alms[i], out=f)
            pl.adjoint(ys[i], out=c)

        seq += time_steps(torch, one, 2, 3, None)
        pl.close()
    torch.cuda.empty_cache()
    return {"workload": "%d transforms, lmax ~ U{256..%d} (seed 0), N_b = 2 lmax_b^2 uniform points "
                        "(%d total), %s, eps %g" % (args.batch_n, args.batch_lmax,
                                                    sum(int(d.shape[0]) for d in dpts),
                                                    "complex128" if fp64 else "complex64", eps),
            "precision": precision,
            "ms_per_step": ms, "sequential_ms_per_step": seq if sequential else None,
            "speedup_vs_sequential": seq / ms if sequential else None,
            "buckets": info["nbuckets"], "bucket_lmax": info["bucket_lmax"], "plan_s": t_plan,
            "eps_eff_max_sampled": par, "clocks": clk.summary()}


def _kernel_hash() -> str:
    import hashlib

    h = hashlib.sha1()
    for f in ("legendre.cu", "recurrence.cuh", "dfloat.cuh"):
        with open(os.path.join(ROOT, "paper_2406_14542_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


if __name__ == "__main__":
    main()
