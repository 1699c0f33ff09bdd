#!/usr/bin/env python
"""Benchmark of the map-maker's hot path on the ACT-like patch (1024 detectors x
2^20 samples, 1200x900 TQU map at 0.5', FP32 time-ordered data with FP64 CG).

A step is one iteration of circulant-preconditioned conjugate gradients: one
application of A = P^T N^-1 P (pointing, gather, noise filter, binning), the
FP64 CG vector updates and one application of the circulant preconditioner
(2-D FFTs and the per-mode 3x3 solve).  ``value`` is samples per second per
A-application inside that loop (N_s / time per iteration), with all inputs
resident in HBM.  The time-ordered spectra streamed every step (4.3 GB) exceed
L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "samples/s per P^T N^-1 P apply (inside circulant PCG)"
UNIT = "samples/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["f32", "f64", "bf16"], default="f32")
    ap.add_argument("--n-det", type=int, default=1024)
    ap.add_argument("--n-t", type=int, default=1 << 20)
    ap.add_argument("--det-chunk", type=int, default=0)
    ap.add_argument("--taper", type=float, default=10.0,
                    help="Gaussian taper of the circulant preconditioner in pixels (10: best of the sweep "
                         "{5, 10, 20, 40, inf} on this scan; the paper's ACT value 20 is solved beside it)")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-1e-6 solves")
    ap.add_argument("--pointing", choices=["cached", "on-the-fly"], default="on-the-fly",
                    help="on-the-fly: pixels recomputed from the boresight and detector offsets in both "
                         "column passes of every application (the method's pointing, no stored P); cached: "
                         "a pixel index per sample stored once (4 B/sample), timed beside it")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--corr-modes", type=int, default=0,
                    help="noise correlated between detectors: r focal-plane modes (common, x, y gradient)")
    ap.add_argument("--workload", choices=["apply", "learned", "batch", "anorm", "spectra", "unet"], default="apply",
                    help="apply: the A-application inside circulant PCG (default); learned: the learned "
                         "correction on 64x64 patches (train on 90 realisations, evaluate on 20)")
    ap.add_argument("--batch", type=int, default=64, help="solves of the batch workload")
    ap.add_argument("--batch-iters", type=int, default=20, help="PCG iterations timed per solve")
    ap.add_argument("--batch-small", action="store_true",
                    help="batch workload at the small corner of its distribution: every solve 128 detectors "
                         "x 2^18 samples on a 256x256 TQU map")
    ap.add_argument("--learned-reals", type=int, default=220,
                    help="realisations of the learned workload (90 percent train: about 20k pairs)")
    ap.add_argument("--learned-epochs", type=int, default=15)
    ap.add_argument("--learned-rounds", type=int, default=2,
                    help="on-policy rounds: pairs from the corrected solves themselves, then more training")
    return ap.parse_args()


def workload(args):
    return {"workload": f"ACT-like patch: {args.n_det} det hex 1 deg, {args.n_t} samples/det at 400 Hz, "
                        f"10 deg throw rising+setting, 1200x900 TQU CAR 0.5'",
            "n_det": args.n_det, "n_samp": args.n_t, "map": [3, 900, 1200],
            "precon": "circulant", "taper_sigma_px": args.taper, "pointing": args.pointing,
            "noise": f"correlated, {args.corr_modes} focal-plane modes" if args.corr_modes > 0 else "independent detectors",
            "l2": "no flush: 4.3 GB of spectra streamed per step exceed the 129 MB L2"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"cmm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is running
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        with open(self.path) as fh:
            lines = fh.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        return summarize_clocks(lines)


def summarize_clocks(lines):
    """Median SM clock under load (samples drawing more than 200 W, else all), the
    maximum SM clock and the throttle reasons seen active, from nvidia-smi rows in
    ClockSampler.FIELDS order (csv, no header, no units); None without a valid row."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
        except ValueError:
            continue
    if not rows:
        return None
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower().startswith("active")})
    loaded = [r for r in rows if r[2] > 200.0] or rows
    return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
            "reasons": reasons, "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


# ---------------------------------------------------------------- oracle timing
ORACLE_DETS = 4   # detectors per worker's sample


def _oracle_worker(job):
    """One host core: the FP64 oracle's A-application on its own ORACLE_DETS
    detectors of the workload, repeated for `seconds` after one untimed warm-up.
    Returns (samples processed, seconds)."""
    n_det, n_t, rank, first, seconds = job
    import numpy as np

    import gen
    from oracle import mapmaker as om
    scan, noise = gen.act_patch(real=rank, n_det=n_det, n_t=n_t)
    dets = (first + np.arange(ORACLE_DETS)) % scan.n_det
    sub, nsub = scan.subset(dets), noise.subset(dets)
    op = om.make_operator(sub, nsub, om.pixel_mask(sub))
    m = gen.sky_map(scan.ny, scan.nx, cfg=2, real=rank)
    om.apply_A(op, m)
    t0 = time.perf_counter()
    reps = 0
    while True:
        om.apply_A(op, m)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps * ORACLE_DETS * scan.n_t, el


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


class OraclePool:
    """Worker processes for the oracle timing, one per host core, started with the
    spawn method (no fork of a process that holds a CUDA context).  Each worker
    runs the plain oracle on a disjoint set of detectors; numpy's threads are
    limited to one per worker."""

    def __init__(self):
        import multiprocessing as mp
        self.cores, self.model = host_cpu()
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(var, "1")
        self.pool = mp.get_context("spawn").Pool(self.cores)

    def rate(self, args, seconds, rank=0):
        jobs = [(args.n_det, args.n_t, rank, k * ORACLE_DETS, seconds) for k in range(self.cores)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t0
        samples = sum(r[0] for r in res)
        span = max(r[1] for r in res)
        rate = samples / span
        sample = (f"{self.cores} processes x FP64 oracle A-applications of {ORACLE_DETS} of {args.n_det} "
                  f"detectors ({ORACLE_DETS * args.n_t} samples each), {samples / (ORACLE_DETS * args.n_t):.0f} "
                  f"applications in {span:.1f} s ({wall:.1f} s with set-up)")
        return rate, sample

    def close(self):
        self.pool.close()
        self.pool.join()

    def baseline(self, rate, sample):
        return {"value": rate, "unit": UNIT, "cores": self.cores, "kind": "oracle", "sample": sample,
                "nproc": self.cores, "cpu_model": self.model}


def oracle_solve_estimate(rate, n_s, solves):
    """The oracle's time to solve the whole workload to 1e-6, estimated (a full FP64
    CPU solve of 10^9 samples over hundreds of iterations takes hours): one
    A-application of all n_s samples at the measured oracle rate, times the
    circulant PCG iterations the GPU needed.  None without that solve."""
    circ = (solves or {}).get("circulant")
    if not circ or not rate:
        return None
    return {"value": n_s / rate * circ["iterations"], "unit": "s", "iterations": circ["iterations"],
            "what": "estimate, not run: oracle samples/s over one A-application of the workload, "
                    "times the GPU's circulant iterations to 1e-6"}


def job_ms(ms, world, device):
    """The job's time: the slowest rank's (max over ranks; the ranks ran after a barrier)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(n_s_per_rank, steps, ms, world):
    """Whole-job throughput: the samples every rank processed over the job's time
    (replicas: each rank solves its own realisation of the same size)."""
    return world * n_s_per_rank * steps / (ms / 1e3)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch

    import gen
    from paper_1309_7473_gb300 import build
    build.build()
    from paper_1309_7473_gb300 import cmm

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    prec = {"f32": cmm.PREC_F32, "f64": cmm.PREC_F64, "bf16": cmm.PREC_BF16}[args.prec]
    t_setup = time.perf_counter()
    scan, noise = gen.act_patch(real=rank, n_det=args.n_det, n_t=args.n_t)
    n_s = scan.n_det * scan.n_t
    with torch.cuda.stream(stream):
        ctx = cmm.Context(dev, stream=stream.cuda_stream)
        op = cmm.Operator(ctx, scan, noise, precision=prec, det_chunk=args.det_chunk,
                          corr=gen.corr_noise(scan.det_off, r=args.corr_modes) if args.corr_modes > 0 else None)
        if args.pointing == "cached" and prec != cmm.PREC_F64:
            op.set_pixel_cache(True)
        m_sky = torch.as_tensor(gen.sky_map(scan.ny, scan.nx, cfg=2, real=rank), device=f"cuda:{dev}")
        tod = op.project(m_sky)                 # noise-free TOD, as in the paper's test
        b = op.rhs(tod)
        del tod
        t_pc = time.perf_counter()
        pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=args.taper)
        stream.synchronize()
        t_pc = time.perf_counter() - t_pc
    setup_s = time.perf_counter() - t_setup

    def iterate(k):
        x = op.new_map()
        # k iterations in one captured graph launch; the exit check of ||b - A x||
        # is not a PCG iteration and stays out of the timed steps
        cmm.cmm_solve(op.h, pc.h, b, x, 0.0, k, k, True, False, None, None, true_resid=False)

    with torch.cuda.stream(stream):
        iterate(args.warmup)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            torch.cuda.synchronize()
            ev0.record(stream)
            iterate(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    ms = job_ms(ms, world, f"cuda:{dev}")
    ms_step = ms / args.steps
    value = job_value(n_s, args.steps, ms, world)

    # per-pass durations of the A-application (CUDA events between its kernels),
    # and the same with the other pointing mode beside it
    with torch.cuda.stream(stream):
        mo = op.new_map()
        prof = cmm.cmm_profile_apply(op.h, b, mo, 5)
        prof_other = None
        prof_single = None
        if prec != cmm.PREC_F64:
            cached = args.pointing == "cached"
            op.set_pixel_cache(not cached)
            prof_other = cmm.cmm_profile_apply(op.h, b, mo, 3)
            op.set_pixel_cache(cached)
            torch.cuda.empty_cache()
            # the one-detector packing of the time-ordered FFTs, timed beside it
            op.set_pair_packing(False)
            prof_single = cmm.cmm_profile_apply(op.h, b, mo, 3)
            op.set_pair_packing(True)
    fast = args.prec != "f64" and (1 << 13) <= scan.n_t <= (1 << 20)   # the register-FFT kernels
    # two detectors per complex FFT unless the noise is correlated between detectors
    pre = ("k_pair_" if args.corr_modes == 0 else "k_fast_") if fast else "k_tod_"
    names = [pre + "fwd (pointing + gather + column FFTs)", pre + "filter (row FFTs + N^-1)",
             pre + "inv_bin (inverse column FFTs + P^T)"]
    chunk_dets = min(op_chunk(op, scan, args), scan.n_det)
    elt = {"f32": 8, "bf16": 4, "f64": 16}[args.prec]
    # filter pass: 8 B/sample; with correlated noise split (r+w) + cross-detector read + merge (r+w)
    filter_bytes = (elt * 5 // 2 if args.corr_modes > 0 else elt) * chunk_dets * scan.n_t
    per_launch_bytes = [elt // 2 * chunk_dets * scan.n_t, filter_bytes, elt // 2 * chunk_dets * scan.n_t]
    dom = int(np.argmax(prof[:3]))
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    achieved = per_launch_bytes[dom] / (prof[dom] / 1e3) / 1e9
    apply_bytes = (elt + per_launch_bytes[1] // (chunk_dets * scan.n_t)) * n_s + 16 * scan.n_t + scan.npix * (3 * 8 * 2 + 16 * 2)
    apply_gbs = apply_bytes / (prof[4] / 1e3) / 1e9
    traffic = measured_traffic(dom, chunk_dets, args)

    cufft = cufft_filter_ms(scan, noise, dev, stream) if args.prec == "f32" else None

    # end to end through the host-buffer solve (cmm_solve_host): the same steps as
    # `value` (K circulant-PCG iterations) with b copied in from pinned host memory
    # and the iterate x copied back, host wall clock around the call
    b_host = torch.empty((3, scan.ny, scan.nx), dtype=torch.float64).pin_memory()
    b_host.copy_(b.cpu())
    x_host = torch.zeros_like(b_host).pin_memory()
    bh, xh = b_host.numpy(), x_host.numpy()
    map_bytes = 3 * scan.npix * 8
    with torch.cuda.stream(stream):
        cmm.cmm_solve_host(op.h, pc.h, bh, xh, tol=0.0, maxit=args.warmup, check_every=args.warmup,
                           true_resid=False)
        t0 = time.perf_counter()
        cmm.cmm_solve_host(op.h, pc.h, bh, xh, tol=0.0, maxit=args.steps, check_every=args.steps,
                           true_resid=False)
        e2e_s = (time.perf_counter() - t0) / args.steps
        # and a whole solve to 1e-6 from host b to host x (preconditioner already built)
        info_e2e, e2e_solve_s = None, None
        if not args.no_solve:
            t0 = time.perf_counter()
            info_e2e = cmm.cmm_solve_host(op.h, pc.h, bh, xh, tol=1e-6, maxit=2000, check_every=10)
            e2e_solve_s = time.perf_counter() - t0

    solves = None
    if not args.no_solve:
        solves = {}
        with torch.cuda.stream(stream):
            for name, kind, kw in (("binned", cmm.PRECON_BINNED, {}),
                                   ("jacobi", cmm.PRECON_JACOBI, {}),
                                   ("circulant", cmm.PRECON_CIRCULANT, {"taper_sigma_px": args.taper}),
                                   ("circulant_taper20", cmm.PRECON_CIRCULANT, {"taper_sigma_px": 20.0}),
                                   ("circulant_tiled_2x2", cmm.PRECON_CIRC_TILED,
                                    {"taper_sigma_px": args.taper, "tiles": (2, 2)})):
                if name == "circulant_taper20" and args.taper == 20.0:
                    continue
                t1 = time.perf_counter()
                p2 = pc if name == "circulant" else cmm.Precon(op, kind, **kw)
                torch.cuda.synchronize()
                build_s = t_pc if name == "circulant" else time.perf_counter() - t1
                x, info, _, _ = cmm.solve(op, p2, b, tol=1e-6, maxit=2000, check_every=10)
                solves[name] = {"iterations": info.iterations, "status": cmm.STATUS[info.status],
                                "seconds": round(info.seconds, 4), "build_seconds": round(build_s, 4),
                                "rel_resid": info.rel_resid, "true_rel_resid": info.true_rel_resid}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f32": "f32 (FP64 CG)", "f64": "f64", "bf16": "bf16-storage/f32"}[args.prec],
        "data": "synthetic (seeded ACT-like scan, C_l ~ l^-2 sky, noise-free TOD as in the paper's test)",
        "config": {**workload(args), "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "global_batch": world, "seq_len": scan.n_t},
        "gpu_launches": None,
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic,
                     # the ncu DRAM bytes of the pass over its CUDA-event time: what HBM actually moved
                     "dram_frac": None if traffic is None else traffic / (prof[dom] / 1e3) / 1e9 / peak,
                     "binding_unit": measured_units(dom, args),
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback",
                     "algorithmic_bytes_per_launch": per_launch_bytes[dom]},
        "apply": {"ms": prof[4], "samples_per_s": n_s / (prof[4] / 1e3), "algorithmic_GBps": apply_gbs,
                  "frac_of_measured_hbm": apply_gbs / peak,
                  "ms_per_pass": {"fwd": prof[0], "filter": prof[1], "inv_bin": prof[2], "map_copies": prof[3]},
                  "det_chunk": chunk_dets, "pointing": args.pointing,
                  ("cached_pointing_ms" if args.pointing != "cached" else "on_the_fly_pointing_ms"):
                      None if prof_other is None else prof_other[4],
                  ("cached_pointing_ms_per_pass" if args.pointing != "cached" else "on_the_fly_ms_per_pass"):
                      None if prof_other is None else {"fwd": prof_other[0], "filter": prof_other[1],
                                                       "inv_bin": prof_other[2]},
                  "packing": "two detectors per complex FFT" if prof_single is not None else "one detector",
                  "one_detector_packing_ms": None if prof_single is None else prof_single[4],
                  "one_detector_packing_ms_per_pass": None if prof_single is None else {
                      "fwd": prof_single[0], "filter": prof_single[1], "inv_bin": prof_single[2]}},
        "e2e": {"value": n_s / e2e_s, "unit": UNIT, "h2d_bytes_per_step": map_bytes / args.steps,
                "d2h_bytes_per_step": map_bytes / args.steps, "ms_per_step": 1e3 * e2e_s,
                "step": f"cmm_solve_host: b H2D from pinned host memory, {args.steps} circulant-PCG iterations "
                        "(the timed steps of value), x D2H; host wall clock; copies per call over the steps",
                "solve_to_1e-6": None if info_e2e is None else {
                    "seconds": round(e2e_solve_s, 4), "iterations": info_e2e.iterations,
                    "status": cmm.STATUS[info_e2e.status],
                    "what": "cmm_solve_host from host b to host x, circulant preconditioner "
                            "built beforehand, exit residual check included"}},
        "solves_to_1e-6": solves,
        "cufft_comparison": cufft,
        "setup_seconds": round(setup_s, 2),
        "clocks": clocks,
    }
    out["gpu_launches"] = launches_per_iteration(scan.n_det, chunk_dets) * args.steps + SETUP_LAUNCHES + CIRC_LAUNCHES
    return out


def run_learned(args):
    """Learned correction on the 32-detector 64x64 patch: pairs from FP64 M_C solves
    (to 1e-12) of the first 90% of the training realisations, Adam on the U-Net,
    then PCG(M_C) and flexible PCG(M_C + U) to 1e-6 on 20 held-out realisations."""
    import torch

    import gen
    from paper_1309_7473_gb300 import build
    build.build()
    from paper_1309_7473_gb300 import cmm, learned
    widths = (16, 32, 48, 96)
    ctx = cmm.Context(0)
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=cmm.PREC_F64)
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=8.0)

    def rhs(real):
        m = torch.as_tensor(gen.sky_map(scan.ny, scan.nx, cfg=5, real=real), device="cuda:0")
        d = op.project(m, dtype=torch.float64)
        d += torch.as_tensor(gen.noise_tod(noise, scan.n_t, scan.f_samp, cfg=5, real=real), device="cuda:0")
        return op.rhs(d)

    t0 = time.perf_counter()
    n_train = max(1, (9 * args.learned_reals) // 10)
    parts = [learned.harvest_pairs(op, pc, rhs(r), max_iter=200, tol=1e-12)[:2] for r in range(args.learned_reals)]
    torch.cuda.synchronize()
    harvest_s = time.perf_counter() - t0
    ti = torch.cat([p[0] for p in parts[:n_train]])
    tt = torch.cat([p[1] for p in parts[:n_train]])
    vi = torch.cat([p[0] for p in parts[n_train:]]) if n_train < len(parts) else ti[:32]
    vt = torch.cat([p[1] for p in parts[n_train:]]) if n_train < len(parts) else tt[:32]
    ti, tt = torch.cat([ti, -ti]), torch.cat([tt, -tt])      # the ideal correction is odd in its input
    net = cmm.UNet(ctx, scan.ny, scan.nx, widths, batch_max=32)
    net.init(seed=2)
    t0 = time.perf_counter()
    hist = learned.train(net, ti, tt, epochs=args.learned_epochs, batch=32, lr=1e-3, val=(vi, vt))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    pcl = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=8.0)
    cmm.cmm_precon_set_correction(pcl.h, net.h)
    pcb = cmm.Precon(op, cmm.PRECON_BINNED)
    held_out = list(range(10_000, 10_020))

    def fcg8_mean():
        its = [cmm.solve(op, pcl, rhs(r), tol=1e-6, maxit=1000, flexible=True, window=8)[1].iterations
               for r in held_out[:10]]
        return sum(its) / len(its)

    # on-policy rounds: pairs harvested along the corrected FCG(8) solves of the
    # training realisations themselves, added to the set, a few more epochs
    rounds = [{"round": 0, "fcg8_iterations_mean_10": fcg8_mean(), "pairs": int(ti.shape[0]) // 2}]
    for rd in range(args.learned_rounds):
        new = [learned.harvest_pairs(op, pc, rhs(r), max_iter=200, tol=1e-12, solve_pc=pcl, window=8)[:2]
               for r in range(n_train)]
        ni = torch.cat([p[0] for p in new])
        nt = torch.cat([p[1] for p in new])
        ti, tt = torch.cat([ti, ni, -ni]), torch.cat([tt, nt, -nt])
        learned.train(net, ti, tt, epochs=max(1, args.learned_epochs // 3), batch=32, lr=3e-4, val=(vi, vt),
                      seed=rd + 1)
        rounds.append({"round": rd + 1, "fcg8_iterations_mean_10": fcg8_mean(), "pairs": int(ti.shape[0]) // 2})
    # on 20 held-out realisations: binned PCG, PCG(M_C), the corrected preconditioner
    # in flexible CG (Polak-Ribiere form and FCG(8)), and PCG(M_C) started from the
    # corrected preconditioner applied to b
    forms = {"binned": [], "plain_mc": [], "learned_fpcg": [], "learned_fcg8": [], "learned_x0": [],
             "control_x0_mc": []}

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        info = fn()
        torch.cuda.synchronize()
        return info.iterations, time.perf_counter() - t, info.status

    for real in held_out:
        b = rhs(real)
        forms["binned"].append(timed(lambda: cmm.solve(op, pcb, b, tol=1e-6, maxit=2000)[1]))
        forms["plain_mc"].append(timed(lambda: cmm.solve(op, pc, b, tol=1e-6, maxit=1000)[1]))
        forms["learned_fpcg"].append(timed(lambda: cmm.solve(op, pcl, b, tol=1e-6, maxit=1000)[1]))
        forms["learned_fcg8"].append(timed(lambda: cmm.solve(op, pcl, b, tol=1e-6, maxit=1000, flexible=True,
                                                             window=8)[1]))

        def from_x0(p0):
            x0 = p0.apply(b)
            return cmm.solve(op, pc, b, x=x0, tol=1e-6, maxit=1000)[1]
        forms["learned_x0"].append(timed(lambda: from_x0(pcl)))
        # control: the same start without the network, x0 = M_C b
        forms["control_x0_mc"].append(timed(lambda: from_x0(pc)))
    summary = {k: {"iterations_mean": sum(r[0] for r in v) / len(v), "seconds_mean": sum(r[1] for r in v) / len(v),
                   "all_converged": all(r[2] == 0 for r in v)} for k, v in forms.items()}
    n = len(forms["plain_mc"])
    return {
        "metric": "iterations to 1e-6, corrected preconditioner (FCG(8) with M_C + U-Net) vs PCG(M_C)",
        "unit": "iterations", "higher_is_better": False, "value": summary["learned_fcg8"]["iterations_mean"],
        "n_gpus": 1, "steps": n, "warmup": 0, "dtype": "f64 solve, bf16 network", "data": "synthetic",
        "config": {"workload": "32 det x 2^16 samples, 64x64 TQU, taper 8 px; U-Net widths 16/32/48/96",
                   "realisations": args.learned_reals, "train_realisations": n_train,
                   "pairs_train": int(ti.shape[0]) // 2, "pairs_train_with_sign_flips": int(ti.shape[0]),
                   "epochs": args.learned_epochs},
        "solves": summary,
        "on_policy_rounds": rounds,
        "val_loss": {"zero_output": float(0.5 * (vt.double() ** 2).mean()), "trained": hist[-1][2]},
        "harvest_seconds": round(harvest_s, 2), "train_seconds": round(train_s, 2),
    }


def run_unet(args):
    """U-Net of the learned correction (widths 16/32/48/96, 64x64 TQU maps, batch 32):
    CUDA-event time of one forward pass and of one training step (forward,
    backward, Adam) with the 3x3 convolutions on the tensor cores (BF16 mma.sync,
    FP32 accumulation) and on the FP32 CUDA cores, on the same weights and data."""
    import torch

    from paper_1309_7473_gb300 import build
    build.build()
    from paper_1309_7473_gb300 import cmm
    widths, hw, B = (16, 32, 48, 96), 64, 32
    ctx = cmm.Context(0)
    net = cmm.UNet(ctx, hw, hw, widths, batch_max=B)
    g = torch.Generator(device="cuda:0").manual_seed(0)
    x = torch.randn((B, 3, hw, hw), device="cuda:0", generator=g)
    t = 0.1 * torch.randn((B, 3, hw, hw), device="cuda:0", generator=g)
    y = torch.empty_like(x)
    # multiply-adds of the 3x3 convolutions of one forward pass (the backward pass does twice as many)
    macs, c = 0, 3
    for l, w in enumerate(widths):
        px = (hw >> l) ** 2
        macs += px * 9 * (c * w + w * w)
        c = w
    for l in range(len(widths) - 2, -1, -1):
        px = (hw >> l) ** 2
        macs += px * 9 * (2 * widths[l] * widths[l] + widths[l] * widths[l])
    macs *= B
    out = {"metric": "U-Net forward and training-step time (64x64 TQU, batch 32)", "unit": "ms",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "bf16 (fp32 accumulate)",
           "config": {"workload": "U-Net widths 16/32/48/96, 299,651 parameters, batch 32 of 3x64x64",
                      "conv3_macs_forward": macs}}
    reps = max(5, args.steps)
    for name, tc in (("tensor_cores", True), ("cuda_cores", False)):
        net.init(seed=2)
        cmm.cmm_unet_set_tensor_cores(net.h, tc)
        for _ in range(3):
            cmm.cmm_unet_forward(net.h, x, y)
            cmm.cmm_unet_train_step(net.h, x, t, 1e-4)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        for _ in range(reps):
            cmm.cmm_unet_forward(net.h, x, y)
        e[1].record()
        for _ in range(reps):
            cmm.cmm_unet_train_step(net.h, x, t, 1e-4)
        e[2].record()
        torch.cuda.synchronize()
        fwd, step = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
        out[name] = {"forward_ms": fwd, "train_step_ms": step, "conv3_tflops_forward": 2 * macs / fwd / 1e9}
    out["value"] = out["tensor_cores"]["train_step_ms"]
    out["speedup_train_step"] = out["cuda_cores"]["train_step_ms"] / out["tensor_cores"]["train_step_ms"]
    return out


def cufft_filter_ms(scan, noise, dev, stream):
    """Timed comparison only: the noise filter N^-1 alone (rfft, multiply by w_d(f),
    irfft) on the same [n_det][n_samp] FP32 time-ordered data through cuFFT
    (torch.fft), without the pointing, the gather and the binning that the
    library's three passes also do."""
    import torch
    with torch.cuda.stream(stream):
        g = torch.Generator(device=f"cuda:{dev}").manual_seed(0)
        d = torch.randn((scan.n_det, scan.n_t), device=f"cuda:{dev}", dtype=torch.float32, generator=g)
        f = torch.arange(scan.n_t // 2 + 1, device=f"cuda:{dev}", dtype=torch.float32) * (scan.f_samp / scan.n_t)
        f[0] = f[1]
        sig = torch.as_tensor(noise.sigma, device=f"cuda:{dev}", dtype=torch.float32)[:, None]
        fk = torch.as_tensor(noise.fknee, device=f"cuda:{dev}", dtype=torch.float32)[:, None]
        al = torch.as_tensor(noise.alpha, device=f"cuda:{dev}", dtype=torch.float32)[:, None]
        w = (1.0 / sig ** 2) / (1.0 + (f[None, :] / fk) ** (-al))
        def run():
            return torch.fft.irfft(torch.fft.rfft(d, dim=1) * w, n=scan.n_t, dim=1)
        for _ in range(2):
            run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        del d, w
        torch.cuda.empty_cache()
    return {"what": "N^-1 only via cuFFT (torch.fft rfft * w irfft), FP32, same n_det x n_samp; "
                    "excludes P and P^T", "ms": ms}


def launches_per_iteration(n_det, chunk):
    """Kernels of one circulant-PCG iteration: the A-application (map copy in, per
    chunk one forward and one filter launch and, per 2048 detectors (eight FP32
    partial maps of 256 detectors), one inverse + binning launch and one flush; map
    copy out), the CG update kernels and the circulant preconditioner (Sigma^-1,
    2-D FFTs, per-mode solve)."""
    a = 2
    maps = min(8, max(1, math.ceil(chunk / 256)))
    for d0 in range(0, n_det, chunk):
        nd = min(chunk, n_det - d0)
        a += 2 + 2 * math.ceil(nd / (256 * maps))
    return a + CG_LAUNCHES + CIRC_LAUNCHES


# kernels per iteration outside the A-application (cmm_solve's FP64 PCG step):
# p^T q partials, alpha, x and r update with ||r||^2, convergence check, beta, p update
CG_LAUNCHES = 6
# the circulant apply: Sigma^-1 into the packed planes, 2 + 2 line-FFT passes, the
# per-mode products, Sigma^-1 out of the planes with the r^T z partials
CIRC_LAUNCHES = 7
# once per cmm_solve call before its iterations: b^T b (partials and sum), r0, the
# solver state (plus one preconditioner apply, CIRC_LAUNCHES)
SETUP_LAUNCHES = 4


# sources of the three A-application kernels of the two-detector path: the traffic
# record holds for them only
TRAFFIC_SOURCES = ("tod_pair.cu", "tod_fast.cuh", "fft_reg.cuh", "fft.cuh", "tod_common.cuh", "common.cuh")


def kernel_sources_digest():
    """SHA-256 over the kernels' sources with comments and blank space removed (the
    counters depend on the code, not on its comments)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1309_7473_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def measured_units(dom, args):
    """L1TEX data-pipe and issue-slot utilisation (% of peak) of the dominant pass
    from the same committed ncu capture as the traffic; None when it does not apply
    to the current kernels or configuration."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
        digest = kernel_sources_digest()
    except (OSError, ValueError):
        return None
    key = f"{args.prec}/{args.pointing}/{args.n_t}"
    if rec.get("kernel_sources_sha256") != digest or key not in rec.get("l1tex_pct_of_peak", {}):
        return None
    return {"l1tex_pct_of_peak": rec["l1tex_pct_of_peak"][key][dom],
            "issue_active_pct": rec["issue_active_pct"][key][dom],
            "source": "ncu --set full, profiles/apply_kernels_64x2p20_full.md"}


def measured_traffic(dom, chunk_dets, args):
    """DRAM bytes of the dominant pass over one chunk of detectors (one launch for
    the forward and filter passes; the inverse pass is one launch per 128
    detectors), from the committed ncu summary (bytes per detector, scaled to the
    chunk); None if the kernels' sources have changed since it was taken or no
    summary covers this configuration."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
        digest = kernel_sources_digest()
    except (OSError, ValueError):
        return None
    key = f"{args.prec}/{args.pointing}/{args.n_t}"
    if rec.get("kernel_sources_sha256") != digest or key not in rec.get("bytes_per_detector", {}):
        return None
    return rec["bytes_per_detector"][key][dom] * chunk_dets


def run_anorm(args):
    """Error A-norm against iteration (the paper's Results metric, Fig. 4 analogue)
    for binned and circulant PCG on the 1024-detector patch, with instant and with
    finite-acceleration (1.5 deg/s^2) turnarounds.  The squared error A-norm at
    iteration i is estimated by the sum of the solver's terms alpha_j r_j^T z_j,
    j = i .. i + 3."""
    import numpy as np
    import torch

    import gen
    from paper_1309_7473_gb300 import build
    build.build()
    from paper_1309_7473_gb300 import cmm
    marks = [0, 25, 50, 100, 200, 300, 400, 600]
    out = {"metric": "iterations to 1e-6 and error A-norm^2 estimate vs iteration", "unit": "iterations",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "1024 det x 2^20 samples, 1200x900 TQU, noise-free TOD, FP32 operator, "
                                  f"circulant taper {args.taper} px", "iterations_marked": marks}, "scans": {}}
    for label, acc in (("instant", None), ("accel_1.5deg_s2", 1.5)):
        scan, noise = gen.act_patch(accel_deg_s2=acc)
        ctx = cmm.Context(0)
        op = cmm.Operator(ctx, scan, noise, precision=cmm.PREC_F32)
        op.set_pixel_cache(True)
        m = torch.as_tensor(gen.sky_map(scan.ny, scan.nx, cfg=2), device="cuda:0")
        b = op.rhs(op.project(m))
        rec = {}
        for name, kind, kw in (("binned", cmm.PRECON_BINNED, {}),
                               ("circulant", cmm.PRECON_CIRCULANT, {"taper_sigma_px": args.taper})):
            pc = cmm.Precon(op, kind, **kw)
            x, info, hist, terms = cmm.solve(op, pc, b, tol=1e-6, maxit=2000, history=True)
            t = terms.cpu().numpy()[: info.iterations]
            an = {i: float(t[i:i + 4].sum()) for i in marks if i + 4 <= len(t)}
            rec[name] = {"iterations": info.iterations, "seconds": round(info.seconds, 3),
                         "anorm2": an, "clamped_modes": pc.clamped() if kind == cmm.PRECON_CIRCULANT else None}
        rec["iteration_ratio"] = rec["circulant"]["iterations"] / rec["binned"]["iterations"]
        out["scans"][label] = rec
        del op, pc, b, m
        torch.cuda.empty_cache()
    out["value"] = out["scans"]["accel_1.5deg_s2"]["circulant"]["iterations"]
    return out


def run_spectra(args):
    """Spectrum convergence (Results section, Figs. 7-9 analogue): binned flat-sky
    TT, EE, BB of the PCG iterates (snapshots every 20 iterations) against the input
    map's, and per multipole bin the first iteration after which the difference stays
    below 0.1 of cosmic variance, for binned and circulant PCG on the 1024-detector
    patch."""
    import numpy as np
    import torch

    import gen
    from paper_1309_7473_gb300 import build, diagnostics
    build.build()
    from paper_1309_7473_gb300 import cmm
    every, maxit, nbins = 20, 1000, 20
    pix = np.deg2rad(0.5 / 60)
    lmax = 20000.0
    scan, noise = gen.act_patch()
    ctx = cmm.Context(0)
    op = cmm.Operator(ctx, scan, noise, precision=cmm.PREC_F32)
    op.set_pixel_cache(True)
    m_np = gen.sky_map(scan.ny, scan.nx, cfg=2)
    mask = op.pointing.mask()[0].reshape(scan.ny, scan.nx)
    m_np[:, ~mask] = 0.0
    m = torch.as_tensor(m_np, device="cuda:0")
    b = op.rhs(op.project(m))
    cls_true, nmodes = cmm.cmm_spectra(ctx.h, m, pix, nbins, lmax)
    cls_true = cls_true[0]
    out = {"metric": "CG steps to 0.1 cosmic variance per multipole bin (TT, EE, BB)", "unit": "iterations",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "1024 det x 2^20 samples, 1200x900 TQU, noise-free TOD, FP32 operator; flat-sky "
                                  f"spectra in {nbins} bins to l = {lmax:.0f}, snapshots every {every} iterations",
                      "l_bin_edges": [lmax * k / nbins for k in range(nbins + 1)]},
           "preconditioners": {}}
    slots = maxit // every + 1
    for name, kind, kw in (("binned", cmm.PRECON_BINNED, {}),
                           ("circulant", cmm.PRECON_CIRCULANT, {"taper_sigma_px": args.taper})):
        pc = cmm.Precon(op, kind, **kw)
        snaps = torch.zeros((slots, 2) + tuple(op.shape), dtype=torch.float64, device="cuda:0")
        x = op.new_map()
        info = cmm.cmm_solve(op.h, pc.h, b, x, 1e-6, maxit, 10, True, False, None, None,
                             snapshots=snaps, snapshot_every=every)
        taken = min(slots, info.iterations // every + 1)
        cls_it, _ = cmm.cmm_spectra(ctx.h, snaps[:taken, 0].contiguous(), pix, nbins, lmax)
        iters = np.arange(taken) * every
        steps = diagnostics.steps_to_converge(cls_it, iters, cls_true, nmodes)
        out["preconditioners"][name] = {"iterations_to_1e-6": info.iterations,
                                        "steps_TT": steps[0].tolist(), "steps_EE": steps[1].tolist(),
                                        "steps_BB": steps[2].tolist()}
        del snaps
        torch.cuda.empty_cache()
    st_b = out["preconditioners"]["binned"]
    st_c = out["preconditioners"]["circulant"]
    ratios = {}
    for key in ("steps_TT", "steps_EE", "steps_BB"):
        r = [c / bb for c, bb in zip(st_c[key], st_b[key]) if c > 0 and bb > 0]
        ratios[key.replace("steps_", "")] = float(np.median(r)) if r else None
    out["median_ratio_circulant_over_binned"] = ratios
    out["value"] = ratios["BB"]
    return out


def run_batch(args):
    """Batched Monte-Carlo solves: args.batch seeded problems of uneven size (detectors,
    samples, map), each with its own sky, circulant preconditioner and context;
    args.batch_iters PCG iterations of all of them through cmm_batch_solve (one CUDA
    graph per check interval, problems as parallel branches) against the same
    iterations solved one after another."""
    import torch

    import gen
    from paper_1309_7473_gb300 import build
    build.build()
    from paper_1309_7473_gb300 import cmm
    small = (128, 1 << 18, 256, 256)
    probs = [gen.uneven_problem(k, sizes=small if args.batch_small else None) for k in range(args.batch)]
    n_s = [sc.n_det * sc.n_t for sc, _ in probs]
    # device memory: spectrum chunk (4 B/sample, at most 8 GB) per operator + tables
    need = sum(min(4 * n, 8 << 30) + 32 * sc.n_t + 200 * sc.npix for n, (sc, _) in zip(n_s, probs))
    free, _ = torch.cuda.mem_get_info()
    if need > 0.6 * free:
        raise SystemExit(f"batch needs ~{need / 1e9:.0f} GB, more than 60% of the {free / 1e9:.0f} GB free")
    cache = args.pointing == "cached" and need + 4 * sum(n_s) <= 0.6 * free   # + 4 B/sample of pixel indices
    t0 = time.perf_counter()
    ctxs, ops, pcs, bs, xs = [], [], [], [], []
    for k, (scan, noise) in enumerate(probs):
        ctx = cmm.Context(0)
        op = cmm.Operator(ctx, scan, noise, precision=cmm.PREC_F32)
        if cache:
            op.set_pixel_cache(True)
        m = torch.as_tensor(gen.sky_map(scan.ny, scan.nx, cfg=4, real=k), device="cuda:0")
        bs.append(op.rhs(op.project(m)))
        pcs.append(cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=args.taper))
        ctxs.append(ctx)
        ops.append(op)
        xs.append(op.new_map())
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    it = args.batch_iters
    hs = [o.h for o in ops]
    ph = [p.h for p in pcs]
    cmm.cmm_batch_solve(hs, ph, bs, xs, tol=0.0, maxit=2, check_every=2, true_resid=False)   # warm-up
    torch.cuda.synchronize()
    by_width = {}
    for w in (0, 2, 4, 8):
        t0 = time.perf_counter()
        cmm.cmm_batch_solve(hs, ph, bs, xs, tol=0.0, maxit=it, check_every=it, width=w, true_resid=False)
        torch.cuda.synchronize()
        by_width["auto" if w == 0 else w] = time.perf_counter() - t0
    batched_s = by_width["auto"]
    t0 = time.perf_counter()
    for o, p, b in zip(ops, pcs, bs):
        cmm.solve(o, p, b, tol=0.0, maxit=it, check_every=it, true_resid=False)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    total = sum(n_s) * it
    return {
        "metric": "samples/s per batched P^T N^-1 P apply (circulant PCG, uneven solves)",
        "value": total / batched_s, "unit": "samples/s", "higher_is_better": True, "n_gpus": 1,
        "steps": it, "warmup": 2, "dtype": "f32 (FP64 CG)", "data": "synthetic",
        "config": {"workload": (f"{args.batch} seeded solves, each 128 det x 2^18 samples on 256x256 TQU"
                                if args.batch_small else
                                f"{args.batch} seeded solves: n_det in {{128..1024}}, n_samp in {{2^18..2^20}}, "
                                f"maps 256x256..1200x900 TQU") + f", circulant taper {args.taper} px",
                   "samples_per_iteration": sum(n_s), "pointing": "cached" if cache else "on-the-fly",
                   "sizes": sorted({(sc.n_det, sc.n_t, sc.ny, sc.nx) for sc, _ in probs})[:8]},
        "batched_seconds": batched_s, "batched_seconds_by_width": by_width, "sequential_seconds": seq_s,
        "sequential_samples_per_s": total / seq_s, "speedup": seq_s / batched_s,
        "setup_seconds": round(setup_s, 1),
    }


def op_chunk(op, scan, args):
    if args.det_chunk > 0:
        return args.det_chunk
    elt = {"f32": 8, "bf16": 4, "f64": 16}[args.prec]
    return max(1, (8 << 30) // (elt * scan.n_t // 2))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        pool = OraclePool()
        rates = []
        t_all = time.perf_counter()
        per = max(1.0, args.cpu_seconds / max(1, args.steps))
        pool.rate(args, 0.1)   # warm-up: workers start, import and build their operators
        sample = ""
        for _ in range(args.steps):
            r, sample = pool.rate(args, per)
            rates.append(r)
        pool.close()
        value = statistics.mean(rates)
        el = time.perf_counter() - t_all
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload(args),
            "cpu_baseline": pool.baseline(value, f"{args.steps} steps of: {sample}"),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return 0
    if args.workload == "learned":
        if rank == 0:
            print(json.dumps(run_learned(args)))
        return 0
    if args.workload == "batch":
        if rank == 0:
            print(json.dumps(run_batch(args)))
        return 0
    if args.workload == "unet":
        if rank == 0:
            print(json.dumps(run_unet(args)))
        return 0
    if args.workload == "anorm":
        if rank == 0:
            print(json.dumps(run_anorm(args)))
        return 0
    if args.workload == "spectra":
        if rank == 0:
            print(json.dumps(run_spectra(args)))
        return 0
    # the oracle's worker processes start before this process touches the GPU
    pool = OraclePool() if rank == 0 and world == 1 else None
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if pool is not None:
        rate, sample = pool.rate(args, args.cpu_seconds)
        pool.close()
        out["cpu_baseline"] = pool.baseline(rate, sample)
        out["cpu_baseline"]["solve_to_1e-6_estimate"] = oracle_solve_estimate(
            rate, args.n_det * args.n_t, out.get("solves_to_1e-6"))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
