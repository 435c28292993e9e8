"""Throughput of the brute-force short-coherence search on B300 (template x SFT evals/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--dtype f16|bf16|f32] [--n-sky 10000] [--no-cpu-baseline] [--no-e2e]
                    [--no-batch] [--batch-steps 2]
                    [--workload search|batch|surrogate|binary|inference]

One step = the whole hot path over the search-shaped workload: for every template of the
bank (180 f0 x 20 f1 x 1e4 sky = 3.6e7 templates) and every SFT (2 detectors x 1 yr at 70%
duty = 24,419 SFTs) the track bin, the power gather and the sum, then the critical ratio
and the top-10 per 0.01 Hz sub-band (ft_topk_per_band: one evaluation kernel with the
selection fused in, plus one merge kernel).  Inputs are synthetic (seeded) and resident in
HBM before timing; L2 is flushed (256 MB write) between timed steps, outside the events.

The same line carries: the precision comparison (FP16, BF16 and plain FP32 storage, each
timed on the full bank; relative error and per-sub-band candidate sets against the oracle on
every template of a 1-in-100 sky sub-bank, which is also the CPU baseline's sample); the end-
to-end rate from host buffers; the weighted searches of the same bank (all-sky weights,
number count, count-gated); the batching workload (64 bands at the stated sky density, one
persistent graph-captured launch per step, against the per-band loop); the binary-orbit
track's search; and the surrogate's BF16 inference on the tensor cores.

Other workloads print their own line: the batch alone at a chosen sky density, the
binary-orbit track over a random hyperbox bank, the learned-surrogate study, and the
surrogate's BF16 inference on the tensor cores alone (`inference`).

Under torchrun (N > 1) every rank runs its own replica of the workload (weak scaling, no
data-path collective); rank 0 prints the JSON line.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "template·SFT evals/s on 1 B300, chosen vs plain FP32 at stated rel. error"
UNIT = "evals/s"
SMEM_BYTES_PER_CLK_PER_SM = 128  # 32 banks x 4 B
ESIZE = {"f32": 4, "f16": 2, "bf16": 2}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_desc(sfts, bank, dtype):
    return {
        "workload": "search-shaped band 200.0-200.1 Hz: 2 detectors x 1 yr of 1800 s SFTs at 70% "
                    f"duty ({sfts.n_total} SFTs, {sfts.n_bins}-bin window incl. Doppler/spindown "
                    f"wings); bank {bank.n_f0} f0 x {bank.n_f1} f1 x {bank.n_sky} Fibonacci sky = "
                    f"{bank.n_templates} templates; top-10 per 0.01 Hz sub-band",
        "n_sft": sfts.n_total,
        "n_templates": bank.n_templates,
        "evals_per_step": bank.n_templates * sfts.n_total,
        "storage": dtype,
        "accumulate": "f32 (compensated across SFT stages)",
        "track_bins": "FP64 eps + exact Q32 integer",
        "l2": "flushed between timed steps (256 MB write, outside the per-step events)",
    }


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms",
                 "100", "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def time_steps(fn, steps, warmup, stream, flush):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        flush()
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def cpu_baseline(sfts, bank, target_s, seed=7):
    """The CPU FP64 oracle, as it stands, on a bounded template sample of the same workload,
    sized to run about target_s seconds."""
    import oracle

    g = np.random.default_rng(seed)
    n = 4096
    for _ in range(3):
        samp = g.choice(bank.n_templates, min(n, bank.n_templates), replace=False)
        t0 = time.perf_counter()
        s_or, _ = oracle.statistic(sfts, bank, samp)
        dt = time.perf_counter() - t0
        if dt >= 0.66 * target_s or len(samp) == bank.n_templates:
            break
        n = int(len(samp) * target_s / max(dt, 1e-3))
    evals = len(samp) * sfts.n_total
    return {"value": evals / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{len(samp)} random templates of the same bank x all {sfts.n_total} SFTs "
                      f"({evals:.3g} evals, {dt:.1f} s, FP64, OpenMP over templates)",
            "seconds": dt}, samp, s_or


def profiled_traffic(dtype):
    """DRAM bytes (read + write) per launch of the evaluation kernel from the committed ncu
    capture of this workload, or None when there is none for this storage type or the
    kernel source changed since it was taken."""
    import hashlib

    path = os.path.join(ROOT, "profiles", f"k_eval_fast_search_10000sky_{dtype}_dram.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith((" ", "#", "`")):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2411_18370_b300", "csrc", "ft_eval.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if fields.get("kernel source sha256 prefix") != sha:
        return None
    try:
        return float(fields["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def profiled_traffic_batch(dtype, sky_scale):
    """DRAM bytes (read + write) per full-density launch of the persistent batch kernel from
    the committed ncu capture, or None for another storage type or density, or when the
    kernel source or the sky order's source changed since it was taken."""
    import hashlib

    path = os.path.join(ROOT, "profiles", f"k_eval_batched_{dtype}_full_dram.md")
    if sky_scale != 1.0 or not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith((" ", "#", "`")):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    csrc = os.path.join(ROOT, "paper_2411_18370_b300", "csrc")
    for key, name in (("kernel source sha256 prefix", "ft_eval.cu"), ("sky order source sha256 prefix", "ft_api.cu")):
        sha = hashlib.sha256(open(os.path.join(csrc, name), "rb").read()).hexdigest()[:16]
        if fields.get(key) != sha:
            return None
    try:
        return float(fields["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def rel_error(s_gpu, s_or):
    r = np.abs(np.asarray(s_gpu, np.float64) - s_or) / np.abs(s_or)
    return {"max": float(r.max()), "rms": float(math.sqrt(np.mean(r * r))), "n": int(len(r))}


def run_reference(args):
    """Reference arm: the CPU FP64 oracle on the host cores, bounded sample per step."""
    import ftsynth
    import oracle

    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    sfts, bank = ftsynth.search_workload(n_sky=args.n_sky)
    g = np.random.default_rng(11)
    per_step = 128
    t0 = time.perf_counter()
    oracle.statistic(sfts, bank, g.choice(bank.n_templates, per_step, replace=False))
    dt = time.perf_counter() - t0
    per_step = int(max(64, per_step * args.ref_step_s / max(dt, 1e-3)))
    for _ in range(args.warmup):
        oracle.statistic(sfts, bank, g.choice(bank.n_templates, per_step, replace=False))
    times = []
    for _ in range(args.steps):
        samp = g.choice(bank.n_templates, per_step, replace=False)
        t0 = time.perf_counter()
        oracle.statistic(sfts, bank, samp)
        times.append(time.perf_counter() - t0)
    evals = per_step * sfts.n_total
    value = evals * len(times) / sum(times)
    cfg = workload_desc(sfts, bank, "f64")
    cfg["storage"] = "f64 (oracle)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{per_step} random templates x {sfts.n_total} SFTs per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_measure(args, ctx, local, sky_scale, steps, warmup, loop_steps, cpu_seconds=None):
    """The batching workload: 64 bands (0.05-0.5 Hz wide, 50-500 Hz, N_sky ~ f^2, 10 f1) on
    the same 1-yr 2-detector timeline, searched by one persistent graph-captured launch,
    against a per-band loop of the single-band path.  Power is chi^2_2 drawn on the device
    with a seeded generator (the band matrices total several GB).  Returns a dict."""
    import torch

    import ftsynth
    import paper_2411_18370_b300 as ft

    T = ftsynth.T_SFT
    n_slots = int(round(ftsynth.YEAR_S / T))
    starts = ftsynth.timeline(2, n_slots, T, 0.7, ftsynth.rng(3, 1))
    t_mid = np.concatenate([st + 0.5 * T for st in starts])
    v = np.concatenate([ftsynth.detector_velocity(st + 0.5 * T, X) for X, st in enumerate(starts)])
    n_sft = [len(st) for st in starts]
    N = len(t_mid)
    specs = ftsynth.batch_bands(64, sky_scale)

    def band_power(b):
        """(power [N, W] on the device, first bin) of band b: chi^2_2 with a seeded generator."""
        sp = specs[b]
        wl, wh = ftsynth.wings_for(sp["f_hi"], -1e-9, n_slots * T, T)
        g = torch.Generator(device="cuda")
        g.manual_seed(ftsynth.derive_seed(3, 1000 + b) & ((1 << 63) - 1))
        P = torch.empty((N, sp["n_bins"] + wl + wh), dtype=torch.float32,
                        device="cuda").exponential_(0.5, generator=g)
        return P, sp["k_band"] - wl

    t_setup = time.perf_counter()
    bands, banks, evals = [], [], 0
    for b, sp in enumerate(specs):
        P, k_lo = band_power(b)
        band = ft.load_sfts(ctx, P, t_mid, v, n_sft, k_lo, T, 0.0, dtype=args.dtype)
        del P
        sky = ftsynth.fibonacci_sky(sp["n_sky"])
        bank = ft.make_bank(ctx, band, sp["k_band"], sp["n_bins"], ftsynth.f1_grid(10, -1e-9, 0.0),
                            sky, 18)
        assert bank.window_safe
        bands.append(band)
        banks.append(bank)
        evals += bank.n_templates * N
    stream = torch.cuda.current_stream()
    k = args.k
    roof_e, _ = ft.gather_roof(ctx, args.dtype)
    cands = [torch.empty(b.n_subbands * k * 16, dtype=torch.uint8, device="cuda") for b in banks]

    def loop_step():
        for band, bank, c in zip(bands, banks, cands):
            ft.topk_per_band(ctx, band, bank, k, c, stream=stream)

    flushbuf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush = lambda: flushbuf.fill_(1)
    t0 = time.perf_counter()
    batch = ft.Batch(ctx, bands, banks, k)
    create_s = time.perf_counter() - t0
    n_sub = sum(b.n_subbands for b in banks)
    out = torch.empty(n_sub * k * 16, dtype=torch.uint8, device="cuda")
    batch_step = lambda: batch.run(out, stream=stream)
    setup_s = time.perf_counter() - t_setup
    with ClockSampler(local) as clk:
        t_batch = time_steps(batch_step, steps, warmup, stream, flush)
    t_loop = time_steps(loop_step, loop_steps, 1, stream, flush)
    ctx.check_status()
    # the two paths must select the same candidates (identical per-tile code, same sums up
    # to accumulation order); report how many sub-bands differ
    got = ft.decode_candidates(out, n_sub, k)[0]
    ref = np.concatenate([ft.decode_candidates(c, b.n_subbands, k)[0] for c, b in zip(cands, banks)])
    differ = int(np.sum(np.any(np.sort(got, 1) != np.sort(ref, 1), axis=1)))
    mb, ml = statistics.mean(t_batch), statistics.mean(t_loop)
    esize = ESIZE[args.dtype]
    achieved_gbs = evals * esize / (mb / 1e3) / 1e9
    peak_max_clk = 148 * SMEM_BYTES_PER_CLK_PER_SM * 2032e6 / 1e9
    res = {
        "value": evals / (mb / 1e3), "unit": UNIT, "ms_per_step": mb, "steps": steps, "warmup": warmup,
        "workload": f"64-band batch: widths 0.05-0.5 Hz, starts 50-500 Hz, N_sky = {sky_scale} x 1e3 "
                    f"(f/50)^2 clamped to [1e3, 1e5], 10 f1, 2 det x 1 yr ({N} SFTs)",
        "storage": args.dtype, "bands": len(bands),
        "templates": int(sum(b.n_templates for b in banks)), "evals_per_step": evals,
        "launch": {"tile_f0": batch.tile_f0, "stages": batch.stages, "rows_per_stage": batch.rows_per_stage,
                   "resident_ctas": batch.n_ctas, "create_s": create_s, "setup_s": setup_s,
                   "gpu_launches_per_step": 2, "kind": "one persistent launch + merge, CUDA graph"},
        "per_band_loop": {"value": evals / (ml / 1e3), "ms_per_step": ml, "steps": loop_steps,
                          "gpu_launches_per_step": 2 * len(bands)},
        "speedup_vs_loop": ml / mb, "subbands_with_different_sets": differ,
        "measured_gather_roof": {"evals_per_s": roof_e, "frac": (evals / (mb / 1e3)) / roof_e,
                                 "entry": "ft_gather_roof", "storage": args.dtype},
        # the timed step is the persistent evaluation plus its merge (under 0.1 % of the step)
        "roofline": {"bound": "smem", "kernel": "k_eval_batched (all bands, fused top-k epilogue)",
                     "achieved": achieved_gbs, "peak": peak_max_clk, "unit": "GB/s",
                     "frac": achieved_gbs / peak_max_clk,
                     "peak_basis": "derived: 148 SMs x 128 B/clk shared-memory load bandwidth x "
                                   "2032 MHz max SM clock",
                     "algorithmic_bytes_per_launch": evals * esize, "bytes_per_eval": esize,
                     # DRAM bytes: the stored rows are 3.2 GB; L2 serves the tiles' re-reads
                     "traffic": profiled_traffic_batch(args.dtype, sky_scale)},
        "l2": "flushed between timed steps",
        "clocks": clk.summary(),
    }
    if cpu_seconds:
        # the oracle on a template sample of the middle band (its power copied to the host)
        b = len(specs) // 2
        sp = specs[b]
        P, k_lo = band_power(b)
        sfts_b = ftsynth.SFTSet(power=P.double().cpu().numpy(), t_mid=t_mid, v=v, s_n=np.ones(N),
                                n_sft=n_sft, k_lo=k_lo, t_sft=T, t0=0.0)
        del P
        bank_b = ftsynth.Bank(k0=sp["k_band"], n_f0=sp["n_bins"], f1=ftsynth.f1_grid(10, -1e-9, 0.0),
                              sky=ftsynth.fibonacci_sky(sp["n_sky"]), subband_bins=18)
        cb, _, _ = cpu_baseline(sfts_b, bank_b, cpu_seconds)
        cb.pop("seconds")
        cb["sample"] = (f"band {b} of the batch ({sp['n_bins']} f0 bins x 10 f1 x {sp['n_sky']} sky "
                        f"points): " + cb["sample"])
        res["cpu_baseline"] = cb
    batch.close()
    for bk in banks:
        bk.close()
    for bd in bands:
        bd.close()
    del flushbuf, out, cands
    torch.cuda.empty_cache()
    return res


def run_batch(args):
    """--workload batch: the batching workload's own JSON line."""
    import torch

    import paper_2411_18370_b300 as ft

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    ctx = ft.create(local)
    r = batch_measure(args, ctx, local, args.sky_scale, max(2, args.steps), args.warmup,
                      max(1, args.steps // 2), None if args.no_cpu_baseline else args.cpu_seconds)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["steps"],
        "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{args.dtype}-storage/f32-accumulate",
        "data": "synthetic",
        "config": {"workload": r["workload"], "storage": r["storage"], "bands": r["bands"],
                   "templates": r["templates"], "evals_per_step": r["evals_per_step"], "l2": r["l2"]},
        "batch": r["launch"], "per_band_loop": r["per_band_loop"], "speedup_vs_loop": r["speedup_vs_loop"],
        "subbands_with_different_sets": r["subbands_with_different_sets"],
        "measured_gather_roof": r["measured_gather_roof"], "roofline": r["roofline"],
        "gpu_launches": 2 * r["steps"], "clocks": r["clocks"],
    }
    if "cpu_baseline" in r:
        line["cpu_baseline"] = r["cpu_baseline"]
    print(json.dumps(line), flush=True)
    return 0


# per (template, SFT) operations of the binary track's FP32 screen and gather: orbit phase
# (three 32-bit multiply-adds: 3), the cosine (convert the phase, scale it to radians, the
# special-function unit's cosine: 3), a.v + y0 (3), y (1), floor, fraction and the two
# boundary tests (4), the bin (2), bounds + out-of-window count (2), address, read, add (3);
# the FP64 decisions (about 2 delta of the evaluations) are not counted
BT_OPS_PER_EVAL = 21
ISSUE_LANES_PER_CLK_PER_SM = 128


def profiled_traffic_binary(dtype):
    """DRAM bytes per launch of k_bt_eval from the committed capture, or None when there is
    none or ft_binary.cu changed since."""
    import hashlib

    path = os.path.join(ROOT, "profiles", f"k_bt_eval_binary_{dtype}_full.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith((" ", "#", "`")):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2411_18370_b300", "csrc", "ft_binary.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if fields.get("kernel source sha256 prefix") != sha:
        return None
    try:
        return float(fields["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def binary_core(args, ctx, local, steps=None):
    """The timed part of the binary-orbit workload (see run_binary): its JSON object and the
    inputs it made."""
    import torch

    import ftsynth
    import paper_2411_18370_b300 as ft

    steps = args.steps if steps is None else steps
    sfts, bank = ftsynth.binary_workload()
    stream = torch.cuda.current_stream()
    P32 = torch.from_numpy(sfts.power.astype(np.float32))
    band = ft.load_sfts(ctx, P32.cuda(), sfts.t_mid, sfts.v, sfts.n_sft, sfts.k_lo, sfts.t_sft,
                        sfts.t0, dtype=args.dtype, s_n=sfts.s_n)
    gb = ft.make_binary_bank(ctx, band, bank.lo, bank.hi, bank.n_div, bank.n_per_box, bank.seed)
    k = 1
    cand = torch.empty(gb.n_boxes * k * 16, dtype=torch.uint8, device="cuda")
    step = lambda: ft.binary_topk_per_box(ctx, band, gb, k, cand, stream=stream)
    flushbuf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush = lambda: flushbuf.fill_(1)
    evals = bank.n_templates * sfts.n_total
    ft.binary_decisions(gb)
    with ClockSampler(local) as clk:
        times = time_steps(step, steps, args.warmup, stream, flush)
    ctx.check_status()
    n64, delta = ft.binary_decisions(gb)
    mean_ms = statistics.mean(times)
    value = evals / (mean_ms / 1e3)
    peak_ops = 148 * ISSUE_LANES_PER_CLK_PER_SM * 2032e6
    achieved = BT_OPS_PER_EVAL * value
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{args.dtype}-storage/f32-accumulate", "data": "synthetic",
        "config": {"workload": f"binary-orbit track, random hyperbox bank: f0 100-100.125 Hz, all sky, "
                               f"a_p 5-15 lt-s, P 7-15 d, phi_b full orbit; {bank.n_templates} templates "
                               f"in {bank.n_boxes} boxes; 2 det x 183 d of 1024 s SFTs at 70% duty "
                               f"({sfts.n_total} SFTs, {sfts.power.shape[1]}-bin window); loudest per box",
                   "n_sft": sfts.n_total, "n_templates": bank.n_templates, "n_boxes": bank.n_boxes,
                   "evals_per_step": evals, "storage": args.dtype,
                   "track_bins": "FP64 bins of Eq. (track): FP32 screen (integer orbit phase, "
                                 "special-function-unit cosine) with a derived error bound delta, FP64 "
                                 "decision within delta of a rounding boundary",
                   "l2": "flushed between timed steps (256 MB write, outside the per-step events)"},
        "roofline": {"bound": "alu", "kernel": "k_bt_eval (per-template track, gather, per-box top-k)",
                     "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Top/s",
                     "frac": achieved / peak_ops,
                     "peak_basis": "derived: 148 SMs x 4 schedulers x 32 lanes x 2032 MHz max SM clock "
                                   "(one operation per lane per clock)",
                     "ops_per_eval": BT_OPS_PER_EVAL, "algorithmic_ops_per_launch": BT_OPS_PER_EVAL * evals,
                     "traffic": profiled_traffic_binary(args.dtype)},
        "gpu_launches": 2 * steps,
        "clocks": clk.summary(),
        "fp64_decisions": {"per_eval": n64 / (evals * (steps + args.warmup)), "delta_bins": delta,
                           "expected_per_eval": 2 * delta},
    }
    # the screen's cosine step over all 2^32 orbit phases against the bound delta assumes
    cos_err, cos_bound = ft.binary_cos_screen_check(ctx)
    out["cos_screen"] = {"max_abs_err": cos_err, "bound": cos_bound, "phases": 1 << 32}
    return out, sfts, bank, band, gb, P32, k


def run_binary(args):
    """The binary-orbit workload: a random hyperbox bank (2^20 templates in 32 boxes) for
    0.125 Hz at 100 Hz, all sky, a_p 5-15 lt-s, P 7-15 d, over 2 detectors x 183 days of 1024 s
    SFTs; one step = the loudest template of every box (evaluation + merge)."""
    import torch

    import ftsynth
    import oracle
    import paper_2411_18370_b300 as ft

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    ctx = ft.create(local)
    out, sfts, bank, band, gb, P32, k = binary_core(args, ctx, local)
    if not args.no_cpu_baseline:
        g = np.random.default_rng(7)
        n = 256
        for _ in range(3):
            samp = g.choice(bank.n_templates, n, replace=False).astype(np.int64)
            t0 = time.perf_counter()
            s_or, _ = oracle.binary_statistic(sfts, bank, samp)
            dt = time.perf_counter() - t0
            if dt >= 0.66 * args.cpu_seconds:
                break
            n = min(bank.n_templates, int(n * args.cpu_seconds / max(dt, 1e-3)))
        ev = len(samp) * sfts.n_total
        out["cpu_baseline"] = {"value": ev / dt, "unit": UNIT, "cores": oracle.num_threads(),
                               "kind": "oracle",
                               "sample": f"{len(samp)} random templates of the same bank x all "
                                         f"{sfts.n_total} SFTs ({ev:.3g} evals, {dt:.1f} s, FP64 sums, "
                                         f"OpenMP over templates)"}
    if not args.no_e2e:
        Ph = P32.pin_memory()
        cand_h = np.zeros((bank.n_boxes, k), dtype=ft.CANDIDATE_DTYPE)
        evals = bank.n_templates * sfts.n_total
        flushbuf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        flush = lambda: flushbuf.fill_(1)

        def e2e_step():
            b2 = ft.load_sfts(ctx, Ph, sfts.t_mid, sfts.v, sfts.n_sft, sfts.k_lo, sfts.t_sft, sfts.t0,
                              dtype=args.dtype, s_n=sfts.s_n)
            g2 = ft.make_binary_bank(ctx, b2, bank.lo, bank.hi, bank.n_div, bank.n_per_box, bank.seed)
            ft.binary_topk_per_box(ctx, b2, g2, k, cand_h)
            g2.close()
            b2.close()

        for _ in range(2):
            e2e_step()
        wall = []
        for _ in range(max(3, args.steps // 4)):
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            wall.append(time.perf_counter() - t0)
        e2e_mean = statistics.mean(wall)
        h2d = P32.numel() * 4 + sfts.t_mid.nbytes + sfts.v.nbytes + sfts.s_n.nbytes + 8 * len(sfts.n_sft)
        out["e2e"] = {"value": evals / e2e_mean, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(cand_h.nbytes + 4), "ms_per_step": 1e3 * e2e_mean,
                      "steps": len(wall), "gpu_launches_per_step": 4}
    print(json.dumps(out), flush=True)
    return 0


def run_surrogate(args):
    """The learned-surrogate workload: injection campaigns across the batching workload's
    bands (per-band duty and PSD), a noise-only threshold per band, an ensemble of 4-layer
    MLPs trained on the pooled outcomes by the library's kernels, and h0 at 90% p_det on
    held-out bands from (a) the surrogate, (b) per-band sigmoid fits with the same per-band
    budget, (c) a high-statistics campaign (the reference)."""
    import torch

    import paper_2411_18370_b300 as ft
    from paper_2411_18370_b300 import study

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    ctx = ft.create(local)
    t0 = time.perf_counter()
    res = study.run_study(ctx, n_bands=args.n_bands, sky_scale=args.sky_scale, n_held=args.n_held,
                          n_noise=args.n_noise, n_train=args.n_train, n_ref=args.n_ref,
                          members=args.members, epochs=args.epochs, k_sky=args.k_sky)
    line = {"workload": "learned p_det surrogate across the batching workload's bands",
            "wall_s": time.perf_counter() - t0}
    line.update(res)
    line["inference"] = inference_rates(ctx, local)
    print(json.dumps(line), flush=True)
    return 0


def run_inference(args):
    """The surrogate's BF16 inference alone (the study's network shape, 4.2e6 samples, device
    input and output), against the measured dense BF16 tensor peak."""
    import torch

    import paper_2411_18370_b300 as ft

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    ctx = ft.create(local)
    r = inference_rates(ctx, local)
    peak = measured_bf16_peak()
    tc = r["tensor_cores"]
    line = {"metric": "p_det surrogate BF16 inference samples/s (width 128, 13 features)",
            "value": tc["samples_per_s"], "unit": "samples/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16-operands/f32-accumulate", "data": "synthetic",
            "config": {"workload": "4-layer MLP, widths 13-128-128-128-1, 4.2e6 samples per call"},
            "gpu_launches_per_call": 1,
            "roofline": {"bound": "tensor", "kernel": "k_infer_tc", "achieved": tc["tflops"],
                         "peak": peak, "unit": "TFLOP/s", "frac": tc["tflops"] / peak if peak else None,
                         "peak_basis": "measured dense BF16 burst (MEASURED_PEAKS.json bf16_tflops)",
                         "flops_per_sample": 2 * (13 * 128 + 2 * 128 * 128 + 128)},
            "inference": r}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def measured_bf16_peak():
    """Dense BF16 TFLOP/s (burst) from MEASURED_PEAKS.json, or the recipe's fallback 1800."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1800.0


def weighted_searches(args, ctx, sfts, bank, P32d, cand, stream, flush, barrier, max_over_ranks, ws, evals):
    """The search of the same bank and storage type with the all-sky weights (a^2 + b^2)/S_n
    of each template's own sky point (Sec. II.B), over the number-count band 1[P > 3.2]
    (Eq. (number_count)), and the loudest s among templates whose weighted count passes the
    noise mean + 3 sigma gate (Sec. VI.B), each timed like the main step."""
    import torch

    import ftsynth
    import paper_2411_18370_b300 as ft

    parts, off = [], 0
    for X, n in enumerate(sfts.n_sft):
        parts.append(ftsynth.detector_tensor(sfts.t_mid[off:off + n], X))
        off += n
    D = np.concatenate(parts)
    steps = max(5, args.steps // 4)

    def timed(step):
        barrier()
        times = time_steps(step, steps, args.warmup, stream, flush)
        barrier()
        ctx.check_status()
        m = max_over_ranks(statistics.mean(times))
        return {"value": ws * evals / (m / 1e3), "unit": UNIT, "ms_per_step": m, "steps": steps}

    def load():
        return ft.load_sfts(ctx, P32d, sfts.t_mid, sfts.v, sfts.n_sft, sfts.k_lo, sfts.t_sft, sfts.t0,
                            dtype=args.dtype, s_n=sfts.s_n)

    out = {}
    # all-sky weights: the producer warp forms a^2 + b^2 per (SFT, sky point) in FP64
    band = load()
    ft.band_set_sky_weights(band, D)
    bk = ft.make_bank(ctx, band, bank.k0, bank.n_f0, bank.f1, bank.sky, bank.subband_bins)
    out["all_sky_weights"] = timed(lambda: ft.topk_per_band(ctx, band, bk, args.k, cand, stream=stream))
    out["all_sky_weights"]["gpu_launches_per_step"] = 2
    # the number count over the same weights, and the count-gated loudest s
    ncb = ft.number_count_band(ctx, band, 3.2)
    nbk = ft.make_bank(ctx, ncb, bank.k0, bank.n_f0, bank.f1, bank.sky, bank.subband_bins)
    out["number_count"] = timed(lambda: ft.topk_per_band(ctx, ncb, nbk, args.k, cand, stream=stream))
    out["number_count"]["gpu_launches_per_step"] = 2
    # the gate is the count's critical ratio (its noise moments depend on the sky point
    # under all-sky weights): templates whose count lies 3 sigma above its noise mean
    count = torch.empty(bank.n_templates, dtype=torch.float32, device="cuda")
    zc = torch.empty(bank.n_templates, dtype=torch.float32, device="cuda")
    ft.eval_statistic(ctx, ncb, nbk, count, zc, stream=stream)
    torch.cuda.synchronize()
    out["count_gated"] = timed(lambda: ft.topk_per_band_gated(ctx, band, bk, args.k, zc, 3.0, cand,
                                                              stream=stream))
    out["count_gated"]["gpu_launches_per_step"] = 2
    out["count_gated"]["gate"] = {"threshold": 3.2, "count_z_min": 3.0,
                                  "templates_passing": int((zc >= 3.0).sum().item())}
    del count, zc
    for b_ in (nbk, ncb, bk, band):
        b_.close()
    return out


def inference_rates(ctx, local, n=1 << 22, d=13, w=128):
    """Samples/s of the surrogate's BF16 inference (the study's network shape: 13 features,
    width 128) on the tensor cores and on the CUDA cores, device input and output; FLOP
    counts 2 (d w + 2 w^2 + w) per sample."""
    import torch

    import paper_2411_18370_b300 as ft

    net = ft.MLP(ctx, d, w, seed=1)
    X = torch.randn(n, d, device="cuda")
    out = {}
    for name, tcores in (("tensor_cores", True), ("cuda_cores", False)):
        for _ in range(3):
            net.predict(X, bf16=True, tensor_cores=tcores)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(5):
            net.predict(X, bf16=True, tensor_cores=tcores)
        ev[1].record()
        torch.cuda.synchronize()
        dt = ev[0].elapsed_time(ev[1]) / 5 / 1e3
        out[name] = {"samples_per_s": n / dt, "ms": 1e3 * dt,
                     "tflops": 2.0 * (d * w + 2 * w * w + w) * n / dt / 1e12}
    out["samples"] = n
    out["speedup"] = out["cuda_cores"]["ms"] / out["tensor_cores"]["ms"]
    net.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f16", choices=["f16", "bf16", "f32"])
    ap.add_argument("--n-sky", type=int, default=10_000)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-weighted", action="store_true")
    ap.add_argument("--no-binary", action="store_true")
    ap.add_argument("--no-inference", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--sub-sky-stride", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=4.0)
    ap.add_argument("--workload", default="search", choices=["search", "batch", "surrogate", "binary", "inference"])
    ap.add_argument("--sky-scale", type=float, default=0.1)
    ap.add_argument("--n-bands", type=int, default=64)
    ap.add_argument("--n-held", type=int, default=4)
    ap.add_argument("--n-noise", type=int, default=2000)
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--members", type=int, default=5)
    ap.add_argument("--n-ref", type=int, default=8000)
    ap.add_argument("--k-sky", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=200)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "binary":
        return run_binary(args)
    if args.workload == "inference":
        return run_inference(args)

    import torch

    import ftsynth
    import paper_2411_18370_b300 as ft

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if pg is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())

    sfts, bank = ftsynth.search_workload(n_sky=args.n_sky)
    ctx = ft.create(local)
    stream = torch.cuda.current_stream()
    P32 = torch.from_numpy(sfts.power.astype(np.float32))
    P32d = P32.cuda()
    flushbuf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def flush():
        flushbuf.fill_(1)

    def mk(dtype, bk_desc=bank):
        band = ft.load_sfts(ctx, P32d, sfts.t_mid, sfts.v, sfts.n_sft, sfts.k_lo, sfts.t_sft,
                            sfts.t0, dtype=dtype, s_n=sfts.s_n)
        bk = ft.make_bank(ctx, band, bk_desc.k0, bk_desc.n_f0, bk_desc.f1, bk_desc.sky, bk_desc.subband_bins)
        return band, bk

    cand = torch.empty(bank.n_subbands * args.k * 16, dtype=torch.uint8, device="cuda")
    evals = bank.n_templates * sfts.n_total
    runs = {}
    # the chosen storage type, then the others of the precision comparison (plain FP32 and
    # BF16), each timed over the full bank
    for dtype in dict.fromkeys([args.dtype, "f32", "bf16", "f16"]):
        band, bk = mk(dtype)
        assert bk.window_safe
        step = lambda: ft.topk_per_band(ctx, band, bk, args.k, cand, stream=stream)
        barrier()
        with ClockSampler(local) as clk:
            times = time_steps(step, args.steps if dtype == args.dtype else max(5, args.steps // 2),
                               args.warmup, stream, flush)
        barrier()
        ctx.check_status()
        mean_ms = statistics.mean(times)
        runs[dtype] = {"band": band, "bank": bk, "times": times, "mean_ms": mean_ms,
                       "mean_ms_max": max_over_ranks(mean_ms), "clocks": clk.summary()}

    # the weighted searches on the same bank and storage type (Sec. II.B, VI.B): all-sky
    # weights, the number count, and the loudest among templates whose count passes the gate
    weighted = {} if args.no_weighted else weighted_searches(args, ctx, sfts, bank, P32d, cand, stream,
                                                               flush, barrier, max_over_ranks, ws, evals)

    chosen = runs[args.dtype]
    value = ws * evals / (chosen["mean_ms_max"] / 1e3)
    clocks = chosen["clocks"] or {}
    sm_mhz = clocks.get("sm_mhz")
    esize = ESIZE[args.dtype]
    achieved_gbs = evals * esize / (chosen["mean_ms"] / 1e3) / 1e9
    peak_max_clk = 148 * SMEM_BYTES_PER_CLK_PER_SM * 2032e6 / 1e9
    roofline = {
        "bound": "smem",
        "kernel": "k_eval (gather-accumulate, fused top-k epilogue)",
        "achieved": achieved_gbs,
        "peak": peak_max_clk,
        "unit": "GB/s",
        "frac": achieved_gbs / peak_max_clk,
        "peak_basis": "derived: 148 SMs x 128 B/clk shared-memory load bandwidth x 2032 MHz max "
                      "SM clock (no measured shared-memory peak exists in MEASURED_PEAKS.json)",
        "algorithmic_bytes_per_launch": evals * esize,
        "bytes_per_eval": esize,
        "frac_at_sampled_clock": (achieved_gbs / (148 * SMEM_BYTES_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e9)
                                  if sm_mhz else None),
        "traffic": profiled_traffic(args.dtype),
    }

    roof_e, roof_c = ft.gather_roof(ctx, args.dtype)
    roof32_e, _ = ft.gather_roof(ctx, "f32")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": chosen["mean_ms_max"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{args.dtype}-storage/f32-accumulate",
        "data": "synthetic",
        "config": workload_desc(sfts, bank, args.dtype),
        "roofline": roofline,
        "gpu_launches": 2 * args.steps,
        "clocks": chosen["clocks"],
        "plain_fp32": {"value": ws * evals / (runs["f32"]["mean_ms_max"] / 1e3),
                       "ms_per_step": runs["f32"]["mean_ms_max"], "clocks": runs["f32"]["clocks"],
                       "frac_of_measured_gather_roof": (evals / (runs["f32"]["mean_ms_max"] / 1e3)) / roof32_e},
        "precision": {d: {"value": ws * evals / (r["mean_ms_max"] / 1e3), "ms_per_step": r["mean_ms_max"],
                          "steps": len(r["times"])} for d, r in runs.items()},
        # the bare inner loop (rows resident in shared memory, no tables or pipeline), run in
        # the same process: the ceiling this kernel's design can reach on this GPU
        "measured_gather_roof": {"evals_per_s": roof_e, "evals_per_clk_per_sm": roof_c,
                                 "frac": (evals / (chosen["mean_ms"] / 1e3)) / roof_e,
                                 "entry": "ft_gather_roof", "storage": args.dtype},
    }
    if weighted:
        out["weighted_searches"] = weighted
        out["gpu_launches"] += sum(w["gpu_launches_per_step"] * w["steps"] for w in weighted.values()
                                   if isinstance(w, dict) and "steps" in w)

    if rank == 0 and not args.no_cpu_baseline:
        # The oracle on every template of a sub-bank of the same bank (every f0 and f1, one
        # sky point in 100): its CPU rate, and for each storage type the GPU's relative error
        # and per-sub-band top-k sets on that sub-bank against the oracle's.
        import oracle

        sub = ftsynth.Bank(k0=bank.k0, n_f0=bank.n_f0, f1=bank.f1, sky=bank.sky[::args.sub_sky_stride],
                           subband_bins=bank.subband_bins)
        t0 = time.perf_counter()
        s_or, _ = oracle.statistic(sfts, sub)
        dt = time.perf_counter() - t0
        ev = sub.n_templates * sfts.n_total
        out["cpu_baseline"] = {"value": ev / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": f"every template of a sub-bank of the same bank ({bank.n_f0} f0 x "
                                         f"{bank.n_f1} f1 x {sub.n_sky} sky points, one in "
                                         f"{args.sub_sky_stride}) x all {sfts.n_total} SFTs ({ev:.3g} evals, "
                                         f"{dt:.1f} s, FP64, OpenMP over templates)"}
        k = args.k
        o_idx, o_val = oracle.topk_per_subband(s_or, sub, k + 1)
        n = sfts.n_total
        # near-tie margins: the oracle's k-th and (k+1)-th values closer than twice the storage
        # type's 6-sigma error of s (one rounding per stored value, unit roundoff u, independent:
        # sigma(s)/s = u sqrt(2 / (3 N)) for exponential power); FP32: 2e-6
        u = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
        agree, errs = {}, {}
        for dtype in runs:
            band_s, bk_s = mk(dtype, sub)
            s_g = np.empty(sub.n_templates, np.float32)
            ft.eval_statistic(ctx, band_s, bk_s, s_g)
            errs[dtype] = rel_error(s_g, s_or)
            c = np.zeros((sub.n_subbands, k), dtype=ft.CANDIDATE_DTYPE)
            ft.topk_per_band(ctx, band_s, bk_s, k, c)
            margin = 2 * 6 * u[dtype] * math.sqrt(2.0 / (3.0 * n)) if dtype in u else 2e-6
            equal, ties, differ = 0, [], 0
            for b in range(sub.n_subbands):
                got = set(int(x) for x in c["template_idx"][b] if x >= 0)
                want = set(int(x) for x in o_idx[b, :k] if x >= 0)
                if got == want:
                    equal += 1
                    continue
                gap = abs(o_val[b, k - 1] - o_val[b, k]) / abs(o_val[b, k - 1])
                if gap < margin:
                    ties.append({"subband": b, "rel_gap_kth_next": float(gap)})
                else:
                    differ += 1
            agree[dtype] = {"subbands": sub.n_subbands, "equal_sets": equal, "near_ties": ties,
                            "differ_beyond_margin": differ, "near_tie_margin_rel": margin}
            bk_s.close()
            band_s.close()
        out["rel_error_vs_oracle"] = errs
        out["candidate_sets_vs_oracle"] = {"sample": f"the {sub.n_templates}-template sub-bank above, "
                                                     f"top-{k} per 0.01 Hz sub-band", **agree}

    if not args.no_e2e:
        # end to end through the C ABI with host buffers: H2D of the SFT power and metadata,
        # bank upload, search, D2H of the candidates; wall clock per step
        Ph = P32.pin_memory()
        cand_h = np.zeros((bank.n_subbands, args.k), dtype=ft.CANDIDATE_DTYPE)

        def e2e_step():
            band = ft.load_sfts(ctx, Ph, sfts.t_mid, sfts.v, sfts.n_sft, sfts.k_lo, sfts.t_sft,
                                sfts.t0, dtype=args.dtype, s_n=sfts.s_n)
            bk = ft.make_bank(ctx, band, bank.k0, bank.n_f0, bank.f1, bank.sky, bank.subband_bins)
            ft.topk_per_band(ctx, band, bk, args.k, cand_h)
            bk.close()
            band.close()

        e2e_steps = args.steps
        for _ in range(args.warmup):
            e2e_step()
        barrier()
        wall = []
        for _ in range(e2e_steps):
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            wall.append(time.perf_counter() - t0)
        barrier()
        e2e_mean = max_over_ranks(statistics.mean(wall))
        h2d = (P32.numel() * 4 + sfts.t_mid.nbytes + sfts.v.nbytes + sfts.s_n.nbytes
               + bank.f1.nbytes + bank.sky.nbytes + 4 * len(sfts.n_sft))
        d2h = cand_h.nbytes + 4
        out["e2e"] = {"value": ws * evals / e2e_mean, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_mean,
                      "steps": e2e_steps, "gpu_launches_per_step": 4}

    for r in runs.values():
        r["bank"].close()
        r["band"].close()
    del P32d
    torch.cuda.empty_cache()
    if not args.no_batch:
        # the batching workload at its stated sky density, one persistent graph-captured
        # launch per step, against the per-band loop (each rank its own replica)
        b = batch_measure(args, ctx, local, 1.0, args.batch_steps, args.warmup, 1)
        b["ms_per_step"] = max_over_ranks(b["ms_per_step"])
        b["value"] = ws * b["evals_per_step"] / (b["ms_per_step"] / 1e3)
        out["batch"] = b
        out["gpu_launches"] += 2 * args.batch_steps

    if not args.no_binary:
        # the binary-orbit track's search (each rank its own replica), its own timed steps
        bt, *_ = binary_core(args, ctx, local, steps=max(5, args.steps // 2))
        out["binary_track"] = {k_: bt[k_] for k_ in ("value", "unit", "ms_per_step", "steps", "roofline",
                                                     "fp64_decisions", "cos_screen", "clocks", "gpu_launches")}
        out["binary_track"]["workload"] = bt["config"]["workload"]
        out["binary_track"]["value"] = ws * bt["value"]
        out["gpu_launches"] += bt["gpu_launches"]
    if not args.no_inference:
        # the surrogate's BF16 inference on the tensor cores (4.2e6 samples per call)
        inf = inference_rates(ctx, local)
        tc = inf["tensor_cores"]
        peak = measured_bf16_peak()
        out["surrogate_inference"] = {
            "value": ws * tc["samples_per_s"], "unit": "samples/s", "tflops": tc["tflops"],
            "roofline": {"bound": "tensor", "kernel": "k_infer_tc", "achieved": tc["tflops"], "peak": peak,
                         "unit": "TFLOP/s", "frac": tc["tflops"] / peak,
                         "peak_basis": "measured dense BF16 burst (MEASURED_PEAKS.json bf16_tflops)"},
            "cuda_cores_samples_per_s": inf["cuda_cores"]["samples_per_s"], "samples": inf["samples"]}

    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
