#!/usr/bin/env python
"""Benchmark: variable-pairs per second of the all-pairs tests with pairwise
deletion (NApy, arXiv 2505.00448) on one GB300, with the cohort resident in HBM.

Workload (default, "mixed-type cohort"): 4,000 continuous FP32 variables (2,000
Gaussian with offsets up to 1e4 sigma, 2,000 lognormal) and 1,000 categorical
ones (2-10 levels) over 50,000 samples, per-column missingness ~ Beta(2,5).
One step runs every test of the cohort's hot path once: all-pairs Pearson
(continuous), ANOVA F (categorical x continuous), Welch t (binary categorical x
continuous) and chi-squared (categorical). value = var-pairs of the step / step
time. The cohort (1 GB) is larger than L2, so no L2 flush is needed between steps.

--workload ranks runs the rank tests (Spearman, Mann-Whitney, Kruskal-Wallis) on
the 1,200-variable x 10,000-sample tied cohort instead (for profiling).

--workload serve runs the request loop on the resident 100,000-sample x 10,000-
variable cohort: Poisson arrivals at 0.25-1.5 x the measured single-request
capacity, each request a random test (Pearson, Spearman, chi-squared,
Kruskal-Wallis), mask (5-80% of samples) and variable subset (50-2,000);
p50/p99 latency and pairs/s per rate.

--workload batch runs 256 sample contexts of uneven size (500-20,000 samples) of
a 20,000-sample cohort (1,600 continuous FP32 + 400 categorical, 25% MCAR):
per context all-pairs Pearson and chi-squared, each test's 256 contexts as one
napg_run_batch call (one captured CUDA graph).

--workload small-pearson times single calls on the 200 x 1,000 plain-FP64
Pearson cohort (p50/p99 latency); --workload paper-sim runs all seven tests on
the paper's simulated data (uniform values, 4 levels, 10% missing; F, S in
250..1,000).

--impl reference times the FP64 CPU oracle (the reference of this method) on
bounded samples of the same workload.

Defaults: 100 timed steps after 10 warm-ups (the p99 over 100 steps).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--precision mixed|fp64]
                       [--workload mixed|ranks|batch|serve|small-pearson|paper-sim]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2505_00448_gb300 import dist as D  # noqa: E402
from paper_2505_00448_gb300 import synth  # noqa: E402

METRIC = "var-pairs/s per test, mixed-precision vs plain FP64 GPU at |dr|<=1e-6; p99 ms"
UNIT = "var-pairs/s"


# ------------------------------------------------------------------ workload --

def make_workload(name, scale=1.0):
    if name == "small-pearson":
        coh = synth.small_pearson_cohort()
        tests = [("pearson", coh["cont"], None)]
        desc = "200 continuous x 1,000 samples, FP64, 20% MCAR; all-pairs Pearson, plain FP64 form"
        return coh, tests, desc
    if name == "ranks":
        coh = synth.rank_cohort() if scale == 1.0 else synth.rank_cohort(n_cont=max(32, int(1000 * scale)),
                                                                   n_cat=max(8, int(200 * scale)))
        cat = coh["cat"]
        bins = cat[coh["nlev"][cat] == 2]
        multi = cat[coh["nlev"][cat] >= 3]
        tests = [("spearman", coh["cont"], None), ("mwu", bins, coh["cont"]), ("kruskal", multi, coh["cont"])]
        desc = ("rank cohort: 1,000 continuous (1-decimal ties, 30% MCAR + block losses) + 200 categorical "
                "(2-8 levels) x 10,000 samples, FP64; Spearman + Mann-Whitney + Kruskal-Wallis")
    else:
        coh = synth.mixed_cohort() if scale == 1.0 else synth.mixed_cohort(n_cont=max(64, int(4000 * scale)),
                                                                   n_cat=max(16, int(1000 * scale)))
        cat = coh["cat"]
        bins = cat[coh["nlev"][cat] == 2]
        tests = [("pearson", coh["cont"], None), ("anova", cat, coh["cont"]), ("ttest", bins, coh["cont"]),
                 ("chi2", cat, None)]
        desc = ("mixed-type cohort: 4,000 continuous FP32 (2,000 Gaussian offsets to 1e4 sigma, 2,000 "
                "lognormal) + 1,000 categorical (2-10 levels) x 50,000 samples, Beta(2,5) missingness; "
                "Pearson + ANOVA + Welch t + chi-squared")
    return coh, tests, desc


def pair_count(test, va, vb):
    if vb is None:
        n = len(va)
        return n * (n - 1) // 2
    return len(va) * len(vb)


# ------------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples during the timed region (every 200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle --

def oracle_sample(coh, tests, budget_s, seed=0, one_thread=True):
    """Time the oracle (as it stands, all host cores) on a bounded random sample
    of each test's pairs; returns per-test pairs/s and the combined rate."""
    from oracle import oracle as O
    O.build()
    rng = np.random.default_rng(seed)
    X = coh["X"].astype(np.float64)
    cores = O.max_threads()
    per_test = {}
    # calibrate: a small sample per test, then scale to the budget
    share = budget_s / len(tests)
    for test, va, vb in tests:
        k = 64
        while True:
            if vb is None:
                pa = rng.choice(va, size=k)
                pb = rng.choice(va, size=k)
            else:
                pa = rng.choice(va, size=k)
                pb = rng.choice(vb, size=k)
            t0 = time.perf_counter()
            O.run_pairs(test, X, coh["missing"], coh["vtype"], coh["nlev"], pa, pb, validate=False)
            dt = time.perf_counter() - t0
            if dt > share / 4 or k >= 1 << 20:
                break
            k = int(k * min(16.0, max(2.0, (share / 4) / max(dt, 1e-3))))
        per_test[test] = {"pairs": int(k), "seconds": dt, "pairs_per_s": k / dt}
        if not one_thread:
            continue
        # the same oracle on one thread, on a sample sized for about a tenth of the share
        k1 = max(8, int(k / dt / max(cores, 1) * share / 10))
        pa, pb = rng.choice(va, size=k1), rng.choice(va if vb is None else vb, size=k1)
        t0 = time.perf_counter()
        O.run_pairs(test, X, coh["missing"], coh["vtype"], coh["nlev"], pa, pb, validate=False, nthreads=1)
        per_test[test]["pairs_per_s_1thread"] = k1 / (time.perf_counter() - t0)
    total_pairs = sum(pair_count(t, va, vb) for t, va, vb in tests)
    total_time = sum(pair_count(t, va, vb) / per_test[t]["pairs_per_s"] for t, va, vb in tests)
    total_time1 = (sum(pair_count(t, va, vb) / per_test[t]["pairs_per_s_1thread"] for t, va, vb in tests)
                   if one_thread else None)
    return {"value": total_pairs / total_time, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "; ".join(f"{t}: {v['pairs']} random pairs in {v['seconds']:.2f}s" for t, v in per_test.items()),
            "sample_seconds": sum(v["seconds"] for v in per_test.values()),
            "sample_pairs": sum(v["pairs"] for v in per_test.values()),
            "per_test": {t: v["pairs_per_s"] for t, v in per_test.items()},
            "value_1thread": total_pairs / total_time1 if one_thread else None}


# ------------------------------------------------------------------ accuracy --

def sampled_accuracy(coh, tests, outs, k, seed=123):
    """Max error of the device outputs against the oracle on k random pairs per
    test: |dr| (Pearson/Spearman), effect-scale difference (F: sqrt(F/(F+n)),
    t: t/sqrt(t^2+n-2)), exactness (chi-squared, U, n), and the p-value's
    relative difference."""
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    X = coh["X"].astype(np.float64)
    res = {}
    for test, va, vb in tests:
        na = len(va)
        nb = na if vb is None else len(vb)
        ia = rng.integers(0, na, k)
        ib = rng.integers(0, nb, k)
        pa = np.asarray(va)[ia]
        pb = (np.asarray(va) if vb is None else np.asarray(vb))[ib]
        st, pv, nn = O.run_pairs(test, X, coh["missing"], coh["vtype"], coh["nlev"], pa, pb, validate=False)
        gs = outs[test]["stat"].cpu().numpy()[ia, ib]
        gp = outs[test]["p"].cpu().numpy()[ia, ib]
        gn = outs[test]["n"].cpu().numpy()[ia, ib]
        fin = np.isfinite(st) & np.isfinite(gs)
        with np.errstate(invalid="ignore", divide="ignore"):
            if test in ("pearson", "spearman"):
                d = np.abs(gs - st)
                kind = "max |d stat|"
            elif test == "anova":
                d = np.abs(np.sqrt(gs / (gs + nn)) - np.sqrt(st / (st + nn)))
                kind = "max |d sqrt(F/(F+n))|"
            elif test == "ttest":
                d = np.abs(gs / np.sqrt(gs * gs + nn - 2) - st / np.sqrt(st * st + nn - 2))
                kind = "max |d t/sqrt(t^2+n-2)|"
            else:
                d = np.abs(gs - st) / np.maximum(np.abs(st), 1e-300)
                kind = "max rel d stat"
            pok = np.isfinite(pv) & (pv > 1e-300)
            pr = np.abs(gp[pok] - pv[pok]) / pv[pok]
        res[test] = {"pairs": int(k), "stat_error": float(np.nanmax(d[fin])) if fin.any() else None, "stat_metric": kind,
                     "p_rel_error_max": float(pr.max()) if pr.size else None,
                     "p_rel_error_median": float(np.median(pr)) if pr.size else None,
                     "n_exact": bool(np.array_equal(gn, nn)),
                     "nan_pattern_equal": bool(np.array_equal(np.isnan(gs), np.isnan(st)))}
    return res


# ---------------------------------------------------------------- roofline --

# stages whose MMAs are all E4M3 (the exact 0/1 count contractions)
FP8_STAGES = ("contingency_tc",)


def stage_rooflines(stage_ms, steps, coh, tests, peaks):
    """Roofline entry per traced stage: algorithmic work of the stage per step
    (the per-unit figures of the hot-path table: 12 S flops per Pearson pair,
    6 S per group-sum pair (issued: the one-hot rows against the B planes), S increments per contingency pair, 16.25 S / 9.125 S
    bytes per rank pair, bytes streamed by the plane builder, FP64 operations per
    p-value) divided by the stage's device time, against the measured peak."""
    S = coh["X"].shape[1]
    S_pad = -(-S // 64) * 64
    nkb = S_pad // 64
    nkb8 = -(-S // 128)

    def count_flops(tiles_a, kb8):
        # the E4M3 counts kernel: 128-row A tiles against 256-row B tiles on the
        # triangle, four MMAs of 128 x 256 x 32 per 128-sample K-block
        tiles_b = -(-tiles_a // 2)
        return sum(tiles_b - i // 2 for i in range(tiles_a)) * kb8 * 4 * 2.0 * 128 * 256 * 32
    # measured denominators, else the fallback figures (one earlier GB300 measurement)
    tens_meas, hbm_meas = peaks.get("bf16_tflops_sustained"), peaks.get("hbm_gbs")
    tens_peak = tens_meas or 1700.0
    hbm_peak = hbm_meas or 6800.0
    esz = coh["X"].dtype.itemsize
    pairs_by = {t: pair_count(t, va, vb) for t, va, vb in tests}
    work = {}
    for test, va, vb in tests:
        na = len(va)
        if test == "pearson":
            T = -(-na // 128)
            # Sxy (triangle, three hi/lo products), the mask against the four value
            # planes (all ordered tile pairs), and n = M M^T on the triangle in E4M3
            # (counted at half its flops: the FP8 MMA runs at twice the f16 rate)
            issued = (T * (T + 1) / 2 * nkb * 12 * 2.0 * 128 * 128 * 16 + T * -(-na // 48) * nkb * 4 * 2.0 * 128 * 192 * 16
                      + count_flops(T, nkb8) / 2)
            work["pearson_moments_tc"] = ("tensor", 12.0 * S * na * (na + 1) / 2, issued)
            work.setdefault("planes_f16", ["hbm", 0.0, None])
            work["planes_f16"][1] += na * (esz * S + S / 8 + 10.0 * S_pad)
        if test in ("anova", "ttest") and vb is not None:
            R = int(coh["nlev"][va].sum())
            if test == "anova":
                # level rows x (count, two sum planes) + observed rows x two square planes
                issued = 2.0 * 128 * -(-R // 128) * 3 * len(vb) * S_pad + 2.0 * 128 * -(-na // 128) * 2 * len(vb) * S_pad
            else:
                # level rows x all five planes
                issued = 2.0 * 128 * -(-R // 128) * 5 * len(vb) * S_pad
            w = work.get("groupsum_tc", ("tensor", 0.0, 0.0))
            work["groupsum_tc"] = ("tensor", w[1] + 6.0 * S * na * len(vb), w[2] + issued)
        if test == "chi2":
            R = int(coh["nlev"][va].sum())
            work["contingency_tc"] = ("tensor", 1.0 * S * na * (na + 1) / 2, count_flops(-(-R // 128), nkb8))
        if test == "pearson":
            work["pearson_moments_fp64"] = ("fp64", 12.0 * S * na * (na + 1) / 2, None)
        if test in ("anova", "ttest") and vb is not None:
            w = work.get("groupsum_fp64", ("fp64", 0.0, None))
            work["groupsum_fp64"] = ("fp64", w[1] + 6.0 * S * na * len(vb), None)
        if test == "spearman":
            work["spearman_rank"] = ("hbm", 16.25 * S * na * (na + 1) / 2, None)
        if test in ("mwu", "kruskal"):
            w = work.get("rank_groups", ("hbm", 0.0, None))
            work["rank_groups"] = ("hbm", w[1] + 9.125 * S * na * len(vb), None)
    work["pvalues"] = ("alu", float(sum(pairs_by.values())), None)
    out = []
    for name, v in stage_ms.items():
        if name not in work:
            continue
        bound, alg, issued = work[name][0], work[name][1], work[name][2]
        secs = v["ms"] / steps / 1000.0
        if secs <= 0 or alg <= 0:
            continue
        e = {"kernel": name, "bound": bound, "ms_per_step": v["ms"] / steps,
             "launches_per_step": max(1, v["launches"] // max(1, steps))}
        if bound == "tensor":
            src = ("measured bf16 dense, sustained (MEASURED_PEAKS; f16 runs at the bf16 rate)"
                   if tens_meas else "fallback 1,700 TFLOP/s bf16 sustained (no measured peak)")
            peak = tens_peak
            if name in FP8_STAGES:
                # E4M3 MMAs (kind::f8f6f4): the bf16 figure times the nominal 2x FP8 ratio
                peak = 2.0 * tens_peak
                src += " x 2, the nominal FP8 (E4M3) to bf16 ratio"
            e.update(achieved=alg / secs / 1e12, peak=peak, unit="TFLOP/s", peak_source=src)
            if issued:
                e["issued_tflops"] = issued / secs / 1e12
                e["issued_frac"] = e["issued_tflops"] / peak
        elif bound == "hbm" and name in ("spearman_rank", "rank_groups"):
            # the rank kernels' byte model (16.25 S or 9.125 S bytes a pair) as an
            # effective rate against the HBM copy rate: their working set stays in
            # L2 and shared memory (DRAM carries under 0.5% of the model), so they
            # are bound by instruction issue, not by HBM
            e.update(bound="alu", achieved=alg / secs / 1e9, peak=hbm_peak, unit="GB/s of the byte model",
                     peak_source=(("measured HBM copy (MEASURED_PEAKS)" if hbm_meas else
                                   "fallback 6,800 GB/s (no measured peak)") +
                                  " as the byte model's reference rate; the kernel is bound by instruction issue "
                                  "(ncu: 65-80% of issue slots)"))
            tr = load_traffic(name)
            e["dram_share_of_model"] = tr / alg if tr else None      # both per step
        elif bound == "hbm":
            e.update(achieved=alg / secs / 1e9, peak=hbm_peak, unit="GB/s",
                     peak_source="measured HBM copy (MEASURED_PEAKS)" if hbm_meas else "fallback 6,800 GB/s (no measured peak)")
        elif bound == "fp64":
            # plain FP64 moments on the CUDA cores: 152 SMs x 2 FP64 FMA per clock x
            # 2.07 GHz = 1.26 TFLOP/s nominal (1.25 TFLOP/s stated for GB300)
            e.update(bound="alu", achieved=alg / secs / 1e9, peak=1250.0, unit="GFLOP/s",
                     peak_source="nominal FP64 rate (152 SMs x 4 flops/clock x 2.07 GHz)")
        else:
            # FP64-pipe bound: the pipe's share is what ncu reports for this kernel
            # (the p-value profile of the mixed cohort); the job count is not known here
            e.update(achieved=sum(pairs_by.values()) / secs / 1e6, peak=None, unit="M p-values/s",
                     peak_source="FP64 pipe (nominal 1.25 TFLOP/s); ncu: FP64 pipe active 84% at 89% lane use")
        e["frac"] = e["achieved"] / e["peak"] if e.get("peak") else None
        e["traffic"] = load_traffic(name)
        out.append(e)
    out.sort(key=lambda e: -e["ms_per_step"])
    return out


def kernel_roofline(stage_ms, steps, coh, tests, peaks):
    """The dominant stage's roofline, plus every modelled stage."""
    if not stage_ms:
        return None
    ents = stage_rooflines(stage_ms, steps, coh, tests, peaks)
    name, ms = max(stage_ms.items(), key=lambda kv: kv[1]["ms"])
    dom = next((e for e in ents if e["kernel"] == name), None)
    if dom is None:
        dom = {"kernel": name, "bound": "unknown", "ms_per_step": ms["ms"] / steps, "traffic": None}
    dom = dict(dom)
    dom["stages"] = ents
    return dom


def load_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if any."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        return json.load(open(p)).get(kernel)
    except Exception:
        return None


def latency_small_pearson(napg, device, reps=100, warm=10):
    """The 200 x 1,000 Pearson cohort (plain FP64): p50 / p99 of one call over
    `reps` calls after `warm`, device time by CUDA events and host wall time."""
    import torch
    coh = synth.small_pearson_cohort()
    ctx = napg.Context(device)
    st = ctx.stream
    ctx.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    va = coh["cont"]
    n = len(va)
    dev = torch.device("cuda", device)
    out = {"stat": torch.empty((n, n), dtype=torch.float64, device=dev),
           "p": torch.empty((n, n), dtype=torch.float64, device=dev),
           "n": torch.empty((n, n), dtype=torch.int32, device=dev)}
    dev_ms, wall_ms = [], []
    for k in range(warm + reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a.record(st)
        ctx.run("pearson", va, outputs=out, sync=False)
        b.record(st)
        b.synchronize()
        t1 = time.perf_counter()
        if k >= warm:
            dev_ms.append(a.elapsed_time(b))
            wall_ms.append(1000.0 * (t1 - t0))
    ctx.close()
    dev_ms.sort()
    wall_ms.sort()
    q = lambda v, f: v[min(len(v) - 1, int(f * len(v)))]
    pairs = n * (n - 1) // 2
    return {"workload": "200 continuous x 1,000 samples, FP64, 20% MCAR; all-pairs Pearson, plain FP64 form",
            "reps": reps, "warmup": warm, "pairs": pairs,
            "device_ms_p50": q(dev_ms, 0.5), "device_ms_p99": q(dev_ms, 0.99),
            "wall_ms_p50": q(wall_ms, 0.5), "wall_ms_p99": q(wall_ms, 0.99),
            "pairs_per_s_p50": pairs / (q(wall_ms, 0.5) / 1000.0)}


# ------------------------------------------------------------ serve workload --

def serve_requests(coh, rng, count):
    """Random requests of the serving workload: test, mask, variable subset."""
    S = coh["X"].shape[1]
    cont, cat = coh["cont"], coh["cat"]
    out = []
    for _ in range(count):
        test = ["pearson", "spearman", "chi2", "kruskal"][int(rng.integers(0, 4))]
        frac = rng.uniform(0.05, 0.8)
        mask = (rng.random(S) < frac).astype(np.uint8)
        k = int(rng.integers(50, 2001))
        if test in ("pearson", "spearman"):
            va, vb = np.sort(rng.choice(cont, k, replace=False)), None
            pairs = k * (k - 1) // 2
        elif test == "chi2":
            va, vb = np.sort(rng.choice(cat, k, replace=False)), None
            pairs = k * (k - 1) // 2
        else:
            va = np.sort(rng.choice(cat, k // 2, replace=False))
            vb = np.sort(rng.choice(cont, k - k // 2, replace=False))
            pairs = len(va) * len(vb)
        out.append((test, va, vb, mask, pairs))
    return out


def serve_main(args, world, rank, local_rank):
    """Request loop on the resident serving cohort; one replica per GPU."""
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    device = local_rank if world > 1 else 0
    torch.cuda.set_device(device)
    from paper_2505_00448_gb300 import napg
    coh = synth.serving_cohort()
    prec = args.precision
    ctx = napg.Context(device)
    ctx.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    rng = np.random.default_rng(5 + rank)
    slots = 4
    t0 = time.perf_counter()
    ctx.serve_start(0, slots)
    t_start = time.perf_counter() - t0
    # warm-up, then the single-request service time (one request in flight at a time)
    for test, va, vb, m, _ in serve_requests(coh, rng, 4):
        ctx.serve_wait(ctx.serve_submit(test, va, vb, mask=m, precision=prec))
    single = []
    for test, va, vb, m, pairs in serve_requests(coh, rng, 12):
        lat, st, _ = ctx.serve_wait(ctx.serve_submit(test, va, vb, mask=m, precision=prec))
        single.append(lat)
    mu = 1000.0 / statistics.mean(single)          # requests per second, one at a time
    launches0 = napg.kernel_launches()
    clocks = ClockSampler(device)
    clocks.start()
    sweep = []
    for f in (0.25, 0.5, 0.75, 0.9, 1.1, 1.5):
        lam = f * mu
        reqs = serve_requests(coh, rng, args.serve_requests)
        gaps = rng.exponential(1.0 / lam, len(reqs))
        pending = {}
        lat = []
        pairs_done = 0
        t_begin = time.perf_counter()
        t_next = t_begin
        i = 0
        while i < len(reqs) or pending:
            now = time.perf_counter()
            while i < len(reqs) and now >= t_next:
                test, va, vb, m, pairs = reqs[i]
                pending[ctx.serve_submit(test, va, vb, mask=m, precision=prec)] = pairs
                t_next += gaps[i]
                i += 1
            for tk in list(pending):
                d, l, st, _ = ctx.serve_poll(tk)
                if d:
                    lat.append(l)
                    pairs_done += pending.pop(tk)
            time.sleep(2e-4)
        wall = time.perf_counter() - t_begin
        lat.sort()
        sweep.append({"load": f, "lambda_per_s": lam, "requests": len(lat), "wall_s": wall,
                      "p50_ms": statistics.median(lat), "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                      "pairs_per_s": pairs_done / wall})
    clk = clocks.stop()
    launches = napg.kernel_launches() - launches0
    ctx.serve_stop()
    ctx.close()
    sat = max(sweep, key=lambda r: r["pairs_per_s"])
    value = sat["pairs_per_s"]
    value = D.sum_over_ranks(value, dist)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.serve_requests,
                "warmup": 4, "ms_per_step": statistics.mean(single), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f16x2-split/f32-acc/f64" if prec == "mixed" else "f64",
                "data": "synthetic",
                "config": {"workload": "serving loop: resident 100,000-sample x 10,000-variable cohort (8,000 "
                           "continuous FP32, 2,000 categorical 2-8 levels, 35% MCAR); Poisson requests, each a "
                           "random test (Pearson, Spearman, chi-squared, Kruskal-Wallis), mask of 5-80% of the "
                           "samples and 50-2,000 variables; value = pairs/s at the best rate of the sweep",
                           "precision": prec, "slots": slots, "serve_start_s": t_start,
                           "single_request_ms_mean": statistics.mean(single),
                           "capacity_req_per_s": mu, "sweep": sweep},
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------ batch workload --

def batch_main(args, world, rank, local_rank):
    """256 sample contexts per test in one napg_run_batch call each; under torchrun
    the contexts are dealt to the ranks block-cyclically (each rank runs its share)."""
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    device = local_rank if world > 1 else 0
    torch.cuda.set_device(device)
    from paper_2505_00448_gb300 import napg
    coh = synth.context_cohort()
    masks = coh["contexts"]
    K, S = masks.shape
    tests = [("pearson", coh["cont"]), ("chi2", coh["cat"])]
    desc = ("batched contexts: 256 sample subsets (500-20,000 of 20,000 samples, log-uniform sizes, random "
            "condition masks) of a 1,600 continuous FP32 + 400 categorical (2-6 levels) cohort, 25% MCAR; "
            "per context all-pairs Pearson + chi-squared; one napg_run_batch call (one captured CUDA graph) per test")
    prec = args.precision
    ctx = napg.Context(device)
    stream = ctx.stream
    torch.cuda.set_stream(stream)
    ctx.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    dev = torch.device("cuda", device)
    dmask = torch.from_numpy(masks).to(dev)
    mine = D.shard_blocks(K, world, rank)          # this rank's contexts (all of them at N = 1)
    mlist = [dmask[k] for k in mine]
    outs = {}
    for test, va in tests:
        n = len(va)
        outs[test] = [{"stat": torch.empty((n, n), dtype=torch.float64, device=dev),
                       "p": torch.empty((n, n), dtype=torch.float64, device=dev),
                       "n": torch.empty((n, n), dtype=torch.int32, device=dev)} for _ in mine]

    def step():
        ctx.release_cache()
        for test, va in tests:
            ctx.run_batch(test, mlist, va, out="cuda", outputs=outs[test], sync=False, precision=prec)

    t_first = time.perf_counter()
    step()                               # sizing run + capture of both graphs
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t_first
    for _ in range(args.warmup - 1):
        step()
    torch.cuda.synchronize()
    launches0 = napg.kernel_launches()
    clocks = ClockSampler(device)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    per_step = []
    ev0.record(stream)
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        per_step.append((a, b))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = napg.kernel_launches() - launches0
    ms_step = ms_total / args.steps
    ms_step = D.max_over_ranks(ms_step, dist)      # the slowest rank sets the time
    step_ms = sorted(a.elapsed_time(b) for a, b in per_step)
    pairs_ctx = {t: len(va) * (len(va) - 1) // 2 for t, va in tests}
    pairs_step = K * sum(pairs_ctx.values())       # every context of the batch, over all ranks
    value = D.split_value(pairs_step, ms_step / 1000.0)

    # accuracy of the timed outputs on a few contexts (random pairs) against the oracle
    accuracy = None
    if rank == 0 and args.accuracy_pairs > 0:
        from oracle import oracle as O
        rng = np.random.default_rng(7)
        X = coh["X"].astype(np.float64)
        accuracy = {}
        for test, va in tests:
            worst, worst_p, n_ok, cnt = 0.0, 0.0, True, 0
            for k in rng.choice(K, size=3, replace=False):
                ia = rng.integers(0, len(va), args.accuracy_pairs // 3)
                ib = rng.integers(0, len(va), args.accuracy_pairs // 3)
                st, pv, nn = O.run_pairs(test, X, coh["missing"], coh["vtype"], coh["nlev"], va[ia], va[ib],
                                         ctx=masks[k], validate=False)
                gs = outs[test][k]["stat"].cpu().numpy()[ia, ib]
                gp = outs[test][k]["p"].cpu().numpy()[ia, ib]
                gn = outs[test][k]["n"].cpu().numpy()[ia, ib]
                fin = np.isfinite(st) & np.isfinite(gs)
                d = np.abs(gs - st)[fin] if test == "pearson" else (np.abs(gs - st) / np.maximum(np.abs(st), 1e-300))[fin]
                worst = max(worst, float(d.max(initial=0.0)))
                pok = np.isfinite(pv) & (pv > 1e-300) & np.isfinite(gp)
                if pok.any():
                    worst_p = max(worst_p, float((np.abs(gp[pok] - pv[pok]) / pv[pok]).max()))
                n_ok = n_ok and bool(np.array_equal(gn, nn))
                cnt += len(ia)
            accuracy[test] = {"pairs": cnt, "contexts": 3, "stat_error": worst,
                              "stat_metric": "max |d r|" if test == "pearson" else "max rel d stat",
                              "p_rel_error_max": worst_p, "n_exact": n_ok}

    # end to end through the public API with host buffers: cohort and masks in, outputs out
    e2e = None
    if not args.no_e2e:
        # pinned host outputs (allocated once, outside the timed region)
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
        host_outs = {t: [{"stat": pin((len(va), len(va)), torch.float64), "p": pin((len(va), len(va)), torch.float64),
                          "n": pin((len(va), len(va)), torch.int32)} for _ in mine] for t, va in tests}
        hmasks = [masks[k] for k in mine]           # this rank's contexts, as in the timed step
        h2d = coh["X"].nbytes + sum(m.nbytes for m in hmasks)
        d2h = sum(sum(a.nbytes for a in o.values()) for v in host_outs.values() for o in v)
        ctx2 = napg.Context(device)
        times = []
        for k in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx2.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
            for test, va in tests:
                ctx2.run_batch(test, hmasks, va, out="numpy", outputs=host_outs[test], precision=prec)
            times.append(time.perf_counter() - t0)
        ctx2.close()
        t_e2e = D.max_over_ranks(statistics.mean(times[1:] or times), dist)    # the slowest rank
        e2e = {"value": pairs_step / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1000 * t_e2e,
               "path": "host outputs: the captured graph writes device buffers, then every context's outputs "
                       "are copied to pinned host arrays"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        rng = np.random.default_rng(11)
        X = coh["X"].astype(np.float64)
        sizes = masks.sum(axis=1)
        est, desc_s = 0.0, []
        for test, va in tests:
            # cost per pair is about proportional to the context size: time random
            # pairs on 3 contexts and scale by the batch's total samples
            per_sample = []
            for k in rng.choice(K, size=3, replace=False):
                m = 2000 if test == "pearson" else 1000
                pa, pb = rng.choice(va, m), rng.choice(va, m)
                t0 = time.perf_counter()
                O.run_pairs(test, X, coh["missing"], coh["vtype"], coh["nlev"], pa, pb, ctx=masks[k], validate=False)
                dt = time.perf_counter() - t0
                per_sample.append(dt / (m * sizes[k]))
                desc_s.append(f"{test}: {m} pairs in context {k} ({sizes[k]} samples) {dt:.2f}s")
            est += statistics.mean(per_sample) * pairs_ctx[test] * float(sizes.sum())
        cpu = {"value": pairs_step / est, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
               "sample": "; ".join(desc_s) + "; extrapolated by pairs x total context samples"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f16x2-split/f32-acc/f64" if prec == "mixed" else "f64",
                "data": "synthetic",
                "config": {"workload": desc, "precision": prec, "contexts": int(K), "pairs_per_step": pairs_step,
                           "parallelism": (f"contexts dealt block-cyclically over {world} GPUs" if world > 1
                                           else "1 GPU"),
                           "context_samples_total": int(masks.sum()),
                           "l2": "cohort (160 MB) and outputs (13.9 GB) larger than L2: no flush between steps",
                           "first_call_s": t_first, "autotuned": ctx.tune_read(), "step_ms_p50": statistics.median(step_ms),
                           "step_ms_p99": step_ms[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
                "roofline": None, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk, "accuracy_vs_oracle": accuracy}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


# -------------------------------------------------------------------- main --

def paper_sim_main(args, world, rank, local_rank):
    """The paper's simulated benchmark (Sec. 4.1.1): uniform continuous, c = 4
    categorical and dichotomous features with 10% missing per feature, on the two
    lines of its runtime figures (S = 1,000 with F in 250..1,000; F = 1,000 with S
    in 250..1,000). Every test in the plain FP64 form; device time per call
    (median of the timed calls after the warm-up ones). Over N GPUs the grid's
    calls are dealt round robin; value = every rank's pairs over the slowest
    rank's summed device time."""
    import torch
    from paper_2505_00448_gb300 import napg
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    device = local_rank if world > 1 else 0
    torch.cuda.set_device(device)
    grid = sorted({(F, 1000) for F in (250, 500, 750, 1000)} | {(1000, S) for S in (250, 500, 750, 1000)})
    rows = []
    skipped = []
    total_pairs = 0
    total_ms = 0.0
    launches0 = napg.kernel_launches()
    for F, S in grid:
        coh = synth.paper_simulation(F, S)
        ctx = napg.Context(device)
        stream = ctx.stream
        ctx.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
        tests = [("pearson", coh["cont"], None), ("spearman", coh["cont"], None), ("chi2", coh["cat"], None),
                 ("ttest", coh["bins"], coh["cont"]), ("mwu", coh["bins"], coh["cont"]),
                 ("anova", coh["cat"], coh["cont"]), ("kruskal", coh["cat"], coh["cont"])]
        for test, va, vb in tests:
            call = len(rows) + len(skipped)
            if call % world != rank:
                skipped.append(call)
                continue
            nb = len(va) if vb is None else len(vb)
            dev = torch.device("cuda", device)
            out = {"stat": torch.empty((len(va), nb), dtype=torch.float64, device=dev),
                   "p": torch.empty((len(va), nb), dtype=torch.float64, device=dev),
                   "n": torch.empty((len(va), nb), dtype=torch.int32, device=dev)}
            opt = {"mwu_mode": "asymptotic"} if test == "mwu" else {}
            ms = []
            for k in range(args.warmup + args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.run(test, va, vb, outputs=out, sync=False, precision="fp64", **opt)
                e1.record(stream)
                e1.synchronize()
                if k >= args.warmup:
                    ms.append(e0.elapsed_time(e1))
            med = statistics.median(ms)
            pairs = pair_count(test, va, vb)
            rows.append({"test": test, "F": F, "S": S, "ms": med, "pairs_per_s": pairs / (med / 1000.0)})
            total_pairs += pairs
            total_ms += med
        ctx.close()
    launches = napg.kernel_launches() - launches0
    total_pairs = D.sum_over_ranks(total_pairs, dist)
    total_ms = D.max_over_ranks(total_ms, dist)
    launches = int(D.sum_over_ranks(launches, dist))
    value = total_pairs / (total_ms / 1000.0)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        coh = synth.paper_simulation(1000, 1000)
        tests = [("pearson", coh["cont"], None), ("spearman", coh["cont"], None), ("chi2", coh["cat"], None),
                 ("ttest", coh["bins"], coh["cont"]), ("mwu", coh["bins"], coh["cont"]),
                 ("anova", coh["cat"], coh["cont"]), ("kruskal", coh["cat"], coh["cont"])]
        cpu = oracle_sample(coh, tests, budget_s=min(args.cpu_budget, 14.0))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"parallelism": (f"the grid's calls dealt round robin over {world} GPUs" if world > 1
                                           else "1 GPU"),
                           "workload": "the paper's simulated benchmark: uniform [0,1] continuous, c = 4 categorical "
                           "and dichotomous features, 10% missing per feature; S = 1,000 with F = 250..1,000 and "
                           "F = 1,000 with S = 250..1,000; all seven tests, plain FP64 form; one step = every "
                           "(test, F, S) call once; value = pairs over the summed device times",
                           "calls": rows},
                "roofline": None, "cpu_baseline": cpu, "e2e": None, "gpu_launches": int(launches), "clocks": None}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100,
                    help="timed steps (the default gives the p99 over 100 steps; about 3 s timed on the mixed cohort)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="mixed", choices=["mixed", "ranks", "batch", "serve", "small-pearson",
                                                             "paper-sim"])
    ap.add_argument("--serve-requests", type=int, default=40, help="requests per arrival rate (serve workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP64 comparator step")
    ap.add_argument("--accuracy-pairs", type=int, default=300)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="variables x scale (profiling captures only; bench lines use 1.0)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world, rank, local_rank = D.env_ranks()

    if args.impl == "reference":
        if rank != 0:
            return
        coh, tests, desc = make_workload(args.workload, args.scale)
        samples = []
        for k in range(args.warmup + args.steps):
            r = oracle_sample(coh, tests, budget_s=max(0.5, 60.0 / (args.warmup + args.steps)), seed=k,
                             one_thread=False)
            if k >= args.warmup:
                samples.append(r)
        v = statistics.mean(r["value"] for r in samples)
        # The oracle cannot run a whole step of this workload in the arm's time:
        # each step times a bounded random sample of its pairs, and ms_per_step is
        # the step's pair count at the sampled rate (an extrapolation); the
        # measured seconds of the sampled pairs are reported beside it.
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * sum(pair_count(t, va, vb) for t, va, vb in tests) / v,
                "ms_per_step_basis": "extrapolated: the step's pairs at the rate measured on sampled pairs",
                "sampled_ms_per_step": 1000.0 * statistics.mean(r["sample_seconds"] for r in samples),
                "sampled_pairs_per_step": int(statistics.mean(r["sample_pairs"] for r in samples)),
                "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": desc, "reference": "plain FP64 CPU oracle (oracle/napg_oracle.c)"},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": samples[0]["cores"], "kind": "oracle",
                                 "sample": samples[0]["sample"]},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if args.workload == "batch":
        return batch_main(args, world, rank, local_rank)
    if args.workload == "serve":
        return serve_main(args, world, rank, local_rank)
    if args.workload == "paper-sim":
        return paper_sim_main(args, world, rank, local_rank)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    device = local_rank if world > 1 else 0
    torch.cuda.set_device(device)
    from paper_2505_00448_gb300 import napg

    coh, tests, desc = make_workload(args.workload, args.scale)
    if args.scale != 1.0:
        desc += f" [variables scaled by {args.scale} for profiling]"
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    ctx = napg.Context(device)
    stream = ctx.stream                     # every kernel of the library runs on this stream
    torch.cuda.set_stream(stream)
    ctx.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    dev = torch.device("cuda", device)
    outs = {}
    for test, va, vb in tests:
        na = len(va)
        nb = na if vb is None else len(vb)
        outs[test] = {"stat": torch.empty((na, nb), dtype=torch.float64, device=dev),
                      "p": torch.empty((na, nb), dtype=torch.float64, device=dev),
                      "n": torch.empty((na, nb), dtype=torch.int32, device=dev)}
    # the small Pearson cohort is the plain FP64 form by definition
    prec = "fp64" if args.workload == "small-pearson" else args.precision

    def step(per_test_events=None):
        # every step builds its own derived data (planes, presort) once and
        # shares it only between that step's tests
        ctx.release_cache()
        for test, va, vb in tests:
            if per_test_events is not None:
                per_test_events[test][0].record(stream)
            if world > 1:
                # this rank's part of the split call (napg_run_part): its output rows' pairs
                ctx.run_part(test, va, vb, part=rank, nparts=world, outputs=outs[test], precision=prec)
            else:
                ctx.run(test, va, vb, outputs=outs[test], sync=False, precision=prec)
            if per_test_events is not None:
                per_test_events[test][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region
    ev = {t: [] for t, _, _ in tests}
    launches0 = napg.kernel_launches()
    ctx.trace(True)
    ctx.trace_read()
    clocks = ClockSampler(device)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    step_events = []
    start.record(stream)
    for _ in range(args.steps):
        pe = {t: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for t, _, _ in tests}
        step(pe)
        step_events.append(pe)
    end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = start.elapsed_time(end)
    clk = clocks.stop()
    launches = napg.kernel_launches() - launches0
    trace = ctx.trace_read()
    ctx.trace(False)
    ms_step = ms_total / args.steps
    ms_step = D.max_over_ranks(ms_step, dist)      # the slowest rank sets the time
    per_test_ms = {t: [pe[t][0].elapsed_time(pe[t][1]) for pe in step_events] for t, _, _ in tests}
    first, last = tests[0][0], tests[-1][0]
    step_ms = sorted(pe[first][0].elapsed_time(pe[last][1]) for pe in step_events)
    pairs_step = sum(pair_count(t, va, vb) for t, va, vb in tests)   # the whole call, over all ranks
    value = D.split_value(pairs_step, ms_step / 1000.0)
    # the split's outputs, gathered once after the timed region: every entry of
    # every test must have been written by exactly its owner
    split_check = None
    if dist:
        for o in outs.values():
            o["n"].fill_(-1)
        step()
        torch.cuda.synchronize()
        complete = True
        for test, va, vb in tests:
            loc = outs[test]["n"]
            allr = [torch.empty_like(loc) for _ in range(world)]
            dist.all_gather(allr, loc)
            if rank == 0:
                parts = [a.cpu().numpy() for a in allr]
                na, nb = loc.shape
                got = D.stitch(parts, na, nb, vb is None)
                complete &= bool((got >= 0).all())
        split_check = {"gathered": True, "every_entry_written_by_its_owner": complete}

    # e2e through the public API with host buffers: upload + run + download per step
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(coh["X"]).pin_memory()
        # pinned host outputs: each test's copies back overlap the next test's kernels
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
        host_out = {t: {"stat": pin(tuple(o["stat"].shape), torch.float64), "p": pin(tuple(o["p"].shape), torch.float64),
                        "n": pin(tuple(o["n"].shape), torch.int32)} for t, o in outs.items()}
        h2d = Xh.numel() * Xh.element_size()
        d2h = sum(sum(a.nbytes for a in v.values()) for v in host_out.values())
        ctx2 = napg.Context(device)
        e2e_steps = max(1, min(args.steps, 5))
        times = []
        for k in range(e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx2.load_cohort(Xh, coh["vtype"], coh["nlev"], coh["missing"])
            for test, va, vb in tests:
                if world > 1:       # this rank's part (synchronous), as in the timed step
                    ctx2.run_part(test, va, vb, part=rank, nparts=world, outputs=host_out[test], precision=prec)
                else:
                    ctx2.run(test, va, vb, outputs=host_out[test], out="numpy", sync=False, precision=prec)
            ctx2.sync()
            dt = time.perf_counter() - t0
            if k > 0:
                times.append(dt)
        ctx2.close()
        if world > 1:
            h2d += d2h      # a part's host outputs are staged on the device first (other parts' entries kept)
        # the median step (a host-timed loop sees the host's own jitter), slowest rank
        t_e2e = D.max_over_ranks(statistics.median(times), dist)
        e2e = {"value": pairs_step / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * t_e2e,
               "ms_steps": [round(1000 * t, 2) for t in times]}

    # error of the timed (last step's) outputs against the FP64 oracle on sampled pairs
    accuracy = None
    if rank == 0 and args.accuracy_pairs > 0:
        accuracy = sampled_accuracy(coh, tests, outs, args.accuracy_pairs)

    # the plain FP64 GPU form of the same step, once, for the comparison the metric names
    comparator = None
    if rank == 0 and prec == "mixed" and not args.no_compare:
        ev_c = {t: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for t, _, _ in tests}
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for test, va, vb in tests:
            ev_c[test][0].record(stream)
            ctx.run(test, va, vb, outputs=outs[test], sync=False, precision="fp64")
            ev_c[test][1].record(stream)
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1)
        comparator = {"precision": "fp64", "value": pairs_step / (cms / 1000.0), "unit": UNIT, "ms_per_step": cms,
                      "per_test_ms": {t: ev_c[t][0].elapsed_time(ev_c[t][1]) for t, _, _ in tests},
                      "speedup_mixed_over_fp64": cms / ms_step}

    roof = kernel_roofline(trace.get("stages", {}), args.steps, coh, tests, peaks)

    # effect sizes and multiple-testing correction after the hot path: the effect
    # stage per test (28 bytes per pair: statistic and n read, two effect sizes
    # written) and a Benjamini-Hochberg pass over the first test's p-values
    post = None
    if rank == 0 and args.scale == 1.0:
        eff = {}
        ctx.trace(True)
        for test, va, vb in tests:
            ctx.trace_read()
            ctx.run(test, va, vb, sync=True, precision=prec, effects=True)
            stg = ctx.trace_read().get("stages", {}).get("effect_sizes")
            if stg:
                pc = pair_count(test, va, vb) if vb is not None else len(va) * len(va)
                eff[test] = {"ms": stg["ms"], "gb_per_s": 28.0 * pc / (stg["ms"] / 1000.0) / 1e9}
        ctx.trace(False)
        p0 = outs[tests[0][0]]["p"]
        ctx.adjust(p0, "bh", symmetric=tests[0][2] is None)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ctx.adjust(p0, "bh", symmetric=tests[0][2] is None)
        a1.record(stream)
        torch.cuda.synchronize()
        m_tests = pair_count(*tests[0])
        post = {"effect_sizes": eff, "adjust_bh": {"matrix": list(p0.shape), "tests": m_tests,
                                                   "ms": a0.elapsed_time(a1),
                                                   "mtests_per_s": m_tests / (a0.elapsed_time(a1) / 1000.0) / 1e6}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(coh, tests, budget_s=args.cpu_budget)
    latency = latency_small_pearson(napg, device) if (rank == 0 and args.workload == "mixed" and args.scale == 1.0) else None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f16x2-split/f32-acc/f64" if prec == "mixed" else "f64",
                "data": "synthetic",
                "config": {"workload": desc, "precision": prec, "pairs_per_step": pairs_step,
                           "parallelism": (f"split over {world} GPUs: napg_run_part, output rows in blocks of "
                                           f"{D.PART_ROWS} dealt back and forth" if world > 1 else "1 GPU"),
                           "split_check": split_check,
                           "l2": "cohort (1.0 GB) larger than L2: no flush between steps",
                           "step_ms_p50": statistics.median(step_ms),
                           "step_ms_p99": step_ms[min(len(step_ms) - 1, int(0.99 * len(step_ms)))],
                           "per_test_ms": {t: statistics.median(v) for t, v in per_test_ms.items()},
                           "per_test_pairs_per_s": {t: pair_count(t, va, vb) / (statistics.median(per_test_ms[t]) / 1e3)
                                                    for t, va, vb in tests},
                           "stage_ms_per_step": {k: v["ms"] / args.steps for k, v in trace.get("stages", {}).items()},
                           "autotuned": ctx.tune_read()},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
                "accuracy_vs_oracle": accuracy, "fp64_plain_gpu": comparator, "latency_small_pearson": latency,
                "postprocess": post}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
