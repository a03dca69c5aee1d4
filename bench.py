"""Benchmark: Kalman propagate + chi2 + update steps/s on one GB300 (or N replicas).

Workload: Phase-2-like events, 64 per batch, 20,000 tracks and 50,000 noise hits each, 10 barrel
cylinders + 2x12 endcap disks, best-N = 6.  One step = one pass of the whole hot path over the
batch: bin every layer's hits, seed, combinatorial forward search, and the Kalman fit of every
track over its known hits.  Kalman steps = candidate-layer steps of the search + track-layer
steps of the fit (crossed layers), counted by the kernels themselves.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Inputs are seeded and synthetic (see paper_2312_11728_gb300/synth.py).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Kalman propagate+χ²+update steps/s on 1 GB300; % of FP32/HBM roofline"
UNIT = "Kalman steps/s"
N_EVENTS, N_TRACKS, N_NOISE = 64, 20000, 50000
WORKLOAD = "phase2_like_{events}ev_20k_tracks_50k_noise_bestN6"

# FP32 operations per unit of work (FMA = 2), counted by ncu's per-thread instruction counters
# (FFMA/FFMA2/FADD/FADD2/FMUL/FMUL2 with true predicates) on the search and fit kernels for the
# 8-event version of this workload, divided by the work counters of the same run:
#   find: per crossed candidate-layer step, k_find's propagation with Jacobian, transport and
#         material, window and chi2 of the window's hits (a4-a9);
#   update: per Kalman update of the search, k_select's merge of the children and the Joseph
#         update (a10-a11);
#   fit: per track-layer step of k_fit (a4-a9, a11 on one hit);
#   seed_fp64, seed_fp32: per seed, the mixed-precision seed fit of every seed plus the FP64 refit
#         of the low-|q/pT| ones (DFMA/DADD/DMUL and the FP32 forms), both kernels of one seed call.
# Multi-function-unit work (sqrt, rsqrt, division seeds, sincos, log, atan2) is not counted.
FLOPS = dict(find=1224.7, update=731.1, fit=1642.6, seed_fp64=1984.8, seed_fp32=1878.1)
# the search and fit kernel sources the counts (and the DRAM traffic in profiles/) belong to
KERNEL_SOURCES = ("paper_2312_11728_gb300/csrc/k_build.cu", "paper_2312_11728_gb300/csrc/kalman.cuh",
                  "paper_2312_11728_gb300/csrc/trig.cuh", "paper_2312_11728_gb300/csrc/dual.cuh",
                  "paper_2312_11728_gb300/csrc/internal.h", "paper_2312_11728_gb300/build.py")


# Algorithmic HBM bytes per unit of work: the data each stage must read and write at least once,
# whatever the kernel design (a state is 27 words = 108 B: 6 parameters + 21 covariance words):
#   search: a crossed candidate-layer step reads the candidate's state (108 B); each kept child
#     with a new state (a hit update, a miss or a stop) writes it (108 B) with its trail entry (the
#     parent slot and hit, 4 B); every hit of the batch is read once (position, 6 covariance words
#     and id, 40 B, with its binned (eta, phi), 8 B) with the bins' offsets (4 B per bin); each
#     seed's start state is read (108 B) and its result written (27 words, chi2, score and two
#     counts, 124 B, plus one hit id per plan step);
#   fit: per track-layer step its hit (40 B) and hit id (4 B); per track its starting state (108 B)
#     and its result (27 words, chi2, status: 116 B);
#   seed: per seed its 3 hit ids (12 B) and hits (3 x 40 B), its state record written (128 B), its
#     ordering key (8 B).
ALG_BYTES = dict(state=108, child=112, hit=48, bin=4, seed_in=108, seed_out=124, hit_id=4,
                 fit_step=44, fit_track=224, seed=268)


def search_bytes(c, n_hits, n_bins, n_seeds, max_plan):
    """c: build counters; c[5] (children with a new state) when reported, else the updates."""
    kept = c[5] if len(c) > 5 else c[2]
    return (ALG_BYTES["state"] * c[0] + ALG_BYTES["child"] * kept + ALG_BYTES["hit"] * n_hits
            + ALG_BYTES["bin"] * n_bins
            + (ALG_BYTES["seed_in"] + ALG_BYTES["seed_out"] + ALG_BYTES["hit_id"] * max_plan) * n_seeds)


def fit_bytes(c, n_tracks):
    return ALG_BYTES["fit_step"] * c[0] + ALG_BYTES["fit_track"] * n_tracks


def roofline(name, ms, flops, nbytes, fp32_peak, hbm, traffic=None, fp64_flops=0.0, fp64_peak=None):
    """Roofline of one stage: its time bound is the slower of the FP32 (or FP64) pipe and the
    HBM bytes, max(F / P, B / BW); frac = that bound / the measured time (the larger of the two
    fractions).  achieved / peak are given in the bound's own unit."""
    t = ms / 1e3
    t_fp32 = flops / (fp32_peak * 1e12)
    t_fp64 = fp64_flops / (fp64_peak * 1e12) if fp64_peak else 0.0
    t_hbm = nbytes / (hbm * 1e9)
    if t_hbm >= max(t_fp32, t_fp64):
        bound, achieved, peak, unit = "hbm", nbytes / t / 1e9, hbm, "GB/s"
    elif t_fp64 > t_fp32:
        bound, achieved, peak, unit = "fp64", fp64_flops / t / 1e12, fp64_peak, "TFLOP/s"
    else:
        bound, achieved, peak, unit = "alu", flops / t / 1e12, fp32_peak, "TFLOP/s"
    r = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
         "traffic": traffic, "stage": name, "measured_ms": ms,
         "bound_ms": {"hbm": t_hbm * 1e3, "fp32": t_fp32 * 1e3},
         "hbm_frac": t_hbm / t, "fp32_frac": t_fp32 / t,
         "algorithmic_bytes": int(nbytes), "algorithmic_fp32_flops": int(flops)}
    if fp64_peak:
        r["bound_ms"]["fp64"] = t_fp64 * 1e3
        r["fp64_frac"] = t_fp64 / t
        r["algorithmic_fp64_flops"] = int(fp64_flops)
    if traffic:
        r["traffic_over_algorithmic"] = traffic / nbytes
    return r


def build_flops(c):
    """c: build counters [steps, chi2 evaluations, updates, hits tested, Newton iterations]."""
    return FLOPS["find"] * c[0] + FLOPS["update"] * c[2]


def fit_flops(c):
    return FLOPS["fit"] * c[0]


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _gen_event(args):
    e, seed = args
    from paper_2312_11728_gb300 import synth as S
    g = S.geometry_phase2()
    return S.simulate_event(g, N_TRACKS, seed, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=N_NOISE)


def _gen_modular_event(args):
    e, seed = args
    from paper_2312_11728_gb300 import synth as S
    g = S.geometry_phase2_modular_disks()
    return S.simulate_event(g, N_TRACKS, seed, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=N_NOISE)


def make_modular_batch(seed, n_events):
    """The same events' recipe on the modular tracker (cylinders 3-5 built from flat and tilted
    modules, the 4th-6th disk of each endcap from planar modules), generated in a spawn pool."""
    from paper_2312_11728_gb300 import synth as S
    g = S.geometry_phase2_modular_disks()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        evs = pool.map(_gen_modular_event, [(e, seed) for e in range(n_events)])
    return g, S.concat_events(evs, g.n_layers)


def make_batch(seed, n_events=N_EVENTS):
    """Events generated in a spawn pool (before any CUDA call in this process)."""
    from paper_2312_11728_gb300 import synth as S
    g = S.geometry_phase2()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        evs = pool.map(_gen_event, [(e, seed) for e in range(n_events)])
    return g, S.concat_events(evs, g.n_layers), evs


def _gen_uneven_event(args):
    e, n, seed = args
    from paper_2312_11728_gb300 import synth as S
    g = S.geometry_phase2()
    return S.simulate_event(g, int(n), seed, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0,
                            noise_total=int(2.5 * n))


def _gen_looper_event(args):
    e, seed = args
    from paper_2312_11728_gb300 import synth as S
    g = S.geometry_phase2()
    return S.simulate_event(g, 20000, seed, e, pt_sampler=S.sample_pt_loopers, eta_max=3.0, noise_total=0)


def make_config_batches(seed):
    """The other configurations' inputs, generated in a spawn pool before any CUDA call:
    the uneven batch (256 events, Poisson(8,000) tracks clipped to [200, 25,000], noise 2.5 per
    track) and the looper sweep (50 events x 20,000 tracks, 10% at 0.5-0.7 GeV, no noise)."""
    from paper_2312_11728_gb300 import synth as S
    g = S.geometry_phase2()
    counts = S.uneven_counts(256, 8000, 200, 25000, seed)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        uneven = pool.map(_gen_uneven_event, [(e, int(n), seed) for e, n in enumerate(counts)])
        loop = pool.map(_gen_looper_event, [(e, seed + 5) for e in range(50)])
    return g, S.concat_events(uneven, g.n_layers), S.concat_events(loop, g.n_layers)


def scan_launches(n):
    """Kernels one device-wide exclusive scan of n ints launches (mirrors csrc/k_hits.cu)."""
    nb = (n + 2047) // 2048
    return 1 if nb <= 1 else 3 + scan_launches(nb)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.rows = [r.split(", ") for r in out.strip().splitlines() if r.count(",") >= 8]

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def cpu_baseline(g, batch, fit, params, n_events_sample=2):
    """The FP64 oracle, as it stands, on a bounded sample: every seed and track of the first events."""
    import oracle
    from oracle import parity as PR
    orc = oracle.Oracle(g, params)
    sel = np.nonzero(batch.seed_event < n_events_sample)[0]
    t0 = time.perf_counter()
    o = PR.oracle_build(orc, batch, sel)
    tsel = np.nonzero(fit.event < n_events_sample)[0]
    r = orc.fit_batch(fit.layers[tsel], fit.hits[tsel], batch.hit_xyz.astype(np.float64),
                      batch.hit_cov.astype(np.float64), fit.p0[tsel].astype(np.float64),
                      fit.c0[tsel].astype(np.float64))
    dt = time.perf_counter() - t0
    steps = int(o["counters"][0] + r["counters"][0])
    return {"value": steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_events_sample} of {batch.n_events} events: {len(sel)} seeds built + {len(tsel)} tracks "
                      f"fitted ({steps} Kalman steps, {dt:.1f} s, FP64, single thread)"}


def _oracle_event(args):
    """One event through the oracle (search of all its seeds, fit of all its tracks) in a worker
    process; returns (Kalman steps, seconds of compute)."""
    g, ev, params, seed = args
    import oracle
    from oracle import parity as PR
    from paper_2312_11728_gb300 import pipeline, synth as S
    b = S.concat_events([ev], g.n_layers)
    fi = pipeline.fit_inputs(b, seed=seed)
    orc = oracle.Oracle(g, params)
    t0 = time.perf_counter()
    o = PR.oracle_build(orc, b)
    r = orc.fit_batch(fi.layers, fi.hits, b.hit_xyz.astype(np.float64), b.hit_cov.astype(np.float64),
                      fi.p0.astype(np.float64), fi.c0.astype(np.float64))
    return int(o["counters"][0] + r["counters"][0]), time.perf_counter() - t0


def cpu_baseline_all_cores(g, evs, params):
    """The same oracle on every host core at once: one event per worker process (spawned), the
    throughput = all workers' steps / the slowest worker's compute time."""
    n = max(1, min(os.cpu_count() or 1, len(evs), 64))
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_event, [(g, evs[e], params, e) for e in range(n)])
    steps = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return {"value": steps / dt, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} of {len(evs)} events, one per process: every seed built and every track fitted "
                      f"({steps} Kalman steps, slowest worker {dt:.1f} s, FP64)"}


def run_reference(args, rank, world=1):
    if rank != 0:   # the oracle baseline runs once, on rank 0's host cores
        return
    from paper_2312_11728_gb300 import pipeline, synth as S
    g, batch, _ = make_batch(0, n_events=2)
    fit = pipeline.fit_inputs(batch)
    params = S.default_params()
    import oracle
    from oracle import parity as PR
    orc = oracle.Oracle(g, params)
    rng = np.random.default_rng(0)
    per_step = 1500
    times, steps = [], []
    for it in range(args.warmup + args.steps):
        sel = np.sort(rng.choice(batch.seed_hits.shape[0], per_step, replace=False))
        tsel = np.sort(rng.choice(fit.layers.shape[0], per_step, replace=False))
        t0 = time.perf_counter()
        o = PR.oracle_build(orc, batch, sel)
        r = orc.fit_batch(fit.layers[tsel], fit.hits[tsel], batch.hit_xyz.astype(np.float64),
                          batch.hit_cov.astype(np.float64), fit.p0[tsel].astype(np.float64),
                          fit.c0[tsel].astype(np.float64))
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            steps.append(int(o["counters"][0] + r["counters"][0]))
    value = sum(steps) / sum(times)
    sample = f"per step {per_step} random seeds built + {per_step} tracks fitted from the same workload"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(events=N_EVENTS), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_e2e(args, ctx, db, batch, fit, g, stream, kalman_steps, world, local, dist):
    """The same pass through the C ABI's host-array call (mkgb_run_host) with page-locked host
    buffers: every step copies its inputs in and its results out inside the timed region (the
    library overlaps the copies with the kernels); host wall-clock time of the synchronous calls."""
    import torch
    from paper_2312_11728_gb300 import mkgb, pipeline
    n_seeds = batch.seed_hits.shape[0]
    n_tracks = fit.layers.shape[0]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h = dict(xyz=pin(batch.hit_xyz), cov=pin(batch.hit_cov), seeds=pin(batch.seed_hits), layers=pin(fit.layers),
             hits=pin(fit.hits), p0=pin(fit.p0), c0=pin(fit.c0))
    ho = {k: torch.from_numpy(v).pin_memory() for k, v in mkgb.alloc_tracks(n_seeds, g.max_plan).items()}
    hf = dict(p=torch.zeros((n_tracks, 6), dtype=torch.float32).pin_memory(),
              c=torch.zeros((n_tracks, 21), dtype=torch.float32).pin_memory(),
              chi2=torch.zeros(n_tracks, dtype=torch.float32).pin_memory(),
              status=torch.zeros(n_tracks, dtype=torch.int32).pin_memory())
    h2d = sum(v.numel() * v.element_size() for v in h.values())
    d2h = sum(v.numel() * v.element_size() for v in ho.values()) + sum(v.numel() * v.element_size() for v in hf.values())

    def e2e_step():
        ctx.run_host(db.n_events, db.seg_off, h["xyz"], h["cov"], h["seeds"], ho, h["layers"], h["hits"], h["p0"],
                     h["c0"], hf["p"], hf["c"], hf["chi2"], hf["status"])

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    n_e2e = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    dt = time.perf_counter() - t0
    # the host results equal the device-resident pass's (same kernels, same inputs)
    same = bool(torch.equal(ho["hits"], db.out["hits"].cpu()) and torch.equal(hf["chi2"], db.fit["chi2"].cpu()))
    value, _, _ = pipeline.replica_throughput(dt, kalman_steps * n_e2e, dist, f"cuda:{local}")
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": dt * 1e3 / n_e2e, "call": "mkgb_run_host (one call per step, page-locked host arrays)",
            "same_results_as_device_pass": same}


def measure_fp64_plain(args, g, params, evs, stream, local, rank, dist):
    """The plain comparison path: every Kalman step (seed, search, fit) in FP64, one event per
    call sequence (no batching across events), on the same events; 1 warm-up + 1 timed pass."""
    import torch
    from paper_2312_11728_gb300 import pipeline, synth as S
    p64 = dict(params, precision=2)
    ctx = pipeline.make_context(g, p64, device=local, stream=stream)
    dbs = []
    for ev in evs:
        b = S.concat_events([ev], g.n_layers)
        dbs.append(pipeline.DeviceBatch(b, pipeline.fit_inputs(b, seed=rank), g.max_plan, f"cuda:{local}"))
    steps = 0
    for db in dbs:                        # warm-up pass, counting the Kalman steps
        pipeline.run_step(ctx, db)
        steps += int(ctx.counters(0)[0] + ctx.counters(1)[0])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for db in dbs:
        pipeline.run_step(ctx, db)
    e1.record(stream)
    torch.cuda.synchronize()
    value, wall, _ = pipeline.replica_throughput(e0.elapsed_time(e1) / 1e3, steps, dist, f"cuda:{local}")
    return {"value": value, "unit": UNIT, "ms_per_step": wall * 1e3, "kalman_steps": steps,
            "mode": "seed, search and fit all in FP64; events one at a time; same events as the FP32 line"}


def measure_fit_backward(ctx, db, fi, stream, dist, local):
    """The backward fit (Sec. 2.2) of the batch's fit workload from its forward fit's results:
    one mkgb_fit_backward call after a warm-up call, CUDA-event timed; one step per listed
    layer (the first an update on the start layer, the others a backward crossing + update)."""
    import torch
    from paper_2312_11728_gb300 import pipeline
    f = db.fit
    n = f["layers"].shape[0]
    o = dict(p=torch.zeros((n, 6), device=f"cuda:{local}"), c=torch.zeros((n, 21), device=f"cuda:{local}"),
             chi2=torch.zeros(n, device=f"cuda:{local}"),
             status=torch.zeros(n, dtype=torch.int32, device=f"cuda:{local}"))
    call = lambda: ctx.fit_backward(f["layers"], f["hits"], f["p"], f["c"], o["p"], o["c"], o["chi2"], o["status"])
    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    call()
    e1.record(stream)
    torch.cuda.synchronize()
    steps = int((fi.layers >= 0).sum())
    value, wall, _ = pipeline.replica_throughput(e0.elapsed_time(e1) / 1e3, steps, dist, f"cuda:{local}")
    ok = float((o["status"] == 0).float().mean().item())
    return {"value": value, "unit": "backward-fit track-layer steps/s", "ms": wall * 1e3, "tracks": n,
            "steps": steps, "status_ok_fraction": ok, "cov_scale": 100.0,
            "workload": "the fit workload of the timed batch, started from its forward fit's results"}


def measure_cleaning(ctx, db, g, stream, local):
    """Seed cleaning over the batch's seeds and the quality filter + duplicate removal over its
    found tracks (seed hits + found hits), one call each after a warm-up, CUDA-event timed."""
    import torch
    n = db.seeds.shape[0]
    keep = torch.zeros(n, dtype=torch.int32, device=f"cuda:{local}")
    hits = torch.cat([db.seeds, torch.where(db.out["hits"] >= 0, db.out["hits"], -1)], dim=1).contiguous()
    score = torch.where(torch.isfinite(db.out["score"]), db.out["score"],
                        torch.full_like(db.out["score"], -1e30)).contiguous()
    calls = {"clean_seeds": lambda: ctx.clean_seeds(db.seeds, keep),
             "remove_duplicates": lambda: ctx.remove_duplicates(hits, score, keep, min_hits=6, frac=0.5)}
    res = {"seeds": int(n), "track_width": int(hits.shape[1])}
    for name, call in calls.items():
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name + "_ms"] = e0.elapsed_time(e1)
        res[name + "_kept"] = int(keep.sum().item())
    return res


def measure_modular(mod, params, shapes, stream, local, dist):
    """The search and the fit on the modular tracker (Sec. 3.1 module planes, the Phase-2 tilted
    barrel; Sec. 2.2 overlap hits): module hits tested and updated on their planes, overlap hits
    picked up.  One warm-up then one CUDA-event timed search and fit; the same hits loaded
    without module ids (every hit taken on its cylinder) give the cost of the plane steps."""
    import torch
    from paper_2312_11728_gb300 import mkgb, pipeline
    g, batch = mod
    fi = pipeline.fit_inputs(batch)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(f"cuda:{local}")
    ctx = pipeline.make_context(g, params, device=local, stream=stream)
    ctx.set_launch(shapes[0], shapes[1])
    xyz, cov, hm, seeds = dev(batch.hit_xyz), dev(batch.hit_cov), dev(batch.hit_mod), dev(batch.seed_hits)
    n, nt = int(batch.seed_hits.shape[0]), int(fi.layers.shape[0])
    out = mkgb.alloc_tracks(n, g.max_plan, device=f"cuda:{local}", ovl=True)
    L, H, P0, C0 = dev(fi.layers), dev(fi.hits), dev(fi.p0), dev(fi.c0)
    fo = [torch.zeros((nt, 6), device=f"cuda:{local}"), torch.zeros((nt, 21), device=f"cuda:{local}"),
          torch.zeros(nt, device=f"cuda:{local}"), torch.zeros(nt, dtype=torch.int32, device=f"cuda:{local}")]
    res = {"events": int(batch.n_events), "seeds": n, "tracks": nt, "modules": int(g.modules.c.shape[0]),
           "modular_layers": sorted(int(l) for l in g.modules.grid)}
    for label, hmod in (("planes", hm), ("cylinders_only", None)):
        ctx.load_hits(batch.n_events, batch.hit_off, xyz, cov, hit_module=hmod)
        ctx.seed(seeds)
        ctx.build(out)
        ctx.fit(L, H, P0, C0, *fo)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        ctx.build(out)
        e[1].record(stream)
        ctx.fit(L, H, P0, C0, *fo)
        e[2].record(stream)
        torch.cuda.synchronize()
        bc, fc = ctx.counters(0), ctx.counters(1)
        ms_s, ms_f = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        steps = int(bc[0] + fc[0])
        value, wall, _ = pipeline.replica_throughput((ms_s + ms_f) / 1e3, steps, dist, f"cuda:{local}")
        r = {"value": value, "unit": UNIT, "search_ms": ms_s, "fit_ms": ms_f, "kalman_steps": steps,
             "search_chi2": int(bc[1]), "search_updates": int(bc[2]),
             "found_fraction": float(torch.isfinite(out["score"]).float().mean().item())}
        if hmod is not None:
            r["overlap_hits"] = int((out["ovl"] >= 0).sum().item())
            r["tracks_with_overlap"] = int((out["ovl"] >= 0).any(1).sum().item())
            r["fit_status_ok_fraction"] = float((fo[3] == 0).float().mean().item())
        res[label] = r
    return res


def _fit_errors(gpu, r, sample):
    """Worst errors of sampled fits against the oracle, in units of the tolerances."""
    from oracle import parity as PR
    rep = PR.compare_fit({k: v[sample] for k, v in gpu.items()}, r)
    return {"tracks_compared": rep["n"], "status_mismatch": rep["status_bad"], "param_bad": rep["param_bad"],
            "cov_bad": rep["cov_bad"], "chi2_bad": rep["chi2_bad"], "worst_param": rep["worst_param"],
            "worst_cov": rep["worst_cov"], "worst_chi2": rep["worst_chi2"]}


def measure_config_small(params, stream, local):
    """1,000 tracks, 10 barrel cylinders, 200 noise hits per layer, one event: the whole pass
    (CUDA events, mean of 10 after 3 warm-ups) and every seed and track against the oracle."""
    import torch
    import oracle
    from oracle import parity as PR
    from paper_2312_11728_gb300 import pipeline, synth as S
    g, ev = S.workload_small_barrel()
    b = S.concat_events([ev], g.n_layers)
    fi = pipeline.fit_inputs(b)
    ctx = pipeline.make_context(g, params, device=local, stream=stream)
    db = pipeline.DeviceBatch(b, fi, g.max_plan, f"cuda:{local}")
    for _ in range(3):
        pipeline.run_step_fused(ctx, db)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    for _ in range(10):
        pipeline.run_step_fused(ctx, db)
    e[1].record(stream)
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / 10
    pipeline.run_step(ctx, db)
    torch.cuda.synchronize()
    steps = int(ctx.counters(0)[0] + ctx.counters(1)[0])
    gpu = {k: v.cpu().numpy() for k, v in db.out.items()}
    orc = oracle.Oracle(g, params)
    t0 = time.perf_counter()
    o = PR.oracle_build(orc, b)
    X, V = b.hit_xyz.astype(np.float64), b.hit_cov.astype(np.float64)
    r = orc.fit_batch(fi.layers, fi.hits, X, V, fi.p0.astype(np.float64), fi.c0.astype(np.float64))
    t_orc = time.perf_counter() - t0
    rep = PR.compare_build(gpu, o)
    gf = {k: db.fit[k].cpu().numpy() for k in ("p", "c", "chi2", "status")}
    return {"value": steps / (ms / 1e3), "unit": UNIT, "ms_per_pass": ms, "kalman_steps": steps,
            "oracle": {"value": int(o["counters"][0] + r["counters"][0]) / t_orc, "unit": UNIT, "cores": 1,
                       "seconds": t_orc},
            "workload": "1,000 tracks, 10 barrel cylinders, 200 noise hits per layer, one event (launch-bound)",
            "build_vs_oracle": {"seeds": rep["n"], "hit_mismatch": int(len(rep["hit_mismatch"])),
                                "near_tie_seeds": rep["n_tie"], "param_bad": rep["param_bad"],
                                "cov_bad": rep["cov_bad"], "chi2_bad": rep["chi2_bad"],
                                "worst_param": rep["worst_param"], "worst_cov": rep["worst_cov"],
                                "worst_chi2": rep["worst_chi2"]},
            "fit_vs_oracle": _fit_errors(gf, r, np.arange(len(gf["chi2"])))}


def measure_config_uneven(batch, g, params, stream, local):
    """256 uneven events (~2.05M tracks) in one call: search shapes autotuned on the batch, then
    the one-call pass timed (CUDA events, mean of 5 after 2 warm-ups)."""
    import torch
    from paper_2312_11728_gb300 import pipeline
    fi = pipeline.fit_inputs(batch)
    ctx = pipeline.make_context(g, params, device=local, stream=stream)
    db = pipeline.DeviceBatch(batch, fi, g.max_plan, f"cuda:{local}")
    pipeline.run_step(ctx, db)
    torch.cuda.synchronize()
    steps = int(ctx.counters(0)[0] + ctx.counters(1)[0])
    f_s, s_s, tune_ms = ctx.autotune(reps=1)
    for _ in range(2):
        pipeline.run_step_fused(ctx, db)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    for _ in range(5):
        pipeline.run_step_fused(ctx, db)
    e[1].record(stream)
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / 5
    return {"value": steps / (ms / 1e3), "unit": UNIT, "ms_per_pass": ms, "kalman_steps": steps,
            "events": int(batch.n_events), "seeds": int(batch.seed_hits.shape[0]), "tracks": int(fi.layers.shape[0]),
            "search_launch": {"find_shape": f_s, "select_shape": s_s, "autotune_ms_per_search": tune_ms},
            "workload": "256 events, Poisson(8,000) tracks clipped to [200, 25,000], 2.5 noise hits per track, "
                        "one call (all events' seeds searched together)"}


def measure_config_loopers(batch, g, params, stream, local):
    """1,000,000 tracks over 34 layers, 10% at 0.5-0.7 GeV: the FP32 fit with the FP64 refit of
    the flagged tracks against the all-FP64 fit (CUDA events, mean of 3 after a warm-up), and
    both against the oracle on 1,000 sampled tracks."""
    import torch
    import oracle
    from paper_2312_11728_gb300 import pipeline
    fi = pipeline.fit_inputs(batch)
    n = fi.layers.shape[0]
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(n, 1000, replace=False))
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    t0 = time.perf_counter()
    r = oracle.Oracle(g, params).fit_batch(fi.layers[sample], fi.hits[sample], X, V,
                                           fi.p0[sample].astype(np.float64), fi.c0[sample].astype(np.float64))
    t_orc = time.perf_counter() - t0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(f"cuda:{local}")
    d = dict(layers=dev(fi.layers), hits=dev(fi.hits), p0=dev(fi.p0), c0=dev(fi.c0))
    res = {"tracks": int(n), "layers": int(g.n_layers), "steps": int((fi.layers >= 0).sum()),
           "oracle": {"value": int(r["counters"][0]) / t_orc, "unit": "fit track-layer steps/s", "cores": 1,
                      "sample": "the 1,000 compared tracks"},
           "workload": "50 events x 20,000 tracks over 34 layers, 10% at 0.5-0.7 GeV (curling), no noise"}
    for name, prec in (("fp32_fp64_refit", 0), ("fp64", 2)):
        ctx = pipeline.make_context(g, dict(params, precision=prec), device=local, stream=stream)
        ctx.load_hits(batch.n_events, batch.hit_off, dev(batch.hit_xyz), dev(batch.hit_cov))
        o = dict(p=torch.zeros((n, 6), device=f"cuda:{local}"), c=torch.zeros((n, 21), device=f"cuda:{local}"),
                 chi2=torch.zeros(n, device=f"cuda:{local}"),
                 status=torch.zeros(n, dtype=torch.int32, device=f"cuda:{local}"))
        call = lambda: ctx.fit(d["layers"], d["hits"], d["p0"], d["c0"], o["p"], o["c"], o["chi2"], o["status"])
        call()
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        for _ in range(3):
            call()
        e[1].record(stream)
        torch.cuda.synchronize()
        ms = e[0].elapsed_time(e[1]) / 3
        gf = {k: v.cpu().numpy() for k, v in o.items()}
        res[name] = {"ms": ms, "value": res["steps"] / (ms / 1e3), "unit": "fit track-layer steps/s",
                     "vs_oracle": _fit_errors(gf, r, sample)}
    res["fp32_over_fp64"] = res["fp64"]["ms"] / res["fp32_fp64_refit"]["ms"]
    return res


def measure_fit_grad(args, local, rank, dist, stream):
    """The fit's derivative on the differentiable-fit workload (100,000 tracks over 22 layers of
    a misaligned detector): one mkgb_fit_grad call after a warm-up call, CUDA-event timed."""
    import torch
    from paper_2312_11728_gb300 import pipeline, synth as S
    g, evs, _, _ = S.workload_aligned_fit(n_tracks=100_000, seed=rank)
    b = S.concat_events(evs, g.n_layers)
    fi = pipeline.fit_inputs(b, seed=rank)
    ctx = pipeline.make_context(g, S.default_params(), device=local, stream=stream)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(f"cuda:{local}")
    ctx.load_hits(b.n_events, b.hit_off, dev(b.hit_xyz), dev(b.hit_cov))
    n, L = fi.layers.shape[0], g.n_layers
    ins = dict(layers=dev(fi.layers), hits=dev(fi.hits), p0=dev(fi.p0), c0=dev(fi.c0),
               align=torch.zeros((L, 6), device=f"cuda:{local}"), xscale=torch.ones(L, device=f"cuda:{local}"))
    outs = dict(chi2=torch.zeros(n, device=f"cuda:{local}"), dp0=torch.zeros((n, 6), device=f"cuda:{local}"),
                dal=torch.zeros((L, 6), device=f"cuda:{local}"), dxs=torch.zeros(L, device=f"cuda:{local}"),
                status=torch.zeros(n, dtype=torch.int32, device=f"cuda:{local}"))
    call = lambda mode: ctx.fit_grad(ins["layers"], ins["hits"], ins["p0"], ins["c0"], ins["align"], ins["xscale"],
                                     outs["chi2"], outs["dp0"], outs["dal"], outs["dxs"], outs["status"], mode=mode)
    steps = int((fi.layers >= 0).sum())
    ms = {}
    for mode in (1, 0):   # forward mode, then the reverse sweep (the default)
        call(mode)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call(mode)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[mode] = e0.elapsed_time(e1)
    value, wall, _ = pipeline.replica_throughput(ms[0] / 1e3, steps, dist, f"cuda:{local}")
    return {"value": value, "unit": "fit track-layer steps/s with derivatives", "ms": wall * 1e3,
            "mode": "reverse sweep over checkpointed steps", "forward_mode_ms": ms[1], "tracks": n,
            "layers": int(np.unique(fi.layers[fi.layers >= 0]).size), "derivatives_per_track": "6 starting parameters + 7 per crossed layer",
            "workload": "100k tracks, 22 layers, misaligned detector (50 um, 0.1 mrad), material x[0.8, 1.2]"}


def spawn_replicas(n):
    """Re-runs this script as n ranks (one process per GPU, rendezvous on 127.0.0.1); rank 0
    prints the line.  Returns the launcher's exit status."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--events", type=int, default=N_EVENTS, help="events per batch (profiling of small cases)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 comparison path")
    ap.add_argument("--no-grad", action="store_true", help="skip the fit-derivative measurement")
    ap.add_argument("--no-modular", action="store_true", help="skip the modular-tracker measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (1,000-track barrel, 256 uneven events, 1M-track sweep)")
    ap.add_argument("--modular-events", type=int, default=16, help="events of the modular-tracker measurement")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes of the search kernels")
    ap.add_argument("--no-graph", action="store_true", help="launch the search rounds one by one")
    ap.add_argument("--shapes", default=None,
                    help="fixed launch shapes 'find,select' of the search kernels (no autotuning)")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # N replicas requested without a launcher: one process per GPU under torch.distributed.run
        sys.exit(spawn_replicas(args.gpus))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    from paper_2312_11728_gb300 import pipeline, synth as S
    g, batch, evs = make_batch(seed=rank, n_events=args.events)   # before the first CUDA call (spawn pool)
    mod = None if args.no_modular else make_modular_batch(rank, args.modular_events)
    cfg = None if args.no_configs else make_config_batches(rank)
    fit = pipeline.fit_inputs(batch, seed=rank)
    params = S.default_params()

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_11728_gb300 import mkgb

    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = pipeline.make_context(g, params, device=local, stream=stream)
    db = pipeline.DeviceBatch(batch, fit, g.max_plan, f"cuda:{local}")
    n_seeds = batch.seed_hits.shape[0]
    n_tracks = fit.layers.shape[0]

    def step(ev=None):
        ctx.load_hits(db.n_events, db.seg_off, db.xyz, db.cov)
        if ev: ev[0].record(stream)
        ctx.seed(db.seeds)
        if ev: ev[1].record(stream)
        ctx.build(db.out)
        if ev: ev[2].record(stream)
        f = db.fit
        ctx.fit(f["layers"], f["hits"], f["p0"], f["c0"], f["p"], f["c"], f["chi2"], f["status"])

    # warm-up with the separate calls (their counters give the work of one pass), then with the
    # one-call pass that the timed steps use
    if args.shapes:   # fixed shapes from the first pass on (profiling runs)
        ctx.set_launch(*(int(x) for x in args.shapes.split(",")), use_graph=not args.no_graph)
    step()
    torch.cuda.synchronize()
    bc = ctx.counters(0)
    fc = ctx.counters(1)
    kalman_steps = int(bc[0] + fc[0])
    shapes = (0, 0, None)
    if args.shapes:
        f_s, s_s = (int(x) for x in args.shapes.split(","))
        shapes = (f_s, s_s, None)
    elif not args.no_autotune:
        shapes = ctx.autotune(reps=2)   # block shapes of the search kernels on this batch
    ctx.set_launch(shapes[0], shapes[1], use_graph=not args.no_graph)
    for _ in range(max(0, args.warmup - 1)):
        pipeline.run_step_fused(ctx, db)
    torch.cuda.synchronize()

    # timed: K passes through mkgb_run (load hits, seed, search, fit in one call)
    ev_step = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            e = ev_step[k]
            e[0].record(stream)
            pipeline.run_step_fused(ctx, db)
            e[1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [e[0].elapsed_time(e[1]) for e in ev_step]
    total_ms = sum(step_ms)

    # stage times from passes through the separate calls (no overlap between stages)
    n_stage = max(1, min(args.steps, 3))
    ev_st = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(n_stage)]
    for e in ev_st:
        e[3].record(stream)
        step(e)
        e[4].record(stream)
    torch.cuda.synchronize()
    build_ms = [e[1].elapsed_time(e[2]) for e in ev_st]
    stage = {"bin_hits": np.mean([e[3].elapsed_time(e[0]) for e in ev_st]),
             "seed": np.mean([e[0].elapsed_time(e[1]) for e in ev_st]),
             "build": np.mean(build_ms),
             "fit": np.mean([e[2].elapsed_time(e[4]) for e in ev_st]),
             "separate_calls_total": np.mean([e[3].elapsed_time(e[4]) for e in ev_st])}
    value, wall, _ = pipeline.replica_throughput(total_ms / 1e3, kalman_steps * args.steps, dist, f"cuda:{local}")

    # ---- the plain all-FP64 path on the same events (the comparison factor)
    fp64 = None
    if not args.no_fp64:
        fp64 = measure_fp64_plain(args, g, params, evs, stream, local, rank, dist)
        fp64["factor"] = value / fp64["value"]

    # the seed fits redone in FP64: the seeds whose mixed-precision fit gives |q/pT| below 0.03
    s_state = torch.zeros((n_seeds, 6), dtype=torch.float32, device=f"cuda:{local}")
    s_cov = torch.zeros((n_seeds, 21), dtype=torch.float32, device=f"cuda:{local}")
    s_info = torch.zeros((n_seeds, 3), dtype=torch.int32, device=f"cuda:{local}")
    ctx.seed(db.seeds, s_state, s_cov, s_info)
    torch.cuda.synchronize()
    ok_seed = s_info[:, 2] == 0
    seed_precision = {
        "mode": "FP32 trajectory and Jacobian, FP64 covariance transport and update; the seeds with "
                "|q/pT| < 0.03 /GeV fitted again entirely in FP64",
        "fp64_redo_fraction": float(((s_state[:, 3].abs() < 0.03) & ok_seed).sum().item() / max(1, n_seeds))}
    del s_state, s_cov, s_info

    bkfit = measure_fit_backward(ctx, db, fit, stream, dist, local)
    cleaning = measure_cleaning(ctx, db, g, stream, local)
    modular = None if mod is None else measure_modular(mod, params, shapes, stream, local, dist)

    grad = None
    if not args.no_grad:
        grad = measure_fit_grad(args, local, rank, dist, stream)

    configs = None
    if cfg is not None:
        cg, uneven, loopers = cfg
        configs = {"small_barrel_1k": measure_config_small(params, stream, local),
                   "uneven_256ev": measure_config_uneven(uneven, cg, params, stream, local),
                   "loopers_1m": measure_config_loopers(loopers, cg, params, stream, local)}

    # ---- end to end through the C ABI with host (pinned) buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, ctx, db, batch, fit, g, stream, kalman_steps, world, local, dist)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    probe = {"fp32_tflops": ctx.probe_peak(0), "fp64_tflops": ctx.probe_peak(1)}
    hbm, sm_max, src = peaks()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = n_sms * 128 * 2 * sm_max * 1e6 / 1e12        # TFLOP/s at the maximum SM clock
    # DRAM bytes of the search kernels per crossed candidate-layer step, from an ncu capture of
    # the same sources (null if the kernels changed since)
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "search_traffic.json")
    if os.path.exists(tr_path) and shapes[0] < 3:   # captured on the two-kernel round
        tr = json.load(open(tr_path))
        if tr.get("sources_sha256_16") == kernel_sources_hash():
            traffic = tr["dram_bytes_per_crossed_step"] * int(bc[0])
    bins_total = batch.n_events * int((g.n_eta.astype(np.int64) * g.n_phi).sum())
    n_hits = int(batch.hit_xyz.shape[0])
    rf_search = roofline("search", stage["build"], build_flops(bc),
                         search_bytes(bc, n_hits, bins_total, n_seeds, g.max_plan), fp32_peak, hbm, traffic)
    rf_search.update({
        "kernel": ("search: k_start, one fused k_round per plan step (k_rescue after it when flagged), k_finish"
                   if shapes[0] >= 3 else
                   "search: k_start, per plan step k_find and k_select (k_rescue after them when flagged), k_finish"),
        "peak_note": f"HBM {hbm:.1f} GB/s ({src} copy bandwidth); FP32 {n_sms} SMs x 128 lanes x 2 x {sm_max:.0f} MHz "
                     f"({src} max clock) = {fp32_peak:.1f} TFLOP/s; FMA probe {probe['fp32_tflops']:.1f} TFLOP/s",
        "launch": "algorithmic bytes and flops of one whole search over its CUDA-event time on the context's "
                  "stream (all its launches, one mkgb_build call, its rounds replayed as a CUDA graph)"})
    rf_fit = roofline("fit", stage["fit"], fit_flops(fc), fit_bytes(fc, n_tracks), fp32_peak, hbm)
    rf_seed = roofline("seed", stage["seed"], FLOPS["seed_fp32"] * n_seeds, ALG_BYTES["seed"] * n_seeds, fp32_peak,
                       hbm, fp64_flops=FLOPS["seed_fp64"] * n_seeds, fp64_peak=probe["fp64_tflops"])
    keys_total = batch.n_events * 32 * 64
    # hits: prep, scatter, scans; seeds: fit, key, scans, scatter; search: start, per plan step of
    # the longest plan the fused round (or find and select) and the FP64 redo, finish; fit: FP32
    # fit and FP64 refit
    redo = 1 if params["kappa_fp64"] > 0 else 0
    per_round = (1 if shapes[0] >= 3 else 2) + redo
    launches_per_step = ((2 + scan_launches(bins_total)) + (2 + scan_launches(keys_total)) + 2
                         + per_round * g.max_plan + 1 + redo)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(events=batch.n_events), "events": batch.n_events, "tracks_per_event": N_TRACKS,
                   "noise_hits_per_event": N_NOISE, "layers": g.n_layers, "best_n": params["max_cands"],
                   "seeds": int(n_seeds), "fit_tracks": int(n_tracks), "hits": int(batch.hit_xyz.shape[0]),
                   "kalman_steps_per_step": kalman_steps, "build_steps": int(bc[0]), "fit_steps": int(fc[0]),
                   "l2": f"inputs larger than L2: {batch.hit_xyz.shape[0] * 92 / 1e9:.2f} GB of hit data resident",
                   "parallelism": f"replicas{world}",
                   "search_launch": {"find_shape": shapes[0], "select_shape": shapes[1],
                                     "autotune_ms_per_search": shapes[2], "cuda_graph": not args.no_graph}},
        "step_ms_spread": {"median": float(np.median(step_ms)), "min": float(np.min(step_ms)),
                           "max": float(np.max(step_ms))},
        "stages_ms": {k: round(float(v), 4) for k, v in stage.items()},
        "roofline": rf_search,
        "roofline_stages": {"seed": rf_seed, "search": {k: rf_search[k] for k in rf_search
                                                        if k not in ("peak_note", "launch", "kernel")},
                            "fit": rf_fit},
        "e2e": e2e,
        "fp64_plain": fp64,
        "seed_precision": seed_precision,
        "fit_grad": grad,
        "configs": configs,
        "fit_backward": bkfit,
        "cleaning": cleaning,
        "modular": modular,
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clocks,
        "counters": {"build": [int(x) for x in bc], "fit": [int(x) for x in fc]},
        # rank 0's timed passes counted in chi2 evaluations and Kalman updates (search + fit)
        "rates_per_gpu": {"chi2_per_s": (int(bc[1]) + int(fc[1])) * args.steps / wall,
                          "updates_per_s": (int(bc[2]) + int(fc[2])) * args.steps / wall},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, batch, fit, params)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(g, evs, params)
    print(json.dumps(line, default=lambda o: o.item() if hasattr(o, "item") else str(o)), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
