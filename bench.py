"""Benchmark of the AMH hot path on GB300.

One step = one Alternating-MH cycle on every chain (10 local sweeps with
window d = 8, then 1 global sweep; Alg. 1) along the annealing schedule of
the L=300, 1024-chain workload (T 2.0 -> 0.05 geometric and sigma 10 -> 4 deg
over 200k proposals per chain), followed by one gradient evaluation dV/ds
of every chain's state (the hand-off to L-BFGS).  Metric: MH proposals per
second over all ranks (weak scaling: each rank owns its own 1024 chains).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on this host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "amh_L300_c1024"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
# FP32 lanes per SM on this part (4 sub-partitions x 32) for the ALU peak
FP32_LANES_PER_SM = 128
# algorithmic FP32 operations of one pair-term evaluation e(|x_a - x_b|):
# 3 sub + 3 mul + 2 add (squared distance), 1 sqrt, 1 sub + 1 mul (bin
# coordinate), 1 sub (fraction), 1 sub + 1 mul + 1 add (interpolation),
# 1 add (accumulate) = 16
FLOP_PER_EVAL = 16
# a term whose distance is formed and found flat (at or past the last bin
# centre in every configuration of its pair, so its entry is not read):
# the squared distance (8), the square root (1) and the bin coordinate (2)
FLOP_PER_FLAT = 11
# DRAM bytes (read + write) of one launch of the global-sweep kernel, from one
# ncu capture (profiles/global_kernel_L300_c1024.md).  Reported only while
# the kernel's sources and launch shape are the ones that were captured.
# DRAM bytes of one global-sweep launch from an ncu capture, per launch shape
# (chains per CTA, threads, staging depth); valid while the kernel's sources
# hash to sources_sha1.
TRAFFIC_CAPTURE = {"sources_sha1": "fa2144c882abdad66e82690a41ef463e56cf9cdf",
                   "sources": ["paper_2211_03193_gb300/csrc/amh_global.cu",
                               "paper_2211_03193_gb300/csrc/amh_device.cuh",
                               "paper_2211_03193_gb300/csrc/amh_internal.h"],
                   "workload": "amh_L300_c1024",
                   "bytes": {(1, 1, 128, 0): 16891136}}


def captured_traffic(workload_name, shape):
    import hashlib
    cap = TRAFFIC_CAPTURE
    if workload_name != cap["workload"] or tuple(shape) not in cap["bytes"]:
        return None
    h = hashlib.sha1()
    for f in cap["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return cap["bytes"][tuple(shape)] if h.hexdigest() == cap["sources_sha1"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--far-pairs", type=int, default=0, choices=[0, 1],
                    help="1: evaluate every straddle pair (no far-field skipping)")
    ap.add_argument("--no-overlap", dest="overlap", action="store_false",
                    help="run the gradient pass after the global sweep instead of beside it")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-target measurement")
    ap.add_argument("--experiment", default="", choices=["", "schemes", "forms", "batched", "grad"],
                    help="schemes: AMH vs plain MH vs MH with noisy restarts (L=150); forms: "
                         "batched FP32 vs one-chain FP64 (L=300); batched: 64 uneven proteins")
    ap.add_argument("--chains-per-cta", type=int, default=0,
                    help="global-sweep chains per CTA (0 = autotuned)")
    ap.add_argument("--threads", type=int, default=0, help="global-sweep threads per CTA")
    ap.add_argument("--texture", type=int, default=0,
                    help="table entries: 0 default (texture when it fits), 1 texture, 2 loads")
    ap.add_argument("--local-chains-per-cta", type=int, default=0,
                    help="local-sweep chains per CTA (0 = chosen from the window)")
    ap.add_argument("--local-threads", type=int, default=0, help="local-sweep threads per CTA")
    ap.add_argument("--stage", type=int, default=0,
                    help="table rows: 0 tuned, 1 staged in shared memory, 2 through L1")
    ap.add_argument("--global-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="global sweeps: 0 tuned, 1 chains of a CTA in lock-step, "
                         "2 one warp per chain")
    ap.add_argument("--warps-per-chain", type=int, default=0, choices=[0, 1, 2, 4],
                    help="chain-group kernel: warps per chain (0 = tuned)")
    ap.add_argument("--per-sweep-calls", action="store_true",
                    help="one library call per local sweep instead of one per run of them")
    ap.add_argument("--clocks-csv", default="",
                    help="keep the nvidia-smi clock samples of the timed region in this file "
                         "(default: a temporary file, removed after it is summarised)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(name):
    from paper_2211_03193_gb300 import synth
    w = dict(synth.WORKLOADS[name])
    L = w["L"]
    n = 2 * L
    w["n"] = n
    w["total_sweeps"] = w["proposals"] // n
    w["cycle"] = w["n_local"] + w["n_global"]
    return w


def schedule_for(w, seed):
    from paper_2211_03193_gb300.sampler import Schedule
    s0, s1 = w["sigma_deg"] if isinstance(w["sigma_deg"], tuple) else (w["sigma_deg"],) * 2
    return Schedule(total_sweeps=w["total_sweeps"], n_local=w["n_local"], n_global=w["n_global"],
                    window=w["window"], T0=w["T0"], T1=w["T1"], sigma0_deg=s0, sigma1_deg=s1,
                    seed=seed)


def pair_evals_per_cycle(w):
    """Pair-term evaluations one chain performs in one cycle."""
    L, n, h = w["L"], w["n"], w["window"] // 2
    glob = 2 * (L ** 3 - L) // 3          # old + new of every straddle pair
    resync = L * (L - 1) // 2             # the exit energy (the entry rebuild forms coordinates only)
    loc = 0
    for k in range(n):
        c, p = k // 2, (k + 1) // 2
        lo, hi = max(0, c - h), min(L - 1, c + h)
        if lo < p <= hi:
            loc += 2 * (p - lo) * (hi - p + 1)
    return w["n_global"] * (glob + resync), w["n_local"] * loc


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        self.keep = bool(path)
        if path:
            self.path = path
        else:
            fd, self.path = tempfile.mkstemp(prefix="amh_clocks_", suffix=".csv")
            os.close(fd)

    def __enter__(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        finally:
            if not self.keep:
                try:
                    os.unlink(self.path)
                except OSError:
                    pass
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(w, seed, budget_s=12.0):
    """The FP64 oracle on this host's cores, on a bounded sample of the
    workload: cycles of the same schedule on as many chains as there are
    cores (OpenMP over chains)."""
    import oracle
    from paper_2211_03193_gb300 import synth
    oracle.build()
    prot = synth.make_protein(w["L"], edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    P = oracle.Problem(prot.L, prot.p, prot.edges)
    cores = oracle.num_threads()
    S = synth.random_torsions(cores, w["L"], seed=w["start_seed"]).astype(np.float64)
    sched = schedule_for(w, seed)
    n = w["n"]
    props = 0
    t0 = time.perf_counter()
    s = 0
    while True:
        mode, T, sigma = sched.params(s)
        S, _ = P.run_chains(S, mode, w["window"], T, sigma, s * n, n, seed, 0)
        props += cores * n
        s += 1
        if time.perf_counter() - t0 > budget_s and s % w["cycle"] == 0:
            break
    dt = time.perf_counter() - t0
    # one core: one chain through one cycle of the same schedule
    s1 = S[0].copy()
    t1 = time.perf_counter()
    for q in range(w["cycle"]):
        mode, T, sigma = sched.params(q)
        s1, _, _ = P.run(s1, mode, w["window"], T, sigma, q * n, n, seed, 0)
    dt1 = time.perf_counter() - t1
    return {"value": props / dt, "unit": "proposals/s", "cores": cores, "kind": "oracle",
            "sample": "%d chains x %d sweeps (%d cycles of %d local + %d global, L=%d) of the "
                      "same schedule, FP64, OpenMP over chains" % (
                          cores, s, s // w["cycle"], w["n_local"], w["n_global"], w["L"]),
            "seconds": dt, "single_core_value": w["cycle"] * n / dt1,
            "single_core_sample": "1 chain x 1 cycle (%d sweeps)" % w["cycle"]}


def measured_peaks():
    """FP32 FMA, MUFU square-root and L2 read rates of this GPU, from the
    microbenchmarks in libamh_peaks.so (or None if it cannot run)."""
    import ctypes
    from paper_2211_03193_gb300 import build
    try:
        lib = ctypes.CDLL(build.PEAKS_LIB)
        f, m, l2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        if lib.amh_measure_peaks(ctypes.byref(f), ctypes.byref(m), ctypes.byref(l2)) != 0:
            return None
    except OSError:
        return None
    return {"fp32_tflops": 2 * f.value / 1e12, "mufu_sqrt_per_s": m.value,
            "l2_read_gbs": l2.value / 1e9,
            "how": "libamh_peaks.so: 8 independent FFMA (or sqrt.approx) chains per thread, "
                   "2048 threads per SM; 16-byte L1-bypassing loads over half the L2"}


def time_to_target():
    """Time to a low-energy structure, after the protocol of Sec. 3 / Fig. 4E,
    over the whole anneal: the CPU (the FP64 oracle, one chain per core, 10
    seeds) runs the full L=150 schedule (2e5 proposals per chain, 10 local :
    1 global, T 2.0 -> 0.05, sigma 10 -> 4 deg); the target E* is the mean
    over the 10 runs of the lowest energy each reached (at global-sweep
    ends).  The GPU then runs 1024 chains of the same schedule until the
    lowest energy over its chains reaches E*.  The target lies at the end of
    the anneal, so the GPU has to anneal towards it (a target taken from a
    short CPU run is met by the spread of 1024 chains at high temperature).
    Returns both wall times and the sweep at which the GPU got there."""
    import torch
    import oracle
    from paper_2211_03193_gb300 import _amh, synth
    from paper_2211_03193_gb300.sampler import Sampler
    w = workload("amh_L150_c1024")
    L, n = w["L"], w["n"]
    total = w["total_sweeps"]
    sched = schedule_for(w, seed=2)
    prot = synth.make_protein(L, edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    P = oracle.Problem(L, prot.p, prot.edges)
    runs = 10
    S = synth.random_torsions(runs, L, seed=w["start_seed"]).astype(np.float64)
    best = np.full(runs, np.inf)
    t0 = time.perf_counter()
    for s in range(total):
        mode, T, sigma = sched.params(s)
        S, _ = P.run_chains(S, mode, w["window"], T, sigma, s * n, n, sched.seed, 0)
        if mode == _amh.AMH_GLOBAL:
            best = np.minimum(best, P.energies(S))
    cpu_s = time.perf_counter() - t0
    target = float(np.mean(best))
    chains = w["chains"]
    stream = torch.cuda.Stream()
    tors = synth.random_torsions(chains, L, seed=w["start_seed"])
    samp = Sampler(prot, chains, tors, stream=stream)
    bE = torch.empty(chains, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reached, s, s_best = False, 0, None
    gpu_s, med_s, s_med = None, None, None
    with torch.cuda.stream(stream):
        for s in range(total):
            mode, T, sigma = sched.params(s)
            _amh.amh_sweeps(samp.ctx, mode, w["window"], T, sigma, 1, sched.seed, None)
            if mode == _amh.AMH_GLOBAL:
                _amh.amh_get_state(samp.ctx, None, None, bE, None)
                now = time.perf_counter() - t0
                if not reached and float(bE.min()) <= target:
                    reached, gpu_s, s_best = True, now, s
                # the median chain: a per-chain measure of the anneal's progress
                if med_s is None and float(bE.median()) <= target:
                    med_s, s_med = now, s
                if reached and med_s is not None:
                    break
    if gpu_s is None:
        gpu_s = time.perf_counter() - t0
    final_best = float(bE.min())
    final_median = float(bE.median())
    samp.close()
    return {"protein": "L=150, 37 bins (amh_L150_c1024 schedule, %d sweeps = 2e5 proposals "
                       "per chain)" % total,
            "target_energy": target, "cpu_runs": runs, "cpu_seconds": cpu_s,
            "cpu_proposals_per_run": total * n, "cpu_best_per_run": [float(v) for v in best],
            "gpu_chains": chains, "gpu_seconds": gpu_s,
            "gpu_sweeps": (s_best + 1) if s_best is not None else total,
            "gpu_sweeps_total": total, "gpu_best_at_end": final_best,
            "reached": reached, "speedup": cpu_s / gpu_s if reached else None,
            "median_chain_seconds": med_s,
            "median_chain_sweeps": (s_med + 1) if s_med is not None else None,
            "median_chain_best_at_end": final_median,
            "median_chain_speedup": cpu_s / med_s if med_s else None,
            "note": "CPU: FP64 oracle, one chain per core, wall time of the 10 parallel runs; "
                    "GPU: wall time from the first sweep until the best of its chains (the "
                    "paper's measure) and until its median chain reach the CPU runs' mean "
                    "lowest energy, checked after every global sweep.  The best of 1024 "
                    "chains reaches it early, in the spread of the chains at high T; the "
                    "median chain has to anneal towards it"}


def run_schemes():
    """The L=150 workload's comparison (Sec. 3, Fig. 3A protocol on synthetic
    data): 1024 chains, 200k proposals each, T 2.0 -> 0.05, sigma 10 -> 4 deg;
    AMH (10 local d=8 : 1 global), plain MH (global only) and MH with noisy
    restarts (N(0, 30 deg) kicks every 20k proposals).  Prints one JSON line
    per scheme with the chains' best energies."""
    import torch
    from paper_2211_03193_gb300 import synth
    from paper_2211_03193_gb300.sampler import Sampler, Schedule, run_schedule
    w = workload("amh_L150_c1024")
    L, n, chains = w["L"], w["n"], w["chains"]
    prot = synth.make_protein(L, edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    tors = synth.random_torsions(chains, L, seed=w["start_seed"])
    total = w["proposals"] // n
    schemes = {
        "amh": dict(n_local=10, n_global=1, noisy_every=0),
        "amh_80g_20l_d5": dict(n_local=20, n_global=80, noisy_every=0, window=5),
        "mh": dict(n_local=0, n_global=1, noisy_every=0),
        "mh_noisy_restarts": dict(n_local=0, n_global=1, noisy_every=max(1, 20000 // n)),
    }
    for name, kw in schemes.items():
        kw = dict(kw)
        win = kw.pop("window", w["window"])
        sched = Schedule(total_sweeps=total, window=win, T0=w["T0"], T1=w["T1"],
                         sigma0_deg=10.0, sigma1_deg=4.0, seed=3, noisy_sd_deg=30.0, **kw)
        stream = torch.cuda.Stream()
        with Sampler(prot, chains, tors, stream=stream) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                run_schedule(s, sched)
            E = s.energy()
            bE = s.state()[2]
            dt = time.perf_counter() - t0
        print(json.dumps({"experiment": "schemes", "scheme": name, "L": L, "chains": chains,
                          "proposals_per_chain": total * n, "seconds": dt,
                          "best_of_chains": float(bE.min()),
                          "median_chain_best": float(np.median(bE)),
                          "median_final_energy": float(np.median(E))}))


def run_forms(name=WORKLOAD):
    """The batched FP32 form against the plain FP64 form (one chain per
    launch) on the same GPU: proposals/s of one AMH cycle of the workload's
    schedule, and the batched FP32 form's end energies against the FP64
    form's energies (FP64 G(s), FP64 terms) of the same states."""
    import torch
    from paper_2211_03193_gb300 import _amh, synth
    from paper_2211_03193_gb300.sampler import Sampler
    w = workload(name)
    L, n, nch = w["L"], w["n"], w["chains"]
    prot = synth.make_protein(L, edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    sched = schedule_for(w, seed=1)
    ends = {}
    for label, chains, prec in (("fp32_batched_%d" % nch, nch, 32), ("fp32_one_chain", 1, 32),
                                ("fp64_one_chain", 1, 64)):
        tors = synth.random_torsions(chains, L, seed=w["start_seed"])
        stream = torch.cuda.Stream()
        with Sampler(prot, chains, tors, precision=prec, stream=stream) as s:
            def cycle():
                for q in range(w["cycle"]):
                    mode, T, sigma = sched.params(q)
                    _amh.amh_sweeps(s.ctx, mode, w["window"], T, sigma, 1, 1, None)
            with torch.cuda.stream(stream):
                cycle()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                cycle()
                e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if chains == nch:
                ends[prec] = s.state()[:2]
        print(json.dumps({"experiment": "forms", "workload": name, "form": label, "L": L,
                          "chains": chains, "precision": prec, "ms_per_cycle": ms,
                          "proposals_per_s": w["cycle"] * n * chains / (ms / 1000.0)}))
    # the FP32 form's energies against the FP64 form's energies of the same states
    th32, E32 = ends[32]
    with Sampler(prot, nch, th32, precision=64) as s64:
        E64 = s64.energy()
    rel = np.abs(E32 - E64) / np.abs(E64)
    print(json.dumps({"experiment": "forms", "workload": name,
                      "fp32_vs_fp64_energy_rel_max": float(rel.max()),
                      "fp32_vs_fp64_energy_rel_median": float(np.median(rel))}))


def run_batched():
    """64 proteins with L uniform in [50, 400], 256 chains each, one context:
    one AMH cycle (10 local + 1 global sweep per chain) through the persistent
    work queue, issued eagerly (one library call per sweep) and replayed from
    a CUDA graph captured from the same calls; proposals/s over all chains."""
    import torch
    from paper_2211_03193_gb300 import _amh, synth
    from paper_2211_03193_gb300.sampler import Sampler, Schedule, capture_schedule
    w = dict(synth.WORKLOADS["amh_batched_64prot"])
    Ls = synth.uneven_lengths(w["nproteins"], w["Lmin"], w["Lmax"], seed=3)
    prots = [synth.make_protein(L, seed=w["seed"] + i) for i, L in enumerate(Ls)]
    chains = [w["chains"]] * len(Ls)
    tors = np.concatenate([synth.random_torsions(w["chains"], L, seed=w["start_seed"] + i).ravel()
                           for i, L in enumerate(Ls)])
    # one cycle at fixed T and sigma, repeated (the schedule's cycle length)
    sched = Schedule(total_sweeps=11, n_local=10, n_global=1, window=w["window"], T0=1.0, T1=1.0,
                     sigma0_deg=10.0, sigma1_deg=10.0, seed=1)
    props = sum(11 * 2 * L * w["chains"] for L in Ls)
    out = {"experiment": "batched", "proteins": len(Ls), "chains": sum(chains),
           "L_range": [min(Ls), max(Ls)], "proposals_per_cycle": props}
    reps = 5
    stream = torch.cuda.Stream()
    with Sampler(prots, chains, tors, resync_every=w["resync_every"], stream=stream) as s:
        def cycle():
            for q in range(11):
                mode, T, sigma = sched.params(q)
                _amh.amh_sweeps(s.ctx, mode, w["window"], T, sigma, 1, 1, None)
        with torch.cuda.stream(stream):
            cycle()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                cycle()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        C, thr, D, K = s.launch_config()
        out.update({"eager_ms_per_cycle": ms, "eager_proposals_per_s": props / (ms / 1000.0),
                    "chains_per_cta": C, "threads_per_cta": thr, "global_kernel": K})
    gstream = torch.cuda.Stream()
    with Sampler(prots, chains, tors, resync_every=w["resync_every"], stream=gstream) as s:
        g = capture_schedule(s, sched, 0, 11, gstream)
        g.replay()  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(gstream):
            e0.record(gstream)
            for _ in range(reps):
                g.replay()
            e1.record(gstream)
        torch.cuda.synchronize()
        ms_g = e0.elapsed_time(e1) / reps
        assert s.counter(0) == (reps + 1) * 11 * 2 * Ls[0]
        out.update({"graph_ms_per_cycle": ms_g, "graph_proposals_per_s": props / (ms_g / 1000.0),
                    "launches_per_cycle": 11})
    print(json.dumps(out))


def run_grad():
    """L=300, 512 torsion vectors: one amh_grad call (energy and dV/ds of all
    512) timed with CUDA events, then AMH (one cycle on 256 chains) and torch
    L-BFGS (500 iterations) on the best 32 states, wall-timed."""
    import torch
    from paper_2211_03193_gb300 import autograd, synth
    from paper_2211_03193_gb300.sampler import Sampler
    w = synth.WORKLOADS["grad_L300_b512"]
    L, batch = w["L"], w["batch"]
    n = 2 * L
    prot = synth.make_protein(L, edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    tors = synth.random_torsions(batch, L, seed=w["start_seed"])
    stream = torch.cuda.Stream()
    with Sampler(prot, 1, tors[:1], stream=stream) as s:
        th = torch.tensor(tors, device="cuda")
        E = torch.empty(batch, dtype=torch.float64, device="cuda")
        G = torch.empty((batch, n), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for _ in range(3):
            s.grad(0, th, E, G)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                s.grad(0, th, E, G)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        # the L-BFGS hand-off's call: 32 vectors, one call at a time
        th32 = th[:32].contiguous()
        E32 = torch.empty(32, dtype=torch.float64, device="cuda")
        G32 = torch.empty((32, n), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        t32 = time.perf_counter()
        for _ in range(50):
            s.grad(0, th32, E32, G32)
            torch.cuda.synchronize()
        ms32 = (time.perf_counter() - t32) / 50 * 1000.0
    chains = 256
    starts = synth.random_torsions(chains, L, seed=w["start_seed"] + 1)
    with Sampler(prot, chains, starts) as s:
        t0 = time.perf_counter()
        for q in range(11):
            s.sweeps(0 if q < 10 else 1, 8, 1.0, math.radians(10.0), 1, 3)
        th_all, E0, _, _ = s.state()
        best = np.argsort(E0)[:32]
        # torch loads its elementwise kernels on first use (seconds on a fresh
        # box): a short L-BFGS run first, outside the timed one
        autograd.lbfgs_refine(s, torch.tensor(th_all.reshape(chains, n)[best], device="cuda"),
                              iterations=3)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        calls = [0]
        plain_grad = s.grad

        def counted(*a, **k):
            calls[0] += 1
            return plain_grad(*a, **k)
        s.grad = counted
        thL, EL = autograd.lbfgs_refine(s, torch.tensor(th_all.reshape(chains, n)[best],
                                                        device="cuda"), iterations=500)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        EL = EL.cpu().numpy()
    print(json.dumps({"experiment": "grad", "L": L, "batch": batch, "ms_per_call": ms,
                      "ms_per_call_32_synchronised": ms32,
                      "vectors_per_s": batch / (ms / 1000.0),
                      "pair_gradients_per_s": batch * L * (L - 1) / (ms / 1000.0),
                      "amh_seconds": t1 - t0, "lbfgs_seconds": t2 - t1,
                      "lbfgs_gradient_calls": calls[0],
                      "best32_energy_before": [float(E0[best].min()), float(E0[best].max())],
                      "best32_energy_after": [float(EL.min()), float(EL.max())]}))


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    w = workload(args.workload)
    n = w["n"]
    # each step is a bounded sample: one cycle on `cores` chains
    import oracle
    from paper_2211_03193_gb300 import synth
    oracle.build()
    prot = synth.make_protein(w["L"], edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    P = oracle.Problem(prot.L, prot.p, prot.edges)
    cores = oracle.num_threads()
    S = synth.random_torsions(cores, w["L"], seed=w["start_seed"]).astype(np.float64)
    sched = schedule_for(w, 1)
    s = 0

    def one_step():
        nonlocal S, s
        for _ in range(w["cycle"]):
            mode, T, sigma = sched.params(s)
            S, _ = P.run_chains(S, mode, w["window"], T, sigma, s * n, n, 1, 0)
            s += 1

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = time.perf_counter() - t0
    props = args.steps * w["cycle"] * n * cores
    val = props / dt
    out = {"metric": "MH proposals/s", "value": val, "unit": "proposals/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload + " (oracle sample: %d chains per step)" % cores,
                      "L": w["L"], "chains_per_step": cores, "schedule": "10 local (d=8) : 1 global"},
           "cpu_baseline": {"value": val, "unit": "proposals/s", "cores": cores, "kind": "oracle",
                            "sample": "%d chains x 1 cycle per step" % cores},
           "e2e": {"value": val, "unit": "proposals/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2211_03193_gb300 import build as b
    b.build()
    from paper_2211_03193_gb300 import _amh, synth
    from paper_2211_03193_gb300.sampler import Sampler

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = workload(args.workload)
    L, n, chains = w["L"], w["n"], w["chains"]
    prot = synth.make_protein(L, edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    tors = synth.random_torsions(chains, L, seed=w["start_seed"] + 1000 * rank)
    # the sweeps run on a high-priority stream; the gradient pass on a second
    # one, so its CTAs take the SMs the global sweep leaves idle
    stream = torch.cuda.Stream(priority=-1)
    aux = torch.cuda.Stream(priority=0)
    samp = Sampler(prot, chains, tors, precision=w["precision"], stream=stream,
                   chains_per_cta=args.chains_per_cta, threads_per_cta=args.threads,
                   stage_table=args.stage, table_texture=args.texture, far_pairs=args.far_pairs,
                   local_chains_per_cta=args.local_chains_per_cta, local_threads=args.local_threads,
                   global_kernel=args.global_kernel, warps_per_chain=args.warps_per_chain)
    # a context for the gradient pass only (fixed launch shape: no autotuning)
    gsamp = Sampler(prot, 1, tors[:1], precision=w["precision"], stream=aux, chains_per_cta=1,
                    threads_per_cta=128)
    C, thr, D, K = samp.launch_config()
    # device table: one 8-byte entry per bin, rows padded to an even bin count
    B = len(synth.edges_by_name(w["bins"])) - 1
    tab_mb = (L * (L - 1) // 2) * ((B + 1) & ~1) * (8 if w["precision"] == 32 else 16) / 1e6
    sched = schedule_for(w, seed=1 + rank)
    cyc = w["cycle"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    theta_dev = torch.empty((chains, n), dtype=torch.float32, device="cuda")
    E_dev = torch.empty(chains, dtype=torch.float64, device="cuda")
    G_dev = torch.empty((chains, n), dtype=torch.float32, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)
    sweep_idx = [0]
    launches = [0]  # library kernel launches (sweep calls and gradient passes)

    def grad_pass():
        _amh.amh_grad(gsamp.ctx, 0, theta_dev, chains, E_dev, G_dev)

    def cycle(glob_events=None):
        """10 local sweeps and the global sweep on every chain, and the
        L-BFGS hand-off: dV/ds of every chain's state.  With --overlap (the
        default) the gradient pass covers the states that ended the previous
        cycle and runs on the second stream beside the global sweep; the
        cycle ends when both are done, and then snapshots its end states."""
        j = 0
        while j < cyc:
            s = sweep_idx[0] % w["total_sweeps"]
            mode, T, sigma = sched.params(s)
            if mode == _amh.AMH_LOCAL and not args.per_sweep_calls:
                # the run of local sweeps up to the global one: one library call,
                # each sweep at its own T and sigma
                Ts, Ss = [], []
                while j < cyc and len(Ts) < _amh.AMH_MAX_SCHED:
                    s = sweep_idx[0] % w["total_sweeps"]
                    m2, T2, sg2 = sched.params(s)
                    if m2 != _amh.AMH_LOCAL or (Ts and s == 0):
                        break
                    Ts.append(T2)
                    Ss.append(sg2)
                    sweep_idx[0] += 1
                    j += 1
                _amh.amh_sweeps_sched(samp.ctx, mode, w["window"], Ts, Ss, sched.seed, None)
                launches[0] += 1
                continue
            launches[0] += 1
            if mode == _amh.AMH_GLOBAL and args.overlap:
                go = torch.cuda.Event()
                go.record(stream)
                aux.wait_event(go)
                grad_pass()
                done = torch.cuda.Event()
                done.record(aux)
            if mode == _amh.AMH_GLOBAL and glob_events is not None:
                e0, e1 = ev(), ev()
                e0.record(stream)
                _amh.amh_sweeps(samp.ctx, mode, w["window"], T, sigma, 1, sched.seed, None)
                e1.record(stream)
                glob_events.append((e0, e1))
            else:
                _amh.amh_sweeps(samp.ctx, mode, w["window"], T, sigma, 1, sched.seed, None)
            if mode == _amh.AMH_GLOBAL and args.overlap:
                stream.wait_event(done)
            sweep_idx[0] += 1
            j += 1
        launches[0] += 1  # the gradient pass
        _amh.amh_get_state(samp.ctx, theta_dev, None, None, None)
        if not args.overlap:
            go = torch.cuda.Event()
            go.record(stream)
            aux.wait_event(go)
            grad_pass()
            done = torch.cuda.Event()
            done.record(aux)
            stream.wait_event(done)

    # the schedule's global sweep is the cycle's last sweep; align to a cycle
    with torch.cuda.stream(stream):
        _amh.amh_get_state(samp.ctx, theta_dev, None, None, None)
        for _ in range(args.warmup):
            cycle()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = []
    glob_ev = []
    launches[0] = 0
    terms0 = samp.pair_terms()  # straddle terms (read, formed) so far (synchronises)
    with Clocks(local, args.clocks_csv or None) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(len(step_ms)))  # evict L2 between timed steps
                e0, e1 = ev(), ev()
                e0.record(stream)
                cycle(glob_ev)
                e1.record(stream)
            step_ms.append((e0, e1))
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    timed_launches = launches[0]
    terms1 = samp.pair_terms()
    # per global sweep, this rank: terms read and interpolated; terms whose
    # distance was formed and found flat
    terms_glob = (terms1[0] - terms0[0]) / args.steps
    flat_glob = ((terms1[1] - terms0[1]) - (terms1[0] - terms0[0])) / args.steps
    total_ms = sum(a.elapsed_time(b_) for a, b_ in step_ms)
    glob_ms = [a.elapsed_time(b_) for a, b_ in glob_ev]
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    props_step = cyc * n * chains
    value = props_step * args.steps * world / (total_ms / 1000.0)
    ev_glob, ev_loc = pair_evals_per_cycle(w)
    evals_step = (ev_glob + ev_loc) * chains

    # e2e through the public API with host buffers: per step, upload the
    # chains' torsions from pinned memory, run the cycle, read back torsions
    # and energies.
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(tors.copy()).pin_memory()
        h_out = torch.empty((chains, n), dtype=torch.float32).pin_memory()
        h_E = torch.empty(chains, dtype=torch.float64).pin_memory()
        h_bE = torch.empty(chains, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            # two pinned buffers in turn: a step's result is the next step's input
            bufs = (h_in, h_out)
            for i in range(args.steps):
                _amh.amh_set_state(samp.ctx, bufs[i % 2])
                cycle()
                _amh.amh_get_state(samp.ctx, bufs[(i + 1) % 2], h_E, h_bE, None)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": props_step * args.steps * world / dt, "unit": "proposals/s",
               "h2d_bytes_per_step": int(h_in.numel() * 4),
               "d2h_bytes_per_step": int(h_out.numel() * 4 + 16 * chains),
               "timing": "host wall clock around set_state + cycle + get_state, synchronised"}

    # the one cross-rank exchange: merge the best states (outside the timed region)
    th_all, _, bE_all, bt_all = samp.state()
    if world > 1:
        from paper_2211_03193_gb300.dist import merge_best
        best_e, _, best_rank = merge_best(bE_all, bt_all, device="cuda")
    else:
        best_e, best_rank = float(np.min(bE_all)), 0
    if rank != 0:
        samp.close()
        gsamp.close()
        if world > 1:
            dist.destroy_process_group()
        return
    pk, src = peaks()
    clocks = clk.summary()
    g_ms = float(np.mean(glob_ms)) if glob_ms else float("nan")
    # terms per global launch: the straddle blocks' terms read (counted by
    # the library: pairs skipped as flat, by chunk or by pair, are not) plus
    # the full energy each call ends with; the flat pairs' formed distances
    # are counted apart at their own cost
    dense = 2 * (L ** 3 - L) // 3 * chains
    resync_terms = (L * (L - 1) // 2) * chains
    evals_glob_launch = int(terms_glob) + resync_terms
    achieved = (evals_glob_launch * FLOP_PER_EVAL + flat_glob * FLOP_PER_FLAT) / (g_ms / 1000.0) / 1e12
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    peak_tf = sm_count * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    fetch = (", table rows staged %d deep" % D if D else
             (", table entries through the texture path" if args.texture != 2
              else ", table entries through L1 loads"))
    if K == 2:
        kname = "gwarp_kernel<%s> (global sweep, chain groups of %d warps, %d chains per CTA%s)" % (
            "true" if args.texture != 2 else "false", thr // (32 * C), C, fetch)
    else:
        kname = "global_kernel<float,%d,%s> (global sweep, %d threads/CTA%s)" % (
            C, "true" if D else "false", thr, fetch)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": achieved / peak_tf,
            "traffic": captured_traffic(args.workload, (K, C, thr, D)),
            "kernel": kname,
            "launch_ms": g_ms, "pair_evals_per_launch": evals_glob_launch,
            "straddle_terms_dense": dense, "straddle_terms_evaluated": int(terms_glob),
            "straddle_terms_flat_tested": int(flat_glob), "flop_per_flat_term": FLOP_PER_FLAT,
            # the rate the same launch time would mean if every straddle pair
            # were evaluated (the skipped ones add exactly zero): a speed
            # figure, not arithmetic the kernel performs
            "dense_equivalent_tflops": (dense + resync_terms) * FLOP_PER_EVAL /
                                       (g_ms / 1000.0) / 1e12,
            "flop_per_eval": FLOP_PER_EVAL,
            "peak_basis": "%d SMs x %d FP32 lanes x 2 (FMA) x %.0f MHz (%s max clock)" % (
                sm_count, FP32_LANES_PER_SM, pk.get("sm_max_mhz", 2070.0), src)}
    mp = measured_peaks()  # after the timed region
    if mp:
        roof["peak_measured"] = mp["fp32_tflops"]
        roof["frac_of_measured"] = achieved / mp["fp32_tflops"]
        evals_s = evals_glob_launch / (g_ms / 1000.0)
        mp["global_sweep_evals_per_s"] = evals_s
        mp["frac_of_mufu_bound"] = evals_s / mp["mufu_sqrt_per_s"]  # one square root per term
    out = {"metric": "MH proposals/s", "value": value, "unit": "proposals/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": args.workload, "L": L, "chains_per_gpu": chains, "bins": w["bins"], "schedule": "10 local (d=8) : 1 global per step, "
                      "T 2.0->0.05, sigma 10->4 deg over %d sweeps" % w["total_sweeps"],
                      "proposals_per_step_per_gpu": props_step, "l2": "flushed between steps "
                      "(256 MB write); the %.1f MB table is read from L2 within a step "
                      "(L2: 129 MB)" % (tab_mb,),
                      "chains_per_cta": C, "threads_per_cta": thr, "stage_depth": D,
                      "global_kernel": ("chain groups of %d warps" % (thr // (32 * C))) if K == 2
                                       else "chains of a CTA in lock-step",
                      "gradient": "dV/ds of all %d states once per step (one amh_grad launch); %s" % (
                          chains, "on a second stream beside the global sweep, over the states "
                          "that ended the previous step" if args.overlap else
                          "after the global sweep, over the step's end states"),
                      "parallelism": "independent chains per GPU (replicas)"},
           # terms computed per second (global sweeps as counted by the library,
           # resyncs, local windows), and the dense count of the same work
           "pair_evals_per_s": (evals_glob_launch + ev_loc * chains) * args.steps * world /
                               (total_ms / 1000.0),
           "pair_evals_dense_per_s": evals_step * args.steps * world / (total_ms / 1000.0),
           "roofline": roof, "gpu_launches": timed_launches,
           "best_energy_all_ranks": best_e, "best_rank": best_rank,
           "clocks": clocks, "e2e": e2e, "measured_peaks": mp}
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(w, seed=1)
    if not args.no_ttt:
        out["time_to_target"] = time_to_target()
    print(json.dumps(out))
    samp.close()
    gsamp.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.experiment:
        if args.experiment == "forms":
            run_forms(args.workload)
            return
        {"schemes": run_schemes, "batched": run_batched, "grad": run_grad}[args.experiment]()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
