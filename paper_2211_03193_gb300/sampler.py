"""Host-side convenience over the C ABI: a context object and the AMH schedule.

``Sampler`` owns one library context (all device memory lives in the
library).  ``Schedule`` is Alg. 1's outer loop: cycles of ``n_local`` local
sweeps (window d) and ``n_global`` global sweeps, with temperature annealed
geometrically and the proposal step sigma linearly from sweep to sweep
(Sec. 2.3: sigma 10 -> 4 deg; Sec. 3: 0.1 < beta < 1), and optional noisy
restarts (the MH-with-noisy-restarts baseline of Sec. 3).  Nothing here
computes part of the method: each sweep is one library call.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import _amh
from ._amh import AMH_GLOBAL, AMH_LOCAL


class Sampler:
    """Chains of one or more proteins on the current CUDA device."""

    def __init__(self, proteins, chains, torsions, precision: int = 32, resync_every: int = 1000,
                 chains_per_cta: int = 0, threads_per_cta: int = 0, trace_chains: int = 0,
                 trace_capacity: int = 0, lattice_K: int = 0, stage_table: int = 0,
                 table_texture: int = 0, far_pairs: int = 0, local_chains_per_cta: int = 0,
                 local_threads: int = 0, keep_coords: int = 0, wait_test: int = 0,
                 global_kernel: int = 0, warps_per_chain: int = 0, stream=None):
        if not isinstance(proteins, (list, tuple)):
            proteins = [proteins]
        chains = list(np.atleast_1d(chains).astype(int))
        if len(chains) == 1 and len(proteins) > 1:
            chains = chains * len(proteins)
        edges = proteins[0].edges
        for p in proteins:
            if not np.array_equal(p.edges, edges):
                raise ValueError("all proteins of one sampler share the bin edges")
        self.proteins = proteins
        self.L = [p.L for p in proteins]
        self.chains = chains
        self.n_chains = int(sum(chains))
        self.offsets = []
        off = 0
        for p, c in zip(proteins, chains):
            self.offsets.append(off)
            off += c * p.n
        self.tors_total = off
        torsions = np.ascontiguousarray(torsions, dtype=np.float32).reshape(-1)
        if torsions.shape[0] != self.tors_total:
            raise ValueError("expected %d torsions, got %d" % (self.tors_total, torsions.shape[0]))
        table = np.concatenate([p.p.reshape(-1) for p in proteins])
        self.trace_capacity = int(trace_capacity)
        opt = _amh.amh_options_default(precision=precision, resync_every=resync_every,
                                       chains_per_cta=chains_per_cta,
                                       threads_per_cta=threads_per_cta, trace_chains=trace_chains,
                                       trace_capacity=trace_capacity, lattice_K=lattice_K,
                                       stage_table=stage_table, table_texture=table_texture,
                                       far_pairs=far_pairs,
                                       local_chains_per_cta=local_chains_per_cta,
                                       local_threads=local_threads, keep_coords=keep_coords,
                                       wait_test=wait_test, global_kernel=global_kernel,
                                       warps_per_chain=warps_per_chain, stream=stream)
        self.ctx = _amh.amh_init(np.array(self.L), np.array(chains), torsions, table, edges, opt)
        self.precision = precision

    # -------------------------------------------------------------- calls
    def energy(self) -> np.ndarray:
        E = np.zeros(self.n_chains)
        _amh.amh_energy(self.ctx, E)
        return E

    def sweep(self, mode: int, window: int, T: float, sigma_rad: float, steps: int, seed: int):
        acc = np.zeros(self.n_chains, dtype=np.int64)
        _amh.amh_sweep(self.ctx, mode, window, T, sigma_rad, steps, seed, acc)
        return acc

    def sweeps(self, mode: int, window: int, T: float, sigma_rad: float, nsweeps: int, seed: int,
               accepted=True):
        acc = np.zeros(self.n_chains, dtype=np.int64) if accepted else None
        _amh.amh_sweeps(self.ctx, mode, window, T, sigma_rad, nsweeps, seed, acc)
        return acc

    def sweeps_sched(self, mode: int, window: int, T, sigma_rad, seed: int, accepted=True):
        """A run of len(T) whole sweeps in one call, sweep q at T[q], sigma_rad[q]."""
        acc = np.zeros(self.n_chains, dtype=np.int64) if accepted else None
        _amh.amh_sweeps_sched(self.ctx, mode, window, T, sigma_rad, seed, acc)
        return acc

    def state(self):
        th = np.zeros(self.tors_total, dtype=np.float32)
        bt = np.zeros(self.tors_total, dtype=np.float32)
        E = np.zeros(self.n_chains)
        bE = np.zeros(self.n_chains)
        _amh.amh_get_state(self.ctx, th, E, bE, bt)
        return th, E, bE, bt

    def torsions(self, protein: int = 0) -> np.ndarray:
        th = self.state()[0]
        o = self.offsets[protein]
        return th[o:o + self.chains[protein] * self.proteins[protein].n].reshape(
            self.chains[protein], self.proteins[protein].n)

    def set_state(self, torsions):
        _amh.amh_set_state(self.ctx, torsions)

    def noisy_restart(self, sd_rad: float, seed: int):
        _amh.amh_noisy_restart(self.ctx, sd_rad, seed)

    def trace(self, chain: int):
        return _amh.amh_get_trace(self.ctx, chain, self.trace_capacity)

    def counter(self, chain: int = 0) -> int:
        return _amh.amh_counter(self.ctx, chain)

    def set_ladder(self, ladder):
        """Parallel tempering: ladders of len(ladder) consecutive chains, slot j
        at T * ladder[j]; None removes it."""
        _amh.amh_set_ladder(self.ctx, ladder)

    def exchange(self, T: float, parity: int, seed: int):
        acc = np.zeros(self.n_chains, dtype=np.int64)
        _amh.amh_exchange(self.ctx, T, parity, seed, acc)
        return acc

    def launch_config(self):
        return _amh.amh_launch_config(self.ctx)

    def grad(self, protein: int, theta, E_out=None, dE=None):
        """theta: CUDA tensor [batch, 2L] (float32, float64 at precision 64)."""
        import torch
        batch = theta.shape[0]
        if E_out is None:
            E_out = torch.empty(batch, dtype=torch.float64, device=theta.device)
        if dE is None:
            dE = torch.empty_like(theta)
        _amh.amh_grad(self.ctx, protein, theta, batch, E_out, dE)
        return E_out, dE

    def coords(self):
        """C-beta coordinates per chain (needs keep_coords=1): a list over
        chains of [L, 3] float64 arrays."""
        X = _amh.amh_get_coords(self.ctx, self.tors_total // 2)
        out, off = [], 0
        for p, c in zip(self.proteins, self.chains):
            for _ in range(c):
                out.append(X[off:off + p.L])
                off += p.L
        return out

    def window_coords(self, chain: int, k: int, window: int):
        """(lo, hi, C-betas) of the window the local sweep scores proposal k
        with, built from the chain's current torsions in residue lo's frame."""
        return _amh.amh_window_coords(self.ctx, chain, k, window)

    def pair_terms(self):
        """(evaluated, formed) straddle-pair terms of the global sweeps so far:
        entries read, and distances formed (see amh_pair_terms)."""
        return _amh.amh_pair_terms(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            _amh.amh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


@dataclass
class Schedule:
    """Alternating MH (Alg. 1, Fig. 1): per cycle n_local local sweeps with
    window d, then n_global global sweeps.  T_s = T0 (T1/T0)^(s/(S-1)) and
    sigma_s linear from sigma0 to sigma1 (degrees) over the S sweeps; both
    constant within a sweep.  n_local = 0 gives plain MH; noisy_every > 0
    adds a Gaussian kick of noisy_sd_deg to every torsion every that many
    sweeps (MH with noisy restarts).  windows (optional) cycles through
    several localization radii in turn (the cascaded radii of Sec. 2.2):
    local sweep j of a cycle uses windows[j % len(windows)]."""
    total_sweeps: int
    n_local: int = 10
    n_global: int = 1
    window: int = 8
    T0: float = 2.0
    T1: float = 0.05
    sigma0_deg: float = 10.0
    sigma1_deg: float = 4.0
    seed: int = 1
    noisy_every: int = 0
    noisy_sd_deg: float = 30.0
    windows: tuple | None = None

    def window_of(self, s: int) -> int:
        if not self.windows:
            return self.window
        j = s % (self.n_local + self.n_global)
        return self.windows[j % len(self.windows)]

    def params(self, s: int):
        S = max(self.total_sweeps - 1, 1)
        f = min(s, S) / S
        T = self.T0 * (self.T1 / self.T0) ** f
        sigma = math.radians(self.sigma0_deg + (self.sigma1_deg - self.sigma0_deg) * f)
        cyc = self.n_local + self.n_global
        mode = AMH_LOCAL if (s % cyc) < self.n_local else AMH_GLOBAL
        return mode, T, sigma


def schedule_runs(sched: Schedule, s0: int, s1: int, limit: int = _amh.AMH_MAX_SCHED):
    """Sweeps [s0, s1) of the schedule as runs that one library call can take:
    consecutive sweeps of one mode and window, at most `limit` of them, a
    run ending where a noisy restart follows.  Yields (mode, window, [s])."""
    run = []
    for s in range(s0, s1):
        mode = sched.params(s)[0]
        win = sched.window_of(s)
        if run and (mode, win) != (sched.params(run[0])[0], sched.window_of(run[0])):
            yield sched.params(run[0])[0], sched.window_of(run[0]), run
            run = []
        run.append(s)
        if len(run) == limit or (sched.noisy_every and (s + 1) % sched.noisy_every == 0):
            yield mode, win, run
            run = []
    if run:
        yield sched.params(run[0])[0], sched.window_of(run[0]), run


def run_schedule(sampler: Sampler, sched: Schedule, s0: int = 0, s1: int | None = None,
                 on_sweep=None):
    """Run sweeps [s0, s1) of the schedule; returns total accepted per chain
    (counted only when on_sweep is given).  Without on_sweep the sweeps go to
    the library in runs (one call per run of same-mode sweeps, each sweep at
    its own T and sigma), which gives the same result as one call per sweep."""
    if s1 is None:
        s1 = sched.total_sweeps
    total = np.zeros(sampler.n_chains, dtype=np.int64)
    if on_sweep is None:
        for mode, win, run in schedule_runs(sched, s0, s1):
            Ts = [sched.params(s)[1] for s in run]
            Ss = [sched.params(s)[2] for s in run]
            sampler.sweeps_sched(mode, win, Ts, Ss, sched.seed, accepted=False)
            last = run[-1]
            if sched.noisy_every and (last + 1) % sched.noisy_every == 0:
                sampler.noisy_restart(math.radians(sched.noisy_sd_deg), sched.seed * 1000003 + last)
        return total
    for s in range(s0, s1):
        mode, T, sigma = sched.params(s)
        acc = sampler.sweeps(mode, sched.window_of(s), T, sigma, 1, sched.seed,
                             accepted=on_sweep is not None)
        if acc is not None:
            total += acc
        if sched.noisy_every and (s + 1) % sched.noisy_every == 0:
            sampler.noisy_restart(math.radians(sched.noisy_sd_deg), sched.seed * 1000003 + s)
        if on_sweep is not None:
            on_sweep(s, mode, T, sigma)
    return total


def capture_schedule(sampler: Sampler, sched: Schedule, s0: int, s1: int, stream):
    """Capture sweeps [s0, s1) of the schedule (one launch per sweep, each with
    its own T and sigma, plus the noisy restarts) into a CUDA graph on
    `stream`, which must be the stream the sampler was created with.  Replay
    runs them again on the device; the chains' proposal counters live in
    device memory, so each replay continues where the previous one ended.
    Capturing runs nothing and counts the sweeps once on the host side.  Runs
    of same-mode sweeps are captured as one launch each (schedule_runs)."""
    import torch
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for mode, win, run in schedule_runs(sched, s0, s1):
            Ts = [sched.params(s)[1] for s in run]
            Ss = [sched.params(s)[2] for s in run]
            _amh.amh_sweeps_sched(sampler.ctx, mode, win, Ts, Ss, sched.seed, None)
            last = run[-1]
            if sched.noisy_every and (last + 1) % sched.noisy_every == 0:
                _amh.amh_noisy_restart(sampler.ctx, math.radians(sched.noisy_sd_deg),
                                       sched.seed * 1000003 + last)
    return g


def restart_from_best(sampler: Sampler, sched: Schedule, runs: int = 10, on_run=None):
    """Sec. 2.3's protocol: the whole schedule is run `runs` times; each run
    starts every chain from the lowest-energy state it has seen (its best
    state at global-sweep ends).  While runs keep lowering the best energy the
    step sigma follows sched (10 -> 4 deg); after F runs without a new lowest
    energy it follows 10/F -> 1/F deg.  "Lower" is judged on the lowest
    energy over all chains.  Returns the best energy after each run."""
    import dataclasses
    history = []
    best = float(np.min(sampler.state()[2]))
    failures = 0
    for r in range(runs):
        if failures:
            sig = (10.0 / failures, 1.0 / failures)
        else:
            sig = (sched.sigma0_deg, sched.sigma1_deg)
        sr = dataclasses.replace(sched, sigma0_deg=sig[0], sigma1_deg=sig[1],
                                 seed=sched.seed + 7919 * r)
        if r:
            sampler.set_state(sampler.state()[3])  # every chain from its best state
        run_schedule(sampler, sr)
        now = float(np.min(sampler.state()[2]))
        if now < best:
            best = now
        else:
            failures += 1
        history.append(best)
        if on_run is not None:
            on_run(r, best, sig)
    return history
