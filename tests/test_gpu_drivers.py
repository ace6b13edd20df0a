"""Host drivers over the C ABI: autograd wrapper, L-BFGS hand-off, the AMH
schedule, and its CUDA-graph capture."""
import math

import numpy as np
import pytest

from paper_2211_03193_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03193_gb300 import build, _amh, sampler, autograd
    build.build()
    _amh.load()
    return torch, sampler, autograd


def test_autograd_backward_is_scaled_amh_grad(env, orc):
    torch, sampler, autograd = env
    L, batch = 30, 5
    prot = synth.make_protein(L, seed=800)
    tors = synth.random_torsions(batch, L, seed=801)
    with sampler.Sampler(prot, 1, tors[:1]) as s:
        th = torch.tensor(tors, device="cuda", requires_grad=True)
        E = autograd.energy(s, th)
        Ed = E.detach()
        w = torch.arange(1, batch + 1, dtype=torch.float64, device="cuda")
        (E * w).sum().backward()
        _, g = s.grad(0, th.detach())
        assert torch.allclose(th.grad, g * w[:, None].float(), rtol=1e-6, atol=1e-6)
        P = orc.Problem(L, prot.p, prot.edges)
        for b in range(batch):
            assert abs(float(Ed[b]) - P.energy(tors[b].astype(np.float64))) <= 1e-5 * abs(float(Ed[b]))


def test_lbfgs_refine_lowers_every_state(env, orc):
    torch, sampler, autograd = env
    L, batch = 40, 4
    prot = synth.make_protein(L, seed=810)
    tors = synth.random_torsions(batch, L, seed=811)
    with sampler.Sampler(prot, 1, tors[:1]) as s:
        th0 = torch.tensor(tors, device="cuda")
        E0, _ = s.grad(0, th0)
        th, E = autograd.lbfgs_refine(s, th0, iterations=60)
    assert torch.all(E < E0 - 1.0)
    P = orc.Problem(L, prot.p, prot.edges)
    for b in range(batch):
        e_orc = P.energy(th[b].cpu().numpy().astype(np.float64))
        assert abs(float(E[b]) - e_orc) <= 1e-5 * abs(e_orc)


def test_lbfgs_with_local_mh_runs_and_improves(env):
    torch, sampler, autograd = env
    L, chains = 36, 4
    prot = synth.make_protein(L, seed=820)
    tors = synth.random_torsions(chains, L, seed=821)
    with sampler.Sampler(prot, chains, tors) as s:
        E0 = s.energy()
        E = autograd.lbfgs_with_local_mh(s, cycles=2, n_lbfgs=20, n_local=2, window=5)
        assert np.all(E < E0)
        assert s.counter(0) == 2 * 2 * 2 * L  # two cycles of two local sweeps


def _wrapped_close(a, b, atol):
    return np.all(np.abs(np.angle(np.exp(1j * (np.asarray(a, np.float64) - b)))) <= atol)


def test_lbfgs_with_local_mh_local_phase_equals_oracle(env, orc):
    """Sec. 3's L-BFGS with localized MH, FP64 form: after every L-BFGS phase
    the oracle replays the localized-MH sweeps from exactly the state L-BFGS
    handed over (the same counter, seed, window, T and sigma) and must end at
    the GPU's torsions; the energies the driver returns are the oracle's V of
    the final torsions."""
    torch, sampler, autograd = env
    L, chains = 28, 4
    n = 2 * L
    prot = synth.make_protein(L, seed=825)
    tors = synth.random_torsions(chains, L, seed=826)
    P = orc.Problem(L, prot.p, prot.edges)
    T, sigma, window, n_local, seed = 0.2, 0.07, 5, 3, 9
    seen = []

    def on_cycle(cyc, handed, t0, after):
        seen.append((handed.copy(), t0, after.copy()))

    with sampler.Sampler(prot, chains, tors, precision=64) as s:
        E = autograd.lbfgs_with_local_mh(s, cycles=3, n_lbfgs=15, n_local=n_local,
                                         window=window, T=T, sigma_rad=sigma, seed=seed,
                                         on_cycle=on_cycle)
        th_end = s.torsions()
    assert len(seen) == 3
    ends = []
    for cyc, (handed, t0, after) in enumerate(seen):
        assert t0 == cyc * n_local * n
        if cyc:  # L-BFGS started from the previous cycle's end state
            assert not np.array_equal(handed, seen[cyc - 1][2])
        for c in range(chains):
            st, _, tr = P.run(handed[c].astype(np.float64), orc.LOCAL, window, T, sigma, t0,
                              n_local * n, seed, c, trace=True)
            # FP64 GPU form: only a near-tie (|ln u + dV/T| < 1e-5) could part
            # the paths; none occurs in this run
            margin = np.abs(tr["lnu"] + tr["dV"] / T)
            assert margin.min() >= 1e-5
            assert _wrapped_close(after[c], st, 1e-6), (cyc, c)
            if cyc == 2:
                ends.append(st)
    # the returned energies are V of the FP64 end states (the torsions read
    # back above passed through the FP32 interface)
    for c in range(chains):
        assert _wrapped_close(th_end[c], ends[c], 1e-6)
        assert abs(E[c] - P.energy(ends[c])) <= 1e-10 * abs(E[c])


def test_restart_from_best_equals_oracle(env, orc):
    """Sec. 2.3's restarts, FP64 form: the oracle replays every run from the
    best state the previous runs reached (kept at global-sweep ends, strictly
    lower energy), with the run's seed and its sigma range (10 -> 4 deg while
    runs improve the lowest energy over the chains, 10/F -> 1/F deg after F
    runs that did not), and must reach the GPU's torsions, best energies and
    sigma ranges run by run."""
    import dataclasses
    torch, sampler, autograd = env
    L, chains = 20, 6
    n = 2 * L
    prot = synth.make_protein(L, seed=855)
    tors = synth.random_torsions(chains, L, seed=856)
    sched = sampler.Schedule(total_sweeps=11, n_local=10, n_global=1, window=8, T0=0.6, T1=0.1,
                             seed=5)
    runs = 5
    P = orc.Problem(L, prot.p, prot.edges)
    gpu = []
    with sampler.Sampler(prot, chains, tors, precision=64) as s:
        sampler.restart_from_best(
            s, sched, runs=runs,
            on_run=lambda r, b, sig: gpu.append((sig, b) + tuple(np.copy(v) for v in s.state())))
    S = tors.astype(np.float64)
    bestE = P.energies(S)
    bestS = S.copy()
    best_all = float(bestE.min())
    failures = 0
    for r in range(runs):
        sig = (10.0 / failures, 1.0 / failures) if failures else (10.0, 4.0)
        sig_gpu, b_gpu, th, E, bE, bt = gpu[r]
        assert sig_gpu == sig, (r, sig_gpu, sig)
        sr = dataclasses.replace(sched, sigma0_deg=sig[0], sigma1_deg=sig[1],
                                 seed=sched.seed + 7919 * r)
        if r:  # every chain from its best state, through the FP32 interface
            S = bestS.astype(np.float32).astype(np.float64)
        for q in range(sched.total_sweeps):
            mode, T, sigma = sr.params(q)
            t0 = (r * sched.total_sweeps + q) * n
            S, _ = P.run_chains(S, orc.LOCAL if mode == 0 else orc.GLOBAL, sr.window_of(q), T,
                                sigma, t0, n, sr.seed, 0)
            if mode == 1:
                Eq = P.energies(S)
                better = Eq < bestE
                bestE[better] = Eq[better]
                bestS[better] = S[better]
        th = th.reshape(chains, n)
        bt = bt.reshape(chains, n)
        for c in range(chains):
            assert _wrapped_close(th[c], S[c], 1e-6), (r, c)
            assert _wrapped_close(bt[c], bestS[c], 1e-6), (r, c)
        assert np.allclose(bE, bestE, rtol=1e-10, atol=0), (r, bE - bestE)
        now = float(bestE.min())
        if now < best_all:
            best_all = now
        else:
            failures += 1
        assert abs(b_gpu - best_all) <= 1e-10 * abs(best_all)


@pytest.mark.parametrize("noisy", [0, 3])
def test_graph_replay_equals_eager_schedule(env, noisy):
    torch, sampler, autograd = env
    L, chains = 26, 12
    prot = synth.make_protein(L, seed=830)
    tors = synth.random_torsions(chains, L, seed=831)
    sched = sampler.Schedule(total_sweeps=22, n_local=3, n_global=1, window=8, T0=1.5,
                             T1=0.1, seed=4, noisy_every=noisy, noisy_sd_deg=20.0)
    eager = torch.cuda.Stream()
    with sampler.Sampler(prot, chains, tors, stream=eager) as s:
        with torch.cuda.stream(eager):
            sampler.run_schedule(s, sched, 0, 8)
            sampler.run_schedule(s, sched, 8, 16)
        torch.cuda.synchronize()
        want = s.state()
    gs = torch.cuda.Stream()
    with sampler.Sampler(prot, chains, tors, stream=gs) as s:
        g1 = sampler.capture_schedule(s, sched, 0, 8, gs)
        g2 = sampler.capture_schedule(s, sched, 8, 16, gs)
        g1.replay()
        g2.replay()
        torch.cuda.synchronize()
        got = s.state()
        assert s.counter(0) == 16 * 2 * L
    for a, b in zip(want, got):
        assert np.array_equal(a, b)


def test_cascaded_windows_follow_the_schedule(env, orc):
    """Local sweep j of a cycle uses windows[j % len(windows)]: the GPU run
    equals the oracle's sweep-by-sweep replay with those windows (FP64)."""
    torch, sampler, autograd = env
    L, chains = 18, 2
    prot = synth.make_protein(L, seed=840)
    tors = synth.random_torsions(chains, L, seed=841)
    sched = sampler.Schedule(total_sweeps=8, n_local=3, n_global=1, windows=(4, 8, 12), T0=1.0,
                             T1=0.5, seed=6)
    n = 2 * L
    P = orc.Problem(L, prot.p, prot.edges)
    with sampler.Sampler(prot, chains, tors, precision=64) as s:
        sampler.run_schedule(s, sched)
        th = s.torsions()
    for c in range(chains):
        st = tors[c].astype(np.float64)
        for q in range(8):
            mode, T, sigma = sched.params(q)
            st, _, _ = P.run(st, orc.LOCAL if mode == 0 else orc.GLOBAL, sched.window_of(q), T,
                             sigma, q * n, n, 6, c)
        assert np.allclose(th[c], st, atol=1e-6)
    assert [sched.window_of(q) for q in range(3)] == [4, 8, 12]


def test_restart_from_best_protocol(env):
    torch, sampler, autograd = env
    L, chains = 24, 64
    prot = synth.make_protein(L, seed=850)
    tors = synth.random_torsions(chains, L, seed=851)
    sched = sampler.Schedule(total_sweeps=11, n_local=10, n_global=1, T0=1.0, T1=0.2, seed=2)
    seen = []
    with sampler.Sampler(prot, chains, tors) as s:
        E0 = float(s.state()[2].min())
        hist = sampler.restart_from_best(s, sched, runs=4,
                                         on_run=lambda r, b, sig: seen.append(sig))
        assert s.counter(0) == 4 * 11 * 2 * L
    assert all(b2 <= b1 for b1, b2 in zip(hist, hist[1:]))
    assert hist[-1] <= E0
    assert seen[0] == (10.0, 4.0)
    for (a, b) in seen[1:]:
        assert (a, b) == (10.0, 4.0) or abs(a / b - 10.0) < 1e-12
