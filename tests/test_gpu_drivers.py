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
