"""Parallel tempering on the GPU: per-slot temperatures in the sweeps and the
replica-exchange step, against the oracle."""
import numpy as np
import pytest

from paper_2211_03193_gb300 import synth
from test_oracle_pins import _lattice_setup, _state_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03193_gb300 import build, _amh, sampler
    build.build()
    _amh.load()
    return sampler


def test_exchange_matches_oracle(amh, orc):
    L, chains, K = 20, 16, 4
    prot = synth.make_protein(L, seed=900)
    tors = synth.random_torsions(chains, L, seed=901)
    ladder = np.array([1.0, 1.3, 1.7, 2.2])
    T = 40.0  # hot enough that some swaps are accepted
    with amh.Sampler(prot, chains, tors, precision=64, trace_chains=chains,
                     trace_capacity=2 * L) as s:
        s.set_ladder(ladder)
        s.sweeps(1, 0, T, 0.3, 1, 5)
        P = orc.Problem(L, prot.p, prot.edges)
        # per-slot temperatures drove the sweep: replay chain by chain
        for c in range(chains):
            tr = s.trace(c)
            _, _, otr = P.run(tors[c].astype(np.float64), orc.GLOBAL, 0, T * ladder[c % K], 0.3,
                              0, 2 * L, 5, c, trace=True, forced=tr["accept"].astype(np.uint8))
            margin = np.abs(otr["lnu"] + otr["dV"] / (T * ladder[c % K]))
            assert np.all((tr["accept"] == otr["accept"]) | (margin < 1e-9))
        th, E, _, _ = s.state()
        S = th.reshape(chains, -1).astype(np.float64)
        for rnd, parity in enumerate((0, 1, 0)):
            sw = s.exchange(T, parity, 77)
            th2, E2, _, _ = s.state()
            Eo, So, acc = orc.exchange(E, S, K, ladder, T, parity, 77, rnd)
            assert np.array_equal(sw, acc.astype(np.int64))
            assert np.array_equal(E2, Eo)
            assert np.array_equal(th2.reshape(chains, -1).astype(np.float64), So)
            E, S = Eo, So


def test_tempering_on_gpu_keeps_each_slot_at_its_boltzmann_law(amh, orc):
    K = 3
    P, prot, n, q, live, Es = _lattice_setup(orc, K=K)
    T0 = float(np.std(Es)) / 2
    ladder = np.array([1.0, 1.6, 2.6, 4.2])
    Kl = len(ladder)
    ladders = 1024
    chains = Kl * ladders
    tors = np.zeros((chains, n), np.float32)
    counts = np.zeros((Kl, K ** len(live)))
    with amh.Sampler(prot, chains, tors, precision=64, lattice_K=K) as s:
        s.set_ladder(ladder)
        for r in range(160):
            s.sweeps(1, 0, T0, 1.5, 1, 11)
            s.exchange(T0, r % 2, 13)
            if r >= 40:
                th = s.torsions().astype(np.float64)
                idx = _state_index(th, live, q, K)
                for j in range(Kl):
                    counts[j] += np.bincount(idx[j::Kl], minlength=K ** len(live))
    for j in range(Kl):
        w = np.exp(-(Es - Es.min()) / (T0 * ladder[j]))
        pi = w / w.sum()
        hist = counts[j] / counts[j].sum()
        mean_exact = float(pi @ Es)
        sd = float(np.sqrt(pi @ (Es - mean_exact) ** 2))
        assert abs(float(hist @ Es) - mean_exact) < 0.03 * sd, j
        tv = 0.5 * np.abs(hist - pi).sum()
        tv_noise = 0.5 * np.sum(np.sqrt(2 * pi * (1 - pi) / (np.pi * counts[j].sum())))
        assert tv < 2.0 * tv_noise, (j, tv, tv_noise)
