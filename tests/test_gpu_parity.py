"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Every case uses seeded synthetic inputs from ``synth``; expected values come
only from ``oracle``.  FP32 runs are compared teacher-forced: the oracle
replays each traced chain adopting the GPU's decisions, recomputes every
Delta-E in FP64 and checks the GPU's value and decision against it.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from paper_2211_03193_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEG = math.pi / 180


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03193_gb300 import build, _amh, sampler
    build.build()
    _amh.load()
    return sampler


def f64(x):
    return np.asarray(x, dtype=np.float64)


# Tolerance of an FP32 Delta-E against the FP64 Delta-E of the GPU's own
# states.  Its parts: a floor for the terms' own rounding (the folded FP32
# entries carry up to ~3e-5 per term); an allowance per straddle pair for the
# coherent error of the moved side (each proposal's FP32 map rounds its
# rotation matrix, and the commits between rebuilds add to it; every pair in
# the table's range feels that shift through its slope); and a relative part
# for the large moves whose long arm carries the map's rounding furthest.
# Measured (GB300, 16 400 global proposals over L = 33, 150 and 300, 37-bin
# and 64-bin-to-66-A tables, random starts, mid-anneal and anneal-tail
# states, with and without periodic rebuilds): at most 1.2e-5 per straddle
# pair where |Delta-E| < 1000, at most 4e-6 of |Delta-E| beyond; the
# constants below sit 1.3x and 2.5x above those.  Only pairs within the
# table's reach (its last bin centre) feel a shift, so the per-pair part
# scales with that reach: x1 for the 37-bin tables (20.25 A), x3.2 for 64
# bins out to 65.5 A, where nearly every straddle pair is in range.
def de_tol(npairs, dE=0.0, reach=1.0):
    return 1e-3 + 1.5e-5 * reach * npairs + 1e-5 * np.abs(dE)


def reach_of(prot):
    """Last bin centre over 20.25 A (the 37-bin tables'), at least 1."""
    e = np.asarray(prot.edges, dtype=np.float64)
    w = e[1] - e[0]
    c_last = e[0] + 0.5 * w + (len(e) - 2) * w
    return max(1.0, c_last / 20.25)


def gpu_advance(s0, tr):
    """The GPU's state after a traced segment: s0 with every accepted
    theta_new applied."""
    g = f64(s0).copy()
    for t in np.flatnonzero(tr["accept"]):
        g[int(tr["k"][t])] = tr["theta_new"][t]
    return g


def gpu_states_delta(P, s0, tr):
    """Eq. 5 Delta-E, in FP64, of each traced proposal from the GPU's own
    states: s0 with every accepted traced theta_new applied (the FP32 values
    the GPU holds).  Returns (Delta-E per step, the final state)."""
    g = f64(s0).copy()
    e = P.energy(g)
    out = np.empty(tr.shape[0])
    for t in range(tr.shape[0]):
        trial = g.copy()
        trial[int(tr["k"][t])] = tr["theta_new"][t]
        e_new = P.energy(trial)
        out[t] = e_new - e
        if tr["accept"][t]:
            g, e = trial, e_new
    return out, g


def replay_and_compare(orc, prot, s0, tr, mode, window, T, sigma, t0, seed, chain, fp64,
                       gpu_s0=None):
    """Teacher-forced replay of one traced GPU chain; returns diagnostics.

    FP32 global sweeps: the GPU holds torsions in FP32, the replay proposes
    in FP64, so their states differ by up to half an FP32 ulp per torsion
    (1.2e-7 rad at |theta| near pi) and, with |dV/dtheta| up to ~1e6 at
    L = 150, their Delta-E by up to ~0.1 for reasons outside the kernel.  The
    GPU's Delta-E is therefore checked against the FP64 Delta-E of its own
    traced states (gpu_s0, default s0, and the accepted theta_new values);
    the replay checks the draws, the proposals and the decisions."""
    P = orc.Problem(prot.L, prot.p, prot.edges)
    steps = tr.shape[0]
    forced = tr["accept"].astype(np.uint8)
    s_end, _, otr = P.run(f64(s0), mode, window, T, sigma, t0, steps, seed, chain,
                          trace=True, forced=forced)
    assert np.array_equal(otr["k"], tr["k"])
    exact = otr["dV"]
    gpu_end = None
    if not fp64 and mode == orc.GLOBAL:
        exact, gpu_end = gpu_states_delta(P, s0 if gpu_s0 is None else gpu_s0, tr)
    emax = float(np.max(-np.log(np.maximum(prot.p, 1e-300))))
    w = float(prot.edges[1] - prot.edges[0])
    k = tr["k"]
    p = (k + 1) // 2
    if mode == orc.GLOBAL:
        npairs = p * (prot.L - p)
    else:
        h = window // 2
        c = k // 2
        lo = np.maximum(0, c - h)
        hi = np.minimum(prot.L - 1, c + h)
        npairs = np.where((p > lo) & (p <= hi), (p - lo) * (hi - p + 1), 0)
    dE_err = np.abs(tr["dE"] - exact)
    if fp64:
        tol = 1e-9 * (1 + np.abs(exact))
        lnu_tol = 1e-12
    else:
        tol = de_tol(npairs, exact, reach_of(prot))
        lnu_tol = 2e-6
    lnu_err = np.abs(tr["lnu"] - otr["lnu"])
    assert np.all(lnu_err <= lnu_tol * (1 + np.abs(otr["lnu"])))
    th_err = np.abs(np.angle(np.exp(1j * (tr["theta_new"] - otr["theta_new"]))))
    assert np.all(th_err <= (1e-12 if fp64 else 2e-6)), th_err.max()
    bad = dE_err > tol
    assert not bad.any(), (np.flatnonzero(bad)[:5], dE_err[bad][:5],
                           tol[bad][:5] if np.ndim(tol) else tol, exact[bad][:5],
                           npairs[bad][:5] if np.ndim(npairs) else npairs)
    # every GPU decision follows Eq. 1 from the GPU's own ln u and Delta-E,
    # in the precision the kernel decides in (the FP32 form: FP32 products;
    # the FP64 form: FP64)
    if not fp64:
        own = (tr["lnu"].astype(np.float32) * np.float32(T)) < -tr["dE"].astype(np.float32)
    else:
        own = tr["lnu"] * T < -tr["dE"]
    assert np.array_equal(tr["accept"].astype(bool), own), np.flatnonzero(tr["accept"] != own)[:5]
    # so a decision can differ from the exact one (the oracle's ln u and the
    # FP64 Delta-E) only within the measured error of those two values: a
    # disagreement is a tie (margin < 1e-5, the contract's allowance) or an
    # FP32 rounding flip (margin below this step's |Delta-E error| / T plus
    # its ln u error); anything else fails
    margin = np.abs(otr["lnu"] + exact / T)
    disagree = tr["accept"] != (otr["lnu"] * T < -exact)
    tie = margin < 1e-5
    explained = margin <= dE_err / T + lnu_err + 1e-12
    assert np.all((tie | explained)[disagree]), np.flatnonzero(disagree & ~(tie | explained))[:5]
    flips = disagree & ~tie
    return dict(max_dE_err=float(dE_err.max()), disagree=int(disagree.sum()),
                ties=int((disagree & tie).sum()), flips=int(flips.sum()), n=steps,
                dE_err=dE_err, npairs=npairs, exact=exact, margin=margin,
                s_end=s_end, gpu_s_end=gpu_end,
                replay_dE_gap=float(np.max(np.abs(otr["dV"] - exact), initial=0.0)))


# ---------------------------------------------------------------- RNG
def test_philox_bit_exact_with_oracle_and_curand(amh, orc, tmp_path):
    from paper_2211_03193_gb300 import _amh
    cases = [(0, 0, 0, 0), (12345, 7, 1 << 33, 0), (2 ** 64 - 1, 2 ** 32 - 1, 2 ** 40 + 5, 1),
             (987654321987, 1023, 99, 2)]
    nvcc = os.environ.get("NVCC", "nvcc")
    so = str(tmp_path / "curand_ref.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                    "-Xcompiler", "-fPIC", "-o", so,
                    os.path.join(ROOT, "tests", "cuda", "curand_philox_ref.cu")], check=True)
    ref = ctypes.CDLL(so)
    for seed, chain, t0, stream in cases:
        words, z, u = _amh.amh_philox(seed, chain, t0, stream, 257)
        ctr = np.zeros((257, 4), np.uint32)
        key = np.zeros((257, 2), np.uint32)
        for i in range(257):
            t = t0 + i
            ctr[i] = (chain, t & 0xFFFFFFFF, (t >> 32) & 0xFFFFFFFF, stream)
            key[i] = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
            want = orc.philox(ctr[i], key[i])
            assert np.array_equal(words[i], want), (seed, chain, t, words[i], want)
            _, zo, uo = orc.draw(seed, chain, t, stream)
            assert float(u[i]) == uo  # 23-bit uniforms are exact in binary32
            assert abs(float(z[i]) - zo) <= 4e-6 * (1 + abs(zo))
        out = np.zeros((257, 4), np.uint32)
        assert ref.curand_philox_ref(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, 257) == 0
        assert np.array_equal(out, words)


# ---------------------------------------------------------------- energy
@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("L,chains,C", [(2, 3, 8), (5, 9, 4), (37, 17, 8), (64, 8, 2), (64, 3, 1)])
def test_energy_matches_oracle(amh, orc, precision, L, chains, C):
    if precision == 64 and C == 8:
        C = 4
    prot = synth.make_protein(L, seed=100 + L)
    tors = synth.random_torsions(chains, L, seed=L)
    with amh.Sampler(prot, chains, tors, precision=precision, chains_per_cta=C) as s:
        E = s.energy()
        P = orc.Problem(L, prot.p, prot.edges)
        want = P.energies(f64(tors))
        rel = 1e-5 if precision == 32 else 1e-12
        assert np.all(np.abs(E - want) <= rel * np.abs(want) + 1e-9), (E, want)
        th, E2, bE, bt = s.state()
        assert np.array_equal(th.reshape(chains, -1), tors)
        assert np.array_equal(bE, E)


def test_energy_uneven_proteins_and_64_bins(amh, orc):
    Ls = [3, 20, 41, 9]
    edges = synth.edges_uniform_64()
    prots = [synth.make_protein(L, edges=edges, sigma_d=1.5, seed=200 + L) for L in Ls]
    chains = [5, 1, 10, 3]
    tors = np.concatenate([synth.random_torsions(c, p.L, seed=c + p.L).ravel()
                           for p, c in zip(prots, chains)])
    with amh.Sampler(prots, chains, tors, chains_per_cta=4) as s:
        E = s.energy()
    want = []
    off = 0
    for p, c in zip(prots, chains):
        P = orc.Problem(p.L, p.p, p.edges)
        want.append(P.energies(f64(tors[off:off + c * p.n])))
        off += c * p.n
    want = np.concatenate(want)
    assert np.allclose(E, want, rtol=1e-5, atol=1e-9)


# ---------------------------------------------------------------- global sweeps
@pytest.mark.parametrize("precision,C,stage,threads,tex", [
    (64, 1, 2, 256, 0), (64, 4, 2, 256, 0), (32, 8, 2, 256, 2), (32, 2, 2, 256, 2),
    (32, 1, 2, 128, 2), (32, 8, 1, 512, 2), (32, 4, 1, 256, 2), (32, 8, 1, 128, 2),
    (32, 8, 2, 512, 1), (32, 4, 2, 256, 1), (32, 2, 2, 256, 0)])
def test_global_sweeps_teacher_forced(amh, orc, precision, C, stage, threads, tex):
    """stage 1: table rows staged in shared memory by bulk async copies;
    stage 2: read through L1; tex 1: entries fetched through a texture, 2:
    global loads, 0: the default (texture)."""
    L, chains = 33, 11
    prot = synth.make_protein(L, seed=300)
    tors = synth.random_torsions(chains, L, seed=301)
    n = 2 * L
    steps = 3 * n + 7  # ragged: ends mid-sweep, with an odd leftover
    T, sigma, seed = 0.8, 25 * DEG, 99
    with amh.Sampler(prot, chains, tors, precision=precision, chains_per_cta=C,
                     threads_per_cta=threads, stage_table=stage, table_texture=tex,
                     trace_chains=chains, trace_capacity=steps, resync_every=50) as s:
        assert s.launch_config()[2] == (0 if stage == 2 else s.launch_config()[2])
        if stage == 1:
            assert s.launch_config()[2] >= 2
        acc = s.sweep(1, 0, T, sigma, steps, seed)
        th, E, bE, bt = s.state()
        for c in range(chains):
            tr = s.trace(c)
            assert tr.shape[0] == steps
            assert acc[c] == tr["accept"].sum()
            d = replay_and_compare(orc, prot, tors[c], tr, orc.GLOBAL, 0, T, sigma, 0, seed, c,
                                   precision == 64)
            if precision == 64:
                assert d["disagree"] == 0
                assert np.allclose(th.reshape(chains, -1)[c], d["s_end"], atol=1e-6)
            # the energy after the call is a fresh FP64 resync of the final
            # state (FP64: the oracle's own end state, as the FP32 interface
            # rounds the torsions the test can read back)
            P = orc.Problem(L, prot.p, prot.edges)
            if precision == 64:
                e_want = P.energy(d["s_end"])
                assert abs(E[c] - e_want) <= 1e-10 * abs(e_want)
            else:
                e_want = P.energy(f64(th.reshape(chains, -1)[c]))
                assert abs(E[c] - e_want) <= 1e-5 * abs(e_want)
        assert np.all(bE <= E + 1e-9)


@pytest.mark.parametrize("W,G,tex,L", [(1, 1, 0, 33), (2, 1, 2, 33), (4, 1, 0, 33), (8, 1, 2, 33),
                                       (4, 2, 0, 33), (2, 4, 2, 33), (1, 2, 0, 150),
                                       (2, 2, 2, 151), (2, 4, 0, 150), (4, 1, 0, 150)])
def test_warp_kernel_teacher_forced(amh, orc, W, G, tex, L):
    """The chain-group global sweep (W chains of a CTA, each on G warps of
    its own): teacher-forced oracle replay of every chain over a ragged run
    that ends mid-sweep with an odd leftover and crosses sweep boundaries."""
    chains = 11
    prot = synth.make_protein(L, seed=300 + L)
    tors = synth.random_torsions(chains, L, seed=301)
    n = 2 * L
    steps = (3 * n + 7) if L < 100 else (n + 5)
    T, sigma, seed = 0.8, 25 * DEG if L < 100 else 10 * DEG, 99
    with amh.Sampler(prot, chains, tors, global_kernel=2, chains_per_cta=W, warps_per_chain=G,
                     table_texture=tex, trace_chains=chains, trace_capacity=steps,
                     resync_every=50) as s:
        assert s.launch_config() == (W, 32 * W * G, 0, 2)
        acc = s.sweep(1, 0, T, sigma, steps, seed)
        th, E, bE, bt = s.state()
        P = orc.Problem(L, prot.p, prot.edges)
        flips = 0
        for c in range(chains):
            tr = s.trace(c)
            assert tr.shape[0] == steps
            assert acc[c] == tr["accept"].sum()
            d = replay_and_compare(orc, prot, tors[c], tr, orc.GLOBAL, 0, T, sigma, 0, seed, c,
                                   False)
            flips += d["flips"]
            e_want = P.energy(f64(th.reshape(chains, -1)[c]))
            assert abs(E[c] - e_want) <= 1e-5 * abs(e_want)
            assert s.counter(c) == steps
        assert np.all(bE <= E + 1e-9)
        print("chain groups W=%d G=%d L=%d: flips %d" % (W, G, L, flips))


def test_warp_and_cta_kernels_agree(amh):
    """The two global-sweep kernels compute the same proposals: from the same
    states and seeds their Delta-E agree within FP32 summation order and
    their decisions agree up to the first near-tie."""
    L, chains = 120, 16
    prot = synth.make_protein(L, seed=340)
    tors = synth.random_torsions(chains, L, seed=341)
    n = 2 * L
    steps = 2 * n + 1
    T, sigma, seed = 0.5, 8 * DEG, 13
    runs = []
    for kw in (dict(global_kernel=2, chains_per_cta=2, warps_per_chain=2),
               dict(global_kernel=1, chains_per_cta=2, threads_per_cta=128)):
        with amh.Sampler(prot, chains, tors, trace_chains=chains, trace_capacity=steps,
                         **kw) as s:
            s.sweep(1, 0, T, sigma, steps, seed)
            runs.append([s.trace(c) for c in range(chains)])
    k = runs[0][0]["k"]
    p = (k + 1) // 2
    npairs = p * (L - p)
    for c in range(chains):
        a, b = runs[0][c], runs[1][c]
        split = np.flatnonzero(a["accept"] != b["accept"])
        upto = split[0] + 1 if split.size else steps
        assert np.array_equal(a["k"][:upto], b["k"][:upto])
        assert np.array_equal(a["lnu"][:upto], b["lnu"][:upto])
        d = np.abs(a["dE"][:upto] - b["dE"][:upto])
        assert np.all(d <= de_tol(npairs[:upto], b["dE"][:upto])), c
        if split.size:
            assert abs(b["lnu"][split[0]] + b["dE"][split[0]] / T) <= 1e-3


def test_warp_kernel_limits(amh):
    from paper_2211_03193_gb300._amh import AmhError
    prot = synth.make_protein(20, seed=345)
    tors = synth.random_torsions(2, 20, seed=346)
    for kw in (dict(precision=64), dict(far_pairs=1), dict(stage_table=1),
               dict(threads_per_cta=128), dict(chains_per_cta=4, warps_per_chain=4)):
        with pytest.raises(AmhError):
            amh.Sampler(prot, 2, tors, global_kernel=2, **kw)
    big = synth.make_protein(800, seed=347)
    with pytest.raises(AmhError):
        amh.Sampler(big, 1, synth.random_torsions(1, 800, seed=348), global_kernel=2)
    # longer chains than the warp kernel's chunk bits take the CTA kernel
    with amh.Sampler(big, 2, synth.random_torsions(2, 800, seed=348)) as s:
        assert s.launch_config()[3] == 1
        s.sweep(1, 0, 1.0, 0.1, 50, 1)


def test_pair_term_counters(amh):
    """amh_pair_terms over one global sweep from a sweep boundary: with every
    pair formed (far_pairs = 1) the distances formed are the straddle terms
    of Sec. 2.4 exactly, 4 per pair of each fused proposal pair, sum over p of
    p (L - p) = (L^3 - L) / 6 pairs, so 2 (L^3 - L) / 3 per chain; the FP32
    form reads the entries of fewer (pairs whose images all lie at or past the
    last bin centre are only tested), the FP64 form of all.  The chunk tests
    (far_pairs = 0) form fewer distances but drop only flat pairs, so the
    terms read are the same whenever the two runs take the same decisions."""
    L, chains = 60, 8
    prot = synth.make_protein(L, seed=371)
    tors = synth.random_torsions(chains, L, seed=372)
    n = 2 * L
    dense = 2 * (L ** 3 - L) // 3 * chains
    got = {}
    for prec, far in ((32, 1), (32, 0), (64, 1)):
        with amh.Sampler(prot, chains, tors, precision=prec, far_pairs=far, chains_per_cta=1,
                         threads_per_cta=128) as s:
            e0, f0 = s.pair_terms()
            s.sweep(1, 0, 0.8, 8 * DEG, n, 12)
            e1, f1 = s.pair_terms()
            got[prec, far] = (e1 - e0, f1 - f0, s.torsions())
    ev, fo, th1 = got[32, 1]
    assert fo == dense
    assert 0 < ev < fo
    ev0, fo0, th0 = got[32, 0]
    assert ev0 <= fo0 < dense
    if np.array_equal(th0, th1):
        assert ev0 == ev
    assert got[64, 1][:2] == (dense, dense)


@pytest.mark.parametrize("C,wide,G", [(8, False, 0), (2, False, 0), (4, True, 0), (2, True, 2),
                                      (2, False, 2)])
def test_far_field_skip_equals_dense(amh, orc, C, wide, G):
    """FP32 global sweeps with the flat far field skipped (the default) and
    with every straddle pair evaluated, from the same states and seeds: the
    same Delta-E within FP32 rounding of the different summation order, the
    same decisions up to the first near-tie, and oracle parity (teacher-forced
    replay) for the skipping run.  L=150 from random starts: with the 37
    bins up to 20 A most (moving atom, chunk) items are far; with 64 bins up
    to 66 A most are kept.  G > 0: the skipping run on the chain-group
    kernel (G warps per chain, C chains per CTA) with its three-level filter."""
    L, chains = 150, 16
    edges = np.linspace(2.0, 66.0, 65) if wide else None
    prot = (synth.make_protein(L, edges=edges, sigma_d=2.0, seed=305) if wide
            else synth.make_protein(L, seed=305))
    tors = synth.random_torsions(chains, L, seed=306)
    n = 2 * L
    steps = n + 3
    T, sigma, seed = 0.6, 10 * DEG, 41
    runs = []
    for far in (0, 1):
        # frequent rebuilds keep the FP32 commits' drift inside the replay's
        # tolerance at this length; with 64 bins up to 66 A nearly every
        # straddle pair is inside the table's range, so the drift of the
        # moving side reaches every term and the rebuilds come twice as often
        kw = dict(global_kernel=2, warps_per_chain=G) if (G and far == 0) else {}
        with amh.Sampler(prot, chains, tors, chains_per_cta=C, far_pairs=far,
                         resync_every=30 if wide else 60,
                         trace_chains=chains, trace_capacity=steps, **kw) as s:
            assert s.launch_config()[3] == (2 if kw else 1)
            s.sweep(1, 0, T, sigma, steps, seed)
            th_end, E_end = s.state()[:2]
            runs.append(([s.trace(c) for c in range(chains)], E_end, th_end.reshape(chains, -1)))
    (tf, Ef, thf), (td, Ed, thd) = runs
    # the energy a call ends with (with skipping: flat chunks added from the
    # protein's flat sums) against the oracle's V of the final torsions
    P = orc.Problem(L, prot.p, prot.edges)
    for c in range(chains):
        for E_end, th_end in ((Ef, thf), (Ed, thd)):
            e = P.energy(f64(th_end[c]))
            assert abs(E_end[c] - e) <= 1e-5 * abs(e), c
    k = tf[0]["k"]
    p = (k + 1) // 2
    npairs = p * (L - p)
    for c in range(chains):
        split = np.flatnonzero(tf[c]["accept"] != td[c]["accept"])
        upto = split[0] + 1 if split.size else steps
        d = np.abs(tf[c]["dE"][:upto] - td[c]["dE"][:upto])
        assert np.all(d <= de_tol(npairs[:upto], td[c]["dE"][:upto], reach_of(prot))), c
        if split.size:
            assert abs(td[c]["lnu"][split[0]] + td[c]["dE"][split[0]] / T) <= 1e-3
    for c in (0, 7, 15):
        replay_and_compare(orc, prot, tors[c], tf[c], orc.GLOBAL, 0, T, sigma, 0, seed, c, False)


def test_global_fp64_untouched_trajectory_equals_oracle(amh, orc):
    """FP64 GPU vs oracle without teacher forcing: identical decisions."""
    L = 24
    prot = synth.make_protein(L, seed=310)
    tors = synth.random_torsions(2, L, seed=311)
    steps = 5 * 2 * L
    with amh.Sampler(prot, 2, tors, precision=64, trace_chains=2, trace_capacity=steps) as s:
        s.sweep(1, 0, 0.5, 15 * DEG, steps, 5)
        th = s.torsions()
        P = orc.Problem(L, prot.p, prot.edges)
        for c in range(2):
            tr = s.trace(c)
            send, acc, otr = P.run(f64(tors[c]), orc.GLOBAL, 0, 0.5, 15 * DEG, 0, steps, 5, c,
                                   trace=True)
            margin = np.abs(otr["lnu"] + otr["dV"] / 0.5)
            diff = np.flatnonzero(tr["accept"] != otr["accept"])
            if diff.size:  # only a near-tie may flip a decision (then paths part)
                assert margin[diff[0]] < 1e-5
            else:
                assert np.allclose(th[c], send, atol=1e-6)


@pytest.mark.parametrize("stage", [1, 2, 0])
def test_split_calls_equal_one_call(amh, stage):
    """stage 0: the warp-per-chain kernel."""
    L, chains = 40, 8
    prot = synth.make_protein(L, seed=320)
    tors = synth.random_torsions(chains, L, seed=321)
    outs = []
    kw = (dict(global_kernel=2, chains_per_cta=2, warps_per_chain=2) if stage == 0
          else dict(chains_per_cta=8, stage_table=stage))
    for split in ([170], [33, 1, 136], [80, 90]):
        with amh.Sampler(prot, chains, tors, **kw) as s:
            for st in split:
                s.sweep(1, 0, 0.6, 0.3, st, 7)
            outs.append(s.state()[0])
            assert s.counter(3) == 170
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_dead_torsions_always_accepted(amh):
    L = 10
    prot = synth.make_protein(L, seed=330)
    tors = synth.random_torsions(4, L, seed=331)
    with amh.Sampler(prot, 4, tors, trace_chains=4, trace_capacity=2 * 2 * L) as s:
        s.sweep(1, 0, 1e-6, 0.5, 2 * 2 * L, 3)
        for c in range(4):
            tr = s.trace(c)
            dead = (tr["k"] == 0) | (tr["k"] == 2 * L - 1)
            assert np.all(tr["accept"][dead] == 1) and np.all(tr["dE"][dead] == 0)


@pytest.mark.parametrize("precision,mode,kw", [
    (32, 0, dict(chains_per_cta=2, threads_per_cta=128)),
    (64, 0, dict(chains_per_cta=2, threads_per_cta=128)),
    (32, 1, dict(global_kernel=1, chains_per_cta=2, threads_per_cta=128)),
    (32, 1, dict(global_kernel=2, chains_per_cta=2, warps_per_chain=2)),
    (64, 1, dict(chains_per_cta=2, threads_per_cta=128))])
def test_sched_run_equals_separate_calls(amh, precision, mode, kw):
    """amh_sweeps_sched: a run of sweeps, each at its own T and sigma, in one
    call gives exactly what one call per sweep gives (state, trace, counts).
    The launch shape is fixed so that both contexts sum their energies in the
    same order."""
    from paper_2211_03193_gb300._amh import AmhError, AMH_EINVAL
    L, chains = 30, 6
    n = 2 * L
    prot = synth.make_protein(L, seed=350)
    tors = synth.random_torsions(chains, L, seed=351)
    Ts = [1.5, 0.9, 0.4, 0.2, 0.1]
    Ss = [0.2, 0.15, 0.1, 0.07, 0.05]
    outs = []
    for sched in (False, True):
        with amh.Sampler(prot, chains, tors, precision=precision, trace_chains=chains,
                         trace_capacity=len(Ts) * n, **kw) as s:
            if sched:
                acc = s.sweeps_sched(mode, 8, Ts, Ss, 11)
            else:
                acc = sum(s.sweeps(mode, 8, T, sg, 1, 11) for T, sg in zip(Ts, Ss))
            outs.append((acc, s.state(), [s.trace(c) for c in range(chains)]))
            assert s.counter(0) == len(Ts) * n
            if sched:
                s.sweep(1, 0, 1.0, 0.1, 5, 1)  # off a sweep boundary
                with pytest.raises(AmhError) as ei:
                    s.sweeps_sched(mode, 8, Ts, Ss, 11)
                assert ei.value.status == AMH_EINVAL
    (a0, st0, tr0), (a1, st1, tr1) = outs
    assert np.array_equal(a0, a1)
    for x, y in zip(st0, st1):
        assert np.array_equal(x, y)
    for x, y in zip(tr0, tr1):
        assert np.array_equal(x, y)


def test_sched_run_limits(amh):
    from paper_2211_03193_gb300._amh import AmhError
    prot = synth.make_protein(12, seed=352)
    with amh.Sampler(prot, 2, synth.random_torsions(2, 12, seed=353)) as s:
        for Ts in ([1.0] * 17, [1.0, -1.0], [], [1.0, float("nan")]):
            with pytest.raises(AmhError):
                s.sweeps_sched(0, 8, Ts, [0.1] * len(Ts), 1)
        assert s.counter(0) == 0


# ---------------------------------------------------------------- local sweeps
@pytest.mark.parametrize("precision,window", [(64, 8), (32, 8), (32, 10), (32, 5), (32, 0),
                                              (32, 3)])
def test_local_sweeps_teacher_forced(amh, orc, precision, window):
    L, chains = 29, 6
    prot = synth.make_protein(L, seed=400)
    tors = synth.random_torsions(chains, L, seed=401)
    n = 2 * L
    steps = 2 * n
    T, sigma, seed = 0.3, 20 * DEG, 17
    with amh.Sampler(prot, chains, tors, precision=precision, trace_chains=chains,
                     trace_capacity=steps) as s:
        acc = s.sweep(0, window, T, sigma, steps, seed)
        th = s.torsions()
        for c in range(chains):
            tr = s.trace(c)
            assert tr.shape[0] == steps and acc[c] == tr["accept"].sum()
            d = replay_and_compare(orc, prot, tors[c], tr, orc.LOCAL, window, T, sigma, 0, seed,
                                   c, precision == 64)
            if precision == 64:
                assert d["disagree"] == 0
                assert np.allclose(th[c], d["s_end"], atol=1e-6)


def test_local_full_window_equals_global_fp64(amh):
    """d >= 2n: a local sweep is a global sweep (same visits, same draws)."""
    L = 8
    prot = synth.make_protein(L, seed=410)
    tors = synth.random_torsions(3, L, seed=411)
    res = []
    for mode, window in ((1, 0), (0, 2 * 2 * L)):
        with amh.Sampler(prot, 3, tors, precision=64) as s:
            s.sweep(mode, window, 0.7, 0.35, 4 * 2 * L, 21)
            res.append(s.torsions())
    assert np.allclose(res[0], res[1], atol=1e-9)


def test_local_requires_whole_sweeps(amh):
    from paper_2211_03193_gb300._amh import AmhError
    prot = synth.make_protein(6, seed=420)
    with amh.Sampler(prot, 2, synth.random_torsions(2, 6, seed=1)) as s:
        with pytest.raises(AmhError):
            s.sweep(0, 8, 1.0, 0.1, 5, 1)
        s.sweep(1, 0, 1.0, 0.1, 5, 1)
        with pytest.raises(AmhError):
            s.sweep(0, 8, 1.0, 0.1, 12, 1)
        with pytest.raises(AmhError):
            s.sweep(0, 66, 1.0, 0.1, 12, 1)


# ---------------------------------------------------------------- gradient
@pytest.mark.parametrize("precision", [32, 64])
def test_grad_matches_oracle(amh, orc, precision):
    import torch
    L, batch = 45, 6
    prot = synth.make_protein(L, seed=500)
    tors = synth.random_torsions(batch, L, seed=501)
    dt = torch.float32 if precision == 32 else torch.float64
    with amh.Sampler(prot, 1, tors[:1], precision=precision) as s:
        th = torch.tensor(tors, dtype=dt, device="cuda")
        E, g = s.grad(0, th)
        E, g = E.cpu().numpy(), g.cpu().numpy()
    P = orc.Problem(L, prot.p, prot.edges)
    for b in range(batch):
        Vo, go = P.grad(f64(tors[b]))
        if precision == 32:
            assert abs(E[b] - Vo) <= 1e-5 * abs(Vo)
            assert np.linalg.norm(g[b] - go) <= 1e-3 * np.linalg.norm(go)
        else:
            assert abs(E[b] - Vo) <= 1e-11 * abs(Vo)
            assert np.linalg.norm(g[b] - go) <= 1e-9 * np.linalg.norm(go)
        assert g[b][0] == 0 and g[b][-1] == 0


# ---------------------------------------------------------------- noisy restart
def test_state_change_energy_on_read(amh, orc):
    """After amh_set_state or a noisy restart, V is computed when next read
    (or by a global sweep): the energies read back are always the oracle's
    V of the torsions read back, with or without sweeps in between."""
    L, chains = 40, 4
    prot = synth.make_protein(L, seed=520)
    tors = synth.random_torsions(chains, L, seed=521)
    new = synth.random_torsions(chains, L, seed=522)
    P = orc.Problem(L, prot.p, prot.edges)

    def check(s):
        th, E = s.state()[:2]
        th = th.reshape(chains, -1)
        for c in range(chains):
            e = P.energy(f64(th[c]))
            assert abs(E[c] - e) <= 1e-5 * abs(e), c
        return th

    with amh.Sampler(prot, chains, tors) as s:
        s.set_state(np.asarray(new, dtype=np.float32).ravel())
        th = check(s)
        assert np.array_equal(th, np.asarray(new, dtype=np.float32))
        s.set_state(np.asarray(tors, dtype=np.float32).ravel())
        s.sweeps(0, 8, 1.0, 10 * DEG, 1, 3)   # a local sweep leaves V to the read
        check(s)
        s.noisy_restart(0.2, 5)
        s.sweeps(1, 0, 1.0, 10 * DEG, 1, 3)   # a global sweep ends with V
        check(s)
        s.noisy_restart(0.2, 6)
        check(s)


def test_noisy_restart_matches_oracle(amh, orc):
    L, chains = 12, 5
    prot = synth.make_protein(L, seed=600)
    tors = synth.random_torsions(chains, L, seed=601)
    with amh.Sampler(prot, chains, tors, precision=64) as s:
        s.noisy_restart(30 * DEG, 77)
        th = s.torsions()
        E = s.state()[1]
    P = orc.Problem(L, prot.p, prot.edges)
    for c in range(chains):
        want = orc.noisy_restart(f64(tors[c]), 30 * DEG, 77, c)
        assert np.allclose(th[c], want, atol=2e-7)  # FP32 interface rounding
        assert abs(E[c] - P.energy(want)) <= 1e-10 * abs(E[c])


# ---------------------------------------------------------------- sampler law
def test_global_mh_on_gpu_samples_exact_boltzmann(amh, orc):
    """Lattice toy (L=4, K=4): the GPU's global MH visits states with
    frequency exp(-V/T)/Z (Eq. 1), Z by enumeration with the oracle."""
    import itertools
    L, K = 4, 4
    prot = synth.make_protein(L, seed=21)
    P = orc.Problem(L, prot.p, prot.edges)
    n = 2 * L
    q = 2 * np.pi / K
    live = list(range(1, n - 1))
    grid = np.array(list(itertools.product(range(K), repeat=len(live))))
    S = np.zeros((grid.shape[0], n))
    S[:, live] = np.angle(np.exp(1j * grid * q))
    E = P.energies(S)
    T = float(np.std(E))
    w = np.exp(-(E - E.min()) / T)
    pi = w / w.sum()
    chains = 4096
    tors = np.zeros((chains, n), np.float32)
    with amh.Sampler(prot, chains, tors, precision=64, lattice_K=K) as s:
        s.sweep(1, 0, T, 1.2, 40 * n, 3)  # burn-in
        counts = np.zeros(K ** len(live))
        for rep in range(150):
            s.sweep(1, 0, T, 1.2, n, 3)
            th = s.torsions()
            m = np.mod(np.rint(th[:, live] / q).astype(np.int64), K)
            idx = (m * K ** np.arange(len(live) - 1, -1, -1)).sum(1)
            counts += np.bincount(idx, minlength=K ** len(live))
    gidx = (np.mod(grid, K) * K ** np.arange(len(live) - 1, -1, -1)).sum(1)
    pi_sorted = pi[np.argsort(gidx)]
    hist = counts / counts.sum()
    tv = 0.5 * np.abs(hist - pi_sorted).sum()
    tv_noise = 0.5 * np.sum(np.sqrt(2 * pi_sorted * (1 - pi_sorted) / (np.pi * counts.sum())))
    assert tv < 1.5 * tv_noise, (tv, tv_noise)
