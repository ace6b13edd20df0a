"""Parity at the workload configurations: the FP64 single chain (exact
trajectory), the bench's L=300 / 1024-chain launch (sampled chains), 64
proteins of uneven length in one context, L=500 with 64 bins (FP32 against
the FP64 GPU form), and the differentiable L=300 / 512-vector batch.
Expected values come from the oracle only."""
import math

import numpy as np
import pytest

from paper_2211_03193_gb300 import synth
from test_gpu_parity import gpu_advance, replay_and_compare

pytestmark = pytest.mark.gpu
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


def test_fp64_single_chain_amh_trajectory_equals_oracle(amh, orc):
    """L=64, one chain, FP64, sigma 15 deg, d=8, T=1, 10 local : 1 global:
    156 whole sweeps (19 968 proposals; a local sweep cannot stop part-way).
    No teacher forcing: every decision must match the oracle's."""
    L = 64
    n = 2 * L
    prot = synth.make_protein(L, seed=1000)
    tors = synth.random_torsions(1, L, seed=8)
    sweeps = 156
    sigma, T, d = 15 * DEG, 1.0, 8
    P = orc.Problem(L, prot.p, prot.edges)
    s_orc = tors[0].astype(np.float64)
    with amh.Sampler(prot, 1, tors, precision=64, trace_chains=1,
                     trace_capacity=sweeps * n) as s:
        trs = []
        for q in range(sweeps):
            mode = 0 if q % 11 < 10 else 1
            s.sweeps(mode, d, T, sigma, 1, 3)
            s_orc, _, tr = P.run(s_orc, orc.LOCAL if mode == 0 else orc.GLOBAL, d, T, sigma,
                                 q * n, n, 3, 0, trace=True)
            trs.append(tr)
        gt = s.trace(0)
        ot = np.concatenate(trs)
        assert gt.shape[0] == sweeps * n
        diff = np.flatnonzero(gt["accept"] != ot["accept"])
        if diff.size:
            j = diff[0]
            assert abs(ot["lnu"][j] + ot["dV"][j] / T) < 1e-5, j
        else:
            assert np.allclose(s.torsions()[0], s_orc, atol=1e-6)
            assert np.allclose(gt["dE"], ot["dV"], atol=1e-8, rtol=1e-9)
        # a local sweep leaves the stored energy at the last global sweep's:
        # recompute it
        E = s.energy()
        assert abs(E[0] - P.energy(s_orc)) <= 1e-10 * abs(E[0])


def test_bench_workload_sampled_parity(amh, orc):
    """L=300, 1024 chains, the autotuned launch shape the bench times, one AMH
    cycle of the bench schedule; chains 0-2 traced and replayed by the oracle,
    eight chains' end energies recomputed by the oracle."""
    import bench
    w = bench.workload("amh_L300_c1024")
    L, n, chains = w["L"], w["n"], w["chains"]
    prot = synth.make_protein(L, edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    tors = synth.random_torsions(chains, L, seed=w["start_seed"])
    sched = bench.schedule_for(w, seed=1)
    P = orc.Problem(L, prot.p, prot.edges)
    with amh.Sampler(prot, chains, tors, trace_chains=3, trace_capacity=w["cycle"] * n) as s:
        for q in range(w["cycle"]):
            mode, T, sigma = sched.params(q)
            s.sweeps(mode, w["window"], T, sigma, 1, sched.seed)
        th, E, bE, _ = s.state()
        th = th.reshape(chains, n)
        for c in range(3):
            tr = s.trace(c)
            st = gst = tors[c]
            for q in range(w["cycle"]):
                mode, T, sigma = sched.params(q)
                seg = tr[q * n:(q + 1) * n]
                d = replay_and_compare(orc, prot, st, seg, orc.LOCAL if mode == 0 else orc.GLOBAL,
                                       w["window"], T, sigma, q * n, sched.seed, c, False,
                                       gpu_s0=gst)
                st = d["s_end"]
                gst = gpu_advance(gst, seg)
                print("chain %d sweep %d (%s, T=%.3f): flips %d ties %d max |dE err| %.3g" % (
                    c, q, "local" if mode == 0 else "global", T, d["flips"], d["ties"],
                    d["max_dE_err"]))
            assert np.allclose(np.angle(np.exp(1j * (th[c] - st))), 0, atol=1e-4)
    for c in (0, 1, 255, 256, 511, 640, 1022, 1023):
        e = P.energy(th[c].astype(np.float64))
        assert abs(E[c] - e) <= 1e-5 * abs(e), c
        assert bE[c] <= E[c] + 1e-9


def test_bench_workload_anneal_tail_parity(amh, orc):
    """The end of the L=300 / 1024-chain anneal, where the optimisation's
    decisions are made: every chain runs the whole schedule (333 sweeps, T
    2.0 -> 0.05, sigma 10 -> 4 deg, Sec. 3's annealing); from the states it
    ends in, a traced context on the autotuned launch shape runs one more
    cycle with the parameters of the schedule's last full cycle (T ~ 0.05,
    sigma ~ 4 deg), and the oracle replays three chains teacher-forced.  No
    decision may differ from the exact one beyond the contract's 1e-5 tie
    margin (FP32 rounding flips: none)."""
    import bench
    w = bench.workload("amh_L300_c1024")
    L, n, chains = w["L"], w["n"], w["chains"]
    prot = synth.make_protein(L, edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    tors = synth.random_torsions(chains, L, seed=w["start_seed"])
    sched = bench.schedule_for(w, seed=1)
    with amh.Sampler(prot, chains, tors) as s:
        amh.run_schedule(s, sched)
        th_end = s.torsions()
        E_end = s.state()[1]
    cyc = w["cycle"]
    last = (sched.total_sweeps // cyc) * cyc - cyc  # first sweep of the last full cycle
    params = [sched.params(last + q) for q in range(cyc)]
    assert params[-1][0] == 1 and params[-1][1] < 0.06 and params[-1][2] < math.radians(4.1)
    stats = []
    with amh.Sampler(prot, chains, th_end, trace_chains=3, trace_capacity=cyc * n) as s:
        for mode, T, sigma in params:
            s.sweeps(mode, w["window"], T, sigma, 1, 77)
        tr_all = [s.trace(c) for c in range(3)]
        C = s.launch_config()
    for c in range(3):
        tr = tr_all[c]
        st = gst = th_end[c]
        for q, (mode, T, sigma) in enumerate(params):
            seg = tr[q * n:(q + 1) * n]
            d = replay_and_compare(orc, prot, st, seg, orc.LOCAL if mode == 0 else orc.GLOBAL,
                                   w["window"], T, sigma, q * n, 77, c, False, gpu_s0=gst)
            st = d["s_end"]
            gst = gpu_advance(gst, seg)
            stats.append((mode, d["flips"], d["ties"], d["max_dE_err"],
                          float(np.max(d["dE_err"] / np.maximum(d["npairs"], 1)))))
    flips = sum(x[1] for x in stats)
    print("anneal tail (T=%.4f, sigma=%.2f deg, launch %r): E_end median %.1f; flips %d, ties %d;"
          " max |dE err| local %.3g global %.3g; per straddle pair (global) %.3g" % (
              params[-1][1], math.degrees(params[-1][2]), C, float(np.median(E_end)), flips,
              sum(x[2] for x in stats), max(x[3] for x in stats if x[0] == 0),
              max(x[3] for x in stats if x[0] == 1), max(x[4] for x in stats if x[0] == 1)))
    assert flips == 0


def test_uneven_proteins_one_context(amh, orc):
    """64 proteins, L uniform in [50, 400], 256 chains each (16 384 chains):
    one local and one global sweep per chain through the persistent queue."""
    Ls = synth.uneven_lengths(64, 50, 400, seed=3)
    prots = [synth.make_protein(L, seed=2000 + i) for i, L in enumerate(Ls)]
    chains = [256] * 64
    tors = np.concatenate([synth.random_torsions(256, L, seed=3000 + i).ravel()
                           for i, L in enumerate(Ls)])
    T, sigma = 1.0, 10 * DEG
    with amh.Sampler(prots, chains, tors, trace_chains=2, trace_capacity=4 * Ls[0]) as s:
        s.sweeps(0, 8, T, sigma, 1, 9)
        s.sweeps(1, 0, T, sigma, 1, 9)
        th, E, bE, _ = s.state()
        for c in range(2):
            tr = s.trace(c)
            n0 = 2 * Ls[0]
            d = replay_and_compare(orc, prots[0], tors[c * n0:(c + 1) * n0], tr[:n0], orc.LOCAL,
                                   8, T, sigma, 0, 9, c, False)
            replay_and_compare(orc, prots[0], d["s_end"], tr[n0:], orc.GLOBAL, 0, T, sigma, n0,
                               9, c, False,
                               gpu_s0=gpu_advance(tors[c * n0:(c + 1) * n0], tr[:n0]))
        for p in (0, 7, 21, 40, 63):
            off = s.offsets[p]
            n = prots[p].n
            P = orc.Problem(prots[p].L, prots[p].p, prots[p].edges)
            for c in (0, 255):
                chain = 256 * p + c
                assert s.counter(chain) == 2 * n
                e = P.energy(th[off + c * n: off + (c + 1) * n].astype(np.float64))
                assert abs(E[chain] - e) <= 1e-5 * abs(e)


def test_l500_64bins_fp32_against_fp64(amh, orc):
    """L=500, 4096 chains, 64 bins of 0.3125 A (sigma_d 1.5 A): after two
    local and one global FP32 sweep, the FP32 energies agree with the FP64
    GPU form's energies of the same states to 1e-4 relative, and both with
    the oracle on sampled chains."""
    L, chains = 500, 4096
    prot = synth.make_protein(L, edges=synth.edges_uniform_64(), sigma_d=1.5, seed=1000)
    tors = synth.random_torsions(chains, L, seed=12)
    with amh.Sampler(prot, chains, tors) as s32:
        s32.sweeps(0, 8, 1.0, 8 * DEG, 2, 5)
        s32.sweeps(1, 0, 1.0, 8 * DEG, 1, 5)
        th, E32, _, _ = s32.state()
    with amh.Sampler(prot, chains, th, precision=64) as s64:
        E64 = s64.energy()
    rel = np.abs(E32 - E64) / np.abs(E64)
    i = int(np.nanargmax(rel))
    assert np.all(rel <= 1e-4), (i, E32[i], E64[i], rel[i], int(np.isnan(E32).sum()))
    P = orc.Problem(L, prot.p, prot.edges)
    th = th.reshape(chains, 2 * L)
    for c in (0, 2047, 4095):
        e = P.energy(th[c].astype(np.float64))
        assert abs(E64[c] - e) <= 1e-11 * abs(e)
        assert abs(E32[c] - e) <= 1e-5 * abs(e)


def test_differentiable_l300_batch512(amh, orc):
    """L=300, 512 torsion vectors: the FP32 energies and dV/ds of all 512 in
    one call; sampled vectors against the oracle's FP64 energy and gradient,
    and sampled components against the oracle's central differences (h =
    1e-4 rad; the analytic derivative lies between the left and right
    differences, which differ where a pair distance crosses a bin centre
    within +-h).  Then the hand-off: a short AMH run, the best 32 states
    through L-BFGS; every state's energy drops and matches the oracle's at
    the end."""
    import torch
    from paper_2211_03193_gb300 import autograd
    w = synth.WORKLOADS["grad_L300_b512"]
    L, batch = w["L"], w["batch"]
    n = 2 * L
    prot = synth.make_protein(L, edges=synth.edges_by_name(w["bins"]), sigma_d=w["sigma_d"],
                              seed=w["seed"])
    tors = synth.random_torsions(batch, L, seed=w["start_seed"])
    P = orc.Problem(L, prot.p, prot.edges)
    with amh.Sampler(prot, 1, tors[:1]) as s:
        th = torch.tensor(tors, device="cuda")
        E, g = s.grad(0, th)
        E, g = E.cpu().numpy(), g.cpu().numpy()
        rng = np.random.default_rng(5)
        h = 1e-4
        for b in (0, 1, 200, 511):
            sb = tors[b].astype(np.float64)
            Vo, go = P.grad(sb)
            assert abs(E[b] - Vo) <= 1e-5 * abs(Vo)
            assert np.linalg.norm(g[b] - go) <= 1e-3 * np.linalg.norm(go)
            tol_g = 2e-3 * np.linalg.norm(go) / math.sqrt(n)
            for k in rng.choice(np.arange(1, n - 1), 24, replace=False):
                sp, sm = sb.copy(), sb.copy()
                sp[k] += h
                sm[k] -= h
                V0, Vp, Vm = P.energy(sb), P.energy(sp), P.energy(sm)
                right, left = (Vp - V0) / h, (V0 - Vm) / h
                tol = tol_g + 1e-3 * max(abs(left), abs(right))
                assert min(left, right) - tol <= g[b][k] <= max(left, right) + tol, (b, k)
    # hand-off: AMH, then L-BFGS on the best 32 states
    chains = 256
    starts = synth.random_torsions(chains, L, seed=w["start_seed"] + 1)
    with amh.Sampler(prot, chains, starts) as s:
        for q in range(11):
            s.sweeps(0 if q < 10 else 1, 8, 1.0, 10 * DEG, 1, 3)
        th, E0, _, _ = s.state()
        best = np.argsort(E0)[:32]
        th0 = torch.tensor(th.reshape(chains, n)[best], device="cuda")
        thL, EL = autograd.lbfgs_refine(s, th0, iterations=500)
        EL = EL.cpu().numpy()
    assert np.all(EL < E0[best])
    for b in (0, 17, 31):
        e = P.energy(thL[b].cpu().numpy().astype(np.float64))
        assert abs(EL[b] - e) <= 1e-5 * abs(e)
