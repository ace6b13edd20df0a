"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, brute force on tiny inputs, an independently written
dihedral formula, or exact enumeration.  None needs a GPU.
"""
import os

import numpy as np
import pytest

from paper_2211_03193_gb300 import synth

DEG = np.pi / 180.0


def dihedral(p0, p1, p2, p3):
    """Independent dihedral formula (atan2 of projected bond vectors)."""
    b0 = p0 - p1
    b1 = p2 - p1
    b2 = p3 - p2
    b1n = b1 / np.linalg.norm(b1)
    v = b0 - np.dot(b0, b1n) * b1n
    w = b2 - np.dot(b2, b1n) * b1n
    return np.arctan2(np.dot(np.cross(b1n, v), w), np.dot(v, w))


def angle(a, b, c):
    u, v = a - b, c - b
    return np.arccos(np.dot(u, v) / np.linalg.norm(u) / np.linalg.norm(v))


def wrapd(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def small_problem(L, seed=5, edges=None, sigma_d=1.0):
    return synth.make_protein(L, edges=edges, sigma_d=sigma_d, seed=seed)


# ---------------------------------------------------------------- G(s)
def test_nerf_recovers_ideal_geometry_and_torsions(orc):
    """Sec. 2.1 / Eq. 3: G(s) reproduces bonds, angles, omega and every live torsion."""
    rng = np.random.default_rng(1)
    L = 24
    s = rng.uniform(-np.pi, np.pi, 2 * L)
    c = orc.build_coords(s)
    N, CA, C, CB = c["N"], c["CA"], c["C"], c["CB"]
    for i in range(L):
        assert abs(np.linalg.norm(CA[i] - N[i]) - 1.458) < 1e-10
        assert abs(np.linalg.norm(C[i] - CA[i]) - 1.525) < 1e-10
        assert abs(angle(N[i], CA[i], C[i]) - 111.2 * DEG) < 1e-10
        assert abs(np.linalg.norm(CB[i] - CA[i]) - 1.52) < 1e-10
        assert abs(angle(C[i], CA[i], CB[i]) - 109.5 * DEG) < 1e-10
        assert abs(wrapd(dihedral(N[i], C[i], CA[i], CB[i]) - 122.6 * DEG)) < 1e-10
        if i + 1 < L:
            assert abs(np.linalg.norm(N[i + 1] - C[i]) - 1.329) < 1e-10
            assert abs(angle(CA[i], C[i], N[i + 1]) - 116.2 * DEG) < 1e-10
            assert abs(angle(C[i], N[i + 1], CA[i + 1]) - 121.7 * DEG) < 1e-10
            # psi_i, omega_i, phi_{i+1}
            assert abs(wrapd(dihedral(N[i], CA[i], C[i], N[i + 1]) - s[2 * i + 1])) < 1e-10
            assert abs(wrapd(dihedral(CA[i], C[i], N[i + 1], CA[i + 1]) - np.pi)) < 1e-10
            assert abs(wrapd(dihedral(C[i], N[i + 1], CA[i + 1], C[i + 1]) - s[2 * i + 2])) < 1e-10


def test_nerf_all_trans_is_planar_zigzag(orc):
    """All torsions 180 deg: the backbone stays in the plane of the first residue
    and is a planar zig-zag that repeats with one fixed translation every two
    residues (a glide), C-beta alternating above and below the plane."""
    L = 12
    s = np.full(2 * L, np.pi)
    c = orc.build_coords(s)
    bb = np.concatenate([c["N"], c["CA"], c["C"]])
    assert np.max(np.abs(bb[:, 2])) < 1e-10
    step = c["CA"][2] - c["CA"][0]
    for i in range(L - 2):
        for nm in ("N", "CA", "C", "CB"):
            assert np.allclose(c[nm][i + 2] - c[nm][i], step, atol=1e-10)
    zc = c["CB"][:, 2]
    assert np.allclose(zc[0::2], zc[0], atol=1e-10) and np.allclose(zc[1::2], -zc[0], atol=1e-10)
    assert abs(zc[0]) > 0.5
    # dead torsions phi_0 and psi_{L-1} move nothing
    s2 = s.copy()
    s2[0] = 0.3
    s2[-1] = -1.1
    c2 = orc.build_coords(s2)
    for nm in ("N", "CA", "C", "CB"):
        assert np.array_equal(c[nm], c2[nm])


def test_pivot_rotation_moves_exactly_far_side(orc):
    """Sec. 2.4 step 2: changing phi_i moves C-beta i.. L-1; psi_i moves i+1.. L-1,
    rigidly (the pivot p(k) = ceil(k/2) used by the straddle block)."""
    rng = np.random.default_rng(2)
    L = 16
    s = rng.uniform(-np.pi, np.pi, 2 * L)
    cb = orc.build_coords(s)["CB"]
    for k in range(1, 2 * L - 1):
        s2 = s.copy()
        s2[k] += 0.7
        cb2 = orc.build_coords(s2)["CB"]
        p = (k + 1) // 2
        assert np.allclose(cb2[:p], cb[:p], atol=1e-12)
        assert not np.allclose(cb2[p:], cb[p:], atol=1e-6)
        D = np.linalg.norm(cb[p:, None] - cb[None, p:], axis=-1)
        D2 = np.linalg.norm(cb2[p:, None] - cb2[None, p:], axis=-1)
        assert np.allclose(D, D2, atol=1e-10)


# ---------------------------------------------------------------- V(x)
def test_pair_term_at_centres_and_flat_ends(orc):
    """Eq. 5 term: -ln p at each centre, linear between, flat outside."""
    prot = small_problem(6)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    c = P.centres()
    assert np.allclose(c[:36], 2.25 + 0.5 * np.arange(36))
    assert abs(c[36] - 20.25) < 1e-12
    a, b = 1, 4
    r = a * prot.L - a * (a + 1) // 2 + (b - a - 1)
    E = -np.log(prot.p[r])
    for j in range(prot.B):
        assert abs(P.pair_term(a, b, c[j]) - E[j]) < 1e-12
    for j in range(prot.B - 1):
        mid = 0.5 * (c[j] + c[j + 1])
        assert abs(P.pair_term(a, b, mid) - 0.5 * (E[j] + E[j + 1])) < 1e-12
    assert P.pair_term(a, b, 0.3) == E[0]
    assert P.pair_term(a, b, 55.0) == E[-1]


def test_one_hot_table_is_a_hat_function(orc):
    """p one-hot at bin j0 (others floored at 1e-300): e(d) is 0 at c_j0 and rises
    linearly to 300 ln 10 at the neighbouring centres."""
    L, B = 3, 37
    edges = synth.edges_af1_37()
    j0 = 10
    p = np.zeros((3, B))
    p[:, j0] = 1.0
    P = orc.Problem(L, p, edges)
    top = 300 * np.log(10.0)
    c0 = 2.25 + 0.5 * j0
    for d in np.linspace(0.0, 25.0, 501):
        hat = top * min(1.0, abs(d - c0) / 0.5)
        assert abs(P.pair_term(0, 2, d) - hat) < 1e-9


def test_row_order_matches_triu(orc):
    """Row r(a,b) = a L - a(a+1)/2 + (b-a-1) is numpy's triu order."""
    L, B = 9, 37
    rows = L * (L - 1) // 2
    vals = np.exp(-np.arange(1, rows + 1) / 7.0)
    p = np.repeat(vals[:, None], B, axis=1)
    P = orc.Problem(L, p, synth.edges_af1_37())
    ia, ib = np.triu_indices(L, 1)
    for r, (a, b) in enumerate(zip(ia, ib)):
        assert abs(P.pair_term(int(a), int(b), 7.7) + np.log(vals[r])) < 1e-12


def test_uniform_table_energy_counts_pairs(orc):
    """p uniform over B bins: every term is ln B, so V = L(L-1)/2 ln B."""
    L, B = 17, 37
    p = np.full((L * (L - 1) // 2, B), 1.0 / B)
    P = orc.Problem(L, p, synth.edges_af1_37())
    s = np.random.default_rng(3).uniform(-np.pi, np.pi, 2 * L)
    assert abs(P.energy(s) - L * (L - 1) / 2 * np.log(B)) < 1e-9


def test_energy_rigid_motion_invariant(orc):
    prot = small_problem(20)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    s = np.random.default_rng(4).uniform(-np.pi, np.pi, prot.n)
    cb = orc.build_coords(s)["CB"]
    q, _ = np.linalg.qr(np.random.default_rng(5).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    cb2 = cb @ q.T + np.array([3.0, -7.0, 11.0])
    e1, e2 = P.energy_cb(cb), P.energy_cb(cb2)
    assert abs(e1 - e2) <= 1e-12 * abs(e1)


def test_af1_layout_roundtrip_same_energy(orc):
    """Storing the open bin first (AlphaFold1 order) and restoring it is lossless."""
    prot = small_problem(10)
    p2 = synth.from_af1_layout(synth.to_af1_layout(prot.p))
    assert np.array_equal(p2, prot.p)
    s = np.random.default_rng(6).uniform(-np.pi, np.pi, prot.n)
    assert orc.Problem(prot.L, p2, prot.edges).energy(s) == orc.Problem(prot.L, prot.p, prot.edges).energy(s)


def test_pivot_block_equals_brute_force_difference(orc):
    """Only pairs a < p(k) <= b change distance: the straddle-block sum equals
    V(G(s')) - V(G(s)) for every k, including the dead phi_0 and psi_{L-1}."""
    prot = small_problem(12)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    rng = np.random.default_rng(7)
    s = rng.uniform(-np.pi, np.pi, prot.n)
    cb = orc.build_coords(s)["CB"]
    for k in range(prot.n):
        s2 = s.copy()
        s2[k] = wrapd(s2[k] + rng.normal(0, 0.5))
        cb2 = orc.build_coords(s2)["CB"]
        p = (k + 1) // 2
        blk = 0.0
        for a in range(p):
            for b in range(max(p, a + 1), prot.L):
                blk += P.pair_term(a, b, np.linalg.norm(cb2[a] - cb2[b])) - \
                    P.pair_term(a, b, np.linalg.norm(cb[a] - cb[b]))
        brute = P.energy(s2) - P.energy(s)
        assert abs(blk - brute) < 1e-9 * (1 + abs(brute))
        if k in (0, prot.n - 1):
            assert brute == 0.0


# ---------------------------------------------------------------- V_local
def test_local_window_clip_and_full_window(orc):
    """Eq. 6: d >= 2n covers the chain, so V_local = V; windows clip at the ends."""
    prot = small_problem(10)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    s = np.random.default_rng(8).uniform(-np.pi, np.pi, prot.n)
    cb = orc.build_coords(s)["CB"]
    V = P.energy_cb(cb)
    for k in range(prot.n):
        assert abs(P.energy_local_cb(cb, k, 2 * prot.n) - V) < 1e-12 * abs(V)
    # k = 1 -> residue 0, d = 4 -> residues [0, 2]
    want = sum(P.pair_term(a, b, np.linalg.norm(cb[a] - cb[b])) for a in range(3) for b in range(a + 1, 3))
    assert abs(P.energy_local_cb(cb, 1, 4) - want) < 1e-12
    # k = 2L-2 -> residue L-1, d = 6 -> residues [L-4, L-1]
    lo = prot.L - 4
    want = sum(P.pair_term(a, b, np.linalg.norm(cb[a] - cb[b])) for a in range(lo, prot.L) for b in range(a + 1, prot.L))
    assert abs(P.energy_local_cb(cb, prot.n - 2, 6) - want) < 1e-12


def test_same_colour_local_moves_commute(orc):
    """Moves whose windows have disjoint torsion sets do not see each other:
    the local Delta-V of k2 is unchanged when k1 (same colour) is applied."""
    prot = small_problem(30)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    rng = np.random.default_rng(9)
    s = rng.uniform(-np.pi, np.pi, prot.n)
    d = 8
    h = d // 2
    ncol = 4 * h
    for k1 in range(0, prot.n - ncol):
        k2 = k1 + ncol
        def dvl(state, k, delta):
            st2 = state.copy()
            st2[k] += delta
            return P.energy_local_cb(orc.build_coords(st2)["CB"], k, d) - \
                P.energy_local_cb(orc.build_coords(state)["CB"], k, d)
        before = dvl(s, k2, 0.4)
        s1 = s.copy()
        s1[k1] += -0.9
        after = dvl(s1, k2, 0.4)
        assert abs(before - after) < 1e-10 * (1 + abs(before))


def test_local_mode_with_full_window_is_global_mode(orc):
    """d >= 2n makes every colour a single torsion in ascending order and
    V_local = V, so a local sweep is a global sweep (same seed, same decisions)."""
    prot = small_problem(8)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    s0 = np.random.default_rng(10).uniform(-np.pi, np.pi, prot.n)
    steps = 4 * prot.n
    sg, ag, tg = P.run(s0, orc.GLOBAL, 0, 0.7, 20 * DEG, 0, steps, 77, 3, trace=True)
    sl, al, tl = P.run(s0, orc.LOCAL, 2 * prot.n, 0.7, 20 * DEG, 0, steps, 77, 3, trace=True)
    assert ag == al
    assert np.array_equal(tg["k"], tl["k"])
    assert np.array_equal(tg["accept"], tl["accept"])
    assert np.allclose(tg["dV"], tl["dV"], atol=1e-9)
    assert np.allclose(sg, sl, atol=0)


def test_local_colour_order_and_counter(orc):
    """Local sweeps visit k by colour (k mod 4h) and draw from Philox index
    q n + k regardless of the visiting order."""
    prot = small_problem(10)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    s0 = np.random.default_rng(11).uniform(-np.pi, np.pi, prot.n)
    n = prot.n
    _, _, tr = P.run(s0, orc.LOCAL, 8, 1.0, 10 * DEG, n, 2 * n, 5, 9, trace=True)
    order = [k for r in range(16) for k in range(r, n, 16)]
    assert list(tr["k"][:n]) == order and list(tr["k"][n:]) == order
    for j in (0, 5, n + 3):
        q = 1 + j // n
        _, z, u = orc.draw(5, 9, q * n + int(tr["k"][j]))
        assert tr["z"][j] == z and tr["lnu"][j] == np.log(u)


def test_split_runs_equal_one_run(orc):
    """The proposal counter continues across calls (exact resume)."""
    prot = small_problem(9)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    s0 = np.random.default_rng(12).uniform(-np.pi, np.pi, prot.n)
    a, _, _ = P.run(s0, orc.GLOBAL, 0, 0.5, 0.2, 0, 50, 3, 1)
    b, _, _ = P.run(s0, orc.GLOBAL, 0, 0.5, 0.2, 0, 21, 3, 1)
    b, _, _ = P.run(b, orc.GLOBAL, 0, 0.5, 0.2, 21, 29, 3, 1)
    assert np.array_equal(a, b)


def test_teacher_forcing_follows_given_decisions(orc):
    prot = small_problem(8)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    s0 = np.random.default_rng(13).uniform(-np.pi, np.pi, prot.n)
    steps = 3 * prot.n
    forced = np.zeros(steps, np.uint8)
    s1, acc, tr = P.run(s0, orc.GLOBAL, 0, 1.0, 0.3, 0, steps, 4, 0, trace=True, forced=forced)
    assert acc == 0 and np.array_equal(s1, s0)
    forced[:] = 1
    s2, acc, tr = P.run(s0, orc.GLOBAL, 0, 1.0, 0.3, 0, steps, 4, 0, trace=True, forced=forced)
    assert acc == steps
    assert np.allclose(s2, tr["theta_new"][-prot.n:])


# ---------------------------------------------------------------- RNG
def test_synthetic_native_has_low_energy(orc):
    """The data model behind the synthetic distograms: each pair's bin
    probabilities peak at the hidden native trace's distance, so V of the
    native C-betas (Eq. 5 on coordinates) lies far below V of random chain
    starts, and below V of the native with its residues shuffled (the same
    bond geometry, the wrong distances)."""
    L = 80
    prot = synth.make_protein(L, seed=1234)
    P = orc.Problem(L, prot.p, prot.edges)
    e_native = P.energy_cb(prot.native)
    starts = synth.random_torsions(8, L, seed=77).astype(np.float64)
    e_random = P.energies(starts)
    assert e_native < 0.5 * e_random.min(), (e_native, e_random.min())
    rng = np.random.default_rng(5)
    e_shuffled = P.energy_cb(prot.native[rng.permutation(L)])
    assert e_native < 0.5 * e_shuffled, (e_native, e_shuffled)


def test_philox_known_answers(orc):
    """The oracle's Philox4x32-10 reproduces the generator's published
    known-answer vectors (tests/golden/philox4x32_10_kat.txt): a wrong
    multiplier, Weyl constant, round count or word order fails every row."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        got = orc.philox(v[0:4], v[4:6])
        assert [int(x) for x in got] == v[6:10], (r, ["%08x" % x for x in got])


def test_philox_words_are_uniform_and_decorrelated(orc):
    words = np.array([orc.philox((c, 7, 0, 0), (123, 456)) for c in range(20000)])
    bytes_ = words.view(np.uint8).ravel()
    cnt = np.bincount(bytes_, minlength=256)
    exp = bytes_.size / 256
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert 180 < chi2 < 340  # 255 dof
    for w in range(4):
        bits = (words[:, w, None] >> np.arange(32)) & 1
        assert np.all(np.abs(bits.mean(0) - 0.5) < 0.02)
    f = words.astype(np.float64) / 2 ** 32
    cc = np.corrcoef(f.T)
    assert np.max(np.abs(cc - np.eye(4))) < 0.03
    assert abs(np.corrcoef(f[:-1, 0], f[1:, 0])[0, 1]) < 0.03
    # the key and every counter word matter
    base = orc.philox((1, 2, 3, 4), (5, 6))
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(orc.philox(c, (5, 6)), base)
    assert not np.array_equal(orc.philox((1, 2, 3, 4), (5, 7)), base)


def test_box_muller_moments(orc):
    zs, us = [], []
    for t in range(40000):
        _, z, u = orc.draw(99, 3, t)
        zs.append(z)
        us.append(u)
    zs, us = np.array(zs), np.array(us)
    assert abs(zs.mean()) < 0.02
    assert abs(zs.var() - 1) < 0.03
    assert abs(np.mean(zs ** 4) - 3) < 0.15
    assert 0 < us.min() and us.max() < 1
    assert abs(us.mean() - 0.5) < 0.01


def test_noisy_restart_moments(orc):
    s = np.zeros(20000)
    s2 = orc.noisy_restart(s, 0.3, 5, 1)
    assert abs(s2.std() - 0.3) < 0.01 and abs(s2.mean()) < 0.01
    assert np.all(np.abs(s2) <= np.pi)


# ---------------------------------------------------------------- Metropolis
@pytest.mark.slow
def test_global_mh_samples_exact_boltzmann_lattice_toy(orc):
    """Eq. 1: on a 4-residue chain whose 6 live torsions move on a K=4 lattice
    (symmetric proposal), global MH visits state x with frequency
    exp(-V(x)/T)/Z, Z by enumerating all K^6 = 4096 states."""
    import itertools
    from concurrent.futures import ThreadPoolExecutor
    L, K = 4, 4
    prot = small_problem(L, seed=21)
    P = orc.Problem(L, prot.p, prot.edges)
    n = 2 * L
    q = 2 * np.pi / K
    live = list(range(1, n - 1))
    grid = np.array(list(itertools.product(range(K), repeat=len(live))))
    S = np.zeros((grid.shape[0], n))
    S[:, live] = wrapd(grid * q)
    E = P.energies(S)
    T = float(np.std(E))
    w = np.exp(-(E - E.min()) / T)
    pi = w / w.sum()
    steps = 4_800_000
    nchains = 8

    def one(c):
        s0 = np.zeros(n)
        _, _, tr = P.run(s0, orc.GLOBAL, 0, T, 1.2, 0, steps, 31, c, lattice_K=K, trace=True)
        # reconstruct the lattice state after every proposal, thinned to one per sweep
        idx = np.zeros(steps // n, dtype=np.int64)
        take = np.arange(n - 1, steps, n)
        for j, k in enumerate(live):
            sel = (tr["k"] == k) & (tr["accept"] == 1)
            pos = np.where(sel, np.arange(steps), -1)
            last = np.maximum.accumulate(pos)[take]
            val = np.where(last >= 0, tr["theta_new"][np.maximum(last, 0)], 0.0)
            m = np.mod(np.rint(val / q).astype(np.int64), K)
            idx += m * K ** (len(live) - 1 - j)
        return idx[200:]

    with ThreadPoolExecutor(nchains) as ex:
        samples = np.concatenate(list(ex.map(one, range(nchains))))
    # enumeration index order: grid row = sum m_j K^(5-j) with m_j = round(theta/q) mod K
    gidx = (np.mod(grid, K) * K ** np.arange(len(live) - 1, -1, -1)).sum(1)
    order = np.argsort(gidx)
    pi_sorted = pi[order]
    hist = np.bincount(samples, minlength=K ** len(live)) / samples.size
    tv = 0.5 * np.abs(hist - pi_sorted).sum()
    # total variation expected from multinomial noise alone at this sample size
    tv_noise = 0.5 * np.sum(np.sqrt(2 * pi_sorted * (1 - pi_sorted) / (np.pi * samples.size)))
    print("TV", tv, "noise level", tv_noise)
    assert tv < 1.5 * tv_noise, (tv, tv_noise)
    # a sign error in the acceptance ratio (Alg. 1 as printed) is far off
    wr = np.exp((E - E.max()) / T)
    tv_wrong = 0.5 * np.abs(hist - (wr / wr.sum())[order]).sum()
    assert tv_wrong > 0.3


# ---------------------------------------------------------------- gradient
def test_gradient_matches_one_sided_differences(orc):
    """dV/ds_k (chain rule) lies between the left and right finite differences
    (V is piecewise smooth in s; kinks where a distance crosses a centre)."""
    prot = small_problem(14, seed=33)
    P = orc.Problem(prot.L, prot.p, prot.edges)
    rng = np.random.default_rng(14)
    h = 1e-6
    for trial in range(3):
        s = rng.uniform(-np.pi, np.pi, prot.n)
        V, g = P.grad(s)
        assert abs(V - P.energy(s)) < 1e-12 * abs(V)
        for k in range(prot.n):
            sp, sm = s.copy(), s.copy()
            sp[k] += h
            sm[k] -= h
            right = (P.energy(sp) - V) / h
            left = (V - P.energy(sm)) / h
            lo, hi = min(left, right), max(left, right)
            tol = 1e-4 * (1 + abs(g[k]))
            assert lo - tol <= g[k] <= hi + tol, (k, g[k], left, right)
        assert g[0] == 0.0 and g[-1] == 0.0


# ---------------------------------------------------------------- parallel tempering
def _lattice_setup(orc, K=3, L=4, seed=21):
    import itertools
    prot = small_problem(L, seed=seed)
    P = orc.Problem(L, prot.p, prot.edges)
    n = 2 * L
    q = 2 * np.pi / K
    live = list(range(1, n - 1))
    grid = np.array(list(itertools.product(range(K), repeat=len(live))))
    S = np.zeros((grid.shape[0], n))
    S[:, live] = wrapd(grid * q)
    E = P.energies(S)
    gidx = (np.mod(grid, K) * K ** np.arange(len(live) - 1, -1, -1)).sum(1)
    order = np.argsort(gidx)
    return P, prot, n, q, live, E[order]


def _state_index(S, live, q, K):
    m = np.mod(np.rint(S[:, live] / q).astype(np.int64), K)
    return (m * K ** np.arange(len(live) - 1, -1, -1)).sum(1)


@pytest.mark.slow
def test_parallel_tempering_keeps_each_slot_at_its_boltzmann_law(orc):
    """Replica exchange (Metropolis rule for swapping replicas of exp(-E/T)):
    with global sweeps and exchanges alternating, every ladder slot samples
    exp(-E/T_j)/Z_j; a sign error in the exchange rule would heat the cold
    slots.  Exact laws by enumerating the 3^6 lattice states."""
    K = 3
    P, prot, n, q, live, Es = _lattice_setup(orc, K=K)
    T0 = float(np.std(Es)) / 2
    ladder = np.array([1.0, 1.6, 2.6, 4.2])
    Kl = len(ladder)
    S = np.zeros((Kl, n))
    rounds = 60000
    counts = np.zeros((Kl, K ** len(live)))
    for r in range(rounds):
        for j in range(Kl):
            S[j], _, _ = P.run(S[j], orc.GLOBAL, 0, T0 * ladder[j], 1.5, r * n, n, 11, j, lattice_K=K)
        E = P.energies(S)
        E, S, _ = orc.exchange(E, S, Kl, ladder, T0, r % 2, 13, r)
        if r >= 500:
            idx = _state_index(S, live, q, K)
            counts[np.arange(Kl), idx] += 1
    for j in range(Kl):
        w = np.exp(-(Es - Es.min()) / (T0 * ladder[j]))
        pi = w / w.sum()
        hist = counts[j] / counts[j].sum()
        mean_exact = float(pi @ Es)
        mean_obs = float(hist @ Es)
        sd = float(np.sqrt(pi @ (Es - mean_exact) ** 2))
        tv = 0.5 * np.abs(hist - pi).sum()
        tv_noise = 0.5 * np.sum(np.sqrt(2 * pi * (1 - pi) / (np.pi * counts[j].sum())))
        print("slot", j, "mean", mean_obs, mean_exact, "sd", sd, "tv", tv, "noise", tv_noise)
        assert abs(mean_obs - mean_exact) < 0.05 * sd, (j, mean_obs, mean_exact, sd)
        # consecutive rounds are correlated: allow twice the independent-sample noise
        assert tv < 2.0 * tv_noise, (j, tv, tv_noise)
