"""Coordinate parity: the C-beta coordinates x = G(s) the CUDA path holds
(Sec. 2.1) against the oracle's NeRF build of the same torsions, read back
through amh_get_coords / amh_window_coords.  V is a sum over pairs and can
hide a coherent frame error; the coordinates cannot.

- a fresh build (after amh_init) is in the canonical frame of residue 0, as
  the oracle's, and is compared atom by atom;
- after global sweeps the coordinates have been turned rigidly by every
  accepted move since the last rebuild (each move turns the smaller side of
  its pivot, so the chain's frame drifts): they are compared by all pair
  distances and, after a least-squares superposition, atom by atom;
- the local sweep's window coordinates are compared in the frame of the
  window's first residue.
Tolerances: 1e-3 A in FP32, 1e-10 A in FP64.
"""
import math

import numpy as np
import pytest

from paper_2211_03193_gb300 import synth

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


def superposed_max_dev(X, Y):
    """Largest atom deviation of X after the least-squares rigid motion onto Y
    (Kabsch, FP64)."""
    xc, yc = X.mean(0), Y.mean(0)
    H = (X - xc).T @ (Y - yc)
    U, _, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(Vt.T @ U.T))
    D = np.diag([1.0, 1.0, d])
    R = Vt.T @ D @ U.T
    return float(np.max(np.linalg.norm((X - xc) @ R.T + yc - Y, axis=1)))


def max_dist_dev(X, Y):
    dX = np.linalg.norm(X[:, None] - X[None], axis=-1)
    dY = np.linalg.norm(Y[:, None] - Y[None], axis=-1)
    return float(np.max(np.abs(dX - dY)))


def frame_of(N, CA, C):
    """Rows: the canonical frame of a residue (x along N->CA, C in the xy-plane
    with y > 0), as the builders' first residue."""
    e1 = (CA - N) / np.linalg.norm(CA - N)
    v = (C - CA) - np.dot(C - CA, e1) * e1
    e2 = v / np.linalg.norm(v)
    return np.stack([e1, e2, np.cross(e1, e2)])


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("L", [150, 300])
def test_fresh_build_equals_oracle(amh, orc, precision, L):
    chains = 6
    prot = synth.make_protein(L, seed=900 + L)
    tors = synth.random_torsions(chains, L, seed=901)
    tol = 1e-3 if precision == 32 else 1e-10
    with amh.Sampler(prot, chains, tors, precision=precision, keep_coords=1) as s:
        X = s.coords()
    worst = 0.0
    for c in range(chains):
        want = orc.build_coords(tors[c].astype(np.float64))["CB"]
        dev = float(np.max(np.linalg.norm(X[c] - want, axis=1)))
        worst = max(worst, dev)
        assert dev <= tol, (c, dev)
    print("fresh build L=%d FP%d: max deviation %.3g A" % (L, precision, worst))


@pytest.mark.parametrize("precision,C,kernel", [(32, 2, 2), (32, 4, 1), (64, 1, 1)])
@pytest.mark.parametrize("L", [150, 300])
def test_coordinates_after_moves_equal_oracle(amh, orc, precision, C, kernel, L):
    """A global sweep of n - 1 proposals (it ends before the next sweep's
    rebuild) with no periodic resync: every accepted move since the entry
    rebuild has turned the coordinates; at the end they must still be G(s) of
    the final torsions up to one rigid motion.  Also after a further call
    that ends part-way through a sweep."""
    chains = 8
    n = 2 * L
    prot = synth.make_protein(L, seed=910 + L)
    tors = synth.random_torsions(chains, L, seed=911)
    tol = 1e-3 if precision == 32 else 1e-10
    P = orc.Problem(L, prot.p, prot.edges)
    s_orc = tors.astype(np.float64)
    t0 = 0
    with amh.Sampler(prot, chains, tors, precision=precision, keep_coords=1,
                     resync_every=1 << 30, chains_per_cta=C, global_kernel=kernel,
                     warps_per_chain=2 if kernel == 2 else 0) as s:
        assert s.launch_config()[3] == kernel
        for steps in (n - 1, n // 2 + 1):
            acc = s.sweep(1, 0, 0.8, 10 * DEG, steps, 17)
            assert acc.min() > steps // 20  # many moves were committed
            X = s.coords()
            th = s.torsions()
            if precision == 64:
                # the FP64 form's torsions are read back through the FP32
                # interface; its own FP64 state is the oracle's trajectory
                # (the FP64 form takes the oracle's decisions)
                s_orc = np.stack([P.run(s_orc[c], orc.GLOBAL, 0, 0.8, 10 * DEG, t0, steps, 17,
                                        c)[0] for c in range(chains)])
                assert np.all(np.abs(np.angle(np.exp(1j * (th - s_orc)))) <= 1e-6)
            t0 += steps
            worst = (0.0, 0.0)
            for c in range(chains):
                want = orc.build_coords(th[c].astype(np.float64) if precision == 32
                                        else s_orc[c])["CB"]
                dd = max_dist_dev(X[c], want)
                sd = superposed_max_dev(X[c], want)
                worst = (max(worst[0], dd), max(worst[1], sd))
                assert dd <= tol and sd <= tol, (steps, c, dd, sd)
            print("after %d proposals L=%d FP%d: distances %.3g A, superposed %.3g A" % (
                steps, L, precision, worst[0], worst[1]))


@pytest.mark.parametrize("precision", [32, 64])
def test_window_coordinates_equal_oracle(amh, orc, precision):
    L, chains = 150, 3
    prot = synth.make_protein(L, seed=920)
    tors = synth.random_torsions(chains, L, seed=921)
    tol = 1e-3 if precision == 32 else 1e-10
    worst = 0.0
    with amh.Sampler(prot, chains, tors, precision=precision) as s:
        for c in range(chains):
            G = orc.build_coords(tors[c].astype(np.float64))
            for k, d in ((0, 8), (1, 8), (77, 8), (150, 10), (201, 5), (298, 8), (299, 3),
                         (120, 0), (64, 64)):
                lo, hi, W = s.window_coords(c, k, d)
                h = d // 2
                assert lo == max(0, k // 2 - h) and hi == min(L - 1, k // 2 + h)
                R = frame_of(G["N"][lo], G["CA"][lo], G["C"][lo])
                want = (G["CB"][lo:hi + 1] - G["N"][lo]) @ R.T
                dev = float(np.max(np.linalg.norm(W - want, axis=1)))
                worst = max(worst, dev)
                assert dev <= tol, (c, k, d, dev)
    print("window coordinates FP%d: max deviation %.3g A" % (precision, worst))
