"""Seeded synthetic inputs for AMH: distogram tables and chain starts.

These stand in for the AlphaFold1 CASP distograms the paper minimises
(Sec. 2.3, Eq. 5), which are not available here.  This module holds none of
the method's arithmetic (no backbone builder, no energy, no sampler, no
random stream of the sampler); it only draws data:

* a hidden "native" C-beta trace: a virtual-bond pseudo-chain, one point per
  residue.  Each residue is helix-like or strand-like with probability 1/2
  (the i.i.d. helix/sheet torsion mixture of the benchmark problem, expressed
  as C-beta virtual-bond length, bond angle and dihedral states whose means
  and spreads are those of ideal-geometry helix (-63, -43 deg) and strand
  (-120, 130 deg) backbones with 10 deg torsion noise);
* per residue pair a<b, logits_j = -(c_j - d_ab)^2 / (2 sigma_d^2) + N(0, 0.3^2)
  over the bin centres c_j and p = softmax(logits), returned in ascending bin
  order with the bin edges (the last bin open-ended);
* chain starts: torsions i.i.d. uniform on (-pi, pi).

Pair rows are ordered a<b lexicographically: r(a,b) = a L - a(a+1)/2 + (b-a-1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# virtual-bond states: (bond A, sd), (angle deg, sd), (dihedral deg, sd)
_STATES = {
    "helix": ((5.32, 0.15), (85.9, 5.6), (36.8, 12.5)),
    "strand": ((5.80, 0.07), (71.8, 3.6), (-161.7, 14.2)),
}


def edges_af1_37() -> np.ndarray:
    """37 bins: 36 of 0.5 A over [2, 20) and one open bin [20, inf)."""
    return np.concatenate([2.0 + 0.5 * np.arange(37), [np.inf]])


def edges_uniform_64() -> np.ndarray:
    """64 bins of 0.3125 A from 2 A, the last one open: [21.6875, inf)."""
    return np.concatenate([2.0 + 0.3125 * np.arange(64), [np.inf]])


def _data_centres(edges: np.ndarray) -> np.ndarray:
    # centres used by the data model only; the open bin sits half a width
    # beyond its lower edge
    lo, hi = edges[:-1], edges[1:].copy()
    hi[-1] = lo[-1] + (lo[-1] - lo[-2])
    return 0.5 * (lo + hi)


def _rot_x(a: float) -> np.ndarray:
    c, s = np.cos(a), np.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def _rot_z(a: float) -> np.ndarray:
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def native_trace(L: int, rng: np.random.Generator) -> np.ndarray:
    """Hidden native C-beta trace [L, 3] as a turtle walk of virtual bonds."""
    helix = rng.random(L) < 0.5
    x = np.zeros((L, 3))
    frame = np.eye(3)
    for i in range(1, L):
        st = _STATES["helix" if helix[i] else "strand"]
        bond = rng.normal(*st[0])
        if i >= 2:
            turn = np.radians(180.0 - rng.normal(*st[1]))
            twist = np.radians(rng.normal(*st[2])) if i >= 3 else 0.0
            frame = frame @ _rot_x(twist) @ _rot_z(turn)
        x[i] = x[i - 1] + bond * frame[:, 0]
    return x


@dataclass
class Protein:
    L: int
    p: np.ndarray        # [L(L-1)/2, B] float64, ascending bins, rows sum to 1
    edges: np.ndarray    # [B+1] float64, last may be +inf
    native: np.ndarray   # [L, 3] hidden C-beta trace (data only)

    @property
    def B(self) -> int:
        return self.edges.shape[0] - 1

    @property
    def n(self) -> int:
        return 2 * self.L


def make_protein(L: int, edges: np.ndarray | None = None, sigma_d: float = 1.0,
                 logit_noise: float = 0.3, seed: int = 1000) -> Protein:
    """A synthetic distogram of L residues (seeded, float64)."""
    if edges is None:
        edges = edges_af1_37()
    rng = np.random.default_rng(seed)
    x = native_trace(L, rng)
    c = _data_centres(edges)
    a, b = np.triu_indices(L, 1)
    p = np.empty((a.shape[0], c.shape[0]))
    chunk = 1 << 15
    for s0 in range(0, a.shape[0], chunk):
        sa, sb = a[s0:s0 + chunk], b[s0:s0 + chunk]
        d = np.linalg.norm(x[sa] - x[sb], axis=1)
        logits = -(c[None, :] - d[:, None]) ** 2 / (2.0 * sigma_d ** 2)
        logits += rng.normal(0.0, logit_noise, logits.shape)
        logits -= logits.max(axis=1, keepdims=True)
        e = np.exp(logits)
        p[s0:s0 + chunk] = e / e.sum(axis=1, keepdims=True)
    return Protein(L=L, p=p, edges=np.asarray(edges, dtype=np.float64), native=x)


def random_torsions(nchains: int, L: int, seed: int) -> np.ndarray:
    """Chain starts [nchains, 2L] float32, i.i.d. uniform on (-pi, pi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi, np.pi, size=(nchains, 2 * L)).astype(np.float32)


def to_af1_layout(p: np.ndarray) -> np.ndarray:
    """Ascending bins -> the AlphaFold1 storage order (open bin first)."""
    return np.concatenate([p[:, -1:], p[:, :-1]], axis=1)


def from_af1_layout(p_af1: np.ndarray) -> np.ndarray:
    """AlphaFold1 storage order (open bin first) -> ascending bins."""
    return np.concatenate([p_af1[:, 1:], p_af1[:, :1]], axis=1)


def uneven_lengths(nproteins: int = 64, lo: int = 50, hi: int = 400, seed: int = 3) -> list[int]:
    """Protein lengths drawn uniformly from [lo, hi] (the batched workload)."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(lo, hi + 1, size=nproteins)]


# Workloads (sizes and schedules; no arithmetic).  Temperatures are in the
# energy's units; sigma in degrees.
WORKLOADS = {
    # one FP64 chain, 20k proposals (small case the oracle finishes quickly)
    "amh_fp64_L64_1chain": dict(L=64, chains=1, bins="af1_37", sigma_d=1.0, n_local=10,
                                n_global=1, window=8, T0=1.0, T1=1.0, sigma_deg=15.0,
                                proposals=20000, precision=64, seed=1000, start_seed=8),
    # the headline: L=300, 1024 chains, 10 local (d=8) : 1 global sweeps
    "amh_L300_c1024": dict(L=300, chains=1024, bins="af1_37", sigma_d=1.0, n_local=10,
                           n_global=1, window=8, T0=2.0, T1=0.05, sigma_deg=(10.0, 4.0),
                           proposals=200000, precision=32, seed=1000, start_seed=9),
    "amh_L150_c1024": dict(L=150, chains=1024, bins="af1_37", sigma_d=1.0, n_local=10,
                           n_global=1, window=8, T0=2.0, T1=0.05, sigma_deg=(10.0, 4.0),
                           proposals=200000, precision=32, seed=1000, start_seed=9),
    "amh_batched_64prot": dict(nproteins=64, Lmin=50, Lmax=400, chains=256, bins="af1_37",
                               sigma_d=1.0, n_local=10, n_global=1, window=8, T0=2.0, T1=0.05,
                               sigma_deg=(10.0, 4.0), proposals=100000, precision=32,
                               resync_every=1000, seed=1000, start_seed=10),
    "grad_L300_b512": dict(L=300, batch=512, bins="af1_37", sigma_d=1.0, seed=1000,
                           start_seed=11),
    "amh_L500_c4096": dict(L=500, chains=4096, bins="uniform_64", sigma_d=1.5, n_local=10,
                           n_global=1, window=8, T0=2.0, T1=0.05, sigma_deg=(10.0, 4.0),
                           proposals=500000, precision=32, seed=1000, start_seed=12),
}


def edges_by_name(name: str) -> np.ndarray:
    return {"af1_37": edges_af1_37, "uniform_64": edges_uniform_64}[name]()
