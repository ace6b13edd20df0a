"""FP64 CPU oracle of the AMH hot path (arXiv 2211.03193) -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It loads ``amh_oracle.c`` (plain C, FP64,
scalar) through ctypes; nothing here is shared with the CUDA library.

Functions (each follows the paper passage cited in ``amh_oracle.c``):
  build_coords   G(s), Sec. 2.1 / Eq. 3 (NeRF with ideal geometry)
  energy         V(x), Eq. 5 over unordered pairs
  energy_local   V_local(x, k, d), Eq. 6
  run            Alg. 1 inner loops (global or local Metropolis sweeps)
  grad           dV/ds by the chain rule
  philox         Philox4x32-10 (Salmon et al., SC'11)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amh_oracle.c")
_SO = os.path.join(_HERE, "_amh_oracle.so")

GLOBAL = 1
LOCAL = 0


def build(force: bool = False) -> str:
    """Compile amh_oracle.c into a shared object beside it (gcc, OpenMP)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class TraceRec(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("accept", ctypes.c_int32), ("z", ctypes.c_double),
                ("lnu", ctypes.c_double), ("dV", ctypes.c_double), ("theta_new", ctypes.c_double)]


TRACE_DTYPE = np.dtype([("k", np.int32), ("accept", np.int32), ("z", np.float64),
                        ("lnu", np.float64), ("dV", np.float64), ("theta_new", np.float64)])

_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_SO)
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_build.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
    L.orc_problem_new.restype = ctypes.c_void_p
    L.orc_problem_new.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
    L.orc_problem_free.argtypes = [ctypes.c_void_p]
    L.orc_problem_centres.argtypes = [ctypes.c_void_p, dp]
    L.orc_pair_term.restype = ctypes.c_double
    L.orc_pair_term.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    L.orc_pair_slope.restype = ctypes.c_double
    L.orc_pair_slope.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    L.orc_energy.restype = ctypes.c_double
    L.orc_energy.argtypes = [ctypes.c_void_p, dp]
    L.orc_energy_local.restype = ctypes.c_double
    L.orc_energy_local.argtypes = [ctypes.c_void_p, dp, ctypes.c_int, ctypes.c_int]
    L.orc_energy_of_torsions.restype = ctypes.c_double
    L.orc_energy_of_torsions.argtypes = [ctypes.c_void_p, dp]
    u32p = ctypes.POINTER(ctypes.c_uint32)
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                           u32p, dp, dp]
    L.orc_run.restype = ctypes.c_longlong
    L.orc_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                          ctypes.c_double, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_uint64,
                          ctypes.c_uint32, ctypes.c_int, dp, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_run_chains.restype = ctypes.c_longlong
    L.orc_run_chains.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_longlong,
                                 ctypes.c_longlong, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                 dp, ctypes.POINTER(ctypes.c_longlong)]
    L.orc_num_threads.restype = ctypes.c_int
    L.orc_noisy_restart.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_uint32]
    L.orc_grad.argtypes = [ctypes.c_void_p, dp, dp, dp]
    L.orc_exchange.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                               ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, dp,
                               dp, ctypes.POINTER(ctypes.c_int)]
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def build_coords(s) -> dict:
    """G(s) for one chain: returns N, CA, C, CB arrays of shape [L, 3]."""
    s = _f64(s)
    L = s.shape[0] // 2
    out = {k: np.zeros((L, 3)) for k in ("N", "CA", "C", "CB")}
    lib().orc_build(L, _dp(s), _dp(out["N"]), _dp(out["CA"]), _dp(out["C"]), _dp(out["CB"]))
    return out


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of a 4-word counter and 2-word key."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def draw(seed: int, chain: int, t: int, stream: int = 0):
    """Raw words, Box-Muller normal and accept uniform of one proposal."""
    o = (ctypes.c_uint32 * 4)()
    z = ctypes.c_double()
    u = ctypes.c_double()
    lib().orc_draw(seed, chain, t, stream, o, ctypes.byref(z), ctypes.byref(u))
    return np.array(list(o), dtype=np.uint32), z.value, u.value


def num_threads() -> int:
    return int(lib().orc_num_threads())


class Problem:
    """One protein: L residues, B bins, table p[rows, B] (ascending bins)."""

    def __init__(self, L: int, p, edges):
        self.L = int(L)
        p = _f64(p)
        edges = _f64(edges)
        self.B = edges.shape[0] - 1
        rows = self.L * (self.L - 1) // 2
        if p.shape != (rows, self.B):
            raise ValueError("table shape %r, expected %r" % (p.shape, (rows, self.B)))
        self._p = p
        self._h = lib().orc_problem_new(self.L, self.B, _dp(p), _dp(edges))
        if not self._h:
            raise ValueError("bad problem")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_problem_free(h)
            self._h = None

    @property
    def n(self) -> int:
        return 2 * self.L

    def centres(self) -> np.ndarray:
        c = np.zeros(self.B)
        lib().orc_problem_centres(self._h, _dp(c))
        return c

    def pair_term(self, a: int, b: int, d: float) -> float:
        return lib().orc_pair_term(self._h, a, b, d)

    def pair_slope(self, a: int, b: int, d: float) -> float:
        return lib().orc_pair_slope(self._h, a, b, d)

    def energy_cb(self, cb) -> float:
        cb = _f64(cb)
        return lib().orc_energy(self._h, _dp(cb))

    def energy_local_cb(self, cb, k: int, d: int) -> float:
        cb = _f64(cb)
        return lib().orc_energy_local(self._h, _dp(cb), k, d)

    def energy(self, s) -> float:
        s = _f64(s)
        return lib().orc_energy_of_torsions(self._h, _dp(s))

    def energies(self, S) -> np.ndarray:
        S = _f64(S)
        return np.array([self.energy(row) for row in S.reshape(-1, self.n)])

    def run(self, s, mode: int, window: int, T: float, sigma: float, t0: int, steps: int,
            seed: int, chain: int, lattice_K: int = 0, trace: bool = False, forced=None):
        """One chain; returns (new s, accepted, trace or None)."""
        s = _f64(s).copy()
        tr = np.zeros(steps, dtype=TRACE_DTYPE) if trace else None
        fz = None
        if forced is not None:
            fz = np.ascontiguousarray(forced, dtype=np.uint8)
            assert fz.shape[0] == steps
        acc = lib().orc_run(self._h, mode, window, T, sigma, t0, steps, seed, chain, lattice_K,
                            _dp(s), tr.ctypes.data if tr is not None else None,
                            fz.ctypes.data if fz is not None else None)
        if acc < 0:
            raise ValueError("bad run arguments")
        return s, int(acc), tr

    def run_chains(self, S, mode: int, window: int, T: float, sigma: float, t0: int, steps: int,
                   seed: int, chain0: int = 0, lattice_K: int = 0):
        """Many chains (OpenMP over chains); returns (new S, accepted[nchains])."""
        S = _f64(S).copy()
        nch = S.shape[0]
        acc = np.zeros(nch, dtype=np.int64)
        r = lib().orc_run_chains(self._h, nch, mode, window, T, sigma, t0, steps, seed, chain0,
                                 lattice_K, _dp(S),
                                 acc.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
        if r < 0:
            raise ValueError("bad run arguments")
        return S, acc

    def grad(self, s):
        """(V, dV/ds) for one chain."""
        s = _f64(s)
        g = np.zeros(self.n)
        V = ctypes.c_double()
        lib().orc_grad(self._h, _dp(s), ctypes.byref(V), _dp(g))
        return V.value, g


def exchange(E, S, K: int, ladder, T_scale: float, parity: int, seed: int, round_: int,
             chain0: int = 0):
    """Replica exchange between neighbouring ladder slots; returns new (E, S,
    accepted) -- see orc_exchange."""
    E = _f64(E).copy()
    S = _f64(S).copy()
    nch = E.shape[0]
    n = S.size // nch
    ladder = _f64(ladder)
    acc = np.zeros(nch, dtype=np.int32)
    lib().orc_exchange(nch, n, K, _dp(ladder), T_scale, parity, seed, round_, chain0, _dp(E),
                       _dp(S), acc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return E, S.reshape(nch, n), acc


def noisy_restart(s, sd: float, seed: int, chain: int) -> np.ndarray:
    s = _f64(s).copy()
    lib().orc_noisy_restart(s.shape[0] // 2, _dp(s), sd, seed, chain)
    return s
