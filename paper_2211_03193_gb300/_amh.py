"""ctypes binding of the AMH C ABI (include/amh.h), argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: NumPy arrays are passed as host pointers, torch CUDA
tensors as device pointers.  If ``libamh.so`` is missing the import fails;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libamh.so")

AMH_OK, AMH_EINVAL, AMH_ENOMEM, AMH_ECUDA, AMH_ETIMEOUT, AMH_ESTATE = range(6)
AMH_LOCAL, AMH_GLOBAL = 0, 1
AMH_MAX_SCHED = 16  # sweeps of one amh_sweeps_sched call at most (amh.h)
_STATUS = {0: "AMH_OK", 1: "AMH_EINVAL", 2: "AMH_ENOMEM", 3: "AMH_ECUDA", 4: "AMH_ETIMEOUT",
           5: "AMH_ESTATE"}


class AmhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class amh_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("resync_every", ctypes.c_int),
                ("chains_per_cta", ctypes.c_int), ("threads_per_cta", ctypes.c_int),
                ("trace_chains", ctypes.c_int), ("trace_capacity", ctypes.c_longlong),
                ("lattice_K", ctypes.c_int), ("table_is_neglog", ctypes.c_int),
                ("stage_table", ctypes.c_int), ("table_texture", ctypes.c_int),
                ("far_pairs", ctypes.c_int), ("local_chains_per_cta", ctypes.c_int),
                ("local_threads", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("keep_coords", ctypes.c_int), ("wait_test", ctypes.c_int),
                ("global_kernel", ctypes.c_int), ("warps_per_chain", ctypes.c_int)]


class amh_trace_rec(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("accept", ctypes.c_int), ("theta_new", ctypes.c_double),
                ("lnu", ctypes.c_double), ("dE", ctypes.c_double)]


TRACE_DTYPE = np.dtype([("k", np.int32), ("accept", np.int32), ("theta_new", np.float64),
                        ("lnu", np.float64), ("dE", np.float64)])

_lib = None


def load() -> ctypes.CDLL:
    """Load libamh.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libamh.so not found at %s: run paper_2211_03193_gb300.build.build()"
                          % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p
    L.amh_options_default.argtypes = [ctypes.POINTER(amh_options)]
    L.amh_options_default.restype = None
    L.amh_init.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ip, ip, vp, vp, vp, ctypes.c_int,
                           ctypes.POINTER(amh_options)]
    L.amh_energy.argtypes = [vp, dp]
    L.amh_sweep.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                            ctypes.c_longlong, ctypes.c_ulonglong, vp]
    L.amh_sweeps.argtypes = L.amh_sweep.argtypes
    L.amh_sweeps_sched.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                   ctypes.c_ulonglong, vp]
    L.amh_grad.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp]
    L.amh_get_state.argtypes = [vp, vp, vp, vp, vp]
    L.amh_set_state.argtypes = [vp, vp]
    L.amh_noisy_restart.argtypes = [vp, ctypes.c_double, ctypes.c_ulonglong]
    L.amh_get_trace.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_longlong)]
    L.amh_counter.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
    L.amh_pair_terms.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong),
                                 ctypes.POINTER(ctypes.c_ulonglong)]
    L.amh_philox.argtypes = [ctypes.c_ulonglong, ctypes.c_uint, ctypes.c_ulonglong, ctypes.c_uint,
                             ctypes.c_longlong, vp, vp, vp]
    L.amh_last_error.argtypes = [vp]
    L.amh_last_error.restype = ctypes.c_char_p
    L.amh_launch_config.argtypes = [vp, ip, ip, ip, ip]
    L.amh_destroy.argtypes = [vp]
    L.amh_destroy.restype = None
    L.amh_set_ladder.argtypes = [vp, ctypes.c_int, vp]
    L.amh_exchange.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_ulonglong, vp]
    L.amh_grad_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp,
                                   ctypes.c_int, vp, vp, vp]
    L.amh_get_coords.argtypes = [vp, vp]
    L.amh_window_coords.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ip, ip]
    for name in ("amh_init", "amh_energy", "amh_sweep", "amh_sweeps", "amh_grad", "amh_get_state",
                 "amh_set_state", "amh_noisy_restart", "amh_get_trace", "amh_counter",
                 "amh_philox", "amh_launch_config", "amh_grad_noalloc", "amh_set_ladder",
                 "amh_exchange", "amh_pair_terms", "amh_get_coords", "amh_window_coords",
                 "amh_sweeps_sched"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(st: int, ctx=None):
    if st != AMH_OK:
        msg = load().amh_last_error(ctx).decode(errors="replace") if st != AMH_ESTATE or ctx is None \
            else load().amh_last_error(ctx).decode(errors="replace")
        raise AmhError(st, msg)


def _ptr(x):
    """Pointer of a NumPy array (host) or torch tensor (host or device), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError("expected a NumPy array, a torch tensor or an int pointer")


def amh_options_default(**kw) -> amh_options:
    o = amh_options()
    load().amh_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # a torch.cuda.Stream
        setattr(o, k, v)
    return o


def amh_init(L, chains, torsions, table, edges, options: amh_options | None = None):
    """Create a context; returns the opaque handle (an int)."""
    L = np.ascontiguousarray(np.atleast_1d(L), dtype=np.int32)
    chains = np.ascontiguousarray(np.atleast_1d(chains), dtype=np.int32)
    torsions = np.ascontiguousarray(torsions, dtype=np.float32)
    table = np.ascontiguousarray(table, dtype=np.float64)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    h = ctypes.c_void_p()
    opt = options if options is not None else amh_options_default()
    st = load().amh_init(ctypes.byref(h), int(L.shape[0]),
                         L.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         chains.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         torsions.ctypes.data, table.ctypes.data, edges.ctypes.data,
                         int(edges.shape[0] - 1), ctypes.byref(opt))
    _check(st, None)
    return h.value


def amh_energy(ctx, E_out):
    _check(load().amh_energy(ctx, _ptr(E_out)), ctx)


def amh_sweep(ctx, mode, window, T, sigma_rad, steps, seed, accepted_out=None):
    _check(load().amh_sweep(ctx, int(mode), int(window), float(T), float(sigma_rad), int(steps),
                            int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(accepted_out)), ctx)


def amh_sweeps(ctx, mode, window, T, sigma_rad, nsweeps, seed, accepted_out=None):
    _check(load().amh_sweeps(ctx, int(mode), int(window), float(T), float(sigma_rad), int(nsweeps),
                             int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(accepted_out)), ctx)


def amh_sweeps_sched(ctx, mode, window, T, sigma_rad, seed, accepted_out=None):
    """A run of len(T) whole sweeps, sweep q at T[q] and sigma_rad[q]."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    S = np.ascontiguousarray(sigma_rad, dtype=np.float64)
    if T.shape != S.shape or T.ndim != 1:
        raise ValueError("T and sigma_rad must be 1-D arrays of one length")
    _check(load().amh_sweeps_sched(ctx, int(mode), int(window), int(T.shape[0]), T.ctypes.data,
                                   S.ctypes.data, int(seed) & 0xFFFFFFFFFFFFFFFF,
                                   _ptr(accepted_out)), ctx)


def amh_grad(ctx, protein, theta, batch, E_out, dE_dtheta):
    _check(load().amh_grad(ctx, int(protein), _ptr(theta), int(batch), _ptr(E_out),
                           _ptr(dE_dtheta)), ctx)


def amh_get_state(ctx, torsions_out=None, E_out=None, best_E=None, best_torsions=None):
    _check(load().amh_get_state(ctx, _ptr(torsions_out), _ptr(E_out), _ptr(best_E),
                                _ptr(best_torsions)), ctx)


def amh_set_state(ctx, torsions):
    if isinstance(torsions, np.ndarray):
        torsions = np.ascontiguousarray(torsions, dtype=np.float32)
    _check(load().amh_set_state(ctx, _ptr(torsions)), ctx)


def amh_noisy_restart(ctx, sd_rad, seed):
    _check(load().amh_noisy_restart(ctx, float(sd_rad), int(seed) & 0xFFFFFFFFFFFFFFFF), ctx)


def amh_get_trace(ctx, chain, capacity):
    out = np.zeros(int(capacity), dtype=TRACE_DTYPE)
    cnt = ctypes.c_longlong()
    _check(load().amh_get_trace(ctx, int(chain), out.ctypes.data if capacity else None,
                                ctypes.byref(cnt)), ctx)
    return out[:cnt.value]


def amh_set_ladder(ctx, ladder):
    """Temperature ladder factors (host array of K >= 2), or None to clear."""
    if ladder is None:
        _check(load().amh_set_ladder(ctx, 0, None), ctx)
        return
    lad = np.ascontiguousarray(ladder, dtype=np.float64)
    _check(load().amh_set_ladder(ctx, int(lad.shape[0]), lad.ctypes.data), ctx)


def amh_exchange(ctx, T, parity, seed, swapped_out=None):
    _check(load().amh_exchange(ctx, float(T), int(parity), int(seed) & 0xFFFFFFFFFFFFFFFF,
                               _ptr(swapped_out)), ctx)


def amh_counter(ctx, chain) -> int:
    t = ctypes.c_longlong()
    _check(load().amh_counter(ctx, int(chain), ctypes.byref(t)), ctx)
    return t.value


def amh_pair_terms(ctx):
    """(evaluated, formed): straddle-pair terms of the context's global sweeps
    so far whose table entries were read, and whose distances were formed."""
    v = ctypes.c_ulonglong()
    f = ctypes.c_ulonglong()
    _check(load().amh_pair_terms(ctx, ctypes.byref(v), ctypes.byref(f)), ctx)
    return v.value, f.value


def amh_philox(seed, chain, t0, stream, count):
    words = np.zeros((count, 4), dtype=np.uint32)
    z = np.zeros(count, dtype=np.float32)
    u = np.zeros(count, dtype=np.float32)
    st = load().amh_philox(int(seed) & 0xFFFFFFFFFFFFFFFF, int(chain), int(t0), int(stream),
                           int(count), words.ctypes.data, z.ctypes.data, u.ctypes.data)
    _check(st, None)
    return words, z, u


def amh_launch_config(ctx):
    """(chains per CTA, threads per CTA, staging depth, kernel: 1 CTA lock-step,
    2 chain groups) of the global sweeps."""
    c, t, d, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().amh_launch_config(ctx, ctypes.byref(c), ctypes.byref(t), ctypes.byref(d),
                                    ctypes.byref(k)), ctx)
    return c.value, t.value, d.value, k.value


def amh_get_coords(ctx, n_residues_total):
    """C-beta coordinates of every chain, [sum of L over chains, 3] float64."""
    out = np.zeros((int(n_residues_total), 3), dtype=np.float64)
    _check(load().amh_get_coords(ctx, out.ctypes.data), ctx)
    return out


def amh_window_coords(ctx, chain, k, window):
    """(lo, hi, C-betas [hi-lo+1, 3]) of proposal k's window, in residue lo's frame."""
    out = np.zeros((int(window) + 1, 3), dtype=np.float64)
    lo, hi = ctypes.c_int(), ctypes.c_int()
    _check(load().amh_window_coords(ctx, int(chain), int(k), int(window), out.ctypes.data,
                                    ctypes.byref(lo), ctypes.byref(hi)), ctx)
    return lo.value, hi.value, out[:hi.value - lo.value + 1].copy()


def amh_last_error(ctx=None) -> str:
    return load().amh_last_error(ctx).decode(errors="replace")


def amh_destroy(ctx):
    if ctx:
        load().amh_destroy(ctx)


def amh_grad_noalloc(L, B, table, table_is_neglog, edges, theta, batch, E_out, dE_dtheta,
                     stream=None):
    """No-allocation gradient: table/theta/E_out/dE_dtheta are device tensors,
    edges a host array; see amh.h."""
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(load().amh_grad_noalloc(int(L), int(B), _ptr(table), int(table_is_neglog),
                                   edges.ctypes.data, _ptr(theta), int(batch), _ptr(E_out),
                                   _ptr(dE_dtheta), stream), None)


EXPORTED = ["amh_options_default", "amh_init", "amh_energy", "amh_sweep", "amh_sweeps",
            "amh_grad", "amh_get_state", "amh_set_state", "amh_noisy_restart", "amh_get_trace",
            "amh_counter", "amh_philox", "amh_last_error", "amh_launch_config", "amh_destroy",
            "amh_grad_noalloc", "amh_set_ladder", "amh_exchange", "amh_pair_terms",
            "amh_get_coords", "amh_window_coords", "amh_sweeps_sched"]
