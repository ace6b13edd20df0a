"""The C-ABI library builds, loads and exports every symbol amh.h declares;
argument checks that need no GPU return AMH_EINVAL."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_03193_gb300 import build, _amh
    build.build()
    return _amh.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "amh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amh_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("amh_init", "amh_energy", "amh_sweep", "amh_grad", "amh_get_state",
                 "amh_set_state", "amh_noisy_restart", "amh_last_error", "amh_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_has_the_same_names(lib):
    from paper_2211_03193_gb300 import _amh
    for name in declared_functions():
        assert callable(getattr(_amh, name)), name


def _init(lib, **over):
    from paper_2211_03193_gb300 import _amh
    L = np.array([over.get("L", 8)], dtype=np.int32)
    ch = np.array([over.get("chains", 2)], dtype=np.int32)
    B = over.get("B", 5)
    edges = np.asarray(over.get("edges", 2.0 + np.arange(B + 1)), dtype=np.float64)
    rows = int(L[0]) * (int(L[0]) - 1) // 2
    table = np.full((max(rows, 1), max(B, 1)), 1.0 / max(B, 1))
    tors = np.zeros(int(ch[0]) * 2 * max(int(L[0]), 1), dtype=np.float32)
    opt = _amh.amh_options_default(**over.get("opt", {}))
    h = ctypes.c_void_p()
    st = lib.amh_init(ctypes.byref(h), 1, L.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      ch.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), tors.ctypes.data,
                      table.ctypes.data, edges.ctypes.data, B, ctypes.byref(opt))
    return st, h


@pytest.mark.parametrize("over", [
    dict(B=1),
    dict(L=1),
    dict(chains=0),
    dict(edges=[2.0, 3.0, 3.5, 5.0, 6.0, 7.0]),     # uneven centres
    dict(edges=[2.0, 3.0, 2.5, 5.0, 6.0, 7.0]),     # not ascending
    dict(opt=dict(precision=16)),
    dict(opt=dict(chains_per_cta=3)),
    dict(opt=dict(threads_per_cta=96)),
    dict(opt=dict(far_pairs=2)),
    dict(opt=dict(local_chains_per_cta=3)),
    dict(opt=dict(local_chains_per_cta=64)),
    dict(opt=dict(local_threads=48)),
    dict(opt=dict(local_threads=512)),
    dict(opt=dict(table_texture=3)),
    dict(opt=dict(stage_table=-1)),
    dict(opt=dict(keep_coords=2)),
    dict(opt=dict(wait_test=-1)),
    dict(opt=dict(global_kernel=3)),
    dict(opt=dict(warps_per_chain=3)),
    dict(opt=dict(global_kernel=2, precision=64)),
    dict(opt=dict(global_kernel=2, far_pairs=1)),
    dict(opt=dict(global_kernel=2, stage_table=1)),
    dict(opt=dict(global_kernel=2, threads_per_cta=128)),
    dict(opt=dict(global_kernel=2, chains_per_cta=4, warps_per_chain=4)),
])
def test_bad_arguments_are_refused_before_any_device_work(lib, over):
    st, h = _init(lib, **over)
    assert st == 1  # AMH_EINVAL
    assert not h.value
    assert lib.amh_last_error(None)


def test_null_context_calls_return_estate(lib):
    assert lib.amh_energy(None, None) == 5
    assert lib.amh_sweep(None, 1, 0, 1.0, 0.1, 10, 1, None) == 5
    v = ctypes.c_ulonglong()
    assert lib.amh_pair_terms(None, ctypes.byref(v), None) == 5
    lib.amh_destroy(None)


def test_binding_constants_match_the_header():
    from paper_2211_03193_gb300 import _amh
    src = open(os.path.join(ROOT, "include", "amh.h")).read()
    m = re.search(r"#define AMH_MAX_SCHED (\d+)", src)
    assert m and int(m.group(1)) == _amh.AMH_MAX_SCHED
    m = re.search(r"#define AMH_NOALLOC_MAX_ENTRIES \(1 << (\d+)\)", src)
    assert m


def test_sched_call_refuses_bad_runs_without_a_device(lib):
    import ctypes as ct
    T = (ct.c_double * 2)(1.0, 1.0)
    assert lib.amh_sweeps_sched(None, 1, 0, 2, T, T, 1, None) == 5  # NULL context


def test_options_default_far_field_skip_on():
    from paper_2211_03193_gb300 import _amh
    o = _amh.amh_options_default()
    assert o.far_pairs == 0 and o.table_texture == 0 and o.threads_per_cta == 0
    assert o.local_chains_per_cta == 0 and o.local_threads == 0


def test_peaks_library_exports_its_symbol():
    """libamh_peaks.so (the roofline microbenchmarks) builds and exports what
    amh_peaks.h declares; nothing runs without a GPU."""
    from paper_2211_03193_gb300 import build
    build.build()
    src = open(os.path.join(ROOT, "include", "amh_peaks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"\b(amh_[a-z_0-9]+)\s*\(", src)))
    assert names == ["amh_measure_peaks"]
    lib = ctypes.CDLL(build.PEAKS_LIB)
    for name in names:
        assert hasattr(lib, name)
