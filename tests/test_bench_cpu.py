"""CPU checks of the benchmark's own arithmetic: the pair-term counts its
roofline divides by, against brute-force enumeration of the pairs each
proposal scores (the straddle block of a global proposal, the window's
straddle pairs of a local one, Eq. 6), and the JSON contract of the
reference arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def brute_counts(L, window, n_local, n_global):
    n = 2 * L
    h = window // 2
    glob = loc = 0
    for k in range(n):
        p = (k + 1) // 2  # first residue whose C-beta moves
        # global: every pair a < p <= b, old and new term
        glob += 2 * sum(1 for a in range(L) for b in range(a + 1, L) if a < p <= b)
        # local: the window around residue k // 2, clipped to the chain
        c = k // 2
        lo, hi = max(0, c - h), min(L - 1, c + h)
        loc += 2 * sum(1 for a in range(lo, hi + 1) for b in range(a + 1, hi + 1) if a < p <= b)
    full = L * (L - 1) // 2  # the energy each global call ends with
    return n_global * (glob + full), n_local * loc


@pytest.mark.parametrize("L,window", [(7, 8), (12, 4), (20, 8), (33, 3), (40, 0)])
def test_pair_counts_match_enumeration(L, window):
    w = dict(L=L, window=window, n_local=10, n_global=1)
    w["n"] = 2 * L
    assert bench.pair_evals_per_cycle(w) == brute_counts(L, window, 10, 1)


def test_headline_workload_counts():
    w = bench.workload("amh_L300_c1024")
    glob, loc = bench.pair_evals_per_cycle(w)
    L = w["L"]
    # the straddle blocks of one sweep hold (L^3 - L) / 3 pairs, scored twice
    assert glob == 2 * (L ** 3 - L) // 3 + L * (L - 1) // 2
    assert glob == 18_000_000 - 200 + 44_850
    assert loc > 0 and w["cycle"] == 11 and w["n"] == 600


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on host cores) prints one JSON
    line with the contract's keys, here on one bounded step."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["metric"] == "MH proposals/s" and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"
