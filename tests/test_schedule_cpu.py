"""CPU checks of the schedule (host logic of Alg. 1's outer loop): which
phase each sweep belongs to, the annealing of T (geometric) and sigma
(linear) over the run, and cascaded localization radii (Sec. 2.2)."""
import math

import pytest

from paper_2211_03193_gb300 import _amh
from paper_2211_03193_gb300.sampler import Schedule


def test_phases_follow_the_cycle():
    sch = Schedule(total_sweeps=33, n_local=10, n_global=1)
    modes = [sch.params(s)[0] for s in range(33)]
    for s, m in enumerate(modes):
        assert m == (_amh.AMH_LOCAL if s % 11 < 10 else _amh.AMH_GLOBAL)
    assert modes.count(_amh.AMH_GLOBAL) == 3


def test_plain_mh_has_no_local_phase():
    sch = Schedule(total_sweeps=5, n_local=0, n_global=1)
    assert all(sch.params(s)[0] == _amh.AMH_GLOBAL for s in range(5))


@pytest.mark.parametrize("S", [2, 7, 333])
def test_anneal_endpoints_and_shape(S):
    sch = Schedule(total_sweeps=S, T0=2.0, T1=0.05, sigma0_deg=10.0, sigma1_deg=4.0)
    _, T_first, sg_first = sch.params(0)
    _, T_last, sg_last = sch.params(S - 1)
    assert T_first == pytest.approx(2.0) and T_last == pytest.approx(0.05)
    assert sg_first == pytest.approx(math.radians(10.0))
    assert sg_last == pytest.approx(math.radians(4.0))
    Ts = [sch.params(s)[1] for s in range(S)]
    sgs = [sch.params(s)[2] for s in range(S)]
    # geometric T: constant ratio between consecutive sweeps; linear sigma
    ratios = [b / a for a, b in zip(Ts, Ts[1:])]
    assert max(ratios) == pytest.approx(min(ratios))
    steps = [b - a for a, b in zip(sgs, sgs[1:])]
    assert max(steps) == pytest.approx(min(steps), abs=1e-15)
    # past the end the schedule holds its last values
    assert sch.params(S + 5)[1] == pytest.approx(0.05)


def test_cascaded_windows():
    sch = Schedule(total_sweeps=12, n_local=3, n_global=1, windows=(4, 8, 12))
    got = [sch.window_of(s) for s in range(12)]
    # local sweep j of each cycle uses windows[j % 3]; the global sweep's entry is unused
    assert [got[s] for s in range(12) if s % 4 < 3] == [4, 8, 12] * 3
    assert Schedule(total_sweeps=3, window=6).window_of(2) == 6
