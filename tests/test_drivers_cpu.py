"""CPU checks of the host drivers above the C ABI, against a stand-in
sampler that records the calls it receives: the schedule's sweep order
with its windows and noisy restarts, and the restart-from-best protocol
(Sec. 2.3): every run after the first starts each chain from its best
state, and the step sigma narrows after runs that find no lower energy."""
import math

import numpy as np

from paper_2211_03193_gb300 import _amh
from paper_2211_03193_gb300.sampler import Schedule, restart_from_best, run_schedule


class Recorder:
    """Duck-typed sampler: records sweeps, noisy restarts and state changes;
    the lowest energy after run r is the scripted per-run value."""

    def __init__(self, per_run_best, total_sweeps, n_chains=3, n=8):
        self.n_chains = n_chains
        self.calls = []
        self.script = list(per_run_best)
        self.total = total_sweeps
        self.sweeps_done = 0
        self.best_t = np.arange(n_chains * n, dtype=np.float32)

    def sweeps(self, mode, window, T, sigma, nsweeps, seed, accepted=True):
        self.calls.append(("sweep", mode, window, T, sigma, seed))
        self.sweeps_done += nsweeps
        return np.ones(self.n_chains, dtype=np.int64) if accepted else None

    def sweeps_sched(self, mode, window, T, sigma, seed, accepted=True):
        assert len(T) == len(sigma) <= _amh.AMH_MAX_SCHED
        for t, sg in zip(T, sigma):
            self.calls.append(("sweep", mode, window, t, sg, seed))
        self.calls.append(("run", len(T)))
        self.sweeps_done += len(T)
        return np.ones(self.n_chains, dtype=np.int64) * len(T) if accepted else None

    def noisy_restart(self, sd, seed):
        self.calls.append(("noisy", sd, seed))

    def set_state(self, t):
        self.calls.append(("set", np.array(t)))

    def state(self):
        runs = self.sweeps_done // self.total
        lo = 10.0 if runs == 0 else self.script[runs - 1]
        bE = np.array([lo + 1.0, lo, lo + 2.0])
        return None, None, bE, self.best_t


def test_run_schedule_order_windows_and_noisy_restarts():
    sch = Schedule(total_sweeps=9, n_local=2, n_global=1, windows=(4, 6), noisy_every=4,
                   noisy_sd_deg=20.0, seed=5)
    rec = Recorder([0.0], total_sweeps=9)
    acc = run_schedule(rec, sch, on_sweep=lambda *a: None)
    sweeps = [c for c in rec.calls if c[0] == "sweep"]
    assert [c[1] for c in sweeps] == [_amh.AMH_LOCAL, _amh.AMH_LOCAL, _amh.AMH_GLOBAL] * 3
    assert [c[2] for c in sweeps if c[1] == _amh.AMH_LOCAL] == [4, 6] * 3
    assert all(c[5] == 5 for c in sweeps)
    for s, c in enumerate(sweeps):
        mode, T, sigma = sch.params(s)
        assert (c[3], c[4]) == (T, sigma)
    noisy = [(i, c) for i, c in enumerate(rec.calls) if c[0] == "noisy"]
    # after sweeps 4 and 8 (s + 1 divisible by 4), with seed * 1000003 + s
    assert [c[2] for _, c in noisy] == [5 * 1000003 + 3, 5 * 1000003 + 7]
    assert all(c[1] == math.radians(20.0) for _, c in noisy)
    assert np.array_equal(acc, np.full(3, 9))


def test_run_schedule_in_runs_of_one_mode():
    """Without a per-sweep callback the schedule goes to the library in runs:
    consecutive sweeps of one mode and window, at most AMH_MAX_SCHED, a run
    ending before each noisy restart; every sweep keeps its own T and sigma."""
    sch = Schedule(total_sweeps=40, n_local=18, n_global=2, windows=(8,), noisy_every=7,
                   noisy_sd_deg=20.0, seed=5)
    rec = Recorder([0.0], total_sweeps=40)
    run_schedule(rec, sch)
    sweeps = [c for c in rec.calls if c[0] == "sweep"]
    assert len(sweeps) == 40
    for s, c in enumerate(sweeps):
        mode, T, sigma = sch.params(s)
        assert (c[1], c[3], c[4]) == (mode, T, sigma)
    runs = [c[1] for c in rec.calls if c[0] == "run"]
    assert sum(runs) == 40 and max(runs) <= _amh.AMH_MAX_SCHED
    # the run boundaries: mode changes (18, 20, 38, 40) and noisy restarts
    # after sweeps 7, 14, 21, 28, 35
    ends = list(np.cumsum(runs))
    assert ends == [7, 14, 18, 20, 21, 28, 35, 38, 40]
    # each noisy restart comes right after its run
    order = [c[0] for c in rec.calls if c[0] in ("run", "noisy")]
    assert order == ["run", "noisy", "run", "noisy", "run", "run", "run", "noisy", "run",
                     "noisy", "run", "noisy", "run", "run"]


def test_restart_from_best_protocol():
    sch = Schedule(total_sweeps=4, n_local=1, n_global=1, sigma0_deg=10.0, sigma1_deg=4.0, seed=3)
    # lowest energy after each run: better, better, worse, worse, better
    rec = Recorder([8.0, 6.0, 6.5, 7.0, 5.0], total_sweeps=4)
    seen = []
    hist = restart_from_best(rec, sch, runs=5, on_run=lambda r, b, sig: seen.append(sig))
    assert hist == [8.0, 6.0, 6.0, 6.0, 5.0]
    # sigma follows the schedule until a run fails; after F failures 10/F -> 1/F deg
    assert seen == [(10.0, 4.0), (10.0, 4.0), (10.0, 4.0), (10.0, 1.0), (5.0, 0.5)]
    sweeps = [c for c in rec.calls if c[0] == "sweep"]
    assert len(sweeps) == 5 * 4
    for r in range(5):
        first = sweeps[4 * r]
        assert math.isclose(first[4], math.radians(seen[r][0]))
        assert first[5] == 3 + 7919 * r
    # runs after the first start from the best states
    sets = [i for i, c in enumerate(rec.calls) if c[0] == "set"]
    assert len(sets) == 4
    for i in sets:
        assert np.array_equal(rec.calls[i][1], rec.best_t)
