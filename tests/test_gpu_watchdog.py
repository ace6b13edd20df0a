"""The bounded-wait watchdog of the staged global sweep (no GPU fault, no
hang): with the wait_test hook every CTA first waits on its staging ring's
first slot before issuing any copy.  Nothing can arrive there, so each wait
gives up after the given number of tries with no copy in flight; the call
reports AMH_ETIMEOUT and the context refuses further work (AMH_ESTATE)."""
import math

import numpy as np
import pytest

from paper_2211_03193_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03193_gb300 import build, _amh, sampler
    build.build()
    _amh.load()
    return _amh, sampler


@pytest.mark.parametrize("C", [4, 8])
def test_staging_wait_gives_up_and_the_context_is_broken(mods, C):
    amh, sampler = mods
    L, chains = 40, 16
    prot = synth.make_protein(L, seed=950)
    tors = synth.random_torsions(chains, L, seed=951)
    with sampler.Sampler(prot, chains, tors, chains_per_cta=C, threads_per_cta=256,
                         stage_table=1, wait_test=64) as s:
        assert s.launch_config()[2] >= 2  # staged
        E0 = s.energy()  # the energy kernel stages nothing: it works
        assert np.all(np.isfinite(E0))
        with pytest.raises(amh.AmhError) as ei:
            s.sweep(1, 0, 1.0, math.radians(10.0), 2 * L, 3)
        assert ei.value.status == amh.AMH_ETIMEOUT
        with pytest.raises(amh.AmhError) as ei2:
            s.energy()
        assert ei2.value.status == amh.AMH_ESTATE
    # the device is still usable: a fresh context without the hook runs
    with sampler.Sampler(prot, chains, tors, chains_per_cta=C, threads_per_cta=256,
                         stage_table=1) as s:
        s.sweep(1, 0, 1.0, math.radians(10.0), 2 * L, 3)
        assert np.all(np.isfinite(s.state()[1]))
