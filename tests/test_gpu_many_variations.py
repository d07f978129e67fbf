"""Parity with the FP64 oracle at large variation counts, up to the ABI's
maximum: the paper's ttH_sci pseudo-experiments (Sect. 4: 1024 variations
of a 1 % resolution smearing) and tiles holding a single event with more
units than the block has threads.  Fast and plain forms, both models."""
import numpy as np
import pytest

import synth
from synth import analyses
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_14346_gb300 import build, Engine
    build.build()
    e = Engine(0)
    yield e
    e.close()


def _check(eng, orc, an, cols, V, seed, model, plain=False):
    from paper_2211_14346_gb300 import DeviceColumns
    aid = eng.define(an)
    g = eng.run_device(aid, DeviceColumns(cols), V=V, seed=seed, first_event_id=5000, plain=plain).numpy()
    assert eng.device_error() == 0
    o = orc.run(an, cols, seed=seed, V=V, first_event_id=5000)
    assert_parity(g, o, model=model, what="%s V=%d plain=%s" % (model, V, plain))
    return g


@pytest.mark.parametrize("V,n", [(257, 120), (1024, 60), (4096, 12)])
@pytest.mark.parametrize("plain", [False, True])
def test_semilep_many_variations(eng, orc, V, n, plain):
    cols = synth.gen_semilep(n, 31)
    g = _check(eng, orc, analyses.config2(), cols, V, 4242, "semilep", plain)
    assert g["cutflow"][0] == n * V


@pytest.mark.parametrize("V,n", [(1024, 80), (4096, 16)])
def test_dilep_paper_resolution_1024(eng, orc, V, n):
    """ttH_sci shape: 1 % jet-energy resolution, 1024 and 4096 variations."""
    cols = synth.gen_dilep(n, 32)
    _check(eng, orc, analyses.tth_sci(), cols, V, 777, "dilep")


def test_semilep_paper_resolution_1024_plain_equals_fast(eng, orc):
    cols = synth.gen_semilep(50, 33)
    an = analyses.semilep(sigma_jet=0.01, sigma_met=1.0)
    a = _check(eng, orc, an, cols, 1024, 99, "semilep")
    b = _check(eng, orc, an, cols, 1024, 99, "semilep", plain=True)
    assert np.array_equal(a["n_surv"], b["n_surv"])
