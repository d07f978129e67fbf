"""Parity of the dilepton ttH path (two-neutrino quartic, Higgs b-jet pair)
with the FP64 oracle: bit-exact mask, cut flow, histogram; reconstructed
masses within 1e-5."""
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


def _run(eng, an, cols, **kw):
    from paper_2211_14346_gb300 import DeviceColumns
    aid = eng.define(an)
    plain = kw.pop("plain", False)
    out = eng.run_device(aid, DeviceColumns(cols), plain=plain, **kw).numpy()
    assert eng.device_error() == 0
    return out


@pytest.mark.parametrize("plain", [False, True])
def test_dilep_smeared_bit_exact(eng, orc, plain):
    """ttH-like dilepton events, 64 smearing variations (jets N(1, 0.10), MET N(0, 10))."""
    cols = synth.gen_dilep(400, 3)
    an = analyses.config3()
    g = _run(eng, an, cols, V=64, seed=1003, plain=plain)
    o = orc.run(an, cols, seed=1003, V=64)
    assert o["cutflow"][-1] > 0
    assert_parity(g, o, model="dilep", what="dilep V=64 plain=%s" % plain)


def test_dilep_unsmeared_and_same_sign(eng, orc):
    cols = synth.gen_dilep(3000, 31, p_same_sign=0.2)
    an = analyses.dilep()
    g = _run(eng, an, cols, V=1)
    o = orc.run(an, cols, V=1)
    assert o["cutflow"][1] < o["cutflow"][0]  # the opposite-sign cut rejects some
    assert_parity(g, o, model="dilep", what="dilep unsmeared")


def test_dilep_many_bjets_and_offsets(eng, orc):
    """More b-tags (up to 12 b-jets: 132 ordered pairings), odd V, event offset."""
    cols = synth.gen_dilep(300, 8, p_btag=0.7)
    an = analyses.dilep(sigma_jet=0.05, sigma_met=5.0)
    g = _run(eng, an, cols, V=7, seed=99, first_event_id=(1 << 33) + 5)
    o = orc.run(an, cols, V=7, seed=99, first_event_id=(1 << 33) + 5)
    assert_parity(g, o, model="dilep", what="dilep many b-jets")


def test_dilep_user_orders(eng, orc):
    cols = synth.gen_dilep(400, 12, p_same_sign=0.1)
    base = analyses.config3()
    rng = np.random.default_rng(5)
    for trial in range(3):
        perm = rng.permutation(len(base["cuts"]))
        an = analyses.with_cuts(base, [base["cuts"][p] for p in perm])
        g = _run(eng, an, cols, V=8, seed=4)
        o = orc.run(an, cols, V=8, seed=4)
        assert_parity(g, o, model="dilep", what="dilep perm %s" % perm)
