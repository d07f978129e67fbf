"""Parity of the full Eq. 1 semileptonic fit (HF_CUT_TTBAR_CHI2_MAX: both
tops, both W bosons, both neutrino solutions) with the FP64 oracle: bit-exact
mask, n_surv, cut flow and histogram; reco (m_top hadronic, m_top leptonic,
p_z, |MET|) within 1e-5."""
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
def test_fullfit_smeared(eng, orc, plain):
    cols = synth.gen_semilep(1500, 41)
    an = analyses.semilep_full(sigma_jet=0.10, sigma_met=10.0)
    g = _run(eng, an, cols, V=16, seed=7, plain=plain)
    o = orc.run(an, cols, seed=7, V=16)
    assert o["cutflow"][-1] > 0
    assert_parity(g, o, what="full fit V=16 plain=%s" % plain)


def test_fullfit_unsmeared_and_offsets(eng, orc):
    cols = synth.gen_semilep(3000, 42)
    an = analyses.semilep_full()
    g = _run(eng, an, cols, V=1, first_event_id=77777)
    o = orc.run(an, cols, V=1, first_event_id=77777)
    assert_parity(g, o, what="full fit unsmeared")


def test_fullfit_all_multiplicities_with_hadtop_cut(eng, orc):
    """Events with 0..12 jets reach the fit (n < 4 is +inf); the hadronic
    triplet cut in the same chain; a loose threshold so that many survive."""
    cols = synth.gen_semilep(1200, 43, n_mean=5.5, n_min=0, n_max=12)
    cuts = [("lep_pt_min", 25.0), ("wnu_solvable",), ("hadtop_chi2_max", 30.0), ("ttbar_chi2_max", 60.0)]
    an = analyses.semilep_full(sigma_jet=0.05, sigma_met=5.0, sigma_t=15.0, sigma_W=10.0, cuts=cuts)
    g = _run(eng, an, cols, V=5, seed=8)
    o = orc.run(an, cols, seed=8, V=5)
    assert_parity(g, o, what="full fit multiplicities")


def test_fullfit_in_a_batch(eng, orc):
    from paper_2211_14346_gb300 import DeviceColumns
    an = analyses.semilep_full(sigma_jet=0.10, sigma_met=10.0)
    aid = eng.define(an)
    aid2 = eng.define(analyses.config2())
    chunks = [synth.gen_semilep(n, 50 + i) for i, n in enumerate((700, 1, 900))]
    items = [dict(aid=aid, cols=DeviceColumns(c), V=8, seed=3, first_event_id=10000 * i) for i, c in enumerate(chunks)]
    items.append(dict(aid=aid2, cols=DeviceColumns(chunks[0]), V=8, seed=3, first_event_id=0))
    res = [o.numpy() for o in eng.run_batch(items)]
    for i, c in enumerate(chunks):
        o = orc.run(an, c, seed=3, V=8, first_event_id=10000 * i)
        assert_parity(res[i], o, what="batched full fit %d" % i)
    o = orc.run(analyses.config2(), chunks[0], seed=3, V=8)
    assert_parity(res[3], o, what="batched hadronic-only beside it")
