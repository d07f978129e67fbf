"""GPU parity of lepton smearing (Sect. 4: every measured object is smeared in
the pseudo-experiments; lepton l of a unit scaled by 1 + sigma_lep z[14 + l])
with the FP64 oracle: bit-exact mask, cut flow, histogram and n_surv, reco
within 1e-5.  With sigma_lep != 0 the lepton pT cut and the W-mass
solvability are decided per unit (stage 2), the p_z of the survivors comes
from FP64, and the full fit and the dilepton solve take the smeared leptons."""
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
def test_semilep_one_percent_leptons(eng, orc, plain):
    cols = synth.gen_semilep(3000, 201)
    an = analyses.semilep(sigma_jet=0.10, sigma_met=10.0, sigma_lep=0.01)
    g = _run(eng, an, cols, V=16, seed=41, plain=plain)
    o = orc.run(an, cols, seed=41, V=16)
    assert_parity(g, o, what="semilep sigma_lep 1%% plain=%s" % plain)


def test_semilep_wide_leptons_and_tight_pt_cut(eng, orc):
    """sigma_lep = 0.15 against a 45 GeV lepton cut moves many units across
    the cut between variations; the cut sits in the user order after the
    MET cut, so it is evaluated per unit in the middle of the chain."""
    cols = synth.gen_semilep(2000, 202)
    cuts = [("njets_min", 4), ("met_min", 20.0), ("lep_pt_min", 45.0), ("nbtag_min", 1),
            ("wnu_solvable",), ("hadtop_chi2_max", 10.0)]
    an = analyses.semilep(sigma_jet=0.05, sigma_met=5.0, sigma_lep=0.15, cuts=cuts)
    g = _run(eng, an, cols, V=12, seed=43, first_event_id=(1 << 33) + 3)
    o = orc.run(an, cols, seed=43, V=12, first_event_id=(1 << 33) + 3)
    assert 0 < o["cutflow"][3] < o["cutflow"][2]  # the smeared lepton cut rejects some units
    assert_parity(g, o, what="semilep sigma_lep 15%")


def test_lepton_only_smearing(eng, orc):
    """Only the lepton is smeared (jets and MET exact)."""
    cols = synth.gen_semilep(2000, 203)
    an = analyses.semilep(sigma_lep=0.05, cuts=[("njets_min", 4), ("lep_pt_min", 35.0), ("wnu_solvable",),
                                                ("hadtop_chi2_max", 10.0)])
    g = _run(eng, an, cols, V=8, seed=45)
    o = orc.run(an, cols, seed=45, V=8)
    assert_parity(g, o, what="lepton-only smearing")


def test_full_fit_with_smeared_leptons(eng, orc):
    cols = synth.gen_semilep(400, 204)
    an = analyses.semilep_full(0.10, 10.0, sigma_lep=0.01)
    g = _run(eng, an, cols, V=8, seed=47)
    o = orc.run(an, cols, seed=47, V=8)
    assert o["cutflow"][-1] > 0
    assert_parity(g, o, what="full fit sigma_lep")


@pytest.mark.parametrize("plain", [False, True])
def test_dilepton_tth_sci_resolution(eng, orc, plain):
    """The paper's ttH_sci resolution: 1 % on jets, leptons and MET (1 GeV),
    with a lepton pT cut added to the chain (now per unit)."""
    cols = synth.gen_dilep(300, 205)
    base = analyses.tth_sci()
    an = analyses.with_cuts(base, [("lep_os",), ("lep_pt_min", 30.0)] + base["cuts"][1:])
    g = _run(eng, an, cols, V=64, seed=49, plain=plain)
    o = orc.run(an, cols, seed=49, V=64)
    assert o["cutflow"][2] < o["cutflow"][1]
    assert_parity(g, o, model="dilep", what="dilep ttH_sci plain=%s" % plain)


def test_many_variations_with_smeared_leptons(eng, orc):
    cols = synth.gen_semilep(60, 206)
    an = analyses.semilep(sigma_jet=0.01, sigma_met=1.0, sigma_lep=0.01)
    g = _run(eng, an, cols, V=1024, seed=51)
    o = orc.run(an, cols, seed=51, V=1024)
    assert_parity(g, o, what="V=1024 sigma_lep")


def test_sigma_lep_rejected_out_of_range(eng):
    from paper_2211_14346_gb300 import HFError
    with pytest.raises(HFError):
        eng.define(analyses.semilep(sigma_lep=0.2))
