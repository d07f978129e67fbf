"""Pins of the oracle's lepton smearing (Sect. 4, ttH_sci: a 1 % resolution
on every measured energy and momentum): lepton l of a unit is scaled by
1 + sigma_lep z[14 + l], z the unit's Philox normals.  Checked through the
published pieces (unit_normals, w_pz, the pT threshold), not through the
unit evaluation."""
import math

import numpy as np
import pytest

import synth
from synth import analyses


def _an(sigma_lep, cuts):
    an = analyses.semilep(sigma_jet=0.01, sigma_met=1.0, cuts=cuts)
    an["sigma_lep"] = sigma_lep
    return an


def test_zero_resolution_changes_nothing(orc):
    cols = synth.gen_semilep(500, 71)
    a = orc.run(analyses.config2(), cols, seed=4, V=8)
    an = analyses.config2()
    an["sigma_lep"] = 0.0
    b = orc.run(an, cols, seed=4, V=8)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_lepton_pt_cut_sees_the_smeared_lepton(orc):
    """Unit passes pT > thr iff s pT > thr, s = 1 + sigma_lep z[14]."""
    cols = synth.gen_semilep(150, 72)
    thr, sl = 40.0, 0.05
    an = _an(sl, [("lep_pt_min", thr), ("wnu_solvable",), ("hadtop_chi2_max", 1e9)])
    V = 8
    r = orc.run(an, cols, seed=8, V=V, unit_passed=True)
    s32 = float(np.float32(sl))
    lep = cols.lep.reshape(-1, 4).astype(np.float64)
    flips = 0
    for e in range(cols.n_events):
        pt = math.hypot(lep[e, 0], lep[e, 1])
        for v in range(V):
            s = 1.0 + s32 * orc.unit_normals(8, e, v)[14]
            if abs(s * pt - thr) < 1e-9 * thr:
                continue  # too close to the threshold for this closed form
            assert (r["unit_passed"][e, v] >= 1) == (s * pt > thr), (e, v)
            flips += (s * pt > thr) != (pt > thr)
    assert flips > 0  # the smearing moves some units across the threshold


def test_neutrino_pz_uses_the_smeared_lepton(orc):
    cols = synth.gen_semilep(60, 73)
    sl = 0.05
    an = _an(sl, [("wnu_solvable",), ("hadtop_chi2_max", 1e9)])
    s32 = float(np.float32(sl))
    sm = float(np.float32(an["sigma_met"]))
    mW = float(np.float32(an["mW"]))
    lep = cols.lep.reshape(-1, 4).astype(np.float64)
    met = cols.met.reshape(-1, 2).astype(np.float64)
    checked = 0
    for e in range(cols.n_events):
        for v in range(3):
            u = orc.unit(an, cols, e, v, seed=12)
            if u["passed"] != 2:
                continue
            z = orc.unit_normals(12, e, v)
            ok, pz, _ = orc.w_pz(lep[e] * (1.0 + s32 * z[14]), met[e, 0] + sm * z[12], met[e, 1] + sm * z[13], mW)
            assert ok and u["q"][2] == pz, (e, v)
            checked += 1
    assert checked > 20


@pytest.mark.parametrize("sl", [0.01, 0.05])
def test_dilepton_leptons_take_their_own_normals(orc, sl):
    """Lepton 1 is scaled by 1 + sigma_lep z[14] and lepton 2 by
    1 + sigma_lep z[15]: the unit's best m_ttbar is the one the pairing
    solver gives for the leptons scaled here by those factors (jets and MET
    unsmeared)."""
    cols = synth.gen_dilep(60, 74)
    an = analyses.dilep(sigma_jet=0.0, sigma_met=0.0)
    an["sigma_lep"] = sl
    seed = 21
    s32 = float(np.float32(sl))
    lep = cols.lep.reshape(-1, 2, 4).astype(np.float64)
    for e in range(cols.n_events):
        z = orc.unit_normals(seed, e, 0)
        lep[e, 0] *= 1.0 + s32 * z[14]
        lep[e, 1] *= 1.0 + s32 * z[15]
    n_ok = 0
    for e in range(cols.n_events):
        u = orc.unit(an, cols, e, 0, seed=seed)
        if u["passed"] < 4 or u["idx"][0] < 0:
            continue
        lo = int(cols.jet_off[e])
        jets = cols.jets.reshape(-1, 4).astype(np.float64)
        b1, b2 = jets[lo + u["idx"][0]], jets[lo + u["idx"][1]]
        met = cols.met.reshape(-1, 2).astype(np.float64)[e]
        sols, _ = orc.dilep_pairing(lep[e, 0], b1, lep[e, 1], b2, met[0], met[1],
                                    float(np.float32(an["mW"])), float(np.float32(an["mt"])))
        mtt = [orc.mass((b1 + lep[e, 0] + s["nu1"]) + (b2 + lep[e, 1] + s["nu2"])) for s in sols]
        # the sums here are grouped differently from the oracle's: equal to rounding
        assert sols and abs(min(mtt) - u["q"][3]) <= 1e-12 * u["q"][3], e
        n_ok += 1
    assert n_ok > 3
