"""Pins of the oracle's best-of-variations reduction (Sect. 4, ttH_sci: only
the most probable solution over the pseudo-experiments is kept)."""
import numpy as np

import synth
from synth import analyses


def test_single_variation_equals_the_mean(orc):
    """V = 1: the best variation is the only one, so the per-event result is
    the run's mean and the histogram the run's."""
    cols = synth.gen_semilep(300, 61)
    an = analyses.config2()
    b = orc.best_of(an, cols, seed=7, V=1)
    r = orc.run(an, cols, seed=7, V=1)
    assert np.array_equal(b["best_v"] >= 0, r["mask"].astype(bool))
    assert np.array_equal(b["reco"], r["reco"])
    assert np.array_equal(b["hist"], r["hist"])


def test_semilep_score_is_the_hadronic_chi2_of_the_smeared_jets(orc):
    """The score, recomputed from the published smearing (jet i scaled by
    1 + sigma_jet z_i, z from the unit's Philox normals) and the hadronic-top
    fit of those jets, is minimal at the chosen variation, ties to the first."""
    cols = synth.gen_semilep(40, 62)
    an = analyses.config2()
    V, seed = 12, 9
    b = orc.best_of(an, cols, seed=seed, V=V)
    nc = len(an["cuts"])
    sj = float(np.float32(an["sigma_jet"]))
    checked = 0
    for e in range(cols.n_events):
        lo, hi = int(cols.jet_off[e]), int(cols.jet_off[e + 1])
        jets = cols.jets.reshape(-1, 4)[lo:hi].astype(np.float64)
        scores = []
        for v in range(V):
            if orc.unit(an, cols, e, v, seed=seed)["passed"] != nc:
                scores.append(np.inf)
                continue
            z = orc.unit_normals(seed, e, v)
            sm = np.array([jets[i] * (1.0 + sj * z[i]) for i in range(len(jets))])
            scores.append(orc.hadtop(sm, float(np.float32(an["mW"])), float(np.float32(an["mt"])),
                                     float(np.float32(an["sigma_W"])), float(np.float32(an["sigma_t"])))["chi2"])
        scores = np.array(scores)
        if np.isinf(scores).all():
            assert b["best_v"][e] == -1
            continue
        want = int(np.argmin(scores))  # first of equal minima
        assert b["best_v"][e] == want, (e, b["best_v"][e], want)
        assert b["score"][e] == scores[want]
        checked += 1
    assert checked >= 10


def test_choice_ignores_the_cut_order(orc):
    """Every cut is a pure predicate of the unit, so the surviving units and
    hence the best one do not depend on the user order of the cuts."""
    cols = synth.gen_semilep(80, 63)
    an = analyses.config2()
    rev = analyses.with_cuts(an, list(reversed(an["cuts"])))
    a = orc.best_of(an, cols, seed=3, V=8)
    b = orc.best_of(rev, cols, seed=3, V=8)
    assert np.array_equal(a["best_v"], b["best_v"])
    assert np.array_equal(a["reco"], b["reco"])
    assert np.array_equal(a["hist"], b["hist"])


def test_dilep_best_is_the_smallest_m_ttbar(orc):
    cols = synth.gen_dilep(30, 64)
    an = analyses.config3()
    V = 6
    b = orc.best_of(an, cols, seed=5, V=V)
    nc = len(an["cuts"])
    for e in range(cols.n_events):
        mtt = [orc.unit(an, cols, e, v, seed=5)["q"][3] if orc.unit(an, cols, e, v, seed=5)["passed"] == nc
               else np.inf for v in range(V)]
        if np.isinf(mtt).all():
            assert b["best_v"][e] == -1
        else:
            assert b["best_v"][e] == int(np.argmin(mtt))
            assert b["reco"][e, 3] == min(mtt)
    assert b["hist"].sum() == (b["best_v"] >= 0).sum() > 0
