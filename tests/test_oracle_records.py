"""Pins of the oracle's per-cut variable records (Sect. 3) against what the
columns and the cut flow fix independently of the unit evaluation."""
import numpy as np

import synth
from synth import analyses


def _with_record(an, levels, vars_):
    an = dict(an)
    an["record"] = dict(levels=levels, vars=vars_)
    return an


def test_stage1_levels_equal_brute_force_predicates(orc):
    """Unsmeared, V = 1, cuts on columns only: level k holds exactly the
    events that satisfy the first k + 1 predicates, computed here from the
    columns directly."""
    cols = synth.gen_semilep(400, 41)
    cuts = [("njets_min", 5), ("nbtag_min", 2), ("lep_pt_min", 40.0), ("hadtop_chi2_max", 10.0)]
    an = _with_record(analyses.semilep(cuts=cuts), [0, 1, 2], ["njets", "nbtag", "lep_pt", "met"])
    r = orc.records(an, cols)
    n = np.diff(cols.jet_off.astype(np.int64))
    nb = np.array([bin(int(b) & ((1 << int(k)) - 1)).count("1") for b, k in zip(cols.btag, n)])
    lep = cols.lep.reshape(-1, 4).astype(np.float64)
    pt = np.sqrt(lep[:, 0] ** 2 + lep[:, 1] ** 2)
    preds = [n >= 5, nb >= 2, pt > np.float32(40.0)]
    for k in range(3):
        want = np.nonzero(np.logical_and.reduce(preds[:k + 1]))[0]
        got = r["event"][r["level"] == k]
        assert np.array_equal(got, want), k
        assert want.size > 0
    sel = r["level"] == 2
    e = r["event"][sel]
    assert np.array_equal(r["value"][sel, 0], n[e].astype(np.float64))
    assert np.array_equal(r["value"][sel, 1], nb[e].astype(np.float64))
    assert np.array_equal(r["value"][sel, 2], pt[e].astype(np.float32).astype(np.float64))
    met = cols.met.reshape(-1, 2).astype(np.float64)
    assert np.array_equal(r["value"][sel, 3], np.sqrt(met[e, 0] ** 2 + met[e, 1] ** 2).astype(np.float32))


def test_single_variation_level_counts_are_the_cut_flow(orc):
    """V = 1: an event is recorded at level k iff its one unit passes cuts
    0..k, so the records per level are the cut flow's entries 1..n."""
    cols = synth.gen_semilep(300, 42)
    an = analyses.config2()
    nc = len(an["cuts"])
    an = _with_record(an, list(range(nc)), ["njets"])
    r = orc.records(an, cols, seed=5, V=1)
    counts = np.bincount(r["level"].astype(np.int64), minlength=nc)
    assert np.array_equal(counts, r["run"]["cutflow"][1:].astype(np.int64))


def test_last_level_is_the_mask_with_the_reco_means(orc):
    cols = synth.gen_semilep(300, 43)
    an = analyses.config2()
    nc = len(an["cuts"])
    an = _with_record(an, [0, nc - 1], ["reco0", "reco1", "reco2", "reco3"])
    r = orc.records(an, cols, seed=6, V=8)
    last = r["level"] == nc - 1
    assert np.array_equal(r["event"][last], np.nonzero(r["run"]["mask"])[0])
    assert np.array_equal(r["value"][last], r["run"]["reco"][r["event"][last]])
    assert not r["value"][~last].any()  # defaults below the last level
    # every event reaching the last level reaches every earlier one
    assert set(r["event"][last]) <= set(r["event"][r["level"] == 0])
