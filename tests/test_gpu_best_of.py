"""GPU parity of best-of-variations (Sect. 4, ttH_sci: of the solutions over
the pseudo-experiments only the most probable is kept) with the FP64 oracle
(oracle.best_of): per event the chosen variation (bit-exact), its
reconstructed quantities (within 1e-5) and the histogram filled once per
selected event (bit-exact); the cut flow, mask and number of surviving
variations are those of the mean mode (oracle.run).  The fit score is the
triplet chi2 of Eq. 1, the full Eq. 1 chi2 with the full fit, and m_ttbar
of the chosen solution in the dilepton model."""
import ctypes as C

import numpy as np
import pytest

import synth
from synth import analyses
from tests.parity import assert_reco

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


def _best(an):
    return dict(an, per_event="best")


def _check(g, an, cols, orc, *, V, seed, first=0, model="semilep", what=""):
    o = orc.run(an, cols, seed=seed, V=V, first_event_id=first)
    b = orc.best_of(an, cols, seed=seed, V=V, first_event_id=first)
    assert np.array_equal(g["cutflow"].astype(np.uint64), o["cutflow"]), what
    assert np.array_equal(g["mask"], o["mask"]), what
    assert np.array_equal(g["n_surv"].astype(np.uint16), o["n_surv"]), what
    want_v = np.where(b["best_v"] >= 0, b["best_v"], 0xffff).astype(np.uint16)
    bad = np.nonzero(g["best_v"] != want_v)[0]
    assert bad.size == 0, "%s: best variation differs at events %s: gpu %s oracle %s (scores %s)" % (
        what, bad[:10], g["best_v"][bad[:5]], want_v[bad[:5]], b["score"][bad[:5]])
    assert np.array_equal(g["hist"].astype(np.uint64), b["hist"]), what
    assert_reco(g["reco"], b["reco"], model=model, what=what)
    return b


def _run(eng, an, cols, **kw):
    from paper_2211_14346_gb300 import DeviceColumns
    aid = eng.define(an)
    out = eng.run_device(aid, DeviceColumns(cols), **kw).numpy()
    assert eng.device_error() == 0
    return out


@pytest.mark.parametrize("V", [1, 5, 16, 40])
def test_semilep_triplet_fit(eng, orc, V):
    cols = synth.gen_semilep(2000, 301)
    an = _best(analyses.semilep(sigma_jet=0.10, sigma_met=10.0))
    g = _run(eng, an, cols, V=V, seed=5)
    b = _check(g, an, cols, orc, V=V, seed=5, what="semilep V=%d" % V)
    assert (b["best_v"] >= 0).sum() > 100


def test_semilep_one_percent_resolution_and_leptons(eng, orc):
    """The ttH_sci resolutions (1 % jets and leptons, 1 GeV MET): the
    variations' chi2 lie close together, so that many events need the FP64
    argmin."""
    cols = synth.gen_semilep(1500, 302)
    an = _best(analyses.semilep(sigma_jet=0.01, sigma_met=1.0, sigma_lep=0.01))
    g = _run(eng, an, cols, V=16, seed=7, first_event_id=(1 << 33) + 11)
    _check(g, an, cols, orc, V=16, seed=7, first=(1 << 33) + 11, what="semilep 1%")


def test_semilep_full_fit(eng, orc):
    cols = synth.gen_semilep(400, 303)
    an = _best(analyses.semilep_full(0.10, 10.0, sigma_lep=0.01))
    g = _run(eng, an, cols, V=8, seed=9)
    b = _check(g, an, cols, orc, V=8, seed=9, what="full fit")
    assert (b["best_v"] >= 0).sum() > 10


def test_dilepton_tth_sci(eng, orc):
    cols = synth.gen_dilep(300, 304)
    an = _best(analyses.tth_sci())
    g = _run(eng, an, cols, V=64, seed=11)
    b = _check(g, an, cols, orc, V=64, seed=11, model="dilep", what="dilep ttH_sci")
    assert (b["best_v"] >= 0).sum() > 5


def test_many_variations(eng, orc):
    cols = synth.gen_semilep(60, 305)
    an = _best(analyses.semilep(sigma_jet=0.01, sigma_met=1.0, sigma_lep=0.01))
    g = _run(eng, an, cols, V=1024, seed=13)
    _check(g, an, cols, orc, V=1024, seed=13, what="V=1024")


def test_identical_variations_tie_to_the_first(eng, orc):
    """Without smearing every variation of an event is the same unit: all
    scores tie and the definition keeps variation 0; the histogram holds each
    selected event once."""
    cols = synth.gen_semilep(1000, 306)
    an = _best(analyses.semilep())
    g = _run(eng, an, cols, V=6, seed=0)
    o = orc.run(analyses.semilep(), cols, seed=0, V=1)
    sel = o["mask"].astype(bool)
    assert sel.sum() > 50
    assert (g["best_v"][sel] == 0).all() and (g["best_v"][~sel] == 0xffff).all()
    assert np.array_equal(g["hist"].astype(np.uint64), o["hist"])
    assert_reco(g["reco"], o["reco"], what="identical variations")


def test_noalloc_and_list_overflow(orc):
    """The allocation-free entry point with best-of, on identical variations
    (every survivor is listed for its FP64 score): 1,500 selected events x 64
    variations exceed the 65,536-entry recheck list, the rest are chosen
    inline."""
    import torch
    from paper_2211_14346_gb300 import build, DeviceColumns, DeviceResults, _lib, CUDA_STREAM_LEGACY
    from paper_2211_14346_gb300 import analysis_desc
    build.build()
    lib = _lib.load()
    an = _best(analyses.semilep())
    cols = synth.gen_semilep(3000, 307)
    d, keep = analysis_desc(an)
    dc = DeviceColumns(cols)
    cs = dc.struct()
    out = DeviceResults(cols.n_events, len(an["cuts"]), an["hist"][0])
    rs = out.struct()
    stream = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
    st = lib.hf_run_device_noalloc(C.byref(d), C.byref(cs), cols.n_events, 0, 3, 64, C.byref(rs), C.c_void_p(stream))
    assert st == _lib.HF_OK, lib.hf_last_error(None)
    torch.cuda.synchronize()
    g = out.numpy()
    o = orc.run(analyses.semilep(), cols, seed=0, V=1)
    sel = o["mask"].astype(bool)
    assert sel.sum() * 64 > 65536
    assert (g["best_v"][sel] == 0).all() and (g["best_v"][~sel] == 0xffff).all()
    assert np.array_equal(g["n_surv"][sel], np.full(sel.sum(), 64, np.uint16))
    assert np.array_equal(g["hist"].astype(np.uint64), o["hist"])
    assert_reco(g["reco"], o["reco"], what="noalloc identical variations")
    # smeared, against the oracle
    cols2 = synth.gen_semilep(1200, 308)
    an2 = _best(analyses.semilep(sigma_jet=0.05, sigma_met=5.0))
    d2, keep2 = analysis_desc(an2)
    dc2 = DeviceColumns(cols2)
    cs2 = dc2.struct()
    out2 = DeviceResults(cols2.n_events, len(an2["cuts"]), an2["hist"][0])
    rs2 = out2.struct()
    st = lib.hf_run_device_noalloc(C.byref(d2), C.byref(cs2), cols2.n_events, 40, 17, 12, C.byref(rs2),
                                   C.c_void_p(stream))
    assert st == _lib.HF_OK, lib.hf_last_error(None)
    torch.cuda.synchronize()
    _check(out2.numpy(), an2, cols2, orc, V=12, seed=17, first=40, what="noalloc smeared")


def test_submit_and_fetch(eng, orc):
    from paper_2211_14346_gb300 import PinnedColumns
    cols = synth.gen_semilep(800, 309)
    an = _best(analyses.semilep(sigma_jet=0.10, sigma_met=10.0))
    aid = eng.define(an)
    t = eng.submit(aid, PinnedColumns(cols), V=16, seed=19, first_event_id=5)
    g = eng.fetch(aid, t, cols.n_events)
    _check(g, an, cols, orc, V=16, seed=19, first=5, what="submit/fetch")


def test_rejected_where_not_supported(eng):
    from paper_2211_14346_gb300 import DeviceColumns, HFError
    cols = synth.gen_semilep(50, 310)
    an = _best(analyses.semilep(sigma_jet=0.10))
    aid = eng.define(an)
    with pytest.raises(HFError):
        eng.run_device(aid, DeviceColumns(cols), V=4, plain=True)
    with pytest.raises(HFError):
        eng.run_batch([dict(aid=aid, cols=DeviceColumns(cols), V=4)])
    rec = dict(an, record=dict(levels=[0], vars=["njets"]))
    aid2 = eng.define(rec)
    with pytest.raises(HFError):
        eng.run_device(aid2, DeviceColumns(cols), V=4)
