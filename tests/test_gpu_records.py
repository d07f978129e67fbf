"""Per-cut variable recording (Sect. 3) on the GPU against the oracle:
the same (event, level) records, in that order, in every device-resident
entry point (fast and plain forms, batched, allocation-free), measured
variables bit-equal, reconstructed means within 1e-5; capacity overflow and
execution-order invariance."""
import ctypes as C

import numpy as np
import pytest

import synth
from synth import analyses
from tests.parity import assert_parity, assert_records

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


def _rec(an, levels, vars_):
    an = dict(an)
    an["record"] = dict(levels=levels, vars=vars_)
    return an


def _run(eng, an, cols, V, seed, plain=False, first=0):
    from paper_2211_14346_gb300 import DeviceColumns
    aid = eng.define(an)
    g = eng.run_device(aid, DeviceColumns(cols), V=V, seed=seed, plain=plain, first_event_id=first).numpy()
    assert eng.device_error() == 0
    return aid, g


@pytest.mark.parametrize("plain", [False, True])
@pytest.mark.parametrize("V", [16, 64])
def test_semilep_all_levels(eng, orc, plain, V):
    cols = synth.gen_semilep(2000, 51)
    an = _rec(analyses.config2(), list(range(6)), ["njets", "lep_pt", "met", "reco0"])
    _, g = _run(eng, an, cols, V, 501, plain)
    o = orc.records(an, cols, seed=501, V=V)
    assert_parity(g, o["run"], what="semilep records run")
    assert g["n_records"] == len(o["event"])
    assert_records(g["records"], o, an, what="semilep V=%d plain=%s" % (V, plain))


@pytest.mark.parametrize("plain", [False, True])
def test_dilep_levels(eng, orc, plain):
    cols = synth.gen_dilep(600, 52)
    an = _rec(analyses.config3(), [1, 3, 4], ["met", "reco0", "reco3", "nbtag"])
    _, g = _run(eng, an, cols, 8, 502, plain)
    o = orc.records(an, cols, seed=502, V=8)
    assert_parity(g, o["run"], model="dilep", what="dilep records run")
    assert_records(g["records"], o, an, what="dilep plain=%s" % plain)


def test_fullfit_and_many_variations(eng, orc):
    cols = synth.gen_semilep(60, 53)
    an = _rec(analyses.semilep_full(0.10, 10.0), [0, 4, 5], ["reco1", "reco2", "njets", "none"])
    _, g = _run(eng, an, cols, 300, 503)
    o = orc.records(an, cols, seed=503, V=300)
    assert_records(g["records"], o, an, what="fullfit V=300")


def test_capacity_overflow_counts_all(eng, orc):
    from paper_2211_14346_gb300 import DeviceColumns
    cols = synth.gen_semilep(500, 54)
    an = _rec(analyses.config2(), [0, 5], ["njets"])
    aid = eng.define(an)
    out = eng.results_for(aid, cols.n_events, record_cap=25)
    g = eng.run_device(aid, DeviceColumns(cols), V=4, seed=7, out=out).numpy()
    o = orc.records(an, cols, seed=7, V=4)
    assert g["n_records"] == len(o["event"]) > 25
    assert len(g["records"]) == 25
    # records come in (event, level) order: the first 25 are written
    assert np.array_equal(g["records"]["event"], o["event"][:25])
    assert np.array_equal(g["records"]["level"], o["level"][:25])


def test_no_levels_no_records(eng):
    from paper_2211_14346_gb300 import DeviceColumns
    cols = synth.gen_semilep(300, 55)
    an = analyses.config2()
    aid = eng.define(an)
    out = eng.results_for(aid, cols.n_events, record_cap=100)
    g = eng.run_device(aid, DeviceColumns(cols), V=4, seed=7, out=out).numpy()
    assert g["n_records"] == 0


def test_records_ignore_execution_order(eng, orc):
    from paper_2211_14346_gb300 import DeviceColumns
    cols = synth.gen_semilep(800, 56)
    an = _rec(analyses.config2(), list(range(6)), ["njets", "met"])
    aid = eng.define(an)
    dc = DeviceColumns(cols)
    a = eng.run_device(aid, dc, V=8, seed=9).numpy()
    eng.set_exec_order(aid, [5, 4, 3, 2, 1, 0])
    b = eng.run_device(aid, dc, V=8, seed=9).numpy()
    assert np.array_equal(a["records"], b["records"])
    assert_records(b["records"], orc.records(an, cols, seed=9, V=8), an, what="reordered")


def test_batched_chunks_record(eng, orc):
    from paper_2211_14346_gb300 import DeviceColumns
    an_s = _rec(analyses.config2(), [2, 5], ["lep_pt", "reco0"])
    an_d = _rec(analyses.config3(), [3, 4], ["reco0", "met"])
    cs, cd = synth.gen_semilep(1500, 57), synth.gen_dilep(300, 58)
    a_s, a_d = eng.define(an_s), eng.define(an_d)
    items = [dict(aid=a_s, cols=DeviceColumns(cs), V=16, seed=11, first_event_id=100),
             dict(aid=a_d, cols=DeviceColumns(cd), V=8, seed=12, first_event_id=200)]
    rs, rd = [x.numpy() for x in eng.run_batch(items)]
    assert eng.device_error() == 0
    assert_records(rs["records"], orc.records(an_s, cs, seed=11, V=16, first_event_id=100), an_s, what="batch s")
    assert_records(rd["records"], orc.records(an_d, cd, seed=12, V=8, first_event_id=200), an_d, what="batch d")


def test_noalloc_records(eng, orc):
    from paper_2211_14346_gb300 import DeviceColumns, _lib, analysis_desc, CUDA_STREAM_LEGACY
    import torch
    cols = synth.gen_semilep(700, 59)
    an = _rec(analyses.config2(), [0, 3, 5], ["nbtag", "reco1"])
    aid = eng.define(an)
    dc = DeviceColumns(cols)
    out = eng.results_for(aid, cols.n_events)
    desc, keep = analysis_desc(an)
    lib = _lib.load()
    st = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
    _lib.check(lib.hf_run_device_noalloc(C.byref(desc), C.byref(dc.struct()), cols.n_events, 0, 13, 4,
                                         C.byref(out.struct()), C.c_void_p(st)))
    torch.cuda.synchronize()
    g = out.numpy()
    assert_records(g["records"], orc.records(an, cols, seed=13, V=4), an, what="noalloc")


def test_many_levels_fill_several_staging_rounds(eng, orc):
    """Sixteen cut levels, ten of them passed by every event: up to 4096
    records per block of 256 events, written in three shared-memory rounds."""
    cols = synth.gen_semilep(1200, 60)
    base = analyses.config2()
    an = analyses.with_cuts(base, [("njets_min", 0)] * 10 + list(base["cuts"]))
    an = _rec(an, list(range(16)), ["njets", "reco0", "met", "nbtag"])
    _, g = _run(eng, an, cols, 4, 504)
    o = orc.records(an, cols, seed=504, V=4)
    assert g["n_records"] == len(o["event"]) > 1200 * 10
    assert_records(g["records"], o, an, what="16 levels")
