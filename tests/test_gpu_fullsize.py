"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (autotuned tiles, device-resident columns):
the whole chunk runs on the GPU, and contiguous blocks of events at seeded
random offsets are compared with the FP64 oracle run on just those events
(their global event ids, hence their smearing, unchanged): bit-exact mask and
surviving-variation counts, reco within 1e-5.  Properties that hold at any
size are checked on the whole chunk: cut flow starts at N V and never
increases, its last entry equals the sum of n_surv and of the histogram, the
mask is n_surv > 0, and the FP64 recheck stays a small fraction."""
import functools

import numpy as np
import pytest

import synth
from synth import analyses
from tests.parity import assert_reco

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=2)
def _semilep_10M():
    return synth.gen_semilep(10_000_000, 2)


@pytest.fixture(scope="module")
def eng():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_14346_gb300 import build, Engine
    build.build()
    e = Engine(0)
    yield e
    e.close()


def _properties(g, N, V, max_recheck_frac):
    cf = g["cutflow"].astype(np.int64)
    assert cf[0] == N * V
    assert np.all(np.diff(cf) <= 0)
    assert cf[-1] == int(g["n_surv"].astype(np.int64).sum()) == int(g["hist"].astype(np.int64).sum())
    assert np.array_equal(g["mask"], (g["n_surv"] > 0).astype(np.uint8))
    assert g["recheck_count"] <= max(max_recheck_frac * N * V, 50)


def _sampled(orc, an, cols, g, *, V, seed, blocks, size, model, rng_seed):
    rng = np.random.default_rng(rng_seed)
    N = cols.n_events
    for lo in rng.integers(0, N - size, blocks):
        lo = int(lo)
        o = orc.run(an, cols.slice(lo, lo + size), seed=seed, V=V, first_event_id=lo)
        sl = slice(lo, lo + size)
        assert np.array_equal(g["mask"][sl], o["mask"]), lo
        assert np.array_equal(g["n_surv"][sl].astype(np.uint16), o["n_surv"]), lo
        assert_reco(g["reco"][sl], o["reco"], o["reco_abs"], model=model, what="events %d.." % lo)


def _run(eng, an, cols, *, V, seed, tune_events):
    from paper_2211_14346_gb300 import DeviceColumns
    aid = eng.define(an)
    dc = DeviceColumns(cols)
    eng.autotune(aid, dc.slice(0, min(cols.n_events, tune_events)), V=V, seed=seed)
    g = eng.run_device(aid, dc, V=V, seed=seed).numpy()
    assert eng.device_error() == 0
    return g


def test_semilep_smeared_10M_x16(eng, orc):
    """The headline: 10,000,000 semileptonic events x 16 variations."""
    N, V, seed = 10_000_000, 16, 1002
    cols = _semilep_10M()
    an = analyses.config2()
    g = _run(eng, an, cols, V=V, seed=seed, tune_events=1_000_000)
    _properties(g, N, V, 0.002)
    _sampled(orc, an, cols, g, V=V, seed=seed, blocks=8, size=64, model="semilep", rng_seed=11)


def test_semilep_smeared_10M_x16_whole_chunk_oracle(eng):
    """The headline step compared whole with the FP64 oracle run in spawned
    processes on the host cores over the same 10,000,000 events x 16
    variations: bit-exact cut flow, histogram, mask and n_surv of every event,
    reco within 1e-5 for every event."""
    from tests import oracle_pool
    N, V, seed = 10_000_000, 16, 1002
    cols = _semilep_10M()
    an = analyses.config2()
    g = _run(eng, an, cols, V=V, seed=seed, tune_events=1_000_000)
    o = oracle_pool.run(an, cols, seed=seed, V=V)
    assert np.array_equal(g["cutflow"].astype(np.uint64), o["cutflow"]), (g["cutflow"], o["cutflow"])
    assert np.array_equal(g["hist"].astype(np.uint64), o["hist"])
    bad = np.nonzero(g["mask"] != o["mask"])[0]
    assert bad.size == 0, bad[:10]
    bad = np.nonzero(g["n_surv"].astype(np.uint16) != o["n_surv"])[0]
    assert bad.size == 0, bad[:10]
    assert_reco(g["reco"], o["reco"], o["reco_abs"], model="semilep", what="10M x 16 whole chunk")


def test_semilep_unsmeared_10M(eng, orc):
    N = 10_000_000
    cols = _semilep_10M()
    an = analyses.config1()
    g = _run(eng, an, cols, V=1, seed=0, tune_events=1_000_000)
    _properties(g, N, 1, 0.002)
    _sampled(orc, an, cols, g, V=1, seed=0, blocks=8, size=256, model="semilep", rng_seed=12)


def test_dilep_2M_x64(eng, orc):
    """The ttH dilepton configuration: 2,000,000 events x 64 variations."""
    N, V, seed = 2_000_000, 64, 1003
    cols = synth.gen_dilep(N, 3)
    an = analyses.config3()
    g = _run(eng, an, cols, V=V, seed=seed, tune_events=50_000)
    _properties(g, N, V, 0.08)
    _sampled(orc, an, cols, g, V=V, seed=seed, blocks=4, size=24, model="dilep", rng_seed=13)


def test_batched_workload_512_chunks(eng, orc):
    """The batched workload of bench.py (512 chunks of 1k-100k events, both
    models, V in {1, 8, 64}) through hf_run_batch: whole-chunk properties for
    every chunk and oracle parity on sampled events of sampled chunks."""
    import bench
    from paper_2211_14346_gb300 import DeviceColumns
    spec = bench.batched_chunks(512, 100000)
    pool_n = max(c["n"] for c in spec)
    pcols = {0: synth.gen_semilep(max(pool_n, 400000), 2), 1: synth.gen_dilep(max(pool_n, 200000), 3)}
    pools = {k: DeviceColumns(v) for k, v in pcols.items()}
    ans = {0: analyses.config2(), 1: analyses.config3()}
    aids = {k: eng.define(v) for k, v in ans.items()}
    seeds = {0: 1002, 1: 1003}
    items, los = [], []
    for c in spec:
        pool = pools[c["model"]]
        lo = int(c["u"] * (pool.n_events - c["n"]))
        los.append(lo)
        items.append(dict(aid=aids[c["model"]], cols=pool.slice(lo, lo + c["n"]), V=c["V"],
                          seed=seeds[c["model"]], first_event_id=c["first"]))
    res = [o.numpy() for o in eng.run_batch(items)]
    assert eng.device_error() == 0
    for c, g in zip(spec, res):
        _properties(g, c["n"], c["V"], 0.08 if c["model"] == 1 else 0.002)
    rng = np.random.default_rng(14)
    for k in rng.choice(len(spec), 12, replace=False):
        c, g, lo = spec[k], res[k], los[k]
        m = c["model"]
        size = 16 if m == 1 else 64
        off = int(rng.integers(0, c["n"] - size))
        sub = pcols[m].slice(lo + off, lo + off + size)
        o = orc.run(ans[m], sub, seed=seeds[m], V=c["V"], first_event_id=c["first"] + off)
        sl = slice(off, off + size)
        assert np.array_equal(g["mask"][sl], o["mask"]), k
        assert np.array_equal(g["n_surv"][sl].astype(np.uint16), o["n_surv"]), k
        assert_reco(g["reco"][sl], o["reco"], o["reco_abs"], model="dilep" if m == 1 else "semilep",
                    what="chunk %d" % k)


def test_fullfit_2M_x16(eng, orc):
    """The full Eq. 1 fit workload of bench.py: 2,000,000 semileptonic events
    x 16 variations with the fit as the last cut."""
    N, V, seed = 2_000_000, 16, 1002
    cols = synth.gen_semilep(N, 2)
    an = analyses.semilep_full(0.10, 10.0)
    g = _run(eng, an, cols, V=V, seed=seed, tune_events=200_000)
    _properties(g, N, V, 0.002)
    _sampled(orc, an, cols, g, V=V, seed=seed, blocks=6, size=48, model="semilep", rng_seed=15)


def test_records_10M_x16_all_levels(eng, orc):
    """The records workload of bench.py: the headline with per-cut recording
    at every level.  Whole chunk: records in (event, level) order, the last
    level's events are the mask's, every recorded event also appears at each
    lower recorded level, and the first level's variables are the columns'.
    Sampled blocks of events: records equal to the oracle's."""
    from paper_2211_14346_gb300 import DeviceColumns
    from tests.parity import assert_records
    N, V, seed = 10_000_000, 16, 1002
    cols = _semilep_10M()
    an = analyses.config2()
    nc = len(an["cuts"])
    an["record"] = dict(levels=list(range(nc)), vars=["njets", "lep_pt", "met", "reco0"])
    aid = eng.define(an)
    dc = DeviceColumns(cols)
    eng.autotune(aid, dc.slice(0, 1_000_000), V=V, seed=seed)
    g = eng.run_device(aid, dc, V=V, seed=seed).numpy()
    assert eng.device_error() == 0
    rec = g["records"]
    assert g["n_records"] == len(rec)
    key = rec["event"].astype(np.int64) * 64 + rec["level"]
    assert np.all(np.diff(key) > 0)
    per_level = np.bincount(rec["level"].astype(np.int64), minlength=nc)
    assert np.all(np.diff(per_level) <= 0)
    assert np.array_equal(rec["event"][rec["level"] == nc - 1], np.nonzero(g["mask"])[0])
    lv0 = rec[rec["level"] == 0]
    n = np.diff(cols.jet_off.astype(np.int64))
    assert np.array_equal(lv0["value"][:, 0], n[lv0["event"]].astype(np.float32))
    rng = np.random.default_rng(16)
    for lo in rng.integers(0, N - 64, 6):
        lo = int(lo)
        sub = cols.slice(lo, lo + 64)
        o = orc.records(an, sub, seed=seed, V=V, first_event_id=lo)
        sel = (rec["event"] >= lo) & (rec["event"] < lo + 64)
        part = rec[sel].copy()
        part["event"] -= lo
        assert_records(part, o, an, what="records events %d.." % lo)
