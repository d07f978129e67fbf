"""Parity of the CUDA path (fast and plain forms, device-resident and
asynchronous host submission) with the FP64 oracle, semileptonic model."""
import copy

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


def _gpu_run(eng, an, cols, *, V=1, seed=0, first_event_id=0, plain=False):
    from paper_2211_14346_gb300 import DeviceColumns
    aid = eng.define(an)
    dc = DeviceColumns(cols)
    out = eng.run_device(aid, dc, V=V, seed=seed, first_event_id=first_event_id, plain=plain)
    res = out.numpy()
    assert eng.device_error() == 0
    return res


@pytest.mark.parametrize("plain", [False, True])
def test_config1_small_bit_exact(eng, orc, plain):
    """10,000 semileptonic events, seed 1, no smearing (the small plain configuration)."""
    cols = synth.gen_semilep(10000, 1)
    an = analyses.config1()
    g = _gpu_run(eng, an, cols, plain=plain)
    o = orc.run(an, cols)
    assert_parity(g, o, what="config1 plain=%s" % plain)


@pytest.mark.parametrize("plain", [False, True])
def test_config2_smeared_bit_exact(eng, orc, plain):
    """Smeared semileptonic (jet scale N(1, 0.10), MET N(0, 10)), V = 16."""
    cols = synth.gen_semilep(3000, 2)
    an = analyses.config2()
    g = _gpu_run(eng, an, cols, V=16, seed=1002, plain=plain)
    o = orc.run(an, cols, seed=1002, V=16)
    assert_parity(g, o, what="config2 plain=%s" % plain)


@pytest.mark.parametrize("V", [1, 3, 5, 33, 64])
def test_variation_counts_and_event_offset(eng, orc, V):
    cols = synth.gen_semilep(700, 17)
    an = analyses.config2()
    g = _gpu_run(eng, an, cols, V=V, seed=77, first_event_id=123456789012)
    o = orc.run(an, cols, seed=77, V=V, first_event_id=123456789012)
    assert_parity(g, o, what="V=%d" % V)


def test_all_multiplicities_and_degenerate_events(eng, orc):
    """Events with 0..12 jets reach the triplet cut (no jet-count cut):
    n < 3 has chi2 = +inf and fails; ragged tails of every bucket."""
    cols = synth.gen_semilep(2600, 5, n_mean=5.0, n_min=0, n_max=12)
    an = analyses.semilep(sigma_jet=0.1, sigma_met=10.0,
                          cuts=[("lep_pt_min", 25.0), ("wnu_solvable",), ("hadtop_chi2_max", 10.0)])
    n = np.diff(cols.jet_off.astype(np.int64))
    assert set(range(0, 13)) <= set(n.tolist())
    g = _gpu_run(eng, an, cols, V=4, seed=9)
    o = orc.run(an, cols, seed=9, V=4)
    assert_parity(g, o, what="multiplicities")


def test_empty_and_single_event(eng, orc):
    an = analyses.config2()
    cols = synth.gen_semilep(1, 3)
    g = _gpu_run(eng, an, cols, V=16, seed=1)
    o = orc.run(an, cols, seed=1, V=16)
    assert_parity(g, o, what="N=1")
    empty = cols.slice(0, 0)
    g = _gpu_run(eng, an, empty, V=16, seed=1)
    assert g["cutflow"].sum() == 0 and g["hist"].sum() == 0


def test_paper_widths_and_loose_chi2(eng, orc):
    """Eq. 1 widths of the paper (11.5, 7.5) and a loose chi2 cut, so that
    many units survive and the histogram and argmin bands are exercised."""
    cols = synth.gen_semilep(2500, 8)
    cuts = [("njets_min", 3), ("wnu_solvable",), ("hadtop_chi2_max", 50.0)]
    an = analyses.semilep(sigma_jet=0.05, sigma_met=5.0, sigma_t=11.5, sigma_W=7.5, cuts=cuts)
    g = _gpu_run(eng, an, cols, V=8, seed=4)
    o = orc.run(an, cols, seed=4, V=8)
    assert_parity(g, o, what="paper widths")


def test_user_order_permutations_and_forced_exec_orders(eng, orc):
    """Any user order: identical selection, user-order cut flow equal to the
    oracle's; any forced execution order of the stage-2 cuts gives the same."""
    import itertools
    from paper_2211_14346_gb300 import DeviceColumns
    cols = synth.gen_semilep(1500, 12)
    base = analyses.config2()
    rng = np.random.default_rng(3)
    dc = DeviceColumns(cols)
    for trial in range(4):
        perm = rng.permutation(len(base["cuts"])) if trial else np.arange(len(base["cuts"]))
        an = analyses.with_cuts(base, [base["cuts"][p] for p in perm])
        o = orc.run(an, cols, seed=11, V=6)
        aid = eng.define(an)
        for order in itertools.permutations(range(len(an["cuts"]))):
            if rng.random() > 0.02 and order != tuple(range(len(an["cuts"]))):
                continue
            eng.set_exec_order(aid, list(order))
            g = eng.run_device(aid, dc, V=6, seed=11).numpy()
            assert_parity(g, o, what="perm %s exec %s" % (perm, order))


def test_scheduler_reorders_without_changing_results(eng, orc):
    """User order puts the triplet chi2 first: the scheduler, fed by measured
    pass rates and costs, runs the cheap MET cut first for the next chunks;
    every chunk still equals the oracle in the user's order."""
    from paper_2211_14346_gb300 import DeviceColumns
    cuts = [("hadtop_chi2_max", 10.0), ("njets_min", 4), ("met_min", 40.0), ("wnu_solvable",)]
    an = analyses.semilep(sigma_jet=0.1, sigma_met=10.0, cuts=cuts)
    aid = eng.define(an)
    for k in range(3):
        cols = synth.gen_semilep(1200, 100 + k)
        g = eng.run_device(aid, DeviceColumns(cols), V=8, seed=5, first_event_id=k * 10000).numpy()
        o = orc.run(an, cols, seed=5, V=8, first_event_id=k * 10000)
        assert_parity(g, o, what="chunk %d" % k)
    st = eng.sched_state(aid)
    assert sorted(st["order"].tolist()) == list(range(len(cuts)))
    assert st["evaluated"][0] > 0


def test_scheduler_with_eight_reorderable_cuts(eng, orc):
    """Eight stage-2 cuts (four triplet chi2 thresholds before four MET
    thresholds in the user order): beyond six cuts the scheduler scores the
    user order, the greedy order by rank and its neighbours.  With the cut
    flow completed in user order every unit must evaluate all cuts up to its
    first user-order failure, so the user order is the cheapest and is kept;
    every chunk equals the oracle."""
    from paper_2211_14346_gb300 import DeviceColumns
    cuts = [("hadtop_chi2_max", 40.0), ("hadtop_chi2_max", 30.0), ("hadtop_chi2_max", 20.0),
            ("hadtop_chi2_max", 10.0), ("met_min", 10.0), ("met_min", 20.0), ("met_min", 30.0),
            ("met_min", 40.0), ("njets_min", 4), ("wnu_solvable",)]
    an = analyses.semilep(sigma_jet=0.1, sigma_met=10.0, cuts=cuts)
    aid = eng.define(an)
    for k in range(3):
        cols = synth.gen_semilep(1500, 110 + k)
        g = eng.run_device(aid, DeviceColumns(cols), V=8, seed=6, first_event_id=k * 10000).numpy()
        o = orc.run(an, cols, seed=6, V=8, first_event_id=k * 10000)
        assert_parity(g, o, what="chunk %d" % k)
    st = eng.sched_state(aid)
    order = st["order"].tolist()
    assert sorted(order) == list(range(len(cuts)))
    stage2 = [c for c in order if cuts[c][0] in ("hadtop_chi2_max", "met_min")]
    assert stage2 == list(range(8)), order
    assert (st["evaluated"][:8] > 0).all() and (st["cost"][:8] > 0).all()


def test_async_submit_poll_fetch(eng, orc):
    """Host columns through hf_submit_chunk / hf_poll / hf_fetch_results with
    several chunks in flight (pinned and pageable host memory)."""
    from paper_2211_14346_gb300 import PinnedColumns, HostColumnsView, HF_STATE_DONE
    an = analyses.config2()
    aid = eng.define(an)
    chunks = [synth.gen_semilep(n, 40 + i) for i, n in enumerate((900, 1, 2500, 1300))]
    tickets = []
    for i, c in enumerate(chunks):
        h = PinnedColumns(c) if i % 2 == 0 else HostColumnsView(c)
        tickets.append((eng.submit(aid, h, V=16, seed=21, first_event_id=1000 * i), h, c, i))
    for t, h, c, i in tickets:
        g = eng.fetch(aid, t, c.n_events)
        assert eng.poll  # ticket released after fetch
        o = orc.run(an, c, seed=21, V=16, first_event_id=1000 * i)
        assert_parity(g, o, what="ticket %d" % i)
    with pytest.raises(Exception):
        eng.poll(tickets[0][0])
    assert HF_STATE_DONE == 2


def test_pinned_staging_ring_for_pageable_columns(orc):
    """A context with a 1 MB pinned staging ring: pageable host columns are
    copied into the ring during hf_submit_chunk, so the caller's buffers may
    be overwritten as soon as the call returns; six chunks cycle through the
    ring (it wraps and waits for earlier copies), a pinned chunk and one
    larger than the ring are copied straight from the caller's memory."""
    from paper_2211_14346_gb300 import Engine, PinnedColumns, HostColumnsView
    an = analyses.config2()
    with Engine(0, staging_bytes=1 << 20) as e:
        aid = e.define(an)
        sizes = (1500, 700, 2600, 1, 1900, 1200, 1000, 12000)
        chunks = [synth.gen_semilep(n, 60 + i) for i, n in enumerate(sizes)]
        tickets = []
        for i, c in enumerate(chunks):
            h = PinnedColumns(c) if i == 6 else HostColumnsView(copy.deepcopy(c))
            t = e.submit(aid, h, V=16, seed=25, first_event_id=5000 * i)
            if i not in (6, 7):  # staged: the caller's buffers are free again
                for a in h._keep:
                    a.view(np.uint8)[...] = 0xA5
            tickets.append((t, h, c, i))
        for t, h, c, i in tickets:
            g = e.fetch(aid, t, c.n_events)
            o = orc.run(an, c, seed=25, V=16, first_event_id=5000 * i)
            assert_parity(g, o, what="staged chunk %d" % i)


def test_fetch_timeout_keeps_the_ticket(eng):
    """hf_fetch_results with timeout_ms = 0 on a ticket still running returns
    HF_ETIMEOUT and keeps the ticket; a later fetch with a long timeout gets
    the results, equal to the device-resident run of the same chunk."""
    from paper_2211_14346_gb300 import PinnedColumns, DeviceColumns, HFError, _lib
    an = analyses.config2()
    aid = eng.define(an)
    cols = synth.gen_semilep(1_000_000, 44)
    h = PinnedColumns(cols)
    t = eng.submit(aid, h, V=64, seed=23)
    with pytest.raises(HFError) as ei:
        eng.fetch(aid, t, cols.n_events, timeout_ms=0)
    assert ei.value.status == _lib.HF_ETIMEOUT
    assert eng.poll(t) in (0, 1, 2)  # the ticket is still known
    g = eng.fetch(aid, t, cols.n_events, timeout_ms=600000)
    ref = eng.run_device(aid, DeviceColumns(cols), V=64, seed=23).numpy()
    assert np.array_equal(g["cutflow"], ref["cutflow"])
    assert np.array_equal(g["mask"], ref["mask"])
    with pytest.raises(HFError):
        eng.poll(t)  # released by the successful fetch


def test_two_contexts_in_one_process(orc):
    """Two contexts open at once on device 0 (per-device kernel attributes and
    scratch are per context): each runs the same chunk, interleaved, and both
    equal the oracle."""
    from paper_2211_14346_gb300 import Engine, DeviceColumns
    an = analyses.config2()
    cols = synth.gen_semilep(3000, 46)
    o = orc.run(an, cols, seed=8, V=16)
    with Engine(0) as a, Engine(0) as b:
        ia, ib = a.define(an), b.define(an)
        dc = DeviceColumns(cols)
        for _ in range(2):
            ga = a.run_device(ia, dc, V=16, seed=8).numpy()
            gb = b.run_device(ib, dc, V=16, seed=8).numpy()
            assert_parity(ga, o, what="context a")
            assert_parity(gb, o, what="context b")


def test_malformed_columns_are_rejected(eng):
    from paper_2211_14346_gb300 import DeviceColumns, HostColumnsView, HFError
    from paper_2211_14346_gb300 import _lib
    cols = synth.gen_semilep(200, 6)
    bad = cols.slice(0, 200)
    # event 10 claims 13 jets: offsets stay monotone and inside the jet array
    off = bad.jet_off.astype(np.int64)
    off[11:] = off[11:] + 0  # keep
    n = np.diff(off)
    k = 10
    extra = 13 - n[k]
    new_off = off.copy()
    new_off[k + 1:] += extra
    jets = np.concatenate([bad.jets[:off[k + 1]], np.tile(bad.jets[:1], (extra, 1)), bad.jets[off[k + 1]:]])
    bad.jet_off = new_off.astype(np.uint32)
    bad.jets = np.ascontiguousarray(jets)
    an = analyses.config2()
    aid = eng.define(an)
    eng.run_device(aid, DeviceColumns(bad), V=2, seed=1)
    assert eng.device_error() & 1
    t = eng.submit(aid, HostColumnsView(bad), V=2, seed=1)
    with pytest.raises(HFError) as ei:
        eng.fetch(aid, t, bad.n_events)
    assert ei.value.status == _lib.HF_EINVAL
    # and a good run afterwards clears the error word
    eng.run_device(aid, DeviceColumns(cols), V=2, seed=1)
    assert eng.device_error() == 0


def test_invalid_descriptors(eng):
    from paper_2211_14346_gb300 import HFError
    an = analyses.config2()
    with pytest.raises(HFError):
        eng.define(analyses.with_cuts(an, [("njets_min", 4)]))  # no reconstruction cuts
    bad = dict(an)
    bad["sigma_jet"] = 0.5
    with pytest.raises(HFError):
        eng.define(bad)
    bad = dict(an)
    bad["hist"] = (0, 0.0, 500.0)
    with pytest.raises(HFError):
        eng.define(bad)
