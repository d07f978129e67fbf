"""Serving with continuous batching (HF_FLAG_BATCHING): chunks submitted
through hf_submit_chunk are admitted by the HBM budget, queued, and launched
together by the context's dispatcher; chunks that arrive while batches run
join the next batch.  Every result must be the same alone and in the mix
(bit-exact mask, n_surv, cut flow, histogram; reco within 1e-5) and equal to
the FP64 oracle's."""
import time

import numpy as np
import pytest

import synth
from synth import analyses
from tests.parity import assert_parity, assert_reco

pytestmark = pytest.mark.gpu


def _requests(seed0, k=12):
    rng = np.random.default_rng(seed0)
    out = []
    for i in range(k):
        model = "dilep" if rng.random() < 0.3 else "semi"
        n = int(rng.integers(1, 3000))
        V = int(rng.integers(1, 65))
        cols = synth.gen_dilep(n, seed0 * 100 + i) if model == "dilep" else synth.gen_semilep(n, seed0 * 100 + i)
        out.append(dict(model=model, cols=cols, V=V, seed=1000 + i, first=10 ** 7 * i))
    return out


def _open(flags_extra=0, budget=0):
    import torch
    assert torch.cuda.is_available()
    from paper_2211_14346_gb300 import build, Engine, HF_FLAG_BATCHING
    build.build()
    eng = Engine(0, flags=HF_FLAG_BATCHING | flags_extra, hbm_budget_bytes=budget)
    aids = {"semi": eng.define(analyses.config2()), "dilep": eng.define(analyses.config3())}
    return eng, aids


def _submit(eng, aids, r):
    from paper_2211_14346_gb300 import PinnedColumns
    h = PinnedColumns(r["cols"])
    t = eng.submit(aids[r["model"]], h, V=r["V"], seed=r["seed"], first_event_id=r["first"])
    return t, h


def test_alone_equals_mix_and_oracle(orc):
    eng, aids = _open()
    reqs = _requests(5)
    alone = []
    for r in reqs:
        t, h = _submit(eng, aids, r)
        alone.append(eng.fetch(aids[r["model"]], t, r["cols"].n_events))
    b_alone = eng.profile()["batches"]
    assert b_alone == len(reqs)
    # the mix: all submitted back to back, fetched afterwards
    hs = [_submit(eng, aids, r) for r in reqs]
    mix = [eng.fetch(aids[r["model"]], t, r["cols"].n_events) for r, (t, h) in zip(reqs, hs)]
    p = eng.profile()
    assert p["batches"] - b_alone < len(reqs), "the mix was not batched"
    for i, (r, a, m) in enumerate(zip(reqs, alone, mix)):
        for key in ("mask", "n_surv", "cutflow", "hist"):
            assert np.array_equal(a[key], m[key]), (i, key)
        assert_reco(m["reco"], a["reco"], model="dilep" if r["model"] == "dilep" else "semilep",
                    what="alone vs mix %d" % i)
    for i in (0, 3, 7):
        r = reqs[i]
        an = analyses.config3() if r["model"] == "dilep" else analyses.config2()
        o = orc.run(an, r["cols"], seed=r["seed"], V=r["V"], first_event_id=r["first"])
        assert_parity(mix[i], o, model="dilep" if r["model"] == "dilep" else "semilep", what="served %d" % i)
    eng.close()


def test_arrivals_while_running_join_later_batches():
    """A large chunk keeps the GPU busy; chunks submitted meanwhile are queued
    (or already batched) and complete; poll states move forward only."""
    from paper_2211_14346_gb300 import HF_STATE_DONE, HF_STATE_QUEUED, HF_STATE_RUNNING
    eng, aids = _open()
    big = dict(model="semi", cols=synth.gen_semilep(400000, 8), V=64, seed=1, first=0)
    tb, hb = _submit(eng, aids, big)
    small = [dict(model="semi", cols=synth.gen_semilep(500, 30 + i), V=8, seed=2, first=10 ** 8 * (i + 1))
             for i in range(6)]
    ts = []
    for r in small:
        ts.append(_submit(eng, aids, r))
        time.sleep(0.002)
    states = [eng.poll(t) for t, _ in ts]
    assert all(s in (HF_STATE_QUEUED, HF_STATE_RUNNING, HF_STATE_DONE) for s in states)
    res = [eng.fetch(aids["semi"], t, r["cols"].n_events) for r, (t, _) in zip(small, ts)]
    eng.fetch(aids["semi"], tb, big["cols"].n_events, fields=("cutflow",))
    assert eng.profile()["batched_chunks"] == 7
    # same results as alone
    eng2, aids2 = _open()
    for r, g in zip(small, res):
        t, h = _submit(eng2, aids2, r)
        a = eng2.fetch(aids2["semi"], t, r["cols"].n_events)
        for key in ("mask", "n_surv", "cutflow", "hist"):
            assert np.array_equal(a[key], g[key])
    eng.close()
    eng2.close()


def test_admission_by_budget():
    """A budget that holds one chunk: the second submission is refused with
    HF_EBUSY until the first is fetched."""
    from paper_2211_14346_gb300 import HFError, _lib
    cols = synth.gen_semilep(20000, 4)
    eng, aids = _open(budget=int(cols.nbytes() * 1.6))
    r = dict(model="semi", cols=cols, V=4, seed=3, first=0)
    t1, h1 = _submit(eng, aids, r)
    with pytest.raises(HFError) as ei:
        _submit(eng, aids, r)
    assert ei.value.status == _lib.HF_EBUSY
    eng.fetch(aids["semi"], t1, cols.n_events)
    t2, h2 = _submit(eng, aids, r)
    eng.fetch(aids["semi"], t2, cols.n_events)
    eng.close()
