"""Batched runs (hf_run_batch): many chunks of uneven size, both event models
and different variation counts through one launch sequence.  Every chunk's
results must equal the FP64 oracle's (bit-exact mask, n_surv, cut flow,
histogram; reco within 1e-5) and those of hf_run_device on the same chunk,
also when the captured launch sequence is replayed for a new batch."""
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


def _mixed_chunks(seed0):
    """(analysis name, columns, V, seed, first_event_id) for a mixed batch:
    ragged sizes (0, 1, a few hundred, a few thousand), both models."""
    spec = [("semi", 1500, 16), ("dilep", 150, 8), ("semi", 0, 4), ("semi", 1, 16), ("semi0", 2500, 1),
            ("dilep", 60, 1), ("semi", 700, 64), ("semi", 333, 3), ("dilep", 1, 64), ("semi", 4000, 8)]
    out = []
    for k, (model, n, V) in enumerate(spec):
        if model == "dilep":
            cols = synth.gen_dilep(n, seed0 + k)
        else:
            cols = synth.gen_semilep(n, seed0 + k)
        out.append((model, cols, V, 500 + k, 1000003 * k + seed0))
    return out


def _analyses(eng):
    ans = {"semi": analyses.config2(), "semi0": analyses.config1(), "dilep": analyses.config3()}
    return ans, {k: eng.define(v) for k, v in ans.items()}


def _run_batch(eng, aids, chunks):
    from paper_2211_14346_gb300 import DeviceColumns
    items = [dict(aid=aids[m], cols=DeviceColumns(c), V=V, seed=s, first_event_id=f) for m, c, V, s, f in chunks]
    outs = eng.run_batch(items)
    res = [o.numpy() for o in outs]
    assert eng.device_error() == 0
    return res


def test_batch_matches_oracle_and_single_runs(eng, orc):
    from paper_2211_14346_gb300 import DeviceColumns
    ans, aids = _analyses(eng)
    chunks = _mixed_chunks(61)
    res = _run_batch(eng, aids, chunks)
    for k, ((m, cols, V, s, f), g) in enumerate(zip(chunks, res)):
        an = ans[m]
        if cols.n_events == 0:
            assert g["cutflow"].sum() == 0 and g["hist"].sum() == 0
            continue
        o = orc.run(an, cols, seed=s, V=V, first_event_id=f)
        assert_parity(g, o, model="dilep" if m == "dilep" else "semilep", what="batch chunk %d (%s V=%d)" % (k, m, V))
        single = eng.run_device(aids[m], DeviceColumns(cols), V=V, seed=s, first_event_id=f).numpy()
        for key in ("mask", "n_surv", "cutflow", "hist"):
            assert np.array_equal(single[key], g[key]), (k, key)


def test_batch_replay_with_new_tables(eng, orc):
    """The second and third batches reuse the captured launch sequence with
    new chunk tables; the repeat of a batch gives identical results."""
    ans, aids = _analyses(eng)
    a = _mixed_chunks(62)
    b = _mixed_chunks(63)
    ra1 = _run_batch(eng, aids, a)
    rb = _run_batch(eng, aids, b)
    ra2 = _run_batch(eng, aids, a)
    for x, y in zip(ra1, ra2):
        for key in ("mask", "n_surv", "cutflow", "hist"):
            assert np.array_equal(x[key], y[key])
    for k, ((m, cols, V, s, f), g) in enumerate(zip(b, rb)):
        if cols.n_events == 0 or k % 3:
            continue
        o = orc.run(ans[m], cols, seed=s, V=V, first_event_id=f)
        assert_parity(g, o, model="dilep" if m == "dilep" else "semilep", what="replayed chunk %d" % k)


def test_batch_many_small_chunks(eng, orc):
    """Hundreds of tiny semileptonic chunks (1..40 events): the tile queue
    crosses chunk boundaries in every block; the sum over chunks equals one
    run over their concatenation."""
    from paper_2211_14346_gb300 import DeviceColumns
    ans, aids = _analyses(eng)
    rng = np.random.default_rng(7)
    sizes = rng.integers(1, 41, 300)
    cols = [synth.gen_semilep(int(n), 9000 + i) for i, n in enumerate(sizes)]
    first = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    items = [dict(aid=aids["semi"], cols=DeviceColumns(c), V=16, seed=77, first_event_id=int(f))
             for c, f in zip(cols, first)]
    res = [o.numpy() for o in eng.run_batch(items)]
    allc = synth.concat(cols)
    whole = eng.run_device(aids["semi"], DeviceColumns(allc), V=16, seed=77).numpy()
    assert np.array_equal(sum(r["cutflow"] for r in res), whole["cutflow"])
    assert np.array_equal(sum(r["hist"] for r in res), whole["hist"])
    assert np.array_equal(np.concatenate([r["mask"] for r in res]), whole["mask"])
    o = orc.run(ans["semi"], allc, seed=77, V=16)
    assert_parity(whole, o, what="concatenation")


def test_batch_rejects_bad_chunks(eng):
    from paper_2211_14346_gb300 import DeviceColumns, HFError
    _, aids = _analyses(eng)
    cols = DeviceColumns(synth.gen_semilep(10, 1))
    with pytest.raises(HFError):
        eng.run_batch([dict(aid=aids["semi"], cols=cols, V=0)])
    with pytest.raises(HFError):
        eng.run_batch([dict(aid=999, cols=cols, V=1, out=eng.results_for(aids["semi"], 10))])
    with pytest.raises(HFError):
        eng.run_batch([dict(aid=aids["semi"], cols=cols, V=5000)])
