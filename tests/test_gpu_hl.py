"""Parity of the HL-LHC multi-region selection (Sect. 6.1) on the GPU with the
FP64 oracle (oracle.hl): bit-exact channel of every unit, per-channel counts
and histograms; hand-built events of every bin and failing requirement,
generated mixes with and without MET smearing, events placed at the decision
boundaries (eta regions, Delta R isolation, MET, M_ll, M_T^W), malformed
columns, and the full-size bench workload on sampled events."""
import math

import numpy as np
import pytest

from synth.hl import HLColumns, gen_hllhc
from tests.test_oracle_hl import CASES, _cols

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


def _gpu(eng, cols, *, V=1, seed=0, sigma_met=0.0, first=0, **kw):
    from paper_2211_14346_gb300 import HLDeviceColumns, hl_desc
    d = hl_desc(sigma_met=sigma_met, **kw)
    out = eng.run_hl(HLDeviceColumns(cols), d, V=V, seed=seed, first_event_id=first)
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r["counts"] = r["counts"].astype(np.uint64)
    r["hist"] = r["hist"].astype(np.uint64)
    return r


def _same(g, o, what):
    bad = np.argwhere(g["channel"] != o["channel"])
    assert bad.size == 0, "%s: channel differs at (event, v) %s: gpu %s oracle %s" % (
        what, bad[:5].tolist(), g["channel"][tuple(bad[:5].T)], o["channel"][tuple(bad[:5].T)])
    assert np.array_equal(g["counts"], o["counts"]), (what, g["counts"], o["counts"])
    assert np.array_equal(g["hist"], o["hist"]), what


def test_hand_built_events(eng, orc):
    cols = _cols([ev for _, ev, _ in CASES])
    g = _gpu(eng, cols)
    o = orc.hl.classify(cols)
    _same(g, o, "hand-built")
    assert g["channel"][:, 0].tolist() == [want for _, _, want in CASES]
    assert eng.device_error() == 0


def test_generated_mix_unsmeared(eng, orc):
    cols = gen_hllhc(20000, 21)
    g = _gpu(eng, cols, V=2)
    o = orc.hl.classify(cols, V=2)
    _same(g, o, "mix unsmeared")
    assert (o["counts"][1:] > 100).all()


def test_generated_mix_smeared(eng, orc):
    cols = gen_hllhc(3000, 22)
    g = _gpu(eng, cols, V=16, seed=31, sigma_met=10.0, first=(1 << 33) + 7)
    o = orc.hl.classify(cols, V=16, seed=31, sigma_met=10.0, first_event_id=(1 << 33) + 7)
    _same(g, o, "mix smeared")


def test_other_thresholds_and_histogram(eng, orc):
    cols = gen_hllhc(5000, 23)
    kw = dict(met_min=45.0, mll_min=60.0, mtw_min=35.0, dr_iso=0.5)
    g = _gpu(eng, cols, V=3, seed=5, sigma_met=4.0, hist=(37, 15.0, 180.0), **kw)
    o = orc.hl.classify(cols, V=3, seed=5, sigma_met=4.0, hist=(37, 15.0, 180.0), **kw)
    _same(g, o, "other thresholds")


def _near_boundary_events(rng, n):
    """Events whose decisions sit at the thresholds: jets at |eta| within
    1e-6 of 2.5, 2.75 and 3.5, a jet at Delta R within 1e-6 of 0.4 from a
    lepton, MET within 1e-5 of 30 GeV, lepton pairs with M_ll near 40 GeV,
    single leptons with M_T^W near 50 GeV."""
    from synth.events import _p4
    jet_off, lep_off, jets, leps, q, fl, bt, met = [0], [0], [], [], [], [], [], []
    for _ in range(n):
        js = []
        for b in (2.5, 2.75, 3.5):
            if rng.random() < 0.5:
                js.append((30.0 + 50 * rng.random(), (b + rng.uniform(-1e-6, 1e-6)) * rng.choice([-1, 1]),
                           rng.uniform(-math.pi, math.pi)))
        for _ in range(int(rng.integers(1, 5))):
            js.append((30.0 + 60 * rng.random(), rng.uniform(-2.4, 2.4), rng.uniform(-math.pi, math.pi)))
        nl = int(rng.integers(1, 3))
        ls = []
        for k in range(nl):
            ls.append((25.0 + 30 * rng.random(), rng.uniform(-2.0, 2.0), rng.uniform(-math.pi, math.pi)))
        if rng.random() < 0.5:
            l = ls[0]
            a = rng.uniform(0, 2 * math.pi)
            dr = 0.4 + rng.uniform(-1e-6, 1e-6)
            js.append((35.0, l[1] + dr * math.cos(a), math.remainder(l[2] + dr * math.sin(a), 2 * math.pi)))
        if nl == 2 and rng.random() < 0.5:
            # M_ll ~ 40: second lepton's pT from the massless two-body mass
            l1, l2 = ls
            c = math.cosh(l1[1] - l2[1]) - math.cos(l1[2] - l2[2])
            pt2 = (40.0 + rng.uniform(-1e-4, 1e-4)) ** 2 / (2.0 * l1[0] * c)
            ls[1] = (pt2, l2[1], l2[2])
        order = sorted(range(len(js)), key=lambda i: -js[i][0])
        js = [js[i] for i in order]
        bits = int(rng.integers(0, 1 << len(js)))
        jets.append(_p4(np.array([j[0] for j in js]), np.array([j[1] for j in js]), np.array([j[2] for j in js]),
                        np.full(len(js), 5.0)))
        leps.append(_p4(np.array([l[0] for l in ls]), np.array([l[1] for l in ls]), np.array([l[2] for l in ls]),
                        np.zeros(nl)))
        q += [1, -1][:nl] if rng.random() < 0.9 else [1, 1][:nl]
        fl += [0, 1][:nl] if rng.random() < 0.9 else [1, 1][:nl]
        jet_off.append(jet_off[-1] + len(js))
        lep_off.append(lep_off[-1] + nl)
        bt.append(bits)
        if nl == 1 and rng.random() < 0.5:
            # M_T^W ~ 50 with |MET| = 40: cos dphi from the transverse mass
            l = ls[0]
            m = 40.0
            cosd = 1.0 - (50.0 + rng.uniform(-1e-4, 1e-4)) ** 2 / (2.0 * l[0] * m)
            phi = l[2] + math.acos(max(-1.0, min(1.0, cosd)))
        else:
            m = 30.0 + rng.uniform(-1e-5, 1e-5)
            phi = rng.uniform(-math.pi, math.pi)
        met.append((m * math.cos(phi), m * math.sin(phi)))
    return HLColumns(np.asarray(jet_off, np.uint32), np.concatenate(jets).astype(np.float32),
                     np.asarray(bt, np.uint16), np.asarray(lep_off, np.uint32),
                     np.concatenate(leps).astype(np.float32), np.asarray(q, np.int8), np.asarray(fl, np.uint8),
                     np.asarray(met, np.float32))


def test_decision_boundaries(eng, orc):
    rng = np.random.default_rng(24)
    cols = _near_boundary_events(rng, 4000)
    g = _gpu(eng, cols, V=2)
    o = orc.hl.classify(cols, V=2)
    _same(g, o, "boundaries")
    gs = _gpu(eng, cols, V=4, seed=3, sigma_met=1e-4)
    os_ = orc.hl.classify(cols, V=4, seed=3, sigma_met=1e-4)
    _same(gs, os_, "boundaries, tiny MET smearing")


def test_malformed_and_empty(eng, orc):
    cols = gen_hllhc(600, 25)
    g0 = _gpu(eng, cols)
    assert eng.device_error() == 0
    bad = HLColumns(**{k: getattr(cols, k).copy() for k in cols.__dataclass_fields__})
    bad.jet_off[101] = bad.jet_off[100] + 17      # event 100: 17 jets; event 101: negative count
    bad.lep_off[300] = bad.lep_off[299] + 20      # event 299: 20 leptons; event 300: negative count
    g = _gpu(eng, bad)
    assert eng.device_error() & 1
    assert int(g["counts"].sum()) == cols.n_events - 4
    good = np.ones(cols.n_events, bool)
    good[[100, 101, 299, 300]] = False
    assert np.array_equal(g["channel"][good], g0["channel"][good])
    assert (g["channel"][~good] == 0).all()
    empty = HLColumns(np.zeros(1, np.uint32), np.zeros((0, 4), np.float32), np.zeros(0, np.uint16),
                      np.zeros(1, np.uint32), np.zeros((0, 4), np.float32), np.zeros(0, np.int8),
                      np.zeros(0, np.uint8), np.zeros((0, 2), np.float32))
    from paper_2211_14346_gb300 import HLDeviceColumns
    out = eng.run_hl(HLDeviceColumns(empty), V=3)
    assert int(out["counts"].sum().item()) == 0


def test_full_size_sampled(eng, orc):
    """The bench workload's size: 10,000,000 events x 4 variations of MET
    smearing; whole-chunk invariants and the oracle on sampled events."""
    N, V = 10_000_000, 4
    cols = gen_hllhc(N, 26)
    g = _gpu(eng, cols, V=V, seed=9, sigma_met=10.0)
    assert eng.device_error() == 0
    assert int(g["counts"].sum()) == N * V
    assert np.array_equal(g["hist"].sum(axis=1), g["counts"][1:])
    assert np.array_equal(np.bincount(g["channel"].reshape(-1).astype(np.int64), minlength=6), g["counts"])
    rng = np.random.default_rng(27)
    for lo in rng.integers(0, N - 500, 6):
        lo = int(lo)
        sub = HLColumns(jet_off=(cols.jet_off[lo:lo + 501] - cols.jet_off[lo]).astype(np.uint32),
                        jets=cols.jets[cols.jet_off[lo]:cols.jet_off[lo + 500]], btag=cols.btag[lo:lo + 500],
                        lep_off=(cols.lep_off[lo:lo + 501] - cols.lep_off[lo]).astype(np.uint32),
                        lep=cols.lep[cols.lep_off[lo]:cols.lep_off[lo + 500]],
                        lep_q=cols.lep_q[cols.lep_off[lo]:cols.lep_off[lo + 500]],
                        lep_flav=cols.lep_flav[cols.lep_off[lo]:cols.lep_off[lo + 500]], met=cols.met[lo:lo + 500])
        o = orc.hl.classify(sub, V=V, seed=9, sigma_met=10.0, first_event_id=lo)
        assert np.array_equal(g["channel"][lo:lo + 500], o["channel"]), lo
