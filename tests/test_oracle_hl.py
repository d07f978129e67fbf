"""Pins of the oracle's HL-LHC multi-region selection (Sect. 6.1) on events
built by hand from (pT, eta, phi): each signal bin, and each requirement
failing on its own, with the expected channel written out here; plus the
closed forms of eta, Delta R and M_T^W."""
import math

import numpy as np
import pytest

from synth.events import _p4
from synth.hl import HLColumns, gen_hllhc

FAR = 2.0  # lepton azimuth, away from every jet below


def _cols(events):
    jet_off, lep_off, jets, leps, q, fl, bt, met = [0], [0], [], [], [], [], [], []
    for ev in events:
        js = sorted(ev["jets"], key=lambda j: -j[0])
        bits = 0
        for i, j in enumerate(js):
            if len(j) > 3 and j[3]:
                bits |= 1 << i
        if js:
            jets.append(_p4(np.array([j[0] for j in js], float), np.array([j[1] for j in js], float),
                            np.array([j[2] for j in js], float), np.full(len(js), 5.0)))
        jet_off.append(jet_off[-1] + len(js))
        bt.append(bits)
        ls = ev.get("leps", [])
        if ls:
            leps.append(_p4(np.array([l[0] for l in ls], float), np.array([l[1] for l in ls], float),
                            np.array([l[2] for l in ls], float), np.zeros(len(ls))))
        q += [l[3] for l in ls]
        fl += [l[4] for l in ls]
        lep_off.append(lep_off[-1] + len(ls))
        mag, phi = ev.get("met", (50.0, -1.0))
        met.append((mag * math.cos(phi), mag * math.sin(phi)))
    z = np.zeros((0, 4), np.float32)
    return HLColumns(np.asarray(jet_off, np.uint32), np.concatenate(jets).astype(np.float32) if jets else z,
                     np.asarray(bt, np.uint16), np.asarray(lep_off, np.uint32),
                     np.concatenate(leps).astype(np.float32) if leps else z, np.asarray(q, np.int8),
                     np.asarray(fl, np.uint8), np.asarray(met, np.float32).reshape(-1, 2))


CENTRAL4 = [(80.0, 0.1, -1.0, 1), (60.0, -0.5, -2.2, 1), (50.0, 1.0, -0.4, 0), (40.0, 2.0, -2.8, 0)]
E1 = (45.0, 0.3, FAR, 1, 0)
MU1 = (35.0, -0.8, FAR + 0.9, -1, 1)

CASES = [
    ("ttbar 1l", dict(jets=CENTRAL4, leps=[E1]), 1),
    ("ttbar 1l, MET 25", dict(jets=CENTRAL4, leps=[E1], met=(25.0, -1.0)), 0),
    ("ttbar 1l + region II jet", dict(jets=CENTRAL4 + [(30.0, 2.6, 0.5, 0)], leps=[E1]), 0),
    ("ttbar 1l + jet beyond 3.5", dict(jets=CENTRAL4 + [(30.0, 3.8, 0.5, 0)], leps=[E1]), 1),
    ("ttbar 1l, lepton beside a jet", dict(jets=CENTRAL4 + [(30.0, 0.5, FAR + 0.1, 0)], leps=[E1]), 0),
    ("ttbar 1l, 3 b", dict(jets=CENTRAL4[:2] + [(50.0, 1.0, -0.4, 1), CENTRAL4[3]], leps=[E1]), 0),
    ("ttbar 2l", dict(jets=CENTRAL4[:2], leps=[E1, MU1]), 2),
    ("ttbar 2l same sign", dict(jets=CENTRAL4[:2], leps=[E1, (35.0, -0.8, FAR + 0.9, 1, 1)]), 0),
    ("ttbar 2l same flavour", dict(jets=CENTRAL4[:2], leps=[E1, (35.0, -0.8, FAR + 0.9, -1, 0)]), 0),
    ("ttbar 2l, M_ll < 40", dict(jets=CENTRAL4[:2], leps=[(20.0, 0.3, FAR, 1, 0), (15.0, 0.5, FAR + 0.2, -1, 1)]), 0),
    ("ttbar 2l + region III jet", dict(jets=CENTRAL4[:2] + [(30.0, -3.0, 0.5, 0)], leps=[E1, MU1]), 0),
    ("t-channel, region III", dict(jets=[(70.0, 0.4, -1.0, 1), (40.0, -3.1, 0.3, 0)], leps=[E1]), 3),
    ("t-channel, region II", dict(jets=[(70.0, 0.4, -1.0, 1), (40.0, 2.6, 0.3, 0)], leps=[E1]), 3),
    ("t-channel, untagged", dict(jets=[(70.0, 0.4, -1.0, 0), (40.0, -3.1, 0.3, 0)], leps=[E1]), 0),
    ("t-channel, 2 central", dict(jets=[(70.0, 0.4, -1.0, 1), (50.0, -1.4, -2.0, 0), (40.0, -3.1, 0.3, 0)],
                                  leps=[E1]), 0),
    ("Wt 1l, back to back", dict(jets=CENTRAL4[1:], leps=[(40.0, 0.3, FAR, 1, 1)], met=(50.0, FAR - math.pi)), 4),
    ("Wt 1l, MET along the lepton", dict(jets=CENTRAL4[1:], leps=[(40.0, 0.3, FAR, 1, 1)], met=(50.0, FAR)), 0),
    ("Wt 2l, 1 jet", dict(jets=[CENTRAL4[0]], leps=[E1, MU1]), 5),
    ("Wt 2l, 2 jets", dict(jets=[CENTRAL4[0], CENTRAL4[2]], leps=[E1, MU1]), 5),
    ("Wt 2l, 3 jets", dict(jets=[CENTRAL4[0], CENTRAL4[2], CENTRAL4[3]], leps=[E1, MU1]), 0),
    ("no lepton", dict(jets=CENTRAL4), 0),
    ("three leptons", dict(jets=CENTRAL4, leps=[E1, MU1, (30.0, -2.0, FAR - 0.8, 1, 1)]), 0),
]


@pytest.mark.parametrize("name,ev,want", CASES, ids=[c[0] for c in CASES])
def test_hand_built_events(orc, name, ev, want):
    r = orc.hl.classify(_cols([ev]))
    assert int(r["channel"][0, 0]) == want, name
    assert int(r["counts"].sum()) == 1 and int(r["counts"][want]) == 1
    if want:
        assert int(r["hist"][want - 1].sum()) == 1


def test_transverse_mass_closed_form(orc):
    """The back-to-back and parallel Wt cases by the textbook form
    M_T = sqrt(2 pT |MET| (1 - cos dphi)): 89.4 and 0 GeV around the 50 GeV cut."""
    assert math.sqrt(2 * 40.0 * 50.0 * (1 - math.cos(math.pi))) > 50.0
    assert math.sqrt(2 * 40.0 * 50.0 * (1 - math.cos(0.0))) < 50.0


def test_eta_is_minus_log_tan_half_theta(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        p = rng.normal(0, 50, 3)
        theta = math.atan2(math.hypot(p[0], p[1]), p[2])
        eta, phi = orc.hl.eta_phi([p[0], p[1], p[2], 0.0])
        assert abs(eta - (-math.log(math.tan(theta / 2)))) < 1e-9 * max(1.0, abs(eta))
        assert abs(phi - math.atan2(p[1], p[0])) < 1e-15


def test_delta_r_wraps_phi(orc):
    assert abs(orc.hl.delta_r((0.0, math.pi - 0.1), (0.0, -math.pi + 0.1)) - 0.2) < 1e-12
    assert abs(orc.hl.delta_r((1.0, 0.0), (-1.0, 0.0)) - 2.0) < 1e-15


def test_generated_mix_fills_every_channel_and_smearing_only_moves_met(orc):
    cols = gen_hllhc(3000, 7)
    r0 = orc.hl.classify(cols, V=3)
    assert (r0["channel"] == r0["channel"][:, :1]).all()  # no smearing: variations agree
    assert (r0["counts"][1:] > 50).all()
    r = orc.hl.classify(cols, seed=11, V=3, sigma_met=10.0)
    assert int(r["counts"].sum()) == 3 * cols.n_events
    assert np.array_equal(r["hist"].sum(axis=1), r["counts"][1:])
    # MET smearing moves units across the MET and M_T cuts only: a unit that
    # changes goes between a signal bin and none, never between two bins
    moved = r["channel"] != r0["channel"]
    assert moved.any()
    assert ((r["channel"][moved] == 0) | (r0["channel"][moved] == 0)).all()
