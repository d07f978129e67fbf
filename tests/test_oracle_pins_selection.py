"""Pins of the oracle's selection steps that sit on top of the pinned
building blocks: the choice of the dilepton b-jet pairing across all ordered
pairings (Sect. 4: the two-neutrino solution of the ttH dilepton analysis),
the Higgs b-pair outside that pairing (Sect. 4) and the per-event mean over
the SURVIVING variations (the pseudo-experiments of Sect. 4).

Each is checked against an independent enumeration written here from the
definitions (numpy, FP64), on hand-built events chosen so that a plausible
mistake -- unordered pairings, untagged jets admitted, max instead of min,
ties not going to the first, the pairing jets not excluded from the Higgs
pair, division by V instead of by the survivors -- changes the answer."""
import itertools

import numpy as np

import synth
from synth import analyses
from synth.events import Columns, DILEP
from tests import kinematics as K

MW, MT, MH = 80.4, 172.5, 125.0


def _mass(v):
    m2 = v[3] * v[3] - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
    return np.sqrt(m2) if m2 >= 0 else -np.sqrt(-m2)


def _dilep_cols(events):
    """Columns of hand-built dilepton events: list of dict(l1, l2, jets
    (n x 4), btag bits, met (2,)); lepton 1 positive."""
    n = np.array([len(ev["jets"]) for ev in events], np.int64)
    off = np.zeros(len(events) + 1, np.uint32)
    off[1:] = np.cumsum(n)
    jets = np.concatenate([np.asarray(ev["jets"], np.float64) for ev in events]).astype(np.float32)
    lep = np.concatenate([np.stack([ev["l1"], ev["l2"]]) for ev in events]).astype(np.float32)
    q = np.tile(np.array([1, -1], np.int8), len(events))
    return Columns(DILEP, off, jets.reshape(-1, 4), np.array([ev["btag"] for ev in events], np.uint16),
                   lep.reshape(-1, 4), q, np.array([ev["met"] for ev in events], np.float32))


def _f64(cols, e):
    """Event e of the columns as the FP64 values the oracle sees."""
    lo, hi = int(cols.jet_off[e]), int(cols.jet_off[e + 1])
    jets = cols.jets.reshape(-1, 4)[lo:hi].astype(np.float64)
    lep = cols.lep.reshape(-1, 2, 4)[e].astype(np.float64)
    met = cols.met.reshape(-1, 2)[e].astype(np.float64)
    return jets, lep[0], lep[1], met, int(cols.btag[e]) & ((1 << (hi - lo)) - 1)


def _enumerate_pairings(orc, jets, l1, l2, met, allowed):
    """Best ordered pairing (b1 with lepton 1, b2 with lepton 2) over distinct
    jets of the `allowed` mask in index order, and each pairing's solutions
    in the order the solver returns them: minimum m_ttbar, ties to the first.
    Returns (b1, b2, m_t1, m_t2, m_tt) or None."""
    best = None
    n = len(jets)
    for b1, b2 in itertools.permutations(range(n), 2):   # (0,1), (0,2), ..., (1,0), ...: index order
        if not (allowed >> b1 & 1 and allowed >> b2 & 1):
            continue
        sols, _ = orc.dilep_pairing(l1, jets[b1], l2, jets[b2], met[0], met[1], np.float32(MW), np.float32(MT))
        for s in sols:
            t1 = jets[b1] + l1 + s["nu1"]
            t2 = jets[b2] + l2 + s["nu2"]
            mtt = _mass(t1 + t2)
            if best is None or mtt < best[4]:
                best = (b1, b2, _mass(t1), _mass(t2), mtt)
    return best


def _planted_dilep_event(rng, n_extra, p_tag_extra):
    l1, b1, n1, l2, b2, n2 = _planted_ttbar(rng)
    jets = [b1, b2]
    for _ in range(n_extra):
        p = rng.normal(0.0, 60.0, 3)
        jets.append(K.p4(p[0], p[1], p[2], 5.0))
    perm = rng.permutation(len(jets))
    jets = [jets[i] for i in perm]
    tags = 0
    for i, src in enumerate(perm):
        if src < 2 or rng.random() < p_tag_extra:
            tags |= 1 << i
    return dict(l1=l1, l2=l2, jets=np.array(jets), btag=tags, met=np.array([n1[0] + n2[0], n1[1] + n2[1]]))


def _planted_ttbar(rng):
    t = K.random_parent(MT, rng, pmax=250)
    tb = K.random_parent(MT, rng, pmax=250)
    b1, W1 = K.two_body(t, 5.0, MW, rng)
    l1, n1 = K.two_body(W1, 0.0, 0.0, rng)
    b2, W2 = K.two_body(tb, 5.0, MW, rng)
    l2, n2 = K.two_body(W2, 0.0, 0.0, rng)
    return l1, b1, n1, l2, b2, n2


def _unsmeared_dilep():
    return analyses.dilep(cuts=[("dilep_solvable",), ("higgs_window", 100.0, 150.0)])


def test_dilep_pairing_choice_enumerated(orc):
    """The unit's pairing is the minimum m_ttbar over ORDERED pairings of
    distinct b-TAGGED jets (independent enumeration over the pinned
    single-pairing solver).  The sample is built so that untagged jets,
    unordered pairings and the maximum would each pick differently on some
    events, and every such mistake is seen at least a few times."""
    rng = np.random.default_rng(101)
    events = [_planted_dilep_event(rng, int(rng.integers(2, 6)), 0.5) for _ in range(160)]
    cols = _dilep_cols(events)
    an = _unsmeared_dilep()
    seen_untagged = seen_order = seen_max = 0
    checked = 0
    for e in range(cols.n_events):
        jets, l1, l2, met, tags = _f64(cols, e)
        u = orc.unit(an, cols, e, 0)
        want = _enumerate_pairings(orc, jets, l1, l2, met, tags)
        if want is None:
            assert u["idx"][0] == -1 and u["idx"][1] == -1
            continue
        checked += 1
        assert (u["idx"][0], u["idx"][1]) == want[:2], (e, u["idx"], want)
        assert u["q"][3] == want[4] and u["q"][1] == want[2] and u["q"][2] == want[3]
        # the alternatives a mistake would produce
        alt = _enumerate_pairings(orc, jets, l1, l2, met, (1 << len(jets)) - 1)
        if alt is not None and alt[:2] != want[:2]:
            seen_untagged += 1
        if want[0] > want[1]:
            seen_order += 1          # an unordered loop (b1 < b2 only) cannot reach this pairing
        worst = None
        for b1, b2 in itertools.permutations(range(len(jets)), 2):
            if tags >> b1 & 1 and tags >> b2 & 1:
                sols, _ = orc.dilep_pairing(l1, jets[b1], l2, jets[b2], met[0], met[1], np.float32(MW),
                                            np.float32(MT))
                for s in sols:
                    m = _mass(jets[b1] + l1 + s["nu1"] + jets[b2] + l2 + s["nu2"])
                    if worst is None or m > worst[2]:
                        worst = (b1, b2, m)
        if worst is not None and worst[:2] != want[:2]:
            seen_max += 1
    assert checked >= 100
    assert seen_untagged >= 5 and seen_order >= 20 and seen_max >= 20


def test_dilep_pairing_tie_goes_to_the_first(orc):
    """Two identical b-tagged jets give two pairings with equal m_ttbar: the
    first in enumeration order wins."""
    rng = np.random.default_rng(102)
    done = 0
    for _ in range(40):
        l1, b1, n1, l2, b2, n2 = _planted_ttbar(rng)
        ev = dict(l1=l1, l2=l2, jets=np.array([b1, b2, b1.copy()]), btag=0b111,
                  met=np.array([n1[0] + n2[0], n1[1] + n2[1]]))
        cols = _dilep_cols([ev])
        u = orc.unit(_unsmeared_dilep(), cols, 0, 0)
        if u["idx"][0] < 0:
            continue
        # jets 0 and 2 are the same four-vector: the winner never uses jet 2 as b1
        # when jet 0 gives the same solutions earlier in the enumeration
        assert u["idx"][0] != 2
        if u["idx"][1] == 2:
            assert u["idx"][0] == 0   # (1, 2) equals the earlier (1, 0): only (0, 2) can end on jet 2
        done += 1
    assert done >= 30


def test_higgs_pair_excludes_the_pairing_jets(orc):
    """The Higgs pair is the minimum |m_bb - 125| over pairs i < j of b-tagged
    jets OUTSIDE the chosen pairing, ties to the first.  Events are built with
    five or six b-tagged jets, one extra jet made to form m = 125 GeV with a
    pairing jet, so the nearest pair over all b-jets uses a pairing jet and
    the oracle must take the next one."""
    rng = np.random.default_rng(103)
    an = _unsmeared_dilep()
    built = checked = 0
    for _ in range(400):
        ev = _planted_dilep_event(rng, int(rng.integers(2, 4)), 1.0)
        cols = _dilep_cols([ev])
        jets, l1, l2, met, tags = _f64(cols, 0)
        best = _enumerate_pairings(orc, jets, l1, l2, met, tags)
        if best is None:
            continue
        pb1 = best[0]
        # a jet h with m(pairing jet + h) = 125: back-to-back in the pairing jet's frame
        b = jets[pb1]
        dirn = rng.normal(size=3)
        dirn /= np.linalg.norm(dirn)
        # energy of a massless-ish jet h with (b + h)^2 = 125^2: m_b^2 + 2 (E_b E_h - p_b.p_h) = 125^2
        mb2 = b[3] ** 2 - b[:3] @ b[:3]
        eh = (MH ** 2 - mb2) / (2.0 * (b[3] - b[:3] @ dirn))
        h = np.concatenate([eh * dirn, [eh]])
        ev2 = dict(ev)
        ev2["jets"] = np.vstack([ev["jets"], h])
        ev2["btag"] = ev["btag"] | (1 << len(ev["jets"]))
        cols2 = _dilep_cols([ev2])
        jets2, l1, l2, met, tags2 = _f64(cols2, 0)
        best2 = _enumerate_pairings(orc, jets2, l1, l2, met, tags2)
        if best2 is None or best2[:2] != best[:2]:
            continue          # the new jet changed the pairing: not the case this test builds
        built += 1
        u = orc.unit(an, cols2, 0, 0)
        assert (u["idx"][0], u["idx"][1]) == best2[:2]
        rest = tags2 & ~(1 << best2[0]) & ~(1 << best2[1])
        want = None
        for i, j in itertools.combinations(range(len(jets2)), 2):
            if rest >> i & 1 and rest >> j & 1:
                m = _mass(jets2[i] + jets2[j])
                if want is None or abs(m - np.float32(MH)) < abs(want[2] - np.float32(MH)):
                    want = (i, j, m)
        everyone = min(((i, j) for i, j in itertools.combinations(range(len(jets2)), 2)
                        if tags2 >> i & 1 and tags2 >> j & 1),
                       key=lambda p: abs(_mass(jets2[p[0]] + jets2[p[1]]) - np.float32(MH)))
        assert pb1 in everyone or best2[1] in everyone     # the trap: the nearest pair uses a pairing jet
        if want is None:
            assert u["idx"][2] == -1
            continue
        checked += 1
        assert (u["idx"][2], u["idx"][3]) == want[:2]
        assert u["q"][0] == want[2]
        if built >= 40:
            break
    assert checked >= 25


def test_higgs_pair_tie_goes_to_the_first(orc):
    """Two non-pairing b-jet pairs with equal mass: the first (i < j in
    lexicographic order) is the Higgs candidate."""
    rng = np.random.default_rng(104)
    done = 0
    for _ in range(60):
        ev = _planted_dilep_event(rng, 0, 0.0)
        x = K.p4(30.0, -20.0, 15.0, 5.0)
        y = K.p4(-25.0, 40.0, -10.0, 5.0)
        ev["jets"] = np.vstack([ev["jets"], x, y, x.copy()])      # pairs (2,3) and (3,4) equal
        ev["btag"] = 0b11111
        cols = _dilep_cols([ev])
        jets, l1, l2, met, tags = _f64(cols, 0)
        best = _enumerate_pairings(orc, jets, l1, l2, met, tags)
        if best is None or best[0] > 1 or best[1] > 1:
            continue
        u = orc.unit(_unsmeared_dilep(), cols, 0, 0)
        # (2,3), (2,4), (3,4): m(2,3) = m(3,4); (2,4) is x + x, mass 2 m_x = 10, far from 125
        assert (u["idx"][2], u["idx"][3]) == (2, 3)
        done += 1
    assert done >= 10


def test_event_mean_divides_by_the_survivors(orc):
    """Per-event reco = mean over the variations that pass every cut (not
    over all V): events of a smeared V = 4 run with exactly 0, 1, 2 and 3
    surviving variations; the means recomputed by hand from the per-unit
    results, and the counts and histogram entries they imply."""
    cols = synth.gen_semilep(600, 105)
    an = analyses.config2()
    V, seed = 4, 17
    r = orc.run(an, cols, seed=seed, V=V)
    nc = len(an["cuts"])
    seen = {0: 0, 1: 0, 2: 0, 3: 0, 4: 0}
    hist = np.zeros_like(r["hist"])
    for e in range(cols.n_events):
        units = [orc.unit(an, cols, e, v, seed=seed) for v in range(V)]
        surv = [u for u in units if u["passed"] == nc]
        k = len(surv)
        seen[k] += 1
        assert r["n_surv"][e] == k and r["mask"][e] == (k > 0)
        for u in surv:
            hist[orc.hist_bin(u["q"][0], an["hist"][0], an["hist"][1], an["hist"][2])] += 1
        if k == 0:
            assert np.all(r["reco"][e] == 0.0)
            continue
        for q in range(4):
            s = 0.0
            for u in surv:          # in variation order, as the oracle sums
                s = s + u["q"][q]
            assert r["reco"][e, q] == s / k, (e, q)
    assert np.array_equal(hist, r["hist"])
    assert seen[1] >= 5 and seen[2] >= 5 and seen[3] >= 5
