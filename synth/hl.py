"""Seeded synthetic events for the HL-LHC multi-region top selection
(Sect. 6.1): one or two leptons of either flavour, jets over three
pseudorapidity regions, b-tags and MET.  This module only draws inputs; it
holds none of the selection arithmetic.

Column layout (N events, J jets, L leptons in total):

    jet_off  uint32[N+1]   CSR offsets into jets
    jets     float32[J,4]  (px, py, pz, E), sorted by pT descending per event
    btag     uint16[N]     bit i <=> jet i of the event is b-tagged
    lep_off  uint32[N+1]   CSR offsets into the lepton columns (0..3 per event)
    lep      float32[L,4]  (px, py, pz, E), massless
    lep_q    int8[L]       charge +-1
    lep_flav uint8[L]      0 electron, 1 muon
    met      float32[N,2]  MET (x, y)

The mix stands in for the HL-LHC samples of the paper (not available):
topologies close to each signal bin (ttbar 1 and 2 leptons, t-channel, Wt 1
and 2 leptons) and unstructured events, each perturbed (an extra jet, a jet
beside a lepton, a flipped b-tag, same-sign or same-flavour leptons, low
MET) so that every requirement of the selection both passes and fails.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .events import _p4


@dataclass
class HLColumns:
    jet_off: np.ndarray
    jets: np.ndarray
    btag: np.ndarray
    lep_off: np.ndarray
    lep: np.ndarray
    lep_q: np.ndarray
    lep_flav: np.ndarray
    met: np.ndarray

    @property
    def n_events(self) -> int:
        return int(self.jet_off.shape[0] - 1)


_P_KIND = np.array([0.24, 0.14, 0.14, 0.16, 0.12, 0.20])  # ttbar 1l, ttbar 2l, t-channel, Wt 1l, Wt 2l, other
_ETA_RANGE = np.array([[0.0, 2.5], [2.5, 2.75], [2.75, 3.5], [3.5, 4.5]])  # regions I, II, III, beyond


def gen_hllhc(n_events: int, seed: int, *, met_mean=55.0) -> HLColumns:
    """A mix of topologies near each signal bin and unstructured events
    (fractions _P_KIND), per kind (jets in region I, II, III; b-tags among the
    region-I jets; leptons): ttbar 1l (4..7, 0, 0; 2; 1), ttbar 2l (2..4, 0,
    0; 2; 2), t-channel (1, one jet in II or in III; 1; 1), Wt 1l (3, 0, 0;
    1; 1), Wt 2l (1..2, 0, 0; 1; 2), other (0..6, 0..1, 0..1; 0..2; 0..3).
    Perturbations: an extra jet in a random region including beyond 3.5
    (12 %), a flipped b-tag of a random jet (8 %), a jet within Delta R < 0.6
    of a random lepton (12 % of events with leptons), same-sign (10 %) and
    same-flavour (12 %) lepton pairs.  Jets: pT 25 + Exp(40), |eta| uniform
    in their region with a random sign, phi uniform, m = 5; leptons: pT
    20 + Exp(30), |eta| < 2.5, massless; MET Exp(met_mean), uniform angle.
    Vectorised over events."""
    r = np.random.Generator(np.random.PCG64(seed))
    N = int(n_events)
    kind = r.choice(6, size=N, p=_P_KIND)
    n1 = np.zeros(N, np.int64)
    n2 = np.zeros(N, np.int64)
    n3 = np.zeros(N, np.int64)
    nb = np.zeros(N, np.int64)
    nl = np.zeros(N, np.int64)
    k = kind == 0
    n1[k], nb[k], nl[k] = r.integers(4, 8, k.sum()), 2, 1
    k = kind == 1
    n1[k], nb[k], nl[k] = r.integers(2, 5, k.sum()), 2, 2
    k = kind == 2
    fwd = r.random(k.sum()) < 0.5
    n1[k], n2[k], n3[k], nb[k], nl[k] = 1, fwd, ~fwd, 1, 1
    k = kind == 3
    n1[k], nb[k], nl[k] = 3, 1, 1
    k = kind == 4
    n1[k], nb[k], nl[k] = r.integers(1, 3, k.sum()), 1, 2
    k = kind == 5
    m = int(k.sum())
    n1[k], n2[k], n3[k], nb[k], nl[k] = (r.integers(0, 7, m), r.integers(0, 2, m), r.integers(0, 2, m),
                                         r.integers(0, 3, m), r.integers(0, 4, m))
    extra = r.random(N) < 0.12
    near = (r.random(N) < 0.12) & (nl > 0)
    # jets in generation order: region I, II, III, the extra one, the one beside a lepton
    nj = n1 + n2 + n3 + extra + near
    J = int(nj.sum())
    ev = np.repeat(np.arange(N), nj)
    first = np.concatenate([[0], np.cumsum(nj)[:-1]])
    loc = np.arange(J) - first[ev]
    reg = np.full(J, -1, np.int64)
    reg[loc < n1[ev]] = 0
    reg[(loc >= n1[ev]) & (loc < (n1 + n2)[ev])] = 1
    reg[(loc >= (n1 + n2)[ev]) & (loc < (n1 + n2 + n3)[ev])] = 2
    is_extra = extra[ev] & (loc == (n1 + n2 + n3)[ev])
    reg[is_extra] = r.integers(0, 4, int(is_extra.sum()))
    is_near = near[ev] & (loc == nj[ev] - 1)
    lo, hi = _ETA_RANGE[np.maximum(reg, 0), 0], _ETA_RANGE[np.maximum(reg, 0), 1]
    eta = r.uniform(lo, hi) * np.where(r.random(J) < 0.5, 1.0, -1.0)
    phi = r.uniform(-np.pi, np.pi, J)
    pt = 25.0 + r.exponential(40.0, J)
    # b-tags: the first nb region-I jets in generation order, then an 8 % flip
    central = reg == 0
    cum = np.cumsum(central)
    base = np.concatenate([[0], cum])[first]
    crank = cum - 1 - base[ev]
    tag = central & (crank < nb[ev])
    flip = (r.random(N) < 0.08) & (nj - near > 0)
    fidx = (r.random(N) * np.maximum(nj - near, 1)).astype(np.int64)
    fj = first[flip] + fidx[flip]
    tag[fj] = ~tag[fj]
    # leptons
    L = int(nl.sum())
    lev = np.repeat(np.arange(N), nl)
    lfirst = np.concatenate([[0], np.cumsum(nl)[:-1]])
    lloc = np.arange(L) - lfirst[lev]
    l_eta = r.uniform(-2.5, 2.5, L)
    l_phi = r.uniform(-np.pi, np.pi, L)
    l_pt = 20.0 + r.exponential(30.0, L)
    q = np.where(r.random(L) < 0.5, 1, -1).astype(np.int8)
    fl = r.integers(0, 2, L).astype(np.uint8)
    two = nl == 2
    ss = r.random(N) < 0.1
    sf = r.random(N) < 0.12
    swap = r.random(N) < 0.5
    t2 = two[lev]
    q[t2] = np.where(lloc[t2] == 0, 1, np.where(ss[lev[t2]], 1, -1))
    f0 = np.where(sf, 1, np.where(swap, 1, 0))
    f1 = np.where(sf, 1, np.where(swap, 0, 1))
    fl[t2] = np.where(lloc[t2] == 0, f0[lev[t2]], f1[lev[t2]]).astype(np.uint8)
    # the jet beside a lepton: Delta R uniform in (0, 0.6) from a random lepton of the event
    ne = np.nonzero(near)[0]
    which = lfirst[ne] + (r.random(ne.size) * nl[ne]).astype(np.int64)
    dr = r.uniform(0.0, 0.6, ne.size)
    ang = r.uniform(0.0, 2.0 * np.pi, ne.size)
    jn = first[ne] + nj[ne] - 1
    eta[jn] = l_eta[which] + dr * np.cos(ang)
    phi[jn] = np.angle(np.exp(1j * (l_phi[which] + dr * np.sin(ang))))
    # sort the jets of each event by pT descending; b-tag bits in that order
    order = np.lexsort((-pt, ev))
    tag_sorted = tag[order]
    new_loc = np.arange(J) - first[ev]
    bits = np.zeros(N, np.uint32)
    np.bitwise_or.at(bits, ev[tag_sorted], (np.uint32(1) << new_loc[tag_sorted].astype(np.uint32)))
    jets = _p4(pt[order], eta[order], phi[order], np.full(J, 5.0))
    leps = _p4(l_pt, l_eta, l_phi, np.zeros(L))
    mag = r.exponential(met_mean, N)
    a = r.uniform(-np.pi, np.pi, N)
    met = np.stack([mag * np.cos(a), mag * np.sin(a)], axis=1).astype(np.float32)
    jet_off = np.zeros(N + 1, np.uint32)
    jet_off[1:] = np.cumsum(nj)
    lep_off = np.zeros(N + 1, np.uint32)
    lep_off[1:] = np.cumsum(nl)
    return HLColumns(jet_off=jet_off, jets=jets.reshape(-1, 4), btag=bits.astype(np.uint16), lep_off=lep_off,
                     lep=leps.reshape(-1, 4), lep_q=q, lep_flav=fl, met=met)
