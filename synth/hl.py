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


# (jets in region I, in II, in III, b-tags among the region-I jets, leptons)
_KINDS = [
    lambda r: (int(r.integers(4, 8)), 0, 0, 2, 1),   # ttbar, one lepton
    lambda r: (int(r.integers(2, 5)), 0, 0, 2, 2),   # ttbar, two leptons
    lambda r: (1, *((1, 0) if r.random() < 0.5 else (0, 1)), 1, 1),  # t-channel
    lambda r: (3, 0, 0, 1, 1),                       # Wt, one lepton
    lambda r: (int(r.integers(1, 3)), 0, 0, 1, 2),   # Wt, two leptons
    lambda r: (int(r.integers(0, 7)), int(r.integers(0, 2)), int(r.integers(0, 2)),
               int(r.integers(0, 3)), int(r.integers(0, 4))),  # unstructured
]
_P_KIND = [0.24, 0.14, 0.14, 0.16, 0.12, 0.20]


def _eta_in(r, region):
    lo, hi = {0: (0.0, 2.5), 1: (2.5, 2.75), 2: (2.75, 3.5), 3: (3.5, 4.5)}[region]
    return float(r.uniform(lo, hi)) * (1.0 if r.random() < 0.5 else -1.0)


def gen_hllhc(n_events: int, seed: int, *, met_mean=55.0) -> HLColumns:
    r = np.random.Generator(np.random.PCG64(seed))
    N = int(n_events)
    jet_off = [0]
    lep_off = [0]
    jets, leps, lq, lf, btag, met = [], [], [], [], [], []
    for _ in range(N):
        kind = int(r.choice(len(_KINDS), p=_P_KIND))
        n1, n2, n3, nb, nl = _KINDS[kind](r)
        regions = [0] * n1 + [1] * n2 + [2] * n3
        if r.random() < 0.12:
            regions.append(int(r.integers(0, 4)))  # an extra jet, possibly beyond 3.5
        eta = [_eta_in(r, g) for g in regions]
        phi = [float(r.uniform(-np.pi, np.pi)) for _ in regions]
        pt = [25.0 + float(r.exponential(40.0)) for _ in regions]
        central = [i for i, g in enumerate(regions) if g == 0]
        tagged = set(central[:nb]) if nb <= len(central) else set(central)
        if r.random() < 0.08 and regions:
            tagged ^= {int(r.integers(0, len(regions)))}  # a flipped or forward tag
        # leptons
        l_eta = [float(r.uniform(-2.5, 2.5)) for _ in range(nl)]
        l_phi = [float(r.uniform(-np.pi, np.pi)) for _ in range(nl)]
        l_pt = [20.0 + float(r.exponential(30.0)) for _ in range(nl)]
        if nl == 2:
            q = [1, -1] if r.random() > 0.1 else [1, 1]
            f = [0, 1] if r.random() > 0.12 else [1, 1]
            if r.random() < 0.5:
                f = f[::-1]
        else:
            q = [1 if r.random() < 0.5 else -1 for _ in range(nl)]
            f = [int(r.integers(0, 2)) for _ in range(nl)]
        if nl and r.random() < 0.12:
            # a jet beside a lepton: Delta R uniform in (0, 0.6)
            k = int(r.integers(0, nl))
            dr, ang = float(r.uniform(0.0, 0.6)), float(r.uniform(0, 2 * np.pi))
            eta.append(l_eta[k] + dr * np.cos(ang))
            phi.append(float(np.angle(np.exp(1j * (l_phi[k] + dr * np.sin(ang))))))
            pt.append(25.0 + float(r.exponential(40.0)))
            regions.append(-1)
        order = sorted(range(len(pt)), key=lambda i: -pt[i])
        bits = 0
        for new, old in enumerate(order):
            if old in tagged:
                bits |= 1 << new
        if order:
            jets.append(_p4(np.array([pt[i] for i in order]), np.array([eta[i] for i in order]),
                            np.array([phi[i] for i in order]), np.full(len(order), 5.0)))
        jet_off.append(jet_off[-1] + len(order))
        btag.append(bits)
        if nl:
            leps.append(_p4(np.array(l_pt), np.array(l_eta), np.array(l_phi), np.zeros(nl)))
            lq += q
            lf += f
        lep_off.append(lep_off[-1] + nl)
        mag = float(r.exponential(met_mean))
        a = float(r.uniform(-np.pi, np.pi))
        met.append((mag * np.cos(a), mag * np.sin(a)))
    z4 = np.zeros((0, 4), np.float32)
    return HLColumns(
        jet_off=np.asarray(jet_off, np.uint32),
        jets=np.concatenate(jets).astype(np.float32) if jets else z4,
        btag=np.asarray(btag, np.uint16),
        lep_off=np.asarray(lep_off, np.uint32),
        lep=np.concatenate(leps).astype(np.float32) if leps else z4,
        lep_q=np.asarray(lq, np.int8),
        lep_flav=np.asarray(lf, np.uint8),
        met=np.asarray(met, np.float32).reshape(N, 2),
    )
