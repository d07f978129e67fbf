"""Seeded synthetic collision events in structure-of-arrays (SoA) columns.

This module only *draws inputs*: it holds none of the analysis arithmetic
(no cut, no mass, no reconstruction).  Both the FP64 oracle and the CUDA path
consume the columns it produces, so neither has to import the other.

The event shapes stand in for the paper's Delphes ttbar(H) samples (Sect. 4,
Sect. 6), which are not available: semileptonic ttbar-like events with one
lepton and 2..12 jets, and ttH-like dilepton events with two opposite-sign
leptons and 4..12 jets.

Column layout (one chunk of N events, J jets in total):

    jet_off  uint32[N+1]   CSR offsets, jet_off[0] = 0, jet_off[N] = J
    jets     float32[J,4]  (px, py, pz, E) per jet, GeV, jets of an event are
                           contiguous and sorted by pT descending
    btag     uint16[N]     bit i set <=> jet i of the event is b-tagged
    lep      float32[N*L,4] (px, py, pz, E) of the L leptons of each event
    lep_q    int8[N*L]     lepton charges (+1 / -1)
    met      float32[N,2]  missing transverse momentum (x, y), GeV

Four-momenta are built in FP64 from (pT, eta, phi, m) and rounded to FP32 per
component; E is the FP64 value sqrt(p^2 + m^2) rounded once.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEMILEP = 1
DILEP = 2


@dataclass
class Columns:
    """One chunk of events as SoA numpy arrays (see module docstring)."""

    model: int
    jet_off: np.ndarray
    jets: np.ndarray
    btag: np.ndarray
    lep: np.ndarray
    lep_q: np.ndarray
    met: np.ndarray

    @property
    def n_events(self) -> int:
        return int(self.jet_off.shape[0] - 1)

    @property
    def n_jets_total(self) -> int:
        return int(self.jet_off[-1])

    @property
    def n_lep(self) -> int:
        return 1 if self.model == SEMILEP else 2

    def nbytes(self) -> int:
        return int(sum(a.nbytes for a in (self.jet_off, self.jets, self.btag,
                                          self.lep, self.lep_q, self.met)))

    def slice(self, lo: int, hi: int) -> "Columns":
        """Events [lo, hi) as a new chunk with offsets rebased to 0."""
        j0, j1 = int(self.jet_off[lo]), int(self.jet_off[hi])
        L = self.n_lep
        return Columns(
            model=self.model,
            jet_off=(self.jet_off[lo:hi + 1] - np.uint32(j0)).astype(np.uint32),
            jets=np.ascontiguousarray(self.jets[j0:j1]),
            btag=np.ascontiguousarray(self.btag[lo:hi]),
            lep=np.ascontiguousarray(self.lep[lo * L:hi * L]),
            lep_q=np.ascontiguousarray(self.lep_q[lo * L:hi * L]),
            met=np.ascontiguousarray(self.met[lo:hi]),
        )


def _p4(pt, eta, phi, m):
    """FP64 (pT, eta, phi, m) -> FP32 (px, py, pz, E)."""
    px = pt * np.cos(phi)
    py = pt * np.sin(phi)
    pz = pt * np.sinh(eta)
    e = np.sqrt(px * px + py * py + pz * pz + m * m)
    out = np.empty((pt.shape[0], 4), dtype=np.float32)
    out[:, 0] = px
    out[:, 1] = py
    out[:, 2] = pz
    out[:, 3] = e
    return out


def _jets(rng, n, pt0, pt_mean, eta_max, mass, p_btag):
    """Jets for events with multiplicities n: sorted by pT desc, b-tag bits."""
    N = n.shape[0]
    J = int(n.sum())
    off = np.zeros(N + 1, dtype=np.uint64)
    np.cumsum(n, out=off[1:])
    ev = np.repeat(np.arange(N, dtype=np.int64), n)
    pt = pt0 + rng.exponential(pt_mean, J)
    eta = rng.uniform(-eta_max, eta_max, J)
    phi = rng.uniform(-np.pi, np.pi, J)
    order = np.lexsort((-pt, ev))          # by event, then pT descending
    pt, eta, phi = pt[order], eta[order], phi[order]
    jets = _p4(pt, eta, phi, np.full(J, float(mass)))
    tag = rng.random(J) < p_btag
    local = np.arange(J, dtype=np.int64) - off[:-1].astype(np.int64)[ev]
    bits = np.zeros(N, dtype=np.uint32)
    np.bitwise_or.at(bits, ev[tag], (np.uint32(1) << local[tag].astype(np.uint32)))
    return off.astype(np.uint32), jets, bits.astype(np.uint16)


def _leptons(rng, count, pt0, pt_mean, eta_max):
    pt = pt0 + rng.exponential(pt_mean, count)
    eta = rng.uniform(-eta_max, eta_max, count)
    phi = rng.uniform(-np.pi, np.pi, count)
    return _p4(pt, eta, phi, np.zeros(count))


def _met(rng, N, mean):
    mag = rng.exponential(mean, N)
    phi = rng.uniform(-np.pi, np.pi, N)
    out = np.empty((N, 2), dtype=np.float32)
    out[:, 0] = mag * np.cos(phi)
    out[:, 1] = mag * np.sin(phi)
    return out


def gen_semilep(n_events: int, seed: int, *, n_mean=6.0, n_min=2, n_max=12,
                jet_pt0=25.0, jet_pt_mean=40.0, eta_max=2.5, jet_mass=5.0,
                p_btag=0.25, lep_pt0=25.0, lep_pt_mean=30.0,
                met_mean=50.0) -> Columns:
    """Semileptonic ttbar-like events: n ~ Poisson(6) clipped to [2, 12],
    jet pT 25 + Exp(40), |eta| < 2.5 uniform, m = 5, b-tag Bernoulli(0.25),
    one massless lepton pT 25 + Exp(30), charge +-1, MET |.| ~ Exp(50)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = int(n_events)
    n = np.clip(rng.poisson(n_mean, N), n_min, n_max).astype(np.int64)
    jet_off, jets, btag = _jets(rng, n, jet_pt0, jet_pt_mean, eta_max,
                                jet_mass, p_btag)
    lep = _leptons(rng, N, lep_pt0, lep_pt_mean, eta_max)
    lep_q = np.where(rng.random(N) < 0.5, 1, -1).astype(np.int8)
    met = _met(rng, N, met_mean)
    return Columns(SEMILEP, jet_off, jets, btag, lep, lep_q, met)


def gen_dilep(n_events: int, seed: int, *, n_mean=7.0, n_min=4, n_max=12,
              jet_pt0=25.0, jet_pt_mean=40.0, eta_max=2.5, jet_mass=5.0,
              p_btag=0.35, lep_pt0=20.0, lep_pt_mean=30.0, met_mean=60.0,
              p_same_sign=0.0) -> Columns:
    """ttH-like dilepton events: two leptons pT 20 + Exp(30), opposite sign
    (the positive one first) unless drawn same-sign with p_same_sign,
    n ~ Poisson(7) clipped to [4, 12], b-tag Bernoulli(0.35), MET Exp(60)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = int(n_events)
    n = np.clip(rng.poisson(n_mean, N), n_min, n_max).astype(np.int64)
    jet_off, jets, btag = _jets(rng, n, jet_pt0, jet_pt_mean, eta_max,
                                jet_mass, p_btag)
    lep = _leptons(rng, 2 * N, lep_pt0, lep_pt_mean, eta_max)
    q = np.empty(2 * N, dtype=np.int8)
    q[0::2] = 1
    q[1::2] = -1
    if p_same_sign > 0:
        ss = rng.random(N) < p_same_sign
        q[1::2][ss] = 1
    met = _met(rng, N, met_mean)
    return Columns(DILEP, jet_off, jets, btag, lep, q, met)


def concat(chunks) -> Columns:
    """Concatenate chunks of one event model into one chunk."""
    model = chunks[0].model
    offs = [np.zeros(1, dtype=np.uint64)]
    base = 0
    for c in chunks:
        offs.append(c.jet_off[1:].astype(np.uint64) + base)
        base += int(c.jet_off[-1])
    return Columns(
        model=model,
        jet_off=np.concatenate(offs).astype(np.uint32),
        jets=np.concatenate([c.jets for c in chunks]),
        btag=np.concatenate([c.btag for c in chunks]),
        lep=np.concatenate([c.lep for c in chunks]),
        lep_q=np.concatenate([c.lep_q for c in chunks]),
        met=np.concatenate([c.met for c in chunks]),
    )
