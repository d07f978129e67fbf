"""FP64 CPU oracle of the HL-LHC multi-region top selection -- TEST
INFRASTRUCTURE (only the tests, the smoke check and the benchmark's CPU
baseline may use it).

Sect. 6.1 of the paper defines the signal regions.  Events are classified
per unit (event, variation); the variation smears only MET, with the
framework's Philox normals z12, z13 (the selection has no jet-pT threshold,
and a jet-energy scale changes neither eta nor the jet counts):

- isolated lepton: no jet within Delta R < 0.4 (Delta R^2 = Delta eta^2 +
  Delta phi^2, Delta phi wrapped to [-pi, pi]);
- transverse magnitudes (pT, |MET|) are sqrt(x^2 + y^2) in FP64;
- eta = asinh(pz / pT) (+-inf for pT = 0); regions by |eta| of the jets: I |eta| < 2.5,
  II 2.5 < |eta| < 2.75, III 2.75 < |eta| < 3.5 (boundaries and |eta| >= 3.5
  in none);
- b-jets: b-tagged jets of region I;
- every signal bin needs |MET| > 30 GeV;
- one isolated lepton: ttbar 1l (>= 4 jets in I, exactly 2 b, none in II or
  III), t-channel (exactly 1 jet in I and exactly 1 in II or III, exactly
  1 b), Wt 1l (exactly 3 jets in I, exactly 1 b, none in II or III,
  M_T^W > 50 GeV);
- two isolated leptons of opposite sign and different flavour: ttbar 2l
  (>= 2 jets in I, exactly 2 b, none in II or III, M_ll > 40 GeV), Wt 2l
  (1 or 2 jets in I, exactly 1 b, none in II or III);
- M_T^W^2 = 2 (pT_l |MET| - pvec_T,l . MET), M_ll the two leptons' mass.

Channel codes: 0 none, 1 ttbar 1l, 2 ttbar 2l, 3 t-channel, 4 Wt 1l,
5 Wt 2l.  Each channel has its own histogram (of the leading isolated
lepton's pT, underflow and overflow bins at the ends).
"""
from __future__ import annotations

import math

import numpy as np

from .oracle import hist_bin, unit_normals

CHANNELS = ("none", "ttbar_1l", "ttbar_2l", "t_channel", "wt_1l", "wt_2l")


def pt_of(x, y):
    """Transverse magnitude sqrt(x^2 + y^2) in FP64 (the formula of the rest
    of the oracle)."""
    x, y = float(x), float(y)
    return math.sqrt(x * x + y * y)


def eta_phi(p):
    """(eta, phi) of a (px, py, pz, E) vector in FP64: eta = asinh(pz / pT),
    +-inf along the beam (pT = 0, a jet in no region)."""
    px, py, pz = float(p[0]), float(p[1]), float(p[2])
    pt = pt_of(px, py)
    eta = math.asinh(pz / pt) if pt > 0.0 else math.copysign(math.inf, pz)
    return eta, math.atan2(py, px)


def delta_r(a, b):
    ea, pa = a
    eb, pb = b
    dphi = pa - pb
    while dphi > math.pi:
        dphi -= 2.0 * math.pi
    while dphi < -math.pi:
        dphi += 2.0 * math.pi
    return math.sqrt((ea - eb) ** 2 + dphi * dphi)


def region(eta):
    a = abs(eta)
    if a < 2.5:
        return 1
    if 2.5 < a < 2.75:
        return 2
    if 2.75 < a < 3.5:
        return 3
    return 0


def _mass(p):
    m2 = p[3] * p[3] - p[0] * p[0] - p[1] * p[1] - p[2] * p[2]
    return math.sqrt(m2) if m2 >= 0.0 else -math.sqrt(-m2)


def classify_event(jets, btag_bits, leps, lq, lflav, metx, mety, *, met_min=30.0, mll_min=40.0, mtw_min=50.0,
                   dr_iso=float(np.float32(0.4))):
    """Channel code of one unit and the leading isolated lepton's pT
    (thresholds as given; classify rounds them to FP32 first)."""
    jep = [eta_phi(j) for j in jets]
    iso = []
    for k, l in enumerate(leps):
        lep = eta_phi(l)
        if all(delta_r(lep, j) >= dr_iso for j in jep):
            iso.append(k)
    n = [0, 0, 0, 0]
    nb = 0
    for i, (eta, _) in enumerate(jep):
        g = region(eta)
        n[g] += 1
        if g == 1 and (btag_bits >> i) & 1:
            nb += 1
    n1, n2, n3 = n[1], n[2], n[3]
    met = pt_of(metx, mety)
    lead = max((pt_of(leps[k][0], leps[k][1]) for k in iso), default=0.0)
    if not met > met_min:
        return 0, lead
    if len(iso) == 1:
        l = leps[iso[0]]
        lx, ly = float(l[0]), float(l[1])
        if n1 >= 4 and nb == 2 and n2 == 0 and n3 == 0:
            return 1, lead
        if n1 == 1 and n2 + n3 == 1 and nb == 1:
            return 3, lead
        if n1 == 3 and nb == 1 and n2 == 0 and n3 == 0:
            mt2 = 2.0 * (pt_of(lx, ly) * met - (lx * metx + ly * mety))
            if math.sqrt(max(mt2, 0.0)) > mtw_min:
                return 4, lead
        return 0, lead
    if len(iso) == 2:
        a, b = iso
        if lq[a] * lq[b] < 0 and lflav[a] != lflav[b]:
            if n1 >= 2 and nb == 2 and n2 == 0 and n3 == 0:
                s = [float(leps[a][c]) + float(leps[b][c]) for c in range(4)]
                if _mass(s) > mll_min:
                    return 2, lead
            if n1 in (1, 2) and nb == 1 and n2 == 0 and n3 == 0:
                return 5, lead
    return 0, lead


def classify(cols, *, seed=0, V=1, sigma_met=0.0, first_event_id=0, hist=(50, 0.0, 500.0), **cuts):
    """All units of a chunk of synth.hl columns.  Returns dict: channel
    (i8[N, V]), counts (u64[6], units per channel code), hist
    (u64[5, nbins + 2], per signal channel)."""
    N = cols.n_events
    nbins, lo, hi = hist
    cuts = {k: float(np.float32(x)) for k, x in cuts.items()}  # the C ABI carries FP32 parameters
    ch = np.zeros((N, V), np.int8)
    counts = np.zeros(6, np.uint64)
    h = np.zeros((5, nbins + 2), np.uint64)
    s_met = float(np.float32(sigma_met))
    for e in range(N):
        jets = cols.jets[cols.jet_off[e]:cols.jet_off[e + 1]]
        l0, l1 = int(cols.lep_off[e]), int(cols.lep_off[e + 1])
        leps, lq, lf = cols.lep[l0:l1], cols.lep_q[l0:l1], cols.lep_flav[l0:l1]
        for v in range(V):
            mx, my = float(cols.met[e, 0]), float(cols.met[e, 1])
            if s_met > 0.0:
                z = unit_normals(seed, first_event_id + e, v)
                mx, my = mx + s_met * z[12], my + s_met * z[13]
            c, lead = classify_event(jets, int(cols.btag[e]), leps, lq, lf, mx, my, **cuts)
            ch[e, v] = c
            counts[c] += 1
            if c:
                h[c - 1, hist_bin(lead, nbins, float(np.float32(lo)), float(np.float32(hi)))] += 1
    return dict(channel=ch, counts=counts, hist=h)
