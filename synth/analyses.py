"""User-level analysis descriptions (plain data, no arithmetic).

An analysis is a dict:

    model      "semilep" | "dilep"
    cuts       list of (name, *params) in USER order
    mW, mt, sigma_t, sigma_W, mH      physics constants (GeV)
    sigma_jet  relative jet-energy resolution of the smearing (0 = none)
    sigma_met  absolute MET resolution per component, GeV (0 = none)
    sigma_lep  relative lepton-energy resolution (0 = none; optional key)
    hist       (nbins, lo, hi) of the reconstructed-mass histogram

Both the C-ABI binding and the oracle binding marshal this dict into their
own layouts; every real parameter is rounded to FP32 first because the C-ABI
carries FP32 parameters.

Cut names: njets_min k | nbtag_min k | lep_pt_min x | met_min x |
wnu_solvable | hadtop_chi2_max x | lep_os | dilep_solvable |
higgs_window lo hi | ttbar_chi2_max x (the full Eq. 1 fit).
"""
from __future__ import annotations

import copy

CUT_NAMES = ("njets_min", "nbtag_min", "lep_pt_min", "met_min", "wnu_solvable",
             "hadtop_chi2_max", "lep_os", "dilep_solvable", "higgs_window", "ttbar_chi2_max")


def semilep(sigma_jet=0.0, sigma_met=0.0, sigma_t=15.0, sigma_W=10.0,
            cuts=None, sigma_lep=0.0):
    """Semileptonic chain C1..C6: >= 4 jets, >= 1 b-tag, lepton pT > 30,
    MET > 20, solvable W-mass neutrino p_z, best hadronic-top chi2 < 10;
    m_W = 80.4, m_t = 172.5, widths 15 / 10, m_top histogram 50 bins 0-500."""
    if cuts is None:
        cuts = [("njets_min", 4), ("nbtag_min", 1), ("lep_pt_min", 30.0),
                ("met_min", 20.0), ("wnu_solvable",), ("hadtop_chi2_max", 10.0)]
    return dict(model="semilep", cuts=list(cuts), mW=80.4, mt=172.5,
                sigma_t=sigma_t, sigma_W=sigma_W, mH=125.0,
                sigma_jet=sigma_jet, sigma_met=sigma_met, sigma_lep=sigma_lep, hist=(50, 0.0, 500.0))


def semilep_full(sigma_jet=0.0, sigma_met=0.0, sigma_t=11.5, sigma_W=7.5, cuts=None, sigma_lep=0.0):
    """Semileptonic chain with the full Eq. 1 fit (both tops, both W bosons,
    both neutrino solutions) in place of the hadronic-top cut: >= 4 jets,
    >= 1 b-tag, lepton pT > 30, MET > 20, solvable W-mass neutrino p_z,
    full chi2 < 20; the paper's widths 11.5 / 7.5; m_top (hadronic)
    histogram 50 bins 0-500."""
    if cuts is None:
        cuts = [("njets_min", 4), ("nbtag_min", 1), ("lep_pt_min", 30.0),
                ("met_min", 20.0), ("wnu_solvable",), ("ttbar_chi2_max", 20.0)]
    return dict(model="semilep", cuts=list(cuts), mW=80.4, mt=172.5,
                sigma_t=sigma_t, sigma_W=sigma_W, mH=125.0,
                sigma_jet=sigma_jet, sigma_met=sigma_met, sigma_lep=sigma_lep, hist=(50, 0.0, 500.0))


def dilep(sigma_jet=0.0, sigma_met=0.0, cuts=None, sigma_lep=0.0):
    """Dilepton ttH chain D1..D5: opposite-sign leptons, >= 4 jets,
    >= 4 b-tags, two-neutrino solution exists, 100 < m_bb < 150;
    m_bb histogram 50 bins 0-500."""
    if cuts is None:
        cuts = [("lep_os",), ("njets_min", 4), ("nbtag_min", 4),
                ("dilep_solvable",), ("higgs_window", 100.0, 150.0)]
    return dict(model="dilep", cuts=list(cuts), mW=80.4, mt=172.5,
                sigma_t=15.0, sigma_W=10.0, mH=125.0,
                sigma_jet=sigma_jet, sigma_met=sigma_met, sigma_lep=sigma_lep, hist=(50, 0.0, 500.0))


def config1():
    """Small plain configuration: semileptonic, no smearing."""
    return semilep()


def config2():
    """Smeared semileptonic: jet scale N(1, 0.10), MET N(0, 10 GeV)."""
    return semilep(sigma_jet=0.10, sigma_met=10.0)


def config3():
    """Smeared dilepton ttH: same smearing model as the semileptonic one."""
    return dilep(sigma_jet=0.10, sigma_met=10.0)


def tth_sci():
    """The paper's ttH_sci resolution model on the dilepton chain: 1 % on
    every measured object -- jet and lepton energies scaled by N(1, 0.01),
    MET shifted by N(0, 1 GeV) per component."""
    return dilep(sigma_jet=0.01, sigma_met=1.0, sigma_lep=0.01)


def with_cuts(an, cuts):
    out = copy.deepcopy(an)
    out["cuts"] = list(cuts)
    return out
