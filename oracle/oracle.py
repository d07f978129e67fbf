"""ctypes binding of the FP64 oracle (hf_oracle.c) -- TEST INFRASTRUCTURE.

Builds liboracle.so with gcc (-O2 -ffp-contract=off, no -march flags) next to
the source on first use.  Imported only by tests, the smoke check and the
benchmark's CPU baseline.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_CUTS = 16
_KIND = {"njets_min": 1, "nbtag_min": 2, "lep_pt_min": 3, "met_min": 4,
         "wnu_solvable": 5, "hadtop_chi2_max": 6, "lep_os": 7,
         "dilep_solvable": 8, "higgs_window": 9, "ttbar_chi2_max": 10}
_MODEL = {"semilep": 1, "dilep": 2}


class _Analysis(C.Structure):
    _fields_ = [("model", C.c_int32), ("n_cuts", C.c_int32),
                ("kind", C.c_int32 * MAX_CUTS),
                ("param", (C.c_double * 2) * MAX_CUTS),
                ("mW", C.c_double), ("mt", C.c_double), ("sigma_t", C.c_double),
                ("sigma_W", C.c_double), ("mH", C.c_double),
                ("sigma_jet", C.c_double), ("sigma_met", C.c_double),
                ("hist_nbins", C.c_int32), ("hist_lo", C.c_double),
                ("hist_hi", C.c_double), ("sigma_lep", C.c_double)]


class _UnitResult(C.Structure):
    _fields_ = [("passed", C.c_int32), ("idx", C.c_int32 * 4),
                ("q", C.c_double * 6)]


class _NuSol(C.Structure):
    _fields_ = [("nu1", C.c_double * 4), ("nu2", C.c_double * 4),
                ("x", C.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so (seconds).  Returns its path."""
    with _lock:
        if force or not os.path.exists(_LIB) or \
                os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off",
                                   "-fno-fast-math", "-D_DEFAULT_SOURCE",
                                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        vp = C.c_void_p
        lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
        lib.orc_unit_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, vp]
        lib.orc_w_pz.argtypes = [vp, C.c_double, C.c_double, C.c_double, vp, vp]
        lib.orc_w_pz.restype = C.c_int
        lib.orc_hadtop.argtypes = [C.c_int, vp, C.c_double, C.c_double, C.c_double,
                                   C.c_double, vp, vp, vp, vp, vp]
        lib.orc_hadtop.restype = C.c_double
        lib.orc_w_pz_both.argtypes = [vp, C.c_double, C.c_double, C.c_double, vp]
        lib.orc_w_pz_both.restype = C.c_int
        lib.orc_ttbar.argtypes = [C.c_int, vp, vp, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_double, vp, vp, vp, vp]
        lib.orc_ttbar.restype = C.c_double
        lib.orc_real_roots.argtypes = [vp, C.c_int, vp]
        lib.orc_real_roots.restype = C.c_int
        lib.orc_dilep_pairing.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double,
                                          C.c_double, C.c_double, vp, vp]
        lib.orc_dilep_pairing.restype = C.c_int
        lib.orc_hist_bin.argtypes = [C.c_double, C.c_int, C.c_double, C.c_double]
        lib.orc_hist_bin.restype = C.c_int
        lib.orc_mass.argtypes = [vp]
        lib.orc_mass.restype = C.c_double
        lib.orc_unit.argtypes = [vp, C.c_uint64, vp, vp, vp, vp, vp, vp,
                                 C.c_uint64, C.c_uint64, C.c_uint32, vp]
        lib.orc_unit.restype = C.c_int
        lib.orc_run.argtypes = [vp, C.c_uint64, vp, vp, vp, vp, vp, vp, C.c_uint64,
                                C.c_uint64, C.c_uint32, vp, vp, vp, vp, vp, vp, vp]
        lib.orc_run.restype = C.c_int
        _lib = lib
    return _lib


def _f32(x) -> float:
    return float(np.float32(x))


def _analysis(an) -> _Analysis:
    a = _Analysis()
    a.model = _MODEL[an["model"]]
    cuts = an["cuts"]
    if len(cuts) > MAX_CUTS:
        raise ValueError("too many cuts")
    a.n_cuts = len(cuts)
    for i, c in enumerate(cuts):
        a.kind[i] = _KIND[c[0]]
        for p in range(2):
            a.param[i][p] = _f32(c[1 + p]) if len(c) > 1 + p else 0.0
    for k in ("mW", "mt", "sigma_t", "sigma_W", "mH", "sigma_jet", "sigma_met"):
        setattr(a, k, _f32(an[k]))
    nb, lo, hi = an["hist"]
    a.hist_nbins = int(nb)
    a.hist_lo = _f32(lo)
    a.hist_hi = _f32(hi)
    a.sigma_lep = _f32(an.get("sigma_lep", 0.0))
    return a


def _ptr(x: np.ndarray):
    return x.ctypes.data_as(C.c_void_p)


def _cols(cols):
    arrs = (np.ascontiguousarray(cols.jet_off, dtype=np.uint32),
            np.ascontiguousarray(cols.jets, dtype=np.float32),
            np.ascontiguousarray(cols.btag, dtype=np.uint16),
            np.ascontiguousarray(cols.lep, dtype=np.float32),
            np.ascontiguousarray(cols.lep_q, dtype=np.int8),
            np.ascontiguousarray(cols.met, dtype=np.float32))
    return arrs


def run(an, cols, *, seed=0, V=1, first_event_id=0, unit_passed=False):
    """Run the oracle over a whole chunk.  Returns a dict with mask (u8[N]),
    cutflow (u64[n_cuts+1]), hist (u64[nbins+2]: under, bins, over),
    n_surv (u16[N]), reco (f64[N,4]), reco_abs (f64[N,4], means of |value|)
    and optionally unit_passed (i8[N,V])."""
    lib = load()
    a = _analysis(an)
    arrs = _cols(cols)
    N = cols.n_events
    nb = an["hist"][0]
    out = dict(mask=np.zeros(N, np.uint8), cutflow=np.zeros(len(an["cuts"]) + 1, np.uint64),
               hist=np.zeros(nb + 2, np.uint64), n_surv=np.zeros(N, np.uint16),
               reco=np.zeros((N, 4), np.float64), reco_abs=np.zeros((N, 4), np.float64))
    up = np.zeros((N, V), np.int8) if unit_passed else None
    rc = lib.orc_run(C.byref(a), N, *[_ptr(x) for x in arrs], first_event_id, seed, V,
                     _ptr(out["mask"]), _ptr(out["cutflow"]), _ptr(out["hist"]),
                     _ptr(out["n_surv"]), _ptr(out["reco"]),
                     _ptr(up) if up is not None else None, _ptr(out["reco_abs"]))
    if rc != 0:
        raise ValueError("oracle: invalid event columns")
    if up is not None:
        out["unit_passed"] = up
    return out


RECORD_VARS = ("none", "njets", "nbtag", "lep_pt", "met", "reco0", "reco1", "reco2", "reco3")


def records(an, cols, *, seed=0, V=1, first_event_id=0):
    """Per-cut variable records (Sect. 3: the variables the user chose are
    stored at every selection level, holding their default where not yet
    updated; Sect. 6.1 example).  an["record"] = dict(levels=[k, ...],
    vars=[name, ...]) with names from RECORD_VARS.

    Event e is recorded at level k when some variation of it passes cuts
    0..k in user order, i.e. when the most leading cuts passed by any of its
    variations exceeds k.  The recorded values are the event's number of
    jets, number of b-tagged jets, first-lepton pT and measured |MET| (FP64,
    rounded to float), and at the last level only the per-event mean
    reconstructed quantities (0 below it).  Returns a dict: event (u32),
    level (u32), value (f64[n, 4]; the reco slots as the FP64 means), sorted
    by (event, level), and the run's result dict."""
    rec = an["record"]
    levels = sorted(set(int(k) for k in rec["levels"]))
    names = list(rec.get("vars", ())) + ["none"] * (4 - len(rec.get("vars", ())))
    r = run(an, cols, seed=seed, V=V, first_event_id=first_event_id, unit_passed=True)
    N = cols.n_events
    maxf = r["unit_passed"].astype(np.int64).max(axis=1) if N else np.zeros(0, np.int64)
    n = np.diff(np.asarray(cols.jet_off, dtype=np.int64))
    btag = np.asarray(cols.btag, dtype=np.int64)
    nb = np.array([bin(int(b) & ((1 << int(k)) - 1)).count("1") for b, k in zip(btag, n)], dtype=np.int64)
    lep = np.asarray(cols.lep, dtype=np.float32).reshape(N, cols.n_lep, 4)[:, 0, :].astype(np.float64)
    met = np.asarray(cols.met, dtype=np.float32).reshape(N, 2).astype(np.float64)
    lep_pt = np.sqrt(lep[:, 0] * lep[:, 0] + lep[:, 1] * lep[:, 1]).astype(np.float32)
    met_abs = np.sqrt(met[:, 0] * met[:, 0] + met[:, 1] * met[:, 1]).astype(np.float32)
    last = len(an["cuts"]) - 1
    ev, lv, val = [], [], []
    for e in range(N):
        for k in levels:
            if maxf[e] <= k:
                continue
            row = []
            for name in names:
                if name == "njets":
                    x = float(n[e])
                elif name == "nbtag":
                    x = float(nb[e])
                elif name == "lep_pt":
                    x = float(lep_pt[e])
                elif name == "met":
                    x = float(met_abs[e])
                elif name.startswith("reco"):
                    x = float(r["reco"][e, int(name[4])]) if k == last else 0.0
                else:
                    x = 0.0
                row.append(x)
            ev.append(e)
            lv.append(k)
            val.append(row)
    return dict(event=np.asarray(ev, np.uint32), level=np.asarray(lv, np.uint32),
                value=np.asarray(val, np.float64).reshape(-1, 4), run=r)


def best_of(an, cols, *, seed=0, V=1, first_event_id=0):
    """Best-of-variations per event (Sect. 4, ttH_sci: of the solutions over
    the pseudo-experiments only the most probable one is kept).  Among the
    variations of event e that pass every cut, the one whose reconstruction
    is most probable: the smallest chi2 of the analysis's fit (the hadronic
    chi2 of Eq. 1, or the full Eq. 1 chi2 when the analysis has the full fit)
    for the semileptonic model, the smallest m_ttbar of the chosen solution
    for the dilepton model (the same criterion that picks the solution within
    a variation); ties go to the lowest variation index.

    Returns dict: best_v (i32[N], -1 without a surviving variation), score
    (f64[N], +inf without one), reco (f64[N, 4], that variation's quantities,
    zeros without one), hist (u64[nbins+2], filled once per selected event
    with its best variation's histogram variable).  Built on unit(): slow,
    for small inputs."""
    N = cols.n_events
    nc = len(an["cuts"])
    nb, lo, hi = an["hist"]
    best_v = np.full(N, -1, np.int32)
    score = np.full(N, np.inf)
    reco = np.zeros((N, 4))
    hist = np.zeros(nb + 2, np.uint64)
    dilep = an["model"] == "dilep"
    for e in range(N):
        for v in range(V):
            u = unit(an, cols, e, v, seed=seed, first_event_id=first_event_id)
            if u["passed"] != nc:
                continue
            sc = u["q"][3] if dilep else u["q"][4]
            if sc < score[e]:
                score[e] = sc
                best_v[e] = v
                reco[e] = u["q"][:4]
        if best_v[e] >= 0:
            hist[hist_bin(reco[e, 0], nb, lo, hi)] += 1
    return dict(best_v=best_v, score=score, reco=reco, hist=hist)


def unit(an, cols, e, v, *, seed=0, first_event_id=0):
    """One unit (event e, variation v): dict(passed, idx[4], q[6])."""
    lib = load()
    a = _analysis(an)
    arrs = _cols(cols)
    r = _UnitResult()
    lib.orc_unit(C.byref(a), e, *[_ptr(x) for x in arrs], first_event_id, seed, v, C.byref(r))
    return dict(passed=r.passed, idx=list(r.idx), q=list(r.q))


def philox4x32_10(ctr, key):
    lib = load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def unit_normals(seed, event, v):
    lib = load()
    z = np.zeros(16, np.float64)
    lib.orc_unit_normals(seed, event, v, _ptr(z))
    return z


def w_pz(lep, metx, mety, mW):
    lib = load()
    l4 = np.ascontiguousarray(lep, dtype=np.float64)
    pz = C.c_double()
    dn = C.c_int()
    ok = lib.orc_w_pz(_ptr(l4), metx, mety, mW, C.byref(pz), C.byref(dn))
    return bool(ok), pz.value, bool(dn.value)


def hadtop(jets, mW, mt, sigma_W, sigma_t):
    lib = load()
    j = np.ascontiguousarray(jets, dtype=np.float64).reshape(-1, 4)
    k, i, jj = C.c_int(), C.c_int(), C.c_int()
    mtop, mw = C.c_double(), C.c_double()
    chi2 = lib.orc_hadtop(j.shape[0], _ptr(j), mW, mt, sigma_W, sigma_t, C.byref(k),
                          C.byref(i), C.byref(jj), C.byref(mtop), C.byref(mw))
    return dict(chi2=chi2, k=k.value, i=i.value, j=jj.value, mtop=mtop.value, mw=mw.value)


def w_pz_both(lep, metx, mety, mW):
    """Neutrino p_z solutions of the W-mass constraint (0, 1 or 2 values)."""
    lib = load()
    l4 = np.ascontiguousarray(lep, dtype=np.float64)
    pz = np.zeros(2, np.float64)
    n = lib.orc_w_pz_both(_ptr(l4), metx, mety, mW, _ptr(pz))
    return pz[:n].copy()


def ttbar(jets, lep, metx, mety, mW, mt, sigma_W, sigma_t):
    """Full Eq. 1 fit: dict(chi2, idx (k, i, j, l, r), mtop_had, mtop_lep, pz)."""
    lib = load()
    j = np.ascontiguousarray(jets, dtype=np.float64).reshape(-1, 4)
    l4 = np.ascontiguousarray(lep, dtype=np.float64)
    idx = np.zeros(5, np.int32)
    mh, ml, pz = C.c_double(), C.c_double(), C.c_double()
    chi2 = lib.orc_ttbar(j.shape[0], _ptr(j), _ptr(l4), metx, mety, mW, mt, sigma_W, sigma_t, _ptr(idx),
                         C.byref(mh), C.byref(ml), C.byref(pz))
    return dict(chi2=chi2, idx=idx.tolist(), mtop_had=mh.value, mtop_lep=ml.value, pz=pz.value)


def real_roots(coeffs):
    """Real roots (ascending) of sum coeffs[i] x^i, degree <= 4."""
    lib = load()
    c = np.zeros(5, np.float64)
    c[:len(coeffs)] = coeffs
    r = np.zeros(4, np.float64)
    n = lib.orc_real_roots(_ptr(c), len(coeffs) - 1, _ptr(r))
    return r[:n].copy()


def dilep_pairing(l1, b1, l2, b2, metx, mety, mW, mt):
    lib = load()
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (l1, b1, l2, b2)]
    sol = (_NuSol * 4)()
    quart = np.zeros(5, np.float64)
    n = lib.orc_dilep_pairing(*[_ptr(x) for x in arrs], metx, mety, mW, mt, sol, _ptr(quart))
    out = [dict(nu1=np.array(sol[s].nu1), nu2=np.array(sol[s].nu2), x=sol[s].x)
           for s in range(n)]
    return out, quart


def hist_bin(x, nbins, lo, hi):
    return load().orc_hist_bin(x, nbins, lo, hi)


def mass(p4):
    v = np.ascontiguousarray(p4, dtype=np.float64)
    return load().orc_mass(_ptr(v))
