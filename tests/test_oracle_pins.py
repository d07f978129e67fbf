"""Pins of the FP64 oracle against facts that do not come from the oracle:
library routines (Triton's Philox, numpy.roots), closed forms, planted-truth
events built by two-body decays, brute force on tiny inputs and invariants.
No GPU needed."""
import itertools
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from synth import analyses
from tests import kinematics as K

HERE = os.path.dirname(os.path.abspath(__file__))
F32 = lambda x: float(np.float32(x))  # noqa: E731


# ---------------------------------------------------------------- Philox
_TRITON_PROBE = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(seed, c_ptr, out_ptr, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    o0, o1, o2, o3 = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, o0)
    tl.store(out_ptr + offs * 4 + 1, o1)
    tl.store(out_ptr + offs * 4 + 2, o2)
    tl.store(out_ptr + offs * 4 + 3, o3)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    c = torch.tensor(np.array(ctrs, dtype=np.uint32).reshape(-1).view(np.int32))
    o = torch.zeros_like(c)
    k[(1,)](seed, c, o, N=len(ctrs))
    res.append(o.numpy().view(np.uint32).reshape(-1, 4).tolist())
print(json.dumps(res))
"""


def test_philox_matches_triton_library(orc):
    """Philox4x32-10 (Salmon et al. SC'11) against Triton's tl.philox run by
    Triton's CPU interpreter (key = (seed_lo32, seed_hi32), 10 rounds)."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    cases = []
    for seed in (0, 1, 1002, 0xFFFFFFFF, 0x123456789ABCDEF, (1 << 63) + 12345):
        ctrs = rng.integers(0, 2 ** 32, size=(8, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = 0xFFFFFFFF
        ctrs[2] = [0, 1, 5, 0]
        cases.append((int(seed), ctrs.tolist()))
    p = subprocess.run([sys.executable, "-c", _TRITON_PROBE], input=json.dumps(cases),
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lib_out = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctrs), ref in zip(cases, lib_out):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, r in zip(ctrs, ref):
            got = orc.philox4x32_10(c, key)
            assert [int(x) for x in got] == [int(x) for x in r], (seed, c)


def test_uniform_conversion_range_and_exactness(orc):
    lib = orc.load()
    import ctypes as C
    lib.orc_u01.argtypes = [C.c_uint32]
    lib.orc_u01.restype = C.c_double
    lo, hi = lib.orc_u01(0), lib.orc_u01(0xFFFFFFFF)
    assert lo == 2.0 ** -24 and hi == 1.0 - 2.0 ** -24
    for x in (0, 511, 512, 0x80000000, 0xFFFFFE00, 12345678):
        u = lib.orc_u01(x)
        assert float(np.float32(u)) == u  # exact in FP32
        assert u == ((x >> 9) + 0.5) / 2 ** 23


def test_box_muller_layout_closed_form(orc):
    """z[2k]^2 + z[2k+1]^2 = -2 ln u(w[2k]) and atan2 gives 2 pi u(w[2k+1]),
    with w the 16 Philox words of blocks (b, v, e_lo, e_hi), key = seed."""
    seed, ev, v = 1002, (1 << 33) + 17, 5
    z = orc.unit_normals(seed, ev, v)
    w = np.concatenate([orc.philox4x32_10([b, v, ev & 0xFFFFFFFF, ev >> 32],
                                          [seed & 0xFFFFFFFF, seed >> 32]) for b in range(4)])
    u = ((w >> 9).astype(np.float64) + 0.5) / 2 ** 23
    for k in range(8):
        r2 = z[2 * k] ** 2 + z[2 * k + 1] ** 2
        assert r2 == pytest.approx(-2 * np.log(u[2 * k]), rel=1e-13)
        ang = np.arctan2(z[2 * k + 1], z[2 * k]) % (2 * np.pi)
        assert ang == pytest.approx(2 * np.pi * u[2 * k + 1], abs=1e-12)


def _ulps(a, b):
    """Distance in units in the last place of b."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_box_muller_functions_within_an_ulp(orc):
    """The fixed-operation ln and sin / cos of 2 pi u that define the normals,
    against numpy's on every kind of uniform they see (multiples of 2^-24 in
    (0, 1), quadrant boundaries, the extremes): within 1.5 ulp (the
    truncation of the series is below 2^-56)."""
    import ctypes as C
    lib = orc.load()
    lib.orc_bm_log.argtypes = [C.c_double]
    lib.orc_bm_log.restype = C.c_double
    lib.orc_bm_sincos2pi.argtypes = [C.c_double, C.c_void_p, C.c_void_p]
    rng = np.random.default_rng(3)
    k = np.concatenate([rng.integers(1, 1 << 24, 200000), [1, 2, 3, (1 << 24) - 1, 1 << 22, 1 << 23, 3 << 22,
                                                           (1 << 22) + 1, (1 << 21) + 1, (1 << 23) - 1]])
    u = k.astype(np.float64) / 2.0 ** 24
    lg = np.array([lib.orc_bm_log(x) for x in u])
    assert _ulps(lg, np.log(u)).max() <= 1.5
    sn, cs = C.c_double(), C.c_double()
    s_, c_ = [], []
    for x in u:
        lib.orc_bm_sincos2pi(x, C.byref(sn), C.byref(cs))
        s_.append(sn.value)
        c_.append(cs.value)
    s_, c_ = np.array(s_), np.array(c_)
    # reference in extended precision of the angle: 2 pi u exactly = 2 pi k / 2^24
    import mpmath
    mpmath.mp.prec = 120
    pick = rng.choice(u.size, 4000, replace=False).tolist() + list(range(u.size - 10, u.size))
    for i in pick:
        th = 2 * mpmath.pi * mpmath.mpf(int(k[i])) / 2 ** 24
        es, ec = float(mpmath.sin(th)), float(mpmath.cos(th))
        tol_s = 1.5 * np.spacing(abs(es)) if abs(es) > 1e-300 else 1e-300
        tol_c = 1.5 * np.spacing(abs(ec)) if abs(ec) > 1e-300 else 1e-300
        assert abs(s_[i] - es) <= max(tol_s, 2.0 ** -60), (k[i], s_[i], es)
        assert abs(c_[i] - ec) <= max(tol_c, 2.0 ** -60), (k[i], c_[i], ec)
    assert np.abs(s_ * s_ + c_ * c_ - 1.0).max() <= 4.5e-16  # two roundings of the squares and the sum


def test_normals_moments(orc):
    """1.6e5 normals: mean, variance, 4th moment within 5 sigma; bounded."""
    zs = np.concatenate([orc.unit_normals(1, e, v) for e in range(2000) for v in range(5)])
    n = zs.size
    assert abs(zs.mean()) < 5 / np.sqrt(n)
    assert abs(zs.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs((zs ** 4).mean() - 3) < 5 * np.sqrt(96 / n)
    assert np.abs(zs).max() <= np.sqrt(-2 * np.log(2.0 ** -24)) + 1e-12


def test_smearing_sigma_zero_is_unsmeared(orc):
    cols = synth.gen_semilep(500, 11)
    base = orc.run(analyses.config1(), cols)
    an0 = analyses.semilep(sigma_jet=0.0, sigma_met=0.0)
    three = orc.run(an0, cols, seed=99, V=3)
    assert np.array_equal(three["cutflow"], 3 * base["cutflow"])
    assert np.array_equal(three["hist"], 3 * base["hist"])
    assert np.array_equal(three["mask"], base["mask"])
    # (x + x + x) / 3 may differ from x in the last bit
    assert np.allclose(three["reco"], base["reco"], rtol=1e-15, atol=0)


# ---------------------------------------------------------------- masses
def test_mass_closed_forms(orc):
    rng = np.random.default_rng(3)
    for _ in range(50):
        v = K.random_parent(5.0, rng)
        assert orc.mass(v) == pytest.approx(5.0, rel=1e-10)
    # negative m^2 -> negative mass (Lorentz-vector convention)
    assert orc.mass([3.0, 0.0, 0.0, 0.0]) == -3.0
    assert orc.mass([0.0, 0.0, 0.0, 2.0]) == 2.0
    # rotation about z and boosts leave the triplet mass unchanged
    jets = [K.random_parent(5.0, rng) for _ in range(3)]
    s = jets[0] + jets[1] + jets[2]
    m0 = orc.mass(s)
    c, sn = np.cos(0.7), np.sin(0.7)
    rot = [np.array([c * j[0] - sn * j[1], sn * j[0] + c * j[1], j[2], j[3]]) for j in jets]
    assert orc.mass(rot[0] + rot[1] + rot[2]) == pytest.approx(m0, rel=1e-12)
    bst = [K.boost(j, [0.3, -0.2, 0.5]) for j in jets]
    assert orc.mass(bst[0] + bst[1] + bst[2]) == pytest.approx(m0, rel=1e-11)


def test_appendix_style_system_sum(orc):
    """Appendix-style sum of three objects: m and pT of t + tbar + H built
    from (pT, eta, phi, m) equal the direct sums."""
    def ptetaphim(pt, eta, phi, m):
        return K.p4(pt * np.cos(phi), pt * np.sin(phi), pt * np.sinh(eta), m)
    t = ptetaphim(120.0, 0.4, 1.0, 172.5)
    tb = ptetaphim(80.0, -1.2, -2.0, 172.5)
    h = ptetaphim(60.0, 2.0, 0.3, 125.0)
    s = t + tb + h
    assert orc.mass(t) == pytest.approx(172.5, rel=1e-12)
    assert orc.mass(h) == pytest.approx(125.0, rel=1e-12)
    assert orc.mass(s) == pytest.approx(np.sqrt(s[3] ** 2 - s[:3] @ s[:3]), rel=1e-13)


# ---------------------------------------------------------------- W p_z
def _planted_w(rng):
    W = K.random_parent(80.4, rng, pmax=150)
    lep, nu = K.two_body(W, 0.0, 0.0, rng)
    return lep, nu


def test_w_pz_planted_truth(orc):
    """Lepton and neutrino from a W(80.4) decay: the true p_z is one of the
    two roots; the returned root is the smaller |p_z| one; both roots meet
    the mass constraint (massless lepton and neutrino)."""
    rng = np.random.default_rng(5)
    hits = 0
    for _ in range(300):
        lep, nu = _planted_w(rng)
        ok, pz, dneg = orc.w_pz(lep, nu[0], nu[1], 80.4)
        assert ok
        # the two roots of a pz^2 - 2 mu pzl pz + (El^2 pT^2 - mu^2)
        mu = 80.4 ** 2 / 2 + lep[0] * nu[0] + lep[1] * nu[1]
        a = lep[3] ** 2 - lep[2] ** 2
        pt2 = nu[0] ** 2 + nu[1] ** 2
        roots = np.roots([a, -2 * mu * lep[2], lep[3] ** 2 * pt2 - mu ** 2])
        if np.all(np.abs(roots.imag) < 1e-9 * np.abs(roots.real).max()):
            roots = roots.real
            assert min(np.abs(roots - nu[2])) < 1e-6 * (1 + abs(nu[2]))
            small = roots[np.argmin(np.abs(roots))]
            assert pz == pytest.approx(small, rel=1e-9, abs=1e-9)
            for r in roots:
                n4 = K.p4(nu[0], nu[1], r, 0.0)
                assert K.minkowski_m2(lep + n4) == pytest.approx(80.4 ** 2, rel=1e-9)
            hits += 1
    assert hits > 250


def test_w_pz_negative_discriminant_real_part(orc):
    """D < 0: the real part of the complex pair (numpy.roots)."""
    rng = np.random.default_rng(6)
    seen = 0
    for _ in range(200):
        lep = K.p4(*rng.uniform(-80, 80, 3), 0.0)
        metx, mety = rng.uniform(-400, 400, 2)
        ok, pz, dneg = orc.w_pz(lep, metx, mety, 80.4)
        if not dneg:
            continue
        seen += 1
        mu = 80.4 ** 2 / 2 + lep[0] * metx + lep[1] * mety
        a = lep[3] ** 2 - lep[2] ** 2
        roots = np.roots([a, -2 * mu * lep[2], lep[3] ** 2 * (metx ** 2 + mety ** 2) - mu ** 2])
        assert np.all(np.abs(roots.imag) > 0)
        assert pz == pytest.approx(roots[0].real, rel=1e-10, abs=1e-9)
    assert seen > 20


# ---------------------------------------------------------------- hadronic top
def _chi2_gram(jets, idx_w, k, mW, mt, sW, sT):
    """chi2 from the Minkowski Gram matrix (sum over pairs), an independent
    formulation of the invariant masses."""
    def m_of(ids):
        G = 0.0
        for a in ids:
            for b in ids:
                va, vb = jets[a], jets[b]
                G += va[3] * vb[3] - va[:3] @ vb[:3]
        return np.sqrt(G) if G >= 0 else -np.sqrt(-G)
    mw = m_of(idx_w)
    mtop = m_of(list(idx_w) + [k])
    return ((mtop - mt) / sT) ** 2 + ((mw - mW) / sW) ** 2


def test_hadtop_brute_force_permutations(orc):
    """All n! jet assignments on n = 3..6 (itertools.permutations, dedup):
    the oracle's minimum and its first-in-order tie rule."""
    rng = np.random.default_rng(8)
    for n in (3, 4, 5, 6):
        for _ in range(15):
            jets = [K.random_parent(5.0, rng, pmax=120) for _ in range(n)]
            best, arg = np.inf, None
            seen = set()
            for perm in itertools.permutations(range(n)):
                k, i, j = perm[0], min(perm[1], perm[2]), max(perm[1], perm[2])
                if (k, i, j) in seen:
                    continue
                seen.add((k, i, j))
                c = _chi2_gram(jets, (i, j), k, 80.4, 172.5, 10.0, 15.0)
                if arg is None or c < best - 1e-9 * max(1.0, best) or (abs(c - best) <= 1e-9 * max(1.0, best)
                                                          and arg is not None and (k, i, j) < arg):
                    best, arg = c, (k, i, j)
            r = orc.hadtop(np.array(jets), 80.4, 172.5, 10.0, 15.0)
            assert len(seen) == n * (n - 1) * (n - 2) // 2
            assert r["chi2"] == pytest.approx(best, rel=1e-9, abs=1e-12)
            assert (r["k"], r["i"], r["j"]) == arg


def test_hadtop_planted_truth(orc):
    """t(172.5) -> b W(80.4), W -> q q', all jets m = 5, plus soft extra jets:
    chi2 ~ 0 and the planted indices win."""
    rng = np.random.default_rng(9)
    for _ in range(40):
        top = K.random_parent(172.5, rng, pmax=200)
        b, W = K.two_body(top, 5.0, 80.4, rng)
        q1, q2 = K.two_body(W, 5.0, 5.0, rng)
        extra = [K.random_parent(5.0, rng, pmax=20) for _ in range(rng.integers(0, 4))]
        jets = [q1, b, q2] + extra
        perm = rng.permutation(len(jets))
        shuffled = [jets[p] for p in perm]
        pos = {orig: new for new, orig in enumerate(perm)}
        r = orc.hadtop(np.array(shuffled), 80.4, 172.5, 10.0, 15.0)
        assert r["chi2"] < 1e-12
        assert r["k"] == pos[1]
        assert {r["i"], r["j"]} == {pos[0], pos[2]}
        assert r["mtop"] == pytest.approx(172.5, rel=1e-12)
        assert r["mw"] == pytest.approx(80.4, rel=1e-12)


def test_hadtop_too_few_jets_is_infinite(orc):
    rng = np.random.default_rng(1)
    jets = np.array([K.random_parent(5.0, rng) for _ in range(2)])
    assert orc.hadtop(jets, 80.4, 172.5, 10.0, 15.0)["chi2"] == np.inf


# ---------------------------------------------------------------- full Eq. 1 fit
def _nu_solutions_numpy(lep, metx, mety, mW):
    """Neutrino p_z of the W-mass constraint by numpy.roots (an independent
    route): real roots ordered by |p_z|, or the real part of a complex pair."""
    mu = mW ** 2 / 2 + lep[0] * metx + lep[1] * mety
    a = lep[3] ** 2 - lep[2] ** 2
    roots = np.roots([a, -2 * mu * lep[2], lep[3] ** 2 * (metx ** 2 + mety ** 2) - mu ** 2])
    if np.any(np.abs(roots.imag) > 0):
        return [roots[0].real]
    return sorted(roots.real.tolist(), key=abs)


def test_w_pz_both_roots(orc):
    """Both solutions: the numpy.roots roots in |p_z| order, each meeting the
    W-mass constraint; the first is orc.w_pz's; D < 0 gives its real part."""
    rng = np.random.default_rng(21)
    n2 = n1 = 0
    for _ in range(300):
        lep = K.p4(*rng.uniform(-90, 90, 3), 0.0)
        metx, mety = rng.uniform(-200, 200, 2)
        sol = orc.w_pz_both(lep, metx, mety, 80.4)
        ref = _nu_solutions_numpy(lep, metx, mety, 80.4)
        ok, pz1, dneg = orc.w_pz(lep, metx, mety, 80.4)
        assert len(sol) == len(ref)
        assert sol[0] == pz1
        for a, b in zip(sol, ref):
            assert a == pytest.approx(b, rel=1e-8, abs=1e-8)
        if len(sol) == 2:
            n2 += 1
            for r in sol:
                assert K.minkowski_m2(lep + K.p4(metx, mety, r, 0.0)) == pytest.approx(80.4 ** 2, rel=1e-9)
        else:
            n1 += 1
    assert n2 > 50 and n1 > 20


def _full_chi2_bruteforce(jets, lep, metx, mety, mW, mt, sW, sT):
    """Every (hadronic b, W pair, leptonic b, neutrino solution) by
    itertools.permutations of four jets, masses from the Minkowski Gram sum
    (independent of the oracle's four-vector sums); returns (chi2, key) of the
    minimum with the oracle's enumeration order as key for ties."""
    nus = _nu_solutions_numpy(lep, metx, mety, mW)

    def m_of(vs):
        G = 0.0
        for va in vs:
            for vb in vs:
                G += va[3] * vb[3] - va[:3] @ vb[:3]
        return np.sqrt(G) if G >= 0 else -np.sqrt(-G)
    best, key = np.inf, None
    seen = set()
    for k, i, j, l in itertools.permutations(range(len(jets)), 4):
        if i > j or (k, i, j, l) in seen:
            continue
        seen.add((k, i, j, l))
        had = ((m_of([jets[i], jets[j], jets[k]]) - mt) / sT) ** 2 + ((m_of([jets[i], jets[j]]) - mW) / sW) ** 2
        for r, pz in enumerate(nus):
            nu = K.p4(metx, mety, pz, 0.0)
            c = had + ((m_of([jets[l], lep, nu]) - mt) / sT) ** 2 + ((m_of([lep, nu]) - mW) / sW) ** 2
            kk = (k, i, j, l, r)
            if key is None or c < best - 1e-9 * max(1.0, best) or (abs(c - best) <= 1e-9 * max(1.0, best) and kk < key):
                best, key = c, kk
    return best, key


def test_ttbar_full_fit_brute_force(orc):
    """n = 4..6 jets: the oracle's minimum of the full Eq. 1 chi2 and its
    assignment equal the brute-force enumeration's."""
    rng = np.random.default_rng(22)
    for n in (4, 5, 6):
        for _ in range(12):
            jets = [K.random_parent(5.0, rng, pmax=120) for _ in range(n)]
            lep = K.p4(*rng.uniform(-60, 60, 3), 0.0)
            metx, mety = rng.uniform(-80, 80, 2)
            best, key = _full_chi2_bruteforce(jets, lep, metx, mety, 80.4, 172.5, 7.5, 11.5)
            r = orc.ttbar(np.array(jets), lep, metx, mety, 80.4, 172.5, 7.5, 11.5)
            assert r["chi2"] == pytest.approx(best, rel=1e-8, abs=1e-10)
            assert tuple(r["idx"]) == key


def test_ttbar_full_fit_planted_truth(orc):
    """ttbar -> (b q q')(b l nu) built by two-body decays, MET = the
    neutrino's pT: chi2 ~ 0 at the planted assignment, with the neutrino
    solution equal to the true p_z and both top masses 172.5."""
    rng = np.random.default_rng(23)
    for _ in range(40):
        th = K.random_parent(172.5, rng, pmax=150)
        tl = K.random_parent(172.5, rng, pmax=150)
        bh, Wh = K.two_body(th, 5.0, 80.4, rng)
        q1, q2 = K.two_body(Wh, 5.0, 5.0, rng)
        bl, Wl = K.two_body(tl, 5.0, 80.4, rng)
        lep, nu = K.two_body(Wl, 0.0, 0.0, rng)
        extra = [K.random_parent(5.0, rng, pmax=15) for _ in range(rng.integers(0, 3))]
        jets = [q1, bh, q2, bl] + extra
        perm = rng.permutation(len(jets))
        shuffled = [jets[p] for p in perm]
        pos = {orig: new for new, orig in enumerate(perm)}
        r = orc.ttbar(np.array(shuffled), lep, nu[0], nu[1], 80.4, 172.5, 7.5, 11.5)
        assert r["chi2"] < 1e-9
        k, i, j, l, sol = r["idx"]
        assert k == pos[1] and {i, j} == {pos[0], pos[2]} and l == pos[3]
        assert r["pz"] == pytest.approx(nu[2], rel=1e-6, abs=1e-6)
        assert r["mtop_had"] == pytest.approx(172.5, rel=1e-10)
        assert r["mtop_lep"] == pytest.approx(172.5, rel=1e-8)


def test_ttbar_needs_four_jets(orc):
    rng = np.random.default_rng(2)
    jets = np.array([K.random_parent(5.0, rng) for _ in range(3)])
    lep = K.p4(30.0, 10.0, 5.0, 0.0)
    assert orc.ttbar(jets, lep, 20.0, -10.0, 80.4, 172.5, 7.5, 11.5)["chi2"] == np.inf


# ---------------------------------------------------------------- quartic
def test_real_roots_from_known_roots(orc):
    """Polynomials built from known real roots times an irreducible
    quadratic: the oracle finds exactly the planted real roots."""
    rng = np.random.default_rng(10)
    for _ in range(300):
        nreal = rng.choice([0, 2, 4])
        rr = np.sort(rng.uniform(-500, 500, nreal))
        if nreal == 4 and np.min(np.diff(rr)) < 1e-3:
            continue
        poly = np.poly1d([1.0])
        for r in rr:
            poly *= np.poly1d([1.0, -r])
        for _ in range((4 - nreal) // 2):
            p, q = rng.uniform(-100, 100), rng.uniform(1, 100)
            poly *= np.poly1d([1.0, p, p * p / 4 + q])
        lead = rng.uniform(0.1, 10) * rng.choice([-1, 1])
        c = (poly.coeffs * lead)[::-1]
        got = orc.real_roots(c)
        assert got.size == nreal
        assert np.allclose(got, rr, rtol=1e-8, atol=1e-7)


def test_real_roots_vs_numpy_roots_random(orc):
    """Random quartic coefficients: real roots equal the real eigenvalues of
    the companion matrix (numpy.roots), away from near-double roots."""
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(2000):
        c = rng.normal(size=5) * 10.0 ** rng.uniform(-2, 2, 5)
        r = np.roots(c[::-1])
        real = np.sort(r[np.abs(r.imag) < 1e-7 * (1 + np.abs(r.real))].real)
        cplx = r[np.abs(r.imag) >= 1e-7 * (1 + np.abs(r.real))]
        if cplx.size and np.min(np.abs(cplx.imag)) < 1e-3 * (1 + np.abs(cplx.real).max()):
            continue
        if real.size > 1 and np.min(np.diff(real)) < 1e-4 * (1 + np.abs(real).max()):
            continue
        got = orc.real_roots(c)
        assert got.size == real.size
        assert np.allclose(got, real, rtol=1e-8, atol=1e-9)
        checked += 1
    assert checked > 1500


def test_real_roots_degenerate_degrees(orc):
    assert np.allclose(orc.real_roots([-6.0, 1.0]), [6.0])
    assert orc.real_roots([1.0, 0.0, 1.0]).size == 0          # x^2 + 1
    assert np.allclose(orc.real_roots([-4.0, 0.0, 1.0, 0.0, 0.0]), [-2.0, 2.0])
    got = orc.real_roots([0.0, 0.0, 1.0])                      # double root at 0
    assert got.size == 1 and got[0] == 0.0
    assert orc.real_roots([5.0]).size == 0


# ---------------------------------------------------------------- dilepton
def _planted_ttbar(rng):
    t = K.random_parent(172.5, rng, pmax=250)
    tb = K.random_parent(172.5, rng, pmax=250)
    b1, W1 = K.two_body(t, 5.0, 80.4, rng)
    l1, n1 = K.two_body(W1, 0.0, 0.0, rng)
    b2, W2 = K.two_body(tb, 5.0, 80.4, rng)
    l2, n2 = K.two_body(W2, 0.0, 0.0, rng)
    return l1, b1, n1, l2, b2, n2


def test_dilep_planted_truth_among_solutions(orc):
    """ttbar -> b l nu b l nu by two-body decays, MET = nu1_T + nu2_T: the true
    neutrinos are among the solutions; every solution meets all constraints
    (two W masses, two top masses, two massless neutrinos; MET exactly).
    The constraint residual is ~1e-14 typically; near-double roots of the
    quartic lose about half the digits, so the bound is 1e-10 for 95 % of
    solutions and 1e-4 for all (a wrong term gives residuals of order 1)."""
    rng = np.random.default_rng(12)
    found = 0
    res = []
    for _ in range(400):
        l1, b1, n1, l2, b2, n2 = _planted_ttbar(rng)
        mx, my = n1[0] + n2[0], n1[1] + n2[1]
        sols, quart = orc.dilep_pairing(l1, b1, l2, b2, mx, my, 80.4, 172.5)
        assert 1 <= len(sols) <= 4
        xs = [s["x"] for s in sols]
        assert xs == sorted(xs)
        for s in sols:
            v1, v2 = s["nu1"], s["nu2"]
            res.append(max(abs(K.minkowski_m2(v1)) / v1[3] ** 2,
                           abs(K.minkowski_m2(v2)) / v2[3] ** 2,
                           abs(K.minkowski_m2(l1 + v1) / 80.4 ** 2 - 1),
                           abs(K.minkowski_m2(l2 + v2) / 80.4 ** 2 - 1),
                           abs(K.minkowski_m2(b1 + l1 + v1) / 172.5 ** 2 - 1),
                           abs(K.minkowski_m2(b2 + l2 + v2) / 172.5 ** 2 - 1)))
            assert v1[0] + v2[0] == pytest.approx(mx, rel=1e-12, abs=1e-9)
            assert v1[1] + v2[1] == pytest.approx(my, rel=1e-12, abs=1e-9)
            assert v1[3] > 0 and v2[3] > 0
        d = [np.max(np.abs(s["nu1"] - n1)) + np.max(np.abs(s["nu2"] - n2)) for s in sols]
        if min(d) < 1e-5 * (1 + np.abs(n1).max() + np.abs(n2).max()):
            found += 1
    res = np.array(res)
    assert res.max() < 1e-4
    assert np.percentile(res, 95) < 1e-10
    # the truth can be lost only when it is an (ill-conditioned) near-double root
    assert found >= 390


def test_dilep_quartic_roots_match_numpy(orc):
    """The x roots used equal numpy.roots of the oracle's own quartic (the
    root finder is pinned separately above; this pins its use)."""
    rng = np.random.default_rng(13)
    for _ in range(100):
        l1, b1, n1, l2, b2, n2 = _planted_ttbar(rng)
        sols, quart = orc.dilep_pairing(l1, b1, l2, b2, n1[0] + n2[0], n1[1] + n2[1],
                                        80.4, 172.5)
        r = np.roots(quart[::-1])
        real = np.sort(r[np.abs(r.imag) < 1e-6 * (1 + np.abs(r))].real)
        xs = np.array([s["x"] for s in sols])
        for x in xs:
            assert np.min(np.abs(real - x)) < 1e-6 * (1 + abs(x))


# ---------------------------------------------------------------- histogram
def test_hist_bin_edges(orc):
    assert orc.hist_bin(-1e-9, 50, 0.0, 500.0) == 0
    assert orc.hist_bin(0.0, 50, 0.0, 500.0) == 1
    assert orc.hist_bin(9.999999999, 50, 0.0, 500.0) == 1
    assert orc.hist_bin(10.0, 50, 0.0, 500.0) == 2
    assert orc.hist_bin(172.5, 50, 0.0, 500.0) == 18
    assert orc.hist_bin(499.99999, 50, 0.0, 500.0) == 50
    assert orc.hist_bin(500.0, 50, 0.0, 500.0) == 51
    assert orc.hist_bin(float("nan"), 50, 0.0, 500.0) == 51
    # non-decimal edges: definition "largest i with x >= lo + i w"
    lo, hi, nb = 0.1, 0.7, 3
    w = (hi - lo) / nb
    for i in range(nb):
        e = lo + i * w
        assert orc.hist_bin(e, nb, lo, hi) == 1 + i
        assert orc.hist_bin(np.nextafter(e, -np.inf), nb, lo, hi) == i


# ---------------------------------------------------------------- chain semantics
def test_cutflow_semantics_against_columns(orc):
    """Config 1: the first four levels of the cut flow counted directly from
    the columns with numpy; invariants of the whole chain."""
    cols = synth.gen_semilep(3000, 21)
    an = analyses.config1()
    r = orc.run(an, cols)
    n = np.diff(cols.jet_off.astype(np.int64))
    nb = np.array([bin(int(b) & ((1 << int(k)) - 1)).count("1") for b, k in zip(cols.btag, n)])
    lpt = np.hypot(cols.lep[:, 0].astype(np.float64), cols.lep[:, 1].astype(np.float64))
    met = np.hypot(cols.met[:, 0].astype(np.float64), cols.met[:, 1].astype(np.float64))
    c1 = n >= 4
    c2 = c1 & (nb >= 1)
    c3 = c2 & (lpt > F32(30.0))
    c4 = c3 & (met > F32(20.0))
    cf = r["cutflow"]
    assert cf[0] == 3000 and cf[1] == c1.sum() and cf[2] == c2.sum()
    assert cf[3] == c3.sum() and cf[4] == c4.sum()
    assert cf[5] == cf[4]          # W p_z always solvable for pT(lepton) > 0
    assert np.all(np.diff(cf.astype(np.int64)) <= 0)
    assert cf[-1] == r["n_surv"].sum() == r["hist"].sum()
    assert np.array_equal(r["mask"], (r["n_surv"] >= 1).astype(np.uint8))


def test_chunk_additivity_and_event_ids(orc):
    """Splitting a chunk (with first_event_id) changes nothing: Philox keys
    by the global event id."""
    cols = synth.gen_semilep(800, 22)
    an = analyses.config2()
    full = orc.run(an, cols, seed=5, V=4)
    a = orc.run(an, cols.slice(0, 300), seed=5, V=4, first_event_id=0)
    b = orc.run(an, cols.slice(300, 800), seed=5, V=4, first_event_id=300)
    assert np.array_equal(full["cutflow"], a["cutflow"] + b["cutflow"])
    assert np.array_equal(full["hist"], a["hist"] + b["hist"])
    assert np.array_equal(full["mask"], np.concatenate([a["mask"], b["mask"]]))
    assert np.array_equal(full["reco"], np.concatenate([a["reco"], b["reco"]]))


def test_cut_order_changes_cutflow_not_selection(orc):
    """Cuts are pure predicates of a unit: any user order selects the same
    units; the cut flow is reported in the user's order."""
    cols = synth.gen_semilep(600, 23)
    an = analyses.config2()
    base = orc.run(an, cols, seed=3, V=3, unit_passed=True)
    rng = np.random.default_rng(0)
    for _ in range(5):
        perm = rng.permutation(len(an["cuts"]))
        an2 = analyses.with_cuts(an, [an["cuts"][p] for p in perm])
        r = orc.run(an2, cols, seed=3, V=3, unit_passed=True)
        assert np.array_equal(r["mask"], base["mask"])
        assert np.array_equal(r["hist"], base["hist"])
        assert np.array_equal(r["reco"], base["reco"])
        assert r["cutflow"][-1] == base["cutflow"][-1]


def test_dilep_chain_invariants(orc):
    cols = synth.gen_dilep(300, 31, p_same_sign=0.2)
    an = analyses.config3()
    r = orc.run(an, cols, seed=1003, V=4)
    q = cols.lep_q.reshape(-1, 2)
    os_ = (q[:, 0] * q[:, 1] < 0)
    assert r["cutflow"][1] == 4 * os_.sum()
    assert np.all(np.diff(r["cutflow"].astype(np.int64)) <= 0)
    assert r["cutflow"][-1] == r["n_surv"].sum() == r["hist"].sum()
    sel = r["mask"] == 1
    # m_bb of selected events inside the window; tops on the mass shell
    assert np.all((r["reco"][sel, 0] > 100) & (r["reco"][sel, 0] < 150))
    assert np.allclose(r["reco"][sel, 1], F32(172.5), rtol=1e-7)
    assert np.allclose(r["reco"][sel, 2], F32(172.5), rtol=1e-7)


def test_paper_constants_golden():
    """Constants printed in the paper (golden fixture with citations) are
    the defaults of the analysis descriptions."""
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as f:
        g = json.load(f)
    an = analyses.semilep()
    assert an["mt"] == g["m_t"]["value"] and an["mW"] == g["m_W"]["value"]
    assert analyses.dilep()["mH"] == g["m_H"]["value"]
    paper = analyses.semilep(sigma_t=g["sigma_t"]["value"], sigma_W=g["sigma_W"]["value"])
    assert (paper["sigma_t"], paper["sigma_W"]) == (11.5, 7.5)
