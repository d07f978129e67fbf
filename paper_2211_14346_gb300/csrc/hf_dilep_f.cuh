// hf_dilep_f.cuh -- fast evaluation of one dilepton unit (device code).
//
// The two-conic resultant amplifies the error of its inputs by several
// orders of magnitude, so an all-FP32 evaluation cannot decide most units.
// The fast path keeps FP64 where the conditioning demands it and moves only
// the long, branchy part -- bracketing the quartic's real roots by bisection
// -- to FP32:
//   * FP64 with the definition's operations: smearing normals of the b-jets
//     and MET, smeared b-jets, both conics of every (lepton, b-jet) pair, the
//     quartic's coefficients of every pairing (these equal the definition's
//     values up to the last bit of the Box-Muller transcendentals), the MET
//     cut and the Higgs pair;
//   * root isolation: x = S t with S a power of two near the Cauchy bound and
//     the coefficients normalised (both exact scalings of the same
//     polynomial); the sign of every level (R, R', R'') at its critical
//     points is evaluated in FP64 and must exceed its rounding bound; each
//     critical point is bracketed by FP32 bisection and the bracket
//     certified by FP64 signs at its ends (else bracketed again in FP64);
//     each root is bracketed by FP32 bisection, polished by FP64 Newton steps
//     and certified by an FP64 sign change across a tiny interval around it;
//   * FP64 back-substitution, E_nu signs and masses at the certified roots.
// Any decision the bounds cannot certify flags the unit for the FP64 recheck
// (the full definition).
#pragma once
#include "hf_dilep.cuh"

namespace hf {

struct SolD {
    double mtt, mt1, mt2;
};

// Horner in FP64 and a bound on its rounding error (coefficients exact).
__device__ __forceinline__ double peval_dd(const double* c, int d, double x, double* bound)
{
    double r = c[d], m = fabs(c[d]);
    const double ax = fabs(x);
    for (int i = d - 1; i >= 0; --i) {
        r = r * x + c[i];
        m = m * ax + fabs(c[i]);
    }
    *bound = (2.0 * d + 2.0) * 1.1102230246251565e-16 * m;
    return r;
}

// Certified real roots of the quartic cq (FP64 coefficients, exact scaling of
// the definition's polynomial).  Returns the number of roots (ascending,
// each within a relative 1e-12 of the definition's), or -1 if uncertain.
__device__ inline int real_roots_mixed(const double* R, float safety, double* roots)
{
    int d = 4;
    while (d > 0 && R[d] == 0.0) --d;  // the definition trims exact zeros only
    if (d <= 0) return 0;
    // scale: x = S t, S = 2^k near the Cauchy bound; normalise by the leading term
    double Bc = 0.0;
    for (int i = 0; i < d; ++i) Bc = fmax(Bc, fabs(R[i] / R[d]));
    Bc = 1.0 + Bc;
    int ex;
    frexp(Bc, &ex);
    const double S = ldexp(1.0, ex);  // power of two >= Bc: all roots |t| < 1
    double c[5];
    double sp = 1.0;
    for (int i = 0; i <= d; ++i) {
        c[i] = R[i] * sp;
        sp *= S;
    }
    const double lead = fabs(c[d]);
    for (int i = 0; i <= d; ++i) c[i] = c[i] / lead;  // |leading| = 1
    // levels: polynomial and derivatives (FP64 exact integer multiples, FP32 copies)
    double lev[4][5];
    float levf[4][5];
    int deg[4];
    for (int i = 0; i <= d; ++i) lev[0][i] = c[i];
    deg[0] = d;
    int L = 0;
    while (deg[L] > 1) {
        const int dd = deg[L] - 1;
        for (int i = 0; i <= dd; ++i) lev[L + 1][i] = (double)(i + 1) * lev[L][i + 1];
        ++L;
        deg[L] = dd;
    }
    for (int l = 0; l <= L; ++l)
        for (int i = 0; i <= deg[l]; ++i) levf[l][i] = (float)lev[l][i];
    double crit[4], crit_w[4], crit_d[4];  // critical points, their widths, a bound on |derivative| there
    int nc = 0;
    for (int l = L; l >= 0; --l) {
        const double* cl = lev[l];
        const float* cf = levf[l];
        const int dl = deg[l];
        double r[4], rw[4], rd[4];
        int nr = 0;
        if (dl == 1) {
            r[0] = -cl[0] / cl[1];
            rw[0] = 4.0e-16 * fabs(r[0]);
            rd[0] = 0.0;
            nr = 1;
        } else {
            double pts[6];
            int np = 0;
            pts[np++] = -1.0;
            for (int i = 0; i < nc; ++i) {
                // sign at a critical point (bracketed to FP32 resolution dc):
                // certain when it exceeds the rounding bound plus the change
                // the slope can make over dc
                double b, bd;
                const double v = peval_dd(cl, dl, crit[i], &b);
                double dv = 0.0, fv = cl[dl];
                for (int k = dl - 1; k >= 0; --k) {
                    dv = dv * crit[i] + fv;
                    fv = fv * crit[i] + cl[k];
                }
                bd = fmax(fabs(dv), crit_d[i]) * crit_w[i];
                if (!(fabs(v) > safety * (b + bd) + 1.0e-300)) return -1;
                if (crit[i] > -1.0 && crit[i] < 1.0) pts[np++] = crit[i];
            }
            pts[np++] = 1.0;
            for (int i = 0; i + 1 < np; ++i) {
                double b0, b1;
                const double flo = peval_dd(cl, dl, pts[i], &b0), fhi = peval_dd(cl, dl, pts[i + 1], &b1);
                if ((flo < 0.0) == (fhi < 0.0)) continue;
                const bool neg = flo < 0.0;
                // bracket in FP32
                float lo = (float)pts[i], hi = (float)pts[i + 1];
                for (int it = 0; it < 40; ++it) {
                    const float mid = 0.5f * (lo + hi);
                    if (!(mid > lo && mid < hi)) break;
                    float v = cf[dl];
                    for (int k = dl - 1; k >= 0; --k) v = fmaf(v, mid, cf[k]);
                    if ((v < 0.0f) == neg) lo = mid;
                    else hi = mid;
                }
                double t = 0.5 * ((double)lo + (double)hi);
                if (l > 0) {
                    // a critical point of the level above.  The FP32 signs near a
                    // root of this level are rounding noise, so the FP32 bracket
                    // counts only when the FP64 signs at its ends, beyond their
                    // rounding bounds, differ as they should; otherwise the root
                    // is bracketed again by FP64 bisection of the monotone
                    // interval, and a bracket that cannot be certified sends the
                    // unit to the FP64 recheck.
                    double dlo = (double)lo, dhi = (double)hi;
                    double bl, bh;
                    double fl = peval_dd(cl, dl, dlo, &bl), fh = peval_dd(cl, dl, dhi, &bh);
                    bool ok = fabs(fl) > safety * bl && fabs(fh) > safety * bh && (fl < 0.0) == neg &&
                              (fh < 0.0) != neg;
                    // widen the FP32 bracket until its ends certify (about one
                    // step when needed), within the monotone interval
                    double w = fmax((double)(hi - lo), 1.0e-300);
                    for (int k = 0; k < 24 && !ok; ++k) {
                        w *= 4.0;
                        dlo = fmax(pts[i], (double)lo - w);
                        dhi = fmin(pts[i + 1], (double)hi + w);
                        fl = peval_dd(cl, dl, dlo, &bl);
                        fh = peval_dd(cl, dl, dhi, &bh);
                        ok = fabs(fl) > safety * bl && fabs(fh) > safety * bh && (fl < 0.0) == neg &&
                             (fh < 0.0) != neg;
                        if (dlo == pts[i] && dhi == pts[i + 1]) break;
                    }
                    if (!ok) {
                        // FP64 bisection of the monotone interval, stopped while
                        // the midpoint's sign is still certain
                        dlo = pts[i];
                        dhi = pts[i + 1];
                        for (int it = 0; it < 64; ++it) {
                            const double mid = 0.5 * (dlo + dhi);
                            if (!(mid > dlo && mid < dhi)) break;
                            double bm;
                            const double fm = peval_dd(cl, dl, mid, &bm);
                            if (!(fabs(fm) > safety * bm)) break;
                            if ((fm < 0.0) == neg) dlo = mid;
                            else dhi = mid;
                        }
                        fl = peval_dd(cl, dl, dlo, &bl);
                        fh = peval_dd(cl, dl, dhi, &bh);
                        ok = fabs(fl) > safety * bl && fabs(fh) > safety * bh && (fl < 0.0) == neg && (fh < 0.0) != neg;
                        if (!ok) return -1;
                    }
                    r[nr] = 0.5 * (dlo + dhi);
                    rw[nr] = (dhi - dlo) + 1.0e-15 * fabs(r[nr]);
                    rd[nr] = fmax(fabs(fl) + bl, fabs(fh) + bh);  // |level| on the bracket (monotone)
                    ++nr;
                    continue;
                }
                // a root of the quartic: polish in FP64 (Newton, kept inside
                // the monotone interval), then certify
                const double ilo = pts[i], ihi = pts[i + 1];
                for (int it = 0; it < 2; ++it) {
                    double fv = cl[dl], dv = 0.0;
                    for (int k = dl - 1; k >= 0; --k) {
                        dv = dv * t + fv;
                        fv = fv * t + cl[k];
                    }
                    if (dv == 0.0) break;
                    const double tn = t - fv / dv;
                    if (!(tn > ilo && tn < ihi)) break;
                    t = tn;
                }
                // certify: a sign change across [t - h, t + h] inside the interval
                const double h = 1.0e-9 * fabs(t) + 1.0e-300;
                double bl, bh;
                const double fl = peval_dd(cl, dl, t - h, &bl), fh = peval_dd(cl, dl, t + h, &bh);
                if (!(t - h > ilo && t + h < ihi)) return -1;
                if (!(fabs(fl) > safety * bl && fabs(fh) > safety * bh) || ((fl < 0.0) == (fh < 0.0))) return -1;
                r[nr] = t;
                rw[nr] = h;
                rd[nr] = 0.0;
                ++nr;
            }
        }
        for (int i = 0; i < nr; ++i) {
            crit[i] = r[i];
            crit_w[i] = rw[i];
            crit_d[i] = rd[i];
        }
        nc = nr;
    }
    for (int i = 0; i < nc; ++i) roots[i] = crit[i] * S;
    return nc;
}

// Solutions of one pairing (FP64 everywhere except the FP32 bracketing).
// Returns the number of solutions (ascending in x), or -1 when uncertain.
__device__ inline int dilep_pairing_mixed(const ConicD& q1, const ConicD& q2, const double* l1, const double* b1,
                                          const double* l2, const double* b2, double MX, double MY, float safety,
                                          SolD* sol)
{
    double A1 = q1.Ayy;
    double B1[2] = {q1.By, q1.Axy};
    double C1[3] = {q1.C0, q1.Bx, q1.Axx};
    double A2 = q2.Ayy;
    double B2[2] = {-q2.Axy * MX - 2.0 * q2.Ayy * MY - q2.By, q2.Axy};
    double C2[3];
    C2[0] = q2.Axx * MX * MX + q2.Axy * MX * MY + q2.Ayy * MY * MY + q2.Bx * MX + q2.By * MY + q2.C0;
    C2[1] = -2.0 * q2.Axx * MX - q2.Axy * MY - q2.Bx;
    C2[2] = q2.Axx;
    double Pd[3], Ld[2], T1[4], T2[4], M[4], PP[5], LM[5], R[5];
    for (int i = 0; i < 3; ++i) Pd[i] = A1 * C2[i] - A2 * C1[i];
    for (int i = 0; i < 2; ++i) Ld[i] = A1 * B2[i] - A2 * B1[i];
    pmul_d(B1, 1, C2, 2, T1);
    pmul_d(B2, 1, C1, 2, T2);
    for (int i = 0; i < 4; ++i) M[i] = T1[i] - T2[i];
    pmul_d(Pd, 2, Pd, 2, PP);
    pmul_d(Ld, 1, M, 3, LM);
    for (int i = 0; i < 5; ++i) R[i] = PP[i] - LM[i];
    double xs[4];
    const int nx = real_roots_mixed(R, safety, xs);
    if (nx < 0) return -1;
    double w1[4], w2[4];
    v4_add_d(b1, l1, w1);
    v4_add_d(b2, l2, w2);
    int ns = 0;
    for (int r = 0; r < nx; ++r) {
        const double x = xs[r];
        const double Pv = (Pd[2] * x + Pd[1]) * x + Pd[0];
        const double Lv = Ld[1] * x + Ld[0];
        if (!(fabs(Lv) > 1.0e-9 * (fabs(Ld[1] * x) + fabs(Ld[0])))) return -1;
        const double y = -Pv / Lv;
        double n1[4], n2[4];
        n1[0] = x;
        n1[1] = y;
        n1[2] = q1.z0 + q1.zx * x + q1.zy * y;
        n1[3] = q1.e0 + q1.ex * x + q1.ey * y;
        const double x2 = MX - x, y2 = MY - y;
        n2[0] = x2;
        n2[1] = y2;
        n2[2] = q2.z0 + q2.zx * x2 + q2.zy * y2;
        n2[3] = q2.e0 + q2.ex * x2 + q2.ey * y2;
        const double s1 = fabs(q1.e0) + fabs(q1.ex * x) + fabs(q1.ey * y);
        const double s2 = fabs(q2.e0) + fabs(q2.ex * x2) + fabs(q2.ey * y2);
        if (!(fabs(n1[3]) > 1.0e-8 * s1) || !(fabs(n2[3]) > 1.0e-8 * s2)) return -1;
        if (!(n1[3] > 0.0) || !(n2[3] > 0.0)) continue;
        double t1[4], t2[4], tt[4];
        v4_add_d(w1, n1, t1);
        v4_add_d(w2, n2, t2);
        v4_add_d(t1, t2, tt);
        sol[ns].mtt = mass_d(tt);
        sol[ns].mt1 = mass_d(t1);
        sol[ns].mt2 = mass_d(t2);
        ++ns;
    }
    return ns;
}

struct DilepRecoF {
    bool unsure, ok, h_ok;
    int pb1, pb2;
    double mtt, mt1, mt2, mbb;
    unsigned pairings;
};

// Best solution over the ordered b-jet pairings and the Higgs pair, with
// certainty of both argmins.  jd: FP64 smeared jets (b-tagged ones set).
__device__ inline DilepRecoF dilep_reco_mixed(const Plan& P, int n, unsigned btag, const double (*jd)[4],
                                              const double* l1, const double* l2, double MX, double MY)
{
    DilepRecoF r;
    r.unsure = false;
    r.ok = r.h_ok = false;
    r.pb1 = r.pb2 = -1;
    r.mtt = r.mt1 = r.mt2 = r.mbb = 0.0;
    r.pairings = 0;
    const float sf = P.safety;
    const unsigned bm = btag & ((1u << n) - 1u);
    ConicD qa[MAX_JETS], qb[MAX_JETS];
    unsigned okA = 0, okB = 0;
    for (int i = 0; i < n; ++i) {
        if (!(bm >> i & 1u)) continue;
        if (conic_d(l1, jd[i], P.dmW, P.dmt, qa[i])) okA |= 1u << i;
        if (conic_d(l2, jd[i], P.dmW, P.dmt, qb[i])) okB |= 1u << i;
    }
    double second = CUDART_INF;
    for (int b1 = 0; b1 < n; ++b1) {
        if (!(bm >> b1 & 1u)) continue;
        for (int b2 = 0; b2 < n; ++b2) {
            if (b2 == b1 || !(bm >> b2 & 1u)) continue;
            ++r.pairings;
            if (!(okA >> b1 & 1u) || !(okB >> b2 & 1u)) continue;  // no conic: no solution
            SolD sol[4];
            const int ns = dilep_pairing_mixed(qa[b1], qb[b2], l1, jd[b1], l2, jd[b2], MX, MY, sf, sol);
            if (ns < 0) {
                r.unsure = true;
                return r;
            }
            for (int s = 0; s < ns; ++s) {
                if (!r.ok || sol[s].mtt < r.mtt) {
                    if (r.ok) second = r.mtt;
                    r.ok = true;
                    r.pb1 = b1;
                    r.pb2 = b2;
                    r.mtt = sol[s].mtt;
                    r.mt1 = sol[s].mt1;
                    r.mt2 = sol[s].mt2;
                } else if (sol[s].mtt < second) {
                    second = sol[s].mtt;
                }
            }
        }
    }
    if (!r.ok) return r;
    if (second - r.mtt <= 1.0e-8 * r.mtt) {  // the argmin must be the definition's
        r.unsure = true;
        return r;
    }
    const unsigned rm = bm & ~(1u << r.pb1) & ~(1u << r.pb2);
    double hb = CUDART_INF, h2 = CUDART_INF;
    for (int i = 0; i < n; ++i) {
        if (!(rm >> i & 1u)) continue;
        for (int j = i + 1; j < n; ++j) {
            if (!(rm >> j & 1u)) continue;
            double h[4];
            v4_add_d(jd[i], jd[j], h);
            const double m = mass_d(h);
            const double d = fabs(m - P.dmH);
            if (d < hb) {
                h2 = hb;
                hb = d;
                r.h_ok = true;
                r.mbb = m;
            } else if (d < h2) {
                h2 = d;
            }
        }
    }
    if (r.h_ok && h2 - hb <= 1.0e-9 * (fabs(r.mbb) + 1.0)) r.unsure = true;
    return r;
}

// Evaluation of one dilepton unit (same protocol as the semileptonic one:
// f = leading cuts passed in user order, -1 = FP64 recheck).
__device__ inline UnitOut dilep_unit_f(const Plan& P, const int* exec, int nexec, const float4* jets, int n,
                                       unsigned btag, float4 lf1, float4 lf2, float2 metf, unsigned s1bits,
                                       uint64_t event_id, uint32_t v, uint64_t seed)
{
    UnitOut out;
    out.f = -1;
    out.reco = make_float4(0.f, 0.f, 0.f, 0.f);
    out.bin = 0;
    out.score = 0.0f;
    out.evald = out.passd = out.cyc_top = out.cyc_met = out.cands = 0;
    const unsigned bm = btag & ((1u << n) - 1u);
    const bool smear = P.smear_jets || P.smear_met || P.smear_lep;
    double z[16];
    unsigned zdone = 0;
    auto pair = [&](int k) {  // FP64 smearing normals z[2k], z[2k+1]
        if (zdone >> k & 1u) return;
        zdone |= 1u << k;
        uint4 w = philox4x32_10(ctr_of((uint32_t)(k / 2), v, event_id), key_of(seed));
        uint32_t w0 = (k & 1) ? w.z : w.x, w1 = (k & 1) ? w.w : w.y;
        box_muller_d(w0, w1, z[2 * k], z[2 * k + 1]);
    };
    double jd[MAX_JETS][4];
    for (int i = 0; i < n; ++i) {
        if (!(bm >> i & 1u)) continue;
        float4 p = jets[i];
        double c[4] = {p.x, p.y, p.z, p.w};
        if (smear) {
            pair(i / 2);
            double s = 1.0 + P.dsigma_jet * z[i];
            for (int k = 0; k < 4; ++k) jd[i][k] = s * c[k];
        } else {
            for (int k = 0; k < 4; ++k) jd[i][k] = c[k];
        }
    }
    double mxd = metf.x, myd = metf.y;
    if (smear) {
        pair(6);
        mxd = (double)metf.x + P.dsigma_met * z[12];
        myd = (double)metf.y + P.dsigma_met * z[13];
    }
    double l1[4] = {lf1.x, lf1.y, lf1.z, lf1.w};
    double l2[4] = {lf2.x, lf2.y, lf2.z, lf2.w};
    if (P.smear_lep) {  // lepton l scaled by 1 + sigma_lep z[14 + l]
        pair(7);
        const double s1 = 1.0 + P.dsigma_lep * z[14], s2 = 1.0 + P.dsigma_lep * z[15];
        for (int k = 0; k < 4; ++k) {
            l1[k] = s1 * l1[k];
            l2[k] = s2 * l2[k];
        }
    }
    DilepRecoF reco;
    bool reco_done = false;
    unsigned evald = 0, passd = 0;
    const unsigned s1fail = P.stage1 & ~s1bits;
    bool phase1 = true;
    int x = 0;
    int f = P.n_cuts;
    while (true) {
        int c;
        unsigned fails = s1fail | (evald & ~passd);
        int kf = fails ? __ffs(fails) - 1 : P.n_cuts;
        if (phase1) {
            if (x >= nexec) {
                phase1 = false;
                continue;
            }
            c = exec[x++];
            if (c > kf) continue;
        } else {
            unsigned below = kf >= 32 ? 0xffffffffu : ((1u << kf) - 1u);
            unsigned todo = P.stage2 & ~evald & below;
            if (!todo) {
                f = kf;
                break;
            }
            c = __ffs(todo) - 1;
        }
        const long long t0 = clock64();
        bool pass = false, unsure = false;
        const int kind = P.kind[c];
        if (kind == CUT_MET_MIN) {
            const double met = sqrt(mxd * mxd + myd * myd);
            pass = met > P.dp0[c];
            unsure = fabs(met - P.dp0[c]) <= 1.0e-9 * P.dp0[c];
        } else if (kind == CUT_LEP_PT_MIN) {
            const double pt = sqrt(l1[0] * l1[0] + l1[1] * l1[1]);
            pass = pt > P.dp0[c];
            unsure = fabs(pt - P.dp0[c]) <= 1.0e-9 * P.dp0[c];
        } else if (kind == CUT_W_NU_SOLVABLE) {
            double pz;
            pass = w_pz_d(l1, mxd, myd, P.dmW, &pz) != 0;  // the definition's FP64 arithmetic
        } else {
            if (!reco_done) {
                reco = dilep_reco_mixed(P, n, btag, jd, l1, l2, mxd, myd);
                reco_done = true;
                out.cands += reco.pairings;
            }
            if (reco.unsure) {
                unsure = true;
            } else if (kind == CUT_DILEP_SOLVABLE) {
                pass = reco.ok;
            } else if (kind == CUT_HIGGS_WINDOW) {
                pass = reco.h_ok && reco.mbb > P.dp0[c] && reco.mbb < P.dp1[c];
                if (reco.h_ok) {
                    const double b = 1.0e-9 * (fabs(reco.mbb) + 1.0);
                    unsure = fabs(reco.mbb - P.dp0[c]) <= b || fabs(reco.mbb - P.dp1[c]) <= b;
                }
            }
        }
        const unsigned dt = (unsigned)(clock64() - t0);
        if (heavy_cut(kind)) out.cyc_top += dt;
        else out.cyc_met += dt;
        evald |= 1u << c;
        if (pass) passd |= 1u << c;
        out.evald = evald;
        out.passd = passd;
        if (unsure) return out;
        if (!pass) phase1 = false;
    }
    if (f == P.n_cuts) {
        if (!reco_done || reco.unsure || !reco.ok || !reco.h_ok) return out;
        const int bin = hist_bin_d(P, reco.mbb);
        const double wd = (P.dhi - P.dlo) / P.nbins;
        const double rel = (reco.mbb - P.dlo) / wd;
        if (fabs(rel - rint(rel)) * wd <= 1.0e-9 * (fabs(reco.mbb) + 1.0)) return out;  // at an edge
        out.bin = bin;
        out.reco = make_float4((float)reco.mbb, (float)reco.mt1, (float)reco.mt2, (float)reco.mtt);
        out.score = (float)reco.mtt;
    }
    out.f = f;
    return out;
}

}  // namespace hf
