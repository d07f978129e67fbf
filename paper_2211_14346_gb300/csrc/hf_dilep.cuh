// hf_dilep.cuh -- dilepton ttH reconstruction on the GPU: the two-neutrino
// solution over b-jet pairings and the Higgs b-jet pair (device code).
//
// Definition (HEP-Frame, arXiv:2211.14346, Sect. 4 and Sect. 6.2): the
// neutrinos of t -> b l nu and tbar -> bbar l nu are massless, each lepton
// with its neutrino reconstructs m_W = 80.4 GeV, adding the b-jet gives
// m_t = 172.5 GeV, and the neutrinos share the missing transverse momentum.
// All pairings of the b-tagged jets with the two leptons are tried; the
// best solution is kept (here: minimum m_ttbar) and an event without any
// solution fails.  The Higgs candidate is the pair of remaining b-jets
// closest to 125 GeV.
//
// Formulation (per pairing): with c = b + l, the constraints l.nu = alpha =
// (m_W^2 - m_l^2)/2 and c.nu = beta = (m_t^2 - m_c^2)/2 are linear in the
// neutrino (E, p); eliminating E gives w.p = k (w = E_l p_c - E_c p_l,
// k = E_c alpha - E_l beta), so p_z and E are linear in (p_x, p_y) and
// masslessness is a conic Q(p_x, p_y) = 0.  With nu_2 = MET - nu_1 in the
// transverse plane, the resultant in y of the two conics is a quartic R(x),
// x = p_x(nu_1); its real roots (isolated between the critical points,
// which come from the derivatives the same way, and bisected) give y, then
// both neutrinos; solutions with E <= 0 for either neutrino are dropped.
//
// This header holds the FP64 evaluation (every operation in the definition's
// order; the recheck of flagged units) and the FP32 building blocks with a
// running absolute error bound on every quantity (Ef), including the
// certified isolation of a quartic's real roots; hf_dilep_f.cuh combines
// them into the fast unit evaluation.
#pragma once
#include "hf_dev.cuh"
#include "hf_fp64.cuh"
#include "hf_semilep.cuh"
#include <math_constants.h>

namespace hf {

// ================================================================== FP64
__device__ __forceinline__ double poly_eval_d(const double* c, int d, double x)
{
    double r = c[d];
    for (int i = d - 1; i >= 0; --i) r = r * x + c[i];
    return r;
}

__device__ inline double bisect_d(const double* c, int d, double lo, double hi, bool neg_lo)
{
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double f = poly_eval_d(c, d, mid);
        if (f == 0.0) return mid;
        if ((f < 0.0) == neg_lo) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// Real roots (ascending) of a polynomial of degree <= 4 with + - * / only:
// the roots of the derivative split (-B, B), B the Cauchy bound, into
// monotone intervals; each strict sign change is bisected; a critical point
// where the value is exactly zero is a root.  Levels are processed from the
// lowest derivative up (the same values as a recursive formulation).
__device__ inline int real_roots_d(const double* c_in, int d_in, double* roots)
{
    double lev[4][5];  // lev[0] = the polynomial, lev[l] = its l-th derivative
    int deg[4];
    int d = d_in;
    for (int i = 0; i <= d; ++i) lev[0][i] = c_in[i];
    while (d > 0 && lev[0][d] == 0.0) --d;
    if (d <= 0) return 0;
    int L = 0;
    deg[0] = d;
    while (deg[L] > 1) {
        int dd = deg[L] - 1;
        for (int i = 0; i <= dd; ++i) lev[L + 1][i] = (double)(i + 1) * lev[L][i + 1];
        while (dd > 0 && lev[L + 1][dd] == 0.0) --dd;
        ++L;
        deg[L] = dd;
        if (dd <= 0) break;
    }
    double crit[4];
    int nc = 0;
    for (int l = L; l >= 0; --l) {
        const double* c = lev[l];
        const int dl = deg[l];
        double r[4];
        int nr = 0;
        if (dl <= 0) {
            nr = 0;
        } else if (dl == 1) {
            r[0] = -c[0] / c[1];
            nr = 1;
        } else {
            double B = 0.0;
            for (int i = 0; i < dl; ++i) {
                double q = fabs(c[i] / c[dl]);
                if (q > B) B = q;
            }
            B = 1.0 + B;
            double pts[6];
            int np = 0;
            pts[np++] = -B;
            for (int i = 0; i < nc; ++i)
                if (crit[i] > -B && crit[i] < B) pts[np++] = crit[i];
            pts[np++] = B;
            for (int i = 0; i + 1 < np; ++i) {
                double lo = pts[i], hi = pts[i + 1];
                double flo = poly_eval_d(c, dl, lo), fhi = poly_eval_d(c, dl, hi);
                if (i > 0 && flo == 0.0) r[nr++] = lo;
                if (flo != 0.0 && fhi != 0.0 && ((flo < 0.0) != (fhi < 0.0))) r[nr++] = bisect_d(c, dl, lo, hi, flo < 0.0);
            }
        }
        for (int i = 0; i < nr; ++i) crit[i] = r[i];
        nc = nr;
    }
    for (int i = 0; i < nc; ++i) roots[i] = crit[i];
    return nc;
}

struct ConicD {
    double z0, zx, zy, e0, ex, ey, Axx, Axy, Ayy, Bx, By, C0;
};

__device__ inline bool conic_d(const double* lep, const double* bjet, double mW, double mt, ConicD& q)
{
    double c[4];
    v4_add_d(bjet, lep, c);
    double alpha = (mW * mW - m2_d(lep)) / 2.0;
    double beta = (mt * mt - m2_d(c)) / 2.0;
    double lE = lep[3], cE = c[3];
    double wx = lE * c[0] - cE * lep[0];
    double wy = lE * c[1] - cE * lep[1];
    double wz = lE * c[2] - cE * lep[2];
    double k = cE * alpha - lE * beta;
    if (wz == 0.0 || lE == 0.0) return false;
    q.z0 = k / wz;
    q.zx = -wx / wz;
    q.zy = -wy / wz;
    q.e0 = (alpha + lep[2] * q.z0) / lE;
    q.ex = (lep[0] + lep[2] * q.zx) / lE;
    q.ey = (lep[1] + lep[2] * q.zy) / lE;
    q.Axx = q.ex * q.ex - 1.0 - q.zx * q.zx;
    q.Ayy = q.ey * q.ey - 1.0 - q.zy * q.zy;
    q.Axy = 2.0 * (q.ex * q.ey - q.zx * q.zy);
    q.Bx = 2.0 * (q.e0 * q.ex - q.z0 * q.zx);
    q.By = 2.0 * (q.e0 * q.ey - q.z0 * q.zy);
    q.C0 = q.e0 * q.e0 - q.z0 * q.z0;
    return true;
}

__device__ inline void pmul_d(const double* a, int da, const double* b, int db, double* o)
{
    for (int i = 0; i <= da + db; ++i) o[i] = 0.0;
    for (int i = 0; i <= da; ++i)
        for (int j = 0; j <= db; ++j) o[i + j] = o[i + j] + a[i] * b[j];
}

// Solutions of one pairing, ascending in x = px(nu_1): nu1, nu2 (px, py, pz, E).
__device__ inline int dilep_pairing_d(const double* l1, const double* b1, const double* l2, const double* b2,
                                      double metx, double mety, double mW, double mt, double (*nu1)[4],
                                      double (*nu2)[4])
{
    ConicD q1, q2;
    if (!conic_d(l1, b1, mW, mt, q1) || !conic_d(l2, b2, mW, mt, q2)) return 0;
    double A1 = q1.Ayy;
    double B1[2] = {q1.By, q1.Axy};
    double C1[3] = {q1.C0, q1.Bx, q1.Axx};
    double MX = metx, MY = mety;
    double A2 = q2.Ayy;
    double B2[2] = {-q2.Axy * MX - 2.0 * q2.Ayy * MY - q2.By, q2.Axy};
    double C2[3];
    C2[0] = q2.Axx * MX * MX + q2.Axy * MX * MY + q2.Ayy * MY * MY + q2.Bx * MX + q2.By * MY + q2.C0;
    C2[1] = -2.0 * q2.Axx * MX - q2.Axy * MY - q2.Bx;
    C2[2] = q2.Axx;
    double P[3], L[2], T1[4], T2[4], M[4], PP[5], LM[5], R[5];
    for (int i = 0; i < 3; ++i) P[i] = A1 * C2[i] - A2 * C1[i];
    for (int i = 0; i < 2; ++i) L[i] = A1 * B2[i] - A2 * B1[i];
    pmul_d(B1, 1, C2, 2, T1);
    pmul_d(B2, 1, C1, 2, T2);
    for (int i = 0; i < 4; ++i) M[i] = T1[i] - T2[i];
    pmul_d(P, 2, P, 2, PP);
    pmul_d(L, 1, M, 3, LM);
    for (int i = 0; i < 5; ++i) R[i] = PP[i] - LM[i];
    double xs[4];
    int nx = real_roots_d(R, 4, xs);
    int ns = 0;
    for (int r = 0; r < nx; ++r) {
        double x = xs[r];
        double Pv = (P[2] * x + P[1]) * x + P[0];
        double Lv = L[1] * x + L[0];
        if (Lv == 0.0) continue;
        double y = -Pv / Lv;
        double n1[4], n2[4];
        n1[0] = x;
        n1[1] = y;
        n1[2] = q1.z0 + q1.zx * x + q1.zy * y;
        n1[3] = q1.e0 + q1.ex * x + q1.ey * y;
        double x2 = MX - x, y2 = MY - y;
        n2[0] = x2;
        n2[1] = y2;
        n2[2] = q2.z0 + q2.zx * x2 + q2.zy * y2;
        n2[3] = q2.e0 + q2.ex * x2 + q2.ey * y2;
        if (!(n1[3] > 0.0) || !(n2[3] > 0.0)) continue;
        for (int c = 0; c < 4; ++c) {
            nu1[ns][c] = n1[c];
            nu2[ns][c] = n2[c];
        }
        ++ns;
    }
    return ns;
}

struct DilepResD {
    bool ok, h_ok;
    int pb1, pb2;
    double m_t1, m_t2, m_tt, m_bb;
};

// Best solution (minimum m_ttbar over ordered pairings of distinct b-tagged
// jets, b1 with lepton 1, in index order, solutions ascending in x, ties to
// the first) and the Higgs pair (minimum |m_bb - m_H| over remaining b-tagged
// jets i < j, ties to the first).  jet(i) gives the smeared jet i.
template <class JetFn>
__device__ inline DilepResD dilep_reco_d(const Plan& P, int n, unsigned btag, const double* l1, const double* l2,
                                         double metx, double mety, JetFn jet)
{
    DilepResD r;
    r.ok = r.h_ok = false;
    r.pb1 = r.pb2 = -1;
    r.m_t1 = r.m_t2 = r.m_tt = r.m_bb = 0.0;
    double best = CUDART_INF;
    unsigned bm = btag & ((1u << n) - 1u);
    double l12[4];
    v4_add_d(l1, l2, l12);
    for (int b1 = 0; b1 < n; ++b1) {
        if (!(bm >> b1 & 1u)) continue;
        for (int b2 = 0; b2 < n; ++b2) {
            if (b2 == b1 || !(bm >> b2 & 1u)) continue;
            double nu1[4][4], nu2[4][4];
            const double* j1 = jet(b1);
            const double* j2 = jet(b2);
            if (r.ok) {
                // every solution of the pairing has m_ttbar >= m_vis (its b-jets
                // and leptons; the neutrinos are future light-like): a pairing
                // whose m_vis is above the best by more than FP64 rounding can
                // neither win nor tie (ties go to the first in this order)
                double v[4], w[4];
                v4_add_d(j1, j2, v);
                v4_add_d(v, l12, w);
                if (mass_d(w) > best * (1.0 + 1.0e-12)) continue;
            }
            int ns = dilep_pairing_d(l1, j1, l2, j2, metx, mety, P.dmW, P.dmt, nu1, nu2);
            for (int s = 0; s < ns; ++s) {
                double t1[4], t2[4], w1[4], w2[4], tt[4];
                v4_add_d(j1, l1, w1);
                v4_add_d(w1, nu1[s], t1);
                v4_add_d(j2, l2, w2);
                v4_add_d(w2, nu2[s], t2);
                v4_add_d(t1, t2, tt);
                double mtt = mass_d(tt);
                if (mtt < best) {
                    best = mtt;
                    r.ok = true;
                    r.pb1 = b1;
                    r.pb2 = b2;
                    r.m_t1 = mass_d(t1);
                    r.m_t2 = mass_d(t2);
                    r.m_tt = mtt;
                }
            }
        }
    }
    if (!r.ok) return r;
    unsigned rm = bm & ~(1u << r.pb1) & ~(1u << r.pb2);
    double bh = CUDART_INF;
    for (int i = 0; i < n; ++i) {
        if (!(rm >> i & 1u)) continue;
        for (int j = i + 1; j < n; ++j) {
            if (!(rm >> j & 1u)) continue;
            double h[4];
            v4_add_d(jet(i), jet(j), h);
            double m = mass_d(h);
            double dd = fabs(m - P.dmH);
            if (dd < bh) {
                bh = dd;
                r.h_ok = true;
                r.m_bb = m;
            }
        }
    }
    return r;
}

// ================================================================== FP32 with error bounds
// A value and an absolute bound on its distance to the value the FP64
// definition computes (first- and second-order terms of every operation plus
// the rounding of the result).
struct Ef {
    float v, e;
};
constexpr float EF_U = 5.9604645e-8f;  // 2^-24
__device__ __forceinline__ Ef efc(float v) { return Ef{v, 0.0f}; }
__device__ __forceinline__ Ef operator+(Ef a, Ef b)
{
    float r = __fadd_rn(a.v, b.v);
    return Ef{r, a.e + b.e + EF_U * fabsf(r)};
}
__device__ __forceinline__ Ef operator-(Ef a, Ef b)
{
    float r = __fsub_rn(a.v, b.v);
    return Ef{r, a.e + b.e + EF_U * fabsf(r)};
}
__device__ __forceinline__ Ef operator-(Ef a) { return Ef{-a.v, a.e}; }
__device__ __forceinline__ Ef operator*(Ef a, Ef b)
{
    float r = __fmul_rn(a.v, b.v);
    return Ef{r, fabsf(a.v) * b.e + fabsf(b.v) * a.e + a.e * b.e + EF_U * fabsf(r)};
}
__device__ __forceinline__ Ef operator*(float s, Ef a)  // exact power-of-two or small integer scale
{
    float r = __fmul_rn(s, a.v);
    return Ef{r, fabsf(s) * a.e + EF_U * fabsf(r)};
}
// a / b; *bad is set when |b| is not certainly away from zero
__device__ __forceinline__ Ef ef_div(Ef a, Ef b, bool* bad)
{
    float den = fabsf(b.v) - b.e;
    if (!(den > 0.0f)) {
        *bad = true;
        return Ef{0.0f, CUDART_INF_F};
    }
    float r = __fdiv_rn(a.v, b.v);
    return Ef{r, (a.e + fabsf(r) * b.e) / den + EF_U * fabsf(r)};
}
__device__ __forceinline__ Ef ef_m2(const Ef* a)
{
    return a[3] * a[3] - ((a[0] * a[0] + a[1] * a[1]) + a[2] * a[2]);
}
// mass of a timelike sum: sqrt(m^2) with the definition's sign convention
__device__ __forceinline__ Ef ef_mass(const Ef* a, bool* bad)
{
    Ef m2 = ef_m2(a);
    if (!(m2.v > m2.e)) {
        *bad = true;
        return Ef{0.0f, CUDART_INF_F};
    }
    float r = sqrtf(m2.v);
    float lo = sqrtf(fmaxf(m2.v - m2.e, 0.0f));
    return Ef{r, m2.e / (r + lo) + EF_U * r};
}
__device__ __forceinline__ void ef_add4(const Ef* a, const Ef* b, Ef* o)
{
    o[0] = a[0] + b[0];
    o[1] = a[1] + b[1];
    o[2] = a[2] + b[2];
    o[3] = a[3] + b[3];
}

struct ConicF {
    Ef z0, zx, zy, e0, ex, ey, Axx, Axy, Ayy, Bx, By, C0;
};

__device__ inline bool conic_f(const Ef* lep, const Ef* bjet, const Ef& mW2h, const Ef& mt2h, ConicF& q)
{
    bool bad = false;
    Ef c[4];
    ef_add4(bjet, lep, c);
    Ef alpha = mW2h - 0.5f * ef_m2(lep);
    Ef beta = mt2h - 0.5f * ef_m2(c);
    Ef lE = lep[3], cE = c[3];
    Ef wx = lE * c[0] - cE * lep[0];
    Ef wy = lE * c[1] - cE * lep[1];
    Ef wz = lE * c[2] - cE * lep[2];
    Ef k = cE * alpha - lE * beta;
    q.z0 = ef_div(k, wz, &bad);
    q.zx = ef_div(-wx, wz, &bad);
    q.zy = ef_div(-wy, wz, &bad);
    q.e0 = ef_div(alpha + lep[2] * q.z0, lE, &bad);
    q.ex = ef_div(lep[0] + lep[2] * q.zx, lE, &bad);
    q.ey = ef_div(lep[1] + lep[2] * q.zy, lE, &bad);
    const Ef one = efc(1.0f);
    q.Axx = (q.ex * q.ex - one) - q.zx * q.zx;
    q.Ayy = (q.ey * q.ey - one) - q.zy * q.zy;
    q.Axy = 2.0f * (q.ex * q.ey - q.zx * q.zy);
    q.Bx = 2.0f * (q.e0 * q.ex - q.z0 * q.zx);
    q.By = 2.0f * (q.e0 * q.ey - q.z0 * q.zy);
    q.C0 = q.e0 * q.e0 - q.z0 * q.z0;
    return !bad;
}

__device__ __forceinline__ void pmul_f(const Ef* a, int da, const Ef* b, int db, Ef* o)
{
    for (int i = 0; i <= da + db; ++i) o[i] = efc(0.0f);
    for (int i = 0; i <= da; ++i)
        for (int j = 0; j <= db; ++j) o[i + j] = o[i + j] + a[i] * b[j];
}

// Value and error bound of a polynomial with uncertain coefficients at an
// uncertain point: Horner in FP32, bound = sum e_i |x|^i + rounding
// (2 d u sum |c_i||x|^i) + |p'| dx.
__device__ __forceinline__ float peval_f(const float* c, int d, float x)
{
    float r = c[d];
    for (int i = d - 1; i >= 0; --i) r = fmaf(r, x, c[i]);
    return r;
}
__device__ __forceinline__ float pbound_f(const float* c, const float* e, int d, float x)
{
    float ax = fabsf(x), s = 0.0f, m = 0.0f, pw = 1.0f;
    for (int i = 0; i <= d; ++i) {
        s = fmaf(e[i], pw, s);
        m = fmaf(fabsf(c[i]), pw, m);
        pw *= ax;
    }
    return s + 2.0f * (float)d * EF_U * m;
}

// Real roots of the quartic R with certainty of the root structure.  Roots
// come with an error bound dx.  Returns -1 when a sign at a critical point
// or the leading coefficient is uncertain (unit goes to the FP64 recheck).
__device__ inline int real_roots_f(const Ef* R, float safety, float* xs, float* dxs)
{
    float lev[4][5], err[4][5];
    int deg[4];
    int d = 4;
    for (int i = 0; i <= 4; ++i) {
        lev[0][i] = R[i].v;
        err[0][i] = R[i].e;
    }
    // the definition trims exact zeros only: a leading term that is not
    // certainly non-zero is undecidable here
    while (d > 0 && fabsf(lev[0][d]) <= safety * err[0][d]) {
        if (lev[0][d] != 0.0f || err[0][d] != 0.0f) return -1;
        --d;
    }
    if (d <= 0) return 0;
    int L = 0;
    deg[0] = d;
    while (deg[L] > 1) {
        int dd = deg[L] - 1;
        for (int i = 0; i <= dd; ++i) {
            lev[L + 1][i] = (float)(i + 1) * lev[L][i + 1];
            err[L + 1][i] = (float)(i + 1) * err[L][i + 1] + EF_U * fabsf(lev[L + 1][i]);
        }
        ++L;
        deg[L] = dd;
    }
    float crit[4];
    int nc = 0;
    for (int l = L; l >= 0; --l) {
        const float* c = lev[l];
        const float* e = err[l];
        const int dl = deg[l];
        float r[4], dr[4];
        int nr = 0;
        if (dl == 1) {
            if (!(fabsf(c[1]) > safety * e[1])) return -1;
            r[0] = -c[0] / c[1];
            dr[0] = (e[0] + fabsf(r[0]) * e[1]) / (fabsf(c[1]) - e[1]) + EF_U * fabsf(r[0]);
            nr = 1;
        } else {
            float B = 0.0f;
            for (int i = 0; i < dl; ++i) B = fmaxf(B, fabsf(c[i] / c[dl]));
            B = (1.0f + B) * 1.0001f;
            float pts[6];
            int np = 0;
            pts[np++] = -B;
            for (int i = 0; i < nc; ++i) {
                // the sign of this level at its critical points must be certain
                float v = peval_f(c, dl, crit[i]);
                if (!(fabsf(v) > safety * pbound_f(c, e, dl, crit[i]))) return -1;
                if (crit[i] > -B && crit[i] < B) pts[np++] = crit[i];
            }
            pts[np++] = B;
            for (int i = 0; i + 1 < np; ++i) {
                float lo = pts[i], hi = pts[i + 1];
                float flo = peval_f(c, dl, lo), fhi = peval_f(c, dl, hi);
                if ((flo < 0.0f) == (fhi < 0.0f)) continue;
                const bool neg = flo < 0.0f;
                for (int it = 0; it < 64; ++it) {
                    float mid = 0.5f * (lo + hi);
                    if (!(mid > lo && mid < hi)) break;
                    if ((peval_f(c, dl, mid) < 0.0f) == neg) lo = mid;
                    else hi = mid;
                }
                float x = 0.5f * (lo + hi);
                // derivative at the root: certainly non-zero, gives the root's error
                float dv = 0.0f, db = 0.0f, pw = 1.0f, apw = 1.0f;
                for (int k = 1; k <= dl; ++k) {
                    dv += (float)k * c[k] * pw;
                    db += (float)k * (e[k] + 2.0f * (float)dl * EF_U * fabsf(c[k])) * apw;
                    pw *= x;
                    apw *= fabsf(x);
                }
                db += 1e-30f;
                if (!(fabsf(dv) > safety * db)) return -1;
                r[nr] = x;
                dr[nr] = (hi - lo) + safety * pbound_f(c, e, dl, x) / (fabsf(dv) - db);
                ++nr;
            }
        }
        for (int i = 0; i < nr; ++i) {
            crit[i] = r[i];
            if (l == 0) {
                xs[i] = r[i];
                dxs[i] = dr[i];
            }
        }
        nc = nr;
    }
    return nc;
}

}  // namespace hf
