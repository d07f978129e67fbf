// hf_fp64.cuh -- FP64 evaluation of one unit on the GPU (the recheck path).
//
// Units whose FP32 evaluation lands within an error band of a decision are
// evaluated again here, in double precision, with the definition's
// formulation and operation order (compiled with -fmad=false: every + - * /
// is one IEEE rounding in the order written; division and sqrt are
// correctly rounded).  The results therefore coincide with any FP64
// implementation of the same formulation, apart from the transcendental
// functions of the Box-Muller transform (log, sin, cos), whose CUDA and host
// implementations may differ in the last bit.
//
// Definitions (HEP-Frame, arXiv:2211.14346): W-mass neutrino p_z with MET as
// the neutrino pT (Sect. 6.2); hadronic-top chi-square, Eq. 1 (Sect. 6.2);
// two-neutrino solution from the W- and top-mass constraints and the Higgs
// b-jet pair (Sect. 4); smearing pseudo-experiments (Sect. 4).
#pragma once
#include "hf_dev.cuh"
#include <math_constants.h>

namespace hf {

struct EvD {
    int n;
    double jet[MAX_JETS][4];  // smeared jets (px, py, pz, E)
    unsigned btag;
    double lep[2][4];
    int q[2];
    double metx, mety;        // smeared MET
};

__device__ __forceinline__ void v4_add_d(const double* a, const double* b, double* o)
{
    o[0] = a[0] + b[0];
    o[1] = a[1] + b[1];
    o[2] = a[2] + b[2];
    o[3] = a[3] + b[3];
}
__device__ __forceinline__ double m2_d(const double* a)
{
    return a[3] * a[3] - (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
}
__device__ __forceinline__ double mass_d(const double* a)
{
    double m2 = m2_d(a);
    return m2 >= 0.0 ? sqrt(m2) : -sqrt(-m2);
}

// ln and the sine / cosine of 2 pi u for the FP64 smearing normals, as the
// definition fixes them: one sequence of IEEE double operations (+, -, *, /;
// every file is compiled with -fmad=false, so none is fused), so that the
// normals are the same bits on every machine that runs it; within about an
// ulp of the exact functions (math libraries differ from one another in the
// last place, enough to move a unit that sits at a near-double root of the
// dilepton quartic).
//
// ln x: x = f 2^e, f in [sqrt(1/2), sqrt(2)) (frexp is exact); ln f =
// 2 atanh(s), s = (f - 1) / (f + 1), |s| <= 0.1716, by the odd series to
// s^23 / 23 (Horner in s^2); plus e ln 2, ln 2 as a 32-bit head (e times it
// exact) and its remainder.
__device__ __forceinline__ double bm_log_d(double x)
{
    const double ln2_hi = 0.6931471806019545, ln2_lo = -4.2009150726810846e-11;
    int e;
    double f = frexp(x, &e);
    if (f < 0.70710678118654752) {
        f = f * 2.0;
        e = e - 1;
    }
    const double s = (f - 1.0) / (f + 1.0);
    const double s2 = s * s;
    double p = 1.0 / 23.0;
    p = 1.0 / 21.0 + s2 * p;
    p = 1.0 / 19.0 + s2 * p;
    p = 1.0 / 17.0 + s2 * p;
    p = 1.0 / 15.0 + s2 * p;
    p = 1.0 / 13.0 + s2 * p;
    p = 1.0 / 11.0 + s2 * p;
    p = 1.0 / 9.0 + s2 * p;
    p = 1.0 / 7.0 + s2 * p;
    p = 1.0 / 5.0 + s2 * p;
    p = 1.0 / 3.0 + s2 * p;
    const double lf = 2.0 * s + (2.0 * s) * (s2 * p);
    return (double)e * ln2_hi + ((double)e * ln2_lo + lf);
}

// sin and cos of 2 pi u, u in [0, 1] a multiple of 2^-24: q = round(4u),
// r = u - q/4 (exact, |r| <= 1/8), x = 2 pi r (2 pi as a 28-bit head, exact
// against r, plus its remainder), |x| <= pi/4; Taylor series of sin to x^19
// and of cos to x^18 in Horner form; quadrant from q.
__device__ __forceinline__ void bm_sincos2pi_d(double u, double& sn, double& cs)
{
    const double two_pi_hi = 6.283185303211212, two_pi_lo = 3.968374318722162e-09;
    const double q = floor(4.0 * u + 0.5);
    const double r = u - 0.25 * q;
    const double x = r * two_pi_hi + r * two_pi_lo;
    const double x2 = x * x;
    double ps = -1.0 / 121645100408832000.0;
    ps = 1.0 / 355687428096000.0 + x2 * ps;
    ps = -1.0 / 1307674368000.0 + x2 * ps;
    ps = 1.0 / 6227020800.0 + x2 * ps;
    ps = -1.0 / 39916800.0 + x2 * ps;
    ps = 1.0 / 362880.0 + x2 * ps;
    ps = -1.0 / 5040.0 + x2 * ps;
    ps = 1.0 / 120.0 + x2 * ps;
    ps = -1.0 / 6.0 + x2 * ps;
    const double s0 = x + x * (x2 * ps);
    double pc = -1.0 / 6402373705728000.0;
    pc = 1.0 / 20922789888000.0 + x2 * pc;
    pc = -1.0 / 87178291200.0 + x2 * pc;
    pc = 1.0 / 479001600.0 + x2 * pc;
    pc = -1.0 / 3628800.0 + x2 * pc;
    pc = 1.0 / 40320.0 + x2 * pc;
    pc = -1.0 / 720.0 + x2 * pc;
    pc = 1.0 / 24.0 + x2 * pc;
    const double c0 = (1.0 - 0.5 * x2) + (x2 * x2) * pc;
    const int quad = (int)q & 3;
    sn = quad == 0 ? s0 : quad == 1 ? c0 : quad == 2 ? -s0 : -c0;
    cs = quad == 0 ? c0 : quad == 1 ? -s0 : quad == 2 ? -c0 : s0;
}

// One FP64 Box-Muller pair from two Philox words: z0 = r cos(2 pi u1),
// z1 = r sin(2 pi u1), r = sqrt(-2 ln u0).
__device__ __forceinline__ void box_muller_d(uint32_t w0, uint32_t w1, double& z0, double& z1)
{
    const double u0 = u01d(w0), u1 = u01d(w1);
    const double r = sqrt(-2.0 * bm_log_d(u0));
    double sn, cs;
    bm_sincos2pi_d(u1, sn, cs);
    z0 = r * cs;
    z1 = r * sn;
}

// Smearing normals of one unit in FP64: Philox words (b, v, e_lo, e_hi),
// Box-Muller pairs z[2k] = r cos(2 pi u1), z[2k+1] = r sin(2 pi u1).
__device__ inline void unit_normals_d(uint64_t seed, uint64_t event, uint32_t v, double z[16])
{
    uint2 key = key_of(seed);
    for (uint32_t b = 0; b < 4; ++b) {
        uint4 w = philox4x32_10(ctr_of(b, v, event), key);
        box_muller_d(w.x, w.y, z[4 * b], z[4 * b + 1]);
        box_muller_d(w.z, w.w, z[4 * b + 2], z[4 * b + 3]);
    }
}

// Loads event e and applies the smearing of variation v.
__device__ inline void load_event_d(const Plan& P, const Cols& C, uint32_t e, uint64_t event_id,
                                    uint64_t seed, uint32_t v, EvD& ev)
{
    uint32_t j0 = C.jet_off[e];
    ev.n = (int)(C.jet_off[e + 1] - j0);
    ev.btag = C.btag[e];
    int L = P.model == MODEL_DILEP ? 2 : 1;
    for (int l = 0; l < L; ++l) {
        float4 lf = C.lep[(uint64_t)e * L + l];
        ev.lep[l][0] = lf.x;
        ev.lep[l][1] = lf.y;
        ev.lep[l][2] = lf.z;
        ev.lep[l][3] = lf.w;
        ev.q[l] = C.lep_q[(uint64_t)e * L + l];
    }
    float2 mf = C.met[e];
    double z[16];
    bool smear = P.dsigma_jet != 0.0 || P.dsigma_met != 0.0;
    if (smear) unit_normals_d(seed, event_id, v, z);
    for (int i = 0; i < ev.n; ++i) {
        float4 jf = C.jets[j0 + i];
        double s = smear ? 1.0 + P.dsigma_jet * z[i] : 1.0;
        double js[4] = {jf.x, jf.y, jf.z, jf.w};
        for (int c = 0; c < 4; ++c) ev.jet[i][c] = smear ? s * js[c] : js[c];
    }
    ev.metx = smear ? (double)mf.x + P.dsigma_met * z[12] : (double)mf.x;
    ev.mety = smear ? (double)mf.y + P.dsigma_met * z[13] : (double)mf.y;
}

// W-mass neutrino p_z (massless lepton and neutrino):
//   mu = mW^2/2 + pT(l).pT(nu), a = E_l^2 - pz_l^2, D = mu^2 - a pT(nu)^2;
// smaller-|p_z| root without cancellation, or the real part mu pz_l / a when
// D < 0; solvable iff a > 0 and the result is finite.
__device__ inline int w_pz_d(const double* lep, double metx, double mety, double mW, double* pz_out)
{
    double lx = lep[0], ly = lep[1], lz = lep[2], lE = lep[3];
    double mu = mW * mW / 2.0 + (lx * metx + ly * mety);
    double a = lE * lE - lz * lz;
    double pt2 = metx * metx + mety * mety;
    double D = mu * mu - a * pt2;
    double pz;
    if (!(a > 0.0)) {
        *pz_out = 0.0;
        return 0;
    }
    if (D < 0.0) {
        pz = mu * lz / a;
    } else {
        double t = mu * lz;
        double sq = lE * sqrt(D);
        double q = t >= 0.0 ? t + sq : t - sq;
        pz = q == 0.0 ? 0.0 : (lE * lE * pt2 - mu * mu) / q;
    }
    *pz_out = pz;
    return isfinite(pz) ? 1 : 0;
}

// Both neutrino solutions of the W-mass constraint (the definition): D >= 0
// the smaller-|p_z| root first, then q / a (one solution 0 when q = 0);
// D < 0 the single real part mu pz_l / a; none when a <= 0 or not finite.
__device__ inline int w_pz_both_d(const double* lep, double metx, double mety, double mW, double pz[2])
{
    double lx = lep[0], ly = lep[1], lz = lep[2], lE = lep[3];
    double mu = mW * mW / 2.0 + (lx * metx + ly * mety);
    double a = lE * lE - lz * lz;
    double pt2 = metx * metx + mety * mety;
    double D = mu * mu - a * pt2;
    if (!(a > 0.0)) return 0;
    if (D < 0.0) {
        pz[0] = mu * lz / a;
        return isfinite(pz[0]) ? 1 : 0;
    }
    double t = mu * lz;
    double sq = lE * sqrt(D);
    double q = t >= 0.0 ? t + sq : t - sq;
    if (q == 0.0) {
        pz[0] = 0.0;
        return 1;
    }
    pz[0] = (lE * lE * pt2 - mu * mu) / q;
    pz[1] = q / a;
    return isfinite(pz[0]) && isfinite(pz[1]) ? 2 : 0;
}

// Hadronic-top triplet chi-square, Eq. 1: enumeration k, then i < j, k not in
// {i, j}; strict minimum, ties to the first; n < 3 -> +inf.
__device__ inline double hadtop_d(const EvD& ev, const Plan& P, double* mtop, double* mw)
{
    double best = CUDART_INF;
    *mtop = 0.0;
    *mw = 0.0;
    for (int k = 0; k < ev.n; ++k)
        for (int i = 0; i < ev.n; ++i) {
            if (i == k) continue;
            for (int j = i + 1; j < ev.n; ++j) {
                if (j == k) continue;
                double W[4], T[4];
                v4_add_d(ev.jet[i], ev.jet[j], W);
                v4_add_d(W, ev.jet[k], T);
                double m_w = mass_d(W);
                double m_t = mass_d(T);
                double dt = (m_t - P.dmt) / P.dsigma_t;
                double dw = (m_w - P.dmW) / P.dsigma_W;
                double chi2 = dt * dt + dw * dw;
                if (chi2 < best) {
                    best = chi2;
                    *mtop = m_t;
                    *mw = m_w;
                }
            }
        }
    return best;
}

// FP64 quantities of one unit, computed on demand: the smearing normals of a
// Box-Muller pair, a smeared jet, the smeared MET (the definition's
// arithmetic, so that they equal those of any FP64 evaluation).
struct LazyUnitD {
    const Plan* P;
    const Cols* C;
    uint64_t event_id, seed;
    uint32_t v, j0;
    int n;
    bool smear;
    unsigned zdone, jdone;
    bool metdone;
    double z[16];
    double jet[MAX_JETS][4];
    double metx, mety;

    const float4* jp;  // the event's jets (FP32 columns)

    __device__ void init(const Plan& P_, const Cols& C_, uint32_t e, uint64_t eid, uint64_t seed_, uint32_t v_)
    {
        P = &P_;
        C = &C_;
        event_id = eid;
        seed = seed_;
        v = v_;
        j0 = C_.jet_off[e];
        n = (int)(C_.jet_off[e + 1] - j0);
        jp = C_.jets + j0;
        smear = P_.dsigma_jet != 0.0 || P_.dsigma_met != 0.0 || P_.dsigma_lep != 0.0;
        zdone = jdone = 0;
        metdone = false;
    }
    // Same from the event's jet row (no column set at hand).
    __device__ void init_jets(const Plan& P_, const float4* jets, int n_, uint64_t eid, uint64_t seed_, uint32_t v_)
    {
        P = &P_;
        C = nullptr;
        event_id = eid;
        seed = seed_;
        v = v_;
        j0 = 0;
        n = n_;
        jp = jets;
        smear = P_.dsigma_jet != 0.0 || P_.dsigma_met != 0.0 || P_.dsigma_lep != 0.0;
        zdone = jdone = 0;
        metdone = false;
    }
    __device__ void pair(int k)  // normals z[2k], z[2k+1]
    {
        if (zdone >> k & 1u) return;
        zdone |= 1u << k;
        uint4 w = philox4x32_10(ctr_of((uint32_t)(k / 2), v, event_id), key_of(seed));
        uint32_t w0 = (k & 1) ? w.z : w.x, w1 = (k & 1) ? w.w : w.y;
        box_muller_d(w0, w1, z[2 * k], z[2 * k + 1]);
    }
    __device__ const double* j(int i)
    {
        if (!(jdone >> i & 1u)) {
            jdone |= 1u << i;
            float4 jf = jp[i];
            double js[4] = {jf.x, jf.y, jf.z, jf.w};
            if (smear) {
                pair(i / 2);
                double s = 1.0 + P->dsigma_jet * z[i];
                for (int c = 0; c < 4; ++c) jet[i][c] = s * js[c];
            } else {
                for (int c = 0; c < 4; ++c) jet[i][c] = js[c];
            }
        }
        return jet[i];
    }
    // Lepton l of the unit: scaled by 1 + sigma_lep z[14 + l] (exactly 1 when
    // sigma_lep = 0, as in the definition).
    __device__ void lepton(int l, float4 lf, double* out)
    {
        const double c[4] = {lf.x, lf.y, lf.z, lf.w};
        if (smear && P->dsigma_lep != 0.0) {  // (the scale is exactly 1 without lepton smearing)
            pair(7);
            const double s = 1.0 + P->dsigma_lep * z[14 + l];
            for (int k = 0; k < 4; ++k) out[k] = s * c[k];
        } else {
            for (int k = 0; k < 4; ++k) out[k] = c[k];
        }
    }
    __device__ void met(float2 mf)
    {
        if (metdone) return;
        metdone = true;
        if (smear) {
            pair(6);
            metx = (double)mf.x + P->dsigma_met * z[12];
            mety = (double)mf.y + P->dsigma_met * z[13];
        } else {
            metx = mf.x;
            mety = mf.y;
        }
    }
};

}  // namespace hf
