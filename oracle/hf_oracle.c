/*
 * hf_oracle.c -- FP64 reference ("oracle") for the per-event cut chain and
 * kinematic reconstruction of HEP-Frame's event analysis.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the test-suite, the smoke check and the CPU
 * baseline of the benchmark do.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * Plain, slow, single-threaded C99 in double precision.  Inputs are the FP32
 * structure-of-arrays columns, upcast exactly.  Build with
 * -ffp-contract=off so that every + - * / is a single IEEE-754 rounding in
 * exactly the order written here.
 *
 * What it computes (paper passages, HEP-Frame, arXiv:2211.14346):
 *   - the ordered cut chain, an event (here: a unit = event x smearing
 *     variation) stops at the first failing cut; an event passing all cuts
 *     is selected (Sect. 3, the pipeline of propositions; Sect. 6.1 cut
 *     example);
 *   - semileptonic reconstruction: neutrino p_z from the W-mass constraint
 *     with the missing transverse momentum as the neutrino p_T (Sect. 6.2),
 *     the hadronic-top jet-triplet chi-square (Eq. 1, hadronic terms) and
 *     the full chi-square of Eq. 1 with both tops and both W bosons;
 *   - dilepton ttH reconstruction: two neutrinos from the W-mass (80.4) and
 *     top-mass (172.5) constraints with MET split between them, over all
 *     b-jet/lepton pairings, the best solution kept, the event rejected when
 *     no solution exists; the Higgs candidate from the two remaining b-jets
 *     closest to 125 GeV (Sect. 4);
 *   - detector-resolution smearing, N pseudo-experiments per event (Sect. 4),
 *     drawn from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 *     numbers: as easy as 1, 2, 3", SC'11) keyed by (seed, event, variation);
 *   - integer histogram of the reconstructed mass (Appendix, user histograms)
 *     and the per-cut event counts (cut flow).
 *
 * Readings where the paper is silent are listed in the design notes; the
 * ones that shape arithmetic are repeated at the function that applies them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Analysis description (the oracle's own layout; marshalled by the     */
/* Python test harness from the same user-level description that the    */
/* C-ABI receives).                                                     */
/* ------------------------------------------------------------------ */
enum {
    ORC_SEMILEP = 1,
    ORC_DILEP = 2
};
enum {
    ORC_NJETS_MIN = 1,       /* n_jets >= p0                                   */
    ORC_NBTAG_MIN = 2,       /* number of b-tagged jets >= p0                  */
    ORC_LEP_PT_MIN = 3,      /* pT(lepton 1) > p0                              */
    ORC_MET_MIN = 4,         /* |MET| > p0 (smeared MET)                        */
    ORC_WNU_SOLVABLE = 5,    /* W-mass neutrino p_z exists (Sect. 6.2)          */
    ORC_HADTOP_CHI2_MAX = 6, /* best triplet chi2 < p0 (Eq. 1, hadronic part)  */
    ORC_LEP_OS = 7,          /* q1 * q2 < 0                                    */
    ORC_DILEP_SOLVABLE = 8,  /* >= 1 two-neutrino solution (Sect. 4)          */
    ORC_HIGGS_WINDOW = 9,    /* p0 < m_bb < p1 (Sect. 4, m_H = 125)           */
    ORC_TTBAR_CHI2_MAX = 10  /* best full Eq. 1 chi2 < p0 (Sect. 6.2)          */
};

#define ORC_MAX_CUTS 16
#define ORC_MAX_JETS 12

typedef struct {
    int32_t model;
    int32_t n_cuts;
    int32_t kind[ORC_MAX_CUTS];
    double param[ORC_MAX_CUTS][2];
    double mW, mt, sigma_t, sigma_W, mH;
    double sigma_jet, sigma_met;
    int32_t hist_nbins;
    double hist_lo, hist_hi;
    double sigma_lep; /* relative lepton-energy resolution (0: leptons unsmeared) */
} orc_analysis;

/* One event, upcast to double. */
typedef struct {
    int n;
    double jet[ORC_MAX_JETS][4]; /* px py pz E */
    unsigned btag;
    double lep[2][4];
    int q[2];
    double met[2];
} orc_event;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).                               */
/* Round: two 32x32->64 multiplications of counter words 0 and 2 by the */
/* round multipliers, outputs permuted and xored with the key; the key  */
/* is advanced by the Weyl increments between rounds.                   */
/* ------------------------------------------------------------------ */
static const uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
static const uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PH_W0;
            k1 += PH_W1;
        }
        uint64_t p0 = (uint64_t)PH_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PH_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 32-bit word -> uniform in [2^-24, 1 - 2^-24]: the top 23 bits, centred.
 * Exactly representable in FP32 and FP64, never 0 or 1. */
double orc_u01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* ln and sin / cos of the smearing normals.  Math libraries round these
 * functions differently in the last place, and a decision that sits at the
 * rounding level of a normal (a near-double root of the dilepton quartic)
 * would then depend on the library.  The definition therefore fixes how they
 * are evaluated: a fixed sequence of IEEE double operations (+, -, *, /, with
 * no fused multiply-add), within about an ulp of the exact functions.
 *
 * ln x: x = f 2^e with f in [sqrt(1/2), sqrt(2)) (frexp, exact), ln f =
 * 2 atanh(s) = 2 (s + s^3/3 + ... + s^23/23) with s = (f - 1) / (f + 1),
 * |s| <= 0.1716 (the next term is below 2^-56 relative), and e ln 2 with ln 2
 * split into a head of 32 significant bits (e times it is exact) and the
 * rest. */
static const double ORC_LN2_HI = 0.6931471806019545;      /* ln 2 rounded to 32 bits */
static const double ORC_LN2_LO = -4.2009150726810846e-11; /* ln 2 - ORC_LN2_HI       */

double orc_bm_log(double x)
{
    int e;
    double f = frexp(x, &e); /* x = f 2^e, f in [1/2, 1) */
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
    return (double)e * ORC_LN2_HI + ((double)e * ORC_LN2_LO + lf);
}

/* sin and cos of 2 pi u for u in [0, 1], u a multiple of 2^-24 (the uniforms
 * here): q = nearest integer to 4u and r = u - q/4 (both exact, |r| <= 1/8),
 * x = 2 pi r with 2 pi split into a head of 28 significant bits (r times it
 * is exact) and the rest, |x| <= pi/4; Taylor series of sin to x^19 and of
 * cos to x^18 (the next terms are below 1e-20); then the quadrant q. */
static const double ORC_2PI_HI = 6.283185303211212;     /* 2 pi rounded to 28 bits */
static const double ORC_2PI_LO = 3.968374318722162e-09; /* 2 pi - ORC_2PI_HI       */

void orc_bm_sincos2pi(double u, double* sn, double* cs)
{
    const double q = floor(4.0 * u + 0.5);
    const double r = u - 0.25 * q;
    const double x = r * ORC_2PI_HI + r * ORC_2PI_LO;
    const double x2 = x * x;
    double ps = -1.0 / 121645100408832000.0;   /* -1/19! */
    ps = 1.0 / 355687428096000.0 + x2 * ps;    /*  1/17! */
    ps = -1.0 / 1307674368000.0 + x2 * ps;     /* -1/15! */
    ps = 1.0 / 6227020800.0 + x2 * ps;         /*  1/13! */
    ps = -1.0 / 39916800.0 + x2 * ps;          /* -1/11! */
    ps = 1.0 / 362880.0 + x2 * ps;             /*  1/9!  */
    ps = -1.0 / 5040.0 + x2 * ps;              /* -1/7!  */
    ps = 1.0 / 120.0 + x2 * ps;                /*  1/5!  */
    ps = -1.0 / 6.0 + x2 * ps;                 /* -1/3!  */
    const double s0 = x + x * (x2 * ps);
    double pc = -1.0 / 6402373705728000.0;     /* -1/18! */
    pc = 1.0 / 20922789888000.0 + x2 * pc;     /*  1/16! */
    pc = -1.0 / 87178291200.0 + x2 * pc;       /* -1/14! */
    pc = 1.0 / 479001600.0 + x2 * pc;          /*  1/12! */
    pc = -1.0 / 3628800.0 + x2 * pc;           /* -1/10! */
    pc = 1.0 / 40320.0 + x2 * pc;              /*  1/8!  */
    pc = -1.0 / 720.0 + x2 * pc;               /* -1/6!  */
    pc = 1.0 / 24.0 + x2 * pc;                 /*  1/4!  */
    const double c0 = (1.0 - 0.5 * x2) + (x2 * x2) * pc;
    switch ((int)q & 3) {
    case 0: *sn = s0; *cs = c0; break;
    case 1: *sn = c0; *cs = -s0; break;
    case 2: *sn = -s0; *cs = -c0; break;
    default: *sn = -c0; *cs = s0; break;
    }
}

/* The 16 standard normals of unit (seed, event, variation).
 * Counter of block b (0..3) = (b, v, event_lo32, event_hi32), key = (seed_lo32,
 * seed_hi32).  Words 2k and 2k+1 of the 16 form one Box-Muller pair:
 *   z[2k] = sqrt(-2 ln u0) cos(2 pi u1),  z[2k+1] = sqrt(-2 ln u0) sin(2 pi u1),
 * ln, cos and sin evaluated as above.
 * z[0..11] scale jets 0..11, z[12], z[13] shift MET x, y; z[14], z[15] scale leptons
 * 0 and 1 when the analysis smears leptons. */
void orc_unit_normals(uint64_t seed, uint64_t event, uint32_t v, double z[16])
{
    uint32_t w[16];
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t b = 0; b < 4; ++b) {
        uint32_t ctr[4] = {b, v, (uint32_t)event, (uint32_t)(event >> 32)};
        orc_philox4x32_10(ctr, key, &w[4 * b]);
    }
    for (int k = 0; k < 8; ++k) {
        double u0 = orc_u01(w[2 * k]);
        double u1 = orc_u01(w[2 * k + 1]);
        double r = sqrt(-2.0 * orc_bm_log(u0));
        double sn, cs;
        orc_bm_sincos2pi(u1, &sn, &cs);
        z[2 * k] = r * cs;
        z[2 * k + 1] = r * sn;
    }
}

/* ------------------------------------------------------------------ */
/* Four-vectors (px, py, pz, E).                                       */
/* ------------------------------------------------------------------ */
static void v4_add(const double* a, const double* b, double* o)
{
    o[0] = a[0] + b[0];
    o[1] = a[1] + b[1];
    o[2] = a[2] + b[2];
    o[3] = a[3] + b[3];
}

double orc_m2(const double* a)
{
    return a[3] * a[3] - (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
}

/* Invariant mass with the signed convention of a Lorentz vector class:
 * m = sqrt(m^2) if m^2 >= 0, else -sqrt(-m^2). */
double orc_mass(const double* a)
{
    double m2 = orc_m2(a);
    return m2 >= 0.0 ? sqrt(m2) : -sqrt(-m2);
}

double orc_pt(const double* a)
{
    return sqrt(a[0] * a[0] + a[1] * a[1]);
}

/* ------------------------------------------------------------------ */
/* Semileptonic: neutrino p_z from the W-mass constraint (Sect. 6.2).  */
/* Massless lepton and neutrino; MET is the neutrino pT.                */
/*   mu = mW^2/2 + pT(l).pT(nu),  a = E_l^2 - pz_l^2,                   */
/*   D  = mu^2 - a pT(nu)^2,  roots (mu pz_l +- E_l sqrt(D)) / a.        */
/* The root of smaller |p_z| is taken (computed without cancellation);  */
/* when D < 0 the real part mu pz_l / a is taken.  Solvable iff a > 0   */
/* and the result is finite.                                            */
/* ------------------------------------------------------------------ */
int orc_w_pz(const double* lep, double metx, double mety, double mW,
             double* pz_out, int* dneg_out)
{
    double lx = lep[0], ly = lep[1], lz = lep[2], lE = lep[3];
    double mu = mW * mW / 2.0 + (lx * metx + ly * mety);
    double a = lE * lE - lz * lz;
    double pt2 = metx * metx + mety * mety;
    double D = mu * mu - a * pt2;
    double pz;
    int dneg = 0;
    if (!(a > 0.0)) {
        *pz_out = 0.0;
        *dneg_out = D < 0.0;
        return 0;
    }
    if (D < 0.0) {
        dneg = 1;
        pz = mu * lz / a;
    } else {
        double t = mu * lz;
        double sq = lE * sqrt(D);
        double q = t >= 0.0 ? t + sq : t - sq;
        if (q == 0.0)
            pz = 0.0;
        else
            pz = (lE * lE * pt2 - mu * mu) / q;
    }
    *pz_out = pz;
    *dneg_out = dneg;
    return isfinite(pz) ? 1 : 0;
}

/* Both neutrino solutions of the W-mass constraint (same mu, a, D as    */
/* orc_w_pz).  D >= 0: the two roots (mu pz_l +- E_l sqrt(D)) / a, the  */
/* smaller-|p_z| one first, both computed without cancellation from     */
/* q = mu pz_l + sgn(mu pz_l) E_l sqrt(D): q / a and (E_l^2 pT^2 - mu^2)/q */
/* (a single solution 0 when q = 0).  D < 0: the single real part        */
/* mu pz_l / a.  a <= 0 or a non-finite value: no solution.  Returns the */
/* number of solutions (0, 1 or 2).                                     */
int orc_w_pz_both(const double* lep, double metx, double mety, double mW, double pz[2])
{
    double lx = lep[0], ly = lep[1], lz = lep[2], lE = lep[3];
    double mu = mW * mW / 2.0 + (lx * metx + ly * mety);
    double a = lE * lE - lz * lz;
    double pt2 = metx * metx + mety * mety;
    double D = mu * mu - a * pt2;
    if (!(a > 0.0))
        return 0;
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

/* ------------------------------------------------------------------ */
/* Semileptonic: hadronic-top triplet chi-square (Eq. 1, hadronic term).*/
/* Candidates (k, {i<j}) with k not in {i, j}: jets i, j form the W,    */
/* jet k the b.  chi2 = ((m_ijk - mt)/sigma_t)^2 + ((m_ij - mW)/sigma_W)^2.*/
/* Enumeration: k ascending, then i ascending, then j ascending; the     */
/* best candidate is the strict minimum, ties go to the first.  Fewer    */
/* than three jets -> chi2 = +inf.                                       */
/* ------------------------------------------------------------------ */
double orc_hadtop(int n, const double (*jet)[4], double mW, double mt,
                  double sigma_W, double sigma_t, int* bk, int* bi, int* bj,
                  double* mtop, double* mw)
{
    double best = INFINITY;
    *bk = *bi = *bj = -1;
    *mtop = 0.0;
    *mw = 0.0;
    for (int k = 0; k < n; ++k) {
        for (int i = 0; i < n; ++i) {
            if (i == k)
                continue;
            for (int j = i + 1; j < n; ++j) {
                if (j == k)
                    continue;
                double W[4], T[4];
                v4_add(jet[i], jet[j], W);
                v4_add(W, jet[k], T);
                double m_w = orc_mass(W);
                double m_t = orc_mass(T);
                double dt = (m_t - mt) / sigma_t;
                double dw = (m_w - mW) / sigma_W;
                double chi2 = dt * dt + dw * dw;
                if (chi2 < best) {
                    best = chi2;
                    *bk = k;
                    *bi = i;
                    *bj = j;
                    *mtop = m_t;
                    *mw = m_w;
                }
            }
        }
    }
    return best;
}

/* ------------------------------------------------------------------ */
/* Semileptonic: the full chi-square of Eq. 1 (Sect. 6.2) for ttbar ->  */
/* (b q q')(b l nu): two top quarks and two W bosons,                   */
/*   chi2 = ((m_kij - mt)/sigma_t)^2 + ((m_ij - mW)/sigma_W)^2           */
/*        + ((m_l,lep,nu - mt)/sigma_t)^2 + ((m_lep,nu - mW)/sigma_W)^2,  */
/* minimised over the hadronic b-jet k, the W jets i < j, the leptonic   */
/* b-jet l (all distinct) and the neutrino solution r (orc_w_pz_both:    */
/* the neutrino is (MET_x, MET_y, p_z, |p|), massless).  Enumeration: k, */
/* then i < j as for the hadronic term, then l ascending, then r in the  */
/* order orc_w_pz_both returns; strict minimum, ties to the first.  Fewer*/
/* than four jets or no neutrino solution -> chi2 = +inf.  Outputs the   */
/* hadronic and leptonic top masses and the chosen p_z.                  */
/* ------------------------------------------------------------------ */
double orc_ttbar(int n, const double (*jet)[4], const double* lep, double metx, double mety,
                 double mW, double mt, double sigma_W, double sigma_t, int idx[5],
                 double* mtop_had, double* mtop_lep, double* pz_out)
{
    double best = INFINITY;
    double pz[2];
    int nr = orc_w_pz_both(lep, metx, mety, mW, pz);
    for (int c = 0; c < 5; ++c)
        idx[c] = -1;
    *mtop_had = *mtop_lep = *pz_out = 0.0;
    if (n < 4 || nr == 0)
        return best;
    double W_lep[2][4], mw_lep[2];
    for (int r = 0; r < nr; ++r) {
        double nu[4] = {metx, mety, pz[r], sqrt(metx * metx + mety * mety + pz[r] * pz[r])};
        v4_add(lep, nu, W_lep[r]);
        mw_lep[r] = orc_mass(W_lep[r]);
    }
    for (int k = 0; k < n; ++k) {
        for (int i = 0; i < n; ++i) {
            if (i == k)
                continue;
            for (int j = i + 1; j < n; ++j) {
                if (j == k)
                    continue;
                double W[4], T[4];
                v4_add(jet[i], jet[j], W);
                v4_add(W, jet[k], T);
                double dt = (orc_mass(T) - mt) / sigma_t;
                double dw = (orc_mass(W) - mW) / sigma_W;
                double had = dt * dt + dw * dw;
                for (int l = 0; l < n; ++l) {
                    if (l == k || l == i || l == j)
                        continue;
                    for (int r = 0; r < nr; ++r) {
                        double TL[4];
                        v4_add(jet[l], W_lep[r], TL);
                        double m_tl = orc_mass(TL);
                        double dtl = (m_tl - mt) / sigma_t;
                        double dwl = (mw_lep[r] - mW) / sigma_W;
                        double chi2 = had + (dtl * dtl + dwl * dwl);
                        if (chi2 < best) {
                            best = chi2;
                            idx[0] = k;
                            idx[1] = i;
                            idx[2] = j;
                            idx[3] = l;
                            idx[4] = r;
                            *mtop_had = orc_mass(T);
                            *mtop_lep = m_tl;
                            *pz_out = pz[r];
                        }
                    }
                }
            }
        }
    }
    return best;
}

/* ------------------------------------------------------------------ */
/* Real roots of a polynomial of degree <= 4 using only + - * / and     */
/* comparisons: the critical points (roots of the derivative, found    */
/* the same way) split (-B, B), B the Cauchy bound, into monotone       */
/* intervals; a strict sign change on an interval is bisected to full  */
/* precision (at most 200 halvings).  A critical point where the value  */
/* is exactly zero is a (multiple) root.  Roots ascending.             */
/* c[0..d] low to high.                                                  */
/* ------------------------------------------------------------------ */
static double poly_eval(const double* c, int d, double x)
{
    double r = c[d];
    for (int i = d - 1; i >= 0; --i)
        r = r * x + c[i];
    return r;
}

static double bisect(const double* c, int d, double lo, double hi, int neg_lo)
{
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi))
            break;
        double f = poly_eval(c, d, mid);
        if (f == 0.0)
            return mid;
        if ((f < 0.0) == neg_lo)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

int orc_real_roots(const double* c_in, int d, double* roots)
{
    double c[5];
    for (int i = 0; i <= d; ++i)
        c[i] = c_in[i];
    while (d > 0 && c[d] == 0.0)
        --d;
    if (d <= 0)
        return 0;
    if (d == 1) {
        roots[0] = -c[0] / c[1];
        return 1;
    }
    double dc[4];
    for (int i = 0; i < d; ++i)
        dc[i] = (double)(i + 1) * c[i + 1];
    double crit[4];
    int nc = orc_real_roots(dc, d - 1, crit);
    double B = 0.0;
    for (int i = 0; i < d; ++i) {
        double r = fabs(c[i] / c[d]);
        if (r > B)
            B = r;
    }
    B = 1.0 + B;
    double pts[6];
    int np = 0;
    pts[np++] = -B;
    for (int i = 0; i < nc; ++i)
        if (crit[i] > -B && crit[i] < B)
            pts[np++] = crit[i];
    pts[np++] = B;
    int nr = 0;
    for (int i = 0; i + 1 < np; ++i) {
        double lo = pts[i], hi = pts[i + 1];
        double flo = poly_eval(c, d, lo), fhi = poly_eval(c, d, hi);
        if (i > 0 && flo == 0.0)
            roots[nr++] = lo; /* root exactly at a critical point */
        if (flo != 0.0 && fhi != 0.0 && ((flo < 0.0) != (fhi < 0.0)))
            roots[nr++] = bisect(c, d, lo, hi, flo < 0.0);
    }
    return nr;
}

/* ------------------------------------------------------------------ */
/* Dilepton: two-neutrino solution for one pairing (Sect. 4, Sect. 6.2).*/
/* Constraints, massless neutrinos nu_a (a = 1, 2):                       */
/*   (l_a + nu_a)^2 = mW^2,  (b_a + l_a + nu_a)^2 = mt^2,                 */
/*   pT(nu_1) + pT(nu_2) = MET.                                           */
/* With c_a = b_a + l_a: l.nu = alpha = (mW^2 - m_l^2)/2 and              */
/* c.nu = beta = (mt^2 - m_c^2)/2 are linear in (E, p) of nu; eliminating */
/* E gives w.p = k with w = E_l p_c - E_c p_l, k = E_c alpha - E_l beta,   */
/* so p_z and E are linear in (px, py) and masslessness is a conic         */
/* Q_a(px, py) = 0.  Substituting nu_2 = MET - nu_1 (transverse), the      */
/* resultant in y of the two conics is a quartic R(x) in x = px(nu_1);     */
/* each real root gives y, then both neutrinos.  Solutions with E <= 0     */
/* for either neutrino are dropped.                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    double z0, zx, zy; /* pz = z0 + zx x + zy y */
    double e0, ex, ey; /* E  = e0 + ex x + ey y */
    double Axx, Axy, Ayy, Bx, By, C0; /* Q = E^2 - px^2 - py^2 - pz^2 */
} orc_conic;

static int conic_of(const double* lep, const double* bjet, double mW, double mt,
                    orc_conic* q)
{
    double c[4];
    v4_add(bjet, lep, c);
    double alpha = (mW * mW - orc_m2(lep)) / 2.0;
    double beta = (mt * mt - orc_m2(c)) / 2.0;
    double lE = lep[3], cE = c[3];
    double wx = lE * c[0] - cE * lep[0];
    double wy = lE * c[1] - cE * lep[1];
    double wz = lE * c[2] - cE * lep[2];
    double k = cE * alpha - lE * beta;
    if (wz == 0.0 || lE == 0.0)
        return 0;
    q->z0 = k / wz;
    q->zx = -wx / wz;
    q->zy = -wy / wz;
    q->e0 = (alpha + lep[2] * q->z0) / lE;
    q->ex = (lep[0] + lep[2] * q->zx) / lE;
    q->ey = (lep[1] + lep[2] * q->zy) / lE;
    q->Axx = q->ex * q->ex - 1.0 - q->zx * q->zx;
    q->Ayy = q->ey * q->ey - 1.0 - q->zy * q->zy;
    q->Axy = 2.0 * (q->ex * q->ey - q->zx * q->zy);
    q->Bx = 2.0 * (q->e0 * q->ex - q->z0 * q->zx);
    q->By = 2.0 * (q->e0 * q->ey - q->z0 * q->zy);
    q->C0 = q->e0 * q->e0 - q->z0 * q->z0;
    return 1;
}

/* Polynomials in x, coefficient arrays low to high. */
static void pmul(const double* a, int da, const double* b, int db, double* o)
{
    for (int i = 0; i <= da + db; ++i)
        o[i] = 0.0;
    for (int i = 0; i <= da; ++i)
        for (int j = 0; j <= db; ++j)
            o[i + j] = o[i + j] + a[i] * b[j];
}

typedef struct {
    double nu1[4], nu2[4];
    double x;
} orc_nusol;

/* Up to 4 solutions, ascending in x = px(nu_1). Returns the count. */
int orc_dilep_pairing(const double* l1, const double* b1, const double* l2,
                      const double* b2, double metx, double mety, double mW,
                      double mt, orc_nusol* sol, double* quartic_out)
{
    orc_conic q1, q2;
    if (!conic_of(l1, b1, mW, mt, &q1) || !conic_of(l2, b2, mW, mt, &q2))
        return 0;
    /* Q1 as A1 y^2 + B1(x) y + C1(x). */
    double A1 = q1.Ayy;
    double B1[2] = {q1.By, q1.Axy};
    double C1[3] = {q1.C0, q1.Bx, q1.Axx};
    /* Q2 at (MX - x, MY - y) as A2 y^2 + B2(x) y + C2(x). */
    double MX = metx, MY = mety;
    double A2 = q2.Ayy;
    double B2[2] = {-q2.Axy * MX - 2.0 * q2.Ayy * MY - q2.By, q2.Axy};
    double C2[3];
    C2[0] = q2.Axx * MX * MX + q2.Axy * MX * MY + q2.Ayy * MY * MY + q2.Bx * MX +
            q2.By * MY + q2.C0;
    C2[1] = -2.0 * q2.Axx * MX - q2.Axy * MY - q2.Bx;
    C2[2] = q2.Axx;
    /* R = (A1 C2 - A2 C1)^2 - (A1 B2 - A2 B1)(B1 C2 - B2 C1). */
    double P[3], L[2], T1[4], T2[4], M[4], PP[5], LM[5], R[5];
    for (int i = 0; i < 3; ++i)
        P[i] = A1 * C2[i] - A2 * C1[i];
    for (int i = 0; i < 2; ++i)
        L[i] = A1 * B2[i] - A2 * B1[i];
    pmul(B1, 1, C2, 2, T1);
    pmul(B2, 1, C1, 2, T2);
    for (int i = 0; i < 4; ++i)
        M[i] = T1[i] - T2[i];
    pmul(P, 2, P, 2, PP);
    pmul(L, 1, M, 3, LM);
    for (int i = 0; i < 5; ++i)
        R[i] = PP[i] - LM[i];
    if (quartic_out)
        for (int i = 0; i < 5; ++i)
            quartic_out[i] = R[i];
    double xs[4];
    int nx = orc_real_roots(R, 4, xs);
    int ns = 0;
    for (int r = 0; r < nx; ++r) {
        double x = xs[r];
        double Pv = (P[2] * x + P[1]) * x + P[0];
        double Lv = L[1] * x + L[0];
        if (Lv == 0.0)
            continue;
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
        if (!(n1[3] > 0.0) || !(n2[3] > 0.0))
            continue;
        memcpy(sol[ns].nu1, n1, sizeof n1);
        memcpy(sol[ns].nu2, n2, sizeof n2);
        sol[ns].x = x;
        ++ns;
    }
    return ns;
}

/* ------------------------------------------------------------------ */
/* Unit evaluation.                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
    double jet[ORC_MAX_JETS][4]; /* smeared jets */
    double lep[2][4];            /* smeared leptons */
    double metx, mety;           /* smeared MET */
    /* semileptonic */
    int w_done, w_ok, dneg;
    double pz;
    int t_done, k, i, j;
    double chi2, mtop, mw;
    int f_done, fidx[5];
    double fchi2, fmtop_had, fmtop_lep, fpz;
    /* dilepton */
    int d_done, d_ok, pb1, pb2;
    double m_t1, m_t2, m_tt;
    int h_done, h_ok, h1, h2;
    double m_bb;
} orc_unit_state;

static void unit_init(const orc_analysis* an, const orc_event* ev, uint64_t seed,
                      uint64_t event_id, uint32_t v, orc_unit_state* st)
{
    memset(st, 0, sizeof *st);
    if (an->sigma_jet != 0.0 || an->sigma_met != 0.0 || an->sigma_lep != 0.0) {
        double z[16];
        orc_unit_normals(seed, event_id, v, z);
        for (int i = 0; i < ev->n; ++i) {
            double s = 1.0 + an->sigma_jet * z[i];
            for (int c = 0; c < 4; ++c)
                st->jet[i][c] = s * ev->jet[i][c];
        }
        /* lepton l scaled by 1 + sigma_lep z[14 + l] (exactly 1 when sigma_lep = 0) */
        for (int l = 0; l < 2; ++l) {
            double s = 1.0 + an->sigma_lep * z[14 + l];
            for (int c = 0; c < 4; ++c)
                st->lep[l][c] = s * ev->lep[l][c];
        }
        st->metx = ev->met[0] + an->sigma_met * z[12];
        st->mety = ev->met[1] + an->sigma_met * z[13];
    } else {
        /* sigma = 0: s_i = 1 and the MET shift is 0 exactly, so the
         * unsmeared event is the same as drawing and applying them. */
        for (int i = 0; i < ev->n; ++i)
            for (int c = 0; c < 4; ++c)
                st->jet[i][c] = ev->jet[i][c];
        for (int l = 0; l < 2; ++l)
            for (int c = 0; c < 4; ++c)
                st->lep[l][c] = ev->lep[l][c];
        st->metx = ev->met[0];
        st->mety = ev->met[1];
    }
}

static void need_w(const orc_analysis* an, const orc_event* ev, orc_unit_state* st)
{
    if (st->w_done)
        return;
    st->w_done = 1;
    st->w_ok = orc_w_pz(st->lep[0], st->metx, st->mety, an->mW, &st->pz, &st->dneg);
}

static void need_top(const orc_analysis* an, const orc_event* ev, orc_unit_state* st)
{
    if (st->t_done)
        return;
    st->t_done = 1;
    st->chi2 = orc_hadtop(ev->n, (const double(*)[4])st->jet, an->mW, an->mt,
                          an->sigma_W, an->sigma_t, &st->k, &st->i, &st->j,
                          &st->mtop, &st->mw);
}

static void need_full(const orc_analysis* an, const orc_event* ev, orc_unit_state* st)
{
    if (st->f_done)
        return;
    st->f_done = 1;
    st->fchi2 = orc_ttbar(ev->n, (const double(*)[4])st->jet, st->lep[0], st->metx, st->mety, an->mW,
                          an->mt, an->sigma_W, an->sigma_t, st->fidx, &st->fmtop_had, &st->fmtop_lep,
                          &st->fpz);
}

/* Best two-neutrino solution over ordered b-jet pairings (b1 with lepton 1,
 * b2 with lepton 2), b1 and b2 distinct b-tagged jets in index order, the
 * solutions of one pairing ascending in px(nu_1); best = minimum m_ttbar,
 * ties to the first. */
static void need_dilep(const orc_analysis* an, const orc_event* ev, orc_unit_state* st)
{
    if (st->d_done)
        return;
    st->d_done = 1;
    st->d_ok = 0;
    double best = INFINITY;
    unsigned bm = ev->btag & ((1u << ev->n) - 1u);
    for (int b1 = 0; b1 < ev->n; ++b1) {
        if (!(bm >> b1 & 1u))
            continue;
        for (int b2 = 0; b2 < ev->n; ++b2) {
            if (b2 == b1 || !(bm >> b2 & 1u))
                continue;
            orc_nusol sol[4];
            int ns = orc_dilep_pairing(st->lep[0], st->jet[b1], st->lep[1], st->jet[b2],
                                       st->metx, st->mety, an->mW, an->mt, sol, NULL);
            for (int s = 0; s < ns; ++s) {
                double t1[4], t2[4], w1[4], w2[4], tt[4];
                v4_add(st->jet[b1], st->lep[0], w1);
                v4_add(w1, sol[s].nu1, t1);
                v4_add(st->jet[b2], st->lep[1], w2);
                v4_add(w2, sol[s].nu2, t2);
                v4_add(t1, t2, tt);
                double mtt = orc_mass(tt);
                if (mtt < best) {
                    best = mtt;
                    st->d_ok = 1;
                    st->pb1 = b1;
                    st->pb2 = b2;
                    st->m_t1 = orc_mass(t1);
                    st->m_t2 = orc_mass(t2);
                    st->m_tt = mtt;
                }
            }
        }
    }
}

/* Higgs candidate: among b-tagged jets outside the best pairing, the pair
 * i < j with minimum |m_bb - mH|, ties to the first. */
static void need_higgs(const orc_analysis* an, const orc_event* ev, orc_unit_state* st)
{
    if (st->h_done)
        return;
    st->h_done = 1;
    need_dilep(an, ev, st);
    st->h_ok = 0;
    if (!st->d_ok)
        return;
    unsigned bm = ev->btag & ((1u << ev->n) - 1u);
    bm &= ~(1u << st->pb1);
    bm &= ~(1u << st->pb2);
    double best = INFINITY;
    for (int i = 0; i < ev->n; ++i) {
        if (!(bm >> i & 1u))
            continue;
        for (int j = i + 1; j < ev->n; ++j) {
            if (!(bm >> j & 1u))
                continue;
            double h[4];
            v4_add(st->jet[i], st->jet[j], h);
            double m = orc_mass(h);
            double d = fabs(m - an->mH);
            if (d < best) {
                best = d;
                st->h_ok = 1;
                st->h1 = i;
                st->h2 = j;
                st->m_bb = m;
            }
        }
    }
}

static int popcount12(unsigned x)
{
    int c = 0;
    for (int i = 0; i < 16; ++i)
        c += (x >> i) & 1u;
    return c;
}

static int cut_pass(const orc_analysis* an, int c, const orc_event* ev, orc_unit_state* st)
{
    double p0 = an->param[c][0], p1 = an->param[c][1];
    switch (an->kind[c]) {
    case ORC_NJETS_MIN:
        return ev->n >= (int)p0;
    case ORC_NBTAG_MIN:
        return popcount12(ev->btag & ((1u << ev->n) - 1u)) >= (int)p0;
    case ORC_LEP_PT_MIN:
        return orc_pt(st->lep[0]) > p0;
    case ORC_MET_MIN:
        return sqrt(st->metx * st->metx + st->mety * st->mety) > p0;
    case ORC_WNU_SOLVABLE:
        need_w(an, ev, st);
        return st->w_ok;
    case ORC_HADTOP_CHI2_MAX:
        need_top(an, ev, st);
        return st->chi2 < p0;
    case ORC_LEP_OS:
        return ev->q[0] * ev->q[1] < 0;
    case ORC_DILEP_SOLVABLE:
        need_dilep(an, ev, st);
        return st->d_ok;
    case ORC_HIGGS_WINDOW:
        need_higgs(an, ev, st);
        return st->h_ok && st->m_bb > p0 && st->m_bb < p1;
    case ORC_TTBAR_CHI2_MAX:
        need_full(an, ev, st);
        return st->fchi2 < p0;
    default:
        return 0;
    }
}

/* Histogram bin of x: 0 = underflow (x < lo), nbins + 1 = overflow
 * (x >= hi or NaN), else 1 + the largest i with x >= lo + i * w,
 * w = (hi - lo) / nbins. */
int orc_hist_bin(double x, int nbins, double lo, double hi)
{
    if (x < lo)
        return 0;
    if (!(x < hi))
        return nbins + 1;
    double w = (hi - lo) / nbins;
    int i = (int)floor((x - lo) / w);
    if (i < 0)
        i = 0;
    if (i > nbins - 1)
        i = nbins - 1;
    while (i > 0 && x < lo + i * w)
        --i;
    while (i < nbins - 1 && x >= lo + (i + 1) * w)
        ++i;
    return 1 + i;
}

static void load_event(const orc_analysis* an, uint64_t e, const uint32_t* jet_off,
                       const float* jets, const uint16_t* btag, const float* lep,
                       const int8_t* lep_q, const float* met, orc_event* ev)
{
    int L = an->model == ORC_DILEP ? 2 : 1;
    uint32_t j0 = jet_off[e];
    memset(ev->lep, 0, sizeof ev->lep); /* the second lepton slot stays 0 for one-lepton events */
    ev->n = (int)(jet_off[e + 1] - j0);
    for (int i = 0; i < ev->n; ++i)
        for (int c = 0; c < 4; ++c)
            ev->jet[i][c] = (double)jets[4 * (uint64_t)(j0 + i) + c];
    ev->btag = btag[e];
    for (int l = 0; l < L; ++l) {
        for (int c = 0; c < 4; ++c)
            ev->lep[l][c] = (double)lep[4 * (e * L + l) + c];
        ev->q[l] = lep_q[e * L + l];
    }
    ev->met[0] = (double)met[2 * e];
    ev->met[1] = (double)met[2 * e + 1];
}

/* Per-unit result for tests: number of leading cuts passed (user order),
 * and the reconstructed quantities (valid when all cuts pass). */
typedef struct {
    int32_t passed;
    int32_t idx[4];   /* semilep: k, i, j, dneg; dilep: b1, b2, h1, h2 */
    double q[6];      /* semilep: mtop, mW, pz, MET', chi2, -; with the full fit: mtop_had, mtop_lep,
                         pz, MET', chi2, neutrino solution;  dilep: m_bb, m_t, m_tbar, m_tt, -, - */
} orc_unit_result;

static int eval_unit(const orc_analysis* an, const orc_event* ev, uint64_t seed,
                     uint64_t event_id, uint32_t v, orc_unit_result* res)
{
    orc_unit_state st;
    unit_init(an, ev, seed, event_id, v, &st);
    int passed = 0;
    for (int c = 0; c < an->n_cuts; ++c) {
        if (!cut_pass(an, c, ev, &st))
            break;
        ++passed;
    }
    if (res) {
        memset(res, 0, sizeof *res);
        res->passed = passed;
        int full = 0;
        for (int c = 0; c < an->n_cuts; ++c)
            full |= an->kind[c] == ORC_TTBAR_CHI2_MAX;
        if (an->model == ORC_SEMILEP && full) {
            /* with the full fit: (m_top hadronic, m_top leptonic, p_z of
             * the chosen neutrino, |MET'|), histogram of the hadronic top */
            need_full(an, ev, &st);
            for (int c = 0; c < 4; ++c)
                res->idx[c] = st.fidx[c];
            res->q[0] = st.fmtop_had;
            res->q[1] = st.fmtop_lep;
            res->q[2] = st.fpz;
            res->q[3] = sqrt(st.metx * st.metx + st.mety * st.mety);
            res->q[4] = st.fchi2;
            res->q[5] = st.fidx[4];
        } else if (an->model == ORC_SEMILEP) {
            need_w(an, ev, &st);
            need_top(an, ev, &st);
            res->idx[0] = st.k;
            res->idx[1] = st.i;
            res->idx[2] = st.j;
            res->idx[3] = st.dneg;
            res->q[0] = st.mtop;
            res->q[1] = st.mw;
            res->q[2] = st.pz;
            res->q[3] = sqrt(st.metx * st.metx + st.mety * st.mety);
            res->q[4] = st.chi2;
        } else {
            need_higgs(an, ev, &st);
            res->idx[0] = st.d_ok ? st.pb1 : -1;
            res->idx[1] = st.d_ok ? st.pb2 : -1;
            res->idx[2] = st.h_ok ? st.h1 : -1;
            res->idx[3] = st.h_ok ? st.h2 : -1;
            res->q[0] = st.m_bb;
            res->q[1] = st.m_t1;
            res->q[2] = st.m_t2;
            res->q[3] = st.m_tt;
        }
    }
    return passed;
}

/* Evaluate one unit of event e of the given columns. */
int orc_unit(const orc_analysis* an, uint64_t e, const uint32_t* jet_off, const float* jets,
             const uint16_t* btag, const float* lep, const int8_t* lep_q, const float* met,
             uint64_t first_event_id, uint64_t seed, uint32_t v, orc_unit_result* res)
{
    orc_event ev;
    load_event(an, e, jet_off, jets, btag, lep, lep_q, met, &ev);
    return eval_unit(an, &ev, seed, first_event_id + e, v, res);
}

/*
 * Whole chunk.  For every event e and variation v < V, the unit's cuts are
 * evaluated in user order until the first failure; cutflow[k] counts the
 * units that passed cuts 1..k (cutflow[0] = N * V).  A unit passing all cuts
 * fills the histogram with its reconstructed mass (m_top semileptonic,
 * m_bb dilepton) and adds its reconstructed quantities, in variation order,
 * to the event's sums; reco[e] = sums / n_surv[e], mask[e] = n_surv[e] >= 1.
 * reco per event (4 values): semilep (m_top, m_W, pz_nu, |MET'|), dilep
 * (m_bb, m_t, m_tbar, m_ttbar); all zero when no unit survives.  reco_abs
 * (optional) receives the means of the absolute values, the magnitude scale
 * of a signed mean such as p_z.
 * Returns 0, or -1 for an invalid event (more than 12 jets).
 */
int orc_run(const orc_analysis* an, uint64_t N, const uint32_t* jet_off, const float* jets,
            const uint16_t* btag, const float* lep, const int8_t* lep_q, const float* met,
            uint64_t first_event_id, uint64_t seed, uint32_t V, uint8_t* mask,
            uint64_t* cutflow, uint64_t* hist, uint16_t* n_surv, double* reco,
            int8_t* unit_passed, double* reco_abs)
{
    for (int c = 0; c <= an->n_cuts; ++c)
        cutflow[c] = 0;
    for (int b = 0; b < an->hist_nbins + 2; ++b)
        hist[b] = 0;
    for (uint64_t e = 0; e < N; ++e) {
        if (jet_off[e + 1] < jet_off[e] || jet_off[e + 1] - jet_off[e] > ORC_MAX_JETS)
            return -1;
        orc_event ev;
        load_event(an, e, jet_off, jets, btag, lep, lep_q, met, &ev);
        double sum[4] = {0.0, 0.0, 0.0, 0.0}, sabs[4] = {0.0, 0.0, 0.0, 0.0};
        int ns = 0;
        for (uint32_t v = 0; v < V; ++v) {
            orc_unit_result r;
            int passed = eval_unit(an, &ev, seed, first_event_id + e, v, &r);
            if (unit_passed)
                unit_passed[e * V + v] = (int8_t)passed;
            for (int c = 0; c <= passed; ++c)
                cutflow[c] += 1;
            if (passed == an->n_cuts) {
                ++ns;
                double x = r.q[0];
                hist[orc_hist_bin(x, an->hist_nbins, an->hist_lo, an->hist_hi)] += 1;
                for (int k = 0; k < 4; ++k) {
                    sum[k] = sum[k] + r.q[k];
                    sabs[k] = sabs[k] + fabs(r.q[k]);
                }
            }
        }
        n_surv[e] = (uint16_t)ns;
        mask[e] = ns >= 1;
        for (int k = 0; k < 4; ++k) {
            reco[4 * e + k] = ns ? sum[k] / (double)ns : 0.0;
            if (reco_abs)
                reco_abs[4 * e + k] = ns ? sabs[k] / (double)ns : 0.0;
        }
    }
    return 0;
}
