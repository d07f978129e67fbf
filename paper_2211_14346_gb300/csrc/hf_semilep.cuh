// hf_semilep.cuh -- FP32 evaluation of one semileptonic unit with error
// bands (device code, templated on the jet multiplicity N so that the
// per-event Gram matrix, the jet scales and the triplet loop live in
// registers).
//
// Definitions (HEP-Frame, arXiv:2211.14346, Sect. 6.2): neutrino p_z from the
// W-mass constraint with MET as the neutrino pT; hadronic-top chi-square of
// Eq. 1: chi2 = ((m_jjj - m_t)/sigma_t)^2 + ((m_jj - m_W)/sigma_W)^2,
// minimised over jet triplets (k the b, {i < j} the W).
//
// GPU formulation: with the Minkowski Gram matrix G_ab = p_a . p_b of the
// event's jets (computed once per event, compensated), a smeared triplet has
//   m^2_ijk = sum_a s_a^2 G_aa + 2 sum_{a<b} s_a s_b G_ab  (a, b in {i, j, k}),
// a sum of non-negative terms for physical jets, so its FP32 relative error
// is a few ulp plus twice the error of the jet scales s; the bands below
// bound |q32 - q64| for every quantity that decides a cut, an argmin, or a
// histogram bin, and a unit inside any band is re-evaluated in FP64.
#pragma once
#include "hf_dev.cuh"
#include "hf_fp64.cuh"
#include <math_constants.h>

namespace hf {

// Cuts whose cost is a reconstruction (charged the unit's reconstruction
// cycles in the scheduler statistics); the others are charged the cheap ones.
__host__ __device__ constexpr bool heavy_cut(int kind)
{
    return kind == CUT_HADTOP_CHI2_MAX || kind == CUT_TTBAR_CHI2_MAX || kind == CUT_DILEP_SOLVABLE ||
           kind == CUT_HIGGS_WINDOW;
}

struct UnitOut {
    int f;             // cuts passed in user order (n_cuts = survives); -1 = recheck
    float4 reco;       // (m_top, m_W, pz_nu, |MET|) when f == n_cuts
    int bin;           // histogram bin when f == n_cuts
    float score;       // fit score when f == n_cuts (FP32; best-of-variations)
    unsigned evald;    // stage-2 cuts evaluated (bit = user index)
    unsigned passd;    // stage-2 cuts passed
    unsigned cyc_top;  // SM cycles spent in the reconstruction cuts (heavy_cut)
    unsigned cyc_met;  // SM cycles spent in the other stage-2 cuts
    unsigned cands;    // triplet candidates evaluated (after pair pruning)
};

// Band of an FP32 chi2 value: |chi2_32 - chi2_64| bound using only the value
// (|dt|, |dw| <= sqrt(chi2); masses <= centre + width sqrt(chi2)).
__device__ __forceinline__ float chi2_band(const Plan& P, float c)
{
    if (!(c < 3.0e38f)) return 0.0f;
    const float u = 5.9604645e-8f;  // 2^-24
    float r = sqrtf(c);
    float ddt = (P.e_m * (P.mt + P.sigma_t * r) + u * P.mt) * P.inv_sigma_t + 2.0f * u * r;
    float ddw = (P.e_m * (P.mW + P.sigma_W * r) + u * P.mW) * P.inv_sigma_W + 2.0f * u * r;
    float d = ddt + ddw;
    return P.safety * (2.0f * r * d + d * d + 3.0f * u * c);
}

// Event stride of the packed Gram matrices of a tile (shared memory): odd, so
// that lanes reading the same entry of different events hit different banks.
__host__ __device__ constexpr int gram_stride(int n) { return ntri(n) | 1; }

// Minimum and second minimum of the triplet chi2, clamped at `cap`, with the
// masses of the minimising candidate.  gf: packed upper triangle of the Gram
// matrix (entry (i, j), i <= j, at tri(i, j)), s: jet scales.  Only candidates
// with chi2 < cap can change any output (cap lies above the cut threshold by
// more than the error bands, so a clamped minimum still decides the cut and
// the argmin gap exactly).  Pairs and b-jets are fully unrolled for the
// multiplicity N, the scaled Gram terms stay in registers, and the loop runs
// over W pairs (j, then i < j) with the b-jet k innermost.  Per W jet j the
// terms u_k = a_k + q_jk are formed once, so a candidate costs two adds for
// m^2 = (m^2_ij + u_k) + q_ik (a sum of non-negative terms in another order
// than the definition's: the same relative error bound), one reciprocal
// square root, one multiply, two fused multiply-adds, and a top-2 update that
// keeps only the winner's m^2 (its mass is formed once at the end with the
// same operations, hence the same value); the winner's W mass is kept per
// pair.  *cands counts the candidates evaluated.
template <int N>
__device__ __forceinline__ void hadtop_f(const Plan& P, const float* __restrict__ gf,
                                         const float (&s)[N > 0 ? N : 1], float cap, float& b1, float& b2,
                                         float& mt_b, float& mw_b, unsigned* cands)
{
    b1 = cap;
    b2 = cap;
    mt_b = 0.0f;
    mw_b = 0.0f;
    if constexpr (N >= 3) {
        float a[N];
        float q2[N * N];
#pragma unroll
        for (int i = 0; i < N; ++i) a[i] = __fmul_rn(__fmul_rn(s[i], s[i]), gf[tri(i, i)]);
#pragma unroll
        for (int j = 1; j < N; ++j)
#pragma unroll
            for (int i = 0; i < j; ++i) q2[i * N + j] = q2[j * N + i] = 2.0f * __fmul_rn(__fmul_rn(s[i], s[j]), gf[tri(i, j)]);
        const float c_t = -P.mt * P.inv_sigma_t;
        const float c_w = -P.mW * P.inv_sigma_W;
        float c1 = cap, c2 = cap, bm2 = 0.0f, bmw = 0.0f;
#pragma unroll
        for (int j = 1; j < N; ++j) {
            float u[N];
#pragma unroll
            for (int k = 0; k < N; ++k) u[k] = k == j ? 0.0f : __fadd_rn(a[k], q2[j * N + k]);
#pragma unroll
            for (int i = 0; i < j; ++i) {
                const float pw = __fadd_rn(__fadd_rn(a[i], a[j]), q2[i * N + j]);
                const float mw = __fmul_rn(pw, rsqrt_approx(pw));
                const float dw = fmaf(mw, P.inv_sigma_W, c_w);
                const float cw = __fmul_rn(dw, dw);
                const float before = c1;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    if (k == i || k == j) continue;
                    const float m2 = __fadd_rn(__fadd_rn(pw, u[k]), q2[i * N + k]);
                    const float mt = __fmul_rn(m2, rsqrt_approx(m2));
                    const float dt = fmaf(mt, P.inv_sigma_t, c_t);
                    const float c = fmaf(dt, dt, cw);
                    bm2 = c < c1 ? m2 : bm2;
                    c2 = fminf(c2, fmaxf(c1, c));
                    c1 = fminf(c1, c);
                }
                bmw = c1 < before ? mw : bmw;
            }
        }
        b1 = c1;
        b2 = c2;
        if (c1 < cap) {
            mt_b = __fmul_rn(bm2, rsqrt_approx(bm2));
            mw_b = bmw;
        }
        *cands += (unsigned)(N * (N - 1) * (N - 2) / 2);
    }
}

// Same result as hadtop_f (clamped minimum and second minimum, the masses of
// the minimising candidate) with the smeared Gram terms in shared memory and
// the W pairs pruned exactly.  A candidate's chi2 is fmaf(dt, dt, cw) >= cw for
// the W term cw of its pair, so a pair with cw >= cap has no candidate below
// the cap and is skipped as a whole; about a third of the pairs remain.  The
// pair phase (unrolled over the N(N-1)/2 pairs) writes the full symmetric
// matrix Q_ik = 2 s_i s_k G_ik with Q_ii = HT_BIG and the diagonal terms
// A_i = s_i^2 G_ii to this thread's column of qs / as (element e at
// e * BLOCK), and marks the pairs below the cap; the candidate loop then runs
// over the marked pairs only (any order: the minimum and the second minimum
// of a set do not depend on it), with the b-jet k unrolled:
//   m^2 = ((m^2_ij + A_k) + Q_ik) + Q_jk,
// a sum of non-negative terms (the hadtop_f error bound holds).  For k = i or
// k = j one term is HT_BIG, so that candidate lands far above the cap and
// never changes the result, without a branch.  Each thread reads only its own
// column, so the loads are free of bank conflicts.  pair_code[p] = i | j << 4
// for the pair index p = j (j - 1) / 2 + i.
constexpr float HT_BIG = 1.0e30f;
constexpr int HT_SLOTS = BLOCK;  // threads (and Q columns) of a chi2 round

__host__ __device__ constexpr int npairs(int n) { return n * (n - 1) / 2; }

template <int N>
__device__ __forceinline__ void hadtop_pruned(const Plan& P, const float* __restrict__ gf,
                                              const float (&s)[N > 0 ? N : 1], float cap, float* qs, float* as,
                                              const uint8_t* pair_code, float& b1, float& b2, float& mt_b,
                                              float& mw_b, unsigned* cands)
{
    b1 = cap;
    b2 = cap;
    mt_b = 0.0f;
    mw_b = 0.0f;
    if constexpr (N >= 3) {
        constexpr int NP = npairs(N);
        const float c_t = -P.mt * P.inv_sigma_t;
        const float c_w = -P.mW * P.inv_sigma_W;
        float a[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            a[i] = __fmul_rn(__fmul_rn(s[i], s[i]), gf[tri(i, i)]);
            as[i * HT_SLOTS] = a[i];
            qs[(i * N + i) * HT_SLOTS] = HT_BIG;
        }
        unsigned long long mlo = 0ull;
        unsigned mhi = 0u;
#pragma unroll
        for (int j = 1; j < N; ++j)
#pragma unroll
            for (int i = 0; i < j; ++i) {
                const float q = 2.0f * __fmul_rn(__fmul_rn(s[i], s[j]), gf[tri(i, j)]);
                qs[(i * N + j) * HT_SLOTS] = q;
                qs[(j * N + i) * HT_SLOTS] = q;
                const float pw = __fadd_rn(__fadd_rn(a[i], a[j]), q);
                const float mw = __fmul_rn(pw, rsqrt_approx(pw));
                const float dw = fmaf(mw, P.inv_sigma_W, c_w);
                const float cw = __fmul_rn(dw, dw);
                const int p = j * (j - 1) / 2 + i;
                if (cw < cap) {
                    if (p < 64) mlo |= 1ull << p;
                    else mhi |= 1u << (p - 64);
                }
            }
        static_assert(NP <= 96, "pair mask");
        *cands += (unsigned)((__popcll(mlo) + __popc(mhi)) * (N - 2));
        float c1 = cap, c2 = cap, bm2 = 0.0f, bmw = 0.0f;
        while (mlo | (unsigned long long)mhi) {
            int p;
            if (mlo) {
                p = __ffsll((long long)mlo) - 1;
                mlo &= mlo - 1ull;
            } else {
                p = 64 + __ffs(mhi) - 1;
                mhi &= mhi - 1u;
            }
            const int code = pair_code[p];
            const int i = code & 15, j = code >> 4;
            const float pw = __fadd_rn(__fadd_rn(as[i * HT_SLOTS], as[j * HT_SLOTS]), qs[(i * N + j) * HT_SLOTS]);
            const float mw = __fmul_rn(pw, rsqrt_approx(pw));
            const float dw = fmaf(mw, P.inv_sigma_W, c_w);
            const float cw = __fmul_rn(dw, dw);
            const float* qi = qs + i * N * HT_SLOTS;
            const float* qj = qs + j * N * HT_SLOTS;
            const float before = c1;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const float m2 = __fadd_rn(__fadd_rn(__fadd_rn(pw, a[k]), qi[k * HT_SLOTS]), qj[k * HT_SLOTS]);
                const float mt = __fmul_rn(m2, rsqrt_approx(m2));
                const float dt = fmaf(mt, P.inv_sigma_t, c_t);
                const float c = fmaf(dt, dt, cw);
                bm2 = c < c1 ? m2 : bm2;
                c2 = fminf(c2, fmaxf(c1, c));
                c1 = fminf(c1, c);
            }
            bmw = c1 < before ? mw : bmw;
        }
        b1 = c1;
        b2 = c2;
        if (c1 < cap) {
            mt_b = __fmul_rn(bm2, rsqrt_approx(bm2));
            mw_b = bmw;
        }
    }
}

// Table of the pair codes i | j << 4 in pair-index order (p = j (j - 1) / 2 + i).
__device__ __forceinline__ void fill_pair_codes(uint8_t* t)
{
    for (int p = threadIdx.x; p < npairs(MAX_JETS); p += blockDim.x) {
        int j = 1;
        while ((j + 1) * j / 2 <= p) ++j;
        const int i = p - j * (j - 1) / 2;
        t[p] = (uint8_t)(i | j << 4);
    }
}

// ------------------------------------------------------------------ full Eq. 1 fit
// Result of the full semileptonic fit of a unit (FP64, the definition's).
struct FullFitD {
    double chi2, mtop_had, mtop_lep, pz;
};

// The full chi-square of Eq. 1 (Sect. 6.2): hadronic top and W from jets
// k, {i < j}, leptonic top from jet l, the lepton and a neutrino solution r
// (w_pz_both_d), leptonic W from the lepton and that neutrino; minimum over
// k, i < j, l (all distinct), r in that enumeration order, strict, ties to
// the first.  n < 4 or no neutrino solution: +inf.  lep: the lepton, metx,
// mety: the smeared MET (FP64).  Candidates are restricted to `list`
// (codes k | i << 4 | j << 8 | l << 12 | r << 16, in enumeration order)
// when nlist >= 0, else all are enumerated.
static __device__ __noinline__ FullFitD ttbar_full_d(const Plan& P, LazyUnitD& U, const double* lep, double metx,
                                                     double mety, const int* list, int nlist)
{
    FullFitD f;
    f.chi2 = CUDART_INF;
    f.mtop_had = f.mtop_lep = f.pz = 0.0;
    const int n = U.n;
    double pz[2];
    const int nr = w_pz_both_d(lep, metx, mety, P.dmW, pz);
    if (n < 4 || nr == 0) return f;
    double Wl[2][4], mwl[2];
    for (int r = 0; r < nr; ++r) {
        const double nu[4] = {metx, mety, pz[r], sqrt(metx * metx + mety * mety + pz[r] * pz[r])};
        v4_add_d(lep, nu, Wl[r]);
        mwl[r] = mass_d(Wl[r]);
    }
    auto eval = [&](int k, int i, int j, int l, int r, double had, const double* T) {
        double TL[4];
        v4_add_d(U.j(l), Wl[r], TL);
        const double m_tl = mass_d(TL);
        const double dtl = (m_tl - P.dmt) / P.dsigma_t;
        const double dwl = (mwl[r] - P.dmW) / P.dsigma_W;
        const double chi2 = had + (dtl * dtl + dwl * dwl);
        if (chi2 < f.chi2) {
            f.chi2 = chi2;
            f.mtop_had = mass_d(T);
            f.mtop_lep = m_tl;
            f.pz = pz[r];
        }
    };
    auto had_of = [&](int k, int i, int j, double* T) {
        double W[4];
        v4_add_d(U.j(i), U.j(j), W);
        v4_add_d(W, U.j(k), T);
        const double dt = (mass_d(T) - P.dmt) / P.dsigma_t;
        const double dw = (mass_d(W) - P.dmW) / P.dsigma_W;
        return dt * dt + dw * dw;
    };
    if (nlist >= 0) {
        int prev = -1;
        double had = 0.0, T[4];
        for (int t = 0; t < nlist; ++t) {
            const int c = list[t];
            const int k = c & 15, i = (c >> 4) & 15, j = (c >> 8) & 15, l = (c >> 12) & 15, r = (c >> 16) & 1;
            if (r >= nr) continue;
            if ((c & 0xfff) != prev) {
                prev = c & 0xfff;
                had = had_of(k, i, j, T);
            }
            eval(k, i, j, l, r, had, T);
        }
        return f;
    }
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            for (int j = i + 1; j < n; ++j) {
                if (j == k) continue;
                double T[4];
                const double had = had_of(k, i, j, T);
                for (int l = 0; l < n; ++l) {
                    if (l == k || l == i || l == j) continue;
                    for (int r = 0; r < nr; ++r) eval(k, i, j, l, r, had, T);
                }
            }
        }
    return f;
}

// The full fit of a unit with little FP64 work: an FP32 screen and the
// definition's FP64 arithmetic on the candidates that survive it.  The
// neutrino solutions and the leptonic terms of every (l, r) are computed in
// FP64 from the FP64-smeared MET (exact) and the FP32 jet scales s (relative
// error <= s_rel), so each leptonic top mass is within (s_rel + 1e-15) of the
// definition's; the hadronic terms come from the FP32 Gram form with the
// chi2 band.  A candidate can be the FP64 minimum only if its screened value
// is within both bands of the screened minimum; those (at most 32, else the
// full enumeration) are evaluated in FP64 in enumeration order.  The result
// is the definition's, so the cut needs no band and no recheck.
// g: the event's packed Gram matrix, s: FP32 jet scales (n entries), mf: the
// event's unsmeared MET.
static __device__ __noinline__ FullFitD ttbar_screened(const Plan& P, LazyUnitD& U, const float* g, const float* s,
                                                       const double* lep, float2 mf)
{
    FullFitD none;
    none.chi2 = CUDART_INF;
    none.mtop_had = none.mtop_lep = none.pz = 0.0;
    const int n = U.n;
    if (n < 4) return none;
    U.met(mf);
    double pz[2];
    const int nr = w_pz_both_d(lep, U.metx, U.mety, P.dmW, pz);
    if (nr == 0) return none;
    // leptonic terms per (l, r) and their bands
    float L[MAX_JETS][2], Lb[MAX_JETS][2];
    {
        double Wl[2][4];
        double cw[2];
        for (int r = 0; r < nr; ++r) {
            const double nu[4] = {U.metx, U.mety, pz[r], sqrt(U.metx * U.metx + U.mety * U.mety + pz[r] * pz[r])};
            v4_add_d(lep, nu, Wl[r]);
            const double dwl = (mass_d(Wl[r]) - P.dmW) / P.dsigma_W;
            cw[r] = dwl * dwl;
        }
        const double rel = 2.0 * (double)P.s_rel + 1.0e-12;
        for (int l = 0; l < n; ++l) {
            const float4 jf = U.jp[l];
            const double sl = (double)s[l];
            const double jl[4] = {sl * jf.x, sl * jf.y, sl * jf.z, sl * jf.w};
            for (int r = 0; r < 2; ++r) {
                if (r >= nr) {
                    L[l][r] = CUDART_INF_F;
                    Lb[l][r] = 0.f;
                    continue;
                }
                double TL[4];
                v4_add_d(jl, Wl[r], TL);
                const double m = mass_d(TL);
                const double d = (m - P.dmt) / P.dsigma_t;
                const double dd = rel * fabs(m) / P.dsigma_t;
                L[l][r] = (float)(d * d + cw[r]);
                Lb[l][r] = (float)(2.0 * fabs(d) * dd + dd * dd) * 1.01f + 2.4e-7f * L[l][r] + 1.0e-30f;
            }
        }
    }
    // hadronic terms in FP32 (Gram form, as in the triplet cut)
    float a[MAX_JETS];
    for (int i = 0; i < n; ++i) a[i] = __fmul_rn(__fmul_rn(s[i], s[i]), g[tri(i, i)]);
    auto q2 = [&](int x, int y) {
        const int lo = x < y ? x : y, hi = x < y ? y : x;
        return 2.0f * __fmul_rn(__fmul_rn(s[lo], s[hi]), g[tri(lo, hi)]);
    };
    const float c_t = -P.mt * P.inv_sigma_t, c_w = -P.mW * P.inv_sigma_W;
    auto had32 = [&](int k, int i, int j) {
        const float pw = __fadd_rn(__fadd_rn(a[i], a[j]), q2(i, j));
        const float mw = __fmul_rn(pw, rsqrt_approx(pw));
        const float dw = fmaf(mw, P.inv_sigma_W, c_w);
        const float m2 = __fadd_rn(__fadd_rn(__fadd_rn(pw, a[k]), q2(i, k)), q2(j, k));
        const float mt = __fmul_rn(m2, rsqrt_approx(m2));
        const float dt = fmaf(mt, P.inv_sigma_t, c_t);
        return fmaf(dt, dt, __fmul_rn(dw, dw));
    };
    // pass 1: the screened minimum; pass 2: the candidates within the bands
    float best = CUDART_INF_F, best_band = 0.f;
    int list[32];
    int nl = 0;
    bool overflow = false;
    for (int pass = 0; pass < 2 && !overflow; ++pass) {
        for (int k = 0; k < n && !overflow; ++k)
            for (int i = 0; i < n && !overflow; ++i) {
                if (i == k) continue;
                for (int j = i + 1; j < n && !overflow; ++j) {
                    if (j == k) continue;
                    const float h = had32(k, i, j);
                    const float hb = chi2_band(P, h);
                    for (int l = 0; l < n && !overflow; ++l) {
                        if (l == k || l == i || l == j) continue;
                        for (int r = 0; r < nr; ++r) {
                            const float c = __fadd_rn(h, L[l][r]);
                            const float cb = hb + Lb[l][r] + 2.4e-7f * c;
                            if (pass == 0) {
                                if (c < best) {
                                    best = c;
                                    best_band = cb;
                                }
                            } else if (c <= best + best_band + cb) {
                                if (nl < 32) list[nl++] = k | i << 4 | j << 8 | l << 12 | r << 16;
                                else overflow = true;
                            }
                        }
                    }
                }
            }
    }
    return ttbar_full_d(P, U, lep, U.metx, U.mety, list, overflow ? -1 : nl);
}

// Cap of the clamped triplet minimum for a chi2 cut at thr: above thr by
// 2.5 bands, so that a minimum at the cap is a certain failure and a second
// minimum at the cap leaves a certain argmin gap.
__device__ __forceinline__ float chi2_cap(const Plan& P, float thr)
{
    return thr + 2.5f * chi2_band(P, thr) + 1.0e-6f * fabsf(thr) + 1.0e-30f;
}

// Float-float (unevaluated sum hi + lo) arithmetic, relative accuracy about
// 2^-44 per operation (Dekker 1971; TwoProduct with fmaf).
struct ff {
    float h, l;
};
__device__ __forceinline__ ff ff_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    return ff{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_norm(float s, float e)
{
    float h = __fadd_rn(s, e);
    return ff{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    return ff_norm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.h, -b.l}); }
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = ff_prod(a.h, b.h);
    return ff_norm(p.h, __fadd_rn(p.l, fmaf(a.h, b.l, __fmul_rn(a.l, b.h))));
}

// W-mass neutrino p_z with mu, D and the numerator in float-float and a
// running error bound that includes the error of the FP32-smeared MET
// (dmx, dmy).  Returns false when the discriminant's sign is uncertain or the
// bound exceeds pz_tol |p(nu)| (|p_z| + pT bounds the neutrino momentum);
// the caller then takes the FP64 value.
__device__ __forceinline__ bool w_pz_f(const Plan& P, float4 l, float mx, float my, float dmx, float dmy,
                                       float& pz)
{
    const float u = 5.9604645e-8f;   // 2^-24
    const float u2 = 9.094947e-13f;  // 2^-40: a few float-float operations
    ff mu = ff_add(ff_add(ff{P.mW2half, P.mW2half_lo}, ff_prod(l.x, mx)), ff_prod(l.y, my));
    ff el2 = ff_prod(l.w, l.w);
    ff a = ff_sub(el2, ff_prod(l.z, l.z));
    ff pt2 = ff_add(ff_prod(mx, mx), ff_prod(my, my));
    ff mu2 = ff_mul(mu, mu);
    ff D = ff_sub(mu2, ff_mul(a, pt2));
    ff num = ff_sub(ff_mul(el2, pt2), mu2);
    const float amu = fabsf(mu.h), af = a.h, apt2 = pt2.h;
    float e_mu = fabsf(l.x) * dmx + fabsf(l.y) * dmy + u2 * (P.mW2half + fabsf(l.x * mx) + fabsf(l.y * my));
    float e_pt2 = 2.0f * (fabsf(mx) * dmx + fabsf(my) * dmy) + dmx * dmx + dmy * dmy + u2 * apt2;
    float e_a = u2 * (el2.h + l.z * l.z);
    float e_D = 2.0f * amu * e_mu + e_mu * e_mu + af * e_pt2 + apt2 * e_a + u2 * (amu * amu + af * apt2);
    float e_num = el2.h * e_pt2 + 2.0f * amu * e_mu + e_mu * e_mu + u2 * (el2.h * apt2 + amu * amu);
    if (!(af > 0.0f)) { pz = 0.0f; return false; }
    const float Df = __fadd_rn(D.h, D.l);
    if (fabsf(Df) <= P.safety * e_D) return false;
    float e_pz;
    if (Df < 0.0f) {
        pz = __fdiv_rn(__fmul_rn(mu.h, l.z), af);
        e_pz = (fabsf(l.z) * e_mu + fabsf(pz) * e_a) / af + 4.0f * u * fabsf(pz);
    } else {
        float sD = sqrtf(Df);
        float e_sD = e_D / (2.0f * sD) + u * sD;
        float t = __fmul_rn(mu.h, l.z);
        float sq = __fmul_rn(l.w, sD);
        float q = t >= 0.0f ? __fadd_rn(t, sq) : __fsub_rn(t, sq);
        if (q == 0.0f) return false;
        float e_q = fabsf(l.z) * e_mu + l.w * e_sD + 3.0f * u * fabsf(q);
        float nf = __fadd_rn(num.h, num.l);
        pz = __fdiv_rn(nf, q);
        e_pz = (e_num + u * fabsf(nf) + fabsf(pz) * e_q) / fabsf(q) + u * fabsf(pz);
    }
    return e_pz <= P.pz_tol * (fabsf(pz) + sqrtf(apt2));
}

// p_z in FP64 with the MET smeared in FP64 (the definition's arithmetic):
// used when the FP32 bound is too wide, typically near D = 0 where p_z is
// ill-conditioned in MET.  Does not affect any cut decision.
static __device__ __noinline__ float w_pz_fp64(const Plan& P, float4 l, float2 met, uint64_t seed, uint64_t event_id,
                                        uint32_t v)
{
    double mx = met.x, my = met.y;
    double lep[4] = {l.x, l.y, l.z, l.w};
    if (P.smear_met || P.smear_jets || P.smear_lep) {
        uint4 w = philox4x32_10(ctr_of(3, v, event_id), key_of(seed));
        double z12, z13;
        box_muller_d(w.x, w.y, z12, z13);
        mx = (double)met.x + P.dsigma_met * z12;
        my = (double)met.y + P.dsigma_met * z13;
        if (P.smear_lep) {
            double z14, z15;
            box_muller_d(w.z, w.w, z14, z15);
            const double sl = 1.0 + P.dsigma_lep * z14;
            for (int k = 0; k < 4; ++k) lep[k] = sl * lep[k];
        }
    }
    double pz;
    w_pz_d(lep, mx, my, P.dmW, &pz);
    return (float)pz;
}

// Per-event inputs of a semileptonic unit.
template <int N>
struct SemiEvent {
    const float* g;  // packed Gram matrix (shared memory, or registers in the plain form)
    const float4* jets;  // the event's jets in global memory (for the full fit in FP64)
    float4 lep;
    float2 met;
    unsigned s1bits;
    uint64_t event_id;
};

// The full Eq. 1 fit of a unit (exact: the FP32 screen and the FP64
// definition on its survivors).
template <int N>
__device__ __noinline__ FullFitD semi_full_fit(const Plan& P, const SemiEvent<N>& ev, const float* s, uint32_t v,
                                               uint64_t seed)
{
    LazyUnitD U;
    U.init_jets(P, ev.jets, N, ev.event_id, seed, v);
    double lep[4];
    U.lepton(0, ev.lep, lep);
    return ttbar_screened(P, U, ev.g, s, lep, ev.met);
}

// Scheduler statistics of one block (shared memory).
struct CutStats {
    unsigned evaluated[MAX_CUTS];
    unsigned passed[MAX_CUTS];
    unsigned long long cost[MAX_CUTS];
    unsigned long long cands;  // triplet candidates evaluated in the block
};

// FP32 jet scales s_i = 1 + sigma_jet z_i of unit (event, v): normals z_0..z_11
// from Philox blocks 0..2 (Box-Muller pairs (z_0, z_1), (z_2, z_3), ... of
// each block); only the first N are formed.
template <int N>
__device__ __forceinline__ void jet_scales_f(const Plan& P, uint32_t v, uint64_t event_id, uint2 key,
                                             float (&s)[N > 0 ? N : 1])
{
#pragma unroll
    for (int b = 0; b < (N + 3) / 4; ++b) {
        uint4 w = philox4x32_10(ctr_of(b, v, event_id), key);
        float z0, z1, z2, z3;
        box_muller_f(w.x, w.y, z0, z1);
        if (4 * b + 0 < N) s[4 * b + 0] = fmaf(P.sigma_jet, z0, 1.0f);
        if (4 * b + 1 < N) s[4 * b + 1] = fmaf(P.sigma_jet, z1, 1.0f);
        if (4 * b + 2 < N) {
            box_muller_f(w.z, w.w, z2, z3);
            s[4 * b + 2] = fmaf(P.sigma_jet, z2, 1.0f);
            if (4 * b + 3 < N) s[4 * b + 3] = fmaf(P.sigma_jet, z3, 1.0f);
        }
    }
}

// Modes of semi_unit_f.  UNIT_WHOLE evaluates everything in the unit's
// thread.  UNIT_PROBE stops where the triplet chi2 is first needed and
// returns f = F_NEED_TOP with the smeared MET state (mx, my, dmx, dmy) in
// reco; the tile then evaluates the chi2 of all such units together and
// completes them with UNIT_RESUME, which takes the MET state and the chi2
// result from a TopIn instead of computing them.
enum : int { UNIT_WHOLE = 0, UNIT_PROBE = 1, UNIT_RESUME = 2 };
constexpr int F_NEED_TOP = -2;

struct TopIn {
    float4 met;        // smeared MET x, y and their error bounds
    float b1, b2;      // clamped minimum and second minimum of the triplet chi2
    float mt, mw;      // masses of the minimising candidate (when b1 < cap)
    unsigned cyc;      // SM cycles of the chi2 evaluation
    unsigned cands;    // candidates evaluated
};

// FP32 evaluation of one semileptonic unit.  exec: stage-2 cuts in execution
// order.  After the first failure in execution order, the stage-2 cuts that
// precede the earliest known failure in USER order and were not evaluated are
// evaluated in user order, so that the reported number of leading cuts passed
// is the user-order one whatever the execution order.
// F: the analysis has the full Eq. 1 fit (instantiated separately, so that the
// triplet-only chain carries none of its code or registers).
template <int N, bool F, int MODE = UNIT_WHOLE>
__device__ UnitOut semi_unit_f(const Plan& P, const int* exec, int nexec, const SemiEvent<N>& ev,
                               uint32_t v, uint64_t seed, const TopIn* tin = nullptr)
{
    static_assert(MODE == UNIT_WHOLE || !F, "the split evaluation serves triplet-only analyses");
    UnitOut out;
    out.f = -1;
    out.reco = make_float4(0.f, 0.f, 0.f, 0.f);
    out.bin = 0;
    out.score = 0.0f;
    out.evald = out.passd = out.cyc_top = out.cyc_met = out.cands = 0;
    float s[N > 0 ? N : 1];
#pragma unroll
    for (int i = 0; i < (N > 0 ? N : 1); ++i) s[i] = 1.0f;
    float mx = ev.met.x, my = ev.met.y, dmx = 0.0f, dmy = 0.0f;
    const uint2 key = key_of(seed);
    // jet scales (Philox blocks 0-2) only once a cut or the fit needs them: a
    // unit that fails a cheaper cut first never draws them
    bool s_todo = MODE == UNIT_WHOLE && P.smear_jets;
    // lepton scale s_l = 1 + sigma_lep z14 and its error bound (Philox block 3,
    // words z, w; the MET shift uses words x, y of the same block)
    float sl = 1.0f, dsl = 0.0f;
    if (MODE == UNIT_RESUME) {
        mx = tin->met.x;
        my = tin->met.y;
        dmx = tin->met.z;
        dmy = tin->met.w;
    }
    if ((MODE != UNIT_RESUME && P.smear_met) || P.smear_lep) {
        uint4 w = philox4x32_10(ctr_of(3, v, ev.event_id), key);
        const float u = 5.9604645e-8f;
        if (MODE != UNIT_RESUME && P.smear_met) {
            float z12, z13;
            box_muller_f(w.x, w.y, z12, z13);
            mx = fmaf(P.sigma_met, z12, ev.met.x);
            my = fmaf(P.sigma_met, z13, ev.met.y);
            dmx = P.sigma_met * P.z_rel * fabsf(z12) + u * fabsf(mx);
            dmy = P.sigma_met * P.z_rel * fabsf(z13) + u * fabsf(my);
        }
        if (P.smear_lep) {
            float z14, z15;
            box_muller_f(w.z, w.w, z14, z15);
            sl = fmaf(P.sigma_lep, z14, 1.0f);
            dsl = P.sigma_lep * P.z_rel * fabsf(z14) + u * sl;
        }
    }
    float b1 = CUDART_INF_F, b2 = CUDART_INF_F, mt_b = 0.f, mw_b = 0.f;
    bool top_done = false;
    FullFitD ff;
    bool full_done = false;
    float met = 0.f, met_err = 0.f;
    bool met_done = false;
    unsigned evald = 0, passd = 0;
    // first stage-1 failure (user order) bounds the cuts that matter
    const unsigned s1fail = P.stage1 & ~ev.s1bits;
    bool phase1 = true;
    int x = 0;
    int f = P.n_cuts;
    while (true) {
        int c;
        unsigned fails = s1fail | (evald & ~passd);
        int kf = fails ? __ffs(fails) - 1 : P.n_cuts;
        if (phase1) {
            if (x >= nexec) { phase1 = false; continue; }
            c = exec[x++];
            if (c > kf) continue;
        } else {
            unsigned below = kf >= 32 ? 0xffffffffu : ((1u << kf) - 1u);
            unsigned todo = P.stage2 & ~evald & below;
            if (!todo) { f = kf; break; }
            c = __ffs(todo) - 1;
        }
        long long t0 = clock64();
        bool pass = false, unsure = false;
        const int kind = P.kind[c];
        if (kind == CUT_MET_MIN) {
            if (!met_done) {
                met = sqrtf(fmaf(mx, mx, __fmul_rn(my, my)));
                met_err = P.safety * (dmx + dmy + 3.6e-7f * met);
                met_done = true;
            }
            pass = met > P.p0[c];
            unsure = fabsf(met - P.p0[c]) <= met_err;
        } else if (kind == CUT_LEP_PT_MIN) {
            // smeared lepton pT = s_l pT: FP32 with the bound of s_l and the rounding
            const float pt = __fmul_rn(sqrtf(fmaf(ev.lep.x, ev.lep.x, __fmul_rn(ev.lep.y, ev.lep.y))), sl);
            pass = pt > P.p0[c];
            unsure = fabsf(pt - P.p0[c]) <= P.safety * (pt * (dsl / sl + 3.6e-7f));
        } else if (kind == CUT_W_NU_SOLVABLE) {
            // E^2 - pz^2 of the smeared lepton is s_l^2 (E^2 - pz^2): the FP32
            // product (E - pz)(E + pz) has its exact sign; near 0 the FP64 one decides
            const float a = __fmul_rn(__fsub_rn(ev.lep.w, ev.lep.z), __fadd_rn(ev.lep.w, ev.lep.z));
            pass = a > 0.0f;
            unsure = fabsf(a) <= 1.0e-6f * __fmul_rn(ev.lep.w, ev.lep.w);
        } else if (kind == CUT_HADTOP_CHI2_MAX) {
            if (!top_done) {
                if constexpr (MODE == UNIT_PROBE) {
                    out.f = F_NEED_TOP;
                    out.reco = make_float4(mx, my, dmx, dmy);
                    return out;
                } else if constexpr (MODE == UNIT_RESUME) {
                    b1 = tin->b1;
                    b2 = tin->b2;
                    mt_b = tin->mt;
                    mw_b = tin->mw;
                    out.cands += tin->cands;
                    out.cyc_top += tin->cyc;
                } else {
                    if (s_todo) {
                        jet_scales_f<N>(P, v, ev.event_id, key, s);
                        s_todo = false;
                    }
                    hadtop_f<N>(P, ev.g, s, chi2_cap(P, P.top_thr), b1, b2, mt_b, mw_b, &out.cands);
                }
                top_done = true;
            }
            pass = b1 < P.p0[c];
            unsure = fabsf(b1 - P.p0[c]) <= chi2_band(P, b1);
        } else if (kind == CUT_TTBAR_CHI2_MAX) {
            if constexpr (F) {
                if (!full_done) {
                    if (s_todo) {
                        jet_scales_f<N>(P, v, ev.event_id, key, s);
                        s_todo = false;
                    }
                    ff = semi_full_fit<N>(P, ev, s, v, seed);
                    full_done = true;
                }
                pass = ff.chi2 < P.dp0[c];  // FP64, the definition's value
            }
        }
        const unsigned dt = (unsigned)(clock64() - t0);
        if (heavy_cut(kind)) out.cyc_top += dt;
        else out.cyc_met += dt;
        evald |= 1u << c;
        if (pass) passd |= 1u << c;
        out.evald = evald;
        out.passd = passd;
        if (unsure) return out;  // f = -1: FP64 recheck
        if (!pass) phase1 = false;
    }
    if constexpr (F) {
        if (f == P.n_cuts) {
            // survivor of an analysis with the full fit: its (exact) values
            if (!full_done) {
                if (s_todo) {
                    jet_scales_f<N>(P, v, ev.event_id, key, s);
                    s_todo = false;
                }
                ff = semi_full_fit<N>(P, ev, s, v, seed);
                full_done = true;
            }
            if (!met_done) met = sqrtf(fmaf(mx, mx, __fmul_rn(my, my)));
            out.bin = hist_bin_d(P, ff.mtop_had);
            out.reco = make_float4((float)ff.mtop_had, (float)ff.mtop_lep, (float)ff.pz, met);
            out.score = (float)ff.chi2;
        }
    } else if (f == P.n_cuts) {
        // survivor: reconstructed quantities must be certain as well
        if (!top_done) return out;  // (the model always has the chi2 cut)
        if (b2 - b1 <= chi2_band(P, b1) + chi2_band(P, b2)) return out;  // argmin near-tie
        float pz;
        // with a smeared lepton the float-float bound does not cover the lepton's
        // error: p_z (a reconstructed value, no decision) comes from FP64
        if (P.smear_lep || !w_pz_f(P, ev.lep, mx, my, dmx, dmy, pz)) pz = w_pz_fp64(P, ev.lep, ev.met, seed, ev.event_id, v);
        if (!met_done) met = sqrtf(fmaf(mx, mx, __fmul_rn(my, my)));
        bool hu = false;
        int bin = hist_bin_f(P, mt_b, P.safety * P.e_m * mt_b, &hu);
        if (hu) return out;
        out.bin = bin;
        out.reco = make_float4(mt_b, mw_b, pz, met);
        out.score = b1;
    }
    out.f = f;
    return out;
}

}  // namespace hf
