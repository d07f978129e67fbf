// hf_common.cuh -- device helpers shared by the kernels of the cut chain:
// exact stage-1 predicates, cut-flow and histogram flushes, the FP64 unit
// evaluation, compensated per-event sums and the pending-event protocol of
// the FP64 recheck.  Header-only; every translation unit gets its own copy.
#pragma once
#include "hf_dev.cuh"
#include "hf_fp64.cuh"
#include "hf_semilep.cuh"
#include "hf_dilep_f.cuh"

namespace hf {

__device__ __forceinline__ void write_zero_event(const Out& O, uint32_t e)
{
    if (O.mask) O.mask[e] = 0;
    if (O.n_surv) O.n_surv[e] = 0;
    if (O.reco) O.reco[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (O.maxf) O.maxf[e] = 0;
    if (O.best_v) O.best_v[e] = 0xffffu;
}

// ------------------------------------------------------------------ per-cut records
// Per-cut variable recording (Sect. 3: the variables the user chose are kept
// at every selection level, at their default where not yet updated).  The
// event paths store maxf, the most cuts (user order) passed by any variation
// of the event; after the run, event e gets one record per recorded level
// k < maxf, written in (event, level) order by k_rec_count / k_rec_scan /
// k_rec_write.
__device__ __forceinline__ unsigned rec_count(const Plan& P, int maxf)
{
    return __popc(P.rec_levels & (maxf >= 32 ? 0xffffffffu : ((1u << (maxf > 0 ? maxf : 0)) - 1u)));
}

// Values of event e's records at level `level` (r: its reconstructed means).
__device__ __forceinline__ void record_values(const Plan& P, const Cols& C, uint32_t e, float4 r, int level,
                                              float* val)
{
    const uint32_t n = C.jet_off[e + 1] - C.jet_off[e];
    for (int i = 0; i < 4; ++i) {
        const int var = P.rec_var[i];
        float x = 0.f;
        if (var == VAR_NJETS) {
            x = (float)n;
        } else if (var == VAR_NBTAG) {
            x = (float)__popc(C.btag[e] & ((1u << n) - 1u));
        } else if (var == VAR_LEP_PT) {
            const float4 l = C.lep[P.model == MODEL_DILEP ? 2 * (uint64_t)e : (uint64_t)e];
            x = (float)__dsqrt_rn((double)l.x * (double)l.x + (double)l.y * (double)l.y);
        } else if (var == VAR_MET) {
            const float2 m = C.met[e];
            x = (float)__dsqrt_rn((double)m.x * (double)m.x + (double)m.y * (double)m.y);
        } else if (var >= VAR_RECO0 && var < VAR_RECO0 + 4 && level == P.n_cuts - 1) {
            x = var == VAR_RECO0 ? r.x : var == VAR_RECO0 + 1 ? r.y : var == VAR_RECO0 + 2 ? r.z : r.w;
        }
        val[i] = x;
    }
}

// Exclusive prefix sum over the threads of a block (blockDim.x a multiple of
// 32, at most 1024); every thread calls.  Returns x's prefix and the total.
__device__ inline unsigned long long block_excl_scan(unsigned long long x, unsigned long long* total)
{
    __shared__ unsigned long long s_w[32];
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (unsigned)o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = lane < nw ? s_w[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= (unsigned)o) t += y;
        }
        if (lane < nw) s_w[lane] = t;  // inclusive prefix of the warp totals
    }
    __syncthreads();
    const unsigned long long before = w ? s_w[w - 1] : 0ull;
    *total = s_w[nw - 1];
    __syncthreads();
    return before + inc - x;
}

// Exact decision of pT(x, y) > thr: FP32 with a rounding band, FP64 inside it.
__device__ __forceinline__ bool pt_gt(float x, float y, float thr, double dthr, float safety)
{
    float pt = sqrtf(fmaf(x, x, __fmul_rn(y, y)));
    float band = safety * 3.6e-7f * pt;
    if (fabsf(pt - thr) > band) return pt > thr;
    double dx = x, dy = y;
    return sqrt(dx * dx + dy * dy) > dthr;
}

__device__ __forceinline__ int popc_n(unsigned bits, int n) { return __popc(bits & ((1u << n) - 1u)); }

// Stage-1 cuts of event e (those that do not depend on the variation).
__device__ inline unsigned stage1_bits(const Plan& P, const Cols& C, uint32_t e, int n)
{
    unsigned bits = 0;
    const int L = P.model == MODEL_DILEP ? 2 : 1;
    for (int c = 0; c < P.n_cuts; ++c) {
        if (!(P.stage1 >> c & 1u)) continue;
        bool pass = false;
        switch (P.kind[c]) {
        case CUT_NJETS_MIN: pass = n >= (int)P.p0[c]; break;
        case CUT_NBTAG_MIN: pass = popc_n(C.btag[e], n) >= (int)P.p0[c]; break;
        case CUT_LEP_PT_MIN: {
            float4 l = C.lep[(uint64_t)e * L];
            pass = pt_gt(l.x, l.y, P.p0[c], P.dp0[c], P.safety);
            break;
        }
        case CUT_MET_MIN: {
            float2 m = C.met[e];
            pass = pt_gt(m.x, m.y, P.p0[c], P.dp0[c], P.safety);
            break;
        }
        case CUT_W_NU_SOLVABLE: {
            // a = E^2 - pz^2 > 0: the FP32 product (E - pz)(E + pz) has the
            // exact sign of E^2 - pz^2 (each correctly rounded factor keeps
            // its sign), as does the FP64 difference of the exact squares.
            float4 l = C.lep[(uint64_t)e * L];
            float a = __fmul_rn(__fsub_rn(l.w, l.z), __fadd_rn(l.w, l.z));
            pass = a > 0.0f;
            break;
        }
        case CUT_LEP_OS: {
            int q0 = C.lep_q[(uint64_t)e * 2], q1 = C.lep_q[(uint64_t)e * 2 + 1];
            pass = q0 * q1 < 0;
            break;
        }
        default: break;
        }
        if (pass) bits |= 1u << c;
    }
    return bits;
}

__device__ __forceinline__ int first_fail_stage1(const Plan& P, unsigned bits)
{
    unsigned fails = P.stage1 & ~bits;
    return fails ? __ffs(fails) - 1 : P.n_cuts;
}

__device__ __forceinline__ bool needs_stage2(const Plan& P, int f1)
{
    unsigned below = f1 >= 32 ? 0xffffffffu : ((1u << f1) - 1u);
    return (P.stage2 & below) != 0u;
}

// Adds the per-block counts of units by first-failure index into the cut flow.
__device__ __forceinline__ void flush_cutflow(const Plan& P, const Out& O, const unsigned long long* fc)
{
    int c = threadIdx.x;
    if (c <= P.n_cuts) {
        unsigned long long s = 0;
        for (int f = c; f <= P.n_cuts; ++f) s += fc[f];
        if (s) atomicAdd(&O.cutflow[c], s);
    }
}

__device__ __forceinline__ void flush_hist(const Plan& P, const Out& O, const unsigned* h)
{
    for (int b = threadIdx.x; b < P.nbins + 2; b += blockDim.x)
        if (h[b]) atomicAdd(&O.hist[b], (unsigned long long)h[b]);
}

// ------------------------------------------------------------------ FP64 unit
// Full unit in FP64 with the definition's formulation (user order; stage-1
// results are already exact and are taken from s1bits).  Returns the number
// of leading cuts passed; reco and bin are set when all pass.

// Exact (definition) triplet minimum of a unit with little FP64 work.  An
// FP32 pass with the stage-2 arithmetic finds the FP32 minimum b and keeps
// the candidates whose FP32 chi2 c satisfies c <= b + band(b) + band(c); since
// |chi2_32 - chi2_64| <= band for every candidate, this set contains every
// candidate that can be the FP64 minimum, including all ties.  Only those are
// evaluated in FP64 with the definition's formulation, in the definition's
// enumeration order (k, then i < j) with a strict minimum.  More than 32
// survivors of the screen fall back to the full FP64 enumeration.
static __device__ __noinline__ double hadtop_screened_d(const Plan& P, LazyUnitD& U, double* mtop, double* mw)
{
    const int n = U.n;
    *mtop = 0.0;
    *mw = 0.0;
    if (n < 3) return CUDART_INF;
    float4 jf[MAX_JETS];
    float s[MAX_JETS];
    for (int i = 0; i < n; ++i) {
        jf[i] = U.jp[i];
        s[i] = 1.0f;
    }
    if (P.smear_jets) {
        const uint2 key = key_of(U.seed);
        for (int b = 0; b < (n + 3) / 4; ++b) {
            uint4 w = philox4x32_10(ctr_of((uint32_t)b, U.v, U.event_id), key);
            float z0, z1, z2, z3;
            box_muller_f(w.x, w.y, z0, z1);
            box_muller_f(w.z, w.w, z2, z3);
            float zz[4] = {z0, z1, z2, z3};
            for (int t = 0; t < 4 && 4 * b + t < n; ++t) s[4 * b + t] = fmaf(P.sigma_jet, zz[t], 1.0f);
        }
    }
    float a[MAX_JETS], q2[MAX_JETS][MAX_JETS];
    for (int i = 0; i < n; ++i) a[i] = __fmul_rn(__fmul_rn(s[i], s[i]), minkowski_dot2(jf[i], jf[i]));
    for (int i = 0; i < n; ++i)
        for (int jj = i + 1; jj < n; ++jj)
            q2[i][jj] = q2[jj][i] = 2.0f * __fmul_rn(__fmul_rn(s[i], s[jj]), minkowski_dot2(jf[i], jf[jj]));
    const float c_t = -P.mt * P.inv_sigma_t, c_w = -P.mW * P.inv_sigma_W;
    // pass 1: FP32 minimum; pass 2: the screened candidates, in enumeration order
    float best = CUDART_INF_F;
    for (int pass = 0; pass < 2; ++pass) {
        int nl = 0;
        int code[32];
        bool overflow = false;
        for (int k = 0; k < n; ++k)
            for (int i = 0; i < n; ++i) {
                if (i == k) continue;
                for (int jj = i + 1; jj < n; ++jj) {
                    if (jj == k) continue;
                    float pw = __fadd_rn(__fadd_rn(a[i], a[jj]), q2[i][jj]);
                    float mwf = __fmul_rn(pw, rsqrt_approx(pw));
                    float dw = fmaf(mwf, P.inv_sigma_W, c_w);
                    float m2 = __fadd_rn(__fadd_rn(__fadd_rn(pw, a[k]), q2[i][k]), q2[jj][k]);
                    float mtf = __fmul_rn(m2, rsqrt_approx(m2));
                    float dt = fmaf(mtf, P.inv_sigma_t, c_t);
                    float c = fmaf(dt, dt, __fmul_rn(dw, dw));
                    if (pass == 0) {
                        best = fminf(best, c);
                    } else if (c <= best + chi2_band(P, best) + chi2_band(P, c)) {
                        if (nl < 32) code[nl++] = (k << 8) | (i << 4) | jj;
                        else overflow = true;
                    }
                }
            }
        if (pass == 0) continue;
        if (overflow) break;  // full enumeration below
        double chi2 = CUDART_INF;
        for (int t = 0; t < nl; ++t) {
            const int k = code[t] >> 8, i = (code[t] >> 4) & 15, jj = code[t] & 15;
            double W[4], T[4];
            v4_add_d(U.j(i), U.j(jj), W);
            v4_add_d(W, U.j(k), T);
            double m_w = mass_d(W), m_t = mass_d(T);
            double dt = (m_t - P.dmt) / P.dsigma_t;
            double dwd = (m_w - P.dmW) / P.dsigma_W;
            double c = dt * dt + dwd * dwd;
            if (c < chi2) {
                chi2 = c;
                *mtop = m_t;
                *mw = m_w;
            }
        }
        return chi2;
    }
    // screen overflow: every candidate in FP64
    double best_d = CUDART_INF;
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            for (int jj = i + 1; jj < n; ++jj) {
                if (jj == k) continue;
                double W[4], T[4];
                v4_add_d(U.j(i), U.j(jj), W);
                v4_add_d(W, U.j(k), T);
                double m_w = mass_d(W), m_t = mass_d(T);
                double dt = (m_t - P.dmt) / P.dsigma_t;
                double dwd = (m_w - P.dmW) / P.dsigma_W;
                double c = dt * dt + dwd * dwd;
                if (c < best_d) {
                    best_d = c;
                    *mtop = m_t;
                    *mw = m_w;
                }
            }
        }
    return best_d;
}

// Dilepton unit with the definition's FP64 arithmetic (user order).
static __device__ __noinline__ int dilep_unit_fp64(const Plan& P, const Cols& C, uint32_t e, LazyUnitD& U,
                                                   unsigned s1bits, float4* reco, int* bin, double* score)
{
    const float2 mf = C.met[e];
    double l1[4], l2[4];
    U.lepton(0, C.lep[2 * (uint64_t)e], l1);
    U.lepton(1, C.lep[2 * (uint64_t)e + 1], l2);
    const unsigned btag = C.btag[e];
    bool done = false;
    DilepResD r;
    auto jet = [&U](int i) { return U.j(i); };
    int f = P.n_cuts;
    for (int c = 0; c < P.n_cuts; ++c) {
        bool pass;
        if (P.stage1 >> c & 1u) {
            pass = s1bits >> c & 1u;
        } else if (P.kind[c] == CUT_MET_MIN) {
            U.met(mf);
            pass = sqrt(U.metx * U.metx + U.mety * U.mety) > P.dp0[c];
        } else if (P.kind[c] == CUT_LEP_PT_MIN) {
            pass = sqrt(l1[0] * l1[0] + l1[1] * l1[1]) > P.dp0[c];
        } else if (P.kind[c] == CUT_W_NU_SOLVABLE) {
            U.met(mf);
            double pz;
            pass = w_pz_d(l1, U.metx, U.mety, P.dmW, &pz) != 0;
        } else {
            if (!done) {
                U.met(mf);
                r = dilep_reco_d(P, U.n, btag, l1, l2, U.metx, U.mety, jet);
                done = true;
            }
            if (P.kind[c] == CUT_DILEP_SOLVABLE) pass = r.ok;
            else if (P.kind[c] == CUT_HIGGS_WINDOW) pass = r.h_ok && r.m_bb > P.dp0[c] && r.m_bb < P.dp1[c];
            else pass = false;
        }
        if (!pass) {
            f = c;
            break;
        }
    }
    if (f == P.n_cuts) {
        if (!done) {
            U.met(mf);
            r = dilep_reco_d(P, U.n, btag, l1, l2, U.metx, U.mety, jet);
        }
        *bin = hist_bin_d(P, r.m_bb);
        *reco = make_float4((float)r.m_bb, (float)r.m_t1, (float)r.m_t2, (float)r.m_tt);
        if (score) *score = r.m_tt;
    }
    return f;
}

// One unit with the definition's FP64 decisions (user order; stage-1
// results are already exact and are taken from s1bits).  Returns the number
// of leading cuts passed; reco, bin and (when given) the fit score -- the
// chi2 of the analysis's fit, or m_ttbar of the dilepton solution -- are set
// when all pass.  Called through unit_fp64 / unit_fp64_scored below.
__device__ __forceinline__ int unit_fp64_body(const Plan& P, const Cols& C, uint32_t e, uint64_t event_id,
                                              uint64_t seed, uint32_t v, unsigned s1bits, float4* reco, int* bin,
                                              double* score)
{
    LazyUnitD U;
    U.init(P, C, e, event_id, seed, v);
    if (P.model == MODEL_DILEP) return dilep_unit_fp64(P, C, e, U, s1bits, reco, bin, score);
    const float2 mf = C.met[e];
    bool top_done = false, full_done = false;
    double chi2 = 0.0, mtop = 0.0, mw = 0.0;
    FullFitD ff;
    double lep[4];
    U.lepton(0, C.lep[e], lep);
    int f = P.n_cuts;
    for (int c = 0; c < P.n_cuts; ++c) {
        bool pass;
        if (P.stage1 >> c & 1u) {
            pass = s1bits >> c & 1u;
        } else if (P.kind[c] == CUT_MET_MIN) {
            U.met(mf);
            pass = sqrt(U.metx * U.metx + U.mety * U.mety) > P.dp0[c];
        } else if (P.kind[c] == CUT_LEP_PT_MIN) {
            pass = sqrt(lep[0] * lep[0] + lep[1] * lep[1]) > P.dp0[c];
        } else if (P.kind[c] == CUT_W_NU_SOLVABLE) {
            U.met(mf);
            double pz;
            pass = w_pz_d(lep, U.metx, U.mety, P.dmW, &pz) != 0;
        } else if (P.kind[c] == CUT_HADTOP_CHI2_MAX) {
            if (!top_done) {
                chi2 = hadtop_screened_d(P, U, &mtop, &mw);
                top_done = true;
            }
            pass = chi2 < P.dp0[c];
        } else if (P.kind[c] == CUT_TTBAR_CHI2_MAX) {
            if (!full_done) {
                U.met(mf);
                ff = ttbar_full_d(P, U, lep, U.metx, U.mety, nullptr, -1);
                full_done = true;
            }
            pass = ff.chi2 < P.dp0[c];
        } else {
            pass = false;
        }
        if (!pass) {
            f = c;
            break;
        }
    }
    if (f == P.n_cuts && P.has_full) {
        U.met(mf);
        if (!full_done) ff = ttbar_full_d(P, U, lep, U.metx, U.mety, nullptr, -1);
        const double met = sqrt(U.metx * U.metx + U.mety * U.mety);
        *bin = hist_bin_d(P, ff.mtop_had);
        *reco = make_float4((float)ff.mtop_had, (float)ff.mtop_lep, (float)ff.pz, (float)met);
        if (score) *score = ff.chi2;
    } else if (f == P.n_cuts) {
        if (!top_done) chi2 = hadtop_screened_d(P, U, &mtop, &mw);
        U.met(mf);
        double pz;
        w_pz_d(lep, U.metx, U.mety, P.dmW, &pz);
        double met = sqrt(U.metx * U.metx + U.mety * U.mety);
        *bin = hist_bin_d(P, mtop);
        *reco = make_float4((float)mtop, (float)mw, (float)pz, (float)met);
        if (score) *score = chi2;
    }
    return f;
}

// Out of line, without and with the score: the stage-2 kernels call the
// former on their rarely taken paths, and an extra argument there cost their
// register allocation spills in the unit loop (measured).
static __device__ __noinline__ int unit_fp64(const Plan& P, const Cols& C, uint32_t e, uint64_t event_id, uint64_t seed,
                                             uint32_t v, unsigned s1bits, float4* reco, int* bin)
{
    return unit_fp64_body(P, C, e, event_id, seed, v, s1bits, reco, bin, nullptr);
}

static __device__ __noinline__ int unit_fp64_scored(const Plan& P, const Cols& C, uint32_t e, uint64_t event_id,
                                                    uint64_t seed, uint32_t v, unsigned s1bits, float4* reco, int* bin,
                                                    double* score)
{
    return unit_fp64_body(P, C, e, event_id, seed, v, s1bits, reco, bin, score);
}

// The records of one block of events (thread = event e, valid if `has`),
// written from `base` on in (event, level) order.  They are assembled in
// shared memory, REC_STAGE at a time, and copied out as consecutive 32-bit
// words, so that a warp's stores cover whole sectors.  Every thread calls.
constexpr int REC_STAGE = 1536;  // records per round (36 KB)

__device__ inline void write_block_records(const Plan& P, const Cols& C, const Out& O, uint32_t e, bool has,
                                           int maxf, unsigned long long base)
{
    __shared__ uint32_t s_rec[REC_STAGE * 6];
    const unsigned cnt = has ? rec_count(P, maxf) : 0u;
    unsigned long long total;
    const unsigned long long excl = block_excl_scan(cnt, &total);
    float vals[4];
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned lv = 0;
    if (cnt) {
        lv = P.rec_levels & (maxf >= 32 ? 0xffffffffu : ((1u << maxf) - 1u));
        if ((lv >> (P.n_cuts - 1) & 1u) && O.reco) r = O.reco[e];
        record_values(P, C, e, r, 0, vals);
    }
    for (unsigned long long r0 = 0; r0 < total; r0 += REC_STAGE) {
        unsigned long long j = excl;
        for (unsigned bits = lv; bits; bits &= bits - 1u, ++j) {
            if (j < r0 || j >= r0 + REC_STAGE) continue;
            const int level = __ffs(bits) - 1;
            uint32_t* w = s_rec + (j - r0) * 6;
            w[0] = e;
            w[1] = (uint32_t)level;
            for (int i = 0; i < 4; ++i) {
                const int var = P.rec_var[i];
                float x = vals[i];
                if (var >= VAR_RECO0 && var < VAR_RECO0 + 4 && level != P.n_cuts - 1) x = 0.f;
                if (var >= VAR_RECO0 && var < VAR_RECO0 + 4 && level == P.n_cuts - 1)
                    x = var == VAR_RECO0 ? r.x : var == VAR_RECO0 + 1 ? r.y : var == VAR_RECO0 + 2 ? r.z : r.w;
                w[2 + i] = __float_as_uint(x);
            }
        }
        __syncthreads();
        const unsigned long long nr = min((unsigned long long)REC_STAGE, total - r0);
        const unsigned long long k0 = base + r0;
        unsigned long long nw = 0;
        if (k0 < O.rec_cap) nw = 6ull * min(nr, O.rec_cap - k0);
        uint32_t* dst = (uint32_t*)O.rec + 6ull * k0;
        for (unsigned long long i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = s_rec[i];
        __syncthreads();
    }
}

// In place: pre[0..n) := exclusive prefix, pre[n] := total (also *total_out
// when given).  One block of 1024 threads, each over a contiguous segment.
__device__ inline void scan_blocks(unsigned long long* pre, unsigned n, unsigned long long* total_out)
{
    const unsigned seg = (n + blockDim.x - 1) / blockDim.x;
    const unsigned lo = min(n, threadIdx.x * seg), hi = min(n, lo + seg);
    unsigned long long sum = 0;
    for (unsigned i = lo; i < hi; ++i) sum += pre[i];
    unsigned long long total;
    unsigned long long run = block_excl_scan(sum, &total);
    for (unsigned i = lo; i < hi; ++i) {
        const unsigned long long x = pre[i];
        pre[i] = run;
        run += x;
    }
    if (threadIdx.x == 0) {
        pre[n] = total;
        if (total_out) *total_out = total;
    }
}

// ------------------------------------------------------------------ pending events
// An event with flagged units keeps the compensated sum of its unflagged
// survivors in a pending slot; its flagged units go to the recheck list,
// contiguous and in variation order.  The recheck stores each unit's FP64
// result per entry, and the completion pass adds them to the slot's partial
// sum in entry order (deterministic, compensated) and writes the event.
__device__ __forceinline__ void write_event(const Out& O, uint32_t e, unsigned cnt, float4 sum, float4 comp)
{
    if (O.mask) O.mask[e] = cnt > 0;
    if (O.n_surv) O.n_surv[e] = (uint16_t)cnt;
    if (O.reco) {
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (cnt) {
            float inv = (float)cnt;
            r.x = __fdiv_rn(__fadd_rn(sum.x, comp.x), inv);
            r.y = __fdiv_rn(__fadd_rn(sum.y, comp.y), inv);
            r.z = __fdiv_rn(__fadd_rn(sum.z, comp.z), inv);
            r.w = __fdiv_rn(__fadd_rn(sum.w, comp.w), inv);
        }
        O.reco[e] = r;
    }
}

// Event e rejected by its stage-1 cuts: every variation passes cuts 0..f1-1.
__device__ __forceinline__ void write_stage1_event(const Plan& P, const Cols& C, const Out& O, uint32_t e, int f1)
{
    write_zero_event(O, e);
    if (O.maxf) O.maxf[e] = (uint8_t)f1;
}

__device__ __forceinline__ void acc4(float4& s, float4& c, float4 x)
{
    float t, e;
    two_sum(s.x, x.x, t, e); s.x = t; c.x = __fadd_rn(c.x, e);
    two_sum(s.y, x.y, t, e); s.y = t; c.y = __fadd_rn(c.y, e);
    two_sum(s.z, x.z, t, e); s.z = t; c.z = __fadd_rn(c.z, e);
    two_sum(s.w, x.w, t, e); s.w = t; c.w = __fadd_rn(c.w, e);
}

// Adds the compensated sum (s2, c2) to (s, c).
__device__ __forceinline__ void merge4(float4& s, float4& c, float4 s2, float4 c2)
{
    float t, e;
    two_sum(s.x, s2.x, t, e); s.x = t; c.x = __fadd_rn(__fadd_rn(c.x, c2.x), e);
    two_sum(s.y, s2.y, t, e); s.y = t; c.y = __fadd_rn(__fadd_rn(c.y, c2.y), e);
    two_sum(s.z, s2.z, t, e); s.z = t; c.z = __fadd_rn(__fadd_rn(c.z, c2.z), e);
    two_sum(s.w, s2.w, t, e); s.w = t; c.w = __fadd_rn(__fadd_rn(c.w, c2.w), e);
}

__device__ __forceinline__ float4 shfl_down4(float4 a, int o)
{
    a.x = __shfl_down_sync(0xffffffffu, a.x, o);
    a.y = __shfl_down_sync(0xffffffffu, a.y, o);
    a.z = __shfl_down_sync(0xffffffffu, a.z, o);
    a.w = __shfl_down_sync(0xffffffffu, a.w, o);
    return a;
}

// Warp-wide compensated sum and count (fixed tree, lane 0 holds the totals);
// every lane of the warp must call it.
__device__ __forceinline__ void warp_merge4(float4& s, float4& c, unsigned& n)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float4 s2 = shfl_down4(s, o), c2 = shfl_down4(c, o);
        const unsigned n2 = __shfl_down_sync(0xffffffffu, n, o);
        merge4(s, c, s2, c2);
        n += n2;
    }
}

// Reserves nflag recheck entries and a pending slot for event e (one thread).
// Returns false when the list is full (the entries must then be evaluated
// by the caller).
__device__ __forceinline__ bool reserve_pending(const Scratch& S, unsigned nflag, unsigned cnt, float4 sum,
                                                float4 comp, unsigned& base, unsigned& slot)
{
    base = atomicAdd(S.rc_count, nflag);
    if (base + nflag > S.rc_cap) {
        atomicOr(S.err, ERR_RECHECK_FULL);
        return false;
    }
    // entries below the largest end of a successful reservation are all
    // written; every reservation after a failed one fails too
    atomicMax(S.rc_valid, base + nflag);
    slot = atomicAdd(S.pend_count, 1u);
    S.pend_cnt[slot] = cnt;
    S.pend_rng[slot] = make_uint2(base, nflag);
    S.pend_sum[slot] = sum;
    S.pend_comp[slot] = comp;
    return true;
}

__device__ __forceinline__ RcEntry rc_entry(const Scratch& S, uint32_t e, uint32_t v, unsigned s1bits, unsigned slot)
{
    RcEntry r;
    r.event = e;
    r.vbits = v | (s1bits << 16);
    r.slot = slot;
    r.chunk = S.chunk;
    return r;
}

// Registers an event with nflag flagged units (their variations in vs[], in
// increasing order).  Evaluates them here in FP64 when the list is full.
static __device__ __noinline__ void pend_event(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t e,
                           uint64_t event_id, uint64_t seed, unsigned s1bits, unsigned cnt, float4 sum,
                           float4 comp, const uint16_t* vs, int nflag, unsigned long long* fc, unsigned* hist)
{
    unsigned base, slot;
    if (reserve_pending(S, (unsigned)nflag, cnt, sum, comp, base, slot)) {
        for (int i = 0; i < nflag; ++i) S.rc[base + i] = rc_entry(S, e, vs[i], s1bits, slot);
        return;
    }
    for (int i = 0; i < nflag; ++i) {
        float4 reco;
        int bin = 0;
        int f = unit_fp64(P, C, e, event_id, seed, vs[i], s1bits, &reco, &bin);
        atomicAdd(&fc[f], 1ull);
        if (O.maxf) O.maxf[e] = (uint8_t)max((int)O.maxf[e], f);
        if (f == P.n_cuts) {
            ++cnt;
            atomicAdd(&hist[bin], 1u);
            acc4(sum, comp, reco);
        }
    }
    atomicAdd(O.rc_total, (unsigned long long)nflag);
    write_event(O, e, cnt, sum, comp);
}

// Completion of pending slot s by one warp: the unflagged partial sum plus the
// passing entries' FP64 results.  Lane 0 returns the totals and the event.
__device__ __forceinline__ void finish_pending(const Scratch& S, int n_cuts, unsigned s, unsigned& cnt, float4& sum,
                                               float4& comp, int& maxf, RcEntry& first)
{
    const unsigned lane = threadIdx.x & 31u;
    const uint2 rg = S.pend_rng[s];
    sum = make_float4(0.f, 0.f, 0.f, 0.f);
    comp = sum;
    cnt = 0;
    maxf = -1;
    for (unsigned i = lane; i < rg.y; i += 32) {
        const int f = S.rc_res[rg.x + i].f;
        maxf = max(maxf, f);
        if (f == n_cuts) {
            ++cnt;
            acc4(sum, comp, S.rc_reco[rg.x + i]);
        }
    }
    warp_merge4(sum, comp, cnt);
    maxf = __reduce_max_sync(0xffffffffu, maxf);
    if (lane == 0) {
        float4 ps = S.pend_sum[s], pc = S.pend_comp[s];
        merge4(ps, pc, sum, comp);
        sum = ps;
        comp = pc;
        cnt += S.pend_cnt[s];
        first = S.rc[rg.x];
    }
}

// ------------------------------------------------------------------ tile epilogues
// Adds a warp's units to the block's cut flow, histogram and scheduler
// statistics with one shared-memory atomic per distinct value (lanes with the
// same first-failure index or bin are combined by __match_any_sync).
template <bool BEST = false>
__device__ __forceinline__ void warp_tally(const Plan& P, const UnitOut& r, unsigned long long* fc, unsigned* hist,
                                           CutStats* st)
{
    const unsigned am = __activemask();
    const unsigned lane = threadIdx.x & 31u;
    const unsigned g = __match_any_sync(am, r.f);
    if (r.f >= 0 && lane == (unsigned)(__ffs(g) - 1)) atomicAdd(&fc[r.f], (unsigned long long)__popc(g));
    const int hb = r.f == P.n_cuts && !BEST ? r.bin : -1;  // best-of: filled per event
    const unsigned gh = __match_any_sync(am, hb);
    if (hb >= 0 && lane == (unsigned)(__ffs(gh) - 1)) atomicAdd(&hist[hb], (unsigned)__popc(gh));
    const bool leader = lane == (unsigned)(__ffs(am) - 1);
    const unsigned ct = __reduce_add_sync(am, r.cyc_top), cm = __reduce_add_sync(am, r.cyc_met);
    const unsigned nc = __reduce_add_sync(am, r.cands);
    if (leader && nc) atomicAdd(&st->cands, (unsigned long long)nc);
    for (unsigned bits = P.stage2; bits; bits &= bits - 1) {
        const int c = __ffs(bits) - 1;
        const unsigned ne = __popc(__ballot_sync(am, r.evald >> c & 1u));
        const unsigned np = __popc(__ballot_sync(am, r.passd >> c & 1u));
        if (leader && ne) {
            atomicAdd(&st->evaluated[c], ne);
            atomicAdd(&st->passed[c], np);
            atomicAdd(&st->cost[c], (unsigned long long)(heavy_cut(P.kind[c]) ? ct : cm));
        }
    }
}

// Per-cut records: the most cuts passed by the event's unflagged units
// (the rechecked ones are added when their event completes).  Out of line:
// inlined into the tile epilogue, this never-taken path cost the stage-2
// kernels about 1 % (measured).  warp: the calling warp shares the work.
static __device__ __noinline__ void store_maxf(const int* uf, uint32_t V, uint8_t* dst, bool warp)
{
    int m = 0;
    if (warp) {
        for (uint32_t v = threadIdx.x & 31u; v < V; v += 32) m = max(m, uf[v]);
        m = __reduce_max_sync(0xffffffffu, m);
        if ((threadIdx.x & 31u) == 0) *dst = (uint8_t)m;
    } else {
        for (uint32_t v = 0; v < V; ++v) m = max(m, uf[v]);
        *dst = (uint8_t)m;
    }
}

// Compensated sum and count over the G lanes of a lane group (G a power of
// two <= 32; fixed tree, the group's first lane holds the totals).  Every
// lane of the warp calls it.
template <int G>
__device__ __forceinline__ void group_merge4(float4& s, float4& c, unsigned& n)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) {
        float4 s2, c2;
        s2.x = __shfl_down_sync(0xffffffffu, s.x, o, G);
        s2.y = __shfl_down_sync(0xffffffffu, s.y, o, G);
        s2.z = __shfl_down_sync(0xffffffffu, s.z, o, G);
        s2.w = __shfl_down_sync(0xffffffffu, s.w, o, G);
        c2.x = __shfl_down_sync(0xffffffffu, c.x, o, G);
        c2.y = __shfl_down_sync(0xffffffffu, c.y, o, G);
        c2.z = __shfl_down_sync(0xffffffffu, c.z, o, G);
        c2.w = __shfl_down_sync(0xffffffffu, c.w, o, G);
        const unsigned n2 = __shfl_down_sync(0xffffffffu, n, o, G);
        merge4(s, c, s2, c2);
        n += n2;
    }
}

template <int G>
__device__ __forceinline__ int group_max(int x)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o, G));
    return x;
}

// Per-event reduction by groups of G lanes (G = 8, 16 or 32): lanes strided
// over the event's variations, a fixed combining tree per group, so that the
// events of a tile are reduced in parallel rather than one thread per event
// in turn.  rank and size describe the calling group of threads (size a
// multiple of 32, every thread calls).
template <int G>
__device__ inline void reduce_events_grp(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                                         uint64_t seed, uint64_t first_id, int ne, const uint32_t* evid,
                                         const uint32_t* bits, const int* uf, const float4* ureco,
                                         unsigned long long* fc, unsigned* hist, int rank, int size)
{
    const unsigned lane = (unsigned)rank & 31u;
    const unsigned gl = lane & (unsigned)(G - 1);
    const unsigned g0 = lane - gl;                            // first lane of the group
    const unsigned gbits = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    const unsigned below = (1u << gl) - 1u;
    constexpr int GPW = 32 / G;                               // groups per warp
    const int gid = (rank >> 5) * GPW + (int)(lane / G);
    const int ngroups = (size >> 5) * GPW;
    for (int ev0 = 0; ev0 < ne; ev0 += ngroups) {
        const int ev = ev0 + gid;
        const bool valid = ev < ne;
        const uint32_t e = valid ? evid[ev] : 0u;
        const int u0 = ev * (int)V;
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f), comp = sum;
        unsigned cnt = 0, nflag = 0;
        int mf = 0;
        for (uint32_t v0 = 0; v0 < V; v0 += G) {
            const uint32_t v = v0 + gl;
            const bool in = valid && v < V;
            const int f = in ? uf[u0 + (int)v] : -1;
            nflag += __popc((__ballot_sync(0xffffffffu, in && f < 0) >> g0) & gbits);
            if (in && f == P.n_cuts) {
                ++cnt;
                acc4(sum, comp, ureco[u0 + (int)v]);
            }
            mf = max(mf, f);
        }
        group_merge4<G>(sum, comp, cnt);
        if (O.maxf) {
            mf = group_max<G>(mf);
            if (valid && gl == 0) O.maxf[e] = (uint8_t)max(mf, 0);
        }
        // nflag and valid are the same on a group's lanes, not across the warp:
        // every lane runs the shuffles and ballots below, the writes are guarded
        if (nflag == 0 && valid && gl == 0) write_event(O, e, cnt, sum, comp);
        if (!__any_sync(0xffffffffu, nflag != 0 && valid)) continue;
        unsigned base = 0, slot = 0;
        int ok = 0;
        if (nflag && valid && gl == 0) ok = reserve_pending(S, nflag, cnt, sum, comp, base, slot);
        ok = __shfl_sync(0xffffffffu, ok, g0);
        base = __shfl_sync(0xffffffffu, base, g0);
        slot = __shfl_sync(0xffffffffu, slot, g0);
        const bool listed = nflag && valid && ok;
        for (uint32_t v0 = 0; v0 < V; v0 += G) {
            const uint32_t v = v0 + gl;
            const bool fl = listed && v < V && uf[u0 + (int)v] < 0;
            const unsigned m = (__ballot_sync(0xffffffffu, fl) >> g0) & gbits;
            if (fl) S.rc[base + __popc(m & below)] = rc_entry(S, e, v, bits[ev], slot);
            base += __popc(m);
        }
        // list full: the group's lanes evaluate the flagged units in FP64
        const bool inline_fp64 = nflag && valid && !ok;
        if (!__any_sync(0xffffffffu, inline_fp64)) continue;
        float4 s2 = make_float4(0.f, 0.f, 0.f, 0.f), c2 = s2;
        unsigned n2 = 0;
        int mf2 = 0;
        for (uint32_t v0 = 0; v0 < V; v0 += G) {
            const uint32_t v = v0 + gl;
            if (inline_fp64 && v < V && uf[u0 + (int)v] < 0) {
                float4 reco;
                int bin = 0;
                const int f2 = unit_fp64(P, C, e, first_id + e, seed, v, bits[ev], &reco, &bin);
                atomicAdd(&fc[f2], 1ull);
                mf2 = max(mf2, f2);
                if (f2 == P.n_cuts) {
                    ++n2;
                    atomicAdd(&hist[bin], 1u);
                    acc4(s2, c2, reco);
                }
            }
        }
        __syncwarp();
        group_merge4<G>(s2, c2, n2);
        mf2 = group_max<G>(mf2);
        if (inline_fp64 && gl == 0) {
            if (O.maxf) O.maxf[e] = (uint8_t)max((int)O.maxf[e], mf2);
            merge4(sum, comp, s2, c2);
            atomicAdd(O.rc_total, (unsigned long long)nflag);
            write_event(O, e, cnt + n2, sum, comp);
        }
    }
}

// ------------------------------------------------------------------ best-of-variations
// Per-event best-of-variations (Sect. 4, ttH_sci): of an event's surviving
// variations the one with the smallest fit score (the triplet chi2 of Eq. 1,
// the full Eq. 1 chi2 with the full fit, m_ttbar of the dilepton solution),
// ties to the lowest variation.  Recheck entries that carry RC_SCORE_ONLY in
// vbits are certain survivors listed only for their FP64 score: the cut flow
// already holds them.
constexpr uint32_t RC_SCORE_ONLY = 0x8000u;

// Half-width of an interval certain to hold the definition's FP64 score of an
// unflagged survivor whose FP32 score is s: the chi2 band of the triplet fit;
// the full fit and the dilepton m_ttbar are FP64 values rounded to FP32
// (2^-24 relative) whose solution choice already keeps a 1e-8 relative margin.
__device__ __forceinline__ float best_band(const Plan& P, float s)
{
    if (P.model == MODEL_SEMILEP && !P.has_full) return chi2_band(P, s);
    return P.safety * (1.2e-7f * fabsf(s)) + 1.0e-30f;
}

__device__ __forceinline__ void write_event_best(const Out& O, uint32_t e, unsigned cnt, unsigned vb, float4 reco)
{
    if (O.mask) O.mask[e] = cnt > 0;
    if (O.n_surv) O.n_surv[e] = (uint16_t)cnt;
    if (O.reco) O.reco[e] = cnt ? reco : make_float4(0.f, 0.f, 0.f, 0.f);
    if (O.best_v) O.best_v[e] = cnt ? (uint16_t)vb : (uint16_t)0xffffu;
}

template <int G>
__device__ __forceinline__ unsigned group_sum(unsigned x)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, G);
    return x;
}

// Lexicographic minimum of (k, v) over a lane group; every lane of the group
// receives it.
template <int G, class T>
__device__ __forceinline__ void group_argmin(T& k, unsigned& v)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) {
        const T k2 = __shfl_xor_sync(0xffffffffu, k, o, G);
        const unsigned v2 = __shfl_xor_sync(0xffffffffu, v, o, G);
        if (k2 < k || (k2 == k && v2 < v)) {
            k = k2;
            v = v2;
        }
    }
}

// Per-event best-of reduction by groups of G lanes (as reduce_events_grp).
// Among the certain survivors, vmin has the smallest upper score bound umin;
// the event is decided here when no unit is flagged and every other
// survivor's lower bound lies above umin.  Otherwise the flagged units and
// the survivors whose interval reaches umin (vmin among them) are listed:
// the best of the event is one of them, chosen in FP64 at completion.
template <int G>
__device__ inline void reduce_events_best(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                                          uint64_t seed, uint64_t first_id, int ne, const uint32_t* evid,
                                          const uint32_t* bits, const int* uf, const float4* ureco,
                                          const float2* usc, unsigned long long* fc, unsigned* hist, int rank,
                                          int size)
{
    const unsigned lane = (unsigned)rank & 31u;
    const unsigned gl = lane & (unsigned)(G - 1);
    const unsigned g0 = lane - gl;
    const unsigned gbits = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    const unsigned below = (1u << gl) - 1u;
    constexpr int GPW = 32 / G;
    const int gid = (rank >> 5) * GPW + (int)(lane / G);
    const int ngroups = (size >> 5) * GPW;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int ev0 = 0; ev0 < ne; ev0 += ngroups) {
        const int ev = ev0 + gid;
        const bool valid = ev < ne;
        const uint32_t e = valid ? evid[ev] : 0u;
        const int u0 = ev * (int)V;
        unsigned cnt = 0, nflag = 0;
        int mf = 0;
        float umin = CUDART_INF_F;
        unsigned vmin = 0xffffffffu;
        for (uint32_t v0 = 0; v0 < V; v0 += G) {
            const uint32_t v = v0 + gl;
            const bool in = valid && v < V;
            const int f = in ? uf[u0 + (int)v] : -1;
            nflag += __popc((__ballot_sync(0xffffffffu, in && f < 0) >> g0) & gbits);
            if (in && f == P.n_cuts) {
                ++cnt;
                const float sc = usc[u0 + (int)v].x;
                const float up = __fadd_ru(sc, best_band(P, sc));
                if (up < umin) {
                    umin = up;
                    vmin = v;
                }
            }
            mf = max(mf, f);
        }
        cnt = group_sum<G>(cnt);
        group_argmin<G>(umin, vmin);
        // a survivor is close when its interval reaches umin
        auto close = [&](uint32_t v) {
            const float sc = usc[u0 + (int)v].x;
            return v == vmin || __fsub_rd(sc, best_band(P, sc)) <= umin;
        };
        unsigned nclose = 0;
        for (uint32_t v0 = 0; v0 < V; v0 += G) {
            const uint32_t v = v0 + gl;
            if (valid && v < V && v != vmin && uf[u0 + (int)v] == P.n_cuts && close(v)) ++nclose;
        }
        nclose = group_sum<G>(nclose);
        if (O.maxf) {
            mf = group_max<G>(mf);
            if (valid && gl == 0) O.maxf[e] = (uint8_t)max(mf, 0);
        }
        const bool certain = nflag == 0 && nclose == 0;
        if (valid && certain && gl == 0) {
            float4 r = zero;
            if (cnt) {
                const int u = u0 + (int)vmin;
                r = ureco[u];
                atomicAdd(&hist[__float_as_int(usc[u].y)], 1u);
            }
            write_event_best(O, e, cnt, vmin, r);
        }
        const bool pend = valid && !certain;
        if (!__any_sync(0xffffffffu, pend)) continue;
        const unsigned nlist = nflag + (cnt ? nclose + 1u : 0u);
        unsigned base = 0, slot = 0;
        int ok = 0;
        if (pend && gl == 0) ok = reserve_pending(S, nlist, cnt, zero, zero, base, slot);
        ok = __shfl_sync(0xffffffffu, ok, g0);
        base = __shfl_sync(0xffffffffu, base, g0);
        slot = __shfl_sync(0xffffffffu, slot, g0);
        const bool listed = pend && ok;
        for (uint32_t v0 = 0; v0 < V; v0 += G) {
            const uint32_t v = v0 + gl;
            const int f = listed && v < V ? uf[u0 + (int)v] : -2;
            const bool fl = f == -1;
            const bool so = f == P.n_cuts && close(v);
            const unsigned m = (__ballot_sync(0xffffffffu, fl || so) >> g0) & gbits;
            if (fl || so) S.rc[base + __popc(m & below)] = rc_entry(S, e, v | (so ? RC_SCORE_ONLY : 0u), bits[ev], slot);
            base += __popc(m);
        }
        // list full: the group's lanes evaluate the listed units in FP64
        const bool inl = pend && !ok;
        if (!__any_sync(0xffffffffu, inl)) continue;
        double bs = CUDART_INF;
        unsigned bv = 0xffffffffu, n2 = 0, nrc = 0;
        float4 br = zero;
        int bb = 0, mf2 = 0;
        for (uint32_t v0 = 0; v0 < V; v0 += G) {
            const uint32_t v = v0 + gl;
            const int f = inl && v < V ? uf[u0 + (int)v] : -2;
            const bool fl = f == -1;
            if (!(fl || (f == P.n_cuts && close(v)))) continue;
            float4 reco;
            int bin = 0;
            double sc = CUDART_INF;
            const int f2 = unit_fp64_scored(P, C, e, first_id + e, seed, v, bits[ev], &reco, &bin, &sc);
            ++nrc;
            if (fl) {
                atomicAdd(&fc[f2], 1ull);
                mf2 = max(mf2, f2);
                if (f2 == P.n_cuts) ++n2;
            }
            if (f2 == P.n_cuts && sc < bs) {  // a lane's variations increase: ties keep the lower
                bs = sc;
                bv = v;
                br = reco;
                bb = bin;
            }
        }
        __syncwarp();
        unsigned kv = bv;
        group_argmin<G>(bs, kv);
        const int wl = (int)(g0 + (kv & (unsigned)(G - 1)));  // the lane that evaluated the winner
        br.x = __shfl_sync(0xffffffffu, br.x, wl);
        br.y = __shfl_sync(0xffffffffu, br.y, wl);
        br.z = __shfl_sync(0xffffffffu, br.z, wl);
        br.w = __shfl_sync(0xffffffffu, br.w, wl);
        bb = __shfl_sync(0xffffffffu, bb, wl);
        n2 = group_sum<G>(n2);
        nrc = group_sum<G>(nrc);
        mf2 = group_max<G>(mf2);
        if (inl && gl == 0) {
            if (O.maxf) O.maxf[e] = (uint8_t)max((int)O.maxf[e], mf2);
            atomicAdd(O.rc_total, (unsigned long long)nrc);
            if (kv != 0xffffffffu) atomicAdd(&hist[bb], 1u);
            write_event_best(O, e, cnt + n2, kv, br);
        }
    }
}

// Completion of best-of pending slot s by one warp: the FP64 argmin over the
// listed survivors; hist is the run's histogram.  Lane 0 writes the event.
__device__ __forceinline__ void finish_pending_best(const Out& O, const Scratch& S, int n_cuts, unsigned s,
                                                    unsigned long long* hist, int& maxf, RcEntry& first)
{
    const unsigned lane = threadIdx.x & 31u;
    const uint2 rg = S.pend_rng[s];
    unsigned cnt = 0, bv = 0xffffffffu, bi = 0;
    double bs = CUDART_INF;
    maxf = -1;
    for (unsigned i = lane; i < rg.y; i += 32) {
        const RcRes q = S.rc_res[rg.x + i];
        const uint32_t vb = S.rc[rg.x + i].vbits;
        const unsigned v = vb & 0x7fffu;
        if (!(vb & RC_SCORE_ONLY)) {
            maxf = max(maxf, q.f);
            if (q.f == n_cuts) ++cnt;
        }
        if (q.f == n_cuts && (q.score < bs || (q.score == bs && v < bv))) {
            bs = q.score;
            bv = v;
            bi = rg.x + i;
        }
    }
    cnt = group_sum<32>(cnt);
    maxf = __reduce_max_sync(0xffffffffu, maxf);
    unsigned key = bv;
    group_argmin<32>(bs, key);
    // the winner's entry index: the lane that held it publishes it
    const unsigned holder = __ballot_sync(0xffffffffu, bv == key && key != 0xffffffffu);
    const unsigned wi = holder ? __shfl_sync(0xffffffffu, bi, __ffs(holder) - 1) : 0u;
    if (lane == 0) {
        first = S.rc[rg.x];
        cnt += S.pend_cnt[s];
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (key != 0xffffffffu) {
            r = S.rc_reco[wi];
            atomicAdd(&hist[S.rc_res[wi].bin], 1ull);
        }
        write_event_best(O, first.event, cnt, key, r);
    }
}

// Per-event reduction of a tile's units (BEST: best-of-variations, above;
// the mean otherwise): compensated sums of the surviving units' reconstructed
// quantities; events without flagged units are written,
// the others get a pending slot and their flagged units go to the recheck
// list.  Fewer than 5 variations: one thread per event, in variation order;
// otherwise a group of 8, 16 or 32 lanes per event (reduce_events_grp), so
// that no thread walks many variations while the others wait.  rank and size
// describe the calling group (size a multiple of 32, every thread calls).
template <bool BEST>
__device__ inline void reduce_tile_events(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                                          uint64_t seed, uint64_t first_id, int ne, const uint32_t* evid,
                                          const uint32_t* bits, const int* uf, const float4* ureco,
                                          const float2* usc, unsigned long long* fc, unsigned* hist, int rank,
                                          int size)
{
    if constexpr (BEST) {
        if (V > 16)
            reduce_events_best<32>(P, C, O, S, V, seed, first_id, ne, evid, bits, uf, ureco, usc, fc, hist, rank, size);
        else if (V > 8)
            reduce_events_best<16>(P, C, O, S, V, seed, first_id, ne, evid, bits, uf, ureco, usc, fc, hist, rank, size);
        else
            reduce_events_best<8>(P, C, O, S, V, seed, first_id, ne, evid, bits, uf, ureco, usc, fc, hist, rank, size);
        return;
    }
    if (V > 16) {
        reduce_events_grp<32>(P, C, O, S, V, seed, first_id, ne, evid, bits, uf, ureco, fc, hist, rank, size);
        return;
    }
    if (V > 8) {
        reduce_events_grp<16>(P, C, O, S, V, seed, first_id, ne, evid, bits, uf, ureco, fc, hist, rank, size);
        return;
    }
    if (V > 4) {
        reduce_events_grp<8>(P, C, O, S, V, seed, first_id, ne, evid, bits, uf, ureco, fc, hist, rank, size);
        return;
    }
    for (int ev = rank; ev < ne; ev += size) {
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f), comp = sum;
        unsigned cnt = 0;
        int nflag = 0;
        uint16_t vs[4];
        const uint32_t e = evid[ev];
        for (uint32_t v = 0; v < V; ++v) {
            const int u = ev * (int)V + (int)v;
            const int f = uf[u];
            if (f < 0) {
                vs[nflag++] = (uint16_t)v;
            } else if (f == P.n_cuts) {
                ++cnt;
                acc4(sum, comp, ureco[u]);
            }
        }
        if (O.maxf) store_maxf(uf + ev * (int)V, V, O.maxf + e, false);
        if (nflag == 0) write_event(O, e, cnt, sum, comp);
        else pend_event(P, C, O, S, e, first_id + e, seed, bits[ev], cnt, sum, comp, vs, nflag, fc, hist);
    }
}

// ------------------------------------------------------------------ thread groups of a tile
// A tile is processed either by the whole block or by one warp (its own
// tile, no block-wide barrier).
struct BlockGroup {
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct WarpGroup {
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ int size() const { return 32; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// ------------------------------------------------------------------ tile shared memory
// Shared memory of one semileptonic stage-2 tile: per event the packed Gram
// matrix (gst floats), lepton, MET, index and stage-1 bits; per unit its
// result.  The layout depends on the tile's (events, units, stride) only.
struct TileSmem {
    float* G;       // [ev][gst]
    float4* lep;    // [ev]
    float2* met;    // [ev]
    uint32_t* evid; // [ev]
    uint32_t* bits; // [ev]
    float4* ureco;  // [unit]
    float2* usc;    // [unit] fit score and (bits of) bin, best-of-variations only
    int* uf;        // [unit] f or -1
    char* top;      // the chi2 step's region (16-byte aligned, after the above)
};

// best: room for the units' scores (best-of-variations runs only).
__host__ __device__ inline size_t tile_smem_bytes(int ev, int units, int gst, bool best)
{
    return (size_t)ev * ((size_t)gst * 4 + 16 + 8 + 4 + 4) + (size_t)units * (16 + (best ? 8 : 0) + 4) + 64;
}

__device__ inline TileSmem carve(char* p, int ev_cap, int unit_cap, int gst, bool best)
{
    TileSmem t;
    t.top = p + ((tile_smem_bytes(ev_cap, unit_cap, gst, best) + 15) & ~(size_t)15);
    t.ureco = (float4*)p; p += (size_t)unit_cap * 16;
    t.lep = (float4*)p; p += (size_t)ev_cap * 16;
    t.met = (float2*)p; p += (size_t)ev_cap * 8;
    t.usc = (float2*)p; p += best ? (size_t)unit_cap * 8 : 0;
    t.G = (float*)p; p += (size_t)ev_cap * gst * 4;
    t.evid = (uint32_t*)p; p += (size_t)ev_cap * 4;
    t.bits = (uint32_t*)p; p += (size_t)ev_cap * 4;
    t.uf = (int*)p;
    return t;
}

// Shared memory of the chi2 step of a tile (after the TileSmem region).
constexpr int HT_UNITS = 256;  // units per sub-batch of the split evaluation

struct TopSmem {
    TopIn* tin;          // [HT_UNITS] MET state in, chi2 result out
    uint32_t* hidx;      // [HT_UNITS] unit (index in the tile) of each listed entry
    float* qs;           // [N * N][HT_SLOTS] smeared Gram terms, one column per thread
    float* as;           // [N][HT_SLOTS]
    uint8_t* pair_code;  // [npairs(MAX_JETS)]
    unsigned* nh;        // listed units
};

// Multiplicities whose triplet-only tiles take the split evaluation (probe,
// chi2 of the listed units, completion).  Below 9 jets the whole unit in one
// thread with the fully unrolled candidate loop measured faster (per-launch
// times of each multiplicity: the split gains from 9 jets on, where the
// candidates outnumber the rest of the unit's work and pair pruning pays).
__host__ __device__ constexpr bool semi_split(int n, bool full) { return !full && n >= 9; }

__host__ __device__ constexpr size_t top_smem_bytes(int n)
{
    return semi_split(n, false) ? (size_t)HT_UNITS * (sizeof(TopIn) + 4) + (size_t)(n * n + n) * HT_SLOTS * 4 + 128
                                : 0;
}

// Byte offset of the Gram-term columns (qs) in the chi2 step's region; the
// stage-2 tile uses that space to stage its events' jets before the chi2 step.
__host__ __device__ constexpr size_t top_qs_offset() { return (size_t)HT_UNITS * sizeof(TopIn); }

__device__ inline TopSmem carve_top(char* p, int n)
{
    TopSmem t;
    t.tin = (TopIn*)p; p += (size_t)HT_UNITS * sizeof(TopIn);
    t.qs = (float*)p; p += (size_t)n * n * HT_SLOTS * 4;
    t.as = (float*)p; p += (size_t)n * HT_SLOTS * 4;
    t.hidx = (uint32_t*)p; p += (size_t)HT_UNITS * 4;
    t.pair_code = (uint8_t*)p; p += 96;
    t.nh = (unsigned*)p;
    return t;
}

// Dynamic shared memory of a semileptonic stage-2 tile (multiplicity n).
__host__ __device__ inline size_t semi_smem_bytes(int n, bool full, int ev, int units, bool best)
{
    const size_t t = (tile_smem_bytes(ev, units, gram_stride(n), best) + 15) & ~(size_t)15;
    return full ? t : t + top_smem_bytes(n);
}

}  // namespace hf
