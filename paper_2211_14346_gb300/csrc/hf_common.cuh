// hf_common.cuh -- device helpers shared by the kernels of the cut chain:
// exact stage-1 predicates, cut-flow and histogram flushes, the FP64 unit
// evaluation, compensated per-event sums and the pending-event protocol of
// the FP64 recheck.  Header-only; every translation unit gets its own copy.
#pragma once
#include "hf_dev.cuh"
#include "hf_fp64.cuh"

namespace hf {

__device__ __forceinline__ void write_zero_event(const Out& O, uint32_t e)
{
    if (O.mask) O.mask[e] = 0;
    if (O.n_surv) O.n_surv[e] = 0;
    if (O.reco) O.reco[e] = make_float4(0.f, 0.f, 0.f, 0.f);
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
static __device__ __noinline__ int unit_fp64(const Plan& P, const Cols& C, uint32_t e, uint64_t event_id, uint64_t seed,
                         uint32_t v, unsigned s1bits, float4* reco, int* bin)
{
    EvD ev;
    load_event_d(P, C, e, event_id, seed, v, ev);
    bool top_done = false;
    double chi2 = 0.0, mtop = 0.0, mw = 0.0;
    int f = P.n_cuts;
    for (int c = 0; c < P.n_cuts; ++c) {
        bool pass;
        if (P.stage1 >> c & 1u) {
            pass = s1bits >> c & 1u;
        } else if (P.kind[c] == CUT_MET_MIN) {
            pass = sqrt(ev.metx * ev.metx + ev.mety * ev.mety) > P.dp0[c];
        } else if (P.kind[c] == CUT_HADTOP_CHI2_MAX) {
            if (!top_done) {
                chi2 = hadtop_d(ev, P, &mtop, &mw);
                top_done = true;
            }
            pass = chi2 < P.dp0[c];
        } else {
            pass = false;
        }
        if (!pass) {
            f = c;
            break;
        }
    }
    if (f == P.n_cuts) {
        if (!top_done) chi2 = hadtop_d(ev, P, &mtop, &mw);
        double pz;
        w_pz_d(ev.lep[0], ev.metx, ev.mety, P.dmW, &pz);
        double met = sqrt(ev.metx * ev.metx + ev.mety * ev.mety);
        *bin = hist_bin_d(P, mtop);
        *reco = make_float4((float)mtop, (float)mw, (float)pz, (float)met);
    }
    return f;
}

// ------------------------------------------------------------------ pending events
// An event with units in the recheck list keeps its partial result in a
// pending slot; the last of its rechecked units writes the event's outputs.
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

__device__ __forceinline__ void acc4(float4& s, float4& c, float4 x)
{
    float t, e;
    two_sum(s.x, x.x, t, e); s.x = t; c.x = __fadd_rn(c.x, e);
    two_sum(s.y, x.y, t, e); s.y = t; c.y = __fadd_rn(c.y, e);
    two_sum(s.z, x.z, t, e); s.z = t; c.z = __fadd_rn(c.z, e);
    two_sum(s.w, x.w, t, e); s.w = t; c.w = __fadd_rn(c.w, e);
}

// Registers an event with nflag flagged units (their variations in vs[]).
// Falls back to evaluating them inline in FP64 when the list is full.
static __device__ __noinline__ void pend_event(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t e,
                           uint64_t event_id, uint64_t seed, unsigned s1bits, unsigned cnt, float4 sum,
                           float4 comp, const uint16_t* vs, int nflag, unsigned long long* fc, unsigned* hist)
{
    unsigned base = atomicAdd(S.rc_count, (unsigned)nflag);
    if (base + (unsigned)nflag <= S.rc_cap) {
        // entries below the largest end of a successful reservation are all
        // written; a reservation crossing rc_cap is never written
        atomicMax(S.rc_valid, base + (unsigned)nflag);
        unsigned slot = atomicAdd(S.pend_count, 1u);
        S.pend_cnt[slot] = cnt;
        S.pend_left[slot] = (unsigned)nflag;
        S.pend_sum[slot] = sum;
        S.pend_comp[slot] = comp;
        for (int i = 0; i < nflag; ++i) {
            RcEntry r;
            r.event = e;
            r.v = vs[i];
            r.s1bits = s1bits;
            r.slot = slot;
            S.rc[base + i] = r;
        }
        return;
    }
    // list full: evaluate here (slow, correct)
    atomicOr(S.err, ERR_RECHECK_FULL);
    for (int i = 0; i < nflag; ++i) {
        float4 reco;
        int bin = 0;
        int f = unit_fp64(P, C, e, event_id, seed, vs[i], s1bits, &reco, &bin);
        atomicAdd(&fc[f], 1ull);
        if (f == P.n_cuts) {
            ++cnt;
            atomicAdd(&hist[bin], 1u);
            acc4(sum, comp, reco);
        }
    }
    atomicAdd(O.rc_total, (unsigned long long)nflag);
    write_event(O, e, cnt, sum, comp);
}

// ------------------------------------------------------------------ tile shared memory
struct TileSmem {
    float4* jets;   // [ev][12]
    float* G;       // [ev][GS]
    float4* lep;    // [ev]
    float2* met;    // [ev]
    uint32_t* evid; // [ev]
    uint32_t* bits; // [ev]
    float4* ureco;  // [unit]
    int* uf;        // [unit] f or -1
};
constexpr int GS = 79;  // padded Gram row stride (odd: conflict-free across events)

__host__ __device__ inline size_t tile_smem_bytes(int ev, int units)
{
    return (size_t)ev * (12 * 16 + GS * 4 + 16 + 8 + 4 + 4) + (size_t)units * (16 + 4) + 64;
}

__device__ inline TileSmem carve(char* p, int ev_cap, int unit_cap)
{
    TileSmem t;
    t.jets = (float4*)p; p += (size_t)ev_cap * 12 * 16;
    t.ureco = (float4*)p; p += (size_t)unit_cap * 16;
    t.lep = (float4*)p; p += (size_t)ev_cap * 16;
    t.met = (float2*)p; p += (size_t)ev_cap * 8;
    t.G = (float*)p; p += (size_t)ev_cap * GS * 4;
    t.evid = (uint32_t*)p; p += (size_t)ev_cap * 4;
    t.bits = (uint32_t*)p; p += (size_t)ev_cap * 4;
    t.uf = (int*)p;
    return t;
}

}  // namespace hf
