// hf_dev.cuh -- device-side data structures and FP32 building blocks of the
// GB300 cut-chain engine.  Internal header of the CUDA library (not part of
// the C ABI).  Every translation unit of the library is compiled with
// -fmad=false: no multiply-add is contracted implicitly, every fused
// multiply-add below is an explicit fmaf(), and FP64 code rounds every
// operation as written.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hf {

constexpr int MAX_CUTS = 16;
constexpr int MAX_JETS = 12;
constexpr int NBUCKET = 13;           // events bucketed by jet multiplicity 0..12
constexpr int BLOCK = 128;            // threads per block of the tile kernels
constexpr int UNITS_PER_TILE = 256;   // units (event x variation) per tile
constexpr int MAX_EV_PER_TILE = 128;  // events per tile cap (V = 1)
constexpr int MAX_BINS = 1024;        // histogram bins

// Cut kinds (same numbering as the C ABI).
enum : int {
    CUT_NJETS_MIN = 1,
    CUT_NBTAG_MIN = 2,
    CUT_LEP_PT_MIN = 3,
    CUT_MET_MIN = 4,
    CUT_W_NU_SOLVABLE = 5,
    CUT_HADTOP_CHI2_MAX = 6,
    CUT_LEP_OS = 7,
    CUT_DILEP_SOLVABLE = 8,
    CUT_HIGGS_WINDOW = 9,
    CUT_TTBAR_CHI2_MAX = 10
};
enum : int { MODEL_SEMILEP = 1, MODEL_DILEP = 2 };

// Profiling counters (device u64[64]).
enum : int { PROF_UNITS = 0, PROF_EVENTS = 1, PROF_PAIRINGS = 2, PROF_CANDS = 3, PROF_TOP = 16, PROF_DILEP = 32 };

// Error word bits (device -> host).
enum : unsigned { ERR_COLUMNS = 1u, ERR_RECHECK_FULL = 2u, ERR_TIMEOUT = 4u };

// Variables of the per-cut recording (values of HF_VAR_*).
enum : int { VAR_NONE = 0, VAR_NJETS = 1, VAR_NBTAG = 2, VAR_LEP_PT = 3, VAR_MET = 4, VAR_RECO0 = 5 };

// Everything a kernel needs to know about an analysis.  Passed by value.
struct Plan {
    int model;
    int n_cuts;
    int kind[MAX_CUTS];
    float p0[MAX_CUTS], p1[MAX_CUTS];
    unsigned stage1;   // bit c: user-order cut c is decided per event in stage 1
    unsigned stage2;   // bit c: decided per unit in stage 2
    int n_exec2;       // stage-2 cuts in default execution order (user order)
    int exec2[MAX_CUTS];
    float mW, mt, sigma_t, sigma_W, inv_sigma_t, inv_sigma_W, mH;
    float top_thr;     // largest threshold of the chi2 cuts (clamp of the triplet minimum)
    int has_full;      // the analysis has a full Eq. 1 fit cut: it supplies the reco and histogram
    float mW2half, mW2half_lo;  // mW*mW/2 (exact in FP64) as a float-float pair
    float sigma_jet, sigma_met, sigma_lep;
    int smear_jets, smear_met, smear_lep;
    int best;          // per-event best-of-variations (HF_PER_EVENT_BEST) instead of the mean
    int nbins;
    float lo, hi, w;   // histogram
    // FP32 error model (relative / absolute bounds vs the FP64 definition)
    float z_rel;       // |z32 - z64| <= z_rel |z|
    float s_rel;       // |s32 - s64| <= s_rel s
    float e_m;         // |m32 - m64| <= e_m m for any FP32 pair / triplet mass
    float safety;      // multiplier on every band
    float pz_tol;      // relative accuracy demanded of p_z before recheck
    // the same in double for the FP64 path
    double dmW, dmt, dsigma_t, dsigma_W, dmH, dsigma_jet, dsigma_met, dsigma_lep;
    double dp0[MAX_CUTS], dp1[MAX_CUTS];
    double dlo, dhi;
    unsigned rec_levels; // per-cut recording: bit k records events passing cuts 0..k
    int rec_var[4];      // HF_VAR_* of each recorded value
};

struct Cols {
    const uint32_t* jet_off;
    const float4* jets;
    const uint16_t* btag;
    const float4* lep;
    const int8_t* lep_q;
    const float2* met;
    uint64_t n_jets_total;
};

// One per-cut record (the layout of hf_record).
struct Record {
    uint32_t event;
    uint32_t level;
    float value[4];
};

struct Out {
    uint8_t* mask;
    uint16_t* n_surv;
    float4* reco;
    unsigned long long* cutflow;  // n_cuts + 1, device accumulators (zeroed per run)
    unsigned long long* hist;     // nbins + 2
    unsigned long long* rc_total; // units rechecked in FP64
    Record* rec;                  // per-cut records (null: none)
    unsigned long long rec_cap;
    unsigned long long* n_rec;    // records produced
    uint8_t* maxf;                // [N] scratch of a recording run: most cuts passed by a variation
    uint16_t* best_v;             // [N] best-of-variations: the chosen variation (or null)
};

// Recheck list entry: one unit whose FP32 evaluation came within an error
// band of a decision (cut threshold, argmin near-tie, histogram edge, ...).
struct RcEntry {
    uint32_t event;   // index within the chunk
    uint32_t vbits;   // variation (low 16 bits) | stage-1 pass bits of the event << 16
    uint32_t slot;    // pending-event slot
    uint32_t chunk;   // chunk of a batched run (0 for a single chunk)
};

// FP64 result of one recheck entry.
struct RcRes {
    int f;         // cuts passed in user order
    int bin;       // histogram bin when f == n_cuts
    double score;  // the unit's fit score (best-of-variations; the definition's FP64 value)
};

struct Scratch {
    unsigned* nhist;      // [16] events per jet multiplicity (bucket capacity)
    unsigned* cursor;     // [16] fill cursor per bucket
    unsigned* tile_ctr;   // [16] persistent-grid tile counter per bucket
    unsigned* rc_count;   // [1]  recheck entries appended
    unsigned* rc_valid;   // [1]  entries [0, rc_valid) of the list are written
    unsigned* pend_count; // [1]  pending-event slots used
    unsigned* err;        // [1]  error word
    uint2* bucket;        // [N]  stage-2 work: (event, stage-1 bits), grouped by n
    RcEntry* rc;          // [rc_cap] flagged units; those of one event are contiguous, in variation order
    unsigned rc_cap;
    float4* rc_reco;      // [rc_cap] FP64 result of entry i: reconstructed quantities
    RcRes* rc_res;        // [rc_cap] FP64 result of entry i: cuts passed, bin, score
    unsigned* pend_cnt;   // [rc_cap] surviving unflagged units of pending event s
    unsigned long long* rec_pre; // [stage-1 blocks + 1] records per block, then their exclusive prefix
    uint2* pend_rng;      // [rc_cap] (first entry, number of entries) of pending event s
    float4* pend_sum;     // [rc_cap] compensated sum over the unflagged survivors
    float4* pend_comp;    // [rc_cap] its compensation terms
    unsigned long long* stats;  // [3*MAX_CUTS] evaluated, passed, cost (cycles)
    unsigned long long* prof;   // [64] profiling counters (PROF_*) or null
    const int* exec2;     // [MAX_CUTS] device execution order of stage-2 cuts (or null)
    int n_exec2;
    uint32_t chunk;       // chunk index recorded in recheck entries (batched runs)
};

// ------------------------------------------------------------------ HL-LHC selection
// The HL-LHC multi-region selection (hf_hl.cu): parameters in FP32 and, for
// the FP64 definition, in double (the same values).
struct HLPlan {
    float met_min, mll_min, mtw_min, dr2;   // dr2 = dr_iso^2 (FP32)
    float dr_iso;
    double dmet_min, dmll_min, dmtw_min, ddr_iso;
    double deta[3];                         // region boundaries of |eta|
    float sh[3];                            // sinh of the boundaries, rounded to FP32
    int smear;
    float sigma_met;
    double dsigma_met;
    float z_rel, safety;
    int nbins;
    float lo, hi, w;
    double dlo, dhi;
};

struct HLCols {
    const uint32_t* jet_off;
    const float4* jets;
    const uint16_t* btag;
    const uint32_t* lep_off;
    const float4* lep;
    const int8_t* lep_q;
    const uint8_t* lep_flav;
    const float2* met;
    uint64_t n_jets, n_leps;
};

struct HLOut {
    unsigned long long* counts;  // [6]
    unsigned long long* hist;    // [5][nbins + 2]
    int8_t* channel;             // [N * V] or null
    unsigned* err;
};

// ------------------------------------------------------------------ batched runs
// One chunk of a batched run (device memory; the table is sorted so that
// semileptonic chunks come first).  Its cut flow, histogram and recheck
// counter pointers are never null (the batch's scratch provides them).
struct BChunk {
    Cols C;
    Out O;
    uint64_t seed, first_id;
    uint32_t V;        // variations per event
    uint32_t n;        // events
    uint32_t plan;     // index into BatchDev::plans
    uint32_t ept;      // events per stage-2 tile
    uint32_t blk0;     // first stage-1 block of the chunk (BLOCK1 events per block)
    uint32_t model;
    uint64_t ev0;      // first bucket slot of the chunk in the batch's bucket array
    unsigned* cnt;     // [32] nhist[16] | cursor[16] of the chunk
    unsigned* err;     // the chunk's own error word, or null
};

constexpr int BLOCK1 = 256;  // events per stage-1 block

// Everything the kernels of a batched run share (passed by value).
struct BatchDev {
    const BChunk* ch;             // n_chunks entries
    const Plan* plans;            // per analysis of the batch
    const int* const* exec;       // [plans] stage-2 execution order of each plan (its scheduler's)
    unsigned long long* stats;    // [plans][3*MAX_CUTS] scheduler statistics of the batch
    unsigned* tpre;               // [NBUCKET][n_chunks+1] tile prefix over chunks per bucket
    unsigned* tctr;               // [32] tile counters: [n] semileptonic multiplicity n, [16 + n] the
                                  // same for full-fit analyses, [15] dilepton
    uint2* bucket;                // stage-2 work of every chunk (chunk c from ev0)
    uint32_t n_chunks, n_semi;    // chunks [0, n_semi) are semileptonic
    uint32_t n_semi0;             // of which [0, n_semi0) without and [n_semi0, n_semi) with the full fit
    uint32_t n_blocks;            // stage-1 blocks of the batch
    uint32_t n_plans;
    unsigned long long* rec_pre;  // [n_blocks + 1] per-cut records per stage-1 block, then their prefix
    Scratch S;                    // recheck list, pending slots, error word of the batch
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products of counter words 0 and 2 by the round multipliers,
// the halves permuted and xored with the key, the key advanced by the Weyl
// increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += W0;
            k.y += W1;
        }
        uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        uint4 n;
        n.x = hi1 ^ c.y ^ k.x;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k.y;
        n.w = lo0;
        c = n;
    }
    return c;
}

// 32-bit word -> uniform in [2^-24, 1 - 2^-24], exact in FP32.
__device__ __forceinline__ float u01f(uint32_t x)
{
    return (__uint2float_rn(x >> 9) + 0.5f) * 1.1920928955078125e-7f;
}
__device__ __forceinline__ double u01d(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

// Box-Muller pair in FP32: r = sqrt(-2 ln u0), angle 2 pi u1 via sincospi
// (2 u1 is exact).  Relative error of each normal <= 2.5 ulp (logf, sqrtf,
// sincospif each within 1 ulp, product 0.5 ulp).
__device__ __forceinline__ void box_muller_f(uint32_t w0, uint32_t w1, float& z0, float& z1)
{
    float u0 = u01f(w0), u1 = u01f(w1);
    float r = sqrtf(-2.0f * logf(u0));
    float s, c;
    sincospif(2.0f * u1, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// Reciprocal square root, one MUFU instruction (PTX rsqrt.approx.ftz.f32,
// relative error below 2^-22; inputs here are normal, positive numbers).
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The Philox counter of block b of unit (event, v) and the seed key.
__device__ __forceinline__ uint4 ctr_of(uint32_t b, uint32_t v, uint64_t event)
{
    return make_uint4(b, v, (uint32_t)event, (uint32_t)(event >> 32));
}
__device__ __forceinline__ uint2 key_of(uint64_t seed)
{
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// ------------------------------------------------------------------ FP32 EFT
// Error-free transformations (Knuth TwoSum; TwoProduct with fmaf) and the
// compensated Minkowski product a.b = aE bE - ax bx - ay by - az bz
// (Ogita, Rump, Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
// 2005, Dot2): result within ~1 ulp of the exact value plus u^2 |a||b|.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float minkowski_dot2(float4 a, float4 b)
{
    float p = __fmul_rn(a.w, b.w);
    float s = fmaf(a.w, b.w, -p);
    float h, r, t, e;
    h = __fmul_rn(-a.x, b.x);
    r = fmaf(-a.x, b.x, -h);
    two_sum(p, h, t, e);
    p = t;
    s = __fadd_rn(s, __fadd_rn(r, e));
    h = __fmul_rn(-a.y, b.y);
    r = fmaf(-a.y, b.y, -h);
    two_sum(p, h, t, e);
    p = t;
    s = __fadd_rn(s, __fadd_rn(r, e));
    h = __fmul_rn(-a.z, b.z);
    r = fmaf(-a.z, b.z, -h);
    two_sum(p, h, t, e);
    p = t;
    s = __fadd_rn(s, __fadd_rn(r, e));
    return __fadd_rn(p, s);
}

// Packed upper triangle of the Gram matrix, diagonal included.
__host__ __device__ constexpr int tri(int i, int j) { return j * (j + 1) / 2 + i; }  // i <= j
__host__ __device__ constexpr int ntri(int n) { return n * (n + 1) / 2; }

// ------------------------------------------------------------------ histogram
// Bin of an FP32 value with a certainty flag: returns 0 = underflow,
// 1..nbins, nbins+1 = overflow, and sets *unsure when x is within `band` of
// an edge (the FP32 value could then fall on the other side of the FP64 one).
__device__ __forceinline__ int hist_bin_f(const Plan& P, float x, float band, bool* unsure)
{
    float eb = band + 2.4e-7f * (fabsf(P.lo) + fabsf(P.hi));
    if (x < P.lo) {
        if (P.lo - x <= eb) *unsure = true;
        return 0;
    }
    if (!(x < P.hi)) {
        if (x - P.hi <= eb) *unsure = true;
        return P.nbins + 1;
    }
    int i = (int)floorf((x - P.lo) / P.w);
    i = i < 0 ? 0 : (i > P.nbins - 1 ? P.nbins - 1 : i);
    float e0 = fmaf((float)i, P.w, P.lo);
    float e1 = fmaf((float)(i + 1), P.w, P.lo);
    if (x < e0 && i > 0) { --i; e1 = e0; e0 = fmaf((float)i, P.w, P.lo); }
    else if (x >= e1 && i < P.nbins - 1) { ++i; e0 = e1; e1 = fmaf((float)(i + 1), P.w, P.lo); }
    if (x - e0 <= eb || e1 - x <= eb) *unsure = true;
    return 1 + i;
}

// Histogram bin in FP64, the definition: largest i with x >= lo + i w.
__device__ __forceinline__ int hist_bin_d(const Plan& P, double x)
{
    if (x < P.dlo) return 0;
    if (!(x < P.dhi)) return P.nbins + 1;
    double w = (P.dhi - P.dlo) / P.nbins;
    int i = (int)floor((x - P.dlo) / w);
    if (i < 0) i = 0;
    if (i > P.nbins - 1) i = P.nbins - 1;
    while (i > 0 && x < P.dlo + i * w) --i;
    while (i < P.nbins - 1 && x >= P.dlo + (i + 1) * w) ++i;
    return 1 + i;
}

}  // namespace hf
