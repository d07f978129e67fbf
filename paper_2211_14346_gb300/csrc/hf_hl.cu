// hf_hl.cu -- the HL-LHC multi-region top selection (Sect. 6.1) on the GPU.
//
// Per unit (event, variation): the jets fall into the pseudorapidity regions
// I |eta| < 2.5, II 2.5 < |eta| < 2.75, III 2.75 < |eta| < 3.5 (a boundary, or
// |eta| >= 3.5, in none); b-jets are the b-tagged jets of region I; a lepton
// is isolated when no jet lies within Delta R < 0.4; every signal bin needs
// |MET| > 30 GeV.  One isolated lepton: ttbar 1l (>= 4 jets in I, exactly 2
// b, none in II or III), t-channel (exactly 1 jet in I and 1 in II or III,
// exactly 1 b), Wt 1l (exactly 3 jets in I, 1 b, none in II or III,
// M_T^W > 50 GeV).  Two isolated leptons of opposite sign and different
// flavour: ttbar 2l (>= 2 jets in I, exactly 2 b, none in II or III,
// M_ll > 40 GeV), Wt 2l (1 or 2 jets in I, exactly 1 b, none in II or III).
// The variations smear MET only (Philox block 3, normals z12 and z13 of the
// unit, as in the other event models): the selection has no jet-pT
// threshold, and jet-energy scales change neither eta nor the jet counts.
// Each signal channel fills its own histogram of the leading isolated
// lepton's pT, once per unit.
//
// Design: a column scan, bound by HBM (about 100 bytes per event).  A
// persistent grid takes tiles of HL_TILE consecutive events; the jet and
// lepton records of a tile (contiguous in the columns) are copied into shared
// memory by one bulk asynchronous copy each (cp.async.bulk completing on an
// mbarrier), double-buffered: the copy of the block's next tile runs while
// the block works on the current one.  One thread per event.
//
// Exactness: every decision is taken in FP32 with an error band and, inside
// the band, again in FP64 with the definition's formulas: a region from
// |pz| against pT sinh(boundary) (monotone in |eta|), FP64
// asinh(pz / sqrt(px^2 + py^2)) inside the band; Delta R^2 from FP32 eta
// (log((|pz| + |p|) / pT)) and the azimuth difference atan2(cross, dot),
// FP64 eta and atan2 differences wrapped to [-pi, pi] inside the band;
// |MET'|, M_T^W^2 and M_ll^2 with bounds on the FP32 smearing and rounding;
// the histogram bin with a band at the edges.
#include <cstdint>
#include <math_constants.h>

#include "hf_common.cuh"
#include "hf_kernels.h"

namespace hf {

namespace {

constexpr int HL_TILE = 256;    // events per tile (one per thread)
constexpr int HL_JCAP = 1280;   // jets of a tile staged in shared memory (else read from global memory)
constexpr int HL_LCAP = 512;    // leptons of a tile staged in shared memory
constexpr unsigned HL_WAIT_LIMIT = 1u << 24;  // bounded waits on the copies

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completing `bytes` on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Waits for phase `parity` of the mbarrier with a bounded number of tries.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity)
{
    for (unsigned it = 0; it < HL_WAIT_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ float hl_pt2(float x, float y) { return fmaf(x, x, __fmul_rn(y, y)); }

// Region of a jet (1 = I, 2 = II, 3 = III, 0 = none): the FP64 definition.
__device__ __noinline__ int region_d(const HLPlan& H, float4 j)
{
    const double px = j.x, py = j.y, pz = j.z;
    const double pt = sqrt(px * px + py * py);
    const double eta = pt > 0.0 ? asinh(pz / pt) : copysign(CUDART_INF, pz);
    const double a = fabs(eta);
    if (a < H.deta[0]) return 1;
    if (H.deta[0] < a && a < H.deta[1]) return 2;
    if (H.deta[1] < a && a < H.deta[2]) return 3;
    return 0;
}

// Region in FP32: |eta| < b <=> |pz| < pT sinh(b); a value within 1e-6 of a
// boundary (about 17 ulp; the FP32 pT and product are within 3 ulp) goes to
// the FP64 definition.
__device__ __forceinline__ int region_f(const HLPlan& H, float4 j)
{
    const float pt = sqrtf(hl_pt2(j.x, j.y));
    const float a = fabsf(j.z);
    bool unsure = !(pt > 0.0f);
    int g = 0;
    float t[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        t[b] = __fmul_rn(pt, H.sh[b]);
        unsure |= fabsf(a - t[b]) <= 1.0e-6f * t[b];
    }
    if (unsure) return region_d(H, j);
    if (a < t[0]) g = 1;
    else if (a < t[1]) g = 2;
    else if (a < t[2]) g = 3;
    return g;
}

// FP64 eta and phi of the definition.
__device__ __forceinline__ void eta_phi_d(float4 p, double& eta, double& phi)
{
    const double px = p.x, py = p.y, pz = p.z;
    const double pt = sqrt(px * px + py * py);
    eta = pt > 0.0 ? asinh(pz / pt) : copysign(CUDART_INF, pz);
    phi = atan2(py, px);
}

// Delta R(lepton, jet) >= dr_iso in FP64, the definition (azimuth difference
// wrapped to [-pi, pi] by steps of 2 pi).
__device__ __noinline__ bool isolated_from_d(const HLPlan& H, float4 l, float4 j)
{
    double el, pl, ej, pj;
    eta_phi_d(l, el, pl);
    eta_phi_d(j, ej, pj);
    double dphi = pl - pj;
    const double pi = 3.141592653589793;
    while (dphi > pi) dphi -= 2.0 * pi;
    while (dphi < -pi) dphi += 2.0 * pi;
    const double de = el - ej;
    return sqrt(de * de + dphi * dphi) >= H.ddr_iso;
}

// FP32 eta = sign(pz) log((|pz| + |p|) / pT) (= asinh(pz / pT)), within about
// 1e-6 of the FP64 value for |eta| < 5 (logf within 1 ulp, its argument
// within 5 ulp).  Returns false for pT = 0.
__device__ __forceinline__ bool eta_f(float4 p, float& eta)
{
    const float pt2 = hl_pt2(p.x, p.y);
    if (!(pt2 > 0.0f)) return false;
    const float pt = sqrtf(pt2);
    const float a = fabsf(p.z);
    const float r = sqrtf(fmaf(a, a, pt2));
    eta = copysignf(logf(__fdiv_rn(__fadd_rn(a, r), pt)), p.z);
    return true;
}

// Isolation of a lepton from one jet: FP32 Delta R^2 against dr_iso^2 with an
// absolute band of 1e-4 (the FP32 Delta eta and Delta phi are within about
// 2e-6 of the FP64 ones near the threshold), the FP64 definition inside it.
// Two cheap certain cases come first: |Delta eta| beyond dr_iso (by more than
// the eta error) and, for dr_iso < pi/2, transverse momenta more than 90
// degrees apart (a negative dot product beyond its rounding bound).
__device__ __forceinline__ bool isolated_from(const HLPlan& H, float4 l, float el, bool lok, float4 j, float ej,
                                              bool jok)
{
    if (!lok || !jok) return isolated_from_d(H, l, j);
    const float de = __fsub_rn(el, ej);
    if (fabsf(de) > H.dr_iso + 1.0e-5f) return true;
    const float dt = fmaf(l.x, j.x, __fmul_rn(l.y, j.y));
    if (H.dr_iso < 1.5f && dt < -2.4e-7f * (fabsf(l.x * j.x) + fabsf(l.y * j.y))) return true;
    // azimuth difference from the transverse cross and dot products
    const float cr = fmaf(l.x, j.y, -__fmul_rn(l.y, j.x));
    const float dphi = atan2f(cr, dt);
    const float dr2 = fmaf(de, de, __fmul_rn(dphi, dphi));
    if (fabsf(dr2 - H.dr2) <= 1.0e-4f) return isolated_from_d(H, l, j);
    return dr2 > H.dr2;
}

// Smeared MET of unit v in FP32 with error bounds (as the semileptonic model).
__device__ __forceinline__ void met_f(const HLPlan& H, float2 m, uint64_t event_id, uint32_t v, uint2 key, float& mx,
                                      float& my, float& dmx, float& dmy)
{
    mx = m.x;
    my = m.y;
    dmx = dmy = 0.0f;
    if (H.smear) {
        const uint4 w = philox4x32_10(ctr_of(3, v, event_id), key);
        float z12, z13;
        box_muller_f(w.x, w.y, z12, z13);
        mx = fmaf(H.sigma_met, z12, m.x);
        my = fmaf(H.sigma_met, z13, m.y);
        const float u = 5.9604645e-8f;
        dmx = H.sigma_met * H.z_rel * fabsf(z12) + u * fabsf(mx);
        dmy = H.sigma_met * H.z_rel * fabsf(z13) + u * fabsf(my);
    }
}

// The same in FP64, the definition (normals z12, z13 of Philox block 3).
__device__ __noinline__ void met_d(const HLPlan& H, float2 m, uint64_t event_id, uint32_t v, uint64_t seed, double& mx,
                                   double& my)
{
    mx = m.x;
    my = m.y;
    if (H.smear) {
        const uint4 w = philox4x32_10(ctr_of(3, v, event_id), key_of(seed));
        double z12, z13;
        box_muller_d(w.x, w.y, z12, z13);
        mx = (double)m.x + H.dsigma_met * z12;
        my = (double)m.y + H.dsigma_met * z13;
    }
}

// |MET'| > met_min: FP32 with the bound of the smeared components, FP64 inside.
__device__ __forceinline__ bool met_pass(const HLPlan& H, float2 m, uint64_t event_id, uint32_t v, uint64_t seed,
                                         float mx, float my, float dmx, float dmy)
{
    const float met = sqrtf(hl_pt2(mx, my));
    const float band = H.safety * (dmx + dmy + 3.6e-7f * met);
    if (fabsf(met - H.met_min) > band) return met > H.met_min;
    double x, y;
    met_d(H, m, event_id, v, seed, x, y);
    return sqrt(x * x + y * y) > H.dmet_min;
}

// M_T^W > mtw_min for the lepton l and the unit's MET.  FP32 M_T^W^2 =
// 2 (pT |MET'| - pT . MET') against mtw_min^2 with a bound that covers the
// smeared components' errors and the rounding; the FP64 definition inside.
__device__ __noinline__ bool mtw_pass_d(const HLPlan& H, float4 l, float2 m, uint64_t event_id, uint32_t v, uint64_t seed)
{
    double x, y;
    met_d(H, m, event_id, v, seed, x, y);
    const double lx = l.x, ly = l.y;
    const double met = sqrt(x * x + y * y);
    const double mt2 = 2.0 * (sqrt(lx * lx + ly * ly) * met - (lx * x + ly * y));
    return sqrt(mt2 > 0.0 ? mt2 : 0.0) > H.dmtw_min;
}

__device__ __forceinline__ bool mtw_pass(const HLPlan& H, float4 l, float2 m, uint64_t event_id, uint32_t v,
                                         uint64_t seed, float mx, float my, float dmx, float dmy)
{
    const float u = 5.9604645e-8f;
    const float pt = sqrtf(hl_pt2(l.x, l.y));
    const float met = sqrtf(hl_pt2(mx, my));
    const float dot = fmaf(l.x, mx, __fmul_rn(l.y, my));
    const float mt2 = 2.0f * __fsub_rn(__fmul_rn(pt, met), dot);
    const float err = 2.0f * (pt * (dmx + dmy + 4.0f * u * met) + fabsf(l.x) * dmx + fabsf(l.y) * dmy +
                              8.0f * u * (pt * met + fabsf(dot))) + 4.0f * u * fabsf(mt2);
    const float thr = H.mtw_min * H.mtw_min;
    if (fabsf(mt2 - thr) > H.safety * err + 1.0e-3f) return mt2 > thr;
    return mtw_pass_d(H, l, m, event_id, v, seed);
}

// M_ll > mll_min of two massless leptons: FP32 m^2 from compensated Minkowski
// products (a . a + b . b + 2 a . b, each within about 2 ulp of |a||b|), the
// FP64 mass of the summed components (the definition) inside the band.
__device__ __noinline__ bool mll_pass_d(const HLPlan& H, float4 a, float4 b)
{
    const double s0 = (double)a.x + (double)b.x, s1 = (double)a.y + (double)b.y, s2 = (double)a.z + (double)b.z,
                 s3 = (double)a.w + (double)b.w;
    const double m2 = s3 * s3 - s0 * s0 - s1 * s1 - s2 * s2;
    const double m = m2 >= 0.0 ? sqrt(m2) : -sqrt(-m2);
    return m > H.dmll_min;
}

__device__ __forceinline__ bool mll_pass(const HLPlan& H, float4 a, float4 b)
{
    const float m2 = __fadd_rn(__fadd_rn(minkowski_dot2(a, a), minkowski_dot2(b, b)), 2.0f * minkowski_dot2(a, b));
    const float e = __fadd_rn(a.w, b.w);
    const float band = 1.0e-5f * e * e + 1.0e-3f;
    const float thr = H.mll_min * H.mll_min;
    if (fabsf(m2 - thr) > band) return m2 > thr;
    return mll_pass_d(H, a, b);
}

// Histogram bin (1..nbins, 0 underflow, nbins + 1 overflow) of the leading
// isolated lepton's pT: FP32 with a band at the edges, the FP64 definition
// (largest i with x >= lo + i w) inside it.
__device__ __noinline__ int lead_bin_d(const HLPlan& H, const float4* leps, unsigned iso, int nl)
{
    double lead = 0.0;
    for (int k = 0; k < nl; ++k)
        if (iso >> k & 1u) {
            const double x = leps[k].x, y = leps[k].y;
            const double pt = sqrt(x * x + y * y);
            lead = pt > lead ? pt : lead;
        }
    if (lead < H.dlo) return 0;
    if (!(lead < H.dhi)) return H.nbins + 1;
    const double w = (H.dhi - H.dlo) / H.nbins;
    int i = (int)floor((lead - H.dlo) / w);
    i = i < 0 ? 0 : (i > H.nbins - 1 ? H.nbins - 1 : i);
    while (i > 0 && lead < H.dlo + i * w) --i;
    while (i < H.nbins - 1 && lead >= H.dlo + (i + 1) * w) ++i;
    return 1 + i;
}

__device__ __forceinline__ int lead_bin(const HLPlan& H, const float4* leps, unsigned iso, int nl)
{
    float lead = 0.0f;
    for (int k = 0; k < nl; ++k)
        if (iso >> k & 1u) lead = fmaxf(lead, sqrtf(hl_pt2(leps[k].x, leps[k].y)));
    const float eb = 2.4e-7f * lead + 2.4e-7f * (fabsf(H.lo) + fabsf(H.hi)) + 1.0e-30f;
    if (lead < H.lo - eb) return 0;
    if (lead >= H.hi + eb) return H.nbins + 1;
    if (lead < H.lo + eb || lead >= H.hi - eb) return lead_bin_d(H, leps, iso, nl);
    int i = (int)floorf((lead - H.lo) / H.w);
    i = i < 0 ? 0 : (i > H.nbins - 1 ? H.nbins - 1 : i);
    const float e0 = fmaf((float)i, H.w, H.lo), e1 = fmaf((float)(i + 1), H.w, H.lo);
    if (lead - e0 <= 4.0f * eb || e1 - lead <= 4.0f * eb) return lead_bin_d(H, leps, iso, nl);
    return 1 + i;
}

struct HLSmem {
    float4 jets[2][HL_JCAP];
    float4 leps[2][HL_LCAP];
    uint64_t bar[2];
    uint32_t jbase[2], lbase[2];  // first jet / lepton of the staged tile
    uint32_t jcnt[2], lcnt[2];    // jets / leptons staged (0 when the tile reads global memory)
    unsigned long long counts[6];
    // per tile (rewritten after each tile's last barrier)
    uint16_t jev[HL_JCAP];        // tile-local event of each staged jet (0xffff: none)
    uint8_t jk[HL_JCAP];          // its index within the event
    uint16_t lev[HL_LCAP];        // tile-local event of each staged lepton
    float leta[HL_LCAP];          // FP32 eta of each staged lepton
    uint8_t lok[HL_LCAP];         // 1: leta valid (pT > 0)
    unsigned cnt4[HL_TILE];       // per event: n1 | n2 << 8 | n3 << 16 | n_b << 24
    unsigned iso[HL_TILE];        // per event: isolation bits of its leptons
    uint16_t lofs[HL_TILE];       // per event: first staged lepton
    uint16_t btag[HL_TILE];
    uint8_t nlep[HL_TILE];
    uint8_t mode[HL_TILE];        // 0: none or malformed, 1: staged, 2: read from global memory
    // followed by the per-channel histograms: unsigned [5][nbins + 2]
};

// Issues the copies of tile t into stage s (one thread).
__device__ __forceinline__ void stage_tile(const HLCols& C, uint32_t N, unsigned t, int s, HLSmem& sm)
{
    const uint32_t e0 = t * HL_TILE, e1 = min(N, e0 + HL_TILE);
    const uint32_t j0 = C.jet_off[e0], j1 = C.jet_off[e1];
    const uint32_t l0 = C.lep_off[e0], l1 = C.lep_off[e1];
    const bool jok = j1 >= j0 && j1 - j0 <= (uint32_t)HL_JCAP && (uint64_t)j1 <= C.n_jets;
    const bool lok = l1 >= l0 && l1 - l0 <= (uint32_t)HL_LCAP && (uint64_t)l1 <= C.n_leps;
    sm.jbase[s] = j0;
    sm.lbase[s] = l0;
    sm.jcnt[s] = jok ? j1 - j0 : 0u;
    sm.lcnt[s] = lok ? l1 - l0 : 0u;
    const unsigned jb = jok ? 16u * (j1 - j0) : 0u, lb = lok ? 16u * (l1 - l0) : 0u;
    mbar_arrive_expect_tx(&sm.bar[s], jb + lb);
    if (jb) bulk_g2s(sm.jets[s], C.jets + j0, jb, &sm.bar[s]);
    if (lb) bulk_g2s(sm.leps[s], C.lep + l0, lb, &sm.bar[s]);
}

// Jet counts per region, b-jets and isolation bits of one event by its own
// thread (events whose records are not staged).
__device__ inline void scan_event_direct(const HLPlan& H, const float4* jp, int n, const float4* lp, int nl,
                                         unsigned bt, unsigned& c4, unsigned& iso)
{
    float el[HF_HL_MAX_LEPTONS];
    bool lk[HF_HL_MAX_LEPTONS];
    iso = 0;
    for (int k = 0; k < nl; ++k) {
        lk[k] = eta_f(lp[k], el[k]);
        iso |= 1u << k;
    }
    c4 = 0;
    for (int q = 0; q < n; ++q) {
        const float4 j = jp[q];
        const int g = region_f(H, j);
        c4 += g == 1 ? 1u + ((bt >> q & 1u) << 24) : g == 2 ? 1u << 8 : g == 3 ? 1u << 16 : 0u;
        if (iso) {
            float ej = 0.0f;
            const bool jok = eta_f(j, ej);
            for (int k = 0; k < nl; ++k)
                if ((iso >> k & 1u) && !isolated_from(H, lp[k], el[k], lk[k], j, ej, jok)) iso &= ~(1u << k);
        }
    }
}

}  // namespace

// One tile in four steps separated by block barriers: (0) one thread per
// event validates its offsets and maps its staged jets and leptons to it;
// (1) one thread per staged lepton forms its eta; (2) one thread per staged
// jet classifies its region, adds it to its event's packed counts and clears
// the isolation bits of the event's leptons it is close to (shared-memory
// atomics); (3) one thread per event takes the channel decisions, MET-
// dependent ones per variation, and counts the units.  Steps 1-2 give every
// lane the same amount of work whatever the events' multiplicities.
__global__ void __launch_bounds__(HL_TILE) k_hl(const HLPlan H, const HLCols C, uint32_t N, uint32_t V, uint64_t seed,
                                               uint64_t first_id, HLOut O)
{
    extern __shared__ __align__(16) char smem_raw[];
    HLSmem& sm = *reinterpret_cast<HLSmem*>(smem_raw);
    unsigned* s_hist = reinterpret_cast<unsigned*>(smem_raw + sizeof(HLSmem));
    const int nb2 = H.nbins + 2;
    for (int b = threadIdx.x; b < 5 * nb2; b += blockDim.x) s_hist[b] = 0;
    if (threadIdx.x < 6) sm.counts[threadIdx.x] = 0;
    const unsigned ntiles = (N + HL_TILE - 1) / HL_TILE;
    unsigned t = blockIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (t < ntiles) stage_tile(C, N, t, 0, sm);
    }
    __syncthreads();
    unsigned long long cnt[6] = {0, 0, 0, 0, 0, 0};
    const uint2 key = key_of(seed);
    bool timed_out = false;
    const int tid = threadIdx.x;
    for (unsigned i = 0; t < ntiles; ++i, t += gridDim.x) {
        const int s = (int)(i & 1u);
        const unsigned tn = t + gridDim.x;
        if (tid == 0 && tn < ntiles) stage_tile(C, N, tn, s ^ 1, sm);
        const uint32_t jbase = sm.jbase[s], lbase = sm.lbase[s], jcnt = sm.jcnt[s], lcnt = sm.lcnt[s];
        for (uint32_t j = tid; j < jcnt; j += HL_TILE) sm.jev[j] = 0xffffu;
        for (uint32_t l = tid; l < lcnt; l += HL_TILE) sm.lev[l] = 0xffffu;
        // (0) per event: validation and the maps of its staged records
        const uint32_t e = t * HL_TILE + tid;
        uint32_t j0 = 0, j1 = 0, l0 = 0, l1 = 0;
        int md = 0;
        if (e < N) {
            j0 = C.jet_off[e];
            j1 = C.jet_off[e + 1];
            l0 = C.lep_off[e];
            l1 = C.lep_off[e + 1];
            if (j1 < j0 || j1 - j0 > HF_HL_MAX_JETS || (uint64_t)j1 > C.n_jets || l1 < l0 ||
                l1 - l0 > HF_HL_MAX_LEPTONS || (uint64_t)l1 > C.n_leps) {
                atomicOr(O.err, ERR_COLUMNS);
                if (O.channel)
                    for (uint32_t v = 0; v < V; ++v) O.channel[(uint64_t)e * V + v] = 0;
            } else {
                const bool js = j0 >= jbase && j1 - jbase <= jcnt;
                const bool ls = l0 >= lbase && l1 - lbase <= lcnt;
                md = js && ls ? 1 : 2;
            }
        }
        __syncthreads();  // the maps are cleared
        const int n = (int)(j1 - j0), nl = (int)(l1 - l0);
        sm.mode[tid] = (uint8_t)md;
        if (md == 1) {
            sm.cnt4[tid] = 0;
            sm.iso[tid] = (1u << nl) - 1u;
            sm.lofs[tid] = (uint16_t)(l0 - lbase);
            sm.nlep[tid] = (uint8_t)nl;
            sm.btag[tid] = C.btag[e];
            for (int q = 0; q < n; ++q) {
                sm.jev[j0 - jbase + q] = (uint16_t)tid;
                sm.jk[j0 - jbase + q] = (uint8_t)q;
            }
            for (int k = 0; k < nl; ++k) sm.lev[l0 - lbase + k] = (uint16_t)tid;
        }
        if (!mbar_wait(&sm.bar[s], (i >> 1) & 1u)) timed_out = true;
        if (__syncthreads_or(timed_out)) {
            timed_out = true;
            break;
        }
        // (1) per staged lepton: eta
        for (uint32_t l = tid; l < lcnt; l += HL_TILE) {
            if (sm.lev[l] == 0xffffu) continue;
            float el = 0.0f;
            sm.lok[l] = eta_f(sm.leps[s][l], el) ? 1 : 0;
            sm.leta[l] = el;
        }
        __syncthreads();
        // (2) per staged jet: region, counts, isolation of its event's leptons
        for (uint32_t j = tid; j < jcnt; j += HL_TILE) {
            const unsigned ev = sm.jev[j];
            if (ev == 0xffffu) continue;
            const float4 jet = sm.jets[s][j];
            const int g = region_f(H, jet);
            const unsigned add = g == 1 ? 1u + ((unsigned)(sm.btag[ev] >> sm.jk[j] & 1u) << 24)
                                        : g == 2 ? 1u << 8 : g == 3 ? 1u << 16 : 0u;
            if (add) atomicAdd(&sm.cnt4[ev], add);
            const int nle = sm.nlep[ev];
            if (nle && sm.iso[ev]) {
                float ej = 0.0f;
                const bool jok = eta_f(jet, ej);
                const int lo = sm.lofs[ev];
                unsigned clear = 0;
                for (int k = 0; k < nle; ++k)
                    if (!isolated_from(H, sm.leps[s][lo + k], sm.leta[lo + k], sm.lok[lo + k] != 0, jet, ej, jok))
                        clear |= 1u << k;
                if (clear) atomicAnd(&sm.iso[ev], ~clear);
            }
        }
        __syncthreads();
        // (3) per event: channel decisions and counts
        if (md) {
            unsigned c4, iso;
            const float4* lp;
            if (md == 1) {
                c4 = sm.cnt4[tid];
                iso = sm.iso[tid];
                lp = sm.leps[s] + (l0 - lbase);
            } else {
                lp = C.lep + l0;
                scan_event_direct(H, C.jets + j0, n, lp, nl, C.btag[e], c4, iso);
            }
            const int n1 = (int)(c4 & 255u), n2 = (int)(c4 >> 8 & 255u), n3 = (int)(c4 >> 16 & 255u);
            const int nbj = (int)(c4 >> 24);
            const int niso = __popc(iso);
            // the signal channel this event can reach, before the MET-dependent requirements
            int ch = 0;
            int ia = -1;
            bool need_mtw = false;
            const bool clean = n2 == 0 && n3 == 0;
            if (niso == 1) {
                ia = __ffs(iso) - 1;
                if (n1 >= 4 && nbj == 2 && clean) ch = 1;
                else if (n1 == 1 && n2 + n3 == 1 && nbj == 1) ch = 3;
                else if (n1 == 3 && nbj == 1 && clean) {
                    ch = 4;
                    need_mtw = true;
                }
            } else if (niso == 2) {
                const int a = __ffs(iso) - 1;
                const int b = __ffs(iso & ~(1u << a)) - 1;
                const uint32_t la = l0 + a, lb = l0 + b;
                if (C.lep_q[la] * C.lep_q[lb] < 0 && C.lep_flav[la] != C.lep_flav[lb]) {
                    if (n1 >= 2 && nbj == 2 && clean && mll_pass(H, lp[a], lp[b])) ch = 2;
                    else if ((n1 == 1 || n1 == 2) && nbj == 1 && clean) ch = 5;
                }
            }
            const float2 m = C.met[e];
            const uint64_t eid = first_id + e;
            unsigned sig = 0;  // units in channel ch
            if (ch == 0) {
                if (O.channel)
                    for (uint32_t v = 0; v < V; ++v) O.channel[(uint64_t)e * V + v] = 0;
            } else if (!H.smear) {
                float mx, my, dmx, dmy;
                met_f(H, m, eid, 0, key, mx, my, dmx, dmy);
                bool pass = met_pass(H, m, eid, 0, seed, mx, my, dmx, dmy);
                if (pass && need_mtw) pass = mtw_pass(H, lp[ia], m, eid, 0, seed, mx, my, dmx, dmy);
                sig = pass ? V : 0;
                if (O.channel)
                    for (uint32_t v = 0; v < V; ++v) O.channel[(uint64_t)e * V + v] = (int8_t)(pass ? ch : 0);
            } else {
                for (uint32_t v = 0; v < V; ++v) {
                    float mx, my, dmx, dmy;
                    met_f(H, m, eid, v, key, mx, my, dmx, dmy);
                    bool pass = met_pass(H, m, eid, v, seed, mx, my, dmx, dmy);
                    if (pass && need_mtw) pass = mtw_pass(H, lp[ia], m, eid, v, seed, mx, my, dmx, dmy);
                    sig += pass;
                    if (O.channel) O.channel[(uint64_t)e * V + v] = (int8_t)(pass ? ch : 0);
                }
            }
            cnt[0] += V - sig;
            if (sig) {
                cnt[ch] += sig;
                float4 leps[HF_HL_MAX_LEPTONS];
                for (int k = 0; k < nl; ++k) leps[k] = lp[k];
                atomicAdd(&s_hist[(ch - 1) * nb2 + lead_bin(H, leps, iso, nl)], sig);
            }
        }
        __syncthreads();  // every thread is done with stage s and the tile's maps
    }
    if (timed_out) {
        // a copy that never completed: record it and give the other stage a
        // bounded chance to land before the block's shared memory goes away
        if (tid == 0) atomicOr(O.err, ERR_TIMEOUT);
        mbar_wait(&sm.bar[0], 0);
        mbar_wait(&sm.bar[1], 0);
        return;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        unsigned long long x = cnt[c];
        for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((tid & 31) == 0 && x) atomicAdd(&sm.counts[c], x);
    }
    __syncthreads();
    if (tid < 6 && sm.counts[tid]) atomicAdd(&O.counts[tid], sm.counts[tid]);
    for (int b = tid; b < 5 * nb2; b += blockDim.x)
        if (s_hist[b]) atomicAdd(&O.hist[b], (unsigned long long)s_hist[b]);
}

cudaError_t launch_hl(const HLPlan& H, const HLCols& C, uint32_t N, uint32_t V, uint64_t seed, uint64_t first_id,
                      const HLOut& O, int sms, cudaStream_t st)
{
    if (N == 0) return cudaSuccess;
    cudaError_t e = ensure_smem_attr((const void*)k_hl);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(HLSmem) + 4 * (size_t)5 * (H.nbins + 2);
    int bs = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_hl, HL_TILE, smem)) != cudaSuccess) return e;
    if (bs < 1) bs = 1;
    const unsigned ntiles = (N + HL_TILE - 1) / HL_TILE;
    const unsigned grid = min(ntiles, (unsigned)(sms * bs));
    k_hl<<<grid, HL_TILE, smem, st>>>(H, C, N, V, seed, first_id, O);
    return cudaGetLastError();
}

}  // namespace hf
