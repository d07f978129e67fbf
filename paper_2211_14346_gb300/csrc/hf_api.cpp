// hf_api.cpp -- host runtime behind the C ABI declared in include/hf.h.
//
// One context per GPU.  A context owns three CUDA streams (host-to-device
// copies, compute, device-to-host copies), the registered analyses with
// their device-side scheduler state, a scratch arena for runs over
// device-resident columns, and the table of asynchronous tickets.  Device
// memory of tickets comes from the stream-ordered allocator
// (cudaMallocAsync), so that admission, copies, kernels and release of many
// in-flight chunks overlap without host synchronisation.
#include "hf.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hf_dev.cuh"
#include "hf_kernels.h"
#include "hf_sched.h"

using namespace hf;

// Message of the last error of the calling thread (fixed storage: reporting
// an error allocates nothing).
namespace {
thread_local char g_err[512] = "";
}  // namespace

namespace hf {
hf_status set_error(hf_status s, const char* msg)
{
    snprintf(g_err, sizeof g_err, "%s", msg);
    return s;
}
hf_status set_cuda_error(cudaError_t e, const char* what)
{
    snprintf(g_err, sizeof g_err, "%s: %s", what, cudaGetErrorString(e));
    return HF_ECUDA;
}
}  // namespace hf

namespace {

hf_status fail(hf_status s, const char* msg) { return hf::set_error(s, msg); }
hf_status cuda_fail(cudaError_t e, const char* what) { return hf::set_cuda_error(e, what); }

#define HF_CUDA(call)                                      \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return cuda_fail(_e, #call); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Analysis {
    Plan plan;
    std::vector<hf_cut> cuts;
    SchedDev* sched = nullptr;  // device
    bool no_sched = false;
};

// Layout of the device memory of one run (scratch + optional columns +
// optional results), carved from one allocation.
struct RunLayout {
    size_t off_small = 0, off_bucket = 0, off_rc = 0, off_pend_cnt = 0, off_pend_rng = 0, off_pend_sum = 0,
           off_rc_reco = 0, off_rc_f = 0, off_maxf = 0, off_rec_pre = 0,
           off_pend_comp = 0, off_stats = 0, off_cutflow = 0, off_hist = 0, off_rctot = 0;
    size_t scratch_bytes = 0;
    unsigned rc_cap = 0;
};

RunLayout layout_for(uint64_t N, uint32_t V)
{
    RunLayout L;
    size_t o = 0;
    L.off_small = o;
    o += 256;
    L.off_bucket = o = align_up(o, 256);
    o += sizeof(uint2) * std::max<uint64_t>(N, 1);
    uint64_t units = N * (uint64_t)V;
    uint64_t cap = std::max<uint64_t>(65536, units / 64);
    cap = std::min<uint64_t>(cap, 1u << 30);
    L.rc_cap = (unsigned)cap;
    L.off_rc = o = align_up(o, 256);
    o += sizeof(RcEntry) * cap;
    L.off_pend_cnt = o = align_up(o, 256);
    o += 4 * cap;
    L.off_pend_rng = o = align_up(o, 256);
    o += 8 * cap;
    L.off_pend_sum = o = align_up(o, 256);
    o += 16 * cap;
    L.off_pend_comp = o = align_up(o, 256);
    o += 16 * cap;
    L.off_rc_reco = o = align_up(o, 256);
    o += 16 * cap;
    L.off_rc_f = o = align_up(o, 256);
    o += sizeof(RcRes) * cap;
    L.off_maxf = o = align_up(o, 256);
    o += std::max<uint64_t>(N, 1);
    L.off_rec_pre = o = align_up(o, 256);
    o += 8 * ((N + 255) / 256 + 1);
    L.off_stats = o = align_up(o, 256);
    o += 8 * 3 * MAX_CUTS;
    L.off_cutflow = o = align_up(o, 256);
    o += 8 * (MAX_CUTS + 1);
    L.off_hist = o = align_up(o, 256);
    o += 8 * (MAX_BINS + 2);
    L.off_rctot = o = align_up(o, 256);
    o += 8;
    L.scratch_bytes = align_up(o, 256);
    return L;
}

// Offsets inside the "small" block: counters zeroed per run.
constexpr size_t SM_NHIST = 0, SM_CURSOR = 64, SM_TILE = 128, SM_RC = 192, SM_RCVALID = 196, SM_PEND = 200,
                 SM_ERR = 204;

Scratch make_scratch(char* base, const RunLayout& L, const Analysis& A)
{
    Scratch S;
    char* sm = base + L.off_small;
    S.nhist = (unsigned*)(sm + SM_NHIST);
    S.cursor = (unsigned*)(sm + SM_CURSOR);
    S.tile_ctr = (unsigned*)(sm + SM_TILE);
    S.rc_count = (unsigned*)(sm + SM_RC);
    S.rc_valid = (unsigned*)(sm + SM_RCVALID);
    S.pend_count = (unsigned*)(sm + SM_PEND);
    S.err = (unsigned*)(sm + SM_ERR);
    S.bucket = (uint2*)(base + L.off_bucket);
    S.rc = (RcEntry*)(base + L.off_rc);
    S.rc_cap = L.rc_cap;
    S.pend_cnt = (unsigned*)(base + L.off_pend_cnt);
    S.pend_rng = (uint2*)(base + L.off_pend_rng);
    S.rc_reco = (float4*)(base + L.off_rc_reco);
    S.rc_res = (RcRes*)(base + L.off_rc_f);
    S.rec_pre = (unsigned long long*)(base + L.off_rec_pre);
    S.pend_sum = (float4*)(base + L.off_pend_sum);
    S.pend_comp = (float4*)(base + L.off_pend_comp);
    S.stats = (unsigned long long*)(base + L.off_stats);
    S.prof = nullptr;
    S.exec2 = A.sched ? A.sched->exec2 : nullptr;
    S.n_exec2 = A.plan.n_exec2;
    S.chunk = 0;
    return S;
}

// Bytes of the device columns of N events with J jets.
struct ColLayout {
    size_t off_jet_off, off_jets, off_btag, off_lep, off_lep_q, off_met, bytes;
};
ColLayout col_layout(uint64_t N, uint64_t J, int L)
{
    ColLayout c;
    size_t o = 0;
    c.off_jets = o;
    o += 16 * J;
    c.off_lep = o = align_up(o, 256);
    o += 16 * (uint64_t)L * N;
    c.off_met = o = align_up(o, 256);
    o += 8 * N;
    c.off_jet_off = o = align_up(o, 256);
    o += 4 * (N + 1);
    c.off_btag = o = align_up(o, 256);
    o += 2 * N;
    c.off_lep_q = o = align_up(o, 256);
    o += (uint64_t)L * N;
    c.bytes = align_up(o, 256);
    return c;
}

struct ResLayout {
    size_t off_mask, off_nsurv, off_reco, off_bestv, bytes;
};
ResLayout res_layout(uint64_t N)
{
    ResLayout r;
    size_t o = 0;
    r.off_reco = o;
    o += 16 * N;
    r.off_nsurv = o = align_up(o, 256);
    o += 2 * N;
    r.off_mask = o = align_up(o, 256);
    o += N;
    r.off_bestv = o = align_up(o, 256);
    o += 2 * N;
    r.bytes = align_up(o, 256);
    return r;
}

struct Ticket {
    uint64_t id = 0;
    uint32_t analysis = 0;
    uint64_t N = 0;
    char* dmem = nullptr;  // one stream-ordered allocation
    size_t bytes = 0;
    RunLayout L;
    ResLayout R;
    cudaEvent_t done = nullptr;
    bool failed_launch = false;
    // continuous batching (HF_FLAG_BATCHING): the dispatcher launches queued
    // tickets together; `done` is then the batch's event, shared by its tickets
    bool batched = false;
    bool launched = false;
    cudaEvent_t h2d = nullptr;  // host-to-device copies of the columns finished
    hf_chunk ch{};              // device view of the chunk (columns, results)
    size_t off_res = 0, off_cf = 0, off_hist = 0, off_rct = 0, off_err = 0;  // the ticket's results
};

}  // namespace

struct hf_ctx {
    int device = 0;
    int sms = 0;
    uint32_t flags = 0;
    uint64_t budget = 0;
    uint32_t max_inflight = 64;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    cudaStream_t user_stream = nullptr;
    SideStreams side{};  // stage-2 kernels of one run overlap on these
    int tune[3][8] = {};  // autotuned units per stage-2 tile by [model][variation class] (0 = default)
    std::mutex mu;
    std::vector<std::unique_ptr<Analysis>> analyses;
    // scratch arena for device-resident runs
    char* arena = nullptr;
    size_t arena_bytes = 0;
    cudaEvent_t arena_free = nullptr;  // last run that used the arena
    // tickets
    std::map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    uint64_t inflight_bytes = 0;
    // batched runs: pinned staging of the batch tables, the captured launch
    // sequence and what it was captured for
    char* bstage = nullptr;
    size_t bstage_bytes = 0;
    // pinned staging ring of pageable host columns (hf_config.staging_bytes)
    struct StageRegion {
        size_t off, bytes;
        cudaEvent_t done;  // the H2D copy out of the region has completed
    };
    char* staging = nullptr;
    size_t staging_bytes = 0, stage_head = 0;
    std::deque<StageRegion> stage_q;  // regions in use, in address order below stage_head
    cudaEvent_t bstage_free = nullptr;  // last upload from the staging buffer
    cudaStream_t s_cap = nullptr;       // capture stream of the batch graphs
    std::map<std::vector<uint64_t>, cudaGraphExec_t> bgraphs;  // captured launch sequences by shape
    // continuous batching (HF_FLAG_BATCHING)
    std::thread dispatcher;
    std::condition_variable cv;
    bool stop = false;
    std::deque<uint64_t> pending;               // submitted, not yet launched
    std::deque<cudaEvent_t> batches;            // done events of launched batches, oldest first
    std::map<cudaEvent_t, int> done_refs;       // tickets still holding a batch's done event
    uint64_t n_batches = 0, n_batched_tickets = 0;
    // profiling (HF_FLAG_PROFILE)
    unsigned long long* prof_dev = nullptr;  // u64[64] device counters
    std::vector<std::array<cudaEvent_t, 4>> prof_events;  // phases of runs not yet summed
    hf_profile_data prof_acc{};
};

namespace {

// Variation class of the autotuner: 0 for V = 1, else floor(log2 V), at most 7.
int vclass(uint32_t V)
{
    int c = 0;
    while (c < 7 && (2u << c) <= V) ++c;
    return V <= 1 ? 0 : c;
}

hf_status submit_batched(hf_ctx* ctx, uint32_t analysis_id, const Analysis& A, const hf_columns* hc, uint64_t N,
                         uint64_t first_event_id, uint64_t seed, uint32_t V, uint64_t* ticket);
void dispatcher_main(hf_ctx* ctx);
void release_done(hf_ctx* ctx, cudaEvent_t ev);

// Chooses the device for the calling thread.
hf_status use_device(hf_ctx* ctx)
{
    HF_CUDA(cudaSetDevice(ctx->device));
    return HF_OK;
}

bool known_kind(int k) { return k >= CUT_NJETS_MIN && k <= CUT_TTBAR_CHI2_MAX; }

}  // namespace

// Validates a descriptor and fills the kernel plan (no allocation).
hf_status hf::build_plan(const hf_analysis_desc* d, Plan& P)
{
    if (!d) return fail(HF_EINVAL, "desc is NULL");
    if (d->event_model != MODEL_SEMILEP && d->event_model != MODEL_DILEP)
        return fail(HF_EINVAL, "unknown event model");
    if (d->n_cuts < 1 || d->n_cuts > (uint32_t)MAX_CUTS || !d->cuts) return fail(HF_EINVAL, "n_cuts must be 1..16");
    if (!(d->sigma_t > 0) || !(d->sigma_W > 0)) return fail(HF_EINVAL, "widths must be > 0");
    if (!(d->sigma_jet >= 0.0f && d->sigma_jet <= 0.15f))
        return fail(HF_EINVAL, "sigma_jet must be in [0, 0.15] (jet scale factors stay positive)");
    if (!(d->sigma_met >= 0.0f) || !std::isfinite(d->sigma_met)) return fail(HF_EINVAL, "sigma_met must be >= 0");
    if (!(d->sigma_lep >= 0.0f && d->sigma_lep <= 0.15f)) return fail(HF_EINVAL, "sigma_lep must be in [0, 0.15]");
    if (d->hist_nbins < 1 || d->hist_nbins > (uint32_t)MAX_BINS || !(d->hist_lo < d->hist_hi))
        return fail(HF_EINVAL, "histogram: 1..1024 bins and lo < hi");
    if (d->record_levels >> d->n_cuts) return fail(HF_EINVAL, "record_levels names a cut level >= n_cuts");
    for (int i = 0; i < 4; ++i)
        if (d->record_vars[i] > HF_VAR_RECO3) return fail(HF_EINVAL, "record_vars: unknown HF_VAR_*");
    memset(&P, 0, sizeof P);
    P.model = d->event_model;
    P.n_cuts = (int)d->n_cuts;
    bool have_top = false, have_w = false, have_dl = false, have_h = false, have_full = false;
    for (int c = 0; c < P.n_cuts; ++c) {
        const hf_cut& cut = d->cuts[c];
        if (!known_kind(cut.kind)) return fail(HF_EINVAL, "unknown cut kind");
        for (int k = 0; k < 4; ++k)
            if (!std::isfinite(cut.params[k])) return fail(HF_EINVAL, "non-finite cut parameter");
        if (cut.dep_mask >> c) return fail(HF_EINVAL, "a cut may depend only on earlier user-order cuts");
        bool semi_only = cut.kind == CUT_W_NU_SOLVABLE || cut.kind == CUT_HADTOP_CHI2_MAX ||
                         cut.kind == CUT_TTBAR_CHI2_MAX;
        bool dl_only = cut.kind == CUT_LEP_OS || cut.kind == CUT_DILEP_SOLVABLE || cut.kind == CUT_HIGGS_WINDOW;
        if (semi_only && P.model != MODEL_SEMILEP) return fail(HF_EINVAL, "semileptonic cut in a dilepton analysis");
        if (dl_only && P.model != MODEL_DILEP) return fail(HF_EINVAL, "dilepton cut in a semileptonic analysis");
        P.kind[c] = cut.kind;
        P.p0[c] = cut.params[0];
        P.p1[c] = cut.params[1];
        P.dp0[c] = cut.params[0];
        P.dp1[c] = cut.params[1];
        have_top |= cut.kind == CUT_HADTOP_CHI2_MAX;
        have_w |= cut.kind == CUT_W_NU_SOLVABLE;
        have_dl |= cut.kind == CUT_DILEP_SOLVABLE;
        have_h |= cut.kind == CUT_HIGGS_WINDOW;
        have_full |= cut.kind == CUT_TTBAR_CHI2_MAX;
    }
    P.top_thr = 0.0f;
    for (int c = 0; c < P.n_cuts; ++c)
        if (P.kind[c] == CUT_HADTOP_CHI2_MAX) P.top_thr = std::max(P.top_thr, P.p0[c]);
    if (P.model == MODEL_SEMILEP && !((have_top || have_full) && have_w))
        return fail(HF_EINVAL, "semileptonic analysis needs HF_CUT_W_NU_SOLVABLE and HF_CUT_HADTOP_CHI2_MAX "
                               "or HF_CUT_TTBAR_CHI2_MAX");
    P.has_full = have_full ? 1 : 0;
    if (P.model == MODEL_DILEP && !(have_dl && have_h))
        return fail(HF_EINVAL, "dilepton analysis needs HF_CUT_DILEP_SOLVABLE and HF_CUT_HIGGS_WINDOW");
    P.mW = d->mW;
    P.mt = d->mt;
    P.sigma_t = d->sigma_t;
    P.sigma_W = d->sigma_W;
    P.inv_sigma_t = 1.0f / d->sigma_t;
    P.inv_sigma_W = 1.0f / d->sigma_W;
    P.mH = d->mH;
    {
        double h = (double)d->mW * (double)d->mW / 2.0;  // exact: 24-bit factors
        P.mW2half = (float)h;
        P.mW2half_lo = (float)(h - (double)P.mW2half);
    }
    P.sigma_jet = d->sigma_jet;
    P.sigma_met = d->sigma_met;
    P.smear_jets = d->sigma_jet != 0.0f;
    P.smear_met = d->sigma_met != 0.0f;
    P.sigma_lep = d->sigma_lep;
    P.smear_lep = d->sigma_lep != 0.0f;
    P.dsigma_lep = d->sigma_lep;
    if (d->per_event > HF_PER_EVENT_BEST) return fail(HF_EINVAL, "per_event must be HF_PER_EVENT_MEAN or _BEST");
    P.best = d->per_event == HF_PER_EVENT_BEST;
    P.nbins = (int)d->hist_nbins;
    P.lo = d->hist_lo;
    P.hi = d->hist_hi;
    P.w = (float)(((double)d->hist_hi - (double)d->hist_lo) / d->hist_nbins);
    P.dmW = d->mW;
    P.dmt = d->mt;
    P.dsigma_t = d->sigma_t;
    P.dsigma_W = d->sigma_W;
    P.dmH = d->mH;
    P.dsigma_jet = d->sigma_jet;
    P.dsigma_met = d->sigma_met;
    P.dlo = d->hist_lo;
    P.dhi = d->hist_hi;
    P.rec_levels = d->record_levels;
    for (int i = 0; i < 4; ++i) P.rec_var[i] = (int)d->record_vars[i];
    // FP32 error model: normals within 2.5 ulp (bound 4e-7 relative), |z| <= 5.8;
    // jet scale s = 1 + sigma z within sigma * 4e-7 * 5.8 / (1 - 5.8 sigma) + 2^-24
    // relative; a Gram-matrix mass squared within 2 s_rel + 12 u, the mass within half of
    // that plus 3 ulp (rsqrtf and the product).
    const double u = 5.9604644775390625e-08;
    P.z_rel = 4.0e-7f;
    double zmax = 5.8;
    double s_rel = (double)d->sigma_jet * 4.0e-7 * zmax / (1.0 - zmax * (double)d->sigma_jet) + u;
    P.s_rel = (float)s_rel;
    P.e_m = (float)(0.5 * (2.0 * s_rel + 12.0 * u) + 6.0 * u);
    P.safety = 4.0f;
    P.pz_tol = 2.5e-6f;
    // stages: cuts whose outcome does not depend on the variation are decided per event
    P.stage1 = 0;
    P.stage2 = 0;
    for (int c = 0; c < P.n_cuts; ++c) {
        int k = P.kind[c];
        // a smeared lepton moves its pT cut and the W-mass solvability to the units
        bool s1 = k == CUT_NJETS_MIN || k == CUT_NBTAG_MIN || k == CUT_LEP_OS ||
                  ((k == CUT_LEP_PT_MIN || k == CUT_W_NU_SOLVABLE) && !P.smear_lep) ||
                  (k == CUT_MET_MIN && !P.smear_met);
        if (s1) P.stage1 |= 1u << c;
        else P.stage2 |= 1u << c;
    }
    P.n_exec2 = 0;
    for (int c = 0; c < P.n_cuts; ++c)
        if (P.stage2 >> c & 1u) P.exec2[P.n_exec2++] = c;
    return HF_OK;
}

namespace {

hf_status ensure_arena(hf_ctx* ctx, size_t bytes)
{
    if (ctx->arena_bytes >= bytes) return HF_OK;
    if (ctx->arena) {
        HF_CUDA(cudaStreamSynchronize(ctx->s_comp));
        if (ctx->arena_free) HF_CUDA(cudaEventSynchronize(ctx->arena_free));
        cudaFree(ctx->arena);
        ctx->arena = nullptr;
        ctx->arena_bytes = 0;
    }
    for (auto& g : ctx->bgraphs) cudaGraphExecDestroy(g.second);  // captured for the old arena
    ctx->bgraphs.clear();
    size_t want = std::max(bytes, (size_t)64 << 20);
    cudaError_t e = cudaMalloc((void**)&ctx->arena, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HF_ENOMEM, "scratch arena allocation failed");
    }
    ctx->arena_bytes = want;
    return HF_OK;
}

// Per-cut records of a device-resident run: only for an analysis that
// records, with a counter to receive their number.
hf_status records_out(const Analysis& A, const hf_results& r, Out& O)
{
    if (!r.records || !A.plan.rec_levels) return HF_OK;
    if (A.plan.best) return fail(HF_EINVAL, "per-cut records are not kept with best-of-variations");
    if (!r.n_records) return fail(HF_EINVAL, "records given without n_records");
    if ((uintptr_t)r.records & 3) return fail(HF_EINVAL, "records must be 4-byte aligned");
    for (int i = 0; i < 4; ++i)
        if (A.plan.rec_var[i] >= VAR_RECO0 && !r.reco)
            return fail(HF_EINVAL, "recording a reconstructed quantity needs the reco output");
    O.rec = (Record*)r.records;
    O.rec_cap = r.record_cap;
    O.n_rec = (unsigned long long*)r.n_records;
    return HF_OK;
}

// Enqueues one run on stream st with the device memory at `scratch`.
hf_status enqueue_run(hf_ctx* ctx, Analysis& A, const Cols& C, uint64_t N, uint32_t V, const Out& Oin,
                      char* scratch, const RunLayout& L, uint64_t seed, uint64_t first_id, bool plain,
                      cudaStream_t st)
{
    Scratch S = make_scratch(scratch, L, A);
    Out O = Oin;
    if (!O.cutflow) O.cutflow = (unsigned long long*)(scratch + L.off_cutflow);
    if (!O.hist) O.hist = (unsigned long long*)(scratch + L.off_hist);
    if (!O.rc_total) O.rc_total = (unsigned long long*)(scratch + L.off_rctot);
    HF_CUDA(cudaMemsetAsync(scratch + L.off_small, 0, 256, st));
    HF_CUDA(cudaMemsetAsync(S.stats, 0, 8 * 3 * MAX_CUTS, st));
    HF_CUDA(cudaMemsetAsync(O.cutflow, 0, 8 * (A.plan.n_cuts + 1), st));
    HF_CUDA(cudaMemsetAsync(O.hist, 0, 8 * (A.plan.nbins + 2), st));
    HF_CUDA(cudaMemsetAsync(O.rc_total, 0, 8, st));
    if (O.rec) {
        O.maxf = (uint8_t*)(scratch + L.off_maxf);
        HF_CUDA(cudaMemsetAsync(O.n_rec, 0, 8, st));
    }
    if (N > 0xFFFFFFFFull) return fail(HF_EINVAL, "at most 2^32 - 1 events per call");
    if (N == 0) return HF_OK;
    bool use_plain = plain || (ctx->flags & HF_FLAG_PLAIN);
    if (use_plain && A.plan.best) return fail(HF_EINVAL, "best-of-variations does not run in the plain form");
    if (use_plain) S.exec2 = nullptr;
    cudaEvent_t* evp = nullptr;
    std::array<cudaEvent_t, 4> ev{};
    if (ctx->prof_dev && !use_plain) {
        S.prof = ctx->prof_dev;
        for (auto& x : ev) HF_CUDA(cudaEventCreate(&x));
        evp = ev.data();
    }
    const int upt = ctx->tune[A.plan.model == MODEL_DILEP ? 2 : 1][vclass(V)];
    HF_CUDA(launch_run(A.plan, C, (uint32_t)N, V, O, S, seed, first_id, use_plain, ctx->sms, st, evp, &ctx->side,
                       upt));
    if (evp) ctx->prof_events.push_back(ev);
    if (!use_plain && A.sched) HF_CUDA(launch_sched_update(A.sched, S.stats, st));
    if (ctx->flags & HF_FLAG_DEBUG_SYNC) HF_CUDA(cudaStreamSynchronize(st));
    return HF_OK;
}

// Host -> device copy on stream st.  Pageable source memory goes through the
// context's pinned staging ring when it has one and the copy fits: the bytes
// are copied on the host into the ring and from there asynchronously, so the
// caller's buffer is free again when this returns.  The ring fills in address
// order; a copy that does not fit before its end starts again at the
// beginning once every copy still in flight out of the ring has completed
// (every region in use lies below the fill point, so nothing else can be
// overwritten).
hf_status copy_h2d(hf_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st)
{
    if (!bytes) return HF_OK;
    if (ctx->staging && bytes <= ctx->staging_bytes) {
        cudaPointerAttributes at;
        const cudaError_t pe = cudaPointerGetAttributes(&at, src);
        if (pe != cudaSuccess) cudaGetLastError();
        if (pe != cudaSuccess || at.type == cudaMemoryTypeUnregistered) {
            if (ctx->stage_head + bytes > ctx->staging_bytes) {
                while (!ctx->stage_q.empty()) {
                    HF_CUDA(cudaEventSynchronize(ctx->stage_q.front().done));
                    cudaEventDestroy(ctx->stage_q.front().done);
                    ctx->stage_q.pop_front();
                }
                ctx->stage_head = 0;
            }
            const size_t lo = ctx->stage_head, hi = lo + bytes;
            memcpy(ctx->staging + lo, src, bytes);
            HF_CUDA(cudaMemcpyAsync(dst, ctx->staging + lo, bytes, cudaMemcpyHostToDevice, st));
            cudaEvent_t ev;
            HF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            HF_CUDA(cudaEventRecord(ev, st));
            ctx->stage_q.push_back(hf_ctx::StageRegion{lo, bytes, ev});
            ctx->stage_head = hi;
            return HF_OK;
        }
    }
    HF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    return HF_OK;
}

hf_status check_cols(const hf_columns* c, uint64_t N, int L)
{
    if (!c) return fail(HF_EINVAL, "columns are NULL");
    if (N > 0 && (!c->jet_off || !c->btag || !c->lep || !c->lep_q || !c->met))
        return fail(HF_EINVAL, "a column pointer is NULL");
    if (N > 0 && c->n_jets_total > 0 && !c->jets) return fail(HF_EINVAL, "jets is NULL");
    if (c->n_jets_total >= (1ull << 32)) return fail(HF_EINVAL, "at most 2^32 - 1 jets per chunk");
    if (((uintptr_t)c->jets & 15) || ((uintptr_t)c->lep & 15) || ((uintptr_t)c->met & 7))
        return fail(HF_EINVAL, "jets/lep must be 16-byte and met 8-byte aligned");
    (void)L;
    return HF_OK;
}

Analysis* get_analysis(hf_ctx* ctx, uint32_t id)
{
    if (id == 0 || id > ctx->analyses.size()) return nullptr;
    return ctx->analyses[id - 1].get();
}

hf_status run_device_impl(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* dev_cols, uint64_t N,
                          uint64_t first_event_id, uint64_t seed, uint32_t V, const hf_results* dev_out,
                          void* stream, bool plain)
{
    if (!ctx) return fail(HF_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    Analysis* A = get_analysis(ctx, analysis_id);
    if (!A) return fail(HF_ENOTFOUND, "unknown analysis id");
    if (V < 1 || V > HF_MAX_VARIATIONS) return fail(HF_EINVAL, "n_variations must be 1..4096");
    int L = A->plan.model == MODEL_DILEP ? 2 : 1;
    if (hf_status s = check_cols(dev_cols, N, L)) return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->s_comp;
    RunLayout RL = layout_for(N, V);
    if (hf_status s = ensure_arena(ctx, RL.scratch_bytes)) return s;
    if (ctx->arena_free) HF_CUDA(cudaStreamWaitEvent(st, ctx->arena_free, 0));
    Cols C;
    C.jet_off = dev_cols->jet_off;
    C.jets = (const float4*)dev_cols->jets;
    C.btag = dev_cols->btag;
    C.lep = (const float4*)dev_cols->lep;
    C.lep_q = dev_cols->lep_q;
    C.met = (const float2*)dev_cols->met;
    C.n_jets_total = dev_cols->n_jets_total;
    Out O;
    memset(&O, 0, sizeof O);
    if (dev_out) {
        O.mask = dev_out->mask;
        O.n_surv = dev_out->n_surv;
        O.reco = (float4*)dev_out->reco;
        O.cutflow = (unsigned long long*)dev_out->cutflow;
        O.hist = (unsigned long long*)dev_out->hist;
        O.rc_total = (unsigned long long*)dev_out->recheck_count;
        if (A->plan.best) O.best_v = dev_out->best_v;
        if (dev_out->reco && ((uintptr_t)dev_out->reco & 15)) return fail(HF_EINVAL, "reco must be 16-byte aligned");
        if (hf_status rs = records_out(*A, *dev_out, O)) return rs;
    }
    hf_status s = enqueue_run(ctx, *A, C, N, V, O, ctx->arena, RL, seed, first_event_id, plain, st);
    if (s) return s;
    if (!ctx->arena_free) HF_CUDA(cudaEventCreateWithFlags(&ctx->arena_free, cudaEventDisableTiming));
    HF_CUDA(cudaEventRecord(ctx->arena_free, st));
    return HF_OK;
}

}  // namespace

extern "C" {

const char* hf_last_error(hf_ctx*) { return g_err; }

hf_status hf_open(const hf_config* cfg, hf_ctx** out)
{
    if (!out) return fail(HF_EINVAL, "out is NULL");
    *out = nullptr;
    hf_config def;
    memset(&def, 0, sizeof def);
    if (!cfg) cfg = &def;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (cfg->device < 0 || cfg->device >= ndev) return fail(HF_EINVAL, "no such device");
    std::unique_ptr<hf_ctx> ctx(new hf_ctx);
    ctx->device = cfg->device;
    ctx->flags = cfg->flags;
    ctx->max_inflight = cfg->max_inflight ? cfg->max_inflight : 64;
    HF_CUDA(cudaSetDevice(ctx->device));
    HF_CUDA(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device));
    HF_CUDA(cudaStreamCreateWithFlags(&ctx->s_h2d, cudaStreamNonBlocking));
    HF_CUDA(cudaStreamCreateWithFlags(&ctx->s_comp, cudaStreamNonBlocking));
    HF_CUDA(cudaStreamCreateWithFlags(&ctx->s_d2h, cudaStreamNonBlocking));
    ctx->side.n = (ctx->flags & HF_FLAG_OVERLAP) ? MAX_SIDE : 0;
    for (int i = 0; i < ctx->side.n; ++i) {
        HF_CUDA(cudaStreamCreateWithFlags(&ctx->side.s[i], cudaStreamNonBlocking));
        HF_CUDA(cudaEventCreateWithFlags(&ctx->side.join[i], cudaEventDisableTiming));
    }
    HF_CUDA(cudaEventCreateWithFlags(&ctx->side.fork, cudaEventDisableTiming));
    ctx->user_stream = (cudaStream_t)cfg->stream;
    if (ctx->flags & HF_FLAG_PROFILE) {
        HF_CUDA(cudaMalloc((void**)&ctx->prof_dev, 64 * sizeof(unsigned long long)));
        HF_CUDA(cudaMemset(ctx->prof_dev, 0, 64 * sizeof(unsigned long long)));
    }
    if (cfg->hbm_budget_bytes) {
        ctx->budget = cfg->hbm_budget_bytes;
    } else {
        size_t fr = 0, tot = 0;
        HF_CUDA(cudaMemGetInfo(&fr, &tot));
        ctx->budget = (uint64_t)(0.8 * (double)fr);
    }
    // keep freed stream-ordered memory cached in the pool
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
        uint64_t thr = ctx->budget;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cfg->staging_bytes) {
        e = cudaHostAlloc((void**)&ctx->staging, cfg->staging_bytes, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(HF_ENOMEM, "pinned staging ring allocation failed");
        }
        ctx->staging_bytes = cfg->staging_bytes;
    }
    if (ctx->flags & HF_FLAG_BATCHING) ctx->dispatcher = std::thread(dispatcher_main, ctx.get());
    *out = ctx.release();
    return HF_OK;
}

hf_status hf_close(hf_ctx* ctx)
{
    if (!ctx) return HF_OK;
    if (ctx->dispatcher.joinable()) {
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->stop = true;
        }
        ctx->cv.notify_all();
        ctx->dispatcher.join();
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        // bounded wait for all streams
        auto t0 = std::chrono::steady_clock::now();
        std::vector<cudaStream_t> ss = {ctx->s_h2d, ctx->s_comp, ctx->s_d2h};
        for (int i = 0; i < ctx->side.n; ++i) ss.push_back(ctx->side.s[i]);
        for (cudaStream_t s : ss) {
            while (cudaStreamQuery(s) == cudaErrorNotReady) {
                if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
                    return fail(HF_ETIMEOUT, "in-flight work did not finish within 60 s");
                std::this_thread::sleep_for(std::chrono::microseconds(200));
            }
        }
        for (auto& kv : ctx->tickets) {
            if (kv.second.dmem) cudaFree(kv.second.dmem);
            if (kv.second.done && !kv.second.batched) cudaEventDestroy(kv.second.done);
        }
        for (auto& a : ctx->analyses)
            if (a->sched) cudaFree(a->sched);
        for (auto& g : ctx->bgraphs) cudaGraphExecDestroy(g.second);
        for (auto& d : ctx->done_refs) cudaEventDestroy(d.first);
        for (auto& kv : ctx->tickets)
            if (kv.second.h2d) cudaEventDestroy(kv.second.h2d);
        if (ctx->bstage) cudaFreeHost(ctx->bstage);
        if (ctx->bstage_free) cudaEventDestroy(ctx->bstage_free);
        for (auto& r : ctx->stage_q) cudaEventDestroy(r.done);
        if (ctx->staging) cudaFreeHost(ctx->staging);
        if (ctx->s_cap) cudaStreamDestroy(ctx->s_cap);
        if (ctx->arena) cudaFree(ctx->arena);
        if (ctx->arena_free) cudaEventDestroy(ctx->arena_free);
        if (ctx->prof_dev) cudaFree(ctx->prof_dev);
        for (auto& ev : ctx->prof_events)
            for (cudaEvent_t x : ev) cudaEventDestroy(x);
        cudaStreamDestroy(ctx->s_h2d);
        cudaStreamDestroy(ctx->s_comp);
        cudaStreamDestroy(ctx->s_d2h);
        for (int i = 0; i < ctx->side.n; ++i) {
            cudaStreamDestroy(ctx->side.s[i]);
            cudaEventDestroy(ctx->side.join[i]);
        }
        if (ctx->side.fork) cudaEventDestroy(ctx->side.fork);
    }
    delete ctx;
    return HF_OK;
}

hf_status hf_define_cuts(hf_ctx* ctx, const hf_analysis_desc* desc, uint32_t* analysis_id)
{
    if (!ctx || !analysis_id) return fail(HF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    std::unique_ptr<Analysis> A(new Analysis);
    if (hf_status s = hf::build_plan(desc, A->plan)) return s;
    A->cuts.assign(desc->cuts, desc->cuts + desc->n_cuts);
    A->no_sched = (ctx->flags & HF_FLAG_NO_SCHED) != 0;
    SchedDev sd;
    memset(&sd, 0, sizeof sd);
    const Plan& P = A->plan;
    sd.n_exec2 = P.n_exec2;
    sd.n_stage2 = P.n_exec2;
    for (int i = 0; i < P.n_exec2; ++i) {
        sd.exec2[i] = P.exec2[i];
        sd.stage2_cuts[i] = P.exec2[i];
    }
    sd.stage2_mask = P.stage2;
    for (int c = 0; c < P.n_cuts; ++c) {
        sd.dep_mask[c] = desc->cuts[c].dep_mask;
        sd.pinned[c] = desc->cuts[c].reorderable ? 0 : 1;
    }
    // implicit dependency: the Higgs window uses the two-neutrino pairing
    for (int c = 0; c < P.n_cuts; ++c)
        if (P.kind[c] == CUT_HIGGS_WINDOW)
            for (int d = 0; d < P.n_cuts; ++d)
                if (P.kind[d] == CUT_DILEP_SOLVABLE && d < c) sd.dep_mask[c] |= 1u << d;
    sd.frozen = A->no_sched ? 1 : 0;
    HF_CUDA(cudaMalloc((void**)&A->sched, sizeof(SchedDev)));
    HF_CUDA(cudaMemcpy(A->sched, &sd, sizeof sd, cudaMemcpyHostToDevice));
    ctx->analyses.push_back(std::move(A));
    *analysis_id = (uint32_t)ctx->analyses.size();
    return HF_OK;
}

hf_status hf_run_device(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* dev_cols, uint64_t n_events,
                        uint64_t first_event_id, uint64_t seed, uint32_t n_variations, const hf_results* dev_out,
                        void* stream)
{
    return run_device_impl(ctx, analysis_id, dev_cols, n_events, first_event_id, seed, n_variations, dev_out,
                           stream, false);
}

hf_status hf_run_device_plain(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* dev_cols, uint64_t n_events,
                              uint64_t first_event_id, uint64_t seed, uint32_t n_variations,
                              const hf_results* dev_out, void* stream)
{
    return run_device_impl(ctx, analysis_id, dev_cols, n_events, first_event_id, seed, n_variations, dev_out,
                           stream, true);
}

hf_status hf_device_error(hf_ctx* ctx, uint32_t* word)
{
    if (!ctx || !word) return fail(HF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    *word = 0;
    if (!ctx->arena) return HF_OK;
    if (ctx->arena_free) HF_CUDA(cudaEventSynchronize(ctx->arena_free));
    HF_CUDA(cudaMemcpy(word, ctx->arena + SM_ERR, 4, cudaMemcpyDeviceToHost));
    return HF_OK;
}

hf_status hf_submit_chunk(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* hc, uint64_t N,
                          uint64_t first_event_id, uint64_t seed, uint32_t V, uint64_t* ticket)
{
    if (!ctx || !ticket) return fail(HF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    Analysis* A = get_analysis(ctx, analysis_id);
    if (!A) return fail(HF_ENOTFOUND, "unknown analysis id");
    if (V < 1 || V > HF_MAX_VARIATIONS) return fail(HF_EINVAL, "n_variations must be 1..4096");
    const int L = A->plan.model == MODEL_DILEP ? 2 : 1;
    if (hf_status s = check_cols(hc, N, L)) return s;
    if (N > 0xFFFFFFFFull) return fail(HF_EINVAL, "at most 2^32 - 1 events per chunk");
    if (N > 0 && hc->jet_off[0] != 0) return fail(HF_EINVAL, "jet_off[0] must be 0");
    if (N > 0 && hc->jet_off[N] != hc->n_jets_total) return fail(HF_EINVAL, "jet_off[N] != n_jets_total");
    if (ctx->tickets.size() >= ctx->max_inflight) return fail(HF_EBUSY, "too many in-flight tickets");
    if (ctx->flags & HF_FLAG_BATCHING) {
        if (A->plan.best) return fail(HF_EINVAL, "best-of-variations analyses do not run batched");
        return submit_batched(ctx, analysis_id, *A, hc, N, first_event_id, seed, V, ticket);
    }
    const uint64_t J = hc->n_jets_total;
    ColLayout CL = col_layout(N, J, L);
    RunLayout RL = layout_for(N, V);
    ResLayout RR = res_layout(N);
    size_t bytes = CL.bytes + RL.scratch_bytes + RR.bytes;
    if (ctx->inflight_bytes + bytes > ctx->budget) return fail(HF_EBUSY, "HBM budget exhausted; retry later");
    Ticket T;
    T.id = ctx->next_ticket++;
    T.analysis = analysis_id;
    T.N = N;
    T.bytes = bytes;
    T.L = RL;
    T.R = RR;
    cudaError_t e = cudaMallocAsync((void**)&T.dmem, bytes, ctx->s_h2d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HF_ENOMEM, "device allocation for the chunk failed");
    }
    char* dc = T.dmem;
    char* dscr = T.dmem + CL.bytes;
    char* dres = dscr + RL.scratch_bytes;
    if (N > 0) {
        const struct {
            size_t off;
            const void* src;
            size_t bytes;
        } cp[6] = {{CL.off_jets, hc->jets, 16 * J},           {CL.off_lep, hc->lep, 16 * (size_t)L * N},
                   {CL.off_met, hc->met, 8 * N},              {CL.off_jet_off, hc->jet_off, 4 * (N + 1)},
                   {CL.off_btag, hc->btag, 2 * N},            {CL.off_lep_q, hc->lep_q, (size_t)L * N}};
        for (const auto& c : cp)
            if (hf_status s = copy_h2d(ctx, dc + c.off, c.src, c.bytes, ctx->s_h2d)) return s;
    }
    cudaEvent_t h2d;
    HF_CUDA(cudaEventCreateWithFlags(&h2d, cudaEventDisableTiming));
    HF_CUDA(cudaEventRecord(h2d, ctx->s_h2d));
    HF_CUDA(cudaStreamWaitEvent(ctx->s_comp, h2d, 0));
    cudaEventDestroy(h2d);
    Cols C;
    C.jet_off = (const uint32_t*)(dc + CL.off_jet_off);
    C.jets = (const float4*)(dc + CL.off_jets);
    C.btag = (const uint16_t*)(dc + CL.off_btag);
    C.lep = (const float4*)(dc + CL.off_lep);
    C.lep_q = (const int8_t*)(dc + CL.off_lep_q);
    C.met = (const float2*)(dc + CL.off_met);
    C.n_jets_total = J;
    Out O;
    memset(&O, 0, sizeof O);
    O.mask = (uint8_t*)(dres + RR.off_mask);
    O.n_surv = (uint16_t*)(dres + RR.off_nsurv);
    O.reco = (float4*)(dres + RR.off_reco);
    if (A->plan.best) O.best_v = (uint16_t*)(dres + RR.off_bestv);
    hf_status s = enqueue_run(ctx, *A, C, N, V, O, dscr, RL, seed, first_event_id, false, ctx->s_comp);
    HF_CUDA(cudaEventCreateWithFlags(&T.done, cudaEventDisableTiming));
    HF_CUDA(cudaEventRecord(T.done, ctx->s_comp));
    if (s) T.failed_launch = true;
    ctx->inflight_bytes += bytes;
    *ticket = T.id;
    ctx->tickets[T.id] = T;
    return s;
}

hf_status hf_poll(hf_ctx* ctx, uint64_t ticket, int32_t* state)
{
    if (!ctx || !state) return fail(HF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(HF_ENOTFOUND, "unknown ticket");
    if (it->second.failed_launch) {
        *state = HF_STATE_FAILED;
        return HF_OK;
    }
    if (it->second.batched && !it->second.launched) {
        *state = HF_STATE_QUEUED;
        return HF_OK;
    }
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaEventQuery(it->second.done);
    if (e == cudaSuccess) *state = HF_STATE_DONE;
    else if (e == cudaErrorNotReady) *state = HF_STATE_RUNNING;
    else {
        *state = HF_STATE_FAILED;
        return cuda_fail(e, "cudaEventQuery");
    }
    return HF_OK;
}

hf_status hf_fetch_results(hf_ctx* ctx, uint64_t ticket, hf_results* out, uint32_t timeout_ms)
{
    if (!ctx) return fail(HF_EINVAL, "ctx is NULL");
    if (out && out->records)
        return fail(HF_EINVAL, "per-cut records come from the device-resident entry points only");
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    while (true) {  // bounded wait: queued (batching) and then running
        cudaEvent_t done = nullptr;
        bool failed = false;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            auto it = ctx->tickets.find(ticket);
            if (it == ctx->tickets.end()) return fail(HF_ENOTFOUND, "unknown ticket");
            failed = it->second.failed_launch;
            if (!it->second.batched || it->second.launched) done = it->second.done;
        }
        if (failed) break;
        if (done) {
            cudaError_t e = cudaEventQuery(done);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) return cuda_fail(e, "waiting for the chunk");
        }
        if (std::chrono::steady_clock::now() - t0 >= std::chrono::milliseconds(timeout_ms))
            return fail(HF_ETIMEOUT, "chunk not finished within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(HF_ENOTFOUND, "unknown ticket");
    Ticket T = it->second;
    ctx->tickets.erase(it);
    ctx->inflight_bytes -= T.bytes;
    Analysis* A = get_analysis(ctx, T.analysis);
    // where this ticket's results live
    const char *d_err, *d_res, *d_cf, *d_hist, *d_rct;
    if (T.batched) {
        d_err = T.dmem + T.off_err;
        d_res = T.dmem + T.off_res;
        d_cf = T.dmem + T.off_cf;
        d_hist = T.dmem + T.off_hist;
        d_rct = T.dmem + T.off_rct;
    } else {
        const char* dscr = T.dmem + (T.bytes - T.L.scratch_bytes - T.R.bytes);
        d_err = dscr + T.L.off_small + SM_ERR;
        d_res = dscr + T.L.scratch_bytes;
        d_cf = dscr + T.L.off_cutflow;
        d_hist = dscr + T.L.off_hist;
        d_rct = dscr + T.L.off_rctot;
    }
    hf_status st = HF_OK;
    unsigned err = 0;
    cudaError_t e = cudaSuccess;
    if (!T.failed_launch) {
        e = cudaMemcpy(&err, d_err, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "reading the error word");
    }
    if (!st && T.failed_launch) st = fail(HF_ECUDA, "the chunk's launch failed");
    if (!st && (err & ERR_COLUMNS)) st = fail(HF_EINVAL, "malformed columns (offsets or n_jets > 12)");
    if (!st && out) {
        const uint64_t N = T.N;
        const int nc = A->plan.n_cuts, nb = A->plan.nbins;
        cudaStream_t s = ctx->s_d2h;
        if (out->mask && N) e = cudaMemcpyAsync(out->mask, d_res + T.R.off_mask, N, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && out->n_surv && N)
            e = cudaMemcpyAsync(out->n_surv, d_res + T.R.off_nsurv, 2 * N, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && out->reco && N)
            e = cudaMemcpyAsync(out->reco, d_res + T.R.off_reco, 16 * N, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && out->best_v && N && A->plan.best && !T.batched)
            e = cudaMemcpyAsync(out->best_v, d_res + T.R.off_bestv, 2 * N, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && out->cutflow)
            e = cudaMemcpyAsync(out->cutflow, d_cf, 8 * (nc + 1), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && out->hist)
            e = cudaMemcpyAsync(out->hist, d_hist, 8 * (nb + 2), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && out->recheck_count)
            e = cudaMemcpyAsync(out->recheck_count, d_rct, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "copying results");
    }
    if (T.batched && !T.launched) {
        // failed before launch: still queued copies may use the memory
        cudaStreamSynchronize(ctx->s_h2d);
    }
    cudaFreeAsync(T.dmem, ctx->s_d2h);
    if (T.batched) {
        if (T.done) release_done(ctx, T.done);
        if (T.h2d) cudaEventDestroy(T.h2d);
    } else if (T.done) {
        cudaEventDestroy(T.done);
    }
    return st;
}

hf_status hf_sched_state(hf_ctx* ctx, uint32_t analysis_id, int32_t* exec_order, uint64_t* evaluated,
                         uint64_t* passed, uint64_t* cost)
{
    if (!ctx) return fail(HF_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    Analysis* A = get_analysis(ctx, analysis_id);
    if (!A) return fail(HF_ENOTFOUND, "unknown analysis id");
    HF_CUDA(cudaStreamSynchronize(ctx->s_comp));
    if (ctx->arena_free) HF_CUDA(cudaEventSynchronize(ctx->arena_free));
    SchedDev sd;
    HF_CUDA(cudaMemcpy(&sd, A->sched, sizeof sd, cudaMemcpyDeviceToHost));
    const Plan& P = A->plan;
    if (exec_order) {
        // full execution order: stage-1 cuts (evaluated together per event) in user
        // order, then the stage-2 cuts in their current execution order
        int k = 0;
        for (int c = 0; c < P.n_cuts; ++c)
            if (P.stage1 >> c & 1u) exec_order[k++] = c;
        for (int i = 0; i < sd.n_exec2; ++i) exec_order[k++] = sd.exec2[i];
    }
    for (int c = 0; c < P.n_cuts; ++c) {
        if (evaluated) evaluated[c] = sd.tot_eval[c];
        if (passed) passed[c] = sd.tot_pass[c];
        if (cost) cost[c] = sd.tot_cost[c];
    }
    return HF_OK;
}

hf_status hf_set_exec_order(hf_ctx* ctx, uint32_t analysis_id, const int32_t* order)
{
    if (!ctx || !order) return fail(HF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    Analysis* A = get_analysis(ctx, analysis_id);
    if (!A) return fail(HF_ENOTFOUND, "unknown analysis id");
    const Plan& P = A->plan;
    unsigned seen = 0;
    for (int x = 0; x < P.n_cuts; ++x) {
        int c = order[x];
        if (c < 0 || c >= P.n_cuts || (seen >> c & 1u)) return fail(HF_EINVAL, "not a permutation of the cuts");
        unsigned deps = A->cuts[c].dep_mask;
        if ((deps & ~seen) != 0u) return fail(HF_EINVAL, "order violates a dependency");
        seen |= 1u << c;
    }
    SchedDev sd;
    HF_CUDA(cudaStreamSynchronize(ctx->s_comp));
    if (ctx->arena_free) HF_CUDA(cudaEventSynchronize(ctx->arena_free));
    HF_CUDA(cudaMemcpy(&sd, A->sched, sizeof sd, cudaMemcpyDeviceToHost));
    int k = 0;
    for (int x = 0; x < P.n_cuts; ++x)
        if (P.stage2 >> order[x] & 1u) sd.exec2[k++] = order[x];
    sd.n_exec2 = k;
    sd.frozen = 1;
    HF_CUDA(cudaMemcpy(A->sched, &sd, sizeof sd, cudaMemcpyHostToDevice));
    return HF_OK;
}

hf_status hf_profile(hf_ctx* ctx, hf_profile_data* out, int32_t reset)
{
    if (!ctx || !out) return fail(HF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    if (!ctx->prof_dev) {
        if (!(ctx->flags & HF_FLAG_BATCHING)) return fail(HF_ESTATE, "context not opened with HF_FLAG_PROFILE");
        memset(out, 0, sizeof *out);
        out->batches = ctx->n_batches;
        out->batched_chunks = ctx->n_batched_tickets;
        return HF_OK;
    }
    hf_profile_data& P = ctx->prof_acc;
    for (auto& ev : ctx->prof_events) {
        HF_CUDA(cudaEventSynchronize(ev[3]));
        float a = 0.f, b = 0.f, c = 0.f;
        HF_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
        HF_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
        HF_CUDA(cudaEventElapsedTime(&c, ev[2], ev[3]));
        P.ms_stage1 += a;
        P.ms_stage2 += b;
        P.ms_recheck += c;
        P.runs += 1;
        P.launches_stage2 += NBUCKET;
        for (cudaEvent_t x : ev) cudaEventDestroy(x);
    }
    ctx->prof_events.clear();
    unsigned long long cnt[64];
    HF_CUDA(cudaMemcpy(cnt, ctx->prof_dev, sizeof cnt, cudaMemcpyDeviceToHost));
    hf_profile_data r = P;
    r.units_stage2 = cnt[PROF_UNITS];
    r.events_stage2 = cnt[PROF_EVENTS];
    r.pairings_dilep = cnt[PROF_PAIRINGS];
    r.cands_top = cnt[PROF_CANDS];
    for (int i = 0; i < 16; ++i) {
        r.units_top[i] = cnt[PROF_TOP + i];
        r.units_dilep[i] = cnt[PROF_DILEP + i];
    }
    r.batches = ctx->n_batches;
    r.batched_chunks = ctx->n_batched_tickets;
    *out = r;
    if (reset) {
        memset(&ctx->prof_acc, 0, sizeof ctx->prof_acc);
        HF_CUDA(cudaMemset(ctx->prof_dev, 0, sizeof cnt));
    }
    return HF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batched runs
namespace {

struct BatchLayout {
    size_t off_dev, off_ch, off_plans, off_exec, off_stats, off_tpre, off_cnt, off_tctr, off_fb, off_bucket, off_rc,
        off_pend_cnt, off_pend_rng, off_pend_sum, off_pend_comp, off_rc_reco, off_rc_f, off_maxf, off_rec_pre, bytes;
    size_t table_bytes;  // [off_dev, off_fb): uploaded from the host
    unsigned rc_cap;
};

}  // namespace

namespace {

// Smallest power of two >= x (at least 4 KB): shared-memory sizes of the
// stage-2 grids are rounded to these classes so that batches with similar
// variation counts share one captured launch sequence.
// Shared-memory class of a batch's stage-2 kernels (part of the captured
// graph's key): rounded up to 4 KB, so that a few classes cover all batches
// while a class never exceeds what the largest tile needs by more than 4 KB
// (powers of two overshot the per-block limit for the largest tiles).
size_t smem_class(size_t x) { return (x + 4095) & ~(size_t)4095; }

// Enqueues one batch on st (ctx->mu held): validation, tables, upload and the
// captured launch sequence (captured on first use of its shape).
hf_status batch_enqueue(hf_ctx* ctx, const hf_chunk* chunks, uint32_t n_chunks, cudaStream_t st,
                        unsigned* const* errs = nullptr)
{
    if (n_chunks == 0) return HF_OK;
    // validate; semileptonic chunks first (the kernels take each model's chunks as one range)
    std::vector<uint32_t> order;
    order.reserve(n_chunks);
    uint32_t n_semi0 = 0;
    for (int pass = 0; pass < 3; ++pass)  // triplet-only semileptonic, full-fit semileptonic, dilepton
        for (uint32_t i = 0; i < n_chunks; ++i) {
            const hf_chunk& k = chunks[i];
            Analysis* A = get_analysis(ctx, k.analysis_id);
            if (!A) return fail(HF_ENOTFOUND, "a chunk names an unknown analysis id");
            const int cls = A->plan.model == MODEL_DILEP ? 2 : (A->plan.has_full ? 1 : 0);
            if (cls != pass) continue;
            if (A->plan.best) return fail(HF_EINVAL, "best-of-variations analyses do not run batched");
            if (pass == 0) ++n_semi0;
            if (k.n_variations < 1 || k.n_variations > HF_MAX_VARIATIONS)
                return fail(HF_EINVAL, "a chunk's n_variations is outside 1..4096");
            if (k.n_events > 0xFFFFFFFFull) return fail(HF_EINVAL, "at most 2^32 - 1 events per chunk");
            if (hf_status s = check_cols(&k.cols, k.n_events, 1)) return s;
            if (k.out.reco && ((uintptr_t)k.out.reco & 15)) return fail(HF_EINVAL, "reco must be 16-byte aligned");
            order.push_back(i);
        }
    // plans of the batch
    std::vector<uint32_t> plan_ids;  // analysis id per plan index
    std::map<uint32_t, uint32_t> plan_of;
    for (uint32_t i : order) {
        uint32_t a = chunks[i].analysis_id;
        if (!plan_of.count(a)) {
            plan_of[a] = (uint32_t)plan_ids.size();
            plan_ids.push_back(a);
        }
    }
    const uint32_t nc = n_chunks, np = (uint32_t)plan_ids.size();
    // host tables
    std::vector<BChunk> tab(nc);
    uint64_t ev_total = 0, blocks = 0, units_semi = 0, units_dl = 0, fb_words = 0;
    uint32_t n_semi = 0;
    BatchLaunch BL;
    memset(&BL, 0, sizeof BL);
    BL.sms = ctx->sms;
    for (uint32_t x = 0; x < nc; ++x) {
        const hf_chunk& k = chunks[order[x]];
        Analysis* A = get_analysis(ctx, k.analysis_id);
        const Plan& P = A->plan;
        BChunk& b = tab[x];
        memset(&b, 0, sizeof b);
        b.C.jet_off = k.cols.jet_off;
        b.C.jets = (const float4*)k.cols.jets;
        b.C.btag = k.cols.btag;
        b.C.lep = (const float4*)k.cols.lep;
        b.C.lep_q = k.cols.lep_q;
        b.C.met = (const float2*)k.cols.met;
        b.C.n_jets_total = k.cols.n_jets_total;
        b.O.mask = k.out.mask;
        b.O.n_surv = k.out.n_surv;
        b.O.reco = (float4*)k.out.reco;
        b.O.cutflow = (unsigned long long*)k.out.cutflow;
        b.O.hist = (unsigned long long*)k.out.hist;
        b.O.rc_total = (unsigned long long*)k.out.recheck_count;
        if (hf_status rs = records_out(*A, k.out, b.O)) return rs;
        if (!b.O.cutflow) fb_words += MAX_CUTS + 1;
        if (!b.O.hist) fb_words += MAX_BINS + 2;
        if (!b.O.rc_total) fb_words += 1;
        b.seed = k.seed;
        b.first_id = k.first_event_id;
        b.V = k.n_variations;
        b.n = (uint32_t)k.n_events;
        b.plan = plan_of[k.analysis_id];
        b.model = (uint32_t)P.model;
        b.blk0 = (uint32_t)blocks;
        b.ev0 = ev_total;
        b.err = errs ? errs[order[x]] : nullptr;
        const uint64_t units = (uint64_t)b.n * b.V;
        if (P.model == MODEL_DILEP) {
            b.ept = (uint32_t)dl_ev_per_tile(b.V, ctx->tune[2][vclass(b.V)]);
            BL.dilep = true;
            BL.smem_dilep = std::max(BL.smem_dilep, smem_class(dl_smem_bytes((int)b.ept, (int)(b.ept * b.V), false)));
            units_dl += units;
        } else {
            b.ept = (uint32_t)ev_per_tile_for(b.V, ctx->tune[1][vclass(b.V)]);
            ++n_semi;
            if (P.has_full) BL.full_mask = (1u << NBUCKET) - 1;
            else BL.semi_mask = (1u << NBUCKET) - 1;
            for (int n = 0; n < NBUCKET; ++n)
                BL.smem_semi[n] = std::max(BL.smem_semi[n],
                                           smem_class(semi_tile_bytes(n, (int)b.ept, (int)(b.ept * b.V))));
            units_semi += units;
        }
        ev_total += b.n;
        blocks += (b.n + BLOCK1 - 1) / BLOCK1;
    }
    if (blocks >= (1ull << 31)) return fail(HF_EINVAL, "batch too large (stage-1 blocks)");
    // device layout (one region of the context's arena)
    BatchLayout L;
    size_t o = 0;
    L.off_dev = o;
    o += sizeof(BatchDev);
    L.off_ch = o = align_up(o, 256);
    o += sizeof(BChunk) * nc;
    L.off_plans = o = align_up(o, 256);
    o += sizeof(Plan) * np;
    L.off_exec = o = align_up(o, 256);
    o += sizeof(void*) * np;
    L.table_bytes = o;
    L.off_stats = o = align_up(o, 256);
    o += 8 * 3 * MAX_CUTS * (size_t)np;
    L.off_tpre = o = align_up(o, 256);
    o += 4 * (size_t)NBUCKET * (nc + 1);
    L.off_cnt = o = align_up(o, 256);
    o += 4 * 32 * (size_t)nc;
    L.off_tctr = o = align_up(o, 256);
    o += 4 * 32;
    L.off_fb = o = align_up(o, 256);
    o += 8 * fb_words;
    L.off_bucket = o = align_up(o, 256);
    o += sizeof(uint2) * std::max<uint64_t>(ev_total, 1);
    // recheck capacity: ~0.05 % of semileptonic and ~5 % of dilepton units are
    // flagged; beyond the list the units are evaluated in place (slower, exact)
    uint64_t cap = 65536 + units_semi / 256 + units_dl / 16;
    cap = std::min<uint64_t>(cap, 1u << 28);
    L.rc_cap = (unsigned)cap;
    L.off_rc = o = align_up(o, 256);
    o += sizeof(RcEntry) * cap;
    L.off_pend_cnt = o = align_up(o, 256);
    o += 4 * cap;
    L.off_pend_rng = o = align_up(o, 256);
    o += 8 * cap;
    L.off_pend_sum = o = align_up(o, 256);
    o += 16 * cap;
    L.off_pend_comp = o = align_up(o, 256);
    o += 16 * cap;
    L.off_rc_reco = o = align_up(o, 256);
    o += 16 * cap;
    L.off_rc_f = o = align_up(o, 256);
    o += sizeof(RcRes) * cap;
    L.off_maxf = o = align_up(o, 256);
    o += std::max<uint64_t>(ev_total, 1);
    L.off_rec_pre = o = align_up(o, 256);
    o += 8 * (blocks + 1);
    L.bytes = align_up(o, 256);
    // the small counter block of single runs (error word at SM_ERR) stays at the
    // arena's start, so that hf_device_error reads batches too
    const size_t base_off = 256;
    if (hf_status s = ensure_arena(ctx, base_off + L.bytes)) return s;
    if (ctx->arena_free) HF_CUDA(cudaStreamWaitEvent(st, ctx->arena_free, 0));
    char* dbase = ctx->arena + base_off;
    // fill in device addresses
    unsigned* cnt = (unsigned*)(dbase + L.off_cnt);
    unsigned long long* fb = (unsigned long long*)(dbase + L.off_fb);
    for (uint32_t x = 0; x < nc; ++x) {
        BChunk& b = tab[x];
        b.cnt = cnt + 32 * (size_t)x;
        if (!b.O.cutflow) { b.O.cutflow = fb; fb += MAX_CUTS + 1; }
        if (!b.O.hist) { b.O.hist = fb; fb += MAX_BINS + 2; }
        if (!b.O.rc_total) { b.O.rc_total = fb; fb += 1; }
        if (b.O.rec) {
            b.O.maxf = (uint8_t*)(dbase + L.off_maxf) + b.ev0;
            BL.records = true;
        }
    }
    BatchDev B;
    memset(&B, 0, sizeof B);
    B.ch = (const BChunk*)(dbase + L.off_ch);
    B.plans = (const Plan*)(dbase + L.off_plans);
    B.exec = (const int* const*)(dbase + L.off_exec);
    B.stats = (unsigned long long*)(dbase + L.off_stats);
    B.tpre = (unsigned*)(dbase + L.off_tpre);
    B.tctr = (unsigned*)(dbase + L.off_tctr);
    B.bucket = (uint2*)(dbase + L.off_bucket);
    B.n_chunks = nc;
    B.n_semi = n_semi;
    B.n_semi0 = n_semi0;
    B.n_blocks = (uint32_t)blocks;
    B.n_plans = np;
    B.rec_pre = (unsigned long long*)(dbase + L.off_rec_pre);
    {
        Scratch& S = B.S;
        char* sm = ctx->arena;  // small counter block of the arena
        S.nhist = S.cursor = S.tile_ctr = nullptr;
        S.rc_count = (unsigned*)(sm + SM_RC);
        S.rc_valid = (unsigned*)(sm + SM_RCVALID);
        S.pend_count = (unsigned*)(sm + SM_PEND);
        S.err = (unsigned*)(sm + SM_ERR);
        S.bucket = B.bucket;
        S.rc = (RcEntry*)(dbase + L.off_rc);
        S.rc_cap = L.rc_cap;
        S.pend_cnt = (unsigned*)(dbase + L.off_pend_cnt);
        S.pend_rng = (uint2*)(dbase + L.off_pend_rng);
        S.rc_reco = (float4*)(dbase + L.off_rc_reco);
        S.rc_res = (RcRes*)(dbase + L.off_rc_f);
        S.pend_sum = (float4*)(dbase + L.off_pend_sum);
        S.pend_comp = (float4*)(dbase + L.off_pend_comp);
        S.stats = nullptr;
        S.prof = nullptr;
        S.exec2 = nullptr;
        S.n_exec2 = 0;
        S.chunk = 0;
    }
    // host staging of the tables (pinned; reused once its last upload is done)
    if (ctx->bstage_free) HF_CUDA(cudaEventSynchronize(ctx->bstage_free));
    if (ctx->bstage_bytes < L.table_bytes) {
        if (ctx->bstage) cudaFreeHost(ctx->bstage);
        ctx->bstage = nullptr;
        ctx->bstage_bytes = 0;
        size_t want = std::max(L.table_bytes, (size_t)1 << 20);
        if (cudaHostAlloc((void**)&ctx->bstage, want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return fail(HF_ENOMEM, "pinned staging of the batch tables failed");
        }
        ctx->bstage_bytes = want;
    }
    char* h = ctx->bstage;
    memcpy(h + L.off_dev, &B, sizeof B);
    memcpy(h + L.off_ch, tab.data(), sizeof(BChunk) * nc);
    for (uint32_t p = 0; p < np; ++p) {
        Analysis* A = get_analysis(ctx, plan_ids[p]);
        memcpy(h + L.off_plans + sizeof(Plan) * p, &A->plan, sizeof(Plan));
        if (!A->sched) return fail(HF_ESTATE, "analysis without scheduler state");
        // device address of the execution order inside the analysis's SchedDev
        const int* ex = (const int*)((const char*)A->sched + offsetof(SchedDev, exec2));
        memcpy(h + L.off_exec + sizeof(void*) * p, &ex, sizeof(void*));
    }
    HF_CUDA(cudaMemcpyAsync(dbase, h, L.table_bytes, cudaMemcpyHostToDevice, st));
    if (!ctx->bstage_free) HF_CUDA(cudaEventCreateWithFlags(&ctx->bstage_free, cudaEventDisableTiming));
    HF_CUDA(cudaEventRecord(ctx->bstage_free, st));
    // the launch sequence: replay the captured graph when it was captured for
    // the same arena, table layout, launch shape and scheduler states
    const BatchDev* Bd = (const BatchDev*)(dbase + L.off_dev);
    std::vector<uint64_t> key = {(uint64_t)(uintptr_t)Bd, (uint64_t)ctx->side.n, BL.semi_mask, BL.full_mask,
                                 BL.dilep, BL.records, BL.smem_dilep, np};
    for (int n = 0; n < NBUCKET; ++n) key.push_back(BL.smem_semi[n]);
    for (uint32_t p = 0; p < np; ++p) {
        Analysis* A = get_analysis(ctx, plan_ids[p]);
        key.push_back((uint64_t)(uintptr_t)A->sched);
        key.push_back(A->no_sched ? 1 : 0);
    }
    auto git = ctx->bgraphs.find(key);
    if (git == ctx->bgraphs.end()) {
        if (ctx->bgraphs.size() >= 32) {  // bounded cache of shapes
            for (auto& g : ctx->bgraphs) cudaGraphExecDestroy(g.second);
            ctx->bgraphs.clear();
        }
        if (!ctx->s_cap) HF_CUDA(cudaStreamCreateWithFlags(&ctx->s_cap, cudaStreamNonBlocking));
        HF_CUDA(cudaStreamBeginCapture(ctx->s_cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_batch(Bd, BL, ctx->s_cap, &ctx->side);
        for (uint32_t p = 0; p < np && e == cudaSuccess; ++p) {
            Analysis* A = get_analysis(ctx, plan_ids[p]);
            e = launch_sched_update(A->sched, B.stats + (size_t)p * 3 * MAX_CUTS, ctx->s_cap);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ctx->s_cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(e != cudaSuccess ? e : e2, "capturing the batch launch sequence");
        }
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(batch)");
        git = ctx->bgraphs.emplace(key, ge).first;
    }
    HF_CUDA(cudaGraphLaunch(git->second, st));
    if (!ctx->arena_free) HF_CUDA(cudaEventCreateWithFlags(&ctx->arena_free, cudaEventDisableTiming));
    HF_CUDA(cudaEventRecord(ctx->arena_free, st));
    if (ctx->flags & HF_FLAG_DEBUG_SYNC) HF_CUDA(cudaStreamSynchronize(st));
    return HF_OK;
}

}  // namespace

extern "C" hf_status hf_run_batch(hf_ctx* ctx, const hf_chunk* chunks, uint32_t n_chunks, void* stream)
{
    if (!ctx) return fail(HF_EINVAL, "ctx is NULL");
    if (n_chunks > 0 && !chunks) return fail(HF_EINVAL, "chunks is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->s_comp;
    return batch_enqueue(ctx, chunks, n_chunks, st);
}

// ------------------------------------------------------------------ continuous batching
namespace {

// hf_submit_chunk with HF_FLAG_BATCHING (ctx->mu held): admission by the HBM
// budget, one allocation for the chunk's columns and results, the copies on
// the H2D stream, and the ticket queued for the dispatcher.
hf_status submit_batched(hf_ctx* ctx, uint32_t analysis_id, const Analysis& A, const hf_columns* hc, uint64_t N,
                         uint64_t first_event_id, uint64_t seed, uint32_t V, uint64_t* ticket)
{
    const int L = A.plan.model == MODEL_DILEP ? 2 : 1;
    const uint64_t J = hc->n_jets_total;
    ColLayout CL = col_layout(N, J, L);
    ResLayout RR = res_layout(N);
    Ticket T;
    T.off_res = CL.bytes;
    T.off_cf = align_up(CL.bytes + RR.bytes, 256);
    T.off_hist = T.off_cf + 8 * (MAX_CUTS + 1);
    T.off_rct = T.off_hist + 8 * (MAX_BINS + 2);
    T.off_err = T.off_rct + 8;
    const size_t bytes = align_up(T.off_err + 4, 256);
    if (ctx->inflight_bytes + bytes > ctx->budget) return fail(HF_EBUSY, "HBM budget exhausted; retry later");
    T.id = ctx->next_ticket++;
    T.analysis = analysis_id;
    T.N = N;
    T.bytes = bytes;
    T.R = RR;
    T.batched = true;
    cudaError_t e = cudaMallocAsync((void**)&T.dmem, bytes, ctx->s_h2d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HF_ENOMEM, "device allocation for the chunk failed");
    }
    char* dc = T.dmem;
    if (N > 0) {
        const struct {
            size_t off;
            const void* src;
            size_t bytes;
        } cp[6] = {{CL.off_jets, hc->jets, 16 * J},           {CL.off_lep, hc->lep, 16 * (size_t)L * N},
                   {CL.off_met, hc->met, 8 * N},              {CL.off_jet_off, hc->jet_off, 4 * (N + 1)},
                   {CL.off_btag, hc->btag, 2 * N},            {CL.off_lep_q, hc->lep_q, (size_t)L * N}};
        for (const auto& c : cp)
            if (hf_status s = copy_h2d(ctx, dc + c.off, c.src, c.bytes, ctx->s_h2d)) return s;
    }
    HF_CUDA(cudaMemsetAsync(dc + T.off_err, 0, 4, ctx->s_h2d));
    HF_CUDA(cudaEventCreateWithFlags(&T.h2d, cudaEventDisableTiming));
    HF_CUDA(cudaEventRecord(T.h2d, ctx->s_h2d));
    hf_chunk& c = T.ch;
    c.analysis_id = analysis_id;
    c.n_variations = V;
    c.n_events = N;
    c.first_event_id = first_event_id;
    c.seed = seed;
    c.cols.jet_off = (const uint32_t*)(dc + CL.off_jet_off);
    c.cols.jets = (const float*)(dc + CL.off_jets);
    c.cols.btag = (const uint16_t*)(dc + CL.off_btag);
    c.cols.lep = (const float*)(dc + CL.off_lep);
    c.cols.lep_q = (const int8_t*)(dc + CL.off_lep_q);
    c.cols.met = (const float*)(dc + CL.off_met);
    c.cols.n_jets_total = J;
    char* dres = dc + T.off_res;
    c.out.mask = (uint8_t*)(dres + RR.off_mask);
    c.out.n_surv = (uint16_t*)(dres + RR.off_nsurv);
    c.out.reco = (float*)(dres + RR.off_reco);
    c.out.cutflow = (uint64_t*)(dc + T.off_cf);
    c.out.hist = (uint64_t*)(dc + T.off_hist);
    c.out.recheck_count = (uint64_t*)(dc + T.off_rct);
    ctx->inflight_bytes += bytes;
    *ticket = T.id;
    ctx->tickets[T.id] = T;
    ctx->pending.push_back(T.id);
    ctx->cv.notify_one();
    return HF_OK;
}

// Drops one reference to a batch's done event (destroyed with the last).
void release_done(hf_ctx* ctx, cudaEvent_t ev)
{
    auto it = ctx->done_refs.find(ev);
    if (it == ctx->done_refs.end()) return;
    if (--it->second == 0) {
        cudaEventDestroy(ev);
        ctx->done_refs.erase(it);
    }
}

// The dispatcher of continuous batching: whenever chunks are queued and at
// most one launched batch is still unfinished, it launches everything queued
// (up to a size limit) as one batch after their copies; chunks that arrive
// while batches run join the next one, and their copies overlap the running
// batch.
void dispatcher_main(hf_ctx* ctx)
{
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (true) {
        ctx->cv.wait(lk, [ctx] { return ctx->stop || !ctx->pending.empty(); });
        if (ctx->stop) break;
        while (true) {
            while (!ctx->batches.empty() && cudaEventQuery(ctx->batches.front()) != cudaErrorNotReady) {
                release_done(ctx, ctx->batches.front());
                ctx->batches.pop_front();
            }
            if (ctx->batches.size() < 2 || ctx->stop) break;
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        }
        if (ctx->stop) break;
        std::vector<hf_chunk> chs;
        std::vector<unsigned*> errs;
        std::vector<uint64_t> ids;
        uint64_t units = 0;
        while (!ctx->pending.empty() && chs.size() < 4096 && units < (1ull << 31)) {
            const uint64_t id = ctx->pending.front();
            ctx->pending.pop_front();
            auto it = ctx->tickets.find(id);
            if (it == ctx->tickets.end()) continue;
            Ticket& T = it->second;
            cudaStreamWaitEvent(ctx->s_comp, T.h2d, 0);
            chs.push_back(T.ch);
            errs.push_back((unsigned*)(T.dmem + T.off_err));
            ids.push_back(id);
            units += T.ch.n_events * T.ch.n_variations;
        }
        if (chs.empty()) continue;
        const hf_status st = batch_enqueue(ctx, chs.data(), (uint32_t)chs.size(), ctx->s_comp, errs.data());
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, ctx->s_comp);
        ctx->done_refs[ev] = (int)ids.size() + 1;  // + the reference of ctx->batches
        ctx->batches.push_back(ev);
        for (uint64_t id : ids) {
            Ticket& T = ctx->tickets[id];
            T.launched = true;
            T.done = ev;
            if (st != HF_OK || e != cudaSuccess) T.failed_launch = true;
        }
        ++ctx->n_batches;
        ctx->n_batched_tickets += ids.size();
    }
}

}  // namespace

// ------------------------------------------------------------------ autotuner
extern "C" hf_status hf_autotune(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* dev_cols, uint64_t n_events,
                                 uint32_t n_variations, uint64_t seed, int32_t* units_per_tile)
{
    if (!ctx || !dev_cols) return fail(HF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    Analysis* A = get_analysis(ctx, analysis_id);
    if (!A) return fail(HF_ENOTFOUND, "unknown analysis id");
    const uint32_t V = n_variations;
    if (V < 1 || V > HF_MAX_VARIATIONS) return fail(HF_EINVAL, "n_variations must be 1..4096");
    if (n_events == 0 || n_events > 0xFFFFFFFFull) return fail(HF_EINVAL, "sample must have 1..2^32-1 events");
    if (hf_status s = check_cols(dev_cols, n_events, 1)) return s;
    const bool dl = A->plan.model == MODEL_DILEP;
    static const int cand_semi[] = {128, 256, 512, 1024};
    static const int cand_dl[] = {32, 64, 128, 256};
    const int* cand = dl ? cand_dl : cand_semi;
    int& slot = ctx->tune[dl ? 2 : 1][vclass(V)];
    const int saved = slot;
    Cols C;
    C.jet_off = dev_cols->jet_off;
    C.jets = (const float4*)dev_cols->jets;
    C.btag = dev_cols->btag;
    C.lep = (const float4*)dev_cols->lep;
    C.lep_q = dev_cols->lep_q;
    C.met = (const float2*)dev_cols->met;
    C.n_jets_total = dev_cols->n_jets_total;
    Out O;
    memset(&O, 0, sizeof O);
    RunLayout RL = layout_for(n_events, V);
    if (hf_status s = ensure_arena(ctx, RL.scratch_bytes)) return s;
    cudaStream_t st = ctx->s_comp;
    if (ctx->arena_free) HF_CUDA(cudaStreamWaitEvent(st, ctx->arena_free, 0));
    cudaEvent_t e0, e1;
    HF_CUDA(cudaEventCreate(&e0));
    HF_CUDA(cudaEventCreate(&e1));
    const int dflt = dl ? 128 : UNITS_PER_TILE;  // the untuned shape (one of the candidates)
    float best_ms = 0.f, dflt_ms = 0.f;
    int best = 0;
    hf_status rs = HF_OK;
    unsigned long long* prof = ctx->prof_dev;
    ctx->prof_dev = nullptr;  // tuning runs are not profiled
    for (int c = 0; c < 4 && rs == HF_OK; ++c) {
        slot = cand[c];
        float t3[3] = {0.f, 0.f, 0.f};
        for (int rep = 0; rep < 4 && rs == HF_OK; ++rep) {  // one warm-up, then the median of three
            cudaEventRecord(e0, st);
            rs = enqueue_run(ctx, *A, C, n_events, V, O, ctx->arena, RL, seed, 0, false, st);
            cudaEventRecord(e1, st);
            if (rs == HF_OK && cudaEventSynchronize(e1) == cudaSuccess && rep > 0)
                cudaEventElapsedTime(&t3[rep - 1], e0, e1);
        }
        std::sort(t3, t3 + 3);
        const float ms = t3[1];
        if (cand[c] == dflt) dflt_ms = ms;
        if (rs == HF_OK && (best == 0 || ms < best_ms)) {
            best = cand[c];
            best_ms = ms;
        }
    }
    // keep the default unless a candidate is clearly faster (timing noise)
    if (best != dflt && dflt_ms > 0.f && best_ms > 0.97f * dflt_ms) best = dflt;
    ctx->prof_dev = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ctx->arena_free) cudaEventCreateWithFlags(&ctx->arena_free, cudaEventDisableTiming);
    cudaEventRecord(ctx->arena_free, st);
    if (rs != HF_OK) {
        slot = saved;
        return rs;
    }
    slot = best;
    if (units_per_tile) *units_per_tile = best;
    return HF_OK;
}

// ------------------------------------------------------------------ HL-LHC selection
extern "C" hf_status hf_run_hl(hf_ctx* ctx, const hf_hl_desc* d, const hf_hl_columns* c, uint64_t N,
                               uint64_t first_event_id, uint64_t seed, uint32_t V, const hf_hl_results* out,
                               void* stream)
{
    if (!ctx || !d || !c) return fail(HF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (hf_status s = use_device(ctx)) return s;
    if (V < 1 || V > HF_MAX_VARIATIONS) return fail(HF_EINVAL, "n_variations must be 1..4096");
    if (N > 0xFFFFFFFFull) return fail(HF_EINVAL, "at most 2^32 - 1 events per call");
    if (d->hist_nbins < 1 || d->hist_nbins > MAX_BINS || !(d->hist_lo < d->hist_hi))
        return fail(HF_EINVAL, "histogram: 1..1024 bins and hist_lo < hist_hi");
    if (!(d->eta_bounds[0] > 0.0f && d->eta_bounds[0] < d->eta_bounds[1] && d->eta_bounds[1] < d->eta_bounds[2] &&
          d->eta_bounds[2] < 20.0f))
        return fail(HF_EINVAL, "eta_bounds must satisfy 0 < b0 < b1 < b2 < 20");
    if (!(d->dr_iso > 0.0f) || !(d->sigma_met >= 0.0f) || !(d->met_min >= 0.0f) || !(d->mll_min >= 0.0f) ||
        !(d->mtw_min >= 0.0f))
        return fail(HF_EINVAL, "thresholds must be >= 0 (dr_iso > 0)");
    if (N > 0 && (!c->jet_off || !c->btag || !c->lep_off || !c->met || (c->n_jets_total && !c->jets) ||
                  (c->n_leptons_total && (!c->lep || !c->lep_q || !c->lep_flav))))
        return fail(HF_EINVAL, "a column pointer is NULL");
    if (((uintptr_t)c->jets & 15) || ((uintptr_t)c->lep & 15) || ((uintptr_t)c->met & 7) ||
        ((uintptr_t)c->jet_off & 3) || ((uintptr_t)c->lep_off & 3) || ((uintptr_t)c->btag & 1))
        return fail(HF_EINVAL, "jets/lep must be 16-byte, met 8-byte, offsets 4-byte and btag 2-byte aligned");
    if (out && (((uintptr_t)out->counts & 7) || ((uintptr_t)out->hist & 7)))
        return fail(HF_EINVAL, "counts and hist must be 8-byte aligned");
    HLPlan H;
    memset(&H, 0, sizeof H);
    H.met_min = d->met_min;
    H.mll_min = d->mll_min;
    H.mtw_min = d->mtw_min;
    H.dr2 = (float)((double)d->dr_iso * (double)d->dr_iso);
    H.dr_iso = d->dr_iso;
    H.dmet_min = d->met_min;
    H.dmll_min = d->mll_min;
    H.dmtw_min = d->mtw_min;
    H.ddr_iso = d->dr_iso;
    for (int b = 0; b < 3; ++b) {
        H.deta[b] = d->eta_bounds[b];
        H.sh[b] = (float)std::sinh((double)d->eta_bounds[b]);
    }
    H.smear = d->sigma_met != 0.0f;
    H.sigma_met = d->sigma_met;
    H.dsigma_met = d->sigma_met;
    H.z_rel = 4.0e-7f;
    H.safety = 4.0f;
    H.nbins = (int)d->hist_nbins;
    H.lo = d->hist_lo;
    H.hi = d->hist_hi;
    H.w = (float)(((double)d->hist_hi - (double)d->hist_lo) / d->hist_nbins);
    H.dlo = d->hist_lo;
    H.dhi = d->hist_hi;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->s_comp;
    // the small counter block at the arena's start holds the error word; the
    // counts and histograms the caller skips go after it
    const size_t off_counts = 256, off_hist = off_counts + 64, bytes = off_hist + 8 * 5 * (MAX_BINS + 2);
    if (hf_status s = ensure_arena(ctx, bytes)) return s;
    if (ctx->arena_free) HF_CUDA(cudaStreamWaitEvent(st, ctx->arena_free, 0));
    HLOut O;
    O.counts = (out && out->counts) ? (unsigned long long*)out->counts : (unsigned long long*)(ctx->arena + off_counts);
    O.hist = (out && out->hist) ? (unsigned long long*)out->hist : (unsigned long long*)(ctx->arena + off_hist);
    O.channel = out ? out->channel : nullptr;
    O.err = (unsigned*)(ctx->arena + SM_ERR);
    HF_CUDA(cudaMemsetAsync(ctx->arena, 0, 256, st));
    HF_CUDA(cudaMemsetAsync(O.counts, 0, 8 * 6, st));
    HF_CUDA(cudaMemsetAsync(O.hist, 0, 8 * 5 * (size_t)(d->hist_nbins + 2), st));
    HLCols C;
    C.jet_off = c->jet_off;
    C.jets = (const float4*)c->jets;
    C.btag = c->btag;
    C.lep_off = c->lep_off;
    C.lep = (const float4*)c->lep;
    C.lep_q = c->lep_q;
    C.lep_flav = c->lep_flav;
    C.met = (const float2*)c->met;
    C.n_jets = c->n_jets_total;
    C.n_leps = c->n_leptons_total;
    HF_CUDA(launch_hl(H, C, (uint32_t)N, V, seed, first_event_id, O, ctx->sms, st));
    if (!ctx->arena_free) HF_CUDA(cudaEventCreateWithFlags(&ctx->arena_free, cudaEventDisableTiming));
    HF_CUDA(cudaEventRecord(ctx->arena_free, st));
    if (ctx->flags & HF_FLAG_DEBUG_SYNC) HF_CUDA(cudaStreamSynchronize(st));
    return HF_OK;
}
