// hf_noalloc.cu -- the run of the whole path with scratch memory in a
// file-scope device array, for callers that cannot allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc at the point where they
// want to run an analysis chunk: code running inside a CUDA stream capture
// (where an allocation would break or be baked into the graph), plug-ins of
// frameworks that own every device allocation themselves, or real-time loops
// that must not risk an allocation's latency or failure.  They can still pass
// their own input and output buffers; hf_run_device_noalloc then needs no
// context and no allocation of its own: its scratch (compaction buckets, the
// FP64-recheck list, pending-event slots, counters) lives in the array below,
// which every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "hf.h"
#include "hf_kernels.h"

namespace {

using namespace hf;

constexpr uint64_t NA_MAX_EVENTS = HF_NOALLOC_MAX_EVENTS;
constexpr unsigned NA_RC_CAP = 1u << 16;  // recheck entries; more are evaluated inline

// Layout of the scratch array (offsets in bytes, 256-byte aligned).
constexpr size_t NA_SMALL = 0;                                      // counters, 256 B
constexpr size_t NA_BUCKET = 256;                                   // uint2[NA_MAX_EVENTS]
constexpr size_t NA_RC = NA_BUCKET + 8 * NA_MAX_EVENTS;             // RcEntry[NA_RC_CAP]
constexpr size_t NA_PEND_CNT = NA_RC + 16 * (size_t)NA_RC_CAP;      // int[NA_RC_CAP]
constexpr size_t NA_PEND_RNG = NA_PEND_CNT + 4 * (size_t)NA_RC_CAP;   // uint2[NA_RC_CAP]
constexpr size_t NA_PEND_SUM = NA_PEND_RNG + 8 * (size_t)NA_RC_CAP;   // float4[NA_RC_CAP]
constexpr size_t NA_PEND_COMP = NA_PEND_SUM + 16 * (size_t)NA_RC_CAP;
constexpr size_t NA_RC_RECO = NA_PEND_COMP + 16 * (size_t)NA_RC_CAP;  // float4[NA_RC_CAP]
constexpr size_t NA_RC_F = NA_RC_RECO + 16 * (size_t)NA_RC_CAP;       // RcRes[NA_RC_CAP]
constexpr size_t NA_MAXF = NA_RC_F + sizeof(RcRes) * (size_t)NA_RC_CAP; // u8[NA_MAX_EVENTS]
constexpr size_t NA_REC_PRE = NA_MAXF + NA_MAX_EVENTS;                 // u64[NA_MAX_EVENTS/256 + 1]
constexpr size_t NA_CUTFLOW = NA_REC_PRE + 8 * (NA_MAX_EVENTS / 256) + 256;  // u64[MAX_CUTS+1]
constexpr size_t NA_HIST = NA_CUTFLOW + 256;                          // u64[MAX_BINS+2]
constexpr size_t NA_RCTOT = NA_HIST + 8 * (MAX_BINS + 2 + 30);        // u64
constexpr size_t NA_BYTES = NA_RCTOT + 256;
static_assert(NA_BYTES == HF_NOALLOC_SCRATCH_BYTES, "scratch size differs from the one hf.h states");

__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Counters inside the small block (same meaning as in the context's runs).
constexpr size_t C_NHIST = 0, C_CURSOR = 64, C_TILE = 128, C_RC = 192, C_RCVALID = 196, C_PEND = 200, C_ERR = 204;

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_addr[MAX_DEVICES];  // device address of the array, per device
int g_sms[MAX_DEVICES];

// Device address of the scratch array on the current device (set up once per
// device: the name g_noalloc_scratch is only a host-side stand-in).  A cached
// address is checked against the runtime's record of device pointers first:
// after a reset of the device (cudaDeviceReset) the module is loaded again,
// the old address no longer belongs to any allocation, and it is looked up
// anew.  Neither call allocates.
hf_status scratch_for_device(int dev, unsigned char** out, int* sms)
{
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(HF_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev]) {
        cudaPointerAttributes pa;
        const cudaError_t e = cudaPointerGetAttributes(&pa, g_addr[dev]);
        if (e != cudaSuccess || pa.type != cudaMemoryTypeDevice || pa.device != dev) {
            cudaGetLastError();
            g_addr[dev] = nullptr;
        }
    }
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress(scratch)");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaDeviceGetAttribute");
        g_addr[dev] = (unsigned char*)p;
        g_sms[dev] = n;
    }
    *out = g_addr[dev];
    *sms = g_sms[dev];
    return HF_OK;
}

}  // namespace

extern "C" hf_status hf_run_device_noalloc(const hf_analysis_desc* desc, const hf_columns* dev_cols,
                                           uint64_t n_events, uint64_t first_event_id, uint64_t seed,
                                           uint32_t n_variations, const hf_results* dev_out, void* stream)
{
    if (!desc || !dev_cols) return set_error(HF_EINVAL, "NULL argument");
    if (n_events > NA_MAX_EVENTS)
        return set_error(HF_EINVAL, "hf_run_device_noalloc: more than HF_NOALLOC_MAX_EVENTS events; "
                                    "split the chunk or use hf_run_device");
    if (n_variations < 1 || n_variations > HF_MAX_VARIATIONS) return set_error(HF_EINVAL, "n_variations must be 1..4096");
    if (n_events > 0 && (!dev_cols->jet_off || !dev_cols->btag || !dev_cols->lep || !dev_cols->lep_q ||
                         !dev_cols->met || (dev_cols->n_jets_total > 0 && !dev_cols->jets)))
        return set_error(HF_EINVAL, "a column pointer is NULL");
    if (((uintptr_t)dev_cols->jets & 15) || ((uintptr_t)dev_cols->lep & 15) || ((uintptr_t)dev_cols->met & 7))
        return set_error(HF_EINVAL, "jets/lep must be 16-byte and met 8-byte aligned");
    if (dev_out && dev_out->reco && ((uintptr_t)dev_out->reco & 15))
        return set_error(HF_EINVAL, "reco must be 16-byte aligned");
    Plan P;
    if (hf_status s = build_plan(desc, P)) return s;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
    unsigned char* base = nullptr;
    int sms = 0;
    if (hf_status s = scratch_for_device(dev, &base, &sms)) return s;
    cudaStream_t st = (cudaStream_t)stream;

    Scratch S;
    memset(&S, 0, sizeof S);
    unsigned char* sm = base + NA_SMALL;
    S.nhist = (unsigned*)(sm + C_NHIST);
    S.cursor = (unsigned*)(sm + C_CURSOR);
    S.tile_ctr = (unsigned*)(sm + C_TILE);
    S.rc_count = (unsigned*)(sm + C_RC);
    S.rc_valid = (unsigned*)(sm + C_RCVALID);
    S.pend_count = (unsigned*)(sm + C_PEND);
    S.err = (unsigned*)(sm + C_ERR);
    S.bucket = (uint2*)(base + NA_BUCKET);
    S.rc = (RcEntry*)(base + NA_RC);
    S.rc_cap = NA_RC_CAP;
    S.pend_cnt = (unsigned*)(base + NA_PEND_CNT);
    S.pend_rng = (uint2*)(base + NA_PEND_RNG);
    S.rc_reco = (float4*)(base + NA_RC_RECO);
    S.rc_res = (RcRes*)(base + NA_RC_F);
    S.rec_pre = (unsigned long long*)(base + NA_REC_PRE);
    S.pend_sum = (float4*)(base + NA_PEND_SUM);
    S.pend_comp = (float4*)(base + NA_PEND_COMP);
    S.stats = nullptr;  // no scheduler: user order
    S.prof = nullptr;
    S.exec2 = nullptr;
    S.n_exec2 = P.n_exec2;

    Out O;
    memset(&O, 0, sizeof O);
    if (dev_out) {
        O.mask = dev_out->mask;
        O.n_surv = dev_out->n_surv;
        O.reco = (float4*)dev_out->reco;
        O.cutflow = (unsigned long long*)dev_out->cutflow;
        O.hist = (unsigned long long*)dev_out->hist;
        O.rc_total = (unsigned long long*)dev_out->recheck_count;
        if (P.best) O.best_v = dev_out->best_v;
        if (dev_out->records && P.rec_levels) {
            if (P.best) return set_error(HF_EINVAL, "per-cut records are not kept with best-of-variations");
            if (!dev_out->n_records || ((uintptr_t)dev_out->records & 3))
                return set_error(HF_EINVAL, "records need n_records and 4-byte alignment");
            for (int i = 0; i < 4; ++i)
                if (P.rec_var[i] >= VAR_RECO0 && !dev_out->reco)
                    return set_error(HF_EINVAL, "recording a reconstructed quantity needs the reco output");
            O.rec = (Record*)dev_out->records;
            O.rec_cap = dev_out->record_cap;
            O.n_rec = (unsigned long long*)dev_out->n_records;
            O.maxf = (uint8_t*)(base + NA_MAXF);
        }
    }
    if (!O.cutflow) O.cutflow = (unsigned long long*)(base + NA_CUTFLOW);
    if (!O.hist) O.hist = (unsigned long long*)(base + NA_HIST);
    if (!O.rc_total) O.rc_total = (unsigned long long*)(base + NA_RCTOT);

    // the array keeps the previous call's contents: clear what starts at zero
    if ((e = cudaMemsetAsync(base + NA_SMALL, 0, 256, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(O.cutflow, 0, 8 * (P.n_cuts + 1), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(O.hist, 0, 8 * (P.nbins + 2), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(O.rc_total, 0, 8, st)) != cudaSuccess ||
        (O.rec && (e = cudaMemsetAsync(O.n_rec, 0, 8, st)) != cudaSuccess))
        return set_cuda_error(e, "cudaMemsetAsync(scratch)");
    if (n_events == 0) return HF_OK;

    Cols C;
    C.jet_off = dev_cols->jet_off;
    C.jets = (const float4*)dev_cols->jets;
    C.btag = dev_cols->btag;
    C.lep = (const float4*)dev_cols->lep;
    C.lep_q = dev_cols->lep_q;
    C.met = (const float2*)dev_cols->met;
    C.n_jets_total = dev_cols->n_jets_total;
    e = launch_run(P, C, (uint32_t)n_events, n_variations, O, S, seed, first_event_id, false, sms, st);
    if (e != cudaSuccess) return set_cuda_error(e, "launching the run");
    return HF_OK;
}
