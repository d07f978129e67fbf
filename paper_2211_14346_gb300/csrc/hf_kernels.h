// hf_kernels.h -- host-side entry points of the device code (internal).
#pragma once
#include <cuda_runtime.h>

#include "hf_dev.cuh"

#include "hf.h"

namespace hf {

// Validates an analysis descriptor and fills the kernel plan (no allocation).
hf_status build_plan(const hf_analysis_desc* d, Plan& P);
// Records the calling thread's error message (fixed storage) and returns s.
hf_status set_error(hf_status s, const char* msg);
hf_status set_cuda_error(cudaError_t e, const char* what);

// Raises the dynamic shared-memory limit of kernel fn to the device's opt-in
// maximum, once per (current device, kernel); thread-safe.  The attribute
// belongs to the device, so every device that launches fn needs its own call.
cudaError_t ensure_smem_attr(const void* fn);

// Events per tile of the semileptonic stage-2 kernels for V variations per
// event and `upt` units per tile (0 = the default, UNITS_PER_TILE).
int ev_per_tile_for(uint32_t V, int upt = 0);

// Enqueues one whole run of the path on stream st.  Scratch counters and the
// output accumulators must be zeroed by the caller beforehand.  If ev is not
// null, ev[0..3] are recorded before stage 1, before stage 2, before the
// recheck and at the end.
template <int N, bool F>
cudaError_t launch_s2_semi(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                           uint64_t seed, uint64_t first_id, int ept, int sms, cudaStream_t st);

cudaError_t launch_s2_dilep(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V, uint64_t seed,
                            uint64_t first_id, int ept, int sms, cudaStream_t st);

cudaError_t launch_plain(const Plan& P, const Cols& C, uint32_t N, uint32_t V, const Out& O, const Scratch& S,
                         uint64_t seed, uint64_t first_id, cudaStream_t st);
cudaError_t launch_plain_dilep(const Plan& P, const Cols& C, uint32_t N, uint32_t V, const Out& O, const Scratch& S,
                               uint64_t seed, uint64_t first_id, cudaStream_t st);

// Side streams on which the per-multiplicity stage-2 kernels of one run
// overlap (fork after stage 1, join before the recheck).  Owned by the caller.
constexpr int MAX_SIDE = 4;
struct SideStreams {
    int n;                     // 0 = everything on the run's stream
    cudaStream_t s[MAX_SIDE];
    cudaEvent_t fork;          // recorded on the run's stream after stage 1
    cudaEvent_t join[MAX_SIDE];
};


cudaError_t launch_run(const Plan& P, const Cols& C, uint32_t N, uint32_t V, const Out& O, const Scratch& S,
                       uint64_t seed, uint64_t first_id, bool plain, int sms, cudaStream_t st,
                       cudaEvent_t* ev = nullptr, const SideStreams* side = nullptr, int upt = 0);

// Batched runs (hf_batch.cu): the host-side shape of one batch's launches.
struct BatchLaunch {
    int sms;
    unsigned semi_mask;            // bit n: launch the multiplicity-n kernel (triplet-only analyses)
    unsigned full_mask;            // the same for analyses with the full Eq. 1 fit
    size_t smem_semi[NBUCKET];     // dynamic shared memory of the multiplicity-n kernels
    bool dilep;                    // the batch has dilepton chunks
    size_t smem_dilep;
    bool records;                  // some chunk records per-cut variables
};
typedef cudaError_t (*BS2Launcher)(const BatchDev*, size_t, int, cudaStream_t);
template <int N, bool F>
cudaError_t launch_bs2_semi(const BatchDev* B, size_t smem, int sms, cudaStream_t st);
cudaError_t launch_bs2_dilep(const BatchDev* B, size_t smem, int sms, cudaStream_t st);
// Enqueues the whole batch (B in device memory) on st; stage-2 kernels overlap
// on the side streams when given.
cudaError_t launch_batch(const BatchDev* B, const BatchLaunch& L, cudaStream_t st, const SideStreams* side);
// Shared memory of one stage-2 tile (semileptonic multiplicity n / dilepton).
size_t semi_tile_bytes(int n, int ept, int units);
size_t dl_smem_bytes(int ev, int units, bool best);
// Events per tile of the dilepton stage-2 kernel (upt: units per tile, 0 = default).
int dl_ev_per_tile(uint32_t V, int upt = 0);

// HL-LHC multi-region selection (hf_hl.cu): one persistent launch.  O.counts,
// O.hist and O.err must be zeroed beforehand.
cudaError_t launch_hl(const HLPlan& H, const HLCols& C, uint32_t N, uint32_t V, uint64_t seed, uint64_t first_id,
                      const HLOut& O, int sms, cudaStream_t st);

// Kernel launches of one fast-path run (count, stage 1, one per multiplicity, recheck).
constexpr int FAST_LAUNCHES = 2 + NBUCKET + 1;

}  // namespace hf
