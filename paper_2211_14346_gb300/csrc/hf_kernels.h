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

// Events per tile of the stage-2 kernels for V variations per event.
int ev_per_tile_for(uint32_t V);

// Enqueues one whole run of the path on stream st.  Scratch counters and the
// output accumulators must be zeroed by the caller beforehand.  If ev is not
// null, ev[0..3] are recorded before stage 1, before stage 2, before the
// recheck and at the end.
template <int N>
cudaError_t launch_s2_semi(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                           uint64_t seed, uint64_t first_id, int ept, int sms, cudaStream_t st);

cudaError_t launch_s2_dilep(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V, uint64_t seed,
                            uint64_t first_id, int sms, cudaStream_t st);

cudaError_t launch_plain(const Plan& P, const Cols& C, uint32_t N, uint32_t V, const Out& O, const Scratch& S,
                         uint64_t seed, uint64_t first_id, cudaStream_t st);

cudaError_t launch_run(const Plan& P, const Cols& C, uint32_t N, uint32_t V, const Out& O, const Scratch& S,
                       uint64_t seed, uint64_t first_id, bool plain, int sms, cudaStream_t st,
                       cudaEvent_t* ev = nullptr);

// Kernel launches of one fast-path run (count, stage 1, one per multiplicity, recheck).
constexpr int FAST_LAUNCHES = 2 + NBUCKET + 1;

}  // namespace hf
