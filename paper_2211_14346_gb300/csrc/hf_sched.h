// hf_sched.h -- device state of the cut scheduler (internal).
#pragma once
#include <cuda_runtime.h>

#include "hf_dev.cuh"

namespace hf {

// Persistent per-analysis scheduler state, in device memory.
struct SchedDev {
    int exec2[MAX_CUTS];        // execution order of the stage-2 cuts (user indices)
    int n_exec2;
    int n_stage2;
    int stage2_cuts[MAX_CUTS];  // stage-2 cuts in user order
    unsigned stage2_mask;
    unsigned dep_mask[MAX_CUTS];
    int pinned[MAX_CUTS];
    int frozen;                 // 1: order fixed (user-forced or scheduling disabled)
    int have[MAX_CUTS];
    float ema_p[MAX_CUTS], ema_c[MAX_CUTS];
    unsigned long long tot_eval[MAX_CUTS], tot_pass[MAX_CUTS], tot_cost[MAX_CUTS];
};

cudaError_t launch_sched_update(SchedDev* sd, const unsigned long long* run_stats, cudaStream_t st);

}  // namespace hf
