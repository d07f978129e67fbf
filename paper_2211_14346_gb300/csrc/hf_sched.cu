// hf_sched.cu -- device-side cut scheduler (between runs).
//
// HEP-Frame measures each cut's filter ratio and execution time at run time
// and reorders the cuts so that cheap, rejecting ones run first while
// respecting dependencies (Sect. 5.2).  Here the per-cut statistics of the
// stage-2 cuts (units evaluated, units passed, clock64 cycles) of each run
// feed exponential moving averages of the pass rate and cost; one block then
// scores every dependency-respecting execution order of the stage-2 cuts by
// its expected cost per unit -- including the cost of completing the
// user-order cut flow (cuts that precede the first failure in user order but
// were skipped by the execution order must still be evaluated) -- under an
// independence assumption, and writes the cheapest order for the next run.
#include "hf_dev.cuh"
#include "hf_sched.h"

namespace hf {

__device__ float order_cost(const int* perm, int k, const int* user_idx, const float* p, const float* c)
{
    // outcome bit i: cut perm-position-independent index i passes
    float total = 0.0f;
    for (unsigned out = 0; out < (1u << k); ++out) {
        float prob = 1.0f;
        for (int i = 0; i < k; ++i) prob *= (out >> i & 1u) ? p[i] : 1.0f - p[i];
        if (prob == 0.0f) continue;
        unsigned evald = 0;
        float cost = 0.0f;
        int fail_u = 1 << 30;  // user index of the first failure found
        for (int x = 0; x < k; ++x) {
            int i = perm[x];
            evald |= 1u << i;
            cost += c[i];
            if (!(out >> i & 1u)) {
                fail_u = user_idx[i];
                break;
            }
        }
        // completion: skipped cuts before the earliest known failure, user order
        while (true) {
            int best = -1;
            for (int i = 0; i < k; ++i)
                if (!(evald >> i & 1u) && user_idx[i] < fail_u && (best < 0 || user_idx[i] < user_idx[best]))
                    best = i;
            if (best < 0) break;
            evald |= 1u << best;
            cost += c[best];
            if (!(out >> best & 1u)) fail_u = user_idx[best];
        }
        total += prob * cost;
    }
    return total;
}

__global__ void k_sched_update(SchedDev* sd, const unsigned long long* run_stats, float alpha)
{
    __shared__ float s_cost[1024];
    
    __shared__ float p[MAX_CUTS], c[MAX_CUTS];
    __shared__ int uidx[MAX_CUTS];
    const int k = sd->n_stage2;
    if (threadIdx.x == 0) {
        for (int i = 0; i < k; ++i) {
            int u = sd->stage2_cuts[i];
            unsigned long long ev = run_stats[u], ps = run_stats[MAX_CUTS + u], cs = run_stats[2 * MAX_CUTS + u];
            sd->tot_eval[u] += ev;
            sd->tot_pass[u] += ps;
            sd->tot_cost[u] += cs;
            if (ev) {
                float pr = (float)ps / (float)ev, co = (float)cs / (float)ev;
                if (sd->have[u]) {
                    sd->ema_p[u] = alpha * pr + (1.0f - alpha) * sd->ema_p[u];
                    sd->ema_c[u] = alpha * co + (1.0f - alpha) * sd->ema_c[u];
                } else {
                    sd->ema_p[u] = pr;
                    sd->ema_c[u] = co;
                    sd->have[u] = 1;
                }
            }
            p[i] = sd->have[u] ? sd->ema_p[u] : 0.5f;
            c[i] = sd->have[u] ? sd->ema_c[u] : 1.0f;
            uidx[i] = u;
        }
    }
    __syncthreads();
    if (sd->frozen || k <= 1 || k > 6) return;
    int nperm = 1;
    for (int i = 2; i <= k; ++i) nperm *= i;
    for (int t = threadIdx.x; t < nperm; t += blockDim.x) {
        int perm[MAX_CUTS], avail[MAX_CUTS];
        for (int i = 0; i < k; ++i) avail[i] = i;
        int r = t, na = k;
        for (int x = 0; x < k; ++x) {
            int f = 1;
            for (int i = 2; i <= na - 1; ++i) f *= i;
            int q = r / f;
            r -= q * f;
            perm[x] = avail[q];
            for (int i = q; i < na - 1; ++i) avail[i] = avail[i + 1];
            --na;
        }
        bool ok = true;
        unsigned placed = 0;  // user indices already executed
        for (int x = 0; x < k && ok; ++x) {
            int u = uidx[perm[x]];
            unsigned need = sd->dep_mask[u] & sd->stage2_mask;
            if ((need & ~placed) != 0u) ok = false;
            if (sd->pinned[u]) {  // a pinned cut keeps its user-order rank among stage-2 cuts
                if (perm[x] != x) ok = false;
            }
            placed |= 1u << u;
        }
        s_cost[t] = ok ? order_cost(perm, k, uidx, p, c) : 3.0e38f;

    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 0;
        for (int t = 1; t < nperm; ++t)
            if (s_cost[t] < s_cost[best] * 0.98f) best = t;  // prefer the user order unless clearly cheaper
        int avail[MAX_CUTS];
        for (int i = 0; i < k; ++i) avail[i] = i;
        int r = best, na = k;
        for (int x = 0; x < k; ++x) {
            int f = 1;
            for (int i = 2; i <= na - 1; ++i) f *= i;
            int q = r / f;
            r -= q * f;
            sd->exec2[x] = uidx[avail[q]];
            for (int i = q; i < na - 1; ++i) avail[i] = avail[i + 1];
            --na;
        }
        sd->n_exec2 = k;
    }
}

cudaError_t launch_sched_update(SchedDev* sd, const unsigned long long* run_stats, cudaStream_t st)
{
    k_sched_update<<<1, 256, 0, st>>>(sd, run_stats, 0.3f);
    return cudaGetLastError();
}

}  // namespace hf
