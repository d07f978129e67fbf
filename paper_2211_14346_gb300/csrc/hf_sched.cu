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
// Up to 6 stage-2 cuts every order is scored (720 at most).  Beyond that the
// candidates are the user order, the greedy order by rank c / (1 - p) (the
// optimal order of independent filters without the completion cost; pinned
// cuts and dependencies respected) and every order one adjacent swap away
// from the greedy one; up to 12 cuts each is scored exactly over the 2^k
// pass / fail outcomes, the block's threads sharing the outcomes, beyond that
// by the sequential expected cost without the completion term.
#include "hf_dev.cuh"
#include "hf_sched.h"

namespace hf {

// Probability-weighted cost of one pass / fail outcome (bit i: cut i passes)
// under execution order perm.
__device__ float outcome_cost(const int* perm, int k, const int* user_idx, const float* p, const float* c,
                              unsigned out)
{
    float prob = 1.0f;
    for (int i = 0; i < k; ++i) prob *= (out >> i & 1u) ? p[i] : 1.0f - p[i];
    if (prob == 0.0f) return 0.0f;
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
    return prob * cost;
}

__device__ float order_cost(const int* perm, int k, const int* user_idx, const float* p, const float* c)
{
    float total = 0.0f;
    for (unsigned out = 0; out < (1u << k); ++out) total += outcome_cost(perm, k, user_idx, p, c, out);
    return total;
}

// Dependencies and pins of an execution order (perm: indices into the
// stage-2 list, which is in user order).
__device__ bool order_valid(const SchedDev* sd, const int* perm, int k, const int* uidx)
{
    unsigned placed = 0;  // user indices already executed
    for (int x = 0; x < k; ++x) {
        const int u = uidx[perm[x]];
        const unsigned need = sd->dep_mask[u] & sd->stage2_mask;
        if ((need & ~placed) != 0u) return false;
        if (sd->pinned[u] && perm[x] != x) return false;  // a pinned cut keeps its rank among stage-2 cuts
        placed |= 1u << u;
    }
    return true;
}

constexpr int SCHED_MAX_CAND = MAX_CUTS + 1;

// k > 6: candidate orders scored exactly, outcomes shared by the block.
__device__ void sched_large(SchedDev* sd, int k, const int* uidx, const float* p, const float* c)
{
    __shared__ int cand[SCHED_MAX_CAND][MAX_CUTS];
    __shared__ int s_nc;
    __shared__ float part[SCHED_MAX_CAND][8];
    if (threadIdx.x == 0) {
        int nc = 0;
        for (int i = 0; i < k; ++i) cand[nc][i] = i;  // user order
        ++nc;
        // greedy by rank: cheapest cost per rejected unit first
        int g[MAX_CUTS];
        unsigned used = 0, placed = 0;
        bool ok = true;
        for (int x = 0; x < k && ok; ++x) {
            int pick = -1;
            if (sd->pinned[uidx[x]]) {
                pick = (used >> x & 1u) ? -1 : x;
            } else {
                float br = 0.0f;
                for (int i = 0; i < k; ++i) {
                    const int u = uidx[i];
                    if ((used >> i & 1u) || sd->pinned[u]) continue;
                    if ((sd->dep_mask[u] & sd->stage2_mask & ~placed) != 0u) continue;
                    const float r = c[i] / fmaxf(1.0f - p[i], 1.0e-6f);
                    if (pick < 0 || r < br) {
                        pick = i;
                        br = r;
                    }
                }
            }
            if (pick < 0) ok = false;
            else {
                g[x] = pick;
                used |= 1u << pick;
                placed |= 1u << uidx[pick];
            }
        }
        if (ok && order_valid(sd, g, k, uidx)) {
            for (int i = 0; i < k; ++i) cand[nc][i] = g[i];
            ++nc;
            for (int x = 0; x + 1 < k && nc < SCHED_MAX_CAND; ++x) {
                int h[MAX_CUTS];
                for (int i = 0; i < k; ++i) h[i] = g[i];
                const int t = h[x];
                h[x] = h[x + 1];
                h[x + 1] = t;
                if (!order_valid(sd, h, k, uidx)) continue;
                for (int i = 0; i < k; ++i) cand[nc][i] = h[i];
                ++nc;
            }
        }
        s_nc = nc;
    }
    __syncthreads();
    const int nc = s_nc;
    const unsigned nout = 1u << k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = 0; q < nc; ++q) {
        float acc = 0.0f;
        if (k <= 12) {
            for (unsigned out = threadIdx.x; out < nout; out += blockDim.x)
                acc += outcome_cost(cand[q], k, uidx, p, c, out);
        } else if (threadIdx.x == 0) {
            // 13..16 cuts: the sequential expected cost sum_x c_x prod_{y<x} p_y
            // (the completion cost left out)
            float reach = 1.0f;
            for (int x = 0; x < k; ++x) {
                acc += reach * c[cand[q][x]];
                reach *= p[cand[q][x]];
            }
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0 && warp < 8) part[q][warp] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float cost0 = 0.0f;
        for (int w = 0; w < nw && w < 8; ++w) cost0 += part[0][w];
        int best = 0;
        float bc = cost0;
        for (int q = 1; q < nc; ++q) {
            float cq = 0.0f;
            for (int w = 0; w < nw && w < 8; ++w) cq += part[q][w];
            if (cq < bc * 0.98f) {  // prefer the user order unless clearly cheaper
                best = q;
                bc = cq;
            }
        }
        for (int x = 0; x < k; ++x) sd->exec2[x] = uidx[cand[best][x]];
        sd->n_exec2 = k;
    }
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
    if (sd->frozen || k <= 1) return;
    if (k > 6) {
        sched_large(sd, k, uidx, p, c);
        return;
    }
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
        s_cost[t] = order_valid(sd, perm, k, uidx) ? order_cost(perm, k, uidx, p, c) : 3.0e38f;

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
