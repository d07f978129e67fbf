// hf_kernels.cu -- scan, compaction and FP64 recheck of the cut chain, and
// the launch sequence of one run.
//
// Pipeline of one run (all on one stream, no host synchronisation):
//   k_count      jet-multiplicity histogram of the chunk (bucket capacities)
//   k_stage1     per event: validation, the cuts that do not depend on the
//                smearing variation (exact: FP32 with an FP64 fallback inside
//                the rounding band), cut flow of the events decided here, and
//                compaction of the rest into per-multiplicity buckets
//                (shared-memory counters, one global atomic per bucket per block)
//   k_stage2_*<N> one persistent grid per jet multiplicity N, largest first
//                (hf_stage2_semi.cuh)
//   k_recheck    FP64 re-evaluation of the listed units
//   k_finish     completion of the events with rechecked units
// Cut flow and histogram are integer counts reduced in shared memory and
// added to global u64 counters once per block.
#include "hf_common.cuh"
#include "hf_kernels.h"

#include <mutex>
#include <set>
#include <utility>

namespace hf {

// ------------------------------------------------------------------ k_count
// Bucket of an event: its jet multiplicity (semileptonic: the triplet loop
// is unrolled per n) or its number of b-tagged jets (dilepton: pairings).
__device__ __forceinline__ int bucket_key(const Plan& P, const Cols& C, uint32_t e, uint32_t n)
{
    return P.model == MODEL_DILEP ? popc_n(C.btag[e], (int)n) : (int)n;
}

__global__ void k_count(const Plan P, const Cols C, uint32_t N, Scratch S)
{
    __shared__ unsigned h[16];
    if (threadIdx.x < 16) h[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
        uint32_t a = C.jet_off[e], b = C.jet_off[e + 1];
        uint32_t n = b - a;
        if (b >= a && n <= MAX_JETS) atomicAdd(&h[bucket_key(P, C, e, n)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NBUCKET && h[threadIdx.x]) atomicAdd(&S.nhist[threadIdx.x], h[threadIdx.x]);
}

// ------------------------------------------------------------------ k_stage1
__global__ void __launch_bounds__(256) k_stage1(const Plan P, const Cols C, uint32_t N, uint32_t V,
                                                const Out O, Scratch S)
{
    __shared__ unsigned s_base[16], s_cnt[16], s_off[16];
    __shared__ unsigned long long s_fc[MAX_CUTS + 1];
    if (threadIdx.x < 16) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x <= MAX_CUTS) s_fc[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = 0; b < NBUCKET; ++b) {
            s_base[b] = acc;
            acc += S.nhist[b];
        }
    }
    __syncthreads();
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    int bucket = -1;
    unsigned loc = 0, bits = 0;
    if (e < N) {
        uint32_t a = C.jet_off[e], b = C.jet_off[e + 1];
        uint32_t n = b - a;
        if (b < a || n > MAX_JETS || (uint64_t)b > C.n_jets_total) {
            atomicOr(S.err, ERR_COLUMNS);
            write_zero_event(O, e);
        } else {
            bits = stage1_bits(P, C, e, (int)n);
            int f1 = first_fail_stage1(P, bits);
            if (needs_stage2(P, f1)) {
                bucket = bucket_key(P, C, e, n);
                loc = atomicAdd(&s_cnt[bucket], 1u);
            } else {
                atomicAdd(&s_fc[f1], (unsigned long long)V);
                write_stage1_event(P, C, O, e, f1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < NBUCKET && s_cnt[threadIdx.x])
        s_off[threadIdx.x] = atomicAdd(&S.cursor[threadIdx.x], s_cnt[threadIdx.x]);
    __syncthreads();
    if (bucket >= 0) S.bucket[s_base[bucket] + s_off[bucket] + loc] = make_uint2(e, bits);
    flush_cutflow(P, O, s_fc);
}

// ------------------------------------------------------------------ recheck
// Compiled for 4 blocks per SM (128 registers): the FP64 re-evaluation is
// latency-bound, and at 168 registers (3 blocks) it measured 35 % slower.
__global__ void __launch_bounds__(BLOCK, 4) k_recheck(const Plan P, const Cols C, const Out O, Scratch S,
                                                   uint64_t seed, uint64_t first_id)
{
    __shared__ unsigned long long s_fc[MAX_CUTS + 1];
    __shared__ unsigned s_hist[MAX_BINS + 2];
    __shared__ unsigned s_n;
    if (threadIdx.x <= MAX_CUTS) s_fc[threadIdx.x] = 0;
    for (int b = threadIdx.x; b < P.nbins + 2; b += blockDim.x) s_hist[b] = 0;
    if (threadIdx.x == 0) s_n = *S.rc_valid;
    __syncthreads();
    const unsigned n = s_n;
    unsigned long long mine = 0;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        RcEntry r = S.rc[i];
        float4 reco;
        int bin = 0;
        double score = 0.0;
        const uint32_t v = r.vbits & 0x7fffu;
        int f = P.best ? unit_fp64_scored(P, C, r.event, first_id + r.event, seed, v, r.vbits >> 16, &reco, &bin, &score)
                       : unit_fp64(P, C, r.event, first_id + r.event, seed, v, r.vbits >> 16, &reco, &bin);
        ++mine;
        // best-of: score-only entries are in the cut flow already, the
        // histogram is filled per event at completion
        if (!(r.vbits & RC_SCORE_ONLY)) atomicAdd(&s_fc[f], 1ull);
        if (f == P.n_cuts && !P.best) atomicAdd(&s_hist[bin], 1u);
        S.rc_reco[i] = reco;
        S.rc_res[i] = RcRes{f, bin, score};
    }
    if (mine) atomicAdd(O.rc_total, mine);
    __syncthreads();
    flush_cutflow(P, O, s_fc);
    flush_hist(P, O, s_hist);
}

// ------------------------------------------------------------------ per-cut records
// Records per block of events (blockDim.x events from blockIdx.x).
__global__ void __launch_bounds__(256) k_rec_count(const Plan P, const Out O, uint32_t N, unsigned long long* pre)
{
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long c = e < N ? rec_count(P, O.maxf[e]) : 0u;
    unsigned long long total;
    block_excl_scan(c, &total);
    if (threadIdx.x == 0) pre[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_rec_scan(unsigned long long* pre, unsigned n,
                                                   unsigned long long* total_out)
{
    scan_blocks(pre, n, total_out);
}

__global__ void __launch_bounds__(256) k_rec_write(const Plan P, const Cols C, const Out O, uint32_t N,
                                                   const unsigned long long* pre)
{
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    const int maxf = e < N ? O.maxf[e] : 0;
    write_block_records(P, C, O, e, e < N, maxf, pre[blockIdx.x]);
}

// ------------------------------------------------------------------ k_finish
// Completion of the pending events after the recheck, one warp per slot.
__global__ void __launch_bounds__(BLOCK) k_finish(const Plan P, const Cols C, const Out O, Scratch S)
{
    const unsigned n = *S.pend_count;
    const unsigned w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (unsigned s = w0; s < n; s += nw) {
        unsigned cnt;
        float4 sum, comp;
        int maxf;
        RcEntry first;
        if (P.best) {
            finish_pending_best(O, S, P.n_cuts, s, O.hist, maxf, first);
            if ((threadIdx.x & 31u) == 0 && O.maxf)
                O.maxf[first.event] = (uint8_t)max((int)O.maxf[first.event], maxf);
            continue;
        }
        finish_pending(S, P.n_cuts, s, cnt, sum, comp, maxf, first);
        if ((threadIdx.x & 31u) == 0) {
            write_event(O, first.event, cnt, sum, comp);
            if (O.maxf) O.maxf[first.event] = (uint8_t)max((int)O.maxf[first.event], maxf);
        }
    }
}

// ------------------------------------------------------------------ host launchers
// The larger of the two layouts (with and without the chi2 step), so that a
// batch's kernels of either kind fit.
size_t semi_tile_bytes(int n, int ept, int units) { return semi_smem_bytes(n, false, ept, units, false); }

cudaError_t ensure_smem_attr(const void* fn)
{
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, fn})) return cudaSuccess;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
    done.insert({dev, fn});
    return cudaSuccess;
}

int ev_per_tile_for(uint32_t V, int upt)
{
    int e = (upt > 0 ? upt : UNITS_PER_TILE) / (int)V;
    if (e < 1) e = 1;
    if (e > MAX_EV_PER_TILE) e = MAX_EV_PER_TILE;
    return e;
}

typedef cudaError_t (*S2Launcher)(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t, uint64_t,
                                  uint64_t, int, int, cudaStream_t);

cudaError_t launch_run(const Plan& P, const Cols& C, uint32_t N, uint32_t V, const Out& O, const Scratch& S,
                       uint64_t seed, uint64_t first_id, bool plain, int sms, cudaStream_t st, cudaEvent_t* ev,
                       const SideStreams* side, int upt)
{
    if (N == 0) return cudaSuccess;
    const unsigned nb = (N + 255) / 256;
    cudaError_t e;
    if (ev) cudaEventRecord(ev[0], st);
    if (plain) {
        e = launch_plain(P, C, N, V, O, S, seed, first_id, st);
        if (e != cudaSuccess) return e;
        if (ev) {
            cudaEventRecord(ev[1], st);
            cudaEventRecord(ev[2], st);
        }
    } else {
        k_count<<<min(nb, 4096u), 256, 0, st>>>(P, C, N, S);
        k_stage1<<<nb, 256, 0, st>>>(P, C, N, V, O, S);
        if (ev) cudaEventRecord(ev[1], st);
        const int ept = ev_per_tile_for(V, upt);
        static const S2Launcher semi_t[NBUCKET] = {
            launch_s2_semi<0, false>,  launch_s2_semi<1, false>,  launch_s2_semi<2, false>,
            launch_s2_semi<3, false>,  launch_s2_semi<4, false>,  launch_s2_semi<5, false>,
            launch_s2_semi<6, false>,  launch_s2_semi<7, false>,  launch_s2_semi<8, false>,
            launch_s2_semi<9, false>,  launch_s2_semi<10, false>, launch_s2_semi<11, false>,
            launch_s2_semi<12, false>};
        static const S2Launcher semi_f[NBUCKET] = {
            launch_s2_semi<0, true>,  launch_s2_semi<1, true>,  launch_s2_semi<2, true>,  launch_s2_semi<3, true>,
            launch_s2_semi<4, true>,  launch_s2_semi<5, true>,  launch_s2_semi<6, true>,  launch_s2_semi<7, true>,
            launch_s2_semi<8, true>,  launch_s2_semi<9, true>,  launch_s2_semi<10, true>, launch_s2_semi<11, true>,
            launch_s2_semi<12, true>};
        const S2Launcher* semi = P.has_full ? semi_f : semi_t;
        if (P.model == MODEL_DILEP) {
            e = launch_s2_dilep(P, C, O, S, V, seed, first_id, dl_ev_per_tile(V, upt), sms, st);
            if (e != cudaSuccess) return e;
        } else {
            // Buckets are independent: on side streams their persistent grids
            // overlap, so that the tail of one multiplicity is filled by the next.
            const bool fork = side && side->n > 0;
            if (fork) {
                if ((e = cudaEventRecord(side->fork, st)) != cudaSuccess) return e;
                for (int i = 0; i < side->n; ++i)
                    if ((e = cudaStreamWaitEvent(side->s[i], side->fork, 0)) != cudaSuccess) return e;
            }
            for (int n = NBUCKET - 1, x = 0; n >= 0; --n, ++x) {
                cudaStream_t sn = fork ? side->s[x % side->n] : st;
                e = semi[n](P, C, O, S, V, seed, first_id, ept, sms, sn);
                if (e != cudaSuccess) return e;
            }
            if (fork) {
                for (int i = 0; i < side->n; ++i) {
                    if ((e = cudaEventRecord(side->join[i], side->s[i])) != cudaSuccess) return e;
                    if ((e = cudaStreamWaitEvent(st, side->join[i], 0)) != cudaSuccess) return e;
                }
            }
        }
        if (ev) cudaEventRecord(ev[2], st);
    }
    k_recheck<<<sms * 4, BLOCK, 0, st>>>(P, C, O, S, seed, first_id);
    k_finish<<<sms * 16, BLOCK, 0, st>>>(P, C, O, S);
    if (O.rec) {
        k_rec_count<<<nb, 256, 0, st>>>(P, O, N, S.rec_pre);
        k_rec_scan<<<1, 1024, 0, st>>>(S.rec_pre, nb, O.n_rec);
        k_rec_write<<<nb, 256, 0, st>>>(P, C, O, N, S.rec_pre);
    }
    if (ev) cudaEventRecord(ev[3], st);
    return cudaGetLastError();
}

}  // namespace hf
