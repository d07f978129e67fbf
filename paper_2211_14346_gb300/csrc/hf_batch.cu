// hf_batch.cu -- batched runs: many chunks of uneven size, of both event
// models and any number of variations, through one fixed sequence of
// persistent kernels (no launch per chunk).
//
//   k_bzero        clears the batch's counters and every chunk's cut flow,
//                  histogram and recheck counter
//   k_bcount       multiplicity (semileptonic) / b-jet count (dilepton)
//                  histogram of every chunk (bucket capacities)
//   k_bstage1      stage-1 cuts and compaction into each chunk's buckets
//   k_btiles       per bucket, the prefix over chunks of their stage-2 tiles
//   k_bstage2_*    persistent grids over the tiles of all chunks
//                  (hf_stage2_semi.cuh, hf_stage2_dilep.cu)
//   k_brecheck     FP64 re-evaluation of the flagged units of all chunks
//   k_bfinish      completion of the events with rechecked units
//
// Every kernel reads the batch description (BatchDev, in device memory) at
// run time and runs a grid that depends only on the GPU, so one captured
// CUDA graph serves every batch laid out in the same arena.
#include "hf_common.cuh"
#include "hf_kernels.h"
#include "hf_sched.h"

namespace hf {

namespace {

// Chunk of stage-1 block blk: largest c with ch[c].blk0 <= blk.
__device__ __forceinline__ unsigned chunk_of_block(const BatchDev& B, unsigned blk)
{
    unsigned lo = 0, hi = B.n_chunks;
    while (hi - lo > 1) {
        unsigned mid = (lo + hi) / 2;
        if (B.ch[mid].blk0 <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int bkey(const Plan& P, const Cols& C, uint32_t e, uint32_t n)
{
    return P.model == MODEL_DILEP ? popc_n(C.btag[e], (int)n) : (int)n;
}

}  // namespace

__global__ void k_bzero(const BatchDev* __restrict__ Bp)
{
    const BatchDev& B = *Bp;
    if (blockIdx.x == 0) {
        if (threadIdx.x < 32) B.tctr[threadIdx.x] = 0;
        if (threadIdx.x < 8) {
            unsigned* w[8] = {B.S.rc_count, B.S.rc_valid, B.S.pend_count, B.S.err, nullptr, nullptr, nullptr,
                              nullptr};
            if (w[threadIdx.x]) *w[threadIdx.x] = 0;
        }
    }
    for (unsigned c = blockIdx.x; c < B.n_chunks; c += gridDim.x) {
        const BChunk& ch = B.ch[c];
        const Plan& P = B.plans[ch.plan];
        if (threadIdx.x < 32) ch.cnt[threadIdx.x] = 0;
        if (threadIdx.x <= (unsigned)P.n_cuts) ch.O.cutflow[threadIdx.x] = 0;
        for (int b = threadIdx.x; b < P.nbins + 2; b += blockDim.x) ch.O.hist[b] = 0;
        if (threadIdx.x == 0) {
            *ch.O.rc_total = 0;
            if (ch.O.rec) *ch.O.n_rec = 0;
        }
    }
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n_plans * 3 * MAX_CUTS;
         i += gridDim.x * blockDim.x)
        B.stats[i] = 0;
}

__global__ void __launch_bounds__(BLOCK1) k_bcount(const BatchDev* __restrict__ Bp)
{
    __shared__ unsigned h[16];
    __shared__ unsigned s_c;
    const BatchDev& B = *Bp;
    for (unsigned blk = blockIdx.x; blk < B.n_blocks; blk += gridDim.x) {
        if (threadIdx.x < 16) h[threadIdx.x] = 0;
        if (threadIdx.x == 0) s_c = chunk_of_block(B, blk);
        __syncthreads();
        const BChunk& ch = B.ch[s_c];
        const Plan& P = B.plans[ch.plan];
        const uint32_t e = (blk - ch.blk0) * BLOCK1 + threadIdx.x;
        if (e < ch.n) {
            const uint32_t a = ch.C.jet_off[e], b = ch.C.jet_off[e + 1];
            const uint32_t n = b - a;
            if (b >= a && n <= MAX_JETS) atomicAdd(&h[bkey(P, ch.C, e, n)], 1u);
        }
        __syncthreads();
        if (threadIdx.x < NBUCKET && h[threadIdx.x]) atomicAdd(&ch.cnt[threadIdx.x], h[threadIdx.x]);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(BLOCK1) k_bstage1(const BatchDev* __restrict__ Bp)
{
    __shared__ unsigned s_base[16], s_cnt[16], s_off[16];
    __shared__ unsigned long long s_fc[MAX_CUTS + 1];
    __shared__ unsigned s_c;
    const BatchDev& B = *Bp;
    for (unsigned blk = blockIdx.x; blk < B.n_blocks; blk += gridDim.x) {
        if (threadIdx.x < 16) s_cnt[threadIdx.x] = 0;
        if (threadIdx.x <= MAX_CUTS) s_fc[threadIdx.x] = 0;
        if (threadIdx.x == 0) s_c = chunk_of_block(B, blk);
        __syncthreads();
        const BChunk& ch = B.ch[s_c];
        const Plan& P = B.plans[ch.plan];
        if (threadIdx.x == 0) {
            unsigned a = 0;
            for (int b = 0; b < NBUCKET; ++b) {
                s_base[b] = a;
                a += ch.cnt[b];
            }
        }
        const uint32_t e = (blk - ch.blk0) * BLOCK1 + threadIdx.x;
        int bucket = -1;
        unsigned loc = 0, bits = 0;
        if (e < ch.n) {
            const uint32_t a = ch.C.jet_off[e], b = ch.C.jet_off[e + 1];
            const uint32_t n = b - a;
            if (b < a || n > MAX_JETS || (uint64_t)b > ch.C.n_jets_total) {
                atomicOr(B.S.err, ERR_COLUMNS);
                if (ch.err) atomicOr(ch.err, ERR_COLUMNS);
                write_zero_event(ch.O, e);
            } else {
                bits = stage1_bits(P, ch.C, e, (int)n);
                const int f1 = first_fail_stage1(P, bits);
                if (needs_stage2(P, f1)) {
                    bucket = bkey(P, ch.C, e, n);
                    loc = atomicAdd(&s_cnt[bucket], 1u);
                } else {
                    atomicAdd(&s_fc[f1], (unsigned long long)ch.V);
                    write_stage1_event(P, ch.C, ch.O, e, f1);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < NBUCKET && s_cnt[threadIdx.x])
            s_off[threadIdx.x] = atomicAdd(&ch.cnt[16 + threadIdx.x], s_cnt[threadIdx.x]);
        __syncthreads();
        if (bucket >= 0) B.bucket[ch.ev0 + s_base[bucket] + s_off[bucket] + loc] = make_uint2(e, bits);
        flush_cutflow(P, ch.O, s_fc);
        __syncthreads();
    }
}

// One block per bucket: tpre[b][c] = tiles of chunks [0, c) in bucket b.
__global__ void __launch_bounds__(1024) k_btiles(const BatchDev* __restrict__ Bp)
{
    __shared__ unsigned s_scan[1024];
    __shared__ unsigned s_carry;
    const BatchDev& B = *Bp;
    const int b = blockIdx.x;
    const unsigned nc = B.n_chunks;
    unsigned* pre = B.tpre + (size_t)b * (nc + 1);
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (unsigned c0 = 0; c0 < nc; c0 += 1024) {
        const unsigned c = c0 + threadIdx.x;
        unsigned t = 0;
        if (c < nc) {
            const BChunk& ch = B.ch[c];
            t = (ch.cnt[16 + b] + ch.ept - 1) / ch.ept;
        }
        s_scan[threadIdx.x] = t;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {  // inclusive Hillis-Steele scan
            unsigned x = threadIdx.x >= (unsigned)d ? s_scan[threadIdx.x - d] : 0u;
            __syncthreads();
            s_scan[threadIdx.x] += x;
            __syncthreads();
        }
        if (c < nc) pre[c] = s_carry + s_scan[threadIdx.x] - t;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry += s_scan[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) pre[nc] = s_carry;
}

__global__ void __launch_bounds__(BLOCK, 4) k_brecheck(const BatchDev* __restrict__ Bp)
{
    const BatchDev& B = *Bp;
    const Scratch& S = B.S;
    const unsigned n = *S.rc_valid;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const RcEntry r = S.rc[i];
        const BChunk& ch = B.ch[r.chunk];
        const Plan& P = B.plans[ch.plan];
        float4 reco;
        int bin = 0;
        const int f = unit_fp64(P, ch.C, r.event, ch.first_id + r.event, ch.seed, r.vbits & 0xffffu, r.vbits >> 16,
                                &reco, &bin);
        for (int k = 0; k <= f; ++k) atomicAdd(&ch.O.cutflow[k], 1ull);
        atomicAdd(ch.O.rc_total, 1ull);
        if (f == P.n_cuts) atomicAdd(&ch.O.hist[bin], 1ull);
        S.rc_reco[i] = reco;
        S.rc_res[i] = RcRes{f, bin, 0.0};
    }
}

// Completion of the pending events of all chunks, one warp per slot.
__global__ void __launch_bounds__(BLOCK) k_bfinish(const BatchDev* __restrict__ Bp)
{
    const BatchDev& B = *Bp;
    const Scratch& S = B.S;
    const unsigned n = *S.pend_count;
    const unsigned w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (unsigned s = w0; s < n; s += nw) {
        // the slot's chunk (read by every lane: the plan sets n_cuts)
        const BChunk& ch = B.ch[S.rc[S.pend_rng[s].x].chunk];
        const Plan& P = B.plans[ch.plan];
        unsigned cnt;
        float4 sum, comp;
        int maxf;
        RcEntry first;
        finish_pending(S, P.n_cuts, s, cnt, sum, comp, maxf, first);
        if ((threadIdx.x & 31u) == 0) {
            write_event(ch.O, first.event, cnt, sum, comp);
            if (ch.O.maxf) ch.O.maxf[first.event] = (uint8_t)max((int)ch.O.maxf[first.event], maxf);
        }
    }
}

// Per-cut records of every recording chunk (stage-1 blocks of BLOCK1 events;
// see k_rec_count / k_rec_write).
__global__ void __launch_bounds__(BLOCK1) k_brec_count(const BatchDev* __restrict__ Bp)
{
    const BatchDev& B = *Bp;
    unsigned long long* pre = B.rec_pre;
    for (unsigned blk = blockIdx.x; blk < B.n_blocks; blk += gridDim.x) {
        const BChunk& ch = B.ch[chunk_of_block(B, blk)];
        const uint32_t e = (blk - ch.blk0) * BLOCK1 + threadIdx.x;
        const unsigned long long c = ch.O.rec && e < ch.n ? rec_count(B.plans[ch.plan], ch.O.maxf[e]) : 0u;
        unsigned long long total;
        block_excl_scan(c, &total);
        if (threadIdx.x == 0) pre[blk] = total;
    }
}

__global__ void __launch_bounds__(1024) k_brec_scan(const BatchDev* __restrict__ Bp)
{
    scan_blocks(Bp->rec_pre, Bp->n_blocks, nullptr);
}

__global__ void __launch_bounds__(BLOCK1) k_brec_write(const BatchDev* __restrict__ Bp)
{
    const BatchDev& B = *Bp;
    const unsigned long long* pre = B.rec_pre;
    for (unsigned blk = blockIdx.x; blk < B.n_blocks; blk += gridDim.x) {
        const BChunk& ch = B.ch[chunk_of_block(B, blk)];
        const Plan& P = B.plans[ch.plan];
        const uint32_t e = (blk - ch.blk0) * BLOCK1 + threadIdx.x;
        if (!ch.O.rec) continue;  // uniform over the block
        const int maxf = e < ch.n ? ch.O.maxf[e] : 0;
        write_block_records(P, ch.C, ch.O, e, e < ch.n, maxf, pre[blk] - pre[ch.blk0]);
        if (blk == ch.blk0 && threadIdx.x == 0)
            *ch.O.n_rec = pre[ch.blk0 + (ch.n + BLOCK1 - 1) / BLOCK1] - pre[ch.blk0];
    }
}

cudaError_t launch_batch(const BatchDev* B, const BatchLaunch& L, cudaStream_t st, const SideStreams* side)
{
    cudaError_t e;
    const int grid1 = L.sms * 8;
    k_bzero<<<L.sms, 256, 0, st>>>(B);
    k_bcount<<<grid1, BLOCK1, 0, st>>>(B);
    k_bstage1<<<grid1, BLOCK1, 0, st>>>(B);
    k_btiles<<<NBUCKET, 1024, 0, st>>>(B);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    static const BS2Launcher semi[NBUCKET] = {
        launch_bs2_semi<0, false>,  launch_bs2_semi<1, false>,  launch_bs2_semi<2, false>,
        launch_bs2_semi<3, false>,  launch_bs2_semi<4, false>,  launch_bs2_semi<5, false>,
        launch_bs2_semi<6, false>,  launch_bs2_semi<7, false>,  launch_bs2_semi<8, false>,
        launch_bs2_semi<9, false>,  launch_bs2_semi<10, false>, launch_bs2_semi<11, false>,
        launch_bs2_semi<12, false>};
    static const BS2Launcher full[NBUCKET] = {
        launch_bs2_semi<0, true>,  launch_bs2_semi<1, true>,  launch_bs2_semi<2, true>,  launch_bs2_semi<3, true>,
        launch_bs2_semi<4, true>,  launch_bs2_semi<5, true>,  launch_bs2_semi<6, true>,  launch_bs2_semi<7, true>,
        launch_bs2_semi<8, true>,  launch_bs2_semi<9, true>,  launch_bs2_semi<10, true>, launch_bs2_semi<11, true>,
        launch_bs2_semi<12, true>};
    const bool fork = side && side->n > 0;
    if (fork) {
        if ((e = cudaEventRecord(side->fork, st)) != cudaSuccess) return e;
        for (int i = 0; i < side->n; ++i)
            if ((e = cudaStreamWaitEvent(side->s[i], side->fork, 0)) != cudaSuccess) return e;
    }
    int x = 0;
    if (L.dilep) {  // the slowest units first
        cudaStream_t sn = fork ? side->s[x++ % side->n] : st;
        if ((e = launch_bs2_dilep(B, L.smem_dilep, L.sms, sn)) != cudaSuccess) return e;
    }
    for (int n = NBUCKET - 1; n >= 0; --n) {
        if (L.full_mask >> n & 1u) {
            cudaStream_t sn = fork ? side->s[x++ % side->n] : st;
            if ((e = full[n](B, L.smem_semi[n], L.sms, sn)) != cudaSuccess) return e;
        }
        if (L.semi_mask >> n & 1u) {
            cudaStream_t sn = fork ? side->s[x++ % side->n] : st;
            if ((e = semi[n](B, L.smem_semi[n], L.sms, sn)) != cudaSuccess) return e;
        }
    }
    if (fork) {
        for (int i = 0; i < side->n; ++i) {
            if ((e = cudaEventRecord(side->join[i], side->s[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, side->join[i], 0)) != cudaSuccess) return e;
        }
    }
    k_brecheck<<<L.sms * 4, BLOCK, 0, st>>>(B);
    k_bfinish<<<L.sms * 16, BLOCK, 0, st>>>(B);
    if (L.records) {
        k_brec_count<<<L.sms * 8, BLOCK1, 0, st>>>(B);
        k_brec_scan<<<1, 1024, 0, st>>>(B);
        k_brec_write<<<L.sms * 8, BLOCK1, 0, st>>>(B);
    }
    return cudaGetLastError();
}

}  // namespace hf
