// hf_stage2_dilep.cu -- stage 2 of the dilepton model: persistent grid over
// tiles of events bucketed by their number of b-tagged jets (the pairings
// solved per unit grow as n_b (n_b - 1)), largest buckets first.  Per tile:
// (A) the events' jets, leptons and MET are staged in shared memory, (B) each
// thread evaluates units (event x variation) with the FP32/FP64 two-neutrino
// solver carrying error bounds, (C) one thread per event reduces its
// surviving units in variation order or registers its flagged units for the
// FP64 recheck.
//
// k_stage2_dilep: the tiles of one chunk.  k_bstage2_dilep: the tiles of every
// dilepton chunk of a batch (buckets of all chunks, largest n_b first; tile ->
// chunk by binary search in the per-chunk tile prefix).
#include "hf_common.cuh"
#include "hf_dilep.cuh"
#include "hf_kernels.h"
#include "hf_stage2_semi.cuh"  // S2Acc, upper_chunk, load_plan

namespace hf {

namespace {

constexpr int DL_UNITS_PER_TILE = 128;

struct DlSmem {
    float4* jets;    // [ev][12]
    float4* lep;     // [ev][2]
    float2* met;     // [ev]
    uint32_t* evid;  // [ev]
    uint32_t* bits;  // [ev]
    uint32_t* nj;    // [ev] jets
    uint32_t* btag;  // [ev]
    float4* ureco;   // [unit]
    float2* usc;     // [unit] fit score and (bits of) bin, best-of-variations only
    int* uf;         // [unit]
};

__device__ inline DlSmem dl_carve(char* p, int ev, int units, bool best)
{
    DlSmem t;
    t.jets = (float4*)p; p += (size_t)ev * 12 * 16;
    t.lep = (float4*)p; p += (size_t)ev * 32;
    t.ureco = (float4*)p; p += (size_t)units * 16;
    t.usc = (float2*)p; p += best ? (size_t)units * 8 : 0;
    t.met = (float2*)p; p += (size_t)ev * 8;
    t.evid = (uint32_t*)p; p += (size_t)ev * 4;
    t.bits = (uint32_t*)p; p += (size_t)ev * 4;
    t.nj = (uint32_t*)p; p += (size_t)ev * 4;
    t.btag = (uint32_t*)p; p += (size_t)ev * 4;
    t.uf = (int*)p;
    return t;
}

// One tile: ne events (ents) of one chunk with all their variations
// (B: best-of-variations per event, else the means).
template <bool B>
__device__ void dilep_tile(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V, uint64_t seed,
                           uint64_t first_id, const uint2* ents, int ne, const DlSmem& sm, const int* exec,
                           int nexec, S2Acc& acc)
{
    // A: stage the tile's events
    for (int t = threadIdx.x; t < ne; t += blockDim.x) {
        uint2 en = ents[t];
        const uint32_t e = en.x;
        sm.evid[t] = e;
        sm.bits[t] = en.y;
        const uint32_t j0 = C.jet_off[e];
        sm.nj[t] = C.jet_off[e + 1] - j0;
        sm.btag[t] = C.btag[e];
        sm.lep[2 * t] = __ldg(&C.lep[2 * (uint64_t)e]);
        sm.lep[2 * t + 1] = __ldg(&C.lep[2 * (uint64_t)e + 1]);
        sm.met[t] = __ldg(&C.met[e]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ne * MAX_JETS; t += blockDim.x) {
        const int ev = t / MAX_JETS, j = t - ev * MAX_JETS;
        if (j < (int)sm.nj[ev]) sm.jets[ev * MAX_JETS + j] = __ldg(&C.jets[C.jet_off[sm.evid[ev]] + j]);
    }
    __syncthreads();
    // B: units
    const int nu = ne * (int)V;
    for (int u = threadIdx.x; u < nu; u += blockDim.x) {
        const int ev = u / (int)V;
        const uint32_t v = (uint32_t)(u - ev * (int)V);
        UnitOut r = dilep_unit_f(P, exec, nexec, sm.jets + ev * MAX_JETS, (int)sm.nj[ev], sm.btag[ev],
                                 sm.lep[2 * ev], sm.lep[2 * ev + 1], sm.met[ev], sm.bits[ev],
                                 first_id + sm.evid[ev], v, seed);
        sm.uf[u] = r.f;
        sm.ureco[u] = r.reco;
        if constexpr (B) sm.usc[u] = make_float2(r.score, __int_as_float(r.bin));
        warp_tally<B>(P, r, acc.fc, acc.hist, &acc.st);
    }
    __syncthreads();
    // C: per-event reduction
    reduce_tile_events<B>(P, C, O, S, V, seed, first_id, ne, sm.evid, sm.bits, sm.uf, sm.ureco, sm.usc, acc.fc, acc.hist,
                       threadIdx.x, blockDim.x);
    __syncthreads();
}

}  // namespace

size_t dl_smem_bytes(int ev, int units, bool best)
{
    return (size_t)ev * (12 * 16 + 32 + 8 + 16) + (size_t)units * (best ? 28 : 20) + 64;
}

int dl_ev_per_tile(uint32_t V, int upt)
{
    int e = (upt > 0 ? upt : DL_UNITS_PER_TILE) / (int)V;
    return e < 1 ? 1 : (e > 64 ? 64 : e);
}

// Compiled for 4 blocks per SM (128 registers; 168 measured 2 % slower).
template <bool B>
__global__ void __launch_bounds__(BLOCK, 4) k_stage2_dilep(const Plan P, const Cols C, const Out O, Scratch S, uint32_t V,
                                                        uint64_t seed, uint64_t first_id, int ept)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ unsigned s_base[16], s_fill[16], s_tiles[17];
    __shared__ S2Acc acc;
    __shared__ int s_exec[MAX_CUTS];
    __shared__ int s_nexec;
    __shared__ unsigned s_tile;
    if (threadIdx.x == 0) {
        unsigned a = 0;
        for (int b = 0; b < NBUCKET; ++b) {
            s_base[b] = a;
            a += S.nhist[b];
            s_fill[b] = S.cursor[b];
        }
        unsigned t = 0;
        for (int b = NBUCKET - 1; b >= 0; --b) {  // largest n_b first
            s_tiles[b] = t;
            t += (s_fill[b] + ept - 1) / ept;
        }
        s_tiles[16] = t;
        s_nexec = S.exec2 ? S.n_exec2 : P.n_exec2;
        for (int x = 0; x < s_nexec; ++x) s_exec[x] = S.exec2 ? S.exec2[x] : P.exec2[x];
    }
    acc.zero();
    __syncthreads();
    DlSmem sm = dl_carve(smem_raw, ept, ept * (int)V, B);
    bool any = false;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(S.tile_ctr, 1u);
        __syncthreads();
        const unsigned tile = s_tile;
        __syncthreads();
        if (tile >= s_tiles[16]) break;
        any = true;
        int b = NBUCKET - 1;
        while (b > 0 && tile >= s_tiles[b - 1]) --b;
        const unsigned first = (tile - s_tiles[b]) * (unsigned)ept;
        const int ne = (int)min((unsigned)ept, s_fill[b] - first);
        dilep_tile<B>(P, C, O, S, V, seed, first_id, S.bucket + s_base[b] + first, ne, sm, s_exec, s_nexec, acc);
    }
    if (!any) return;
    acc.flush(P, O, S.stats);
    if (S.prof && threadIdx.x == 0 && acc.st.cands) atomicAdd(&S.prof[PROF_PAIRINGS], acc.st.cands);
}

__global__ void __launch_bounds__(BLOCK) k_bstage2_dilep(const BatchDev* __restrict__ Bp)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ S2Acc acc;
    __shared__ __align__(8) Plan s_plan;
    __shared__ int s_exec[MAX_CUTS];
    __shared__ int s_nexec;
    __shared__ unsigned s_seg[NBUCKET + 1];  // tile segments, largest n_b first
    __shared__ unsigned s_tile, s_chunk, s_bucket, s_tg;
    const BatchDev& B = *Bp;
    const unsigned nc = B.n_chunks, ns = B.n_semi;
    if (ns == nc) return;
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int b = NBUCKET - 1; b >= 0; --b) {
            const unsigned* pre = B.tpre + (size_t)b * (nc + 1);
            s_seg[b] = t;
            t += pre[nc] - pre[ns];
        }
        s_seg[NBUCKET] = t;
    }
    acc.zero();
    __syncthreads();
    const unsigned total = s_seg[NBUCKET];
    if (total == 0) return;
    int cur = -1;
    while (true) {
        if (threadIdx.x == 0) {
            const unsigned t = atomicAdd(&B.tctr[15], 1u);
            s_tile = t;
            if (t < total) {
                int b = NBUCKET - 1;
                while (b > 0 && t >= s_seg[b - 1]) --b;
                const unsigned* pre = B.tpre + (size_t)b * (nc + 1);
                const unsigned tg = t - s_seg[b] + pre[ns];  // tile index in the bucket's prefix
                const unsigned c = upper_chunk(pre, ns, nc, tg);
                s_bucket = (unsigned)b;
                s_chunk = c;
                s_tg = tg - pre[c];  // tile within the chunk's bucket
            }
        }
        __syncthreads();
        if (s_tile >= total) break;
        const int c = (int)s_chunk;
        const int b = (int)s_bucket;
        const unsigned tl = s_tg;
        const BChunk& ch = B.ch[c];
        if (c != cur) {
            if (cur >= 0) {
                const BChunk& pc = B.ch[cur];
                acc.flush(s_plan, pc.O, B.stats + (size_t)pc.plan * 3 * MAX_CUTS);
                __syncthreads();
                acc.zero();
            }
            load_plan(&s_plan, &B.plans[ch.plan]);
            if (threadIdx.x == 0) {
                s_nexec = B.plans[ch.plan].n_exec2;
                const int* ex = B.exec[ch.plan];
                for (int x = 0; x < s_nexec; ++x) s_exec[x] = ex[x];
            }
            cur = c;
            __syncthreads();
        }
        const unsigned ept = ch.ept;
        unsigned base = 0;
        for (int k = 0; k < b; ++k) base += ch.cnt[k];
        const unsigned first = tl * ept;
        const int ne = (int)min(ept, ch.cnt[16 + b] - first);
        Scratch S = B.S;
        S.chunk = (uint32_t)c;
        DlSmem sm = dl_carve(smem_raw, (int)ept, (int)(ept * ch.V), false);
        dilep_tile<false>(s_plan, ch.C, ch.O, S, ch.V, ch.seed, ch.first_id, B.bucket + ch.ev0 + base + first, ne, sm,
                   s_exec, s_nexec, acc);
    }
    if (cur >= 0) {
        const BChunk& pc = B.ch[cur];
        acc.flush(s_plan, pc.O, B.stats + (size_t)pc.plan * 3 * MAX_CUTS);
    }
}

cudaError_t launch_bs2_dilep(const BatchDev* B, size_t smem, int sms, cudaStream_t st)
{
    cudaError_t e = ensure_smem_attr((const void*)k_bstage2_dilep);
    if (e != cudaSuccess) return e;
    int bs = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_bstage2_dilep, BLOCK, smem);
    if (bs < 1) bs = 1;
    k_bstage2_dilep<<<sms * bs, BLOCK, smem, st>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_s2_dilep(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V, uint64_t seed,
                            uint64_t first_id, int ept, int sms, cudaStream_t st)
{
    const size_t smem = dl_smem_bytes(ept, ept * (int)V, P.best);
    auto k = P.best ? k_stage2_dilep<true> : k_stage2_dilep<false>;
    cudaError_t e = ensure_smem_attr((const void*)k);
    if (e != cudaSuccess) return e;
    int bs = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k, BLOCK, smem);
    if (bs < 1) bs = 1;
    k<<<sms * bs, BLOCK, smem, st>>>(P, C, O, S, V, seed, first_id, ept);
    return cudaGetLastError();
}

}  // namespace hf
