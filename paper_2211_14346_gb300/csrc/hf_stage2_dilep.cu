// hf_stage2_dilep.cu -- stage 2 of the dilepton model: persistent grid over
// tiles of events bucketed by their number of b-tagged jets (the pairings
// solved per unit grow as n_b (n_b - 1)), largest buckets first.  Per tile:
// (A) the events' jets, leptons and MET are staged in shared memory, (B) each
// thread evaluates units (event x variation) with the FP32 two-neutrino solver
// carrying error bounds, (C) one thread per event reduces its surviving units
// in variation order or registers its flagged units for the FP64 recheck.
#include "hf_common.cuh"
#include "hf_dilep.cuh"
#include "hf_kernels.h"

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
    int* uf;         // [unit]
};

__host__ __device__ inline size_t dl_smem_bytes(int ev, int units)
{
    return (size_t)ev * (12 * 16 + 32 + 8 + 16) + (size_t)units * 20 + 64;
}

__device__ inline DlSmem dl_carve(char* p, int ev, int units)
{
    DlSmem t;
    t.jets = (float4*)p; p += (size_t)ev * 12 * 16;
    t.lep = (float4*)p; p += (size_t)ev * 32;
    t.ureco = (float4*)p; p += (size_t)units * 16;
    t.met = (float2*)p; p += (size_t)ev * 8;
    t.evid = (uint32_t*)p; p += (size_t)ev * 4;
    t.bits = (uint32_t*)p; p += (size_t)ev * 4;
    t.nj = (uint32_t*)p; p += (size_t)ev * 4;
    t.btag = (uint32_t*)p; p += (size_t)ev * 4;
    t.uf = (int*)p;
    return t;
}

int dl_ev_per_tile(uint32_t V)
{
    int e = DL_UNITS_PER_TILE / (int)V;
    return e < 1 ? 1 : (e > 64 ? 64 : e);
}

}  // namespace

__global__ void __launch_bounds__(BLOCK) k_stage2_dilep(const Plan P, const Cols C, const Out O, Scratch S, uint32_t V,
                                                        uint64_t seed, uint64_t first_id, int ept)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ unsigned s_base[16], s_fill[16], s_tiles[17];
    __shared__ unsigned long long s_fc[MAX_CUTS + 1];
    __shared__ unsigned s_hist[MAX_BINS + 2];
    __shared__ CutStats s_st;
    __shared__ int s_exec[MAX_CUTS];
    __shared__ int s_nexec;
    __shared__ unsigned s_tile;
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = 0; b < NBUCKET; ++b) {
            s_base[b] = acc;
            acc += S.nhist[b];
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
        s_st.cands = 0;
    }
    if (threadIdx.x <= MAX_CUTS) s_fc[threadIdx.x] = 0;
    for (int b = threadIdx.x; b < P.nbins + 2; b += blockDim.x) s_hist[b] = 0;
    if (threadIdx.x < MAX_CUTS) {
        s_st.evaluated[threadIdx.x] = 0;
        s_st.passed[threadIdx.x] = 0;
        s_st.cost[threadIdx.x] = 0;
    }
    __syncthreads();
    DlSmem sm = dl_carve(smem_raw, ept, ept * (int)V);
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
        const uint2* ents = S.bucket + s_base[b] + first;
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
            UnitOut r = dilep_unit_f(P, s_exec, s_nexec, sm.jets + ev * MAX_JETS, (int)sm.nj[ev], sm.btag[ev],
                                     sm.lep[2 * ev], sm.lep[2 * ev + 1], sm.met[ev], sm.bits[ev],
                                     first_id + sm.evid[ev], v, seed);
            sm.uf[u] = r.f;
            sm.ureco[u] = r.reco;
            warp_tally(P, r, s_fc, s_hist, &s_st);
        }
        __syncthreads();
        // C: per-event reduction
        reduce_tile_events(P, C, O, S, V, seed, first_id, ne, sm.evid, sm.bits, sm.uf, sm.ureco, s_fc, s_hist);
        __syncthreads();
    }
    if (!any) return;
    flush_cutflow(P, O, s_fc);
    flush_hist(P, O, s_hist);
    if (threadIdx.x < P.n_cuts && S.stats) {
        const int c = threadIdx.x;
        if (s_st.evaluated[c]) atomicAdd(&S.stats[c], (unsigned long long)s_st.evaluated[c]);
        if (s_st.passed[c]) atomicAdd(&S.stats[MAX_CUTS + c], (unsigned long long)s_st.passed[c]);
        if (s_st.cost[c]) atomicAdd(&S.stats[2 * MAX_CUTS + c], s_st.cost[c]);
    }
    if (S.prof && threadIdx.x == 0 && s_st.cands) atomicAdd(&S.prof[PROF_PAIRINGS], s_st.cands);
}

cudaError_t launch_s2_dilep(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V, uint64_t seed,
                            uint64_t first_id, int sms, cudaStream_t st)
{
    const int ept = dl_ev_per_tile(V);
    const size_t smem = dl_smem_bytes(ept, ept * (int)V);
    int bs = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_stage2_dilep, BLOCK, smem);
    if (bs < 1) bs = 1;
    k_stage2_dilep<<<sms * bs, BLOCK, smem, st>>>(P, C, O, S, V, seed, first_id, ept);
    return cudaGetLastError();
}

}  // namespace hf
