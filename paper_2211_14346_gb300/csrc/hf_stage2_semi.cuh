// hf_stage2_semi.cuh -- stage-2 kernel of the semileptonic model for one
// jet multiplicity N (instantiated per N in separate translation units so
// that each gets its own register allocation and the build runs in parallel).
//
// Persistent grid over the tiles of bucket N: a tile is up to ev_per_tile
// events of the bucket with all their variations.  Per tile: (A) the jets,
// lepton and MET of its events are staged in shared memory and each event's
// Gram matrix is computed once (compensated FP32), (B) every unit is
// evaluated in FP32 registers (Philox smearing, MET cut, triplet chi2, W p_z)
// with error bands, (C) one thread per event reduces its surviving units in
// variation order and writes the event's outputs, or registers its flagged
// units for the FP64 recheck.
#pragma once
#include "hf_common.cuh"
#include "hf_semilep.cuh"

namespace hf {

template <int N>
__device__ void semi_tile(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                          uint64_t seed, uint64_t first_id, const uint2* ents, int ne, TileSmem& sm,
                          const int* exec, int nexec, unsigned long long* fc, unsigned* hist, CutStats* st)
{
    // A: stage jets / lepton / MET, then the Gram matrices
    if constexpr (N > 0) {
        for (int t = threadIdx.x; t < ne * N; t += blockDim.x) {
            int ev = t / N, j = t - ev * N;
            uint32_t e = ents[ev].x;
            sm.jets[ev * 12 + j] = __ldg(&C.jets[C.jet_off[e] + j]);
        }
    }
    for (int t = threadIdx.x; t < ne; t += blockDim.x) {
        uint2 en = ents[t];
        sm.evid[t] = en.x;
        sm.bits[t] = en.y;
        sm.lep[t] = __ldg(&C.lep[en.x]);
        sm.met[t] = __ldg(&C.met[en.x]);
    }
    __syncthreads();
    constexpr int NT = ntri(N);
    constexpr int GST = GramLayout<N>::STRIDE;
    if constexpr (NT > 0) {
        for (int t = threadIdx.x; t < ne * NT; t += blockDim.x) {
            int ev = t / NT, k = t - ev * NT;
            int j = 0;
            while ((j + 1) * (j + 2) / 2 <= k) ++j;
            int i = k - j * (j + 1) / 2;
            const float g = minkowski_dot2(sm.jets[ev * 12 + i], sm.jets[ev * 12 + j]);
            sm.G[ev * GST + i * N + j] = g;
            sm.G[ev * GST + j * N + i] = g;
        }
    }
    __syncthreads();
    // B: units
    const int nu = ne * (int)V;
    for (int u = threadIdx.x; u < nu; u += blockDim.x) {
        int ev = u / (int)V;
        uint32_t v = (uint32_t)(u - ev * (int)V);
        SemiEvent<N> se;
        se.g = sm.G + ev * GST;
        se.lep = sm.lep[ev];
        se.met = sm.met[ev];
        se.s1bits = sm.bits[ev];
        se.event_id = first_id + sm.evid[ev];
        UnitOut r = semi_unit_f<N>(P, exec, nexec, se, v, seed);
        sm.uf[u] = r.f;
        sm.ureco[u] = r.reco;
        warp_tally(P, r, fc, hist, st);
    }
    __syncthreads();
    // C: per-event reduction in variation order
    reduce_tile_events(P, C, O, S, V, seed, first_id, ne, sm.evid, sm.bits, sm.uf, sm.ureco, fc, hist);
    __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(BLOCK, N >= 9 ? 3 : 4) k_stage2_semi(const Plan P, const Cols C, const Out O, Scratch S,
                                                       uint32_t V, uint64_t seed, uint64_t first_id,
                                                       int ev_per_tile)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ unsigned long long s_fc[MAX_CUTS + 1];
    __shared__ unsigned s_hist[MAX_BINS + 2];
    __shared__ CutStats s_st;
    __shared__ int s_exec[MAX_CUTS];
    __shared__ int s_nexec;
    __shared__ unsigned s_tile, s_base, s_fill;
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = 0; b < N; ++b) acc += S.nhist[b];
        s_base = acc;
        s_fill = S.cursor[N];
        s_nexec = S.exec2 ? S.n_exec2 : P.n_exec2;
        for (int x = 0; x < s_nexec; ++x) s_exec[x] = S.exec2 ? S.exec2[x] : P.exec2[x];
    }
    if (threadIdx.x <= MAX_CUTS) s_fc[threadIdx.x] = 0;
    for (int b = threadIdx.x; b < P.nbins + 2; b += blockDim.x) s_hist[b] = 0;
    if (threadIdx.x < MAX_CUTS) {
        s_st.evaluated[threadIdx.x] = 0;
        s_st.passed[threadIdx.x] = 0;
        s_st.cost[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) s_st.cands = 0;
    __syncthreads();
    if (s_fill == 0) return;
    const unsigned ntiles = (s_fill + ev_per_tile - 1) / ev_per_tile;
    TileSmem sm = carve(smem_raw, ev_per_tile, ev_per_tile * (int)V);
    bool any = false;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&S.tile_ctr[N], 1u);
        __syncthreads();
        const unsigned tile = s_tile;
        __syncthreads();
        if (tile >= ntiles) break;
        any = true;
        unsigned first = tile * (unsigned)ev_per_tile;
        int ne = (int)min((unsigned)ev_per_tile, s_fill - first);
        semi_tile<N>(P, C, O, S, V, seed, first_id, S.bucket + s_base + first, ne, sm, s_exec, s_nexec, s_fc,
                     s_hist, &s_st);
    }
    if (!any) return;
    flush_cutflow(P, O, s_fc);
    flush_hist(P, O, s_hist);
    if (threadIdx.x < P.n_cuts && S.stats) {
        int c = threadIdx.x;
        if (s_st.evaluated[c]) atomicAdd(&S.stats[c], (unsigned long long)s_st.evaluated[c]);
        if (s_st.passed[c]) atomicAdd(&S.stats[MAX_CUTS + c], (unsigned long long)s_st.passed[c]);
        if (s_st.cost[c]) atomicAdd(&S.stats[2 * MAX_CUTS + c], s_st.cost[c]);
        if (S.prof && P.kind[c] == CUT_HADTOP_CHI2_MAX && s_st.evaluated[c])
            atomicAdd(&S.prof[PROF_TOP + N], (unsigned long long)s_st.evaluated[c]);
    }
    if (S.prof && threadIdx.x == 0 && s_st.cands) atomicAdd(&S.prof[PROF_CANDS], s_st.cands);
    if (S.prof && threadIdx.x == 0 && blockIdx.x == 0) {
        atomicAdd(&S.prof[PROF_UNITS], (unsigned long long)s_fill * V);
        atomicAdd(&S.prof[PROF_EVENTS], (unsigned long long)s_fill);
    }
}

// Launches the kernel of multiplicity N as a persistent grid (one wave).
template <int N>
cudaError_t launch_s2_semi(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                           uint64_t seed, uint64_t first_id, int ept, int sms, cudaStream_t st)
{
    size_t smem = tile_smem_bytes(ept, ept * (int)V);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_stage2_semi<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr = true;
    }
    int bs = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_stage2_semi<N>, BLOCK, smem);
    if (bs < 1) bs = 1;
    k_stage2_semi<N><<<sms * bs, BLOCK, smem, st>>>(P, C, O, S, V, seed, first_id, ept);
    return cudaGetLastError();
}

}  // namespace hf
