// hf_stage2_semi.cuh -- stage-2 kernels of the semileptonic model for one
// jet multiplicity N (instantiated per N in separate translation units so
// that each gets its own register allocation and the build runs in parallel).
//
// A tile is up to `ept` events of bucket N of one chunk with all their
// variations.  Per tile: (A) the lepton and MET of its events are staged in
// shared memory and each event's packed Gram matrix is computed once
// (compensated FP32) from the jets in global memory, (B) every unit is
// evaluated in FP32 (Philox smearing, MET cut, triplet chi2, W p_z) with
// error bands, (C) one thread per event reduces its surviving units in
// variation order and writes the event's outputs, or registers its flagged
// units for the FP64 recheck.
//
// (B) for triplet-only analyses with N >= 9 jets runs in sub-batches of HT_UNITS
// units and three steps: (B1) one thread per unit smears the MET and runs
// the cut state machine up to the point where the triplet chi2 is needed
// (UNIT_PROBE); those units are compacted into a list by warp ballot and a
// prefix over the warp's lanes (one shared-memory atomic per warp); (B2) one
// thread per listed unit smears the jets and evaluates the chi2 with the
// smeared Gram terms in its own shared-memory column and the W pairs pruned
// (hadtop_pruned), so every lane of a warp works on a unit that needs it,
// and (B3) the same thread completes that unit (UNIT_RESUME) right away.  Analyses with
// the full Eq. 1 fit, and N < 9, evaluate each unit whole in its thread.
//
// k_stage2_semi<N>: persistent grid over the tiles of one chunk.
// k_bstage2_semi<N>: persistent grid over the tiles of every semileptonic
// chunk of a batch (a device work queue: one atomic tile counter per
// multiplicity, tile -> chunk by binary search in the per-chunk tile prefix).
#pragma once
#include "hf_common.cuh"
#include "hf_kernels.h"
#include "hf_semilep.cuh"

namespace hf {

// (B) of a tile of a triplet-only analysis: B1 probe, B2 chi2 of the listed
// units, B3 completion, per sub-batch of HT_UNITS units (B: best-of-variations).
template <int N, bool B, class Grp>
__device__ void semi_units_split(const Grp& g, const Plan& P, const Scratch& S, uint32_t V, uint64_t seed,
                                 uint64_t first_id, int ne, TileSmem& sm, const int* exec, int nexec,
                                 unsigned long long* fc, unsigned* hist, CutStats* st)
{
    const int r0 = g.rank(), gs = g.size();
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = (1u << lane) - 1u;
    constexpr int GST = gram_stride(N);
    TopSmem ts = carve_top(sm.top, N);
    const float cap = chi2_cap(P, P.top_thr);
    const uint2 key = key_of(seed);
    const int nu = ne * (int)V;
    for (int u0 = 0; u0 < nu; u0 += HT_UNITS) {
        const int u1 = min(nu, u0 + HT_UNITS);
        if (r0 == 0) *ts.nh = 0;
        if (u0 == 0) fill_pair_codes(ts.pair_code);
        g.sync();
        // B1: probe every unit; list the ones that need the chi2
        for (int u = u0 + r0; u < u1; u += gs) {
            const int ev = u / (int)V;
            const uint32_t v = (uint32_t)(u - ev * (int)V);
            SemiEvent<N> se;
            se.g = sm.G + ev * GST;
            se.jets = nullptr;
            se.lep = sm.lep[ev];
            se.met = sm.met[ev];
            se.s1bits = sm.bits[ev];
            se.event_id = first_id + sm.evid[ev];
            UnitOut r = semi_unit_f<N, false, UNIT_PROBE>(P, exec, nexec, se, v, seed);
            const bool need = r.f == F_NEED_TOP;
            const unsigned am = __activemask();
            const unsigned bal = __ballot_sync(am, need);
            const unsigned leader = (unsigned)__ffs(am) - 1u;
            unsigned base = 0;
            if (lane == leader && bal) base = atomicAdd(ts.nh, (unsigned)__popc(bal));
            base = __shfl_sync(am, base, leader);
            if (need) {
                const unsigned h = base + (unsigned)__popc(bal & lt);
                ts.hidx[h] = (uint32_t)u;
                ts.tin[h].met = r.reco;
            } else {
                sm.uf[u] = r.f;
                sm.ureco[u] = r.reco;
                if constexpr (B) sm.usc[u] = make_float2(r.score, __int_as_float(r.bin));
                warp_tally<B>(P, r, fc, hist, st);
            }
        }
        g.sync();
        const int nh = (int)*ts.nh;
        // B2 + B3: the chi2 of the listed units, one per thread, and at once the
        // completion of the same unit (no block barrier between the two)
        for (int h0 = 0; h0 < nh; h0 += gs) {
            const int h = h0 + r0;
            if (h < nh) {
                const int u = (int)ts.hidx[h];
                const int ev = u / (int)V;
                const uint32_t v = (uint32_t)(u - ev * (int)V);
                float s[N];
#pragma unroll
                for (int i = 0; i < N; ++i) s[i] = 1.0f;
                if (P.smear_jets) jet_scales_f<N>(P, v, first_id + sm.evid[ev], key, s);
                const long long t0 = clock64();
                TopIn t;
                t.met = ts.tin[h].met;
                t.cands = 0;
                hadtop_pruned<N>(P, sm.G + ev * GST, s, cap, ts.qs + r0, ts.as + r0, ts.pair_code, t.b1, t.b2, t.mt,
                                 t.mw, &t.cands);
                t.cyc = (unsigned)(clock64() - t0);
                SemiEvent<N> se;
                se.g = sm.G + ev * GST;
                se.jets = nullptr;
                se.lep = sm.lep[ev];
                se.met = sm.met[ev];
                se.s1bits = sm.bits[ev];
                se.event_id = first_id + sm.evid[ev];
                UnitOut r = semi_unit_f<N, false, UNIT_RESUME>(P, exec, nexec, se, v, seed, &t);
                sm.uf[u] = r.f;
                sm.ureco[u] = r.reco;
                if constexpr (B) sm.usc[u] = make_float2(r.score, __int_as_float(r.bin));
                warp_tally<B>(P, r, fc, hist, st);
            }
        }
        g.sync();
    }
}

template <int N, bool F, bool B, class Grp>
__device__ void semi_tile(const Grp& g, const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                          uint64_t seed, uint64_t first_id, const uint2* ents, int ne, TileSmem& sm,
                          const int* exec, int nexec, unsigned long long* fc, unsigned* hist, CutStats* st)
{
    const int r0 = g.rank(), gs = g.size();
    // A: stage lepton / MET, then the packed Gram matrices
    constexpr int NT = ntri(N);
    constexpr int GST = gram_stride(N);
    if constexpr (semi_split(N, F)) {
        // the jets of the tile's events are first copied into the chi2 step's
        // shared-memory region (free until then), every load independent of the
        // others, so that the Gram terms wait for one round of global loads
        // instead of one per entry
        float4* sj = (float4*)(sm.top + top_qs_offset());
        __shared__ uint32_t s_j0[MAX_EV_PER_TILE];
        for (int t = r0; t < ne; t += gs) {
            uint2 en = ents[t];
            sm.evid[t] = en.x;
            sm.bits[t] = en.y;
            sm.lep[t] = __ldg(&C.lep[en.x]);
            sm.met[t] = __ldg(&C.met[en.x]);
            s_j0[t] = __ldg(&C.jet_off[en.x]);
        }
        g.sync();
        for (int t = r0; t < ne * N; t += gs) {
            const int ev = t / N, k = t - ev * N;
            sj[t] = __ldg(&C.jets[s_j0[ev] + k]);
        }
        g.sync();
        for (int t = r0; t < ne * NT; t += gs) {
            int ev = t / NT, k = t - ev * NT;
            int j = 0;
            while ((j + 1) * (j + 2) / 2 <= k) ++j;
            int i = k - j * (j + 1) / 2;
            sm.G[ev * GST + k] = minkowski_dot2(sj[ev * N + i], sj[ev * N + j]);
        }
        g.sync();
    } else {
    for (int t = r0; t < ne; t += gs) {
        uint2 en = ents[t];
        sm.evid[t] = en.x;
        sm.bits[t] = en.y;
        sm.lep[t] = __ldg(&C.lep[en.x]);
        sm.met[t] = __ldg(&C.met[en.x]);
    }
    g.sync();
    if constexpr (NT > 0) {
        for (int t = r0; t < ne * NT; t += gs) {
            int ev = t / NT, k = t - ev * NT;
            int j = 0;
            while ((j + 1) * (j + 2) / 2 <= k) ++j;
            int i = k - j * (j + 1) / 2;
            const uint32_t j0 = __ldg(&C.jet_off[sm.evid[ev]]);
            sm.G[ev * GST + k] = minkowski_dot2(__ldg(&C.jets[j0 + i]), __ldg(&C.jets[j0 + j]));
        }
    }
    g.sync();
    }
    const int nu = ne * (int)V;
    if constexpr (semi_split(N, F)) {
        semi_units_split<N, B>(g, P, S, V, seed, first_id, ne, sm, exec, nexec, fc, hist, st);
    } else {
    // B: units
    for (int u = r0; u < nu; u += gs) {
        int ev = u / (int)V;
        uint32_t v = (uint32_t)(u - ev * (int)V);
        SemiEvent<N> se;
        se.g = sm.G + ev * GST;
        se.jets = F ? C.jets + __ldg(&C.jet_off[sm.evid[ev]]) : nullptr;
        se.lep = sm.lep[ev];
        se.met = sm.met[ev];
        se.s1bits = sm.bits[ev];
        se.event_id = first_id + sm.evid[ev];
        UnitOut r = semi_unit_f<N, F>(P, exec, nexec, se, v, seed);
        sm.uf[u] = r.f;
        sm.ureco[u] = r.reco;
        if constexpr (B) sm.usc[u] = make_float2(r.score, __int_as_float(r.bin));
        warp_tally<B>(P, r, fc, hist, st);
    }
    }
    g.sync();
    // C: per-event reduction in variation order
    reduce_tile_events<B>(P, C, O, S, V, seed, first_id, ne, sm.evid, sm.bits, sm.uf, sm.ureco, sm.usc, fc, hist, r0,
                          gs);
    g.sync();
}

// Blocks per SM the stage-2 kernels are compiled for (the register budget):
// the shared memory of a split triplet-only tile (the smeared Gram terms of
// the chi2 step) allows at most 2 blocks per SM, so those get the registers
// of that occupancy.  The whole-unit kernels are latency-bound, and more
// warps measured faster than fewer spills: 8 blocks per SM (64 registers) up
// to 5 jets, 7 at 6 jets, 6 at 7-8 jets -- 7 % less stage-2 time than 4
// blocks (128 registers) for all of them.  The full fit keeps 4 (3 from 9 jets).
__host__ __device__ constexpr int s2_min_blocks(int n, bool full)
{
    return full ? (n >= 9 ? 3 : 4) : (semi_split(n, full) ? 2 : n <= 5 ? 8 : n == 6 ? 7 : 6);
}

// Block-level accumulators of the stage-2 kernels (shared memory).
struct S2Acc {
    unsigned long long fc[MAX_CUTS + 1];
    unsigned hist[MAX_BINS + 2];
    CutStats st;
    __device__ void zero()
    {
        if (threadIdx.x <= MAX_CUTS) fc[threadIdx.x] = 0;
        for (int b = threadIdx.x; b < MAX_BINS + 2; b += blockDim.x) hist[b] = 0;
        if (threadIdx.x < MAX_CUTS) {
            st.evaluated[threadIdx.x] = 0;
            st.passed[threadIdx.x] = 0;
            st.cost[threadIdx.x] = 0;
        }
        if (threadIdx.x == 0) st.cands = 0;
    }
    // Adds the block's counts to the chunk's cut flow and histogram and to the
    // scheduler statistics (stats may be null).
    __device__ void flush(const Plan& P, const Out& O, unsigned long long* stats)
    {
        flush_cutflow(P, O, fc);
        flush_hist(P, O, hist);
        if (threadIdx.x < P.n_cuts && stats) {
            int c = threadIdx.x;
            if (st.evaluated[c]) atomicAdd(&stats[c], (unsigned long long)st.evaluated[c]);
            if (st.passed[c]) atomicAdd(&stats[MAX_CUTS + c], (unsigned long long)st.passed[c]);
            if (st.cost[c]) atomicAdd(&stats[2 * MAX_CUTS + c], st.cost[c]);
        }
    }
};

// Single chunk: the block takes tiles of bucket N from its tile counter.  The
// block-wide barriers between the phases of a tile keep the block's warps at
// nearby code addresses of the (long, fully unrolled) unit evaluation, which
// measured faster than independent per-warp tiles.  B: best-of-variations
// (a kernel of its own, so that the per-event means carry none of its code).
template <int N, bool F, bool B>
__global__ void __launch_bounds__(BLOCK, s2_min_blocks(N, F)) k_stage2_semi(const Plan P, const Cols C, const Out O, Scratch S,
                                                       uint32_t V, uint64_t seed, uint64_t first_id,
                                                       int ev_per_tile)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ S2Acc acc;
    __shared__ int s_exec[MAX_CUTS];
    __shared__ int s_nexec;
    __shared__ unsigned s_tile, s_base, s_fill;
    if (threadIdx.x == 0) {
        unsigned a = 0;
        for (int b = 0; b < N; ++b) a += S.nhist[b];
        s_base = a;
        s_fill = S.cursor[N];
        s_nexec = S.exec2 ? S.n_exec2 : P.n_exec2;
        for (int x = 0; x < s_nexec; ++x) s_exec[x] = S.exec2 ? S.exec2[x] : P.exec2[x];
    }
    acc.zero();
    __syncthreads();
    if (s_fill == 0) return;
    const unsigned ntiles = (s_fill + ev_per_tile - 1) / ev_per_tile;
    TileSmem sm = carve(smem_raw, ev_per_tile, ev_per_tile * (int)V, gram_stride(N), B);
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
        semi_tile<N, F, B>(BlockGroup(), P, C, O, S, V, seed, first_id, S.bucket + s_base + first, ne, sm, s_exec,
                           s_nexec, acc.fc, acc.hist, &acc.st);
    }
    if (!any) return;
    acc.flush(P, O, S.stats);
    if (threadIdx.x < P.n_cuts && S.prof && P.kind[threadIdx.x] == CUT_HADTOP_CHI2_MAX &&
        acc.st.evaluated[threadIdx.x])
        atomicAdd(&S.prof[PROF_TOP + N], (unsigned long long)acc.st.evaluated[threadIdx.x]);
    if (S.prof && threadIdx.x == 0 && acc.st.cands) atomicAdd(&S.prof[PROF_CANDS], acc.st.cands);
    if (S.prof && threadIdx.x == 0 && blockIdx.x == 0) {
        atomicAdd(&S.prof[PROF_UNITS], (unsigned long long)s_fill * V);
        atomicAdd(&S.prof[PROF_EVENTS], (unsigned long long)s_fill);
    }
}

// Largest c in [lo, hi) with pre[c] <= t (pre non-decreasing, pre[lo] <= t).
__device__ __forceinline__ unsigned upper_chunk(const unsigned* pre, unsigned lo, unsigned hi, unsigned t)
{
    while (hi - lo > 1) {
        unsigned mid = (lo + hi) / 2;
        if (pre[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Copies a Plan into shared memory (all threads of the block).
__device__ __forceinline__ void load_plan(Plan* dst, const Plan* src)
{
    const int* s = (const int*)src;
    int* d = (int*)dst;
    for (int i = threadIdx.x; i < (int)(sizeof(Plan) / 4); i += blockDim.x) d[i] = s[i];
}

// F = false: the chunks [0, n_semi0) (triplet-only analyses); F = true: the
// chunks [n_semi0, n_semi) (analyses with the full fit), each with its own
// tile counter.
template <int N, bool F>
__global__ void __launch_bounds__(BLOCK, s2_min_blocks(N, F)) k_bstage2_semi(const BatchDev* __restrict__ Bp)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ S2Acc acc;
    __shared__ __align__(8) Plan s_plan;
    __shared__ int s_exec[MAX_CUTS];
    __shared__ int s_nexec;
    __shared__ unsigned s_tile, s_chunk;
    const BatchDev& B = *Bp;
    const unsigned nc = B.n_chunks;
    const unsigned c0 = F ? B.n_semi0 : 0u, c1 = F ? B.n_semi : B.n_semi0;
    if (c0 == c1) return;
    const unsigned* pre = B.tpre + (size_t)N * (nc + 1);
    const unsigned t0 = pre[c0], total = pre[c1] - t0;
    if (total == 0) return;
    acc.zero();
    int cur = -1;
    while (true) {
        if (threadIdx.x == 0) {
            unsigned t = atomicAdd(&B.tctr[N + (F ? 16 : 0)], 1u);
            s_tile = t;
            if (t < total) s_chunk = upper_chunk(pre, c0, c1, t + t0);
        }
        __syncthreads();
        const unsigned t = s_tile;
        const int c = (int)s_chunk;
        if (t >= total) break;
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
        for (int b = 0; b < N; ++b) base += ch.cnt[b];
        const unsigned fill = ch.cnt[16 + N];
        const unsigned first = (t + t0 - pre[c]) * ept;
        const int ne = (int)min(ept, fill - first);
        Scratch S = B.S;
        S.chunk = (uint32_t)c;
        TileSmem sm = carve(smem_raw, (int)ept, (int)(ept * ch.V), gram_stride(N), false);
        semi_tile<N, F, false>(BlockGroup(), s_plan, ch.C, ch.O, S, ch.V, ch.seed, ch.first_id,
                               B.bucket + ch.ev0 + base + first, ne, sm, s_exec, s_nexec, acc.fc, acc.hist, &acc.st);
    }
    if (cur >= 0) {
        const BChunk& pc = B.ch[cur];
        acc.flush(s_plan, pc.O, B.stats + (size_t)pc.plan * 3 * MAX_CUTS);
    }
}

// Launches the kernel of multiplicity N as a persistent grid (one wave).
template <int N, bool F>
cudaError_t launch_s2_semi(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t V,
                           uint64_t seed, uint64_t first_id, int ept, int sms, cudaStream_t st)
{
    const size_t smem = semi_smem_bytes(N, F, ept, ept * (int)V, P.best);
    auto k = P.best ? k_stage2_semi<N, F, true> : k_stage2_semi<N, F, false>;
    cudaError_t e = ensure_smem_attr((const void*)k);
    if (e != cudaSuccess) return e;
    int bs = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k, BLOCK, smem);
    if (bs < 1) bs = 1;
    k<<<sms * bs, BLOCK, smem, st>>>(P, C, O, S, V, seed, first_id, ept);
    return cudaGetLastError();
}

// Batched form: smem = the largest tile of the batch at this multiplicity.
template <int N, bool F>
cudaError_t launch_bs2_semi(const BatchDev* B, size_t smem, int sms, cudaStream_t st)
{
    cudaError_t e = ensure_smem_attr((const void*)k_bstage2_semi<N, F>);
    if (e != cudaSuccess) return e;
    int bs = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_bstage2_semi<N, F>, BLOCK, smem);
    if (bs < 1) bs = 1;
    k_bstage2_semi<N, F><<<sms * bs, BLOCK, smem, st>>>(B);
    return cudaGetLastError();
}

}  // namespace hf
