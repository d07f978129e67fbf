// hf_plain.cu -- the plain form of the path, the comparison baseline: one
// thread per event runs the whole chain in user order for each of its
// variations, with the event's jets read from global memory into registers;
// no compaction, no shared-memory staging, no bucketing by multiplicity and
// no reordering.  It uses the same FP32 unit evaluation, error bands and FP64
// recheck as the fast path, so its results are identical.
#include "hf_common.cuh"
#include "hf_kernels.h"
#include "hf_semilep.cuh"

namespace hf {

// ------------------------------------------------------------------ plain form
// One thread per event, all cuts in user order, jets read from global memory
// into registers, no compaction, no staging, no reordering.
template <int N, bool F>
__device__ __noinline__ void plain_semi_event(const Plan& P, const Cols& C, const Out& O, const Scratch& S, uint32_t e,
                                 uint32_t V, uint64_t seed, uint64_t first_id, unsigned bits,
                                 unsigned long long* fc, unsigned* hist)
{
    constexpr int NT = ntri(N);
    SemiEvent<N> se;
    float g[NT > 0 ? NT : 1];
    float4 jet[N > 0 ? N : 1];
    const uint32_t j0 = C.jet_off[e];
#pragma unroll
    for (int i = 0; i < N; ++i) jet[i] = C.jets[j0 + i];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i <= j; ++i) g[tri(i, j)] = minkowski_dot2(jet[i], jet[j]);
    if (NT == 0) g[0] = 0.f;
    se.g = g;
    se.jets = C.jets + j0;
    se.lep = C.lep[e];
    se.met = C.met[e];
    se.s1bits = bits;
    se.event_id = first_id + e;
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f), comp = sum;
    unsigned cnt = 0;
    int nflag = 0, maxf = -1;
    uint16_t vs[64];
    for (uint32_t v = 0; v < V; ++v) {
        UnitOut r = semi_unit_f<N, F>(P, P.exec2, P.n_exec2, se, v, seed);
        if (r.f < 0) {
            if (nflag < 64) {
                vs[nflag++] = (uint16_t)v;
                continue;
            }
            float4 reco;  // more than 64 flagged units: evaluate the excess here
            int bin = 0;
            r.f = unit_fp64(P, C, e, first_id + e, seed, v, bits, &reco, &bin);
            r.reco = reco;
            r.bin = bin;
            atomicAdd(O.rc_total, 1ull);
        }
        maxf = max(maxf, r.f);
        atomicAdd(&fc[r.f], 1ull);
        if (r.f == P.n_cuts) {
            ++cnt;
            atomicAdd(&hist[r.bin], 1u);
            acc4(sum, comp, r.reco);
        }
    }
    if (O.maxf) O.maxf[e] = (uint8_t)max(maxf, 0);
    if (nflag == 0) write_event(O, e, cnt, sum, comp);
    else pend_event(P, C, O, S, e, first_id + e, seed, bits, cnt, sum, comp, vs, nflag, fc, hist);
}

template <int N, bool F>
__device__ __forceinline__ void plain_dispatch(int n, const Plan& P, const Cols& C, const Out& O, const Scratch& S,
                                               uint32_t e, uint32_t V, uint64_t seed, uint64_t first_id,
                                               unsigned bits, unsigned long long* fc, unsigned* hist)
{
    if (n == N) {
        plain_semi_event<N, F>(P, C, O, S, e, V, seed, first_id, bits, fc, hist);
    }
    if constexpr (N > 0) plain_dispatch<N - 1, F>(n, P, C, O, S, e, V, seed, first_id, bits, fc, hist);
}

// Semileptonic model (the dilepton plain kernel is in hf_plain_dilep.cu).
__global__ void __launch_bounds__(BLOCK) k_plain(const Plan P, const Cols C, uint32_t N, uint32_t V,
                                                 const Out O, Scratch S, uint64_t seed, uint64_t first_id)
{
    __shared__ unsigned long long s_fc[MAX_CUTS + 1];
    __shared__ unsigned s_hist[MAX_BINS + 2];
    if (threadIdx.x <= MAX_CUTS) s_fc[threadIdx.x] = 0;
    for (int b = threadIdx.x; b < P.nbins + 2; b += blockDim.x) s_hist[b] = 0;
    __syncthreads();
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < N) {
        uint32_t a = C.jet_off[e], b = C.jet_off[e + 1];
        uint32_t n = b - a;
        if (b < a || n > MAX_JETS || (uint64_t)b > C.n_jets_total) {
            atomicOr(S.err, ERR_COLUMNS);
            write_zero_event(O, e);
        } else {
            unsigned bits = stage1_bits(P, C, e, (int)n);
            int f1 = first_fail_stage1(P, bits);
            if (!needs_stage2(P, f1)) {
                atomicAdd(&s_fc[f1], (unsigned long long)V);
                write_stage1_event(P, C, O, e, f1);
            } else {
                if (P.has_full)
                    plain_dispatch<MAX_JETS, true>((int)n, P, C, O, S, e, V, seed, first_id, bits, s_fc, s_hist);
                else
                    plain_dispatch<MAX_JETS, false>((int)n, P, C, O, S, e, V, seed, first_id, bits, s_fc, s_hist);
            }
        }
    }
    __syncthreads();
    flush_cutflow(P, O, s_fc);
    flush_hist(P, O, s_hist);
}

cudaError_t launch_plain(const Plan& P, const Cols& C, uint32_t N, uint32_t V, const Out& O, const Scratch& S,
                         uint64_t seed, uint64_t first_id, cudaStream_t st)
{
    if (P.model == MODEL_DILEP) return launch_plain_dilep(P, C, N, V, O, S, seed, first_id, st);
    k_plain<<<(N + BLOCK - 1) / BLOCK, BLOCK, 0, st>>>(P, C, N, V, O, S, seed, first_id);
    return cudaGetLastError();
}

}  // namespace hf
