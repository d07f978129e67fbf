// hf_plain_dilep.cu -- plain form of the dilepton model (the comparison
// baseline): one thread per event runs the whole chain in user order for each
// of its variations, reading the event's jets from global memory; no
// compaction, no shared-memory staging, no bucketing by b-jet count and no
// reordering.  Same FP32/FP64 unit evaluation, bands and recheck as the fast
// path, so its results are identical.
#include "hf_common.cuh"
#include "hf_kernels.h"

namespace hf {

__global__ void __launch_bounds__(BLOCK) k_plain_dilep(const Plan P, const Cols C, uint32_t N, uint32_t V,
                                                       const Out O, Scratch S, uint64_t seed, uint64_t first_id)
{
    __shared__ unsigned long long s_fc[MAX_CUTS + 1];
    __shared__ unsigned s_hist[MAX_BINS + 2];
    __shared__ int s_exec[MAX_CUTS];
    if (threadIdx.x <= MAX_CUTS) s_fc[threadIdx.x] = 0;
    if (threadIdx.x < MAX_CUTS) s_exec[threadIdx.x] = P.exec2[threadIdx.x];
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
                const float4* jet = C.jets + a;
                const float4 l1 = C.lep[2 * (uint64_t)e], l2 = C.lep[2 * (uint64_t)e + 1];
                const float2 met = C.met[e];
                const unsigned btag = C.btag[e];
                float4 sum = make_float4(0.f, 0.f, 0.f, 0.f), comp = sum;
                unsigned cnt = 0;
                int nflag = 0, maxf = -1;
                uint16_t vs[64];
                for (uint32_t v = 0; v < V; ++v) {
                    UnitOut r = dilep_unit_f(P, s_exec, P.n_exec2, jet, (int)n, btag, l1, l2, met, bits, first_id + e, v, seed);
                    if (r.f < 0) {
                        if (nflag < 64) {
                            vs[nflag++] = (uint16_t)v;
                            continue;
                        }
                        float4 reco;
                        int bin = 0;
                        r.f = unit_fp64(P, C, e, first_id + e, seed, v, bits, &reco, &bin);
                        r.reco = reco;
                        r.bin = bin;
                        atomicAdd(O.rc_total, 1ull);
                    }
                    maxf = max(maxf, r.f);
                    atomicAdd(&s_fc[r.f], 1ull);
                    if (r.f == P.n_cuts) {
                        ++cnt;
                        atomicAdd(&s_hist[r.bin], 1u);
                        acc4(sum, comp, r.reco);
                    }
                }
                if (O.maxf) O.maxf[e] = (uint8_t)max(maxf, 0);
                if (nflag == 0) write_event(O, e, cnt, sum, comp);
                else pend_event(P, C, O, S, e, first_id + e, seed, bits, cnt, sum, comp, vs, nflag, s_fc, s_hist);
            }
        }
    }
    __syncthreads();
    flush_cutflow(P, O, s_fc);
    flush_hist(P, O, s_hist);
}


cudaError_t launch_plain_dilep(const Plan& P, const Cols& C, uint32_t N, uint32_t V, const Out& O, const Scratch& S,
                               uint64_t seed, uint64_t first_id, cudaStream_t st)
{
    k_plain_dilep<<<(N + BLOCK - 1) / BLOCK, BLOCK, 0, st>>>(P, C, N, V, O, S, seed, first_id);
    return cudaGetLastError();
}

}  // namespace hf
