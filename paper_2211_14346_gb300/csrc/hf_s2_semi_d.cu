// hf_s2_semi_d.cu -- instantiations of the semileptonic stage-2 kernels (single
// chunk and batched, triplet-only analyses) for jet multiplicities 6, 7.
#include "hf_stage2_semi.cuh"

namespace hf {
template cudaError_t launch_s2_semi<6, false>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<6, false>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<7, false>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<7, false>(const BatchDev*, size_t, int, cudaStream_t);
}  // namespace hf
