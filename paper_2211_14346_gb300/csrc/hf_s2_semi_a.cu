// hf_s2_semi_a.cu -- instantiations of the semileptonic stage-2 kernels (single
// chunk and batched, triplet-only analyses) for jet multiplicities 0, 1, 2, 3, 4, 5.
#include "hf_stage2_semi.cuh"

namespace hf {
template cudaError_t launch_s2_semi<0, false>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<0, false>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<1, false>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<1, false>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<2, false>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<2, false>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<3, false>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<3, false>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<4, false>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<4, false>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<5, false>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<5, false>(const BatchDev*, size_t, int, cudaStream_t);
}  // namespace hf
