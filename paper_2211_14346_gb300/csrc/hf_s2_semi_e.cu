// hf_s2_semi_e.cu -- instantiations of the semileptonic stage-2 kernels (single
// chunk and batched, with the full Eq. 1 fit) for jet multiplicities 0, 1, 2, 3, 4, 5, 6, 7.
#include "hf_stage2_semi.cuh"

namespace hf {
template cudaError_t launch_s2_semi<0, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<0, true>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<1, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<1, true>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<2, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<2, true>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<3, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<3, true>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<4, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<4, true>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<5, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<5, true>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<6, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<6, true>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<7, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<7, true>(const BatchDev*, size_t, int, cudaStream_t);
}  // namespace hf
