// hf_s2_semi_f.cu -- instantiations of the semileptonic stage-2 kernels (single
// chunk and batched, with the full Eq. 1 fit) for jet multiplicities 8, 9.
#include "hf_stage2_semi.cuh"

namespace hf {
template cudaError_t launch_s2_semi<8, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<8, true>(const BatchDev*, size_t, int, cudaStream_t);
template cudaError_t launch_s2_semi<9, true>(const Plan&, const Cols&, const Out&, const Scratch&, uint32_t,
                                           uint64_t, uint64_t, int, int, cudaStream_t);
template cudaError_t launch_bs2_semi<9, true>(const BatchDev*, size_t, int, cudaStream_t);
}  // namespace hf
