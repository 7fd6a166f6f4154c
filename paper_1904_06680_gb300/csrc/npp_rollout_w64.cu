// Instantiation of the batched rollout kernel for the 8-64-64-2 network.
#include "npp_rollout.cuh"

namespace npp {

using KW64 = RolloutKernel<64, 8, 4>;

cudaError_t launch_rollout_w64(const RolloutArgs& a, cudaStream_t s, int* smem_needed)
{
    return launch_rollout<64, 8, 4>(a, s, smem_needed);
}

int rollout_max_points_w64(int smem_limit)
{
    return (smem_limit - KW64::fixed_bytes()) / 16;
}

}  // namespace npp
