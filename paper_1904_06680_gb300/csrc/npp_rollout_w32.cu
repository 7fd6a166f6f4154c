// Instantiation of the batched rollout kernel for the 8-32-32-2 network.
#include "npp_rollout.cuh"

namespace npp {

using KW32 = RolloutKernel<32, 8, 8>;

cudaError_t launch_rollout_w32(const RolloutArgs& a, cudaStream_t s, int* smem_needed)
{
    return launch_rollout<32, 8, 8>(a, s, smem_needed);
}

int rollout_max_points_w32(int smem_limit)
{
    return (smem_limit - KW32::fixed_bytes()) / 16;
}

}  // namespace npp
