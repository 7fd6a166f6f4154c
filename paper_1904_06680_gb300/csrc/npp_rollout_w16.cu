// Instantiation of the batched rollout kernel for the 8-16-16-2 network.
#include "npp_rollout.cuh"

namespace npp {

using KW16 = RolloutKernel<16, 8, 8>;

cudaError_t launch_rollout_w16(const RolloutArgs& a, cudaStream_t s, int* smem_needed)
{
    return launch_rollout<16, 8, 8>(a, s, smem_needed);
}

int rollout_max_points_w16(int smem_limit)
{
    return (smem_limit - KW16::fixed_bytes()) / 16;
}

}  // namespace npp
