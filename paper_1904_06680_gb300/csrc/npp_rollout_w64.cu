// Trajectory kernel for the 8-64-64-2 network: variant 0 holds 2 hidden
// units per lane (32 lanes per sample), variant 1 holds 4 (16 lanes); both
// compute identical values.
#include "npp_rollout.cuh"

namespace npp {

cudaError_t launch_traj_w64(const RolloutArgs& a, cudaStream_t s, int variant)
{
    return variant ? launch_traj<64, 16, 8>(a, s) : launch_traj<64, 32, 8>(a, s);
}

}  // namespace npp
