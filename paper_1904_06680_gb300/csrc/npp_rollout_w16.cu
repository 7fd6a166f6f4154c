// Trajectory kernel for the 8-16-16-2 network: variant 0 holds 2 hidden
// units per lane (8 lanes per sample), variant 1 holds 4 (4 lanes); both
// compute identical values.
#include "npp_rollout.cuh"

namespace npp {

cudaError_t launch_traj_w16(const RolloutArgs& a, cudaStream_t s, int variant)
{
    return variant ? launch_traj<16, 4, 8>(a, s) : launch_traj<16, 8, 8>(a, s);
}

}  // namespace npp
