// Trajectory kernel for the 8-16-16-2 network.  Launch shapes (all compute
// identical values): 0 (default) <16, 8, 8, 3>, eight-warp blocks at three
// per SM (24 warps) -- measured on GB300 8-11 % faster than <16, 8, 4, 4>
// (16 warps per SM) on the parking scene (N = 16384, T = 60), the road at
// the paper's horizon (N = 20480, T = 200) and the course (N = 16384,
// T = 40); 1 four hidden units per lane, 2 eight-warp blocks with no
// occupancy hint, 3 <16, 8, 4, 4>; template arguments <width, lanes per
// sample, warps per block, blocks per SM hint>.
#include "npp_rollout.cuh"

namespace npp {

cudaError_t launch_traj_w16(const RolloutArgs& a, cudaStream_t s, int variant)
{
    // rollout variants run in the default shape
    if (uses_variants(a.c)) return launch_traj<16, 8, 4, 4, true>(a, s);
    switch (variant) {
    case 1: return launch_traj<16, 4, 8>(a, s);
    case 2: return launch_traj<16, 8, 8>(a, s);
    case 3: return launch_traj<16, 8, 4, 4>(a, s);
    default: return launch_traj<16, 8, 8, 3>(a, s);
    }
}

// Trajectories with the windowed binned check (fused_kernel; template
// arguments after the trajectory kernel's: window of states, candidates
// loaded ahead per lane)
cudaError_t launch_fused_w16(const RolloutArgs& a, cudaStream_t s, int variant)
{
    if (uses_variants(a.c)) return launch_fused<16, 8, 4, 4, true, 0, 16, 4>(a, s);
    switch (variant) {
    case 2: return launch_fused<16, 8, 4, 4, false, 0, 8, 4>(a, s);
    case 3: return launch_fused<16, 8, 4, 4, false, 0, 16, 2>(a, s);
    default: return launch_fused<16, 8, 4, 4, false, 0, 16, 4>(a, s);
    }
}

}  // namespace npp
