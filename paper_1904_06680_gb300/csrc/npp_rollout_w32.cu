// Trajectory kernel for the 8-32-32-2 network.  Launch shapes (all compute
// identical values): 0 (default, fastest measured on GB300) <32, 16, 4, 4>,
// 1 four hidden units per lane, 2 eight-warp blocks, 3 <32, 16, 8, 3>, 4 the
// last 5 of each lane's 8 W2 input quads in shared memory (5 KB per warp;
// parameters generated by rolled loops through those slots) so that 20
// warps fit per SM (measured 0.161 against 0.164 ms on the course: this
// width is not bound by occupancy, so it is not the default);
// template arguments <width, lanes per sample, warps per block, blocks per SM hint>.
#include "npp_rollout.cuh"

namespace npp {

cudaError_t launch_traj_w32(const RolloutArgs& a, cudaStream_t s, int variant)
{
    // rollout variants run in the default shape
    if (uses_variants(a.c)) return launch_traj<32, 16, 4, 4, true>(a, s);
    switch (variant) {
    case 1: return launch_traj<32, 8, 8>(a, s);
    case 2: return launch_traj<32, 16, 8>(a, s);
    case 3: return launch_traj<32, 16, 8, 3>(a, s);
    case 4: return launch_traj<32, 16, 4, 5, false, 5>(a, s);
    default: return launch_traj<32, 16, 4, 4>(a, s);
    }
}

// Trajectories with the windowed binned check (fused_kernel; template
// arguments after the trajectory kernel's: window of states, candidates
// loaded ahead per lane).  Not the library's choice at this width: on the
// course (N = 16384, T = 40, M = 2000) the default shape, 5 of 8 W2 quads in
// shared memory and windows of 8, took 0.311 ms per plan step against 0.258
// in two kernels (1: 0.348, 3: 0.330).
cudaError_t launch_fused_w32(const RolloutArgs& a, cudaStream_t s, int variant)
{
    if (uses_variants(a.c)) return launch_fused<32, 16, 4, 5, true, 5, 8, 4>(a, s);
    switch (variant) {
    case 1: return launch_fused<32, 16, 4, 4, false, 0, 16, 4>(a, s);
    case 2: return launch_fused<32, 16, 4, 4, false, 0, 8, 4>(a, s);
    case 3: return launch_fused<32, 16, 4, 3, false, 0, 16, 4>(a, s);
    case 4: return launch_fused<32, 16, 4, 5, false, 5, 16, 4>(a, s);
    default: return launch_fused<32, 16, 4, 5, false, 5, 8, 4>(a, s);
    }
}

}  // namespace npp
