// Trajectory kernel for the 8-64-64-2 network.  Launch shapes (all compute
// identical values): 0 (default, fastest measured on GB300: 3.29 against
// 4.02 ms at N = 65536, T = 100) the last 8 of each lane's 16 W2 input quads
// in shared memory (8 KB per warp), so that 127 registers without spills
// and 16 one-warp blocks fit per SM, parameters generated by rolled loops; 1 four hidden units per lane, 2
// eight-warp blocks, 3 <64, 32, 2, 5>, 4 every weight in registers
// <64, 32, 1, 10> (168 registers with spills, 12 warps per SM);
// template arguments <width, lanes per sample, warps per block, blocks per SM hint>.
#include "npp_rollout.cuh"

namespace npp {

cudaError_t launch_traj_w64(const RolloutArgs& a, cudaStream_t s, int variant)
{
    // rollout variants run in the default shape
    if (uses_variants(a.c)) return launch_traj<64, 32, 1, 16, true, 8>(a, s);
    switch (variant) {
    case 1: return launch_traj<64, 16, 8>(a, s);
    case 2: return launch_traj<64, 32, 8>(a, s);
    case 3: return launch_traj<64, 32, 2, 5>(a, s);
    case 4: return launch_traj<64, 32, 1, 10>(a, s);
    default: return launch_traj<64, 32, 1, 16, false, 8>(a, s);
    }
}

// Trajectories with the windowed binned check (fused_kernel; template
// arguments after the trajectory kernel's: window of states, candidates
// loaded ahead per lane).  Measured on GB300 at N = 65536, T = 100,
// M = 8192 (ms per plan step): 0 (default) 12 W2 quads of 16 in shared
// memory, windows of 8 states: 2.68; 1 10 quads, windows of 16: 2.76;
// 2 12 quads, windows of 16: 2.73; 3 and 4 with 8 candidates ahead: 2.94 -
// 2.98 (no register left for them without spills).
cudaError_t launch_fused_w64(const RolloutArgs& a, cudaStream_t s, int variant)
{
    if (uses_variants(a.c)) return launch_fused<64, 32, 1, 16, true, 12, 8, 4>(a, s);
    switch (variant) {
    case 1: return launch_fused<64, 32, 1, 16, false, 10, 16, 4>(a, s);
    case 2: return launch_fused<64, 32, 1, 16, false, 12, 16, 4>(a, s);
    case 3: return launch_fused<64, 32, 1, 16, false, 12, 16, 8>(a, s);
    case 4: return launch_fused<64, 32, 1, 16, false, 8, 8, 4>(a, s);
    default: return launch_fused<64, 32, 1, 16, false, 12, 8, 4>(a, s);
    }
}

}  // namespace npp
