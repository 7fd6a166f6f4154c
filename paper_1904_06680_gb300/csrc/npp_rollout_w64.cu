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

cudaError_t launch_fused_w64(const RolloutArgs& a, cudaStream_t s, int variant)
{
    if (uses_variants(a.c)) return launch_fused<64, 32, 1, 10, true>(a, s);
    switch (variant) {
    case 1: return launch_fused<64, 16, 8>(a, s);
    case 2: return launch_fused<64, 32, 8>(a, s);
    case 3: return launch_fused<64, 32, 2, 5>(a, s);
    default: return launch_fused<64, 32, 1, 10>(a, s);
    }
}

cudaError_t launch_reroll_w64(const RolloutArgs& a, const EpilogueArgs& e, cudaStream_t s)
{
    return launch_reroll<64, 32>(a, e, s);
}

}  // namespace npp
