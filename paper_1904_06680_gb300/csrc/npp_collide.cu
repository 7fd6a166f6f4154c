// Collision kernels with all obstacle points resident in shared memory.
// Variants compute the same values: 0 block-balanced (16 warps, one block per
// SM, items of up to 128 samples); 1 block-balanced with 8 warps and two
// blocks per SM; 2 warp-owned items of 8 samples pulled from a queue; 3 / 4
// items of 8 samples on 4 / 2 point slices, two / four items per 8-warp
// block sharing one staged copy of the points (two blocks per SM).
#include "npp_rollout.cuh"

namespace npp {

using CollideResident = CollideBlockKernel<16, 128>;

cudaError_t launch_collide_resident(const RolloutArgs& a, cudaStream_t s, int variant)
{
    switch (variant) {
    case 0: return launch_collide_block<16, 128, 1>(a, s);
    case 1: return launch_collide_block<8, 64, 2>(a, s);
    case 2: return launch_collide_warp<8, 2>(a, s);
    case 3: return launch_collide_slice<4, 2, 2>(a, s);
    default: return launch_collide_slice<2, 2, 4>(a, s);
    }
}

int collide_resident_blocks_per_sm(int M, int variant)
{
    switch (variant) {
    case 0: return collide_block_blocks_per_sm<16, 128, 1>(M);
    case 1: return collide_block_blocks_per_sm<8, 64, 2>(M);
    case 2: return collide_warp_blocks_per_sm<8, 2>(M);
    case 3: return collide_slice_blocks_per_sm<4, 2, 2>(M);
    default: return collide_slice_blocks_per_sm<2, 2, 4>(M);
    }
}

cudaError_t launch_collide_global(const RolloutArgs& a, cudaStream_t s)
{
    return launch_collide_slice_global<4, 4>(a, s);
}

int collide_global_blocks_per_sm()
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, collide_slice_kernel<4, 4, true>, 128,
                                                  CollideSliceKernel<4>::fixed_bytes());
    return nb > 0 ? nb : 1;
}

// points whose pair blocks fit beside the largest fixed part (and the
// staging barrier, static shared memory)
int collide_max_points(int smem_limit)
{
    return 64 * ((smem_limit - CollideResident::fixed_bytes() - 16) / 1024);
}

}  // namespace npp
