// npp_binned.cu -- collision checks through per-timestep spatial binning
// (the grid build, and the check over stored trajectories; the check fused
// into the trajectory kernel lives in npp_rollout.cuh).
//
// For every horizon step h the obstacle points at time h Ts (EV frame,
// p + tau v with the brute-force kernels' arithmetic) are counting-sorted into
// a uniform grid of BIN_DIM x BIN_DIM cells centred on the vehicle.  A cell is
// wider than half the radius of the vehicle rectangle's circumscribed disk
// (plus a rounding margin), so a state's disk overlaps at most 5 x 5 cells
// (rows of cells are contiguous runs: at most five per query, `cand_rows`); every
// point inside the rectangle lies in the disk, and cell indices of
// points and of the query are clamped to the grid the same (monotone) way,
// so the queried cells hold every point that can be inside.  The per-point
// test is the brute-force one (same coefficients, same fma sequence), hence
// the collision flags are identical to checking all points.
#include <cmath>

#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_rollout.cuh"

using namespace npp;

namespace {

constexpr int BIN_THREADS = 1024;

// one block per horizon step
__global__ void __launch_bounds__(BIN_THREADS) bin_build_kernel(const RolloutArgs a, BinView g, int* __restrict__ cell_start,
                                                                float2* __restrict__ binned)
{
    extern __shared__ int cnt[];             // [BIN_NCELL]
    __shared__ int run_tot[BIN_THREADS];
    const int h = blockIdx.x;
    const StepIn si = step_in(a);
    float s0, c0;
    sincosf(si.phi0, &s0, &c0);
    build_step_bins<BIN_THREADS>(a.obs, a.M, si.x0, si.y0, s0, c0, (float)h * a.c.Ts, g,
                                 cell_start + (size_t)h * BIN_CS_STRIDE, binned + (size_t)h * a.M, cnt, run_tot);
}

// One warp per sample over its stored states (each step's inequality rows
// recomputed from the state).  The warp checks BIN_SB consecutive steps at
// once, an 8-lane group per step: a step's candidates are the points of at
// most five cell rows, each row's cells contiguous in the sorted array; the
// group's lanes stride through each row's run, one candidate per row and
// lane loaded ahead (binned_item_inside_rows; longer rows one pass at a time
// after them).  The chunk's first colliding step, if any, ends the sample.  Steps
// are independent given the stored states, so checking a few past the first
// collision changes nothing; it replaces one chain of two dependent loads
// per step (cell bounds, then candidates) by one per chunk.
constexpr int BINNED_WARPS = 8;
constexpr int BIN_SB = 32 / BIN_ITEM_LANES; // steps per chunk
constexpr int BIN_GS = BIN_ITEM_LANES;      // lanes per step

__global__ void __launch_bounds__(BINNED_WARPS * 32, 5) collide_binned_kernel(const RolloutArgs a)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane / BIN_GS, gl = lane % BIN_GS;
    const BinView& g = a.bins;
    const int T = a.T, N = a.N, M = a.M;
    int n = blockIdx.x * BINNED_WARPS + warp;
    bool valid = n < N;
    if (a.live_in) {
        const int cnt = *a.live_n_in;
        valid = n < cnt;
        n = valid ? a.live_in[n] : 0;
    }
    // the states of this launch: all (0 .. T), or those of one chunk
    // (0 .. chunk_hi for the first, chunk_lo + 1 .. chunk_hi after it)
    const bool chunked = a.chunk_hi > 0;
    const int hs = chunked && a.chunk_lo > 0 ? a.chunk_lo + 1 : 0;
    const int he = chunked ? a.chunk_hi : T;
    unsigned long long key = ~0ull;
    bool fold = false;                       // lane 0: this warp's sample ended here (key to fold)
    unsigned ntest = 0, nstate = 0;          // this lane's candidate tests and states (measurement)
    if (valid) {
        int fh = -1;
        for (int h0 = hs; h0 <= he; h0 += BIN_SB) {
            const int h = h0 + gid;
            const bool ok = h <= he;
            // the rectangle lies in the disk of radius reach around the
            // reference point (reach covers the centre offset)
            const float4 z = ok ? a.traj[(size_t)h * N + n] : make_float4(0.f, 0.f, 0.f, 0.f);
            nstate += (ok && gl == 0) ? 1u : 0u;
            const bool inside = binned_item_inside_rows<1>(a.c, g, z, h, ok, gl, ntest);
            const unsigned bal = __ballot_sync(FULL, inside);
            unsigned steps_hit = 0;
#pragma unroll
            for (int s = 0; s < BIN_SB; ++s)
                if ((bal >> (s * BIN_GS)) & ((1u << BIN_GS) - 1u)) steps_hit |= 1u << s;
            if (steps_hit) {
                fh = h0 + __ffs(steps_hit) - 1;
                break;
            }
        }
        if (lane == 0) {
            fh = discard_step(a.vfirst, n, fh);
            if (fh < 0 && he < T) {
                // collision-free so far: on to the next chunk
                a.live_out[atomicAdd(a.live_n_out, 1)] = n;
            } else {
                float J = __int_as_float(0x7f800000);
                if (fh < 0) {
                    J = a.jfree[n];
                    key = ((unsigned long long)__float_as_uint(J) << 32) | (unsigned)n;
                } else {
                    key = (1ull << 63) | ((unsigned long long)(T - fh) << 32) | (unsigned)n;
                }
                if (a.costs) a.costs[n] = J;
                if (a.first_hit) a.first_hit[n] = fh;
                fold = true;
            }
        }
    }
    if (a.counts) {
        unsigned long long t = ntest, s = nstate;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            t += __shfl_xor_sync(FULL, t, off);
            s += __shfl_xor_sync(FULL, s, off);
        }
        if (lane == 0 && valid) {
            atomicAdd(a.counts, t);
            atomicAdd(a.counts + 1, s);
        }
    }
    // each warp folds its key into the minimum on its own (no block barrier:
    // samples end at different steps); the read skips atomics that cannot win
    if (fold && a.best_key && key < *reinterpret_cast<volatile unsigned long long*>(a.best_key))
        atomicMin(a.best_key, key);
}

}  // namespace

namespace npp {

// bytes of the per-step grids: (T+1) cell-start tables and (T+1) x M points
size_t binned_workspace_bytes(int max_T, int max_M)
{
    return (size_t)(max_T + 1) * BIN_CS_STRIDE * sizeof(int) + (size_t)(max_T + 1) * max_M * sizeof(float2);
}

// Cells wider than half the radius of the query disk (circumradius of the
// rectangle plus |c_off|, plus a margin against rounding of positions of
// O(100) m), a grid of BIN_DIM^2 cells centred on the vehicle.
cudaError_t build_bins(RolloutArgs& a, float half_len, float half_wid, float c_off, void* workspace, cudaStream_t s)
{
    return build_bins_radius(a, std::sqrt((double)half_len * half_len + (double)half_wid * half_wid) +
                                    std::fabs((double)c_off), workspace, s);
}

// grids for a footprint inside the disk of the given radius around the
// reference point
cudaError_t build_bins_radius(RolloutArgs& a, double radius, void* workspace, cudaStream_t s)
{
    BinView g = make_bin_grid_radius(radius);
    int* cell_start = static_cast<int*>(workspace);
    float2* binned = reinterpret_cast<float2*>(cell_start + (size_t)(a.T + 1) * BIN_CS_STRIDE);
    g.cell_start = cell_start;
    g.pts = binned;
    g.M = a.M;
    const int smem = BIN_NCELL * (int)sizeof(int);
    cudaError_t e = ensure_smem(bin_build_kernel, smem);
    if (e != cudaSuccess) return e;
    bin_build_kernel<<<a.T + 1, BIN_THREADS, smem, s>>>(a, g, cell_start, binned);
    e = cudaGetLastError();
    if (e == cudaSuccess) a.bins = g;
    return e;
}

cudaError_t launch_collide_binned(const RolloutArgs& a, cudaStream_t s)
{
    collide_binned_kernel<<<(a.N + BINNED_WARPS - 1) / BINNED_WARPS, BINNED_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace npp
