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

// one warp per sample over the stored states (each step's inequality rows
// recomputed from the state), h in order: the candidates of a step are the
// points of at most five cell
// rows, each row's cells contiguous in the sorted array; the lanes stride
// through them (coalesced loads) and a ballot ends the sample at its first
// colliding step
constexpr int BINNED_WARPS = 8;

__global__ void __launch_bounds__(BINNED_WARPS * 32) collide_binned_kernel(const RolloutArgs a)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const BinView& g = a.bins;
    const int T = a.T, N = a.N, M = a.M;
    const int n = blockIdx.x * BINNED_WARPS + warp;
    unsigned long long key = ~0ull;
    if (n < N) {
        int fh = -1;
        // the next step's state is loaded while the current step is checked
        float4 nz = a.traj[n];
        for (int h = 0; h <= T; ++h) {
            // the rectangle lies in the disk of radius reach around the
            // reference point (reach covers the centre offset)
            const float4 z = nz;
            if (h < T) nz = a.traj[(size_t)(h + 1) * N + n];
            float4 ca;
            float2 cb;
            rows_of_state(a.c, z, ca, cb);
            const CandRows cr = cand_rows(g.cell_start + (size_t)h * BIN_CS_STRIDE, g, z.x, z.y, g.reach);
            const float2* pts = g.pts + (size_t)h * M;
            const int total = cr.total;
            bool hit = false;
            for (int base = 0; base < total && !hit; base += 32) {
                const int k = base + lane;
                bool inside = false;
                if (k < total) {
                    const float2 p = pts[cr.index(k)];
                    const float xi = fmaf(ca.x, p.x, fmaf(ca.y, p.y, ca.z));
                    const float et = fmaf(ca.w, p.x, fmaf(cb.x, p.y, cb.y));
                    inside = !(((__float_as_uint(xi) | __float_as_uint(et)) >> 30) & 1u);
                }
                hit = __any_sync(FULL, inside);
            }
            if (hit) { fh = h; break; }
        }
        if (lane == 0) {
            fh = discard_step(a.vfirst, n, fh);
            float J = __int_as_float(0x7f800000);
            if (fh < 0) {
                J = a.jfree[n];
                key = ((unsigned long long)__float_as_uint(J) << 32) | (unsigned)n;
            } else {
                key = (1ull << 63) | ((unsigned long long)(T - fh) << 32) | (unsigned)n;
            }
            if (a.costs) a.costs[n] = J;
            if (a.first_hit) a.first_hit[n] = fh;
        }
    }
    // each warp folds its key into the minimum on its own (no block barrier:
    // samples end at different steps); the read skips atomics that cannot win
    if (lane == 0 && n < N && a.best_key && key < *reinterpret_cast<volatile unsigned long long*>(a.best_key))
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
