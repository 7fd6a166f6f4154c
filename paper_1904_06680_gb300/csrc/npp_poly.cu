// npp_poly.cu -- the collision check of a general footprint (Sect. II-D:
// the EV as an arbitrarily refined polytope, convex or non-convex, checked
// by the linear inequalities A(phi)(p - [x, y]) < b(phi)): the union of
// convex pieces given as half-planes in the vehicle's frame, over the
// per-step grids of npp_binned.cu or over every point.
#include <cmath>

#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_rollout.cuh"

using namespace npp;

namespace {

constexpr int POLY_WARPS = 8;

// Whether point p (EV frame at the step's time) is inside the general
// footprint at pose (x, y) with heading cosine and sine (cp, sp): p moved
// into the vehicle's frame, q = R(-phi) (p - [x, y]), is inside a convex
// piece when n . q < b holds strictly for all of its faces (Eq. of the
// polytope check, Sect. II-D); the footprint is the union of its pieces.
__device__ __forceinline__ bool poly_inside(const float4* faces, int n_faces, float r2, float2 p, float x,
                                            float y, float cp, float sp)
{
    const float dx = p.x - x, dy = p.y - y;
    const float qx = fmaf(cp, dx, __fmul_rn(sp, dy));
    const float qy = fmaf(-sp, dx, __fmul_rn(cp, dy));
    // outside the footprint's bounding disk (r2 is its squared radius,
    // enlarged beyond any rounding of q): no face test needed
    if (fmaf(qx, qx, __fmul_rn(qy, qy)) >= r2) return false;
    bool any = false, in = true;
    for (int f = 0; f < n_faces; ++f) {
        const float4 F = faces[f];
        in = in & (fmaf(F.x, qx, __fmul_rn(F.y, qy)) < F.z);
        if (F.w != 0.0f) {
            any = any | in;
            in = true;
        }
    }
    return any;
}

// Polygon footprint check, one warp per sample over the stored states, h in
// order: the candidates are the points of the (at most five) cell rows the
// footprint's bounding disk overlaps (binned), or every point of the step
// (brute force, the same per-point test); the lanes stride through them and
// a ballot ends the sample at its first colliding step.  Faces are staged in
// shared memory (uniform reads).
__global__ void __launch_bounds__(POLY_WARPS * 32) collide_poly_kernel(const RolloutArgs a)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ float4 faces[FP_MAX_FACES];
    const int nf = a.poly.n_faces;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) faces[i] = a.poly.faces[i];
    __syncthreads();
    const BinView& g = a.bins;
    const int T = a.T, N = a.N, M = a.M;
    const bool brute = a.poly.brute != 0;
    const int n = blockIdx.x * POLY_WARPS + warp;
    unsigned long long key = ~0ull;
    if (n < N) {
        int fh = -1;
        float4 nz = a.traj[n];
        for (int h = 0; h <= T; ++h) {
            const float4 z = nz;
            if (h < T) nz = a.traj[(size_t)(h + 1) * N + n];
            float sp, cp;
            sincos_r(z.z, sp, cp);
            const float2* pts = g.pts + (size_t)h * M;
            // brute force: every point, as one run
            CandRows cr = {};
            if (brute) {
                cr.total = M;
#pragma unroll
                for (int k = 0; k < BIN_MAX_ROWS; ++k) cr.e[k] = M;
            } else {
                cr = cand_rows(g.cell_start + (size_t)h * BIN_CS_STRIDE, g, z.x, z.y, g.reach);
            }
            const int total = cr.total;
            bool hit = false;
            for (int base = 0; base < total && !hit; base += 32) {
                const int k = base + lane;
                bool inside = false;
                if (k < total)
                    inside = poly_inside(faces, nf, a.poly.r2, pts[cr.index(k)], z.x, z.y, cp, sp);
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

cudaError_t launch_collide_poly(const RolloutArgs& a, cudaStream_t s)
{
    collide_poly_kernel<<<(a.N + POLY_WARPS - 1) / POLY_WARPS, POLY_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace npp
