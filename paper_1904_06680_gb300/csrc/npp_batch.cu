// npp_batch.cu -- many independent plan steps (scenes of different N, T, M
// and network width) in one batch of persistent launches:
//   prologue      every scene's obstacle points into its EV frame, as pairs;
//   trajectories  one persistent launch per network width, blocks pulling
//                 (scene, sample block) items, costliest scenes first;
//   collisions    one persistent launch over all scenes, blocks of S warps
//                 pulling (scene, 8-sample) items; a scene's points are
//                 staged in shared memory while the block works on it (read
//                 from global memory when they do not fit);
//   epilogue      one block per scene: decode the winner, re-roll it for
//                 its controls and trajectory, regenerate its parameters.
// Per-sample arithmetic is the single-scene plan step's, so every scene's
// result equals npp_plan_step on that scene alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_internal.h"
#include "npp_rollout.cuh"

using namespace npp;

namespace {

struct SceneDev {
    float x0, y0, phi0, v0, ap0, ap1, gx, gy, gphi, gv;
    int N, T, M, width;
    long long obs_off;       // first input point
    long long pair_off;      // first transformed pair
    long long coef_off;      // first coefficient row
    long long samp_off;      // first sample (costs, first_hit, jfree)
    long long params_off, ctrl_off, traj_off;
    long long tile_off;      // first point tile (32 pairs)
    long long bin_off;       // first int of the scene's per-step cell tables
    long long bpts_off;      // first float2 of the scene's per-step sorted points
    uint32_t k0, k1, t_index, pad;
};

struct BatchArgs {
    DevCfg c;
    const SceneDev* scenes;
    int S;
    const float4* obs;               // input points (world frame)
    float4* pXY;                     // transformed pairs, sorted by cell (static points first)
    float4* pV;
    float4* tileP;                   // per tile of 32 pairs: (min x, max x, min y, max y) of its points
    float4* tileV;                   // (min vx, max vx, min vy, max vy)
    float reach;                     // radius around a rectangle's centre that holds it, plus a margin
    int windowed64;                  // width-64 scenes checked inside their trajectory kernel
    // binned collision check (per scene and horizon step)
    BinView grid;                    // geometry (cell_start, pts, M unused here)
    int* bin_cs;                     // cell tables, scene s at bin_off
    float2* bin_pts;                 // sorted points, scene s at bpts_off
    const long long* bstep_prefix;   // prefix over scenes of T + 1 (grid-build blocks)
    float4* coefA;
    float2* coefB;
    float* jfree;
    int* vfirst;                     // first speed-violating step per sample, or null (limits off)
    unsigned long long* keys;        // [S]
    unsigned* counters;              // [4] work queues: widths 16, 32, 64, collisions
    // item lists
    const int* order;                // scenes by decreasing cost
    const long long* titem_prefix[3];  // per width: prefix of trajectory items over order_w
    const int* torder[3];            // per width: scenes of that width by decreasing cost
    int n_torder[3];
    const long long* citem_prefix;   // prefix of 8-sample items over `order`
    int resident_pairs;              // pairs that fit in shared memory
    // outputs
    npp_best* best;
    float* params;
    float* controls;
    float* trajectory;
    float* costs;
    int* first_hit;
};

__device__ __forceinline__ int find_slot(const long long* prefix, int n, long long item)
{
    // largest s with prefix[s] <= item (prefix[0] = 0, prefix[n] = total)
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ StepIn scene_step_in(const SceneDev& s)
{
    StepIn si;
    si.x0 = s.x0; si.y0 = s.y0; si.phi0 = s.phi0; si.v0 = s.v0; si.ap0 = s.ap0; si.ap1 = s.ap1;
    si.gx = s.gx; si.gy = s.gy; si.gphi = s.gphi; si.gv = s.gv;
    si.t_index = s.t_index;
    si.warm_ok = false;
    return si;
}

// World -> EV frame, as pairs, ordered for tile culling: a counting sort by
// a coarse cell of the EV-frame position (4 m cells, 64 x 64 around the
// vehicle, clamped), static points before moving ones (the order of the
// points does not change any result: a collision is "some point inside").
// The odd tail is padded with a far point.  Then per tile of 32 pairs the
// bounds of its real points' positions and velocities.
constexpr int SORT_THREADS = 1024;
constexpr int SORT_DIM = 64;
constexpr int SORT_KEYS = 2 * SORT_DIM * SORT_DIM;   // static cells, then moving cells

__device__ __forceinline__ int sort_key(float px, float py, float vx, float vy)
{
    const int cx = (int)fminf(fmaxf(floorf((px + 128.0f) * 0.25f), 0.0f), (float)(SORT_DIM - 1));
    const int cy = (int)fminf(fmaxf(floorf((py + 128.0f) * 0.25f), 0.0f), (float)(SORT_DIM - 1));
    const bool moving = vx != 0.0f || vy != 0.0f;
    return (moving ? SORT_DIM * SORT_DIM : 0) + cy * SORT_DIM + cx;
}

__global__ void __launch_bounds__(SORT_THREADS) batch_prologue_kernel(const BatchArgs b)
{
    extern __shared__ int cnt[];                       // [SORT_KEYS]
    __shared__ int run_tot[SORT_THREADS];
    const SceneDev& s = b.scenes[blockIdx.x];
    const int M = s.M;
    if (M == 0) return;
    const int npairs = (M + 1) / 2;
    float sn, cs;
    sincosf(s.phi0, &sn, &cs);
    for (int i = threadIdx.x; i < SORT_KEYS; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        float px, py, vx, vy;
        ev_point(b.obs[s.obs_off + j], s.x0, s.y0, sn, cs, px, py, vx, vy);
        atomicAdd(&cnt[sort_key(px, py, vx, vy)], 1);
    }
    __syncthreads();
    constexpr int RUN = SORT_KEYS / SORT_THREADS;
    const int base = threadIdx.x * RUN;
    int acc = 0;
    for (int k = 0; k < RUN; ++k) { const int v = cnt[base + k]; cnt[base + k] = acc; acc += v; }
    run_tot[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int PER = SORT_THREADS / 32;
        int local = 0;
        for (int k = 0; k < PER; ++k) local += run_tot[threadIdx.x * PER + k];
        int incl = local;
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, off);
            if ((int)threadIdx.x >= off) incl += v;
        }
        int run = incl - local;
        for (int k = 0; k < PER; ++k) {
            const int v = run_tot[threadIdx.x * PER + k];
            run_tot[threadIdx.x * PER + k] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int k = 0; k < RUN; ++k) cnt[base + k] += run_tot[threadIdx.x];
    __syncthreads();
    float* xy = reinterpret_cast<float*>(b.pXY + s.pair_off);
    float* vv = reinterpret_cast<float*>(b.pV + s.pair_off);
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        float px, py, vx, vy;
        ev_point(b.obs[s.obs_off + j], s.x0, s.y0, sn, cs, px, py, vx, vy);
        const int pos = atomicAdd(&cnt[sort_key(px, py, vx, vy)], 1);
        const int q = pos >> 1, o = pos & 1;
        xy[4 * q + o] = px;
        xy[4 * q + 2 + o] = py;
        vv[4 * q + o] = vx;
        vv[4 * q + 2 + o] = vy;
    }
    if (threadIdx.x == 0 && (M & 1)) {
        const int q = M >> 1;
        xy[4 * q + 1] = 1e15f;
        xy[4 * q + 3] = 1e15f;
        vv[4 * q + 1] = 0.0f;
        vv[4 * q + 3] = 0.0f;
    }
    __syncthreads();
    // tile bounds over the real points (the pad point is never inside)
    const int ntiles = (npairs + 31) / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = warp; t < ntiles; t += SORT_THREADS / 32) {
        float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
        float mnvx = INFINITY, mxvx = -INFINITY, mnvy = INFINITY, mxvy = -INFINITY;
        const int q = t * 32 + lane;
        for (int o = 0; o < 2; ++o) {
            const int j = 2 * q + o;
            if (q < npairs && j < M) {
                const float px = xy[4 * q + o], py = xy[4 * q + 2 + o];
                const float vx = vv[4 * q + o], vy = vv[4 * q + 2 + o];
                mnx = fminf(mnx, px); mxx = fmaxf(mxx, px); mny = fminf(mny, py); mxy = fmaxf(mxy, py);
                mnvx = fminf(mnvx, vx); mxvx = fmaxf(mxvx, vx); mnvy = fminf(mnvy, vy); mxvy = fmaxf(mxvy, vy);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            mnx = fminf(mnx, __shfl_xor_sync(FULL, mnx, off));
            mxx = fmaxf(mxx, __shfl_xor_sync(FULL, mxx, off));
            mny = fminf(mny, __shfl_xor_sync(FULL, mny, off));
            mxy = fmaxf(mxy, __shfl_xor_sync(FULL, mxy, off));
            mnvx = fminf(mnvx, __shfl_xor_sync(FULL, mnvx, off));
            mxvx = fmaxf(mxvx, __shfl_xor_sync(FULL, mxvx, off));
            mnvy = fminf(mnvy, __shfl_xor_sync(FULL, mnvy, off));
            mxvy = fmaxf(mxvy, __shfl_xor_sync(FULL, mxvy, off));
        }
        if (lane == 0) {
            b.tileP[s.tile_off + t] = make_float4(mnx, mxx, mny, mxy);
            b.tileV[s.tile_off + t] = make_float4(mnvx, mxvx, mnvy, mxvy);
        }
    }
}

// The pair loop of one warp's tiles (t0, t0 + tstep, ...) for CC live
// samples staged in the warp's slots, skipping tiles whose points, at time
// tau, cannot reach the box around the live samples (box: xmin, xmax, ymin,
// ymax).  fma rounding is monotone, so every point's extrapolated position
// lies in the tile's extrapolated bounds; the per-point test is the
// brute-force one.  Returns the hit bits in slot order.
template <int CC>
__device__ __forceinline__ unsigned check_slots_tiles(const float4* __restrict__ XY, const float4* __restrict__ V,
                                                      int npairs, float tau, const float4* __restrict__ sA,
                                                      const float2* __restrict__ sB, int L, int lane,
                                                      const float4* __restrict__ tP, const float4* __restrict__ tV,
                                                      int ntiles, int t0, int tstep, float4 box)
{
    unsigned long long A[CC], B[CC], NC[CC], D[CC], E[CC], NF[CC];
#pragma unroll
    for (int k = 0; k < CC; ++k) {
        const int slot = k < L ? k : 0;
        const float4 qa = sA[slot];
        const float2 qb = sB[slot];
        A[k] = pk(qa.x, qa.x); B[k] = pk(qa.y, qa.y); NC[k] = pk(qa.z, qa.z);
        D[k] = pk(qa.w, qa.w); E[k] = pk(qb.x, qb.x); NF[k] = pk(qb.y, qb.y);
    }
    unsigned long long acc[CC];
#pragma unroll
    for (int k = 0; k < CC; ++k) acc[k] = 0ull;
    const unsigned long long TT = pk(tau, tau);
    for (int t = t0; t < ntiles; t += tstep) {
        const float4 P = tP[t], Q = tV[t];
        if (fmaf(tau, Q.x, P.x) > box.y || fmaf(tau, Q.y, P.y) < box.x ||
            fmaf(tau, Q.z, P.z) > box.w || fmaf(tau, Q.w, P.w) < box.z)
            continue;
        const int q = t * 32 + lane;
        if (q < npairs) {
            const float4 xy = XY[q];
            const float4 vv = V[q];
            const unsigned long long PX = fma2(TT, pk(vv.x, vv.y), pk(xy.x, xy.y));
            const unsigned long long PY = fma2(TT, pk(vv.z, vv.w), pk(xy.z, xy.w));
#pragma unroll
            for (int k = 0; k < CC; ++k) {
                const unsigned long long xi = fma2(A[k], PX, fma2(B[k], PY, NC[k]));
                const unsigned long long et = fma2(D[k], PX, fma2(E[k], PY, NF[k]));
                acc[k] |= ~(xi | et);
            }
        }
    }
    unsigned bits = 0;
#pragma unroll
    for (int k = 0; k < CC; ++k) {
        const bool inside = ((((unsigned)acc[k]) | (unsigned)(acc[k] >> 32)) >> 30) & 1u;
        if (k < L && __any_sync(FULL, inside)) bits |= 1u << k;
    }
    return bits;
}

// one culled step of an 8-sample item for one warp (see warp_step)
__device__ __forceinline__ unsigned warp_step_tiles(const float4* XY, const float4* V, int npairs, float tau,
                                                    float4 ca, float2 cb, unsigned live, float4* sA, float2* sB,
                                                    int lane, const float4* tP, const float4* tV, int ntiles,
                                                    int t0, int tstep, float4 box)
{
    const bool owner = lane < 8 && ((live >> lane) & 1u);
    const int rank = __popc(live & ((1u << lane) - 1u));
    if (owner) { sA[rank] = ca; sB[rank] = cb; }
    __syncwarp();
    const int L = __popc(live);
    unsigned bits;
    if (L > 4)      bits = check_slots_tiles<8>(XY, V, npairs, tau, sA, sB, L, lane, tP, tV, ntiles, t0, tstep, box);
    else if (L > 2) bits = check_slots_tiles<4>(XY, V, npairs, tau, sA, sB, L, lane, tP, tV, ntiles, t0, tstep, box);
    else if (L > 1) bits = check_slots_tiles<2>(XY, V, npairs, tau, sA, sB, L, lane, tP, tV, ntiles, t0, tstep, box);
    else            bits = check_slots_tiles<1>(XY, V, npairs, tau, sA, sB, L, lane, tP, tV, ntiles, t0, tstep, box);
    __syncwarp();
    return __ballot_sync(FULL, owner && ((bits >> rank) & 1u));
}

// Box (xmin, xmax, ymin, ymax) around the rectangles of the live samples of
// an item (owner lanes 0..7), from their scaled inequality rows: the centre
// is R^T (along, across) with cos, sin = A / sl, B / sl, along = -C' / sl,
// across = -F' / sw; plus `reach` (the rectangle's circumradius and a margin
// far above the rounding of this reconstruction).  Uniform over the warp.
__device__ __forceinline__ float4 live_box(const DevCfg& c, float4 ca, float2 cb, bool owner, float reach)
{
    float xmn = INFINITY, xmx = -INFINITY, ymn = INFINITY, ymx = -INFINITY;
    if (owner) {
        const float isl = 1.0f / (2.0f * c.ihl), isw = 1.0f / (2.0f * c.ihw);
        const float cp = ca.x * isl, sp = ca.y * isl;
        const float along = -ca.z * isl, across = -cb.y * isw;
        const float xc = cp * along - sp * across, yc = sp * along + cp * across;
        xmn = xc - reach; xmx = xc + reach; ymn = yc - reach; ymx = yc + reach;
    }
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
        xmn = fminf(xmn, __shfl_xor_sync(FULL, xmn, off));
        xmx = fmaxf(xmx, __shfl_xor_sync(FULL, xmx, off));
        ymn = fminf(ymn, __shfl_xor_sync(FULL, ymn, off));
        ymx = fmaxf(ymx, __shfl_xor_sync(FULL, ymx, off));
    }
    return make_float4(__shfl_sync(FULL, xmn, 0), __shfl_sync(FULL, xmx, 0), __shfl_sync(FULL, ymn, 0),
                       __shfl_sync(FULL, ymx, 0));
}

// KSQ > 0: the last KSQ layer-2 input quads of each lane in shared memory
// (as the single-scene width-64 kernel: 128 registers and MINB blocks per
// SM instead of every weight in registers at 250)
// WIN: the scene's binned check done window by window inside the kernel
// (traj_sample_windowed, windows of BATCH_CW states, the scene's grids built
// before the launch): each sample's cost, first collision and the scene's
// key are written here, nothing per step is stored
constexpr int BATCH_CW = 8;
template <int W, int G, int NW, bool VAR = false, int KSQ = 0, int MINB = 1, bool WIN = false>
__global__ void __launch_bounds__(NW * 32, MINB) batch_traj_kernel(const BatchArgs b, int wi)
{
    constexpr int B = TrajKernel<W, G, NW>::B;
    __shared__ __align__(16) float hx_all[B * W];
    __shared__ long long qslot;
    // [LaneNet::SLOTS][NW * 32] floats when W == 32 (KSQ = 0); the shared W2
    // quads [group][U][KSQ][G] of 16 bytes when KSQ > 0
    extern __shared__ __align__(16) float stage_all[];
    const int tid = threadIdx.x;
    const int bi = tid / G, gl = tid % G;
    const int n_sc = b.n_torder[wi];
    const long long total = n_sc > 0 ? __ldg(b.titem_prefix[wi] + n_sc) : 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) qslot = (long long)atomicAdd(b.counters + wi, 1u);
        __syncthreads();
        const long long item = qslot;
        if (item >= total) break;
        const int r = find_slot(b.titem_prefix[wi], n_sc, item);
        const SceneDev& s = b.scenes[b.torder[wi][r]];
        const int n = (int)(item - __ldg(b.titem_prefix[wi] + r)) * B + bi;
        TrajJob job;
        job.si = scene_step_in(s);
        job.key.k0 = s.k0; job.key.k1 = s.k1; job.key.t_index = s.t_index; job.key.stream_id = 0u;
        job.theta = nullptr;
        job.warm = nullptr;
        job.prop = Proposal{ nullptr, nullptr, 0, 1u };
        job.bins = nullptr;
        job.stage = stage_all + tid;
        job.w2s = nullptr;
        if constexpr (KSQ > 0)
            job.w2s = reinterpret_cast<ulonglong2*>(stage_all) + (size_t)bi * (Shape<W, G>::U * KSQ * G) + gl;
        job.N = s.N;
        job.T = s.T;
        job.traj = nullptr;
        job.ctrl = nullptr;
        job.rec_stride = 0;
        job.rec_shift = 0;
        job.coefA = b.coefA;
        job.coefB = b.coefB;
        job.coef_base = s.coef_off;
        job.jfree = b.jfree + s.samp_off;
        job.vfirst = b.vfirst ? b.vfirst + s.samp_off : nullptr;
        constexpr int STAGE_TH = (W == 32 && KSQ == 0) ? NW * 32 : 0;     // as traj_kernel
        if constexpr (WIN) {
            const int si = b.torder[wi][r];
            BinView bv = b.grid;
            bv.cell_start = b.bin_cs + s.bin_off;
            bv.pts = b.bin_pts + s.bpts_off;
            bv.M = s.M;
            job.bins = &bv;
            job.coefA = nullptr;
            job.coefB = nullptr;
            job.jfree = nullptr;
            job.vfirst = nullptr;
            float4* wnd = reinterpret_cast<float4*>(reinterpret_cast<char*>(stage_all) +
                                                    NW * 32 * Shape<W, G>::U * KSQ * 16) +
                          (size_t)(tid / 32) * (32 / G) * BATCH_CW;
            unsigned steps = 0, ntest = 0, nstate = 0;
            const bool valid = n < s.N;
            const FusedOut o = traj_sample_windowed<W, G, STAGE_TH, VAR, KSQ, BATCH_CW, 4>(
                b.c, job, n, valid, gl, hx_all + bi * W, wnd, steps, ntest, nstate);
            if (valid && gl == 0) {
                unsigned long long key;
                if (o.first_hit < 0)
                    key = ((unsigned long long)__float_as_uint(o.cost) << 32) | (unsigned)n;
                else
                    key = (1ull << 63) | ((unsigned long long)(s.T - o.first_hit) << 32) | (unsigned)n;
                if (b.costs) b.costs[s.samp_off + n] = o.cost;
                if (b.first_hit) b.first_hit[s.samp_off + n] = o.first_hit;
                if (key < *reinterpret_cast<volatile unsigned long long*>(b.keys + si)) atomicMin(b.keys + si, key);
            }
        } else {
            traj_sample<W, G, STAGE_TH, VAR, KSQ>(b.c, job, n, n < s.N, gl, hx_all + bi * W);
        }
    }
}

template <int S>
struct BatchCollide {
    static constexpr int THREADS = S * 32;
    static constexpr int fixed_bytes() { return S * 8 * 24 + 8 * 4 + 16 + S * 8 + 64; }
};

template <int S>
__global__ void __launch_bounds__(S * 32) batch_collide_kernel(const BatchArgs b)
{
    using K = BatchCollide<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RP = b.resident_pairs;
    float4* sXY = reinterpret_cast<float4*>(smem_raw);
    float4* sV = sXY + RP;
    float4* slotA = sV + RP;                                     // [S][8]
    float2* slotB = reinterpret_cast<float2*>(slotA + S * 8);    // [S][8]
    int* dead_at = reinterpret_cast<int*>(slotB + S * 8);        // [8]
    long long* qslot = reinterpret_cast<long long*>(dead_at + 8);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    float4* sA = slotA + warp * 8;
    float2* sB = slotB + warp * 8;
    const long long total = __ldg(b.citem_prefix + b.S);
    int staged = -1;
    for (;;) {
        __syncthreads();
        if (tid == 0) *qslot = (long long)atomicAdd(b.counters + 3, 1u);
        if (tid < 8) dead_at[tid] = 0x7fffffff;
        __syncthreads();
        const long long item = *qslot;
        if (item >= total) break;
        const int r = find_slot(b.citem_prefix, b.S, item);
        const int si = b.order[r];
        const SceneDev& s = b.scenes[si];
        const int npairs = (s.M + 1) / 2;
        const bool resident = npairs <= RP;
        if (resident && staged != si) {
            for (int q = tid; q < npairs; q += K::THREADS) {
                sXY[q] = b.pXY[s.pair_off + q];
                sV[q] = b.pV[s.pair_off + q];
            }
            staged = si;
            __syncthreads();
        }
        const float4* XY = resident ? sXY : b.pXY + s.pair_off;
        const float4* V = resident ? sV : b.pV + s.pair_off;
        const int ntiles = (npairs + 31) / 32;
        const float4* tP = b.tileP + s.tile_off;
        const float4* tV = b.tileV + s.tile_off;
        const int T = s.T, N = s.N;
        const int n0 = (int)(item - __ldg(b.citem_prefix + r)) * 8;
        const int cnt = min(8, N - n0);
        const int n = n0 + lane;
        const bool mine = lane < cnt;
        unsigned live = (1u << cnt) - 1u;
        float4 ca = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 cb = make_float2(0.f, 0.f);
        if (mine) { ca = b.coefA[s.coef_off + n]; cb = b.coefB[s.coef_off + n]; }
        for (int h = 0; h <= T; ++h) {
            const float4 cur_a = ca;
            const float2 cur_b = cb;
            if (mine && h < T) {
                const long long idx = s.coef_off + (long long)(h + 1) * N + n;
                ca = b.coefA[idx];
                cb = b.coefB[idx];
            }
            const unsigned gone = __ballot_sync(FULL, lane < 8 && *(volatile int*)&dead_at[lane] <= h);
            live &= ~gone;
            if (live == 0u || ntiles <= warp) break;
            const float4 box = live_box(b.c, cur_a, cur_b, lane < 8 && ((live >> lane) & 1u), b.reach);
            const unsigned hits = warp_step_tiles(XY, V, npairs, (float)h * b.c.Ts, cur_a, cur_b, live, sA, sB,
                                                  lane, tP, tV, ntiles, warp, S, box);
            if ((hits >> lane) & 1u) atomicMin(&dead_at[lane], h);
            live &= ~hits;
        }
        __syncthreads();
        if (warp == 0) {
            unsigned long long key = ~0ull;
            if (mine) {
                const int d = dead_at[lane];
                const int fh = discard_step(b.vfirst ? b.vfirst + s.samp_off : nullptr, n, d <= T ? d : -1);
                float J = __int_as_float(0x7f800000);
                if (fh < 0) {
                    J = b.jfree[s.samp_off + n];
                    key = ((unsigned long long)__float_as_uint(J) << 32) | (unsigned)n;
                } else {
                    key = (1ull << 63) | ((unsigned long long)(T - fh) << 32) | (unsigned)n;
                }
                if (b.costs) b.costs[s.samp_off + n] = J;
                if (b.first_hit) b.first_hit[s.samp_off + n] = fh;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(FULL, key, off);
                key = o < key ? o : key;
            }
            if (lane == 0) atomicMin(b.keys + si, key);
        }
    }
}

// Grids of every scene and horizon step: block b -> (scene, h).
__global__ void __launch_bounds__(1024) batch_bin_build_kernel(const BatchArgs b)
{
    extern __shared__ int cnt[];             // [BIN_NCELL]
    __shared__ int run_tot[1024];
    const long long blk = blockIdx.x;
    const int si = find_slot(b.bstep_prefix, b.S, blk);
    const SceneDev& s = b.scenes[si];
    const int h = (int)(blk - __ldg(b.bstep_prefix + si));
    float sn, cs;
    sincosf(s.phi0, &sn, &cs);
    build_step_bins<1024>(b.obs + s.obs_off, s.M, s.x0, s.y0, sn, cs, (float)h * b.c.Ts, b.grid,
                          b.bin_cs + s.bin_off + (size_t)h * BIN_CS_STRIDE, b.bin_pts + s.bpts_off + (size_t)h * s.M,
                          cnt, run_tot);
}

// Binned check of an 8-sample item per block, one warp per sample, over the
// stored inequality rows: four steps at once, eight lanes per step, each
// cell row's run of candidates taken directly (binned_rows_inside, as the
// single-scene check); the query disk around the rectangle's centre
// recovered from its rows (as in live_box).  The chunk's first colliding
// step ends the sample; one key minimum per block.
__global__ void __launch_bounds__(256) batch_binned_kernel(const BatchArgs b)
{
    __shared__ unsigned long long red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane / BIN_ITEM_LANES, gl = lane % BIN_ITEM_LANES;
    constexpr int SB = 32 / BIN_ITEM_LANES;            // steps per chunk
    const long long item = blockIdx.x;
    const int r = find_slot(b.citem_prefix, b.S, item);
    const int si = b.order[r];
    const SceneDev& s = b.scenes[si];
    if (b.windowed64 && s.width == 64) return;       // checked inside the trajectory kernel (block-uniform)
    const int T = s.T, N = s.N, M = s.M;
    const int n = (int)(item - __ldg(b.citem_prefix + r)) * 8 + warp;
    const BinView& g = b.grid;
    const float isl = 1.0f / (2.0f * b.c.ihl), isw = 1.0f / (2.0f * b.c.ihw);
    unsigned long long key = ~0ull;
    if (n < N) {
        int fh = -1;
        for (int h0 = 0; h0 <= T; h0 += SB) {
            const int h = h0 + gid;
            const bool ok = h <= T;
            float4 ca = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 cb = make_float2(0.f, 0.f);
            if (ok) {
                const long long idx = s.coef_off + (long long)h * N + n;
                ca = b.coefA[idx];
                cb = b.coefB[idx];
            }
            const float cp = ca.x * isl, sp = ca.y * isl;
            const float along = -ca.z * isl, across = -cb.y * isw;
            const float xc = cp * along - sp * across, yc = sp * along + cp * across;
            const int hq = ok ? h : 0;
            unsigned ntest = 0;
            const bool inside = binned_rows_inside<1>(g, b.bin_cs + s.bin_off + (size_t)hq * BIN_CS_STRIDE,
                                                      b.bin_pts + s.bpts_off + (size_t)hq * M, ca, cb, xc, yc,
                                                      b.reach, ok, gl, ntest);
            const unsigned bal = __ballot_sync(FULL, inside);
            unsigned steps_hit = 0;
#pragma unroll
            for (int k = 0; k < SB; ++k)
                if ((bal >> (k * BIN_ITEM_LANES)) & ((1u << BIN_ITEM_LANES) - 1u)) steps_hit |= 1u << k;
            if (steps_hit) {
                fh = h0 + __ffs(steps_hit) - 1;
                break;
            }
        }
        if (lane == 0) {
            fh = discard_step(b.vfirst ? b.vfirst + s.samp_off : nullptr, n, fh);
            float J = __int_as_float(0x7f800000);
            if (fh < 0) {
                J = b.jfree[s.samp_off + n];
                key = ((unsigned long long)__float_as_uint(J) << 32) | (unsigned)n;
            } else {
                key = (1ull << 63) | ((unsigned long long)(T - fh) << 32) | (unsigned)n;
            }
            if (b.costs) b.costs[s.samp_off + n] = J;
            if (b.first_hit) b.first_hit[s.samp_off + n] = fh;
        }
    }
    if (lane == 0) red[warp] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long k = red[0];
        for (int w = 1; w < 8; ++w) k = red[w] < k ? red[w] : k;
        atomicMin(b.keys + si, k);
    }
}

// one warp per scene: winner summary, parameters, re-rolled controls and
// trajectory (EV frame, then converted to the world frame in place).  Every
// group of G lanes of the warp computes the winner (the warp-wide shuffles
// need all lanes); the groups write identical values.
template <int W, int G, bool VAR>
__device__ void batch_reroll(const BatchArgs& b, const SceneDev& s, int idx, float* hrows)
{
    const int lane = threadIdx.x & 31;
    TrajJob job;
    job.si = scene_step_in(s);
    job.key.k0 = s.k0; job.key.k1 = s.k1; job.key.t_index = s.t_index; job.key.stream_id = 0u;
    job.theta = nullptr;
    job.warm = nullptr;
    job.prop = Proposal{ nullptr, nullptr, 0, 1u };
    job.bins = nullptr;
    job.stage = nullptr;
    job.w2s = nullptr;
    job.N = s.N;
    job.T = s.T;
    job.traj = b.trajectory ? reinterpret_cast<float4*>(b.trajectory) + s.traj_off : nullptr;
    job.ctrl = b.controls ? reinterpret_cast<float2*>(b.controls) + s.ctrl_off : nullptr;
    job.rec_stride = 1;
    job.rec_shift = idx;
    job.coefA = nullptr;
    job.coefB = nullptr;
    job.coef_base = 0;
    job.jfree = nullptr;
    job.vfirst = nullptr;
    traj_sample<W, G, 0, VAR>(b.c, job, idx, true, lane % G, hrows + (lane / G) * W);
}

__global__ void batch_epilogue_kernel(const BatchArgs b)
{
    __shared__ __align__(16) float hrow[64];
    const int si = blockIdx.x;
    const SceneDev& s = b.scenes[si];
    const int lane = threadIdx.x;
    const unsigned long long key = b.keys[si];
    const int idx = (int)(key & 0xffffffffull);
    const bool dead = (key >> 63) != 0;
    const unsigned hi = (unsigned)((key >> 32) & 0x7fffffffu);
    const int fh = dead ? s.T - (int)hi : -1;
    const int last = dead ? fh : s.T;
    if (lane == 0) {
        npp_best* o = b.best + si;
        o->best_idx = idx;
        o->status = dead ? NPP_INFEASIBLE : NPP_OK;
        o->best_cost = dead ? __int_as_float(0x7f800000) : __uint_as_float(hi);
        o->first_hit = fh;
        o->reserved[0] = o->reserved[1] = o->reserved[2] = o->reserved[3] = 0;
    }
    const bool var = uses_variants(b.c);
    switch (s.width) {
    case 16: if (var) batch_reroll<16, 8, true>(b, s, idx, hrow); else batch_reroll<16, 8, false>(b, s, idx, hrow); break;
    case 32: if (var) batch_reroll<32, 16, true>(b, s, idx, hrow); else batch_reroll<32, 16, false>(b, s, idx, hrow); break;
    default: if (var) batch_reroll<64, 32, true>(b, s, idx, hrow); else batch_reroll<64, 32, false>(b, s, idx, hrow); break;
    }
    __syncwarp();
    // world frame; rows after an infeasible winner's first collision repeat
    // the colliding state, its controls there are zero
    float sn, cs;
    sincosf(s.phi0, &sn, &cs);
    if (b.trajectory) {
        float4* tr = reinterpret_cast<float4*>(b.trajectory) + s.traj_off;
        const float4 zl = tr[last];
        __syncwarp();                        // every lane has zl before rows change
        for (int h = lane; h <= s.T; h += 32) {
            const float4 z = h <= last ? tr[h] : zl;
            float4 w;
            w.x = s.x0 + cs * z.x - sn * z.y;
            w.y = s.y0 + sn * z.x + cs * z.y;
            w.z = s.phi0 + z.z;
            w.w = z.w;
            tr[h] = w;                       // each lane converts only its own rows
        }
    }
    if (b.controls) {
        float2* ct = reinterpret_cast<float2*>(b.controls) + s.ctrl_off;
        for (int h = lane; h < s.T; h += 32)
            if (h >= last) ct[h] = make_float2(0.f, 0.f);
    }
    if (b.params) {
        SamplerKey k;
        k.k0 = s.k0; k.k1 = s.k1; k.t_index = s.t_index; k.stream_id = 0u;
        const int nt = 12 * s.width + s.width * s.width + 2;
        float* pr = b.params + s.params_off;
        for (int q = lane; 4 * q < nt; q += 32) {
            const float4 v = sample_quad(k, (uint32_t)q, (uint32_t)idx);
            const float vv[4] = { v.x, v.y, v.z, v.w };
            for (int j = 0; j < 4 && 4 * q + j < nt; ++j) pr[4 * q + j] = vv[j];
        }
    }
}

int n_theta_w(int w) { return 12 * w + w * w + 2; }

}  // namespace

struct npp_batch {
    npp_handle* h;
    int S;
    std::vector<npp_scene> scenes;
    std::vector<long long> offs;     // per scene: params, controls, traj, samples
    SceneDev* d_scenes;
    int* d_order;
    long long* d_citem_prefix;
    int* d_torder[3];
    long long* d_titem_prefix[3];
    int n_torder[3];
    float4* d_pXY;
    float4* d_pV;
    float4* d_tileP;
    float4* d_tileV;
    int* d_bin_cs;
    float2* d_bin_pts;
    long long* d_bstep_prefix;
    long long bin_blocks;    // sum over scenes of T + 1
    long long total_items;   // sum over scenes of ceil(N / 8)
    int binned;              // collision check: 0 brute force (tile-culled), 1 per-step bins
    float4* d_coefA;
    float2* d_coefB;
    float* d_jfree;
    int* d_vfirst;           // [samples] when the handle's speed limits are on
    unsigned long long* d_keys;
    unsigned* d_counters;
    int resident_pairs;
    int max_pairs;
    long long total_pairs, total_rows, total_samples;
    int grid_traj[3], grid_collide;
    int slices;              // warps per collision item (point slices): 2, 4, 8
    int traj_warps;          // warps per trajectory block: 4, 8
    int smem_optin;
};

namespace {

constexpr int MAX_SLICES = 8;

void free_batch(npp_batch* B)
{
    if (!B) return;
    void* ptrs[] = { B->d_scenes, B->d_order, B->d_citem_prefix, B->d_torder[0], B->d_torder[1],
                     B->d_torder[2], B->d_titem_prefix[0], B->d_titem_prefix[1], B->d_titem_prefix[2],
                     B->d_pXY, B->d_pV, B->d_tileP, B->d_tileV, B->d_bin_cs, B->d_bin_pts, B->d_bstep_prefix,
                     B->d_coefA, B->d_coefB, B->d_jfree, B->d_vfirst, B->d_keys, B->d_counters };
    for (void* p : ptrs) if (p) cudaFree(p);
    delete B;
}

npp_status upload_scenes(npp_batch* B)
{
    npp_handle* h = B->h;
    std::vector<SceneDev> sd(B->S);
    long long pair = 0, rows = 0, samp = 0, par = 0, ctl = 0, trj = 0, tiles = 0, bcs = 0, bpts = 0;
    std::vector<long long> bstep(B->S + 1, 0);
    for (int i = 0; i < B->S; ++i) {
        const npp_scene& s = B->scenes[i];
        SceneDev& d = sd[i];
        d.x0 = s.state.x; d.y0 = s.state.y; d.phi0 = s.state.phi; d.v0 = s.state.v;
        d.ap0 = s.state.a_prev0; d.ap1 = s.state.a_prev1;
        d.gx = s.goal.x; d.gy = s.goal.y; d.gphi = s.goal.phi; d.gv = s.goal.v;
        d.N = s.N; d.T = s.T; d.M = s.M; d.width = s.width;
        d.obs_off = s.obs_offset;
        d.pair_off = pair; pair += (s.M + 1) / 2;
        d.tile_off = tiles; tiles += ((s.M + 1) / 2 + 31) / 32;
        d.bin_off = bcs; bcs += (long long)(s.T + 1) * BIN_CS_STRIDE;
        d.bpts_off = bpts; bpts += (long long)(s.T + 1) * s.M;
        bstep[i + 1] = bstep[i] + s.T + 1;
        d.coef_off = rows; rows += (long long)s.N * (s.T + 1);
        d.samp_off = samp; samp += s.N;
        d.params_off = par; par += n_theta_w(s.width);
        d.ctrl_off = ctl; ctl += s.T;
        d.traj_off = trj; trj += s.T + 1;
        d.k0 = (uint32_t)(s.seed & 0xffffffffu);
        d.k1 = (uint32_t)(s.seed >> 32);
        d.t_index = s.t_index;
        d.pad = 0;
    }
    CUDA_TRY(h, cudaMemcpy(B->d_scenes, sd.data(), sizeof(SceneDev) * B->S, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(B->d_bstep_prefix, bstep.data(), sizeof(long long) * (B->S + 1), cudaMemcpyHostToDevice));
    B->bin_blocks = bstep[B->S];
    return NPP_OK;
}


template <int S>
cudaError_t collide_grid(npp_batch* B, int* grid)
{
    const int smem = B->resident_pairs * 32 + BatchCollide<S>::fixed_bytes();
    cudaError_t e = ensure_smem(batch_collide_kernel<S>, smem);
    int nb = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_collide_kernel<S>,
                                                          BatchCollide<S>::THREADS, smem);
    *grid = B->h->sm_count * std::max(1, nb);
    return e;
}

template <int W, int G>
constexpr int batch_stage_bytes(int nw) { return W == 32 ? LaneNet<W, G>::SLOTS * nw * 32 * (int)sizeof(float) : 0; }

// width 64: 8 of 16 layer-2 input quads per lane in shared memory, 16 warps
// per SM (the single-scene default; 250 registers and 8 warps per SM with
// every weight in registers)
constexpr int BATCH_KSQ64 = 8;
constexpr int batch_w2s_bytes64(int nw) { return nw * 32 * 2 * BATCH_KSQ64 * 16; }
// with the windowed check: the W2 quads of 12 inputs per lane in shared
// memory (registers for the check, as the single-scene kernel) and the
// warps' windows of states
constexpr int BATCH_KSQ64W = 12;
constexpr int batch_w64w_bytes(int nw) { return nw * 32 * 2 * BATCH_KSQ64W * 16 + nw * BATCH_CW * 16; }

template <int NW>
void traj_grids(npp_batch* B)
{
    int nt = 0;
    const int s16 = batch_stage_bytes<16, 8>(NW), s32 = batch_stage_bytes<32, 16>(NW);
    ensure_smem(batch_traj_kernel<16, 8, NW>, s16);
    ensure_smem(batch_traj_kernel<32, 16, NW, false, 0, 16 / NW>, s32);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nt, batch_traj_kernel<16, 8, NW>, NW * 32, s16);
    B->grid_traj[0] = B->h->sm_count * std::max(1, nt);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nt, batch_traj_kernel<32, 16, NW, false, 0, 16 / NW>, NW * 32, s32);
    B->grid_traj[1] = B->h->sm_count * std::max(1, nt);
    auto k64 = batch_traj_kernel<64, 32, NW, false, BATCH_KSQ64, 16 / NW>;
    ensure_smem(k64, batch_w2s_bytes64(NW));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nt, k64, NW * 32, batch_w2s_bytes64(NW));
    B->grid_traj[2] = B->h->sm_count * std::max(1, nt);
}

// work order (costliest scenes first), item prefixes for the current block
// shapes, persistent grids
npp_status plan_work(npp_batch* B)
{
    npp_handle* h = B->h;
    const int S = B->S;
    const std::vector<npp_scene>& sc = B->scenes;
    std::vector<int> order(S);
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int i) { return (double)sc[i].N * (sc[i].T + 1) * (1.0 + sc[i].M); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<long long> cpre(S + 1, 0);
    for (int r = 0; r < S; ++r) cpre[r + 1] = cpre[r] + (sc[order[r]].N + 7) / 8;
    CUDA_TRY(h, cudaMemcpy(B->d_order, order.data(), sizeof(int) * S, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(B->d_citem_prefix, cpre.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice));
    const int widths[3] = { 16, 32, 64 };
    for (int w = 0; w < 3; ++w) {
        const int Bsz = B->traj_warps * 32 / (widths[w] / 2);
        std::vector<int> v;
        for (int r = 0; r < S; ++r) if (sc[order[r]].width == widths[w]) v.push_back(order[r]);
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
            return (double)sc[a].N * sc[a].T > (double)sc[b].N * sc[b].T; });
        std::vector<long long> pre(v.size() + 1, 0);
        for (size_t r = 0; r < v.size(); ++r) pre[r + 1] = pre[r] + (sc[v[r]].N + Bsz - 1) / Bsz;
        B->n_torder[w] = (int)v.size();
        if (!v.empty()) CUDA_TRY(h, cudaMemcpy(B->d_torder[w], v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(h, cudaMemcpy(B->d_titem_prefix[w], pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice));
    }
    cudaError_t e;
    switch (B->slices) {
    case 2: e = collide_grid<2>(B, &B->grid_collide); break;
    case 8: e = collide_grid<8>(B, &B->grid_collide); break;
    default: e = collide_grid<4>(B, &B->grid_collide); break;
    }
    if (e != cudaSuccess) return fail(h, NPP_CUDA_ERROR, "batch collision set-up: %s", cudaGetErrorString(e));
    if (B->traj_warps == 4) traj_grids<4>(B); else traj_grids<8>(B);
    return NPP_OK;
}

template <int S>
void launch_batch_collide(npp_batch* B, const BatchArgs& b, cudaStream_t s)
{
    const int smem = B->resident_pairs * 32 + BatchCollide<S>::fixed_bytes();
    batch_collide_kernel<S><<<B->grid_collide, BatchCollide<S>::THREADS, smem, s>>>(b);
}

template <int NW, bool VAR>
void launch_batch_traj_v(npp_batch* B, const BatchArgs& b, cudaStream_t s)
{
    if (B->n_torder[0]) {
        ensure_smem(batch_traj_kernel<16, 8, NW, VAR>, batch_stage_bytes<16, 8>(NW));
        batch_traj_kernel<16, 8, NW, VAR><<<B->grid_traj[0], NW * 32, batch_stage_bytes<16, 8>(NW), s>>>(b, 0);
    }
    if (B->n_torder[1]) {
        ensure_smem(batch_traj_kernel<32, 16, NW, VAR, 0, 16 / NW>, batch_stage_bytes<32, 16>(NW));
        batch_traj_kernel<32, 16, NW, VAR, 0, 16 / NW><<<B->grid_traj[1], NW * 32, batch_stage_bytes<32, 16>(NW), s>>>(b, 1);
    }
    if (B->n_torder[2] && b.windowed64) {
        auto k64 = batch_traj_kernel<64, 32, NW, VAR, BATCH_KSQ64W, 16 / NW, true>;
        ensure_smem(k64, batch_w64w_bytes(NW));
        k64<<<B->grid_traj[2], NW * 32, batch_w64w_bytes(NW), s>>>(b, 2);
    } else if (B->n_torder[2]) {
        auto k64 = batch_traj_kernel<64, 32, NW, VAR, BATCH_KSQ64, 16 / NW>;
        ensure_smem(k64, batch_w2s_bytes64(NW));
        k64<<<B->grid_traj[2], NW * 32, batch_w2s_bytes64(NW), s>>>(b, 2);
    }
}

// rollout variants (body-frame features, speed limits) in their own kernels
template <int NW>
void launch_batch_traj(npp_batch* B, const BatchArgs& b, cudaStream_t s)
{
    if (uses_variants(b.c)) launch_batch_traj_v<NW, true>(B, b, s);
    else launch_batch_traj_v<NW, false>(B, b, s);
}

}  // namespace

extern "C" {

npp_status npp_batch_create(npp_handle* h, const npp_scene* scenes, int32_t S, npp_batch** out)
{
    if (!h || !out || !scenes || S < 1) return fail(h, NPP_INVALID_ARG, "batch: bad arguments");
    *out = nullptr;
    if (h->fp_faces > 0)
        return fail(h, NPP_UNSUPPORTED, "batch: a general footprint is checked by the single-scene entry points only");
    long long pairs = 0, rows = 0, samples = 0, tiles_total = 0, bin_ints = 0, bin_pts = 0, items = 0;
    int max_pairs = 0;
    for (int i = 0; i < S; ++i) {
        const npp_scene& s = scenes[i];
        if (s.N < 1 || s.T < 1 || s.M < 0 || s.obs_offset < 0 ||
            (s.width != 16 && s.width != 32 && s.width != 64))
            return fail(h, NPP_INVALID_ARG, "batch: scene %d has bad N, T, M, width or offset", i);
        const float* f = &s.state.x;
        for (int k = 0; k < 6; ++k) if (!std::isfinite(f[k])) return fail(h, NPP_INVALID_ARG, "batch: scene %d state", i);
        const float* g = &s.goal.x;
        for (int k = 0; k < 4; ++k) if (!std::isfinite(g[k])) return fail(h, NPP_INVALID_ARG, "batch: scene %d goal", i);
        if (std::fabs(s.state.a_prev0) > 1.f || std::fabs(s.state.a_prev1) > 1.f)
            return fail(h, NPP_INVALID_ARG, "batch: scene %d previous controls outside [-1, 1]", i);
        pairs += (s.M + 1) / 2;
        tiles_total += ((s.M + 1) / 2 + 31) / 32;
        bin_ints += (long long)(s.T + 1) * BIN_CS_STRIDE;
        bin_pts += (long long)(s.T + 1) * s.M;
        items += (s.N + 7) / 8;
        rows += (long long)s.N * (s.T + 1);
        samples += s.N;
        max_pairs = std::max(max_pairs, (s.M + 1) / 2);
    }
    CUDA_TRY(h, cudaSetDevice(h->device));
    npp_batch* B = new npp_batch();
    B->h = h;
    B->S = S;
    B->scenes.assign(scenes, scenes + S);
    B->total_pairs = pairs;
    B->total_rows = rows;
    B->total_samples = samples;
    B->max_pairs = max_pairs;
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    const int cap = (smem_optin - BatchCollide<MAX_SLICES>::fixed_bytes()) / 32;
    B->resident_pairs = std::min(max_pairs, cap);

    B->smem_optin = smem_optin;
    B->slices = 4;
    B->traj_warps = 8;
    B->binned = 1;
    B->total_items = items;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16); };
    A((void**)&B->d_scenes, sizeof(SceneDev) * S);
    A((void**)&B->d_order, sizeof(int) * S);
    A((void**)&B->d_citem_prefix, sizeof(long long) * (S + 1));
    for (int w = 0; w < 3; ++w) {
        A((void**)&B->d_torder[w], sizeof(int) * S);
        A((void**)&B->d_titem_prefix[w], sizeof(long long) * (S + 1));
    }
    A((void**)&B->d_pXY, sizeof(float4) * std::max(1LL, pairs));
    A((void**)&B->d_pV, sizeof(float4) * std::max(1LL, pairs));
    A((void**)&B->d_tileP, sizeof(float4) * std::max(1LL, tiles_total));
    A((void**)&B->d_tileV, sizeof(float4) * std::max(1LL, tiles_total));
    A((void**)&B->d_bin_cs, sizeof(int) * std::max(1LL, bin_ints));
    A((void**)&B->d_bin_pts, sizeof(float2) * std::max(1LL, bin_pts));
    A((void**)&B->d_bstep_prefix, sizeof(long long) * (S + 1));
    A((void**)&B->d_coefA, sizeof(float4) * rows);
    A((void**)&B->d_coefB, sizeof(float2) * rows);
    A((void**)&B->d_jfree, sizeof(float) * samples);
    if (h->cfg.v_limits) A((void**)&B->d_vfirst, sizeof(int) * samples);
    A((void**)&B->d_keys, sizeof(unsigned long long) * S);
    A((void**)&B->d_counters, 64);
    if (e != cudaSuccess) {
        free_batch(B);
        return fail(h, NPP_CUDA_ERROR, "batch allocation failed: %s", cudaGetErrorString(e));
    }
    npp_status st = upload_scenes(B);
    if (st == NPP_OK) st = plan_work(B);
    if (st != NPP_OK) { free_batch(B); return st; }
    *out = B;
    return NPP_OK;
}

npp_status npp_batch_update(npp_batch* B, const npp_scene* scenes)
{
    if (!B || !scenes) return fail(B ? B->h : nullptr, NPP_INVALID_ARG, "batch: bad arguments");
    for (int i = 0; i < B->S; ++i) {
        const npp_scene& a = B->scenes[i];
        const npp_scene& s = scenes[i];
        if (a.N != s.N || a.T != s.T || a.M != s.M || a.width != s.width || a.obs_offset != s.obs_offset)
            return fail(B->h, NPP_INVALID_ARG, "batch: scene %d changed its sizes (create a new batch)", i);
    }
    CUDA_TRY(B->h, cudaSetDevice(B->h->device));
    B->scenes.assign(scenes, scenes + B->S);
    return upload_scenes(B);
}

npp_status npp_batch_offsets(npp_batch* B, int64_t* offsets)
{
    if (!B || !offsets) return fail(B ? B->h : nullptr, NPP_INVALID_ARG, "batch: bad arguments");
    long long par = 0, ctl = 0, trj = 0, smp = 0;
    for (int i = 0; i < B->S; ++i) {
        const npp_scene& s = B->scenes[i];
        offsets[4 * i + 0] = par;
        offsets[4 * i + 1] = ctl;
        offsets[4 * i + 2] = trj;
        offsets[4 * i + 3] = smp;
        par += n_theta_w(s.width);
        ctl += s.T;
        trj += s.T + 1;
        smp += s.N;
    }
    offsets[4 * B->S + 0] = par;
    offsets[4 * B->S + 1] = ctl;
    offsets[4 * B->S + 2] = trj;
    offsets[4 * B->S + 3] = smp;
    return NPP_OK;
}

npp_status npp_plan_batch(npp_batch* B, const float* obs_dev, const npp_batch_outputs* out, void* stream)
{
    if (!B || !out || !out->best) return fail(B ? B->h : nullptr, NPP_INVALID_ARG, "batch: outputs.best required");
    npp_handle* h = B->h;
    if (B->total_pairs > 0 && (!obs_dev || (reinterpret_cast<uintptr_t>(obs_dev) & 15u)))
        return fail(h, NPP_INVALID_ARG, "batch: obstacle array NULL or not 16-byte aligned");
    CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BatchArgs b;
    memset(&b, 0, sizeof b);
    b.c = h->dc;
    b.scenes = B->d_scenes;
    b.S = B->S;
    b.obs = reinterpret_cast<const float4*>(obs_dev);
    b.pXY = B->d_pXY;
    b.pV = B->d_pV;
    b.tileP = B->d_tileP;
    b.tileV = B->d_tileV;
    b.reach = (float)(std::sqrt((double)h->cfg.half_len * h->cfg.half_len + (double)h->cfg.half_wid * h->cfg.half_wid)
                      + std::fabs((double)h->cfg.c_off) + 0.1);
    b.grid = make_bin_grid(h->cfg.half_len, h->cfg.half_wid, h->cfg.c_off);
    b.windowed64 = B->binned ? 1 : 0;
    b.bin_cs = B->d_bin_cs;
    b.bin_pts = B->d_bin_pts;
    b.bstep_prefix = B->d_bstep_prefix;
    b.coefA = B->d_coefA;
    b.coefB = B->d_coefB;
    b.jfree = B->d_jfree;
    b.vfirst = B->d_vfirst;
    b.keys = B->d_keys;
    b.counters = B->d_counters;
    b.order = B->d_order;
    for (int w = 0; w < 3; ++w) {
        b.titem_prefix[w] = B->d_titem_prefix[w];
        b.torder[w] = B->d_torder[w];
        b.n_torder[w] = B->n_torder[w];
    }
    b.citem_prefix = B->d_citem_prefix;
    b.resident_pairs = B->resident_pairs;
    b.best = out->best;
    b.params = out->params;
    b.controls = out->controls;
    b.trajectory = out->trajectory;
    b.costs = out->costs;
    b.first_hit = out->first_hit;
    if (h->timing) {
        CUDA_TRY(h, record_event(h->ev[0], s));
        h->last_chunks = 1;
    }
    CUDA_TRY(h, cudaMemsetAsync(B->d_keys, 0xff, sizeof(unsigned long long) * B->S, s));
    CUDA_TRY(h, cudaMemsetAsync(B->d_counters, 0, 64, s));
    if (B->max_pairs > 0) {
        const int smem = SORT_KEYS * (int)sizeof(int);
        CUDA_TRY(h, ensure_smem(batch_prologue_kernel, smem));
        batch_prologue_kernel<<<B->S, SORT_THREADS, smem, s>>>(b);
        CUDA_TRY(h, cudaGetLastError());
    }
    // with the binned check the grids come first: the width-64 scenes are
    // checked inside their trajectory kernel (windowed), the others after
    if (B->binned && B->bin_blocks > 0) {
        const int smem = BIN_NCELL * (int)sizeof(int);
        CUDA_TRY(h, ensure_smem(batch_bin_build_kernel, smem));
        batch_bin_build_kernel<<<(unsigned)B->bin_blocks, 1024, smem, s>>>(b);
        CUDA_TRY(h, cudaGetLastError());
    }
    if (B->traj_warps == 4) launch_batch_traj<4>(B, b, s); else launch_batch_traj<8>(B, b, s);
    CUDA_TRY(h, cudaGetLastError());
    if (h->timing) CUDA_TRY(h, record_event(h->ev[1], s));
    if (B->binned) {
        batch_binned_kernel<<<(unsigned)B->total_items, 256, 0, s>>>(b);
    } else {
        switch (B->slices) {
        case 2: launch_batch_collide<2>(B, b, s); break;
        case 8: launch_batch_collide<8>(B, b, s); break;
        default: launch_batch_collide<4>(B, b, s); break;
        }
    }
    CUDA_TRY(h, cudaGetLastError());
    if (h->timing) CUDA_TRY(h, record_event(h->ev[2], s));
    batch_epilogue_kernel<<<B->S, 32, 0, s>>>(b);
    CUDA_TRY(h, cudaGetLastError());
    if (h->timing) CUDA_TRY(h, record_event(h->ev[3], s));
    return NPP_OK;
}

npp_status npp_batch_set_option(npp_batch* B, const char* name, int32_t value)
{
    if (!B || !name) return fail(B ? B->h : nullptr, NPP_INVALID_ARG, "batch: bad arguments");
    if (std::strcmp(name, "slices") == 0) {
        if (value != 2 && value != 4 && value != 8) return fail(B->h, NPP_INVALID_ARG, "slices is 2, 4 or 8");
        B->slices = value;
    } else if (std::strcmp(name, "traj_warps") == 0) {
        if (value != 4 && value != 8) return fail(B->h, NPP_INVALID_ARG, "traj_warps is 4 or 8");
        B->traj_warps = value;
    } else if (std::strcmp(name, "collide") == 0) {
        if (value != 0 && value != 1) return fail(B->h, NPP_INVALID_ARG, "collide is 0 or 1");
        B->binned = value;
    } else {
        return fail(B->h, NPP_INVALID_ARG, "unknown batch option '%s'", name);
    }
    CUDA_TRY(B->h, cudaSetDevice(B->h->device));
    return plan_work(B);
}

npp_status npp_batch_destroy(npp_batch* B)
{
    if (!B) return NPP_OK;
    cudaSetDevice(B->h->device);
    cudaDeviceSynchronize();
    free_batch(B);
    return NPP_OK;
}

}  // extern "C"
