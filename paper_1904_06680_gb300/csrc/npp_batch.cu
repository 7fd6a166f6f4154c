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
    uint32_t k0, k1, t_index, pad;
};

struct BatchArgs {
    DevCfg c;
    const SceneDev* scenes;
    int S;
    const float4* obs;               // input points (world frame)
    float4* pXY;                     // transformed pairs
    float4* pV;
    float4* coefA;
    float2* coefB;
    float* jfree;
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

// world -> EV frame, as pairs (odd tail padded with a far point)
__global__ void batch_prologue_kernel(const BatchArgs b)
{
    const SceneDev& s = b.scenes[blockIdx.y];
    const int npairs = (s.M + 1) / 2;
    float sn, cs;
    sincosf(s.phi0, &sn, &cs);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += gridDim.x * blockDim.x) {
        float px[2], py[2], vx[2], vy[2];
        for (int o = 0; o < 2; ++o) {
            const int j = 2 * q + o;
            px[o] = 1e15f; py[o] = 1e15f; vx[o] = 0.f; vy[o] = 0.f;
            if (j < s.M) {
                ev_point(b.obs[s.obs_off + j], s.x0, s.y0, sn, cs, px[o], py[o], vx[o], vy[o]);
            }
        }
        b.pXY[s.pair_off + q] = make_float4(px[0], px[1], py[0], py[1]);
        b.pV[s.pair_off + q] = make_float4(vx[0], vx[1], vy[0], vy[1]);
    }
}

template <int W, int G, int NW>
__global__ void __launch_bounds__(NW * 32) batch_traj_kernel(const BatchArgs b, int wi)
{
    constexpr int B = TrajKernel<W, G, NW>::B;
    __shared__ __align__(16) float hx_all[B * W];
    __shared__ long long qslot;
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
        job.prop = Proposal{ nullptr, nullptr, 0 };
        job.bins = nullptr;
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
        traj_sample<W, G>(b.c, job, n, n < s.N, gl, hx_all + bi * W);
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
        const int per = (npairs + S - 1) / S;
        const int q0 = min(npairs, warp * per), q1 = min(npairs, q0 + per);
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
            if (live == 0u || q1 <= q0) break;
            const unsigned hits = warp_step(XY + q0, V + q0, q1 - q0, (float)h * b.c.Ts, cur_a, cur_b,
                                            live, sA, sB, lane);
            if ((hits >> lane) & 1u) atomicMin(&dead_at[lane], h);
            live &= ~hits;
        }
        __syncthreads();
        if (warp == 0) {
            unsigned long long key = ~0ull;
            if (mine) {
                const int d = dead_at[lane];
                const int fh = d <= T ? d : -1;
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

// one warp per scene: winner summary, parameters, re-rolled controls and
// trajectory (EV frame, then converted to the world frame in place).  Every
// group of G lanes of the warp computes the winner (the warp-wide shuffles
// need all lanes); the groups write identical values.
template <int W, int G>
__device__ void batch_reroll(const BatchArgs& b, const SceneDev& s, int idx, float* hrows)
{
    const int lane = threadIdx.x & 31;
    TrajJob job;
    job.si = scene_step_in(s);
    job.key.k0 = s.k0; job.key.k1 = s.k1; job.key.t_index = s.t_index; job.key.stream_id = 0u;
    job.theta = nullptr;
    job.warm = nullptr;
    job.prop = Proposal{ nullptr, nullptr, 0 };
    job.bins = nullptr;
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
    traj_sample<W, G>(b.c, job, idx, true, lane % G, hrows + (lane / G) * W);
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
    switch (s.width) {
    case 16: batch_reroll<16, 8>(b, s, idx, hrow); break;
    case 32: batch_reroll<32, 16>(b, s, idx, hrow); break;
    default: batch_reroll<64, 32>(b, s, idx, hrow); break;
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
    float4* d_coefA;
    float2* d_coefB;
    float* d_jfree;
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
                     B->d_pXY, B->d_pV, B->d_coefA, B->d_coefB, B->d_jfree, B->d_keys, B->d_counters };
    for (void* p : ptrs) if (p) cudaFree(p);
    delete B;
}

npp_status upload_scenes(npp_batch* B)
{
    npp_handle* h = B->h;
    std::vector<SceneDev> sd(B->S);
    long long pair = 0, rows = 0, samp = 0, par = 0, ctl = 0, trj = 0;
    for (int i = 0; i < B->S; ++i) {
        const npp_scene& s = B->scenes[i];
        SceneDev& d = sd[i];
        d.x0 = s.state.x; d.y0 = s.state.y; d.phi0 = s.state.phi; d.v0 = s.state.v;
        d.ap0 = s.state.a_prev0; d.ap1 = s.state.a_prev1;
        d.gx = s.goal.x; d.gy = s.goal.y; d.gphi = s.goal.phi; d.gv = s.goal.v;
        d.N = s.N; d.T = s.T; d.M = s.M; d.width = s.width;
        d.obs_off = s.obs_offset;
        d.pair_off = pair; pair += (s.M + 1) / 2;
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

template <int NW>
void traj_grids(npp_batch* B)
{
    int nt = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nt, batch_traj_kernel<16, 8, NW>, NW * 32, 0);
    B->grid_traj[0] = B->h->sm_count * std::max(1, nt);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nt, batch_traj_kernel<32, 16, NW>, NW * 32, 0);
    B->grid_traj[1] = B->h->sm_count * std::max(1, nt);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nt, batch_traj_kernel<64, 32, NW>, NW * 32, 0);
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

template <int NW>
void launch_batch_traj(npp_batch* B, const BatchArgs& b, cudaStream_t s)
{
    if (B->n_torder[0]) batch_traj_kernel<16, 8, NW><<<B->grid_traj[0], NW * 32, 0, s>>>(b, 0);
    if (B->n_torder[1]) batch_traj_kernel<32, 16, NW><<<B->grid_traj[1], NW * 32, 0, s>>>(b, 1);
    if (B->n_torder[2]) batch_traj_kernel<64, 32, NW><<<B->grid_traj[2], NW * 32, 0, s>>>(b, 2);
}

}  // namespace

extern "C" {

npp_status npp_batch_create(npp_handle* h, const npp_scene* scenes, int32_t S, npp_batch** out)
{
    if (!h || !out || !scenes || S < 1) return fail(h, NPP_INVALID_ARG, "batch: bad arguments");
    *out = nullptr;
    long long pairs = 0, rows = 0, samples = 0;
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
    A((void**)&B->d_coefA, sizeof(float4) * rows);
    A((void**)&B->d_coefB, sizeof(float2) * rows);
    A((void**)&B->d_jfree, sizeof(float) * samples);
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
    b.coefA = B->d_coefA;
    b.coefB = B->d_coefB;
    b.jfree = B->d_jfree;
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
    if (h->timing) CUDA_TRY(h, record_event(h->ev[0], s));
    CUDA_TRY(h, cudaMemsetAsync(B->d_keys, 0xff, sizeof(unsigned long long) * B->S, s));
    CUDA_TRY(h, cudaMemsetAsync(B->d_counters, 0, 64, s));
    if (B->max_pairs > 0) {
        dim3 grid((unsigned)std::min(64, (B->max_pairs + 255) / 256), (unsigned)B->S);
        batch_prologue_kernel<<<grid, 256, 0, s>>>(b);
        CUDA_TRY(h, cudaGetLastError());
    }
    if (B->traj_warps == 4) launch_batch_traj<4>(B, b, s); else launch_batch_traj<8>(B, b, s);
    CUDA_TRY(h, cudaGetLastError());
    if (h->timing) CUDA_TRY(h, record_event(h->ev[1], s));
    switch (B->slices) {
    case 2: launch_batch_collide<2>(B, b, s); break;
    case 8: launch_batch_collide<8>(B, b, s); break;
    default: launch_batch_collide<4>(B, b, s); break;
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
