// npp_api.cu -- handle, argument validation, small kernels (winner epilogue,
// parameter sampler) and the extern "C" entry points declared in npp.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_device.cuh"
#include "npp_internal.h"

using namespace npp;

static std::string g_err;

npp_status fail(npp_handle* h, npp_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    g_err = buf;                       // npp_last_error(NULL): the most recent failure
    return s;
}

static int n_theta_of(int width) { return 12 * width + width * width + 2; }

static bool finite_all(const float* p, int n)
{
    for (int i = 0; i < n; ++i) if (!std::isfinite(p[i])) return false;
    return true;
}

// ------------------------------------------------------------------ kernels
namespace {

// Winner epilogue: decode the packed key, write the summary record, the
// winner's world-frame trajectory and controls, and regenerate its
// parameters from Philox (or copy the warm start).
__global__ void epilogue_kernel(const EpilogueArgs e)
{
    float x0 = e.x0, y0 = e.y0, phi0 = e.phi0;
    SamplerKey skey = e.key;
    bool warm_ok = true;
    if (e.dyn) {
        x0 = e.dyn->x0; y0 = e.dyn->y0; phi0 = e.dyn->phi0;
        skey.t_index = e.dyn->t_index;
        warm_ok = e.dyn->warm_valid != 0 || e.warm_force != 0;
    }
    const unsigned long long key = *e.best_key;
    const int idx = (int)(key & 0xffffffffull);
    const bool dead = (key >> 63) != 0;
    const unsigned hi = (unsigned)((key >> 32) & 0x7fffffffu);
    const int fh = dead ? e.T - (int)hi : -1;
    const int last = dead ? fh : e.T;
    if (threadIdx.x == 0) {
        npp_best* b = reinterpret_cast<npp_best*>(e.best);
        b->best_idx = idx;
        b->status = dead ? NPP_INFEASIBLE : NPP_OK;
        if (e.fault && *e.fault) {
            // a bounded wait of this step's kernels gave up: no valid result
            b->status = NPP_DEVICE_TIMEOUT;
            *e.fault = 0u;
        }
        b->best_cost = dead ? __int_as_float(0x7f800000) : __uint_as_float(hi);
        b->first_hit = fh;
        b->reserved[0] = b->reserved[1] = b->reserved[2] = b->reserved[3] = 0;
    }
    float s0, c0;
    sincosf(phi0, &s0, &c0);
    if (e.trajectory) {
        for (int h = threadIdx.x; h <= e.T; h += blockDim.x) {
            const float4 z = e.traj[(size_t)min(h, last) * e.N + idx];
            float4 w;
            w.x = x0 + c0 * z.x - s0 * z.y;
            w.y = y0 + s0 * z.x + c0 * z.y;
            w.z = phi0 + z.z;
            w.w = z.w;
            reinterpret_cast<float4*>(e.trajectory)[h] = w;
        }
    }
    if (e.controls) {
        for (int h = threadIdx.x; h < e.T; h += blockDim.x) {
            float2 a = make_float2(0.f, 0.f);
            if (h < last) a = e.ctrl[(size_t)h * e.N + idx];
            reinterpret_cast<float2*>(e.controls)[h] = a;
        }
    }
    if (e.params) {
        if (e.warm && idx == 0 && warm_ok) {
            if (e.params != e.warm)
                for (int i = threadIdx.x; i < e.n_theta; i += blockDim.x) e.params[i] = e.warm[i];
        } else {
            for (int q = threadIdx.x; 4 * q < e.n_theta; q += blockDim.x) {
                const float4 v = sample_quad_mixed_tail(skey, e.prop, (uint32_t)q, (uint32_t)idx, e.n_theta);
                const float vv[4] = { v.x, v.y, v.z, v.w };
                for (int j = 0; j < 4 && 4 * q + j < e.n_theta; ++j) e.params[4 * q + j] = vv[j];
            }
        }
    }
}

__global__ void sample_params_kernel(SamplerKey key, int n0, int K, int nt, float* out)
{
    const int nq = (nt + 3) / 4;
    const long long total = (long long)K * nq;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / nq), q = (int)(t % nq);
        const float4 v = sample_quad(key, (uint32_t)q, (uint32_t)(n0 + k));
        const float vv[4] = { v.x, v.y, v.z, v.w };
        float* row = out + (size_t)k * nt;
        for (int j = 0; j < 4 && 4 * q + j < nt; ++j) row[4 * q + j] = vv[j];
    }
}

__global__ void math_eval_kernel(int fn, const float* x, int n, float* y, float* y2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float v = x[i];
        if (fn == 0) {
            y[i] = tanh_r(v);
        } else if (fn == 1) {
            y[i] = tan_r(v);
        } else {
            float s, c;
            sincos_r(v, s, c);
            y[i] = s;
            y2[i] = c;
        }
    }
}

}  // namespace

namespace npp {
// Message for npp_last_error(NULL) from entry points without a handle.
void set_global_error(const char* msg) { g_err = msg; }

// The winner epilogue for callers outside this file (one block of 256).
cudaError_t launch_epilogue(const EpilogueArgs& e, cudaStream_t s)
{
    epilogue_kernel<<<1, 256, 0, s>>>(e);
    return cudaGetLastError();
}
}  // namespace npp

// ------------------------------------------------------------------ helpers
namespace {
__global__ void fill_value_kernel(float* p, int n, float v)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}
}  // namespace

cudaError_t stage_times(const cudaEvent_t* ev, const cudaEvent_t* cev, int nch, float t[4])
{
    cudaError_t e = cudaSuccess;
    if (nch > 1) {
        t[0] = t[1] = 0.f;
        for (int k = 0; k < nch && e == cudaSuccess; ++k) {
            float a = 0.f, b = 0.f;
            e = cudaEventElapsedTime(&a, cev[2 * k], cev[2 * k + 1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&b, cev[2 * k + 1], cev[2 * k + 2]);
            t[0] += a;
            t[1] += b;
        }
    } else {
        e = cudaEventElapsedTime(&t[0], ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t[1], ev[1], ev[2]);
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t[2], ev[2], ev[3]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t[3], ev[0], ev[3]);
    return e;
}

cudaError_t fill_floats(float* p, int n, float v, cudaStream_t s)
{
    fill_value_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

static cudaError_t launch_traj(const npp_handle* h, const RolloutArgs& a, cudaStream_t s)
{
    switch (h->cfg.width) {
    case 16: return launch_traj_w16(a, s, h->traj_variant);
    case 32: return launch_traj_w32(a, s, h->traj_variant);
    default: return launch_traj_w64(a, s, h->traj_variant);
    }
}

// trajectories, then collision checks; events around both when timing
static cudaError_t launch_fused(const npp_handle* h, const RolloutArgs& a, cudaStream_t s)
{
    switch (h->cfg.width) {
    case 16: return launch_fused_w16(a, s, h->traj_variant);
    case 32: return launch_fused_w32(a, s, h->traj_variant);
    default: return launch_fused_w64(a, s, h->traj_variant);
    }
}

// Step chunks of a binned plan step: 1 (one trajectory launch and one check)
// when the caller wants every sample's records or chooses so, else the
// handle's setting or the automatic choice, at most one per step.  Each
// chunk regenerates its samples' parameters (measured on GB300 at N = 65536,
// T = 100, width 64: 0.59 ms per full generation, 0.12 ms of launch and tail
// per chunk, 0.027 ms per step of all samples), so two chunks pay at width
// 64 (3.83 -> 3.31 ms per plan step; 3, 4, 6 chunks: 3.50, 3.87, 4.69 ms)
// and none at width 32 and T = 40 (0.258 ms in one launch, 0.293 in two).
static int chunk_count(const npp_handle* h, const RolloutArgs& a, bool no_records)
{
    if (!no_records || h->chunks == 1 || a.T < 2) return 1;
    const int k = h->chunks > 1 ? h->chunks : (h->cfg.width == 64 ? 2 : 1);
    return std::min(k, a.T);
}

// The binned plan step in K chunks of the horizon: chunk k rolls the
// samples still collision-free from the states chunk k - 1 stored over
// steps [T k / K, T (k + 1) / K) and checks the states it produced; a
// sample ends with its chunk's first collision, so no sample is rolled out
// more than one chunk past its first collision.  Per sample the arithmetic
// and the results are those of the single launch (the carried values are
// the FP32 values the single loop holds); only the records past a sample's
// last chunk are not written.  The grids are being built on the side
// stream (join_ev) while chunk 0's trajectories run.
static npp_status run_chunked(npp_handle* h, RolloutArgs& a, cudaStream_t s, int K)
{
    CUDA_TRY(h, cudaMemsetAsync(h->d_live_n, 0, NPP_MAX_CHUNKS * sizeof(int), s));
    a.carry = h->d_carry;
    const size_t half = (size_t)h->cfg.max_N;
    for (int k = 0; k < K; ++k) {
        a.chunk_lo = (int)((long long)a.T * k / K);
        a.chunk_hi = (int)((long long)a.T * (k + 1) / K);
        a.live_in = k > 0 ? h->d_live + ((k - 1) % 2) * half : nullptr;
        a.live_n_in = k > 0 ? h->d_live_n + (k - 1) : nullptr;
        a.live_out = k + 1 < K ? h->d_live + (k % 2) * half : nullptr;
        a.live_n_out = k + 1 < K ? h->d_live_n + k : nullptr;
        if (h->timing) CUDA_TRY(h, record_event(h->cev[2 * k], s));
        CUDA_TRY(h, launch_traj(h, a, s));
        if (h->timing) CUDA_TRY(h, record_event(h->cev[2 * k + 1], s));
        if (k == 0) CUDA_TRY(h, cudaStreamWaitEvent(s, h->join_ev, 0));
        CUDA_TRY(h, launch_collide_binned(a, s));
    }
    if (h->timing) {
        CUDA_TRY(h, record_event(h->cev[2 * K], s));
        CUDA_TRY(h, record_event(h->ev[2], s));
        h->last_chunks = K;
    }
    a.chunk_lo = a.chunk_hi = 0;
    a.live_in = a.live_n_in = nullptr;
    a.live_out = a.live_n_out = nullptr;
    a.carry = nullptr;
    a.counts = nullptr;
    return NPP_OK;
}

npp_status run_rollout(npp_handle* h, RolloutArgs& a, cudaStream_t s, bool no_records)
{
    // no rows are stored: every collision kernel recomputes them from the
    // stored states
    a.coefA = nullptr;
    a.coefB = nullptr;
    a.work = h->d_work;
    if (h->timing) h->last_chunks = 1;
    if (h->fp_faces > 0) {
        // general footprint: grids sized by its radius (side stream, as
        // below), trajectories without the rectangle's rows, polygon check
        a.coefA = nullptr;
        a.coefB = nullptr;
        a.poly.faces = h->d_fp;
        a.poly.n_faces = h->fp_faces;
        a.poly.brute = (h->collide_variant >= 0 && h->collide_variant < COLLIDE_BINNED) ? 1 : 0;
        // enlarged by 1e-3 relative and 1e-6 m^2: larger than any rounding of
        // a point's squared distance, so no inside point is skipped
        a.poly.r2 = (float)(h->fp_radius * h->fp_radius * 1.001 + 1e-6);
        if (h->timing) CUDA_TRY(h, record_event(h->ev[0], s));
        CUDA_TRY(h, cudaEventRecord(h->fork_ev, s));
        CUDA_TRY(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));
        CUDA_TRY(h, build_bins_radius(a, h->fp_radius, h->d_bins, h->side));
        CUDA_TRY(h, cudaEventRecord(h->join_ev, h->side));
        CUDA_TRY(h, launch_traj(h, a, s));
        if (h->timing) CUDA_TRY(h, record_event(h->ev[1], s));
        CUDA_TRY(h, cudaStreamWaitEvent(s, h->join_ev, 0));
        CUDA_TRY(h, launch_collide_poly(a, s));
        if (h->timing) CUDA_TRY(h, record_event(h->ev[2], s));
        return NPP_OK;
    }
    // automatic choice (measured on GB300): many points -> spatial binning,
    // else the brute-force variant by points and samples (brute_auto); at
    // width 64 the binned check runs window by window inside the
    // trajectory kernel unless the caller wants every sample's records
    // (measured at N = 65536, T = 100, M = 8192: 2.72 ms per plan step
    // against 3.83 in two kernels and 3.31 in two step chunks; at width 32,
    // T = 40 the two kernels stay faster, 0.258 against 0.311 ms)
    const int v = h->collide_variant >= 0 ? h->collide_variant
                : (binned_auto(a.M, a.N) ? COLLIDE_BINNED : brute_auto(a.M, a.N));
    if (v == COLLIDE_BINNED) {
        if (h->timing) CUDA_TRY(h, record_event(h->ev[0], s));
        const bool fuse = no_records && (h->fuse == 1 || (h->fuse < 0 && h->cfg.width == 64));
        if (!fuse) {
            if (h->timing) {
                // measurement counters (candidate tests, states checked,
                // sample-steps rolled out)
                CUDA_TRY(h, cudaMemsetAsync(h->d_counts, 0, 4 * sizeof(unsigned long long), s));
                a.counts = h->d_counts;
            }
            // the grids depend only on the points: build them on the side
            // stream while the trajectories run (fork/join events; under
            // stream capture this makes two graph branches)
            CUDA_TRY(h, cudaEventRecord(h->fork_ev, s));
            CUDA_TRY(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));
            CUDA_TRY(h, build_bins(a, h->cfg.half_len, h->cfg.half_wid, h->cfg.c_off, h->d_bins, h->side));
            CUDA_TRY(h, cudaEventRecord(h->join_ev, h->side));
            const int K = chunk_count(h, a, no_records);
            if (K > 1) return run_chunked(h, a, s, K);
            CUDA_TRY(h, launch_traj(h, a, s));
            if (h->timing) CUDA_TRY(h, record_event(h->ev[1], s));
            CUDA_TRY(h, cudaStreamWaitEvent(s, h->join_ev, 0));
            CUDA_TRY(h, launch_collide_binned(a, s));
            a.counts = nullptr;
            if (h->timing) CUDA_TRY(h, record_event(h->ev[2], s));
            return NPP_OK;
        }
        // fused: the grids first, then the trajectories with the windowed
        // check inside (timing: [0] the grid build, [1] the fused kernel)
        if (h->timing) {
            CUDA_TRY(h, cudaMemsetAsync(h->d_counts, 0, 4 * sizeof(unsigned long long), s));
            a.counts = h->d_counts;
        }
        CUDA_TRY(h, build_bins(a, h->cfg.half_len, h->cfg.half_wid, h->cfg.c_off, h->d_bins, s));
        if (h->timing) CUDA_TRY(h, record_event(h->ev[1], s));
        CUDA_TRY(h, launch_fused(h, a, s));
        a.counts = nullptr;
        if (h->timing) CUDA_TRY(h, record_event(h->ev[2], s));
        return NPP_OK;
    }
    // points beyond shared memory: point-sliced kernel on an L2-resident copy
    const bool global_pts = a.M > h->max_points;
    if (global_pts) {
        a.pXY = h->d_pXY;
        a.grid_collide = h->sm_count * collide_global_blocks_per_sm();
    } else {
        if (h->occ_M != a.M || h->collide_active != v) {
            h->occ_blocks = collide_resident_blocks_per_sm(a.M, v);
            h->occ_M = a.M;
            h->collide_active = v;
        }
        a.grid_collide = h->sm_count * h->occ_blocks;
    }
    CUDA_TRY(h, cudaMemsetAsync(h->d_work, 0, sizeof(unsigned), s));
    if (h->timing) CUDA_TRY(h, record_event(h->ev[0], s));
    CUDA_TRY(h, launch_traj(h, a, s));
    if (h->timing) CUDA_TRY(h, record_event(h->ev[1], s));
    CUDA_TRY(h, global_pts ? launch_collide_global(a, s) : launch_collide_resident(a, s, h->collide_active));
    if (h->timing) CUDA_TRY(h, record_event(h->ev[2], s));
    return NPP_OK;
}


static SamplerKey make_key(uint64_t seed, uint32_t t_index, uint32_t stream_id)
{
    SamplerKey k;
    k.k0 = (uint32_t)(seed & 0xffffffffu);
    k.k1 = (uint32_t)(seed >> 32);
    k.t_index = t_index;
    k.stream_id = stream_id;
    return k;
}

static npp_status check_state_goal(npp_handle* h, const npp_state* s, const npp_goal* g)
{
    if (!s || !g) return fail(h, NPP_INVALID_ARG, "state and goal must not be NULL");
    if (!finite_all(&s->x, 6)) return fail(h, NPP_INVALID_ARG, "state has a non-finite entry");
    if (!finite_all(&g->x, 4)) return fail(h, NPP_INVALID_ARG, "goal has a non-finite entry");
    if (std::fabs(s->a_prev0) > 1.0f || std::fabs(s->a_prev1) > 1.0f)
        return fail(h, NPP_INVALID_ARG, "previous controls must lie in [-1, 1]");
    return NPP_OK;
}

static npp_status check_sizes(npp_handle* h, int32_t M, int32_t N, int32_t T, const void* obs,
                              bool device_obs)
{
    const npp_config& c = h->cfg;
    if (N < 1 || N > c.max_N) return fail(h, NPP_INVALID_ARG, "N=%d outside [1, %d]", N, c.max_N);
    if (T < 1 || T > c.max_T) return fail(h, NPP_INVALID_ARG, "T=%d outside [1, %d]", T, c.max_T);
    if (M < 0 || M > c.max_M) return fail(h, NPP_INVALID_ARG, "M=%d outside [0, %d]", M, c.max_M);
    if (M > 0 && !obs) return fail(h, NPP_INVALID_ARG, "obstacle pointer is NULL with M=%d", M);
    if (device_obs && obs && (reinterpret_cast<uintptr_t>(obs) & 15u))
        return fail(h, NPP_INVALID_ARG, "obstacle array must be 16-byte aligned");
    return NPP_OK;
}

static void fill_rollout_args(const npp_handle* h, RolloutArgs& a, const npp_state* s,
                              const npp_goal* g, const float* obs, int32_t M, int32_t N, int32_t T)
{
    memset(&a, 0, sizeof a);
    a.c = h->dc;
    a.x0 = s->x; a.y0 = s->y; a.phi0 = s->phi; a.v0 = s->v; a.ap0 = s->a_prev0; a.ap1 = s->a_prev1;
    a.gx = g->x; a.gy = g->y; a.gphi = g->phi; a.gv = g->v;
    a.obs = reinterpret_cast<const float4*>(obs);
    a.M = M; a.N = N; a.T = T;
    a.vfirst = h->d_vfirst;
    a.fault = h->d_fault;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int32_t npp_n_theta(const npp_config* cfg)
{
    if (!cfg || cfg->n_in != 8) return -1;
    if (cfg->width != 16 && cfg->width != 32 && cfg->width != 64) return -1;
    return n_theta_of(cfg->width);
}

const char* npp_last_error(const npp_handle* h)
{
    return h ? h->err.c_str() : g_err.c_str();
}

npp_status npp_create(npp_handle** out, const npp_config* cfg, int32_t device)
{
    if (!out) return fail(nullptr, NPP_INVALID_ARG, "handle pointer is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, NPP_INVALID_ARG, "config is NULL");
    if (npp_n_theta(cfg) < 0)
        return fail(nullptr, NPP_UNSUPPORTED, "network [%d, %d, %d, 2] is not built (n_in 8; width 16, 32, 64)",
                    cfg->n_in, cfg->width, cfg->width);
    if (const char* ce = config_error(*cfg)) return fail(nullptr, NPP_INVALID_ARG, "%s", ce);
    if (cfg->max_N < 1 || cfg->max_T < 1 || cfg->max_M < 0)
        return fail(nullptr, NPP_INVALID_ARG, "capacity max_N, max_T >= 1, max_M >= 0 required");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(nullptr, NPP_CUDA_ERROR, "CUDA device %d not available", device);
    if (cudaSetDevice(device) != cudaSuccess)
        return fail(nullptr, NPP_CUDA_ERROR, "cudaSetDevice(%d) failed", device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    int max_points = collide_max_points(smem_optin);
    if ((double)(cfg->max_T + 1) * cfg->max_N * 24.0 > 64e9)
        return fail(nullptr, NPP_INVALID_ARG, "workspace for max_N x max_T too large");

    npp_handle* h = new npp_handle();
    h->cfg = *cfg;
    h->collide_variant = -1;
    h->fuse = -1;
    h->chunks = 0;
    h->last_chunks = 1;
    h->loop_restarts = 1;
    h->loop_sigma = 0.0f;
    h->collide_active = -1;
    h->occ_M = -1;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (h->sm_count < 1) h->sm_count = 1;
    h->device = device;
    h->n_theta = n_theta_of(cfg->width);
    h->max_points = max_points;
    h->dc = devcfg_from(*cfg);

    const size_t NT1 = (size_t)(cfg->max_T + 1) * cfg->max_N;
    const size_t NT = (size_t)cfg->max_T * cfg->max_N;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16); };
    A((void**)&h->d_key, 64);
    A((void**)&h->d_traj, NT1 * sizeof(float4));
    A((void**)&h->d_ctrl, NT * sizeof(float2));
    A((void**)&h->d_jfree, (size_t)cfg->max_N * sizeof(float));
    if (cfg->v_limits) A((void**)&h->d_vfirst, (size_t)cfg->max_N * sizeof(int));
    A((void**)&h->d_work, 64);
    A((void**)&h->d_counts, 64);
    A((void**)&h->d_fault, sizeof(unsigned));
    A((void**)&h->d_live, (size_t)2 * cfg->max_N * sizeof(int));
    A((void**)&h->d_live_n, NPP_MAX_CHUNKS * sizeof(int));
    A((void**)&h->d_carry, (size_t)cfg->max_N * sizeof(float4));
    A(&h->d_bins, binned_workspace_bytes(cfg->max_T, cfg->max_M));
    if (cfg->max_M > max_points) {
        A((void**)&h->d_pXY, (size_t)64 * pair_blocks(cfg->max_M) * sizeof(float4));
    }
    A((void**)&h->d_obs, (size_t)cfg->max_M * sizeof(float4));
    A((void**)&h->d_warm, (size_t)h->n_theta * sizeof(float));
    A((void**)&h->d_sigma, (size_t)h->n_theta * sizeof(float));
    A((void**)&h->d_best, sizeof(npp_best));
    A((void**)&h->d_params, (size_t)h->n_theta * sizeof(float));
    A((void**)&h->d_controls, (size_t)cfg->max_T * 2 * sizeof(float));
    A((void**)&h->d_trajectory, (size_t)(cfg->max_T + 1) * 4 * sizeof(float));
    A((void**)&h->d_costs, (size_t)cfg->max_N * sizeof(float));
    A((void**)&h->d_fh, (size_t)cfg->max_N * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(h->d_fault, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev[i]);
    for (int i = 0; i < NPP_CHUNK_EVENTS && e == cudaSuccess; ++i) e = cudaEventCreate(&h->cev[i]);
    if (e != cudaSuccess) {
        g_err = std::string("workspace allocation failed: ") + cudaGetErrorString(e);
        npp_destroy(h);
        return NPP_CUDA_ERROR;
    }
    *out = h;
    return NPP_OK;
}

npp_status npp_destroy(npp_handle* h)
{
    if (!h) return NPP_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    void* ptrs[] = { h->d_key, h->d_traj, h->d_ctrl, h->d_jfree, h->d_vfirst, h->d_fp, h->d_work, h->d_counts,
                     h->d_live, h->d_live_n, h->d_carry,
                     h->d_pXY, h->d_fault, h->d_bins,
                     h->d_obs, h->d_warm, h->d_sigma, h->d_best, h->d_params, h->d_controls, h->d_trajectory,
                     h->d_costs, h->d_fh };
    for (void* p : ptrs) if (p) cudaFree(p);
    if (h->stream) cudaStreamDestroy(h->stream);
    if (h->side) { cudaStreamSynchronize(h->side); cudaStreamDestroy(h->side); }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    for (int i = 0; i < 4; ++i) if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    for (int i = 0; i < NPP_CHUNK_EVENTS; ++i) if (h->cev[i]) cudaEventDestroy(h->cev[i]);
    delete h;
    return NPP_OK;
}

static npp_status plan_step_impl(npp_handle* h, const npp_state* state, const npp_goal* goal,
                                 const float* obs_dev, int32_t M, int32_t N, int32_t T, uint64_t seed,
                                 uint32_t t_index, const float* warm_dev, const Proposal& prop,
                                 const npp_outputs* out, void* stream)
{
    npp_status st;
    if ((st = check_state_goal(h, state, goal)) != NPP_OK) return st;
    if ((st = check_sizes(h, M, N, T, obs_dev, true)) != NPP_OK) return st;
    if (!out || !out->best) return fail(h, NPP_INVALID_ARG, "outputs.best must not be NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(h, cudaSetDevice(h->device));

    RolloutArgs a;
    fill_rollout_args(h, a, state, goal, obs_dev, M, N, T);
    a.key = make_key(seed, t_index, 0u);
    a.warm = warm_dev;
    a.prop = prop;
    a.costs = out->costs;
    a.first_hit = out->first_hit;
    a.traj = out->sample_traj ? reinterpret_cast<float4*>(out->sample_traj) : h->d_traj;
    a.ctrl = out->sample_ctrl ? reinterpret_cast<float2*>(out->sample_ctrl) : h->d_ctrl;
    a.jfree = h->d_jfree;
    a.best_key = h->d_key;
    CUDA_TRY(h, cudaMemsetAsync(h->d_key, 0xff, sizeof(unsigned long long), s));
    const bool records = out->sample_traj != nullptr || out->sample_ctrl != nullptr;
    if ((st = run_rollout(h, a, s, !records)) != NPP_OK) return st;

    EpilogueArgs e;
    memset(&e, 0, sizeof e);
    e.x0 = state->x; e.y0 = state->y; e.phi0 = state->phi;
    e.N = N; e.T = T; e.n_theta = h->n_theta;
    e.key = a.key;
    e.warm = warm_dev;
    e.prop = prop;
    e.traj = a.traj;
    e.ctrl = a.ctrl;
    e.best_key = h->d_key;
    e.fault = h->d_fault;
    e.best = out->best;
    e.params = out->params;
    e.controls = out->controls;
    e.trajectory = out->trajectory;
    CUDA_TRY(h, launch_epilogue(e, s));
    if (h->timing) CUDA_TRY(h, record_event(h->ev[3], s));
    return NPP_OK;
}

npp_status npp_plan_step(npp_handle* h, const npp_state* state, const npp_goal* goal,
                         const float* obs_dev, int32_t M, int32_t N, int32_t T, uint64_t seed,
                         uint32_t t_index, const float* warm_dev, const npp_outputs* out,
                         void* stream)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    return plan_step_impl(h, state, goal, obs_dev, M, N, T, seed, t_index, warm_dev,
                          Proposal{ nullptr, nullptr, 0, 1u }, out, stream);
}

npp_status npp_plan_step_proposal(npp_handle* h, const npp_state* state, const npp_goal* goal,
                                  const float* obs_dev, int32_t M, int32_t N, int32_t T, uint64_t seed,
                                  uint32_t t_index, const float* warm_dev, const float* mean_dev,
                                  const float* std_dev, int32_t N_prop, const npp_outputs* out,
                                  void* stream)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    if (N_prop < 0 || N_prop > N) return fail(h, NPP_INVALID_ARG, "N_prop=%d outside [0, N=%d]", N_prop, N);
    if (N_prop > 0 && (!mean_dev || !std_dev))
        return fail(h, NPP_INVALID_ARG, "mean and std must not be NULL with N_prop > 0");
    return plan_step_impl(h, state, goal, obs_dev, M, N, T, seed, t_index, warm_dev,
                          Proposal{ N_prop > 0 ? mean_dev : nullptr, std_dev, N_prop, 1u }, out, stream);
}

__global__ void fill_kernel(float* p, int n, float v)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

npp_status npp_set_loop_restarts(npp_handle* h, int32_t n_restarts, float sigma_pert)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    if (n_restarts < 1 || n_restarts > 64) return fail(h, NPP_INVALID_ARG, "n_restarts=%d outside [1, 64]", n_restarts);
    if (n_restarts > 1 && (!(sigma_pert > 0.0f) || !std::isfinite(sigma_pert)))
        return fail(h, NPP_INVALID_ARG, "sigma_pert must be finite and > 0");
    h->loop_restarts = n_restarts;
    h->loop_sigma = n_restarts > 1 ? sigma_pert : 0.0f;
    return NPP_OK;
}

npp_status npp_plan_tshc(npp_handle* h, const npp_state* state, const npp_goal* goal, const float* obs_dev,
                         int32_t M, int32_t N, int32_t T, uint64_t seed, uint32_t t_index, const float* warm_dev,
                         int32_t n_restarts, float sigma_pert, const npp_outputs* out, void* stream)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    if (n_restarts < 1) return fail(h, NPP_INVALID_ARG, "n_restarts=%d must be >= 1", n_restarts);
    if (!(sigma_pert > 0.0f) || !std::isfinite(sigma_pert))
        return fail(h, NPP_INVALID_ARG, "sigma_pert must be finite and > 0");
    if (!out || !out->params) return fail(h, NPP_INVALID_ARG, "outputs.params must not be NULL (the running best)");
    npp_status st = plan_step_impl(h, state, goal, obs_dev, M, N, T, seed, t_index, warm_dev,
                                   Proposal{ nullptr, nullptr, 0, 1u }, out, stream);
    if (st != NPP_OK || n_restarts == 1) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    fill_kernel<<<(h->n_theta + 255) / 256, 256, 0, s>>>(h->d_sigma, h->n_theta, sigma_pert);
    CUDA_TRY(h, cudaGetLastError());
    for (int r = 1; r < n_restarts && st == NPP_OK; ++r)
        st = plan_step_impl(h, state, goal, obs_dev, M, N, T, seed, t_index, out->params,
                            Proposal{ out->params, h->d_sigma, N, (uint32_t)r }, out, stream);
    return st;
}

npp_status npp_plan_step_host(npp_handle* h, const npp_state* state, const npp_goal* goal,
                              const float* obs_host, int32_t M, int32_t N, int32_t T,
                              uint64_t seed, uint32_t t_index, const float* warm_host,
                              const npp_outputs* out_host)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    if (!out_host || !out_host->best) return fail(h, NPP_INVALID_ARG, "outputs.best must not be NULL");
    if (out_host->sample_traj || out_host->sample_ctrl)
        return fail(h, NPP_INVALID_ARG, "per-sample outputs are device-only");
    npp_status st;
    if ((st = check_state_goal(h, state, goal)) != NPP_OK) return st;
    if ((st = check_sizes(h, M, N, T, obs_host, false)) != NPP_OK) return st;
    CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    if (M > 0) CUDA_TRY(h, cudaMemcpyAsync(h->d_obs, obs_host, (size_t)M * 16, cudaMemcpyHostToDevice, s));
    if (warm_host)
        CUDA_TRY(h, cudaMemcpyAsync(h->d_warm, warm_host, (size_t)h->n_theta * 4, cudaMemcpyHostToDevice, s));
    npp_outputs d;
    memset(&d, 0, sizeof d);
    d.best = h->d_best;
    d.params = out_host->params ? h->d_params : nullptr;
    d.controls = out_host->controls ? h->d_controls : nullptr;
    d.trajectory = out_host->trajectory ? h->d_trajectory : nullptr;
    d.costs = out_host->costs ? h->d_costs : nullptr;
    d.first_hit = out_host->first_hit ? h->d_fh : nullptr;
    st = npp_plan_step(h, state, goal, reinterpret_cast<const float*>(h->d_obs), M, N, T, seed, t_index,
                       warm_host ? h->d_warm : nullptr, &d, s);
    if (st != NPP_OK) return st;
    CUDA_TRY(h, cudaMemcpyAsync(out_host->best, h->d_best, sizeof(npp_best), cudaMemcpyDeviceToHost, s));
    if (out_host->params)
        CUDA_TRY(h, cudaMemcpyAsync(out_host->params, h->d_params, (size_t)h->n_theta * 4, cudaMemcpyDeviceToHost, s));
    if (out_host->controls)
        CUDA_TRY(h, cudaMemcpyAsync(out_host->controls, h->d_controls, (size_t)T * 8, cudaMemcpyDeviceToHost, s));
    if (out_host->trajectory)
        CUDA_TRY(h, cudaMemcpyAsync(out_host->trajectory, h->d_trajectory, (size_t)(T + 1) * 16, cudaMemcpyDeviceToHost, s));
    if (out_host->costs)
        CUDA_TRY(h, cudaMemcpyAsync(out_host->costs, h->d_costs, (size_t)N * 4, cudaMemcpyDeviceToHost, s));
    if (out_host->first_hit)
        CUDA_TRY(h, cudaMemcpyAsync(out_host->first_hit, h->d_fh, (size_t)N * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    const int32_t st_best = out_host->best->status;
    return st_best == NPP_INFEASIBLE || st_best == NPP_DEVICE_TIMEOUT ? (npp_status)st_best : NPP_OK;
}

npp_status npp_rollout_params(npp_handle* h, const npp_state* state, const npp_goal* goal,
                              const float* obs_dev, int32_t M, const float* theta_dev, int32_t K,
                              int32_t T, float* costs_dev, int32_t* first_hit_dev,
                              float* sample_traj_dev, float* sample_ctrl_dev, void* stream)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    npp_status st;
    if ((st = check_state_goal(h, state, goal)) != NPP_OK) return st;
    if ((st = check_sizes(h, M, K, T, obs_dev, true)) != NPP_OK) return st;
    if (!theta_dev) return fail(h, NPP_INVALID_ARG, "theta must not be NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(h, cudaSetDevice(h->device));
    RolloutArgs a;
    fill_rollout_args(h, a, state, goal, obs_dev, M, K, T);
    a.theta = theta_dev;
    a.costs = costs_dev;
    a.first_hit = first_hit_dev;
    a.traj = sample_traj_dev ? reinterpret_cast<float4*>(sample_traj_dev) : h->d_traj;
    a.ctrl = sample_ctrl_dev ? reinterpret_cast<float2*>(sample_ctrl_dev) : h->d_ctrl;
    a.jfree = h->d_jfree;
    a.best_key = nullptr;
    if ((st = run_rollout(h, a, s, !sample_traj_dev && !sample_ctrl_dev)) != NPP_OK) return st;
    if (h->timing) CUDA_TRY(h, record_event(h->ev[3], s));
    return NPP_OK;
}

npp_status npp_set_footprint(npp_handle* h, const float* verts_host, const int32_t* piece_start_host,
                             int32_t n_pieces)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    if (n_pieces < 0 || n_pieces > FP_MAX_PIECES)
        return fail(h, NPP_INVALID_ARG, "n_pieces is 0..%d", FP_MAX_PIECES);
    if (n_pieces == 0) {
        h->fp_faces = 0;
        return NPP_OK;
    }
    if (!verts_host || !piece_start_host) return fail(h, NPP_INVALID_ARG, "vertices and piece starts required");
    if (piece_start_host[0] != 0) return fail(h, NPP_INVALID_ARG, "piece_start[0] must be 0");
    const int nv = piece_start_host[n_pieces];
    if (nv > FP_MAX_FACES) return fail(h, NPP_INVALID_ARG, "at most %d vertices in total", FP_MAX_FACES);
    float4 faces[FP_MAX_FACES];
    double radius = 0.0;
    const double TWO_PI = 6.283185307179586;
    for (int k = 0; k < n_pieces; ++k) {
        const int b = piece_start_host[k], e = piece_start_host[k + 1], n = e - b;
        if (n < 3 || b < 0 || e > nv) return fail(h, NPP_INVALID_ARG, "piece %d needs >= 3 vertices", k);
        double turn = 0.0;
        for (int i = 0; i < n; ++i) {
            const float* v0 = verts_host + 2 * (b + i);
            const float* v1 = verts_host + 2 * (b + (i + 1) % n);
            const float* v2 = verts_host + 2 * (b + (i + 2) % n);
            if (!std::isfinite(v0[0]) || !std::isfinite(v0[1]))
                return fail(h, NPP_INVALID_ARG, "non-finite vertex in piece %d", k);
            const double ax = (double)v1[0] - v0[0], ay = (double)v1[1] - v0[1];
            const double bx = (double)v2[0] - v1[0], by = (double)v2[1] - v1[1];
            const double cr = ax * by - ay * bx;
            if (!(cr > 0.0))
                return fail(h, NPP_INVALID_ARG, "piece %d is not strictly convex and counter-clockwise", k);
            turn += std::atan2(cr, ax * bx + ay * by);
            const double len = std::sqrt(ax * ax + ay * ay);
            // outward unit normal of edge v0 -> v1 and its offset
            const double nx = ay / len, ny = -ax / len;
            faces[b + i] = make_float4((float)nx, (float)ny, (float)(nx * v0[0] + ny * v0[1]),
                                       i == n - 1 ? 1.0f : 0.0f);
            radius = std::fmax(radius, std::sqrt((double)v0[0] * v0[0] + (double)v0[1] * v0[1]));
        }
        if (std::fabs(turn - TWO_PI) > 1e-6)
            return fail(h, NPP_INVALID_ARG, "piece %d winds more than once", k);
    }
    CUDA_TRY(h, cudaSetDevice(h->device));
    if (!h->d_fp) CUDA_TRY(h, cudaMalloc((void**)&h->d_fp, sizeof(float4) * FP_MAX_FACES));
    CUDA_TRY(h, cudaMemcpy(h->d_fp, faces, sizeof(float4) * nv, cudaMemcpyHostToDevice));
    h->fp_faces = nv;
    h->fp_radius = radius;
    return NPP_OK;
}

npp_status npp_set_option(npp_handle* h, const char* name, int32_t value)
{
    if (!h || !name) return fail(h, NPP_INVALID_ARG, "handle and name must not be NULL");
    if (std::strcmp(name, "collide_variant") == 0) {
        if (value < -1 || value > COLLIDE_BINNED)
            return fail(h, NPP_INVALID_ARG, "collide_variant is -1..%d", COLLIDE_BINNED);
        h->collide_variant = value;
        h->occ_M = -1;
        return NPP_OK;
    }
    if (std::strcmp(name, "fuse") == 0) {
        if (value < -1 || value > 1) return fail(h, NPP_INVALID_ARG, "fuse is -1, 0 or 1");
        h->fuse = value;
        return NPP_OK;
    }
    if (std::strcmp(name, "chunks") == 0) {
        if (value < 0 || value > NPP_MAX_CHUNKS) return fail(h, NPP_INVALID_ARG, "chunks is 0..%d", NPP_MAX_CHUNKS);
        h->chunks = value;
        return NPP_OK;
    }
    if (std::strcmp(name, "traj_variant") == 0) {
        if (value < 0 || value > 4) return fail(h, NPP_INVALID_ARG, "traj_variant is 0..4");
        h->traj_variant = value;
        return NPP_OK;
    }
    return fail(h, NPP_INVALID_ARG, "unknown option '%s'", name);
}

npp_status npp_inject_fault(npp_handle* h)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    CUDA_TRY(h, cudaSetDevice(h->device));
    const unsigned one = 1u;
    CUDA_TRY(h, cudaMemcpy(h->d_fault, &one, sizeof one, cudaMemcpyHostToDevice));
    return NPP_OK;
}

npp_status npp_set_timing(npp_handle* h, int32_t enable)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    h->timing = enable != 0;
    return NPP_OK;
}

npp_status npp_last_counts(npp_handle* h, uint64_t* counts, int32_t n)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    if (!h->timing) return fail(h, NPP_INVALID_ARG, "timing is not enabled on this handle");
    if (!counts || n < 1) return fail(h, NPP_INVALID_ARG, "counts must hold n >= 1 values");
    CUDA_TRY(h, cudaSetDevice(h->device));
    CUDA_TRY(h, cudaDeviceSynchronize());
    unsigned long long c[3] = { 0ull, 0ull, 0ull };
    CUDA_TRY(h, cudaMemcpy(c, h->d_counts, sizeof c, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n && i < 3; ++i) counts[i] = c[i];
    return NPP_OK;
}

npp_status npp_last_timing(npp_handle* h, float* stage_ms, int32_t n)
{
    if (!h) return fail(nullptr, NPP_INVALID_ARG, "handle is NULL");
    if (!h->timing) return fail(h, NPP_INVALID_ARG, "timing is not enabled on this handle");
    if (!stage_ms || n < 1) return fail(h, NPP_INVALID_ARG, "stage_ms must hold n >= 1 values");
    CUDA_TRY(h, cudaSetDevice(h->device));
    CUDA_TRY(h, cudaEventSynchronize(h->ev[3]));
    float t[4] = { 0.f, 0.f, 0.f, 0.f };
    CUDA_TRY(h, stage_times(h->ev, h->cev, h->last_chunks, t));
    for (int i = 0; i < n && i < 4; ++i) stage_ms[i] = t[i];
    return NPP_OK;
}


npp_status npp_sample_params(uint64_t seed, uint32_t t_index, uint32_t stream_id, int32_t n0,
                             int32_t K, int32_t n_theta, float* out_dev, void* stream)
{
    if (n0 < 0 || K < 1 || n_theta < 1 || !out_dev)
        return fail(nullptr, NPP_INVALID_ARG, "npp_sample_params: bad arguments");
    const long long quads = (long long)K * ((n_theta + 3) / 4);
    const int grid = (int)std::min<long long>((quads + 255) / 256, 65536);
    sample_params_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        make_key(seed, t_index, stream_id), n0, K, n_theta, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, NPP_CUDA_ERROR, "sampler launch: %s", cudaGetErrorString(e));
    return NPP_OK;
}

npp_status npp_math_eval(int32_t fn, const float* x_dev, int32_t n, float* y_dev, float* y2_dev,
                         void* stream)
{
    if (fn < 0 || fn > 2 || n < 0 || (n > 0 && (!x_dev || !y_dev || (fn == 2 && !y2_dev))))
        return fail(nullptr, NPP_INVALID_ARG, "npp_math_eval: bad arguments");
    if (n == 0) return NPP_OK;
    const int grid = std::min((n + 255) / 256, 4096);
    math_eval_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(fn, x_dev, n, y_dev, y2_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, NPP_CUDA_ERROR, "math_eval launch: %s", cudaGetErrorString(e));
    return NPP_OK;
}

}  // extern "C"
