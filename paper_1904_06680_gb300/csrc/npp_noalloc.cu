// npp_noalloc.cu -- a plan step that allocates no memory.
//
// Some callers cannot call cudaMalloc: a plugin whose host application owns
// every device allocation, or a real-time control loop that must not
// allocate once it runs, because cudaMalloc may synchronise the device and
// take unbounded time.  npp_plan_step_noalloc serves them: it runs the
// trajectory kernel and the winner epilogue of npp_plan_step, with one
// collision check -- the brute-force check with the points held in shared
// memory (items of 8 samples on 4 or 2 point slices) -- whatever M and N
// are.  It never uses the spatial binning that npp_plan_step picks for many
// points, so M is limited to the points shared memory holds (about 14,000
// with the 227 KB of a GB300 block) and a large M * N runs slower than
// through a handle.  Every collision check gives the same flags, so the
// results equal npp_plan_step's.  Its workspace is one file-scope
// __device__ array of fixed size instead of handle-owned cudaMalloc buffers.
//
// The array (NOALLOC_BYTES, about 17 MB) exists on every GPU on which this
// library's module is loaded, until the process exits.  All calls share it,
// so calls that overlap on the GPU (on different streams, or from different
// threads) race; each call clears the parts that must start at zero.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_device.cuh"

using namespace npp;

namespace {

// capacity: N <= NOALLOC_MAX_N samples and N * (T + 1) <= NOALLOC_MAX_STEPS
constexpr int NOALLOC_MAX_N = 16384;
constexpr long long NOALLOC_MAX_STEPS = 16384LL * 42;     // 688,128 sample-steps
// layout: [key, work counter | pad to 256] [cost if free, N floats]
//         [first speed-violating step, N ints] [states float4] [controls float2]
constexpr size_t OFF_JFREE = 256;
constexpr size_t OFF_VFIRST = OFF_JFREE + (size_t)NOALLOC_MAX_N * 4;
constexpr size_t OFF_TRAJ = OFF_VFIRST + (size_t)NOALLOC_MAX_N * 4;
constexpr size_t OFF_CTRL = OFF_TRAJ + (size_t)NOALLOC_MAX_STEPS * 16;
constexpr size_t NOALLOC_BYTES = OFF_CTRL + (size_t)NOALLOC_MAX_STEPS * 8;

static __device__ __align__(256) unsigned char g_scratch[NOALLOC_BYTES];

// host-side device address of g_scratch per device (the symbol itself names
// a host stand-in; only cudaGetSymbolAddress yields the device address)
constexpr int MAX_DEVICES = 64;
static unsigned char* g_scratch_dev[MAX_DEVICES];

npp_status fail_noalloc(npp_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_global_error(buf);
    return s;
}

bool finite_n(const float* p, int n)
{
    for (int i = 0; i < n; ++i) if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

extern "C" npp_status npp_plan_step_noalloc(const npp_config* cfg, const npp_state* state,
                                            const npp_goal* goal, const float* obs_dev, int32_t M,
                                            int32_t N, int32_t T, uint64_t seed, uint32_t t_index,
                                            const float* warm_dev, const npp_outputs* out,
                                            void* stream)
{
    if (!cfg || !state || !goal || !out || !out->best)
        return fail_noalloc(NPP_INVALID_ARG, "noalloc: cfg, state, goal and outputs.best must not be NULL");
    if (cfg->n_in != 8 || (cfg->width != 16 && cfg->width != 32 && cfg->width != 64))
        return fail_noalloc(NPP_UNSUPPORTED, "noalloc: network [%d, %d, %d, 2] is not built",
                            cfg->n_in, cfg->width, cfg->width);
    // the same checks as npp_create
    if (const char* ce = config_error(*cfg)) return fail_noalloc(NPP_INVALID_ARG, "noalloc: %s", ce);
    if (!finite_n(&state->x, 6) || !finite_n(&goal->x, 4) ||
        std::fabs(state->a_prev0) > 1.0f || std::fabs(state->a_prev1) > 1.0f)
        return fail_noalloc(NPP_INVALID_ARG, "noalloc: non-finite state/goal or |a_prev| > 1");
    if (N < 1 || N > NOALLOC_MAX_N)
        return fail_noalloc(NPP_INVALID_ARG, "noalloc: N=%d outside [1, %d]", N, NOALLOC_MAX_N);
    if (T < 1 || (long long)N * (T + 1) > NOALLOC_MAX_STEPS)
        return fail_noalloc(NPP_INVALID_ARG,
                            "noalloc: N*(T+1)=%lld exceeds the %lld sample-steps of the static workspace",
                            (long long)N * (T + 1), NOALLOC_MAX_STEPS);
    if (M < 0 || (M > 0 && !obs_dev) || (obs_dev && (reinterpret_cast<uintptr_t>(obs_dev) & 15u)))
        return fail_noalloc(NPP_INVALID_ARG, "noalloc: bad obstacle array (M=%d)", M);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return fail_noalloc(NPP_CUDA_ERROR, "noalloc: no current CUDA device");
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (M > collide_max_points(smem_optin))
        return fail_noalloc(NPP_UNSUPPORTED, "noalloc: M=%d exceeds the %d points held in shared memory",
                            M, collide_max_points(smem_optin));
    // set-up, once per device, with that device current
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail_noalloc(NPP_CUDA_ERROR, "noalloc: cudaGetSymbolAddress failed: %s",
                                cudaGetErrorString(e));
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    unsigned char* base = g_scratch_dev[dev];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    const DevCfg d = devcfg_from(*cfg);

    RolloutArgs a;
    memset(&a, 0, sizeof a);
    a.c = d;
    a.x0 = state->x; a.y0 = state->y; a.phi0 = state->phi; a.v0 = state->v;
    a.ap0 = state->a_prev0; a.ap1 = state->a_prev1;
    a.gx = goal->x; a.gy = goal->y; a.gphi = goal->phi; a.gv = goal->v;
    a.obs = reinterpret_cast<const float4*>(obs_dev);
    a.M = M; a.N = N; a.T = T;
    a.key.k0 = (uint32_t)(seed & 0xffffffffu);
    a.key.k1 = (uint32_t)(seed >> 32);
    a.key.t_index = t_index;
    a.key.stream_id = 0u;
    a.warm = warm_dev;
    a.costs = out->costs;
    a.first_hit = out->first_hit;
    a.traj = out->sample_traj ? reinterpret_cast<float4*>(out->sample_traj)
                              : reinterpret_cast<float4*>(base + OFF_TRAJ);
    a.ctrl = out->sample_ctrl ? reinterpret_cast<float2*>(out->sample_ctrl)
                              : reinterpret_cast<float2*>(base + OFF_CTRL);
    a.jfree = reinterpret_cast<float*>(base + OFF_JFREE);
    a.vfirst = cfg->v_limits ? reinterpret_cast<int*>(base + OFF_VFIRST) : nullptr;
    a.coefA = nullptr;                   // the collision kernels recompute the rows from the states
    a.coefB = nullptr;
    a.best_key = reinterpret_cast<unsigned long long*>(base);
    a.work = reinterpret_cast<unsigned*>(base + 8);
    a.fault = reinterpret_cast<unsigned*>(base + 12);
    int sm_count = 1;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    const int variant = N <= 8192 ? 3 : 4;
    a.grid_collide = (sm_count > 0 ? sm_count : 1) * collide_resident_blocks_per_sm(M, variant);

    // the best key starts at all ones, the work counter and fault flag at zero
    e = cudaMemsetAsync(base, 0xff, 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + 8, 0, 8, s);
    if (e == cudaSuccess) {
        switch (cfg->width) {
        case 16: e = launch_traj_w16(a, s, 0); break;
        case 32: e = launch_traj_w32(a, s, 0); break;
        default: e = launch_traj_w64(a, s, 0); break;
        }
    }
    if (e == cudaSuccess) e = launch_collide_resident(a, s, variant);
    if (e == cudaSuccess) {
        EpilogueArgs ep;
        memset(&ep, 0, sizeof ep);
        ep.x0 = state->x; ep.y0 = state->y; ep.phi0 = state->phi;
        ep.N = N; ep.T = T; ep.n_theta = 12 * cfg->width + cfg->width * cfg->width + 2;
        ep.key = a.key;
        ep.warm = warm_dev;
        ep.traj = a.traj;
        ep.ctrl = a.ctrl;
        ep.best_key = a.best_key;
        ep.fault = a.fault;
        ep.best = out->best;
        ep.params = out->params;
        ep.controls = out->controls;
        ep.trajectory = out->trajectory;
        e = launch_epilogue(ep, s);
    }
    if (e != cudaSuccess)
        return fail_noalloc(NPP_CUDA_ERROR, "noalloc: launch failed: %s", cudaGetErrorString(e));
    return NPP_OK;
}
