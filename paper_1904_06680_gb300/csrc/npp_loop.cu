// npp_loop.cu -- the closed-loop control algorithm (Alg. 1 of the paper) run
// on the device: one CUDA graph per sampling time holds the plan step
// (Step 5) and an advance kernel that applies the winner's first control to
// the simulated vehicle (Step 6), moves the obstacle points, switches to the
// next waypoint once the current one is reached within the tolerances of
// Table hyperparameters (Steps 4 and 7) and keeps the winner's parameters as
// the next warm start (Sect. II-D "Fifth").  With restarts set on the handle
// (npp_set_loop_restarts) the plan step of every sampling time is the hill
// climb of Sect. II-D: after the first round, each further round samples
// theta = theta_best + sigma_pert eps around the best so far (kept as sample
// 0), as npp_plan_tshc does.  The host only replays the graph.
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_device.cuh"
#include "npp_internal.h"

using namespace npp;

// loop entry points report errors on their handle and in npp_last_error(NULL)
#define LOOP_TRY(h, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            npp_status s_ = fail((h), NPP_CUDA_ERROR, "%s failed: %s", #call,               \
                                 cudaGetErrorString(e_));                                   \
            set_global_error(npp_last_error(h));                                            \
            return s_;                                                                      \
        }                                                                                   \
    } while (0)

struct npp_loop {
    npp_handle* h;
    int M, N, T, n_wp, max_log;
    LoopDev* d_dyn;
    float4* d_wp;            // [n_wp] waypoints
    float4* d_obs0;          // [M] obstacle points at the start (world frame)
    float4* d_obs;           // [M] obstacle points at the current sampling time
    float* d_warm;           // [n_theta] warm start = winner of the last step
    npp_best* d_best;
    float* d_controls;       // [T][2]
    float* d_trajectory;     // [T+1][4]
    float* d_log;            // [max_log][8]
    float* d_costs;          // [N] per-sample costs of the last step
    int32_t* d_fh;           // [N] per-sample first collisions of the last step
    int restarts;            // hill-climb rounds per sampling time (1: the plan step alone)
    float* d_sigma;          // [n_theta] their perturbation scale
    cudaEvent_t ev[4];       // captured: start, after trajectories, after collisions, end
    cudaEvent_t cev[NPP_CHUNK_EVENTS];  // captured chunk stage events (plan step in chunks)
    int nch;                 // chunks of the captured plan step
    cudaStream_t cap;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

// where points outside the range field are parked (world frame, at rest):
// farther from any vehicle pose than a plan step can reach
constexpr float HIDDEN_POINT = 1.0e7f;

struct PlantCfg {
    double lf, lr, delta_max, u_min, u_max, Ts;
};

// ---- mission layer (Alg. 1 Steps 3, 4, 7; Sect. II-B to II-D), FP64 on the
// simulated vehicle's pose.  Readings: setpoints with v = 0 and the last
// one are stop setpoints that must be reached within eps before the path
// beyond them is used (the last one completes the mission); the space index
// is the setpoint closest to the vehicle among idx .. min(idx + window,
// stop), ties to the lowest; the goal is the furthest setpoint from the
// space index on, up to the stop, with it and all before it within or on the
// range field xi in [-back, front], |eta| <= side (EV frame at t).

// (xi, eta) of a world point in the vehicle's frame
__device__ __forceinline__ void ev_of(const LoopDev* d, double px, double py, double& xi, double& eta)
{
    const double c = cos(d->pphi), s = sin(d->pphi);
    const double dx = px - d->px, dy = py - d->py;
    xi = c * dx + s * dy;
    eta = -s * dx + c * dy;
}

__device__ __forceinline__ bool in_field(const LoopDev* d, double px, double py)
{
    double xi, eta;
    ev_of(d, px, py, xi, eta);
    return -(double)d->field[1] <= xi && xi <= (double)d->field[0] && fabs(eta) <= (double)d->field[2];
}

__device__ __forceinline__ bool is_stop(const float4* ref, int n, int k) { return k == n - 1 || ref[k].w == 0.0f; }

__device__ __forceinline__ int next_stop(const float4* ref, int n, int k)
{
    while (!is_stop(ref, n, k)) ++k;
    return k;
}

// the tolerances of Table hyperparameters at the vehicle's pose and speed
__device__ __forceinline__ bool reached(const LoopDev* d, const float4 g)
{
    double dxi, deta;
    ev_of(d, g.x, g.y, dxi, deta);
    const double dphi = remainder((double)g.z - d->pphi, 2.0 * M_PI);
    return fabs(dxi) <= d->eps[0] && fabs(deta) <= d->eps[1] && fabs(dphi) <= d->eps[2] &&
           fabs((double)g.w - d->pv) <= d->eps[3];
}

__device__ void select_goal(LoopDev* d, const float4* ref)
{
    int k = d->idx;
    if (in_field(d, ref[k].x, ref[k].y))
        while (k + 1 <= d->stop && in_field(d, ref[k + 1].x, ref[k + 1].y)) ++k;
    d->goal_k = k;
}

// Step 7 (stop setpoints, completion) and Steps 3-4 (space index, goal) at
// the vehicle's current pose
__device__ void mission_update(LoopDev* d, const float4* ref)
{
    if (d->done) return;
    const int n = d->n_wp;
    int best = d->idx;
    double bd = INFINITY;
    const int last = min(d->idx + d->window, d->stop);
    for (int k = d->idx; k <= last; ++k) {
        const double dd = hypot((double)ref[k].x - d->px, (double)ref[k].y - d->py);
        if (dd < bd) { best = k; bd = dd; }
    }
    d->idx = best;
    if (reached(d, ref[d->stop])) {
        if (d->stop == n - 1) {
            d->done = 1;
        } else {
            d->idx = d->stop;
            d->stop = next_stop(ref, n, d->stop + 1);
        }
    }
    select_goal(d, ref);
}

// mission start: first stop, goal at the initial pose
__global__ void mission_init_kernel(LoopDev* d, const float4* __restrict__ ref)
{
    d->idx = 0;
    d->stop = next_stop(ref, d->n_wp, 0);
    select_goal(d, ref);
    const float4 g = ref[d->goal_k];
    d->gx = g.x; d->gy = g.y; d->gphi = g.z; d->gv = g.w;
}

// Obstacle points at the current sampling time t (the state kernel has
// advanced t): p0 + tau v, tau = t Ts; with hide, points outside the range
// field at t are moved far away (at rest), so no plan step sees them.
__global__ void advance_obstacles_kernel(const LoopDev* d, const float4* __restrict__ obs0,
                                         float4* __restrict__ obs, int M, float Ts)
{
    const float tau = (float)d->t * Ts;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const float4 o = obs0[j];
        const float px = fmaf(tau, o.z, o.x), py = fmaf(tau, o.w, o.y);
        if (d->hide && !in_field(d, px, py)) obs[j] = make_float4(HIDDEN_POINT, HIDDEN_POINT, 0.0f, 0.0f);
        else obs[j] = make_float4(px, py, o.z, o.w);
    }
}

// Steps 6 and 7 of Alg. 1: one sampling time of the simulated vehicle (the
// kinematic bicycle of Sect. IV, FP64, explicit Euler on the old state) under
// the winner's first applied control; waypoint switch or mission update;
// log row (x, y, phi, v, a0, a1, best cost, goal index).  One thread.
__global__ void advance_state_kernel(LoopDev* d, const float* __restrict__ controls,
                                     const npp_best* __restrict__ best, const float4* __restrict__ wps,
                                     float* __restrict__ log, int max_log, PlantCfg pc)
{
    const double a0 = controls[0], a1 = controls[1];
    d->status = best->status;
    d->best_idx = best->best_idx;
    d->best_cost = best->best_cost;
    if (best->status == NPP_INFEASIBLE) d->n_infeasible += 1;
    if (d->t < max_log) {
        float* row = log + 8 * d->t;
        row[0] = (float)d->px; row[1] = (float)d->py; row[2] = (float)d->pphi; row[3] = (float)d->pv;
        row[4] = (float)a0; row[5] = (float)a1; row[6] = best->best_cost;
        row[7] = (float)(d->mission ? d->goal_k : d->waypoint);
    }
    const double L = pc.lf + pc.lr;
    const double delta = pc.delta_max * a0;
    const double u = pc.u_min + 0.5 * (a1 + 1.0) * (pc.u_max - pc.u_min);
    const double beta = atan(pc.lr * tan(delta) / L);
    const double x = d->px, y = d->py, ph = d->pphi, v = d->pv;
    d->px = x + pc.Ts * v * cos(ph + beta) / cos(beta);
    d->py = y + pc.Ts * v * sin(ph + beta) / cos(beta);
    d->pphi = ph + pc.Ts * v * tan(delta) / L;
    d->pv = v + pc.Ts * u;
    d->t += 1;
    d->t_index += 1;
    if (d->mission) {
        mission_update(d, wps);
        const float4 g = wps[d->goal_k];
        d->gx = g.x; d->gy = g.y; d->gphi = g.z; d->gv = g.w;
        d->x0 = (float)d->px; d->y0 = (float)d->py; d->phi0 = (float)d->pphi; d->v0 = (float)d->pv;
        d->ap0 = (float)a0; d->ap1 = (float)a1;
        d->warm_valid = 1;
        return;
    }
    // completion check against the current waypoint (Table hyperparameters)
    if (!d->done) {
        const float4 g = wps[d->waypoint];
        const double c = cos(d->pphi), s = sin(d->pphi);
        const double dx = g.x - d->px, dy = g.y - d->py;
        const double dxi = c * dx + s * dy, deta = -s * dx + c * dy;
        const double dphi = remainder((double)g.z - d->pphi, 2.0 * M_PI);
        if (fabs(dxi) <= d->eps[0] && fabs(deta) <= d->eps[1] && fabs(dphi) <= d->eps[2] &&
            fabs((double)g.w - d->pv) <= d->eps[3]) {
            if (d->waypoint + 1 < d->n_wp) d->waypoint += 1;
            else d->done = 1;
        }
    }
    const float4 g = wps[d->waypoint];
    d->gx = g.x; d->gy = g.y; d->gphi = g.z; d->gv = g.w;
    d->x0 = (float)d->px; d->y0 = (float)d->py; d->phi0 = (float)d->pphi; d->v0 = (float)d->pv;
    d->ap0 = (float)a0; d->ap1 = (float)a1;
    d->warm_valid = 1;
}

void free_loop(npp_loop* L)
{
    if (!L) return;
    if (L->exec) cudaGraphExecDestroy(L->exec);
    if (L->graph) cudaGraphDestroy(L->graph);
    if (L->cap) cudaStreamDestroy(L->cap);
    void* ptrs[] = { L->d_dyn, L->d_wp, L->d_obs0, L->d_obs, L->d_warm, L->d_best, L->d_controls,
                     L->d_trajectory, L->d_log, L->d_costs, L->d_fh, L->d_sigma };
    for (void* p : ptrs) if (p) cudaFree(p);
    for (int i = 0; i < 4; ++i) if (L->ev[i]) cudaEventDestroy(L->ev[i]);
    for (int i = 0; i < NPP_CHUNK_EVENTS; ++i) if (L->cev[i]) cudaEventDestroy(L->cev[i]);
    delete L;
}

// queue one sampling time on stream s (captured into the graph)
npp_status enqueue_step(npp_loop* L, uint64_t seed)
{
    npp_handle* h = L->h;
    cudaStream_t s = L->cap;
    RolloutArgs a;
    memset(&a, 0, sizeof a);
    a.c = h->dc;
    a.obs = L->d_obs;
    a.M = L->M; a.N = L->N; a.T = L->T;
    a.key.k0 = (uint32_t)(seed & 0xffffffffu);
    a.key.k1 = (uint32_t)(seed >> 32);
    a.key.stream_id = 0u;
    a.warm = L->d_warm;
    a.traj = h->d_traj;
    a.ctrl = h->d_ctrl;
    a.jfree = h->d_jfree;
    a.vfirst = h->d_vfirst;
    a.best_key = h->d_key;
    a.fault = h->d_fault;
    a.dyn = L->d_dyn;
    a.costs = L->d_costs;
    a.first_hit = L->d_fh;
    CUDA_TRY(h, cudaMemsetAsync(h->d_key, 0xff, sizeof(unsigned long long), s));
    npp_status st = run_rollout(h, a, s, true);
    if (st != NPP_OK) return st;
    EpilogueArgs e;
    memset(&e, 0, sizeof e);
    e.N = L->N; e.T = L->T; e.n_theta = h->n_theta;
    e.key = a.key;
    e.warm = L->d_warm;
    e.traj = a.traj;
    e.ctrl = a.ctrl;
    e.best_key = h->d_key;
    e.fault = h->d_fault;
    e.best = L->d_best;
    e.params = L->d_warm;
    e.controls = L->d_controls;
    e.trajectory = L->d_trajectory;
    e.dyn = L->d_dyn;
    CUDA_TRY(h, launch_epilogue(e, s));
    // restart rounds: the winner so far is sample 0 (warm start, valid even
    // at the loop's first step), every other sample a perturbation of it on
    // the round's own Philox stream; the winner's parameters, controls and
    // trajectory are overwritten by each round's (never worse) winner.  The
    // stage events time the first round; the end event the whole step.
    const bool timing = h->timing;
    h->timing = false;
    for (int r = 1; r < L->restarts; ++r) {
        RolloutArgs ar = a;
        ar.prop = Proposal{ L->d_warm, L->d_sigma, L->N, (uint32_t)r };
        ar.warm = L->d_warm;
        ar.warm_force = 1;
        CUDA_TRY(h, cudaMemsetAsync(h->d_key, 0xff, sizeof(unsigned long long), s));
        st = run_rollout(h, ar, s, true);
        if (st != NPP_OK) {
            h->timing = timing;
            return st;
        }
        EpilogueArgs er = e;
        er.prop = ar.prop;
        er.warm_force = 1;
        cudaError_t ce = launch_epilogue(er, s);
        if (ce != cudaSuccess) {
            h->timing = timing;
            return fail(h, NPP_CUDA_ERROR, "restart epilogue: %s", cudaGetErrorString(ce));
        }
    }
    h->timing = timing;
    PlantCfg pc;
    pc.lf = h->cfg.lf; pc.lr = h->cfg.lr; pc.delta_max = h->cfg.delta_max;
    pc.u_min = h->cfg.u_min; pc.u_max = h->cfg.u_max; pc.Ts = h->cfg.Ts;
    advance_state_kernel<<<1, 1, 0, s>>>(L->d_dyn, L->d_controls, L->d_best, L->d_wp, L->d_log,
                                         L->max_log, pc);
    CUDA_TRY(h, cudaGetLastError());
    if (L->M > 0) {
        advance_obstacles_kernel<<<(L->M + 255) / 256, 256, 0, s>>>(L->d_dyn, L->d_obs0, L->d_obs, L->M,
                                                                     (float)pc.Ts);
        CUDA_TRY(h, cudaGetLastError());
    }
    CUDA_TRY(h, record_event(L->ev[3], s));
    return NPP_OK;
}

npp_status loop_create(npp_handle* h, const npp_state* s0, const float* waypoints_host, int32_t n_wp,
                       const npp_mission* mission, const float* eps_host, const float* obs_dev, int32_t M,
                       int32_t N, int32_t T, uint64_t seed, int32_t max_log, npp_loop** out)
{
    if (!h || !out) return fail(h, NPP_INVALID_ARG, "handle and output pointer must not be NULL");
    *out = nullptr;
    if (!s0 || !waypoints_host || n_wp < 1 || !eps_host || max_log < 0)
        return fail(h, NPP_INVALID_ARG, "loop: state, waypoints (n_wp >= 1), eps and max_log >= 0 required");
    for (int i = 0; i < 4 * n_wp; ++i)
        if (!std::isfinite(waypoints_host[i])) return fail(h, NPP_INVALID_ARG, "loop: non-finite waypoint");
    const float* sv = &s0->x;
    for (int i = 0; i < 6; ++i) if (!std::isfinite(sv[i])) return fail(h, NPP_INVALID_ARG, "loop: non-finite state");
    if (std::fabs(s0->a_prev0) > 1.f || std::fabs(s0->a_prev1) > 1.f)
        return fail(h, NPP_INVALID_ARG, "loop: previous controls must lie in [-1, 1]");
    for (int i = 0; i < 4; ++i)
        if (!(eps_host[i] >= 0.f)) return fail(h, NPP_INVALID_ARG, "loop: tolerances must be >= 0");
    if (mission) {
        const float f[3] = { mission->range_front, mission->range_back, mission->range_side };
        for (int i = 0; i < 3; ++i)
            if (!(f[i] >= 0.f) || !std::isfinite(f[i]))
                return fail(h, NPP_INVALID_ARG, "mission: range field extents must be finite and >= 0");
        if (mission->window < 1 || (mission->hide_outside != 0 && mission->hide_outside != 1))
            return fail(h, NPP_INVALID_ARG, "mission: window >= 1 and hide_outside 0 or 1 required");
    }
    const npp_config& c = h->cfg;
    if (N < 1 || N > c.max_N || T < 1 || T > c.max_T || M < 0 || M > c.max_M)
        return fail(h, NPP_INVALID_ARG, "loop: N=%d T=%d M=%d outside the handle's capacity", N, T, M);
    if (M > 0 && (!obs_dev || (reinterpret_cast<uintptr_t>(obs_dev) & 15u)))
        return fail(h, NPP_INVALID_ARG, "loop: obstacle array NULL or not 16-byte aligned");
    CUDA_TRY(h, cudaSetDevice(h->device));

    npp_loop* L = new npp_loop();
    L->h = h; L->M = M; L->N = N; L->T = T; L->n_wp = n_wp; L->max_log = max_log;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16); };
    A((void**)&L->d_dyn, sizeof(LoopDev));
    A((void**)&L->d_wp, (size_t)n_wp * sizeof(float4));
    A((void**)&L->d_obs0, (size_t)(M > 0 ? M : 1) * sizeof(float4));
    A((void**)&L->d_obs, (size_t)(M > 0 ? M : 1) * sizeof(float4));
    A((void**)&L->d_warm, (size_t)h->n_theta * sizeof(float));
    A((void**)&L->d_best, sizeof(npp_best));
    A((void**)&L->d_controls, (size_t)T * 2 * sizeof(float));
    A((void**)&L->d_trajectory, (size_t)(T + 1) * 4 * sizeof(float));
    A((void**)&L->d_log, (size_t)(max_log > 0 ? max_log : 1) * 8 * sizeof(float));
    A((void**)&L->d_costs, (size_t)N * sizeof(float));
    A((void**)&L->d_fh, (size_t)N * sizeof(int32_t));
    L->restarts = h->loop_restarts;
    if (L->restarts > 1) A((void**)&L->d_sigma, (size_t)h->n_theta * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&L->ev[i]);
    for (int i = 0; i < NPP_CHUNK_EVENTS && e == cudaSuccess; ++i) e = cudaEventCreate(&L->cev[i]);
    if (e != cudaSuccess) {
        free_loop(L);
        return fail(h, NPP_CUDA_ERROR, "loop allocation failed: %s", cudaGetErrorString(e));
    }
    LoopDev d;
    memset(&d, 0, sizeof d);
    d.px = s0->x; d.py = s0->y; d.pphi = s0->phi; d.pv = s0->v;
    d.x0 = s0->x; d.y0 = s0->y; d.phi0 = s0->phi; d.v0 = s0->v; d.ap0 = s0->a_prev0; d.ap1 = s0->a_prev1;
    d.gx = waypoints_host[0]; d.gy = waypoints_host[1]; d.gphi = waypoints_host[2]; d.gv = waypoints_host[3];
    d.n_wp = n_wp;
    for (int i = 0; i < 4; ++i) d.eps[i] = eps_host[i];
    d.status = NPP_OK;
    if (mission) {
        d.mission = 1;
        d.window = mission->window;
        d.hide = mission->hide_outside;
        d.field[0] = mission->range_front;
        d.field[1] = mission->range_back;
        d.field[2] = mission->range_side;
    }
    e = cudaMemcpy(L->d_dyn, &d, sizeof d, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_wp, waypoints_host, (size_t)n_wp * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && M > 0) e = cudaMemcpy(L->d_obs0, obs_dev, (size_t)M * sizeof(float4), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && M > 0) e = cudaMemcpy(L->d_obs, obs_dev, (size_t)M * sizeof(float4), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && L->restarts > 1) {
        e = fill_floats(L->d_sigma, h->n_theta, h->loop_sigma, L->cap);
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->cap);
    }
    if (e == cudaSuccess && mission) {
        // the first goal and the points seen at t = 0
        mission_init_kernel<<<1, 1, 0, L->cap>>>(L->d_dyn, L->d_wp);
        e = cudaGetLastError();
        if (e == cudaSuccess && M > 0) {
            advance_obstacles_kernel<<<(M + 255) / 256, 256, 0, L->cap>>>(L->d_dyn, L->d_obs0, L->d_obs, M,
                                                                           (float)h->cfg.Ts);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->cap);
    }
    if (e != cudaSuccess) {
        free_loop(L);
        return fail(h, NPP_CUDA_ERROR, "loop set-up copy failed: %s", cudaGetErrorString(e));
    }
    // capture one sampling time; the kernels' launch shapes depend only on
    // N, T, M, which the loop fixes
    // the plan step records its stage events (the loop's own) into the graph
    const bool timing = h->timing;
    cudaEvent_t hev[4], hcev[NPP_CHUNK_EVENTS];
    for (int i = 0; i < 4; ++i) { hev[i] = h->ev[i]; h->ev[i] = L->ev[i]; }
    for (int i = 0; i < NPP_CHUNK_EVENTS; ++i) { hcev[i] = h->cev[i]; h->cev[i] = L->cev[i]; }
    const int h_last_chunks = h->last_chunks;
    h->timing = true;
    e = cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal);
    npp_status st = NPP_OK;
    if (e == cudaSuccess) st = enqueue_step(L, seed);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(L->cap, &g);
    h->timing = timing;
    L->nch = h->last_chunks;
    h->last_chunks = h_last_chunks;
    for (int i = 0; i < 4; ++i) h->ev[i] = hev[i];
    for (int i = 0; i < NPP_CHUNK_EVENTS; ++i) h->cev[i] = hcev[i];
    if (e != cudaSuccess || st != NPP_OK || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        free_loop(L);
        if (st != NPP_OK) return st;
        return fail(h, NPP_CUDA_ERROR, "loop graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    L->graph = g;
    e = cudaGraphInstantiate(&L->exec, g, 0);
    if (e != cudaSuccess) {
        free_loop(L);
        return fail(h, NPP_CUDA_ERROR, "loop graph instantiation failed: %s", cudaGetErrorString(e));
    }
    *out = L;
    return NPP_OK;
}

}  // namespace

extern "C" {

npp_status npp_loop_create(npp_handle* h, const npp_state* s0, const float* waypoints_host,
                           int32_t n_wp, const float* eps_host, const float* obs_dev, int32_t M,
                           int32_t N, int32_t T, uint64_t seed, int32_t max_log, npp_loop** out)
{
    return loop_create(h, s0, waypoints_host, n_wp, nullptr, eps_host, obs_dev, M, N, T, seed, max_log, out);
}

npp_status npp_loop_create_mission(npp_handle* h, const npp_state* s0, const float* ref_host, int32_t n_ref,
                                   const npp_mission* mission, const float* eps_host, const float* obs_dev,
                                   int32_t M, int32_t N, int32_t T, uint64_t seed, int32_t max_log,
                                   npp_loop** out)
{
    if (!mission) return fail(h, NPP_INVALID_ARG, "mission is NULL");
    return loop_create(h, s0, ref_host, n_ref, mission, eps_host, obs_dev, M, N, T, seed, max_log, out);
}

npp_status npp_loop_points(npp_loop* L, float* obs_host)
{
    if (!L || (!obs_host && L->M > 0)) return fail(L ? L->h : nullptr, NPP_INVALID_ARG, "loop: bad arguments");
    npp_handle* h = L->h;
    LOOP_TRY(h, cudaSetDevice(h->device));
    LOOP_TRY(h, cudaDeviceSynchronize());
    if (L->M > 0) LOOP_TRY(h, cudaMemcpy(obs_host, L->d_obs, (size_t)L->M * sizeof(float4), cudaMemcpyDeviceToHost));
    return NPP_OK;
}

npp_status npp_loop_run(npp_loop* L, int32_t steps, void* stream)
{
    if (!L || steps < 0) return fail(L ? L->h : nullptr, NPP_INVALID_ARG, "loop: bad arguments");
    npp_handle* h = L->h;
    LOOP_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < steps; ++i) LOOP_TRY(h, cudaGraphLaunch(L->exec, s));
    return NPP_OK;
}

npp_status npp_loop_read(npp_loop* L, npp_loop_state* out_host)
{
    if (!L || !out_host) return fail(L ? L->h : nullptr, NPP_INVALID_ARG, "loop: bad arguments");
    npp_handle* h = L->h;
    LOOP_TRY(h, cudaSetDevice(h->device));
    LoopDev d;
    LOOP_TRY(h, cudaDeviceSynchronize());
    LOOP_TRY(h, cudaMemcpy(&d, L->d_dyn, sizeof d, cudaMemcpyDeviceToHost));
    memset(out_host, 0, sizeof *out_host);
    out_host->x = (float)d.px; out_host->y = (float)d.py; out_host->phi = (float)d.pphi;
    out_host->v = (float)d.pv; out_host->a_prev0 = d.ap0; out_host->a_prev1 = d.ap1;
    out_host->t = d.t; out_host->waypoint = d.waypoint; out_host->done = d.done;
    out_host->status = d.status; out_host->best_idx = d.best_idx;
    out_host->n_infeasible = d.n_infeasible; out_host->best_cost = d.best_cost;
    if (d.mission) {
        out_host->waypoint = d.goal_k;
        out_host->space_index = d.idx;
        out_host->stop = d.stop;
    }
    return NPP_OK;
}

npp_status npp_loop_log(npp_loop* L, float* log_host, int32_t max_rows, int32_t* rows_out)
{
    if (!L || !log_host || max_rows < 0) return fail(L ? L->h : nullptr, NPP_INVALID_ARG, "loop: bad arguments");
    npp_handle* h = L->h;
    LOOP_TRY(h, cudaSetDevice(h->device));
    LoopDev d;
    LOOP_TRY(h, cudaDeviceSynchronize());
    LOOP_TRY(h, cudaMemcpy(&d, L->d_dyn, sizeof d, cudaMemcpyDeviceToHost));
    int rows = d.t < L->max_log ? d.t : L->max_log;
    if (rows > max_rows) rows = max_rows;
    if (rows > 0) LOOP_TRY(h, cudaMemcpy(log_host, L->d_log, (size_t)rows * 8 * sizeof(float), cudaMemcpyDeviceToHost));
    if (rows_out) *rows_out = rows;
    return NPP_OK;
}

npp_status npp_loop_samples(npp_loop* L, float* costs_host, int32_t* first_hit_host)
{
    if (!L) return fail(nullptr, NPP_INVALID_ARG, "loop is NULL");
    npp_handle* h = L->h;
    LOOP_TRY(h, cudaSetDevice(h->device));
    LOOP_TRY(h, cudaDeviceSynchronize());
    if (costs_host)
        LOOP_TRY(h, cudaMemcpy(costs_host, L->d_costs, (size_t)L->N * sizeof(float), cudaMemcpyDeviceToHost));
    if (first_hit_host)
        LOOP_TRY(h, cudaMemcpy(first_hit_host, L->d_fh, (size_t)L->N * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return NPP_OK;
}

npp_status npp_loop_last_timing(npp_loop* L, float* stage_ms, int32_t n)
{
    if (!L || !stage_ms || n < 1) return fail(L ? L->h : nullptr, NPP_INVALID_ARG, "loop: bad arguments");
    npp_handle* h = L->h;
    LOOP_TRY(h, cudaSetDevice(h->device));
    LOOP_TRY(h, cudaEventSynchronize(L->ev[3]));
    float t[4] = { 0.f, 0.f, 0.f, 0.f };
    LOOP_TRY(h, stage_times(L->ev, L->cev, L->nch, t));
    for (int i = 0; i < n && i < 4; ++i) stage_ms[i] = t[i];
    return NPP_OK;
}

npp_status npp_loop_destroy(npp_loop* L)
{
    if (!L) return NPP_OK;
    cudaSetDevice(L->h->device);
    cudaDeviceSynchronize();
    free_loop(L);
    return NPP_OK;
}

}  // extern "C"
