/*
 * npp.h -- C ABI of the GB300 planner library (libnpp.so).
 *
 * The library implements the per-sampling-time batched rollout of Plessen,
 * "Online Sampling in the Parameter Space of a Neural Network for
 * GPU-accelerated Motion Planning of Autonomous Vehicles" (arXiv 1904.06680):
 * N neural-network controller parameter vectors are sampled, each one is held
 * fixed over a T-step horizon while the evolving feature vector drives it
 * (Sect. II-D "Sixth", Eq. eq_def_stph), the controls are integrated through
 * the kinematic vehicle model (Sect. IV), every state is checked against
 * obstacle points extrapolated at constant velocity with the polytope
 * inequalities of Eq. eq_Apsietc_collAvoidIneqs, and the best sample is
 * returned (a_t = X(s_t, theta*), Eq. eq_def_at_mathcalXetc).
 *
 * Conventions shared by every entry point:
 *  - Plain C types only.  Pointers named *_dev are device pointers on the
 *    handle's device; pointers named *_host are host pointers.  The caller
 *    owns every buffer it passes; the handle owns its own workspaces.
 *  - Calls taking a `stream` are asynchronous on that CUDA stream (a
 *    cudaStream_t passed as void*, NULL = legacy default stream); their
 *    device outputs are valid once the stream has reached that point.
 *    Calls without a stream are synchronous.
 *  - World frame: x, y in m, heading phi in rad (counter-clockwise from +x),
 *    speed v in m/s (negative = reverse).  Obstacle points are 4 floats
 *    (x, y, vx, vy): position and constant velocity (Sect. II-D item (i)
 *    describes points by position, heading and speed; vx = speed cos heading,
 *    vy = speed sin heading).  Arrays of points are [M][4], 16-byte aligned.
 *  - Parameter vectors theta hold, per layer, W[out][in] row-major then
 *    b[out], for the network [n_in = 8, width, width, 2], tanh on every
 *    layer; n_theta = 12 width + width^2 + 2 (450, 1410, 4866 for widths
 *    16, 32, 64).
 *  - Sampling: theta_n[i] is entry (i mod 4) of the Box-Muller normals made
 *    from Philox4x32-10(counter = (i / 4, n, t_index, stream_id),
 *    key = (seed & 0xffffffff, seed >> 32)); words 0,1 give entries 0,1 and
 *    words 2,3 give entries 2,3; within a pair the first word sets the radius
 *    sqrt(-2 ln u) and the second the angle 2 pi u, with
 *    u = (2 (w >> 9) + 1) 2^-24.  The results are reproducible bit for bit.
 *  - Results are a pure function of the inputs, seed and t_index: the launch
 *    shape does not change any per-sample arithmetic, and ties in cost go to
 *    the lowest sample index.
 *  - Errors: every call returns an npp_status; npp_last_error(h) gives a
 *    human-readable message for the last failing call on that handle.
 *    Invalid arguments are rejected before any work is queued.
 */
#ifndef NPP_H_
#define NPP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NPP_OK = 0,
    NPP_INVALID_ARG = 1,    /* bad size, pointer, alignment or non-finite scalar */
    NPP_INFEASIBLE = 2,     /* not an error: every sample collided (Sect. II-D
                               "Third": no collision-free trajectory is
                               guaranteed); the result is the sample whose
                               first collision comes last */
    NPP_CUDA_ERROR = 3,     /* a CUDA runtime call failed */
    NPP_DEVICE_TIMEOUT = 4, /* a bounded device-side wait gave up */
    NPP_UNSUPPORTED = 5     /* configuration outside what the library builds */
} npp_status;

/* Vehicle, footprint, feature, cost and network constants.  The model
 * constants play the role of the paper's Table veh and Table
 * hyperparameters; they are fixed per handle ("defined directly on the
 * GPU", Sect. II-D "First" and "Fourth"). */
typedef struct {
    float lf, lr;              /* CoG to front / rear axle [m]                   */
    float delta_max;           /* steering limit [rad]; delta = delta_max a[0]   */
    float delta_rate_max;      /* steering-rate limit [rad/s]                    */
    float u_min, u_max;        /* acceleration range; u = u_min + (a[1]+1)/2 (u_max-u_min) */
    float Ts;                  /* sampling time and Euler step [s]               */
    float half_len, half_wid;  /* rectangle half length / half width [m]        */
    float c_off;               /* rectangle centre ahead of the reference point [m] */
    float dxi_n, deta_n, dphi_n, dv_n; /* feature normalisation (Delta constants) */
    float w_pos, w_phi, w_v, w_effort; /* cost weights                          */
    int32_t n_in;              /* network inputs: must be 8                      */
    int32_t width;             /* hidden width: 16, 32 or 64                     */
    int32_t max_N, max_T, max_M; /* workspace capacity of the handle             */
    /* Variants of Sect. V (a zero-filled tail keeps the defaults): */
    int32_t feature_frame;     /* goal offsets s0, s1 of the features (Eq. of s_{t+h}):
                                  0 = in the EV frame at t (default), 1 = in the
                                  vehicle's own frame at t+h                       */
    int32_t v_limits;          /* 1 = velocity constraints by discarding samples: a
                                  sample is discarded at the first state h >= 1 it
                                  reaches whose speed is outside [v_min, v_max],
                                  exactly as if it collided there (first_hit = h);
                                  0 = off (default)                                */
    float v_min, v_max;        /* speed limits [m/s] when v_limits = 1; v_min <= v_max */
} npp_config;

/* Vehicle state at the sampling time (world frame) with the controls applied
 * at the previous sampling time, a_{t-1} (normalised, in [-1, 1]). */
typedef struct { float x, y, phi, v, a_prev0, a_prev1; } npp_state;

/* Goal setpoint zeta_goal = [x, y, phi, v] (world frame). */
typedef struct { float x, y, phi, v; } npp_goal;

/* Device-side summary of one plan step. */
typedef struct {
    int32_t best_idx;   /* winning sample index                              */
    int32_t status;     /* NPP_OK or NPP_INFEASIBLE; NPP_DEVICE_TIMEOUT when a
                           bounded device-side wait of this step (the bulk
                           copy staging the obstacle points of a brute-force
                           check, about a second) gave up: the step's results
                           are then not valid                                */
    float best_cost;    /* its cost (+inf when infeasible)                   */
    int32_t first_hit;  /* its first colliding (or, with v_limits, speed-violating)
                           horizon index, -1 if none                         */
    int32_t reserved[4];
} npp_best;

/* Output buffers of a plan step; all device pointers, any may be NULL except
 * `best`.  Trajectory and controls are those of the winning sample in the
 * world frame; for an infeasible winner the rows after its first collision
 * repeat the colliding state and the controls there are 0. */
typedef struct {
    npp_best* best;          /* [1]                                          */
    float* params;           /* [n_theta]   winning parameter vector         */
    float* controls;         /* [T][2]      applied normalised controls      */
    float* trajectory;       /* [T+1][4]    (x, y, phi, v)                   */
    float* costs;            /* [N]         per-sample cost, +inf if collided */
    int32_t* first_hit;      /* [N]         first colliding (or speed-violating) h, -1 if none */
    float* sample_traj;      /* [T+1][N][4] every sample's states, EV frame at t
                                (origin at the vehicle, x along its heading);
                                rows after a sample's first collision continue
                                its dynamics and carry no meaning */
    float* sample_ctrl;      /* [T][N][2]   every sample's applied controls   */
} npp_outputs;

typedef struct npp_handle npp_handle;

/* Create a handle on CUDA device `device`: validates the configuration and
 * allocates device workspaces for up to max_N samples, max_T steps and max_M
 * obstacle points (point sets larger than shared memory, about 14,000
 * points, are read from an L2-resident copy instead).  *h is set to NULL on
 * failure. */
npp_status npp_create(npp_handle** h, const npp_config* cfg, int32_t device);

/* Free the handle and its workspaces (waits for its device work). */
npp_status npp_destroy(npp_handle* h);

/* Message for the last failing call on h; with h = NULL, the most recent
 * failure of any call.  The pointer stays valid until the next failure. */
const char* npp_last_error(const npp_handle* h);

/* General vehicle footprint (Sect. II-D: the EV modelled as an arbitrarily
 * refined polytope, convex or non-convex, checked by the linear inequalities
 * A(phi)(p - [x, y]) < b(phi)): the union of n_pieces convex polygons.
 * Piece k has the vertices verts_host[2*piece_start_host[k] ..
 * 2*piece_start_host[k+1]) as (x, y) pairs in the vehicle's frame (x along
 * the heading, origin at the reference point), counter-clockwise and
 * strictly convex; piece_start_host[0] = 0.  A point collides when it is
 * strictly inside some piece.  At most 16 pieces and 64 vertices in total.
 * Host arrays, copied synchronously: call between plan steps, and before
 * npp_loop_create.  n_pieces = 0 restores the rectangle of the config.  The
 * plan-step, closed-loop, hill-climb and proposal entry points of h then use
 * the polygon check (per-step spatial bins; collide_variant 0..4 selects a
 * brute-force check over every point instead, with identical results);
 * npp_batch_create on such a handle returns NPP_UNSUPPORTED.
 * NPP_INVALID_ARG for a piece that is not strictly convex and
 * counter-clockwise, winds more than once, or has fewer than 3 vertices. */
npp_status npp_set_footprint(npp_handle* h, const float* verts_host, const int32_t* piece_start_host,
                             int32_t n_pieces);

/* Number of network parameters of cfg's network, or -1 if unsupported. */
int32_t npp_n_theta(const npp_config* cfg);

/* One plan step (Step 5 of Alg. 1): sample N parameter vectors (sample 0 is
 * warm_dev when non-NULL, the warm start theta*_{t-1} of Sect. II-D "Fifth"),
 * roll each out over T steps from `state` towards `goal` among the M
 * obstacle points obs_dev (world frame, [M][4], may be NULL when M = 0), and
 * reduce to the best sample.  1 <= N <= max_N, 1 <= T <= max_T,
 * 0 <= M <= max_M.  Asynchronous on `stream`; outputs as in npp_outputs. */
npp_status npp_plan_step(npp_handle* h, const npp_state* state, const npp_goal* goal,
                         const float* obs_dev, int32_t M, int32_t N, int32_t T,
                         uint64_t seed, uint32_t t_index, const float* warm_dev,
                         const npp_outputs* out, void* stream);

/* The same plan step with HOST buffers: copies obs_host (and warm_host) to
 * the device, runs npp_plan_step on the handle's own stream, copies the
 * summary and the requested outputs back to the host pointers in out_host
 * (fields as in npp_outputs, host memory; sample_traj and sample_ctrl must
 * be NULL) and synchronises.  Returns NPP_INFEASIBLE when every sample
 * collided. */
npp_status npp_plan_step_host(npp_handle* h, const npp_state* state, const npp_goal* goal,
                              const float* obs_host, int32_t M, int32_t N, int32_t T,
                              uint64_t seed, uint32_t t_index, const float* warm_host,
                              const npp_outputs* out_host);

/* The sampling loop of the paper's hill climb (TSHC, Sect. II-D "Fourth"-
 * "Sixth": a restart perturbs the current best parameters by sigma_pert
 * times normal noise) run on the device: round 0 is npp_plan_step; round
 * r = 1 .. n_restarts-1 keeps the best so far as sample 0 and draws the other
 * samples as theta_best + sigma_pert eps with eps the normals of Philox
 * stream r (same counter layout), so the best cost never increases.  The
 * paper leaves the update of sigma_pert to its cited work; here it is fixed
 * per call.  out->params must be a device buffer of n_theta floats (it holds
 * the running best); the outputs describe the final round (its winner is the
 * best of all rounds).  NPP_INVALID_ARG for n_restarts < 1 or sigma_pert not
 * finite and positive, otherwise as npp_plan_step. */
npp_status npp_plan_tshc(npp_handle* h, const npp_state* state, const npp_goal* goal,
                         const float* obs_dev, int32_t M, int32_t N, int32_t T, uint64_t seed,
                         uint32_t t_index, const float* warm_dev, int32_t n_restarts, float sigma_pert,
                         const npp_outputs* out, void* stream);

/* Roll out K explicit parameter vectors theta_dev[K][n_theta] (no sampling,
 * no selection): writes costs[K], first_hit[K] and, when non-NULL, every
 * rollout's states sample_traj[T+1][K][4] and controls sample_ctrl[T][K][2]
 * in the EV frame at t.  For closed-form and regression checks. */
npp_status npp_rollout_params(npp_handle* h, const npp_state* state, const npp_goal* goal,
                              const float* obs_dev, int32_t M, const float* theta_dev,
                              int32_t K, int32_t T, float* costs_dev, int32_t* first_hit_dev,
                              float* sample_traj_dev, float* sample_ctrl_dev, void* stream);

/* The sampled parameter vectors of samples n0 .. n0+K-1 (see "Sampling"
 * above) written to out_dev[K][n_theta], rows of exactly n_theta entries.
 * 0 <= n0, 1 <= K, 1 <= n_theta. */
npp_status npp_sample_params(uint64_t seed, uint32_t t_index, uint32_t stream_id,
                             int32_t n0, int32_t K, int32_t n_theta, float* out_dev,
                             void* stream);

/* Diagnostics (no counterpart in the paper): evaluates the FP32 function
 * approximations the rollout uses on x_dev[n] (device): fn 0 tanh of the
 * network layers -> y_dev; 1 tan of the steering angle -> y_dev; 2 sin and
 * cos of a heading -> y_dev, y2_dev.  Lets callers bound their error against
 * correctly rounded values.  NPP_INVALID_ARG for an unknown fn, n < 0 or a
 * NULL output that fn writes. */
npp_status npp_math_eval(int32_t fn, const float* x_dev, int32_t n, float* y_dev, float* y2_dev,
                         void* stream);

/* Measurement (no counterpart in the paper): FP32 fused multiply-adds per
 * second that device `device` sustains on streams of independent FMA chains
 * (packed = 0: scalar FFMA; 1: packed FP32x2 FMA, two per instruction), every
 * SM filled, best of three timed runs after a warm-up; the denominator of
 * the rollout kernels' roofline next to the figure derived from SM count,
 * FP32 lanes and clock.  Synchronous, on the default stream; takes a few
 * milliseconds.  NPP_INVALID_ARG for a NULL output or packed not 0/1,
 * NPP_CUDA_ERROR if the device is unavailable. */
npp_status npp_measure_fma_peak(int32_t device, int32_t packed, double* fma_per_s);

/* Failure detection (no counterpart in the paper).  npp_wait_probe runs the
 * library's bounded mbarrier wait (the one of the obstacle-point staging and
 * the GEMM pipeline) in one block on the current device, on a barrier whose
 * single expected arrival happens (arrive = 1) or never happens (arrive =
 * 0), with a limit of limit_cycles clock cycles (1 .. 4e9); writes 1 to
 * *completed_host if the wait saw the phase complete, 0 if it gave up.  The
 * context stays usable either way.  Synchronous.
 * npp_inject_fault sets the handle's device fault flag exactly as a timed-out
 * wait of a plan step's kernels does: the next plan step reports
 * NPP_DEVICE_TIMEOUT in its npp_best.status (npp_plan_step_host returns it)
 * and clears the flag. */
npp_status npp_wait_probe(int64_t limit_cycles, int32_t arrive, int32_t* completed_host);
npp_status npp_inject_fault(npp_handle* h);

/* ---------------------------------------------------------------------
 * Device-resident closed loop (Alg. 1): each sampling time is one CUDA graph
 * replay holding the plan step and an advance kernel that applies the
 * winner's first control to a simulated vehicle (the kinematic bicycle of
 * Sect. IV in FP64, explicit Euler with Ts), moves the obstacle points at
 * their velocities, switches to the next waypoint once the current one is
 * reached within eps = (eps_xi, eps_eta, eps_phi, eps_v) (position error along
 * and across the vehicle heading; Table hyperparameters), and keeps the
 * winner's parameters as the next step's sample 0 (warm start, Sect. II-D
 * "Fifth").  The sampling time t is the Philox t_index.
 * --------------------------------------------------------------------- */
typedef struct npp_loop npp_loop;

typedef struct {
    float x, y, phi, v, a_prev0, a_prev1;  /* simulated vehicle after the last step */
    int32_t t;            /* sampling times completed                         */
    int32_t waypoint;     /* index of the current waypoint (mission mode: of the
                             goal setpoint on the reference path)              */
    int32_t done;         /* 1 once the last waypoint has been reached         */
    int32_t status;       /* status of the last plan step (OK / INFEASIBLE)    */
    int32_t best_idx;     /* winner of the last plan step                      */
    int32_t n_infeasible; /* plan steps that ended infeasible                  */
    float best_cost;      /* cost of the last winner                           */
    int32_t space_index;  /* mission mode: progress index on the reference path */
    int32_t stop;         /* mission mode: next stop setpoint to reach          */
    int32_t reserved;
} npp_loop_state;

/* The hill climb of Sect. II-D (TSHC, N_restarts rounds; Table
 * hyperparameters) in every sampling time of the loops created on h after
 * this call: round 0 is the plan step (warm start = the last winner); each
 * of the n_restarts - 1 further rounds draws N samples theta = theta_best +
 * sigma_pert eps (eps the normals of Philox stream r, r = round) with
 * theta_best -- the winner so far -- as sample 0, so the best cost never
 * increases; the last round's winner is applied.  The same rounds as
 * npp_plan_tshc.  The paper takes sigma_pert from its cited work; here it is
 * one fixed scale.  n_restarts in [1, 64] (1, the default: the plan step
 * alone); sigma_pert > 0 and finite when n_restarts > 1.  Loops created
 * earlier keep their setting. */
npp_status npp_set_loop_restarts(npp_handle* h, int32_t n_restarts, float sigma_pert);

/* Create a loop on handle h (which it uses; keep h alive): initial state s0,
 * waypoints_host[n_wp][4] (x, y, phi, v), eps_host[4], obstacle points
 * obs_dev[M][4] at t = 0 (copied; the caller's array is not modified), N
 * samples and horizon T per plan step (within the handle's capacity), and a
 * device log of up to max_log rows.  Captures the step graph (synchronous). */
npp_status npp_loop_create(npp_handle* h, const npp_state* s0, const float* waypoints_host,
                           int32_t n_wp, const float* eps_host, const float* obs_dev, int32_t M,
                           int32_t N, int32_t T, uint64_t seed, int32_t max_log, npp_loop** out);

/* Mission layer of Alg. 1 (Steps 3, 4 and 7; Sect. II-B to II-D) on the
 * device, for a loop created by npp_loop_create_mission. */
typedef struct {
    float range_front, range_back, range_side; /* range field visible at t, EV frame:
                                                  xi in [-back, front], |eta| <= side [m] */
    int32_t window;        /* setpoints searched ahead of the space index, >= 1        */
    int32_t hide_outside;  /* 1: obstacle points outside the range field at t are not
                              seen by that sampling time's plan step                 */
} npp_mission;

/* A loop that follows a reference path ref_host[n_ref][4] (x, y, phi, v,
 * world frame; mission data of Sect. II-B) instead of a waypoint list.
 * Setpoints with v = 0 and the last one are stop setpoints (a cusp, a parking
 * position) that must be reached within eps before the path beyond them is
 * used; reaching the last one completes the mission (npp_loop_state.done).
 * At every sampling time, on the simulated vehicle's pose: the space index
 * (Sect. II-C) is the setpoint closest to the vehicle among index ..
 * min(index + window, next stop), ties to the lowest; the goal setpoint
 * (Step 4; Sect. II-D (iv)) is the furthest setpoint from the space index on,
 * up to the next stop, with it and every setpoint before it within or on the
 * range field (the space index itself when even that one is outside).
 * With hide_outside the points outside the range field at t are parked far
 * away (at rest) for that plan step.  Log rows and npp_loop_state.waypoint
 * carry the goal setpoint's index.  Other arguments and behaviour as
 * npp_loop_create; NPP_INVALID_ARG for a negative or non-finite field
 * extent, window < 1 or hide_outside not 0/1. */
npp_status npp_loop_create_mission(npp_handle* h, const npp_state* s0, const float* ref_host, int32_t n_ref,
                                   const npp_mission* mission, const float* eps_host, const float* obs_dev,
                                   int32_t M, int32_t N, int32_t T, uint64_t seed, int32_t max_log,
                                   npp_loop** out);

/* Synchronise and copy the M obstacle points the next plan step of L sees
 * (world frame at the current sampling time, (x, y, vx, vy); hidden points
 * parked at (1e7, 1e7) at rest) into obs_host[M][4]. */
npp_status npp_loop_points(npp_loop* L, float* obs_host);

/* Run `steps` sampling times (graph replays), asynchronous on `stream`.
 * A loop's steps must not run concurrently with other work on its handle. */
npp_status npp_loop_run(npp_loop* L, int32_t steps, void* stream);

/* Synchronise the device and read the loop state. */
npp_status npp_loop_read(npp_loop* L, npp_loop_state* out_host);

/* Synchronise and copy up to max_rows log rows of 8 floats (one per completed
 * step: x, y, phi, v before the step, applied a0, a1, winner cost, waypoint
 * index) into log_host; *rows_out receives the number copied. */
npp_status npp_loop_log(npp_loop* L, float* log_host, int32_t max_rows, int32_t* rows_out);

/* Synchronise and copy the last step's per-sample costs[N] and first
 * collisions first_hit[N] (either pointer may be NULL). */
npp_status npp_loop_samples(npp_loop* L, float* costs_host, int32_t* first_hit_host);

/* Stage times of the last replayed step in ms (events captured in the
 * graph): [0] trajectory kernel, [1] collision kernel, [2] selection
 * epilogue + advance, [3] whole step; writes up to n values.  When the
 * binned check runs fused into the trajectory kernel ("fuse"), [0] is the
 * grid build and [1] the fused kernel; in step chunks ("chunks"), [0] and
 * [1] are summed over the chunks. */
npp_status npp_loop_last_timing(npp_loop* L, float* stage_ms, int32_t n);

/* Free the loop (after synchronising the device). */
npp_status npp_loop_destroy(npp_loop* L);

/* ---------------------------------------------------------------------
 * Batched planning: many independent plan steps ("scenes", each with its own
 * state, goal, obstacle points, N, T and network width 16, 32 or 64; the
 * vehicle/cost constants are the handle's) run as one batch of persistent
 * launches -- a point transform, one trajectory launch per width, one
 * collision launch over all scenes (work queues, costliest scenes first) and
 * one epilogue -- with no host work between them, so the batch can be
 * captured in a CUDA graph by the caller.  Each scene's result equals
 * npp_plan_step on that scene (same arithmetic per sample).
 * --------------------------------------------------------------------- */
typedef struct {
    npp_state state;
    npp_goal goal;
    int32_t N, T, M, width;   /* samples, horizon, obstacle points, hidden width */
    int64_t obs_offset;       /* index of the scene's first point in the batch's
                                 obstacle array ([total][4] floats)              */
    uint64_t seed;
    uint32_t t_index;
    int32_t reserved;
} npp_scene;

/* Outputs of a batch (device pointers; all but `best` may be NULL).  Scene s
 * starts at the offsets npp_batch_offsets returns: parameters (n_theta of its
 * width), control rows [T][2], trajectory rows [T+1][4], samples [N]. */
typedef struct {
    npp_best* best;          /* [S]                                           */
    float* params;           /* [sum n_theta]                                 */
    float* controls;         /* [sum T][2]                                    */
    float* trajectory;       /* [sum (T+1)][4]                                */
    float* costs;            /* [sum N]                                       */
    int32_t* first_hit;      /* [sum N]                                       */
} npp_batch_outputs;

typedef struct npp_batch npp_batch;

/* Validate the S scene descriptors, order the work, allocate the batch's
 * workspaces (24 bytes per sample-step plus the points) and upload the scene
 * table (synchronous).  The batch uses h's constants and keeps a pointer to h. */
npp_status npp_batch_create(npp_handle* h, const npp_scene* scenes, int32_t S, npp_batch** out);

/* New states, goals, seeds and t_index for the same scenes (sizes, widths and
 * obstacle offsets must not change); synchronous upload. */
npp_status npp_batch_update(npp_batch* B, const npp_scene* scenes);

/* offsets_host[S+1][4]: per scene the first parameter, control row,
 * trajectory row and sample of its outputs; row S holds the totals. */
npp_status npp_batch_offsets(npp_batch* B, int64_t* offsets_host);

/* Queue the whole batch on `stream` (kernels and memsets only).  obs_dev is
 * the [total points][4] world-frame obstacle array, 16-byte aligned. */
npp_status npp_plan_batch(npp_batch* B, const float* obs_dev, const npp_batch_outputs* out,
                          void* stream);

/* Launch shapes of the batch (no result changes): "collide" = collision
 * check: 1 (default) per-scene, per-step spatial bins (one warp per sample,
 * the points of the cells its rectangle's disk overlaps), 0 brute force over
 * the scene's points, sorted by cell so that tiles out of reach of an
 * item's live samples are skipped; "slices" = warps that share one 8-sample
 * brute-force item, each on an interleaved share of the point tiles (2, 4 or
 * 8; default 4); "traj_warps" = warps per trajectory block (4 or 8; default 8).
 * Synchronous (re-plans the work lists). */
npp_status npp_batch_set_option(npp_batch* B, const char* name, int32_t value);

/* Free the batch (after synchronising the device). */
npp_status npp_batch_destroy(npp_batch* B);

/* The plan step of npp_plan_step for callers that cannot allocate device
 * memory -- for instance a plugin whose host application owns every device
 * allocation, or a real-time control loop that must not call cudaMalloc once
 * it runs, because cudaMalloc may synchronise the device and take unbounded
 * time.  There is no counterpart in the paper; it is a deployment variant.
 *
 * It runs npp_plan_step's trajectory kernel and winner epilogue with one
 * collision check whatever M and N are: the brute-force check with all
 * points in shared memory (collide_variant 3 for N <= 8192, else 4), never
 * the spatial binning a handle picks for many points.  So M is limited to
 * the points shared memory holds (about 14,000 on GB300; more returns
 * NPP_UNSUPPORTED) and a large M * N runs slower than npp_plan_step.  All
 * collision checks give the same flags, so the outputs equal
 * npp_plan_step's.
 *
 * No handle: the constants come from cfg (its max_* fields are ignored and
 * it is checked as npp_create checks it), the
 * workspace is one fixed file-scope device array of about 17 MB that every
 * GPU loading this part of the library holds until the process exits.
 * Limits: 1 <= N <= 16384 and N * (T + 1) <= 688128 sample-steps (for
 * example N = 16384 with T <= 41); larger requests return NPP_INVALID_ARG
 * with a message in npp_last_error(NULL).  Inputs and outputs are as in
 * npp_plan_step (device pointers; out->best required), and the launch is
 * asynchronous on `stream` on the current device.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents; every call resets what must start at
 * zero, but calls that overlap on the GPU (other streams or threads) race.
 * Nothing here calls cudaMalloc, cudaFree or an allocating library routine. */
npp_status npp_plan_step_noalloc(const npp_config* cfg, const npp_state* state,
                                 const npp_goal* goal, const float* obs_dev, int32_t M,
                                 int32_t N, int32_t T, uint64_t seed, uint32_t t_index,
                                 const float* warm_dev, const npp_outputs* out, void* stream);

/* Launch options that do not change any result (they choose among kernels
 * computing identical values).  "collide_variant" in -1..5: 0 the
 * block-balanced collision kernel with 16 warps and one block per SM, 1 the
 * same with 8 warps and two blocks per SM, 2 warp-owned items of 8 samples,
 * 3 / 4 items of 8 samples checked by 4 / 2 warps each taking a slice of the
 * points, 5 per-step spatial binning: the points extrapolated to each step
 * are counting-sorted into a uniform grid around the vehicle and each state
 * is tested only against the cells its bounding disk overlaps (the same
 * per-point test, so the same flags as checking every point); -1 (default)
 * takes 5 from 128 points and below that 2 for N >= 6144 or at most 64
 * points, else 3.
 * "fuse" -1 (default), 0 or 1: with the binned check (5) and no per-sample
 * records requested, 1 runs the check inside the trajectory kernel: each
 * warp rolls its samples through a window of steps, checks the window's
 * states itself (the same grids and per-point test) and stops a sample
 * within one window of its first collision, storing states and controls up
 * to that window (every row the winner's outputs need).  Same results;
 * -1 takes it at width 64 (measured on GB300 at N = 65536, T = 100,
 * M = 8192: 2.72 ms per plan step against 3.83 in two kernels), 0 never.
 * "chunks" 0..8: with the binned check (5) and no per-sample records
 * requested (sample_traj and sample_ctrl NULL, and the closed loop), roll
 * the horizon out in that many chunks of steps, each followed by the check
 * of the states it produced; only the samples still collision-free go on to
 * the next chunk, so no sample is rolled out more than one chunk past its
 * first collision.  Each chunk regenerates its samples' parameters and
 * continues from the stored state and the carried FP32 values, so every
 * output (costs, first_hit, the winner and its rows) is the one of a single
 * launch.  0 (default): automatic (2 at width 64, else 1), 1: one launch
 * each; at most T chunks.
 * "traj_variant" 0..4: launch shape of the trajectory kernel -- 0 (default)
 * 2 hidden units per lane in blocks sized for occupancy, 1 four hidden units
 * per lane, 2 eight-warp blocks, 3 another block size, 4 at width 64 every
 * weight in registers (12 warps per SM; the width-64 default keeps half of
 * each lane's layer-2 weights in shared memory so that 16 fit), at width 32
 * 5 of each lane's 8 layer-2 input quads in shared memory (20 warps per
 * SM), at width 16 the default shape.
 * Returns NPP_INVALID_ARG for an unknown name or value. */
npp_status npp_set_option(npp_handle* h, const char* name, int32_t value);

/* Kernel timing for measurement: when enabled, npp_plan_step and
 * npp_rollout_params record CUDA events on their stream around each stage.
 * npp_last_timing synchronises on the last recorded event and writes up to n
 * durations in milliseconds: [0] trajectory kernel, [1] collision kernel,
 * [2] selection epilogue, [3] the whole call (npp_rollout_params has no
 * epilogue: [2] is 0); with the fused binned check, [0] is the grid build
 * and [1] the fused trajectory-and-check kernel; with the step chunks
 * ("chunks"), [0] and [1] are the sums over the chunks' trajectory and check
 * launches.  Disabled by default; enabling it adds four event records per
 * call (and two per chunk). */
npp_status npp_set_timing(npp_handle* h, int32_t enable);
npp_status npp_last_timing(npp_handle* h, float* stage_ms, int32_t n);

/* Work counters of the last timed plan step's binned collision check (also
 * of the first round of a closed loop's sampling time created with timing
 * on): [0] candidate point tests (each one evaluation of the rectangle's
 * inequalities), [1] states checked, [2] sample-steps the trajectory kernel
 * rolled out (N T in one launch, fewer with the step chunks).  Zero when
 * that step used another collision check.  Synchronises the device; needs
 * timing enabled; writes up to n (at most 3) values. */
npp_status npp_last_counts(npp_handle* h, uint64_t* counts, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* NPP_H_ */
