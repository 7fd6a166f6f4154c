// npp_device.cuh -- device-side building blocks of the planner library:
// the counter-based parameter sampler, the per-handle constants and the
// kernel argument blocks shared by the kernels and their launchers.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/npp.h"

namespace npp {

constexpr int NIN = 8;               // network inputs (features)
constexpr uint32_t FULL = 0xffffffffu;

// Constants derived once per handle from npp_config (FP32, device side).
struct DevCfg {
    float delta_max, r_rate;         // steering limit, rate limit per step (normalised)
    float lrL, iL;                   // l_r / (l_f + l_r), 1 / (l_f + l_r)
    float umid, uhalf;               // u = umid + uhalf a1
    float Ts;
    float ihl, ihw, c_off;           // 1/half_len, 1/half_wid, centre offset
    float idxi, ideta, idphi, idv;   // 1 / feature normalisation constants
    float w_pos, w_phi, w_v, w_effort;
    int body_frame;                  // goal offsets of the features in the frame at t+h
    int vlim;                        // speed limits on: discard at the first h >= 1 outside
    float v_lo, v_hi;                // [v_lo, v_hi]
};

// The device constants of a validated configuration (host side).
inline DevCfg devcfg_from(const npp_config& cfg)
{
    DevCfg d;
    const double L = (double)cfg.lf + cfg.lr;
    d.delta_max = cfg.delta_max;
    d.r_rate = (float)((double)cfg.delta_rate_max * cfg.Ts / cfg.delta_max);
    d.lrL = (float)(cfg.lr / L);
    d.iL = (float)(1.0 / L);
    d.umid = (float)(0.5 * ((double)cfg.u_min + cfg.u_max));
    d.uhalf = (float)(0.5 * ((double)cfg.u_max - cfg.u_min));
    d.Ts = cfg.Ts;
    d.ihl = (float)(1.0 / cfg.half_len);
    d.ihw = (float)(1.0 / cfg.half_wid);
    d.c_off = cfg.c_off;
    d.idxi = (float)(1.0 / cfg.dxi_n);
    d.ideta = (float)(1.0 / cfg.deta_n);
    d.idphi = (float)(1.0 / cfg.dphi_n);
    d.idv = (float)(1.0 / cfg.dv_n);
    d.w_pos = cfg.w_pos; d.w_phi = cfg.w_phi; d.w_v = cfg.w_v; d.w_effort = cfg.w_effort;
    d.body_frame = cfg.feature_frame;
    d.vlim = cfg.v_limits;
    d.v_lo = cfg.v_min;
    d.v_hi = cfg.v_max;
    return d;
}

// Range check of the variant fields of a configuration; null when valid.
inline const char* variant_error(const npp_config& cfg)
{
    if (cfg.feature_frame != 0 && cfg.feature_frame != 1) return "feature_frame is 0 or 1";
    if (cfg.v_limits != 0 && cfg.v_limits != 1) return "v_limits is 0 or 1";
    if (cfg.v_limits == 1 && !(std::isfinite(cfg.v_min) && std::isfinite(cfg.v_max) && cfg.v_min <= cfg.v_max))
        return "v_limits needs finite v_min <= v_max";
    return nullptr;
}

// Range check of the vehicle, feature and cost constants and the variant
// fields of a configuration (not the network shape, not the capacities);
// null when valid.  Every entry point that takes a configuration uses it.
inline const char* config_error(const npp_config& cfg)
{
    const float* f = &cfg.lf;                // the 18 float constants lf .. w_effort
    for (int i = 0; i < 18; ++i)
        if (!std::isfinite(f[i])) return "config has a non-finite constant";
    if (!(cfg.lf + cfg.lr > 0.f) || !(cfg.lr >= 0.f) || !(cfg.delta_max > 0.f) ||
        !(cfg.delta_rate_max > 0.f) || !(cfg.u_max >= cfg.u_min) || !(cfg.Ts > 0.f) ||
        !(cfg.half_len > 0.f) || !(cfg.half_wid > 0.f) || !(cfg.dxi_n > 0.f) ||
        !(cfg.deta_n > 0.f) || !(cfg.dphi_n > 0.f) || !(cfg.dv_n > 0.f))
        return "config constant out of range";
    return variant_error(cfg);
}

// ------------------------------------------------------------------ sampler
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
// published multipliers, key bumped by the published Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Natural log of u in (0,1) (the FP32 sampler specification): u = 2^e f with
// f in [sqrt(1/2), sqrt(2)), ln f = 2 atanh(s), s = (f-1)/(f+1), odd Taylor
// terms up to s^11, Cody-Waite split of ln 2.  Every operation is a single
// IEEE round-to-nearest step so that the value is reproducible bit for bit.
__device__ __forceinline__ float spec_ln(float u)
{
    uint32_t b = __float_as_uint(u);
    int e = (int)(b >> 23) - 127;
    const uint32_t m = b & 0x7FFFFFu;
    float f;
    if (m > 0x3504F3u) { f = __uint_as_float(m | 0x3F000000u); e += 1; }
    else               { f = __uint_as_float(m | 0x3F800000u); }
    const float num = __fsub_rn(f, 1.0f);
    const float den = __fadd_rn(f, 1.0f);
    const float s = __fdiv_rn(num, den);
    const float z = __fmul_rn(s, s);
    float p = __fmaf_rn(z, 0x1.745d18p-3f, 0x1.c71c72p-3f);   // 2/11, 2/9
    p = __fmaf_rn(z, p, 0x1.24924ap-2f);                        // 2/7
    p = __fmaf_rn(z, p, 0x1.99999ap-2f);                        // 2/5
    p = __fmaf_rn(z, p, 0x1.555556p-1f);                        // 2/3
    const float t = __fmul_rn(s, z);
    const float lnf = __fmaf_rn(t, p, __fmul_rn(2.0f, s));
    const float ef = __int2float_rn(e);
    return __fmaf_rn(ef, 0x1.62e400p-1f, __fmaf_rn(ef, 0x1.7f7d1cp-20f, lnf));
}

// sin and cos of 2 pi K 2^-24 for odd K in [1, 2^24): quarter-turn reduction
// in integers (exact), Taylor polynomials of degree 9 / 10 on |x| <= pi/4.
__device__ __forceinline__ void spec_sincos2pi(uint32_t K, float& s_out, float& c_out)
{
    const int q = (int)((K + (1u << 21)) >> 22);
    const int k = (int)K - q * (1 << 22);
    const float x = __fmul_rn(__int2float_rn(k), 0x1.921fb6p-22f);
    const float z = __fmul_rn(x, x);
    float ps = __fmaf_rn(z, 0x1.71de3ap-19f, -0x1.a01a02p-13f);
    ps = __fmaf_rn(z, ps, 0x1.111112p-7f);
    ps = __fmaf_rn(z, ps, -0x1.555556p-3f);
    const float sx = __fmaf_rn(__fmul_rn(x, z), ps, x);
    float pc = __fmaf_rn(z, -0x1.27e4fcp-22f, 0x1.a01a02p-16f);
    pc = __fmaf_rn(z, pc, -0x1.6c16c2p-10f);
    pc = __fmaf_rn(z, pc, 0x1.555556p-5f);
    pc = __fmaf_rn(z, pc, -0.5f);
    const float cx = __fmaf_rn(z, pc, 1.0f);
    switch (q & 3) {
    case 0: s_out = sx;  c_out = cx;  break;
    case 1: s_out = cx;  c_out = -sx; break;
    case 2: s_out = -sx; c_out = -cx; break;
    default: s_out = -cx; c_out = sx; break;
    }
}

// Box-Muller pair from two Philox words: radius from `a`, angle from `b`.
__device__ __forceinline__ float2 spec_normal_pair(uint32_t a, uint32_t b)
{
    const float u1 = __fmul_rn(__uint2float_rn(((a >> 9) << 1) | 1u), 0x1p-24f);
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, spec_ln(u1)));
    float s, c;
    spec_sincos2pi(((b >> 9) << 1) | 1u, s, c);
    return make_float2(__fmul_rn(r, c), __fmul_rn(r, s));
}

struct SamplerKey {
    uint32_t k0, k1, t_index, stream_id;
};

// theta_n[4q .. 4q+3]
__device__ __forceinline__ float4 sample_quad(const SamplerKey& key, uint32_t q, uint32_t n)
{
    const uint4 w = philox4x32_10(make_uint4(q, n, key.t_index, key.stream_id), key.k0, key.k1);
    const float2 a = spec_normal_pair(w.x, w.y);
    const float2 b = spec_normal_pair(w.z, w.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

// theta_n[i], theta_n[i+1] for even i (one Box-Muller pair)
__device__ __forceinline__ float2 sample_pair(const SamplerKey& key, uint32_t i, uint32_t n)
{
    const uint4 w = philox4x32_10(make_uint4(i >> 2, n, key.t_index, key.stream_id), key.k0, key.k1);
    return (i & 2u) ? spec_normal_pair(w.z, w.w) : spec_normal_pair(w.x, w.y);
}

// Gaussian sampling proposal of a plan step: samples n < n_prop take
// theta_i = fma(sigma_i, eps_i, mu_i) with eps the normals of stream
// `stream` (1 for the learned proposal; the restart rounds of the hill
// climb use 1, 2, ...) rounded once to FP32; the others are the isotropic
// samples.  mu and sigma hold n_theta FP32 values.
struct Proposal {
    const float* mu;
    const float* sigma;
    int n_prop;
    uint32_t stream;      // Philox stream of the proposal's normals (1 unless set)
};

__device__ __forceinline__ bool proposal_sample(const Proposal& p, uint32_t n)
{
    return p.mu != nullptr && (long long)n < (long long)p.n_prop;
}

// theta_n[4q .. 4q+3] of a plan step with proposal p (all four indices
// below n_theta)
__device__ __forceinline__ float4 sample_quad_mixed(const SamplerKey& key, const Proposal& p, uint32_t q,
                                                    uint32_t n)
{
    if (!proposal_sample(p, n)) return sample_quad(key, q, n);
    SamplerKey k1 = key;
    k1.stream_id = p.stream;
    const float4 e = sample_quad(k1, q, n);
    const int i = 4 * (int)q;
    return make_float4(fmaf(p.sigma[i], e.x, p.mu[i]), fmaf(p.sigma[i + 1], e.y, p.mu[i + 1]),
                       fmaf(p.sigma[i + 2], e.z, p.mu[i + 2]), fmaf(p.sigma[i + 3], e.w, p.mu[i + 3]));
}

// theta_n[i], theta_n[i+1] for even i
__device__ __forceinline__ float2 sample_pair_mixed(const SamplerKey& key, const Proposal& p, uint32_t i,
                                                    uint32_t n)
{
    if (!proposal_sample(p, n)) return sample_pair(key, i, n);
    SamplerKey k1 = key;
    k1.stream_id = p.stream;
    const float2 e = sample_pair(k1, i, n);
    return make_float2(fmaf(p.sigma[i], e.x, p.mu[i]), fmaf(p.sigma[i + 1], e.y, p.mu[i + 1]));
}

// Obstacle point o = (x, y, vx, vy) in the EV frame of the plan step (origin
// (x0, y0), heading with sine s0 and cosine c0), rounding fixed by explicit
// fmas so every collision path sees the same FP32 positions.
__device__ __forceinline__ void ev_point(const float4& o, float x0, float y0, float s0, float c0,
                                         float& px, float& py, float& vx, float& vy)
{
    const float dx = o.x - x0, dy = o.y - y0;
    px = fmaf(c0, dx, __fmul_rn(s0, dy));
    py = fmaf(-s0, dx, __fmul_rn(c0, dy));
    vx = fmaf(c0, o.z, __fmul_rn(s0, o.w));
    vy = fmaf(-s0, o.z, __fmul_rn(c0, o.w));
}

// theta[4q .. 4q+3] where the quad may run past n_theta (the proposal
// arrays hold exactly n_theta values)
__device__ __forceinline__ float4 sample_quad_mixed_tail(const SamplerKey& key, const Proposal& p, uint32_t q,
                                                         uint32_t n, int n_theta)
{
    if (4 * (int)q + 3 < n_theta || !proposal_sample(p, n)) return sample_quad_mixed(key, p, q, n);
    SamplerKey k1 = key;
    k1.stream_id = p.stream;
    const float4 e = sample_quad(k1, q, n);
    const float ev[4] = { e.x, e.y, e.z, e.w };
    float r[4] = { 0.f, 0.f, 0.f, 0.f };
    for (int j = 0; j < 4 && 4 * (int)q + j < n_theta; ++j) {
        const int i = 4 * (int)q + j;
        r[j] = fmaf(p.sigma[i], ev[j], p.mu[i]);
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}

// ------------------------------------------------------------------ spatial bins
// Per-step grids of the binned collision check: for step h, cell_start[h]
// [BIN_DIM^2 + 1 entries, stride BIN_CS_STRIDE] indexes the points of
// step h sorted by cell, pts + h M.  A query disk of radius `reach` around a
// state spans at most five cells per axis.
constexpr int BIN_DIM = 128;
constexpr int BIN_NCELL = BIN_DIM * BIN_DIM;
constexpr int BIN_CS_STRIDE = BIN_NCELL + 4;    // 16-byte multiple: the float2 points that follow stay aligned

struct BinView {
    float x0;              // lower-left corner of the grid (EV frame, both axes)
    float inv_cell;
    float reach;           // query radius
    const int* cell_start; // null: no grids
    const float2* pts;
    int M;
};

// General footprint: the union of convex pieces, each the intersection of
// half-planes n . q < b in the vehicle's frame (q relative to the reference
// point, x along the heading), faces of one piece consecutive, w = 1 on the
// last face of a piece.
constexpr int FP_MAX_FACES = 64;
constexpr int FP_MAX_PIECES = 16;
struct PolyView {
    const float4* faces;   // [n_faces] (nx, ny, b, last) with |n| = 1
    int n_faces;           // 0: the rectangle
    int brute;             // 1: every point each step (no grid cells)
    float r2;              // squared radius of a disk around the reference point holding the footprint
};

__device__ __forceinline__ int bin_cell(float x, const BinView& g)
{
    const float f = floorf((x - g.x0) * g.inv_cell);
    return (int)fminf(fmaxf(f, 0.0f), (float)(BIN_DIM - 1));
}

// The candidate points of a query disk in one step's grid: the cells of the
// (at most five) cell rows its bounding square overlaps, each row's cells
// one contiguous run of the cell-sorted points.  Cells are at least half as
// wide as the query radius, so the square spans at most five cells per axis;
// indices are clamped monotonically at the grid border, so every point that
// can lie in the disk is a candidate.
constexpr int BIN_MAX_ROWS = 5;      // cell rows a query can span (cells >= half the query radius)
struct CandRows {
    int b[BIN_MAX_ROWS];             // first sorted point of each row's run
    int e[BIN_MAX_ROWS];             // candidates before the end of each run (inclusive prefix)
    int total;
    // index (into the step's sorted points) of candidate k < total
    __device__ __forceinline__ int index(int k) const
    {
        int i = b[0] + k;
#pragma unroll
        for (int r = 1; r < BIN_MAX_ROWS; ++r)
            if (k >= e[r - 1]) i = b[r] + (k - e[r - 1]);
        return i;
    }
};

__device__ __forceinline__ CandRows cand_rows(const int* __restrict__ cs, const BinView& g, float x, float y,
                                              float r)
{
    const int ix0 = bin_cell(x - r, g), ix1 = bin_cell(x + r, g);
    const int iy0 = bin_cell(y - r, g), iy1 = bin_cell(y + r, g);
    CandRows c;
    int acc = 0;
#pragma unroll
    for (int k = 0; k < BIN_MAX_ROWS; ++k) {
        int beg = 0, len = 0;
        if (iy0 + k <= iy1) {
            beg = cs[(iy0 + k) * BIN_DIM + ix0];
            len = cs[(iy0 + k) * BIN_DIM + ix1 + 1] - beg;
        }
        c.b[k] = beg;
        acc += len;
        c.e[k] = acc;
    }
    c.total = acc;
    return c;
}

// ------------------------------------------------------------------ rollout math
// FP32 functions of the rollout step built on the SFU's approximate base-2
// exponential, reciprocal, sine and cosine (PTX ex2/rcp/sin/cos .approx).
// Absolute errors (measured against the correctly rounded values on a dense
// grid of arguments, see the diagnostics entry point): tanh below 5e-7 for
// every finite x; tan below 2e-6 for |z| <= 1; sin/cos of the heading below
// 1e-6 for |phi| <= 1e3.

__device__ __forceinline__ float sfu_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sfu_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sfu_sin(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sfu_cos(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// tanh x = 1 - 2 / (e^{2x} + 1); e^{2x} = 2^{x * 2/ln 2}.  Saturates to
// +-1 (e^{2x} = inf gives 1, e^{2x} = 0 gives -1).
__device__ __forceinline__ float tanh_r(float x)
{
    const float e = sfu_ex2(x * 2.88539008177792681f);
    return fmaf(-2.0f, sfu_rcp(e + 1.0f), 1.0f);
}

// tan z = sin z / cos z for the steering angle (|z| <= delta_max < pi/2)
__device__ __forceinline__ float tan_r(float z)
{
    return sfu_sin(z) * sfu_rcp(sfu_cos(z));
}

// sin and cos of a heading: Cody-Waite reduction by 2 pi (two-part constant,
// 2 pi = TWO_PI_HI + TWO_PI_LO) to |r| <= pi, then the SFU on r
__device__ __forceinline__ void sincos_r(float phi, float& s, float& c)
{
    const float TWO_PI_HI = 6.28318548202514648f;      // float nearest 2 pi
    const float TWO_PI_LO = -1.74845553146951715e-7f;  // 2 pi - TWO_PI_HI
    const float k = rintf(phi * 0.159154943091895336f);
    float r = fmaf(-k, TWO_PI_HI, phi);
    r = fmaf(-k, TWO_PI_LO, r);
    s = sfu_sin(r);
    c = sfu_cos(r);
}

// ------------------------------------------------------------------ kernels
// State of a device-resident closed loop (Alg. 1 run inside a CUDA graph).
// The plan-step kernels read the planner's view of it; the advance kernel
// moves the simulated vehicle and the mission forward.
struct LoopDev {
    float x0, y0, phi0, v0, ap0, ap1;  // vehicle state at this sampling time (FP32 view)
    float gx, gy, gphi, gv;            // current goal setpoint
    uint32_t t_index;                  // sampling time (Philox counter word)
    int warm_valid;                    // the warm-start buffer holds theta*_{t-1}
    double px, py, pphi, pv;           // simulated vehicle (FP64)
    int waypoint, n_wp, done, t;
    int status, best_idx, n_infeasible;
    float best_cost;
    float eps[4];                      // completion tolerances (xi, eta, phi, v)
    // mission mode (reference path): space index, next stop setpoint, goal
    // setpoint index, range field (front, back, side), index search window,
    // points outside the range field hidden from the plan step
    int mission, idx, stop, goal_k, window, hide;
    float field[3];
};

// Per-step scalars of a plan step, from the arguments or from a LoopDev.
struct StepIn {
    float x0, y0, phi0, v0, ap0, ap1, gx, gy, gphi, gv;
    uint32_t t_index;
    bool warm_ok;
};

// blocks of 32 point pairs (64 points) holding M obstacle points in the
// brute-force checks' layout (XY entries of a block, then its V entries)
__host__ __device__ constexpr int pair_blocks(int M) { return (M + 63) / 64; }

struct RolloutArgs {
    DevCfg c;
    float x0, y0, phi0, v0, ap0, ap1;  // world-frame state and last controls
    float gx, gy, gphi, gv;            // world-frame goal
    const float4* obs;                 // [M] world frame (x, y, vx, vy)
    int M, N, T;
    SamplerKey key;
    const float* theta;                // explicit parameters [N][n_theta] or null
    const float* warm;                 // replaces sample 0 when non-null
    Proposal prop;                     // sampling proposal (mu null: isotropic only)
    float* costs;                      // [N] or null
    int* first_hit;                    // [N] or null
    float4* traj;                      // [T+1][N] EV frame (always written)
    float2* ctrl;                      // [T][N]
    float* jfree;                      // [N] cost of each sample if collision-free
    int* vfirst;                       // [N] first speed-violating step (-1 none), written by the
                                       // trajectory kernel when c.vlim; null otherwise
    float4* coefA;                     // [T+1][N] (A, B, -C, D) scaled inequality rows
    float2* coefB;                     // [T+1][N] (E, -F)
    unsigned long long* best_key;      // packed (class, cost, index) minimum
    unsigned* work;                    // work-queue counter of the persistent collision kernel
    int grid_collide;                  // persistent grid size
    const LoopDev* dyn;                // when set, per-step scalars come from here
    int warm_force;                    // the warm start replaces sample 0 even before the loop's
                                       // first step (restart rounds: it is the incumbent)
    float4* pXY;                       // EV-frame point pairs in global memory when the points
                                       // exceed shared memory: 64 pair_blocks(M) entries, the
                                       // shared-memory staging's blocked layout
    unsigned* fault;                   // set when a bounded device wait gave up (read and
                                       // cleared by the winner epilogue), or null
    BinView bins;                      // per-step grids (binned and fused collision checks)
    unsigned long long* counts;        // measurement counters, or null: [0] candidate point tests
                                       // and [1] states checked by the binned check, [2] sample-steps
                                       // computed by the trajectory kernel
    // Step chunks (binned check, no per-sample records wanted): a
    // trajectory launch computes steps chunk_lo .. chunk_hi - 1 (states up to
    // chunk_hi), the check covers the states the chunk produced; chunk_hi 0:
    // the whole horizon in one launch each.  live_in (length *live_n_in)
    // lists the samples still collision-free before the chunk (null: all N);
    // the check appends the chunk's survivors to live_out, counting in
    // *live_n_out.  carry: [N] values carried between chunks.
    int chunk_lo, chunk_hi;
    const int* live_in;
    const int* live_n_in;
    int* live_out;
    int* live_n_out;
    float4* carry;
    PolyView poly;                     // general footprint (polygon checks)
};

__device__ __forceinline__ StepIn step_in(const RolloutArgs& a)
{
    StepIn s;
    if (a.dyn) {
        const LoopDev& d = *a.dyn;
        s.x0 = d.x0; s.y0 = d.y0; s.phi0 = d.phi0; s.v0 = d.v0; s.ap0 = d.ap0; s.ap1 = d.ap1;
        s.gx = d.gx; s.gy = d.gy; s.gphi = d.gphi; s.gv = d.gv;
        s.t_index = d.t_index;
        s.warm_ok = d.warm_valid != 0 || a.warm_force != 0;
    } else {
        s.x0 = a.x0; s.y0 = a.y0; s.phi0 = a.phi0; s.v0 = a.v0; s.ap0 = a.ap0; s.ap1 = a.ap1;
        s.gx = a.gx; s.gy = a.gy; s.gphi = a.gphi; s.gv = a.gv;
        s.t_index = a.key.t_index;
        s.warm_ok = true;
    }
    return s;
}

struct EpilogueArgs {
    float x0, y0, phi0;
    int N, T, n_theta;
    SamplerKey key;
    const float* warm;
    Proposal prop;
    const float4* traj;
    const float2* ctrl;
    const unsigned long long* best_key;
    void* best;                        // npp_best*
    float* params;
    float* controls;
    float* trajectory;
    const LoopDev* dyn;                // when set, x0, y0, phi0, t_index, warm validity from here
    int warm_force;                    // as RolloutArgs::warm_force
    unsigned* fault;                   // as RolloutArgs::fault: nonzero turns the result's status
                                       // into NPP_DEVICE_TIMEOUT (and is cleared), or null
};

// launchers: trajectory kernel per network width, one collision kernel
cudaError_t launch_traj_w16(const RolloutArgs& a, cudaStream_t s, int variant);
cudaError_t launch_traj_w32(const RolloutArgs& a, cudaStream_t s, int variant);
cudaError_t launch_traj_w64(const RolloutArgs& a, cudaStream_t s, int variant);
// trajectories with the binned collision check done window by window by
// the trajectory warps (a.bins set): each sample stops within one window
// of its first collision; writes costs, first hits, the key and the states
// and controls up to that window
cudaError_t launch_fused_w16(const RolloutArgs& a, cudaStream_t s, int variant);
cudaError_t launch_fused_w32(const RolloutArgs& a, cudaStream_t s, int variant);
cudaError_t launch_fused_w64(const RolloutArgs& a, cudaStream_t s, int variant);
cudaError_t launch_collide_resident(const RolloutArgs& a, cudaStream_t s, int variant);
cudaError_t launch_collide_global(const RolloutArgs& a, cudaStream_t s);
int collide_global_blocks_per_sm();
int collide_resident_blocks_per_sm(int M, int variant);
int collide_max_points(int smem_limit);
// collisions through per-step spatial binning of the points (any M): builds
// the grids in `workspace` (binned_workspace_bytes) and checks every sample
// against the points of the cells its bounding disk overlaps
size_t binned_workspace_bytes(int max_T, int max_M);
cudaError_t build_bins(RolloutArgs& a, float half_len, float half_wid, float c_off, void* workspace,
                       cudaStream_t s);          // fills a.bins
cudaError_t launch_collide_binned(const RolloutArgs& a, cudaStream_t s);
cudaError_t launch_collide_poly(const RolloutArgs& a, cudaStream_t s);
cudaError_t build_bins_radius(RolloutArgs& a, double radius, void* workspace, cudaStream_t s);
cudaError_t launch_epilogue(const EpilogueArgs& e, cudaStream_t s);
void set_global_error(const char* msg);

}  // namespace npp
