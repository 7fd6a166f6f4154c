// npp_rollout.cuh -- the two kernels of one plan step, instantiated per
// network width by npp_rollout_w{16,32,64}.cu.
//
// The rollout of a sample (Sect. II-D "Sixth", Sect. IV) does not depend on
// its collision checks: a collision only ends the sample (cost +inf).  The
// step is therefore split into
//
//   traj_kernel    -- per sample: features (Eq. eq_def_stph), MLP
//                     a = X(s, theta) (Eq. eq_def_at), rate-limited controls,
//                     Euler step of the kinematic bicycle on the old state,
//                     for h = 0..T; writes the states [T+1][N], the applied
//                     controls [T][N] and the cost the sample has if it is
//                     collision-free.  A group of G lanes of one warp holds
//                     one sample's network in registers (each lane W/G hidden
//                     units: its rows of W1, W2 and columns of W3), generated
//                     straight from Philox and never stored.
//   collide_kernel -- per block of SB samples: the M obstacle points staged in
//                     shared memory in the EV-aligned frame at t, then for
//                     h = 0..T the still-live samples are checked against the
//                     points extrapolated at constant velocity (Sect. II-D
//                     items (i)-(iv)) with the polytope inequalities of Eq.
//                     eq_Apsietc_collAvoidIneqs; a sample leaves the live list
//                     at its first collision.  Finally the (class, cost,
//                     index) keys are reduced and folded into the global
//                     minimum with one 64-bit atomicMin per block.
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_device.cuh"
#include "npp_async.cuh"

namespace npp {

template <int W, int G_>
struct Shape {
    static constexpr int G = G_;                                     // lanes per sample
    static constexpr int U = W / G;                                  // hidden units per lane
    static constexpr int NT = 12 * W + W * W + 2;                    // parameters
    static constexpr int OFF_B1 = NIN * W;
    static constexpr int OFF_W2 = OFF_B1 + W;
    static constexpr int OFF_B2 = OFF_W2 + W * W;
    static constexpr int OFF_W3 = OFF_B2 + W;
    static constexpr int OFF_B3 = OFF_W3 + 2 * W;
    static_assert(U == 2 || U == 4, "2 or 4 hidden units per lane");
    static_assert(G <= 32 && (32 % G) == 0, "a group lives in one warp");
};

// Parameter source: Philox (sampled, optionally through the proposal) or
// memory (explicit / warm start).
struct ThetaSrc {
    const float* mem;     // row of this sample, or null -> sample
    SamplerKey key;
    Proposal prop;
    uint32_t n;
    // rows from memory are read element by element: a row of n_theta floats
    // starts at any 4-byte boundary
    __device__ __forceinline__ float4 quad(int i) const {     // i % 4 == 0
        if (mem) return make_float4(mem[i], mem[i + 1], mem[i + 2], mem[i + 3]);
        return sample_quad_mixed(key, prop, (uint32_t)i >> 2, n);
    }
    __device__ __forceinline__ float2 pair(int i) const {     // i % 2 == 0
        if (mem) return make_float2(mem[i], mem[i + 1]);
        return sample_pair_mixed(key, prop, (uint32_t)i, n);
    }
};

// Two FP32 values in one 64-bit register pair, for the packed FP32x2
// instructions: fma.rn.f32x2 rounds each half exactly as fmaf does.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi)
{
    unsigned long long d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// The weights of one lane: rows of W1 and W2 as packed pairs of adjacent
// inputs (2k, 2k + 1), the operands of the FP32x2 FMAs of the step.  With
// KSQ > 0 the last KSQ input quads of each W2 row live in shared memory
// instead of registers (fewer registers per thread, more warps per SM):
// unit j's quad QR + q of this lane at w2s[(j KSQ + q) G] as two packed
// pairs, lanes of a group adjacent (conflict-free 16-byte loads).
template <int W, int G, int KSQ = 0>
struct LaneNet {
    using S = Shape<W, G>;
    static constexpr int U = S::U;
    static constexpr int QR = W / 4 - KSQ;        // W2 input quads per unit in registers
    static_assert(KSQ >= 0 && KSQ < W / 4, "some quads in registers");
    unsigned long long w1p[U][NIN / 2];
    float b1[U];
    unsigned long long w2p[U][2 * QR];
    float b2[U];
    float w3[2][U], b3[2];
    ulonglong2* w2s;                              // this lane's slot of the shared part (KSQ > 0)

    __device__ __forceinline__ void put_w2(int j, int qi, float4 q) {
        if (qi < QR) {
            w2p[j][2 * qi] = f2_pack(q.x, q.y);
            w2p[j][2 * qi + 1] = f2_pack(q.z, q.w);
        } else {
            w2s[(j * KSQ + (qi - QR)) * G] = make_ulonglong2(f2_pack(q.x, q.y), f2_pack(q.z, q.w));
        }
    }
    // the packed pairs (4 qi, 4 qi + 1) and (4 qi + 2, 4 qi + 3) of unit j
    __device__ __forceinline__ ulonglong2 get_w2(int j, int qi) const {
        if (qi < QR) return make_ulonglong2(w2p[j][2 * qi], w2p[j][2 * qi + 1]);
        return w2s[(j * KSQ + (qi - QR)) * G];
    }

    // With KSQ > 0: the same values as load(), generated by rolled loops
    // (one copy of the sampler's code per loop instead of one per quad, so
    // the kernel's code stays small) and staged through this lane's own
    // shared W2 slots, which no other lane reads: first the W2 quads held in
    // registers, then the W1 quads and the bias / W3 pairs, last the shared
    // W2 quads straight into their slots.
    __device__ __forceinline__ void load_rolled(const ThetaSrc& src, int gl) {
        static_assert(KSQ > 0 && QR <= KSQ && U * (NIN / 4) + 2 * U + 1 <= U * KSQ, "staging fits the slots");
        constexpr int QW1 = NIN / 4;
#pragma unroll 1
        for (int it = 0; it < U * QR; ++it) {
            const int j = it / QR, qi = it - j * QR;
            const float4 q = src.quad(S::OFF_W2 + (gl * U + j) * W + 4 * qi);
            w2s[it * G] = make_ulonglong2(f2_pack(q.x, q.y), f2_pack(q.z, q.w));
        }
#pragma unroll
        for (int j = 0; j < U; ++j)
#pragma unroll
            for (int qi = 0; qi < QR; ++qi) {
                const ulonglong2 t = w2s[(j * QR + qi) * G];
                w2p[j][2 * qi] = t.x;
                w2p[j][2 * qi + 1] = t.y;
            }
#pragma unroll 1
        for (int it = 0; it < U * QW1 + 2 * U + 1; ++it) {
            if (it < U * QW1) {
                const int j = it / QW1, qi = it - j * QW1;
                const float4 q = src.quad((gl * U + j) * NIN + 4 * qi);
                w2s[it * G] = make_ulonglong2(f2_pack(q.x, q.y), f2_pack(q.z, q.w));
            } else {
                const int pj = it - U * QW1;
                int pidx = S::OFF_B3;
                if (pj < 2 * U) {
                    const int jj = gl * U + (pj >> 2) * 2, kind = pj & 3;
                    pidx = kind == 0 ? S::OFF_B1 + jj : kind == 1 ? S::OFF_B2 + jj
                         : kind == 2 ? S::OFF_W3 + jj : S::OFF_W3 + W + jj;
                }
                const float2 p = src.pair(pidx);
                w2s[it * G] = make_ulonglong2(f2_pack(p.x, p.y), 0ull);
            }
        }
#pragma unroll
        for (int j = 0; j < U; ++j)
#pragma unroll
            for (int qi = 0; qi < QW1; ++qi) {
                const ulonglong2 t = w2s[(j * QW1 + qi) * G];
                w1p[j][2 * qi] = t.x;
                w1p[j][2 * qi + 1] = t.y;
            }
#pragma unroll
        for (int j = 0; j < U; j += 2) {
            const int p0 = U * QW1 + (j >> 1) * 4;
            const float2 pb1 = f2_unpack(w2s[(p0 + 0) * G].x), pb2 = f2_unpack(w2s[(p0 + 1) * G].x);
            const float2 pw0 = f2_unpack(w2s[(p0 + 2) * G].x), pw1 = f2_unpack(w2s[(p0 + 3) * G].x);
            b1[j] = pb1.x; b1[j + 1] = pb1.y;
            b2[j] = pb2.x; b2[j + 1] = pb2.y;
            w3[0][j] = pw0.x; w3[0][j + 1] = pw0.y;
            w3[1][j] = pw1.x; w3[1][j + 1] = pw1.y;
        }
        const float2 pb3 = f2_unpack(w2s[(U * QW1 + 2 * U) * G].x);
        b3[0] = pb3.x; b3[1] = pb3.y;
#pragma unroll 1
        for (int it = 0; it < U * KSQ; ++it) {
            const int j = it / KSQ, qs = it - j * KSQ;
            const float4 q = src.quad(S::OFF_W2 + (gl * U + j) * W + 4 * (QR + qs));
            w2s[it * G] = make_ulonglong2(f2_pack(q.x, q.y), f2_pack(q.z, q.w));
        }
    }

    // lane gl of the group holds hidden units gl*U .. gl*U + U - 1
    __device__ __forceinline__ void load(const ThetaSrc& src, int gl) {
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int u = gl * U + j;
#pragma unroll
            for (int i = 0; i < NIN; i += 4) {
                const float4 q = src.quad(u * NIN + i);
                w1p[j][i / 2] = f2_pack(q.x, q.y);
                w1p[j][i / 2 + 1] = f2_pack(q.z, q.w);
            }
#pragma unroll
            for (int i = 0; i < W; i += 4) put_w2(j, i / 4, src.quad(S::OFF_W2 + u * W + i));
        }
#pragma unroll
        for (int j = 0; j < U; j += 2) {
            const float2 pb1 = src.pair(S::OFF_B1 + gl * U + j);
            b1[j] = pb1.x; b1[j + 1] = pb1.y;
            const float2 pb2 = src.pair(S::OFF_B2 + gl * U + j);
            b2[j] = pb2.x; b2[j + 1] = pb2.y;
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const float2 p = src.pair(S::OFF_W3 + o * W + gl * U + j);
                w3[o][j] = p.x; w3[o][j + 1] = p.y;
            }
        }
        const float2 pb3 = src.pair(S::OFF_B3);
        b3[0] = pb3.x; b3[1] = pb3.y;
    }

    // Parameters generated by a rolled loop into this lane's slots of a
    // shared staging area (slot k of the lane at st[k * TH]), then loaded
    // into registers: the same values as load(), with one copy of the
    // sampler's code instead of one per parameter quad.
    static constexpr int QW1 = NIN / 4, QW2 = W / 4, QPU = QW1 + QW2;
    static constexpr int NQUAD = U * QPU;                  // quads: W1 and W2 rows of the lane's units
    static constexpr int NPAIR = 2 * U + 1;                // pairs: b1, b2, W3 rows (per unit pair), b3
    static constexpr int SLOTS = 4 * NQUAD + 2 * NPAIR;

    template <int TH>
    __device__ __forceinline__ void load_staged(const ThetaSrc& src, int gl, float* st) {
        static_assert(KSQ == 0, "staged loading keeps every weight in registers");
#pragma unroll 1
        for (int it = 0; it < NQUAD; ++it) {
            const int j = it / QPU, q = it - j * QPU;
            const int u = gl * U + j;
            const int pidx = q < QW1 ? u * NIN + 4 * q : S::OFF_W2 + u * W + 4 * (q - QW1);
            const float4 v = src.quad(pidx);
            st[(4 * it + 0) * TH] = v.x;
            st[(4 * it + 1) * TH] = v.y;
            st[(4 * it + 2) * TH] = v.z;
            st[(4 * it + 3) * TH] = v.w;
        }
#pragma unroll 1
        for (int pj = 0; pj < NPAIR; ++pj) {
            int pidx = S::OFF_B3;
            if (pj < 2 * U) {
                const int jj = gl * U + (pj >> 2) * 2, kind = pj & 3;
                pidx = kind == 0 ? S::OFF_B1 + jj : kind == 1 ? S::OFF_B2 + jj
                     : kind == 2 ? S::OFF_W3 + jj : S::OFF_W3 + W + jj;
            }
            const float2 v = src.pair(pidx);
            st[(4 * NQUAD + 2 * pj + 0) * TH] = v.x;
            st[(4 * NQUAD + 2 * pj + 1) * TH] = v.y;
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
#pragma unroll
            for (int i = 0; i < NIN; i += 2)
                w1p[j][i / 2] = f2_pack(st[(4 * (j * QPU + i / 4) + i % 4) * TH],
                                        st[(4 * (j * QPU + i / 4) + i % 4 + 1) * TH]);
#pragma unroll
            for (int i = 0; i < W; i += 2)
                w2p[j][i / 2] = f2_pack(st[(4 * (j * QPU + QW1 + i / 4) + i % 4) * TH],
                                        st[(4 * (j * QPU + QW1 + i / 4) + i % 4 + 1) * TH]);
        }
#pragma unroll
        for (int j = 0; j < U; j += 2) {
            const int p0 = 4 * NQUAD + 2 * ((j >> 1) * 4);
            b1[j] = st[(p0 + 0) * TH]; b1[j + 1] = st[(p0 + 1) * TH];
            b2[j] = st[(p0 + 2) * TH]; b2[j + 1] = st[(p0 + 3) * TH];
            w3[0][j] = st[(p0 + 4) * TH]; w3[0][j + 1] = st[(p0 + 5) * TH];
            w3[1][j] = st[(p0 + 6) * TH]; w3[1][j + 1] = st[(p0 + 7) * TH];
        }
        b3[0] = st[(4 * NQUAD + 2 * (2 * U)) * TH];
        b3[1] = st[(4 * NQUAD + 2 * (2 * U) + 1) * TH];
    }
};

// Every rounding of the rollout step below is written out (fmaf, __fmul_rn,
// __fadd_rn, __fsub_rn): the compiler may not contract a product and a sum
// differently in different kernels, so every kernel that rolls a sample out
// (trajectories, fused check, batch, winner re-roll) produces the same bits.
__device__ __forceinline__ float wrap_pi(float a)
{
    const float TWO_PI = 6.28318530717958647692f;
    const float INV_TWO_PI = 0.15915494309189533577f;
    return fmaf(-TWO_PI, floorf(__fmul_rn(__fadd_rn(a, 3.14159265358979323846f), INV_TWO_PI)), a);
}

// The rectangle's four inequalities at state (x, y, phi), scaled so that a
// point p is inside iff |A px + B py - C| < 2 and |D px + E py - F| < 2: rows
// along and across the heading divided by the half length / width, times 2
// (an exact scaling).  |v| < 2 holds exactly when bit 30 of v's IEEE pattern
// is clear, so "both inside" is bit 30 of (xi | eta) clear: one 3-input logic
// op per point-sample pair accumulates "some point inside".
// (Rounding fixed by explicit fmas and round-to-nearest products, so that the
// rows stored by the trajectory kernel and the rows the fused check computes
// are the same bits.)
__device__ __forceinline__ void coef_rows(const DevCfg& c, float x, float y, float sp, float cp, float4& A,
                                          float2& B)
{
    const float sl = 2.0f * c.ihl, sw = 2.0f * c.ihw;
    const float along = fmaf(cp, x, fmaf(sp, y, c.c_off));
    const float across = fmaf(-sp, x, __fmul_rn(cp, y));
    A = make_float4(__fmul_rn(cp, sl), __fmul_rn(sp, sl), -__fmul_rn(along, sl), -__fmul_rn(sp, sw));
    B = make_float2(__fmul_rn(cp, sw), -__fmul_rn(across, sw));
}

// The rows of a stored state z = (x, y, phi, v): the trajectory kernel's own
// arithmetic on the same FP32 values, so a collision kernel that recomputes
// them from the stored state gets the same bits the rollout had (and no
// rows need to be stored).
__device__ __forceinline__ void rows_of_state(const DevCfg& c, const float4& z, float4& A, float2& B)
{
    float sp, cp;
    sincos_r(z.z, sp, cp);
    coef_rows(c, z.x, z.y, sp, cp, A, B);
}

__device__ __forceinline__ void write_coef(float4* coefA, float2* coefB, const DevCfg& c,
                                           long long idx, float x, float y, float sp, float cp)
{
    float4 A;
    float2 B;
    coef_rows(c, x, y, sp, cp, A, B);
    coefA[idx] = A;
    coefB[idx] = B;
}

// The step at which a sample is discarded: the earlier of its first colliding
// step fh and its first speed-violating step vfirst[n] (either -1 for none;
// vfirst null when speed limits are off).
__device__ __forceinline__ int discard_step(const int* vfirst, long long n, int fh)
{
    if (!vfirst) return fh;
    const int hv = vfirst[n];
    return (hv >= 0 && (fh < 0 || hv < fh)) ? hv : fh;
}

// One state of one sample against one step's grid, checked by an 8-lane
// group of a warp (four such items per warp at a time): the candidates of
// the at most five cell rows the state's disk overlaps, strided over the
// group's lanes, each lane first issuing the loads of up to R candidates and
// then testing them with the brute-force kernels' per-point test (the rest,
// rarely any, one by one).  Every lane of the warp calls it (warp-wide
// reduction inside); the lanes of an item that is not ok test nothing.
// Returns the lane's verdict (the item's is the OR over its 8 lanes) and
// counts the lane's candidate tests in ntest.
constexpr int BIN_ITEM_LANES = 8;

__device__ __forceinline__ bool inside_rows(const float4& A, const float2& B, float2 p)
{
    const float xi = fmaf(A.x, p.x, fmaf(A.y, p.y, A.z));
    const float et = fmaf(A.w, p.x, fmaf(B.x, p.y, B.y));
    return !(((__float_as_uint(xi) | __float_as_uint(et)) >> 30) & 1u);
}

template <int R>
__device__ __forceinline__ bool binned_item_inside(const DevCfg& c, const BinView& g, const float4& z, int h,
                                                   bool ok, int gl, unsigned& ntest)
{
    constexpr int L = BIN_ITEM_LANES;
    float4 ca;
    float2 cb;
    rows_of_state(c, z, ca, cb);
    CandRows cr = {};
    if (ok) cr = cand_rows(g.cell_start + (size_t)h * BIN_CS_STRIDE, g, z.x, z.y, g.reach);
    const float2* pts = g.pts + (size_t)(ok ? h : 0) * g.M;
    const int total = cr.total;
    float2 pr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = gl + r * L;
        pr[r] = k < total ? pts[cr.index(k)] : make_float2(0.f, 0.f);
    }
    bool inside = false;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (gl + r * L < total) {
            inside |= inside_rows(ca, cb, pr[r]);
            ++ntest;
        }
    constexpr int PRE = R * L;
    const int rest = total > PRE ? (total - PRE + L - 1) / L : 0;
    const int maxr = __reduce_max_sync(FULL, rest);
    for (int it = 0; it < maxr; ++it) {
        const int k = PRE + it * L + gl;
        if (it < rest && k < total) {
            inside |= inside_rows(ca, cb, pts[cr.index(k)]);
            ++ntest;
        }
    }
    return inside;
}


// The same item check with the candidates taken row by row: each of the
// (at most five) cell rows' runs strided over the item's 8 lanes, RR
// candidates per row and lane loaded ahead (longer rows one pass at a time
// after them).  No candidate index search (the run of a row is contiguous),
// at the cost of lanes idle in short rows; the same candidates, tests and
// verdict as binned_item_inside.  Measured on GB300 in the two-kernel check:
// 0.32 against 0.43 ms at the large workload (8 candidates per state), 0.077
// against 0.078 ms on the course (25); inside the trajectory kernel's
// window check it costs registers (spills) and is not used there.
template <int RR>
__device__ __forceinline__ bool binned_rows_inside(const BinView& g, const int* __restrict__ cs,
                                                   const float2* __restrict__ pts, const float4& ca,
                                                   const float2& cb, float qx, float qy, float reach, bool ok,
                                                   int gl, unsigned& ntest)
{
    constexpr int L = BIN_ITEM_LANES;
    CandRows cr = {};
    if (ok) cr = cand_rows(cs, g, qx, qy, reach);
    int len[BIN_MAX_ROWS];
#pragma unroll
    for (int r = 0; r < BIN_MAX_ROWS; ++r) len[r] = cr.e[r] - (r > 0 ? cr.e[r - 1] : 0);
    float2 pr[BIN_MAX_ROWS][RR];
#pragma unroll
    for (int r = 0; r < BIN_MAX_ROWS; ++r)
#pragma unroll
        for (int t = 0; t < RR; ++t) {
            const int k = gl + t * L;
            pr[r][t] = k < len[r] ? pts[cr.b[r] + k] : make_float2(0.f, 0.f);
        }
    bool inside = false;
    int rest = 0;
#pragma unroll
    for (int r = 0; r < BIN_MAX_ROWS; ++r) {
#pragma unroll
        for (int t = 0; t < RR; ++t)
            if (gl + t * L < len[r]) {
                inside |= inside_rows(ca, cb, pr[r][t]);
                ++ntest;
            }
        rest = max(rest, len[r] - RR * L);
    }
    const int maxr = __reduce_max_sync(FULL, (rest + L - 1) / L);
    for (int it = 0; it < maxr; ++it) {
#pragma unroll
        for (int r = 0; r < BIN_MAX_ROWS; ++r) {
            const int k = RR * L + it * L + gl;
            if (k < len[r]) {
                inside |= inside_rows(ca, cb, pts[cr.b[r] + k]);
                ++ntest;
            }
        }
    }
    return inside;
}

// the row-wise item check of state z at step h of grid g (its rows
// recomputed, the query disk around its reference point)
template <int RR>
__device__ __forceinline__ bool binned_item_inside_rows(const DevCfg& c, const BinView& g, const float4& z, int h,
                                                        bool ok, int gl, unsigned& ntest)
{
    float4 ca;
    float2 cb;
    rows_of_state(c, z, ca, cb);
    return binned_rows_inside<RR>(g, g.cell_start + (size_t)(ok ? h : 0) * BIN_CS_STRIDE,
                                  g.pts + (size_t)(ok ? h : 0) * g.M, ca, cb, z.x, z.y, g.reach, ok, gl, ntest);
}

// ------------------------------------------------------------------ bins
// The grid of one horizon step (time tau) built by one block of THREADS
// threads: counting sort of the extrapolated EV-frame points by cell (counts
// in shared memory cnt[BIN_NCELL], exclusive scan, scatter).  Writes the
// step's cell-start table cs[BIN_NCELL + 1] and the sorted points out[M].
template <int THREADS>
__device__ __forceinline__ void build_step_bins(const float4* __restrict__ obs, int M, float x0, float y0, float s0,
                                                float c0, float tau, const BinView& g, int* __restrict__ cs,
                                                float2* __restrict__ out, int* cnt, int* run_tot)
{
    for (int i = threadIdx.x; i < BIN_NCELL; i += THREADS) cnt[i] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < M; j += THREADS) {
        float ex, ey, evx, evy;
        ev_point(obs[j], x0, y0, s0, c0, ex, ey, evx, evy);
        const float px = fmaf(tau, evx, ex), py = fmaf(tau, evy, ey);
        atomicAdd(&cnt[bin_cell(py, g) * BIN_DIM + bin_cell(px, g)], 1);
    }
    __syncthreads();
    // exclusive scan: each thread scans a contiguous run, then warp 0 scans
    // the run totals
    constexpr int RUN = BIN_NCELL / THREADS;
    const int base = threadIdx.x * RUN;
    int acc = 0;
    for (int k = 0; k < RUN; ++k) { const int v = cnt[base + k]; cnt[base + k] = acc; acc += v; }
    run_tot[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int PER = THREADS / 32;
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
    for (int i = threadIdx.x; i < BIN_NCELL; i += THREADS) cs[i] = cnt[i];
    if (threadIdx.x == 0) cs[BIN_NCELL] = M;
    __syncthreads();
    // scatter (order within a cell is arbitrary; the test is an OR)
    for (int j = threadIdx.x; j < M; j += THREADS) {
        float ex, ey, evx, evy;
        ev_point(obs[j], x0, y0, s0, c0, ex, ey, evx, evy);
        const float px = fmaf(tau, evx, ex), py = fmaf(tau, evy, ey);
        const int pos = atomicAdd(&cnt[bin_cell(py, g) * BIN_DIM + bin_cell(px, g)], 1);
        out[pos] = make_float2(px, py);
    }
}

// A grid whose cell exceeds the diameter of the query disk: the rectangle's
// circumradius plus |c_off|, plus a margin against rounding of positions of
// O(100) m (host side).
inline BinView make_bin_grid_radius(double R)
{
    // query radius R + 0.05 (rounding of positions of O(100) m); cells a
    // little wider than half of it, so a query spans at most five cells per
    // axis (a query square of side 2r over cells of width c covers (2r + c)^2
    // of candidates on average: 6.25 r^2 here against 16 r^2 for c = 2r;
    // measured on GB300: c = r/2 beats c = r and c = 2r)
    const double cell = 0.5 * (R + 0.15);
    BinView g;
    g.inv_cell = (float)(1.0 / cell);
    g.x0 = (float)(-0.5 * BIN_DIM * cell);
    g.reach = (float)(R + 0.05);
    g.cell_start = nullptr;
    g.pts = nullptr;
    g.M = 0;
    return g;
}

// the rectangle lies in the disk of its circumradius plus |c_off|
inline BinView make_bin_grid(float half_len, float half_wid, float c_off)
{
    return make_bin_grid_radius(std::sqrt((double)half_len * half_len + (double)half_wid * half_wid) +
                                std::fabs((double)c_off));
}

// ------------------------------------------------------------------ traj
template <int W, int G, int NW>
struct TrajKernel {
    static constexpr int THREADS = NW * 32;
    static constexpr int B = THREADS / G;             // samples per block
};

// One planning instance as the trajectory code sees it.  Records of sample n
// at step h go to index h * rec_stride + n - rec_shift (states, controls);
// coefficient rows to coef_base + h * N + n; the free cost to jfree[n].  Any
// pointer may be null (nothing written).
struct TrajJob {
    StepIn si;
    SamplerKey key;               // t_index resolved
    const float* theta;           // explicit rows [N][n_theta] or null
    const float* warm;            // replaces sample 0 when non-null (and si.warm_ok)
    Proposal prop;                // sampling proposal (mu null: none)
    int N, T;
    float4* traj;                 // [T+1] x stride
    float2* ctrl;                 // [T] x stride
    long long rec_stride, rec_shift;
    float4* coefA;                // coefficient rows (scaled inequalities)
    float2* coefB;
    long long coef_base;
    float* jfree;
    int* vfirst;                  // first speed-violating step per sample (speed limits on), or null
    const BinView* bins;          // grids of the windowed check (traj_sample_windowed)
    ulonglong2* w2s;              // this lane's slot of the shared W2 quads (LaneNet KSQ > 0), or null
    float* stage;                 // this thread's slot 0 of a staging area (stride stage_th), or null
    // One chunk of the horizon: steps h_lo .. h_hi - 1 from the stored state
    // h_lo and the carried (last controls, effort, first speed violation);
    // h_hi < 0: the whole horizon from the initial state
    int h_lo = 0, h_hi = -1;
    float4* carry = nullptr;      // [N] carried values between chunks
};

// Result of a fused rollout, uniform over the sample's group: the first
// colliding step (-1 if none) and the cost if collision-free.
struct FusedOut {
    int first_hit;
    float cost;
};

// The goal in the EV frame at t and the constants of one rollout.
struct GoalEV {
    float xi, eta, phi, v;
};

__device__ __forceinline__ GoalEV goal_ev(const StepIn& si)
{
    float s0, c0;
    sincosf(si.phi0, &s0, &c0);
    const float gdx = __fsub_rn(si.gx, si.x0), gdy = __fsub_rn(si.gy, si.y0);
    GoalEV g;
    g.xi = fmaf(c0, gdx, __fmul_rn(s0, gdy));
    g.eta = fmaf(-s0, gdx, __fmul_rn(c0, gdy));
    g.phi = __fsub_rn(si.gphi, si.phi0);
    g.v = si.gv;
    return g;
}

// The network of sample n (valid: n < N) loaded into the lanes of its group.
template <int W, int G, int STAGE_TH, int KSQ = 0>
__device__ __forceinline__ void load_net(LaneNet<W, G, KSQ>& net, const TrajJob& job, int n, bool valid, int gl)
{
    net.w2s = job.w2s;
    ThetaSrc src;
    src.key = job.key;
    src.prop = job.prop;
    src.n = (uint32_t)(valid ? n : 0);
    src.mem = nullptr;
    if (job.theta) src.mem = job.theta + (size_t)(valid ? n : 0) * Shape<W, G>::NT;
    else if (job.warm && n == 0 && job.si.warm_ok) src.mem = job.warm;
    if constexpr (STAGE_TH > 0) net.template load_staged<STAGE_TH>(src, gl, job.stage);
    else if constexpr (KSQ > 0) net.load_rolled(src, gl);
    else net.load(src, gl);
}

// One control step h from state (x, y, ph, v) whose heading has sine sp and
// cosine cp: features (Eq. eq_def_stph), network a = X(s, theta) (Eq.
// eq_def_at) by the G lanes of the group (hrow: the group's W-float shared
// exchange row), rate-limited controls, effort, Euler step of the kinematic
// bicycle on the old state (Sect. IV).  Updates the state, the last
// controls, the effort E and rem = T - h; returns the applied controls.
template <int W, int G, bool VAR, int KSQ = 0>
__device__ __forceinline__ float2 control_step(const DevCfg& c, const LaneNet<W, G, KSQ>& net, const GoalEV& g,
                                               float invT, int gl, float* hrow, float sp, float cp, float& x,
                                               float& y, float& ph, float& v, float& ap0, float& ap1, float& E,
                                               float& rem)
{
    constexpr int U = Shape<W, G>::U;
    float s[NIN];
    if (VAR && c.body_frame) {
        // goal offset in the vehicle's frame at t+h
        const float dgx = __fsub_rn(g.xi, x), dgy = __fsub_rn(g.eta, y);
        s[0] = __fmul_rn(fmaf(cp, dgx, __fmul_rn(sp, dgy)), c.idxi);
        s[1] = __fmul_rn(fmaf(-sp, dgx, __fmul_rn(cp, dgy)), c.ideta);
    } else {
        s[0] = __fmul_rn(__fsub_rn(g.xi, x), c.idxi);
        s[1] = __fmul_rn(__fsub_rn(g.eta, y), c.ideta);
    }
    s[2] = __fmul_rn(wrap_pi(__fsub_rn(g.phi, ph)), c.idphi);
    s[3] = __fmul_rn(__fsub_rn(g.v, v), c.idv);
    s[4] = ap0;
    s[5] = ap1;
    s[6] = __fmul_rn(v, c.idv);
    s[7] = __fmul_rn(rem, invT);
    rem = __fsub_rn(rem, 1.0f);
    // layer 1: the even and odd inputs as the two halves of FP32x2 FMAs,
    // then their sum and the bias
    unsigned long long sp2[NIN / 2];
#pragma unroll
    for (int i = 0; i < NIN / 2; ++i) sp2[i] = f2_pack(s[2 * i], s[2 * i + 1]);
    float h1[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
        unsigned long long q = f2_fma(net.w1p[j][0], sp2[0], 0ull);
#pragma unroll
        for (int i = 1; i < NIN / 2; ++i) q = f2_fma(net.w1p[j][i], sp2[i], q);
        const float2 qq = f2_unpack(q);
        h1[j] = tanh_r(__fadd_rn(__fadd_rn(qq.x, qq.y), net.b1[j]));
    }
#pragma unroll
    for (int j = 0; j < U; ++j) hrow[gl * U + j] = h1[j];
    __syncwarp();
    // layer 2: each unit's dot product as four interleaved partial sums
    // (inputs i = 4q + r go to partial r), added pairwise with the bias
    // last: independent FMA chains keep the pipe busy
    // (partials 0, 1 and 2, 3 as packed pairs: two FP32x2 FMAs per input
    // quad, each half rounded as a separate fmaf)
    unsigned long long p01[U], p23[U];
#pragma unroll
    for (int j = 0; j < U; ++j) p01[j] = p23[j] = 0ull;
    const float4* hrow4 = reinterpret_cast<const float4*>(hrow);
#pragma unroll
    for (int i = 0; i < W / 4; ++i) {
        const float4 hv = hrow4[i];
        const unsigned long long h01 = f2_pack(hv.x, hv.y), h23 = f2_pack(hv.z, hv.w);
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const ulonglong2 w = net.get_w2(j, i);
            p01[j] = f2_fma(w.x, h01, p01[j]);
            p23[j] = f2_fma(w.y, h23, p23[j]);
        }
    }
    __syncwarp();
    float acc2[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
        const float2 q01 = f2_unpack(p01[j]), q23 = f2_unpack(p23[j]);
        acc2[j] = __fadd_rn(__fadd_rn(__fadd_rn(q01.x, q01.y), __fadd_rn(q23.x, q23.y)), net.b2[j]);
    }
    // layer 3: a fixed pairwise tree over the hidden units -- leaves
    // w_2i h_2i + w_2i+1 h_2i+1 (one fma), then sums of neighbours -- so
    // the value does not depend on how many units a lane holds
    float h2[U];
#pragma unroll
    for (int j = 0; j < U; ++j) h2[j] = tanh_r(acc2[j]);
    float p0 = fmaf(net.w3[0][1], h2[1], __fmul_rn(net.w3[0][0], h2[0]));
    float p1 = fmaf(net.w3[1][1], h2[1], __fmul_rn(net.w3[1][0], h2[0]));
    if constexpr (U == 4) {
        p0 = __fadd_rn(p0, fmaf(net.w3[0][3], h2[3], __fmul_rn(net.w3[0][2], h2[2])));
        p1 = __fadd_rn(p1, fmaf(net.w3[1][3], h2[3], __fmul_rn(net.w3[1][2], h2[2])));
    }
#pragma unroll
    for (int off = 1; off < G; off <<= 1) {
        p0 = __fadd_rn(p0, __shfl_xor_sync(FULL, p0, off));
        p1 = __fadd_rn(p1, __shfl_xor_sync(FULL, p1, off));
    }
    const float ar0 = tanh_r(__fadd_rn(net.b3[0], p0));
    const float ar1 = tanh_r(__fadd_rn(net.b3[1], p1));
    float a0 = fminf(fmaxf(ar0, __fsub_rn(ap0, c.r_rate)), __fadd_rn(ap0, c.r_rate));
    a0 = fminf(fmaxf(a0, -1.0f), 1.0f);
    const float a1 = ar1;
    E = __fadd_rn(E, fmaf(a0, a0, __fmul_rn(a1, a1)));
    const float td = tan_r(__fmul_rn(c.delta_max, a0));
    const float tb = __fmul_rn(c.lrL, td);
    const float dv = __fmul_rn(c.Ts, v);
    x = fmaf(dv, fmaf(-sp, tb, cp), x);
    y = fmaf(dv, fmaf(cp, tb, sp), y);
    ph = fmaf(__fmul_rn(dv, td), c.iL, ph);
    v = fmaf(c.Ts, fmaf(c.uhalf, a1, c.umid), v);
    ap0 = a0;
    ap1 = a1;
    return make_float2(a0, a1);
}

// cost of a collision-free rollout from its final state and effort
__device__ __forceinline__ float final_cost(const DevCfg& c, const GoalEV& g, float x, float y, float ph, float v,
                                            float E, float invT)
{
    const float dx = __fsub_rn(x, g.xi), dy = __fsub_rn(y, g.eta);
    const float d = __fsqrt_rn(fmaf(dx, dx, __fmul_rn(dy, dy)));
    const float e = __fmul_rn(__fmul_rn(c.w_effort, E), invT);
    return fmaf(c.w_pos, d, fmaf(c.w_phi, fabsf(wrap_pi(__fsub_rn(ph, g.phi))),
                                 fmaf(c.w_v, fabsf(__fsub_rn(v, g.v)), e)));
}

// The trajectory of sample n (valid: n < N) computed by the G lanes of a
// group (lane gl); hrow is the group's W-float shared exchange row.  Writes
// the records the job asks for (states, controls, scaled inequality rows,
// cost if collision-free, first speed-violating step).  VAR: the variants
// of c (body-frame goal offsets, speed limits) are honoured; without it the
// kernel is the plain rollout, and the launchers pick VAR whenever c turns
// a variant on.
template <int W, int G, int STAGE_TH = 0, bool VAR = false, int KSQ = 0>
__device__ __forceinline__ void traj_sample(const DevCfg& c, const TrajJob& job, int n, bool valid, int gl,
                                            float* hrow)
{
    const GoalEV g = goal_ev(job.si);
    LaneNet<W, G, KSQ> net;
    load_net<W, G, STAGE_TH, KSQ>(net, job, n, valid, gl);

    float x = 0.f, y = 0.f, ph = 0.f, v = job.si.v0, ap0 = job.si.ap0, ap1 = job.si.ap1, E = 0.f;
    const int T = job.T, N = job.N;
    const float invT = 1.0f / (float)T;
    const bool writer = valid && gl == 0;
    const long long rec = (long long)n - job.rec_shift;
    int vbad = -1;                       // first state h >= 1 whose speed is outside the limits
    const int h_lo = job.h_lo, h_hi = job.h_hi < 0 ? T : job.h_hi;
    if (h_lo > 0) {
        // a later chunk: the state the previous chunk stored, and what it
        // carried (the same FP32 values the whole-horizon loop would hold)
        const float4 z = job.traj[h_lo * job.rec_stride + (valid ? rec : 0)];
        const float4 cv = job.carry[valid ? n : 0];
        x = z.x; y = z.y; ph = z.z; v = z.w;
        ap0 = cv.x; ap1 = cv.y; E = cv.z;
        vbad = __float_as_int(cv.w);
    }
    float rem = (float)(T - h_lo);       // T - h, exact in FP32
    for (int h = h_lo; h < h_hi; ++h) {
        float sp, cp;
        sincos_r(ph, sp, cp);
        if constexpr (VAR) {
            if (c.vlim && h > 0 && vbad < 0 && !(v >= c.v_lo && v <= c.v_hi)) vbad = h;
        }
        // pointer tests are uniform over the kernel; only the stores
        // depend on the writer lane
        if (job.traj && writer) job.traj[h * job.rec_stride + rec] = make_float4(x, y, ph, v);
        if (job.coefA) {
            float4 A;
            float2 B;
            coef_rows(c, x, y, sp, cp, A, B);
            if (writer) {
                const long long ci = job.coef_base + (long long)h * N + n;
                job.coefA[ci] = A;
                job.coefB[ci] = B;
            }
        }
        const float2 a = control_step<W, G, VAR, KSQ>(c, net, g, invT, gl, hrow, sp, cp, x, y, ph, v, ap0, ap1,
                                                      E, rem);
        if (writer && job.ctrl) job.ctrl[h * job.rec_stride + rec] = a;
    }
    if (h_hi < T) {
        // end of a chunk: state h_hi (checked with this chunk, the next
        // chunk's start) and the carried values
        if (writer) {
            job.traj[h_hi * job.rec_stride + rec] = make_float4(x, y, ph, v);
            job.carry[n] = make_float4(ap0, ap1, E, __int_as_float(vbad));
            if constexpr (VAR) {
                if (job.vfirst) job.vfirst[n] = vbad;
            }
        }
        return;
    }
    if constexpr (VAR) {
        if (c.vlim && T > 0 && vbad < 0 && !(v >= c.v_lo && v <= c.v_hi)) vbad = T;
    }
    if (writer) {
        if constexpr (VAR) {
            if (job.vfirst) job.vfirst[n] = vbad;
        }
        float sp, cp;
        sincos_r(ph, sp, cp);
        if (job.traj) job.traj[T * job.rec_stride + rec] = make_float4(x, y, ph, v);
        if (job.coefA) write_coef(job.coefA, job.coefB, c, job.coef_base + (long long)T * N + n, x, y, sp, cp);
        if (job.jfree) job.jfree[n] = final_cost(c, g, x, y, ph, v, E, invT);
    }
}

// ------------------------------------------------------------------ fused: windowed check
// The rollout of sample n with the binned check done by the trajectory
// warp itself, one window of CW states at a time: the group rolls its
// sample through steps h0 .. h0 + CW - 1 (storing the states and controls
// the caller asked for, and the states in the warp's shared window), then
// the warp checks the window's states of every group still alive, four
// (group, state) items at a time with the binned check's item code
// (binned_item_inside: the same grids, rows and per-point test, so the same
// flags), the earliest colliding state of a group ending its sample.  A
// sample is therefore rolled out at most CW - 1 steps past its first
// collision, its parameters generated once, and the loop ends once no group
// of the warp is alive.  VAR as in traj_sample (a sample is discarded at its
// first state h >= 1 whose speed is out of range, unless an earlier state
// collides).  wnd: the warp's [32/G][CW] states; steps counts the control
// steps the warp computed (lane 0 of each valid group), ntest / nstate the
// check's candidate tests and states.
template <int W, int G, int STAGE_TH, bool VAR, int KSQ, int CW, int R>
__device__ __forceinline__ FusedOut traj_sample_windowed(const DevCfg& c, const TrajJob& job, int n, bool valid,
                                                         int gl, float* hrow, float4* wnd, unsigned& steps,
                                                         unsigned& ntest, unsigned& nstate)
{
    constexpr int NG = 32 / G;                 // groups (samples) per warp
    constexpr int SPI = 4 / NG;                // states of a group per check round
    static_assert(NG <= 4 && 32 % G == 0, "at most four groups per warp");
    const int lane = threadIdx.x & 31, grp = lane / G;
    const GoalEV g = goal_ev(job.si);
    LaneNet<W, G, KSQ> net;
    load_net<W, G, STAGE_TH, KSQ>(net, job, n, valid, gl);
    const BinView& bv = *job.bins;

    float x = 0.f, y = 0.f, ph = 0.f, v = job.si.v0, ap0 = job.si.ap0, ap1 = job.si.ap1, E = 0.f;
    const int T = job.T;
    const float invT = 1.0f / (float)T;
    const bool writer = valid && gl == 0;
    const long long rec = n;
    int vbad = -1;
    float rem = (float)T;
    bool alive = valid;
    int fh = -1;
    for (int h0 = 0; h0 <= T && __any_sync(FULL, alive); h0 += CW) {
        const int ns = min(CW, T + 1 - h0);    // states h0 .. h0 + ns - 1
        for (int j = 0; j < ns; ++j) {
            const int h = h0 + j;
            float sp, cp;
            sincos_r(ph, sp, cp);
            if constexpr (VAR) {
                if (c.vlim && h > 0 && vbad < 0 && !(v >= c.v_lo && v <= c.v_hi)) vbad = h;
            }
            const float4 z = make_float4(x, y, ph, v);
            if (gl == 0) wnd[grp * CW + j] = z;
            if (writer && alive && job.traj) job.traj[h * job.rec_stride + rec] = z;
            if (h < T) {
                const float2 a = control_step<W, G, VAR, KSQ>(c, net, g, invT, gl, hrow, sp, cp, x, y, ph, v,
                                                              ap0, ap1, E, rem);
                if (writer && alive && job.ctrl) job.ctrl[h * job.rec_stride + rec] = a;
                ++steps;
            }
        }
        __syncwarp();
        // the window's check: round si0 takes items q = lane / 8 (group
        // q % NG, state si0 + q / NG), so a group's items come in order
        const unsigned amask = __ballot_sync(FULL, alive);
        int first = -1;                        // earliest colliding state of this lane's group (slot)
        for (int si0 = 0; si0 < ns; si0 += SPI) {
            const int q = lane / BIN_ITEM_LANES, il = lane % BIN_ITEM_LANES;
            const int bi = q % NG, si = si0 + q / NG;
            const bool ok = si < ns && ((amask >> (bi * G)) & 1u) != 0u;
            const float4 z = ok ? wnd[bi * CW + si] : make_float4(0.f, 0.f, 0.f, 0.f);
            nstate += (ok && il == 0) ? 1u : 0u;
            const bool in = binned_item_inside<R>(c, bv, z, h0 + si, ok, il, ntest);
            const unsigned bal = __ballot_sync(FULL, in);
            if (first < 0) {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
                    if (first < 0 && qq % NG == grp && ((bal >> (qq * BIN_ITEM_LANES)) & 0xFFu) != 0u)
                        first = si0 + qq / NG;
            }
            if (__all_sync(FULL, !alive || first >= 0)) break;
        }
        __syncwarp();                          // the window is rewritten next
        int d = first >= 0 ? h0 + first : -1;
        if constexpr (VAR) {
            if (vbad >= 0 && (d < 0 || vbad < d)) d = vbad;
        }
        if (alive && d >= 0) {
            alive = false;
            fh = d;
        }
    }
    FusedOut out;
    out.first_hit = valid ? fh : -1;
    out.cost = __int_as_float(0x7f800000);
    if (valid && alive) out.cost = final_cost(c, g, x, y, ph, v, E, invT);
    return out;
}

template <int W, int G, int NW, int MINB = 1, bool VAR = false, int KSQ = 0>
__global__ void __launch_bounds__(NW * 32, MINB) traj_kernel(const RolloutArgs a)
{
    constexpr int B = TrajKernel<W, G, NW>::B;
    __shared__ __align__(16) float hx_all[B * W];
    // [LaneNet::SLOTS][NW * 32] floats of parameter staging when W == 32;
    // with KSQ > 0 the shared W2 quads, [group][U][KSQ][G] of 16 bytes
    extern __shared__ __align__(16) float stage_all[];
    const int tid = threadIdx.x;
    const int b = tid / G, gl = tid % G;
    int n = blockIdx.x * B + b;
    bool valid = n < a.N;
    if (a.live_in) {
        // a later chunk: the samples still collision-free, listed
        const int cnt = *a.live_n_in;
        if ((int)blockIdx.x * B >= cnt) return;            // the whole block idle (no block barrier below)
        valid = n < cnt;
        n = valid ? a.live_in[n] : 0;
    }
    TrajJob job;
    job.si = step_in(a);
    job.key = a.key;
    job.key.t_index = job.si.t_index;
    job.theta = a.theta;
    job.warm = a.warm;
    job.prop = a.prop;
    job.N = a.N;
    job.T = a.T;
    job.traj = a.traj;
    job.ctrl = a.ctrl;
    job.rec_stride = a.N;
    job.rec_shift = 0;
    job.coefA = a.coefA;
    job.coefB = a.coefB;
    job.coef_base = 0;
    job.jfree = a.jfree;
    job.vfirst = a.c.vlim ? a.vfirst : nullptr;
    job.bins = nullptr;
    job.stage = stage_all + tid;
    job.w2s = nullptr;
    if constexpr (KSQ > 0)
        job.w2s = reinterpret_cast<ulonglong2*>(stage_all) + (size_t)b * (Shape<W, G>::U * KSQ * G) + gl;
    // staged parameter generation pays at W = 32 (measured on GB300: 11 %
    // faster at T = 40); at W = 16 and 64 the direct load is faster
    constexpr int STAGE_TH = (W == 32 && KSQ == 0) ? NW * 32 : 0;
    if (a.chunk_hi > 0) {
        job.h_lo = a.chunk_lo;
        job.h_hi = a.chunk_hi;
        job.carry = a.carry;
    }
    traj_sample<W, G, STAGE_TH, VAR, KSQ>(a.c, job, n, valid, gl, hx_all + b * W);
    // measurement: sample-steps computed (timing on)
    if (a.counts && valid && gl == 0)
        atomicAdd(a.counts + 2, (unsigned long long)((a.chunk_hi > 0 ? a.chunk_hi : a.T) - a.chunk_lo));
}

// Shared memory a trajectory block needs beyond its hidden rows: the
// parameter staging (width 32, every weight in registers) or the shared
// layer-2 quads (KSQ > 0), in bytes.
template <int W, int G, int NW, int KSQ>
__host__ __device__ constexpr int traj_stage_bytes()
{
    return KSQ > 0 ? NW * 32 * Shape<W, G>::U * KSQ * 16
         : W == 32 ? LaneNet<W, G>::SLOTS * NW * 32 * (int)sizeof(float) : 0;
}

// Trajectories with the binned check done window by window by the
// trajectory warps themselves (traj_sample_windowed; the grids are built
// before the launch): per sample its first collision and cost, written and
// folded into the (class, cost, index) minimum; states and controls stored
// up to the window of a sample's first collision, which holds every row the
// winner epilogue reads.
template <int W, int G, int NW, int MINB = 1, bool VAR = false, int KSQ = 0, int CW = 16, int R = 4>
__global__ void __launch_bounds__(NW * 32, MINB) fused_kernel(const RolloutArgs a)
{
    constexpr int B = TrajKernel<W, G, NW>::B;
    __shared__ __align__(16) float hx_all[B * W];
    // the staging or shared W2 quads of traj_kernel, then each warp's window
    extern __shared__ __align__(16) float stage_all[];
    const int tid = threadIdx.x;
    const int b = tid / G, gl = tid % G;
    const int n = blockIdx.x * B + b;
    const bool valid = n < a.N;
    TrajJob job;
    job.si = step_in(a);
    job.key = a.key;
    job.key.t_index = job.si.t_index;
    job.theta = a.theta;
    job.warm = a.warm;
    job.prop = a.prop;
    job.N = a.N;
    job.T = a.T;
    job.traj = a.traj;
    job.ctrl = a.ctrl;
    job.rec_stride = a.N;
    job.rec_shift = 0;
    job.coefA = nullptr;
    job.coefB = nullptr;
    job.coef_base = 0;
    job.jfree = nullptr;
    job.vfirst = nullptr;
    job.bins = &a.bins;
    job.stage = stage_all + tid;
    job.w2s = nullptr;
    if constexpr (KSQ > 0)
        job.w2s = reinterpret_cast<ulonglong2*>(stage_all) + (size_t)b * (Shape<W, G>::U * KSQ * G) + gl;
    constexpr int STAGE_TH = (W == 32 && KSQ == 0) ? NW * 32 : 0;
    float4* wnd = reinterpret_cast<float4*>(reinterpret_cast<char*>(stage_all) + traj_stage_bytes<W, G, NW, KSQ>()) +
                  (size_t)(tid / 32) * (32 / G) * CW;
    unsigned steps = 0, ntest = 0, nstate = 0;
    const FusedOut r = traj_sample_windowed<W, G, STAGE_TH, VAR, KSQ, CW, R>(a.c, job, n, valid, gl,
                                                                              hx_all + b * W, wnd, steps, ntest,
                                                                              nstate);
    if (valid && gl == 0) {
        unsigned long long key;
        if (r.first_hit < 0)
            key = ((unsigned long long)__float_as_uint(r.cost) << 32) | (unsigned)n;
        else
            key = (1ull << 63) | ((unsigned long long)(a.T - r.first_hit) << 32) | (unsigned)n;
        if (a.costs) a.costs[n] = r.cost;
        if (a.first_hit) a.first_hit[n] = r.first_hit;
        // the read skips atomics that cannot win
        if (a.best_key && key < *reinterpret_cast<volatile unsigned long long*>(a.best_key))
            atomicMin(a.best_key, key);
    }
    if (a.counts) {
        unsigned long long t = ntest, s = nstate;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            t += __shfl_xor_sync(FULL, t, off);
            s += __shfl_xor_sync(FULL, s, off);
        }
        if ((tid & 31) == 0) {
            atomicAdd(a.counts, t);
            atomicAdd(a.counts + 1, s);
        }
        if (valid && gl == 0) atomicAdd(a.counts + 2, (unsigned long long)steps);
    }
}

// ------------------------------------------------------------------ collide
// Points live in shared memory as pairs: XY_q = (x_2q, x_2q+1, y_2q, y_2q+1),
// V_q = (vx_2q, vx_2q+1, vy_2q, vy_2q+1), so that one packed FP32x2 FMA
// handles the same sample against two points.  The pairs come in blocks of
// 32: block b holds its 32 XY entries, then its 32 V entries (XY_q at
// pair_index(q), V_q 32 entries later) -- the same 1024 bytes as the
// block's 64 raw points, so the staging moves them into the EV frame in
// place, and a warp reads 32 consecutive XY (or V) entries at once.
__device__ __forceinline__ int pair_index(int q) { return q + (q & ~31); }
__device__ __forceinline__ unsigned long long pk(float lo, float hi)
{
    return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// One work unit: CC live samples (compact coefficient slots cs .. cs+CC-1, at
// most `nvalid` real; the rest repeat slot cs) against point pairs [q0, q1)
// at time tau.  Each lane keeps m = min over its points of max(|xi''|,
// |eta''|); a sample collides iff some lane has m < 1.  Returns the hit bits
// of the CC slots.
template <int CC>
__device__ __forceinline__ unsigned check_unit(const float4* __restrict__ P, int q0, int q1, float tau,
                                               const float4* __restrict__ cfA, const float2* __restrict__ cfB,
                                               int cs, int nvalid, int lane)
{
    unsigned long long A[CC], B[CC], NC[CC], D[CC], E[CC], NF[CC];
#pragma unroll
    for (int k = 0; k < CC; ++k) {
        const int slot = cs + (k < nvalid ? k : 0);
        const float4 qa = cfA[slot];
        const float2 qb = cfB[slot];
        A[k] = pk(qa.x, qa.x); B[k] = pk(qa.y, qa.y); NC[k] = pk(qa.z, qa.z);
        D[k] = pk(qa.w, qa.w); E[k] = pk(qb.x, qb.x); NF[k] = pk(qb.y, qb.y);
    }
    unsigned long long acc[CC];
#pragma unroll
    for (int k = 0; k < CC; ++k) acc[k] = 0ull;
    const unsigned long long TT = pk(tau, tau);
#pragma unroll 2
    for (int q = q0 + lane, i = pair_index(q0 + lane); q < q1; q += 32, i += 64) {
        const float4 xy = P[i];
        const float4 vv = P[i + 32];
        const unsigned long long PX = fma2(TT, pk(vv.x, vv.y), pk(xy.x, xy.y));
        const unsigned long long PY = fma2(TT, pk(vv.z, vv.w), pk(xy.z, xy.w));
#pragma unroll
        for (int k = 0; k < CC; ++k) {
            const unsigned long long xi = fma2(A[k], PX, fma2(B[k], PY, NC[k]));
            const unsigned long long et = fma2(D[k], PX, fma2(E[k], PY, NF[k]));
            acc[k] |= ~(xi | et);
        }
    }
    unsigned bits = 0;
#pragma unroll
    for (int k = 0; k < CC; ++k) {
        const bool inside = ((((unsigned)acc[k]) | (unsigned)(acc[k] >> 32)) >> 30) & 1u;
        if (k < nvalid && __any_sync(FULL, inside)) bits |= 1u << k;
    }
    return bits;
}


// Staging of the M obstacle points in shared memory P (pair_blocks(M)
// blocks of 64 points): one bulk copy by the copy engine (TMA) of the
// world-frame points, 16 bytes each, to the start of P, then each warp
// moves whole blocks into the EV frame in place (ev_point on the point's
// owner lane, the pairs assembled by shuffles).  Points past M (an odd tail
// and the rest of the last block) are placed 1e15 m away (never inside).
// Returns the number of pairs, or -1 when the copy's bounded wait ran out:
// *a.fault is then set and the whole block must return.
template <int THREADS>
__device__ __forceinline__ int stage_points(const RolloutArgs& a, float4* P)
{
    __shared__ uint64_t bar;
    const int M = a.M, nb = pair_blocks(M);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0 && M > 0) {
        mbar_expect_tx(&bar, (uint32_t)M * 16u);
        bulk_load(P, a.obs, (uint32_t)M * 16u, &bar);
    }
    const bool ok = M == 0 || mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0 && a.fault) atomicOr(a.fault, 1u);
        return -1;
    }
    const StepIn si = step_in(a);
    float s0, c0;
    sincosf(si.phi0, &s0, &c0);
    for (int b = warp; b < nb; b += THREADS / 32) {
        // lane l moves points j0 = 64 b + l and j1 = j0 + 32
        const int j0 = 64 * b + lane, j1 = j0 + 32;
        float x0 = 1e15f, y0 = 1e15f, u0 = 0.f, w0 = 0.f;
        float x1 = 1e15f, y1 = 1e15f, u1 = 0.f, w1 = 0.f;
        if (j0 < M) ev_point(P[j0], si.x0, si.y0, s0, c0, x0, y0, u0, w0);
        if (j1 < M) ev_point(P[j1], si.x0, si.y0, s0, c0, x1, y1, u1, w1);
        // pair r = lane of the block: its points 2r, 2r + 1 sit on lanes
        // 2r mod 32 and 2r + 1 mod 32, in the second half for r >= 16
        // (a shuffle reads the source lane's variable, so both halves travel
        // and the receiving lane picks)
        const int l0 = (2 * lane) & 31, l1 = l0 + 1;
        const bool hi = lane >= 16;
        const auto pick = [&](float lo_v, float hi_v, int src) {
            const float a_ = __shfl_sync(FULL, lo_v, src), b_ = __shfl_sync(FULL, hi_v, src);
            return hi ? b_ : a_;
        };
        const float ax0 = pick(x0, x1, l0), ax1 = pick(x0, x1, l1);
        const float ay0 = pick(y0, y1, l0), ay1 = pick(y0, y1, l1);
        const float au0 = pick(u0, u1, l0), au1 = pick(u0, u1, l1);
        const float aw0 = pick(w0, w1, l0), aw1 = pick(w0, w1, l1);
        __syncwarp();                         // every raw point of the block read
        P[64 * b + lane] = make_float4(ax0, ax1, ay0, ay1);
        P[64 * b + 32 + lane] = make_float4(au0, au1, aw0, aw1);
    }
    return (M + 1) / 2;
}

// Point slices per chunk for this step: the count whose units spread best
// over the NW warps (ties to fewer slices), each slice keeping at least
// `min_pairs` point pairs.
template <int NW>
__device__ __forceinline__ int choose_slices(int nch, int npairs)
{
    const int cand[8] = { 1, 2, 3, 4, 6, 8, 12, 16 };
    int best_s = 1;
    float best_e = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int S = cand[i];
        if (S > 1 && npairs / S < 96) break;
        const int units = nch * S;
        const int rounds = (units + NW - 1) / NW;
        const float e = (float)units / (float)(NW * rounds);
        if (e > best_e + 1e-3f) { best_e = e; best_s = S; }
    }
    return best_s;
}

template <int NW, int SBMAX>
struct CollideBlockKernel {
    static constexpr int THREADS = NW * 32;
    static_assert(SBMAX <= 128 && SBMAX % 32 == 0, "live list of at most 128 slots");
    static constexpr int fixed_bytes() {
        return 2 * SBMAX * 16 + 2 * SBMAX * 8 + 2 * SBMAX * 4 + NW * 8 + 64;
    }
    static int smem_bytes(int M) { return pair_blocks(M) * 1024 + fixed_bytes(); }
};

// Block-balanced collision kernel.  Block b owns an equal contiguous share of
// the samples and processes it in items of at most SBMAX samples; within an
// item all live samples advance through h = 0..T together.  The live list is
// kept compact and in sample order: slot r holds the r-th live sample, whose
// owner thread knows its rank; after each step the hit slots are removed and
// every rank shifts down by the number of hits below it.  The next step's
// coefficient rows are prefetched by the owners during the checks.
template <int NW, int SBMAX, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) collide_block_kernel(const RolloutArgs a)
{
    using K = CollideBlockKernel<NW, SBMAX>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* P = reinterpret_cast<float4*>(smem_raw);           // the point pairs
    float4* cfA = P + 64 * pair_blocks(a.M);                   // [2][SBMAX]
    float2* cfB = reinterpret_cast<float2*>(cfA + 2 * SBMAX);  // [2][SBMAX]
    int* hitf = reinterpret_cast<int*>(cfB + 2 * SBMAX);       // [2][SBMAX]
    unsigned long long* red = reinterpret_cast<unsigned long long*>(hitf + 2 * SBMAX);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const DevCfg& c = a.c;
    const int T = a.T, N = a.N;
    const int npairs = stage_points<K::THREADS>(a, P);
    if (npairs < 0) return;                                    // the staging copy gave up (a.fault set)

    // this block's share of the samples
    const int per_block = (N + gridDim.x - 1) / gridDim.x;
    const int b_begin = min(N, blockIdx.x * per_block);
    const int b_end = min(N, b_begin + per_block);
    const int nitems = (b_end - b_begin + SBMAX - 1) / SBMAX;
    unsigned long long best = ~0ull;

    for (int it = 0; it < nitems; ++it) {
        const int i_begin = b_begin + (int)(((long long)(b_end - b_begin) * it) / nitems);
        const int i_end = b_begin + (int)(((long long)(b_end - b_begin) * (it + 1)) / nitems);
        const int cnt = i_end - i_begin;
        const bool owner = tid < cnt;
        const int n = i_begin + tid;
        bool alive = owner;
        int fh = -1;
        int rank = tid;
        int L = cnt;
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (owner) z = a.traj[n];
        __syncthreads();                      // points staged / previous item done
        for (int h = 0; h <= T; ++h) {
            const int buf = h & 1;
            if (alive) {
                float4 ca;
                float2 cb;
                rows_of_state(c, z, ca, cb);
                cfA[buf * SBMAX + rank] = ca;
                cfB[buf * SBMAX + rank] = cb;
                hitf[buf * SBMAX + rank] = 0;
                if (h < T) z = a.traj[(size_t)(h + 1) * N + n];
            }
            __syncthreads();
            const int nch = (L + 7) / 8;
            const int S = choose_slices<NW>(nch, npairs);
            const int nunits = nch * S;
            const int per = (npairs + S - 1) / S;
            const float tau = (float)h * c.Ts;
            const float4* A_ = cfA + buf * SBMAX;
            const float2* B_ = cfB + buf * SBMAX;
            for (int u = warp; u < nunits; u += NW) {
                const int ch = u % nch, sl = u / nch;
                const int q0 = sl * per, q1 = min(npairs, q0 + per);
                const int cs = ch * 8;
                const int nv = min(8, L - cs);
                unsigned bits;
                if (nv > 4)      bits = check_unit<8>(P, q0, q1, tau, A_, B_, cs, nv, lane);
                else if (nv > 2) bits = check_unit<4>(P, q0, q1, tau, A_, B_, cs, nv, lane);
                else if (nv > 1) bits = check_unit<2>(P, q0, q1, tau, A_, B_, cs, nv, lane);
                else             bits = check_unit<1>(P, q0, q1, tau, A_, B_, cs, nv, lane);
                if (lane < 8 && ((bits >> lane) & 1u)) hitf[buf * SBMAX + cs + lane] = 1;
            }
            __syncthreads();
            // hit mask over the (at most 128) live slots, identical in every warp
            unsigned hm[SBMAX / 32];
#pragma unroll
            for (int w = 0; w < SBMAX / 32; ++w) {
                const int r = 32 * w + lane;
                hm[w] = __ballot_sync(FULL, r < L && hitf[buf * SBMAX + r] != 0);
            }
            int nhits = 0;
#pragma unroll
            for (int w = 0; w < SBMAX / 32; ++w) nhits += __popc(hm[w]);
            if (alive) {
                const int w = rank >> 5, bit = rank & 31;
                if ((hm[w] >> bit) & 1u) {
                    alive = false;
                    fh = h;
                } else {
                    int below = __popc(hm[w] & ((1u << bit) - 1u));
#pragma unroll
                    for (int ww = 0; ww < SBMAX / 32; ++ww) if (ww < w) below += __popc(hm[ww]);
                    rank -= below;
                }
            }
            L -= nhits;
            if (L == 0) break;
        }
        if (owner) {
            fh = discard_step(a.vfirst, n, fh);
            float J = __int_as_float(0x7f800000);
            unsigned long long key;
            if (fh < 0) {
                J = a.jfree[n];
                key = ((unsigned long long)__float_as_uint(J) << 32) | (unsigned)n;
            } else {
                key = (1ull << 63) | ((unsigned long long)(T - fh) << 32) | (unsigned)n;
            }
            if (a.costs) a.costs[n] = J;
            if (a.first_hit) a.first_hit[n] = fh;
            best = key < best ? key : best;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(FULL, best, off);
        best = o < best ? o : best;
    }
    __syncthreads();
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (tid == 0 && a.best_key) {
        unsigned long long k = red[0];
        for (int w = 1; w < NW; ++w) k = red[w] < k ? red[w] : k;
        atomicMin(a.best_key, k);
    }
}

// ------------------------------------------------------------------ collide (warp items)
// Barrier-free variant: each warp owns an item of 8 consecutive samples and
// checks them against all points, pulling items from the same atomic queue.
// The next horizon step's coefficient rows are prefetched (lanes 0..7 hold
// one sample each) while the current step is checked; the live samples are
// gathered into 8/4/2/1 slots by shuffles so that dead ones cost nothing.
// The live samples' coefficient rows sit in a warp-private shared slot array
// (slot r = the r-th live sample, written by its owner lane); every lane
// reads the CC slots with broadcast loads.  Returns the hit bits in slot
// order.
template <int CC>
__device__ __forceinline__ unsigned check_slots(const float4* __restrict__ P, int q0, int q1, float tau,
                                                const float4* __restrict__ sA,
                                                const float2* __restrict__ sB, int L, int lane)
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
#pragma unroll 2
    for (int q = q0 + lane, i = pair_index(q0 + lane); q < q1; q += 32, i += 64) {
        const float4 xy = P[i];
        const float4 vv = P[i + 32];
        const unsigned long long PX = fma2(TT, pk(vv.x, vv.y), pk(xy.x, xy.y));
        const unsigned long long PY = fma2(TT, pk(vv.z, vv.w), pk(xy.z, xy.w));
#pragma unroll
        for (int k = 0; k < CC; ++k) {
            const unsigned long long xi = fma2(A[k], PX, fma2(B[k], PY, NC[k]));
            const unsigned long long et = fma2(D[k], PX, fma2(E[k], PY, NF[k]));
            acc[k] |= ~(xi | et);
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

// One step of an 8-sample item for one warp: the owner lanes (lane < 8 with
// their bit in `live`) stage their coefficient rows, the warp checks the
// point pairs [q0, q1), and the hits come back as a lane mask.
__device__ __forceinline__ unsigned warp_step(const float4* P, int q0, int q1, float tau,
                                              float4 ca, float2 cb, unsigned live, float4* sA,
                                              float2* sB, int lane)
{
    const bool owner = lane < 8 && ((live >> lane) & 1u);
    const int rank = __popc(live & ((1u << lane) - 1u));
    if (owner) { sA[rank] = ca; sB[rank] = cb; }
    __syncwarp();
    const int L = __popc(live);
    unsigned bits;
    if (L > 4)      bits = check_slots<8>(P, q0, q1, tau, sA, sB, L, lane);
    else if (L > 2) bits = check_slots<4>(P, q0, q1, tau, sA, sB, L, lane);
    else if (L > 1) bits = check_slots<2>(P, q0, q1, tau, sA, sB, L, lane);
    else            bits = check_slots<1>(P, q0, q1, tau, sA, sB, L, lane);
    __syncwarp();
    return __ballot_sync(FULL, owner && ((bits >> rank) & 1u));
}

template <int NW>
struct CollideWarpKernel {
    static constexpr int THREADS = NW * 32;
    static constexpr int fixed_bytes() { return NW * 8 * 24 + NW * 8 + 64; }
    static int smem_bytes(int M) { return pair_blocks(M) * 1024 + fixed_bytes(); }
};

template <int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) collide_warp_kernel(const RolloutArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* P = reinterpret_cast<float4*>(smem_raw);             // the point pairs
    float4* slotA = P + 64 * pair_blocks(a.M);                   // [NW][8]
    float2* slotB = reinterpret_cast<float2*>(slotA + NW * 8);   // [NW][8]
    unsigned long long* red = reinterpret_cast<unsigned long long*>(slotB + NW * 8);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const DevCfg& c = a.c;
    const int T = a.T, N = a.N;
    const int npairs = stage_points<NW * 32>(a, P);
    if (npairs < 0) return;                                      // the staging copy gave up (a.fault set)
    __syncthreads();
    float4* sA = slotA + warp * 8;
    float2* sB = slotB + warp * 8;
    __syncthreads();

    unsigned long long best = ~0ull;
    const int nitems = (N + 7) / 8;
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(a.work, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= nitems) break;
        const int n0 = item * 8;
        const int cnt = min(8, N - n0);
        const int n = n0 + lane;
        const bool mine = lane < cnt;
        unsigned live = (1u << cnt) - 1u;
        int fh = -1;
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mine) z = a.traj[n];
        for (int h = 0; h <= T; ++h) {
            float4 cur_a;
            float2 cur_b;
            rows_of_state(c, z, cur_a, cur_b);
            if (mine && h < T) z = a.traj[(size_t)(h + 1) * N + n];
            const unsigned hits = warp_step(P, 0, npairs, (float)h * c.Ts, cur_a, cur_b, live,
                                            sA, sB, lane);
            if ((hits >> lane) & 1u) fh = h;
            live &= ~hits;
            if (live == 0u) break;
        }
        if (mine) {
            fh = discard_step(a.vfirst, n, fh);
            float J = __int_as_float(0x7f800000);
            unsigned long long key;
            if (fh < 0) {
                J = a.jfree[n];
                key = ((unsigned long long)__float_as_uint(J) << 32) | (unsigned)n;
            } else {
                key = (1ull << 63) | ((unsigned long long)(T - fh) << 32) | (unsigned)n;
            }
            if (a.costs) a.costs[n] = J;
            if (a.first_hit) a.first_hit[n] = fh;
            best = key < best ? key : best;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(FULL, best, off);
        best = o < best ? o : best;
    }
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (tid == 0 && a.best_key) {
        unsigned long long k = red[0];
        for (int w = 1; w < NW; ++w) k = red[w] < k ? red[w] : k;
        atomicMin(a.best_key, k);
    }
}

// ------------------------------------------------------------------ collide (sliced items)
// An item of 8 samples is checked by a block of S warps, warp s against the
// s-th slice of the points.  The warps run through h independently; they
// share, per sample, the earliest step at which any slice found a collision
// (dead_at, shared-memory atomicMin) and stop checking a sample at steps at
// or after it.  The item's first collision per sample is the minimum over
// the slices, identical to checking all points at once.  A block holds P
// such item groups of S warps: they share one staged copy of the points (so
// the staging does not cap the warps per SM) and each group synchronises on
// its own named barrier.
template <int S, int P = 1>
struct CollideSliceKernel {
    static constexpr int THREADS = P * S * 32;
    static constexpr int fixed_bytes() { return P * S * 8 * 24 + P * (8 * 4 + 16) + P * S * 8 + 64; }
    static int smem_bytes(int M) { return pair_blocks(M) * 1024 + fixed_bytes(); }
};

// barrier of one item group (named barrier 1 + group, its S warps; the
// whole block when the block is one group)
template <int S, int P>
__device__ __forceinline__ void group_sync(int grp)
{
    if constexpr (P == 1) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "n"(S * 32) : "memory");
}

template <int S, int MINB, bool GLOBAL_PTS = false, int P = 1>
__global__ void __launch_bounds__(P * S * 32, MINB) collide_slice_kernel(const RolloutArgs a)
{
    static_assert(P >= 1 && P <= 15, "one named barrier per item group");
    using K = CollideSliceKernel<S, P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int npairs = (a.M + 1) / 2;
    const int sb = GLOBAL_PTS ? 0 : pair_blocks(a.M);            // pair blocks held in shared memory
    const float4* Pts = GLOBAL_PTS ? a.pXY : reinterpret_cast<float4*>(smem_raw);
    float4* slotA = reinterpret_cast<float4*>(smem_raw) + 64 * sb;  // [P S][8]
    float2* slotB = reinterpret_cast<float2*>(slotA + P * S * 8);  // [P S][8]
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int grp = warp / S, ws = warp % S, gtid = tid - grp * S * 32;
    int* dead_at = reinterpret_cast<int*>(slotB + P * S * 8) + grp * 12;   // [P][8] (+ qslot, pad)
    int* qslot = dead_at + 8;
    unsigned long long* red = reinterpret_cast<unsigned long long*>(
        reinterpret_cast<int*>(slotB + P * S * 8) + P * 12);             // [P S]
    const DevCfg& c = a.c;
    const int T = a.T, N = a.N;
    if (!GLOBAL_PTS) {
        if (stage_points<K::THREADS>(a, reinterpret_cast<float4*>(smem_raw)) < 0) return;   // a.fault set
        if constexpr (P > 1) __syncthreads();
    }
    const int per = (npairs + S - 1) / S;
    const int q0 = min(npairs, ws * per), q1 = min(npairs, q0 + per);
    const int nslice = q1 - q0;
    float4* sA = slotA + warp * 8;
    float2* sB = slotB + warp * 8;

    unsigned long long best = ~0ull;
    const int nitems = (N + 7) / 8;
    for (;;) {
        if (gtid < 8) dead_at[gtid] = T + 1;
        if (gtid == 0) *qslot = (int)atomicAdd(a.work, 1u);
        group_sync<S, P>(grp);
        const int item = *qslot;
        if (item >= nitems) break;
        const int n0 = item * 8;
        const int cnt = min(8, N - n0);
        const int n = n0 + lane;
        const bool mine = lane < cnt;
        unsigned live = (1u << cnt) - 1u;
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mine) z = a.traj[n];
        for (int h = 0; h <= T; ++h) {
            float4 cur_a;
            float2 cur_b;
            rows_of_state(c, z, cur_a, cur_b);
            if (mine && h < T) z = a.traj[(size_t)(h + 1) * N + n];
            // drop samples another slice already found colliding at or before h
            const unsigned gone = __ballot_sync(FULL, lane < 8 && *(volatile int*)&dead_at[lane] <= h);
            live &= ~gone;
            if (live == 0u || nslice <= 0) break;
            const unsigned hits = warp_step(Pts, q0, q1, (float)h * c.Ts, cur_a, cur_b,
                                            live, sA, sB, lane);
            if ((hits >> lane) & 1u) atomicMin(&dead_at[lane], h);
            live &= ~hits;
        }
        group_sync<S, P>(grp);
        if (ws == 0 && mine) {
            const int d = dead_at[lane];
            const int fh = discard_step(a.vfirst, n, d <= T ? d : -1);
            float J = __int_as_float(0x7f800000);
            unsigned long long key;
            if (fh < 0) {
                J = a.jfree[n];
                key = ((unsigned long long)__float_as_uint(J) << 32) | (unsigned)n;
            } else {
                key = (1ull << 63) | ((unsigned long long)(T - fh) << 32) | (unsigned)n;
            }
            if (a.costs) a.costs[n] = J;
            if (a.first_hit) a.first_hit[n] = fh;
            best = key < best ? key : best;
        }
        group_sync<S, P>(grp);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(FULL, best, off);
        best = o < best ? o : best;
    }
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (tid == 0 && a.best_key) {
        unsigned long long k = red[0];
        for (int w = 1; w < P * S; ++w) k = red[w] < k ? red[w] : k;
        atomicMin(a.best_key, k);
    }
}

// ------------------------------------------------------------------ launchers
// opt in to more than 48 KB of dynamic shared memory for kernel fn (a host
// call; repeated on every launch that needs it, since the setting is per
// function and per device)
template <typename KernelFn>
inline cudaError_t ensure_smem(KernelFn fn, int smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// Whether a configuration turns on a rollout variant (VAR kernels).
__host__ __device__ inline bool uses_variants(const DevCfg& c) { return c.body_frame != 0 || c.vlim != 0; }

template <int W, int G, int NW, int MINB = 1, bool VAR = false, int KSQ = 0>
cudaError_t launch_traj(const RolloutArgs& a, cudaStream_t stream)
{
    using K = TrajKernel<W, G, NW>;
    const int grid = (a.N + K::B - 1) / K::B;
    const int smem = traj_stage_bytes<W, G, NW, KSQ>();
    cudaError_t e = ensure_smem(traj_kernel<W, G, NW, MINB, VAR, KSQ>, smem);
    if (e != cudaSuccess) return e;
    traj_kernel<W, G, NW, MINB, VAR, KSQ><<<grid, K::THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int W, int G, int NW, int MINB = 1, bool VAR = false, int KSQ = 0, int CW = 16, int R = 4>
cudaError_t launch_fused(const RolloutArgs& a, cudaStream_t stream)
{
    using K = TrajKernel<W, G, NW>;
    const int grid = (a.N + K::B - 1) / K::B;
    const int smem = traj_stage_bytes<W, G, NW, KSQ>() + NW * (32 / G) * CW * (int)sizeof(float4);
    cudaError_t e = ensure_smem(fused_kernel<W, G, NW, MINB, VAR, KSQ, CW, R>, smem);
    if (e != cudaSuccess) return e;
    fused_kernel<W, G, NW, MINB, VAR, KSQ, CW, R><<<grid, K::THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int NW, int SBMAX, int MINB>
cudaError_t launch_collide_block(const RolloutArgs& a, cudaStream_t stream)
{
    using K = CollideBlockKernel<NW, SBMAX>;
    const int smem = K::smem_bytes(a.M);
    cudaError_t e = ensure_smem(collide_block_kernel<NW, SBMAX, MINB>, smem);
    if (e != cudaSuccess) return e;
    const int grid = max(1, min((a.N + 7) / 8, a.grid_collide));
    collide_block_kernel<NW, SBMAX, MINB><<<grid, K::THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int NW, int SBMAX, int MINB>
int collide_block_blocks_per_sm(int M)
{
    using K = CollideBlockKernel<NW, SBMAX>;
    int nb = 0;
    const int smem = K::smem_bytes(M);
    if (ensure_smem(collide_block_kernel<NW, SBMAX, MINB>, smem) != cudaSuccess) return 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, collide_block_kernel<NW, SBMAX, MINB>,
                                                  K::THREADS, smem);
    return nb > 0 ? nb : 1;
}

template <int NW, int MINB>
cudaError_t launch_collide_warp(const RolloutArgs& a, cudaStream_t stream)
{
    using K = CollideWarpKernel<NW>;
    const int smem = K::smem_bytes(a.M);
    cudaError_t e = ensure_smem(collide_warp_kernel<NW, MINB>, smem);
    if (e != cudaSuccess) return e;
    const int nwarps_needed = (a.N + 7) / 8;
    const int grid = min((nwarps_needed + NW - 1) / NW, a.grid_collide);
    collide_warp_kernel<NW, MINB><<<grid, K::THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int NW, int MINB>
int collide_warp_blocks_per_sm(int M)
{
    using K = CollideWarpKernel<NW>;
    int nb = 0;
    const int smem = K::smem_bytes(M);
    if (ensure_smem(collide_warp_kernel<NW, MINB>, smem) != cudaSuccess) return 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, collide_warp_kernel<NW, MINB>, K::THREADS, smem);
    return nb > 0 ? nb : 1;
}

// EV-frame point pairs written to global memory in the staging's blocked
// layout (for point sets larger than shared memory); same arithmetic as
// stage_points.
static __global__ void transform_pairs_kernel(const RolloutArgs a)
{
    const int npairs = 32 * pair_blocks(a.M);
    const StepIn si = step_in(a);
    float s0, c0;
    sincosf(si.phi0, &s0, &c0);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += gridDim.x * blockDim.x) {
        float px[2], py[2], vx[2], vy[2];
        for (int o = 0; o < 2; ++o) {
            const int j = 2 * q + o;
            px[o] = 1e15f; py[o] = 1e15f; vx[o] = 0.f; vy[o] = 0.f;
            if (j < a.M) {
                ev_point(a.obs[j], si.x0, si.y0, s0, c0, px[o], py[o], vx[o], vy[o]);
            }
        }
        a.pXY[pair_index(q)] = make_float4(px[0], px[1], py[0], py[1]);
        a.pXY[pair_index(q) + 32] = make_float4(vx[0], vx[1], vy[0], vy[1]);
    }
}

template <int S, int MINB>
cudaError_t launch_collide_slice_global(const RolloutArgs& a, cudaStream_t stream)
{
    using K = CollideSliceKernel<S>;
    const int npairs = 32 * pair_blocks(a.M);
    transform_pairs_kernel<<<max(1, min(1024, (npairs + 255) / 256)), 256, 0, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int smem = K::fixed_bytes();
    const int grid = max(1, min((a.N + 7) / 8, a.grid_collide));
    collide_slice_kernel<S, MINB, true><<<grid, K::THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int S, int MINB, int P = 1>
cudaError_t launch_collide_slice(const RolloutArgs& a, cudaStream_t stream)
{
    using K = CollideSliceKernel<S, P>;
    const int smem = K::smem_bytes(a.M);
    cudaError_t e = ensure_smem(collide_slice_kernel<S, MINB, false, P>, smem);
    if (e != cudaSuccess) return e;
    const int grid = max(1, min(((a.N + 7) / 8 + P - 1) / P, a.grid_collide));
    collide_slice_kernel<S, MINB, false, P><<<grid, K::THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int S, int MINB, int P = 1>
int collide_slice_blocks_per_sm(int M)
{
    using K = CollideSliceKernel<S, P>;
    int nb = 0;
    const int smem = K::smem_bytes(M);
    if (ensure_smem(collide_slice_kernel<S, MINB, false, P>, smem) != cudaSuccess) return 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, collide_slice_kernel<S, MINB, false, P>, K::THREADS, smem);
    return nb > 0 ? nb : 1;
}

}  // namespace npp
