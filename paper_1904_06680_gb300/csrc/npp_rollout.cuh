// npp_rollout.cuh -- the batched rollout kernel (one template per network
// width), instantiated by npp_rollout_w{16,32,64}.cu.
//
// What one block does (paper: Sect. II-D "First".."Sixth", Sect. IV):
//   * stages the M obstacle points in shared memory, rotated into the
//     EV-aligned frame at t (Sect. II-C, m^ext in (xi, eta) coordinates);
//   * owns B samples; a group of G lanes of one warp holds one sample's
//     network in registers (each lane two hidden units: its rows of W1, W2,
//     its columns of W3), generated straight from Philox, never stored;
//   * steps all its samples through h = 0..T in lockstep.  Per step:
//       collision phase -- the block's warps split the M points, each lane
//         tests its points against a chunk of C live samples at once
//         (Eq. eq_Apsietc_collAvoidIneqs with the rectangle's inequalities
//         scaled to |xi''| < 1, |eta''| < 1: 4 FMA + 2 min/max per pair),
//         points extrapolated at constant velocity (Sect. II-D (ii)-(iv));
//       control phase -- features (Eq. eq_def_stph), MLP with the hidden
//         vector exchanged through shared memory, rate-limited controls,
//         one Euler step of the kinematic bicycle on the old state;
//   * reduces (class, cost, index) keys to the block minimum and folds it
//     into the global minimum with one 64-bit atomicMin.
#pragma once

#include <cfloat>
#include <cstdint>
#include <cuda_runtime.h>

#include "npp_device.cuh"

namespace npp {

template <int W>
struct Shape {
    static constexpr int G = (W == 16) ? 8 : (W == 32) ? 16 : 32;   // lanes per sample
    static constexpr int U = W / G;                                  // hidden units per lane
    static constexpr int NT = 12 * W + W * W + 2;                    // parameters
    static constexpr int OFF_B1 = NIN * W;
    static constexpr int OFF_W2 = OFF_B1 + W;
    static constexpr int OFF_B2 = OFF_W2 + W * W;
    static constexpr int OFF_W3 = OFF_B2 + W;
    static constexpr int OFF_B3 = OFF_W3 + 2 * W;
    static_assert(U == 2, "two hidden units per lane");
};

// Parameter source: Philox (sampled) or memory (explicit / warm start).
struct ThetaSrc {
    const float* mem;     // row of this sample, or null -> sample
    SamplerKey key;
    uint32_t n;
    __device__ __forceinline__ float4 quad(int i) const {     // i % 4 == 0
        if (mem) return make_float4(mem[i], mem[i + 1], mem[i + 2], mem[i + 3]);
        return sample_quad(key, (uint32_t)i >> 2, n);
    }
    __device__ __forceinline__ float2 pair(int i) const {     // i % 2 == 0
        if (mem) return make_float2(mem[i], mem[i + 1]);
        return sample_pair(key, (uint32_t)i, n);
    }
};

template <int W>
struct LaneNet {
    using S = Shape<W>;
    float w1[S::U][NIN], b1[S::U];
    float w2[S::U][W], b2[S::U];
    float w3[2][S::U], b3[2];

    // lane gl of the group holds hidden units 2 gl and 2 gl + 1
    __device__ __forceinline__ void load(const ThetaSrc& src, int gl) {
#pragma unroll
        for (int j = 0; j < S::U; ++j) {
            const int u = gl * S::U + j;
#pragma unroll
            for (int i = 0; i < NIN; i += 4) {
                const float4 q = src.quad(u * NIN + i);
                w1[j][i] = q.x; w1[j][i + 1] = q.y; w1[j][i + 2] = q.z; w1[j][i + 3] = q.w;
            }
#pragma unroll
            for (int i = 0; i < W; i += 4) {
                const float4 q = src.quad(S::OFF_W2 + u * W + i);
                w2[j][i] = q.x; w2[j][i + 1] = q.y; w2[j][i + 2] = q.z; w2[j][i + 3] = q.w;
            }
        }
        const float2 pb1 = src.pair(S::OFF_B1 + gl * S::U);
        b1[0] = pb1.x; b1[1] = pb1.y;
        const float2 pb2 = src.pair(S::OFF_B2 + gl * S::U);
        b2[0] = pb2.x; b2[1] = pb2.y;
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            const float2 p = src.pair(S::OFF_W3 + o * W + gl * S::U);
            w3[o][0] = p.x; w3[o][1] = p.y;
        }
        const float2 pb3 = src.pair(S::OFF_B3);
        b3[0] = pb3.x; b3[1] = pb3.y;
    }
};

__device__ __forceinline__ float wrap_pi(float a)
{
    const float TWO_PI = 6.28318530717958647692f;
    const float INV_TWO_PI = 0.15915494309189533577f;
    return a - TWO_PI * floorf((a + 3.14159265358979323846f) * INV_TWO_PI);
}

// Collision phase: warps split the points; every lane tests its points
// against chunks of C live samples.  Sets hit[b] for samples that collide.
template <int NW, int C>
__device__ __forceinline__ void collide_phase(const float4* __restrict__ pts, int M, float tau,
                                              const float4* __restrict__ coef,
                                              int* __restrict__ hit, unsigned live,
                                              int warp, int lane)
{
    const int per = (M + NW - 1) / NW;
    const int j0 = warp * per;
    const int j1 = min(M, j0 + per);
    while (live) {
        int sidx[C];
        float cA[C], cB[C], cC[C], cD[C], cE[C], cF[C];
#pragma unroll
        for (int k = 0; k < C; ++k) {
            if (live) {
                const int s = __ffs(live) - 1;
                live &= live - 1;
                sidx[k] = s;
                const float4 q0 = coef[2 * s], q1 = coef[2 * s + 1];
                cA[k] = q0.x; cB[k] = q0.y; cC[k] = q0.z; cD[k] = q0.w; cE[k] = q1.x; cF[k] = q1.y;
            } else {
                sidx[k] = -1;                 // padding slot: |xi''| = 2, never inside
                cA[k] = 0.f; cB[k] = 0.f; cC[k] = -2.f; cD[k] = 0.f; cE[k] = 0.f; cF[k] = 0.f;
            }
        }
        float m[C];
#pragma unroll
        for (int k = 0; k < C; ++k) m[k] = FLT_MAX;
        for (int j = j0 + lane; j < j1; j += 32) {
            const float4 p = pts[j];
            const float px = fmaf(tau, p.z, p.x);
            const float py = fmaf(tau, p.w, p.y);
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const float xi = fmaf(cA[k], px, fmaf(cB[k], py, -cC[k]));
                const float et = fmaf(cD[k], px, fmaf(cE[k], py, -cF[k]));
                m[k] = fminf(m[k], fmaxf(fabsf(xi), fabsf(et)));
            }
        }
#pragma unroll
        for (int k = 0; k < C; ++k) {
            if (sidx[k] >= 0 && __any_sync(FULL, m[k] < 1.0f) && lane == 0) hit[sidx[k]] = 1;
        }
    }
}

template <int W, int NW, int C>
struct RolloutKernel {
    using S = Shape<W>;
    static constexpr int G = S::G;
    static constexpr int U = S::U;
    static constexpr int THREADS = NW * 32;
    static constexpr int B = THREADS / G;            // samples per block
    static_assert(B <= 32, "live mask is one warp ballot");

    // shared memory carve-up (bytes), points first
    static constexpr int fixed_bytes() {
        return B * 32 /*coef*/ + B * 4 /*hit*/ + B * 4 /*alive*/ + B * W * 4 /*hidden*/
             + NW * 8 /*reduction*/ + 64;
    }
    static int smem_bytes(int M) { return M * 16 + fixed_bytes(); }
};

template <int W, int NW, int C>
__global__ void __launch_bounds__(NW * 32, 1) rollout_kernel(const RolloutArgs a)
{
    using K = RolloutKernel<W, NW, C>;
    using S = Shape<W>;
    constexpr int G = K::G, U = K::U, B = K::B;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* pts = reinterpret_cast<float4*>(smem_raw);
    float4* coef = pts + a.M;
    int* hit = reinterpret_cast<int*>(coef + 2 * B);
    int* alive_f = hit + B;
    float* hx = reinterpret_cast<float*>(alive_f + B);
    unsigned long long* red = reinterpret_cast<unsigned long long*>(hx + B * W);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int b = tid / G, gl = tid % G;
    const int n = blockIdx.x * B + b;
    const bool valid = n < a.N;
    const DevCfg& c = a.c;

    // frame of the vehicle at time t
    float s0, c0;
    sincosf(a.phi0, &s0, &c0);
    for (int j = tid; j < a.M; j += K::THREADS) {
        const float4 o = a.obs[j];
        const float dx = o.x - a.x0, dy = o.y - a.y0;
        pts[j] = make_float4(c0 * dx + s0 * dy, -s0 * dx + c0 * dy,
                             c0 * o.z + s0 * o.w, -s0 * o.z + c0 * o.w);
    }
    const float gdx = a.gx - a.x0, gdy = a.gy - a.y0;
    const float gxi = c0 * gdx + s0 * gdy, geta = -s0 * gdx + c0 * gdy;
    const float gph = a.gphi - a.phi0, gv = a.gv;

    // this lane's slice of the sample's network
    LaneNet<W> net;
    {
        ThetaSrc src;
        src.key = a.key;
        src.n = (uint32_t)(valid ? n : 0);
        src.mem = nullptr;
        if (a.theta) src.mem = a.theta + (size_t)(valid ? n : 0) * S::NT;
        else if (a.warm && n == 0) src.mem = a.warm;
        net.load(src, gl);
    }

    float x = 0.f, y = 0.f, ph = 0.f, v = a.v0, ap0 = a.ap0, ap1 = a.ap1, E = 0.f;
    bool alive = valid;
    int fh = -1;
    const int T = a.T, N = a.N;
    const float invT = 1.0f / (float)T;

    for (int h = 0;; ++h) {
        float sp, cp;
        sincosf(ph, &sp, &cp);
        if (gl == 0) {
            if (alive) a.traj[(size_t)h * N + n] = make_float4(x, y, ph, v);
            coef[2 * b] = make_float4(cp * c.ihl, sp * c.ihl, (cp * x + sp * y + c.c_off) * c.ihl,
                                      -sp * c.ihw);
            coef[2 * b + 1] = make_float4(cp * c.ihw, (-sp * x + cp * y) * c.ihw, 0.f, 0.f);
            hit[b] = 0;
            alive_f[b] = alive ? 1 : 0;
        }
        __syncthreads();
        {
            const unsigned live = __ballot_sync(FULL, lane < B && alive_f[lane] != 0);
            collide_phase<NW, C>(pts, a.M, (float)h * c.Ts, coef, hit, live, warp, lane);
        }
        __syncthreads();
        if (alive && hit[b]) { alive = false; fh = h; }
        if (h == T) break;
        if (!__syncthreads_or(alive)) break;

        // ---- control phase: features, network, controls, Euler step
        float s[NIN];
        s[0] = (gxi - x) * c.idxi;
        s[1] = (geta - y) * c.ideta;
        s[2] = wrap_pi(gph - ph) * c.idphi;
        s[3] = (gv - v) * c.idv;
        s[4] = ap0;
        s[5] = ap1;
        s[6] = v * c.idv;
        s[7] = (float)(T - h) * invT;
        float h1[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            float acc = net.b1[j];
#pragma unroll
            for (int i = 0; i < NIN; ++i) acc = fmaf(net.w1[j][i], s[i], acc);
            h1[j] = tanhf(acc);
        }
        float* hrow = hx + b * W;
        *reinterpret_cast<float2*>(hrow + gl * U) = make_float2(h1[0], h1[1]);
        __syncwarp();
        float acc2[U];
#pragma unroll
        for (int j = 0; j < U; ++j) acc2[j] = net.b2[j];
        const float4* hrow4 = reinterpret_cast<const float4*>(hrow);
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
            const float4 hv = hrow4[i];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                acc2[j] = fmaf(net.w2[j][4 * i + 0], hv.x, acc2[j]);
                acc2[j] = fmaf(net.w2[j][4 * i + 1], hv.y, acc2[j]);
                acc2[j] = fmaf(net.w2[j][4 * i + 2], hv.z, acc2[j]);
                acc2[j] = fmaf(net.w2[j][4 * i + 3], hv.w, acc2[j]);
            }
        }
        __syncwarp();
        float h2[U];
#pragma unroll
        for (int j = 0; j < U; ++j) h2[j] = tanhf(acc2[j]);
        float p0 = fmaf(net.w3[0][1], h2[1], net.w3[0][0] * h2[0]);
        float p1 = fmaf(net.w3[1][1], h2[1], net.w3[1][0] * h2[0]);
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
            p0 += __shfl_xor_sync(FULL, p0, off);
            p1 += __shfl_xor_sync(FULL, p1, off);
        }
        const float ar0 = tanhf(net.b3[0] + p0);
        const float ar1 = tanhf(net.b3[1] + p1);
        if (alive) {
            float a0 = fminf(fmaxf(ar0, ap0 - c.r_rate), ap0 + c.r_rate);
            a0 = fminf(fmaxf(a0, -1.0f), 1.0f);
            const float a1 = ar1;
            E += a0 * a0 + a1 * a1;
            if (gl == 0) a.ctrl[(size_t)h * N + n] = make_float2(a0, a1);
            const float td = tanf(c.delta_max * a0);
            const float tb = c.lrL * td;
            const float dv = c.Ts * v;
            x += dv * (cp - sp * tb);
            y += dv * (sp + cp * tb);
            ph += dv * td * c.iL;
            v += c.Ts * (c.umid + c.uhalf * a1);
            ap0 = a0;
            ap1 = a1;
        }
    }

    // ---- cost and packed selection key
    unsigned long long key = ~0ull;
    if (valid && gl == 0) {
        float J = __int_as_float(0x7f800000);
        if (alive) {
            const float dx = x - gxi, dy = y - geta;
            J = c.w_pos * sqrtf(dx * dx + dy * dy) + c.w_phi * fabsf(wrap_pi(ph - gph))
              + c.w_v * fabsf(v - gv) + c.w_effort * E * invT;
            key = ((unsigned long long)__float_as_uint(J) << 32) | (unsigned)n;
        } else {
            key = (1ull << 63) | ((unsigned long long)(T - fh) << 32) | (unsigned)n;
        }
        if (a.costs) a.costs[n] = J;
        if (a.first_hit) a.first_hit[n] = alive ? -1 : fh;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(FULL, key, off);
        key = o < key ? o : key;
    }
    if (lane == 0) red[warp] = key;
    __syncthreads();
    if (tid == 0) {
        unsigned long long k = red[0];
        for (int w = 1; w < NW; ++w) k = red[w] < k ? red[w] : k;
        if (a.best_key) atomicMin(a.best_key, k);
    }
}

template <int W, int NW, int C>
cudaError_t launch_rollout(const RolloutArgs& a, cudaStream_t stream, int* smem_needed)
{
    using K = RolloutKernel<W, NW, C>;
    const int smem = K::smem_bytes(a.M);
    if (smem_needed) *smem_needed = smem;
    // opt in to large dynamic shared memory once per device (idempotent)
    static int configured[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (configured[dev] < smem) {
        e = cudaFuncSetAttribute(rollout_kernel<W, NW, C>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured[dev] = smem;
    }
    const int grid = (a.N + K::B - 1) / K::B;
    rollout_kernel<W, NW, C><<<grid, K::THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace npp
