// npp_proposal.cu -- the learned sampling proposal: scene encoding, the
// 72-256-256-900 network on BF16 tensor-core GEMMs (forward, backward),
// Gaussian negative log-likelihood, Adam, and the standalone GEMM entry.
//
// The paper samples theta ~ N(0, I) every sampling time (Sect. II-D
// "Fourth") and lists guiding the sampling as future work (Sect. V); this
// file is that guide, built so that it never bends the method: its output
// (mean, std) only feeds npp_plan_step_proposal, whose proposal samples
// are mixed with isotropic ones and judged by the exact rollout cost.
//
// Layout of the FP32 master parameters (padded for the GEMM tiles):
//   W1 [256][128] (inputs 72..127 zero), b1 [256], W2 [256][256], b2 [256],
//   W3 [1024][256] (rows 900..1023 zero), b3 [1024]
// BF16 copies W1, W2, W2^T, W3, W3^T are refreshed after every update.
#include <cmath>
#include <cstring>
#include <string>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/npp_proposal.h"
#include "npp_gemm.cuh"
#include "npp_internal.h"

using namespace npp;

namespace {

constexpr int NIN_X = NPP_PROP_NIN;        // 72
constexpr int D0 = 128;                    // padded input width
constexpr int HID = NPP_PROP_HIDDEN;       // 256
constexpr int NTH = NPP_PROP_NTHETA;       // 450
constexpr int D3 = 1024;                   // padded output width (900 used)
constexpr int NBINS = 64;
constexpr float R_HIST = 20.0f;

// offsets into the flat master / gradient / moment buffers
constexpr size_t OFF_W1 = 0;
constexpr size_t OFF_B1 = OFF_W1 + (size_t)HID * D0;
constexpr size_t OFF_W2 = OFF_B1 + HID;
constexpr size_t OFF_B2 = OFF_W2 + (size_t)HID * HID;
constexpr size_t OFF_W3 = OFF_B2 + HID;
constexpr size_t OFF_B3 = OFF_W3 + (size_t)D3 * HID;
constexpr size_t N_FLAT = OFF_B3 + D3;
// packed (unpadded) parameter count of the public layout
constexpr int N_PACKED = HID * NIN_X + HID + HID * HID + HID + 2 * NTH * HID + 2 * NTH;

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ encoding
// One block per scene: nearness-weighted polar histogram of the points in
// the EV-aligned frame at t (fixed-point sums, so the result does not
// depend on the order of the atomic adds), squashed h / (1 + h), then the
// rollout's 8 network inputs at h = 0.
__global__ void __launch_bounds__(256) encode_kernel(const DevCfg c, const npp_scene* __restrict__ scenes,
                                                     const float4* __restrict__ obs, float* __restrict__ x)
{
    __shared__ unsigned long long hist[NBINS];
    const npp_scene sc = scenes[blockIdx.x];
    for (int k = threadIdx.x; k < NBINS; k += blockDim.x) hist[k] = 0ull;
    __syncthreads();
    float s0, c0;
    sincosf(sc.state.phi, &s0, &c0);
    const float4* p = obs + sc.obs_offset;
    for (int j = threadIdx.x; j < sc.M; j += blockDim.x) {
        float px, py, vx, vy;
        ev_point(p[j], sc.state.x, sc.state.y, s0, c0, px, py, vx, vy);
        const float d = sqrtf(fmaf(px, px, py * py));
        const float w = 1.0f - d / R_HIST;
        if (w > 0.0f) {
            const float u = (atan2f(py, px) + 3.14159265358979323846f) * (NBINS / 6.28318530717958647692f);
            const int k = min(max((int)floorf(u), 0), NBINS - 1);
            atomicAdd(&hist[k], (unsigned long long)__float2ull_rn(w * 4294967296.0f));
        }
    }
    __syncthreads();
    float* xr = x + (size_t)blockIdx.x * NIN_X;
    for (int k = threadIdx.x; k < NBINS; k += blockDim.x) {
        const float h = (float)((double)hist[k] * (1.0 / 4294967296.0));
        xr[k] = h / (1.0f + h);
    }
    if (threadIdx.x == 0) {
        const float gdx = sc.goal.x - sc.state.x, gdy = sc.goal.y - sc.state.y;
        const float gxi = c0 * gdx + s0 * gdy, geta = -s0 * gdx + c0 * gdy;
        float* s = xr + NBINS;
        s[0] = gxi * c.idxi;
        s[1] = geta * c.ideta;
        const float dph = sc.goal.phi - sc.state.phi;
        s[2] = (dph - 6.28318530717958647692f * floorf((dph + 3.14159265358979323846f) *
                                                       0.15915494309189533577f)) * c.idphi;
        s[3] = (sc.goal.v - sc.state.v) * c.idv;
        s[4] = sc.state.a_prev0;
        s[5] = sc.state.a_prev1;
        s[6] = sc.state.v * c.idv;
        s[7] = (float)sc.T * (1.0f / (float)sc.T);
    }
}

// x [n][72] FP32 -> X [B][128] BF16 and its transpose XT [128][B] (zero
// rows beyond n, zero inputs beyond 72).  A block takes PX_TB rows: X is
// written along the inputs, the tile staged in shared memory and XT written
// along the batch, so both stores are coalesced.
constexpr int PX_TB = 32;
__global__ void __launch_bounds__(256) pack_x_kernel(const float* __restrict__ x, int n, int B,
                                                     bf16* __restrict__ X, bf16* __restrict__ XT)
{
    __shared__ bf16 tile[D0][PX_TB + 2];                  // input x batch row
    const int b0 = blockIdx.x * PX_TB;
    for (int e = threadIdx.x; e < PX_TB * D0; e += blockDim.x) {
        const int k = e % D0, bb = e / D0, b = b0 + bb;
        const float v = (b < n && k < NIN_X) ? x[(size_t)b * NIN_X + k] : 0.0f;
        const bf16 q = __float2bfloat16_rn(v);
        X[(size_t)b * D0 + k] = q;
        tile[k][bb] = q;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < PX_TB * D0; e += blockDim.x) {
        const int bb = e % PX_TB, k = e / PX_TB;
        XT[(size_t)k * B + b0 + bb] = tile[k][bb];
    }
}

// Gaussian NLL of theta under (mu, exp(clamp(raw))) and its gradient with
// respect to the network output, both layouts in BF16; the loss (mean over
// B x 450) is added to *loss.  A block takes a tile of NLL_TB batch rows x
// NLL_TI parameters: the row-major gradient is written along the
// parameters, the tile is staged in shared memory and the transposed
// gradient written along the batch, so both stores are coalesced.  The
// padding outputs 900..1023 are never written: their gradient rows stay at
// the zeros the handle set at creation.
constexpr int NLL_TB = 64;
constexpr int NLL_TI = 32;
__global__ void __launch_bounds__(256) nll_kernel(const float* __restrict__ Y, const float* __restrict__ theta, int B,
                                                  float ls_min, float ls_max, bf16* __restrict__ dY,
                                                  bf16* __restrict__ dYT, float* __restrict__ loss)
{
    __shared__ float red[8];
    __shared__ bf16 tile[2][NLL_TI][NLL_TB + 2];          // (mu, log-std) x parameter x batch row
    const float scale = 1.0f / ((float)B * (float)NTH);
    const int i0 = blockIdx.x * NLL_TI, b0 = blockIdx.y * NLL_TB;
    float acc = 0.0f;
    for (int e = threadIdx.x; e < NLL_TI * NLL_TB; e += blockDim.x) {
        const int ii = e % NLL_TI, bb = e / NLL_TI;
        const int i = i0 + ii, b = b0 + bb;
        if (i < NTH) {
            const float mu = Y[(size_t)b * D3 + i];
            const float raw = Y[(size_t)b * D3 + NTH + i];
            const float ls = fminf(fmaxf(raw, ls_min), ls_max);
            const float r = theta[(size_t)b * NTH + i] - mu;
            const float e2 = expf(-2.0f * ls);
            acc += ls + 0.5f * r * r * e2;
            const float dmu = -r * e2 * scale;
            const float dls = (raw > ls_min && raw < ls_max) ? (1.0f - r * r * e2) * scale : 0.0f;
            const bf16 qm = __float2bfloat16_rn(dmu), ql = __float2bfloat16_rn(dls);
            dY[(size_t)b * D3 + i] = qm;
            dY[(size_t)b * D3 + NTH + i] = ql;
            tile[0][ii][bb] = qm;
            tile[1][ii][bb] = ql;
        }
    }
    __syncthreads();
    // transposed rows i and NTH + i, NLL_TB consecutive batch entries each
    for (int e = threadIdx.x; e < 2 * NLL_TI * NLL_TB; e += blockDim.x) {
        const int bb = e % NLL_TB, k = e / NLL_TB, half = k / NLL_TI, ii = k % NLL_TI;
        const int i = i0 + ii;
        if (i < NTH) dYT[(size_t)(half * NTH + i) * B + b0 + bb] = tile[half][ii][bb];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s * scale);
    }
}

// bias gradients: row sums of dY^T (1024 rows), dZ2^T and dZ1^T (256 each);
// one warp per row, each lane summing 8 consecutive entries per 16-byte
// load, then the lanes in a fixed tree: a fixed summation order
__global__ void bias_grad_kernel(const bf16* __restrict__ dYT, const bf16* __restrict__ dZ2T,
                                 const bf16* __restrict__ dZ1T, int B, float* __restrict__ g)
{
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= D3 + 2 * HID) return;
    const bf16* src;
    float* dst;
    if (row < D3) { src = dYT + (size_t)row * B; dst = g + OFF_B3 + row; }
    else if (row < D3 + HID) { src = dZ2T + (size_t)(row - D3) * B; dst = g + OFF_B2 + (row - D3); }
    else { src = dZ1T + (size_t)(row - D3 - HID) * B; dst = g + OFF_B1 + (row - D3 - HID); }
    float s = 0.0f;
    const uint4* src8 = reinterpret_cast<const uint4*>(src);      // B is a multiple of 128
    for (int q = lane; q < B / 8; q += 32) {
        const uint4 u = src8[q];
        const uint32_t w[4] = { u.x, u.y, u.z, u.w };
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s += __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[k] & 0xFFFFu)));
            s += __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[k] >> 16)));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) *dst = s;
}

// weight gradients summed over the K slices of the split GEMMs, in slice
// order (deterministic): segment k has n[k] outputs at dst[k] and n[k] x
// splits[k] partials at src[k] (slice z at src[k] + z n[k])
struct SplitSum {
    const float* src[3];
    float* dst[3];
    int n[3];
    int splits[3];
};
__global__ void __launch_bounds__(256) splitk_sum_kernel(const SplitSum a)
{
    const int total = a.n[0] + a.n[1] + a.n[2];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int k = 0, i = t;
        if (i >= a.n[0]) { i -= a.n[0]; k = 1; if (i >= a.n[1]) { i -= a.n[1]; k = 2; } }
        const float* p = a.src[k] + i;
        const size_t st = (size_t)a.n[k];
        const int S = a.splits[k];
        float s = 0.0f;
        int z = 0;
        // eight loads in flight, added in slice order
        for (; z + 8 <= S; z += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = p[(size_t)(z + u) * st];
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; z < S; ++z) s += p[(size_t)z * st];
        a.dst[k][i] = s;
    }
}

// Adam with bias correction on the flat FP32 masters
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, size_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mhat = mi / c1, vhat = vi / c2;
        w[i] -= lr * mhat / (sqrtf(vhat) + eps);
    }
}

// BF16 copies of the weight matrices (row-major and, for W2, W3, transposed)
__global__ void convert_kernel(const float* __restrict__ w, bf16* __restrict__ W1, bf16* __restrict__ W2,
                               bf16* __restrict__ W2T, bf16* __restrict__ W3, bf16* __restrict__ W3T)
{
    const int n1 = HID * D0, n2 = HID * HID, n3 = D3 * HID;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n1 + n2 + n3; t += gridDim.x * blockDim.x) {
        if (t < n1) {
            W1[t] = __float2bfloat16_rn(w[OFF_W1 + t]);
        } else if (t < n1 + n2) {
            const int u = t - n1, r = u / HID, k = u % HID;
            const bf16 q = __float2bfloat16_rn(w[OFF_W2 + u]);
            W2[u] = q;
            W2T[(size_t)k * HID + r] = q;
        } else {
            const int u = t - n1 - n2, r = u / HID, k = u % HID;
            const bf16 q = __float2bfloat16_rn(w[OFF_W3 + u]);
            W3[u] = q;
            W3T[(size_t)k * D3 + r] = q;
        }
    }
}

// mean and std of rows 0..n-1 from the network output
__global__ void mean_std_kernel(const float* __restrict__ Y, int n, float ls_min, float ls_max,
                                float* __restrict__ mean, float* __restrict__ sd)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * NTH; t += gridDim.x * blockDim.x) {
        const int b = t / NTH, i = t % NTH;
        mean[t] = Y[(size_t)b * D3 + i];
        sd[t] = expf(fminf(fmaxf(Y[(size_t)b * D3 + NTH + i], ls_min), ls_max));
    }
}

__device__ int g_gemm_err;

std::string g_prop_err;

npp_status perr(npp_status s, const std::string& msg)
{
    g_prop_err = msg;
    set_global_error(msg.c_str());
    return s;
}

}  // namespace

struct npp_proposal {
    npp_proposal_config cfg;
    int B;
    int t;                                  // Adam steps taken
    float* w; float* m; float* v; float* g; // flat FP32 [N_FLAT]
    bf16 *W1, *W2, *W2T, *W3, *W3T;
    bf16 *X, *XT, *H1, *H1T, *H2, *H2T, *dY, *dYT, *dZ2, *dZ2T, *dZ1T;
    float* Y;
    float* loss;                            // scratch loss when the caller passes none
    int* err;
    // the weight-gradient GEMMs (K = batch) split K into sp[k] slices, each
    // slice's FP32 partial in ws (dW3, dW2, dW1 at ws_off[k]), summed by
    // splitk_sum_kernel
    float* ws;
    int sp[3];
    size_t ws_off[3];
    CUtensorMap tX, tW1, tH1, tW2, tH2, tW3, tdY, tW3T, tdZ2, tW2T, tdYT, tH2T, tdZ2T, tH1T, tdZ1T, tXT;
};

namespace {

// K slices of a weight-gradient GEMM with `tiles` output tiles and nk K
// blocks: doubled while the CTAs stay within about one wave of the 152 SMs
// and every slice keeps two K blocks or more
int grad_splits(int tiles, int nk)
{
    int sp = 1;
    while (2 * sp * tiles <= 160 && nk % (2 * sp) == 0 && nk / (2 * sp) >= 2) sp *= 2;
    return sp;
}

cudaError_t forward_gemms(npp_proposal* P, cudaStream_t s)
{
    const int B = P->B;
    GemmEpilogue e;
    memset(&e, 0, sizeof e);
    e.err = P->err;
    e.mode = EPI_BIAS_RELU_BF16;
    e.bias = P->w + OFF_B1; e.out_bf16 = P->H1; e.ldo = HID; e.out_t = P->H1T; e.ldt = B;
    cudaError_t r = launch_gemm(P->tX, P->tW1, B, HID, D0, 128, e, s);
    if (r != cudaSuccess) return r;
    e.bias = P->w + OFF_B2; e.out_bf16 = P->H2; e.out_t = P->H2T;
    r = launch_gemm(P->tH1, P->tW2, B, HID, HID, 128, e, s);
    if (r != cudaSuccess) return r;
    memset(&e, 0, sizeof e);
    e.err = P->err;
    e.mode = EPI_BIAS_F32;
    e.bias = P->w + OFF_B3; e.out_f32 = P->Y; e.ldo = D3;
    return launch_gemm(P->tH2, P->tW3, B, D3, HID, 256, e, s);
}

cudaError_t backward_gemms(npp_proposal* P, cudaStream_t s)
{
    const int B = P->B;
    GemmEpilogue e;
    memset(&e, 0, sizeof e);
    e.err = P->err;
    // dZ2 = (dY W3) masked by H2 > 0
    e.mode = EPI_MASK_BF16;
    e.mask = P->H2; e.ldm = HID; e.out_bf16 = P->dZ2; e.ldo = HID; e.out_t = P->dZ2T; e.ldt = B;
    cudaError_t r = launch_gemm(P->tdY, P->tW3T, B, HID, D3, 128, e, s);
    if (r != cudaSuccess) return r;
    // dZ1 = (dZ2 W2) masked by H1 > 0 (transposed only)
    e.mask = P->H1; e.out_bf16 = nullptr; e.out_t = P->dZ1T;
    r = launch_gemm(P->tdZ2, P->tW2T, B, HID, HID, 128, e, s);
    if (r != cudaSuccess) return r;
    // weight gradients (K = B): K split into slices (partials in ws), then
    // summed in slice order into the flat gradient
    memset(&e, 0, sizeof e);
    e.err = P->err;
    e.mode = EPI_F32;
    e.out_f32 = P->ws + P->ws_off[0]; e.ldo = HID; e.split_stride = (size_t)D3 * HID;
    r = launch_gemm(P->tdYT, P->tH2T, D3, HID, B, 256, e, s, P->sp[0]);          // dW3 = dY^T H2
    if (r != cudaSuccess) return r;
    e.out_f32 = P->ws + P->ws_off[1]; e.ldo = HID; e.split_stride = (size_t)HID * HID;
    r = launch_gemm(P->tdZ2T, P->tH1T, HID, HID, B, 256, e, s, P->sp[1]);        // dW2 = dZ2^T H1
    if (r != cudaSuccess) return r;
    e.out_f32 = P->ws + P->ws_off[2]; e.ldo = D0; e.split_stride = (size_t)HID * D0;
    r = launch_gemm(P->tdZ1T, P->tXT, HID, D0, B, 128, e, s, P->sp[2]);          // dW1 = dZ1^T X
    if (r != cudaSuccess) return r;
    SplitSum ss;
    ss.src[0] = P->ws + P->ws_off[0]; ss.dst[0] = P->g + OFF_W3; ss.n[0] = D3 * HID; ss.splits[0] = P->sp[0];
    ss.src[1] = P->ws + P->ws_off[1]; ss.dst[1] = P->g + OFF_W2; ss.n[1] = HID * HID; ss.splits[1] = P->sp[1];
    ss.src[2] = P->ws + P->ws_off[2]; ss.dst[2] = P->g + OFF_W1; ss.n[2] = HID * D0; ss.splits[2] = P->sp[2];
    splitk_sum_kernel<<<(D3 * HID + HID * HID + HID * D0 + 255) / 256, 256, 0, s>>>(ss);
    return cudaGetLastError();
}

cudaError_t refresh_bf16(npp_proposal* P, cudaStream_t s)
{
    convert_kernel<<<512, 256, 0, s>>>(P->w, P->W1, P->W2, P->W2T, P->W3, P->W3T);
    return cudaGetLastError();
}

// packed public layout <-> padded flat layout
void packed_to_flat(const float* src, float* flat)
{
    std::memset(flat, 0, N_FLAT * sizeof(float));
    size_t o = 0;
    for (int r = 0; r < HID; ++r)
        for (int k = 0; k < NIN_X; ++k) flat[OFF_W1 + (size_t)r * D0 + k] = src[o++];
    for (int r = 0; r < HID; ++r) flat[OFF_B1 + r] = src[o++];
    for (int i = 0; i < HID * HID; ++i) flat[OFF_W2 + i] = src[o++];
    for (int r = 0; r < HID; ++r) flat[OFF_B2 + r] = src[o++];
    for (int i = 0; i < 2 * NTH * HID; ++i) flat[OFF_W3 + i] = src[o++];
    for (int r = 0; r < 2 * NTH; ++r) flat[OFF_B3 + r] = src[o++];
}

void flat_to_packed(const float* flat, float* dst)
{
    size_t o = 0;
    for (int r = 0; r < HID; ++r)
        for (int k = 0; k < NIN_X; ++k) dst[o++] = flat[OFF_W1 + (size_t)r * D0 + k];
    for (int r = 0; r < HID; ++r) dst[o++] = flat[OFF_B1 + r];
    for (int i = 0; i < HID * HID; ++i) dst[o++] = flat[OFF_W2 + i];
    for (int r = 0; r < HID; ++r) dst[o++] = flat[OFF_B2 + r];
    for (int i = 0; i < 2 * NTH * HID; ++i) dst[o++] = flat[OFF_W3 + i];
    for (int r = 0; r < 2 * NTH; ++r) dst[o++] = flat[OFF_B3 + r];
}

npp_status read_flat(npp_proposal* P, const float* dev, float* host_packed)
{
    float* flat = new float[N_FLAT];
    cudaError_t e = cudaMemcpy(flat, dev, N_FLAT * sizeof(float), cudaMemcpyDeviceToHost);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, P->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) flat_to_packed(flat, host_packed);
    delete[] flat;
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("proposal read: ") + cudaGetErrorString(e));
    if (err) return perr(NPP_DEVICE_TIMEOUT, "a proposal GEMM pipeline wait timed out");
    return NPP_OK;
}

}  // namespace

extern "C" {

int32_t npp_proposal_n_params(void) { return N_PACKED; }

npp_status npp_proposal_create(const npp_proposal_config* cfg, npp_proposal** out)
{
    if (!cfg || !out) return perr(NPP_INVALID_ARG, "npp_proposal_create: NULL argument");
    *out = nullptr;
    if (cfg->batch < 128 || cfg->batch % 128 || cfg->batch > 65536)
        return perr(NPP_INVALID_ARG, "proposal batch must be a multiple of 128 in [128, 65536]");
    if (!(cfg->ls_min < cfg->ls_max) || !(cfg->beta1 >= 0 && cfg->beta1 < 1) || !(cfg->beta2 >= 0 && cfg->beta2 < 1) ||
        !(cfg->eps > 0))
        return perr(NPP_INVALID_ARG, "proposal config: need ls_min < ls_max, 0 <= beta < 1, eps > 0");
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    npp_proposal* P = new npp_proposal;
    memset(P, 0, sizeof *P);
    P->cfg = *cfg;
    P->B = cfg->batch;
    const size_t B = (size_t)cfg->batch;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    A((void**)&P->w, N_FLAT * 4); A((void**)&P->m, N_FLAT * 4); A((void**)&P->v, N_FLAT * 4); A((void**)&P->g, N_FLAT * 4);
    A((void**)&P->W1, (size_t)HID * D0 * 2); A((void**)&P->W2, (size_t)HID * HID * 2); A((void**)&P->W2T, (size_t)HID * HID * 2);
    A((void**)&P->W3, (size_t)D3 * HID * 2); A((void**)&P->W3T, (size_t)D3 * HID * 2);
    A((void**)&P->X, B * D0 * 2); A((void**)&P->XT, B * D0 * 2);
    A((void**)&P->H1, B * HID * 2); A((void**)&P->H1T, B * HID * 2);
    A((void**)&P->H2, B * HID * 2); A((void**)&P->H2T, B * HID * 2);
    A((void**)&P->dY, B * D3 * 2); A((void**)&P->dYT, B * D3 * 2);
    A((void**)&P->dZ2, B * HID * 2); A((void**)&P->dZ2T, B * HID * 2); A((void**)&P->dZ1T, B * HID * 2);
    A((void**)&P->Y, B * D3 * 4);
    A((void**)&P->loss, sizeof(float));
    A((void**)&P->err, sizeof(int));
    const int nkb = cfg->batch / 64;
    P->sp[0] = grad_splits((D3 / 128) * (HID / 256), nkb);
    P->sp[1] = grad_splits((HID / 128) * (HID / 256), nkb);
    P->sp[2] = grad_splits((HID / 128) * (D0 / 128), nkb);
    P->ws_off[0] = 0;
    P->ws_off[1] = P->ws_off[0] + (size_t)P->sp[0] * D3 * HID;
    P->ws_off[2] = P->ws_off[1] + (size_t)P->sp[1] * HID * HID;
    A((void**)&P->ws, (P->ws_off[2] + (size_t)P->sp[2] * HID * D0) * 4);
    if (e == cudaSuccess) e = cudaMemset(P->w, 0, N_FLAT * 4);
    if (e == cudaSuccess) e = cudaMemset(P->m, 0, N_FLAT * 4);
    if (e == cudaSuccess) e = cudaMemset(P->v, 0, N_FLAT * 4);
    if (e == cudaSuccess) e = cudaMemset(P->g, 0, N_FLAT * 4);
    if (e == cudaSuccess) e = cudaMemset(P->err, 0, sizeof(int));
    // the padding outputs' gradient rows stay zero (the loss kernel writes 0..899)
    if (e == cudaSuccess) e = cudaMemset(P->dY, 0, B * D3 * 2);
    if (e == cudaSuccess) e = cudaMemset(P->dYT, 0, B * D3 * 2);
    if (e != cudaSuccess) {
        npp_proposal_destroy(P);
        return perr(NPP_CUDA_ERROR, std::string("proposal allocation: ") + cudaGetErrorString(e));
    }
    const int b = cfg->batch;
    // A operands: boxes of 128 rows; B operands: boxes of the tile width
    // (128 for the N = 256 products over the batch: twice the CTAs of
    // 256-wide tiles, on 152 SMs)
    struct M { CUtensorMap* map; const void* base; int rows, cols, box; } maps[] = {
        { &P->tX, P->X, b, D0, 128 },     { &P->tW1, P->W1, HID, D0, 128 },
        { &P->tH1, P->H1, b, HID, 128 },  { &P->tW2, P->W2, HID, HID, 128 },
        { &P->tH2, P->H2, b, HID, 128 },  { &P->tW3, P->W3, D3, HID, 256 },
        { &P->tdY, P->dY, b, D3, 128 },   { &P->tW3T, P->W3T, HID, D3, 128 },
        { &P->tdZ2, P->dZ2, b, HID, 128 }, { &P->tW2T, P->W2T, HID, HID, 128 },
        { &P->tdYT, P->dYT, D3, b, 128 }, { &P->tH2T, P->H2T, HID, b, 256 },
        { &P->tdZ2T, P->dZ2T, HID, b, 128 }, { &P->tH1T, P->H1T, HID, b, 256 },
        { &P->tdZ1T, P->dZ1T, HID, b, 128 }, { &P->tXT, P->XT, D0, b, 128 },
    };
    for (auto& mp : maps) {
        e = make_tmap_bf16(mp.map, mp.base, mp.rows, mp.cols, mp.box);
        if (e != cudaSuccess) {
            npp_proposal_destroy(P);
            return perr(NPP_CUDA_ERROR, std::string("tensor map: ") + cudaGetErrorString(e));
        }
    }
    e = refresh_bf16(P, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        npp_proposal_destroy(P);
        return perr(NPP_CUDA_ERROR, std::string("proposal init: ") + cudaGetErrorString(e));
    }
    *out = P;
    return NPP_OK;
}

npp_status npp_proposal_destroy(npp_proposal* P)
{
    if (!P) return NPP_OK;
    cudaSetDevice(P->cfg.device);
    cudaDeviceSynchronize();
    void* ptrs[] = { P->w, P->m, P->v, P->g, P->W1, P->W2, P->W2T, P->W3, P->W3T, P->X, P->XT, P->H1, P->H1T,
                     P->H2, P->H2T, P->dY, P->dYT, P->dZ2, P->dZ2T, P->dZ1T, P->Y, P->loss, P->err, P->ws };
    for (void* p : ptrs) if (p) cudaFree(p);
    delete P;
    return NPP_OK;
}

npp_status npp_proposal_set_params(npp_proposal* P, const float* params_host)
{
    if (!P || !params_host) return perr(NPP_INVALID_ARG, "npp_proposal_set_params: NULL argument");
    for (int i = 0; i < N_PACKED; ++i)
        if (!std::isfinite(params_host[i])) return perr(NPP_INVALID_ARG, "proposal parameters must be finite");
    cudaSetDevice(P->cfg.device);
    float* flat = new float[N_FLAT];
    packed_to_flat(params_host, flat);
    cudaError_t e = cudaMemcpy(P->w, flat, N_FLAT * 4, cudaMemcpyHostToDevice);
    delete[] flat;
    if (e == cudaSuccess) e = cudaMemset(P->m, 0, N_FLAT * 4);
    if (e == cudaSuccess) e = cudaMemset(P->v, 0, N_FLAT * 4);
    if (e == cudaSuccess) e = refresh_bf16(P, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("proposal set: ") + cudaGetErrorString(e));
    P->t = 0;
    return NPP_OK;
}

npp_status npp_proposal_get_params(npp_proposal* P, float* params_host)
{
    if (!P || !params_host) return perr(NPP_INVALID_ARG, "npp_proposal_get_params: NULL argument");
    cudaSetDevice(P->cfg.device);
    return read_flat(P, P->w, params_host);
}

npp_status npp_proposal_get_grads(npp_proposal* P, float* grads_host)
{
    if (!P || !grads_host) return perr(NPP_INVALID_ARG, "npp_proposal_get_grads: NULL argument");
    cudaSetDevice(P->cfg.device);
    return read_flat(P, P->g, grads_host);
}

npp_status npp_proposal_encode(const npp_handle* h, const npp_scene* scenes_dev, int32_t S, const float* obs_dev,
                               float* x_dev, void* stream)
{
    if (!h || !scenes_dev || !x_dev || S < 0) return perr(NPP_INVALID_ARG, "npp_proposal_encode: bad arguments");
    if (S == 0) return NPP_OK;
    if (!obs_dev || (reinterpret_cast<uintptr_t>(obs_dev) & 15u))
        return perr(NPP_INVALID_ARG, "npp_proposal_encode: obstacle array must be non-NULL and 16-byte aligned");
    cudaSetDevice(h->device);
    encode_kernel<<<S, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        h->dc, scenes_dev, reinterpret_cast<const float4*>(obs_dev), x_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("encode launch: ") + cudaGetErrorString(e));
    return NPP_OK;
}

npp_status npp_proposal_forward(npp_proposal* P, const float* x_dev, int32_t n, float* mean_dev, float* std_dev,
                                void* stream)
{
    if (!P || !x_dev || !mean_dev || !std_dev) return perr(NPP_INVALID_ARG, "npp_proposal_forward: NULL argument");
    if (n < 1 || n > P->B) return perr(NPP_INVALID_ARG, "npp_proposal_forward: n outside [1, batch]");
    cudaSetDevice(P->cfg.device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pack_x_kernel<<<P->B / PX_TB, 256, 0, s>>>(x_dev, n, P->B, P->X, P->XT);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward_gemms(P, s);
    if (e == cudaSuccess) {
        mean_std_kernel<<<256, 256, 0, s>>>(P->Y, n, P->cfg.ls_min, P->cfg.ls_max, mean_dev, std_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("proposal forward: ") + cudaGetErrorString(e));
    return NPP_OK;
}

npp_status npp_proposal_train_step(npp_proposal* P, const float* x_dev, const float* theta_dev, float lr,
                                   float* loss_dev, void* stream)
{
    if (!P || !x_dev || !theta_dev) return perr(NPP_INVALID_ARG, "npp_proposal_train_step: NULL argument");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return perr(NPP_INVALID_ARG, "learning rate must be finite and >= 0");
    cudaSetDevice(P->cfg.device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int B = P->B;
    pack_x_kernel<<<B / PX_TB, 256, 0, s>>>(x_dev, B, B, P->X, P->XT);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward_gemms(P, s);
    float* lp = loss_dev ? loss_dev : P->loss;
    if (e == cudaSuccess) e = cudaMemsetAsync(lp, 0, sizeof(float), s);
    if (e == cudaSuccess) {
        nll_kernel<<<dim3((NTH + NLL_TI - 1) / NLL_TI, B / NLL_TB), 256, 0, s>>>(P->Y, theta_dev, B, P->cfg.ls_min,
                                                                        P->cfg.ls_max, P->dY, P->dYT, lp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward_gemms(P, s);
    if (e == cudaSuccess) {
        bias_grad_kernel<<<(D3 + 2 * HID) / 8, 256, 0, s>>>(P->dYT, P->dZ2T, P->dZ1T, B, P->g);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        P->t += 1;
        const double c1 = 1.0 - std::pow((double)P->cfg.beta1, P->t);
        const double c2 = 1.0 - std::pow((double)P->cfg.beta2, P->t);
        adam_kernel<<<512, 256, 0, s>>>(P->w, P->m, P->v, P->g, N_FLAT, lr, P->cfg.beta1, P->cfg.beta2, P->cfg.eps,
                                        (float)c1, (float)c2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = refresh_bf16(P, s);
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("proposal train step: ") + cudaGetErrorString(e));
    return NPP_OK;
}

npp_status npp_gemm_bf16(const uint16_t* A_dev, const uint16_t* B_dev, float* C_dev, int32_t M, int32_t N,
                         int32_t K, void* stream)
{
    if (!A_dev || !B_dev || !C_dev) return perr(NPP_INVALID_ARG, "npp_gemm_bf16: NULL argument");
    if (M < 128 || M % 128 || N < 128 || N % 128 || K < 64 || K % 64)
        return perr(NPP_INVALID_ARG, "npp_gemm_bf16: M, N multiples of 128 and K a multiple of 64");
    const int bn = (N % 256 == 0) ? 256 : 128;
    CUtensorMap ta, tb;
    cudaError_t e = make_tmap_bf16(&ta, A_dev, M, K, 128);
    if (e == cudaSuccess) e = make_tmap_bf16(&tb, B_dev, N, K, bn);
    if (e != cudaSuccess) return perr(NPP_INVALID_ARG, "npp_gemm_bf16: operands must be 16-byte aligned");
    int* err = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_gemm_err);
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("gemm error flag: ") + cudaGetErrorString(e));
    GemmEpilogue ep;
    memset(&ep, 0, sizeof ep);
    ep.mode = EPI_F32;
    ep.out_f32 = C_dev;
    ep.ldo = N;
    ep.err = err;
    e = launch_gemm(ta, tb, M, N, K, bn, ep, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("gemm launch: ") + cudaGetErrorString(e));
    return NPP_OK;
}

npp_status npp_gemm_status(void)
{
    int err = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&err, g_gemm_err, sizeof(int));
    if (e != cudaSuccess) return perr(NPP_CUDA_ERROR, std::string("gemm status: ") + cudaGetErrorString(e));
    if (err) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_gemm_err, &zero, sizeof(int));
        return perr(NPP_DEVICE_TIMEOUT, "a GEMM pipeline wait timed out");
    }
    return NPP_OK;
}

}  // extern "C"
