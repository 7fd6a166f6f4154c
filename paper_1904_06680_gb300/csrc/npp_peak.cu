// npp_peak.cu -- FP32 fused multiply-add throughput of the device, the
// denominator of the rollout kernels' roofline: every thread runs eight
// independent FMA chains (or four packed FP32x2 chains, eight FMAs per
// step), enough blocks to fill every SM, timed with CUDA events.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_internal.h"
#include "npp_async.cuh"

namespace {

// The bounded mbarrier wait of the staging copies and the GEMM pipeline on
// a barrier of one expected arrival: with `arrive` the block's first thread
// arrives and the phase completes; without it nothing ever arrives and the
// wait must give up after `limit` cycles and report it.
__global__ void wait_probe_kernel(long long limit, int arrive, int* out)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        npp::mbar_init(&bar, 1);
        npp::mbar_init_fence();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) npp::mbar_arrive(&bar);
    const bool done = npp::mbar_wait(&bar, 0, limit);
    if (threadIdx.x == 0) *out = done ? 1 : 0;
}

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;

template <bool PACKED>
__global__ void __launch_bounds__(PEAK_THREADS) fma_peak_kernel(float* __restrict__ sink, int iters, float m, float c)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    if constexpr (PACKED) {
        unsigned long long p[4], mm, cc;
        asm("mov.b64 %0, {%1, %1};" : "=l"(mm) : "f"(m));
        asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
        for (int k = 0; k < 4; ++k) asm("mov.b64 %0, {%1, %2};" : "=l"(p[k]) : "f"(a[2 * k]), "f"(a[2 * k + 1]));
#pragma unroll 4
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 4; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[k]) : "l"(mm), "l"(cc));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) asm("mov.b64 {%0, %1}, %2;" : "=f"(a[2 * k]), "=f"(a[2 * k + 1]) : "l"(p[k]));
    } else {
#pragma unroll 4
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 123456.0f) sink[blockIdx.x * PEAK_THREADS + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" npp_status npp_measure_fma_peak(int32_t device, int32_t packed, double* fma_per_s)
{
    if (!fma_per_s || (packed != 0 && packed != 1)) {
        npp::set_global_error("npp_measure_fma_peak: NULL output or packed not 0/1");
        return NPP_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
        cudaSetDevice(device) != cudaSuccess) {
        npp::set_global_error("npp_measure_fma_peak: CUDA device not available");
        return NPP_CUDA_ERROR;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (sms < 1) return NPP_CUDA_ERROR;
    const int blocks = sms * PEAK_BLOCKS_PER_SM;
    const int iters = 8192;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&sink, sizeof(float) * blocks * PEAK_THREADS);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {     // rep 0 warms up
        cudaEventRecord(e0);
        if (packed) fma_peak_kernel<true><<<blocks, PEAK_THREADS>>>(sink, iters, 0.999f, 1e-3f);
        else fma_peak_kernel<false><<<blocks, PEAK_THREADS>>>(sink, iters, 0.999f, 1e-3f);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best_ms == 0.0f || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess || !(best_ms > 0.0f)) {
        npp::set_global_error("npp_measure_fma_peak: timed launch failed");
        return NPP_CUDA_ERROR;
    }
    *fma_per_s = (double)blocks * PEAK_THREADS * (double)iters * 8.0 / (best_ms * 1e-3);
    return NPP_OK;
}

extern "C" npp_status npp_wait_probe(int64_t limit_cycles, int32_t arrive, int32_t* completed_host)
{
    if (!completed_host || limit_cycles < 1 || limit_cycles > 4000000000LL || (arrive != 0 && arrive != 1)) {
        npp::set_global_error("npp_wait_probe: limit outside [1, 4e9] cycles, arrive not 0/1 or NULL output");
        return NPP_INVALID_ARG;
    }
    int* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        wait_probe_kernel<<<1, 32>>>((long long)limit_cycles, arrive, d);
        e = cudaGetLastError();
    }
    int v = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&v, d, sizeof(int), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        npp::set_global_error("npp_wait_probe: launch or copy failed");
        return NPP_CUDA_ERROR;
    }
    *completed_host = v;
    return NPP_OK;
}
