// Test helper: raw Philox4x32-10 blocks from cuRAND's device API, an
// independent implementation to pin the oracle's generator against.
// Input (stdin): lines "seed subsequence offset"; output: the first
// curand4() block after curand_init(seed, subsequence, offset) as four
// unsigned integers per line.
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void first_block(const unsigned long long* args, uint4* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(args[3 * i], args[3 * i + 1], args[3 * i + 2], &st);
    out[i] = curand4(&st);
}

int main()
{
    std::vector<unsigned long long> a;
    unsigned long long s, q, o;
    while (std::scanf("%llu %llu %llu", &s, &q, &o) == 3) { a.push_back(s); a.push_back(q); a.push_back(o); }
    const int n = (int)(a.size() / 3);
    if (n == 0) return 1;
    unsigned long long* d_a = nullptr;
    uint4* d_o = nullptr;
    if (cudaMalloc(&d_a, a.size() * sizeof(unsigned long long)) != cudaSuccess) return 2;
    if (cudaMalloc(&d_o, n * sizeof(uint4)) != cudaSuccess) return 2;
    cudaMemcpy(d_a, a.data(), a.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    first_block<<<(n + 127) / 128, 128>>>(d_a, d_o, n);
    std::vector<uint4> h(n);
    if (cudaMemcpy(h.data(), d_o, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    for (int i = 0; i < n; ++i) std::printf("%u %u %u %u\n", h[i].x, h[i].y, h[i].z, h[i].w);
    cudaFree(d_a);
    cudaFree(d_o);
    return 0;
}
