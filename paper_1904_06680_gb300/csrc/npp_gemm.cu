// npp_gemm.cu -- BF16 GEMM on the fifth-generation tensor cores.
//
// A persistent kernel: one CTA of 192 threads per SM walks 128 x BN tiles
// of C (and, with split K, slices of their K blocks):
//   warp 0, one lane   TMA producer: K blocks of 64 (128 bytes of BF16, the
//                      128-byte swizzle atom) of A and B into a ring of
//                      STAGES shared-memory stages, completion counted by
//                      the stage's "full" mbarrier;
//   warp 1, one lane   MMA issuer: four tcgen05.mma (M = 128, N = BN,
//                      K = 16) per stage into one of two TMEM accumulators
//                      of BN FP32 columns (alternating by tile), then
//                      tcgen05.commit frees the stage ("empty"); after a
//                      tile's last stage a commit hands the accumulator to
//                      the epilogue ("tfull");
//   warps 2-5          epilogue: warp w reads TMEM lanes 32 (w % 4) ..
//                      32 (w % 4) + 31 (rows) with tcgen05.ld, applies the
//                      fused epilogue, stores, and returns the accumulator
//                      ("tempty") -- while the MMAs of the next tile run on
//                      the other one.
// Every wait on an mbarrier is bounded (about a second of clock): on a
// timeout the CTA records an error code, stops issuing, waits (bounded) for
// the copies it issued, frees its TMEM and returns.
#include "npp_gemm.cuh"
#include "npp_async.cuh"

#include <cudaTypedefs.h>

#include <algorithm>

namespace npp {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int STAGES = 4;

template <int BN>
struct GemmShape {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 128;   // + alignment slack + barriers
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major operand in 128-byte swizzle
// atoms (8 rows x 128 bytes, atoms 1024 bytes apart along the rows)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);         // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = bn
__host__ __device__ constexpr uint32_t mma_idesc(int bn)
{
    return (1u << 4)                  // D: FP32
         | (1u << 7)                  // A: BF16
         | (1u << 10)                 // B: BF16
         | ((uint32_t)(bn >> 3) << 17)
         | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int GEMM_GROUP_M = 16;
constexpr int GEMM_THREADS = 192;

// one 128 x BN tile's accumulator rows (TMEM lanes 32 q .. 32 q + 31 at
// trow, this thread's row `row`) through the fused epilogue to global memory
template <int BN>
__device__ __forceinline__ void store_rows(const GemmEpilogue& ep, uint32_t trow, int row, int n0, int z)
{
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld16(trow + c, v);
        const int n = n0 + c;
        if (ep.mode == EPI_F32 || ep.mode == EPI_BIAS_F32) {
            if (ep.mode == EPI_BIAS_F32)
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += ep.bias[n + i];
            float4* o = reinterpret_cast<float4*>(ep.out_f32 + (size_t)z * ep.split_stride + (size_t)row * ep.ldo + n);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        } else {
            __nv_bfloat16 hb[16];
            if (ep.mode == EPI_BIAS_RELU_BF16) {
#pragma unroll
                for (int i = 0; i < 16; ++i) hb[i] = __float2bfloat16_rn(fmaxf(v[i] + ep.bias[n + i], 0.0f));
            } else {
                const __nv_bfloat16* mk = ep.mask + (size_t)row * ep.ldm + n;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    hb[i] = __float2bfloat16_rn(__bfloat162float(mk[i]) > 0.0f ? v[i] : 0.0f);
            }
            if (ep.out_bf16) {
                uint4* o = reinterpret_cast<uint4*>(ep.out_bf16 + (size_t)row * ep.ldo + n);
                const uint4* src = reinterpret_cast<const uint4*>(hb);
                o[0] = src[0];
                o[1] = src[1];
            }
            if (ep.out_t) {
#pragma unroll
                for (int i = 0; i < 16; ++i) ep.out_t[(size_t)(n + i) * ep.ldt + row] = hb[i];
            }
        }
    }
}

// Work unit u = (tile, K slice): tile u % tiles in the grouped order
// (consecutive units walk GEMM_GROUP_M row tiles before the next column
// tile, so the CTAs busy at once share a few tiles of A and of B in L2),
// slice u / tiles.
__device__ __forceinline__ void unit_coords(int u, int tiles, int n_tiles, int m_tiles, int bn, int& m0, int& n0,
                                            int& z)
{
    const int pid = u % tiles;
    z = u / tiles;
    const int per_group = GEMM_GROUP_M * n_tiles;
    const int first_m = (pid / per_group) * GEMM_GROUP_M;
    const int gsize = min(m_tiles - first_m, GEMM_GROUP_M);
    const int in_group = pid % per_group;
    m0 = (first_m + in_group % gsize) * BM;
    n0 = (in_group / gsize) * bn;
}

// Persistent GEMM: each CTA (one per SM) walks the work units
// blockIdx.x, blockIdx.x + gridDim.x, ...  The MMAs of a CTA's i-th unit go
// to TMEM accumulator i % 2 (BN columns each) while warps 2-5 drain the
// other one through the epilogue, so a tile's epilogue overlaps the next
// tile's MMAs; the operand ring and its barrier phases run on across units.
template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N, int K,
            int splits, const GemmEpilogue ep)
{
    using S = GemmShape<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * S::STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;          // [2] accumulator ready for the epilogue
    uint64_t* tempty = tfull + 2;              // [2] accumulator drained by the epilogue (128 arrivals)
    uint64_t* done = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* flags = reinterpret_cast<int*>(tmem_slot + 1);      // [0] abort, [1] issued, [2] consumed

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = N / BN, m_tiles = M / BM, tiles = n_tiles * m_tiles;
    const int units = tiles * splits;
    const int nk = K / BK / splits;            // K blocks per unit

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 128);
        }
        mbar_init(done, 1);
        flags[0] = 0;
        flags[1] = 0;
        flags[2] = 0;
        mbar_init_fence();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(2 * BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

    if (warp == 0 && lane == 0) {
        // TMA producer
        int g = 0;                             // K blocks issued by this CTA
        bool stop = false;
        for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
            int m0, n0, z;
            unit_coords(u, tiles, n_tiles, m_tiles, BN, m0, n0, z);
            for (int kb = 0; kb < nk; ++kb, ++g) {
                const int s = g % STAGES;
                if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1)) {
                    atomicExch(&flags[0], 1);
                    stop = true;
                    break;
                }
                if (*reinterpret_cast<volatile int*>(&flags[0])) {
                    stop = true;
                    break;
                }
                uint8_t* st = smem + s * S::STAGE_BYTES;
                const int kc = (z * nk + kb) * BK;
                mbar_expect_tx(&full[s], S::STAGE_BYTES);
                tma_load_2d(st, &ta, kc, m0, &full[s]);
                tma_load_2d(st + S::A_BYTES, &tb, kc, n0, &full[s]);
            }
        }
        flags[1] = g;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = mma_idesc(BN);
        int g = 0, i = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < units && !stop; u += gridDim.x, ++i) {
            const int b = i & 1;
            // the accumulator's previous tile drained (its first use passes at once)
            if (!mbar_wait(&tempty[b], ((i >> 1) & 1) ^ 1)) {
                atomicExch(&flags[0], 1);
                break;
            }
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)(b * BN);
            for (int kb = 0; kb < nk; ++kb, ++g) {
                const int s = g % STAGES;
                if (!mbar_wait(&full[s], (g / STAGES) & 1)) {
                    atomicExch(&flags[0], 1);
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(smem + s * S::STAGE_BYTES);
                const uint32_t b0 = a0 + S::A_BYTES;
#pragma unroll
                for (int j = 0; j < BK / 16; ++j)
                    mma_bf16(acc, sw128_desc(a0 + j * 32), sw128_desc(b0 + j * 32), idesc, (kb | j) != 0);
                mma_commit(&empty[s]);
            }
            if (!stop) mma_commit(&tfull[b]);  // arrives once this unit's MMAs have completed
        }
        flags[2] = g;
        mma_commit(done);
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31
        const int q = warp & 3;
        int i = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++i) {
            const int b = i & 1;
            const bool ok = mbar_wait(&tfull[b], (i >> 1) & 1);
            if (!__all_sync(0xffffffffu, ok) || *reinterpret_cast<volatile int*>(&flags[0])) {
                atomicExch(&flags[0], 1);
                break;
            }
            tc_fence_after();
            int m0, n0, z;
            unit_coords(u, tiles, n_tiles, m_tiles, BN, m0, n0, z);
            store_rows<BN>(ep, tmem + (uint32_t)(b * BN) + ((uint32_t)(q * 32) << 16), m0 + q * 32 + lane, n0, z);
            tc_fence_before();
            mbar_arrive(&tempty[b]);
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0) {
        // every MMA complete before the TMEM goes back; after a timeout the
        // copies issued but never consumed land first (bounded waits)
        const bool ok = mbar_wait(done, 0);
        if (!ok || *reinterpret_cast<volatile int*>(&flags[0])) {
            if (ep.err) atomicExch(ep.err, 1);
            for (int g = flags[2]; g < flags[1]; ++g) mbar_wait(&full[g % STAGES], (g / STAGES) & 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
    }
}

int sm_count()
{
    static int cnt[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (cnt[dev] == 0) {
        int c = 0;
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 148;
        cnt[dev] = c;
    }
    return cnt[dev];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

cudaError_t make_tmap_bf16(CUtensorMap* map, const void* base, int rows, int cols, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || cols % 64 || rows % box_rows) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = { (cuuint64_t)cols, (cuuint64_t)rows };
    cuuint64_t strides[1] = { (cuuint64_t)cols * 2 };
    cuuint32_t box[2] = { 64u, (cuuint32_t)box_rows };
    cuuint32_t estr[2] = { 1u, 1u };
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int bn,
                        const GemmEpilogue& ep, cudaStream_t s, int splits)
{
    if (M % BM || K % BK || K < BK || (bn != 128 && bn != 256) || N % bn) return cudaErrorInvalidValue;
    if (splits < 1 || (K / BK) % splits || (splits > 1 && (ep.mode != EPI_F32 || ep.split_stride == 0)))
        return cudaErrorInvalidValue;
    const int units = (M / BM) * (N / bn) * splits;
    const int grid = std::min(units, sm_count());
    if (bn == 256) {
        const int smem = GemmShape<256>::SMEM;
        cudaError_t e = cudaFuncSetAttribute(gemm_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        gemm_kernel<256><<<grid, GEMM_THREADS, smem, s>>>(ta, tb, M, N, K, splits, ep);
    } else {
        const int smem = GemmShape<128>::SMEM;
        cudaError_t e = cudaFuncSetAttribute(gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        gemm_kernel<128><<<grid, GEMM_THREADS, smem, s>>>(ta, tb, M, N, K, splits, ep);
    }
    return cudaGetLastError();
}

}  // namespace npp
