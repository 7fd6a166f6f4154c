// npp_gemm.cuh -- BF16 tensor-core GEMM (tcgen05 + TMA) with the fused
// epilogues the sampling-proposal network needs.
//
//   C[m][n] = sum_k A[m][k] B[n][k]      A: M x K, B: N x K, both BF16 with K
//                                        contiguous ("K-major"), FP32 sums
//
// M a multiple of 128, N of the tile width BN (128 or 256), K of 64.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace npp {

enum GemmEpi {
    EPI_F32 = 0,             // out_f32[m][n] = acc
    EPI_BIAS_F32 = 1,        // out_f32[m][n] = acc + bias[n]
    EPI_BIAS_RELU_BF16 = 2,  // h = bf16(max(acc + bias[n], 0)) -> out_bf16[m][n], out_t[n][m]
    EPI_MASK_BF16 = 3,       // g = bf16(mask[m][n] > 0 ? acc : 0) -> out_bf16[m][n], out_t[n][m]
};

struct GemmEpilogue {
    int mode;
    float* out_f32;                  // row-major, leading dimension ldo
    __nv_bfloat16* out_bf16;         // row-major, leading dimension ldo (may be null)
    __nv_bfloat16* out_t;            // transposed [n][m], leading dimension ldt (may be null)
    const float* bias;               // [N]
    const __nv_bfloat16* mask;       // row-major, leading dimension ldm
    int ldo, ldt, ldm;
    int* err;                        // set to a nonzero code if a pipeline wait timed out
    size_t split_stride;             // split K (EPI_F32 only): slice z of K writes out_f32 + z split_stride
};

// TMA descriptor of a row-major BF16 matrix [rows][cols] (cols contiguous,
// a multiple of 64; base 16-byte aligned) read in boxes of box_rows x 64.
cudaError_t make_tmap_bf16(CUtensorMap* map, const void* base, int rows, int cols, int box_rows);

// C = A B^T with the epilogue; ta boxes of 128 rows, tb boxes of bn rows.
// splits > 1 (EPI_F32 only; K / 64 a multiple of splits): slice z of the K
// blocks is summed into its own FP32 partial C at out_f32 + z split_stride,
// for the caller to add up.
cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int bn,
                        const GemmEpilogue& ep, cudaStream_t s, int splits = 1);

}  // namespace npp
