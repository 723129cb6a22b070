// FP32-accurate dense products on the tensor cores (csrc/mlp.cu): operands
// split three ways into BF16 (x = x1 + x2 + x3) and the six significant
// cross products accumulated in FP32 by two tcgen05 launches (a1 b1, then
// the five smaller products added to it).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace scs {
namespace mlp {

// dst (rows x 3 Kp BF16, row-major: chunks x1 | x2 | x3, each zero-padded
// from K to Kp columns) from src rows x K, element (r, k) at src[r ld + k]
// (trans = 0) or src[k ld + r] (trans = 1).  Enqueued on `stream`.
void split3_bf16(const float *src, int rows, int K, int64_t ld, int trans, int Kp, __nv_bfloat16 *dst,
                 cudaStream_t stream);

// C'(r, c) = alpha sum_k A(r, k) B(c, k) + beta C'(r, c) for r < rows_a,
// c < rows_b, stored at C[r ldc + c]; A3, B3 split by split3_bf16 with the
// same Kp (a multiple of 64).  *err (device) is set if a bounded wait of the
// kernel timed out.  Throws CudaError on bad arguments.
void gemm_fp32x3(const __nv_bfloat16 *A3, int rows_a, const __nv_bfloat16 *B3, int rows_b, int Kp, float *C,
                 int64_t ldc, float alpha, float beta, int *err, cudaStream_t stream);

}  // namespace mlp
}  // namespace scs
