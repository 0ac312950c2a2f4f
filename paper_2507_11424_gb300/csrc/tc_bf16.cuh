// BF16 tensor-core GEMM with the learned proposal's epilogue.  See tc_bf16.cu.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace tns {

// C = A B^T over K (A: M x K, B: N x K, BF16, K contiguous; pitches lda / ldb in
// elements, multiples of 8; 16-byte aligned bases).  Epilogue per element (m, n):
//   v = C + bias[n] (bias optional); v = 0 where gate[m * ldc + n] <= 0 (gate
//   optional); Cf[m * ldc + n] = v (optional); Cb[m * ldcb + n] = bf16(relu ?
//   max(v, 0) : v) (optional).  err: device flag set when a pipeline wait timed out.
struct Bf16Gemm {
  int M, N, K;
  float* Cf;
  __nv_bfloat16* Cb;
  long long ldc, ldcb;
  const float* bias;
  int relu;
  const float* gate;
  int* err;
};

cudaError_t tc_gemm_bf16(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B, long long ldb,
                         const Bf16Gemm& g, cudaStream_t st);
// out[c][r] = in[r][c] (rows x cols of `in`, pitches in elements).
cudaError_t bf16_transpose(const __nv_bfloat16* in, long long ldi, int rows, int cols, __nv_bfloat16* out,
                           long long ldo, cudaStream_t st);

}  // namespace tns
