// Tensor-core (tcgen05, kind::tf32, three-pass split) complex contraction.  See tc_gemm.cu.
#pragma once
#include "common.cuh"

namespace tns {

// C[M x Nr] = A[M x Kr] * B[Nr x Kr]^T in real FP32 storage, where A is a complex
// M x (Kr/2) matrix read as interleaved reals and B the real block expansion of a
// complex (Nr/2) x (Kr/2) operand (expand_b).  Alo is the TF32 remainder of A
// (tf32_lo); Bhi/Blo come from expand_b.  Row strides in floats.  err: device int
// set to 1 if a pipeline wait timed out (results then invalid).
cudaError_t tc_gemm_tf32x3(const float* A, const float* Alo, long long M, int Kr, long long lda, const float* Bhi,
                           const float* Blo, int Nr, long long ldb, float* C, long long ldc, int* err,
                           cudaStream_t st);
bool tc_gemm_supported(long long M, int Nr, int Kr, long long lda, long long ldb, long long ldc);

cudaError_t tf32_lo(const float* x, float* lo, long long n, cudaStream_t st);

// Expand a complex operand E (complex64, element (n, k) at n1*sN1 + n2*sN2 + k1*sK1 +
// k2*sK2 with n = n1*N2 + n2, k = k1*K2 + k2) into the real 2N x 2K block matrix.
cudaError_t expand_b(const void* E, int N1, int N2, long long sN1, long long sN2, int K1, int K2, long long sK1,
                     long long sK2, float* Bhi, float* Blo, cudaStream_t st);

}  // namespace tns
