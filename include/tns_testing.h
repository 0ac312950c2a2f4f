/*
 * tns_testing.h -- test-only entry points of libtns.so that expose internal
 * device primitives, so the test suite can check them against the CPU oracle
 * one by one.  Not part of the sampling API; same conventions as tns.h
 * (caller-owned device buffers, tns_status return codes).
 */
#ifndef TNS_TESTING_H
#define TNS_TESTING_H

#include <stdint.h>
#include "tns.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 (Salmon et al., SC'11) evaluated on the device.
 *   ctr_key_dev  device uint32 [n][6]: counter words 0..3, key words 0..1
 *   out_dev      device uint32 [n][4]: output words */
tns_status tns_test_philox(int64_t n, const uint32_t* ctr_key_dev, uint32_t* out_dev, void* cuda_stream);

/* Batched FP64 Hermitian eigendecomposition by parallel Jacobi.
 *   A_dev    device complex128 [batch][n][n] (read only)
 *   lam_dev  device float64 [batch][n], descending
 *   V_dev    device complex128 [batch][n][n], column j = eigenvector j */
tns_status tns_test_eigh(int32_t batch, int32_t n, const double* A_dev, double* lam_dev, double* V_dev,
                         void* cuda_stream);

/* The FP32 variant of the eigensolver used by the mixed-precision truncation:
 * A_dev complex64 [batch][n][n] Hermitian (read only), lam_dev float64 [batch][n]
 * descending, V_dev complex128 [batch][n][n] (column j = eigenvector j).  Sweep
 * counts are reported through tns_test_eigh_sweeps like tns_test_eigh's. */
tns_status tns_test_eigh32(int32_t batch, int32_t n, const float* A_dev, double* lam_dev, double* V_dev,
                           void* cuda_stream);

/* Sweeps used by each matrix of the last tns_test_eigh call (host int32 [batch]);
 * a value of 0 or less means the sweep cap was reached. */
tns_status tns_test_eigh_sweeps(int32_t batch, int32_t* sweeps_host);

/* Orthonormalising map of the range finder: W = L^{-H} with
 * L L^H = G + shift * max_i G_ii * I.
 *   G_dev  device complex128 [batch][n][n] Hermitian PSD; W_dev complex128 [batch][n][n] */
tns_status tns_test_cholw(int32_t batch, int32_t n, double shift, const double* G_dev, double* W_dev,
                          void* cuda_stream);

/* Tensor-core complex GEMM used by the mixed-precision contractions:
 * C = A B^T with A complex64 [M][K], B complex64 [N][K] (K contiguous), C complex64
 * [M][N], computed by tcgen05 kind::tf32 with a three-pass hi/lo split.
 * Returns TNS_ERR_STATE when the shape is not supported by the tensor-core path
 * and TNS_ERR_NUMERIC when a pipeline wait timed out. */
tns_status tns_test_tcgemm(int64_t M, int32_t N, int32_t K, const float* A_dev, const float* B_dev, float* C_dev,
                           void* cuda_stream);

/* Force the tensor-core GEMM's tile variant for later launches: 128 or 256 real
 * columns with a pipelined ring of stages, 129 for 128 columns with one stage and
 * three CTAs per SM, or 0 for the variant the library's timing-based choice picks per
 * shape class (256 is taken as 128 for outputs of up to 64 complex columns). */
tns_status tns_test_tc_tile(int32_t bn);

/* The library's labelled tensor contraction C[c] = sum A[a] B[b] (einsum over the
 * label strings: labels in all three operands are batch indices, labels in one
 * input and C are free, labels in both inputs only are summed).  Each operand is
 * given by its labels (one char per axis), extents and strides (in complex
 * elements) and a conjugation flag; C is overwritten.
 *   mode 0: complex64 on the CUDA cores; 1: complex64 on the tensor cores
 *           (TNS_ERR_STATE if the contraction does not fit that path);
 *           2: complex128 on the CUDA cores. */
tns_status tns_test_contract(const char* labels_a, const int64_t* dims_a, const int64_t* strides_a, int32_t conj_a,
                             const void* A_dev, const char* labels_b, const int64_t* dims_b, const int64_t* strides_b,
                             int32_t conj_b, const void* B_dev, const char* labels_c, const int64_t* dims_c,
                             const int64_t* strides_c, void* C_dev, int32_t mode, void* cuda_stream);

/* The contraction planner's decision for tns_test_contract's mode 1 (tensor cores),
 * computed on the host without touching a device (operand pointers are not
 * needed).  out (host int64 [11]): [0] 1 = tensor cores, 0 = CUDA cores (too small
 * or not expressible); [1] operand roles swapped (C^T = B^T A^T); [2] the A-side
 * operand read in place; [3] / [4] A / B side shared by every batch entry; [5] batch
 * rows merged into one launch; [6] tile width in real columns (128 or 256); [7] M,
 * [8] N (complex, after any swap); [9] K; [10] batch entries. */
tns_status tns_test_plan(const char* labels_a, const int64_t* dims_a, const int64_t* strides_a, int32_t conj_a,
                         const char* labels_b, const int64_t* dims_b, const int64_t* strides_b, int32_t conj_b,
                         const char* labels_c, const int64_t* dims_c, const int64_t* strides_c, int64_t* out);

/* Batched FP64 thin SVD A = U diag(s) V^H (m >= n) by one-sided Jacobi.
 *   A_dev  device complex128 [batch][m][n] (read only); s_dev float64 [batch][n];
 *   U_dev  complex128 [batch][m][n]; V_dev complex128 [batch][n][n] */
tns_status tns_test_svd(int32_t batch, int32_t m, int32_t n, const double* A_dev, double* s_dev, double* U_dev,
                        double* V_dev, void* cuda_stream);

/* One site of a cached bottom norm environment E[b] (built by the last tns_log_norm
 * or tns_sample call), in its stored form: dims_out (host int64 [4]) receives its
 * left bond, its two physical dims and its right bond in storage order;
 * reversed_out (host, may be NULL) whether the environment is stored in reversed
 * column order (stored site k is column W-1-k with bonds swapped); out_host (host
 * complex128, row-major, may be NULL to query dims) the entries, widened from the
 * working precision.  TNS_ERR_STATE when no environment is cached. */
tns_status tns_test_env_site(tns_state* s, int32_t b, int32_t k, int64_t* dims_out, int32_t* reversed_out,
                             double* out_host);

#ifdef __cplusplus
}
#endif
#endif /* TNS_TESTING_H */
