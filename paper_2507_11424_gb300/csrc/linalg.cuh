// Batched small dense linear algebra in FP64 (Jacobi methods), sm_103a.
#pragma once
#include "common.cuh"

namespace tns {

// Hermitian eigendecomposition of a batch of n x n matrices by cyclic parallel
// Jacobi (round-robin pair ordering, one thread block per matrix).
//   A   : input, row-major, leading dim lda, batch stride sA (complex); destroyed
//   lam : [batch][n] eigenvalues, descending
//   V   : [batch] n x n row-major, column j = eigenvector j (batch stride sV)
//   work: >= batch * 2 * np * np complex (np = n rounded up to even), used when the
//         matrix does not fit in shared memory; may be null otherwise
//   status: [batch] 0 = converged, 1 = sweep cap reached (result still returned)
//   sweeps_out: optional [batch] number of sweeps used.  n <= 512.
cudaError_t eigh_batched(cd* A, long long sA, int lda, int n, int batch, double* lam, cd* V, long long sV,
                         cd* work, int* status, cudaStream_t st, int* sweeps_out = nullptr);

// The same solver in FP32 for a complex64 input (the mixed-precision truncation):
// thresholds scaled to FP32 rounding; lam and V written as float64 / complex128.
// work: >= batch * 2 * np * np complex64 when !jacobi_fits_smem_f32(n).
cudaError_t eigh_batched_f32(const cf* A, long long sA, int lda, int n, int batch, double* lam, cd* V, long long sV,
                             cf* work, int* status, cudaStream_t st, int* sweeps_out = nullptr);
bool jacobi_fits_smem_f32(int n);

// Orthonormalising map from a Gram matrix: W = L^{-H} with
// L L^H = G + shift * max_i G_ii * I, batched n x n (contiguous).  G complex128
// (g_f64) or complex64, W complex128 (w_f64) or complex64.  The factorisation runs
// in FP64, except for complex64 G and W with fp32_factor (then FP32).  A pivot below
// the shift (a Gram made indefinite by its rounding) is set to sqrt(shift) and its
// column decoupled, so W stays bounded.  work: >= batch * n (n + 1) complex128 unless
// chol_fits_smem(n) (callers may pass more).  n <= 512.
cudaError_t chol_w_batched(const void* G, bool g_f64, int n, int batch, double shift, void* W, bool w_f64, void* work,
                           cudaStream_t st, bool fp32_factor = false);
bool chol_fits_smem(int n);

// Thin SVD A = U diag(sigma) V^H of a batch of m x n matrices with m >= n by
// one-sided (Hestenes) Jacobi.  A (row-major, lda, batch stride sA) is destroyed.
//   sigma: [batch][n] descending;  U: [batch] m x n row-major (zero columns where
//   sigma = 0);  V: [batch] n x n row-major.  work as for eigh (m*np + np*np).
cudaError_t svd_batched(cd* A, long long sA, int lda, int m, int n, int batch, double* sigma, cd* U, long long sU,
                        cd* V, long long sV, cd* work, int* status, cudaStream_t st);

// Whether svd_batched of an m x n matrix runs from shared memory (else it needs work).
bool jacobi_fits_smem(int m, int n);
// Whether eigh_batched of an n x n matrix runs from shared memory (else it needs work).
bool eigh_fits_smem(int n);

}  // namespace tns
