// Tensor-core (tcgen05, kind::tf32, three-pass split) batched complex GEMM.  See tc_gemm.cu.
#pragma once
#include "common.cuh"
#include <string.h>
#include <cuda.h>

namespace tns {

// Output layout: element (batch b, row m, column n) of C (complex64) lives at
//   C + boff(b) + sum_g (m_g * sCm[g]) + sum_g (n_g * sCn[g])
// where m = m_0 + mdim[0] * (m_1 + mdim[1] * ...), likewise n and b, and boff adds
// coff[b_{coff_grp}] when coff is set.  Strides in complex elements.
struct TcEpilogue {
  float2* C;
  long long M;          // rows of one batch entry
  int N;                // complex columns
  int nm, nn, nb;
  int mdim[4], ndim[4], bdim[2];
  long long sCm[4], sCn[4], sCb[2];
  const long long* coff;
  int coff_grp;
};

struct TcArgs {
  TcEpilogue e;
  long long nbatch;     // batch entries
  int merged;           // 1: A rows run over nbatch * M (B shared by every entry)
  int a_batched;        // A holds one M-row block per batch entry (else one, shared)
  int b_batched;        // B holds one 2N-row block per batch entry (else one, shared)
  int Kr;               // real K extent (2K); columns beyond the operands' widths read as 0
  int tiles_m, tiles_n; // filled by tc_gemm_tf32x3
  int* err;             // device flag set to 1 when a pipeline wait timed out
};

// A: [rowsA][Kr] FP32 (interleaved complex) with row pitch lda floats (its TF32
// remainder is formed in shared memory); Bhi/Blo: [rowsB][Kr] expanded operand and
// its TF32 remainder, pitch ldb.  Pitches must be multiples of 4 floats and
// pointers 16-byte aligned.
struct TcOperands {
  const float *A, *Bhi, *Blo;
  long long lda, ldb;
};

// x rounded to the nearest TF32 value (ties to even): 13 low mantissa bits cleared.
__host__ __device__ inline float tf32_rn(float x) {
#ifdef __CUDA_ARCH__
  uint32_t u = __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
#endif
  u += 0x0FFFu + ((u >> 13) & 1u);
  u &= 0xFFFFE000u;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float r;
  memcpy(&r, &u, 4);
  return r;
#endif
}

// Tile width (real output columns) for an output of n complex columns.
inline int tc_tile_n(long long n_complex) { return 2 * n_complex <= 128 ? 128 : 256; }

bool tc_available();
// 2-D TMA descriptor (128B swizzle, zero fill out of bounds) over a row-major
// [rows][cols] FP32 or BF16 array with a row pitch of ld_bytes (multiple of 16).
bool tma_map_2d(CUtensorMap* map, bool bf16, const void* ptr, long long rows, long long cols, long long ld_bytes,
                int box_cols, int box_rows);
// cudaErrorNotSupported when the shape or alignment does not fit the kernel.
cudaError_t tc_gemm_tf32x3(const TcOperands& op, const TcArgs& a, cudaStream_t st);
// Testing: force the tile width of later launches (128 or 256; 0 = the tuned choice).
// Testing: force the tile variant of later launches (128, 256 or TC_TILE_128_SINGLE;
// 0 = the timing-based choice).
constexpr int TC_TILE_128_SINGLE = 129;
void tc_force_tile(int bn);
// Per-device error flag shared by every tensor-core launch (lazily allocated).
int* tc_error_flag();

}  // namespace tns
