// BF16 tensor-core GEMM (tcgen05 kind::f16, FP32 accumulation in TMEM) for the
// learned proposal's training and inference, with the network's fused epilogue.
//
//   C[m][n] = sum_k A[m][k] B[n][k]      (A: M x K, B: N x K, both BF16, K contiguous)
//   v = C[m][n] + bias[n];  v = 0 where gate[m][n] <= 0;  Cf = v;  Cb = bf16(relu ? max(v, 0) : v)
//
// One 128 x 128 output tile per CTA, 128 threads.  Thread 0 issues TMA loads
// (128B swizzle, 64 BF16 of K per row) of A and B into a 4-stage ring; thread 32
// issues four M=128, N=128, K=16 MMAs per stage into one FP32 TMEM accumulator and
// frees the stage with tcgen05.commit; after the last stage all four warps read
// the accumulator (warp w owns TMEM lanes 32w..32w+31 = tile rows) and apply the
// epilogue.  Every wait is bounded (1 s of %globaltimer), after which the kernel
// raises the error flag, lets in-flight copies land and frees TMEM.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_bf16.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace tns {

namespace {
constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4, THREADS = 128;
constexpr size_t TILE_BYTES = (size_t)BM * BK * sizeof(__nv_bfloat16);        // 16 KB (A and B alike)
constexpr size_t SMEM = STAGES * 2 * TILE_BYTES + 1024 + 256;
constexpr unsigned long long WAIT_NS = 1000000000ull;

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
}  // namespace
using namespace ptx;

__global__ void __launch_bounds__(THREADS, 1)
tc_gemm_bf16_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, const Bf16Gemm p) {
  extern __shared__ unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
  unsigned char* sA = reinterpret_cast<unsigned char*>(base);            // [STAGES][BM][BK] bf16, swizzled
  unsigned char* sB = sA + STAGES * TILE_BYTES;                          // [STAGES][BN][BK]
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * TILE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nkb = (p.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned long long deadline = gtimer() + WAIT_NS;

  if (threadIdx.x == 0) {
    int issued = 0;
    for (int it = 0; it < nkb; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1, deadline)) { *abort_flag = 1; break; }
      mbar_expect_tx(&full[s], (uint32_t)(2 * TILE_BYTES));
      tma_load_2d(sA + s * TILE_BYTES, &mA, &full[s], it * BK, m0);
      tma_load_2d(sB + s * TILE_BYTES, &mB, &full[s], it * BK, n0);
      issued = it + 1;
    }
    if (*abort_flag) {
      const unsigned long long d2 = gtimer() + WAIT_NS / 10;
      for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; ++it)
        mbar_wait(&full[it % STAGES], (it / STAGES) & 1, d2);
    }
  } else if (threadIdx.x == 32) {
    const uint32_t idesc = idesc_bf16(BM, BN);
    bool ok = true;
    for (int it = 0; it < nkb; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (*abort_flag || !mbar_wait(&full[s], ph, deadline)) {
        *abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * TILE_BYTES), b0 = smem_u32(sB + s * TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)      // 16 BF16 = 32 bytes of each 128-byte row per MMA
        mma_bf16(tmem, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc, (it > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
    if (!ok) *abort_flag = 1;
  }
  __syncwarp();
  const bool ready = mbar_wait(done, 0, deadline) && !*abort_flag;
  tc_fence_after();
  if (ready) {
    const int m = m0 + warp * 32 + lane;
    const bool valid = m < p.M;
#pragma unroll 1
    for (int cb = 0; cb < BN; cb += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      if (!valid) continue;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int n = n0 + cb + i;
        if (n >= p.N) break;
        float x = __uint_as_float(v[i]) + (p.bias ? p.bias[n] : 0.f);
        const long long o = (long long)m * p.ldc + n;
        if (p.gate && !(p.gate[o] > 0.f)) x = 0.f;
        if (p.Cf) p.Cf[o] = x;
        if (p.Cb) p.Cb[(long long)m * p.ldcb + n] = __float2bfloat16(p.relu ? fmaxf(x, 0.f) : x);
      }
    }
  } else if (threadIdx.x == 0 && p.err) {
    atomicExch(p.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

// out[c][r] = in[r][c] for r < rows, c < cols (BF16, row pitches ldi / ldo), through
// 32 x 32 shared-memory tiles.
__global__ void bf16_transpose_kernel(const __nv_bfloat16* __restrict__ in, long long ldi, int rows, int cols,
                                      __nv_bfloat16* __restrict__ out, long long ldo) {
  __shared__ __nv_bfloat16 tile[32][34];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int rr = r0 + r, cc = c0 + threadIdx.x;
    if (rr < rows && cc < cols) tile[r][threadIdx.x] = in[(long long)rr * ldi + cc];
  }
  __syncthreads();
  for (int c = threadIdx.y; c < 32; c += blockDim.y) {
    const int cc = c0 + c, rr = r0 + threadIdx.x;
    if (rr < rows && cc < cols) out[(long long)cc * ldo + rr] = tile[threadIdx.x][c];
  }
}

cudaError_t tc_gemm_bf16(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B, long long ldb,
                         const Bf16Gemm& g, cudaStream_t st) {
  if (g.M < 1 || g.N < 1 || g.K < 1) return cudaSuccess;
  if (!tc_available()) return cudaErrorNotSupported;
  if ((lda * 2) % 16 || (ldb * 2) % 16 || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!tma_map_2d(&ma, true, A, g.M, g.K, lda * 2, BK, BM) || !tma_map_2d(&mb, true, B, g.N, g.K, ldb * 2, BK, BN))
    return cudaErrorInvalidValue;
  cudaError_t e = smem_optin((const void*)tc_gemm_bf16_kernel, (int)SMEM);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + BN - 1) / BN));
  if (grid.y > 65535) return cudaErrorInvalidValue;
  tc_gemm_bf16_kernel<<<grid, THREADS, SMEM, st>>>(ma, mb, g);
  return cudaGetLastError();
}

cudaError_t bf16_transpose(const __nv_bfloat16* in, long long ldi, int rows, int cols, __nv_bfloat16* out,
                           long long ldo, cudaStream_t st) {
  if (rows < 1 || cols < 1) return cudaSuccess;
  const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  if (grid.y > 65535) return cudaErrorInvalidValue;
  bf16_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, ldi, rows, cols, out, ldo);
  return cudaGetLastError();
}

}  // namespace tns
