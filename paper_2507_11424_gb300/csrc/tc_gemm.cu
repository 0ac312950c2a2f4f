// Tensor-core (tcgen05) complex contraction for the environment GEMMs of the
// marginal sweeps, C = A B^T with A: M x K complex, B: N x K complex (both
// K-contiguous), C: M x N complex, all complex64.
//
// Complex arithmetic runs as one real GEMM: A is read as M x 2K real (interleaved
// re/im), B is expanded once into the 2N x 2K real block matrix
//   [ Br  -Bi ]   rows 2n   (real part of column n)
//   [ Bi   Br ]   rows 2n+1 (imaginary part)
// interleaved by k, so C comes out interleaved.  Precision: kind::tf32 with a
// three-pass split product A_hi B_hi + A_hi B_lo + A_lo B_hi, where the hi part
// is the FP32 value itself (the tensor core reads its top 19 bits) and the lo
// part the exact FP32 remainder; all passes accumulate in one FP32 TMEM tile.
//
// Kernel: one 128 x 256 output tile per CTA, 128 threads.  Thread 0 issues TMA
// loads (128B-swizzled, 32 FP32 of K per row) into a 4-stage ring guarded by
// mbarriers; thread 32 issues tcgen05.mma (M=128, N=256, K=8 per instruction)
// and releases each stage with tcgen05.commit; all four warps then read the
// accumulator from TMEM (each warp its 32 lanes) and store it.  Every wait has
// a 1 s time limit after which the kernel raises an error flag and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace tns {

namespace {
constexpr int BM = 128, BN = 256, BKF = 32, STAGES = 4;
constexpr int TMEM_COLS = 256;
constexpr size_t TILE_A = (size_t)BM * BKF * sizeof(float);   // 16 KB
constexpr size_t TILE_B = (size_t)BN * BKF * sizeof(float);   // 32 KB
constexpr size_t SMEM_BYTES = STAGES * (TILE_A + TILE_B) + 1024 + 256;
constexpr unsigned long long WAIT_NS = 1000000000ull;          // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false when the deadline passes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long deadline) {
  while (!mbar_try(bar, parity)) {
    if (gtimer() > deadline) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile, 128B swizzle: 128-byte rows, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);        // start address
  d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)2 << 61;                         // SWIZZLE_128B
  return d;
}
// Instruction descriptor: D = F32, A = B = TF32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
}  // namespace

__global__ void __launch_bounds__(128, 1)
tc_gemm_tf32x3_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mAlo,
                      const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, float* C,
                      long long ldc, long long M, int Nr, int Kr, int* err) {
  extern __shared__ unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
  float* sA = reinterpret_cast<float*>(base);
  float* sB = sA + STAGES * BM * BKF;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * BN * BKF);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // linear grid, N tiles fastest: the CTAs sharing an A row-block run together and
  // read it from L2 instead of re-reading it from HBM once per N tile
  const int ntn = (Nr + BN - 1) / BN;
  const long long m0 = (long long)(blockIdx.x / ntn) * BM;
  const int n0 = (int)(blockIdx.x % ntn) * BN;
  const int nkb = (Kr + BKF - 1) / BKF;
  const int nsteps = 3 * nkb;

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
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned long long deadline = gtimer() + WAIT_NS;

  if (threadIdx.x == 0) {
    // producer: TMA loads of (A or A_lo, B_hi or B_lo) per k-step
    int issued = 0;
    for (int it = 0; it < nsteps; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1, deadline)) { *abort_flag = 1; break; }
      const int pass = it / nkb, kb = it % nkb;
      const CUtensorMap* ma = (pass == 2) ? &mAlo : &mA;
      const CUtensorMap* mb = (pass == 1) ? &mBlo : &mBhi;
      mbar_expect_tx(&full[s], (uint32_t)(TILE_A + TILE_B));
      tma_load_2d(sA + s * BM * BKF, ma, &full[s], kb * BKF, (int)m0);
      tma_load_2d(sB + s * BN * BKF, mb, &full[s], kb * BKF, n0);
      issued = it + 1;
    }
    if (*abort_flag) {
      // let copies already in flight land before the CTA exits (bounded)
      const unsigned long long d2 = gtimer() + WAIT_NS / 10;
      for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; ++it)
        mbar_wait(&full[it % STAGES], (it / STAGES) & 1, d2);
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer
    const uint32_t idesc = idesc_tf32(BM, BN);
    bool ok = true;
    for (int it = 0; it < nsteps; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (*abort_flag || !mbar_wait(&full[s], ph, deadline)) { *abort_flag = 1; ok = false; break; }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * BM * BKF), b0 = smem_u32(sB + s * BN * BKF);
#pragma unroll
      for (int kk = 0; kk < BKF / 8; ++kk)
        mma_tf32(tmem, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc, (it > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    // always signal `done`: it completes once every MMA issued above has finished,
    // so TMEM is never released under an MMA still in flight
    mma_commit(done);
    if (!ok) *abort_flag = 1;
  }
  __syncwarp();
  const bool ready = mbar_wait(done, 0, deadline) && !*abort_flag;
  tc_fence_after();
  if (ready) {
    const long long row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int cb = 0; cb < BN; cb += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, r);
      if (row < M) {
        float* dst = C + row * ldc + n0 + cb;
        const int lim = Nr - (n0 + cb);
        if (lim >= 32) {
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4*>(dst + j) =
                make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                            __uint_as_float(r[j + 3]));
        } else {
          for (int j = 0; j < 32 && j < lim; ++j) dst[j] = __uint_as_float(r[j]);
        }
      }
    }
  } else if (threadIdx.x == 0 && err) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// lo = x - (x with its low 13 mantissa bits cleared): the part of x a TF32 read drops.
__global__ void tf32_lo_kernel(const float* __restrict__ x, float* __restrict__ lo, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float v = x[i];
    float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    lo[i] = v - h;
  }
}

// Real block expansion of a complex N x K operand read through two sub-indices
// per dimension: value E[n1*sN1 + n2*sN2 + k1*sK1 + k2*sK2], n = n1*N2 + n2,
// k = k1*K2 + k2.  Writes hi (the value) and lo (its TF32 remainder).
__global__ void expand_b_kernel(const float2* __restrict__ E, int N1, int N2, long long sN1, long long sN2, int K1,
                                int K2, long long sK1, long long sK2, float* __restrict__ Bhi,
                                float* __restrict__ Blo) {
  const long long N = (long long)N1 * N2, K = (long long)K1 * K2;
  const long long Kr = 2 * K;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N * K;
       idx += (long long)gridDim.x * blockDim.x) {
    long long n = idx / K, k = idx % K;
    long long n1 = n / N2, n2 = n % N2, k1 = k / K2, k2 = k % K2;
    float2 v = E[n1 * sN1 + n2 * sN2 + k1 * sK1 + k2 * sK2];
    float q[4] = {v.x, -v.y, v.y, v.x};
    long long o[4] = {(2 * n) * Kr + 2 * k, (2 * n) * Kr + 2 * k + 1, (2 * n + 1) * Kr + 2 * k,
                      (2 * n + 1) * Kr + 2 * k + 1};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float h = __uint_as_float(__float_as_uint(q[t]) & 0xFFFFE000u);
      Bhi[o[t]] = q[t];
      Blo[o[t]] = q[t] - h;
    }
  }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

static bool make_map(CUtensorMap* map, const float* ptr, long long rows, int cols, long long ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)BKF, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_gemm_supported(long long M, int Nr, int Kr, long long lda, long long ldb, long long ldc) {
  if (!encode_fn()) return false;
  if (M < 1 || Nr < 1 || Kr < BKF || M >= (1LL << 31)) return false;
  if ((lda * 4) % 16 || (ldb * 4) % 16 || (ldc % 4) || (Kr % 4)) return false;
  return true;
}

cudaError_t tc_gemm_tf32x3(const float* A, const float* Alo, long long M, int Kr, long long lda, const float* Bhi,
                           const float* Blo, int Nr, long long ldb, float* C, long long ldc, int* err,
                           cudaStream_t st) {
  if (!tc_gemm_supported(M, Nr, Kr, lda, ldb, ldc)) return cudaErrorNotSupported;
  CUtensorMap ma, malo, mbhi, mblo;
  if (!make_map(&ma, A, M, Kr, lda, BM) || !make_map(&malo, Alo, M, Kr, lda, BM) ||
      !make_map(&mbhi, Bhi, Nr, Kr, ldb, BN) || !make_map(&mblo, Blo, Nr, Kr, ldb, BN))
    return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long tiles = ((M + BM - 1) / BM) * ((Nr + BN - 1) / BN);
  if (tiles >= (1LL << 31)) return cudaErrorInvalidValue;
  tc_gemm_tf32x3_kernel<<<(unsigned)tiles, 128, SMEM_BYTES, st>>>(ma, malo, mbhi, mblo, C, ldc, M, Nr, Kr, err);
  return cudaGetLastError();
}

cudaError_t tf32_lo(const float* x, float* lo, long long n, cudaStream_t st) {
  long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  tf32_lo_kernel<<<(unsigned)std::max<long long>(1, blocks), 256, 0, st>>>(x, lo, n);
  return cudaGetLastError();
}

cudaError_t expand_b(const void* E, int N1, int N2, long long sN1, long long sN2, int K1, int K2, long long sK1,
                     long long sK2, float* Bhi, float* Blo, cudaStream_t st) {
  long long n = (long long)N1 * N2 * K1 * K2;
  long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  expand_b_kernel<<<(unsigned)std::max<long long>(1, blocks), 256, 0, st>>>(
      static_cast<const float2*>(E), N1, N2, sN1, sN2, K1, K2, sK1, sK2, Bhi, Blo);
  return cudaGetLastError();
}

}  // namespace tns
