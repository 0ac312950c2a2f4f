// Strided tensor-contraction GEMM (SIMT) and the host planner.  See contract.cuh.
#include "contract.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <atomic>
#include <cstdio>

namespace tns {

// Launches of this thread's contractions (the API entry points attribute the
// difference across a call to the state they run on).
static thread_local long long g_launches = 0;
long long contract_launches() { return g_launches; }

TView view(void* p, const std::string& labels, const std::vector<long long>& dims, bool conj) {
  TView v;
  v.ptr = p;
  v.labels = labels;
  v.dim = dims;
  v.conj = conj;
  v.stride.resize(dims.size());
  long long s = 1;
  for (int i = (int)dims.size() - 1; i >= 0; --i) {
    v.stride[i] = s;
    s *= dims[i];
  }
  return v;
}

TView& bcast(TView& v, char label, long long dim) {
  v.labels.push_back(label);
  v.dim.push_back(dim);
  v.stride.push_back(0);
  return v;
}

struct GemmParams {
  long long M;
  int N, K;
  int nm, nn, nk, nb;
  int mdim[4], ndim[4], kdim[4], bdim[2];
  long long sAm[4], sCm[4], sBn[4], sCn[4], sAk[4], sBk[4];
  long long sAb[2], sBb[2], sCb[2];
  const uint8_t* aidx;
  long long a_idx_ld, a_idx_stride;
  int a_idx_grp;
  const uint8_t* bidx;
  long long b_idx_ld, b_idx_stride;
  int b_idx_grp;
  const long long* aoff;
  const long long* boffs;
  const long long* coff;
  int aoff_grp, boff_grp, coff_grp;
  const void* A;
  const void* B;
  void* C;
  int conjA, conjB;
  double2 alpha, beta;
  int beta_zero;
  int a_kfast, b_kfast;
  // split-K: blocks of one output tile share blockIdx.x/y and split the K loop;
  // partial tiles go to `partial` and a second kernel reduces them in order
  int splits, kchunk;
  void* partial;
};

template <typename T> __device__ inline T ld_in(const T* p, bool cj) {
  T v = *p;
  return cj ? cconj(v) : v;
}

__device__ inline void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ inline void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ inline double2 widen(double2 a, double2) { return a; }
__device__ inline double2 widen(float2 a, double2) { return make_double2(a.x, a.y); }
__device__ inline float2 widen(float2 a, float2) { return a; }

template <typename TO> __device__ inline TO narrow(double2 a);
template <> __device__ inline double2 narrow<double2>(double2 a) { return a; }
template <> __device__ inline float2 narrow<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <typename TO> __device__ inline TO narrow(float2 a);
template <> __device__ inline float2 narrow<float2>(float2 a) { return a; }

// 64x64 output tile per 256-thread block; each thread owns a 4x4 sub-tile on a
// stride-16 lattice.  Operand tiles are staged through shared memory with
// addresses decoded from the sub-index strides.
template <typename TI, typename TACC, typename TO, int BK>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmParams p) {
  constexpr int BM = 64, BN = 64;
  __shared__ TI As[BK][BM + 1];
  __shared__ TI Bs[BK][BN + 1];
  __shared__ long long rowA[BM], rowC[BM], colB[BN], colC[BN];
  __shared__ long long kA[BK], kB[BK];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;

  long long offA = 0, offB = 0, offC = 0;
  int bi[2] = {0, 0};
  const int ks = blockIdx.z % p.splits;
  const int bz = blockIdx.z / p.splits;
  {
    int r = bz;
    for (int g = 0; g < p.nb; ++g) {
      bi[g] = r % p.bdim[g];
      r /= p.bdim[g];
      offA += bi[g] * p.sAb[g];
      offB += bi[g] * p.sBb[g];
      offC += bi[g] * p.sCb[g];
    }
  }
  if (p.aidx) offA += (long long)p.aidx[(long long)bi[p.a_idx_grp] * p.a_idx_ld] * p.a_idx_stride;
  if (p.bidx) offB += (long long)p.bidx[(long long)bi[p.b_idx_grp] * p.b_idx_ld] * p.b_idx_stride;
  if (p.aoff) offA += p.aoff[bi[p.aoff_grp]];
  if (p.boffs) offB += p.boffs[bi[p.boff_grp]];
  if (p.coff) offC += p.coff[bi[p.coff_grp]];
  const TI* A = (const TI*)p.A + offA;
  const TI* B = (const TI*)p.B + offB;
  TO* C = (TO*)p.C + offC;

  if (tid < BM) {
    long long m = m0 + tid, oa = 0, oc = 0;
    if (m < p.M) {
      long long r = m;
      for (int g = 0; g < p.nm; ++g) {
        long long i = r % p.mdim[g];
        r /= p.mdim[g];
        oa += i * p.sAm[g];
        oc += i * p.sCm[g];
      }
    }
    rowA[tid] = oa;
    rowC[tid] = oc;
  } else if (tid < BM + BN) {
    int t = tid - BM;
    long long n = n0 + t, ob = 0, oc = 0;
    if (n < p.N) {
      long long r = n;
      for (int g = 0; g < p.nn; ++g) {
        long long i = r % p.ndim[g];
        r /= p.ndim[g];
        ob += i * p.sBn[g];
        oc += i * p.sCn[g];
      }
    }
    colB[t] = ob;
    colC[t] = oc;
  }

  TACC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<TACC>();

  const bool cjA = p.conjA != 0, cjB = p.conjB != 0;
  const int kbeg = ks * p.kchunk;
  const int kend = min(p.K, kbeg + p.kchunk);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    __syncthreads();
    if (tid < BK) {
      long long k = k0 + tid, oa = 0, ob = 0;
      if (k < kend) {
        long long r = k;
        for (int g = 0; g < p.nk; ++g) {
          long long i = r % p.kdim[g];
          r /= p.kdim[g];
          oa += i * p.sAk[g];
          ob += i * p.sBk[g];
        }
      }
      kA[tid] = oa;
      kB[tid] = ob;
    }
    __syncthreads();
    for (int e = tid; e < BM * BK; e += 256) {
      int mm, kk;
      if (p.a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      TI v = czero<TI>();
      if (m0 + mm < p.M && k0 + kk < kend) v = ld_in(A + rowA[mm] + kA[kk], cjA);
      As[kk][mm] = v;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int nn, kk;
      if (p.b_kfast) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      TI v = czero<TI>();
      if (n0 + nn < p.N && k0 + kk < kend) v = ld_in(B + kB[kk] + colB[nn], cjB);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TACC a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = widen(As[kk][ty + 16 * i], TACC());
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = widen(Bs[kk][tx + 16 * j], TACC());
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
  }

  if (p.splits > 1) {
    TACC* part = (TACC*)p.partial +
                 (((long long)bz * p.splits + ks) * gridDim.x * gridDim.y + (long long)blockIdx.x * gridDim.y +
                  blockIdx.y) * (BM * BN);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[(ty + 16 * i) * BN + tx + 16 * j] = acc[i][j];
    return;
  }
  TACC al = narrow<TACC>(p.alpha), be = narrow<TACC>(p.beta);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long m = m0 + ty + 16 * i;
    if (m >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= p.N) continue;
      TO* dst = C + rowC[ty + 16 * i] + colC[tx + 16 * j];
      TACC v = cmul(al, acc[i][j]);
      if (!p.beta_zero) v = cadd(v, cmul(be, widen(*dst, TACC())));
      *dst = narrow<TO>(v);
    }
  }
}

// Sums the split-K partial tiles in a fixed order (deterministic) and writes C.
template <typename TACC, typename TO>
__global__ void __launch_bounds__(256) splitk_reduce_kernel(const GemmParams p, unsigned gx, unsigned gy) {
  const long long tile = blockIdx.x;                 // over batch * gx * gy
  const long long bz = tile / ((long long)gx * gy);
  const long long txy = tile % ((long long)gx * gy);
  const long long bx = txy / gy, by = txy % gy;
  long long offC = 0;
  int bi[2] = {0, 0};
  {
    long long r = bz;
    for (int g = 0; g < p.nb; ++g) {
      bi[g] = (int)(r % p.bdim[g]);
      r /= p.bdim[g];
      offC += bi[g] * p.sCb[g];
    }
  }
  if (p.coff) offC += p.coff[bi[p.coff_grp]];
  TO* C = (TO*)p.C + offC;
  const TACC* part = (const TACC*)p.partial;
  TACC al = narrow<TACC>(p.alpha), be = narrow<TACC>(p.beta);
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    long long m = bx * 64 + e / 64;
    long long n = by * 64 + e % 64;
    if (m >= p.M || n >= p.N) continue;
    TACC acc = czero<TACC>();
    for (int ks = 0; ks < p.splits; ++ks)
      acc = cadd(acc, part[((bz * p.splits + ks) * gx * gy + bx * gy + by) * 4096 + e]);
    long long oc = 0, r = m;
    for (int g = 0; g < p.nm; ++g) { oc += (r % p.mdim[g]) * p.sCm[g]; r /= p.mdim[g]; }
    r = n;
    for (int g = 0; g < p.nn; ++g) { oc += (r % p.ndim[g]) * p.sCn[g]; r /= p.ndim[g]; }
    TO* dst = C + oc;
    TACC v = cmul(al, acc);
    if (!p.beta_zero) v = cadd(v, cmul(be, widen(*dst, TACC())));
    *dst = narrow<TO>(v);
  }
}

// ------------------------------------------------------ tensor-core operand packing
// Operand offsets of batch entry b (A side when which == 0, B side otherwise).
__device__ inline long long batch_off(const GemmParams& p, long long b, int which) {
  long long o = 0;
  int bi[2] = {0, 0};
  for (int g = 0; g < p.nb; ++g) {
    bi[g] = (int)(b % p.bdim[g]);
    b /= p.bdim[g];
    o += bi[g] * (which == 0 ? p.sAb[g] : p.sBb[g]);
  }
  if (which == 0) {
    if (p.aidx) o += (long long)p.aidx[(long long)bi[p.a_idx_grp] * p.a_idx_ld] * p.a_idx_stride;
    if (p.aoff) o += p.aoff[bi[p.aoff_grp]];
  } else {
    if (p.bidx) o += (long long)p.bidx[(long long)bi[p.b_idx_grp] * p.b_idx_ld] * p.b_idx_stride;
    if (p.boffs) o += p.boffs[bi[p.boff_grp]];
  }
  return o;
}
__device__ inline long long decomp(long long i, int n, const int* dim, const long long* stride) {
  long long o = 0;
  for (int g = 0; g < n; ++g) {
    o += (i % dim[g]) * stride[g];
    i /= dim[g];
  }
  return o;
}
// TF32 split of an FP32 value: hi = tf32_rn(v), lo = tf32_rn(v - hi).
__device__ inline float tf32_lo_rn(float v) { return tf32_rn(v - tf32_rn(v)); }

// A side: [nbA][M][Kp] interleaved complex, zero beyond 2K.
__global__ void pack_a_kernel(const GemmParams p, long long nbA, int Kp, float* __restrict__ out) {
  const int Kc = Kp / 2;
  const long long tot = nbA * p.M * Kc;
  const float2* A = (const float2*)p.A;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int kc = (int)(i % Kc);
    const long long r = i / Kc;
    float2 v = make_float2(0.f, 0.f);
    if (kc < p.K) {
      const long long b = r / p.M, m = r % p.M;
      v = A[batch_off(p, b, 0) + decomp(m, p.nm, p.mdim, p.sAm) + decomp(kc, p.nk, p.kdim, p.sAk)];
      if (p.conjA) v.y = -v.y;
    }
    *reinterpret_cast<float2*>(out + r * Kp + 2 * kc) = v;
  }
}

// B side: the real block expansion, hi/lo [nbB][2N][Kp] (TF32 split, see
// tc_gemm.cu); rows 2n / 2n+1 hold (Br, -Bi) / (Bi, Br) of column n interleaved by k.
__global__ void pack_b_kernel(const GemmParams p, long long nbB, int Kp, float* __restrict__ hi, float* __restrict__ lo) {
  const int Kc = Kp / 2;
  const long long tot = nbB * (long long)p.N * Kc;
  const float2* B = (const float2*)p.B;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int kc = (int)(i % Kc);
    const long long r = i / Kc;            // b * N + n
    float2 v = make_float2(0.f, 0.f);
    if (kc < p.K) {
      const long long b = r / p.N, n = r % p.N;
      v = B[batch_off(p, b, 1) + decomp(n, p.nn, p.ndim, p.sBn) + decomp(kc, p.nk, p.kdim, p.sBk)];
      if (p.conjB) v.y = -v.y;
    }
    const long long o0 = (2 * r) * Kp + 2 * kc, o1 = o0 + Kp;
    const float hx = tf32_rn(v.x), hy = tf32_rn(v.y), lx = tf32_lo_rn(v.x), ly = tf32_lo_rn(v.y);
    *reinterpret_cast<float2*>(hi + o0) = make_float2(hx, -hy);
    *reinterpret_cast<float2*>(hi + o1) = make_float2(hy, hx);
    *reinterpret_cast<float2*>(lo + o0) = make_float2(lx, -ly);
    *reinterpret_cast<float2*>(lo + o1) = make_float2(ly, lx);
  }
}

static unsigned grid_for(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 32));
}

// Swap the roles of A and B (C^T = B^T A^T): M <-> N.
static void swap_roles(GemmParams& p) {
  GemmParams q = p;
  q.M = p.N;
  q.N = (int)p.M;
  q.nm = p.nn; q.nn = p.nm;
  for (int g = 0; g < 4; ++g) {
    q.mdim[g] = p.ndim[g]; q.ndim[g] = p.mdim[g];
    q.sAm[g] = p.sBn[g]; q.sCm[g] = p.sCn[g];
    q.sBn[g] = p.sAm[g]; q.sCn[g] = p.sCm[g];
    q.sAk[g] = p.sBk[g]; q.sBk[g] = p.sAk[g];
  }
  for (int g = 0; g < 2; ++g) { q.sAb[g] = p.sBb[g]; q.sBb[g] = p.sAb[g]; }
  q.aidx = p.bidx; q.a_idx_ld = p.b_idx_ld; q.a_idx_stride = p.b_idx_stride; q.a_idx_grp = p.b_idx_grp;
  q.bidx = p.aidx; q.b_idx_ld = p.a_idx_ld; q.b_idx_stride = p.a_idx_stride; q.b_idx_grp = p.a_idx_grp;
  q.aoff = p.boffs; q.aoff_grp = p.boff_grp;
  q.boffs = p.aoff; q.boff_grp = p.aoff_grp;
  q.A = p.B; q.B = p.A;
  q.conjA = p.conjB; q.conjB = p.conjA;
  p = q;
}

// Stable insertion sort of index groups by the key stride `key`, carrying the other arrays.
// Reference batch at which the tensor-core operand roles are weighed.
static constexpr long long TC_ROLE_REF_BATCH = 128;

static void sort_groups(int n, int* dim, long long* key, long long* o1, long long* o2) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && key[j] < key[j - 1]; --j) {
      std::swap(dim[j], dim[j - 1]);
      std::swap(key[j], key[j - 1]);
      if (o1) std::swap(o1[j], o1[j - 1]);
      if (o2) std::swap(o2[j], o2[j - 1]);
    }
}

static bool operand_shared(const GemmParams& p, int which) {
  for (int g = 0; g < p.nb; ++g)
    if ((which == 0 ? p.sAb[g] : p.sBb[g]) != 0) return false;
  return which == 0 ? (!p.aidx && !p.aoff) : (!p.bidx && !p.boffs);
}

// A usable in place: row m of batch entry b at (b * M + m) * K, its K entries contiguous.
static bool dense_a(const GemmParams& p) {
  if (p.conjA || (p.K & 1) || p.aidx || p.aoff) return false;
  long long want = 1;
  for (int g = 0; g < p.nk; ++g) {
    if (p.sAk[g] != want) return false;
    want *= p.kdim[g];
  }
  for (int g = 0; g < p.nm; ++g) {
    if (p.sAm[g] != want) return false;
    want *= p.mdim[g];
  }
  if (!operand_shared(p, 0))
    for (int g = 0; g < p.nb; ++g) {
      if (p.sAb[g] != want) return false;
      want *= p.bdim[g];
    }
  return (reinterpret_cast<uintptr_t>(p.A) & 15) == 0;
}

struct TcRole {
  GemmParams q;
  bool a_sh, b_sh, ad, ok, swapped;
  double cost;   // bytes written by the operand packing
};

// Orders the index groups for the tensor-core path: K by the A-side stride, M by
// the A-side stride when A can be used in place (else by the output stride), N
// by the output stride (so each thread's 16 columns are, where possible, one
// contiguous run of the output).
static TcRole tc_role(const GemmParams& p, long long nbatch, bool swapped) {
  TcRole r;
  r.q = p;
  r.swapped = swapped;
  if (swapped) swap_roles(r.q);
  GemmParams& q = r.q;
  sort_groups(q.nk, q.kdim, q.sAk, q.sBk, nullptr);
  sort_groups(q.nm, q.mdim, q.sAm, q.sCm, nullptr);
  r.ad = dense_a(q);
  if (!r.ad) sort_groups(q.nm, q.mdim, q.sCm, q.sAm, nullptr);
  sort_groups(q.nn, q.ndim, q.sCn, q.sBn, nullptr);
  r.a_sh = operand_shared(q, 0);
  r.b_sh = operand_shared(q, 1);
  r.ok = !(r.a_sh && r.b_sh && nbatch > 1);
  // the packing cost is weighed at a fixed reference batch, not the call's: the role
  // decides which operand's rounding is split, so it must not change with the number
  // of batch entries (a sample drawn in a chunk of any size gets the same bits)
  const double nref = (double)TC_ROLE_REF_BATCH;
  const double rowsA = (r.a_sh ? 1.0 : nref) * q.M, rowsB = (r.b_sh ? 1.0 : nref) * q.N;
  r.cost = rowsA * q.K * (r.ad ? 0.0 : 8.0) + rowsB * q.K * 32.0;
  return r;
}

// The role assignment the tensor-core path uses (the cheaper packing of the two),
// or false when neither fits the kernel (both operands shared across a batch, or
// more rows than a TMA coordinate holds).
static bool pick_role(const GemmParams& p0, long long nbatch, TcRole& r) {
  if (p0.M < 1 || p0.N < 1 || p0.K < 1) return false;
  const TcRole r0 = tc_role(p0, nbatch, false), r1 = tc_role(p0, nbatch, true);
  if (!r0.ok && !r1.ok) return false;
  r = (!r0.ok || (r1.ok && r1.cost < r0.cost)) ? r1 : r0;
  const long long rowsA = (r.a_sh ? 1 : nbatch) * r.q.M, rowsB = (r.b_sh ? 1 : nbatch) * 2LL * r.q.N;
  return rowsA + 128 < (1LL << 31) && rowsB + 256 < (1LL << 31);
}

// Whether a contraction of this size goes to the tensor cores (else the SIMT kernel).
// Decided per batch entry (2^18 MACs, i.e. 2^24 at the reference batch of 64 entries),
// never by the batch count: the two paths round differently, and a batch entry's
// result must not depend on how many entries share its launch.
static bool tc_worth_it(const GemmParams& p, long long nbatch) {
  (void)nbatch;
  const double macs = (double)p.M * (double)p.N * (double)p.K;
  return macs >= 262144.0 && p.K >= 8;
}

// Run the contraction on the tensor cores.  *handled = false (and nothing
// launched) when the contraction does not fit the kernel.
static cudaError_t contract_tc(const GemmParams& p0, long long nbatch, cudaStream_t st, ContractTiming* tm,
                               bool* handled) {
  *handled = false;
  if (!tc_available()) return cudaSuccess;
  TcRole r;
  if (!pick_role(p0, nbatch, r)) return cudaSuccess;
  const GemmParams& p = r.q;
  const bool a_sh = r.a_sh, b_sh = r.b_sh, ad = r.ad;
  const int Kr = 2 * p.K;
  const int Kp = (Kr + 31) / 32 * 32;
  const long long nbA = a_sh ? 1 : nbatch, nbB = b_sh ? 1 : nbatch;
  const long long rowsA = nbA * p.M, rowsB = nbB * 2LL * p.N;
  TcArgs a{};
  a.e.C = (float2*)p.C;
  a.e.M = p.M;
  a.e.N = p.N;
  a.e.nm = p.nm;
  a.e.nn = p.nn;
  a.e.nb = p.nb;
  for (int g = 0; g < 4; ++g) {
    a.e.mdim[g] = p.mdim[g]; a.e.ndim[g] = p.ndim[g];
    a.e.sCm[g] = p.sCm[g]; a.e.sCn[g] = p.sCn[g];
  }
  for (int g = 0; g < 2; ++g) { a.e.bdim[g] = p.bdim[g]; a.e.sCb[g] = p.sCb[g]; }
  a.e.coff = p.coff;
  a.e.coff_grp = p.coff_grp;
  a.nbatch = nbatch;
  a.a_batched = a_sh ? 0 : 1;
  a.b_batched = b_sh ? 0 : 1;
  a.merged = (b_sh && !a_sh) ? 1 : 0;
  a.Kr = Kr;
  a.err = tc_error_flag();
  if (!a.err) return cudaSuccess;
  // scratch: A (unless it is used in place), B hi/lo
  const long long lda = ad ? Kr : Kp;
  const size_t a_floats = ad ? 0 : (size_t)rowsA * Kp;
  const size_t b_floats = (size_t)rowsB * Kp;
  const size_t b_al = (b_floats + 63) / 64 * 64;
  float* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, sizeof(float) * (a_floats + 2 * b_al), st);
  if (e != cudaSuccess) return e;
  float* Blo_ = buf;
  float* Bhi_ = buf + b_al;
  float* Ahi_ = ad ? (float*)p.A : buf + 2 * b_al;
  *handled = true;
  if (!ad) {
    pack_a_kernel<<<grid_for(rowsA * (Kp / 2)), 256, 0, st>>>(p, nbA, Kp, Ahi_);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    pack_b_kernel<<<grid_for(nbB * (long long)p.N * (Kp / 2)), 256, 0, st>>>(p, nbB, Kp, Bhi_, Blo_);
    e = cudaGetLastError();
  }
  g_launches += ad ? 1 : 2;
  if (e == cudaSuccess && tm && tm->mma_begin) e = cudaEventRecord(tm->mma_begin, st);
  TcOperands op{Ahi_, Bhi_, Blo_, lda, (long long)Kp};
  if (e == cudaSuccess) e = tc_gemm_tf32x3(op, a, st);
  g_launches++;
  if (e == cudaSuccess && tm && tm->mma_end) e = cudaEventRecord(tm->mma_end, st);
  if (tm && e == cudaSuccess) tm->used_tc = true;
  cudaFreeAsync(buf, st);
  return e;
}

// ------------------------------------------------------------------ planner
namespace {
struct Lab {
  char c;
  long long d;
  long long sa = 0, sb = 0, sc = 0;
  bool inA = false, inB = false, inC = false;
};
struct Grp {
  long long d;
  long long s0, s1, s2;   // strides in the (up to) three operands of the group
};

// Sort by the first stride and merge runs that are contiguous in every operand.
std::vector<Grp> merge(std::vector<Grp> g, int nops) {
  std::sort(g.begin(), g.end(), [](const Grp& a, const Grp& b) { return a.s0 < b.s0; });
  std::vector<Grp> out;
  for (auto& x : g) {
    if (!out.empty()) {
      Grp& c = out.back();
      bool ok = (x.s0 == c.s0 * c.d) && (x.s1 == c.s1 * c.d) && (nops < 3 || x.s2 == c.s2 * c.d);
      if (ok) {
        c.d *= x.d;
        continue;
      }
    }
    out.push_back(x);
  }
  return out;
}
}  // namespace

// Label analysis of C = alpha sum A B + beta C: batch / M / N / K index groups
// (contiguous runs merged), their strides in each operand, and per-batch offsets.
// *empty = true when the contraction or its output is empty (nothing to launch).
static cudaError_t plan_params(const TView& A, const TView& B, const TView& C, double2 alpha, double2 beta,
                               GemmParams& p, long long& nbatch, bool* empty) {
  *empty = false;
  std::vector<Lab> labs;
  auto find = [&](char c) -> Lab& {
    for (auto& l : labs)
      if (l.c == c) return l;
    labs.push_back(Lab{c, -1});
    return labs.back();
  };
  auto add = [&](const TView& v, int which) -> bool {
    if (v.labels.size() != v.dim.size() || v.dim.size() != v.stride.size()) return false;
    for (size_t i = 0; i < v.labels.size(); ++i) {
      Lab& l = find(v.labels[i]);
      if (l.d >= 0 && l.d != v.dim[i]) return false;
      l.d = v.dim[i];
      if (which == 0) { l.inA = true; l.sa = v.stride[i]; }
      if (which == 1) { l.inB = true; l.sb = v.stride[i]; }
      if (which == 2) { l.inC = true; l.sc = v.stride[i]; }
    }
    return true;
  };
  if (!add(A, 0) || !add(B, 1) || !add(C, 2)) {
    fprintf(stderr, "tns contract: inconsistent views (%s,%s->%s)\n", A.labels.c_str(), B.labels.c_str(),
            C.labels.c_str());
    return cudaErrorInvalidValue;
  }
  std::vector<Grp> gm, gn, gk, gb;
  char a_idx_label = A.idx ? A.idx_label : 0, b_idx_label = B.idx ? B.idx_label : 0;
  std::string off_labels;
  for (const TView* v : {&A, &B, &C})
    if (v->boff && off_labels.find(v->boff_label) == std::string::npos) off_labels.push_back(v->boff_label);
  std::vector<Grp> gb_idx;  // batch labels carrying an index offset (kept unmerged, first)
  std::vector<char> gb_idx_lab;
  long long Mtot = 1, Ntot = 1, Ktot = 1;
  for (auto& l : labs) {
    if (l.d == 0) { *empty = true; return cudaSuccess; }  // empty contraction or empty output
    bool idxl = (l.c == a_idx_label || l.c == b_idx_label || off_labels.find(l.c) != std::string::npos);
    if (l.d == 1 && !idxl) continue;
    if (l.inA && l.inB && l.inC) {
      if (idxl) { gb_idx.push_back(Grp{l.d, l.sc, l.sa, l.sb}); gb_idx_lab.push_back(l.c); }
      else gb.push_back(Grp{l.d, l.sc, l.sa, l.sb});
    } else if (l.inA && l.inC && !l.inB) { gm.push_back(Grp{l.d, l.sa, l.sc, 0}); Mtot *= l.d; }
    else if (l.inB && l.inC && !l.inA) { gn.push_back(Grp{l.d, l.sb, l.sc, 0}); Ntot *= l.d; }
    else if (l.inA && l.inB && !l.inC) { gk.push_back(Grp{l.d, l.sa, l.sb, 0}); Ktot *= l.d; }
    else {
      fprintf(stderr, "tns contract: label '%c' appears in one operand only (%s,%s->%s)\n", l.c,
              A.labels.c_str(), B.labels.c_str(), C.labels.c_str());
      return cudaErrorInvalidValue;
    }
  }
  gm = merge(gm, 2);
  gn = merge(gn, 2);
  gk = merge(gk, 2);
  gb = merge(gb, 3);
  std::vector<Grp> batch = gb_idx;
  for (auto& g : gb) batch.push_back(g);
  if (gm.size() > 4 || gn.size() > 4 || gk.size() > 4 || batch.size() > 2) {
    fprintf(stderr, "tns contract: too many index groups m%zu n%zu k%zu b%zu (%s,%s->%s)\n", gm.size(), gn.size(),
            gk.size(), batch.size(), A.labels.c_str(), B.labels.c_str(), C.labels.c_str());
    return cudaErrorInvalidValue;
  }
  p = GemmParams{};
  p.M = Mtot;
  p.N = (int)Ntot;
  p.K = (int)Ktot;
  if (Ntot > (1LL << 30) || Ktot > (1LL << 30)) return cudaErrorInvalidValue;
  p.nm = (int)gm.size();
  p.nn = (int)gn.size();
  p.nk = (int)gk.size();
  p.nb = (int)batch.size();
  for (int i = 0; i < p.nm; ++i) { p.mdim[i] = (int)gm[i].d; p.sAm[i] = gm[i].s0; p.sCm[i] = gm[i].s1; }
  for (int i = 0; i < p.nn; ++i) { p.ndim[i] = (int)gn[i].d; p.sBn[i] = gn[i].s0; p.sCn[i] = gn[i].s1; }
  for (int i = 0; i < p.nk; ++i) { p.kdim[i] = (int)gk[i].d; p.sAk[i] = gk[i].s0; p.sBk[i] = gk[i].s1; }
  nbatch = 1;
  for (int i = 0; i < p.nb; ++i) {
    p.bdim[i] = (int)batch[i].d;
    p.sCb[i] = batch[i].s0;
    p.sAb[i] = batch[i].s1;
    p.sBb[i] = batch[i].s2;
    nbatch *= batch[i].d;
  }
  if (nbatch > 65535) return cudaErrorInvalidValue;
  p.aidx = nullptr;
  p.bidx = nullptr;
  for (size_t i = 0; i < gb_idx_lab.size(); ++i) {
    if (gb_idx_lab[i] == a_idx_label) { p.aidx = A.idx; p.a_idx_ld = A.idx_ld; p.a_idx_stride = A.idx_stride; p.a_idx_grp = (int)i; }
    if (gb_idx_lab[i] == b_idx_label) { p.bidx = B.idx; p.b_idx_ld = B.idx_ld; p.b_idx_stride = B.idx_stride; p.b_idx_grp = (int)i; }
  }
  if ((A.idx && !p.aidx) || (B.idx && !p.bidx)) return cudaErrorInvalidValue;
  p.aoff = p.boffs = p.coff = nullptr;
  for (size_t i = 0; i < gb_idx_lab.size(); ++i) {
    if (A.boff && gb_idx_lab[i] == A.boff_label) { p.aoff = A.boff; p.aoff_grp = (int)i; }
    if (B.boff && gb_idx_lab[i] == B.boff_label) { p.boffs = B.boff; p.boff_grp = (int)i; }
    if (C.boff && gb_idx_lab[i] == C.boff_label) { p.coff = C.boff; p.coff_grp = (int)i; }
  }
  if ((A.boff && !p.aoff) || (B.boff && !p.boffs) || (C.boff && !p.coff)) return cudaErrorInvalidValue;
  p.A = A.ptr;
  p.B = B.ptr;
  p.C = C.ptr;
  p.conjA = A.conj;
  p.conjB = B.conj;
  p.alpha = alpha;
  p.beta = beta;
  p.beta_zero = (beta.x == 0.0 && beta.y == 0.0);
  p.a_kfast = (p.nk > 0 && p.sAk[0] == 1 && !(p.nm > 0 && p.sAm[0] == 1));
  p.b_kfast = false;
  if (p.nk > 0) {
    long long mk = p.sBk[0];
    for (int i = 0; i < p.nk; ++i) mk = std::min(mk, p.sBk[i]);
    p.b_kfast = (mk == 1 && !(p.nn > 0 && p.sBn[0] == 1));
    // B innermost K group must be the decomposition's first: re-sort K by B stride when B is k-fast
    if (p.b_kfast && p.sBk[0] != 1 && !p.a_kfast) {
      std::sort(gk.begin(), gk.end(), [](const Grp& a, const Grp& b) { return a.s1 < b.s1; });
      for (int i = 0; i < p.nk; ++i) { p.kdim[i] = (int)gk[i].d; p.sAk[i] = gk[i].s0; p.sBk[i] = gk[i].s1; }
    }
    p.b_kfast = (p.sBk[0] == 1 && !(p.nn > 0 && p.sBn[0] == 1));
  }
  if (p.M == 0 || p.N == 0) *empty = true;
  return cudaSuccess;
}

cudaError_t contract(const TView& A, const TView& B, const TView& C, Prec prec, cudaStream_t st, double2 alpha,
                     double2 beta, double* flops_out, ContractTiming* timing) {
  if (flops_out) *flops_out = 0.0;
  GemmParams p{};
  long long nbatch = 1;
  bool empty = false;
  cudaError_t pe = plan_params(A, B, C, alpha, beta, p, nbatch, &empty);
  if (pe != cudaSuccess || empty) return pe;
  if (flops_out) *flops_out = 8.0 * (double)p.M * (double)p.N * (double)p.K * (double)nbatch;
  if (prec == Prec::TF32X3) {
    // small contractions stay on the SIMT kernel (packing and tile waste dominate)
    const bool force = timing && timing->force_tc;
    if (p.beta_zero && alpha.x == 1.0 && alpha.y == 0.0 && (force || tc_worth_it(p, nbatch))) {
      bool handled = false;
      cudaError_t e = contract_tc(p, nbatch, st, timing, &handled);
      if (handled || e != cudaSuccess) return e;
    }
    if (force) return cudaErrorNotSupported;
    prec = Prec::F32;
  }
  long long gx = (p.M + 63) / 64;
  int gy = (p.N + 63) / 64;
  if (gx > 2147483647LL || gy > 65535) return cudaErrorInvalidValue;
  // split K when one batch entry's output has too few tiles to fill the GPU.  The
  // split count sets the summation order, so it follows the entry's shape only (at most
  // 15 splits: grids of up to 4096 entries fit), never the batch count; only batches
  // beyond 65535 / 15 entries cap it further.
  const long long tiles = gx * gy * nbatch;
  const long long tiles_e = gx * gy;
  int splits = 1;
  if (tiles_e < 2 * 152 && p.K >= 1024) {
    splits = (int)std::min<long long>(std::min<long long>(15, p.K / 512), (4 * 152 + tiles_e - 1) / tiles_e);
    splits = std::max(1, std::min<int>(splits, (int)(65535 / std::max<long long>(1, nbatch))));
  }
  const int bk = (prec == Prec::F32) ? 16 : 8;
  p.splits = splits;
  p.kchunk = splits > 1 ? (int)(((p.K + splits - 1) / splits + bk - 1) / bk * bk) : p.K;
  p.partial = nullptr;
  const size_t acc_bytes = (prec == Prec::F32) ? sizeof(float2) : sizeof(double2);
  if (splits > 1) {
    cudaError_t e = cudaMallocAsync(&p.partial, acc_bytes * 4096 * (size_t)tiles * splits, st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)(nbatch * splits));
  switch (prec) {
    case Prec::F64: gemm_kernel<double2, double2, double2, 8><<<grid, 256, 0, st>>>(p); break;
    case Prec::F32: gemm_kernel<float2, float2, float2, 16><<<grid, 256, 0, st>>>(p); break;
    case Prec::F32_ACC64: gemm_kernel<float2, double2, double2, 8><<<grid, 256, 0, st>>>(p); break;
  }
  g_launches++;
  if (splits > 1) {
    switch (prec) {
      case Prec::F64: splitk_reduce_kernel<double2, double2><<<(unsigned)tiles, 256, 0, st>>>(p, (unsigned)gx, gy); break;
      case Prec::F32: splitk_reduce_kernel<float2, float2><<<(unsigned)tiles, 256, 0, st>>>(p, (unsigned)gx, gy); break;
      case Prec::F32_ACC64: splitk_reduce_kernel<double2, double2><<<(unsigned)tiles, 256, 0, st>>>(p, (unsigned)gx, gy); break;
    }
    g_launches++;
    cudaFreeAsync(p.partial, st);
  }
  return cudaGetLastError();
}

cudaError_t contract_plan(const TView& A, const TView& B, const TView& C, long long* out) {
  for (int i = 0; i < 11; ++i) out[i] = 0;
  GemmParams p{};
  long long nbatch = 1;
  bool empty = false;
  cudaError_t e = plan_params(A, B, C, make_double2(1.0, 0.0), make_double2(0.0, 0.0), p, nbatch, &empty);
  if (e != cudaSuccess || empty) return e;
  out[7] = p.M;
  out[8] = p.N;
  out[9] = p.K;
  out[10] = nbatch;
  TcRole r;
  if (!tc_worth_it(p, nbatch) || !pick_role(p, nbatch, r)) return cudaSuccess;
  out[0] = 1;
  out[1] = r.swapped ? 1 : 0;
  out[2] = r.ad;
  out[3] = r.a_sh;
  out[4] = r.b_sh;
  out[5] = (r.b_sh && !r.a_sh) ? 1 : 0;
  out[6] = tc_tile_n(r.q.N);
  out[7] = r.q.M;
  out[8] = r.q.N;
  return cudaSuccess;
}

}  // namespace tns
