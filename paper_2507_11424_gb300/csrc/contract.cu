// Strided tensor-contraction GEMM (SIMT) and the host planner.  See contract.cuh.
#include "contract.cuh"

#include <algorithm>
#include <atomic>
#include <cstdio>

namespace tns {

static std::atomic<long long> g_launches{0};
long long contract_launches() { return g_launches.load(); }

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

cudaError_t contract(const TView& A, const TView& B, const TView& C, Prec prec, cudaStream_t st, double2 alpha,
                     double2 beta, double* flops_out) {
  if (flops_out) *flops_out = 0.0;
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
    if (l.d == 0) return cudaSuccess;  // empty contraction or empty output
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
  GemmParams p{};
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
  long long nbatch = 1;
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
  if (p.M == 0 || p.N == 0) return cudaSuccess;
  if (flops_out) *flops_out = 8.0 * (double)p.M * (double)p.N * (double)p.K * (double)nbatch;
  long long gx = (p.M + 63) / 64;
  int gy = (p.N + 63) / 64;
  if (gx > 2147483647LL || gy > 65535) return cudaErrorInvalidValue;
  // split K when the output has too few tiles to fill the GPU
  const long long tiles = gx * gy * nbatch;
  int splits = 1;
  if (tiles < 2 * 152 && p.K >= 1024) {
    splits = (int)std::min<long long>(std::min<long long>(64, p.K / 512), (4 * 152 + tiles - 1) / tiles);
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

}  // namespace tns
