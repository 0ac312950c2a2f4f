// Generalized boundary-MPS sampler (Appendix "Sampling from a Tensor Network
// State", Fig. 7) and single-layer amplitudes, batched over samples.
//
// Partitions are grid rows b = 0..H-1.  The norm environments E[b] (the paper's
// M_{b -> b-1}) are contracted once from the bottom: absorb the ket row then the
// bra row, each followed by a zip-up compression to rank R.  Each chunk of
// samples then sweeps the rows: absorb row b into the sample's boundary MPS and
// compress (zip-up; the truncated SVD of every site is taken by a randomized
// range finder with one subspace iteration and a shared Philox test matrix),
// contract the right environments F, and draw the row's qubits left to right
// from their one-site conditionals, projecting as it goes.  Rows alternate
// direction so every zip starts at the orthogonality centre the previous one
// left behind.
#include <cmath>
#include <cstdio>
#include <functional>
#include <vector>

#include "linalg.cuh"
#include "state.h"
#include "tc_gemm.cuh"

namespace tns {

// Shifts of the Cholesky orthonormalisation, relative to the largest diagonal entry of
// the Gram matrix.  In the mixed path the Gram matrices are FP32 sums over up to ~10^4
// rows, whose rounding (~sqrt(rows) eps_32 ~ 10^-5) must stay below the shift of every
// pass, or the shifted Gram can be indefinite; the later passes restore orthonormality
// to that level.
static constexpr double ORTH_SHIFT_FP64 = 1e-14;
static constexpr double ORTH_SHIFT_CQR_FIRST = 1e-5;
static constexpr double ORTH_SHIFT_CQR_NEXT = 1e-5;

static inline int nblk(long long n, int t = 256) { return (int)std::min<long long>((n + t - 1) / t, 1 << 20); }

// ------------------------------------------------------------------ kernels
template <typename C> __global__ void convert_kernel(const cd* in, C* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = from_cd<C>(in[i]);
}

template <typename C> __global__ void fill_kernel(C* out, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = from_cd<C>(mk(v, 0.0));
}

// Range-finder test matrix Omega[i][j] (n x kk): Philox counter (i, j, row*4096+site,
// 0x80000000 | stage), key = seed; Re from words 0,1 and Im from words 2,3, each 2u-1.
template <typename C>
__global__ void omega_kernel(C* out, int n, int kk, uint64_t seed_arg, const uint64_t* seed_dev, int stage, int row,
                             int site) {
  const uint64_t seed = seed_dev ? *seed_dev : seed_arg;
  long long tot = (long long)n * kk;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    uint32_t i = (uint32_t)(idx / kk), j = (uint32_t)(idx % kk);
    Philox4 w = philox4x32_10(i, j, (uint32_t)(row * 4096 + site), 0x80000000u | (uint32_t)stage,
                              (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    double re = 2.0 * u53(w.v[0], w.v[1]) - 1.0, im = 2.0 * u53(w.v[2], w.v[3]) - 1.0;
    out[idx] = from_cd<C>(mk(re, im));
  }
}


// UBt[b][i][r] = UB[b][i][r] for r < Rk (first Rk eigenvectors, descending).
template <typename C> __global__ void take_cols_kernel(const cd* UB, int n, int Rk, C* out, int batch) {
  long long tot = (long long)batch * n * Rk;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    long long b = idx / ((long long)n * Rk);
    int rem = (int)(idx % ((long long)n * Rk));
    int i = rem / Rk, r = rem % Rk;
    out[idx] = from_cd<C>(UB[b * n * n + (long long)i * n + r]);
  }
}

// Column phase convention: make sum_i K[i][col] / sqrt(i+1) real positive; when
// that sum is below 1e-8, make the first largest-magnitude entry real positive.
// Block (g, b) handles columns 32g .. 32g+31 of batch entry b: lane = column, warp =
// row group (rows w, w + PF_GROUPS, ...), so every warp load is one coalesced run of
// 32 consecutive columns of a row; the row groups' partial sums are combined in a
// fixed order, then the same walk applies the phase.
constexpr int PF_GROUPS = 16;
template <typename C> __global__ void __launch_bounds__(32 * PF_GROUPS) phase_fix_kernel(C* K, int M, int Rk) {
  const long long b = blockIdx.y;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool active = col < Rk;
  C* k = K + b * (long long)M * Rk + col;
  __shared__ double sx[PF_GROUPS][32], sy[PF_GROUPS][32], sm[PF_GROUPS][32];
  __shared__ int si[PF_GROUPS][32];
  __shared__ cd ph[32];
  double cx = 0.0, cy = 0.0, best = -1.0;
  int bi = 0x7fffffff;
  if (active)
    for (int i = grp; i < M; i += PF_GROUPS) {
      cd v = to_cd(k[(long long)i * Rk]);
      double w = 1.0 / sqrt((double)i + 1.0);
      cx += w * v.x;
      cy += w * v.y;
      double a = cabs2(v);
      if (a > best) { best = a; bi = i; }       // rows ascend: the first largest wins ties
    }
  sx[grp][lane] = cx; sy[grp][lane] = cy; sm[grp][lane] = best; si[grp][lane] = bi;
  __syncthreads();
  if (grp == 0 && active) {
    double ax = 0.0, ay = 0.0, m = -1.0;
    int mi = 0x7fffffff;
    for (int g = 0; g < PF_GROUPS; ++g) {
      ax += sx[g][lane];
      ay += sy[g][lane];
      const double m2 = sm[g][lane];
      const int i2 = si[g][lane];
      if (m2 > m || (m2 == m && i2 < mi)) { m = m2; mi = i2; }
    }
    const double a = sqrt(ax * ax + ay * ay);
    cd p = mk(1.0, 0.0);
    if (a > 1e-8) p = mk(ax / a, -ay / a);
    else if (m > 0.0 && mi < M) {
      cd v = to_cd(k[(long long)mi * Rk]);
      double av = sqrt(cabs2(v));
      p = mk(v.x / av, -v.y / av);
    }
    ph[lane] = p;
  }
  __syncthreads();
  if (!active) return;
  const cd p = ph[lane];
  for (int i = grp; i < M; i += PF_GROUPS) {
    cd v = to_cd(k[(long long)i * Rk]);
    k[(long long)i * Rk] = from_cd<C>(cmul(v, p));
  }
}

// K = T / |T| per batch entry; logscale[b] += log|T| (or -inf).
template <typename C> __global__ void normalize_last_kernel(const C* T, long long M, C* K, double* logscale) {
  const long long b = blockIdx.x;
  __shared__ double red[256];
  double s2 = 0.0;
  for (long long i = threadIdx.x; i < M; i += blockDim.x) s2 += cabs2(to_cd(T[b * M + i]));
  red[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  double nrm = sqrt(red[0]);
  double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (long long i = threadIdx.x; i < M; i += blockDim.x) K[b * M + i] = from_cd<C>(cscale(to_cd(T[b * M + i]), inv));
  if (threadIdx.x == 0 && logscale) logscale[b] += nrm > 0.0 ? log(nrm) : -INFINITY;
}

// Scale each batch entry of F to unit Frobenius norm (conditionals are scale free),
// in two kernels with NRM_SPLIT blocks per batch entry: norm_partial_kernel sums
// |F|^2 over its slice into part[b][k]; normalize_apply_kernel adds the NRM_SPLIT
// partials in index order (the same total in every block) and scales its slice.
constexpr int NRM_SPLIT = 16;
template <typename C> __global__ void norm_partial_kernel(const C* F, long long n, double* part) {
  const long long b = blockIdx.y;
  const long long chunk = (n + NRM_SPLIT - 1) / NRM_SPLIT;
  const long long lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  __shared__ double red[256];
  double s2 = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s2 += cabs2(to_cd(F[b * n + i]));
  red[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[b * NRM_SPLIT + blockIdx.x] = red[0];
}
template <typename C> __global__ void normalize_apply_kernel(C* F, long long n, const double* part) {
  const long long b = blockIdx.y;
  const long long chunk = (n + NRM_SPLIT - 1) / NRM_SPLIT;
  const long long lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double s2 = 0.0;
  for (int k = 0; k < NRM_SPLIT; ++k) s2 += part[b * NRM_SPLIT + k];
  const double nrm = sqrt(s2);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) F[b * n + i] = from_cd<C>(cscale(to_cd(F[b * n + i]), inv));
}

// Per-call arguments of the sampler's chunk, read on the device so that one captured
// launch sequence serves every call: the sampling seed (also the key of the
// range-finder test matrices), the chunk's first sample index and the output buffers.
struct SampleCall {
  uint64_t seed;
  long long sample0;     // the chunk's first row of the output buffers
  long long first;       // stream index of output row 0 (Philox counter = first + row)
  uint8_t* bits;
  const uint8_t* forced;
  double* logq;
  double* cond;
};

// Conditional marginals of one qubit for every sample of the chunk, in two
// kernels with MARG_SPLIT blocks per sample (enough blocks to fill the GPU at any
// chunk size):
//   marginal_partial_kernel: block (k, i) sums its slice of
//     rho_s = Re sum_e G[i][s][e] F[i][e]  (s = 0, 1) into part[i][k][s];
//   marginal_draw_kernel: every block of sample i adds the MARG_SPLIT partials in
//     index order (the same total in every block), forms q0 = rho0 / (rho0 + rho1)
//     (negative rho clamped to 0), takes x from the Philox uniform u (x = [u >= q0])
//     or the forced bit, and copies its slice of L_next = G[x] / (rho0 + rho1) and
//     of m_next = K'[:, x, :, :]; block 0 writes the bit, q0 and log q(x).
constexpr int MARG_SPLIT = 8;
template <typename C>
__global__ void __launch_bounds__(256)
marginal_partial_kernel(const C* __restrict__ G, int P, long long nel, const C* __restrict__ F, long long fstride,
                        double* __restrict__ part) {
  const long long sidx = blockIdx.y;
  const int k = blockIdx.x;
  const long long per = (nel + MARG_SPLIT - 1) / MARG_SPLIT;
  const long long e0 = k * per, e1 = min(nel, e0 + per);
  const C* g = G + sidx * P * nel;
  const C* f = F + sidx * fstride;
  __shared__ double r0[256], r1[256];
  double a0 = 0.0, a1 = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const cd fv = to_cd(f[e]);
    const cd g0 = to_cd(g[e]);
    a0 += g0.x * fv.x - g0.y * fv.y;
    if (P > 1) {
      const cd g1 = to_cd(g[nel + e]);
      a1 += g1.x * fv.x - g1.y * fv.y;
    }
  }
  r0[threadIdx.x] = a0;
  r1[threadIdx.x] = a1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { r0[threadIdx.x] += r0[threadIdx.x + o]; r1[threadIdx.x] += r1[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[(sidx * MARG_SPLIT + k) * 2] = r0[0];
    part[(sidx * MARG_SPLIT + k) * 2 + 1] = r1[0];
  }
}

template <typename C>
__global__ void __launch_bounds__(256)
marginal_draw_kernel(const double* __restrict__ part, const C* __restrict__ G, int P, long long nel,
                     const C* __restrict__ Kp, long long kstride, int ka, int Dd, int kb, C* __restrict__ Lnext,
                     C* __restrict__ mnext, const SampleCall* __restrict__ call, int n_sites, int qubit) {
  const long long sidx = blockIdx.y;
  uint8_t* bits = call->bits;
  const uint8_t* forced = call->forced;
  double* logq = call->logq;
  double* cond = call->cond;
  const uint64_t seed = call->seed;
  const long long sample0 = call->sample0;
  const long long first = call->first;
  const int k = blockIdx.x;
  __shared__ int xs;
  __shared__ double invs;
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < MARG_SPLIT; ++i) {
      s0 += part[(sidx * MARG_SPLIT + i) * 2];
      s1 += part[(sidx * MARG_SPLIT + i) * 2 + 1];
    }
    const double p0 = fmax(s0, 0.0), p1 = (P > 1) ? fmax(s1, 0.0) : 0.0;
    const double tot = p0 + p1;
    int x = 0;
    if (P > 1) {
      const double q0 = tot > 0.0 ? p0 / tot : 0.5;
      const long long gs = sample0 + sidx;
      if (forced) {
        x = forced[gs * n_sites + qubit] ? 1 : 0;
      } else {
        const uint64_t ctr = (uint64_t)(first + gs);
        Philox4 w = philox4x32_10((uint32_t)(ctr & 0xffffffffu), (uint32_t)(ctr >> 32),
                                  (uint32_t)qubit, 0u, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
        const double u = u53(w.v[0], w.v[1]);
        x = (u >= q0) ? 1 : 0;
      }
      if (k == 0) {
        if (!forced) bits[gs * n_sites + qubit] = (uint8_t)x;
        const double qx = x ? 1.0 - q0 : q0;
        logq[gs] += qx > 0.0 ? log(qx) : -INFINITY;
        if (cond) cond[gs * n_sites + qubit] = q0;
      }
    }
    xs = x;
    invs = tot > 0.0 ? 1.0 / tot : 1.0;
  }
  __syncthreads();
  const int x = xs;
  const double inv = invs;
  const long long per = (nel + MARG_SPLIT - 1) / MARG_SPLIT;
  const long long e1 = min(nel, (k + 1) * per);
  const C* g = G + (sidx * P + x) * nel;
  for (long long e = k * per + threadIdx.x; e < e1; e += blockDim.x)
    Lnext[sidx * nel + e] = from_cd<C>(cscale(to_cd(g[e]), inv));
  const C* kp = Kp + sidx * kstride;
  const long long nm = (long long)ka * Dd * kb;
  const long long mper = (nm + MARG_SPLIT - 1) / MARG_SPLIT;
  const long long m1 = min(nm, (k + 1) * mper);
  for (long long e = k * mper + threadIdx.x; e < m1; e += blockDim.x) {
    const long long a = e / ((long long)Dd * kb), rem = e % ((long long)Dd * kb);
    mnext[sidx * nm + e] = kp[((a * P + x) * Dd) * kb + rem];
  }
}

// Amplitude of the final (all dimension 1) boundary MPS: product of W scalars.
template <typename C>
__global__ void amp_final_kernel(const C* const* sites, int W, long long S, double* log_abs, double* phase) {
  long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= S) return;
  cd z = mk(1.0, 0.0);
  for (int j = 0; j < W; ++j) z = cmul(z, to_cd(sites[j][b]));
  double a = sqrt(cabs2(z));
  if (a > 0.0 && isfinite(log_abs[b])) {
    log_abs[b] += log(a);
    phase[b] = atan2(z.y, z.x);
  } else {
    log_abs[b] = -INFINITY;
    phase[b] = 0.0;
  }
}

// ------------------------------------------------------------------ host side
enum ProfClass {
  PC_ENV = 0, PC_SWEEP = 1, PC_ZIP = 2, PC_EIGH = 3, PC_MARG = 4,
  PC_PREP = 5, PC_PREP_SWEEP = 6, PC_PREP_ZIP = 7,    // tensor-core operand packing per contraction class
  PC_ZIP_SIMT = 8, PC_SWEEP_SIMT = 9                  // zip / sweep contractions that ran on the CUDA cores
};

// contract() bracketed by the state's profiler (no-op when profiling is off).
// Th[b][n][m] = conj(T[b][m][n]) through 32 x 32 shared-memory tiles (both sides coalesced).
template <typename C>
__global__ void transpose_conj_kernel(const C* __restrict__ T, C* __restrict__ Th, long long M, long long N) {
  __shared__ C tile[32][33];
  const long long b = blockIdx.z;
  const long long m0 = (long long)blockIdx.y * 32, n0 = (long long)blockIdx.x * 32;
  const C* src = T + b * M * N;
  C* dst = Th + b * M * N;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const long long m = m0 + r, n = n0 + threadIdx.x;
    if (m < M && n < N) tile[r][threadIdx.x] = src[m * N + n];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const long long n = n0 + r, m = m0 + threadIdx.x;
    if (m < M && n < N) dst[n * M + m] = cconj(tile[threadIdx.x][r]);
  }
}

// Gram matrices of tall complex64 panels: G[b] = Y[b]^H Y[b] with Y [b][M][n]
// (row-major), G [b][n][n], FP32 accumulation on the CUDA cores.  Block (split,
// b) sums rows [split * rows_per, ...) of entry b into P[b][split]; thread (x, y)
// of the (nb x nb) block, nb = ceil(n / 4), owns the 4 x 4 tile G[4y.., 4x..]; Y
// streams through shared memory 32 rows at a time.  gram_reduce_kernel adds the
// splits in index order (deterministic).
constexpr int GRAM_MAX_N = 128;
// G is Hermitian: block (split, b) computes only the 4 x 4 tiles on and above the
// diagonal, one tile per thread (threadIdx.x enumerates them row by row), and the
// reduction fills the lower triangle by conjugation.
__global__ void __launch_bounds__(528) gram_partial_kernel(const cf* __restrict__ Y, long long M, int n,
                                                            long long rows_per, cf* __restrict__ P) {
  __shared__ cf ys[32][GRAM_MAX_N];
  const long long b = blockIdx.y;
  const int split = blockIdx.x;
  const long long r0 = split * rows_per, r1 = min(M, r0 + rows_per);
  const cf* src = Y + b * M * n;
  const int nb = (n + 3) / 4;
  int ty = 0, tx = threadIdx.x;                 // upper-triangular tile (ty <= tx)
  while (ty < nb && tx >= nb - ty) { tx -= nb - ty; ++ty; }
  tx += ty;
  const bool active = ty < nb;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (long long m0 = r0; m0 < r1; m0 += 32) {
    const int rows = (int)(r1 - m0 < 32 ? r1 - m0 : 32);
    for (int e = threadIdx.x; e < 32 * n; e += blockDim.x) {
      const int r = e / n, c = e % n;
      ys[r][c] = r < rows ? src[(m0 + r) * n + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (active) {
      for (int r = 0; r < rows; ++r) {
        float2 a[4], v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int ci = 4 * ty + i, cj = 4 * tx + i;
          a[i] = ci < n ? ys[r][ci] : make_float2(0.f, 0.f);
          v[i] = cj < n ? ys[r][cj] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {          // acc += conj(a_i) v_j
            acc[i][j].x = fmaf(a[i].x, v[j].x, fmaf(a[i].y, v[j].y, acc[i][j].x));
            acc[i][j].y = fmaf(a[i].x, v[j].y, fmaf(-a[i].y, v[j].x, acc[i][j].y));
          }
      }
    }
    __syncthreads();
  }
  if (!active) return;
  cf* dst = P + (b * gridDim.x + split) * (long long)n * n;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ci = 4 * ty + i, cj = 4 * tx + j;
      if (ci < n && cj < n) dst[(long long)ci * n + cj] = acc[i][j];
    }
}

// G[b][i][j] = sum of the splits' partial Grams in index order, read from the computed
// upper triangle of 4 x 4 tiles (conjugated for entries below it).
__global__ void gram_reduce_kernel(const cf* __restrict__ P, int splits, int n, long long total, cf* __restrict__ G) {
  const long long nn = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / nn, e = i % nn;
    const int r = (int)(e / n), c = (int)(e % n);
    const bool upper = (r / 4) <= (c / 4);
    const long long src = upper ? e : (long long)c * n + r;
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < splits; ++k) {
      const float2 v = P[(b * splits + k) * nn + src];
      acc.x += v.x;
      acc.y += v.y;
    }
    if (!upper) acc.y = -acc.y;
    G[i] = acc;
  }
}

static cudaError_t pcontract(tns_state* s, int cls, const TView& A, const TView& B, const TView& C, Prec p) {
  cudaEvent_t ev = s->prof.begin(s->st);
  double fl = 0.0;
  ContractTiming tm;
  if (ev && p == Prec::TF32X3 &&
      (cudaEventCreate(&tm.mma_begin) != cudaSuccess || cudaEventCreate(&tm.mma_end) != cudaSuccess)) {
    if (tm.mma_begin) cudaEventDestroy(tm.mma_begin);
    tm.mma_begin = tm.mma_end = nullptr;
  }
  cudaError_t e = contract(A, B, C, p, s->st, make_double2(1.0, 0.0), make_double2(0.0, 0.0), &fl, &tm);
  if (tm.used_tc && ev) {
    // operand packing counts as tensor-core preparation, the GEMM kernel as the class
    const int prep = cls == PC_ENV ? PC_PREP : (cls == PC_SWEEP ? PC_PREP_SWEEP : PC_PREP_ZIP);
    s->prof.span(prep, ev, tm.mma_begin, 0.0, true, false);
    s->prof.span(cls, tm.mma_begin, tm.mma_end, fl, true, true);
  } else {
    if (tm.mma_begin) cudaEventDestroy(tm.mma_begin);
    if (tm.mma_end) cudaEventDestroy(tm.mma_end);
    int c = cls;
    if (p == Prec::TF32X3 && cls == PC_ZIP) c = PC_ZIP_SIMT;
    if (p == Prec::TF32X3 && cls == PC_SWEEP) c = PC_SWEEP_SIMT;
    s->prof.end(c, ev, fl, s->st);
  }
  return e;
}

// G = Y^H Y per batch entry (Y: S x M x n): the dedicated Gram kernels for complex64
// panels with n <= 128, else the general contraction.
static cudaError_t pgram(tns_state* s, Prec p, const void* Y, long long S, long long M, int n, void* G) {
  if (p == Prec::F64 || n > GRAM_MAX_N || S > 65535)
    return pcontract(s, PC_ZIP, view(const_cast<void*>(Y), "Smc", {S, M, n}, true),
                     view(const_cast<void*>(Y), "Sme", {S, M, n}), view(G, "Sce", {S, n, n}), p);
  // row splits from the panel height only (at least 256 rows each, at most 8): the
  // split sets the summation order, which must not depend on the chunk size
  int splits = (int)std::max<long long>(1, std::min<long long>((M + 255) / 256, 8));
  const long long rows_per = (M + splits - 1) / splits;
  splits = (int)((M + rows_per - 1) / rows_per);
  cudaEvent_t ev = s->prof.begin(s->st);
  cf* P = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&P, sizeof(cf) * (size_t)S * splits * n * n, s->st);
  if (e != cudaSuccess) return e;
  const int nb = (n + 3) / 4;
  gram_partial_kernel<<<dim3((unsigned)splits, (unsigned)S), nb * (nb + 1) / 2, 0, s->st>>>((const cf*)Y, M, n,
                                                                                           rows_per, P);
  s->launches++;
  e = cudaGetLastError();
  const long long total = S * (long long)n * n;
  if (e == cudaSuccess) gram_reduce_kernel<<<nblk(total), 256, 0, s->st>>>(P, splits, n, total, (cf*)G);
  s->launches++;
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFreeAsync(P, s->st);
  s->prof.end(PC_ZIP_SIMT, ev, 8.0 * (double)S * M * n * n, s->st);
  return e;
}

static cudaError_t peigh(tns_state* s, cd* A, int n, int batch, double* lam, cd* V, cd* work, int* status) {
  cudaEvent_t ev = s->prof.begin(s->st);
  cudaError_t e = eigh_batched(A, (long long)n * n, n, n, batch, lam, V, (long long)n * n, work, status, s->st);
  s->prof.end(PC_EIGH, ev, 0.0, s->st);
  return e;
}

struct Ctx {
  tns_state* s;
  cudaStream_t st;
  bool f64;
  Prec gp;
  size_t esz;
  uint64_t seed;
  int R;
  const uint64_t* seed_dev = nullptr;   // when set, kernels read the seed here (graph replays)
  int p = 8;      // range-finder oversampling: k = R + p columns
  int q = 1;      // subspace iterations (T T^H applications)
};

template <typename F> static void dispatch(bool f64, F&& f) {
  if (f64) f((cd*)nullptr);
  else f((cf*)nullptr);
}

static tns_status ensure_work_cells(tns_state* s, bool f64) {
  int want = f64 ? 0 : 1;
  if (s->work_prec == want && s->work_version == s->version && !s->work_cells.empty()) return TNS_OK;
  if (s->work_cells.empty()) s->work_cells.assign(s->cell.size(), nullptr);
  for (size_t ci = 0; ci < s->cell.size(); ++ci) {
    Cell& c = s->cell[ci];
    if (f64) {
      s->work_cells[ci] = nullptr;  // FP64 reads the master copy
      continue;
    }
    if (!s->work_cells[ci]) TNS_TRY_CUDA(cudaMalloc(&s->work_cells[ci], sizeof(cf) * c.cap));
    convert_kernel<cf><<<nblk(c.size()), 256, 0, s->st>>>(c.t, (cf*)s->work_cells[ci], c.size());
    s->launches++;
  }
  s->work_prec = want;
  s->work_gen++;
  s->work_version = s->version;
  return TNS_OK;
}

static void* cell_ptr(tns_state* s, int ci, bool f64) { return f64 ? (void*)s->cell[ci].t : s->work_cells[ci]; }

// Row b, logical site j (rev: right to left); labels for (s, u, logical-left, d, logical-right).
static TView cell_view(tns_state* s, bool f64, int b, int j, bool rev, char ls, char lu, char la, char ld, char lb,
                       bool conj = false) {
  int c = rev ? s->W - 1 - j : j;
  int ci = s->cidx(b, c);
  const Cell& cc = s->cell[ci];
  std::string lab = {ls, lu, rev ? lb : la, ld, rev ? la : lb};
  return view(cell_ptr(s, ci, f64), lab, {cc.dim[0], cc.dim[1], cc.dim[2], cc.dim[3], cc.dim[4]}, conj);
}

// Site of a stored MPS seen at logical site j of a row swept in direction rev,
// labels (logical-left, phys..., logical-right); optional leading sample axis.
static TView mps_view(const StoredMPS& m, int W, int j, bool rev, char la, const std::string& phys, char lb,
                      long long S, long long sstride, bool conj = false) {
  int c = rev ? W - 1 - j : j;
  int i = m.reversed ? W - 1 - c : c;
  bool same = (m.reversed == rev);
  std::string lab;
  std::vector<long long> dims;
  lab.push_back(same ? la : lb);
  dims.push_back(m.bond[i]);
  for (size_t k = 0; k < phys.size(); ++k) { lab.push_back(phys[k]); dims.push_back(m.phys[i][k]); }
  lab.push_back(same ? lb : la);
  dims.push_back(m.bond[i + 1]);
  TView v = view(m.site[i], lab, dims, conj);
  if (S > 0) {
    v.labels.insert(v.labels.begin(), 'S');
    v.dim.insert(v.dim.begin(), S);
    v.stride.insert(v.stride.begin(), sstride);
  }
  return v;
}

// Elements of logical site j (row direction rev) of a stored MPS.
static long long mps_site_size(const StoredMPS& m, int W, int j, bool rev) {
  int c = rev ? W - 1 - j : j;
  int i = m.reversed ? W - 1 - c : c;
  long long n = m.bond[i] * m.bond[i + 1];
  for (auto d : m.phys[i]) n *= d;
  return n;
}

static long long vdim(const TView& v, char l) {
  for (size_t i = 0; i < v.labels.size(); ++i)
    if (v.labels[i] == l) return v.dim[i];
  return -1;
}

static long long vsize_nos(const TView& v) {
  long long n = 1;
  for (size_t i = 0; i < v.labels.size(); ++i)
    if (v.labels[i] != 'S') n *= v.dim[i];
  return n;
}

struct ZipSpec {
  long long S;                                  // batch of the zip (1 = shared)
  std::function<TView(int)> mview;              // labels S a Pm b
  std::function<TView(int)> wview;              // labels l Pw r (+ S)
  std::string out_phys;                         // labels of the output physical legs
  int stage, row;
  bool rev;
  StoredMPS* out;                               // site buffers preassigned, S*cap each
  double* logscale;                             // device [S], += log |T_last| (may be null)
};

// Workspace request helper with a per-sample capacity.
static tns_status wsget(tns_state* s, const char* nm, size_t bytes, void** p) {
  TNS_TRY_CUDA(s->ws.get(nm, bytes, p));
  return TNS_OK;
}

// Q = orthonormal basis of range(Y) for each batch entry (Y, Q: S x M x kk).
// FP64 path: W = L^{-H} with L L^H = Y^H Y + 1e-14 max_i G_ii (the shift only
// regularises rank-deficient Y), Q = Y W.  Mixed path: shifted CholeskyQR3 in
// FP32 (Gram and products in FP32, the first pass's kk x kk Cholesky in FP64, the
// later two in FP32), every pass with
// shift 1e-5: the first gives a well-conditioned basis of the same range, the two
// more restore orthonormality to ~1e-5 (directions with Gram eigenvalue below the
// shift are damped, not lost).
static tns_status orth(Ctx& cx, void* Y, long long S, long long M, int kk, void* Qout, bool span_only = false) {
  tns_state* s = cx.s;
  void *G, *Wm;
  TNS_TRY(wsget(s, "z_G", sizeof(cd) * S * kk * kk, &G));
  TNS_TRY(wsget(s, "z_W", cx.esz * S * kk * kk, &Wm));
  cd* work = nullptr;
  if (!chol_fits_smem(kk)) TNS_TRY(wsget(s, "z_cwork", sizeof(cd) * S * 2 * kk * kk, (void**)&work));
  auto pass = [&](void* src, void* dst, double shift, bool fp32_factor) -> tns_status {
    TNS_TRY_CUDA(pgram(s, cx.gp, src, S, M, kk, G));
    cudaEvent_t ev = s->prof.begin(cx.st);
    TNS_TRY_CUDA(chol_w_batched(G, cx.f64, kk, (int)S, shift, Wm, cx.f64, work, cx.st, fp32_factor));
    s->prof.end(PC_EIGH, ev, 0.0, cx.st);
    s->launches++;
    TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(src, "Smc", {S, M, kk}), view(Wm, "Sce", {S, kk, kk}),
                           view(dst, "Sme", {S, M, kk}), cx.gp));
    return TNS_OK;
  };
  if (cx.f64) return pass(Y, Qout, ORTH_SHIFT_FP64, false);
  // between subspace iterations only the span matters: one pass, factorised in FP32,
  // gives a bounded basis of the same range
  if (span_only) return pass(Y, Qout, ORTH_SHIFT_CQR_FIRST, true);
  void* tmp;
  TNS_TRY(wsget(s, "z_Q2", cx.esz * S * M * kk, &tmp));
  // the first pass sees the Gram of Y (condition up to ~1/shift) and factorises in
  // FP64; the two more see the Gram of an already well-conditioned basis (close to
  // the identity), whose FP32 Cholesky is as accurate as the FP32 Gram it factorises
  TNS_TRY(pass(Y, Qout, ORTH_SHIFT_CQR_FIRST, false));
  TNS_TRY(pass(Qout, tmp, ORTH_SHIFT_CQR_NEXT, true));
  return pass(tmp, Qout, ORTH_SHIFT_CQR_NEXT, true);
}

// Rank-R factorisation T = K C of each batch entry (T: S x M x N): randomized
// range finder with q subspace iterations (Halko, Martinsson, Tropp 2011, Alg. 4.4),
// orthonormalising after every application:
//   Y = T Omega (k = R + p columns); q times { Z = orth(T^H orth(Y)), Y = T Z };
//   Q = orth(Y),
// then the truncated SVD of B = Q^H T from the eigendecomposition of B B^H (FP64
// path: FP64; mixed path: FP32, the precision B carries):
//   K = Q U_B[:, :R] (column phases fixed), C = K^H T (returned conjugate-transposed).
// The error of the kept subspace shrinks like (sigma_{k+1} / sigma_R)^(2q+1), so
// flat spectra at the cut need k well above R and a few iterations.  The products
// that contract over M read T^H from one transposed copy.  With k >= N the test
// matrix is the identity and Y = T: the step is an exact truncated SVD.
static tns_status truncate(Ctx& cx, void* T, long long S, long long M, long long N, int stage, int row, int site,
                           void* Kout, void* Cout, int* Rk_out) {
  tns_state* s = cx.s;
  const int kk = (int)std::min<long long>(std::min<long long>(cx.R + cx.p, M), N);
  const int Rk = (int)std::min<long long>(std::min<long long>(cx.R, M), N);
  *Rk_out = Rk;
  void *Y, *Q, *Z, *B, *UBt, *om;
  TNS_TRY(wsget(s, "z_Y", cx.esz * S * M * kk, &Y));
  TNS_TRY(wsget(s, "z_Q", cx.esz * S * M * kk, &Q));
  TNS_TRY(wsget(s, "z_Z", cx.esz * S * N * kk, &Z));
  TNS_TRY(wsget(s, "z_B", cx.esz * S * N * kk, &B));
  TNS_TRY(wsget(s, "z_UBt", cx.esz * S * kk * kk, &UBt));
  // Th = T^H (per batch entry), read in place by the products that contract over M
  void* Th;
  TNS_TRY(wsget(s, "z_Th", cx.esz * S * M * N, &Th));
  dispatch(cx.f64, [&](auto* tp) {
    using C = std::remove_pointer_t<decltype(tp)>;
    dim3 g((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32), (unsigned)S);
    transpose_conj_kernel<C><<<g, dim3(32, 8), 0, cx.st>>>((const C*)T, (C*)Th, M, N);
  });
  s->launches++;
  void* Ymat = Y;
  if (kk == N) {
    Ymat = T;  // test matrix = identity: the range of T is captured exactly
  } else {
    TNS_TRY(wsget(s, "z_om", cx.esz * N * kk, &om));
    dispatch(cx.f64, [&](auto* tp) {
      using C = std::remove_pointer_t<decltype(tp)>;
      omega_kernel<C><<<nblk(N * kk), 256, 0, cx.st>>>((C*)om, (int)N, kk, cx.seed, cx.seed_dev, stage, row, site);
    });
    s->launches++;
    TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(T, "Smn", {S, M, N}), view(om, "nc", {N, kk}), view(Y, "Smc", {S, M, kk}),
                           cx.gp));
    for (int it = 0; it < cx.q; ++it) {
      TNS_TRY(orth(cx, Y, S, M, kk, Q, true));
      TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(Th, "Snm", {S, N, M}), view(Q, "Sme", {S, M, kk}),
                             view(Z, "Sne", {S, N, kk}), cx.gp));
      TNS_TRY(orth(cx, Z, S, N, kk, B, true));
      TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(T, "Smn", {S, M, N}), view(B, "Sne", {S, N, kk}),
                             view(Y, "Sme", {S, M, kk}), cx.gp));
    }
  }
  TNS_TRY(orth(cx, Ymat, S, M, kk, Q));
  // Bt = T^H Q = conj(B)^T with B = Q^H T; read T^H in place from Th
  TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(Th, "Snm", {S, N, M}), view(Q, "Sme", {S, M, kk}),
                         view(B, "Sne", {S, N, kk}), cx.gp));
  cd *Hm, *V;
  double* mu;
  int* status;
  TNS_TRY(wsget(s, "z_H", sizeof(cd) * S * kk * kk, (void**)&Hm));
  TNS_TRY(wsget(s, "z_V2", sizeof(cd) * S * kk * kk, (void**)&V));
  TNS_TRY(wsget(s, "z_mu", sizeof(double) * S * kk, (void**)&mu));
  TNS_TRY(wsget(s, "z_status2", sizeof(int) * S, (void**)&status));
  // B B^H and its eigendecomposition: FP64 in the FP64 path; FP32 (the precision B
  // carries) in the mixed path
  const long long np = kk + (kk & 1);
  if (cx.f64) {
    TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(B, "Sne", {S, N, kk}, true), view(B, "Snf", {S, N, kk}),
                           view(Hm, "Sef", {S, kk, kk}), cx.gp));
    cd* work = nullptr;
    if (!eigh_fits_smem(kk)) TNS_TRY(wsget(s, "z_jwork", sizeof(cd) * S * 2 * np * np, (void**)&work));
    TNS_TRY_CUDA(peigh(s, Hm, kk, (int)S, mu, V, work, status));
  } else {
    void* H32;
    TNS_TRY(wsget(s, "z_H32", sizeof(cf) * S * kk * kk, &H32));
    TNS_TRY_CUDA(pgram(s, cx.gp, B, S, N, kk, H32));
    cf* work = nullptr;
    if (!jacobi_fits_smem_f32(kk)) TNS_TRY(wsget(s, "z_jwork32", sizeof(cf) * S * 2 * np * np, (void**)&work));
    cudaEvent_t ev = s->prof.begin(s->st);
    TNS_TRY_CUDA(eigh_batched_f32((const cf*)H32, kk * kk, kk, kk, (int)S, mu, V, kk * kk, work, status, s->st));
    s->prof.end(PC_EIGH, ev, 0.0, s->st);
    s->launches++;
  }
  dispatch(cx.f64, [&](auto* tp) {
    using C = std::remove_pointer_t<decltype(tp)>;
    take_cols_kernel<C><<<nblk(S * kk * Rk), 256, 0, cx.st>>>(V, kk, Rk, (C*)UBt, (int)S);
  });
  TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(Q, "Sme", {S, M, kk}), view(UBt, "Ser", {S, kk, Rk}),
                         view(Kout, "Smr", {S, M, Rk}), cx.gp));
  dispatch(cx.f64, [&](auto* tp) {
    using C = std::remove_pointer_t<decltype(tp)>;
    phase_fix_kernel<C><<<dim3((Rk + 31) / 32, (unsigned)S), 32 * PF_GROUPS, 0, cx.st>>>((C*)Kout, (int)M, Rk);
  });
  // C = K^H T, stored conjugate-transposed: Cout[S][n][r] = conj(C[r][n]) = (T^H K)[n][r]
  TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(Th, "Snm", {S, N, M}), view(Kout, "Smr", {S, M, Rk}),
                         view(Cout, "Snr", {S, N, Rk}), cx.gp));
  s->launches += 2;
  return TNS_OK;
}

// Zip-up compression of (MPS . MPO) to rank R along the spec's logical order.
static tns_status zip(Ctx& cx, ZipSpec& zs) {
  tns_state* s = cx.s;
  const int W = s->W;
  const long long S = zs.S;
  StoredMPS& out = *zs.out;
  out.reversed = zs.rev;
  out.bond.assign(W + 1, 1);
  out.phys.assign(W, {});
  void *Cp, *Cn, *X, *T;
  long long kprev = 1;
  // C_{-1} = 1
  long long chi = 1;
  for (auto& c : s->cell)
    for (int leg = 1; leg <= 4; ++leg) chi = std::max<long long>(chi, c.dim[leg]);
  const long long Ccap = (long long)cx.R * cx.R * chi;   // C[k][a][l]: k, a <= R, l <= chi
  TNS_TRY(wsget(s, "zip_C0", cx.esz * S * Ccap, &Cp));
  TNS_TRY(wsget(s, "zip_C1", cx.esz * S * Ccap, &Cn));
  dispatch(cx.f64, [&](auto* tp) {
    using C = std::remove_pointer_t<decltype(tp)>;
    fill_kernel<C><<<nblk(S), 256, 0, cx.st>>>((C*)Cp, S, 1.0);
  });
  s->launches++;
  long long a_prev = 1, l_prev = 1;
  for (int j = 0; j < W; ++j) {
    TView mv = zs.mview(j);
    TView wv = zs.wview(j);
    // labels of m: [S] a Pm b ; w: l Pw r [S]
    std::string Pm, Pw;
    for (char c : mv.labels)
      if (c != 'S' && c != 'a' && c != 'b') Pm.push_back(c);
    for (char c : wv.labels)
      if (c != 'S' && c != 'l' && c != 'r') Pw.push_back(c);
    const long long a = vdim(mv, 'a'), bdm = vdim(mv, 'b'), l = vdim(wv, 'l'), r = vdim(wv, 'r');
    if (a != a_prev || l != l_prev) {
      set_error("zip: bond mismatch at site %d (a %lld/%lld, l %lld/%lld)", j, a, a_prev, l, l_prev);
      return TNS_ERR_STATE;
    }
    // X[S][k][b][l][Pm] = sum_a C[S][k][a][l] m[S][a][Pm][b]  (rows (k,b), contiguous (l,Pm): the
    // next contraction reads X in place)
    std::vector<long long> xd = {S, kprev, bdm, l};
    std::string xl = "Skbl";
    long long xsz = kprev * bdm * l;
    for (char c : Pm) { xl.push_back(c); long long d = vdim(mv, c); xd.push_back(d); xsz *= d; }
    TNS_TRY(wsget(s, "zip_X", cx.esz * S * xsz, &X));
    // C is held conjugate-transposed ([S][a][l][k] = conj C[k][a][l]), see truncate()
    TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(Cp, "Salk", {S, a, l, kprev}, true), mv, view(X, xl, xd), cx.gp));
    // T[S][k][out][b][r] = sum_{l, Pc} X w
    std::vector<long long> td = {S, kprev};
    std::string tl = "Sk";
    long long Mrow = kprev;
    std::vector<long long> pdims;
    for (char c : zs.out_phys) {
      long long d = vdim(mv, c);
      if (d < 0) d = vdim(wv, c);
      tl.push_back(c);
      td.push_back(d);
      pdims.push_back(d);
      Mrow *= d;
    }
    tl += "br";
    td.push_back(bdm);
    td.push_back(r);
    const long long Ncol = bdm * r;
    TNS_TRY(wsget(s, "zip_T", cx.esz * S * Mrow * Ncol, &T));
    TNS_TRY_CUDA(pcontract(s, PC_ZIP, view(X, xl, xd), wv, view(T, tl, td), cx.gp));
    out.phys[j] = pdims;
    if (j == W - 1) {
      if (Ncol != 1) { set_error("zip: open right bond at the last site"); return TNS_ERR_STATE; }
      dispatch(cx.f64, [&](auto* tp) {
        using C = std::remove_pointer_t<decltype(tp)>;
        normalize_last_kernel<C><<<(unsigned)S, 256, 0, cx.st>>>((C*)T, Mrow, (C*)out.site[j], zs.logscale);
      });
      s->launches++;
      out.bond[j] = kprev;
      out.bond[j + 1] = 1;
      break;
    }
    int Rk = 0;
    TNS_TRY(truncate(cx, T, S, Mrow, Ncol, zs.stage, zs.row, j, out.site[j], Cn, &Rk));
    out.bond[j] = kprev;
    out.bond[j + 1] = Rk;
    std::swap(Cp, Cn);
    kprev = Rk;
    a_prev = bdm;
    l_prev = r;
  }
  return TNS_OK;
}

static void free_mps(StoredMPS& m) {
  for (auto p : m.site)
    if (p) cudaFree(p);
  m.site.clear();
}

// Bottom norm environments E[b], b = H..0 (E[0] gives <psi|psi>), at rank R.  With
// top = true, the same construction on the state read upside down (row b of that
// frame is row H-1-b, up and down legs exchanged): Et[H-b] is then the environment
// of rows 0..b-1 on the up legs of row b.  Test matrices are keyed by the row index
// of the frame the environments are built in.
static tns_status build_envs(Ctx& cx_in, bool top = false) {
  // environment test matrices use key 0, independent of the sampling seed
  Ctx cx = cx_in;
  cx.seed = 0;
  cx.seed_dev = nullptr;
  tns_state* s = cx.s;
  cx.q = s->rf_q_env;
  EnvCache& ec = top ? s->env_top : s->env;
  const int prec = cx.f64 ? 0 : 1;
  if (ec.valid && ec.chi_b == cx.R && ec.prec == prec && ec.version == s->version && ec.p == cx.p && ec.q == cx.q)
    return TNS_OK;
  for (auto& E : ec.E) free_mps(E);
  ec.E.assign(s->H + 1, StoredMPS());
  ec.valid = false;
  const int H = s->H, W = s->W;
  // E[H]: trivial
  StoredMPS& EH = ec.E[H];
  EH.reversed = true;
  EH.bond.assign(W + 1, 1);
  EH.phys.assign(W, {1, 1});
  EH.site.assign(W, nullptr);
  for (int c = 0; c < W; ++c) {
    TNS_TRY_CUDA(cudaMalloc(&EH.site[c], cx.esz));
    dispatch(cx.f64, [&](auto* tp) {
      using C = std::remove_pointer_t<decltype(tp)>;
      fill_kernel<C><<<1, 32, 0, cx.st>>>((C*)EH.site[c], 1, 1.0);
    });
  }
  double* dlog;
  TNS_TRY(wsget(s, "env_log", sizeof(double), (void**)&dlog));
  TNS_TRY_CUDA(cudaMemsetAsync(dlog, 0, sizeof(double), cx.st));
  StoredMPS Z;
  const long long R = cx.R;
  const char KU = top ? 'd' : 'u', KD = top ? 'u' : 'd', BU = top ? 'D' : 'U', BD = top ? 'U' : 'D';
  for (int b = H - 1; b >= 0; --b) {
    const int r = top ? H - 1 - b : b;      // the grid row absorbed at this step
    // capacity per site: R * phys * R
    long long chi = 1;
    for (int c = 0; c < W; ++c)
      for (int leg = 1; leg <= 4; ++leg) chi = std::max<long long>(chi, s->cell[s->cidx(r, c)].dim[leg]);
    Z.site.assign(W, nullptr);
    for (int c = 0; c < W; ++c) {
      char nm[32];
      snprintf(nm, sizeof nm, "env_Z%d", c);
      TNS_TRY(wsget(s, nm, cx.esz * R * R * 2 * chi * chi, &Z.site[c]));
    }
    ZipSpec ket;
    ket.S = 1;
    ket.mview = [&, b](int j) { return mps_view(ec.E[b + 1], W, j, false, 'a', "Dd", 'b', 0, 0); };
    ket.wview = [&, r](int j) { return cell_view(s, cx.f64, r, j, false, 's', KU, 'l', KD, 'r'); };
    ket.out_phys = "suD";
    ket.stage = STAGE_ENV_KET;
    ket.row = b;
    ket.rev = false;
    ket.out = &Z;
    ket.logscale = dlog;
    TNS_TRY(zip(cx, ket));
    StoredMPS& Eb = ec.E[b];
    Eb.site.assign(W, nullptr);
    long long Du = 1;
    for (int c = 0; c < W; ++c) Du = std::max<long long>(Du, s->cell[s->cidx(r, c)].dim[top ? LEG_D : LEG_U]);
    for (int c = 0; c < W; ++c) TNS_TRY_CUDA(cudaMalloc(&Eb.site[c], cx.esz * R * R * Du * Du));
    ZipSpec bra;
    bra.S = 1;
    bra.mview = [&](int j) { return mps_view(Z, W, j, true, 'a', "suD", 'b', 0, 0); };
    bra.wview = [&, r](int j) { return cell_view(s, cx.f64, r, j, true, 's', BU, 'l', BD, 'r', true); };
    bra.out_phys = "Uu";  // E[b] sites [e][bra][ket][e']
    bra.stage = STAGE_ENV_BRA;
    bra.row = b;
    bra.rev = true;
    bra.out = &Eb;
    bra.logscale = dlog;
    TNS_TRY(zip(cx, bra));
  }
  // <psi|psi> = exp(sum of scales) * prod of the (1x1x1x1) sites of E[0]
  std::vector<double> h(2 * W);
  for (int c = 0; c < W; ++c) {
    if (cx.f64) {
      TNS_TRY_CUDA(cudaMemcpyAsync(&h[2 * c], ec.E[0].site[c], sizeof(cd), cudaMemcpyDeviceToHost, cx.st));
    } else {
      float tmp[2];
      TNS_TRY_CUDA(cudaMemcpyAsync(tmp, ec.E[0].site[c], sizeof(cf), cudaMemcpyDeviceToHost, cx.st));
      TNS_TRY_CUDA(cudaStreamSynchronize(cx.st));
      h[2 * c] = tmp[0];
      h[2 * c + 1] = tmp[1];
    }
  }
  double lg = 0.0;
  TNS_TRY_CUDA(cudaMemcpyAsync(&lg, dlog, sizeof(double), cudaMemcpyDeviceToHost, cx.st));
  TNS_TRY_CUDA(cudaStreamSynchronize(cx.st));
  double zr = 1.0, zi = 0.0;
  for (int c = 0; c < W; ++c) {
    double a = h[2 * c], bb = h[2 * c + 1];
    double nr = zr * a - zi * bb, ni = zr * bb + zi * a;
    zr = nr;
    zi = ni;
  }
  ec.log_norm = lg + 0.5 * std::log(zr * zr + zi * zi);
  ec.valid = true;
  s->env_builds++;
  ec.chi_b = cx.R;
  ec.prec = prec;
  ec.version = s->version;
  ec.p = cx.p;
  ec.q = cx.q;
  return TNS_OK;
}

static tns_status make_ctx(tns_state* s, int chi_b, uint64_t seed, Ctx& cx) {
  cx.s = s;
  cx.st = s->st;
  cx.f64 = (s->prec == TNS_PREC_FP64);
  cx.gp = cx.f64 ? Prec::F64 : (s->tensor_cores ? Prec::TF32X3 : Prec::F32);
  cx.esz = cx.f64 ? sizeof(cd) : sizeof(cf);
  cx.seed = seed;
  cx.R = chi_b;
  cx.p = s->rf_p;
  cx.q = s->rf_q;
  return ensure_work_cells(s, cx.f64);
}

// Reads and clears the tensor-core timeout flag (stream already synchronised).
static tns_status check_tc_error(const Ctx& cx) {
  if (cx.gp != Prec::TF32X3) return TNS_OK;
  int* f = tc_error_flag();
  if (!f) return TNS_OK;
  int h = 0;
  TNS_TRY_CUDA(cudaMemcpy(&h, f, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return TNS_OK;
  TNS_TRY_CUDA(cudaMemset(f, 0, sizeof(int)));
  set_error("tensor-core GEMM pipeline wait timed out");
  return TNS_ERR_NUMERIC;
}

tns_status log_norm(tns_state* s, int chi_b, double* out) {
  Ctx cx;
  TNS_TRY(make_ctx(s, chi_b, 0, cx));
  TNS_TRY(build_envs(cx));
  TNS_TRY_CUDA(cudaStreamSynchronize(cx.st));
  TNS_TRY(check_tc_error(cx));
  *out = s->env.log_norm;
  return TNS_OK;
}

// Largest physical/bond dimension of a row.
static long long row_chi(tns_state* s, int b) {
  long long chi = 1;
  for (int c = 0; c < s->W; ++c)
    for (int leg = 1; leg <= 4; ++leg) chi = std::max<long long>(chi, s->cell[s->cidx(b, c)].dim[leg]);
  return chi;
}

static long long env_rank(const StoredMPS& m) {
  long long r = 1;
  for (auto x : m.bond) r = std::max(r, x);
  return r;
}

// Per-sample device bytes of the sampler working set (used to pick the chunk).
static long long sampler_bytes_per_sample(tns_state* s, const Ctx& cx) {
  long long R = cx.R, chi = 1, rho = 1;
  for (int b = 0; b < s->H; ++b) chi = std::max(chi, row_chi(s, b));
  for (auto& E : s->env.E) rho = std::max(rho, env_rank(E));
  long long kk = R + cx.p;
  long long big = R * 2 * R * chi * rho;                 // marginal intermediates
  long long Tm = R * 2 * chi * R * chi;                  // zip matrix
  long long site = R * 2 * chi * R;                      // K' site
  long long per = 2 * big + Tm + 2 * R * 2 * chi * kk + 2 * R * chi * kk + s->W * site * 2 + s->W * R * rho * R +
                  3 * R * rho * R + 2 * R * chi * R * s->W + R * 4096 * 2 + R * chi * chi * R;
  if (cx.gp == Prec::TF32X3) per += 2 * Tm;            // tensor-core operand packing
  return per * (long long)cx.esz + 64 * kk * kk * 16;
}

tns_status sample(tns_state* s, int chi_b, long long n, uint64_t seed, const uint8_t* forced, uint8_t* bits,
                  double* logq, double* cond, long long first) {
  if (n == 0) return TNS_OK;
  Ctx cx;
  TNS_TRY(make_ctx(s, chi_b, seed, cx));
  TNS_TRY(build_envs(cx));
  const int H = s->H, W = s->W;
  TNS_TRY_CUDA(cudaMemsetAsync(logq, 0, sizeof(double) * n, cx.st));
  // chunk size from free memory
  size_t fr = 0, tot = 0;
  TNS_TRY_CUDA(cudaMemGetInfo(&fr, &tot));
  long long per = sampler_bytes_per_sample(s, cx);
  long long chunk = std::max<long long>(1, std::min<long long>(n, (long long)(0.45 * (double)fr) / per));
  chunk = std::min<long long>(chunk, 4096);
  const long long R = cx.R;
  long long chimax = 1, rhomax = 1;
  for (int b = 0; b < H; ++b) chimax = std::max(chimax, row_chi(s, b));
  for (auto& E : s->env.E) rhomax = std::max(rhomax, env_rank(E));
  const long long site_cap = R * 2 * chimax * R;         // K' site per sample
  const long long msite_cap = R * chimax * R;            // projected m site per sample
  const long long F_cap = R * rhomax * R;
  const long long big_cap = R * 2 * R * chimax * rhomax;
  // persistent per-chunk buffers
  std::vector<void*> Ksite(W), Fs(W + 1), mA(W), mB(W);
  void *L0, *L1, *Gb, *bigA, *bigB, *ones;
  for (int j = 0; j < W; ++j) {
    char nm[32];
    snprintf(nm, sizeof nm, "s_K%d", j);
    TNS_TRY(wsget(s, nm, cx.esz * chunk * site_cap, &Ksite[j]));
    snprintf(nm, sizeof nm, "s_F%d", j);
    TNS_TRY(wsget(s, nm, cx.esz * chunk * F_cap, &Fs[j]));
    snprintf(nm, sizeof nm, "s_mA%d", j);
    TNS_TRY(wsget(s, nm, cx.esz * chunk * msite_cap, &mA[j]));
    snprintf(nm, sizeof nm, "s_mB%d", j);
    TNS_TRY(wsget(s, nm, cx.esz * chunk * msite_cap, &mB[j]));
  }
  TNS_TRY(wsget(s, "s_ones", cx.esz * chunk, &ones));
  Fs[W] = ones;
  TNS_TRY(wsget(s, "s_L0", cx.esz * chunk * F_cap, &L0));
  TNS_TRY(wsget(s, "s_L1", cx.esz * chunk * F_cap, &L1));
  TNS_TRY(wsget(s, "s_G", cx.esz * chunk * 2 * F_cap, &Gb));
  TNS_TRY(wsget(s, "s_bigA", cx.esz * chunk * big_cap, &bigA));
  TNS_TRY(wsget(s, "s_bigB", cx.esz * chunk * big_cap, &bigB));
  double* mpart;
  TNS_TRY(wsget(s, "s_mpart", sizeof(double) * 2 * MARG_SPLIT * chunk, (void**)&mpart));
  dispatch(cx.f64, [&](auto* tp) {
    using C = std::remove_pointer_t<decltype(tp)>;
    fill_kernel<C><<<nblk(chunk), 256, 0, cx.st>>>((C*)ones, chunk, 1.0);
  });
  s->launches++;

  // The per-chunk launch sequence: everything in it depends on the state, the
  // settings and the chunk size S only; the call's seed, first sample and output
  // buffers come from the device block `dcall`.
  SampleCall* dcall;
  TNS_TRY(wsget(s, "s_call", sizeof(SampleCall), (void**)&dcall));
  cx.seed_dev = &dcall->seed;
  auto run_chunk = [&](long long S) -> tns_status {
    // m_0: trivial, shared by all samples
    StoredMPS mcur;
    mcur.reversed = false;
    mcur.bond.assign(W + 1, 1);
    mcur.phys.assign(W, {1});
    mcur.site.assign(W, ones);
    bool mshared = true;
    StoredMPS mnext;
    for (int b = 0; b < H; ++b) {
      const bool rev = (b % 2 == 1);
      const bool shared = mshared;            // the row's zip is the same for every sample
      const long long Sz = shared ? 1 : S;
      StoredMPS Kp;
      Kp.site = Ksite;
      ZipSpec zs;
      zs.S = Sz;
      zs.mview = [&, rev, Sz](int j) {
        long long mst = mshared ? 0 : mps_site_size(mcur, W, j, rev);
        return mps_view(mcur, W, j, rev, 'a', "u", 'b', Sz, mst);
      };
      zs.wview = [&, b, rev](int j) { return cell_view(s, cx.f64, b, j, rev, 's', 'u', 'l', 'd', 'r'); };
      zs.out_phys = "sd";
      zs.stage = STAGE_SAMPLE;
      zs.row = b;
      zs.rev = rev;
      zs.out = &Kp;
      zs.logscale = nullptr;
      TNS_TRY(zip(cx, zs));
      const StoredMPS& E = s->env.E[b + 1];
      auto Eview = [&](int j) { return mps_view(E, W, j, rev, 'e', "Dd", 'f', 0, 0); };
      auto Kview = [&](int j, char la, char ls, char ld, char lb, long long SS, bool conj) {
        // K' site j stored [S][k][s][d][k'] in this row's logical order
        std::string lab = {'S', la, ls, ld, lb};
        long long sz = Kp.bond[j] * Kp.phys[j][0] * Kp.phys[j][1] * Kp.bond[j + 1];
        TView v = view(Kp.site[j], lab, {SS, Kp.bond[j], Kp.phys[j][0], Kp.phys[j][1], Kp.bond[j + 1]}, conj);
        v.stride[0] = shared ? 0 : sz;
        v.dim[0] = SS;
        return v;
      };
      // right environments F_j, j = W-1..1 (batch Sz)
      std::vector<long long> fdim(W + 1, 1);
      for (int j = W - 1; j >= 1; --j) {
        const long long ka = Kp.bond[j], P = Kp.phys[j][0], Dd = Kp.phys[j][1], kb = Kp.bond[j + 1];
        TView Ev = Eview(j);
        const long long re = vdim(Ev, 'e'), rf = vdim(Ev, 'f');
        // R1: T1[S][a][s][B][d][f] = sum_A K'[a,s,d,A] F_{j+1}[A,f,B]
        TView Fv = view(Fs[j + 1], "SAfB", {Sz, kb, rf, kb});
        if (j + 1 == W) Fv.stride[0] = 0;
        TNS_TRY_CUDA(pcontract(s, PC_SWEEP, Kview(j, 'a', 's', 'd', 'A', Sz, false), Fv,
                              view(bigA, "SasBdf", {Sz, ka, P, kb, Dd, rf}), cx.gp));
        // R2: T2[S][a][e][s][B][D] = sum_{d,f} T1 E[e,d,D,f]  (rows (a,e) of T2 are the next step's K-contiguous rows)
        TNS_TRY_CUDA(pcontract(s, PC_ENV, view(bigA, "SasBdf", {Sz, ka, P, kb, Dd, rf}), Ev,
                               view(bigB, "SaesBD", {Sz, ka, re, P, kb, Dd}), cx.gp));
        // R3: F_j[S][a][e][c] = sum_{s,B,D} T2 conj K'[c,s,D,B]
        TNS_TRY_CUDA(pcontract(s, PC_SWEEP, view(bigB, "SaesBD", {Sz, ka, re, P, kb, Dd}), Kview(j, 'c', 's', 'D', 'B', Sz, true),
                              view(Fs[j], "Saec", {Sz, ka, re, ka}), cx.gp));
        double* nrm_part = nullptr;
        TNS_TRY(wsget(s, "z_nrm", sizeof(double) * Sz * NRM_SPLIT, (void**)&nrm_part));
        dispatch(cx.f64, [&](auto* tp) {
          using C = std::remove_pointer_t<decltype(tp)>;
          const dim3 g(NRM_SPLIT, (unsigned)Sz);
          norm_partial_kernel<C><<<g, 256, 0, cx.st>>>((const C*)Fs[j], ka * re * ka, nrm_part);
          normalize_apply_kernel<C><<<g, 256, 0, cx.st>>>((C*)Fs[j], ka * re * ka, nrm_part);
        });
        s->launches += 2;
        fdim[j] = re;
      }
      // left sweep: draw the row's qubits
      mnext.reversed = rev;
      mnext.bond = Kp.bond;
      mnext.phys.assign(W, {});
      mnext.site = (mcur.site[0] == mA[0]) ? mB : mA;
      dispatch(cx.f64, [&](auto* tp) {
        using C = std::remove_pointer_t<decltype(tp)>;
        fill_kernel<C><<<nblk(S), 256, 0, cx.st>>>((C*)L0, S, 1.0);
      });
      s->launches++;
      void* Lc = L0;
      void* Ln = L1;
      for (int j = 0; j < W; ++j) {
        const long long ka = Kp.bond[j], P = Kp.phys[j][0], Dd = Kp.phys[j][1], kb = Kp.bond[j + 1];
        TView Ev = Eview(j);
        const long long re = vdim(Ev, 'e'), rf = vdim(Ev, 'f');
        // L1: U1[S][c][s][A][e][d] = sum_a L[a,e,c] K'[a,s,d,A]
        TNS_TRY_CUDA(pcontract(s, PC_SWEEP, view(Lc, "Saec", {S, ka, re, ka}), Kview(j, 'a', 's', 'd', 'A', S, false),
                              view(bigA, "ScsAed", {S, ka, P, kb, re, Dd}), cx.gp));
        // L2: U2[S][s][A][f][c][D] = sum_{e,d} U1 E[e,d,D,f]  (rows (A,f) of U2 are the next step's K-contiguous rows)
        TNS_TRY_CUDA(pcontract(s, PC_ENV, view(bigA, "ScsAed", {S, ka, P, kb, re, Dd}), Ev,
                               view(bigB, "SsAfcD", {S, P, kb, rf, ka, Dd}), cx.gp));
        // L3: G[S][s][A][f][B] = sum_{c,D} U2 conj K'[c,s,D,B]
        TNS_TRY_CUDA(pcontract(s, PC_SWEEP, view(bigB, "SsAfcD", {S, P, kb, rf, ka, Dd}), Kview(j, 'c', 's', 'D', 'B', S, true),
                              view(Gb, "SsAfB", {S, P, kb, rf, kb}), cx.gp));
        const int c = rev ? W - 1 - j : j;
        const int q = s->cell[s->cidx(b, c)].qubit;
        const long long nel = kb * rf * kb;
        const long long fst = (j + 1 == W || shared) ? 0 : kb * rf * kb;
        const long long kst = shared ? 0 : ka * P * Dd * kb;
        cudaEvent_t mev = s->prof.begin(cx.st);
        dispatch(cx.f64, [&](auto* tp) {
          using C = std::remove_pointer_t<decltype(tp)>;
          const dim3 grid(MARG_SPLIT, (unsigned)S);
          marginal_partial_kernel<C><<<grid, 256, 0, cx.st>>>((const C*)Gb, (int)P, nel, (const C*)Fs[j + 1], fst,
                                                              mpart);
          marginal_draw_kernel<C><<<grid, 256, 0, cx.st>>>(
              mpart, (const C*)Gb, (int)P, nel, (const C*)Kp.site[j], kst, (int)ka, (int)Dd, (int)kb, (C*)Ln,
              (C*)mnext.site[j], dcall, s->n, q < 0 ? 0 : q);
        });
        s->launches++;
        s->prof.end(PC_MARG, mev, 0.0, cx.st);
        s->launches++;
        mnext.phys[j] = {Dd};
        std::swap(Lc, Ln);
      }
      mcur = mnext;
      mshared = false;
    }
    return TNS_OK;
  };
  for (long long s0 = 0; s0 < n; s0 += chunk) {
    const long long S = std::min(chunk, n - s0);
    SampleCall hc{seed, s0, first, bits, forced, logq, cond};
    static_assert(sizeof(SampleCall) <= sizeof(s->host_call), "call block staging");
    memcpy(s->host_call, &hc, sizeof hc);
    TNS_TRY_CUDA(cudaMemcpyAsync(dcall, s->host_call, sizeof hc, cudaMemcpyHostToDevice, cx.st));
    if (!s->use_graphs || s->prof.on) {
      TNS_TRY(run_chunk(S));
      continue;
    }
    // everything the launch sequence depends on (buffer addresses included, through the
    // generation counters of the workspace, environments and working copies)
    const std::vector<long long> key = {s->version, R, S, cx.f64 ? 1 : 0, (long long)cx.gp, cx.p, cx.q,
                                        s->tensor_cores ? 1 : 0, s->ws.gen, s->env_builds, s->work_gen};
    auto it = s->graphs.find(key);
    if (it == s->graphs.end() && !s->graph_seen.count(key)) {   // first time: run eagerly (sizes every buffer)
      s->graph_seen.insert(key);
      TNS_TRY(run_chunk(S));
      continue;
    }
    // Graphs are captured and replayed on a private stream (the caller's may be the legacy
    // default stream, which cannot be captured), ordered after and before the caller's
    // stream by events.
    if (!s->gstream) {
      TNS_TRY_CUDA(cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
      for (auto& e : s->gev) TNS_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    cudaStream_t caller = s->st;
    TNS_TRY_CUDA(cudaEventRecord(s->gev[0], caller));
    TNS_TRY_CUDA(cudaStreamWaitEvent(s->gstream, s->gev[0], 0));
    if (it == s->graphs.end()) {
      const long long l0 = s->launches, c0 = contract_launches();
      s->st = cx.st = s->gstream;
      cudaError_t eb = cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeThreadLocal);
      tns_status rs = eb == cudaSuccess ? run_chunk(S) : TNS_OK;
      cudaGraph_t g = nullptr;
      cudaError_t ec = eb == cudaSuccess ? cudaStreamEndCapture(s->gstream, &g) : eb;
      s->st = cx.st = caller;
      if (rs != TNS_OK) {
        if (g) cudaGraphDestroy(g);
        return rs;
      }
      TNS_TRY_CUDA(ec);
      // kernels recorded during capture were counted but not launched (the contraction
      // layer's count reaches s->launches when the API call returns); the graph's
      // launches are counted on every replay instead
      tns_state::GraphEntry en;
      const long long cdelta = contract_launches() - c0;
      en.launches = (s->launches - l0) + cdelta;
      s->launches = l0 - cdelta;
      ec = cudaGraphInstantiate(&en.exec, g, 0);
      cudaGraphDestroy(g);
      TNS_TRY_CUDA(ec);
      if (s->ws.gen != key[8]) {                   // a buffer moved during capture: do not keep it
        cudaGraphExecDestroy(en.exec);
        set_error("workspace changed while capturing the sampler's launch sequence");
        return TNS_ERR_STATE;
      }
      it = s->graphs.emplace(key, en).first;
    }
    TNS_TRY_CUDA(cudaGraphLaunch(it->second.exec, s->gstream));
    s->launches += it->second.launches;
    TNS_TRY_CUDA(cudaEventRecord(s->gev[1], s->gstream));
    TNS_TRY_CUDA(cudaStreamWaitEvent(caller, s->gev[1], 0));
  }
  TNS_TRY_CUDA(cudaStreamSynchronize(cx.st));
  s->prof.resolve();
  return check_tc_error(cx);
}

tns_status amplitude(tns_state* s, int chi_b, long long n, const uint8_t* bits, double* log_abs, double* phase) {
  if (n == 0) return TNS_OK;
  Ctx cx;
  TNS_TRY(make_ctx(s, chi_b, 0, cx));
  const int H = s->H, W = s->W;
  const long long R = cx.R;
  long long chimax = 1;
  for (int b = 0; b < H; ++b) chimax = std::max(chimax, row_chi(s, b));
  size_t fr = 0, tot = 0;
  TNS_TRY_CUDA(cudaMemGetInfo(&fr, &tot));
  long long per = (R * chimax * R * W * 2 + R * chimax * R * chimax * 2 + R * 8 * R * chimax * 6) * (long long)cx.esz;
  long long chunk = std::max<long long>(1, std::min<long long>(n, (long long)(0.4 * (double)fr) / std::max(per, 1LL)));
  chunk = std::min<long long>(chunk, 16384);
  const long long msite_cap = R * chimax * R;
  std::vector<void*> mA(W), mB(W);
  void* ones;
  for (int j = 0; j < W; ++j) {
    char nm[32];
    snprintf(nm, sizeof nm, "a_mA%d", j);
    TNS_TRY(wsget(s, nm, cx.esz * chunk * msite_cap, &mA[j]));
    snprintf(nm, sizeof nm, "a_mB%d", j);
    TNS_TRY(wsget(s, nm, cx.esz * chunk * msite_cap, &mB[j]));
  }
  TNS_TRY(wsget(s, "a_ones", cx.esz * chunk, &ones));
  dispatch(cx.f64, [&](auto* tp) {
    using C = std::remove_pointer_t<decltype(tp)>;
    fill_kernel<C><<<nblk(chunk), 256, 0, cx.st>>>((C*)ones, chunk, 1.0);
  });
  void** dsites;
  TNS_TRY(wsget(s, "a_sites", sizeof(void*) * W, (void**)&dsites));
  for (long long s0 = 0; s0 < n; s0 += chunk) {
    const long long S = std::min(chunk, n - s0);
    double* la = log_abs + s0;
    TNS_TRY_CUDA(cudaMemsetAsync(la, 0, sizeof(double) * S, cx.st));
    StoredMPS mcur;
    mcur.reversed = false;
    mcur.bond.assign(W + 1, 1);
    mcur.phys.assign(W, {1});
    mcur.site.assign(W, ones);
    bool first = true;
    StoredMPS out;
    for (int b = 0; b < H; ++b) {
      const bool rev = (b % 2 == 1);
      out.site = (mcur.site[0] == mA[0]) ? mB : mA;
      ZipSpec zs;
      zs.S = S;
      zs.mview = [&, rev, first](int j) {
        // per-sample stride of the stored MPS site (0 for the shared trivial row)
        long long st = first ? 0 : mps_site_size(mcur, W, j, rev);
        return mps_view(mcur, W, j, rev, 'a', "u", 'b', S, st);
      };
      zs.wview = [&, b, rev](int j) {
        // psi[x_q] projected per sample: the physical axis is replaced by an index offset
        TView v = cell_view(s, cx.f64, b, j, rev, 's', 'u', 'l', 'd', 'r');
        int c = rev ? W - 1 - j : j;
        int q = s->cell[s->cidx(b, c)].qubit;
        long long sstride = v.stride[0];
        v.labels.erase(v.labels.begin());
        v.dim.erase(v.dim.begin());
        v.stride.erase(v.stride.begin());
        v.labels.insert(v.labels.begin(), 'S');
        v.dim.insert(v.dim.begin(), S);
        v.stride.insert(v.stride.begin(), 0);
        if (q >= 0) {
          v.idx = bits + s0 * s->n + q;
          v.idx_ld = s->n;
          v.idx_stride = sstride;
          v.idx_label = 'S';
        }
        return v;
      };
      zs.out_phys = "d";
      zs.stage = STAGE_AMPLITUDE;
      zs.row = b;
      zs.rev = rev;
      zs.out = &out;
      zs.logscale = la;
      TNS_TRY(zip(cx, zs));
      for (int j = 0; j < W; ++j)
        if (out.bond[j] * out.phys[j][0] * out.bond[j + 1] > msite_cap) { set_error("amplitude: site capacity"); return TNS_ERR_STATE; }
      mcur = out;
      first = false;
    }
    TNS_TRY_CUDA(cudaMemcpyAsync(dsites, mcur.site.data(), sizeof(void*) * W, cudaMemcpyHostToDevice, cx.st));
    dispatch(cx.f64, [&](auto* tp) {
      using C = std::remove_pointer_t<decltype(tp)>;
      amp_final_kernel<C><<<nblk(S), 256, 0, cx.st>>>((const C* const*)dsites, W, S, la, phase + s0);
    });
    s->launches++;
  }
  TNS_TRY_CUDA(cudaStreamSynchronize(cx.st));
  return check_tc_error(cx);
}

// ------------------------------------------------------- direct marginals
// Single-block reductions used between the row-contraction steps (vectors of at
// most a few million entries; one block keeps the summation order fixed).
template <typename C> __global__ void __launch_bounds__(1024) vec_normalize_kernel(C* v, long long n, double* nrm_out) {
  __shared__ double red[1024];
  double s2 = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s2 += cabs2(to_cd(v[i]));
  red[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double nrm = sqrt(red[0]);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) v[i] = from_cd<C>(cscale(to_cd(v[i]), inv));
  if (threadIdx.x == 0) *nrm_out = nrm;
}

// out = sum_i a[i] b[i] (no conjugation: a full tensor contraction), as (re, im).
template <typename C>
__global__ void __launch_bounds__(1024) vec_dot_kernel(const C* a, const C* b, long long n, double* out) {
  __shared__ double rr[1024], ri[1024];
  double sr = 0.0, si = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const cd x = cmul(to_cd(a[i]), to_cd(b[i]));
    sr += x.x;
    si += x.y;
  }
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { rr[threadIdx.x] += rr[threadIdx.x + o]; ri[threadIdx.x] += ri[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = rr[0]; out[1] = ri[0]; }
}

namespace {
// One row of the norm network <psi|psi> between its top environment U (sites
// [e][bra][ket][e']) and bottom environment D (sites [f][bra][ket][f']), contracted
// site by site.  Vectors carry the four bonds cut between two columns:
// [top env][ket horizontal][bra horizontal][bottom env].
struct RowNet {
  tns_state* s;
  Ctx* cx;
  int b;                          // grid row
  const StoredMPS* U;             // top environment of row b (flipped-frame storage)
  const StoredMPS* D;             // bottom environment E[b+1]
  void *X1, *X2, *X3;             // intermediates

  // ket (and, with proj, its bra) view of column c; proj = physical index fixed to 1
  TView ket(int c, char ls, char lu, char ll, char ld, char lr, bool conj, bool proj) const {
    TView v = cell_view(s, cx->f64, b, c, false, ls, lu, ll, ld, lr, conj);
    if (proj && v.dim[0] == 2) {
      v.ptr = (char*)v.ptr + cx->esz * v.stride[0];
      v.dim[0] = 1;
    }
    return v;
  }
  long long bond(const StoredMPS& m, int c, bool right) const {
    const int i = m.reversed ? s->W - 1 - c : c;
    return m.bond[right ? (m.reversed ? i : i + 1) : (m.reversed ? i + 1 : i)];
  }
  // out[E][r][R][F] = sum in[e][l][L][f] U[e][B][u][E] psi[s][u][l][d][r] conj psi[s][B][L][Dd][R] D[f][Dd][d][F]
  tns_status grow_left(int c, const void* in, void* out, bool proj) {
    const Cell& cl = s->cell[s->cidx(b, c)];
    const long long e = bond(*U, c, false), E = bond(*U, c, true), f = bond(*D, c, false), F = bond(*D, c, true);
    const long long l = cl.dim[LEG_L], r = cl.dim[LEG_R], u = cl.dim[LEG_U], d = cl.dim[LEG_D];
    const long long sp = (proj && cl.dim[0] == 2) ? 1 : cl.dim[0];
    TView Uv = mps_view(*U, s->W, c, false, 'e', "Bu", 'E', 0, 0);
    TView Dv = mps_view(*D, s->W, c, false, 'f', "Yd", 'F', 0, 0);
    TNS_TRY_CUDA(pcontract(s, PC_ENV, view(const_cast<void*>(in), "elLf", {e, l, l, f}), Uv,
                           view(X1, "lLfBuE", {l, l, f, u, u, E}), cx->gp));
    TNS_TRY_CUDA(pcontract(s, PC_ENV, view(X1, "lLfBuE", {l, l, f, u, u, E}), ket(c, 's', 'u', 'l', 'd', 'r', false, proj),
                           view(X2, "LfBEsdr", {l, f, u, E, sp, d, r}), cx->gp));
    TNS_TRY_CUDA(pcontract(s, PC_ENV, view(X2, "LfBEsdr", {l, f, u, E, sp, d, r}),
                           ket(c, 's', 'B', 'L', 'Y', 'R', true, proj), view(X3, "fEdrYR", {f, E, d, r, d, r}), cx->gp));
    TNS_TRY_CUDA(pcontract(s, PC_ENV, view(X3, "fEdrYR", {f, E, d, r, d, r}), Dv, view(out, "ErRF", {E, r, r, F}),
                           cx->gp));
    return TNS_OK;
  }
  // out[e][l][L][f] = sum U[e][B][u][E] psi[s][u][l][d][r] conj psi[s][B][L][Dd][R] D[f][Dd][d][F] in[E][r][R][F]
  tns_status grow_right(int c, const void* in, void* out) {
    const Cell& cl = s->cell[s->cidx(b, c)];
    const long long e = bond(*U, c, false), E = bond(*U, c, true), f = bond(*D, c, false), F = bond(*D, c, true);
    const long long l = cl.dim[LEG_L], r = cl.dim[LEG_R], u = cl.dim[LEG_U], d = cl.dim[LEG_D], sp = cl.dim[0];
    TView Uv = mps_view(*U, s->W, c, false, 'e', "Bu", 'E', 0, 0);
    TView Dv = mps_view(*D, s->W, c, false, 'f', "Yd", 'F', 0, 0);
    TNS_TRY_CUDA(pcontract(s, PC_ENV, Uv, view(const_cast<void*>(in), "ErRF", {E, r, r, F}),
                           view(X1, "eBurRF", {e, u, u, r, r, F}), cx->gp));
    TNS_TRY_CUDA(pcontract(s, PC_ENV, view(X1, "eBurRF", {e, u, u, r, r, F}), ket(c, 's', 'u', 'l', 'd', 'r', false, false),
                           view(X2, "eBRFsld", {e, u, r, F, sp, l, d}), cx->gp));
    TNS_TRY_CUDA(pcontract(s, PC_ENV, view(X2, "eBRFsld", {e, u, r, F, sp, l, d}),
                           ket(c, 's', 'B', 'L', 'Y', 'R', true, false), view(X3, "eFldLY", {e, F, l, d, l, d}), cx->gp));
    TNS_TRY_CUDA(pcontract(s, PC_ENV, view(X3, "eFldLY", {e, F, l, d, l, d}), Dv, view(out, "elLf", {e, l, l, f}),
                           cx->gp));
    return TNS_OK;
  }
};
}  // namespace

// Sample-free marginals <n_q> for every qubit and <n_q n_q'> for every pair in the
// same grid row (Methods, expectation values from the boundary-MPS contraction of
// <psi|psi>): row b is contracted exactly between its top and bottom environments
// at rank chi_b, from the left and from the right, with P1 = |1><1| (the physical
// index fixed to 1 in ket and bra) on the marginal's qubits.  Every partial vector
// is stored at unit norm and its scale kept as a log on the host, so no contraction
// over- or underflows.  one: host [n]; two: host [n][n] or NULL (NaN off the rows).
tns_status direct_marginals(tns_state* s, int chi_b, double* one, double* two) {
  Ctx cx;
  TNS_TRY(make_ctx(s, chi_b, 0, cx));
  TNS_TRY(build_envs(cx, false));
  TNS_TRY(build_envs(cx, true));
  const int H = s->H, W = s->W;
  for (int q = 0; q < s->n; ++q) one[q] = NAN;
  if (two)
    for (long long i = 0; i < (long long)s->n * s->n; ++i) two[i] = NAN;
  // workspace: vectors (R * chi * chi * R) and the three intermediates
  long long chi = 1, rho = 1;
  for (auto& c : s->cell)
    for (int leg = 1; leg <= 4; ++leg) chi = std::max<long long>(chi, c.dim[leg]);
  for (auto* ec : {&s->env, &s->env_top})
    for (auto& E : ec->E) rho = std::max(rho, env_rank(E));
  const long long vcap = rho * chi * chi * rho, xcap = 2 * rho * chi * chi * chi * chi * rho;
  RowNet net;
  net.s = s;
  net.cx = &cx;
  TNS_TRY(wsget(s, "dm_X1", cx.esz * xcap, &net.X1));
  TNS_TRY(wsget(s, "dm_X2", cx.esz * xcap * chi, &net.X2));
  TNS_TRY(wsget(s, "dm_X3", cx.esz * xcap, &net.X3));
  std::vector<void*> left(W + 1), right(W + 1);
  for (int c = 0; c <= W; ++c) {
    char nm[32];
    snprintf(nm, sizeof nm, "dm_L%d", c);
    TNS_TRY(wsget(s, nm, cx.esz * vcap, &left[c]));
    snprintf(nm, sizeof nm, "dm_R%d", c);
    TNS_TRY(wsget(s, nm, cx.esz * vcap, &right[c]));
  }
  void *v0, *v1;
  TNS_TRY(wsget(s, "dm_v0", cx.esz * vcap, &v0));
  TNS_TRY(wsget(s, "dm_v1", cx.esz * vcap, &v1));
  double* dscal;
  TNS_TRY(wsget(s, "dm_scal", sizeof(double) * 2, (void**)&dscal));
  // vector element counts at the cut left of column c (c = W: the trivial right end)
  auto vlen = [&](const RowNet& rn, int c) -> long long {
    if (c == 0 || c == W) return 1;
    const Cell& cl = s->cell[s->cidx(rn.b, c)];
    return rn.bond(*rn.U, c, false) * cl.dim[LEG_L] * cl.dim[LEG_L] * rn.bond(*rn.D, c, false);
  };
  auto normalize = [&](void* v, long long n, double* log_scale) -> tns_status {
    dispatch(cx.f64, [&](auto* tp) {
      using C = std::remove_pointer_t<decltype(tp)>;
      vec_normalize_kernel<C><<<1, 1024, 0, cx.st>>>((C*)v, n, dscal);
    });
    s->launches++;
    double h = 0.0;
    TNS_TRY_CUDA(cudaMemcpyAsync(&h, dscal, sizeof(double), cudaMemcpyDeviceToHost, cx.st));
    TNS_TRY_CUDA(cudaStreamSynchronize(cx.st));
    *log_scale = h > 0.0 ? std::log(h) : -INFINITY;
    return TNS_OK;
  };
  auto dot = [&](const void* a, const void* bb, long long n, double* re) -> tns_status {
    dispatch(cx.f64, [&](auto* tp) {
      using C = std::remove_pointer_t<decltype(tp)>;
      vec_dot_kernel<C><<<1, 1024, 0, cx.st>>>((const C*)a, (const C*)bb, n, dscal);
    });
    s->launches++;
    double h[2];
    TNS_TRY_CUDA(cudaMemcpyAsync(h, dscal, sizeof(double) * 2, cudaMemcpyDeviceToHost, cx.st));
    TNS_TRY_CUDA(cudaStreamSynchronize(cx.st));
    *re = h[0];
    return TNS_OK;
  };
  for (int b = 0; b < H; ++b) {
    net.b = b;
    net.U = &s->env_top.E[H - b];
    net.D = &s->env.E[b + 1];
    std::vector<double> la(W + 1, 0.0), lb(W + 1, 0.0);
    dispatch(cx.f64, [&](auto* tp) {
      using C = std::remove_pointer_t<decltype(tp)>;
      fill_kernel<C><<<1, 32, 0, cx.st>>>((C*)left[0], 1, 1.0);
      fill_kernel<C><<<1, 32, 0, cx.st>>>((C*)right[W], 1, 1.0);
    });
    s->launches += 2;
    for (int c = 0; c < W; ++c) {
      TNS_TRY(net.grow_left(c, left[c], left[c + 1], false));
      double g;
      TNS_TRY(normalize(left[c + 1], vlen(net, c + 1), &g));
      la[c + 1] = la[c] + g;
    }
    for (int c = W - 1; c >= 0; --c) {
      TNS_TRY(net.grow_right(c, right[c + 1], right[c]));
      double g;
      TNS_TRY(normalize(right[c], vlen(net, c), &g));
      lb[c] = lb[c + 1] + g;
    }
    const double log_norm = la[W];            // left[W] = <psi|psi> of this row's network, at unit norm
    double zW;
    TNS_TRY(dot(left[W], right[W], 1, &zW));
    // <P> at columns (ci[, cj]) = e^{scales - log_norm} Re(v . right) / zW
    for (int ci = 0; ci < W; ++ci) {
      const int qi = s->cell[s->cidx(b, ci)].qubit;
      if (qi < 0) continue;
      TNS_TRY(net.grow_left(ci, left[ci], v0, true));
      double gv;
      TNS_TRY(normalize(v0, vlen(net, ci + 1), &gv));
      double lv = la[ci] + gv, val;
      TNS_TRY(dot(v0, right[ci + 1], vlen(net, ci + 1), &val));
      one[qi] = std::exp(lv + lb[ci + 1] - log_norm) * val / zW;
      if (!two) continue;
      two[(long long)qi * s->n + qi] = one[qi];
      void* vc = v0;
      void* vn = v1;
      for (int c = ci + 1; c < W; ++c) {
        const int q = s->cell[s->cidx(b, c)].qubit;
        if (q >= 0) {
          TNS_TRY(net.grow_left(c, vc, vn, true));
          double gp, vv;
          TNS_TRY(normalize(vn, vlen(net, c + 1), &gp));
          TNS_TRY(dot(vn, right[c + 1], vlen(net, c + 1), &vv));
          const double x = std::exp(lv + gp + lb[c + 1] - log_norm) * vv / zW;
          two[(long long)qi * s->n + q] = two[(long long)q * s->n + qi] = x;
        }
        if (c + 1 < W) {
          TNS_TRY(net.grow_left(c, vc, vn, false));
          double gi;
          TNS_TRY(normalize(vn, vlen(net, c + 1), &gi));
          lv += gi;
          std::swap(vc, vn);
        }
      }
    }
  }
  TNS_TRY_CUDA(cudaStreamSynchronize(cx.st));
  return check_tc_error(cx);
}

// ------------------------------------------------------- sample certification
// log p(x) = 2 log|<x|psi>| - log <psi|psi> at the certification rank; the ratio
// w = p / q and the per-sample log q - log p, reduced (one block, fixed order) to
// sum w, sum w^2, sum (log q - log p) and the number of samples with p > 0.
__global__ void __launch_bounds__(1024) certify_kernel(const double* log_abs, double log_norm, const double* logq,
                                                       long long n, double* logp, double* stats) {
  __shared__ double r0[1024], r1[1024], r2[1024], r3[1024];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double lp = 2.0 * log_abs[i] - log_norm;
    logp[i] = lp;
    if (isfinite(lp)) {
      const double w = exp(lp - logq[i]);
      s0 += w;
      s1 += w * w;
      s2 += logq[i] - lp;
      s3 += 1.0;
    }
  }
  r0[threadIdx.x] = s0; r1[threadIdx.x] = s1; r2[threadIdx.x] = s2; r3[threadIdx.x] = s3;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o]; r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o]; r3[threadIdx.x] += r3[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { stats[0] = r0[0]; stats[1] = r1[0]; stats[2] = r2[0]; stats[3] = r3[0]; }
}

tns_status certify(tns_state* s, int chi_b, long long n, const uint8_t* bits, const double* logq, double* logp,
                   double* stats_host) {
  double ln = 0.0;
  TNS_TRY(log_norm(s, chi_b, &ln));
  double *la, *ph, *st;
  TNS_TRY(wsget(s, "c_la", sizeof(double) * std::max<long long>(n, 1), (void**)&la));
  TNS_TRY(wsget(s, "c_ph", sizeof(double) * std::max<long long>(n, 1), (void**)&ph));
  TNS_TRY(wsget(s, "c_stats", sizeof(double) * 4, (void**)&st));
  TNS_TRY(amplitude(s, chi_b, n, bits, la, ph));
  certify_kernel<<<1, 1024, 0, s->st>>>(la, ln, logq, n, logp, st);
  s->launches++;
  TNS_TRY_CUDA(cudaGetLastError());
  double h[4];
  TNS_TRY_CUDA(cudaMemcpyAsync(h, st, sizeof h, cudaMemcpyDeviceToHost, s->st));
  TNS_TRY_CUDA(cudaStreamSynchronize(s->st));
  const double m = h[3] > 0 ? h[3] : 1.0;
  stats_host[0] = h[0] / m;                                                   // mean p/q
  stats_host[1] = h[3] > 1 ? std::sqrt(std::max(0.0, h[1] / m - stats_host[0] * stats_host[0]) / (m - 1)) : NAN;
  stats_host[2] = h[2] / m;                                                   // KLD estimate
  stats_host[3] = h[3];
  stats_host[4] = ln;
  return TNS_OK;
}
}  // namespace tns
