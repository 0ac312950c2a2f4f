// Batched FP64 Jacobi eigensolver and one-sided Jacobi SVD.  See linalg.cuh.
//
// Both use the round-robin ("chess tournament") ordering of index pairs, so the
// n/2 rotations of a round act on disjoint indices and run in parallel.  Every
// sweep loop is bounded (MAX_SWEEPS); a matrix that has not converged is
// returned as is with status 1, never spun on.
#include "linalg.cuh"

namespace tns {

static constexpr int JAC_THREADS = 256;
// The eigensolver applies up to n/2 independent rotations per round, one warp each:
// 32 warps keep the rotation phases short at the truncation sizes (n ~ 100).
static constexpr int EIG_THREADS = 1024;
static constexpr int MAX_SWEEPS = 40;
static constexpr size_t SMEM_LIMIT = 200 * 1024;
// Largest Cholesky order (the in-place inverse stages one column of n entries).
static constexpr int CHOL_MAX_N = 512;

bool jacobi_fits_smem(int m, int n) {
  size_t np = n + (n & 1);
  size_t need = ((size_t)m * np + np * np) * sizeof(cd) + 1024;
  return need <= SMEM_LIMIT;
}

__device__ inline void rr_pair(int r, int i, int np, int& p, int& q) {
  int k = i, l = np - 1 - i;
  p = (k == 0) ? 0 : 1 + (k - 1 + r) % (np - 1);
  q = (l == 0) ? 0 : 1 + (l - 1 + r) % (np - 1);
}

// Rotation J = [[c, s], [-s conj(e), c conj(e)]] on (p, q) that zeroes the (p, q)
// entry of J^H A J for the Hermitian 2x2 block [[app, apq], [conj(apq), aqq]]
// (phase-reduce to a real symmetric block, then the symmetric Schur rotation).
template <typename T, typename C>
__device__ inline void herm_rot(T app, T aqq, C apq, T& c, T& s, C& e) {
  const T tiny = sizeof(T) == 8 ? (T)1e-300 : (T)1e-37;
  T ab = sqrt(cabs2(apq));
  if (!(ab > tiny)) {
    c = 1; s = 0; e = mk((T)1, (T)0);
    return;
  }
  e = mk(apq.x / ab, apq.y / ab);
  T tau = (aqq - app) / (2 * ab);
  T t = (tau >= 0 ? (T)1 : (T)-1) / (fabs(tau) + hypot((T)1, tau));
  c = 1 / hypot((T)1, t);
  s = t * c;
}

template <typename T> __device__ inline T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Precision-dependent Jacobi thresholds: a pair is rotated while
// |a_pq| > REL * max(|a_pp|, |a_qq|) and |a_pq| > FLOOR * ||A||_F (a few units of
// rounding: rotating below that level cannot converge).
template <typename T> struct JacTol;
template <> struct JacTol<double> { static constexpr double REL = 1e-15, FLOOR = 1e-17; };
template <> struct JacTol<float> { static constexpr float REL = 3e-7f, FLOOR = 1e-9f; };

// T = double: the FP64 solver.  T = float: the same algorithm in FP32 (complex64
// input), eigenvalues and eigenvectors written widened to FP64 storage.
template <typename T>
__global__ void __launch_bounds__(EIG_THREADS)
eigh_kernel(const typename CplxOf<T>::type* Ain, long long sA, int lda, int n, double* lam, cd* Vout, long long sV,
            typename CplxOf<T>::type* work, int* status, int use_smem, int* sweeps_out) {
  typedef typename CplxOf<T>::type C;
  extern __shared__ double4 smraw4[];
  __shared__ T cs_c[256], cs_s[256], cs_d[256];
  __shared__ C cs_e[256];
  __shared__ int cs_p[256], cs_q[256];
  __shared__ T red[EIG_THREADS / 32];
  __shared__ T floor_s;
  __shared__ int nrot;
  const int b = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  const int np = n + (n & 1), half = np / 2;
  // row pitch: np + 1 in shared memory (odd, so the column phase's strided walks are
  // free of bank conflicts), np in global memory
  const int ld = use_smem ? np + 1 : np;
  C* a = use_smem ? reinterpret_cast<C*>(smraw4) : work + (long long)b * 2 * np * np;
  C* v = a + (long long)np * ld;
  const C* src = Ain + (long long)b * sA;
  T tot = 0;
  for (int idx = tid; idx < np * np; idx += blockDim.x) {
    int i = idx / np, j = idx % np;
    C x = (i < n && j < n) ? src[(long long)i * lda + j] : mk((T)0, (T)0);
    if (i == j) x.y = 0;            // Hermitian: real diagonal
    a[i * ld + j] = x;
    tot += cabs2(x);
    v[i * ld + j] = mk(i == j ? (T)1 : (T)0, (T)0);
  }
  tot = warp_sum(tot);
  if ((tid & 31) == 0) red[tid >> 5] = tot;
  __syncthreads();
  if (tid == 0) {
    T t = 0;
    for (int w = 0; w < EIG_THREADS / 32; ++w) t += red[w];
    floor_s = JacTol<T>::FLOOR * sqrt(t);     // absolute floor below which a pair counts as rotated
  }
  __syncthreads();
  bool conv = (np <= 1);
  int sweeps_done = 0;
  for (int sweep = 0; sweep < MAX_SWEEPS && !conv; ++sweep) {
    ++sweeps_done;
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int i = tid; i < half; i += blockDim.x) {
        int p, q;
        rr_pair(r, i, np, p, q);
        cs_p[i] = p;
        cs_q[i] = q;
        T app = a[p * ld + p].x, aqq = a[q * ld + q].x;
        C apq = a[p * ld + q];
        T ab = sqrt(cabs2(apq));
        T c = 1, s = 0, dl = 0;
        C e = mk((T)1, (T)0);
        // rounding leaves off-diagonal noise ~ eps * max(|app|, |aqq|): rotating below
        // that level cannot converge, and leaving it perturbs eigenvectors by ~eps
        if (ab > floor_s && ab > JacTol<T>::REL * fmax(fabs(app), fabs(aqq))) {
          herm_rot(app, aqq, apq, c, s, e);
          dl = (s / c) * ab;        // app' = app - t|apq|, aqq' = aqq + t|apq|
          atomicAdd(&nrot, 1);
        }
        cs_c[i] = c; cs_s[i] = s; cs_e[i] = e; cs_d[i] = dl;
      }
      __syncthreads();
      // one warp per rotation, lanes along the row / column (no index division)
      for (int i = warp; i < half; i += nwarp) {                       // rows: J^H A
        if (cs_s[i] == 0) continue;
        const int p = cs_p[i], q = cs_q[i];
        const T c = cs_c[i], s = cs_s[i];
        const C e = cs_e[i];
        for (int j = lane; j < np; j += 32) {
          C ap = a[p * ld + j], aq = a[q * ld + j];
          C eaq = cmul(e, aq);
          a[p * ld + j] = mk(c * ap.x - s * eaq.x, c * ap.y - s * eaq.y);
          a[q * ld + j] = mk(s * ap.x + c * eaq.x, s * ap.y + c * eaq.y);
        }
      }
      __syncthreads();
      for (int i = warp; i < half; i += nwarp) {                       // columns: (J^H A) J and V J
        if (cs_s[i] == 0) continue;
        const int p = cs_p[i], q = cs_q[i];
        const T c = cs_c[i], s = cs_s[i];
        const C ec = cconj(cs_e[i]);
        for (int j = lane; j < np; j += 32) {
          C ap = a[j * ld + p], aq = a[j * ld + q];
          C eaq = cmul(ec, aq);
          a[j * ld + p] = mk(c * ap.x - s * eaq.x, c * ap.y - s * eaq.y);
          a[j * ld + q] = mk(s * ap.x + c * eaq.x, s * ap.y + c * eaq.y);
          C vp = v[j * ld + p], vq = v[j * ld + q];
          C evq = cmul(ec, vq);
          v[j * ld + p] = mk(c * vp.x - s * evq.x, c * vp.y - s * evq.y);
          v[j * ld + q] = mk(s * vp.x + c * evq.x, s * vp.y + c * evq.y);
        }
      }
      __syncthreads();
      for (int i = tid; i < half; i += blockDim.x) {                   // exact 2x2 result
        if (cs_s[i] == 0) continue;
        const int p = cs_p[i], q = cs_q[i];
        a[p * ld + q] = mk((T)0, (T)0);
        a[q * ld + p] = mk((T)0, (T)0);
      }
      __syncthreads();
    }
    conv = (nrot == 0);
    __syncthreads();
  }
  if (tid == 0 && status) status[b] = conv ? 0 : 1;
  if (tid == 0 && sweeps_out) sweeps_out[b] = sweeps_done;
  for (int i = tid; i < n; i += blockDim.x) {
    T li = a[i * ld + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      T lj = a[j * ld + j].x;
      if (lj > li || (lj == li && j < i)) ++rank;
    }
    lam[(long long)b * n + rank] = (double)li;
    cd* vo = Vout + (long long)b * sV;
    for (int row = 0; row < n; ++row) vo[(long long)row * n + rank] = to_cd(v[row * ld + i]);
  }
}

__global__ void __launch_bounds__(JAC_THREADS)
svd_kernel(cd* Ain, long long sA, int lda, int m, int n, double* sigma, cd* Uout, long long sU, cd* Vout,
           long long sV, cd* work, int* status, int use_smem) {
  extern __shared__ double4 smraw4[];
  __shared__ double wred[JAC_THREADS / 32];
  __shared__ double sig[1024];
  __shared__ int flag;
  const int b = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nw = blockDim.x >> 5;
  const int np = n + (n & 1), half = np / 2;
  cd* a = use_smem ? reinterpret_cast<cd*>(smraw4) : work + (long long)b * ((long long)m * np + (long long)np * np);
  cd* v = a + (long long)m * np;
  const cd* src = Ain + (long long)b * sA;
  for (long long idx = tid; idx < (long long)m * np; idx += blockDim.x) {
    int i = (int)(idx / np), j = (int)(idx % np);
    a[idx] = (j < n) ? src[(long long)i * lda + j] : mk(0.0, 0.0);
  }
  for (int idx = tid; idx < np * np; idx += blockDim.x) v[idx] = mk((idx / np == idx % np) ? 1.0 : 0.0, 0.0);
  __shared__ double floor_s;
  {
    double t = 0.0;
    for (long long idx = tid; idx < (long long)m * np; idx += blockDim.x) t += cabs2(a[idx]);
    t = warp_sum(t);
    if (lane == 0) wred[warp] = t;
    __syncthreads();
    if (tid == 0) {
      double tt = 0.0;
      for (int w = 0; w < nw; ++w) tt += wred[w];
      floor_s = 1e-17 * tt;          // |gamma| scale is a squared column norm
    }
  }
  __syncthreads();
  const double tol = 1e-15 * sqrt((double)m);   // orthogonality threshold ~ sqrt(m) eps (LAPACK zgesvj style)
  bool conv = (np <= 1);
  for (int sweep = 0; sweep < MAX_SWEEPS && !conv; ++sweep) {
    double wmax = 0.0;
    for (int r = 0; r < np - 1; ++r) {
      for (int i = warp; i < half; i += nw) {
        int p, q;
        rr_pair(r, i, np, p, q);
        double al = 0.0, be = 0.0, gx = 0.0, gy = 0.0;
        for (int row = lane; row < m; row += 32) {
          cd x = a[(long long)row * np + p], y = a[(long long)row * np + q];
          al += cabs2(x);
          be += cabs2(y);
          gx += x.x * y.x + x.y * y.y;     // conj(x) * y
          gy += x.x * y.y - x.y * y.x;
        }
        al = warp_sum(al); be = warp_sum(be); gx = warp_sum(gx); gy = warp_sum(gy);
        double gab = sqrt(gx * gx + gy * gy);
        double den = sqrt(al * be);
        if (gab > floor_s && den > 0.0 && gab > tol * den) {
          wmax = fmax(wmax, gab / den);
          cd ec = mk(gx / gab, -gy / gab);        // conj(e)
          double tau = (be - al) / (2.0 * gab);
          double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
          double c = 1.0 / hypot(1.0, t), s = t * c;
          for (int row = lane; row < m; row += 32) {
            cd x = a[(long long)row * np + p], y = a[(long long)row * np + q];
            cd ey = cmul(ec, y);
            a[(long long)row * np + p] = mk(c * x.x - s * ey.x, c * x.y - s * ey.y);
            a[(long long)row * np + q] = mk(s * x.x + c * ey.x, s * x.y + c * ey.y);
          }
          for (int row = lane; row < np; row += 32) {
            cd x = v[row * np + p], y = v[row * np + q];
            cd ey = cmul(ec, y);
            v[row * np + p] = mk(c * x.x - s * ey.x, c * x.y - s * ey.y);
            v[row * np + q] = mk(s * x.x + c * ey.x, s * x.y + c * ey.y);
          }
        }
      }
      __syncthreads();
    }
    wmax = warp_max(wmax);
    if (lane == 0) wred[warp] = wmax;
    __syncthreads();
    if (tid == 0) {
      double mx = 0.0;
      for (int w = 0; w < nw; ++w) mx = fmax(mx, wred[w]);
      flag = (mx == 0.0) ? 1 : 0;
    }
    __syncthreads();
    conv = flag != 0;
  }
  if (tid == 0 && status) status[b] = conv ? 0 : 1;
  for (int i = warp; i < n; i += nw) {
    double s2 = 0.0;
    for (int row = lane; row < m; row += 32) s2 += cabs2(a[(long long)row * np + i]);
    s2 = warp_sum(s2);
    if (lane == 0) sig[i] = sqrt(s2);
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    double si = sig[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double sj = sig[j];
      if (sj > si || (sj == si && j < i)) ++rank;
    }
    sigma[(long long)b * n + rank] = si;
    double inv = si > 0.0 ? 1.0 / si : 0.0;
    cd* uo = Uout + (long long)b * sU;
    for (int row = 0; row < m; ++row) uo[(long long)row * n + rank] = cscale(a[(long long)row * np + i], inv);
    cd* vo = Vout + (long long)b * sV;
    for (int row = 0; row < n; ++row) vo[(long long)row * n + rank] = v[row * np + i];
  }
}

// W = L^{-H} with L L^H = G + shift * max_i G_ii * I (G Hermitian PSD, n x n).
// One block per matrix, the factor held in one n x n buffer with row pitch n + 1
// (an odd pitch keeps the column walks of both phases free of shared-memory bank
// conflicts): right-looking Cholesky, then the triangular inverse in place
// (columns from the last to the first: column j of L^{-1} is -L^{-1}[j+1:, j+1:]
// L[j+1:, j] / L[j, j], from the already inverted trailing block).  Used so that
// Y W has orthonormal columns when G = Y^H Y; the shift keeps it well defined for
// rank-deficient Y and damps directions below shift * max G_ii smoothly.
// use_smem: 1 = the buffer in shared memory, 0 = in work (n (n + 1) per matrix).
template <typename C, typename GIN, typename T>
__global__ void __launch_bounds__(JAC_THREADS)
chol_w_kernel(const GIN* Gin, int n, double shift, C* Wout, typename CplxOf<T>::type* work, int use_smem) {
  typedef typename CplxOf<T>::type CT;
  extern __shared__ double4 smraw4[];
  __shared__ T red[JAC_THREADS / 32];
  __shared__ T sh_s;
  __shared__ CT xs[CHOL_MAX_N];
  const int b = blockIdx.x, tid = threadIdx.x;
  const int ld = n + 1;
  CT* L = use_smem ? reinterpret_cast<CT*>(smraw4) : work + (long long)b * n * ld;
  const GIN* G = Gin + (long long)b * n * n;
  T mx = 0;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    int i = idx / n, j = idx % n;
    const GIN gi = G[idx];
    CT g = mk((T)gi.x, (T)gi.y);
    L[i * ld + j] = (j <= i) ? g : mk((T)0, (T)0);
    if (i == j) mx = fmax(mx, g.x);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    T m = 0;
    for (int w = 0; w < JAC_THREADS / 32; ++w) m = fmax(m, red[w]);
    sh_s = (T)shift * m;
  }
  __syncthreads();
  const T sft = sh_s;
  C* W = Wout + (long long)b * n * n;
  if (!(sft > 0)) {                // Y = 0: no directions
    for (int idx = tid; idx < n * n; idx += blockDim.x) W[idx] = from_cd<C>(mk(0.0, 0.0));
    return;
  }
  for (int i = tid; i < n; i += blockDim.x) L[i * ld + i].x += sft;
  __syncthreads();
  __shared__ int broke;
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      // Every pivot of G + sft I (G PSD) is >= sft in exact arithmetic.  A smaller
      // computed pivot means the Gram's rounding has made it indefinite in this
      // direction: the pivot is set to sqrt(sft) and the column decoupled from the
      // rest (zeroed below the diagonal), so the factor and its inverse stay bounded
      // by 1/sqrt(sft) instead of growing through the remaining columns.
      T d = L[j * ld + j].x;
      broke = !(d > sft);
      L[j * ld + j] = mk(sqrt(broke ? sft : d), (T)0);
    }
    __syncthreads();
    const T inv = 1 / L[j * ld + j].x;
    for (int i = j + 1 + tid; i < n; i += blockDim.x)
      L[i * ld + j] = broke ? mk((T)0, (T)0) : cscale(L[i * ld + j], inv);
    __syncthreads();
    const int m = n - j - 1;
    for (int idx = tid; idx < m * m; idx += blockDim.x) {        // trailing lower triangle
      int i = j + 1 + idx / m, k = j + 1 + idx % m;
      if (k > i) continue;
      L[i * ld + k] = csub(L[i * ld + k], cmul(L[i * ld + j], cconj(L[k * ld + j])));
    }
    __syncthreads();
  }
  // L <- L^{-1} in place, last column first
  for (int j = n - 1; j >= 0; --j) {
    const T d = 1 / L[j * ld + j].x;
    for (int i = j + 1 + tid; i < n; i += blockDim.x) xs[i] = L[i * ld + j];
    __syncthreads();
    for (int i = j + 1 + tid; i < n; i += blockDim.x) {
      CT acc = mk((T)0, (T)0);
      for (int k = j + 1; k <= i; ++k) acc = cadd(acc, cmul(L[i * ld + k], xs[k]));
      L[i * ld + j] = cscale(acc, -d);
    }
    if (tid == 0) L[j * ld + j] = mk(d, (T)0);
    __syncthreads();
  }
  for (int idx = tid; idx < n * n; idx += blockDim.x) {          // W = (L^{-1})^H
    int i = idx / n, j = idx % n;
    W[idx] = from_cd<C>(to_cd(j >= i ? cconj(L[j * ld + i]) : mk((T)0, (T)0)));
  }
}

cudaError_t chol_w_batched(const void* G, bool g_f64, int n, int batch, double shift, void* W, bool w_f64, void* work,
                           cudaStream_t st, bool fp32_factor) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  // Complex64 in and out (the mixed path's CholeskyQR passes): the factorisation and
  // the triangular inverse run in FP64 unless fp32_factor (passes where only the span
  // of the result matters).  In FP32 their rounding (~n eps_32 of the largest pivot)
  // reaches the shifts used at n ~ 100, which the pivot guard then absorbs.
  const bool c64 = !g_f64 && !w_f64;
  const bool f32 = c64 && fp32_factor;
  if (n > CHOL_MAX_N) return cudaErrorInvalidValue;
  const size_t esz = f32 ? sizeof(cf) : sizeof(cd);
  const size_t need = (size_t)n * (n + 1) * esz;
  const int use_smem = need <= SMEM_LIMIT ? 1 : 0;
  if (!use_smem && !work) return cudaErrorInvalidValue;
  const size_t sm = use_smem ? need : 0;
  cudaError_t ea = cudaSuccess;
  if (w_f64 && g_f64) ea = smem_optin((const void*)chol_w_kernel<cd, cd, double>, (int)SMEM_LIMIT);
  else if (g_f64) ea = smem_optin((const void*)chol_w_kernel<cf, cd, double>, (int)SMEM_LIMIT);
  else if (f32) ea = smem_optin((const void*)chol_w_kernel<cf, cf, float>, (int)SMEM_LIMIT);
  else if (c64) ea = smem_optin((const void*)chol_w_kernel<cf, cf, double>, (int)SMEM_LIMIT);
  if (ea != cudaSuccess) return ea;
  if (w_f64 && g_f64)
    chol_w_kernel<cd, cd, double><<<batch, JAC_THREADS, sm, st>>>((const cd*)G, n, shift, (cd*)W, (cd*)work, use_smem);
  else if (g_f64)
    chol_w_kernel<cf, cd, double><<<batch, JAC_THREADS, sm, st>>>((const cd*)G, n, shift, (cf*)W, (cd*)work, use_smem);
  else if (f32)
    chol_w_kernel<cf, cf, float><<<batch, JAC_THREADS, sm, st>>>((const cf*)G, n, shift, (cf*)W, (cf*)work, use_smem);
  else if (c64)
    chol_w_kernel<cf, cf, double><<<batch, JAC_THREADS, sm, st>>>((const cf*)G, n, shift, (cf*)W, (cd*)work, use_smem);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

bool chol_fits_smem(int n) { return (size_t)n * (n + 1) * sizeof(cd) <= SMEM_LIMIT; }

cudaError_t eigh_batched(cd* A, long long sA, int lda, int n, int batch, double* lam, cd* V, long long sV, cd* work,
                         int* status, cudaStream_t st, int* sweeps_out) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  if (n > 512) return cudaErrorInvalidValue;  // round parameters held in 256-entry tables
  int np = n + (n & 1);
  size_t bytes = (size_t)2 * np * (np + 1) * sizeof(cd);
  int use_smem = bytes <= SMEM_LIMIT;
  if (!use_smem && !work) return cudaErrorInvalidValue;
  cudaError_t ea = smem_optin((const void*)eigh_kernel<double>, (int)SMEM_LIMIT);
  if (ea != cudaSuccess) return ea;
  eigh_kernel<double><<<batch, EIG_THREADS, use_smem ? bytes : 0, st>>>(A, sA, lda, n, lam, V, sV, work, status,
                                                                        use_smem, sweeps_out);
  return cudaGetLastError();
}

cudaError_t eigh_batched_f32(const cf* A, long long sA, int lda, int n, int batch, double* lam, cd* V, long long sV,
                             cf* work, int* status, cudaStream_t st, int* sweeps_out) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  if (n > 512) return cudaErrorInvalidValue;
  int np = n + (n & 1);
  size_t bytes = (size_t)2 * np * (np + 1) * sizeof(cf);
  int use_smem = bytes <= SMEM_LIMIT;
  if (!use_smem && !work) return cudaErrorInvalidValue;
  cudaError_t ea = smem_optin((const void*)eigh_kernel<float>, (int)SMEM_LIMIT);
  if (ea != cudaSuccess) return ea;
  eigh_kernel<float><<<batch, EIG_THREADS, use_smem ? bytes : 0, st>>>(A, sA, lda, n, lam, V, sV, work, status,
                                                                       use_smem, sweeps_out);
  return cudaGetLastError();
}

bool eigh_fits_smem(int n) {
  size_t np = n + (n & 1);
  return (size_t)2 * np * (np + 1) * sizeof(cd) <= SMEM_LIMIT;
}

bool jacobi_fits_smem_f32(int n) {
  size_t np = n + (n & 1);
  return (size_t)2 * np * (np + 1) * sizeof(cf) <= SMEM_LIMIT;
}

cudaError_t svd_batched(cd* A, long long sA, int lda, int m, int n, int batch, double* sigma, cd* U, long long sU,
                        cd* V, long long sV, cd* work, int* status, cudaStream_t st) {
  if (batch <= 0 || n <= 0 || m <= 0) return cudaSuccess;
  if (n > 1024 || m < n) return cudaErrorInvalidValue;
  int np = n + (n & 1);
  size_t bytes = ((size_t)m * np + (size_t)np * np) * sizeof(cd);
  int use_smem = bytes <= SMEM_LIMIT;
  if (!use_smem && !work) return cudaErrorInvalidValue;
  cudaError_t ea = smem_optin((const void*)svd_kernel, (int)SMEM_LIMIT);
  if (ea != cudaSuccess) return ea;
  svd_kernel<<<batch, JAC_THREADS, use_smem ? bytes : 0, st>>>(A, sA, lda, m, n, sigma, U, sU, V, sV, work, status,
                                                              use_smem);
  return cudaGetLastError();
}

}  // namespace tns
