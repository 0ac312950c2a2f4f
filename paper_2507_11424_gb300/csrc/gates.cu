// BP-gauged simple update (Methods, Eqs. 1-2; Appendix Fig. 8d) and belief
// propagation (Appendix Fig. 8c) on the device.  Gates are FP64 throughout; BP is
// FP64 in the FP64 path and complex64 contractions with FP64 normalisation in the
// mixed path.
#include <cctype>
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "linalg.cuh"
#include "state.h"

namespace tns {

static const char LEGCH[5] = {'s', 'u', 'l', 'd', 'r'};

// Mixed-path BP (complex64 contractions, FP64 normalisation): smallest tolerance
// honoured, and the stall rule that detects the FP32 rounding floor.
static constexpr double BP_MIXED_FLOOR = 1e-6;
static constexpr double BP_MIXED_STALL_BELOW = 1e-3;
static constexpr int BP_MIXED_STALL_ITERS = 5;

static std::vector<long long> dims5(const int d[5]) { return {d[0], d[1], d[2], d[3], d[4]}; }

// X = V diag(f(lam_c)) V^H with lam_c = max(lam, 1e-12 lam_max): f = sqrt (X) and 1/sqrt (Xi).
__global__ void gauge_from_eig_kernel(const double* lam, const cd* V, int D, cd* X, cd* Xi) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= D * D) return;
  int i = idx / D, j = idx % D;
  double lmax = lam[0];
  cd x = mk(0.0, 0.0), xi = mk(0.0, 0.0);
  for (int k = 0; k < D; ++k) {
    double l = lmax > 0.0 ? fmax(lam[k], 1e-12 * lmax) : 1.0;
    double sq = sqrt(l);
    cd p = cmul(V[i * D + k], cconj(V[j * D + k]));
    x = cadd(x, cscale(p, sq));
    xi = cadd(xi, cscale(p, 1.0 / sq));
  }
  X[idx] = x;
  Xi[idx] = xi;
}

// W = V diag(lam^{-1/2}) keeping eigenvalues above cut * lam_max (others -> zero column).
__global__ void gram_w_kernel(const double* lam, const cd* V, int n, double cut, cd* Wm) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int c = idx % n;
  double l = lam[c], lmax = lam[0];
  double f = (lmax > 0.0 && l > cut * lmax) ? 1.0 / sqrt(l) : 0.0;
  Wm[idx] = cscale(V[idx], f);
}

// out[(row), b] = in[row, b] * sqrt(sigma_b) (optionally conjugated), b < k; in has ld cols.
__global__ void scale_cols_kernel(const cd* in, int rows, int ld, int k, const double* sigma, int conj_in, cd* out) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * k) return;
  int r = idx / k, b = idx % k;
  cd v = in[(long long)r * ld + b];
  if (conj_in) v = cconj(v);
  out[idx] = cscale(v, sqrt(sigma[b]));
}

__global__ void diag_msg_kernel(const double* sigma, int k, cd* m1, cd* m2) {
  __shared__ double nrm;
  if (threadIdx.x == 0) {
    double s2 = 0;
    for (int i = 0; i < k; ++i) s2 += sigma[i] * sigma[i];
    nrm = sqrt(s2);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    int i = idx / k, j = idx % k;
    cd v = mk(i == j && nrm > 0 ? sigma[i] / nrm : 0.0, 0.0);
    m1[idx] = v;
    m2[idx] = v;
  }
}

struct MsgDesc {
  cd* cur;
  cd* nw;
  int D;
  const cf* nw32;    // mixed path: the new message in complex64 (read instead of nw)
};

__device__ __forceinline__ cd bp_new_entry(const MsgDesc& d, int idx) {
  if (d.nw32) {
    const cf v = d.nw32[idx];
    return mk((double)v.x, (double)v.y);
  }
  return d.nw[idx];
}

// Hermitise and normalise every new message in FP64, write it over the current
// one and record |m_new - m_old|_F per message.  One block per message.
__global__ void bp_finish_kernel(const MsgDesc* md, double* resid) {
  MsgDesc d = md[blockIdx.x];
  __shared__ double red[256];
  const int D = d.D;
  double s2 = 0.0;
  for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
    int i = idx / D, j = idx % D;
    cd a = bp_new_entry(d, i * D + j), b = cconj(bp_new_entry(d, j * D + i));
    s2 += cabs2(cscale(cadd(a, b), 0.5));
  }
  red[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  double nrm = sqrt(red[0]);
  double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  __syncthreads();
  double df = 0.0;
  for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
    int i = idx / D, j = idx % D;
    cd a = bp_new_entry(d, i * D + j), b = cconj(bp_new_entry(d, j * D + i));
    cd h = cscale(cadd(a, b), 0.5 * inv);
    cd o = d.cur[idx];
    df += cabs2(csub(h, o));
    d.cur[idx] = h;
  }
  red[threadIdx.x] = df;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) resid[blockIdx.x] = sqrt(red[0]);
}

static inline int blocks(long long n, int t = 256) { return (int)((n + t - 1) / t); }

// complex128 -> complex64 copy (the mixed path's BP operands)
__global__ void bp_to_c64_kernel(const cd* __restrict__ in, cf* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cd v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

static inline int grid_stride_blocks(long long n) { return (int)std::min<long long>(4 * 152, std::max(1LL, (n + 255) / 256)); }

// t'[.. J ..] = sum_j t[.. j ..] M[j, J] on axis `leg` of a [s][u][l][d][r] tensor.
static cudaError_t apply_leg(const cd* src, const int d[5], int leg, const cd* M, cd* dst, cudaStream_t st) {
  std::string lab = "suldr";
  std::string out = lab;
  out[leg] = (char)toupper(lab[leg]);
  TView A = view((void*)src, lab, dims5(d));
  TView B = view((void*)M, std::string() + lab[leg] + out[leg], {d[leg], d[leg]});
  TView C = view(dst, out, dims5(d));
  return contract(A, B, C, Prec::F64, st);
}

// Buffers of one gate slot.  The gates of a layer are vertex-disjoint, so up to
// GATE_SLOTS of them run at once, each on its own stream with its own buffers.
constexpr int GATE_SLOTS = 8;
struct GateBufs {
  cd *t1, *t2, *G, *V, *Wm, *QA, *QB, *RA, *RB, *P, *theta, *U, *VV, *Us, *gm, *gA, *gB, *X[10], *Xi[10];
  double *lam, *sig;
  int* status;
  cudaStream_t st;
  int slot;
};

static tns_status gate_buffers(tns_state* s, GateBufs& b, int slot) {
  const long long chi = s->chi_max;
  long long tmax = 2;
  for (auto& c : s->cell) tmax = std::max(tmax, c.cap);
  const long long n = 2 * chi, m2 = 2 * n;  // R-factor rank and theta side
  b.slot = slot;
  auto get = [&](const char* nm, size_t bytes, void** p) {
    return s->ws.get(std::string(nm) + "#" + std::to_string(slot), bytes, p);
  };
  TNS_TRY_CUDA(get("g_t1", sizeof(cd) * tmax, (void**)&b.t1));
  TNS_TRY_CUDA(get("g_t2", sizeof(cd) * tmax, (void**)&b.t2));
  TNS_TRY_CUDA(get("g_G", sizeof(cd) * m2 * m2, (void**)&b.G));
  TNS_TRY_CUDA(get("g_V", sizeof(cd) * m2 * m2, (void**)&b.V));
  TNS_TRY_CUDA(get("g_W", sizeof(cd) * m2 * m2, (void**)&b.Wm));
  TNS_TRY_CUDA(get("g_QA", sizeof(cd) * tmax, (void**)&b.QA));
  TNS_TRY_CUDA(get("g_QB", sizeof(cd) * tmax, (void**)&b.QB));
  TNS_TRY_CUDA(get("g_RA", sizeof(cd) * n * n, (void**)&b.RA));
  TNS_TRY_CUDA(get("g_RB", sizeof(cd) * n * n, (void**)&b.RB));
  TNS_TRY_CUDA(get("g_P", sizeof(cd) * m2 * m2, (void**)&b.P));
  TNS_TRY_CUDA(get("g_theta", sizeof(cd) * m2 * m2, (void**)&b.theta));
  TNS_TRY_CUDA(get("g_U", sizeof(cd) * m2 * m2, (void**)&b.U));
  TNS_TRY_CUDA(get("g_VV", sizeof(cd) * m2 * m2, (void**)&b.VV));
  TNS_TRY_CUDA(get("g_Us", sizeof(cd) * m2 * m2, (void**)&b.Us));
  TNS_TRY_CUDA(get("g_gm", sizeof(cd) * 16 * 1024, (void**)&b.gm));
  TNS_TRY_CUDA(get("g_lam", sizeof(double) * m2, (void**)&b.lam));
  TNS_TRY_CUDA(get("g_sig", sizeof(double) * m2, (void**)&b.sig));
  TNS_TRY_CUDA(get("g_status", sizeof(int) * 64, (void**)&b.status));
  TNS_TRY_CUDA(get("g_gA", sizeof(cd) * tmax, (void**)&b.gA));
  TNS_TRY_CUDA(get("g_gB", sizeof(cd) * tmax, (void**)&b.gB));
  for (int i = 0; i < 10; ++i) {
    char nm[32];
    snprintf(nm, sizeof nm, "g_X%d", i);
    TNS_TRY_CUDA(get(nm, sizeof(cd) * chi * chi, (void**)&b.X[i]));
    snprintf(nm, sizeof nm, "g_Xi%d", i);
    TNS_TRY_CUDA(get(nm, sizeof(cd) * chi * chi, (void**)&b.Xi[i]));
  }
  return TNS_OK;
}

// work buffer (of the slot) for Jacobi problems that do not fit in shared memory
static tns_status jacobi_work(tns_state* s, const GateBufs& b, int m, int n, int batch, cd** w) {
  *w = nullptr;
  if (jacobi_fits_smem(m, n)) return TNS_OK;
  long long np = n + (n & 1);
  TNS_TRY_CUDA(s->ws.get("jac_work#" + std::to_string(b.slot),
                         sizeof(cd) * batch * ((long long)m * np + np * np + 2 * np * np), (void**)w));
  return TNS_OK;
}

// Gram-matrix orthonormalisation of the columns (s, j) of t viewed as
// A[(others), (s, j)]: two passes of Q = A V Lambda^{-1/2}; R = Q^H A.
static tns_status reduce_side(tns_state* s, GateBufs& b, const cd* t, const int d[5], int j, cd* Q, cd* R) {
  cudaStream_t st = b.st;
  const int n = d[0] * d[j];
  std::string lab = "suldr";
  std::string others;
  std::vector<long long> odims;
  for (int leg = 1; leg <= 4; ++leg)
    if (leg != j) { others.push_back(lab[leg]); odims.push_back(d[leg]); }
  std::string labA = lab, labB = lab;
  labA[0] = 'S';
  labA[j] = 'J';
  // G[(S,J),(s,j)] = sum_others conj t t
  TNS_TRY_CUDA(contract(view((void*)t, labA, dims5(d), true), view((void*)t, labB, dims5(d)),
                        view(b.G, std::string("SJ") + 's' + lab[j], {d[0], d[j], d[0], d[j]}), Prec::F64, st));
  cd* work = nullptr;
  TNS_TRY(jacobi_work(s, b, n, n, 1, &work));
  TNS_TRY_CUDA(eigh_batched(b.G, (long long)n * n, n, n, 1, b.lam, b.V, (long long)n * n, work, b.status, st));
  gram_w_kernel<<<blocks((long long)n * n), 256, 0, st>>>(b.lam, b.V, n, 1e-30, b.Wm);
  s->launches += 2;
  // Q1[others, c] = sum_{s,j} t W1
  std::vector<long long> qd = odims;
  qd.push_back(n);
  TNS_TRY_CUDA(contract(view((void*)t, lab, dims5(d)),
                        view(b.Wm, std::string("s") + lab[j] + 'c', {d[0], d[j], n}),
                        view(b.t2, others + 'c', qd), Prec::F64, st));
  // second pass: G2 = Q1^H Q1, Q = Q1 W2
  TNS_TRY_CUDA(contract(view(b.t2, others + 'C', qd, true), view(b.t2, others + 'c', qd), view(b.G, "Cc", {n, n}),
                        Prec::F64, st));
  TNS_TRY_CUDA(eigh_batched(b.G, (long long)n * n, n, n, 1, b.lam, b.V, (long long)n * n, work, b.status, st));
  gram_w_kernel<<<blocks((long long)n * n), 256, 0, st>>>(b.lam, b.V, n, 1e-24, b.Wm);
  s->launches += 2;
  TNS_TRY_CUDA(contract(view(b.t2, others + 'c', qd), view(b.Wm, "cC", {n, n}), view(Q, others + 'C', qd),
                        Prec::F64, st));
  // R[c, (s, j)] = sum_others conj Q t
  TNS_TRY_CUDA(contract(view(Q, others + 'c', qd, true), view((void*)t, lab, dims5(d)),
                        view(R, std::string("cs") + lab[j], {n, d[0], d[j]}), Prec::F64, st));
  return TNS_OK;
}

// Rebuild one side: new[others, o, b'] = sum_x Q[others, x] Us[x, o, b'] with Q of
// n columns; then ungauge the external legs with the inverse square roots (the
// last step writes the cell's storage).  c.dim already holds the new bond k.
static tns_status rebuild_side(tns_state* s, GateBufs& b, Cell& c, int j, int n, const cd* Q, const cd* Us,
                               const std::vector<int>& glegs, cd* const* Xi) {
  cudaStream_t st = b.st;
  const std::string lab = "suldr";
  std::string others;
  std::vector<long long> qd;
  for (int leg = 1; leg <= 4; ++leg)
    if (leg != j) { others.push_back(lab[leg]); qd.push_back(c.dim[leg]); }
  qd.push_back(n);
  const int k = c.dim[j];
  cd* bufs[2] = {b.t1, b.t2};
  cd* cur = glegs.empty() ? c.t : bufs[0];
  TNS_TRY_CUDA(contract(view((void*)Q, others + 'x', qd),
                        view((void*)Us, std::string("xs") + lab[j], {n, c.dim[0], k}),
                        view(cur, lab, dims5(c.dim)), Prec::F64, st));
  for (size_t i = 0; i < glegs.size(); ++i) {
    cd* dst = (i + 1 == glegs.size()) ? c.t : bufs[(i + 1) & 1];
    TNS_TRY_CUDA(apply_leg(cur, c.dim, glegs[i], Xi[i], dst, st));
    cur = dst;
  }
  return TNS_OK;
}

// psi_tilde = psi x_l X_l over the listed legs; result in `out` (or psi itself if no legs).
static tns_status gauge_side(tns_state* s, GateBufs& b, const Cell& c, const std::vector<int>& glegs, cd* const* X,
                             cd* out, const cd** res) {
  if (glegs.empty()) { *res = c.t; return TNS_OK; }
  cd* bufs[2] = {b.t1, b.t2};
  const cd* cur = c.t;
  for (size_t i = 0; i < glegs.size(); ++i) {
    cd* dst = (i + 1 == glegs.size()) ? out : bufs[i & 1];
    TNS_TRY_CUDA(apply_leg(cur, c.dim, glegs[i], X[i], dst, b.st));
    cur = dst;
  }
  *res = out;
  return TNS_OK;
}

static tns_status gauge_mats(tns_state* s, GateBufs& b, int ci, const std::vector<int>& glegs, cd* const* X,
                             cd* const* Xi) {
  for (size_t i = 0; i < glegs.size(); ++i) {
    int leg = glegs[i];
    int D = s->cell[ci].dim[leg];
    const cd* m = s->msg[ci * 5 + leg];
    cd* work = nullptr;
    TNS_TRY(jacobi_work(s, b, D, D, 1, &work));
    TNS_TRY_CUDA(eigh_batched((cd*)m, (long long)D * D, D, D, 1, b.lam, b.V, (long long)D * D, work, b.status, b.st));
    gauge_from_eig_kernel<<<blocks((long long)D * D), 256, 0, b.st>>>(b.lam, b.V, D, X[i], Xi[i]);
    s->launches += 2;
  }
  return TNS_OK;
}

static int leg_between(const tns_state* s, int ca, int cb) {
  int ra = ca / s->W, xa = ca % s->W, rb = cb / s->W, xb = cb % s->W;
  if (rb == ra - 1 && xb == xa) return LEG_U;
  if (rb == ra + 1 && xb == xa) return LEG_D;
  if (rb == ra && xb == xa - 1) return LEG_L;
  if (rb == ra && xb == xa + 1) return LEG_R;
  return -1;
}

// A two-qubit gate in two halves.  gate_begin enqueues, on the slot's stream, the
// gauging, the QR reduction of both sides, theta = G R_A R_B and its SVD, and copies
// the singular values and the SVD status to the slot's pinned host block (event
// recorded after the copy); it never waits.  gate_end waits for that event, picks the
// kept rank and epsilon (Eq. 1) on the host, and enqueues the rebuild of both sides and
// the bond messages.
struct GateJob {
  int q0, q1, ca, cb, j, jb, n, m2;
  std::vector<int> ga, gb;
  double* h_sig;                 // pinned: m2 singular values, then the status word
};

static tns_status gate_begin(tns_state* s, GateBufs& b, GateJob& jb_, const cd* gmat, cudaEvent_t ev) {
  cudaStream_t st = b.st;
  jb_.ca = s->qcell[jb_.q0];
  jb_.cb = s->qcell[jb_.q1];
  jb_.j = leg_between(s, jb_.ca, jb_.cb);
  jb_.jb = opp_leg(jb_.j);
  Cell& A = s->cell[jb_.ca];
  Cell& B = s->cell[jb_.cb];
  jb_.ga.clear();
  jb_.gb.clear();
  for (int leg = 1; leg <= 4; ++leg) {
    if (leg != jb_.j && A.edge[leg]) jb_.ga.push_back(leg);
    if (leg != jb_.jb && B.edge[leg]) jb_.gb.push_back(leg);
  }
  TNS_TRY(gauge_mats(s, b, jb_.ca, jb_.ga, b.X, b.Xi));
  TNS_TRY(gauge_mats(s, b, jb_.cb, jb_.gb, b.X + 5, b.Xi + 5));
  const cd *tA = nullptr, *tB = nullptr;
  TNS_TRY(gauge_side(s, b, A, jb_.ga, b.X, b.gA, &tA));
  TNS_TRY(gauge_side(s, b, B, jb_.gb, b.X + 5, b.gB, &tB));
  const int Dj = A.dim[jb_.j];
  const int n = A.dim[0] * Dj;  // = B.dim[0] * Dj
  jb_.n = n;
  TNS_TRY(reduce_side(s, b, tA, A.dim, jb_.j, b.QA, b.RA));
  TNS_TRY(reduce_side(s, b, tB, B.dim, jb_.jb, b.QB, b.RB));
  TNS_TRY_CUDA(contract(view(b.RA, "xsb", {n, 2, Dj}), view(b.RB, "ytb", {n, 2, Dj}), view(b.P, "xsyt", {n, 2, n, 2}),
                        Prec::F64, st));
  TNS_TRY_CUDA(contract(view((void*)gmat, "opst", {2, 2, 2, 2}), view(b.P, "xsyt", {n, 2, n, 2}),
                        view(b.theta, "xoyp", {n, 2, n, 2}), Prec::F64, st));
  const int m2 = 2 * n;
  jb_.m2 = m2;
  cd* work = nullptr;
  TNS_TRY(jacobi_work(s, b, m2, m2, 1, &work));
  TNS_TRY_CUDA(svd_batched(b.theta, (long long)m2 * m2, m2, m2, m2, 1, b.sig, b.U, (long long)m2 * m2, b.VV,
                           (long long)m2 * m2, work, b.status, st));
  s->launches += 1;
  TNS_TRY_CUDA(cudaMemcpyAsync(jb_.h_sig, b.sig, sizeof(double) * m2, cudaMemcpyDeviceToHost, st));
  TNS_TRY_CUDA(cudaMemcpyAsync(jb_.h_sig + m2, b.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  TNS_TRY_CUDA(cudaEventRecord(ev, st));
  return TNS_OK;
}

static tns_status gate_end(tns_state* s, GateBufs& b, GateJob& jb_, cudaEvent_t ev, int chi, double cutoff,
                           double* eps_out) {
  cudaStream_t st = b.st;
  TNS_TRY_CUDA(cudaEventSynchronize(ev));
  const int m2 = jb_.m2, n = jb_.n;
  const double* sig = jb_.h_sig;
  int status = 0;
  std::memcpy(&status, jb_.h_sig + m2, sizeof(int));
  double tot = 0.0;
  for (int i = 0; i < m2; ++i) tot += sig[i] * sig[i];
  if (!std::isfinite(tot)) {
    set_error("non-finite singular values in gate on qubits %d,%d", jb_.q0, jb_.q1);
    return TNS_ERR_NUMERIC;
  }
  int keep = 0;
  for (int i = 0; i < m2; ++i)
    if (sig[0] > 0 && sig[i] > cutoff * sig[0]) ++keep;
  int k = std::max(1, std::min(chi, keep));
  double disc = 0.0;
  for (int i = k; i < m2; ++i) disc += sig[i] * sig[i];
  double eps = tot > 0.0 ? disc / tot : 0.0;
  Cell& A = s->cell[jb_.ca];
  Cell& B = s->cell[jb_.cb];
  // side A
  scale_cols_kernel<<<blocks((long long)m2 * k), 256, 0, st>>>(b.U, m2, m2, k, b.sig, 0, b.Us);
  A.dim[jb_.j] = k;
  TNS_TRY(rebuild_side(s, b, A, jb_.j, n, b.QA, b.Us, jb_.ga, b.Xi));
  scale_cols_kernel<<<blocks((long long)m2 * k), 256, 0, st>>>(b.VV, m2, m2, k, b.sig, 1, b.Us);
  B.dim[jb_.jb] = k;
  TNS_TRY(rebuild_side(s, b, B, jb_.jb, n, b.QB, b.Us, jb_.gb, b.Xi + 5));
  diag_msg_kernel<<<1, 256, 0, st>>>(b.sig, k, s->msg[jb_.ca * 5 + jb_.j], s->msg[jb_.cb * 5 + jb_.jb]);
  s->launches += 3;
  s->log_f += (eps < 1.0) ? std::log1p(-eps) : -INFINITY;
  if (eps_out) *eps_out = eps;
  if (status != 0) {
    set_error("SVD sweep cap reached in gate on qubits %d,%d", jb_.q0, jb_.q1);
    return TNS_ERR_NUMERIC;
  }
  return TNS_OK;
}

// GATE_SLOTS streams, their events and the pinned host blocks, created on first use.
static tns_status gate_slots(tns_state* s) {
  const size_t per = (size_t)4 * s->chi_max + 2;
  if ((int)s->gate_streams.size() < GATE_SLOTS) {
    for (int i = (int)s->gate_streams.size(); i < GATE_SLOTS; ++i) {
      cudaStream_t q = nullptr;
      cudaEvent_t e = nullptr;
      TNS_TRY_CUDA(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
      s->gate_streams.push_back(q);
      TNS_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      s->gate_events.push_back(e);
    }
  }
  if (s->gate_host_n < per * GATE_SLOTS) {
    if (s->gate_host) cudaFreeHost(s->gate_host);
    s->gate_host = nullptr;
    s->gate_host_n = 0;
    TNS_TRY_CUDA(cudaMallocHost((void**)&s->gate_host, sizeof(double) * per * GATE_SLOTS));
    s->gate_host_n = per * GATE_SLOTS;
  }
  return TNS_OK;
}

tns_status apply_gate_layer(tns_state* s, int n_gates, const int32_t* sites, const double* mats, int chi,
                            double cutoff, double* eps_out) {
  std::vector<char> used(s->n, 0);
  for (int g = 0; g < n_gates; ++g) {
    int a = sites[2 * g], bq = sites[2 * g + 1];
    if (a < 0 || a >= s->n || bq < -1 || bq >= s->n || a == bq) {
      set_error("gate %d: invalid qubits (%d,%d)", g, a, bq);
      return TNS_ERR_ARG;
    }
    if (used[a] || (bq >= 0 && used[bq])) {
      set_error("gate %d overlaps another gate of the layer", g);
      return TNS_ERR_ARG;
    }
    used[a] = 1;
    if (bq >= 0) {
      used[bq] = 1;
      int j = leg_between(s, s->qcell[a], s->qcell[bq]);
      if (j < 0 || !s->cell[s->qcell[a]].edge[j]) {
        set_error("gate %d acts on qubits %d,%d that share no bond", g, a, bq);
        return TNS_ERR_ARG;
      }
    }
    for (int i = 0; i < 32; ++i)
      if (!std::isfinite(mats[32 * g + i])) { set_error("gate %d has non-finite entries", g); return TNS_ERR_ARG; }
  }
  if (n_gates == 0) return TNS_OK;
  TNS_TRY(gate_slots(s));
  GateBufs bufs[GATE_SLOTS];
  for (int i = 0; i < GATE_SLOTS; ++i) {
    TNS_TRY(gate_buffers(s, bufs[i], i));
    bufs[i].st = s->gate_streams[i];
  }
  cd* gm = nullptr;
  TNS_TRY_CUDA(s->ws.get("g_gates", sizeof(cd) * 16 * n_gates, (void**)&gm));
  TNS_TRY_CUDA(cudaMemcpyAsync(gm, mats, sizeof(cd) * 16 * n_gates, cudaMemcpyHostToDevice, s->st));
  // the slots start after everything already on the state's stream (the gate
  // matrices, earlier layers, BP) and the state's stream waits for all slots at the end
  cudaEvent_t fork = nullptr;
  TNS_TRY_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  struct EvGuard {
    cudaEvent_t e;
    ~EvGuard() { if (e) cudaEventDestroy(e); }
  } fork_guard{fork};
  TNS_TRY_CUDA(cudaEventRecord(fork, s->st));
  for (int i = 0; i < GATE_SLOTS; ++i) TNS_TRY_CUDA(cudaStreamWaitEvent(bufs[i].st, fork, 0));
  const size_t per = (size_t)4 * s->chi_max + 2;
  tns_status result = TNS_OK;
  auto join = [&]() -> tns_status {
    for (int i = 0; i < GATE_SLOTS; ++i) {
      TNS_TRY_CUDA(cudaEventRecord(s->gate_events[i], bufs[i].st));
      TNS_TRY_CUDA(cudaStreamWaitEvent(s->st, s->gate_events[i], 0));
    }
    return TNS_OK;
  };
  // gates in rounds of GATE_SLOTS: every gate's first half is enqueued (they overlap on
  // the GPU), then the second halves in gate order as their singular values arrive
  std::vector<GateJob> jobs(GATE_SLOTS);
  for (int g0 = 0; g0 < n_gates; g0 += GATE_SLOTS) {
    const int g1 = std::min(n_gates, g0 + GATE_SLOTS);
    for (int g = g0; g < g1; ++g) {
      const int slot = g - g0;
      GateBufs& b = bufs[slot];
      int a = sites[2 * g], bq = sites[2 * g + 1];
      if (bq < 0) {
        Cell& c = s->cell[s->qcell[a]];
        tns_status r = TNS_OK;
        cudaError_t e = contract(view(gm + 16 * g, "os", {2, 2}), view(c.t, "suldr", dims5(c.dim)),
                                 view(b.t1, "ouldr", dims5(c.dim)), Prec::F64, b.st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.t, b.t1, sizeof(cd) * c.size(), cudaMemcpyDeviceToDevice, b.st);
        if (e != cudaSuccess) r = cuda_status(e, "one-qubit gate");
        if (r != TNS_OK) { join(); return r; }
        continue;
      }
      GateJob& jb_ = jobs[slot];
      jb_.q0 = a;
      jb_.q1 = bq;
      jb_.h_sig = s->gate_host + per * slot;
      tns_status r = gate_begin(s, b, jb_, gm + 16 * g, s->gate_events[slot]);
      if (r != TNS_OK) { join(); return r; }
    }
    for (int g = g0; g < g1; ++g) {
      const int slot = g - g0;
      double eps = 0.0;
      if (sites[2 * g + 1] >= 0) {
        tns_status r = gate_end(s, bufs[slot], jobs[slot], s->gate_events[slot], chi, cutoff, &eps);
        if (r == TNS_ERR_NUMERIC) result = r;
        else if (r != TNS_OK) { join(); return r; }
      }
      if (eps_out) eps_out[g] = eps;
    }
  }
  TNS_TRY(join());
  s->version++;
  TNS_TRY_CUDA(cudaStreamSynchronize(s->st));
  return result;
}

// ---------------------------------------------------------------- BP
// Directed edges (v -> v') are grouped by the shape of psi_v and the outgoing
// leg; each group runs as one batched contraction chain that gathers the cell
// tensors and messages of its members through per-member offset arrays:
//   X = psi_v x_l m_{l -> v} for every other bonded leg l, then
//   m_new[k, kbar] = sum X[.. k ..] conj(psi_v[.. kbar ..]).
tns_status bp_gauge(tns_state* s, int max_iter, double tol, int* iters, double* resid) {
  cudaStream_t st = s->st;
  struct Group {
    int dims[5];
    int edges;
    int j;
    std::vector<long long> cell_off, dst_off, moff[5];
    long long* d_cell = nullptr;
    long long* d_dst = nullptr;
    long long* d_moff[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  };
  std::vector<Group> groups;
  std::vector<MsgDesc> md;
  const long long mslot = (long long)s->chi_max * s->chi_max;
  for (int ci = 0; ci < (int)s->cell.size(); ++ci) {
    const Cell& c = s->cell[ci];
    int eb = 0;
    for (int leg = 1; leg <= 4; ++leg) eb |= (c.edge[leg] ? 1 : 0) << leg;
    for (int j = 1; j <= 4; ++j) {
      if (!c.edge[j]) continue;
      int r2, c2;
      s->nbr(ci, j, r2, c2);
      int dst = s->cidx(r2, c2) * 5 + opp_leg(j);
      Group* g = nullptr;
      for (auto& gg : groups)
        if (gg.j == j && gg.edges == eb && std::equal(gg.dims, gg.dims + 5, c.dim)) { g = &gg; break; }
      if (!g) {
        groups.emplace_back();
        g = &groups.back();
        std::copy(c.dim, c.dim + 5, g->dims);
        g->edges = eb;
        g->j = j;
      }
      g->cell_off.push_back(c.off);
      g->dst_off.push_back((long long)dst * mslot);
      for (int leg = 1; leg <= 4; ++leg) g->moff[leg].push_back((long long)(ci * 5 + leg) * mslot);
      md.push_back({s->msg[dst], s->msg_new[dst], c.dim[j]});
    }
  }
  *iters = 0;
  *resid = 0.0;
  s->bp_last_ms = s->bp_last_bytes = s->bp_last_flops = 0.0;
  if (md.empty()) return TNS_OK;
  // Precision: FP64 path, every contraction in FP64.  Mixed path, the message
  // contractions run on complex64 copies of the cells and messages (TF32x3 tensor
  // cores where the planner finds them worth it, FP32 CUDA cores otherwise, FP32
  // accumulation) and the Hermitisation, normalisation and residual stay FP64; the
  // residual then cannot fall much below the FP32 rounding of the contractions, so
  // the tolerance is raised to BP_MIXED_FLOOR.
  const bool mixed = s->prec == TNS_PREC_MIXED;
  const Prec bp_prec = mixed ? (s->tensor_cores ? Prec::TF32X3 : Prec::F32) : Prec::F64;
  const double tol_eff = mixed ? std::max(tol, BP_MIXED_FLOOR) : tol;
  const size_t esz = mixed ? sizeof(cf) : sizeof(cd);
  // upload the offset tables once
  std::vector<long long> table;
  for (auto& g : groups) {
    table.insert(table.end(), g.cell_off.begin(), g.cell_off.end());
    table.insert(table.end(), g.dst_off.begin(), g.dst_off.end());
    for (int leg = 1; leg <= 4; ++leg) table.insert(table.end(), g.moff[leg].begin(), g.moff[leg].end());
  }
  long long* dtab = nullptr;
  TNS_TRY_CUDA(s->ws.get("bp_tab", sizeof(long long) * table.size(), (void**)&dtab));
  TNS_TRY_CUDA(cudaMemcpyAsync(dtab, table.data(), sizeof(long long) * table.size(), cudaMemcpyHostToDevice, st));
  long long pos = 0, xmax = 1;
  double bytes_it = 0.0;
  for (auto& g : groups) {
    const long long G = (long long)g.cell_off.size();
    g.d_cell = dtab + pos; pos += G;
    g.d_dst = dtab + pos; pos += G;
    for (int leg = 1; leg <= 4; ++leg) { g.d_moff[leg] = dtab + pos; pos += G; }
    long long sz = (long long)g.dims[0] * g.dims[1] * g.dims[2] * g.dims[3] * g.dims[4];
    xmax = std::max(xmax, G * sz);
    // algorithmic bytes: every member reads its site tensor (ket and bra side of the
    // same array, counted once), its incoming messages, and writes one message
    long long mb = 0;
    for (int leg = 1; leg <= 4; ++leg)
      if (leg != g.j && (g.edges >> leg & 1)) mb += (long long)g.dims[leg] * g.dims[leg];
    mb += (long long)g.dims[g.j] * g.dims[g.j];
    bytes_it += (double)G * (double)(sz + mb) * (double)esz;
  }
  void *X0, *X1;
  TNS_TRY_CUDA(s->ws.get("bp_X0", esz * xmax, &X0));
  TNS_TRY_CUDA(s->ws.get("bp_X1", esz * xmax, &X1));
  void* cells = s->cell_arena;
  void* msgs = s->msg_arena;
  void* msgs_new = s->msg_new_arena;
  const long long msg_elems = mslot * (long long)s->cell.size() * 5;
  cf* m32 = nullptr;
  if (mixed) {
    long long arena = 0;
    for (auto& c : s->cell) arena = std::max(arena, c.off + c.cap);
    cf *c32 = nullptr, *mn32 = nullptr;
    TNS_TRY_CUDA(s->ws.get("bp_c32", sizeof(cf) * arena, (void**)&c32));
    TNS_TRY_CUDA(s->ws.get("bp_m32", sizeof(cf) * msg_elems, (void**)&m32));
    TNS_TRY_CUDA(s->ws.get("bp_mn32", sizeof(cf) * msg_elems, (void**)&mn32));
    bp_to_c64_kernel<<<grid_stride_blocks(arena), 256, 0, st>>>(s->cell_arena, c32, arena);
    s->launches++;
    cells = c32;
    msgs = m32;
    msgs_new = mn32;
    for (auto& d : md) d.nw32 = mn32 + (d.nw - s->msg_new_arena);
  }
  MsgDesc* dmd = nullptr;
  double* dres = nullptr;
  const size_t nmsg = md.size();
  TNS_TRY_CUDA(s->ws.get("bp_desc", sizeof(MsgDesc) * nmsg, (void**)&dmd));
  TNS_TRY_CUDA(s->ws.get("bp_res", sizeof(double) * nmsg, (void**)&dres));
  TNS_TRY_CUDA(cudaMemcpyAsync(dmd, md.data(), sizeof(MsgDesc) * nmsg, cudaMemcpyHostToDevice, st));
  if (s->bp_host_n < 2 * nmsg) {
    if (s->bp_host) cudaFreeHost(s->bp_host);
    s->bp_host = nullptr;
    s->bp_host_n = 0;
    TNS_TRY_CUDA(cudaMallocHost((void**)&s->bp_host, sizeof(double) * 2 * nmsg));
    s->bp_host_n = 2 * nmsg;
  }
  double* hres[2] = {s->bp_host, s->bp_host + nmsg};
  // events: two per iteration slot (residual copy landed), plus the timing pair
  cudaEvent_t ev[2] = {nullptr, nullptr}, t0 = nullptr, t1 = nullptr;
  struct EvGuard {
    cudaEvent_t* e[4];
    ~EvGuard() {
      for (auto p : e)
        if (*p) cudaEventDestroy(*p);
    }
  } guard{{&ev[0], &ev[1], &t0, &t1}};
  for (auto& e : ev) TNS_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  TNS_TRY_CUDA(cudaEventCreate(&t0));
  TNS_TRY_CUDA(cudaEventCreate(&t1));
  TNS_TRY_CUDA(cudaEventRecord(t0, st));
  double flops_it = 0.0;
  const std::string lab = "suldr";
  // one BP iteration: contractions for every directed edge, FP64 finish, residuals
  // copied to hres[slot] (pinned) and ev[slot] recorded; nothing waits on the host
  auto enqueue = [&](int slot) -> tns_status {
    if (mixed) {
      bp_to_c64_kernel<<<grid_stride_blocks(msg_elems), 256, 0, st>>>(s->msg_arena, m32, msg_elems);
      s->launches++;
    }
    double fl_total = 0.0;
    for (auto& g : groups) {
      const long long G = (long long)g.cell_off.size();
      std::vector<long long> d5 = dims5(g.dims);
      std::vector<long long> gd = {G};
      gd.insert(gd.end(), d5.begin(), d5.end());
      // current operand: the cells themselves (gathered) or a workspace buffer
      TView cur = view(cells, "G" + lab, gd);
      cur.stride[0] = 0;
      cur.boff = g.d_cell;
      cur.boff_label = 'G';
      void* bufs[2] = {X0, X1};
      int nb = 0;
      double fl = 0.0;
      for (int leg = 1; leg <= 4; ++leg) {
        if (leg == g.j || !(g.edges >> leg & 1)) continue;
        std::string out = "G" + lab;
        out[leg + 1] = (char)toupper(lab[leg]);
        TView M = view(msgs, std::string("G") + lab[leg] + out[leg + 1], {G, d5[leg], d5[leg]});
        M.stride[0] = 0;
        M.boff = g.d_moff[leg];
        M.boff_label = 'G';
        void* dst = bufs[nb & 1];
        TNS_TRY_CUDA(contract(cur, M, view(dst, out, gd), bp_prec, st, make_double2(1.0, 0.0),
                              make_double2(0.0, 0.0), &fl));
        fl_total += fl;
        cur = view(dst, "G" + lab, gd);   // labels restart for the next leg
        ++nb;
      }
      std::string la = "G" + lab, lb = "G" + lab;
      la[g.j + 1] = 'a';
      lb[g.j + 1] = 'b';
      cur.labels = la;
      TView bra = view(cells, lb, gd, true);
      bra.stride[0] = 0;
      bra.boff = g.d_cell;
      bra.boff_label = 'G';
      const long long D = d5[g.j];
      TView out = view(msgs_new, "Gab", {G, D, D});
      out.stride[0] = 0;
      out.boff = g.d_dst;
      out.boff_label = 'G';
      TNS_TRY_CUDA(contract(cur, bra, out, bp_prec, st, make_double2(1.0, 0.0), make_double2(0.0, 0.0), &fl));
      fl_total += fl;
    }
    flops_it = fl_total;
    bp_finish_kernel<<<(unsigned)nmsg, 256, 0, st>>>(dmd, dres);
    s->launches++;
    TNS_TRY_CUDA(cudaMemcpyAsync(hres[slot], dres, sizeof(double) * nmsg, cudaMemcpyDeviceToHost, st));
    TNS_TRY_CUDA(cudaEventRecord(ev[slot], st));
    return TNS_OK;
  };
  // residual of the iteration whose copy went to hres[slot] (waits for that copy only)
  auto residual = [&](int slot, double* r) -> tns_status {
    TNS_TRY_CUDA(cudaEventSynchronize(ev[slot]));
    double mx = 0.0;
    for (size_t i = 0; i < nmsg; ++i) {
      const double x = hres[slot][i];
      if (!std::isfinite(x)) { *r = x; set_error("non-finite BP message"); return TNS_ERR_NUMERIC; }
      mx = std::max(mx, x);
    }
    *r = mx;
    return TNS_OK;
  };
  auto finish = [&](int it, double r) {
    *iters = it;
    *resid = r;
    float ms = 0.f;
    if (cudaEventRecord(t1, st) == cudaSuccess && cudaEventSynchronize(t1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess)
      s->bp_last_ms = ms;
    s->bp_last_bytes = bytes_it * it;
    s->bp_last_flops = flops_it * it;
  };
  // Iteration it is checked while iteration it + 1 runs, so the host never idles the
  // GPU; convergence is declared on the last enqueued iteration.  Mixed path: once the
  // residual is below BP_MIXED_STALL_BELOW and has stopped falling (no 10% gain over
  // the best for BP_MIXED_STALL_ITERS checks) it sits at the FP32 rounding floor, which
  // also counts as converged.
  double best = 1e300;
  int stall = 0;
  for (int it = 1;; ++it) {
    TNS_TRY(enqueue(it & 1));
    double r = 0.0;
    if (it > 1) {
      TNS_TRY(residual((it - 1) & 1, &r));
      bool floor_hit = false;
      if (mixed) {
        stall = (r < BP_MIXED_STALL_BELOW && r > 0.9 * best) ? stall + 1 : 0;
        best = std::min(best, r);
        floor_hit = stall >= BP_MIXED_STALL_ITERS;
      }
      if (r < tol_eff || floor_hit) {
        double r2 = 0.0;
        TNS_TRY(residual(it & 1, &r2));
        if (r2 < tol_eff || floor_hit) {
          finish(it, r2);
          return TNS_OK;
        }
      }
    }
    if (it >= max_iter) {
      TNS_TRY(residual(it & 1, &r));
      finish(it, r);
      if (r < tol_eff) return TNS_OK;
      set_error("BP not converged after %d iterations (residual %.3e)", max_iter, r);
      return TNS_ERR_NOT_CONVERGED;
    }
  }
}

}  // namespace tns
