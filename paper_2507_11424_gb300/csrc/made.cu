// Learned proposal on the device: MADE network trained by maximum likelihood with
// BF16 GEMMs on the tcgen05 tensor cores (FP32 accumulation in TMEM, fused bias /
// ReLU / ReLU-gate epilogues; tc_bf16.cu), FP32 master weights and Adam,
// ancestral sampling with Philox draws, and independent Metropolis-Hastings.
// Not part of the paper; see include/tns.h (tns_made_*, tns_mh_independent).
//
// Layouts: every BF16 GEMM operand is row-major with its contraction index
// contiguous and a row pitch that is a multiple of 8 elements (TMA): activations
// [B][hp] and [B][np] (hp, np = hidden width and qubit count rounded up to 8),
// masked weights W1 [h][np], W2, W3 [h][hp], W4 [n][hp] and their transposes
// W2^T, W3^T [h][hp], W4^T [h][np]; weight gradients contract over the batch and
// read transposed activation copies [rows][Bp].
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "../../include/tns.h"
#include "common.cuh"
#include "state.h"
#include "tc_bf16.cuh"
#include "tc_gemm.cuh"

typedef __nv_bfloat16 bf16;

struct tns_made {
  int n = 0, h = 0;
  int np = 0, hp = 0;               // n and h rounded up to multiples of 8 (row pitches)
  cudaStream_t st = nullptr;
  long long P = 0;
  long long off[8] = {};            // W1, b1, W2, b2, W3, b3, W4, b4 in the packed vector
  long long woff[4] = {};           // masked bf16 weights W1..W4 (pitches np, hp, hp, hp)
  long long wtoff[3] = {};          // their transposes W2^T, W3^T (pitch hp), W4^T (pitch np)
  float* theta = nullptr;           // FP32 master parameters
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  bf16* wb = nullptr;
  long long t = 0;                  // Adam steps taken
  long long launches = 0;
  tns::Workspace ws;
};

namespace tns {

__device__ __forceinline__ int hdeg(int k, int n) { return 1 + (k % (n > 1 ? n - 1 : 1)); }

// Layer L (0..3) weight mask at (row r, col c): hidden rows need deg(r) >= deg(c),
// output rows need r+1 > deg(c) (MADE connectivity, natural order).
__device__ __forceinline__ bool made_mask(int L, int r, int c, int n) {
  if (L == 0) return hdeg(r, n) >= c + 1;
  if (L == 3) return r + 1 > hdeg(c, n);
  return hdeg(r, n) >= hdeg(c, n);
}

struct MadeLayout {
  long long off[8];
  int rows[4], cols[4], pitch[4];
  int n;
};

// Masked BF16 copies of the four weight matrices (row pitches lay.pitch[L]).
__global__ void made_prep_weights_kernel(const float* theta, MadeLayout lay, bf16* wb, long long w1, long long w2,
                                         long long w3, long long w4) {
  const long long wo[4] = {w1, w2, w3, w4};
  for (int L = 0; L < 4; ++L) {
    const long long cnt = (long long)lay.rows[L] * lay.cols[L];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x) {
      int r = (int)(i / lay.cols[L]), c = (int)(i % lay.cols[L]);
      float val = made_mask(L, r, c, lay.n) ? theta[lay.off[2 * L] + i] : 0.f;
      wb[wo[L] + (long long)r * lay.pitch[L] + c] = __float2bfloat16(val);
    }
  }
}

// X[b][j] (pitch np) and xb[b][j] (pitch n) from row order[i0 + b] (or i0 + b) of bits.
__global__ void made_gather_bits_kernel(const uint8_t* bits, const int32_t* order, long long i0, int B, int n, int np,
                                        bf16* X, uint8_t* xb) {
  long long tot = (long long)B * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    long long b = i / n;
    int j = (int)(i % n);
    long long row = order ? order[i0 + b] : i0 + b;
    uint8_t x = bits[row * n + j] ? 1 : 0;
    X[b * np + j] = __float2bfloat16(x ? 1.f : 0.f);
    xb[i] = x;
  }
}

__device__ __forceinline__ double softplus_d(double z) { return fmax(z, 0.0) + log1p(exp(-fabs(z))); }

// Row log g(x) = -sum_i softplus(-(2x_i - 1) l_i); dL = (sigmoid(l) - x) / B (FP32 and BF16).
// L, dLf, dLb have pitch np; xb has pitch n.
__global__ void made_loss_grad_kernel(const float* L, const uint8_t* xb, int B, int n, int np, double* logg, float* dLf,
                                      bf16* dLb) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double lp = 0.0;
  for (int i = 0; i < n; ++i) {
    long long o = (long long)b * np + i;
    double l = L[o];
    int x = xb[(long long)b * n + i];
    lp -= softplus_d(x ? -l : l);
    if (dLf) {
      float d = (float)((1.0 / (1.0 + exp(-l)) - x) / B);
      dLf[o] = d;
      dLb[o] = __float2bfloat16(d);
    }
  }
  logg[b] = lp;
}

// out[j] = sum_b X[b][j] (pitch ld), for the bias gradients.
__global__ void colsum_kernel(const float* X, int B, int N, long long ld, float* out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += X[(long long)b * ld + j];
  out[j] = s;
}

// Zero the gradient of masked-out weights (they stay at their initial values).
__global__ void made_mask_grad_kernel(float* grad, MadeLayout lay) {
  for (int L = 0; L < 4; ++L) {
    const long long cnt = (long long)lay.rows[L] * lay.cols[L];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
      if (!made_mask(L, (int)(i / lay.cols[L]), (int)(i % lay.cols[L]), lay.n)) grad[lay.off[2 * L] + i] = 0.f;
  }
}

// Adam (Kingma & Ba 2015) with bias corrections c1 = 1/(1-b1^t), c2 = 1/(1-b2^t).
__global__ void made_adam_kernel(float* theta, float* m, float* v, const float* grad, long long P, float lr, float b1,
                                 float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// Draw column i of every proposal: x_i = 1 iff u >= g(x_i = 0 | x_<i), u from the
// Philox counter (sample lo, sample hi, i, 1); log g accumulates in FP64.
__global__ void made_draw_kernel(const float* L, int B, int n, int np, int i, uint64_t seed, long long s0, bf16* X,
                                 uint8_t* bits, double* logg) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double l = L[(long long)b * np + i];
  double p0 = 1.0 / (1.0 + exp(l));
  unsigned long long sid = (unsigned long long)(s0 + b);
  Philox4 w = philox4x32_10((uint32_t)(sid & 0xffffffffu), (uint32_t)(sid >> 32), (uint32_t)i, 1u,
                            (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  int x = u53(w.v[0], w.v[1]) >= p0 ? 1 : 0;
  X[(long long)b * np + i] = __float2bfloat16(x ? 1.f : 0.f);
  bits[(s0 + b) * (long long)n + i] = (uint8_t)x;
  logg[s0 + b] += -softplus_d(x ? -l : l);
}

// Independent MH, one thread per chain: accept iff u < exp(lp' - lp + lg - lg'),
// u from the Philox counter (chain, step, 0, 2).
__global__ void mh_kernel(int C, int T, const double* lpp, const double* lgp, const double* lp0, const double* lg0,
                          uint64_t seed, int32_t* state, int64_t* acc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double lp = lp0[c], lg = lg0[c];
  int cur = -1;
  long long na = 0;
  for (int t = 0; t < T; ++t) {
    long long o = (long long)c * T + t;
    Philox4 w = philox4x32_10((uint32_t)c, (uint32_t)t, 0u, 2u, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    double u = u53(w.v[0], w.v[1]);
    double a = (lpp[o] - lp) + (lg - lgp[o]);
    if (u == 0.0 || log(u) < a) {
      lp = lpp[o];
      lg = lgp[o];
      cur = t;
      ++na;
    }
    state[o] = cur;
  }
  acc[c] = na;
}

static inline unsigned blk(long long n, int t = 256) { return (unsigned)std::max<long long>(1, std::min<long long>((n + t - 1) / t, 152LL * 32)); }

static MadeLayout layout(const tns_made* md) {
  MadeLayout L;
  for (int i = 0; i < 8; ++i) L.off[i] = md->off[i];
  const int n = md->n, h = md->h;
  int rows[4] = {h, h, h, n}, cols[4] = {n, h, h, h}, pitch[4] = {md->np, md->hp, md->hp, md->hp};
  for (int i = 0; i < 4; ++i) { L.rows[i] = rows[i]; L.cols[i] = cols[i]; L.pitch[i] = pitch[i]; }
  L.n = n;
  return L;
}

static inline long long round8(long long x) { return (x + 7) / 8 * 8; }

// Tensor-core GEMM C = A B^T over K with the fused epilogue (see tc_bf16.cuh).
static cudaError_t gemm(tns_made* md, int M, int N, int K, const bf16* A, long long lda, const bf16* B, long long ldb,
                        float* Cf, bf16* Cb, long long ldc, const float* bias, int relu, const float* gate) {
  Bf16Gemm g{M, N, K, Cf, Cb, ldc, ldc, bias, relu, gate, tc_error_flag()};
  if (!g.err) return cudaErrorMemoryAllocation;
  md->launches++;
  return tc_gemm_bf16(A, lda, B, ldb, g, md->st);
}

static cudaError_t transpose(tns_made* md, const bf16* in, long long ldi, int rows, int cols, bf16* out,
                             long long ldo) {
  md->launches++;
  return bf16_transpose(in, ldi, rows, cols, out, ldo, md->st);
}

struct MadeBufs {
  bf16 *X, *A1, *A2, *A3, *dLb, *dZb, *T1, *T2;
  float *Z1, *Z2, *Z3, *L, *dLf, *dZf;
  uint8_t* xb;
  double* logg;
  long long Bp;                    // pitch of the transposed activation copies T1, T2
};

static tns_status made_bufs(tns_made* md, long long B, MadeBufs& b) {
  const long long n = md->n, np = md->np, hp = md->hp;
  const long long rmax = std::max<long long>(np, hp);
  b.Bp = round8(B);
  auto get = [&](const char* nm, size_t bytes, void** p) { return md->ws.get(nm, bytes, p); };
  TNS_TRY_CUDA(get("X", sizeof(bf16) * B * np, (void**)&b.X));
  TNS_TRY_CUDA(get("A1", sizeof(bf16) * B * hp, (void**)&b.A1));
  TNS_TRY_CUDA(get("A2", sizeof(bf16) * B * hp, (void**)&b.A2));
  TNS_TRY_CUDA(get("A3", sizeof(bf16) * B * hp, (void**)&b.A3));
  TNS_TRY_CUDA(get("dLb", sizeof(bf16) * B * np, (void**)&b.dLb));
  TNS_TRY_CUDA(get("dZb", sizeof(bf16) * B * hp, (void**)&b.dZb));
  TNS_TRY_CUDA(get("T1", sizeof(bf16) * rmax * b.Bp, (void**)&b.T1));
  TNS_TRY_CUDA(get("T2", sizeof(bf16) * rmax * b.Bp, (void**)&b.T2));
  TNS_TRY_CUDA(get("Z1", sizeof(float) * B * hp, (void**)&b.Z1));
  TNS_TRY_CUDA(get("Z2", sizeof(float) * B * hp, (void**)&b.Z2));
  TNS_TRY_CUDA(get("Z3", sizeof(float) * B * hp, (void**)&b.Z3));
  TNS_TRY_CUDA(get("L", sizeof(float) * B * np, (void**)&b.L));
  TNS_TRY_CUDA(get("dLf", sizeof(float) * B * np, (void**)&b.dLf));
  TNS_TRY_CUDA(get("dZf", sizeof(float) * B * hp, (void**)&b.dZf));
  TNS_TRY_CUDA(get("xb", B * n, (void**)&b.xb));
  TNS_TRY_CUDA(get("logg", sizeof(double) * B, (void**)&b.logg));
  return TNS_OK;
}

// Masked BF16 weights and the transposes the backward pass reads.
static tns_status prep_weights(tns_made* md) {
  made_prep_weights_kernel<<<blk((long long)md->h * md->h), 256, 0, md->st>>>(md->theta, layout(md), md->wb, md->woff[0],
                                                                            md->woff[1], md->woff[2], md->woff[3]);
  md->launches++;
  TNS_TRY_CUDA(cudaGetLastError());
  const int n = md->n, h = md->h;
  TNS_TRY_CUDA(transpose(md, md->wb + md->woff[1], md->hp, h, h, md->wb + md->wtoff[0], md->hp));
  TNS_TRY_CUDA(transpose(md, md->wb + md->woff[2], md->hp, h, h, md->wb + md->wtoff[1], md->hp));
  TNS_TRY_CUDA(transpose(md, md->wb + md->woff[3], md->hp, n, h, md->wb + md->wtoff[2], md->np));
  return TNS_OK;
}

// Forward pass of B rows held in b.X: Z1..Z3 (FP32), A1..A3 (BF16 relu), logits L.
static tns_status forward(tns_made* md, int B, MadeBufs& b) {
  const int n = md->n, h = md->h;
  const long long np = md->np, hp = md->hp;
  const float* th = md->theta;
  TNS_TRY_CUDA(gemm(md, B, h, n, b.X, np, md->wb + md->woff[0], np, b.Z1, b.A1, hp, th + md->off[1], 1, nullptr));
  TNS_TRY_CUDA(gemm(md, B, h, h, b.A1, hp, md->wb + md->woff[1], hp, b.Z2, b.A2, hp, th + md->off[3], 1, nullptr));
  TNS_TRY_CUDA(gemm(md, B, h, h, b.A2, hp, md->wb + md->woff[2], hp, b.Z3, b.A3, hp, th + md->off[5], 1, nullptr));
  TNS_TRY_CUDA(gemm(md, B, n, h, b.A3, hp, md->wb + md->woff[3], hp, b.L, nullptr, np, th + md->off[7], 0, nullptr));
  return TNS_OK;
}

// Gradient of the mean NLL of the B rows in b.X / b.xb into md->grad; row log g into b.logg.
// Weight gradients dW = dZ^T A contract over the batch: both operands are read from
// transposed copies (rows = output units, contiguous batch index).
static tns_status backward(tns_made* md, int B, MadeBufs& b) {
  const int n = md->n, h = md->h;
  const long long np = md->np, hp = md->hp, Bp = b.Bp;
  float* g = md->grad;
  made_loss_grad_kernel<<<blk(B), 256, 0, md->st>>>(b.L, b.xb, B, n, md->np, b.logg, b.dLf, b.dLb);
  md->launches++;
  // layer 4: dW4 = dL^T A3, db4 = colsum dL, dZ3 = (dL W4) * [Z3 > 0]
  TNS_TRY_CUDA(transpose(md, b.dLb, np, B, n, b.T1, Bp));
  TNS_TRY_CUDA(transpose(md, b.A3, hp, B, h, b.T2, Bp));
  TNS_TRY_CUDA(gemm(md, n, h, B, b.T1, Bp, b.T2, Bp, g + md->off[6], nullptr, h, nullptr, 0, nullptr));
  colsum_kernel<<<blk(n), 256, 0, md->st>>>(b.dLf, B, n, np, g + md->off[7]);
  TNS_TRY_CUDA(gemm(md, B, h, n, b.dLb, np, md->wb + md->wtoff[2], np, b.dZf, b.dZb, hp, nullptr, 0, b.Z3));
  // layer 3
  TNS_TRY_CUDA(transpose(md, b.dZb, hp, B, h, b.T1, Bp));
  TNS_TRY_CUDA(transpose(md, b.A2, hp, B, h, b.T2, Bp));
  TNS_TRY_CUDA(gemm(md, h, h, B, b.T1, Bp, b.T2, Bp, g + md->off[4], nullptr, h, nullptr, 0, nullptr));
  colsum_kernel<<<blk(h), 256, 0, md->st>>>(b.dZf, B, h, hp, g + md->off[5]);
  // dZ2 = (dZ3 W3) * [Z2 > 0]; A3 is no longer needed and holds the BF16 copy of dZ2
  TNS_TRY_CUDA(gemm(md, B, h, h, b.dZb, hp, md->wb + md->wtoff[1], hp, b.dZf, b.A3, hp, nullptr, 0, b.Z2));
  TNS_TRY_CUDA(transpose(md, b.A3, hp, B, h, b.T1, Bp));
  TNS_TRY_CUDA(transpose(md, b.A1, hp, B, h, b.T2, Bp));
  TNS_TRY_CUDA(gemm(md, h, h, B, b.T1, Bp, b.T2, Bp, g + md->off[2], nullptr, h, nullptr, 0, nullptr));
  colsum_kernel<<<blk(h), 256, 0, md->st>>>(b.dZf, B, h, hp, g + md->off[3]);
  // dZ1 = (dZ2 W2) * [Z1 > 0]
  TNS_TRY_CUDA(gemm(md, B, h, h, b.A3, hp, md->wb + md->wtoff[0], hp, b.dZf, b.dZb, hp, nullptr, 0, b.Z1));
  TNS_TRY_CUDA(transpose(md, b.dZb, hp, B, h, b.T1, Bp));
  TNS_TRY_CUDA(transpose(md, b.X, np, B, n, b.T2, Bp));
  TNS_TRY_CUDA(gemm(md, h, n, B, b.T1, Bp, b.T2, Bp, g + md->off[0], nullptr, n, nullptr, 0, nullptr));
  colsum_kernel<<<blk(h), 256, 0, md->st>>>(b.dZf, B, h, hp, g + md->off[1]);
  made_mask_grad_kernel<<<blk((long long)h * h), 256, 0, md->st>>>(g, layout(md));
  md->launches += 5;
  TNS_TRY_CUDA(cudaGetLastError());
  return TNS_OK;
}

// Reads and clears the tensor-core timeout flag after the stream has drained.
static tns_status check_tc_flag() {
  int* f = tc_error_flag();
  if (!f) return TNS_OK;
  int hf = 0;
  TNS_TRY_CUDA(cudaMemcpy(&hf, f, sizeof(int), cudaMemcpyDeviceToHost));
  if (!hf) return TNS_OK;
  TNS_TRY_CUDA(cudaMemset(f, 0, sizeof(int)));
  set_error("tensor-core GEMM pipeline wait timed out");
  return TNS_ERR_NUMERIC;
}

}  // namespace tns

using namespace tns;

extern "C" tns_status tns_made_create(int32_t n_sites, int32_t hidden, const float* params_host, void* stream,
                                      tns_made** out) {
  if (!out || n_sites < 2 || hidden < 1 || !params_host) { set_error("invalid argument to tns_made_create"); return TNS_ERR_ARG; }
  *out = nullptr;
  tns_made* md = new tns_made();
  md->n = n_sites;
  md->h = hidden;
  md->st = (cudaStream_t)stream;
  const long long n = n_sites, h = hidden;
  const long long sz[8] = {h * n, h, h * h, h, h * h, h, n * h, n};
  long long o = 0;
  for (int i = 0; i < 8; ++i) { md->off[i] = o; o += sz[i]; }
  md->P = o;
  md->np = (int)round8(n);
  md->hp = (int)round8(h);
  const long long np = md->np, hp = md->hp;
  // every block starts on a multiple of 8 elements (16 bytes) for the TMA descriptors
  md->woff[0] = 0;
  md->woff[1] = md->woff[0] + h * np;
  md->woff[2] = md->woff[1] + h * hp;
  md->woff[3] = md->woff[2] + h * hp;
  md->wtoff[0] = md->woff[3] + n * hp;
  md->wtoff[1] = md->wtoff[0] + h * hp;
  md->wtoff[2] = md->wtoff[1] + h * hp;
  const long long nw = md->wtoff[2] + h * np;
  cudaError_t e = cudaMalloc(&md->theta, sizeof(float) * md->P);
  if (e == cudaSuccess) e = cudaMalloc(&md->m, sizeof(float) * md->P);
  if (e == cudaSuccess) e = cudaMalloc(&md->v, sizeof(float) * md->P);
  if (e == cudaSuccess) e = cudaMalloc(&md->grad, sizeof(float) * md->P);
  if (e == cudaSuccess) e = cudaMalloc(&md->wb, sizeof(bf16) * nw);
  if (e == cudaSuccess) e = cudaMemcpy(md->theta, params_host, sizeof(float) * md->P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemsetAsync(md->m, 0, sizeof(float) * md->P, md->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(md->v, 0, sizeof(float) * md->P, md->st);
  if (e != cudaSuccess) { tns_status r = cuda_status(e, "tns_made_create"); tns_made_destroy(md); return r; }
  tns_status r = prep_weights(md);
  if (r != TNS_OK) { tns_made_destroy(md); return r; }
  *out = md;
  return TNS_OK;
}

extern "C" void tns_made_destroy(tns_made* md) {
  if (!md) return;
  cudaStreamSynchronize(md->st);
  cudaFree(md->theta);
  cudaFree(md->m);
  cudaFree(md->v);
  cudaFree(md->grad);
  cudaFree(md->wb);
  md->ws.release();
  delete md;
}

extern "C" tns_status tns_made_params(const tns_made* md, float* params_host) {
  if (!md || !params_host) { set_error("invalid argument to tns_made_params"); return TNS_ERR_ARG; }
  TNS_TRY_CUDA(cudaStreamSynchronize(md->st));
  TNS_TRY_CUDA(cudaMemcpy(params_host, md->theta, sizeof(float) * md->P, cudaMemcpyDeviceToHost));
  return TNS_OK;
}

extern "C" tns_status tns_made_logprob(tns_made* md, const uint8_t* bits_dev, int64_t n, double* logg_dev) {
  if (!md || n < 0 || (n > 0 && (!bits_dev || !logg_dev))) { set_error("invalid argument to tns_made_logprob"); return TNS_ERR_ARG; }
  const long long CH = 65536;
  MadeBufs b;
  TNS_TRY(made_bufs(md, std::min<long long>(std::max<long long>(n, 1), CH), b));
  for (long long s0 = 0; s0 < n; s0 += CH) {
    const int B = (int)std::min<long long>(CH, n - s0);
    made_gather_bits_kernel<<<blk((long long)B * md->n), 256, 0, md->st>>>(bits_dev, nullptr, s0, B, md->n, md->np,
                                                                           b.X, b.xb);
    TNS_TRY(forward(md, B, b));
    made_loss_grad_kernel<<<blk(B), 256, 0, md->st>>>(b.L, b.xb, B, md->n, md->np, logg_dev + s0, nullptr, nullptr);
    md->launches += 2;
  }
  TNS_TRY_CUDA(cudaGetLastError());
  TNS_TRY_CUDA(cudaStreamSynchronize(md->st));
  return check_tc_flag();
}

extern "C" tns_status tns_made_grad(tns_made* md, const uint8_t* bits_dev, int64_t n, float* grad_host, double* loss) {
  if (!md || n < 1 || n > (1 << 20) || !bits_dev) { set_error("invalid argument to tns_made_grad"); return TNS_ERR_ARG; }
  MadeBufs b;
  TNS_TRY(made_bufs(md, n, b));
  made_gather_bits_kernel<<<blk(n * md->n), 256, 0, md->st>>>(bits_dev, nullptr, 0, (int)n, md->n, md->np, b.X, b.xb);
  TNS_TRY(forward(md, (int)n, b));
  TNS_TRY(backward(md, (int)n, b));
  std::vector<double> lg(n);
  TNS_TRY_CUDA(cudaMemcpyAsync(lg.data(), b.logg, sizeof(double) * n, cudaMemcpyDeviceToHost, md->st));
  if (grad_host) TNS_TRY_CUDA(cudaMemcpyAsync(grad_host, md->grad, sizeof(float) * md->P, cudaMemcpyDeviceToHost, md->st));
  TNS_TRY_CUDA(cudaStreamSynchronize(md->st));
  TNS_TRY(check_tc_flag());
  if (loss) {
    double s = 0;
    for (double x : lg) s -= x;
    *loss = s / n;
  }
  return TNS_OK;
}

extern "C" tns_status tns_made_train(tns_made* md, const uint8_t* bits_dev, int64_t n, int32_t batch, int32_t epochs,
                                     const int32_t* orders_host, float lr, double* loss_host) {
  if (!md || n < 1 || batch < 1 || epochs < 0 || !bits_dev || !(lr > 0)) { set_error("invalid argument to tns_made_train"); return TNS_ERR_ARG; }
  MadeBufs b;
  TNS_TRY(made_bufs(md, std::min<long long>(batch, n), b));
  int32_t* order = nullptr;
  if (orders_host) TNS_TRY_CUDA(md->ws.get("order", sizeof(int32_t) * n * epochs, (void**)&order));
  if (orders_host)
    TNS_TRY_CUDA(cudaMemcpyAsync(order, orders_host, sizeof(int32_t) * n * epochs, cudaMemcpyHostToDevice, md->st));
  double* lsum = nullptr;
  TNS_TRY_CUDA(md->ws.get("lsum", sizeof(double) * n, (void**)&lsum));
  std::vector<double> rows(n);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int e = 0; e < epochs; ++e) {
    for (long long i0 = 0; i0 < n; i0 += batch) {
      const int B = (int)std::min<long long>(batch, n - i0);
      made_gather_bits_kernel<<<blk((long long)B * md->n), 256, 0, md->st>>>(
          bits_dev, order ? order + (long long)e * n : nullptr, i0, B, md->n, md->np, b.X, b.xb);
      md->launches++;
      TNS_TRY(forward(md, B, b));
      TNS_TRY(backward(md, B, b));
      TNS_TRY_CUDA(cudaMemcpyAsync(lsum + i0, b.logg, sizeof(double) * B, cudaMemcpyDeviceToDevice, md->st));
      md->t += 1;
      const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)md->t)));
      const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)md->t)));
      made_adam_kernel<<<blk(md->P), 256, 0, md->st>>>(md->theta, md->m, md->v, md->grad, md->P, lr, b1, b2, eps, c1,
                                                       c2);
      md->launches++;
      TNS_TRY(prep_weights(md));
    }
    TNS_TRY_CUDA(cudaMemcpyAsync(rows.data(), lsum, sizeof(double) * n, cudaMemcpyDeviceToHost, md->st));
    TNS_TRY_CUDA(cudaStreamSynchronize(md->st));
    if (loss_host) {
      double s = 0;
      for (double x : rows) s -= x;
      loss_host[e] = s / n;
    }
  }
  TNS_TRY_CUDA(cudaGetLastError());
  TNS_TRY_CUDA(cudaStreamSynchronize(md->st));
  return check_tc_flag();
}

extern "C" tns_status tns_made_sample(tns_made* md, int64_t n, uint64_t seed, uint8_t* bits_dev, double* logg_dev) {
  if (!md || n < 0 || (n > 0 && (!bits_dev || !logg_dev))) { set_error("invalid argument to tns_made_sample"); return TNS_ERR_ARG; }
  const long long CH = 65536;
  MadeBufs b;
  TNS_TRY(made_bufs(md, std::min<long long>(std::max<long long>(n, 1), CH), b));
  TNS_TRY_CUDA(cudaMemsetAsync(logg_dev, 0, sizeof(double) * n, md->st));
  for (long long s0 = 0; s0 < n; s0 += CH) {
    const int B = (int)std::min<long long>(CH, n - s0);
    TNS_TRY_CUDA(cudaMemsetAsync(b.X, 0, sizeof(bf16) * B * md->np, md->st));
    for (int i = 0; i < md->n; ++i) {
      TNS_TRY(forward(md, B, b));
      made_draw_kernel<<<blk(B), 256, 0, md->st>>>(b.L, B, md->n, md->np, i, seed, s0, b.X, bits_dev, logg_dev);
      md->launches++;
    }
  }
  TNS_TRY_CUDA(cudaGetLastError());
  TNS_TRY_CUDA(cudaStreamSynchronize(md->st));
  return check_tc_flag();
}

extern "C" tns_status tns_mh_independent(int32_t n_chains, int32_t n_steps, const double* logp_prop_dev,
                                         const double* logg_prop_dev, const double* logp0_dev, const double* logg0_dev,
                                         uint64_t seed, int32_t* state_dev, int64_t* accepted_dev, void* stream) {
  if (n_chains < 0 || n_steps < 0 || (n_chains > 0 && !accepted_dev) ||
      (n_chains > 0 && n_steps > 0 && (!logp_prop_dev || !logg_prop_dev || !logp0_dev || !logg0_dev || !state_dev))) {
    set_error("invalid argument to tns_mh_independent");
    return TNS_ERR_ARG;
  }
  if (n_chains == 0) return TNS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (n_steps == 0) {
    TNS_TRY_CUDA(cudaMemsetAsync(accepted_dev, 0, sizeof(int64_t) * n_chains, st));
    TNS_TRY_CUDA(cudaStreamSynchronize(st));
    return TNS_OK;
  }
  mh_kernel<<<(n_chains + 127) / 128, 128, 0, st>>>(n_chains, n_steps, logp_prop_dev, logg_prop_dev, logp0_dev,
                                                    logg0_dev, seed, state_dev, accepted_dev);
  TNS_TRY_CUDA(cudaGetLastError());
  TNS_TRY_CUDA(cudaStreamSynchronize(st));
  return TNS_OK;
}
