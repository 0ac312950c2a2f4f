// Test-only entry points (include/tns_testing.h): device primitives exposed
// through the C ABI so they can be compared with the CPU oracle in isolation.
#include "../../include/tns_testing.h"
#include "linalg.cuh"
#include "tc_gemm.cuh"
#include "contract.cuh"
#include "state.h"

#include <vector>

namespace tns {
__global__ void philox_test_kernel(long long n, const uint32_t* ck, uint32_t* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* c = ck + 6 * i;
  Philox4 w = philox4x32_10(c[0], c[1], c[2], c[3], c[4], c[5]);
  for (int k = 0; k < 4; ++k) out[4 * i + k] = w.v[k];
}
}  // namespace tns

using namespace tns;

extern "C" tns_status tns_test_philox(int64_t n, const uint32_t* ck, uint32_t* out, void* stream) {
  if (n < 0 || (n > 0 && (!ck || !out))) { set_error("invalid argument"); return TNS_ERR_ARG; }
  if (n == 0) return TNS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  philox_test_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ck, out);
  TNS_TRY_CUDA(cudaGetLastError());
  TNS_TRY_CUDA(cudaStreamSynchronize(st));
  return TNS_OK;
}

static std::vector<int> g_last_sweeps;

extern "C" tns_status tns_test_eigh(int32_t batch, int32_t n, const double* A, double* lam, double* V, void* stream) {
  if (batch < 0 || n < 1 || n > 512 || !A || !lam || !V) { set_error("invalid argument"); return TNS_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  cd* work = nullptr;
  int* status = nullptr;
  int* sweeps = nullptr;
  TNS_TRY_CUDA(cudaMalloc(&status, sizeof(int) * (batch > 0 ? batch : 1)));
  TNS_TRY_CUDA(cudaMalloc(&sweeps, sizeof(int) * (batch > 0 ? batch : 1)));
  if (!eigh_fits_smem(n)) {
    long long np = n + (n & 1);
    TNS_TRY_CUDA(cudaMalloc(&work, sizeof(cd) * batch * 2 * np * np));
  }
  cudaError_t e = eigh_batched((cd*)A, (long long)n * n, n, n, batch, lam, (cd*)V, (long long)n * n, work, status, st,
                               sweeps);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  std::vector<int> hs(batch > 0 ? batch : 1), hw(batch > 0 ? batch : 1);
  if (e == cudaSuccess && batch > 0) {
    cudaMemcpy(hs.data(), status, sizeof(int) * batch, cudaMemcpyDeviceToHost);
    cudaMemcpy(hw.data(), sweeps, sizeof(int) * batch, cudaMemcpyDeviceToHost);
    g_last_sweeps.assign(batch, 0);
    for (int b = 0; b < batch; ++b) g_last_sweeps[b] = hs[b] == 0 ? hw[b] : -hw[b];
  }
  cudaFree(work);
  cudaFree(status);
  cudaFree(sweeps);
  TNS_TRY_CUDA(e);
  return TNS_OK;
}

extern "C" tns_status tns_test_eigh32(int32_t batch, int32_t n, const float* A, double* lam, double* V,
                                      void* stream) {
  if (batch < 0 || n < 1 || n > 512 || !A || !lam || !V) { set_error("invalid argument"); return TNS_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  cf* work = nullptr;
  int* status = nullptr;
  int* sweeps = nullptr;
  TNS_TRY_CUDA(cudaMalloc(&status, sizeof(int) * (batch > 0 ? batch : 1)));
  TNS_TRY_CUDA(cudaMalloc(&sweeps, sizeof(int) * (batch > 0 ? batch : 1)));
  if (!jacobi_fits_smem_f32(n)) {
    long long np = n + (n & 1);
    TNS_TRY_CUDA(cudaMalloc(&work, sizeof(cf) * batch * 2 * np * np));
  }
  cudaError_t e = eigh_batched_f32((const cf*)A, (long long)n * n, n, n, batch, lam, (cd*)V, (long long)n * n, work,
                                   status, st, sweeps);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  std::vector<int> hs(batch > 0 ? batch : 1), hw(batch > 0 ? batch : 1);
  if (e == cudaSuccess && batch > 0) {
    cudaMemcpy(hs.data(), status, sizeof(int) * batch, cudaMemcpyDeviceToHost);
    cudaMemcpy(hw.data(), sweeps, sizeof(int) * batch, cudaMemcpyDeviceToHost);
    g_last_sweeps.assign(batch, 0);
    for (int b = 0; b < batch; ++b) g_last_sweeps[b] = hs[b] == 0 ? hw[b] : -hw[b];
  }
  cudaFree(work);
  cudaFree(status);
  cudaFree(sweeps);
  TNS_TRY_CUDA(e);
  return TNS_OK;
}

extern "C" tns_status tns_test_eigh_sweeps(int32_t batch, int32_t* out) {
  if (!out || batch < 0 || (size_t)batch > g_last_sweeps.size()) { set_error("invalid argument"); return TNS_ERR_ARG; }
  for (int b = 0; b < batch; ++b) out[b] = g_last_sweeps[b];
  return TNS_OK;
}

extern "C" tns_status tns_test_cholw(int32_t batch, int32_t n, double shift, const double* G, double* W, void* stream) {
  if (batch < 0 || n < 1 || !G || !W || !(shift > 0.0)) { set_error("invalid argument"); return TNS_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  cd* work = nullptr;
  if (!chol_fits_smem(n)) TNS_TRY_CUDA(cudaMalloc(&work, sizeof(cd) * batch * 2 * (long long)n * n));
  cudaError_t e = chol_w_batched(G, true, n, batch, shift, W, true, work, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(work);
  TNS_TRY_CUDA(e);
  return TNS_OK;
}

extern "C" tns_status tns_test_svd(int32_t batch, int32_t m, int32_t n, const double* A, double* s, double* U,
                                   double* V, void* stream) {
  if (batch < 0 || n < 1 || m < n || n > 1024 || !A || !s || !U || !V) { set_error("invalid argument"); return TNS_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  cd* work = nullptr;
  int* status = nullptr;
  TNS_TRY_CUDA(cudaMalloc(&status, sizeof(int) * (batch > 0 ? batch : 1)));
  if (!jacobi_fits_smem(m, n)) {
    long long np = n + (n & 1);
    TNS_TRY_CUDA(cudaMalloc(&work, sizeof(cd) * batch * ((long long)m * np + np * np)));
  }
  cudaError_t e = svd_batched((cd*)A, (long long)m * n, n, m, n, batch, s, (cd*)U, (long long)m * n, (cd*)V,
                              (long long)n * n, work, status, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(work);
  cudaFree(status);
  TNS_TRY_CUDA(e);
  return TNS_OK;
}

extern "C" tns_status tns_test_tcgemm(int64_t M, int32_t N, int32_t K, const float* A, const float* B, float* C,
                                      void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) { set_error("invalid argument"); return TNS_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  ContractTiming tm;
  tm.force_tc = true;
  cudaError_t e = contract(view((void*)A, "mk", {M, K}), view((void*)B, "nk", {N, K}), view(C, "mn", {M, N}),
                           Prec::TF32X3, st, make_double2(1.0, 0.0), make_double2(0.0, 0.0), nullptr, &tm);
  if (e == cudaErrorNotSupported) { set_error("shape not supported by the tensor-core path"); return TNS_ERR_STATE; }
  TNS_TRY_CUDA(e);
  TNS_TRY_CUDA(cudaStreamSynchronize(st));
  int* f = tc_error_flag();
  int herr = 0;
  if (f) {
    TNS_TRY_CUDA(cudaMemcpy(&herr, f, sizeof(int), cudaMemcpyDeviceToHost));
    TNS_TRY_CUDA(cudaMemset(f, 0, sizeof(int)));
  }
  if (herr) { set_error("tensor-core GEMM pipeline wait timed out"); return TNS_ERR_NUMERIC; }
  return TNS_OK;
}

extern "C" tns_status tns_test_tc_tile(int32_t bn) {
  if (bn != 0 && bn != 128 && bn != 256 && bn != TC_TILE_128_SINGLE) {
    set_error("tile variant must be 0, 128, 129 or 256");
    return TNS_ERR_ARG;
  }
  tc_force_tile(bn);
  return TNS_OK;
}

extern "C" tns_status tns_test_contract(const char* labels_a, const int64_t* dims_a, const int64_t* strides_a,
                                        int32_t conj_a, const void* A, const char* labels_b, const int64_t* dims_b,
                                        const int64_t* strides_b, int32_t conj_b, const void* B, const char* labels_c,
                                        const int64_t* dims_c, const int64_t* strides_c, void* C, int32_t mode,
                                        void* stream) {
  if (!labels_a || !labels_b || !labels_c || !A || !B || !C || mode < 0 || mode > 2) {
    set_error("invalid argument");
    return TNS_ERR_ARG;
  }
  auto mk = [](const char* lab, const int64_t* d, const int64_t* st, int cj, const void* p) {
    TView v;
    v.ptr = const_cast<void*>(p);
    v.labels = lab;
    for (size_t i = 0; i < v.labels.size(); ++i) {
      v.dim.push_back(d[i]);
      v.stride.push_back(st[i]);
    }
    v.conj = cj != 0;
    return v;
  };
  cudaStream_t st = (cudaStream_t)stream;
  ContractTiming tm;
  tm.force_tc = (mode == 1);
  const Prec pr = mode == 0 ? Prec::F32 : (mode == 1 ? Prec::TF32X3 : Prec::F64);
  cudaError_t e = contract(mk(labels_a, dims_a, strides_a, conj_a, A), mk(labels_b, dims_b, strides_b, conj_b, B),
                           mk(labels_c, dims_c, strides_c, 0, C), pr, st, make_double2(1.0, 0.0),
                           make_double2(0.0, 0.0), nullptr, &tm);
  if (e == cudaErrorNotSupported) { set_error("contraction not supported by the tensor-core path"); return TNS_ERR_STATE; }
  if (e == cudaErrorInvalidValue) { set_error("inconsistent contraction views"); return TNS_ERR_ARG; }
  TNS_TRY_CUDA(e);
  TNS_TRY_CUDA(cudaStreamSynchronize(st));
  if (mode == 1) {
    int* f = tc_error_flag();
    int herr = 0;
    if (f) {
      TNS_TRY_CUDA(cudaMemcpy(&herr, f, sizeof(int), cudaMemcpyDeviceToHost));
      TNS_TRY_CUDA(cudaMemset(f, 0, sizeof(int)));
    }
    if (herr) { set_error("tensor-core GEMM pipeline wait timed out"); return TNS_ERR_NUMERIC; }
  }
  return TNS_OK;
}

extern "C" tns_status tns_test_plan(const char* labels_a, const int64_t* dims_a, const int64_t* strides_a,
                                    int32_t conj_a, const char* labels_b, const int64_t* dims_b,
                                    const int64_t* strides_b, int32_t conj_b, const char* labels_c,
                                    const int64_t* dims_c, const int64_t* strides_c, int64_t* out) {
  if (!labels_a || !labels_b || !labels_c || !dims_a || !dims_b || !dims_c || !strides_a || !strides_b ||
      !strides_c || !out) {
    set_error("invalid argument");
    return TNS_ERR_ARG;
  }
  auto mk = [](const char* lab, const int64_t* d, const int64_t* st, int cj) {
    TView v;
    v.labels = lab;
    for (size_t i = 0; i < v.labels.size(); ++i) {
      v.dim.push_back(d[i]);
      v.stride.push_back(st[i]);
    }
    v.conj = cj != 0;
    return v;
  };
  long long o[11];
  cudaError_t e = contract_plan(mk(labels_a, dims_a, strides_a, conj_a), mk(labels_b, dims_b, strides_b, conj_b),
                                mk(labels_c, dims_c, strides_c, 0), o);
  if (e != cudaSuccess) { set_error("inconsistent contraction views"); return TNS_ERR_ARG; }
  for (int i = 0; i < 11; ++i) out[i] = o[i];
  return TNS_OK;
}

extern "C" tns_status tns_test_env_site(tns_state* s, int32_t b, int32_t k, int64_t* dims_out, int32_t* reversed_out,
                                        double* out_host) {
  if (!s || !dims_out) { set_error("invalid argument"); return TNS_ERR_ARG; }
  const EnvCache& ec = s->env;
  if (!ec.valid) { set_error("no environment cached"); return TNS_ERR_STATE; }
  if (b < 0 || b >= (int)ec.E.size() || k < 0 || k >= (int)ec.E[b].site.size()) {
    set_error("env site index out of range");
    return TNS_ERR_ARG;
  }
  const StoredMPS& m = ec.E[b];
  if (m.phys[k].size() != 2) { set_error("env site with %zu physical legs", m.phys[k].size()); return TNS_ERR_STATE; }
  dims_out[0] = m.bond[k];
  dims_out[1] = m.phys[k][0];
  dims_out[2] = m.phys[k][1];
  dims_out[3] = m.bond[k + 1];
  if (reversed_out) *reversed_out = m.reversed ? 1 : 0;
  if (!out_host) return TNS_OK;
  const long long n = dims_out[0] * dims_out[1] * dims_out[2] * dims_out[3];
  TNS_TRY_CUDA(cudaStreamSynchronize(s->st));
  if (ec.prec == 0) {
    TNS_TRY_CUDA(cudaMemcpy(out_host, m.site[k], sizeof(cd) * n, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(2 * n);
    TNS_TRY_CUDA(cudaMemcpy(tmp.data(), m.site[k], sizeof(cf) * n, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < 2 * n; ++i) out_host[i] = tmp[i];
  }
  return TNS_OK;
}
