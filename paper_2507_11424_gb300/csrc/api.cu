// C ABI entry points: state construction, persistence, queries (include/tns.h).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <set>

#include "state.h"

namespace tns {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

tns_status cuda_status(cudaError_t e, const char* where) {
  set_error("CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), where);
  return e == cudaErrorMemoryAllocation ? TNS_ERR_OOM : TNS_ERR_CUDA;
}

cudaError_t Workspace::get(const std::string& name, size_t bytes, void** out) {
  auto it = slots.find(name);
  if (it != slots.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return cudaSuccess;
  }
  if (it != slots.end()) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    cudaFree(it->second.first);
    slots.erase(it);
    ++gen;
  }
  void* p = nullptr;
  size_t nb = bytes < 256 ? 256 : bytes;
  cudaError_t e = cudaMalloc(&p, nb);
  if (e != cudaSuccess) return e;
  slots[name] = std::make_pair(p, nb);
  *out = p;
  return cudaSuccess;
}

cudaEvent_t Profiler::begin(cudaStream_t st) {
  if (!on) return nullptr;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, st);
  return e;
}

void Profiler::end(int cls, cudaEvent_t a, double fl, cudaStream_t st) {
  if (!on || !a) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaEventDestroy(a); return; }
  cudaEventRecord(e, st);
  pending.push_back({cls, a, e, fl});
}

void Profiler::span(int cls, cudaEvent_t a, cudaEvent_t b, double fl, bool own_a, bool own_b) {
  if (!on || !a || !b) return;
  Rec r{cls, a, b, fl};
  r.own_a = own_a;
  r.own_b = own_b;
  pending.push_back(r);
}

void Profiler::resolve() {
  for (auto& r : pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms[r.cls] += t;
      flops[r.cls] += r.flops;
      n[r.cls] += 1;
    }
  }
  // destroy after every interval is read (an event may end one span and start the next)
  for (auto& r : pending) {
    if (r.own_a) cudaEventDestroy(r.a);
    if (r.own_b) cudaEventDestroy(r.b);
  }
  pending.clear();
}

void Profiler::clear() {
  resolve();
  for (int i = 0; i < NCLASS; ++i) { ms[i] = 0; flops[i] = 0; n[i] = 0; }
}

void Workspace::release() {
  for (auto& kv : slots) cudaFree(kv.second.first);
  slots.clear();
}

__global__ void init_product_kernel(cd* t, int bit) {
  t[0] = mk(bit == 0 ? 1.0 : 0.0, 0.0);
  t[1] = mk(bit == 1 ? 1.0 : 0.0, 0.0);
}
__global__ void fill_one_kernel(cd* t) { t[0] = mk(1.0, 0.0); }

// Cells and messages live in two arenas so batched kernels can gather them by offset.
static tns_status alloc_state(tns_state* s) {
  const int nc = s->H * s->W;
  s->msg.assign((size_t)nc * 5, nullptr);
  s->msg_new.assign((size_t)nc * 5, nullptr);
  long long total = 0;
  for (int ci = 0; ci < nc; ++ci) {
    Cell& c = s->cell[ci];
    long long cap = (c.qubit >= 0) ? 2 : 1;
    for (int leg = 1; leg <= 4; ++leg) cap *= c.edge[leg] ? s->chi_max : 1;
    c.cap = cap;
    c.off = total;
    total += (cap + 31) / 32 * 32;
  }
  TNS_TRY_CUDA(cudaMalloc(&s->cell_arena, sizeof(cd) * total));
  const long long mslot = (long long)s->chi_max * s->chi_max;
  TNS_TRY_CUDA(cudaMalloc(&s->msg_arena, sizeof(cd) * mslot * nc * 5));
  TNS_TRY_CUDA(cudaMalloc(&s->msg_new_arena, sizeof(cd) * mslot * nc * 5));
  for (int ci = 0; ci < nc; ++ci) {
    Cell& c = s->cell[ci];
    c.t = s->cell_arena + c.off;
    for (int leg = 1; leg <= 4; ++leg) {
      if (!c.edge[leg]) continue;
      s->msg[ci * 5 + leg] = s->msg_arena + (long long)(ci * 5 + leg) * mslot;
      s->msg_new[ci * 5 + leg] = s->msg_new_arena + (long long)(ci * 5 + leg) * mslot;
    }
  }
  return TNS_OK;
}

static void free_state(tns_state* s) {
  if (s->cell_arena) cudaFree(s->cell_arena);
  if (s->msg_arena) cudaFree(s->msg_arena);
  if (s->msg_new_arena) cudaFree(s->msg_new_arena);
  for (auto p : s->work_cells)
    if (p) cudaFree(p);
  for (auto& g : s->graphs)
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
  s->graphs.clear();
  for (auto& e : s->gev)
    if (e) cudaEventDestroy(e);
  if (s->gstream) cudaStreamDestroy(s->gstream);
  if (s->bp_host) cudaFreeHost(s->bp_host);
  s->bp_host = nullptr;
  for (auto e : s->gate_events)
    if (e) cudaEventDestroy(e);
  s->gate_events.clear();
  for (auto q : s->gate_streams)
    if (q) cudaStreamDestroy(q);
  s->gate_streams.clear();
  if (s->gate_host) cudaFreeHost(s->gate_host);
  s->gate_host = nullptr;
  for (auto* ec : {&s->env, &s->env_top})
    for (auto& E : ec->E)
      for (auto p : E.site)
        if (p) cudaFree(p);
  s->ws.release();
}

}  // namespace tns

using namespace tns;

extern "C" const char* tns_last_error(void) { return g_err; }

extern "C" tns_status tns_build_lattice(int32_t n_sites, const int32_t* grid_rc, int32_t n_edges,
                                        const int32_t* edges, const uint8_t* init_bits, int32_t chi_max,
                                        tns_prec prec, void* cuda_stream, tns_state** out) {
  if (!out) { set_error("out is NULL"); return TNS_ERR_ARG; }
  *out = nullptr;
  if (n_sites < 1 || !grid_rc || !init_bits || (n_edges > 0 && !edges) || n_edges < 0 || chi_max < 1 ||
      (prec != TNS_PREC_FP64 && prec != TNS_PREC_MIXED)) {
    set_error("invalid argument to tns_build_lattice");
    return TNS_ERR_ARG;
  }
  int H0 = 0, W0 = 0;
  for (int q = 0; q < n_sites; ++q) {
    if (grid_rc[2 * q] < 0 || grid_rc[2 * q + 1] < 0 || grid_rc[2 * q] > 4096 || grid_rc[2 * q + 1] > 4096) {
      set_error("grid coordinate of qubit %d out of range", q);
      return TNS_ERR_ARG;
    }
    if (init_bits[q] > 1) { set_error("init_bits[%d] is not 0/1", q); return TNS_ERR_ARG; }
    H0 = std::max(H0, grid_rc[2 * q] + 1);
    W0 = std::max(W0, grid_rc[2 * q + 1] + 1);
  }
  tns_state* s = new tns_state();
  s->transposed = W0 > H0;
  s->H = s->transposed ? W0 : H0;
  s->W = s->transposed ? H0 : W0;
  s->n = n_sites;
  s->chi_max = chi_max;
  s->prec = prec;
  s->st = (cudaStream_t)cuda_stream;
  cudaGetDevice(&s->device);
  s->cell.assign((size_t)s->H * s->W, Cell());
  s->qcell.assign(n_sites, -1);
  for (int q = 0; q < n_sites; ++q) {
    int r = grid_rc[2 * q], c = grid_rc[2 * q + 1];
    if (s->transposed) std::swap(r, c);
    int ci = s->cidx(r, c);
    if (s->cell[ci].qubit >= 0) {
      set_error("qubits %d and %d share grid cell", s->cell[ci].qubit, q);
      delete s;
      return TNS_ERR_ARG;
    }
    s->cell[ci].qubit = q;
    s->cell[ci].dim[0] = 2;
    s->qcell[q] = ci;
  }
  std::set<std::pair<int, int>> seen;
  for (int e = 0; e < n_edges; ++e) {
    int a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= n_sites || b >= n_sites || a == b) {
      set_error("edge %d has invalid qubits", e);
      delete s;
      return TNS_ERR_ARG;
    }
    if (!seen.insert({std::min(a, b), std::max(a, b)}).second) {
      set_error("duplicate edge %d", e);
      delete s;
      return TNS_ERR_ARG;
    }
    int ca = s->qcell[a], cb = s->qcell[b];
    int ra = ca / s->W, cca = ca % s->W, rb = cb / s->W, ccb = cb % s->W;
    int leg = -1;
    if (rb == ra - 1 && ccb == cca) leg = LEG_U;
    else if (rb == ra + 1 && ccb == cca) leg = LEG_D;
    else if (rb == ra && ccb == cca - 1) leg = LEG_L;
    else if (rb == ra && ccb == cca + 1) leg = LEG_R;
    if (leg < 0) {
      set_error("edge %d joins qubits %d,%d that are not grid neighbours", e, a, b);
      delete s;
      return TNS_ERR_ARG;
    }
    s->cell[ca].edge[leg] = true;
    s->cell[cb].edge[opp_leg(leg)] = true;
  }
  tns_status st = alloc_state(s);
  if (st != TNS_OK) {
    free_state(s);
    delete s;
    return st;
  }
  for (size_t ci = 0; ci < s->cell.size(); ++ci) {
    Cell& c = s->cell[ci];
    if (c.qubit >= 0) init_product_kernel<<<1, 1, 0, s->st>>>(c.t, init_bits[c.qubit]);
    else fill_one_kernel<<<1, 1, 0, s->st>>>(c.t);
    for (int leg = 1; leg <= 4; ++leg)
      if (c.edge[leg]) fill_one_kernel<<<1, 1, 0, s->st>>>(s->msg[ci * 5 + leg]);
  }
  cudaError_t e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) {
    tns_status r = cuda_status(e, "tns_build_lattice");
    free_state(s);
    delete s;
    return r;
  }
  *out = s;
  return TNS_OK;
}

extern "C" void tns_destroy(tns_state* s) {
  if (!s) return;
  cudaStreamSynchronize(s->st);
  free_state(s);
  delete s;
}

extern "C" tns_status tns_apply_gate_layer(tns_state* s, int32_t n_gates, const int32_t* sites, const double* mats,
                                           int32_t chi, double svd_cutoff, double* eps_out) {
  LaunchScope ls_(s);
  if (!s || n_gates < 0 || (n_gates > 0 && (!sites || !mats)) || chi < 1 || chi > s->chi_max ||
      !(svd_cutoff >= 0.0)) {
    set_error("invalid argument to tns_apply_gate_layer");
    return TNS_ERR_ARG;
  }
  return apply_gate_layer(s, n_gates, sites, mats, chi, svd_cutoff, eps_out);
}

extern "C" tns_status tns_bp_gauge(tns_state* s, int32_t max_iter, double tol, int32_t* iters_out,
                                   double* residual_out) {
  LaunchScope ls_(s);
  if (!s || max_iter < 1 || !(tol >= 0.0)) { set_error("invalid argument to tns_bp_gauge"); return TNS_ERR_ARG; }
  int it = 0;
  double res = 0.0;
  tns_status r = bp_gauge(s, max_iter, tol, &it, &res);
  if (iters_out) *iters_out = it;
  if (residual_out) *residual_out = res;
  return r;
}

extern "C" tns_status tns_sample(tns_state* s, int32_t chi_b, int64_t n_samples, uint64_t seed, uint8_t* bits_dev,
                                 double* logq_dev, double* cond_dev) {
  LaunchScope ls_(s);
  if (!s || chi_b < 1 || n_samples < 0 || (n_samples > 0 && (!bits_dev || !logq_dev))) {
    set_error("invalid argument to tns_sample");
    return TNS_ERR_ARG;
  }
  return sample(s, chi_b, n_samples, seed, nullptr, bits_dev, logq_dev, cond_dev);
}

extern "C" tns_status tns_sample_range(tns_state* s, int32_t chi_b, int64_t first, int64_t n_samples, uint64_t seed,
                                       uint8_t* bits_dev, double* logq_dev, double* cond_dev) {
  LaunchScope ls_(s);
  if (!s || chi_b < 1 || first < 0 || n_samples < 0 || (n_samples > 0 && (!bits_dev || !logq_dev))) {
    set_error("invalid argument to tns_sample_range");
    return TNS_ERR_ARG;
  }
  return sample(s, chi_b, n_samples, seed, nullptr, bits_dev, logq_dev, cond_dev, first);
}

extern "C" tns_status tns_sample_replay(tns_state* s, int32_t chi_b, int64_t n, uint64_t seed,
                                        const uint8_t* bits_dev, double* logq_dev, double* cond_dev) {
  LaunchScope ls_(s);
  if (!s || chi_b < 1 || n < 0 || (n > 0 && (!bits_dev || !logq_dev))) {
    set_error("invalid argument to tns_sample_replay");
    return TNS_ERR_ARG;
  }
  return sample(s, chi_b, n, seed, bits_dev, nullptr, logq_dev, cond_dev);
}

extern "C" tns_status tns_amplitude(tns_state* s, int32_t chi_b, int64_t n, const uint8_t* bits_dev,
                                    double* log_abs_dev, double* phase_dev) {
  LaunchScope ls_(s);
  if (!s || chi_b < 1 || n < 0 || (n > 0 && (!bits_dev || !log_abs_dev || !phase_dev))) {
    set_error("invalid argument to tns_amplitude");
    return TNS_ERR_ARG;
  }
  return amplitude(s, chi_b, n, bits_dev, log_abs_dev, phase_dev);
}

extern "C" tns_status tns_certify(tns_state* s, int32_t chi_b, int64_t n, const uint8_t* bits_dev,
                                  const double* logq_dev, double* logp_dev, double* stats_host) {
  LaunchScope ls_(s);
  if (!s || chi_b < 1 || n < 0 || !stats_host || (n > 0 && (!bits_dev || !logq_dev || !logp_dev))) {
    set_error("invalid argument to tns_certify");
    return TNS_ERR_ARG;
  }
  return certify(s, chi_b, n, bits_dev, logq_dev, logp_dev, stats_host);
}

extern "C" tns_status tns_bp_stats(const tns_state* s, double* ms, double* bytes, double* flops) {
  if (!s) { set_error("invalid argument to tns_bp_stats"); return TNS_ERR_ARG; }
  if (ms) *ms = s->bp_last_ms;
  if (bytes) *bytes = s->bp_last_bytes;
  if (flops) *flops = s->bp_last_flops;
  return TNS_OK;
}

extern "C" tns_status tns_log_fidelity(const tns_state* s, double* log_f) {
  if (!s || !log_f) { set_error("invalid argument to tns_log_fidelity"); return TNS_ERR_ARG; }
  *log_f = s->log_f;
  return TNS_OK;
}

extern "C" tns_status tns_log_norm(tns_state* s, int32_t chi_b, double* out) {
  LaunchScope ls_(s);
  if (!s || !out || chi_b < 1) { set_error("invalid argument to tns_log_norm"); return TNS_ERR_ARG; }
  return log_norm(s, chi_b, out);
}

extern "C" tns_status tns_direct_marginals(tns_state* s, int32_t chi_b, double* one_host, double* two_host) {
  LaunchScope ls_(s);
  if (!s || !one_host || chi_b < 1) { set_error("invalid argument to tns_direct_marginals"); return TNS_ERR_ARG; }
  return direct_marginals(s, chi_b, one_host, two_host);
}

extern "C" tns_status tns_set_precision(tns_state* s, tns_prec prec) {
  LaunchScope ls_(s);
  if (!s || (prec != TNS_PREC_FP64 && prec != TNS_PREC_MIXED)) { set_error("invalid precision"); return TNS_ERR_ARG; }
  s->prec = prec;
  return TNS_OK;
}

extern "C" tns_status tns_set_tensor_cores(tns_state* s, int32_t enable) {
  if (!s) { set_error("state is NULL"); return TNS_ERR_ARG; }
  s->tensor_cores = enable != 0;
  return TNS_OK;
}

extern "C" tns_status tns_set_graphs(tns_state* s, int32_t enable) {
  if (!s) { set_error("state is NULL"); return TNS_ERR_ARG; }
  s->use_graphs = enable != 0;
  return TNS_OK;
}

extern "C" tns_status tns_set_compression(tns_state* s, int32_t oversample, int32_t power_iters,
                                          int32_t env_power_iters) {
  if (!s || oversample < 0 || oversample > 4096 || power_iters < 0 || power_iters > 64 || env_power_iters < 0 ||
      env_power_iters > 64) {
    set_error("invalid argument to tns_set_compression");
    return TNS_ERR_ARG;
  }
  s->rf_p = oversample;
  s->rf_q = power_iters;
  s->rf_q_env = env_power_iters;
  return TNS_OK;
}

extern "C" tns_status tns_query(const tns_state* s, int32_t* H, int32_t* W, int32_t* transposed, int32_t* chi_now) {
  if (!s) { set_error("state is NULL"); return TNS_ERR_ARG; }
  int chi = 1;
  for (auto& c : s->cell)
    for (int leg = 1; leg <= 4; ++leg) chi = std::max(chi, c.dim[leg]);
  if (H) *H = s->H;
  if (W) *W = s->W;
  if (transposed) *transposed = s->transposed ? 1 : 0;
  if (chi_now) *chi_now = chi;
  return TNS_OK;
}

extern "C" tns_status tns_launch_count(const tns_state* s, int64_t* launches) {
  if (!s || !launches) { set_error("invalid argument"); return TNS_ERR_ARG; }
  *launches = s->launches;
  return TNS_OK;
}

extern "C" tns_status tns_profile_enable(tns_state* s, int32_t enable) {
  if (!s) { set_error("state is NULL"); return TNS_ERR_ARG; }
  TNS_TRY_CUDA(cudaStreamSynchronize(s->st));
  s->prof.clear();
  s->prof.on = enable != 0;
  return TNS_OK;
}

extern "C" tns_status tns_profile_read(tns_state* s, int32_t cls, double* ms, int64_t* launches, double* flops) {
  if (!s || cls < 0 || cls >= Profiler::NCLASS) { set_error("invalid argument to tns_profile_read"); return TNS_ERR_ARG; }
  TNS_TRY_CUDA(cudaStreamSynchronize(s->st));
  s->prof.resolve();
  if (ms) *ms = s->prof.ms[cls];
  if (launches) *launches = s->prof.n[cls];
  if (flops) *flops = s->prof.flops[cls];
  return TNS_OK;
}

// ---------------------------------------------------------------- save / load
namespace {
struct FileW {
  FILE* f;
  bool ok = true;
  void u32(uint32_t v) { ok &= fwrite(&v, 4, 1, f) == 1; }
  void f64(double v) { ok &= fwrite(&v, 8, 1, f) == 1; }
  void raw(const void* p, size_t n) { if (n) ok &= fwrite(p, 1, n, f) == n; }
};
struct FileR {
  FILE* f;
  bool ok = true;
  uint32_t u32() { uint32_t v = 0; ok &= fread(&v, 4, 1, f) == 1; return v; }
  double f64() { double v = 0; ok &= fread(&v, 8, 1, f) == 1; return v; }
  void raw(void* p, size_t n) { if (n) ok &= fread(p, 1, n, f) == n; }
};
}  // namespace

extern "C" tns_status tns_save(const tns_state* s, const char* path) {
  if (!s || !path) { set_error("invalid argument to tns_save"); return TNS_ERR_ARG; }
  TNS_TRY_CUDA(cudaStreamSynchronize(s->st));
  FILE* f = fopen(path, "wb");
  if (!f) { set_error("cannot open %s", path); return TNS_ERR_ARG; }
  FileW w{f};
  w.raw("TNSF", 4);
  w.u32(1);
  w.u32(s->H); w.u32(s->W); w.u32(s->n); w.u32(s->transposed ? 1 : 0);
  w.f64(s->log_f);
  for (int q = 0; q < s->n; ++q) { w.u32(s->qcell[q] / s->W); w.u32(s->qcell[q] % s->W); }
  for (auto& c : s->cell)
    for (int leg = 1; leg <= 4; ++leg) w.u32(c.edge[leg] ? 1 : 0);
  std::vector<cd> buf;
  for (size_t ci = 0; ci < s->cell.size(); ++ci) {
    const Cell& c = s->cell[ci];
    for (int k = 0; k < 5; ++k) w.u32(c.dim[k]);
    buf.resize(c.size());
    if (cudaMemcpy(buf.data(), c.t, sizeof(cd) * c.size(), cudaMemcpyDeviceToHost) != cudaSuccess) w.ok = false;
    w.raw(buf.data(), sizeof(cd) * c.size());
  }
  for (size_t ci = 0; ci < s->cell.size(); ++ci) {
    const Cell& c = s->cell[ci];
    for (int leg = 1; leg <= 4; ++leg) {
      if (!c.edge[leg]) continue;
      int D = c.dim[leg];
      w.u32(D);
      buf.resize((size_t)D * D);
      if (cudaMemcpy(buf.data(), s->msg[ci * 5 + leg], sizeof(cd) * D * D, cudaMemcpyDeviceToHost) != cudaSuccess)
        w.ok = false;
      w.raw(buf.data(), sizeof(cd) * D * D);
    }
  }
  fclose(f);
  if (!w.ok) { set_error("write failed: %s", path); return TNS_ERR_ARG; }
  return TNS_OK;
}

extern "C" tns_status tns_load(const char* path, void* cuda_stream, tns_state** out) {
  if (!path || !out) { set_error("invalid argument to tns_load"); return TNS_ERR_ARG; }
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) { set_error("cannot open %s", path); return TNS_ERR_ARG; }
  FileR r{f};
  char magic[4];
  r.raw(magic, 4);
  if (!r.ok || memcmp(magic, "TNSF", 4) != 0 || r.u32() != 1) {
    fclose(f);
    set_error("%s is not a TNSF v1 file", path);
    return TNS_ERR_STATE;
  }
  tns_state* s = new tns_state();
  s->H = r.u32(); s->W = r.u32(); s->n = r.u32(); s->transposed = r.u32() != 0;
  s->log_f = r.f64();
  s->st = (cudaStream_t)cuda_stream;
  cudaGetDevice(&s->device);
  if (!r.ok || s->H < 1 || s->W < 1 || s->H > 4096 || s->W > 4096 || s->n < 1) {
    fclose(f); delete s; set_error("corrupt header in %s", path); return TNS_ERR_STATE;
  }
  s->cell.assign((size_t)s->H * s->W, Cell());
  s->qcell.assign(s->n, -1);
  for (int q = 0; q < s->n; ++q) {
    int rr = r.u32(), cc = r.u32();
    if (rr >= s->H || cc >= s->W) { fclose(f); delete s; set_error("bad cell in %s", path); return TNS_ERR_STATE; }
    s->qcell[q] = s->cidx(rr, cc);
    s->cell[s->qcell[q]].qubit = q;
    s->cell[s->qcell[q]].dim[0] = 2;
  }
  for (auto& c : s->cell)
    for (int leg = 1; leg <= 4; ++leg) c.edge[leg] = r.u32() != 0;
  // first pass: dims and data on the host to size chi_max
  std::vector<std::vector<cd>> data(s->cell.size());
  int chi = 1;
  for (size_t ci = 0; ci < s->cell.size(); ++ci) {
    Cell& c = s->cell[ci];
    for (int k = 0; k < 5; ++k) c.dim[k] = (int)r.u32();
    if (!r.ok || c.size() <= 0 || c.size() > (1LL << 34)) { fclose(f); delete s; set_error("bad dims in %s", path); return TNS_ERR_STATE; }
    for (int leg = 1; leg <= 4; ++leg) chi = std::max(chi, c.dim[leg]);
    data[ci].resize(c.size());
    r.raw(data[ci].data(), sizeof(cd) * c.size());
  }
  s->chi_max = chi;
  tns_status st = alloc_state(s);
  if (st != TNS_OK || !r.ok) { fclose(f); free_state(s); delete s; if (st == TNS_OK) set_error("truncated %s", path); return st == TNS_OK ? TNS_ERR_STATE : st; }
  for (size_t ci = 0; ci < s->cell.size(); ++ci)
    cudaMemcpy(s->cell[ci].t, data[ci].data(), sizeof(cd) * data[ci].size(), cudaMemcpyHostToDevice);
  std::vector<cd> buf;
  for (size_t ci = 0; ci < s->cell.size(); ++ci) {
    Cell& c = s->cell[ci];
    for (int leg = 1; leg <= 4; ++leg) {
      if (!c.edge[leg]) continue;
      int D = (int)r.u32();
      if (D != c.dim[leg]) r.ok = false;
      if (!r.ok) break;
      buf.resize((size_t)D * D);
      r.raw(buf.data(), sizeof(cd) * D * D);
      cudaMemcpy(s->msg[ci * 5 + leg], buf.data(), sizeof(cd) * D * D, cudaMemcpyHostToDevice);
    }
  }
  fclose(f);
  if (!r.ok) { free_state(s); delete s; set_error("truncated or inconsistent %s", path); return TNS_ERR_STATE; }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { tns_status rr = cuda_status(e, "tns_load"); free_state(s); delete s; return rr; }
  *out = s;
  return TNS_OK;
}
