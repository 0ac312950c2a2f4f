// Internal state of the tensor-network library (host side).
#pragma once
#include <map>
#include <set>
#include <string>
#include <vector>

#include "../../include/tns.h"
#include "common.cuh"
#include "contract.cuh"

namespace tns {

enum Leg { LEG_S = 0, LEG_U = 1, LEG_L = 2, LEG_D = 3, LEG_R = 4 };
inline int opp_leg(int leg) { return leg == LEG_U ? LEG_D : leg == LEG_D ? LEG_U : leg == LEG_L ? LEG_R : LEG_L; }

// One grid cell: tensor psi[s][u][l][d][r] (FP64 master copy on the device).
struct Cell {
  int qubit = -1;            // -1: empty cell (physical dimension 1)
  int dim[5] = {1, 1, 1, 1, 1};
  bool edge[5] = {false, false, false, false, false};
  cd* t = nullptr;           // device, capacity cap complex elements (inside the cell arena)
  long long cap = 0;
  long long off = 0;         // element offset of t in the cell arena
  long long size() const { return (long long)dim[0] * dim[1] * dim[2] * dim[3] * dim[4]; }
};

// Named, grow-only device buffers reused across calls.
struct Workspace {
  std::map<std::string, std::pair<void*, size_t>> slots;
  long long gen = 0;                    // bumped whenever a buffer is reallocated
  cudaError_t get(const std::string& name, size_t bytes, void** out);
  void release();
};

// A boundary MPS stored site by site in the logical order of the sweep that
// produced it.  Site i has layout [left][phys...][right] in that logical order;
// `reversed` says whether logical order runs right-to-left over the grid.
struct StoredMPS {
  std::vector<void*> site;              // device pointers (working precision)
  std::vector<long long> bond;          // W+1 bond dims in logical order
  std::vector<std::vector<long long>> phys;  // per site physical dims (in stored order)
  bool reversed = false;
};

// Event-bracketed timing of kernel classes (see tns_profile_enable).
struct Profiler {
  static constexpr int NCLASS = 10;
  bool on = false;
  struct Rec { int cls; cudaEvent_t a, b; double flops; bool own_a = true, own_b = true; };
  std::vector<Rec> pending;
  double ms[NCLASS] = {};
  double flops[NCLASS] = {};
  long long n[NCLASS] = {};
  cudaEvent_t begin(cudaStream_t st);
  void end(int cls, cudaEvent_t a, double fl, cudaStream_t st);
  // Record the interval between two already-recorded events; own_* = destroy the event when resolved.
  void span(int cls, cudaEvent_t a, cudaEvent_t b, double fl, bool own_a, bool own_b);
  void resolve();   // after the stream is synchronised
  void clear();
};

struct EnvCache {
  bool valid = false;
  int chi_b = 0;
  int prec = -1;
  long long version = -1;
  int p = -1, q = -1;                   // range-finder settings the environments were built with
  std::vector<StoredMPS> E;             // E[b], b = 1..H (index b); each stored right-to-left
  double log_norm = 0.0;
};

}  // namespace tns

struct tns_state {
  int H = 0, W = 0, n = 0;
  bool transposed = false;
  int chi_max = 1;
  tns_prec prec = TNS_PREC_MIXED;
  cudaStream_t st = nullptr;
  int device = 0;
  std::vector<tns::Cell> cell;          // H*W, row-major
  std::vector<int> qcell;               // qubit -> cell index
  std::vector<cd*> msg;                 // (cell*5 + leg): message into cell across leg, chi_max^2 capacity
  std::vector<cd*> msg_new;
  cd* cell_arena = nullptr;             // every cell tensor, cell ci at cell[ci].off
  cd* msg_arena = nullptr;              // message slot (cell*5 + leg) at slot * chi_max^2
  cd* msg_new_arena = nullptr;
  double log_f = 0.0;
  long long version = 0;                // bumped whenever site tensors change
  long long launches = 0;
  tns::Workspace ws;
  tns::EnvCache env;                    // bottom environments E[b] (rows b..H-1)
  tns::EnvCache env_top;                // top environments, built on the flipped frame
  tns::Profiler prof;
  std::vector<void*> work_cells;        // working-precision copies of the cell tensors
  int work_prec = -1;
  bool tensor_cores = true;             // mixed path: environment GEMMs on tcgen05
  int rf_p = 48;                        // range-finder oversampling (k = chi_b + rf_p columns)
  int rf_q = 3;                         // subspace iterations of the sampler and amplitude zips
  int rf_q_env = 6;                     // subspace iterations of the norm-environment zips
  // CUDA graphs of the sampler's per-chunk launch sequence, keyed by everything the
  // sequence depends on (see sample()); a key seen once runs eagerly, the second time
  // it is captured, then replayed.
  bool use_graphs = true;
  struct GraphEntry { cudaGraphExec_t exec = nullptr; long long launches = 0; };
  std::map<std::vector<long long>, GraphEntry> graphs;
  std::set<std::vector<long long>> graph_seen;
  long long env_builds = 0;             // bumped when norm environments are rebuilt
  long long work_gen = 0;               // bumped when the working-precision cell copies change
  unsigned char host_call[64] = {};     // staging for the per-call parameter block
  cudaStream_t gstream = nullptr;       // private stream that graphs are captured and replayed on
  cudaEvent_t gev[2] = {nullptr, nullptr};
  long long work_version = -1;
  // gate layers: the gates of a group run concurrently on these streams (one slot per
  // stream: its own buffers, a pinned host block for the singular values, an event)
  std::vector<cudaStream_t> gate_streams;
  std::vector<cudaEvent_t> gate_events;
  double* gate_host = nullptr;          // [slots][4 chi_max + 1] singular values + status
  size_t gate_host_n = 0;
  // pinned host buffer for BP's per-message residuals (two iterations in flight)
  double* bp_host = nullptr;
  size_t bp_host_n = 0;
  // BP timing of the last tns_bp_gauge call: iterations and device milliseconds of the
  // message contractions + normalisation (events on the state's stream)
  double bp_last_ms = 0.0;
  double bp_last_bytes = 0.0;   // algorithmic bytes of the last call (site tensors + messages)
  double bp_last_flops = 0.0;

  int cidx(int r, int c) const { return r * W + c; }
  void nbr(int ci, int leg, int& r2, int& c2) const {
    int r = ci / W, c = ci % W;
    r2 = r + (leg == tns::LEG_D) - (leg == tns::LEG_U);
    c2 = c + (leg == tns::LEG_R) - (leg == tns::LEG_L);
  }
};

namespace tns {
void set_error(const char* fmt, ...);
tns_status cuda_status(cudaError_t e, const char* where);
#define TNS_TRY_CUDA(expr)                                         \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return ::tns::cuda_status(_e, #expr);   \
  } while (0)
#define TNS_TRY(expr)                      \
  do {                                     \
    tns_status _s = (expr);                \
    if (_s != TNS_OK) return _s;           \
  } while (0)

// gates.cu
tns_status apply_gate_layer(tns_state* s, int n_gates, const int32_t* sites, const double* mats, int chi,
                            double cutoff, double* eps_out);
tns_status bp_gauge(tns_state* s, int max_iter, double tol, int* iters, double* resid);
// sampler.cu
// Attributes the contraction launches made by this thread during an API call to
// the call's state (the contraction layer counts per thread, not per state).
struct LaunchScope {
  tns_state* s;
  long long c0;
  explicit LaunchScope(tns_state* st) : s(st), c0(contract_launches()) {}
  ~LaunchScope() {
    if (s) s->launches += contract_launches() - c0;
  }
};

tns_status sample(tns_state* s, int chi_b, long long n, uint64_t seed, const uint8_t* forced, uint8_t* bits,
                  double* logq, double* cond, long long first = 0);
tns_status amplitude(tns_state* s, int chi_b, long long n, const uint8_t* bits, double* log_abs, double* phase);
tns_status log_norm(tns_state* s, int chi_b, double* out);
tns_status direct_marginals(tns_state* s, int chi_b, double* one, double* two);
tns_status certify(tns_state* s, int chi_b, long long n, const uint8_t* bits, const double* logq, double* logp,
                   double* stats_host);
}  // namespace tns
