// Strided tensor-contraction GEMM (SIMT) and its host-side planner.
//
// Every tensor contraction of the library is written as an einsum over labelled
// strided views; the planner classifies labels into batch / M / N / K groups,
// merges contiguous runs, and launches one batched complex GEMM whose operand
// addresses are decoded from up to four sub-indices per dimension.  This avoids
// explicit permutes: outputs are written straight into the layout the next
// step reads.
#pragma once
#include "common.cuh"
#include <vector>
#include <string>

namespace tns {

enum class Prec { F64 = 0, F32 = 1, F32_ACC64 = 2 };   // F32_ACC64: float2 inputs, double accumulate + output

struct TView {
  void* ptr = nullptr;            // device base pointer (complex elements)
  std::string labels;             // one char per axis
  std::vector<long long> dim;     // extents
  std::vector<long long> stride;  // strides in complex elements
  bool conj = false;
  // optional per-batch offset: ptr += idx[b * idx_ld] * idx_stride where b is the
  // index of batch label idx_label (used to project physical legs per sample)
  const uint8_t* idx = nullptr;
  long long idx_ld = 0, idx_stride = 0;
  char idx_label = 0;
  // optional per-batch element offsets (device int64): ptr += boff[b] where b is the
  // index of batch label boff_label (gathers operands that are not equally spaced)
  const long long* boff = nullptr;
  char boff_label = 0;
};

// Row-major contiguous view helper.
TView view(void* p, const std::string& labels, const std::vector<long long>& dims, bool conj = false);
// Add a broadcast (stride 0) axis.
TView& bcast(TView& v, char label, long long dim);

// C = alpha * sum_K A * B + beta * C  (labels of C decide the output layout).
// Returns cudaSuccess or an error; throws nothing.
// flops_out (optional) receives 8 * M * N * K * batch, the algorithmic real FLOPs.
cudaError_t contract(const TView& A, const TView& B, const TView& C, Prec prec, cudaStream_t st,
                     double2 alpha = make_double2(1.0, 0.0), double2 beta = make_double2(0.0, 0.0),
                     double* flops_out = nullptr);

// Number of GEMM launches issued so far (for launch accounting).
long long contract_launches();

}  // namespace tns
