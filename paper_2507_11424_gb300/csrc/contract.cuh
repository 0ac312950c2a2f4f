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

// F32_ACC64: float2 inputs, double accumulate + output.  TF32X3: complex64 on the
// tensor cores (tcgen05 kind::tf32, three-pass split; FP32-level accuracy) when
// the contraction is large enough and alpha = 1, beta = 0; SIMT F32 otherwise.
enum class Prec { F64 = 0, F32 = 1, F32_ACC64 = 2, TF32X3 = 3 };

// Optional timing hooks for the tensor-core path: when the contraction runs on
// the tensor cores, `mma_begin` / `mma_end` (caller-created events) are recorded
// around the GEMM kernel (operand packing runs before mma_begin) and used_tc is set.
struct ContractTiming {
  cudaEvent_t mma_begin = nullptr, mma_end = nullptr;
  bool used_tc = false;
  bool force_tc = false;     // fail with cudaErrorNotSupported instead of falling back (tests)
};

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
                     double* flops_out = nullptr, ContractTiming* timing = nullptr);

// The planner's decision for a contraction in the TF32X3 precision, without
// launching anything (host only): out[0] tensor cores used (1) or CUDA cores (0),
// [1] operand roles swapped, [2] A read in place, [3] A shared by the batch, [4] B
// shared, [5] batch rows merged into one launch, [6] tile width in real columns,
// [7] M, [8] N (complex, after any swap), [9] K, [10] batch entries.
cudaError_t contract_plan(const TView& A, const TView& B, const TView& C, long long* out);

// Number of GEMM launches issued so far (for launch accounting).
long long contract_launches();

}  // namespace tns
