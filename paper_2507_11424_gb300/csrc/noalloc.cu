// Batched Hermitian eigensolver that allocates nothing (tns_eigh_noalloc).
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// owned by another allocator (a framework that reserves all of HBM up front and
// hands out sub-buffers), and latency-critical callers that cannot accept the
// device-wide synchronisation a cudaMalloc/cudaFree may imply.  This entry point
// runs the library's FP64 Jacobi eigensolver with its scratch (the working copy
// of matrices too large for shared memory, and the per-matrix status words) in
// a file-scope device array instead of allocated memory.
#include <map>
#include <mutex>

#include "../../include/tns.h"
#include "linalg.cuh"
#include "state.h"

namespace tns {

// Fixed scratch, resident on every GPU that loads the library until the process exits.
static constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device addresses of the array, looked up once per CUDA context with its device
// current.  In host code the symbol name is only a host-side stand-in: the kernel
// must receive the address that cudaGetSymbolAddress returns.  The cache is keyed
// by the context's unique id, so a second device, or the same device after
// cudaDeviceReset (new primary context, module loaded again, possibly at another
// address), looks the address up again instead of reusing a stale one.
// Next to each address: the batch of the last call in that context, whose status
// words (at the start of the array) tns_eigh_noalloc_status reads back.
struct ScratchEntry {
  void* addr;
  int last_batch;
};
static std::map<unsigned long long, ScratchEntry> g_scratch_addr;
static std::mutex g_scratch_mu;

static tns_status scratch_entry(ScratchEntry** out) {
  unsigned long long ctx = 0;
  TNS_TRY_CUDA(current_context_id(&ctx));
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  auto it = g_scratch_addr.find(ctx);
  if (it == g_scratch_addr.end()) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    it = g_scratch_addr.emplace(ctx, ScratchEntry{p, 0}).first;
  }
  *out = &it->second;   // std::map nodes do not move
  return TNS_OK;
}

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace tns

using namespace tns;

extern "C" tns_status tns_eigh_noalloc(int32_t batch, int32_t n, const double* A_dev, double* lam_dev, double* V_dev,
                                       void* cuda_stream) {
  if (batch < 0 || n < 1 || n > 512 || (batch > 0 && (!A_dev || !lam_dev || !V_dev))) {
    set_error("invalid argument to tns_eigh_noalloc");
    return TNS_ERR_ARG;
  }
  if (batch == 0) return TNS_OK;
  const size_t np = (size_t)n + (n & 1);
  const size_t status_bytes = align256(sizeof(int) * (size_t)batch);
  const size_t work_bytes = eigh_fits_smem(n) ? 0 : (size_t)batch * 2 * np * np * sizeof(cd);
  if (status_bytes + work_bytes > NOALLOC_SCRATCH_BYTES) {
    set_error("tns_eigh_noalloc: batch %d of %dx%d matrices needs %zu bytes of scratch, above the %zu-byte "
              "static limit",
              batch, n, n, status_bytes + work_bytes, NOALLOC_SCRATCH_BYTES);
    return TNS_ERR_ARG;
  }
  ScratchEntry* se = nullptr;
  TNS_TRY(scratch_entry(&se));
  void* base = se->addr;
  int* status = static_cast<int*>(base);
  cd* work = work_bytes ? reinterpret_cast<cd*>(static_cast<unsigned char*>(base) + status_bytes) : nullptr;
  // Nothing in the scratch needs to start at zero: the kernel overwrites its
  // working copy from A and writes every status word.
  TNS_TRY_CUDA(eigh_batched(const_cast<cd*>(reinterpret_cast<const cd*>(A_dev)), (long long)n * n, n, n, batch, lam_dev,
                            reinterpret_cast<cd*>(V_dev), (long long)n * n, work, status,
                            static_cast<cudaStream_t>(cuda_stream)));
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    se->last_batch = batch;
  }
  return TNS_OK;
}

extern "C" tns_status tns_eigh_noalloc_status(int32_t batch, int32_t* status_dev, void* cuda_stream) {
  if (batch < 0 || (batch > 0 && !status_dev)) {
    set_error("invalid argument to tns_eigh_noalloc_status");
    return TNS_ERR_ARG;
  }
  if (batch == 0) return TNS_OK;
  ScratchEntry* se = nullptr;
  TNS_TRY(scratch_entry(&se));
  int last;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    last = se->last_batch;
  }
  if (batch > last) {
    set_error("tns_eigh_noalloc_status: %d status words asked, the last tns_eigh_noalloc call on this device "
              "wrote %d",
              batch, last);
    return TNS_ERR_ARG;
  }
  // stream-ordered device-to-device copy of the status words: no allocation, no host wait
  TNS_TRY_CUDA(cudaMemcpyAsync(status_dev, se->addr, sizeof(int32_t) * (size_t)batch, cudaMemcpyDeviceToDevice,
                               static_cast<cudaStream_t>(cuda_stream)));
  return TNS_OK;
}
