// Per-context bookkeeping shared by the launchers: the identity of the current
// CUDA context, and a thread-safe record of which kernels already have their
// dynamic shared-memory opt-in on it.
//
// A kernel attribute such as cudaFuncAttributeMaxDynamicSharedMemorySize belongs
// to one device's context: a second GPU used from the same process, or the same
// GPU after cudaDeviceReset (which creates a new primary context), starts without
// it.  Keying the record by the context's unique id covers both.
#include <mutex>
#include <set>
#include <tuple>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace tns {

namespace {
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct DriverFns {
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
};

const DriverFns& driver_fns() {
  static DriverFns f;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  return f;
}
}  // namespace

cudaError_t current_context_id(unsigned long long* id) {
  const DriverFns& f = driver_fns();
  if (!f.get_current || !f.get_id) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (f.get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (!ctx) {
    // no context bound to this thread yet: cudaSetDevice on the current device makes
    // the runtime create and bind its primary context (CUDA 12 and later), without
    // touching any allocator (only on this first call, never during a capture)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) return e;
    if (f.get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  }
  if (f.get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

cudaError_t smem_optin(const void* fn, int bytes) {
  static std::mutex mu;
  static std::set<std::tuple<unsigned long long, const void*, int>> done;
  unsigned long long ctx = 0;
  cudaError_t e = current_context_id(&ctx);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(ctx, fn, bytes);
  if (done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  // kernels that opt in use large shared-memory footprints: prefer the largest
  // shared-memory carveout so that as many CTAs as fit can be resident per SM
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) done.insert(key);
  return e;
}

}  // namespace tns
