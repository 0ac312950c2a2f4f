// Shared device helpers for the boundary-MPS sampler library (sm_103a).
// Complex numbers are interleaved (re, im) pairs: double2 (FP64 master data and
// small cores) and float2 (working copies of the mixed-precision path).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

typedef double2 cd;
typedef float2 cf;

template <typename T> struct CplxOf;
template <> struct CplxOf<double> { typedef double2 type; };
template <> struct CplxOf<float> { typedef float2 type; };

__host__ __device__ inline double2 mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline float2 mk(float r, float i) { return make_float2(r, i); }

template <typename C> __host__ __device__ inline C czero();
template <> __host__ __device__ inline double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __host__ __device__ inline float2 czero<float2>() { return make_float2(0.f, 0.f); }

__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// conversions between precisions
__host__ __device__ inline double2 to_cd(double2 a) { return a; }
__host__ __device__ inline double2 to_cd(float2 a) { return make_double2(a.x, a.y); }
template <typename C> __host__ __device__ inline C from_cd(double2 a);
template <> __host__ __device__ inline double2 from_cd<double2>(double2 a) { return a; }
template <> __host__ __device__ inline float2 from_cd<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 4x32-bit counter, 2x32-bit
// key, ten rounds of multiply/xor mixing with a Weyl key schedule.
struct Philox4 { uint32_t v[4]; };

__host__ __device__ inline Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    if (r < 9) { k0 += W0; k1 += W1; }
  }
  Philox4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// Uniform in [0,1) from the top 53 bits of the 64-bit word hi:lo (exact in FP64).
__host__ __device__ inline double u53(uint32_t hi, uint32_t lo) {
  uint64_t x = (((uint64_t)hi << 32) | lo) >> 11;
  return (double)x * (1.0 / 9007199254740992.0);
}

// Stage codes of the range-finder test matrices (mirror the documented counter layout).
enum { STAGE_SAMPLE = 0, STAGE_ENV_KET = 1, STAGE_ENV_BRA = 2, STAGE_AMPLITUDE = 3 };

#define TNS_CUDA_OK(x) ((x) == cudaSuccess)

namespace tns {
// Unique id of the CUDA context current on this thread (binding the device's
// primary context first).  Ids are never reused within a process, so a cache
// keyed by it goes stale neither across devices nor across cudaDeviceReset.
cudaError_t current_context_id(unsigned long long* id);
// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes) once per context
// (thread-safe); later calls with the same (context, fn, bytes) return at once.
cudaError_t smem_optin(const void* fn, int bytes);
}  // namespace tns
