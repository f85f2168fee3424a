// Shared device/host helpers of the AFQMC library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <cstdio>

#include "../../include/afqmc.h"

namespace afq {

// ---------------------------------------------------------------- errors --
void set_error(const char* fmt, ...);
extern int64_t g_launches;

#define AFQ_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ::afq::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call,           \
                       cudaGetErrorString(e_));                               \
      return AFQMC_ECUDA;                                                     \
    }                                                                         \
  } while (0)

// Checked launch: counts the kernel and turns a launch error into ECUDA.
#define AFQ_LAUNCH(kernel, grid, block, smem, stream, ...)                    \
  do {                                                                        \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);               \
    ++::afq::g_launches;                                                      \
    cudaError_t e_ = cudaGetLastError();                                      \
    if (e_ != cudaSuccess) {                                                  \
      ::afq::set_error("%s:%d: launch %s: %s", __FILE__, __LINE__, #kernel,  \
                       cudaGetErrorString(e_));                               \
      return AFQMC_ECUDA;                                                     \
    }                                                                         \
  } while (0)

#define AFQ_TRY(expr)                                                         \
  do {                                                                        \
    int r_ = (expr);                                                          \
    if (r_ != AFQMC_OK) return r_;                                            \
  } while (0)

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit on the current device, once per
// device: the attribute belongs to each device's context, so a process that
// drives several GPUs sets it on each (bit d of `done` = set on device d).
// A cudaDeviceReset() drops it with the rest of that device's context.
template <typename F>
inline int smem_attr_once(F* kern, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  AFQ_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return AFQMC_OK;
  AFQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_release);
  return AFQMC_OK;
}

// -------------------------------------------------------------- Philox -----
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
// (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2, c = (hi1^c1^k0, lo1, hi0^c3^k1, lo0),
// with the key advanced by the Weyl constants before every round but the
// first.
struct u32x4 {
  uint32_t x, y, z, w;
};

__host__ __device__ inline void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

__host__ __device__ inline u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, c.x, &hi0, &lo0);
    mulhilo32(M1, c.z, &hi1, &lo1);
    u32x4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

// u in (0, 1]: a = (hi >> 5) * 2^26 + (lo >> 6), u = fl(fl(a + 0.5) * 2^-53).
__host__ __device__ inline double uniform53(uint32_t hi, uint32_t lo) {
  uint64_t a = ((uint64_t)(hi >> 5) << 26) + (uint64_t)(lo >> 6);
#ifdef __CUDA_ARCH__
  return __dmul_rn(__dadd_rn((double)a, 0.5), 1.1102230246251565e-16);
#else
  volatile double t = (double)a + 0.5;
  return t * 1.1102230246251565e-16;
#endif
}

// The two standard normals of field pair k (fields 2k and 2k+1) of a walker
// at one step: counter (k, walker, step, 0), key (seed lo, seed hi),
// Box-Muller on (u1, u2).
__device__ inline void field_pair(uint64_t seed, uint32_t step, uint32_t walker, uint32_t k,
                                  double* xa, double* xb) {
  u32x4 c = {k, walker, step, 0u};
  u32x4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  double u1 = uniform53(r.x, r.y);
  double u2 = uniform53(r.z, r.w);
  double rad = sqrt(-2.0 * log(u1));
  double s, co;
  sincos(__dmul_rn(6.283185307179586, u2), &s, &co);
  *xa = rad * co;
  *xb = rad * s;
}

// The same pair from the same Philox words with the Box-Muller transform taken
// in FP32 (mixed path: the fields only feed BF16/TF32 contractions, and
// float64 log/sincos run on GB300's slow FP64 pipe).
__device__ inline void field_pair_f32(uint64_t seed, uint32_t step, uint32_t walker, uint32_t k,
                                      double* xa, double* xb) {
  u32x4 c = {k, walker, step, 0u};
  u32x4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u1 = (float)uniform53(r.x, r.y);
  const float u2 = (float)uniform53(r.z, r.w);
  const float rad = sqrtf(-2.f * logf(u1));
  float s, co;
  sincospif(2.f * u2, &s, &co);
  *xa = (double)(rad * co);
  *xb = (double)(rad * s);
}

// ------------------------------------------------------------ reductions --
template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order (deterministic); blockDim.x multiple of 32.
template <typename T>
__device__ inline T block_sum(T v, T* sh /* >= 32 */) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

__host__ __device__ inline double wrap_pi(double a) {
  // (-pi, pi]
  const double PI = 3.141592653589793, TWO_PI = 6.283185307179586;
  double w = fmod(a + PI, TWO_PI);
  if (w < 0) w += TWO_PI;
  w -= PI;
  if (w == -PI) w = PI;
  return w;
}

}  // namespace afq
