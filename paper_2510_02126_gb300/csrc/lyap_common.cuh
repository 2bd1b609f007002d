// Shared device helpers for liblyap (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <math.h>
#include <algorithm>
#include <atomic>

#include "../../include/liblyap.h"

#define LYAP_CUDA_TRY(expr)                                                     \
  do {                                                                          \
    cudaError_t _e = (expr);                                                    \
    if (_e != cudaSuccess) {                                                    \
      lyap_set_error_message(cudaGetErrorString(_e), __FILE__, __LINE__);       \
      return LYAP_ERR_CUDA;                                                     \
    }                                                                           \
  } while (0)

#define LYAP_TRY(expr)                  \
  do {                                  \
    int _s = (expr);                    \
    if (_s < 0) return _s;              \
  } while (0)

void lyap_set_error_message(const char* what, const char* file, int line);
// Counts kernel launches made by the library (reported in lyap_info_t).
void lyap_count_launch(int k = 1);

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// One-time host actions per device: kernel attributes set with cudaFuncSetAttribute apply
// to the device that is current at the call, so a flag shared by the whole process would
// skip them on every device but the first.  need() is true until set() has run with the
// same device current.
constexpr int LYAP_MAX_DEVICES = 64;
struct DeviceOnce {
  std::atomic<bool> done[LYAP_MAX_DEVICES] = {};
  static int device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) { cudaGetLastError(); return -1; }
    return d;
  }
  bool need() const {
    const int d = device();
    return d < 0 || d >= LYAP_MAX_DEVICES || !done[d].load();
  }
  void set() {
    const int d = device();
    if (d >= 0 && d < LYAP_MAX_DEVICES) done[d].store(true);
  }
};

// Device spin-waits never run unbounded: after this many polls a kernel records
// LYAP_ERR_TIMEOUT in its status word and returns.
#define LYAP_SPIN_LIMIT (1u << 26)

// ---------------------------------------------------------------------------
// warp reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// argmax of (val, idx): larger val wins; ties -> smaller idx.  idx < 0 = empty.
template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, i, o);
    bool take = (oi >= 0) && (i < 0 || ov > v || (ov == v && oi < i));
    if (take) { v = ov; i = oi; }
  }
}

// ---------------------------------------------------------------------------
// thread-block cluster helpers (distributed shared memory)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t dsmem_map(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ float dsmem_ld_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double dsmem_ld_f64(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int dsmem_ld_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
template <typename T> __device__ __forceinline__ T dsmem_ld(uint32_t addr);
template <> __device__ __forceinline__ float dsmem_ld<float>(uint32_t a) { return dsmem_ld_f32(a); }
template <> __device__ __forceinline__ double dsmem_ld<double>(uint32_t a) { return dsmem_ld_f64(a); }

// ---------------------------------------------------------------------------
// precision helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline double unit_roundoff(int prec) {
  switch (prec) {
    case LYAP_FP64: return 1.1102230246251565e-16;  // 2^-53
    case LYAP_FP32: return 5.9604644775390625e-08;  // 2^-24
    case LYAP_FP16: return 4.8828125e-04;           // 2^-11
    case LYAP_BF16: return 3.90625e-03;             // 2^-8
  }
  return 0.0;
}

template <typename H> __device__ __forceinline__ H to_half(float x);
template <> __device__ __forceinline__ __half to_half<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_half<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// power of two 2^e with e chosen so that amax * 2^-e lies in [1, 2)
__device__ __forceinline__ int pow2_exponent(double amax) {
  if (!(amax > 0.0) || !isfinite(amax)) return 0;
  int e;
  frexp(amax, &e);  // amax = f * 2^e, f in [0.5, 1)
  return e - 1;
}
