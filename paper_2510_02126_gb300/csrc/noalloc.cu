// lyap_invert_noalloc: the Gauss-Jordan inversion of lyap_invert without any device
// allocation.  Its workspace is one file-scope __device__ array sized for
// LYAP_NOALLOC_MAX_N; the array's address is looked up once per device (with that
// device current) and carved into the GJWork buffers on every call.
#include <atomic>

#include "dense.cuh"
#include "gj_inverse.cuh"

namespace lyap {

constexpr int64_t NA_ALIGN = 256;
constexpr int64_t na_round(int64_t b) { return (b + NA_ALIGN - 1) / NA_ALIGN * NA_ALIGN; }
// Bytes of the workspace for order n in FP64 (the larger of the two working types).
constexpr int64_t na_bytes(int64_t n) {
  return 2 * na_round(n * n * 8)          // ping-pong working matrices
         + 2 * na_round(n * GJ_BS * 8)    // panel operands P' and R^T
         + 3 * na_round(n * 4)            // orig, perm[0], perm[1]
         + na_round(n * 8)                // pivots / log|pivot|
         + na_round(4)                    // status word
         + na_round(2 * ((n + GJ_BS - 1) / GJ_BS) * 4)  // per-step exponents (unused by SIMT)
         + na_round(64 * 4)               // amax scratch
         + na_round(8);                   // log|det|
}
constexpr int64_t NA_BYTES = na_bytes(LYAP_NOALLOC_MAX_N);

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
static std::atomic<void*> g_na_ptr[NA_MAX_DEVICES];

// Address of this device's copy of the workspace (looked up once per device).
static int na_scratch(int dev, unsigned char** out) {
  void* p = g_na_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      lyap_set_error_message("cudaGetSymbolAddress of the static workspace failed", __FILE__, __LINE__);
      return LYAP_ERR_CUDA;
    }
    g_na_ptr[dev].store(p, std::memory_order_release);
  }
  *out = static_cast<unsigned char*>(p);
  return LYAP_OK;
}

__global__ void na_iota_kernel(int* p, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

template <typename T>
__global__ void na_unpermute_kernel(const T* __restrict__ X, const int* __restrict__ perm, int n,
                                    double* __restrict__ Ainv, int64_t ld) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    Ainv[i + (int64_t)perm[c] * ld] = (double)X[i * n + c];
  }
}

static unsigned na_blocks(int64_t total) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, ceil_div(total, 256))); }

template <typename T>
static int na_run(const double* A, int n, int64_t lda, int prec, double* Ainv, int64_t ldai, int32_t* ipiv,
                  double* logabsdet, unsigned char* ws, cudaStream_t s) {
  GJWork W;
  W.n = n;
  W.elt = sizeof(T);
  unsigned char* p = ws;
  auto take = [&](int64_t bytes) { unsigned char* q = p; p += na_round(bytes); return q; };
  W.M[0] = take((int64_t)n * n * 8);
  W.M[1] = take((int64_t)n * n * 8);
  W.Pp = take((int64_t)n * GJ_BS * 8);
  W.Rt = take((int64_t)n * GJ_BS * 8);
  W.orig = reinterpret_cast<int*>(take((int64_t)n * 4));
  W.perm[0] = reinterpret_cast<int*>(take((int64_t)n * 4));
  W.perm[1] = reinterpret_cast<int*>(take((int64_t)n * 4));
  W.logpiv = reinterpret_cast<double*>(take((int64_t)n * 8));
  W.status = reinterpret_cast<int*>(take(4));
  W.exps = reinterpret_cast<int*>(take(2 * ceil_div(n, GJ_BS) * 4));
  W.amax = reinterpret_cast<float*>(take(64 * 4));
  double* ld = reinterpret_cast<double*>(take(8));
  W.ipiv = ipiv;
  W.cur = 0;
  // the status word is the only state that must start at zero
  LYAP_CUDA_TRY(cudaMemsetAsync(W.status, 0, sizeof(int), s));
  LYAP_TRY(cm64_to_rm<T>(A, n, lda, 1.0, (T*)W.M[0], s));
  na_iota_kernel<<<na_blocks(n), 256, 0, s>>>(W.perm[0], n);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  LYAP_TRY(gj_invert_run(W, prec, s));
  na_unpermute_kernel<T><<<na_blocks((int64_t)n * n), 256, 0, s>>>((const T*)W.M[W.cur], W.perm[W.cur], n, Ainv, ldai);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  LYAP_TRY(pivot_logs(W, ld, s));
  double h_ld = 0.0;
  int h_st = 0;
  LYAP_CUDA_TRY(cudaMemcpyAsync(&h_ld, ld, sizeof(double), cudaMemcpyDeviceToHost, s));
  LYAP_CUDA_TRY(cudaMemcpyAsync(&h_st, W.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  LYAP_CUDA_TRY(cudaStreamSynchronize(s));
  if (logabsdet) *logabsdet = h_ld;
  return h_st;
}

}  // namespace lyap

extern "C" int lyap_invert_noalloc(const double* A, int64_t n, int64_t lda, int prec, double* Ainv, int64_t ldai,
                                   int32_t* ipiv, double* logabsdet, void* stream) {
  using namespace lyap;
  if (!A || !Ainv || n <= 0 || lda < n || ldai < n) return LYAP_ERR_ARG;
  if (n > LYAP_NOALLOC_MAX_N) {
    lyap_set_error_message("lyap_invert_noalloc: n exceeds LYAP_NOALLOC_MAX_N", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  if (prec != LYAP_FP64 && prec != LYAP_FP32) {
    lyap_set_error_message("lyap_invert_noalloc: only LYAP_FP64 and LYAP_FP32", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  int dev = 0;
  LYAP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return LYAP_ERR_ARG;
  unsigned char* ws = nullptr;
  LYAP_TRY(na_scratch(dev, &ws));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == LYAP_FP64) return na_run<double>(A, (int)n, lda, prec, Ainv, ldai, ipiv, logabsdet, ws, s);
  return na_run<float>(A, (int)n, lda, prec, Ainv, ldai, ipiv, logabsdet, ws, s);
}
