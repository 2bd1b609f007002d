// Dense helpers: SIMT GEMM (FP32/FP64), reductions, layout and precision casts.
#pragma once
#include "lyap_common.cuh"

namespace lyap {

// How gemm<double> / gemm_sym<double> compute FP64 products on the calling host thread:
// DGEMM_AUTO (the FP16 tensor-core emulation of ozaki.cuh above a size threshold, the FP64
// SIMT kernel below it), DGEMM_SIMT, DGEMM_TENSOR.
enum { DGEMM_AUTO = 0, DGEMM_SIMT = 1, DGEMM_TENSOR = 2 };
void set_dgemm_method(int method);
int dgemm_method();

// C = alpha op(A) op(B) + beta C, column-major, op = identity ('N') or transpose ('T').
template <typename T>
int gemm(char ta, char tb, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda,
         const T* B, int64_t ldb, T beta, T* C, int64_t ldc, cudaStream_t s);
// C (N x N) = alpha op(A) op(B) + beta C for a product known to be symmetric (e.g. X^T X,
// X^T (H X) with H symmetric): only the upper triangle is computed and mirrored; when
// beta != 0 C must be symmetric on entry.
template <typename T>
int gemm_sym(char ta, char tb, int64_t N, int64_t K, T alpha, const T* A, int64_t lda, const T* B, int64_t ldb,
             T beta, T* C, int64_t ldc, cudaStream_t s);

// Deterministic reductions into a device double (fixed block count, fixed order).
// out[0] = sum_i x_i^2 over an m x n column-major matrix (ld).
template <typename T>
int sumsq(const T* x, int64_t m, int64_t n, int64_t ld, double* out, double* part, cudaStream_t s);
// out[0] = max |x_i|
template <typename T>
int maxabs(const T* x, int64_t m, int64_t n, int64_t ld, double* out, double* part, cudaStream_t s);

constexpr int RED_BLOCKS = 256;  // partial-sum buffer length needed by the reductions

// Bounded grid-wide barrier for cooperative launches.  Returns false (and sets
// *status = LYAP_ERR_TIMEOUT) if the other blocks did not arrive within ~2 s.
struct GridBar {
  unsigned count;
  unsigned gen;
};
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_sync(GridBar* bar, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* genp = &bar->gen;
    const unsigned g = *genp;
    __threadfence();
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nb - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned polls = 0;
      while (*genp == g) {
        if (((++polls) & 255u) == 0 && global_ns() - t0 > 2000000000ull) {
          atomicCAS(status, 0, LYAP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (*(volatile int*)status != 0) { ok = 0; break; }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}


// Copy/convert helpers (all launched on stream s)
// dst (row-major n x n, type T) = scale * src (column-major FP64, lda)   (transpose + cast)
template <typename T>
int cm64_to_rm(const double* src, int64_t n, int64_t lda, double scale, T* dst, cudaStream_t s);
// dst (column-major m x n, ldd, type D) = scale * src (column-major, lds, type S)
template <typename S, typename D>
int copy_cast(const S* src, int64_t m, int64_t n, int64_t lds, D* dst, int64_t ldd, double scale,
              cudaStream_t s);
// round every entry of a FP64 matrix to precision prec (with a power-of-two range
// shift for FP16), in place
int round_to_prec(double* x, int64_t m, int64_t n, int64_t ld, int prec, double* scratch, cudaStream_t s);
// scale columns: x[:, j] *= d[j]  (d device FP64)
template <typename T>
int scale_cols(T* x, int64_t m, int64_t n, int64_t ld, const double* d, cudaStream_t s);
// set matrix to zero / identity
template <typename T>
int set_zero(T* x, int64_t m, int64_t n, int64_t ld, cudaStream_t s);
template <typename T>
int set_identity(T* x, int64_t n, int64_t ld, cudaStream_t s);

// Check an FP64 matrix for NaN/Inf; *flag (device int) becomes 1 if any.
int check_finite(const double* x, int64_t m, int64_t n, int64_t ld, int* flag, cudaStream_t s);

}  // namespace lyap
