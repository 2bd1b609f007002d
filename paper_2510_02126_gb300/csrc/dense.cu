#include "dense.cuh"
#include "ozaki.cuh"

namespace lyap {

// ---------------------------------------------------------------------------
// SIMT GEMM: 64 x 64 output tile, 16-deep K slices, 256 threads with 4 x 4 outputs.
// Thread (tx, ty) owns rows tx + 16 a and columns ty + 16 b, so that every store
// of a half warp covers 16 consecutive rows of the column-major C.
// ---------------------------------------------------------------------------
// TILE x TILE output tile (TILE = 64 or 32), 16-deep K slices, 256 threads, each owning
// (TILE/16) x (TILE/16) outputs.
// SYM: the result is symmetric (M == N, e.g. X^T X or X^T (H X) with H symmetric): only
// tiles on or above the diagonal are computed; each writes its upper-triangle entries
// (i <= j) and mirrors the strictly upper ones to (j, i), so every entry is written once.
template <typename T, bool TA, bool TB, int TILE, bool SYM = false>
__global__ void __launch_bounds__(256)
gemm_kernel(int64_t M, int64_t N, int64_t K, T alpha, const T* __restrict__ A, int64_t lda,
            const T* __restrict__ B, int64_t ldb, T beta, T* __restrict__ C, int64_t ldc) {
  if (SYM && blockIdx.x > blockIdx.y) return;
  constexpr int RA = TILE / 16;            // outputs per thread along each dimension
  constexpr int LD = TILE * 16 / 256;      // loads per thread per operand slice
  __shared__ T As[16][TILE + 1];
  __shared__ T Bs[16][TILE + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * TILE, n0 = (int64_t)blockIdx.y * TILE;
  T acc[RA][RA];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < RA; ++b) acc[a][b] = T(0);
  for (int64_t k0 = 0; k0 < K; k0 += 16) {
    // A tile: As[p][i] = op(A)(m0 + i, k0 + p)
#pragma unroll
    for (int e = 0; e < LD; ++e) {
      const int idx = tid + e * 256;
      int i, p;
      if (TA) { p = idx & 15; i = idx >> 4; } else { i = idx % TILE; p = idx / TILE; }
      const int64_t gi = m0 + i, gp = k0 + p;
      T v = T(0);
      if (gi < M && gp < K) v = TA ? A[gp + gi * lda] : A[gi + gp * lda];
      As[p][i] = v;
    }
    // B tile: Bs[p][j] = op(B)(k0 + p, n0 + j)
#pragma unroll
    for (int e = 0; e < LD; ++e) {
      const int idx = tid + e * 256;
      int j, p;
      if (TB) { j = idx % TILE; p = idx / TILE; } else { p = idx & 15; j = idx >> 4; }
      const int64_t gj = n0 + j, gp = k0 + p;
      T v = T(0);
      if (gj < N && gp < K) v = TB ? B[gj + gp * ldb] : B[gp + gj * ldb];
      Bs[p][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 16; ++p) {
      T av[RA], bv[RA];
#pragma unroll
      for (int a = 0; a < RA; ++a) av[a] = As[p][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < RA; ++b) bv[b] = Bs[p][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < RA; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < RA; ++b) {
    const int64_t j = n0 + ty + 16 * b;
    if (j >= N) continue;
#pragma unroll
    for (int a = 0; a < RA; ++a) {
      const int64_t i = m0 + tx + 16 * a;
      if (i >= M) continue;
      if (SYM && i > j) continue;  // written by the mirror of (j, i)
      T* c = C + i + j * ldc;
      const T v = (beta == T(0)) ? alpha * acc[a][b] : alpha * acc[a][b] + beta * *c;
      *c = v;
      if (SYM && i < j) C[j + i * ldc] = v;  // C was symmetric on entry when beta != 0
    }
  }
}

static int g_num_sms = 0;
static int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

static thread_local int g_dgemm_method = DGEMM_AUTO;
void set_dgemm_method(int method) { g_dgemm_method = method; }
int dgemm_method() { return g_dgemm_method; }

// FP64 products large enough for the tensor-core emulation (or forced to it)
static bool use_tensor_fp64(int64_t M, int64_t N, int64_t K) {
  if (g_dgemm_method == DGEMM_SIMT) return false;
  if (g_dgemm_method == DGEMM_TENSOR) return true;
  // enough work, a K worth the digit split, and enough (128 x 32 tile, K split) pairs to occupy
  // the GPU: ozaki_dgemm splits K into up to 16 ranges of at least 256 when tiles are few
  const int64_t tiles = ceil_div(M, 128) * ceil_div(N, 32);
  const int64_t splits = std::max<int64_t>(1, std::min<int64_t>(16, K / 256));
  return (double)M * (double)N * (double)K >= OZ_MIN_MACS && K >= 128 && tiles * splits >= 48;
}

// C[j, i] = C[i, j] for i < j (the upper triangle of a symmetric product is the result)
__global__ void mirror_upper_kernel(double* __restrict__ C, int64_t N, int64_t ldc) {
  const int64_t total = N * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / N, i = e - j * N;
    if (i > j) C[i + j * ldc] = C[j + i * ldc];
  }
}

template <typename T, int TILE>
static void gemm_launch(bool TA, bool TB, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda,
                        const T* B, int64_t ldb, T beta, T* C, int64_t ldc, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(M, TILE), (unsigned)ceil_div(N, TILE));
  if (!TA && !TB) gemm_kernel<T, false, false, TILE><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (TA && !TB) gemm_kernel<T, true, false, TILE><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (!TA && TB) gemm_kernel<T, false, true, TILE><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else gemm_kernel<T, true, true, TILE><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

template <typename T>
int gemm(char ta, char tb, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda,
         const T* B, int64_t ldb, T beta, T* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return LYAP_OK;
  if (K <= 0) {
    if (beta == T(0)) return set_zero<T>(C, M, N, ldc, s);
    return scale_cols<T>(C, M, N, ldc, nullptr, s);  // beta must be 0 or 1 here
  }
  if constexpr (sizeof(T) == 8) {
    if (use_tensor_fp64(M, N, K)) return ozaki_dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  }
  const bool TA = (ta == 'T' || ta == 't'), TB = (tb == 'T' || tb == 't');
  // 64-wide tiles when they already give every SM two tiles, 32-wide tiles otherwise
  if (ceil_div(M, 64) * ceil_div(N, 64) >= 2 * num_sms())
    gemm_launch<T, 64>(TA, TB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  else
    gemm_launch<T, 32>(TA, TB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}
template int gemm<float>(char, char, int64_t, int64_t, int64_t, float, const float*, int64_t, const float*,
                         int64_t, float, float*, int64_t, cudaStream_t);

template <typename T>
int gemm_sym(char ta, char tb, int64_t N, int64_t K, T alpha, const T* A, int64_t lda, const T* B, int64_t ldb,
             T beta, T* C, int64_t ldc, cudaStream_t s) {
  if (N <= 0) return LYAP_OK;
  if (K <= 0) return gemm<T>(ta, tb, N, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  if constexpr (sizeof(T) == 8) {
    if (use_tensor_fp64(N, N, K)) {
      // the full product, then its upper triangle mirrored (exact symmetry, as below)
      LYAP_TRY(ozaki_dgemm(ta, tb, N, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s));
      mirror_upper_kernel<<<(unsigned)std::min<int64_t>(4096, ceil_div(N * N, 256)), 256, 0, s>>>(C, N, ldc);
      LYAP_CUDA_TRY(cudaGetLastError());
      lyap_count_launch();
      return LYAP_OK;
    }
  }
  const bool TA = (ta == 'T' || ta == 't'), TB = (tb == 'T' || tb == 't');
  constexpr int TILE = 32;
  dim3 grid((unsigned)ceil_div(N, TILE), (unsigned)ceil_div(N, TILE));
  if (TA && !TB) gemm_kernel<T, true, false, TILE, true><<<grid, 256, 0, s>>>(N, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (!TA && TB) gemm_kernel<T, false, true, TILE, true><<<grid, 256, 0, s>>>(N, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (!TA && !TB) gemm_kernel<T, false, false, TILE, true><<<grid, 256, 0, s>>>(N, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else gemm_kernel<T, true, true, TILE, true><<<grid, 256, 0, s>>>(N, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}
template int gemm_sym<double>(char, char, int64_t, int64_t, double, const double*, int64_t, const double*, int64_t,
                              double, double*, int64_t, cudaStream_t);
template int gemm<double>(char, char, int64_t, int64_t, int64_t, double, const double*, int64_t,
                          const double*, int64_t, double, double*, int64_t, cudaStream_t);

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename T, int OPK>  // OPK 0 = sum of squares, 1 = max abs
__global__ void __launch_bounds__(256) reduce_kernel(const T* __restrict__ x, int64_t m, int64_t n,
                                                     int64_t ld, double* __restrict__ part) {
  const int64_t total = m * n;
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
    const int64_t j = e / m, i = e - j * m;
    const double v = (double)x[i + j * ld];
    if (OPK == 0) acc = fma(v, v, acc); else acc = fmax(acc, fabs(v));
  }
  __shared__ double sh[8];
  acc = (OPK == 0) ? warp_sum(acc) : warp_max(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < 8) ? sh[threadIdx.x] : 0.0;
    v = (OPK == 0) ? warp_sum(v) : warp_max(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}
template <int OPK>
__global__ void reduce_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) acc = (OPK == 0) ? acc + part[i] : fmax(acc, part[i]);
  acc = (OPK == 0) ? warp_sum(acc) : warp_max(acc);
  if (threadIdx.x == 0) *out = acc;
}

template <typename T, int OPK>
static int reduce_run(const T* x, int64_t m, int64_t n, int64_t ld, double* out, double* part, cudaStream_t s) {
  if (m <= 0 || n <= 0) {
    LYAP_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
    return LYAP_OK;
  }
  const int64_t total = m * n;
  int nb = (int)std::min<int64_t>(RED_BLOCKS, ceil_div(total, 256));
  reduce_kernel<T, OPK><<<nb, 256, 0, s>>>(x, m, n, ld, part);
  reduce_final<OPK><<<1, 32, 0, s>>>(part, nb, out);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch(2);
  return LYAP_OK;
}
template <typename T>
int sumsq(const T* x, int64_t m, int64_t n, int64_t ld, double* out, double* part, cudaStream_t s) {
  return reduce_run<T, 0>(x, m, n, ld, out, part, s);
}
template <typename T>
int maxabs(const T* x, int64_t m, int64_t n, int64_t ld, double* out, double* part, cudaStream_t s) {
  return reduce_run<T, 1>(x, m, n, ld, out, part, s);
}
template int sumsq<float>(const float*, int64_t, int64_t, int64_t, double*, double*, cudaStream_t);
template int sumsq<double>(const double*, int64_t, int64_t, int64_t, double*, double*, cudaStream_t);
template int maxabs<float>(const float*, int64_t, int64_t, int64_t, double*, double*, cudaStream_t);
template int maxabs<double>(const double*, int64_t, int64_t, int64_t, double*, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// grid barrier
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// copies and casts
// ---------------------------------------------------------------------------
template <typename T>
__global__ void cm64_to_rm_kernel(const double* __restrict__ src, int64_t n, int64_t lda, double scale,
                                  T* __restrict__ dst) {
  __shared__ double tile[32][33];
  const int64_t bi = (int64_t)blockIdx.y * 32, bj = (int64_t)blockIdx.x * 32;
  // read column-major: consecutive threads -> consecutive rows i
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = bi + threadIdx.x, j = bj + r;
    tile[r][threadIdx.x] = (i < n && j < n) ? src[i + j * lda] : 0.0;
  }
  __syncthreads();
  // write row-major: consecutive threads -> consecutive columns j
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = bi + r, j = bj + threadIdx.x;
    if (i < n && j < n) dst[i * n + j] = (T)(scale * tile[threadIdx.x][r]);
  }
}
template <typename T>
int cm64_to_rm(const double* src, int64_t n, int64_t lda, double scale, T* dst, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(n, 32));
  cm64_to_rm_kernel<T><<<grid, dim3(32, 8), 0, s>>>(src, n, lda, scale, dst);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}
template int cm64_to_rm<float>(const double*, int64_t, int64_t, double, float*, cudaStream_t);
template int cm64_to_rm<double>(const double*, int64_t, int64_t, double, double*, cudaStream_t);

template <typename S, typename D>
__global__ void copy_cast_kernel(const S* __restrict__ src, int64_t m, int64_t n, int64_t lds, D* __restrict__ dst,
                                 int64_t ldd, double scale) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    dst[i + j * ldd] = (D)(scale * (double)src[i + j * lds]);
  }
}
template <typename S, typename D>
int copy_cast(const S* src, int64_t m, int64_t n, int64_t lds, D* dst, int64_t ldd, double scale, cudaStream_t s) {
  if (m <= 0 || n <= 0) return LYAP_OK;
  const int64_t total = m * n;
  const int nb = (int)std::min<int64_t>(4096, ceil_div(total, 256));
  copy_cast_kernel<S, D><<<nb, 256, 0, s>>>(src, m, n, lds, dst, ldd, scale);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}
template int copy_cast<double, double>(const double*, int64_t, int64_t, int64_t, double*, int64_t, double, cudaStream_t);
template int copy_cast<double, float>(const double*, int64_t, int64_t, int64_t, float*, int64_t, double, cudaStream_t);
template int copy_cast<float, double>(const float*, int64_t, int64_t, int64_t, double*, int64_t, double, cudaStream_t);
template int copy_cast<float, float>(const float*, int64_t, int64_t, int64_t, float*, int64_t, double, cudaStream_t);

__global__ void round_prec_kernel(double* __restrict__ x, int64_t m, int64_t n, int64_t ld, int prec,
                                  const double* __restrict__ amax) {
  const int64_t total = m * n;
  int e = 0;
  if (prec == LYAP_FP16) e = pow2_exponent(*amax);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / m, i = idx - j * m;
    double v = x[i + j * ld];
    if (prec == LYAP_FP32) v = (double)(float)v;
    else if (prec == LYAP_BF16) v = (double)__bfloat162float(__float2bfloat16_rn((float)v));
    else if (prec == LYAP_FP16) v = ldexp((double)__half2float(__float2half_rn((float)ldexp(v, -e))), e);
    x[i + j * ld] = v;
  }
}
int round_to_prec(double* x, int64_t m, int64_t n, int64_t ld, int prec, double* scratch, cudaStream_t s) {
  if (prec == LYAP_FP64 || m <= 0 || n <= 0) return LYAP_OK;
  LYAP_TRY(maxabs<double>(x, m, n, ld, scratch, scratch + 1, s));
  const int nb = (int)std::min<int64_t>(4096, ceil_div(m * n, 256));
  round_prec_kernel<<<nb, 256, 0, s>>>(x, m, n, ld, prec, scratch);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}

template <typename T>
__global__ void scale_cols_kernel(T* __restrict__ x, int64_t m, int64_t n, int64_t ld, const double* __restrict__ d) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    if (d) x[i + j * ld] = (T)((double)x[i + j * ld] * d[j]);
  }
}
template <typename T>
int scale_cols(T* x, int64_t m, int64_t n, int64_t ld, const double* d, cudaStream_t s) {
  if (m <= 0 || n <= 0 || d == nullptr) return LYAP_OK;
  const int nb = (int)std::min<int64_t>(4096, ceil_div(m * n, 256));
  scale_cols_kernel<T><<<nb, 256, 0, s>>>(x, m, n, ld, d);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}
template int scale_cols<float>(float*, int64_t, int64_t, int64_t, const double*, cudaStream_t);
template int scale_cols<double>(double*, int64_t, int64_t, int64_t, const double*, cudaStream_t);

template <typename T>
__global__ void set_kernel(T* __restrict__ x, int64_t m, int64_t n, int64_t ld, int ident) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    x[i + j * ld] = (ident && i == j) ? T(1) : T(0);
  }
}
template <typename T>
int set_zero(T* x, int64_t m, int64_t n, int64_t ld, cudaStream_t s) {
  if (m <= 0 || n <= 0) return LYAP_OK;
  const int nb = (int)std::min<int64_t>(4096, ceil_div(m * n, 256));
  set_kernel<T><<<nb, 256, 0, s>>>(x, m, n, ld, 0);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}
template <typename T>
int set_identity(T* x, int64_t n, int64_t ld, cudaStream_t s) {
  if (n <= 0) return LYAP_OK;
  const int nb = (int)std::min<int64_t>(4096, ceil_div(n * n, 256));
  set_kernel<T><<<nb, 256, 0, s>>>(x, n, n, ld, 1);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}
template int set_zero<float>(float*, int64_t, int64_t, int64_t, cudaStream_t);
template int set_zero<double>(double*, int64_t, int64_t, int64_t, cudaStream_t);
template int set_identity<float>(float*, int64_t, int64_t, cudaStream_t);
template int set_identity<double>(double*, int64_t, int64_t, cudaStream_t);

__global__ void check_finite_kernel(const double* __restrict__ x, int64_t m, int64_t n, int64_t ld, int* flag) {
  const int64_t total = m * n;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    if (!isfinite(x[i + j * ld])) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}
int check_finite(const double* x, int64_t m, int64_t n, int64_t ld, int* flag, cudaStream_t s) {
  if (m <= 0 || n <= 0) return LYAP_OK;
  const int nb = (int)std::min<int64_t>(1024, ceil_div(m * n, 256));
  check_finite_kernel<<<nb, 256, 0, s>>>(x, m, n, ld, flag);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}

}  // namespace lyap
