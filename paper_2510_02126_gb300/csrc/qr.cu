// Householder QR kernels.  Both factorisations are cooperative launches: the
// columns are distributed cyclically over the CTAs (one warp per column at a
// time) and the CTAs meet at a bounded grid barrier between reflectors, so the
// FP64 arithmetic of the trailing updates runs on many SMs at once.
#include "qr.cuh"

#include <atomic>

namespace lyap {

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T t = (lane < nw) ? red[lane] : T(0);
  t = warp_sum(t);
  return t;  // valid in every warp
}

// ---------------------------------------------------------------------------
// thin Householder QR (cooperative, with lookahead)
//
// Column l is owned by CTA l mod G.  Reflector j is published behind a per-column flag
// instead of a grid barrier: the owner of column j+1 applies H_j to that column first
// (the whole CTA on one column), forms reflector j+1, publishes it, and only then applies
// H_j to its other columns; every CTA waits (bounded) for flag j before applying H_j.
// The critical path per column is thus one column update and one reflector, not a grid
// barrier plus the slowest CTA's update.
// ---------------------------------------------------------------------------
// Reflector of column j (rows j..m-1) in place, by the whole CTA: v below the diagonal
// (unit leading entry implicit), beta on the diagonal, tau[j].
template <typename T>
__device__ void hqr_reflector(T* __restrict__ F, int64_t m, int64_t ld, int64_t j, T* __restrict__ tau, T* red) {
  T* x = F + j + j * ld;
  T sig = T(0);
  for (int64_t i = 1 + threadIdx.x; i < m - j; i += blockDim.x) sig = fma(x[i], x[i], sig);
  sig = block_sum(sig, red);
  const T alpha = x[0];
  T beta, tj, scale;
  if (sig == T(0)) {
    tj = T(0);
    beta = alpha;
    scale = T(0);
  } else {
    const T nrm = sqrt(alpha * alpha + sig);
    beta = (alpha <= T(0)) ? nrm : -nrm;
    tj = (beta - alpha) / beta;
    scale = T(1) / (alpha - beta);
  }
  __syncthreads();
  for (int64_t i = 1 + threadIdx.x; i < m - j; i += blockDim.x) x[i] *= scale;
  if (threadIdx.x == 0) { x[0] = beta; tau[j] = tj; }
}

// y <- H_j y for one column y (rows j..m-1), by one warp (v, tj read L2-coherently)
template <typename T>
__device__ __forceinline__ void hqr_apply_warp(const T* __restrict__ v, T tj, T* __restrict__ y, int64_t len) {
  const int lane = threadIdx.x & 31;
  T w = T(0);
  for (int64_t i = 1 + lane; i < len; i += 32) w = fma(__ldcg(&v[i]), y[i], w);
  w = (warp_sum(w) + y[0]) * tj;
  __syncwarp();
  if (lane == 0) y[0] -= w;
  for (int64_t i = 1 + lane; i < len; i += 32) y[i] = fma(-w, __ldcg(&v[i]), y[i]);
}

// H_j applied to the owned columns lg, lg + G, ..., lg + (nc - 1) G (nc <= HQR_NC) by the whole
// CTA: thread t takes rows 1 + t, 1 + t + blockDim.x, ... of every column of the group, so a
// group costs one pass for the dot products, one block reduction and one pass for the
// updates -- not one warp's pass over all m - j rows per column.  v and tj: reflector j;
// y0 = F + j (row j of the matrix).
constexpr int HQR_NC = 8;
constexpr int64_t QR_GROUP_MIN_M = 2048;  // the CTA-wide forms above this many rows
template <typename T>
__device__ __forceinline__ void hqr_apply_group(const T* __restrict__ v, T tj, T* __restrict__ y0, int64_t len,
                                                int64_t ld, int64_t lg, int G, int nc, T* redc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T part[HQR_NC];
#pragma unroll
  for (int c = 0; c < HQR_NC; ++c) part[c] = T(0);
  for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) {
    const T vi = __ldcg(&v[i]);
#pragma unroll
    for (int c = 0; c < HQR_NC; ++c)
      if (c < nc) part[c] = fma(vi, y0[i + (lg + (int64_t)c * G) * ld], part[c]);
  }
#pragma unroll
  for (int c = 0; c < HQR_NC; ++c) part[c] = warp_sum(part[c]);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < HQR_NC; ++c) redc[warp * HQR_NC + c] = part[c];
  __syncthreads();
  T w[HQR_NC];
#pragma unroll
  for (int c = 0; c < HQR_NC; ++c) {
    T t = T(0);
    if (c < nc) {
      for (int k = 0; k < nw; ++k) t += redc[k * HQR_NC + c];
      t = (t + y0[(lg + (int64_t)c * G) * ld]) * tj;
    }
    w[c] = t;
  }
  __syncthreads();  // every thread has read the row-j entries and redc
#pragma unroll
  for (int c = 0; c < HQR_NC; ++c)
    if (c < nc && threadIdx.x == c) y0[(lg + (int64_t)c * G) * ld] -= w[c];
  for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) {
    const T vi = __ldcg(&v[i]);
#pragma unroll
    for (int c = 0; c < HQR_NC; ++c)
      if (c < nc) {
        T* y = y0 + i + (lg + (int64_t)c * G) * ld;
        *y = fma(-w[c], vi, *y);
      }
  }
}

// GROUP: the columns a CTA owns beyond the lookahead column take each reflector in groups of
// HQR_NC by the whole CTA (tall matrices); else one warp per column (cheaper per reflector
// while a warp's pass over the m - j rows is short).
template <typename T, bool GROUP>
__global__ void __launch_bounds__(256)
hqr_kernel(T* __restrict__ F, int64_t m, int64_t q, int64_t ld, T* __restrict__ tau, int* __restrict__ flags,
           int* status) {
  __shared__ T red[32];
  __shared__ T redc[8 * HQR_NC];
  __shared__ int ok_s;
  const int G = gridDim.x, b = blockIdx.x;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t kmax = (m < q) ? m : q;
  if (kmax <= 0) return;
  auto publish = [&](int64_t j) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(&flags[j], 1);
    }
  };
  if (b == 0) {
    hqr_reflector<T>(F, m, ld, 0, tau, red);
    publish(0);
  }
  for (int64_t j = 0; j < kmax; ++j) {
    // wait for reflector j (bounded)
    if ((j % G) != b) {
      if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = global_ns();
        unsigned polls = 0;
        while (atomicAdd(&flags[j], 0) == 0) {
          if (((++polls) & 255u) == 0 && global_ns() - t0 > 2000000000ull) {
            atomicCAS(status, 0, LYAP_ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
        ok_s = ok;
      }
      __syncthreads();
      if (!ok_s) return;
    }
    const T tj = __ldcg(&tau[j]);
    const T* v = F + j + j * ld;
    const int64_t len = m - j;
    // lookahead: the owner of column j+1 updates it with the whole CTA, then publishes
    // reflector j+1 before touching its other columns
    const int64_t l1 = j + 1;
    if (l1 < q && (l1 % G) == b) {
      T* y = F + j + l1 * ld;
      T w = T(0);
      for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) w = fma(__ldcg(&v[i]), y[i], w);
      w = block_sum(w, red);
      w = (w + y[0]) * tj;
      __syncthreads();  // every thread has read y[0]
      if (threadIdx.x == 0) y[0] -= w;
      for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) y[i] = fma(-w, __ldcg(&v[i]), y[i]);
      __syncthreads();
      if (l1 < kmax) {
        hqr_reflector<T>(F, m, ld, l1, tau, red);
        publish(l1);
      }
    }
    // the remaining owned columns l > j + 1
    if (GROUP) {
      int64_t lstart = b;
      if (lstart <= l1) lstart += ((l1 - lstart) / G + 1) * G;
      for (int64_t lg = lstart; lg < q; lg += (int64_t)G * HQR_NC) {
        const int64_t left = (q - lg + G - 1) / G;
        const int nc = (int)(left < HQR_NC ? left : HQR_NC);
        hqr_apply_group<T>(v, tj, F + j, len, ld, lg, G, nc, redc);
        __syncthreads();  // redc is reused by the next group
      }
    } else {
      int slot = 0;
      for (int64_t l = b; l < q; l += G) {
        if (l <= l1) continue;
        if ((slot++ % nw) != warp) continue;
        hqr_apply_warp<T>(v, tj, F + j + l * ld, len);
      }
    }
    __syncthreads();
  }
}

template <typename T>
static int hqr_unblocked(T* F, int64_t m, int64_t q, int64_t ld, T* tau, QRScratch& sc, cudaStream_t s) {
  if (m <= 0 || q <= 0) return LYAP_OK;
  int G = (int)std::min<int64_t>(q, sc.num_sms);
  if (G < 1) G = 1;
  const int64_t kmax = std::min(m, q);
  LYAP_CUDA_TRY(cudaMemsetAsync(sc.flags, 0, sizeof(int) * (size_t)kmax, s));
  void* args[] = {&F, &m, &q, &ld, &tau, &sc.flags, &sc.status};
  // measured: the grouped form cuts the time per reflector at m = 4096 (24 -> 17 us) and
  // loses about a fifth at m = 1024
  void* fn = (m > QR_GROUP_MIN_M) ? (void*)hqr_kernel<T, true> : (void*)hqr_kernel<T, false>;
  LYAP_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(256), args, 0, s));
  lyap_count_launch();
  return LYAP_OK;
}

// ---------------------------------------------------------------------------
// Y = H_0 ... H_{k-1} [C; 0]: the columns of Y are independent.  Tall Q: a CTA takes NC of
// them and applies the reflectors in reverse order, each as one pass of dot products over
// the rows (all threads), one block reduction and one pass of updates.
// ---------------------------------------------------------------------------
template <typename T, int NC>
__global__ void __launch_bounds__(256)
apply_q_kernel(const T* __restrict__ F, int64_t m, int64_t k, int64_t ldf, const T* __restrict__ tau,
               const T* __restrict__ C, int64_t ldc, int64_t r, T* __restrict__ Y, int64_t ldy) {
  __shared__ T redc[8 * NC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * NC;
  if (c0 >= r) return;
  const int nc = (int)((r - c0 < NC) ? r - c0 : NC);
  T* y0 = Y + c0 * ldy;
  for (int c = 0; c < nc; ++c)
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x)
      y0[i + c * ldy] = (i < k) ? C[i + (c0 + c) * ldc] : T(0);
  __syncthreads();
  for (int64_t j = k - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj == T(0)) continue;  // H_j = I
    const T* v = F + j + j * ldf;
    T* yj = y0 + j;
    const int64_t len = m - j;
    T part[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) part[c] = T(0);
    for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) {
      const T vi = v[i];
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < nc) part[c] = fma(vi, yj[i + c * ldy], part[c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) part[c] = warp_sum(part[c]);
    if (lane == 0)
#pragma unroll
      for (int c = 0; c < NC; ++c) redc[warp * NC + c] = part[c];
    __syncthreads();
    T w[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T t = T(0);
      if (c < nc) {
        for (int q = 0; q < nw; ++q) t += redc[q * NC + c];
        t = (t + yj[c * ldy]) * tj;
      }
      w[c] = t;
    }
    __syncthreads();  // every thread has read yj[0] and redc
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < nc && threadIdx.x == c) yj[c * ldy] -= w[c];
    for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) {
      const T vi = v[i];
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < nc) yj[i + c * ldy] = fma(-w[c], vi, yj[i + c * ldy]);
    }
    __syncthreads();  // the next reflector reads rows written here by other threads
  }
}

// the same with one warp per column of Y (short columns: a warp's pass is cheaper than a
// block reduction per reflector)
template <typename T>
__global__ void __launch_bounds__(32)
apply_q_warp_kernel(const T* __restrict__ F, int64_t m, int64_t k, int64_t ldf, const T* __restrict__ tau,
               const T* __restrict__ C, int64_t ldc, int64_t r, T* __restrict__ Y, int64_t ldy) {
  const int64_t col = blockIdx.x;
  if (col >= r) return;
  const int lane = threadIdx.x;
  T* y = Y + col * ldy;
  for (int64_t i = lane; i < m; i += 32) y[i] = (i < k) ? C[i + col * ldc] : T(0);
  __syncwarp();
  for (int64_t j = k - 1; j >= 0; --j) {
    const T* v = F + j + j * ldf;
    T* yj = y + j;
    T w = T(0);
    for (int64_t i = 1 + lane; i < m - j; i += 32) w = fma(v[i], yj[i], w);
    w = warp_sum(w) + yj[0];
    w *= tau[j];
    __syncwarp();
    if (lane == 0) yj[0] -= w;
    for (int64_t i = 1 + lane; i < m - j; i += 32) yj[i] = fma(-w, v[i], yj[i]);
    __syncwarp();
  }
}

template <typename T>
static int apply_q_unblocked(const T* F, int64_t m, int64_t k, int64_t ldf, const T* tau, const T* C, int64_t ldc,
                             int64_t r, T* Y, int64_t ldy, cudaStream_t s) {
  if (r <= 0 || m <= 0) return LYAP_OK;
  if (m <= QR_GROUP_MIN_M) {
    apply_q_warp_kernel<T><<<(unsigned)r, 32, 0, s>>>(F, m, k, ldf, tau, C, ldc, r, Y, ldy);
  } else {
    // one column per CTA while that keeps the SMs busy, more per CTA for wide Y (shared
    // loads of v); measured at 4096 x 543 with 270 columns: 6.3 -> 3.2 ms
    int dev = 0, sms = 1;
    LYAP_CUDA_TRY(cudaGetDevice(&dev));
    LYAP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (r <= 2 * (int64_t)sms)
      apply_q_kernel<T, 1><<<(unsigned)r, 256, 0, s>>>(F, m, k, ldf, tau, C, ldc, r, Y, ldy);
    else if (r <= 4 * (int64_t)sms)
      apply_q_kernel<T, 2><<<(unsigned)ceil_div(r, 2), 256, 0, s>>>(F, m, k, ldf, tau, C, ldc, r, Y, ldy);
    else
      apply_q_kernel<T, 4><<<(unsigned)ceil_div(r, 4), 256, 0, s>>>(F, m, k, ldf, tau, C, ldc, r, Y, ldy);
  }
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}

// The factorisation and the application of Q stay unblocked: their cost is the chain of
// reflectors (a reduction each on the critical path), which a blocked (compact WY) variant
// keeps in its panels while adding the trailing products -- measured slower at the orders
// of the refinement (1024 x 846 and 4096 x 547: about 1.5-2x).
template <typename T>
int householder_qr(T* F, int64_t m, int64_t q, int64_t ld, T* tau, QRScratch& sc, cudaStream_t s) {
  return hqr_unblocked<T>(F, m, q, ld, tau, sc, s);
}
template int householder_qr<float>(float*, int64_t, int64_t, int64_t, float*, QRScratch&, cudaStream_t);
template int householder_qr<double>(double*, int64_t, int64_t, int64_t, double*, QRScratch&, cudaStream_t);

template <typename T>
int apply_q(const T* F, int64_t m, int64_t k, int64_t ldf, const T* tau, const T* C, int64_t ldc,
            int64_t r, T* Y, int64_t ldy, cudaStream_t s) {
  return apply_q_unblocked<T>(F, m, k, ldf, tau, C, ldc, r, Y, ldy, s);
}
template int apply_q<float>(const float*, int64_t, int64_t, int64_t, const float*, const float*, int64_t,
                            int64_t, float*, int64_t, cudaStream_t);
template int apply_q<double>(const double*, int64_t, int64_t, int64_t, const double*, const double*, int64_t,
                             int64_t, double*, int64_t, cudaStream_t);

// ---------------------------------------------------------------------------
// QR with column pivoting of M = Z^T (c x n); columns of M = rows of Z
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
qrcp_kernel(T* __restrict__ Z, int64_t n, int64_t c, int64_t ldz, double tol, T* __restrict__ M,
            T* __restrict__ nrm, T* __restrict__ nrm_ref, int* __restrict__ piv, T* __restrict__ rdiag,
            double* __restrict__ cand, int* __restrict__ rank_out, GridBar* bar, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* v = reinterpret_cast<T*>(smem_raw);  // reflector, length c
  __shared__ T red[32];
  __shared__ double redd[32];
  __shared__ int redi[32];
  __shared__ double r11_s;
  const int G = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

  // copy-in: M[:, i] = Z[i, :], norms, identity pivots (owned columns i = b mod G)
  for (int64_t i = b; i < n; i += G) {
    T acc = T(0);
    for (int64_t l = threadIdx.x; l < c; l += blockDim.x) {
      const T z = Z[i + l * ldz];
      M[l + i * c] = z;
      acc = fma(z, z, acc);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) { nrm[i] = acc; nrm_ref[i] = acc; piv[i] = (int)i; }
  }
  const int64_t kmax = (c < n) ? c : n;
  int64_t r = kmax;
  for (int64_t j = 0; j < kmax; ++j) {
    // (1) local argmax and tail sum over owned columns i >= j
    double bv = -1.0, ts = 0.0;
    int bi = -1;
    for (int64_t i = b + (int64_t)threadIdx.x * G; i < n; i += (int64_t)blockDim.x * G) {
      if (i < j) continue;
      const double w = (double)nrm[i];
      ts += w;
      if (bi < 0 || w > bv) { bv = w; bi = (int)i; }
    }
    warp_argmax(bv, bi);
    ts = warp_sum(ts);
    __syncthreads();
    if (lane == 0) { redd[warp] = bv; redi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      double v2 = (lane < nw) ? redd[lane] : -1.0;
      int i2 = (lane < nw) ? redi[lane] : -1;
      warp_argmax(v2, i2);
      if (lane == 0) { cand[3 * b] = v2; cand[3 * b + 1] = (double)i2; }
    }
    __syncthreads();
    if (lane == 0) redd[warp] = ts;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += redd[w];
      cand[3 * b + 2] = t;
    }
    if (!grid_sync(bar, status)) return;
    // (2) global pivot + truncation test (identical in every block)
    double pv = -1.0, tail = 0.0;
    int p = -1;
    for (int e = lane; e < G; e += 32) {
      const double cv = cand[3 * e];
      const int ci = (int)cand[3 * e + 1];
      if (ci >= 0 && (p < 0 || cv > pv || (cv == pv && ci < p))) { pv = cv; p = ci; }
    }
    warp_argmax(pv, p);
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int e = lane; e < G; e += 32) t += cand[3 * e + 2];
      t = warp_sum(t);
      if (threadIdx.x == 0) redd[0] = t;
    }
    __syncthreads();
    tail = redd[0];
    __syncthreads();
    if (j == 0 && !(tail > 0.0)) { r = 0; break; }
    if (j >= 1 && sqrt(fmax(tail, 0.0)) <= tol * r11_s) { r = j; break; }
    // (3) swap columns j <-> p (block 0), then everybody reads column j
    if (b == 0 && p != (int)j) {
      for (int64_t l = threadIdx.x; l < c; l += blockDim.x) {
        const T a = M[l + j * c];
        M[l + j * c] = M[l + (int64_t)p * c];
        M[l + (int64_t)p * c] = a;
      }
      if (threadIdx.x == 0) {
        T t = nrm[j]; nrm[j] = nrm[p]; nrm[p] = t;
        t = nrm_ref[j]; nrm_ref[j] = nrm_ref[p]; nrm_ref[p] = t;
        const int q = piv[j]; piv[j] = piv[p]; piv[p] = q;
      }
    }
    if (!grid_sync(bar, status)) return;
    // (4) reflector from column j (computed redundantly, kept in shared memory)
    const T* x = M + j + j * c;
    T sig = T(0);
    for (int64_t l = 1 + threadIdx.x; l < c - j; l += blockDim.x) sig = fma(x[l], x[l], sig);
    sig = block_sum(sig, red);
    const T alpha = x[0];
    T beta, tj, scale;
    if (sig == T(0)) { beta = alpha; tj = T(0); scale = T(0); }
    else {
      const T nrmx = sqrt(alpha * alpha + sig);
      beta = (alpha <= T(0)) ? nrmx : -nrmx;
      tj = (beta - alpha) / beta;
      scale = T(1) / (alpha - beta);
    }
    for (int64_t l = 1 + threadIdx.x; l < c - j; l += blockDim.x) v[l] = x[l] * scale;
    if (threadIdx.x == 0) {
      v[0] = T(1);
      if (j == 0) r11_s = fabs((double)beta);
      if (b == 0) rdiag[j] = beta;
    }
    __syncthreads();
    // (5) apply to owned columns i > j (one warp per column) + norm downdate
    int slot = 0;
    for (int64_t i = b; i < n; i += G) {
      if (i <= j) continue;
      if ((slot++ % nw) != warp) continue;
      T* y = M + j + i * c;
      T w = T(0);
      for (int64_t l = 1 + lane; l < c - j; l += 32) w = fma(v[l], y[l], w);
      w = (warp_sum(w) + y[0]) * tj;
      const T top = y[0] - w;
      T tail2 = T(0);
      for (int64_t l = 1 + lane; l < c - j; l += 32) {
        const T nv = fma(-w, v[l], y[l]);
        y[l] = nv;
        tail2 = fma(nv, nv, tail2);
      }
      if (lane == 0) y[0] = top;
      // downdate ||M[j+1:, i]||^2 ; recompute when cancellation is severe
      T nn = nrm[i] - top * top;
      const T eps = (sizeof(T) == 8) ? T(1.5e-8) : T(3.5e-4);  // ~ sqrt(machine eps)
      if (!(nn > eps * nrm_ref[i])) {
        nn = warp_sum(tail2);
        if (lane == 0) nrm_ref[i] = nn;
      }
      if (lane == 0) nrm[i] = (nn > T(0)) ? nn : T(0);
    }
    __syncthreads();
  }
  if (!grid_sync(bar, status)) return;
  // (6) output: Z[piv[i], l] = R[l, i] for l < r
  for (int64_t i = b; i < n; i += G) {
    const int pi = piv[i];
    for (int64_t l = threadIdx.x; l < r; l += blockDim.x) {
      T val;
      if (l < i) val = M[l + i * c];
      else if (l == i) val = rdiag[i];
      else val = T(0);
      Z[pi + l * ldz] = val;
    }
  }
  if (b == 0 && threadIdx.x == 0) *rank_out = (int)r;
}

// ---------------------------------------------------------------------------
// The same QR with column pivoting with M = Z^T resident in the distributed shared
// memory of one thread-block cluster: CTA `rank` owns columns [rank nc, rank nc + nc).
// Columns are never swapped: each records the step at which it became the pivot, and
// the output is assembled from that at the end.  Every CTA forms the reflector itself
// from the pivot column (read from its owner through DSMEM), so a step takes a single
// cluster barrier (after the candidates of the step are published; the candidate
// slots are double-buffered by step parity).
// ---------------------------------------------------------------------------
// odd column pitch: threads walking different columns of the same row hit distinct banks
__host__ __device__ inline int64_t qrcp_cluster_ld(int64_t c) { return c | 1; }
template <typename T>
__host__ __device__ inline size_t qrcp_cluster_smem(int64_t c, int64_t nc) {
  return sizeof(T) * ((size_t)qrcp_cluster_ld(c) * nc + 3 * (size_t)nc + (size_t)c) + sizeof(int) * (size_t)nc + 64;
}

template <typename T>
__global__ void __launch_bounds__(256, 1)
qrcp_cluster_kernel(T* __restrict__ Z, int n, int c, int64_t ldz, int nc, double tol, int* __restrict__ rank_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ldm = (int)qrcp_cluster_ld(c);
  T* Ms = reinterpret_cast<T*>(smem_raw);  // c x nc, column-major (ld = ldm)
  T* nrm = Ms + (size_t)ldm * nc;
  T* nref = nrm + nc;
  T* bdg = nref + nc;                      // beta of a column chosen as pivot
  T* v = bdg + nc;                         // the step's reflector (length c)
  int* stepof = reinterpret_cast<int*>(v + c);  // step at which the column was chosen, -1 if not
  __shared__ double slot_v[2], slot_t[2];
  __shared__ int slot_i[2];
  __shared__ double redd[8], redt[8];
  __shared__ int redi[8];
  __shared__ T red[32];
  const int rk = (int)cluster_ctarank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int col0 = rk * nc;
  const int ncl = max(0, min(nc, n - col0));
  for (int e = tid; e < c * ncl; e += blockDim.x) {
    const int l = e / ncl, i = e - l * ncl;
    Ms[l + (size_t)i * ldm] = Z[col0 + i + l * ldz];
  }
  __syncthreads();
  for (int i = tid; i < ncl; i += blockDim.x) {
    T acc = T(0);
    for (int l = 0; l < c; ++l) acc = fma(Ms[l + (size_t)i * ldm], Ms[l + (size_t)i * ldm], acc);
    nrm[i] = acc;
    nref[i] = acc;
    stepof[i] = -1;
  }
  __syncthreads();
  const int kmax = min(c, n);
  int r = kmax;
  double r11 = 0.0;
  for (int j = 0; j < kmax; ++j) {
    const int par = j & 1;
    // (1) local candidate: largest remaining norm (lowest index on ties) and tail sum
    double bv = -1.0, ts = 0.0;
    int bi = -1;
    for (int i = tid; i < ncl; i += blockDim.x) {
      if (stepof[i] >= 0) continue;
      const double w = (double)nrm[i];
      ts += w;
      if (bi < 0 || w > bv) { bv = w; bi = col0 + i; }
    }
    warp_argmax(bv, bi);
    ts = warp_sum(ts);
    if (lane == 0) { redd[warp] = bv; redi[warp] = bi; redt[warp] = ts; }
    __syncthreads();
    if (warp == 0) {
      double v2 = (lane < nw) ? redd[lane] : -1.0;
      int i2 = (lane < nw) ? redi[lane] : -1;
      double t2 = (lane < nw) ? redt[lane] : 0.0;
      warp_argmax(v2, i2);
      t2 = warp_sum(t2);
      if (lane == 0) { slot_v[par] = v2; slot_i[par] = i2; slot_t[par] = t2; }
    }
    cluster_sync_all();
    // (2) pivot and truncation test (every CTA alike)
    double pv = -1.0, tail = 0.0;
    int p = -1;
    if (lane < (int)gridDim.x) {
      pv = dsmem_ld_f64(dsmem_map(&slot_v[par], lane));
      p = dsmem_ld_s32(dsmem_map(&slot_i[par], lane));
      tail = dsmem_ld_f64(dsmem_map(&slot_t[par], lane));
    }
    warp_argmax(pv, p);
    tail = warp_sum(tail);
    if (j == 0 && !(tail > 0.0)) { r = 0; break; }
    if (j >= 1 && sqrt(fmax(tail, 0.0)) <= tol * r11) { r = j; break; }
    // (3) reflector from rows j.. of the pivot column
    const int po = p / nc, pl = p - po * nc;
    for (int l = tid; l < c - j; l += blockDim.x) v[l] = dsmem_ld<T>(dsmem_map(&Ms[j + l + (size_t)pl * ldm], po));
    __syncthreads();
    T sig = T(0);
    for (int l = 1 + tid; l < c - j; l += blockDim.x) sig = fma(v[l], v[l], sig);
    sig = block_sum(sig, red);
    const T alpha = v[0];
    T beta, tj, scale;
    if (sig == T(0)) { beta = alpha; tj = T(0); scale = T(0); }
    else {
      const T nrmx = sqrt(alpha * alpha + sig);
      beta = (alpha <= T(0)) ? nrmx : -nrmx;
      tj = (beta - alpha) / beta;
      scale = T(1) / (alpha - beta);
    }
    __syncthreads();
    for (int l = 1 + tid; l < c - j; l += blockDim.x) v[l] *= scale;
    if (tid == 0) {
      v[0] = T(1);
      if (rk == po) { stepof[pl] = j; bdg[pl] = beta; }
    }
    if (j == 0) r11 = fabs((double)beta);
    __syncthreads();
    // (4) apply to the remaining owned columns (two threads per column, rows split by
    //     parity, combined by one shuffle) + norm downdate
    for (int t0 = 0; t0 < 2 * ncl; t0 += blockDim.x) {  // warp-uniform trip count (shuffles below)
      const int t = t0 + tid;
      const int i = min(t >> 1, ncl - 1), h = t & 1;
      const bool live = (t < 2 * ncl) && stepof[i] < 0;
      T* y = Ms + j + (size_t)i * ldm;
      const int len = c - j;
      // four independent partial sums per thread (rows l, l + 2, l + 4, l + 6): the
      // dependent chains are a quarter as long
      T w0 = T(0), w1 = T(0), w2 = T(0), w3 = T(0);
      int l = 1 + h;
      if (live) {
        for (; l + 6 < len; l += 8) {
          w0 = fma(v[l], y[l], w0);
          w1 = fma(v[l + 2], y[l + 2], w1);
          w2 = fma(v[l + 4], y[l + 4], w2);
          w3 = fma(v[l + 6], y[l + 6], w3);
        }
        for (; l < len; l += 2) w0 = fma(v[l], y[l], w0);
      }
      T w = (w0 + w1) + (w2 + w3);
      w += __shfl_xor_sync(0xffffffffu, w, 1);
      const T y0 = live ? y[0] : T(0);
      w = (w + y0) * tj;
      const T top = y0 - w;
      T t0s = T(0), t1s = T(0), t2s = T(0), t3s = T(0);
      l = 1 + h;
      if (live) {
        for (; l + 6 < len; l += 8) {
          const T n0 = fma(-w, v[l], y[l]), n1 = fma(-w, v[l + 2], y[l + 2]);
          const T n2 = fma(-w, v[l + 4], y[l + 4]), n3 = fma(-w, v[l + 6], y[l + 6]);
          y[l] = n0;
          y[l + 2] = n1;
          y[l + 4] = n2;
          y[l + 6] = n3;
          t0s = fma(n0, n0, t0s);
          t1s = fma(n1, n1, t1s);
          t2s = fma(n2, n2, t2s);
          t3s = fma(n3, n3, t3s);
        }
        for (; l < len; l += 2) {
          const T nv = fma(-w, v[l], y[l]);
          y[l] = nv;
          t0s = fma(nv, nv, t0s);
        }
      }
      T tail2 = (t0s + t1s) + (t2s + t3s);
      tail2 += __shfl_xor_sync(0xffffffffu, tail2, 1);
      if (live && h == 0) {
        y[0] = top;
        T nn = nrm[i] - top * top;
        const T eps = (sizeof(T) == 8) ? T(1.5e-8) : T(3.5e-4);
        if (!(nn > eps * nref[i])) {
          nn = tail2;
          nref[i] = nn;
        }
        nrm[i] = (nn > T(0)) ? nn : T(0);
      }
    }
    __syncthreads();
  }
  cluster_sync_all();  // keep this CTA's columns readable until every CTA is done
  // (5) output rows l < r of R in original column order: Z[o, l] = R[l, position of o]
  for (int e = tid; e < r * ncl; e += blockDim.x) {
    const int l = e / ncl, i = e - l * ncl;
    const int st = stepof[i];
    T val;
    if (st < 0 || l < st) val = Ms[l + (size_t)i * ldm];
    else if (l == st) val = bdg[i];
    else val = T(0);
    Z[col0 + i + l * ldz] = val;
  }
  if (rk == 0 && tid == 0) *rank_out = r;
}

constexpr size_t QRCP_CLUSTER_SMEM = 225 * 1024;  // dynamic shared memory cap per CTA (of 227 KB)

// Cluster size for the resident variant, or 0 when M = Z^T does not fit.
template <typename T>
static int qrcp_cluster_size(int64_t n, int64_t c) {
  for (int C : {8, 16}) {
    const int64_t nc = ceil_div(n, C);
    if (qrcp_cluster_smem<T>(c, nc) <= QRCP_CLUSTER_SMEM) return C;
  }
  return 0;
}

template <typename T>
int qrcp_truncate(T* Z, int64_t n, int64_t c, int64_t ldz, double tol, QRScratch& sc, cudaStream_t s) {
  if (n <= 0 || c <= 0) {
    LYAP_CUDA_TRY(cudaMemsetAsync(sc.rank, 0, sizeof(int), s));
    return LYAP_OK;
  }
  const int CL = (n >= 64) ? qrcp_cluster_size<T>(n, c) : 0;
  if (CL > 0) {
    const int nc = (int)ceil_div(n, CL);
    const size_t smem = qrcp_cluster_smem<T>(c, nc);
    auto kc = qrcp_cluster_kernel<T>;
    // attributes are set once, to their largest value: concurrent callers (batched
    // solves) must never lower them between another caller's set and launch
    static DeviceOnce attr_c;
    if (attr_c.need()) {
      LYAP_CUDA_TRY(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)QRCP_CLUSTER_SMEM));
      LYAP_CUDA_TRY(cudaFuncSetAttribute(kc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
      attr_c.set();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LYAP_CUDA_TRY(cudaLaunchKernelEx(&cfg, kc, Z, (int)n, (int)c, ldz, nc, tol, sc.rank));
    lyap_count_launch();
    return LYAP_OK;
  }
  int G = (int)std::min<int64_t>(ceil_div(n, 8), sc.num_sms);
  G = std::min(G, 256);
  if (G < 1) G = 1;
  const size_t smem = sizeof(T) * (size_t)c;
  auto kern = qrcp_kernel<T>;
  if (smem > QRCP_CLUSTER_SMEM) {
    lyap_set_error_message("QR with column pivoting: factor too wide", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  static DeviceOnce attr_g;
  if (smem > 48 * 1024 && attr_g.need()) {
    LYAP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)QRCP_CLUSTER_SMEM));
    attr_g.set();
  }
  LYAP_CUDA_TRY(cudaMemsetAsync(sc.bar, 0, sizeof(GridBar), s));
  T* M = (T*)sc.work;
  T* nrm = (T*)sc.norms;
  T* nrm_ref = nrm + n;
  T* rdiag = (T*)sc.rdiag;
  double* cand = (double*)sc.cand;
  void* args[] = {&Z, &n, &c, &ldz, &tol, &M, &nrm, &nrm_ref, &sc.piv, &rdiag, &cand, &sc.rank, &sc.bar, &sc.status};
  LYAP_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(G), dim3(256), args, smem, s));
  lyap_count_launch();
  return LYAP_OK;
}
template int qrcp_truncate<float>(float*, int64_t, int64_t, int64_t, double, QRScratch&, cudaStream_t);
template int qrcp_truncate<double>(double*, int64_t, int64_t, int64_t, double, QRScratch&, cudaStream_t);

}  // namespace lyap
