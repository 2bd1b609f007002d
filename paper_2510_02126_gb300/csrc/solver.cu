// Host driver and C-ABI of liblyap: the sign-function Newton solver (Sec. 3) and
// mixed-precision iterative refinement (Sec. 2) on one GPU.  Every arithmetic
// step runs in this library's kernels; the host only sequences launches and
// reads back the device-computed scalars that steer the loops.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>
#include <thread>
#include <cstring>
#include <vector>

#include "dense.cuh"
#include "eig.cuh"
#include "gj_inverse.cuh"
#include "qr.cuh"
#include "tc_gemm.cuh"

// ---------------------------------------------------------------------------
// process-wide diagnostics
// ---------------------------------------------------------------------------
// last error message and kernel-launch count of the calling host thread (a call runs on
// one thread; batched solves run their equations on worker threads)
static thread_local char g_err[512] = "";
static thread_local int64_t g_launches = 0;

void lyap_set_error_message(const char* what, const char* file, int line) {
  snprintf(g_err, sizeof(g_err), "%s (%s:%d)", what, file, line);
}
void lyap_count_launch(int k) { g_launches += k; }

namespace lyap {

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

static int ensure(Buf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return LYAP_OK;
  if (b.p) {
    // work queued on this context's (non-blocking) stream may still use the old buffer;
    // cudaFree does not wait for it, and another context's next cudaMalloc may reuse the
    // memory at once (batched solves grow buffers on several streams concurrently)
    LYAP_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes + bytes / 4 + 256;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    lyap_set_error_message("device allocation failed", __FILE__, __LINE__);
    return LYAP_ERR_NOMEM;
  }
  // zero-filled, and complete before any kernel of any stream touches it: status words and
  // flags are read as "no error" before their first write (memory freed by an earlier
  // context comes back holding its old contents)
  LYAP_CUDA_TRY(cudaMemset(b.p, 0, want));
  LYAP_CUDA_TRY(cudaDeviceSynchronize());
  b.cap = want;
  return LYAP_OK;
}
template <typename T>
static T* P(Buf& b) { return reinterpret_cast<T*>(b.p); }

// Device-side state of one sign-Newton run (read back by the host after each step).
struct NewtonState {
  double ssA, ssX, maxX, mu, ssA1, ssD, ssE, stopv, delta, delta_prev, logdet, nrmA, nrmX;
  double meas[64];
  int scaling_on, fired, prev_unscaled, done, k, eX, status, pad;
};

}  // namespace lyap

struct lyap_ctx {
  int device = 0;
  cudaStream_t s = nullptr;
  int num_sms = 0;
  lyap::Buf state, scal, part, hist;
  // inversion
  lyap::GJWork gj;
  lyap::Buf gjM0, gjM1, gjPp, gjRt, gjOrig, gjPerm0, gjPerm1, gjLog, gjIpiv, gjStatus, gjExps, gjAmax;
  // Newton working buffers
  lyap::Buf A0, A1, pinv, colsum, Zw, Zw2, Zh, eZ, yv, yv2;
  // stored inverse sequence (Sec. 3.4)
  lyap::Buf store, dmu, dex;
  int store_n = 0, store_prec = -1, store_count = 0, store_e0 = 0;
  bool store_t = false;  // the stored inverses are transposed (the adjoint's replay)
  double store_fp = 0.0;   // fingerprint of the matrix whose inverse sequence is stored
  size_t store_elt = 0;
  int64_t store_ld = 0;    // row pitch (elements) of a stored inverse
  int64_t store_rows = 0;  // rows allocated per stored inverse
  // checkpointed sequence (opts.ckpt_every / opts.mem_budget): the store holds the Newton
  // iterates A_0, A_c, A_2c, ... (working precision, row-major n x n) instead of the
  // inverses; every use recomputes the inverses of a segment from its checkpoint, using
  // the recorded mu_k and storage exponents, into the one-slot buffer inv1
  int store_ckpt = 0;       // 0: inverses stored; c > 0: checkpoint every c steps
  size_t store_welt = 0;    // element size of a checkpoint (working precision)
  lyap::Buf inv1;           // the inverse of the current step (checkpoint mode)
  int64_t recomputed = 0;   // inversions recomputed from checkpoints by the current call
  // FP64 refinement buffers
  lyap::Buf F, tau, Tm, TP, H, w, Qh, Csel, Lp, Lm, Zs, Zbest, G, gram, ysol, ybest, ytmp, Lw, Sd, Vs, Lst, Rtau, Bm, VB;
  // scratch of the QR and eigen kernels
  lyap::QRScratch qr;
  lyap::Buf qrBar, qrStatus, qrCand, qrNorms, qrPiv, qrRdiag, qrWork, qrRank;
  lyap::EigScratch eig;
  // adjoint: A^T, C^T, the adjoint factor and the gradient products
  lyap::Buf At, Ct, ZY, adjT;
  lyap::Buf tl;  // trace loss: C Z and C Z diag(D)
  lyap::Buf Hf;  // FP32 copy of the residual core for its range finder
  lyap::Buf pnw; // power-iteration vectors of the 2-norm / spectral-radius scalings
  lyap::Buf adiW, adiY, adiG;  // low-rank ADI: [W, V] (working precision), weights of W, W^T W
  std::vector<double> adi_p;   // low-rank ADI: the shifts of the stored inverses
  // extended Krylov: basis, A times basis, new block, right-hand side, projected matrices
  lyap::Buf ekV, ekAV, ekW, ekL, ekT, ekE, ekS, ekZY, ekD, ekH, ekTau, ekP, ekQ, ekR;
  lyap_ctx* sub = nullptr;     // context of the projected (small) Lyapunov solves
  lyap::Buf eigWork32, eigBig, eigX, eigR, eigS, eigHX, eigE, eigLam, eigRed, eigW, eigPv, eigInt;
  void* hpin = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // phase profiling (opts.profile): events recorded at phase boundaries
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> marks_phase;
  size_t marks_used = 0;
  double flops[LYAP_NUM_PHASES] = {};  // algorithmic flops per phase (host-side count)
  // batched solves: worker contexts, each on its own non-blocking stream
  std::vector<lyap_ctx*> pool;
  std::vector<cudaStream_t> pool_streams;
};

namespace lyap {

using Ctx = lyap_ctx;

static bool is16(int prec) { return prec == LYAP_FP16 || prec == LYAP_BF16; }

// Start of a phase on the context stream (no-op unless profiling).
static void mark(Ctx& C, int phase) {
  if (!C.profile) return;
  if (C.marks_used == C.ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    C.ev_pool.push_back(e);
  }
  cudaEventRecord(C.ev_pool[C.marks_used], C.s);
  if (C.marks_phase.size() <= C.marks_used) C.marks_phase.resize(C.marks_used + 1);
  C.marks_phase[C.marks_used] = phase;
  ++C.marks_used;
}
// mark() for the eigensolver (EigScratch::mark)
static void mark_cb(void* ctx, int phase) { mark(*static_cast<Ctx*>(ctx), phase); }
static void collect_marks(Ctx& C, lyap_info_t* info) {
  for (int p = 0; p < LYAP_NUM_PHASES; ++p) info->phase_flops[p] += C.flops[p];
  if (!C.profile) return;
  mark(C, LYAP_PHASE_OTHER);
  cudaEventSynchronize(C.ev_pool[C.marks_used - 1]);
  for (size_t i = 0; i + 1 < C.marks_used; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, C.ev_pool[i], C.ev_pool[i + 1]);
    const int ph = C.marks_phase[i];
    info->phase_ms[ph] += ms;
    info->phase_calls[ph] += 1;
  }
  C.marks_used = 0;
}

// ---------------------------------------------------------------------------
// small kernels of the Newton step (Eq. (3.1a)-(3.3))
// ---------------------------------------------------------------------------
__global__ void iota_kernel(int* p, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}
__global__ void pinv_kernel(const int* __restrict__ perm, int* __restrict__ pinv, int n) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) pinv[perm[c]] = c;
}

__global__ void newton_init_kernel(NewtonState* st, int scaling) {
  st->scaling_on = (scaling != LYAP_SCALE_NONE);
  st->fired = 0;
  st->prev_unscaled = 0;
  st->done = 0;
  st->k = 0;
  st->eX = 0;
  st->status = 0;
  st->delta_prev = -1.0;
  st->mu = 1.0;
}

// mu_k (Frobenius: (||A^-1||_F/||A||_F)^{1/2}; determinantal: |det A|^{-1/n} from the
// pivots in logarithms; 1 once scaling is off) and the storage exponent of A_k^{-1}.
__global__ void newton_mu_kernel(NewtonState* st, int n, int scaling, int store16) {
  double mu = 1.0;
  if (st->scaling_on) {
    if (scaling == LYAP_SCALE_FROB) mu = sqrt(sqrt(st->ssX) / sqrt(st->ssA));
    else if (scaling == LYAP_SCALE_DET) mu = exp(-st->logdet / (double)n);
    else if (scaling == LYAP_SCALE_NORM2 || scaling == LYAP_SCALE_SPECTRAL) mu = sqrt(st->nrmX / st->nrmA);
  }
  if (!isfinite(mu) || !(mu > 0.0) || !isfinite(st->ssX)) atomicCAS(&st->status, 0, LYAP_ERR_NONFINITE);
  st->mu = mu;
  st->eX = store16 ? pow2_exponent(st->maxX) : 0;
}

// mu_k and the storage exponent of A_k^{-1} as recorded by the first solve (recomputation
// of an inverse from a checkpoint reproduces the recorded sequence)
__global__ void newton_recorded_mu_kernel(NewtonState* st, const double* __restrict__ dmu, const int* __restrict__ dex,
                                          int kk) {
  st->mu = dmu[kk];
  st->eX = dex[kk];
}

// A_{k+1} = (mu A_k + mu^{-1} A_k^{-1}) / 2 with A_k^{-1}[i, j] = X[i, pinv[j]];
// also stores A_k^{-1} (scaled by 2^-eX) and the partial sums of
// ||A_{k+1}||_F^2, ||A_{k+1} - A_k||_F^2 and ||A_{k+1} + I||_F^2.
template <typename T, typename ST>
__global__ void __launch_bounds__(256)
newton_update_kernel(int n, const T* __restrict__ Ak, const T* __restrict__ X, const int* __restrict__ pinv,
                     const NewtonState* __restrict__ st, T* __restrict__ An, ST* __restrict__ Xs, int64_t ldx,
                     double* __restrict__ part) {
  const double mu = st->mu, imu = 1.0 / st->mu;
  const double sx = ldexp(1.0, -st->eX);
  const int64_t total = (int64_t)n * n;
  double s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const double x = (double)X[i * n + pinv[j]];
    const double a = (double)Ak[e];
    const double an_d = 0.5 * (mu * a + imu * x);
    const T an = (T)an_d;
    An[e] = an;
    Xs[i * ldx + j] = (ST)(x * sx);
    const double av = (double)an;
    s1 = fma(av, av, s1);
    const double d = av - a;
    s2 = fma(d, d, s2);
    const double ep = av + (i == j ? 1.0 : 0.0);
    s3 = fma(ep, ep, s3);
  }
  __shared__ double sh[3][8];
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  s3 = warp_sum(s3);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sh[0][warp] = s1; sh[1][warp] = s2; sh[2][warp] = s3; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[threadIdx.x][w];
    part[threadIdx.x * RED_BLOCKS + blockIdx.x] = t;
  }
}
// ---- 2-norm and spectral-radius estimates of a row-major n x n matrix M (FP32 power
// iteration; v, u: n floats; part: PN_SPLIT x n floats; hist: PN_STEPS + 1 doubles)
constexpr int PN_STEPS_NORM2 = 12;     // power steps on M^T M
constexpr int PN_STEPS_SPECTRAL = 24;  // power steps on M (the geometric mean of the second half)
constexpr int PN_SPLIT = 16;           // row chunks of the M^T u partial sums
// v = a fixed non-degenerate start; hist[0] = ||v||^2
__global__ void pn_init_kernel(int n, float* __restrict__ v, double* __restrict__ hist) {
  __shared__ double red[32];
  double t = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float x = 1.0f + 0.01f * (float)(j % 7);
    v[j] = x;
    t += (double)x * x;
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    hist[0] = s;
  }
}
// u = M P v / ||v|| (one warp per row; (P v)_p = v[cmap[p]], cmap == NULL: identity)
template <typename T>
__global__ void __launch_bounds__(256) pn_mv_kernel(const T* __restrict__ M, int n, const int* __restrict__ cmap,
                                                    const float* __restrict__ v, const double* __restrict__ vn2,
                                                    float* __restrict__ u) {
  const int lane = threadIdx.x & 31;
  const float inv = (float)(1.0 / sqrt(*vn2));
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
    const T* row = M + (int64_t)i * n;
    float t = 0.f;
    for (int p = lane; p < n; p += 32) t = fmaf((float)row[p], v[cmap ? cmap[p] : p], t);
    t = warp_sum(t);
    if (lane == 0) u[i] = t * inv;
  }
}
// part[s n + j] = sum over the rows i of chunk s of M[i, j] u_i (M^T u in PN_SPLIT row chunks)
template <typename T>
__global__ void __launch_bounds__(256) pn_mtv_kernel(const T* __restrict__ M, int n, const float* __restrict__ u,
                                                     float* __restrict__ part) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int s = blockIdx.y, i0 = (int)((int64_t)n * s / PN_SPLIT), i1 = (int)((int64_t)n * (s + 1) / PN_SPLIT);
  float t = 0.f;
  for (int i = i0; i < i1; ++i) t = fmaf((float)M[(int64_t)i * n + j], u[i], t);
  part[(int64_t)s * n + j] = t;
}
// v = sum of the nparts rows of part (fixed order); out = ||v||^2 (one CTA)
__global__ void pn_sum_kernel(const float* __restrict__ part, int n, int nparts, float* __restrict__ v,
                              double* __restrict__ out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    float x = 0.f;
    for (int s = 0; s < nparts; ++s) x += part[(int64_t)s * n + j];
    v[j] = x;
    t += (double)x * x;
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    *out = s;
  }
}
// *est from the recorded norms: 2-norm ||M^T M v^|| ^ (1/2) of the last step; spectral
// radius exp(mean of log ||M v^|| over the second half of the steps)
__global__ void pn_final_kernel(const double* __restrict__ hist, int steps, int spectral, double* __restrict__ est) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!spectral) {
    *est = sqrt(sqrt(hist[steps]));
  } else {
    double l = 0.0;
    const int h = steps / 2;
    for (int k = steps - h + 1; k <= steps; ++k) l += 0.5 * log(hist[k]);
    *est = exp(l / h);
  }
}

// ---- low-rank ADI (real cyclic shifts) ----
// M = A0 + p I (row-major n x n, working precision)
template <typename T>
__global__ void adi_shift_kernel(const T* __restrict__ A0, int n, double p, T* __restrict__ M) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    M[e] = (T)((double)A0[e] + (i == j ? p : 0.0));
  }
}
// storage exponent of inverse j (16-bit storage only), as the Newton step records it
__global__ void adi_exp_kernel(const double* __restrict__ maxX, int j, int store16, int* __restrict__ dex,
                               double* __restrict__ dmu) {
  dex[j] = store16 ? pow2_exponent(*maxX) : 0;
  dmu[j] = 1.0;
}
// slot j of the store = (A0 + p_j I)^{-1} (X row-major with columns permuted: X[i, pinv[c]])
template <typename T, typename ST>
__global__ void adi_store_kernel(int n, const T* __restrict__ X, const int* __restrict__ pinv,
                                 const int* __restrict__ dex, int j, ST* __restrict__ Xs, int64_t ldx) {
  const double sx = ldexp(1.0, -dex[j]);
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, c = e - i * n;
    Xs[i * ldx + c] = (ST)((double)X[i * n + pinv[c]] * sx);
  }
}
// Z[:, c0 + t] = sZ V[:, t], W[:, t] -= 2 p V[:, t] (t < m; Y = [W, V], ld n); LDL^T weights
// y[c0 + t] = -2 p y0[t]
template <typename T>
__global__ void adi_step_kernel(T* __restrict__ Y, int n, int m, double p, double sZ, T* __restrict__ Z, int c0,
                                const double* __restrict__ y0, double* __restrict__ y) {
  const int64_t total = (int64_t)n * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / n, i = e - t * n;
    const double v = (double)Y[i + (t + m) * (int64_t)n];
    Z[i + (c0 + t) * (int64_t)n] = (T)(sZ * v);
    Y[e] = (T)((double)Y[e] - 2.0 * p * v);
    if (y && i == 0) y[c0 + t] = -2.0 * p * y0[t];
  }
}
// out = ||W diag(y0) W^T||_F^2 = sum_ij (G_ij)^2 y0_i y0_j for G = W^T W (m x m; y0 == NULL: 1)
__global__ void adi_resnorm_kernel(const double* __restrict__ G, int m, const double* __restrict__ y0,
                                   double* __restrict__ out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int j = e / m, i = e - j * m;
    const double g = G[e];
    t += g * g * (y0 ? y0[i] * y0[j] : 1.0);
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    *out = s;
  }
}

__global__ void newton_sums_kernel(const double* __restrict__ part, int nb, NewtonState* st) {
  // fixed-order sums of the three partial vectors
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < 3) {
    double t = 0.0;
    for (int i = lane; i < nb; i += 32) t += part[w * RED_BLOCKS + i];
    t = warp_sum(t);
    if (lane == 0) {
      if (w == 0) st->ssA1 = t;
      else if (w == 1) st->ssD = t;
      else st->ssE = t;
    }
  }
}
// column sums of |A + I| (row-major A) -> colsum[j]
template <typename T>
__global__ void colsum_kernel(int n, const T* __restrict__ A, double* __restrict__ colsum) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += fabs((double)A[(int64_t)i * n + j] + (i == j ? 1.0 : 0.0));
    colsum[j] = t;
  }
}
// stop test of Eq. (3.4) (or the Frobenius variant), Higham's delta rule, scaling switch-off
__global__ void newton_test_kernel(NewtonState* st, double tau, int norm_fro, int stop_after, int delta_rule,
                                   double scale_off, double* dmu, int* dex, int kidx) {
  const double delta = sqrt(st->ssD) / sqrt(st->ssA1);
  const double meas = norm_fro ? sqrt(st->ssE) : st->stopv;
  const int unscaled = (st->mu == 1.0);
  if (st->fired == 0) {
    bool fire = meas <= tau;
    if (delta_rule && unscaled && st->prev_unscaled && st->delta_prev >= 0.0 && delta > 0.5 * st->delta_prev)
      fire = true;
    if (fire) st->fired = 1;
  } else {
    st->fired += 1;
  }
  st->done = (st->fired >= (stop_after > 1 ? stop_after : 1));
  if (st->scaling_on && delta < scale_off) st->scaling_on = 0;
  st->delta = delta;
  st->delta_prev = delta;
  st->prev_unscaled = unscaled;
  st->ssA = st->ssA1;
  if (kidx < 64) st->meas[kidx] = meas;
  dmu[kidx] = st->mu;
  dex[kidx] = st->eX;
  st->k = kidx + 1;
  if (!isfinite(meas) || !isfinite(delta)) atomicCAS(&st->status, 0, LYAP_ERR_NONFINITE);
}
__global__ void sum_vec_kernel(const double* __restrict__ v, int n, double* out) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) t += v[i];
  t = warp_sum(t);
  if (threadIdx.x == 0) *out = t;
}
// Cholesky type (Eq. (3.2)):  Z[:, :c] *= sqrt(mu/2),  Z[:, c:2c] *= 1/sqrt(2 mu)
// LDL^T type (Eq. (3.3)):    y[c + j] = y[j] / (2 mu),  y[j] *= mu / 2
template <typename T>
__global__ void factor_scale_kernel(T* __restrict__ Z, int64_t ld, int n, int c, const double* __restrict__ mu_p,
                                    int ldlt, double* __restrict__ y) {
  const double mu = *mu_p;
  if (!ldlt) {
    const double a = sqrt(0.5 * mu), b = 1.0 / sqrt(2.0 * mu);
    const int64_t total = (int64_t)n * 2 * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t j = e / n, i = e - j * n;
      Z[i + j * ld] = (T)((double)Z[i + j * ld] * (j < c ? a : b));
    }
  } else if (blockIdx.x == 0) {
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
      const double yj = y[j];
      y[c + j] = yj / (2.0 * mu);
      y[j] = 0.5 * mu * yj;
    }
  }
}

// ---------------------------------------------------------------------------
// small kernels of the refinement (Fragments ResFac*/SolUpt*)
// ---------------------------------------------------------------------------
// Tm (kr x q) = upper trapezoid of F's leading rows
__global__ void extract_r_kernel(const double* __restrict__ F, int64_t ldf, int kr, int q, double* __restrict__ Tm) {
  const int64_t total = (int64_t)kr * q;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / kr, i = e - j * kr;
    Tm[i + j * kr] = (i <= j) ? F[i + j * ldf] : 0.0;
  }
}
// TP = T * middle, middle = [[0, Y, 0], [Y, 0, 0], [0, 0, S]] (Y = diag(y) or I, S = diag(sd) or I)
__global__ void core_right_kernel(const double* __restrict__ Tm, int kr, int c, int m, const double* __restrict__ y,
                                  const double* __restrict__ sd, double* __restrict__ TP) {
  const int q = 2 * c + m;
  const int64_t total = (int64_t)kr * q;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / kr, i = e - j * kr;
    double v;
    if (j < c) v = Tm[i + (j + c) * kr] * (y ? y[j] : 1.0);
    else if (j < 2 * c) v = Tm[i + (j - c) * kr] * (y ? y[j - c] : 1.0);
    else v = Tm[i + j * kr] * (sd ? sd[j - 2 * c] : 1.0);
    TP[i + j * kr] = v;
  }
}
// Gamma * J with J = diag(sign) (SolUptChol: +1 for Z, Z+, -1 for Z-) or diag(ups) (SolUptLdlt)
__global__ void scale_cols_dev_kernel(const double* __restrict__ A, int kr, int q, int cneg_start,
                                      const double* __restrict__ d, double* __restrict__ B) {
  const int64_t total = (int64_t)kr * q;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / kr, i = e - j * kr;
    double f = d ? d[j] : (j >= cneg_start ? -1.0 : 1.0);
    B[i + j * kr] = A[i + j * kr] * f;
  }
}
// Ranges of an ascending spectrum w[0..q): out[0] = #(w <= -thr), out[1] = first index with w >= thr,
// thr = eta * max|w|.  Also out[2] = first index with |w| > thr (magnitude mode helper not needed).
__global__ void select_kernel(const double* __restrict__ w, int q, double eta, int strict, int* __restrict__ out,
                              double* __restrict__ thr_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mx = 0.0;
  for (int i = 0; i < q; ++i) mx = fmax(mx, fabs(w[i]));
  const double thr = eta * mx;
  int nneg = 0;
  while (nneg < q && (strict ? (w[nneg] < -thr) : (w[nneg] <= -thr))) ++nneg;
  int pos = q;
  while (pos > 0 && (strict ? (w[pos - 1] > thr) : (w[pos - 1] >= thr))) --pos;
  if (!(mx > 0.0)) { nneg = 0; pos = q; }
  if (pos < nneg) pos = nneg;
  out[0] = nneg;
  out[1] = pos;
  *thr_out = thr;
}
// C[:, t] = Q[:, i0 + t] * f(w[i0 + t]), f = sqrt(|w|) (Cholesky types) or 1 (LDL^T, value copied to yo)
__global__ void gather_cols_kernel(const double* __restrict__ Q, int64_t ldq, int kr, const double* __restrict__ w,
                                   int i0, int cnt, int use_sqrt, double* __restrict__ C, int64_t ldc,
                                   double* __restrict__ yo) {
  const int64_t total = (int64_t)kr * cnt;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / kr, i = e - t * kr;
    const double wv = w[i0 + t];
    const double f = use_sqrt ? sqrt(fabs(wv)) : 1.0;
    C[i + t * ldc] = Q[i + (i0 + t) * ldq] * f;
    if (yo && i == 0) yo[t] = wv;
  }
}
// normalised residual of Eq. (4.1) from ||H||_F^2, ||W||_F, ||A||_F and ||X||_F^2
__global__ void resid_kernel(const double* ssH, const double* wF, const double* aF2, const double* ssX,
                             double* out) {
  const double num = sqrt(*ssH);
  const double den = *wF + 2.0 * sqrt(*ssX) * sqrt(*aF2);
  out[0] = num / den;
  out[1] = num;
}
// ||Z Y Z^T||_F^2 = sum_ij G_ij^2 y_i y_j from G = Z^T Z (y == NULL: Z Z^T)
__global__ void gram_norm_kernel(const double* __restrict__ G, int c, const double* __restrict__ y, double* out) {
  double t = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)c * c; e += blockDim.x) {
    const int64_t j = e / c, i = e - j * c;
    const double g = G[e];
    t += g * g * (y ? y[i] * y[j] : 1.0);
  }
  __shared__ double sh[32];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    *out = fmax(s, 0.0);
  }
}
__global__ void scale_vec_kernel(double* v, int n, double f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] *= f;
}
// trace(C X C^T) = sum_j d_j sum_k T[k, j]^2 with T = C Z (q x r, column-major); d == NULL
// means d = 1.  Also TD = T diag(d).  One block, fixed order (the same bits every call).
__global__ void trace_loss_kernel(const double* __restrict__ Tm, int q, int r, const double* __restrict__ d,
                                  double* __restrict__ TD, double* __restrict__ out) {
  __shared__ double sh[32];
  double t = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)q * r; e += blockDim.x) {
    const int64_t j = e / q;
    const double v = Tm[e], dj = d ? d[j] : 1.0;
    t = fma(dj * v, v, t);
    TD[e] = dj * v;
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += sh[w];
    *out = u;
  }
}
// Ainv (column-major, ld) [i, perm[c]] = X[i, c] (X row-major)
template <typename T>
__global__ void unpermute_kernel(const T* __restrict__ X, const int* __restrict__ perm, int n, double* __restrict__ Ainv,
                                 int64_t ld) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    Ainv[i + (int64_t)perm[c] * ld] = (double)X[i * n + c];
  }
}

static unsigned nblk(int64_t total, int64_t per = 256, int64_t cap = 4096) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, ceil_div(total, per)));
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct Sizes {
  int n, m, zcap_w, fcap;
};

template <typename T>
static int prepare_newton(Ctx& C, int n, int m, int prec) {
  const size_t nn = (size_t)n * n;
  const int zcap = 2 * n + 2 * m + 8;
  const size_t elt = sizeof(T);
  LYAP_TRY(ensure(C.gjM0, nn * elt));
  LYAP_TRY(ensure(C.gjM1, nn * elt));
  LYAP_TRY(ensure(C.gjPp, (size_t)tc_rows(n) * GJ_KLD16 * 2 + (size_t)n * GJ_BS * elt));
  LYAP_TRY(ensure(C.gjRt, (size_t)tc_rows(n) * GJ_KLD16 * 2 + (size_t)n * GJ_BS * elt));
  LYAP_TRY(ensure(C.gjOrig, (size_t)n * 4));
  LYAP_TRY(ensure(C.gjPerm0, (size_t)n * 4));
  LYAP_TRY(ensure(C.gjPerm1, (size_t)n * 4));
  LYAP_TRY(ensure(C.gjLog, (size_t)n * 8));
  LYAP_TRY(ensure(C.gjIpiv, (size_t)n * 4));
  LYAP_TRY(ensure(C.gjStatus, 16));
  LYAP_TRY(ensure(C.gjExps, (size_t)(2 * ceil_div(n, GJ_BS) + 2) * 4));
  LYAP_TRY(ensure(C.gjAmax, 64));
  LYAP_TRY(ensure(C.A0, nn * elt));
  LYAP_TRY(ensure(C.A1, nn * elt));
  LYAP_TRY(ensure(C.pinv, (size_t)n * 4));
  LYAP_TRY(ensure(C.colsum, (size_t)n * 8));
  LYAP_TRY(ensure(C.Zw, (size_t)n * zcap * elt));
  LYAP_TRY(ensure(C.Zw2, (size_t)n * zcap * elt));
  if (C.Zh.cap < (size_t)tc_rows(zcap) * tc_kpitch(n) * 2 + 256) {
    LYAP_TRY(ensure(C.Zh, (size_t)tc_rows(zcap) * tc_kpitch(n) * 2 + 256));
    LYAP_CUDA_TRY(cudaMemsetAsync(C.Zh.p, 0, C.Zh.cap, C.s));  // padding rows stay finite
  }
  LYAP_TRY(ensure(C.eZ, (size_t)zcap * 4));
  LYAP_TRY(ensure(C.yv, (size_t)zcap * 8));
  LYAP_TRY(ensure(C.yv2, (size_t)zcap * 8));
  LYAP_TRY(ensure(C.state, sizeof(NewtonState)));
  LYAP_TRY(ensure(C.scal, 4096));
  LYAP_TRY(ensure(C.part, (size_t)6 * RED_BLOCKS * 8));
  LYAP_TRY(ensure(C.dmu, 64 * 8));
  LYAP_TRY(ensure(C.dex, 64 * 4));
  // QR scratch (working precision and FP64 share it; size for FP64)
  LYAP_TRY(ensure(C.qrBar, sizeof(GridBar)));
  LYAP_TRY(ensure(C.qrStatus, 16));
  LYAP_TRY(ensure(C.qrCand, 3 * 256 * 8));
  LYAP_TRY(ensure(C.qrNorms, (size_t)2 * n * 8 + 64));
  LYAP_TRY(ensure(C.qrPiv, (size_t)n * 4 + 64));
  LYAP_TRY(ensure(C.qrRdiag, (size_t)zcap * 8 + 64));
  LYAP_TRY(ensure(C.qrWork, (size_t)n * zcap * 8));
  LYAP_TRY(ensure(C.qrRank, 16));
  C.qr.bar = P<GridBar>(C.qrBar);
  C.qr.status = P<int>(C.qrStatus);
  C.qr.cand = C.qrCand.p;
  C.qr.norms = C.qrNorms.p;
  C.qr.piv = P<int>(C.qrPiv);
  C.qr.flags = P<int>(C.qrPiv);  // shares the pivot buffer: QRCP and QR never run at the same time
  C.qr.rdiag = C.qrRdiag.p;
  C.qr.work = C.qrWork.p;
  C.qr.rank = P<int>(C.qrRank);
  C.qr.num_sms = C.num_sms;
  GJWork& W = C.gj;
  W.n = n;
  W.elt = (int)elt;
  W.M[0] = C.gjM0.p;
  W.M[1] = C.gjM1.p;
  W.Pp = C.gjPp.p;
  W.Rt = C.gjRt.p;
  W.orig = P<int>(C.gjOrig);
  W.perm[0] = P<int>(C.gjPerm0);
  W.perm[1] = P<int>(C.gjPerm1);
  W.logpiv = P<double>(C.gjLog);
  W.ipiv = nullptr;
  W.status = P<int>(C.gjStatus);
  W.exps = P<int>(C.gjExps);
  W.amax = P<float>(C.gjAmax);
  (void)prec;
  return LYAP_OK;
}

static int prepare_eig(Ctx& C, int q) {
  const size_t qq = (size_t)q * q;
  LYAP_TRY(ensure(C.eigWork32, std::max(2 * qq, bjac_work_floats(q)) * 4 + 64));
  if (eig_big_floats(q) > 0) {
    LYAP_TRY(ensure(C.eigBig, eig_big_floats(q) * 4 + 64));
    C.eig.big = P<float>(C.eigBig);
  }
  LYAP_TRY(ensure(C.eigX, qq * 8 + 64));
  LYAP_TRY(ensure(C.eigR, qq * 8 + 64));
  LYAP_TRY(ensure(C.eigS, qq * 8 + 64));
  LYAP_TRY(ensure(C.eigHX, qq * 8 + 64));
  LYAP_TRY(ensure(C.eigE, qq * 8 + 64));
  LYAP_TRY(ensure(C.eigLam, (size_t)q * 8 + 64));
  LYAP_TRY(ensure(C.eigRed, (size_t)(16 + RED_BLOCKS + 128) * 8));
  LYAP_TRY(ensure(C.eigW, qq * 8 + 64));
  LYAP_TRY(ensure(C.eigPv, (size_t)2 * q * 8 + 64));
  LYAP_TRY(ensure(C.eigInt, (size_t)(3 * q + 16) * 4));
  C.eig.work32 = P<float>(C.eigWork32);
  C.eig.X = P<double>(C.eigX);
  C.eig.R = P<double>(C.eigR);
  C.eig.S = P<double>(C.eigS);
  C.eig.HX = P<double>(C.eigHX);
  C.eig.E = P<double>(C.eigE);
  C.eig.lam = P<double>(C.eigLam);
  C.eig.red = P<double>(C.eigRed);
  C.eig.W = P<double>(C.eigW);
  C.eig.pv = P<double>(C.eigPv);
  C.eig.order = P<int>(C.eigInt);
  C.eig.coff = P<int>(C.eigInt) + q;
  C.eig.cidx = P<int>(C.eigInt) + 2 * q + 1;
  C.eig.cinfo = P<int>(C.eigInt) + 3 * q + 4;
  LYAP_TRY(ensure(C.qrBar, sizeof(GridBar)));
  LYAP_TRY(ensure(C.qrStatus, 16));
  C.eig.bar = P<GridBar>(C.qrBar);
  C.eig.status = P<int>(C.qrStatus);
  C.eig.num_sms = C.num_sms;
  C.eig.mark = mark_cb;
  C.eig.mark_ctx = &C;
  C.eig.flops = C.flops;
  return LYAP_OK;
}

// ---------------------------------------------------------------------------
// adjoint support
// ---------------------------------------------------------------------------
// Partial sums of sum_ij a_ij w_ij with fixed pseudo-random weights in [1, 2): a
// fingerprint that identifies the matrix whose inverse sequence is stored.
__global__ void fingerprint_kernel(const double* __restrict__ A, int n, int64_t lda, double* __restrict__ part) {
  __shared__ double red[32];
  double t = 0.0;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    const uint32_t h = ((uint32_t)i * 2654435761u) ^ ((uint32_t)j * 40503u + 0x9e3779b9u);
    t += A[i + j * lda] * (1.0 + (double)(h % 1009u) / 1009.0);
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
    part[blockIdx.x] = u;
  }
}
__global__ void sum_parts_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double u = 0.0;
    for (int b = 0; b < nb; ++b) u += part[b];  // fixed order: the same bits every call
    *out = u;
  }
}
// In-place transpose of `count` square n x n matrices (row pitch ld, slot stride) of
// U-sized elements; 32 x 32 tiles, the tile pair (bi, bj), bi <= bj, per CTA.
template <typename U>
__global__ void transpose_slots_kernel(U* __restrict__ M, int n, int64_t ld, size_t slot) {
  __shared__ U t1[32][33], t2[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  U* Ms = M + (size_t)blockIdx.z * slot;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int i1 = bi * 32 + r, j1 = bj * 32 + tx;
    if (i1 < n && j1 < n) t1[r][tx] = Ms[(int64_t)i1 * ld + j1];
    const int i2 = bj * 32 + r, j2 = bi * 32 + tx;
    if (bi != bj && i2 < n && j2 < n) t2[r][tx] = Ms[(int64_t)i2 * ld + j2];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    // tile (bi, bj) <- transpose of tile (bj, bi); tile (bj, bi) <- transpose of tile (bi, bj)
    const int i1 = bi * 32 + r, j1 = bj * 32 + tx;
    if (i1 < n && j1 < n) Ms[(int64_t)i1 * ld + j1] = (bi != bj) ? t2[tx][r] : t1[tx][r];
    const int i2 = bj * 32 + r, j2 = bi * 32 + tx;
    if (bi != bj && i2 < n && j2 < n) Ms[(int64_t)i2 * ld + j2] = t1[tx][r];
  }
}
// B (n x m, ld n) = A^T for A (m x n, lda), FP64 column-major
__global__ void transpose64_kernel(const double* __restrict__ A, int m, int n, int64_t lda, double* __restrict__ B) {
  __shared__ double t[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;  // block of A: rows i0.., cols j0..
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = i0 + threadIdx.x, j = j0 + r;
    if (i < m && j < n) t[r][threadIdx.x] = A[i + (int64_t)j * lda];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int j = j0 + threadIdx.x, i = i0 + r;  // B[j, i] = A[i, j]
    if (i < m && j < n) B[j + (int64_t)i * n] = t[threadIdx.x][r];
  }
}

static int sync_read(Ctx& C, const void* dev, void* host, size_t bytes) {
  LYAP_CUDA_TRY(cudaMemcpyAsync(C.hpin, dev, bytes, cudaMemcpyDeviceToHost, C.s));
  LYAP_CUDA_TRY(cudaStreamSynchronize(C.s));
  memcpy(host, C.hpin, bytes);
  return LYAP_OK;
}

static int fingerprint(Ctx& C, const double* A, int n, int64_t lda, double* out) {
  fingerprint_kernel<<<RED_BLOCKS, 256, 0, C.s>>>(A, n, lda, P<double>(C.part) + 5 * RED_BLOCKS);
  sum_parts_kernel<<<1, 32, 0, C.s>>>(P<double>(C.part) + 5 * RED_BLOCKS, RED_BLOCKS, P<double>(C.scal) + 310);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch(2);
  return sync_read(C, P<double>(C.scal) + 310, out, sizeof(double));
}

// Transpose every stored inverse in place: A_k^{-1} -> A_k^{-T} (and back).
static int transpose_store(Ctx& C) {
  if (C.store_count == 0) return LYAP_OK;
  C.store_t = !C.store_t;
  const int n = C.store_n;
  const unsigned nt = (unsigned)ceil_div(n, 32);
  // checkpoint mode: the iterates are transposed (A_k -> A_k^T); the inverses recomputed
  // from them are then those of A_k^T = (A_k^{-1})^T
  const int count = C.store_ckpt ? (int)ceil_div(C.store_count, C.store_ckpt) : C.store_count;
  const int64_t ld = C.store_ckpt ? n : C.store_ld;
  const size_t slot = C.store_ckpt ? (size_t)n * n : (size_t)C.store_rows * C.store_ld;
  const size_t elt = C.store_ckpt ? C.store_welt : C.store_elt;
  dim3 grid(nt, nt, (unsigned)count), block(32, 8);
  if (elt == 2) transpose_slots_kernel<uint16_t><<<grid, block, 0, C.s>>>((uint16_t*)C.store.p, n, ld, slot);
  else if (elt == 4) transpose_slots_kernel<uint32_t><<<grid, block, 0, C.s>>>((uint32_t*)C.store.p, n, ld, slot);
  else transpose_slots_kernel<uint64_t><<<grid, block, 0, C.s>>>((uint64_t*)C.store.p, n, ld, slot);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}

// Slot of the inverse used at Newton step kk: the stored one, or the recomputed one.
static void* inv_slot(Ctx& C, int kk) {
  if (C.store_ckpt) return C.inv1.p;
  return (char*)C.store.p + (size_t)kk * (size_t)C.store_rows * C.store_ld * C.store_elt;
}
// Checkpoint j (iterate A_{j c}) in checkpoint mode.
static void* ckpt_slot(Ctx& C, int j) { return (char*)C.store.p + (size_t)j * C.store_n * C.store_n * C.store_welt; }

// ---------------------------------------------------------------------------
// the inversion (K1-K3) on the current Newton iterate
// ---------------------------------------------------------------------------
template <typename T>
static int invert_current(Ctx& C, const T* Acur, int n, int prec) {
  GJWork& W = C.gj;
  W.cur = 0;
  LYAP_CUDA_TRY(cudaMemcpyAsync(W.M[0], Acur, sizeof(T) * (size_t)n * n, cudaMemcpyDeviceToDevice, C.s));
  iota_kernel<<<nblk(n), 256, 0, C.s>>>(W.perm[0], n);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  C.flops[LYAP_PHASE_INVERT] += 2.0 * (double)n * n * n;
  return gj_invert_run(W, prec, C.s);
}

// ---------------------------------------------------------------------------
// one factor step of the Newton iteration, given the stored A_k^{-1} (slot kk)
// ---------------------------------------------------------------------------
template <typename T>
static int factor_product(Ctx& C, int n, int c, int prec, int kk, T* Z) {
  if (is16(prec)) {
    const void* Xs = inv_slot(C, kk);
    LYAP_TRY(factor_to_16(prec, (const float*)Z, n, c, n, C.Zh.p, P<int>(C.eZ), C.s));
    LYAP_TRY(tc_product(prec, n, c, Xs, P<int>(C.dex) + kk, C.Zh.p, P<int>(C.eZ), (float*)Z + (size_t)c * n, n,
                        C.s));
  } else {
    const T* Xs = (const T*)inv_slot(C, kk);
    // Xs is row-major, i.e. the transpose of a column-major n x n matrix
    LYAP_TRY(gemm<T>('T', 'N', n, c, n, T(1), Xs, n, Z, n, T(0), Z + (size_t)c * n, n, C.s));
  }
  return LYAP_OK;
}

// RankTruncLdlt in working precision T (Sec. 3.2): Z = QR, R Y R^T = V L V^T, keep |l| > tol max|l|.
template <typename T>
static int rank_trunc_ldlt(Ctx& C, T* Z, int n, int c, double* y, double tol, int* r_out) {
  // thin QR of Z (in place in a copy, T precision)
  T* Fz = (T*)C.qrWork.p;
  LYAP_TRY((copy_cast<T, T>(Z, n, c, n, Fz, n, 1.0, C.s)));
  LYAP_TRY(ensure(C.tau, (size_t)(c + 8) * 8));
  LYAP_TRY(householder_qr<T>(Fz, n, c, n, (T*)C.tau.p, C.qr, C.s));
  const int kr = std::min(n, c);
  LYAP_TRY(ensure(C.Tm, (size_t)kr * c * 8 + 64));
  LYAP_TRY(ensure(C.TP, (size_t)kr * c * 8 + 64));
  LYAP_TRY(ensure(C.H, (size_t)kr * kr * 8 + 64));
  LYAP_TRY(ensure(C.w, (size_t)kr * 8 + 64));
  LYAP_TRY(ensure(C.Qh, (size_t)kr * kr * 8 + 64));
  LYAP_TRY(ensure(C.Csel, (size_t)kr * kr * 8 + 64));
  double* R64 = P<double>(C.Tm);
  // R (kr x c) in FP64
  {
    double* tmp = P<double>(C.TP);
    LYAP_TRY((copy_cast<T, double>(Fz, kr, c, n, tmp, kr, 1.0, C.s)));
    extract_r_kernel<<<nblk((int64_t)kr * c), 256, 0, C.s>>>(tmp, kr, kr, c, R64);
    lyap_count_launch();
  }
  // M = R diag(y) R^T
  double* RY = P<double>(C.TP);
  scale_cols_dev_kernel<<<nblk((int64_t)kr * c), 256, 0, C.s>>>(R64, kr, c, c + 1, y, RY);
  lyap_count_launch();
  LYAP_TRY(gemm<double>('N', 'T', kr, kr, c, 1.0, RY, kr, R64, kr, 0.0, P<double>(C.H), kr, C.s));
  LYAP_TRY(prepare_eig(C, kr));
  LYAP_TRY(sym_eig(P<double>(C.H), kr, kr, P<double>(C.w), P<double>(C.Qh), kr, sizeof(T) == 8 ? 1 : 0, C.eig, C.s));
  int* sel = P<int>(C.scal) + 64;
  select_kernel<<<1, 32, 0, C.s>>>(P<double>(C.w), kr, tol, 1, sel, P<double>(C.scal) + 100);
  lyap_count_launch();
  int hs[2];
  LYAP_TRY(sync_read(C, sel, hs, sizeof(hs)));
  const int nneg = hs[0], pos = hs[1];
  const int r = nneg + (kr - pos);
  // V_t (kr x r) = [Q[:, 0:nneg], Q[:, pos:kr]], y_t = eigenvalues
  double* Vt = P<double>(C.Csel);
  double* yt = P<double>(C.yv2);
  if (nneg > 0) {
    gather_cols_kernel<<<nblk((int64_t)kr * nneg), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), 0, nneg, 0,
                                                                 Vt, kr, yt);
    lyap_count_launch();
  }
  if (kr - pos > 0) {
    gather_cols_kernel<<<nblk((int64_t)kr * (kr - pos)), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), pos,
                                                                       kr - pos, 0, Vt + (size_t)nneg * kr, kr,
                                                                       yt + nneg);
    lyap_count_launch();
  }
  LYAP_CUDA_TRY(cudaGetLastError());
  // Z_new = Q [V_t; 0] (working precision)
  T* Vw = (T*)C.Zw2.p;
  LYAP_TRY((copy_cast<double, T>(Vt, kr, r, kr, Vw, kr, 1.0, C.s)));
  LYAP_TRY(apply_q<T>(Fz, n, kr, n, (const T*)C.tau.p, Vw, kr, r, Z, n, C.s));
  LYAP_CUDA_TRY(cudaMemcpyAsync(y, yt, sizeof(double) * r, cudaMemcpyDeviceToDevice, C.s));
  *r_out = r;
  return LYAP_OK;
}

struct NewtonOpts {
  int prec, scaling, norm_fro, stop_after, delta_rule, kmax;
  double tau, scale_off, rank_tol, rho;
};

// ||M||_2 (spectral = false; 12 power steps on M^T M) or the spectral radius of M P
// (spectral = true; (P v)_p = v[cmap[p]], cmap == NULL: P = I) of the row-major n x n M,
// written to *est on the device (FP32 iteration, FP64 norms).
template <typename T>
static int norm_estimate(Ctx& C, const T* M, int n, const int* cmap, bool spectral, double* est) {
  const int steps = spectral ? PN_STEPS_SPECTRAL : PN_STEPS_NORM2;
  const size_t hb = (size_t)(PN_STEPS_SPECTRAL + 2) * 8;
  LYAP_TRY(ensure(C.pnw, hb + (size_t)(2 + PN_SPLIT) * n * 4 + 64));
  double* hist = P<double>(C.pnw);
  float* v = reinterpret_cast<float*>(static_cast<char*>(C.pnw.p) + hb);
  float* u = v + n;
  float* part = u + n;
  pn_init_kernel<<<1, 1024, 0, C.s>>>(n, v, hist);
  const unsigned rows = (unsigned)std::min<int64_t>(4096, ceil_div((int64_t)n, 8));
  for (int k = 1; k <= steps; ++k) {
    pn_mv_kernel<T><<<rows, 256, 0, C.s>>>(M, n, spectral ? cmap : nullptr, v, hist + k - 1, u);
    if (spectral) {
      pn_sum_kernel<<<1, 1024, 0, C.s>>>(u, n, 1, v, hist + k);
    } else {
      pn_mtv_kernel<T><<<dim3((unsigned)ceil_div((int64_t)n, 256), PN_SPLIT), 256, 0, C.s>>>(M, n, u, part);
      pn_sum_kernel<<<1, 1024, 0, C.s>>>(part, n, PN_SPLIT, v, hist + k);
    }
  }
  pn_final_kernel<<<1, 32, 0, C.s>>>(hist, steps, spectral ? 1 : 0, est);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch(2 + steps * (spectral ? 2 : 3));
  return LYAP_OK;
}

struct AdiOpts {
  int shifts, maxit;
  double tol;
};

// Low-rank ADI on Z (working precision; the right-hand side factor L in C.Zw, n x m, weights
// in C.yv for LDL^T).  compute == true: estimate a = 1/||A0^-1||_2 and b = ||A0||_2 (power
// iteration), place the real shifts, and store the shifted inverses (A0 + p_j I)^{-1}
// (A0 = the prescaled working matrix in C.A0); else reuse them.  Then the iteration of
// LYAP_INNER_ADI until ||W S W^T||_F <= tol ||L S L^T||_F, with the truncations of the Newton
// solver whenever cols(Z) > rho n.  *c_out: columns of Z (in C.Zw, weights in C.yv).
template <typename T>
static int adi_run(Ctx& C, int n, int m, bool ldlt, const NewtonOpts& o, const AdiOpts& ao, bool compute, int* c_out,
                   lyap_info_t* info) {
  NewtonState* st = P<NewtonState>(C.state);
  T* Z = P<T>(C.Zw);
  double* y = P<double>(C.yv);
  const bool s16 = is16(o.prec);
  if (compute) {
    const int ns = ao.shifts;
    if (ns < 1 || ns > o.kmax) {
      lyap_set_error_message("adi_shifts must lie in 1..kmax", __FILE__, __LINE__);
      return LYAP_ERR_ARG;
    }
    mark(C, LYAP_PHASE_NEWTON);
    T* A0 = P<T>(C.A0);
    T* M = P<T>(C.A1);
    LYAP_TRY(norm_estimate<T>(C, A0, n, nullptr, false, &st->nrmA));
    mark(C, LYAP_PHASE_INVERT);
    LYAP_TRY(invert_current<T>(C, A0, n, o.prec));
    mark(C, LYAP_PHASE_NEWTON);
    LYAP_TRY(norm_estimate<T>(C, (const T*)C.gj.M[C.gj.cur], n, nullptr, false, &st->nrmX));
    NewtonState hst;
    LYAP_TRY(sync_read(C, st, &hst, sizeof(NewtonState)));
    int gjs = 0;
    LYAP_TRY(sync_read(C, C.gj.status, &gjs, sizeof(int)));
    if (gjs) return gjs;
    const double b = hst.nrmA, a = 1.0 / hst.nrmX;
    if (!std::isfinite(a) || !std::isfinite(b) || !(a > 0.0) || !(b > 0.0)) return LYAP_ERR_NONFINITE;
    C.adi_p.assign(ns, 0.0);
    for (int j = 0; j < ns; ++j) C.adi_p[j] = -b * std::pow(std::min(a, b) / b, (2.0 * j + 1.0) / (2.0 * ns));
    for (int j = 0; j < ns; ++j) {
      adi_shift_kernel<T><<<nblk((int64_t)n * n), 256, 0, C.s>>>(A0, n, C.adi_p[j], M);
      lyap_count_launch();
      mark(C, LYAP_PHASE_INVERT);
      LYAP_TRY(invert_current<T>(C, M, n, o.prec));
      mark(C, LYAP_PHASE_NEWTON);
      const T* X = (const T*)C.gj.M[C.gj.cur];
      pinv_kernel<<<nblk(n), 256, 0, C.s>>>(C.gj.perm[C.gj.cur], P<int>(C.pinv), n);
      LYAP_TRY(maxabs<T>(X, n, n, n, &st->maxX, P<double>(C.part), C.s));
      adi_exp_kernel<<<1, 1, 0, C.s>>>(&st->maxX, j, s16 ? 1 : 0, P<int>(C.dex), P<double>(C.dmu));
      void* slot = inv_slot(C, j);
      const unsigned nb = (unsigned)std::min<int64_t>(4096, ceil_div((int64_t)n * n, 256));
      switch (o.prec) {
        case LYAP_FP64:
          adi_store_kernel<double, double><<<nb, 256, 0, C.s>>>(n, (const double*)X, P<int>(C.pinv), P<int>(C.dex), j,
                                                              (double*)slot, C.store_ld);
          break;
        case LYAP_FP32:
          adi_store_kernel<float, float><<<nb, 256, 0, C.s>>>(n, (const float*)X, P<int>(C.pinv), P<int>(C.dex), j,
                                                            (float*)slot, C.store_ld);
          break;
        case LYAP_FP16:
          adi_store_kernel<float, __half><<<nb, 256, 0, C.s>>>(n, (const float*)X, P<int>(C.pinv), P<int>(C.dex), j,
                                                             (__half*)slot, C.store_ld);
          break;
        case LYAP_BF16:
          adi_store_kernel<float, __nv_bfloat16><<<nb, 256, 0, C.s>>>(n, (const float*)X, P<int>(C.pinv),
                                                                    P<int>(C.dex), j, (__nv_bfloat16*)slot,
                                                                    C.store_ld);
          break;
      }
      LYAP_CUDA_TRY(cudaGetLastError());
      lyap_count_launch(3);
      LYAP_TRY(sync_read(C, C.gj.status, &gjs, sizeof(int)));
      if (gjs) return gjs;
      if (info && j < 64) info->mu[j] = C.adi_p[j];
    }
    C.store_count = ns;
  } else if ((int)C.adi_p.size() != C.store_count) {
    lyap_set_error_message("no stored ADI shifts for this problem", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  const int ns = C.store_count;
  // [W, V] and the weights of W
  LYAP_TRY(ensure(C.adiW, (size_t)n * 2 * m * sizeof(T) + 64));
  LYAP_TRY(ensure(C.adiY, (size_t)m * 8 + 64));
  LYAP_TRY(ensure(C.adiG, (size_t)m * m * 8 + 64));
  T* Y = P<T>(C.adiW);
  double* y0 = P<double>(C.adiY);
  LYAP_CUDA_TRY(cudaMemcpyAsync(Y, Z, sizeof(T) * (size_t)n * m, cudaMemcpyDeviceToDevice, C.s));
  if (ldlt) LYAP_CUDA_TRY(cudaMemcpyAsync(y0, y, sizeof(double) * m, cudaMemcpyDeviceToDevice, C.s));
  double* sc = P<double>(C.scal) + 48;
  auto resnorm = [&](double* out) -> int {
    // ||W diag(y0) W^T||_F^2 through the m x m Gram matrix of W (FP64; C.Lst is free here)
    LYAP_TRY(ensure(C.Lst, (size_t)n * m * 8 + 64));
    double* W64 = P<double>(C.Lst);
    LYAP_TRY((copy_cast<T, double>(Y, n, m, n, W64, n, 1.0, C.s)));
    LYAP_TRY(gemm<double>('T', 'N', m, m, n, 1.0, W64, n, W64, n, 0.0, P<double>(C.adiG), m, C.s));
    adi_resnorm_kernel<<<1, 256, 0, C.s>>>(P<double>(C.adiG), m, ldlt ? y0 : nullptr, out);
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
    return LYAP_OK;
  };
  mark(C, LYAP_PHASE_FACTOR);
  LYAP_TRY(resnorm(sc));
  double r0 = 0.0;
  LYAP_TRY(sync_read(C, sc, &r0, sizeof(double)));
  int c = 0;
  for (int it = 0; it < ao.maxit && r0 > 0.0; ++it) {
    const int j = it % ns;
    const double p = C.adi_p[j];
    if (c + m > 2 * n + 8) {
      lyap_set_error_message("ADI factor exceeds its capacity", __FILE__, __LINE__);
      return LYAP_ERR_CAPACITY;
    }
    mark(C, LYAP_PHASE_FACTOR);
    // V = (A0 + p_j I)^{-1} W into the second half of Y
    LYAP_TRY(factor_product<T>(C, n, m, o.prec, j, Y));
    adi_step_kernel<T><<<nblk((int64_t)n * m), 256, 0, C.s>>>(Y, n, m, p, ldlt ? 1.0 : std::sqrt(-2.0 * p), Z, c, y0,
                                                             ldlt ? y : nullptr);
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
    c += m;
    if ((double)c > o.rho * (double)n) {
      mark(C, LYAP_PHASE_COMPRESS);
      int r = 0;
      if (!ldlt) {
        LYAP_TRY(qrcp_truncate<T>(Z, n, c, n, o.rank_tol, C.qr, C.s));
        LYAP_TRY(sync_read(C, C.qr.rank, &r, sizeof(int)));
      } else {
        LYAP_TRY(rank_trunc_ldlt<T>(C, Z, n, c, y, o.rank_tol, &r));
      }
      c = r;
    }
    mark(C, LYAP_PHASE_FACTOR);
    LYAP_TRY(resnorm(sc));
    double rj = 0.0;
    LYAP_TRY(sync_read(C, sc, &rj, sizeof(double)));
    if (!std::isfinite(rj)) return LYAP_ERR_NONFINITE;
    if (std::sqrt(rj) <= ao.tol * std::sqrt(r0)) break;
  }
  mark(C, LYAP_PHASE_OTHER);
  int qrs = 0, tcs = 0;
  LYAP_TRY(sync_read(C, C.qr.status, &qrs, sizeof(int)));
  if (qrs) return qrs;
  if (s16) {
    LYAP_TRY(tc_status_read(&tcs));
    if (tcs) return tcs;
  }
  *c_out = c;
  return LYAP_OK;
}

static int solve_entry(lyap_ctx_t* C, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl,
                       int64_t m, const double* S, int64_t lds, const lyap_opts_t* opts, double* Z, int64_t ldz,
                       int64_t z_cap, double* D, int64_t* rank_out, lyap_info_t* info, bool refine);

// diag(R) of the leading q columns of a Householder-factored F (ld): out[j] = |F[j, j]|
template <typename T>
__global__ void ek_rdiag_kernel(const T* __restrict__ F, int64_t ld, int q, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x)
    out[j] = fabs((double)F[j + (int64_t)j * ld]);
}

// Extended Krylov (Galerkin) on Z (working precision; the right-hand side factor L in C.Zw,
// n x m, weights in C.yv for LDL^T).  compute == true: A0^{-1} (A0 = the prescaled working
// matrix) is inverted at u_s and stored in slot 0, as the Newton sequence; else reused.  The
// basis V = [U_1, U_2, ...] (orthonormal blocks of 2m columns): U_1 = orth([L, A0^{-1} L]),
// U_{j+1} = orth([A0 U_j^(1), A0^{-1} U_j^(2)] minus its projection on V, twice).  With
// T = V^T A0 V and E = V^T L the projected equation T Y + Y T^T + E S E^T = 0 is solved by
// the FP64 sign-Newton solver on a context of its own (T must be stable: A0 + A0^T < 0
// guarantees it); the residual norm is sqrt(2) ||U_{j+1}^T A0 V Y||_F, and the iteration
// stops once it is <= tol ||L S L^T||_F (or on breakdown of the new block, or at maxit).
// Result Z = V Z_Y (weights D_Y) in C.Zw / C.yv, *c_out its columns.
template <typename T>
static int eksm_run(Ctx& C, int n, int m, bool ldlt, const NewtonOpts& o, int maxit, double tol, bool compute,
                    int* c_out) {
  NewtonState* st = P<NewtonState>(C.state);
  T* Z = P<T>(C.Zw);
  double* y = P<double>(C.yv);
  const bool s16 = is16(o.prec);
  T* A0 = P<T>(C.A0);
  if (compute) {
    mark(C, LYAP_PHASE_INVERT);
    LYAP_TRY(invert_current<T>(C, A0, n, o.prec));
    mark(C, LYAP_PHASE_NEWTON);
    const T* X = (const T*)C.gj.M[C.gj.cur];
    pinv_kernel<<<nblk(n), 256, 0, C.s>>>(C.gj.perm[C.gj.cur], P<int>(C.pinv), n);
    LYAP_TRY(maxabs<T>(X, n, n, n, &st->maxX, P<double>(C.part), C.s));
    adi_exp_kernel<<<1, 1, 0, C.s>>>(&st->maxX, 0, s16 ? 1 : 0, P<int>(C.dex), P<double>(C.dmu));
    void* slot = inv_slot(C, 0);
    const unsigned nb = (unsigned)std::min<int64_t>(4096, ceil_div((int64_t)n * n, 256));
    switch (o.prec) {
      case LYAP_FP64:
        adi_store_kernel<double, double><<<nb, 256, 0, C.s>>>(n, (const double*)X, P<int>(C.pinv), P<int>(C.dex), 0,
                                                            (double*)slot, C.store_ld);
        break;
      case LYAP_FP32:
        adi_store_kernel<float, float><<<nb, 256, 0, C.s>>>(n, (const float*)X, P<int>(C.pinv), P<int>(C.dex), 0,
                                                          (float*)slot, C.store_ld);
        break;
      case LYAP_FP16:
        adi_store_kernel<float, __half><<<nb, 256, 0, C.s>>>(n, (const float*)X, P<int>(C.pinv), P<int>(C.dex), 0,
                                                           (__half*)slot, C.store_ld);
        break;
      case LYAP_BF16:
        adi_store_kernel<float, __nv_bfloat16><<<nb, 256, 0, C.s>>>(n, (const float*)X, P<int>(C.pinv),
                                                                  P<int>(C.dex), 0, (__nv_bfloat16*)slot,
                                                                  C.store_ld);
        break;
    }
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch(3);
    int gjs = 0;
    LYAP_TRY(sync_read(C, C.gj.status, &gjs, sizeof(int)));
    if (gjs) return gjs;
    C.store_count = 1;
  } else if (C.store_count != 1) {
    lyap_set_error_message("no stored inverse for the extended Krylov solver", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  if (!C.sub) LYAP_TRY(lyap_ctx_create(&C.sub, C.s));
  LYAP_TRY(lyap_ctx_set_stream(C.sub, C.s));
  const int b = 2 * m;                                    // block width
  const int kcap = std::min(n, b * (maxit + 1));
  const size_t te = sizeof(T);
  LYAP_TRY(ensure(C.ekV, (size_t)n * (kcap + b) * te + 64));
  LYAP_TRY(ensure(C.ekAV, (size_t)n * (kcap + b) * te + 64));
  LYAP_TRY(ensure(C.ekW, (size_t)n * 2 * b * te + 64));
  LYAP_TRY(ensure(C.ekL, (size_t)n * m * te + 64));
  LYAP_TRY(ensure(C.ekT, (size_t)kcap * kcap * 8 + 64));
  LYAP_TRY(ensure(C.ekE, (size_t)kcap * m * 8 + 64));
  LYAP_TRY(ensure(C.ekS, (size_t)m * m * 8 + 64));
  LYAP_TRY(ensure(C.ekZY, (size_t)kcap * kcap * 8 + 64));
  LYAP_TRY(ensure(C.ekD, (size_t)kcap * 8 + 64));
  LYAP_TRY(ensure(C.ekH, (size_t)(kcap + b) * b * te + 64));
  LYAP_TRY(ensure(C.ekTau, (size_t)(b + 8) * te));
  LYAP_TRY(ensure(C.ekP, (size_t)b * kcap * 8 + 64));
  LYAP_TRY(ensure(C.ekQ, (size_t)std::max<int64_t>((int64_t)kcap * kcap, (int64_t)b * kcap) * 8 + 64));
  LYAP_TRY(ensure(C.ekR, (size_t)(b + 8) * 8));
  LYAP_TRY(ensure(C.qrWork, (size_t)n * b * te + 64));
  T* V = P<T>(C.ekV);
  T* AV = P<T>(C.ekAV);
  T* W = P<T>(C.ekW);       // [W | scratch] n x 2b
  T* Lr = P<T>(C.ekL);
  T* H = P<T>(C.ekH);
  T* tauq = P<T>(C.ekTau);
  double* sc = P<double>(C.scal) + 56;
  LYAP_CUDA_TRY(cudaMemcpyAsync(Lr, Z, te * (size_t)n * m, cudaMemcpyDeviceToDevice, C.s));
  // weights of the right-hand side (S = diag(y0)) as an m x m FP64 matrix for the small solves
  std::vector<double> y0(m, 1.0);
  if (ldlt) LYAP_TRY(sync_read(C, y, y0.data(), sizeof(double) * m));
  {
    std::vector<double> Sh((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Sh[(size_t)i * m + i] = y0[i];
    LYAP_CUDA_TRY(cudaMemcpyAsync(C.ekS.p, Sh.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice, C.s));
    LYAP_CUDA_TRY(cudaStreamSynchronize(C.s));
  }
  // ||L S L^T||_F^2 through the Gram matrix of L
  double nrm0 = 0.0;
  {
    LYAP_TRY(ensure(C.Lst, (size_t)n * m * 8 + 64));
    double* L64 = P<double>(C.Lst);
    LYAP_TRY((copy_cast<T, double>(Lr, n, m, n, L64, n, 1.0, C.s)));
    LYAP_TRY(gemm<double>('T', 'N', m, m, n, 1.0, L64, n, L64, n, 0.0, P<double>(C.ekP), m, C.s));
    adi_resnorm_kernel<<<1, 256, 0, C.s>>>(P<double>(C.ekP), m, ldlt ? y : nullptr, sc);
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
    LYAP_TRY(sync_read(C, sc, &nrm0, sizeof(double)));
    nrm0 = std::sqrt(nrm0);
  }
  if (!(nrm0 > 0.0)) {
    *c_out = 0;
    return LYAP_OK;
  }
  mark(C, LYAP_PHASE_FACTOR);
  double ek_last_min = 0.0, ek_last_rms = 0.0;
  // orthonormalise the n x b block Wb (in W) against V[:, :k] (twice) and into V[:, k:k+b];
  // false on breakdown (a column of the new block below 1e-10 of its size before projection)
  auto next_block = [&](int k, bool* broke) -> int {
    double pre = 0.0;
    LYAP_TRY(sumsq<T>(W, n, b, n, sc, P<double>(C.part), C.s));
    LYAP_TRY(sync_read(C, sc, &pre, sizeof(double)));
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      LYAP_TRY(gemm<T>('T', 'N', k, b, n, T(1), V, n, W, n, T(0), H, k, C.s));
      LYAP_TRY(gemm<T>('N', 'N', n, b, k, T(-1), V, n, H, k, T(1), W, n, C.s));
    }
    T* F = (T*)C.qrWork.p;
    LYAP_TRY((copy_cast<T, T>(W, n, b, n, F, n, 1.0, C.s)));
    LYAP_CUDA_TRY(cudaMemsetAsync(C.qr.status, 0, sizeof(int), C.s));
    LYAP_TRY(householder_qr<T>(F, n, b, n, tauq, C.qr, C.s));
    ek_rdiag_kernel<T><<<1, 128, 0, C.s>>>(F, n, b, P<double>(C.ekR));
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
    std::vector<double> rd(b);
    LYAP_TRY(sync_read(C, C.ekR.p, rd.data(), sizeof(double) * b));
    int qs = 0;
    LYAP_TRY(sync_read(C, C.qr.status, &qs, sizeof(int)));
    if (qs) return qs;
    double mn = rd[0];
    for (double v : rd) mn = std::min(mn, v);
    ek_last_min = mn;
    ek_last_rms = std::sqrt(pre / b);
    *broke = !(mn > 1e-10 * std::sqrt(pre / b));
    if (*broke) return LYAP_OK;
    // explicit Q: V[:, k:k+b] = Q [I; 0]
    LYAP_TRY(set_identity<T>(H, b, b, C.s));
    LYAP_TRY(apply_q<T>(F, n, b, n, tauq, H, b, b, V + (size_t)k * n, n, C.s));
    // A0 times the new block (A0 is row-major: the transpose of a column-major matrix; while
    // the store is transposed for the adjoint, the operator is A0^T)
    LYAP_TRY(gemm<T>(C.store_t ? 'N' : 'T', 'N', n, b, n, T(1), A0, n, V + (size_t)k * n, n, T(0),
                     AV + (size_t)k * n, n, C.s));
    return LYAP_OK;
  };
  // U_1 = orth([L, A0^{-1} L]); when it has n columns or more the space is all of R^n and the
  // projected equation is the equation itself (V = I)
  const bool full = (b >= n);
  bool broke = false;
  if (full) {
    LYAP_TRY(set_identity<T>(V, n, n, C.s));
    LYAP_TRY(gemm<T>(C.store_t ? 'N' : 'T', 'N', n, n, n, T(1), A0, n, V, n, T(0), AV, n, C.s));
  } else {
    LYAP_CUDA_TRY(cudaMemcpyAsync(W, Lr, te * (size_t)n * m, cudaMemcpyDeviceToDevice, C.s));
    LYAP_TRY(factor_product<T>(C, n, m, o.prec, 0, W));   // W[:, m:2m] = A0^{-1} L
    LYAP_TRY(next_block(0, &broke));
    if (broke) {
      char msg[160];
      snprintf(msg, sizeof(msg), "extended Krylov: the first block [L, A^-1 L] is rank deficient (n %d, m %d, "
               "min |r_jj| %.3e, rms column %.3e)", n, m, ek_last_min, ek_last_rms);
      lyap_set_error_message(msg, __FILE__, __LINE__);
      return LYAP_ERR_NOCONV;
    }
  }
  int k = full ? n : b;  // columns of V in the current projection
  int kY = k;            // columns of V that Z_Y belongs to
  int rY = 0;            // columns of Z_Y
  lyap_opts_t so;
  lyap_opts_default(&so);
  so.u_s = LYAP_FP64;
  so.rho = 0.0;
  for (int it = 0; it < maxit; ++it) {
    broke = full;
    if (!full) {
      // the next block from U_j = V[:, k-b:k]: [A0 U^(1), A0^{-1} U^(2)]
      LYAP_CUDA_TRY(cudaMemcpyAsync(W, AV + (size_t)(k - b) * n, te * (size_t)n * m, cudaMemcpyDeviceToDevice, C.s));
      T* Ws = W + (size_t)b * n;  // scratch [U^(2) | A0^{-1} U^(2)]
      LYAP_CUDA_TRY(cudaMemcpyAsync(Ws, V + (size_t)(k - m) * n, te * (size_t)n * m, cudaMemcpyDeviceToDevice, C.s));
      LYAP_TRY(factor_product<T>(C, n, m, o.prec, 0, Ws));
      LYAP_CUDA_TRY(cudaMemcpyAsync(W + (size_t)m * n, Ws + (size_t)m * n, te * (size_t)n * m,
                                    cudaMemcpyDeviceToDevice, C.s));
      const bool room = (k + b <= n) && (k + b <= kcap);
      broke = !room;
      if (room) LYAP_TRY(next_block(k, &broke));
    }
    // projected equation on V[:, :k]: T = V^T A0 V, E = V^T L (FP64)
    {
      T* Tw = (T*)C.ekQ.p;  // k x k
      LYAP_TRY(gemm<T>('T', 'N', k, k, n, T(1), V, n, AV, n, T(0), Tw, k, C.s));
      LYAP_TRY((copy_cast<T, double>(Tw, k, k, k, P<double>(C.ekT), k, 1.0, C.s)));
      LYAP_TRY(gemm<T>('T', 'N', k, m, n, T(1), V, n, Lr, n, T(0), Tw, k, C.s));
      LYAP_TRY((copy_cast<T, double>(Tw, k, m, k, P<double>(C.ekE), k, 1.0, C.s)));
    }
    int64_t r64 = 0;
    lyap_info_t sinfo;
    LYAP_TRY(solve_entry(C.sub, P<double>(C.ekT), k, k, P<double>(C.ekE), k, m, ldlt ? P<double>(C.ekS) : nullptr, m,
                         &so, P<double>(C.ekZY), k, k, ldlt ? P<double>(C.ekD) : nullptr, &r64, &sinfo, false));
    rY = (int)r64;
    kY = k;
    if (broke) break;  // invariant subspace, all of R^n, or no room: the projection on V is the answer
    // residual: sqrt(2) ||U_{j+1}^T A0 V Y||_F with Y = Z_Y D Z_Y^T
    {
      T* Tw = (T*)C.ekQ.p;
      LYAP_TRY(gemm<T>('T', 'N', b, k, n, T(1), V + (size_t)k * n, n, AV, n, T(0), Tw, b, C.s));  // tau (b x k)
      double* tau64 = P<double>(C.ekP);
      LYAP_TRY((copy_cast<T, double>(Tw, b, k, b, tau64, b, 1.0, C.s)));
      double* PZ = P<double>(C.ekQ);
      LYAP_TRY(gemm<double>('N', 'N', b, rY, k, 1.0, tau64, b, P<double>(C.ekZY), k, 0.0, PZ, b, C.s));
      if (ldlt) LYAP_TRY(scale_cols<double>(PZ, b, rY, b, P<double>(C.ekD), C.s));
      double* PY = P<double>(C.ekP);
      LYAP_TRY(gemm<double>('N', 'T', b, k, rY, 1.0, PZ, b, P<double>(C.ekZY), k, 0.0, PY, b, C.s));
      LYAP_TRY(sumsq<double>(PY, b, k, b, sc, P<double>(C.part), C.s));
      double r2 = 0.0;
      LYAP_TRY(sync_read(C, sc, &r2, sizeof(double)));
      if (!std::isfinite(r2)) return LYAP_ERR_NONFINITE;
      if (std::sqrt(2.0 * r2) <= tol * nrm0) break;
    }
    k += b;
  }
  // Z = V[:, :k] Z_Y (working precision), weights D_Y
  if (rY > 2 * n + 8) {
    lyap_set_error_message("extended Krylov factor exceeds its capacity", __FILE__, __LINE__);
    return LYAP_ERR_CAPACITY;
  }
  {
    T* ZYw = (T*)C.ekQ.p;
    LYAP_TRY((copy_cast<double, T>(P<double>(C.ekZY), kY, rY, kY, ZYw, kY, 1.0, C.s)));
    LYAP_TRY(gemm<T>('N', 'N', n, rY, kY, T(1), V, n, ZYw, kY, T(0), Z, n, C.s));
    if (ldlt) LYAP_CUDA_TRY(cudaMemcpyAsync(y, C.ekD.p, sizeof(double) * rY, cudaMemcpyDeviceToDevice, C.s));
  }
  mark(C, LYAP_PHASE_OTHER);
  if (s16) {
    int tcs = 0;
    LYAP_TRY(tc_status_read(&tcs));
    if (tcs) return tcs;
  }
  *c_out = rY;
  return LYAP_OK;
}

// Run the sign-Newton factor iteration on Z (working precision, n x c0 in C.Zw, column-major).
// compute == true: compute and store the inverse sequence from the working
// matrix in C.A0 (row-major, already scaled); else replay the stored sequence.
template <typename T>
static int newton_run(Ctx& C, int n, int c0, bool ldlt, const NewtonOpts& o, bool compute, int* c_out,
                      lyap_info_t* info) {
  NewtonState* st = P<NewtonState>(C.state);
  const size_t nn = (size_t)n * n;
  int c = c0;
  T* Z = P<T>(C.Zw);
  double* y = P<double>(C.yv);
  int K = compute ? o.kmax : C.store_count;
  if (compute) {
    C.store_count = 0;
    // the compressions below report through the QR status word: clear what an earlier call
    // left in it
    LYAP_CUDA_TRY(cudaMemsetAsync(C.qr.status, 0, sizeof(int), C.s));
    newton_init_kernel<<<1, 1, 0, C.s>>>(st, o.scaling);
    lyap_count_launch();
    LYAP_TRY(sumsq<T>(P<T>(C.A0), n, n, n, &st->ssA, P<double>(C.part), C.s));
  }
  T* Acur = P<T>(C.A0);
  T* Anext = P<T>(C.A1);
  bool finished = false;
  // the 2-norm / spectral scalings need norm estimates while scaling is on (the host learns
  // of its switch-off from the state read back after each step)
  bool est_norms = compute && (o.scaling == LYAP_SCALE_NORM2 || o.scaling == LYAP_SCALE_SPECTRAL);
  const int ce = C.store_ckpt;
  if (!compute && ce) LYAP_CUDA_TRY(cudaMemsetAsync(C.gj.status, 0, sizeof(int), C.s));
  for (int kk = 0; kk < K; ++kk) {
    // the inverse of step kk: computed (first solve), or recomputed from the last checkpoint
    // with the recorded mu_kk and storage exponent (checkpoint mode); a plain replay reads it
    // from the store
    if (compute || ce) {
      if (kk >= 64) {
        lyap_set_error_message("more than 64 Newton steps", __FILE__, __LINE__);
        return LYAP_ERR_NOCONV;
      }
      if (ce && kk % ce == 0) {
        void* cp = ckpt_slot(C, kk / ce);
        if (compute) LYAP_CUDA_TRY(cudaMemcpyAsync(cp, Acur, sizeof(T) * nn, cudaMemcpyDeviceToDevice, C.s));
        else LYAP_CUDA_TRY(cudaMemcpyAsync(Acur, cp, sizeof(T) * nn, cudaMemcpyDeviceToDevice, C.s));
      }
      if (compute) LYAP_CUDA_TRY(cudaMemsetAsync(C.gj.status, 0, sizeof(int), C.s));
      mark(C, LYAP_PHASE_INVERT);
      LYAP_TRY(invert_current<T>(C, Acur, n, o.prec));
      if (!compute) C.recomputed += 1;
      mark(C, LYAP_PHASE_NEWTON);
      const T* X = (const T*)C.gj.M[C.gj.cur];
      const int* perm = C.gj.perm[C.gj.cur];
      pinv_kernel<<<nblk(n), 256, 0, C.s>>>(perm, P<int>(C.pinv), n);
      lyap_count_launch();
      if (compute) {
        LYAP_TRY(sumsq<T>(X, n, n, n, &st->ssX, P<double>(C.part), C.s));
        LYAP_TRY(maxabs<T>(X, n, n, n, &st->maxX, P<double>(C.part), C.s));
        if (o.scaling == LYAP_SCALE_DET) LYAP_TRY(pivot_logs(C.gj, &st->logdet, C.s));
        if (est_norms) {
          const bool sp = (o.scaling == LYAP_SCALE_SPECTRAL);
          LYAP_TRY(norm_estimate<T>(C, Acur, n, nullptr, sp, &st->nrmA));
          LYAP_TRY(norm_estimate<T>(C, X, n, perm, sp, &st->nrmX));
        }
        newton_mu_kernel<<<1, 1, 0, C.s>>>(st, n, o.scaling, is16(o.prec) ? 1 : 0);
      } else {
        newton_recorded_mu_kernel<<<1, 1, 0, C.s>>>(st, P<double>(C.dmu), P<int>(C.dex), kk);
      }
      lyap_count_launch();
      void* slot = inv_slot(C, kk);
      const unsigned nb = RED_BLOCKS;
      switch (o.prec) {
        case LYAP_FP64:
          newton_update_kernel<double, double><<<nb, 256, 0, C.s>>>(n, (const double*)Acur, (const double*)X,
                                                                    P<int>(C.pinv), st, (double*)Anext,
                                                                    (double*)slot, C.store_ld, P<double>(C.part));
          break;
        case LYAP_FP32:
          newton_update_kernel<float, float><<<nb, 256, 0, C.s>>>(n, (const float*)Acur, (const float*)X,
                                                                  P<int>(C.pinv), st, (float*)Anext, (float*)slot, C.store_ld,
                                                                  P<double>(C.part));
          break;
        case LYAP_FP16:
          newton_update_kernel<float, __half><<<nb, 256, 0, C.s>>>(n, (const float*)Acur, (const float*)X,
                                                                   P<int>(C.pinv), st, (float*)Anext,
                                                                   (__half*)slot, C.store_ld, P<double>(C.part));
          break;
        case LYAP_BF16:
          newton_update_kernel<float, __nv_bfloat16><<<nb, 256, 0, C.s>>>(n, (const float*)Acur, (const float*)X,
                                                                          P<int>(C.pinv), st, (float*)Anext,
                                                                          (__nv_bfloat16*)slot, C.store_ld, P<double>(C.part));
          break;
      }
      LYAP_CUDA_TRY(cudaGetLastError());
      lyap_count_launch();
      if (compute) {
        newton_sums_kernel<<<1, 96, 0, C.s>>>(P<double>(C.part), nb, st);
        lyap_count_launch();
        if (!o.norm_fro) {
          colsum_kernel<T><<<nblk(n, 128), 128, 0, C.s>>>(n, Anext, P<double>(C.colsum));
          lyap_count_launch();
          LYAP_TRY(maxabs<double>(P<double>(C.colsum), n, 1, n, &st->stopv, P<double>(C.part) + 3 * RED_BLOCKS, C.s));
        }
        newton_test_kernel<<<1, 1, 0, C.s>>>(st, o.tau, o.norm_fro, o.stop_after, o.delta_rule, o.scale_off,
                                             P<double>(C.dmu), P<int>(C.dex), kk);
        lyap_count_launch();
        C.store_count = kk + 1;
      }
      std::swap(Acur, Anext);
    }
    // factor update with the stored A_kk^{-1}
    if (2 * c + 8 > 2 * n + 8) {
      lyap_set_error_message("Newton factor exceeds its capacity", __FILE__, __LINE__);
      return LYAP_ERR_CAPACITY;
    }
    mark(C, LYAP_PHASE_FACTOR);
    LYAP_TRY(factor_product<T>(C, n, c, o.prec, kk, Z));
    factor_scale_kernel<T><<<ldlt ? 1 : nblk((int64_t)n * 2 * c), 256, 0, C.s>>>(Z, n, n, c, P<double>(C.dmu) + kk,
                                                                                ldlt ? 1 : 0, y);
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
    c *= 2;
    if ((double)c > o.rho * (double)n) {
      mark(C, LYAP_PHASE_COMPRESS);
      int r = 0;
      if (!ldlt) {
        LYAP_TRY(qrcp_truncate<T>(Z, n, c, n, o.rank_tol, C.qr, C.s));
        LYAP_TRY(sync_read(C, C.qr.rank, &r, sizeof(int)));
      } else {
        LYAP_TRY(rank_trunc_ldlt<T>(C, Z, n, c, y, o.rank_tol, &r));
      }
      c = r;
    }
    mark(C, LYAP_PHASE_OTHER);
    if (compute) {
      NewtonState hst;
      LYAP_TRY(sync_read(C, st, &hst, sizeof(NewtonState)));
      int gjs = 0, qrs = 0, tcs = 0;
      LYAP_TRY(sync_read(C, C.gj.status, &gjs, sizeof(int)));
      LYAP_TRY(sync_read(C, C.qr.status, &qrs, sizeof(int)));
      if (is16(o.prec)) {
        LYAP_TRY(tc_status_read(&tcs));
        if (tcs) return tcs;
      }
      if (info && kk < 64) info->mu[kk] = hst.mu;
      if (!hst.scaling_on) est_norms = false;
      if (gjs) return gjs;
      if (qrs) return qrs;
      if (hst.status) return hst.status;
      if (hst.done) {
        finished = true;
        break;
      }
    }
  }
  if (compute && !finished) {
    lyap_set_error_message("sign-Newton reached kmax without meeting its stop test", __FILE__, __LINE__);
    return LYAP_ERR_NOCONV;
  }
  if (!compute) {
    int qrs = 0;
    LYAP_TRY(sync_read(C, C.qr.status, &qrs, sizeof(int)));
    if (qrs) return qrs;
    if (ce) {
      int gjs = 0;
      LYAP_TRY(sync_read(C, C.gj.status, &gjs, sizeof(int)));
      if (gjs) return gjs;
    }
  }
  *c_out = c;
  return LYAP_OK;
}

// ---- kappa_sign(B) for B = [[A, W], [0, -A^T]] (Sec. 4.2) ----
// B (N x N, N = 2n, column-major) from A (lda) and W (n x n)
__global__ void sign_block_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ W, int n,
                                  double* __restrict__ B) {
  const int64_t N = 2 * (int64_t)n, total = N * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / N, i = e - j * N;
    double v;
    if (i < n) v = (j < n) ? A[i + j * lda] : W[i + (j - n) * n];
    else v = (j < n) ? 0.0 : -A[(j - n) + (i - n) * lda];
    B[e] = v;
  }
}
// Y = a X + b Z (N x N, contiguous); D = Y - X when D != NULL
__global__ void axpby_kernel(int64_t total, double a, const double* __restrict__ X, double b,
                             const double* __restrict__ Z, double* __restrict__ Y, double* __restrict__ D) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = X[e], y = a * x + b * Z[e];
    Y[e] = y;
    if (D) D[e] = y - x;
  }
}
// deterministic start of the power method: entries uniform in [-1, 1) from a counter hash
// (splitmix64 of seed + index)
__global__ void hash_fill_kernel(int64_t total, uint64_t seed, double* __restrict__ E) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(e + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    E[e] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}

}  // namespace lyap

// ===========================================================================
// C ABI
// ===========================================================================
using namespace lyap;

extern "C" {

const char* lyap_last_error(void) { return g_err; }

const char* lyap_version(void) { return "liblyap 0.1 (sm_103a)"; }

const char* lyap_status_string(int s) {
  switch (s) {
    case LYAP_OK: return "ok";
    case LYAP_ERR_ARG: return "invalid argument";
    case LYAP_ERR_NONFINITE: return "non-finite value";
    case LYAP_ERR_SINGULAR: return "singular pivot";
    case LYAP_ERR_NOCONV: return "sign-Newton did not converge";
    case LYAP_ERR_CAPACITY: return "output capacity too small";
    case LYAP_ERR_TIMEOUT: return "device wait timed out";
    case LYAP_ERR_CUDA: return "CUDA error";
    case LYAP_ERR_NOMEM: return "out of device memory";
    case LYAP_WARN_STAGNATED: return "refinement stagnated";
    case LYAP_WARN_MAXIT: return "refinement reached imax";
  }
  return "unknown status";
}

int lyap_opts_default(lyap_opts_t* o) {
  if (!o) return LYAP_ERR_ARG;
  memset(o, 0, sizeof(*o));
  o->u_s = LYAP_FP16;
  o->scaling = LYAP_SCALE_FROB;
  o->tau_newton = 0.0;
  o->newton_norm_fro = 0;
  o->stop_after = 2;
  o->delta_rule = 1;
  o->scale_off = 1e-2;
  o->rank_tol = 0.0;
  o->rho = 0.1;
  o->kmax = 50;
  o->imax = 50;
  o->tau_ir = 0.0;
  o->eta_r = 1e-4;
  o->eta_s = 0.0;
  o->stag_theta = 0.9;
  o->stag_count = 2;
  o->project_psd = 1;
  o->inner = LYAP_INNER_SIGN;
  o->adi_shifts = 8;
  o->adi_maxit = 200;
  o->eksm_maxit = 60;
  return LYAP_OK;
}

int lyap_ctx_create(lyap_ctx_t** out, void* stream) {
  if (!out) return LYAP_ERR_ARG;
  *out = nullptr;
  int dev = 0;
  LYAP_CUDA_TRY(cudaGetDevice(&dev));
  int sms = 0;
  LYAP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  lyap_ctx* C = new lyap_ctx();
  C->device = dev;
  C->s = (cudaStream_t)stream;
  C->num_sms = sms;
  if (cudaMallocHost(&C->hpin, 1 << 16) != cudaSuccess) {
    delete C;
    lyap_set_error_message("pinned host allocation failed", __FILE__, __LINE__);
    return LYAP_ERR_NOMEM;
  }
  cudaEventCreate(&C->e0);
  cudaEventCreate(&C->e1);
  *out = C;
  return LYAP_OK;
}

static void free_buf(Buf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

int lyap_ctx_destroy(lyap_ctx_t* C) {
  if (!C) return LYAP_OK;
  cudaStreamSynchronize(C->s);
  Buf* all[] = {&C->state, &C->scal, &C->part, &C->hist, &C->gjM0, &C->gjM1, &C->gjPp, &C->gjRt, &C->gjOrig,
                &C->gjPerm0, &C->gjPerm1, &C->gjLog, &C->gjIpiv, &C->gjStatus, &C->gjExps, &C->gjAmax, &C->A0,
                &C->A1, &C->pinv, &C->colsum, &C->Zw, &C->Zw2, &C->Zh, &C->eZ, &C->yv, &C->yv2, &C->store,
                &C->dmu, &C->dex, &C->F, &C->tau, &C->Tm, &C->TP, &C->H, &C->w, &C->Qh, &C->Csel, &C->Lp,
                &C->Lm, &C->Zs, &C->Zbest, &C->G, &C->gram, &C->ysol, &C->ybest, &C->ytmp, &C->Lw, &C->Sd,
                &C->Vs, &C->Lst, &C->Rtau, &C->Bm, &C->VB, &C->qrBar, &C->qrStatus, &C->qrCand, &C->qrNorms, &C->qrPiv, &C->qrRdiag, &C->qrWork,
                &C->qrRank, &C->eigWork32, &C->eigBig, &C->eigX, &C->eigR, &C->eigS, &C->eigHX, &C->eigE, &C->eigLam,
                &C->eigRed, &C->eigW, &C->eigPv, &C->eigInt, &C->At, &C->Ct, &C->ZY, &C->adjT, &C->Hf, &C->tl, &C->inv1, &C->pnw, &C->adiW, &C->adiY, &C->adiG, &C->ekV, &C->ekAV, &C->ekW, &C->ekL,
                &C->ekT, &C->ekE, &C->ekS, &C->ekZY, &C->ekD, &C->ekH, &C->ekTau, &C->ekP, &C->ekQ, &C->ekR};
  for (Buf* b : all) free_buf(*b);
  if (C->sub) lyap_ctx_destroy(C->sub);
  for (lyap_ctx* w : C->pool) lyap_ctx_destroy(w);
  for (cudaStream_t st : C->pool_streams) cudaStreamDestroy(st);
  if (C->hpin) cudaFreeHost(C->hpin);
  if (C->e0) cudaEventDestroy(C->e0);
  if (C->e1) cudaEventDestroy(C->e1);
  for (cudaEvent_t e : C->ev_pool) cudaEventDestroy(e);
  delete C;
  return LYAP_OK;
}

int lyap_ctx_set_stream(lyap_ctx_t* C, void* stream) {
  if (!C) return LYAP_ERR_ARG;
  C->s = (cudaStream_t)stream;
  return LYAP_OK;
}

int lyap_invert(lyap_ctx_t* C, const double* A, int64_t n, int64_t lda, int prec, double* Ainv, int64_t ldai,
                int32_t* ipiv, double* logabsdet) {
  if (!C || !A || !Ainv || n <= 0 || lda < n || ldai < n || prec < 0 || prec > 3) return LYAP_ERR_ARG;
  const int ni = (int)n;
  if (prec == LYAP_FP64) LYAP_TRY(prepare_newton<double>(*C, ni, 1, prec));
  else LYAP_TRY(prepare_newton<float>(*C, ni, 1, prec));
  GJWork& W = C->gj;
  W.cur = 0;
  W.ipiv = ipiv;
  LYAP_CUDA_TRY(cudaMemsetAsync(W.status, 0, sizeof(int), C->s));
  if (prec == LYAP_FP64) LYAP_TRY(cm64_to_rm<double>(A, n, lda, 1.0, (double*)W.M[0], C->s));
  else LYAP_TRY(cm64_to_rm<float>(A, n, lda, 1.0, (float*)W.M[0], C->s));
  iota_kernel<<<nblk(n), 256, 0, C->s>>>(W.perm[0], ni);
  lyap_count_launch();
  int st = gj_invert_run(W, prec, C->s);
  W.ipiv = nullptr;
  if (st < 0) return st;
  if (prec == LYAP_FP64)
    unpermute_kernel<double><<<nblk(n * n), 256, 0, C->s>>>((const double*)W.M[W.cur], W.perm[W.cur], ni, Ainv, ldai);
  else
    unpermute_kernel<float><<<nblk(n * n), 256, 0, C->s>>>((const float*)W.M[W.cur], W.perm[W.cur], ni, Ainv, ldai);
  lyap_count_launch();
  double* ld = P<double>(C->scal);
  LYAP_TRY(pivot_logs(W, ld, C->s));
  LYAP_CUDA_TRY(cudaGetLastError());
  struct { double ld; } h;
  LYAP_TRY(sync_read(*C, ld, &h, sizeof(h)));
  int gs = 0;
  LYAP_TRY(sync_read(*C, W.status, &gs, sizeof(int)));
  if (logabsdet) *logabsdet = h.ld;
  return gs;
}

int lyap_rank_trunc(lyap_ctx_t* C, double* Z, int64_t n, int64_t c, int64_t ldz, double tol, int64_t* rank_out) {
  if (!C || !Z || n <= 0 || c < 0 || ldz < n || !rank_out) return LYAP_ERR_ARG;
  LYAP_TRY(prepare_newton<double>(*C, (int)n, (int)std::max<int64_t>(1, c), LYAP_FP64));
  LYAP_TRY(ensure(C->qrWork, (size_t)n * c * 8 + 64));
  C->qr.work = C->qrWork.p;
  LYAP_TRY(ensure(C->qrRdiag, (size_t)c * 8 + 64));
  C->qr.rdiag = C->qrRdiag.p;
  LYAP_CUDA_TRY(cudaMemsetAsync(C->qr.status, 0, sizeof(int), C->s));
  LYAP_TRY(qrcp_truncate<double>(Z, n, c, ldz, tol, C->qr, C->s));
  int r = 0, qs = 0;
  LYAP_TRY(sync_read(*C, C->qr.rank, &r, sizeof(int)));
  LYAP_TRY(sync_read(*C, C->qr.status, &qs, sizeof(int)));
  *rank_out = r;
  return qs;
}

int lyap_sym_eig(lyap_ctx_t* C, double* H, int64_t q, int64_t ldh, double* w, double* Q, int64_t ldq,
                 int fp64_refine) {
  if (!C || !H || !w || !Q || q <= 0 || ldh < q || ldq < q) return LYAP_ERR_ARG;
  LYAP_TRY(prepare_eig(*C, (int)q));
  LYAP_TRY(sym_eig(H, q, ldh, w, Q, ldq, fp64_refine, C->eig, C->s));
  LYAP_CUDA_TRY(cudaStreamSynchronize(C->s));
  return LYAP_OK;
}

}  // extern "C"

// ===========================================================================
// solver driver
// ===========================================================================
namespace lyap {

struct Problem {
  const double* A;
  int n;
  int64_t lda;
  const double* L;
  int64_t ldl;
  int m;
  const double* S;
  int64_t lds;
};

static NewtonOpts make_newton_opts(const lyap_opts_t& o, int n, bool ldlt) {
  NewtonOpts no;
  no.prec = o.u_s;
  no.scaling = o.scaling;
  no.norm_fro = o.newton_norm_fro;
  no.stop_after = o.stop_after;
  no.delta_rule = o.delta_rule;
  no.kmax = std::min(o.kmax, 64);
  const double us = unit_roundoff(o.u_s);
  no.tau = o.tau_newton > 0 ? o.tau_newton : 10.0 * sqrt((double)n * us);
  no.scale_off = o.scale_off;
  no.rank_tol = o.rank_tol > 0 ? o.rank_tol : (ldlt ? us : sqrt(us));
  no.rho = o.rho;
  return no;
}

// Prepare S: diagonalise (S = V diag(s) V^T, L <- L V) so that every inner factor is
// diagonal.  Returns Lw (n x m FP64, device) and sd (m, device).
static int prepare_rhs(Ctx& C, const Problem& pb, double** Lw_out, double** sd_out, bool* indefinite) {
  const int n = pb.n, m = pb.m;
  LYAP_TRY(ensure(C.Lw, (size_t)n * m * 8 + 64));
  LYAP_TRY(ensure(C.Sd, (size_t)m * 8 + 64));
  *indefinite = false;
  if (!pb.S) {
    LYAP_TRY((copy_cast<double, double>(pb.L, n, m, pb.ldl, P<double>(C.Lw), n, 1.0, C.s)));
    *Lw_out = P<double>(C.Lw);
    *sd_out = nullptr;
    return LYAP_OK;
  }
  LYAP_TRY(ensure(C.Vs, (size_t)m * m * 8 + 64));
  LYAP_TRY(ensure(C.H, (size_t)m * m * 8 + 64));
  LYAP_TRY((copy_cast<double, double>(pb.S, m, m, pb.lds, P<double>(C.H), m, 1.0, C.s)));
  LYAP_TRY(prepare_eig(C, m));
  LYAP_TRY(sym_eig(P<double>(C.H), m, m, P<double>(C.Sd), P<double>(C.Vs), m, 1, C.eig, C.s));
  LYAP_TRY(gemm<double>('N', 'N', n, m, m, 1.0, pb.L, pb.ldl, P<double>(C.Vs), m, 0.0, P<double>(C.Lw), n, C.s));
  std::vector<double> sd(m);
  LYAP_TRY(sync_read(C, C.Sd.p, sd.data(), sizeof(double) * m));
  for (double v : sd)
    if (v < 0) *indefinite = true;
  *Lw_out = P<double>(C.Lw);
  *sd_out = P<double>(C.Sd);
  return LYAP_OK;
}

// Solve A X + X A^T + Lr diag(yr) Lr^T = 0 with the sign-Newton iteration at u_s;
// result (FP64, column-major) into Zout (n x r), yout (LDL^T).  Lr is rounded to u_s.
// compute: build the inverse sequence from A (first solve) or replay it.
template <typename T>
static int newton_solve(Ctx& C, const Problem& pb, const double* Lr, int mr, const double* yr, bool ldlt,
                        const lyap_opts_t& o, bool compute, double* Zout, int64_t ldo, int zcap_out,
                        double* yout, int* r_out, lyap_info_t* info, int* iters) {
  const int n = pb.n;
  NewtonOpts no = make_newton_opts(o, n, ldlt);
  LYAP_TRY(prepare_newton<T>(C, n, std::max(mr, pb.m), o.u_s));
  const size_t nn = (size_t)n * n;
  if (compute) {
    const size_t selt = (o.u_s == LYAP_FP64) ? 8 : (o.u_s == LYAP_FP32 ? 4 : 2);
    // 16-bit inverses are tensor-core A operands: row pitch and row count follow tc_kpitch / tc_rows
    C.store_ld = (selt == 2) ? tc_kpitch(n) : n;
    C.store_rows = (selt == 2) ? tc_rows(n) : n;
    const size_t inv_bytes = (size_t)C.store_rows * C.store_ld * selt;
    const bool padded = selt == 2 && (C.store_ld != n || C.store_rows != n);  // K padding must read as zero
    // checkpoints every ckpt_every steps when asked, or (every 4 steps) when the full
    // sequence of kmax inverses would exceed mem_budget
    int ce = o.ckpt_every > 0 ? o.ckpt_every : 0;
    if (ce == 0 && o.mem_budget > 0 && (double)no.kmax * (double)inv_bytes > (double)o.mem_budget) ce = 4;
    if (o.inner != LYAP_INNER_SIGN) ce = 0;  // the (shifted) inverses of ADI / EKSM are always stored
    C.store_ckpt = ce;
    C.store_welt = sizeof(T);
    if (ce) {
      LYAP_TRY(ensure(C.store, (size_t)ceil_div(no.kmax, ce) * nn * sizeof(T)));
      LYAP_TRY(ensure(C.inv1, inv_bytes));
      if (padded) LYAP_CUDA_TRY(cudaMemsetAsync(C.inv1.p, 0, inv_bytes, C.s));
    } else {
      LYAP_TRY(ensure(C.store, (size_t)no.kmax * inv_bytes));
      if (padded) LYAP_CUDA_TRY(cudaMemsetAsync(C.store.p, 0, (size_t)no.kmax * inv_bytes, C.s));
    }
    C.store_elt = selt;
    C.store_t = false;
    C.store_n = n;
    C.store_prec = o.u_s;
    C.store_count = 0;
    // A_0 = 2^-e0 A (exact power-of-two prescaling: ||A_0||_F in [1, 2))
    double* sc = P<double>(C.scal);
    LYAP_TRY(sumsq<double>(pb.A, n, n, pb.lda, sc, P<double>(C.part), C.s));
    double ssA = 0;
    LYAP_TRY(sync_read(C, sc, &ssA, sizeof(double)));
    int e0 = 0;
    frexp(sqrt(ssA), &e0);
    e0 -= 1;
    C.store_e0 = e0;
    LYAP_TRY(fingerprint(C, pb.A, n, pb.lda, &C.store_fp));
    LYAP_TRY(cm64_to_rm<T>(pb.A, n, pb.lda, ldexp(1.0, -e0), P<T>(C.A0), C.s));
  } else if (C.store_n != n || C.store_prec != o.u_s || C.store_count == 0) {
    lyap_set_error_message("no stored inverse sequence for this problem", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  if (mr == 0) {
    *r_out = 0;
    if (iters) *iters = C.store_count;
    return LYAP_OK;
  }
  // Z_0 = L rounded to u_s (working precision)
  {
    LYAP_TRY(ensure(C.Lst, (size_t)n * mr * 8 + 64));
    double* tmp = P<double>(C.Lst);
    LYAP_TRY((copy_cast<double, double>(Lr, n, mr, n, tmp, n, 1.0, C.s)));
    LYAP_TRY(round_to_prec(tmp, n, mr, n, o.u_s, P<double>(C.part) + 4 * RED_BLOCKS, C.s));
    LYAP_TRY((copy_cast<double, T>(tmp, n, mr, n, P<T>(C.Zw), n, 1.0, C.s)));
    if (ldlt) {
      if (yr) {
        LYAP_CUDA_TRY(cudaMemcpyAsync(C.yv.p, yr, sizeof(double) * mr, cudaMemcpyDeviceToDevice, C.s));
      } else {
        std::vector<double> ones(mr, 1.0);
        LYAP_CUDA_TRY(cudaMemcpyAsync(C.yv.p, ones.data(), sizeof(double) * mr, cudaMemcpyHostToDevice, C.s));
        LYAP_CUDA_TRY(cudaStreamSynchronize(C.s));
      }
    }
  }
  int c = 0;
  // ADI and EKSM iterates approximate X itself (no final factor of the Newton form)
  const bool adi = (o.inner != LYAP_INNER_SIGN);
  const double itol = o.adi_tol > 0 ? o.adi_tol : std::max(10.0 * unit_roundoff(o.u_s), 1e-14);
  if (o.inner == LYAP_INNER_ADI) {
    AdiOpts ao;
    ao.shifts = o.adi_shifts > 0 ? o.adi_shifts : 8;
    ao.maxit = o.adi_maxit > 0 ? o.adi_maxit : 200;
    ao.tol = itol;
    LYAP_TRY(adi_run<T>(C, n, mr, ldlt, no, ao, compute, &c, info));
  } else if (o.inner == LYAP_INNER_EKSM) {
    LYAP_TRY(eksm_run<T>(C, n, mr, ldlt, no, o.eksm_maxit > 0 ? o.eksm_maxit : 60, itol, compute, &c));
  } else {
    LYAP_TRY(newton_run<T>(C, n, mr, ldlt, no, compute, &c, info));
  }
  if (iters) *iters = C.store_count;
  if (c > zcap_out) {
    *r_out = c;
    lyap_set_error_message("factor capacity too small", __FILE__, __LINE__);
    return LYAP_ERR_CAPACITY;
  }
  // undo the prescaling: X = 2^-e0 X'  ->  Z = 2^{-e0/2} Z' (Cholesky, with the final 1/sqrt 2),
  // Y = 2^-e0 Y'/2 (LDL^T)
  // (ADI and EKSM factors carry no final 1/sqrt 2 / 1/2: their iterates approximate X itself)
  const double e0 = (double)C.store_e0;
  if (!ldlt) {
    LYAP_TRY((copy_cast<T, double>(P<T>(C.Zw), n, c, n, Zout, ldo, pow(2.0, -0.5 * e0) / (adi ? 1.0 : sqrt(2.0)),
                                   C.s)));
  } else {
    LYAP_TRY((copy_cast<T, double>(P<T>(C.Zw), n, c, n, Zout, ldo, 1.0, C.s)));
    LYAP_CUDA_TRY(cudaMemcpyAsync(yout, C.yv.p, sizeof(double) * c, cudaMemcpyDeviceToDevice, C.s));
    scale_vec_kernel<<<1, 256, 0, C.s>>>(yout, c, (adi ? 1.0 : 0.5) * pow(2.0, -e0));
    lyap_count_launch();
  }
  *r_out = c;
  return LYAP_OK;
}

static int newton_solve_any(Ctx& C, const Problem& pb, const double* Lr, int mr, const double* yr, bool ldlt,
                            const lyap_opts_t& o, bool compute, double* Zout, int64_t ldo, int zcap_out,
                            double* yout, int* r_out, lyap_info_t* info, int* iters) {
  if (o.u_s == LYAP_FP64)
    return newton_solve<double>(C, pb, Lr, mr, yr, ldlt, o, compute, Zout, ldo, zcap_out, yout, r_out, info, iters);
  return newton_solve<float>(C, pb, Lr, mr, yr, ldlt, o, compute, Zout, ldo, zcap_out, yout, r_out, info, iters);
}

// ---------------------------------------------------------------------------
// residual factorisation (FP64): Fragment ResFacChol / ResFacLdlt
// Returns the normalised residual (device scal[40]) and, if want_split, the
// truncated factors: Cholesky: L+ (n x r+) in C.Lp, L- (n x r-) in C.Lm;
// LDL^T: L^Delta in C.Lp with values in C.ytmp (r+ = count, r- = 0).
// ---------------------------------------------------------------------------
struct ResOut {
  double res, resF;
  int rp, rm;
};

// y == NULL: X = Z Z^T; sd == NULL: W = L L^T.  ldlt selects the split of Fragment ResFacLdlt.
static int res_fac(Ctx& C, const Problem& pb, const double* Lw, const double* sd, const double* Z, int c,
                   const double* y, bool ldlt, double eta_r, bool want_split, ResOut* out) {
  const int n = pb.n, m = pb.m;
  const int q = 2 * c + m;
  mark(C, LYAP_PHASE_RESFAC);
  LYAP_TRY(ensure(C.F, (size_t)n * q * 8 + 64));
  LYAP_TRY(ensure(C.tau, (size_t)(q + 8) * 8));
  double* F = P<double>(C.F);
  // F = [Z, A Z, L]
  LYAP_TRY((copy_cast<double, double>(Z, n, c, n, F, n, 1.0, C.s)));
  LYAP_TRY(gemm<double>('N', 'N', n, c, n, 1.0, pb.A, pb.lda, Z, n, 0.0, F + (size_t)c * n, n, C.s));
  LYAP_TRY((copy_cast<double, double>(Lw, n, m, n, F + (size_t)2 * c * n, n, 1.0, C.s)));
  LYAP_CUDA_TRY(cudaMemsetAsync(C.qr.status, 0, sizeof(int), C.s));
  LYAP_TRY(householder_qr<double>(F, n, q, n, P<double>(C.tau), C.qr, C.s));
  const int kr = std::min(n, q);
  LYAP_TRY(ensure(C.Tm, (size_t)kr * q * 8 + 64));
  LYAP_TRY(ensure(C.TP, (size_t)kr * q * 8 + 64));
  LYAP_TRY(ensure(C.H, (size_t)kr * kr * 8 + 64));
  extract_r_kernel<<<nblk((int64_t)kr * q), 256, 0, C.s>>>(F, n, kr, q, P<double>(C.Tm));
  core_right_kernel<<<nblk((int64_t)kr * q), 256, 0, C.s>>>(P<double>(C.Tm), kr, c, m, y, sd, P<double>(C.TP));
  lyap_count_launch(2);
  LYAP_TRY(gemm<double>('N', 'T', kr, kr, q, 1.0, P<double>(C.TP), kr, P<double>(C.Tm), kr, 0.0, P<double>(C.H), kr,
                        C.s));
  double* sc = P<double>(C.scal);
  // sc[20] = ||H||_F^2 ; sc[21] = ||X||_F^2 ; sc[22] = ||W||_F ; sc[23] = ||A||_F^2 ; sc[24..25] = res
  LYAP_TRY(sumsq<double>(P<double>(C.H), kr, kr, kr, sc + 20, P<double>(C.part), C.s));
  LYAP_TRY(ensure(C.gram, (size_t)std::max(c, m) * std::max(c, m) * 8 + 64));
  LYAP_TRY(gemm<double>('T', 'N', c, c, n, 1.0, Z, n, Z, n, 0.0, P<double>(C.gram), c, C.s));
  gram_norm_kernel<<<1, 256, 0, C.s>>>(P<double>(C.gram), c, y, sc + 21);
  lyap_count_launch();
  resid_kernel<<<1, 1, 0, C.s>>>(sc + 20, sc + 22, sc + 23, sc + 21, sc + 24);
  lyap_count_launch();
  double hres[2];
  LYAP_TRY(sync_read(C, sc + 24, hres, sizeof(hres)));
  int qs = 0;
  LYAP_TRY(sync_read(C, C.qr.status, &qs, sizeof(int)));
  if (qs) return qs;
  out->res = hres[0];
  out->resF = hres[1];
  out->rp = out->rm = 0;
  if (!want_split) return LYAP_OK;
  // eigen-split of H (FP32 accuracy suffices: the split is truncated at eta_r >> u_fp32).
  // Cores above the eigensolver's order limit: the range of H is first found by QR with
  // column pivoting truncated at eta_r / 10 (everything dropped lies far below the
  // truncation level of the split), and the eigenpairs come from the Rayleigh-Ritz matrix
  // on that range.  Below it the direct FP32 eigensolver is cheaper: the range found is
  // typically most of H (805 of 950 at n = 1024) and costs two QRs and three products.
  LYAP_TRY(ensure(C.w, (size_t)kr * 8 + 64));
  LYAP_TRY(ensure(C.Qh, (size_t)kr * kr * 8 + 64));
  LYAP_TRY(ensure(C.Csel, (size_t)kr * kr * 8 + 64));
  int neig = kr;
  if (kr > EIG_MAX_Q) {
    // the range is found in FP32 (the split needs FP32 accuracy at most, and the FP32 copy
    // fits the cluster-resident QRCP); the Rayleigh-Ritz step below uses the FP64 H
    double* Zr = P<double>(C.Csel);
    LYAP_TRY(ensure(C.Hf, (size_t)kr * kr * 4 + 64));
    float* Hf = P<float>(C.Hf);
    LYAP_TRY((copy_cast<double, float>(P<double>(C.H), kr, kr, kr, Hf, kr, 1.0, C.s)));
    LYAP_TRY(qrcp_truncate<float>(Hf, kr, kr, kr, 0.1 * eta_r, C.qr, C.s));
    int r = 0;
    LYAP_TRY(sync_read(C, C.qr.rank, &r, sizeof(int)));
    r = std::max(r, 1);
    LYAP_TRY((copy_cast<float, double>(Hf, kr, r, kr, Zr, kr, 1.0, C.s)));
    LYAP_TRY(ensure(C.Rtau, (size_t)(r + 8) * 8));
    LYAP_TRY(ensure(C.Bm, (size_t)r * r * 8 + 64));
    LYAP_TRY(ensure(C.VB, (size_t)r * r * 8 + 64));
    LYAP_TRY(householder_qr<double>(Zr, kr, r, kr, P<double>(C.Rtau), C.qr, C.s));
    LYAP_TRY(set_identity<double>(P<double>(C.Bm), r, r, C.s));
    double* Qb = P<double>(C.TP);
    LYAP_TRY(apply_q<double>(Zr, kr, r, kr, P<double>(C.Rtau), P<double>(C.Bm), r, r, Qb, kr, C.s));
    double* HQ = P<double>(C.Tm);
    LYAP_TRY(gemm<double>('N', 'N', kr, r, kr, 1.0, P<double>(C.H), kr, Qb, kr, 0.0, HQ, kr, C.s));
    LYAP_TRY(gemm<double>('T', 'N', r, r, kr, 1.0, Qb, kr, HQ, kr, 0.0, P<double>(C.Bm), r, C.s));
    LYAP_TRY(prepare_eig(C, r));
    mark(C, LYAP_PHASE_EIG);
    LYAP_TRY(sym_eig(P<double>(C.Bm), r, r, P<double>(C.w), P<double>(C.VB), r, 0, C.eig, C.s));
    mark(C, LYAP_PHASE_RESFAC);
    LYAP_TRY(gemm<double>('N', 'N', kr, r, r, 1.0, Qb, kr, P<double>(C.VB), r, 0.0, P<double>(C.Qh), kr, C.s));
    neig = r;
  } else {
    LYAP_TRY(prepare_eig(C, kr));
    mark(C, LYAP_PHASE_EIG);
    LYAP_TRY(sym_eig(P<double>(C.H), kr, kr, P<double>(C.w), P<double>(C.Qh), kr, 0, C.eig, C.s));
    mark(C, LYAP_PHASE_RESFAC);
  }
  int* sel = P<int>(C.scal) + 64;
  select_kernel<<<1, 32, 0, C.s>>>(P<double>(C.w), neig, eta_r, 0, sel, sc + 30);
  lyap_count_launch();
  int hs[2];
  LYAP_TRY(sync_read(C, sel, hs, sizeof(hs)));
  const int nneg = hs[0], pos = hs[1];
  const int npos = neig - pos;
  double* Cs = P<double>(C.Csel);
  if (!ldlt) {
    LYAP_TRY(ensure(C.Lp, (size_t)n * std::max(npos, 1) * 8 + 64));
    LYAP_TRY(ensure(C.Lm, (size_t)n * std::max(nneg, 1) * 8 + 64));
    if (npos > 0) {
      gather_cols_kernel<<<nblk((int64_t)kr * npos), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), pos, npos,
                                                                     1, Cs, kr, nullptr);
      lyap_count_launch();
      LYAP_TRY(apply_q<double>(F, n, kr, n, P<double>(C.tau), Cs, kr, npos, P<double>(C.Lp), n, C.s));
    }
    if (nneg > 0) {
      gather_cols_kernel<<<nblk((int64_t)kr * nneg), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), 0, nneg,
                                                                     1, Cs, kr, nullptr);
      lyap_count_launch();
      LYAP_TRY(apply_q<double>(F, n, kr, n, P<double>(C.tau), Cs, kr, nneg, P<double>(C.Lm), n, C.s));
    }
    out->rp = npos;
    out->rm = nneg;
  } else {
    const int r = nneg + npos;
    LYAP_TRY(ensure(C.Lp, (size_t)n * std::max(r, 1) * 8 + 64));
    LYAP_TRY(ensure(C.Lm, (size_t)(r + 8) * 8));
    double* yd = P<double>(C.Lm);
    if (nneg > 0) {
      gather_cols_kernel<<<nblk((int64_t)kr * nneg), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), 0, nneg,
                                                                     0, Cs, kr, yd);
      lyap_count_launch();
    }
    if (npos > 0) {
      gather_cols_kernel<<<nblk((int64_t)kr * npos), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), pos, npos,
                                                                     0, Cs + (size_t)nneg * kr, kr, yd + nneg);
      lyap_count_launch();
    }
    if (r > 0) LYAP_TRY(apply_q<double>(F, n, kr, n, P<double>(C.tau), Cs, kr, r, P<double>(C.Lp), n, C.s));
    out->rp = r;
    out->rm = 0;
  }
  LYAP_CUDA_TRY(cudaGetLastError());
  return LYAP_OK;
}

// ---------------------------------------------------------------------------
// projected solution update (FP64): Fragment SolUptChol / SolUptLdlt.
// G = [Z, Z+, Z-] (Cholesky) or [Z, Z^Delta] with weights ups (LDL^T), in C.G.
// ---------------------------------------------------------------------------
static int sol_upt(Ctx& C, int n, int qg, int cneg_start, const double* ups, bool psd_keep_positive,
                   double eta_s, double res_next, double* Zout, double* yout, int* r_out) {
  double* G = P<double>(C.G);
  mark(C, LYAP_PHASE_SOLUPT);
  LYAP_TRY(ensure(C.tau, (size_t)(qg + 8) * 8));
  LYAP_CUDA_TRY(cudaMemsetAsync(C.qr.status, 0, sizeof(int), C.s));
  LYAP_TRY(householder_qr<double>(G, n, qg, n, P<double>(C.tau), C.qr, C.s));
  const int kr = std::min(n, qg);
  LYAP_TRY(ensure(C.Tm, (size_t)kr * qg * 8 + 64));
  LYAP_TRY(ensure(C.TP, (size_t)kr * qg * 8 + 64));
  LYAP_TRY(ensure(C.H, (size_t)kr * kr * 8 + 64));
  LYAP_TRY(ensure(C.w, (size_t)kr * 8 + 64));
  LYAP_TRY(ensure(C.Qh, (size_t)kr * kr * 8 + 64));
  LYAP_TRY(ensure(C.Csel, (size_t)kr * kr * 8 + 64));
  extract_r_kernel<<<nblk((int64_t)kr * qg), 256, 0, C.s>>>(G, n, kr, qg, P<double>(C.Tm));
  scale_cols_dev_kernel<<<nblk((int64_t)kr * qg), 256, 0, C.s>>>(P<double>(C.Tm), kr, qg, cneg_start, ups,
                                                                P<double>(C.TP));
  lyap_count_launch(2);
  LYAP_TRY(gemm<double>('N', 'T', kr, kr, qg, 1.0, P<double>(C.TP), kr, P<double>(C.Tm), kr, 0.0, P<double>(C.H), kr,
                        C.s));
  LYAP_TRY(prepare_eig(C, kr));
  mark(C, LYAP_PHASE_EIG);
  // the eigendecomposition of K defines X_{i+1}: its error enters the next residual, so the
  // fast refinement runs until its coupling is below 1/100 of the residual this step is
  // expected to reach (res_next), and at most to FP64 level
  C.eig.target = std::max(1e-15, 1e-2 * res_next);
  const int est = sym_eig(P<double>(C.H), kr, kr, P<double>(C.w), P<double>(C.Qh), kr, 2, C.eig, C.s);
  C.eig.target = 0.0;
  LYAP_TRY(est);
  mark(C, LYAP_PHASE_SOLUPT);
  int* sel = P<int>(C.scal) + 64;
  select_kernel<<<1, 32, 0, C.s>>>(P<double>(C.w), kr, eta_s, 0, sel, P<double>(C.scal) + 31);
  lyap_count_launch();
  int hs[2];
  LYAP_TRY(sync_read(C, sel, hs, sizeof(hs)));
  int qs = 0;
  LYAP_TRY(sync_read(C, C.qr.status, &qs, sizeof(int)));
  if (qs) return qs;
  const int nneg = hs[0], pos = hs[1];
  const int npos = kr - pos;
  double* Cs = P<double>(C.Csel);
  int r = 0;
  if (psd_keep_positive) {
    if (npos > 0) {
      gather_cols_kernel<<<nblk((int64_t)kr * npos), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), pos, npos,
                                                                     yout ? 0 : 1, Cs, kr, yout);
      lyap_count_launch();
    }
    r = npos;
  } else {
    if (nneg > 0) {
      gather_cols_kernel<<<nblk((int64_t)kr * nneg), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), 0, nneg,
                                                                     0, Cs, kr, yout);
      lyap_count_launch();
    }
    if (npos > 0) {
      gather_cols_kernel<<<nblk((int64_t)kr * npos), 256, 0, C.s>>>(P<double>(C.Qh), kr, kr, P<double>(C.w), pos, npos,
                                                                     0, Cs + (size_t)nneg * kr, kr,
                                                                     yout ? yout + nneg : nullptr);
      lyap_count_launch();
    }
    r = nneg + npos;
  }
  if (r > 0) LYAP_TRY(apply_q<double>(G, n, kr, n, P<double>(C.tau), Cs, kr, r, Zout, n, C.s));
  LYAP_CUDA_TRY(cudaGetLastError());
  *r_out = r;
  return LYAP_OK;
}

static int check_problem(const Problem& pb, const lyap_opts_t* o, double* Z, int64_t ldz, int64_t z_cap) {
  if (!pb.A || !pb.L || !o || !Z) return LYAP_ERR_ARG;
  if (pb.n <= 0 || pb.m <= 0 || pb.lda < pb.n || pb.ldl < pb.n || ldz < pb.n || z_cap <= 0) return LYAP_ERR_ARG;
  if (pb.S && pb.lds < pb.m) return LYAP_ERR_ARG;
  if (o->u_s < 0 || o->u_s > 3 || o->scaling < 0 || o->scaling > 4 || o->kmax <= 0 || o->imax < 0) return LYAP_ERR_ARG;
  if (o->inner != LYAP_INNER_SIGN && o->inner != LYAP_INNER_ADI && o->inner != LYAP_INNER_EKSM) return LYAP_ERR_ARG;
  if (o->u != o->u_r || o->u != o->u_c || (o->u != LYAP_FP64 && o->u != LYAP_FP32)) {
    lyap_set_error_message("u = u_r = u_c must be LYAP_FP64 or LYAP_FP32", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  return LYAP_OK;
}

static int check_inputs_finite(Ctx& C, const Problem& pb) {
  int* flag = P<int>(C.scal) + 300;
  LYAP_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), C.s));
  LYAP_TRY(check_finite(pb.A, pb.n, pb.n, pb.lda, flag, C.s));
  LYAP_TRY(check_finite(pb.L, pb.n, pb.m, pb.ldl, flag, C.s));
  if (pb.S) LYAP_TRY(check_finite(pb.S, pb.m, pb.m, pb.lds, flag, C.s));
  int f = 0;
  LYAP_TRY(sync_read(C, flag, &f, sizeof(int)));
  return f ? LYAP_ERR_NONFINITE : LYAP_OK;
}

static int solve_common(Ctx& C, const Problem& pb, const lyap_opts_t& o, bool refine, double* Z, int64_t ldz,
                        int64_t z_cap, double* D, int64_t* rank_out, lyap_info_t* info, bool replay_first = false) {
  const int n = pb.n, m = pb.m;
  const bool ldlt = (pb.S != nullptr);
  LYAP_TRY(ensure(C.scal, 4096));
  LYAP_TRY(ensure(C.part, (size_t)6 * RED_BLOCKS * 8));
  LYAP_TRY(check_inputs_finite(C, pb));
  double* Lw = nullptr;
  double* sd = nullptr;
  bool indefinite = false;
  LYAP_TRY(prepare_rhs(C, pb, &Lw, &sd, &indefinite));
  const int zcap_ir = n + 8;
  LYAP_TRY(ensure(C.Zs, (size_t)n * (zcap_ir) * 8));
  LYAP_TRY(ensure(C.Zbest, (size_t)n * (zcap_ir) * 8));
  LYAP_TRY(ensure(C.ysol, (size_t)(zcap_ir) * 8));
  LYAP_TRY(ensure(C.ybest, (size_t)(zcap_ir) * 8));
  // first solve (computes and stores the inverse sequence, or replays a stored one)
  int c = 0, iters = 0;
  LYAP_TRY(newton_solve_any(C, pb, Lw, m, sd, ldlt, o, !replay_first, P<double>(C.Zs), n, zcap_ir,
                            P<double>(C.ysol), &c, info, &iters));
  info->newton_calls = 1;
  info->newton_total = iters;
  info->newton_max = iters;
  info->n_inversions = replay_first ? 0 : iters;
  // normalisation constants
  double* sc = P<double>(C.scal);
  {
    // ||W||_F from the Gram matrix of L (with the diagonal S), ||A||_F^2
    LYAP_TRY(ensure(C.gram, (size_t)m * m * 8 + 64));
    LYAP_TRY(gemm<double>('T', 'N', m, m, n, 1.0, Lw, n, Lw, n, 0.0, P<double>(C.gram), m, C.s));
    gram_norm_kernel<<<1, 256, 0, C.s>>>(P<double>(C.gram), m, sd, sc + 26);
    lyap_count_launch();
    LYAP_TRY(sumsq<double>(pb.A, n, n, pb.lda, sc + 23, P<double>(C.part), C.s));
    double h[1];
    LYAP_TRY(sync_read(C, sc + 26, h, sizeof(double)));
    h[0] = sqrt(h[0]);
    LYAP_CUDA_TRY(cudaMemcpyAsync(sc + 22, h, sizeof(double), cudaMemcpyHostToDevice, C.s));
    LYAP_CUDA_TRY(cudaStreamSynchronize(C.s));
  }
  // working precision u = u_r = u_c (Table 2.1): the residual factors and the updated solution
  // factor are stored in it (rounded when it is FP32; the products themselves run in FP64)
  const int wu = o.u;
  double* rscr = P<double>(C.part) + 4 * RED_BLOCKS;
  auto to_u = [&](double* x, int64_t rows, int64_t cols) { return round_to_prec(x, rows, cols, rows, wu, rscr, C.s); };
  LYAP_TRY(to_u(P<double>(C.Zs), n, c));
  if (ldlt) LYAP_TRY(to_u(P<double>(C.ysol), c, 1));
  const double tau_ir = o.tau_ir > 0 ? o.tau_ir : (double)n * unit_roundoff(wu);
  const double eta_s = o.eta_s > 0 ? o.eta_s : 10.0 * unit_roundoff(wu);
  const bool project = (o.project_psd != 0) && !indefinite;
  double best = 1e300;
  int best_c = 0;
  int stag = 0;
  double res_prev = -1.0;
  int status = LYAP_OK;
  info->n_res = 0;
  const int imax = refine ? o.imax : 0;
  for (int i = 1; i <= imax + 1; ++i) {
    ResOut ro;
    const bool last = (i == imax + 1);
    // (the eigen-split of R stays at the FP32 Jacobi's default accuracy, 1e-6: a split as
    // loose as the next step's contraction, 1e-2 for FP16, was measured to raise the ranks of
    // the corrections -- 411 -> 483 at n = 1024 -- and with them the cost of every step)
    LYAP_TRY(res_fac(C, pb, Lw, sd, P<double>(C.Zs), c, ldlt ? P<double>(C.ysol) : nullptr, ldlt, o.eta_r, !last, &ro));
    if (info->n_res < 64) info->res_hist[info->n_res++] = ro.res;
    if (ro.res < best) {
      best = ro.res;
      best_c = c;
      LYAP_CUDA_TRY(cudaMemcpyAsync(C.Zbest.p, C.Zs.p, sizeof(double) * (size_t)n * c, cudaMemcpyDeviceToDevice, C.s));
      if (ldlt) LYAP_CUDA_TRY(cudaMemcpyAsync(C.ybest.p, C.ysol.p, sizeof(double) * c, cudaMemcpyDeviceToDevice, C.s));
    }
    if (ro.res <= tau_ir) {
      info->converged = 1;
      break;
    }
    if (!refine) break;
    if (res_prev > 0 && ro.res / res_prev > o.stag_theta) ++stag;
    else stag = 0;
    // the residual this step is expected to reach: the last observed contraction (first step:
    // a guess from u_s -- roughly the contraction of the inner solves at moderate kappa)
    double contraction = (o.u_s == LYAP_FP64) ? 1e-8 : (o.u_s == LYAP_FP32) ? 1e-5 : (o.u_s == LYAP_FP16) ? 1e-2 : 1e-1;
    if (res_prev > 0) contraction = std::min(1.0, std::max(1e-8, ro.res / res_prev));
    const double res_next = ro.res * contraction;
    res_prev = ro.res;
    if (stag >= o.stag_count) {
      info->stagnated = 1;
      status = LYAP_WARN_STAGNATED;
      break;
    }
    if (last) {
      status = LYAP_WARN_MAXIT;
      break;
    }
    // correction solves replay the stored inverse sequence (Sec. 3.4)
    const int rp = ro.rp, rm = ro.rm;
    const int qg = c + rp + rm;
    LYAP_TRY(ensure(C.G, (size_t)n * (qg + 4 * n + 16) * 8));
    double* G = P<double>(C.G);
    LYAP_TRY((copy_cast<double, double>(P<double>(C.Zs), n, c, n, G, n, 1.0, C.s)));
    int cp = 0, cm = 0, it2 = 0;
    if (!ldlt) {
      // copy L+, L- aside (the Newton solve reuses scratch buffers)
      LYAP_TRY(ensure(C.Vs, (size_t)n * (rp + rm + 1) * 8 + 64));
      double* Lpm = P<double>(C.Vs);
      LYAP_TRY((copy_cast<double, double>(P<double>(C.Lp), n, rp, n, Lpm, n, 1.0, C.s)));
      LYAP_TRY((copy_cast<double, double>(P<double>(C.Lm), n, rm, n, Lpm + (size_t)n * rp, n, 1.0, C.s)));
      LYAP_TRY(to_u(Lpm, n, rp + rm));
      LYAP_TRY(newton_solve_any(C, pb, Lpm, rp, nullptr, false, o, false, G + (size_t)n * c, n, 2 * n, nullptr, &cp,
                                nullptr, &it2));
      LYAP_TRY(newton_solve_any(C, pb, Lpm + (size_t)n * rp, rm, nullptr, false, o, false, G + (size_t)n * (c + cp), n,
                                2 * n, nullptr, &cm, nullptr, &it2));
      info->newton_calls += 1;
      info->newton_total += C.store_count;
      int rnew = 0;
      LYAP_TRY(sol_upt(C, n, c + cp + cm, c + cp, nullptr, true, eta_s, res_next, P<double>(C.Zs), nullptr, &rnew));
      c = rnew;
      LYAP_TRY(to_u(P<double>(C.Zs), n, c));
    } else {
      LYAP_TRY(ensure(C.Vs, (size_t)n * (rp + 1) * 8 + 64));
      double* Ld = P<double>(C.Vs);
      LYAP_TRY((copy_cast<double, double>(P<double>(C.Lp), n, rp, n, Ld, n, 1.0, C.s)));
      LYAP_TRY(ensure(C.ytmp, (size_t)(2 * n + rp + 16) * 8 * 2 + (size_t)n * rp * 8));
      // values of S^Delta rounded to u_s
      double* ups = P<double>(C.ytmp);
      LYAP_CUDA_TRY(cudaMemcpyAsync(ups, C.ysol.p, sizeof(double) * c, cudaMemcpyDeviceToDevice, C.s));
      double* sdel = ups + c + 2 * n + 8;
      LYAP_CUDA_TRY(cudaMemcpyAsync(sdel, C.Lm.p, sizeof(double) * rp, cudaMemcpyDeviceToDevice, C.s));
      LYAP_TRY(to_u(Ld, n, rp));
      LYAP_TRY(to_u(sdel, rp, 1));
      LYAP_TRY(round_to_prec(sdel, rp, 1, rp, o.u_s, P<double>(C.part) + 4 * RED_BLOCKS, C.s));
      LYAP_TRY(newton_solve_any(C, pb, Ld, rp, sdel, true, o, false, G + (size_t)n * c, n, 2 * n, ups + c, &cp, nullptr,
                                &it2));
      info->newton_calls += 1;
      info->newton_total += C.store_count;
      int rnew = 0;
      LYAP_TRY(sol_upt(C, n, c + cp, c + cp, ups, project, eta_s, res_next, P<double>(C.Zs), P<double>(C.ysol), &rnew));
      c = rnew;
      LYAP_TRY(to_u(P<double>(C.Zs), n, c));
      LYAP_TRY(to_u(P<double>(C.ysol), c, 1));
    }
    info->ir_steps = i;
    if (c > n) c = n;
  }
  // return the best factor
  if (best_c > z_cap) {
    *rank_out = best_c;
    lyap_set_error_message("output capacity too small", __FILE__, __LINE__);
    return LYAP_ERR_CAPACITY;
  }
  LYAP_TRY((copy_cast<double, double>(P<double>(C.Zbest), n, best_c, n, Z, ldz, 1.0, C.s)));
  if (ldlt && D) LYAP_CUDA_TRY(cudaMemcpyAsync(D, C.ybest.p, sizeof(double) * best_c, cudaMemcpyDeviceToDevice, C.s));
  LYAP_CUDA_TRY(cudaStreamSynchronize(C.s));
  *rank_out = best_c;
  info->rank = best_c;
  info->res_final = best;
  info->n_inversions += (int)C.recomputed;
  C.recomputed = 0;
  return status;
}

static int solve_entry(lyap_ctx_t* C, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl, int64_t m,
                       const double* S, int64_t lds, const lyap_opts_t* opts, double* Z, int64_t ldz, int64_t z_cap,
                       double* D, int64_t* rank_out, lyap_info_t* info, bool refine) {
  if (!C || !rank_out) return LYAP_ERR_ARG;
  Problem pb{A, (int)n, lda, L, ldl, (int)m, S, lds};
  LYAP_TRY(check_problem(pb, opts, Z, ldz, z_cap));
  if (S && !D) return LYAP_ERR_ARG;
  lyap_info_t local;
  lyap_info_t* inf = info ? info : &local;
  memset(inf, 0, sizeof(*inf));
  const int64_t l0 = g_launches;
  C->profile = opts->profile != 0;
  C->marks_used = 0;
  C->recomputed = 0;
  for (double& f : C->flops) f = 0.0;
  const int dgemm_prev = dgemm_method();
  set_dgemm_method(opts->fp64_products);
  cudaEventRecord(C->e0, C->s);
  mark(*C, LYAP_PHASE_OTHER);
  int st = solve_common(*C, pb, *opts, refine, Z, ldz, z_cap, D, rank_out, inf);
  set_dgemm_method(dgemm_prev);
  if (st >= 0) {
    int tcs = 0;  // a bounded wait of a tensor-core product that gave up
    if (tc_status_read(&tcs) == LYAP_OK && tcs) st = tcs;
  }
  collect_marks(*C, inf);
  C->profile = false;
  cudaEventRecord(C->e1, C->s);
  cudaEventSynchronize(C->e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, C->e0, C->e1);
  inf->device_ms = ms;
  inf->kernel_launches = g_launches - l0;
  inf->status = st;
  return st;
}


// Adjoint of the last solve (not in the paper): Y = Z_Y Z_Y^T solves A^T Y + Y A + C^T C = 0
// by the same refinement, its Newton solves replaying the stored A_k^{-1} transposed (the
// sign-Newton sequence of A^T is the transposed sequence of A with the same mu_k, since
// the Frobenius norm and determinant are transpose-invariant); then
// dl/dA = 2 Y X, dl/dL = 2 Y L S, dl/dS = L^T Y L for X = Z D Z^T.
static int adjoint_entry(lyap_ctx_t* Cp, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl,
                         int64_t m, const double* S, int64_t lds, const double* Z, int64_t ldz, int64_t r,
                         const double* D, const double* Cm, int64_t ldc, int64_t q, const lyap_opts_t* opts,
                         double* dA, int64_t ldda, double* dL, int64_t lddl, double* dS, int64_t ldds, double* Zy,
                         int64_t ldzy, int64_t zy_cap, int64_t* rank_y, lyap_info_t* info) {
  if (!Cp || !A || !L || !Z || !Cm || !opts || n <= 0 || m <= 0 || r < 0 || q <= 0) return LYAP_ERR_ARG;
  if (opts->u != LYAP_FP64 || opts->u_r != LYAP_FP64 || opts->u_c != LYAP_FP64) return LYAP_ERR_ARG;
  if (lda < n || ldl < n || ldz < n || ldc < q || (S && lds < m)) return LYAP_ERR_ARG;
  if ((dA && ldda < n) || (dL && lddl < n) || (dS && ldds < m) || (Zy && (ldzy < n || !rank_y))) return LYAP_ERR_ARG;
  Ctx& C = *Cp;
  const int ni = (int)n, mi = (int)m, qi = (int)q, ri = (int)r;
  lyap_info_t local;
  lyap_info_t* inf = info ? info : &local;
  memset(inf, 0, sizeof(*inf));
  const int64_t l0 = g_launches;
  C.profile = opts->profile != 0;
  C.marks_used = 0;
  C.recomputed = 0;
  for (double& f : C.flops) f = 0.0;
  const int dgemm_prev = dgemm_method();
  set_dgemm_method(opts->fp64_products);
  cudaEventRecord(C.e0, C.s);
  mark(C, LYAP_PHASE_OTHER);
  int st = LYAP_OK;
  bool transposed = false;
  do {
    LYAP_TRY(ensure(C.scal, 4096));
    LYAP_TRY(ensure(C.part, (size_t)6 * RED_BLOCKS * 8));
    LYAP_TRY(ensure(C.At, (size_t)n * n * 8));
    LYAP_TRY(ensure(C.Ct, (size_t)n * q * 8));
    const int64_t cap = n + 8;
    LYAP_TRY(ensure(C.ZY, (size_t)n * cap * 8));
    dim3 blk(32, 8);
    transpose64_kernel<<<dim3((unsigned)ceil_div(n, 32), (unsigned)ceil_div(n, 32)), blk, 0, C.s>>>(A, ni, ni, lda,
                                                                                                  P<double>(C.At));
    transpose64_kernel<<<dim3((unsigned)ceil_div(n, 32), (unsigned)ceil_div(q, 32)), blk, 0, C.s>>>(Cm, qi, ni, ldc,
                                                                                                  P<double>(C.Ct));
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch(2);
    // C = 0: Y = 0 and every gradient vanishes
    {
      double cc = 0.0;
      LYAP_TRY(sumsq<double>(P<double>(C.Ct), n, q, n, P<double>(C.scal) + 312, P<double>(C.part), C.s));
      LYAP_TRY(sync_read(C, P<double>(C.scal) + 312, &cc, sizeof(double)));
      if (cc == 0.0) {
        if (dL) LYAP_TRY(set_zero<double>(dL, n, m, lddl, C.s));
        if (dS) LYAP_TRY(set_zero<double>(dS, m, m, ldds, C.s));
        if (dA) LYAP_TRY(set_zero<double>(dA, n, n, ldda, C.s));
        if (rank_y) *rank_y = 0;
        inf->converged = 1;
        break;
      }
    }
    // replay the forward inverse sequence if it belongs to this A, else build one for A^T
    double fp = 0.0;
    LYAP_TRY(fingerprint(C, A, ni, lda, &fp));
    const bool replay = C.store_count > 0 && C.store_n == ni && C.store_prec == opts->u_s && fp == C.store_fp;
    if (replay) {
      LYAP_TRY(transpose_store(C));
      transposed = true;
    }
    Problem pbY{P<double>(C.At), ni, n, P<double>(C.Ct), n, qi, nullptr, 0};
    int64_t ry = 0;
    st = solve_common(C, pbY, *opts, true, P<double>(C.ZY), n, cap, nullptr, &ry, inf, replay);
    if (st < 0) break;
    if (transposed) {
      LYAP_TRY(transpose_store(C));
      transposed = false;
    }
    if (rank_y) *rank_y = ry;
    if (Zy) {
      if (ry > zy_cap) {
        lyap_set_error_message("adjoint factor capacity too small", __FILE__, __LINE__);
        st = LYAP_ERR_CAPACITY;
        break;
      }
      LYAP_TRY((copy_cast<double, double>(P<double>(C.ZY), n, ry, n, Zy, ldzy, 1.0, C.s)));
    }
    // gradient products (FP64)
    const int ryi = (int)ry;
    LYAP_TRY(ensure(C.adjT, (size_t)(std::max(ryi, 1) * (mi + ri) + n * (mi + ri) + 64) * 8));
    double* T1 = P<double>(C.adjT);                               // Z_Y^T L      (ry x m)
    double* T2 = T1 + (size_t)std::max(ryi, 1) * mi;              // Z_Y T1       (n x m)
    double* T3 = T2 + (size_t)n * mi;                             // Z_Y^T Z      (ry x r)
    double* T4 = T3 + (size_t)std::max(ryi, 1) * std::max(ri, 1); // Z_Y T3 D     (n x r)
    const double* Yf = P<double>(C.ZY);
    if (ryi == 0) {
      if (dL) LYAP_TRY(set_zero<double>(dL, n, m, lddl, C.s));
      if (dS) LYAP_TRY(set_zero<double>(dS, m, m, ldds, C.s));
      if (dA) LYAP_TRY(set_zero<double>(dA, n, n, ldda, C.s));
      break;
    }
    LYAP_TRY(gemm<double>('T', 'N', ryi, mi, ni, 1.0, Yf, n, L, ldl, 0.0, T1, ryi, C.s));
    if (dL) {
      if (S) {
        LYAP_TRY(gemm<double>('N', 'N', ni, mi, ryi, 1.0, Yf, n, T1, ryi, 0.0, T2, n, C.s));
        LYAP_TRY(gemm<double>('N', 'N', ni, mi, mi, 2.0, T2, n, S, lds, 0.0, dL, lddl, C.s));
      } else {
        LYAP_TRY(gemm<double>('N', 'N', ni, mi, ryi, 2.0, Yf, n, T1, ryi, 0.0, dL, lddl, C.s));
      }
    }
    if (dS) LYAP_TRY(gemm<double>('T', 'N', mi, mi, ryi, 1.0, T1, ryi, T1, ryi, 0.0, dS, ldds, C.s));
    if (dA) {
      if (ri == 0) {
        LYAP_TRY(set_zero<double>(dA, n, n, ldda, C.s));
      } else {
        LYAP_TRY(gemm<double>('T', 'N', ryi, ri, ni, 1.0, Yf, n, Z, ldz, 0.0, T3, ryi, C.s));
        LYAP_TRY(gemm<double>('N', 'N', ni, ri, ryi, 1.0, Yf, n, T3, ryi, 0.0, T4, n, C.s));
        if (D) {
          scale_cols_dev_kernel<<<nblk((int64_t)n * r), 256, 0, C.s>>>(T4, ni, ri, ri + 1, D, T4);
          LYAP_CUDA_TRY(cudaGetLastError());
          lyap_count_launch();
        }
        LYAP_TRY(gemm<double>('N', 'T', ni, ni, ri, 2.0, T4, n, Z, ldz, 0.0, dA, ldda, C.s));
      }
    }
  } while (false);
  if (transposed) {
    const int t = transpose_store(C);
    if (st >= 0 && t < 0) st = t;
  }
  set_dgemm_method(dgemm_prev);
  collect_marks(C, inf);
  C.profile = false;
  cudaEventRecord(C.e1, C.s);
  cudaEventSynchronize(C.e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, C.e0, C.e1);
  inf->device_ms = ms;
  inf->kernel_launches = g_launches - l0;
  inf->status = st;
  return st;
}

// Independent Cholesky-type IR solves (config of many small equations) run concurrently:
// worker host threads, each with its own context and non-blocking stream, take the
// equations largest-n^3 first from a shared counter.  Every solve is the single-equation
// lyap_solve_ir path, so each result equals what a lone call would return.
static int batched_entry(lyap_ctx_t* C, int nb, const double* const* A, const int64_t* n, const double* const* L,
                         const int64_t* m, const lyap_opts_t* opts, double* const* Z, const int64_t* z_cap,
                         int64_t* rank_out, lyap_info_t* info, int workers) {
  if (!C || nb < 0 || !opts) return LYAP_ERR_ARG;
  if (nb == 0) return LYAP_OK;
  if (!A || !n || !L || !m || !Z || !z_cap || !rank_out) return LYAP_ERR_ARG;
  for (int e = 0; e < nb; ++e)
    if (!A[e] || !L[e] || !Z[e] || n[e] <= 0 || m[e] <= 0 || z_cap[e] <= 0) return LYAP_ERR_ARG;
  if (workers <= 0) workers = 8;
  workers = std::max(1, std::min({workers, nb, 32}));
  // inputs were produced on the caller's stream
  LYAP_CUDA_TRY(cudaStreamSynchronize(C->s));
  while ((int)C->pool.size() < workers) {
    cudaStream_t st = nullptr;
    LYAP_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    lyap_ctx_t* w = nullptr;
    const int r = lyap_ctx_create(&w, st);
    if (r < 0) {
      cudaStreamDestroy(st);
      return r;
    }
    C->pool.push_back(w);
    C->pool_streams.push_back(st);
  }
  std::vector<int> order(nb);
  for (int e = 0; e < nb; ++e) order[e] = e;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::atomic<int> next{0};
  std::vector<int> status(nb, 0);
  std::mutex mu;
  std::string first_err;
  const int dev = C->device;
  auto work = [&](int wi) {
    cudaSetDevice(dev);
    lyap_ctx_t* W = C->pool[wi];
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= nb) break;
      const int e = order[k];
      lyap_info_t* inf = info ? &info[e] : nullptr;
      const int st = solve_entry(W, A[e], n[e], n[e], L[e], n[e], m[e], nullptr, 0, opts, Z[e], n[e], z_cap[e],
                                 nullptr, &rank_out[e], inf, true);
      status[e] = st;
      if (st < 0) {
        std::lock_guard<std::mutex> g(mu);
        if (first_err.empty()) first_err = std::string("equation ") + std::to_string(e) + ": " + g_err;
      }
    }
    // every solve of this thread has completed (solve_entry waits for its last event)
    tc_release_thread_state();
  };
  std::vector<std::thread> th;
  for (int wi = 0; wi < workers; ++wi) th.emplace_back(work, wi);
  for (auto& t : th) t.join();
  int ret = LYAP_OK;
  for (int e = 0; e < nb; ++e) {
    if (status[e] < 0 && ret >= 0) ret = status[e];
    else if (status[e] > 0 && ret == LYAP_OK) ret = status[e];
  }
  if (!first_err.empty()) snprintf(g_err, sizeof(g_err), "%s", first_err.c_str());
  return ret;
}
}  // namespace lyap

extern "C" {

int lyap_sign_solve(lyap_ctx_t* C, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl, int64_t m,
                    const double* S, int64_t lds, const lyap_opts_t* opts, double* Z, int64_t ldz, int64_t z_cap,
                    double* D, int64_t* rank_out, lyap_info_t* info) {
  return solve_entry(C, A, n, lda, L, ldl, m, S, lds, opts, Z, ldz, z_cap, D, rank_out, info, false);
}

int lyap_solve_ir(lyap_ctx_t* C, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl, int64_t m,
                  const double* S, int64_t lds, const lyap_opts_t* opts, double* Z, int64_t ldz, int64_t z_cap,
                  double* D, int64_t* rank_out, lyap_info_t* info) {
  return solve_entry(C, A, n, lda, L, ldl, m, S, lds, opts, Z, ldz, z_cap, D, rank_out, info, true);
}

int lyap_solve_ir_batched(lyap_ctx_t* C, int nb, const double* const* A, const int64_t* n, const double* const* L,
                          const int64_t* m, const lyap_opts_t* opts, double* const* Z, const int64_t* z_cap,
                          int64_t* rank_out, lyap_info_t* info, int workers) {
  return batched_entry(C, nb, A, n, L, m, opts, Z, z_cap, rank_out, info, workers);
}

int lyap_adjoint(lyap_ctx_t* C, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl, int64_t m,
                 const double* S, int64_t lds, const double* Z, int64_t ldz, int64_t r, const double* D,
                 const double* Cm, int64_t ldc, int64_t q, const lyap_opts_t* opts, double* dA, int64_t ldda,
                 double* dL, int64_t lddl, double* dS, int64_t ldds, double* Zy, int64_t ldzy, int64_t zy_cap,
                 int64_t* rank_y, lyap_info_t* info) {
  return adjoint_entry(C, A, n, lda, L, ldl, m, S, lds, Z, ldz, r, D, Cm, ldc, q, opts, dA, ldda, dL, lddl, dS, ldds,
                       Zy, ldzy, zy_cap, rank_y, info);
}

int lyap_residual(lyap_ctx_t* C, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl, int64_t m,
                  const double* S, int64_t lds, const double* Z, int64_t ldz, int64_t r, const double* D,
                  double* res_out) {
  if (!C || !A || !L || !Z || !res_out || n <= 0 || m <= 0 || r < 0 || lda < n || ldl < n || ldz < n) return LYAP_ERR_ARG;
  Ctx& X = *C;
  Problem pb{A, (int)n, lda, L, ldl, (int)m, S, lds};
  LYAP_TRY(ensure(X.scal, 4096));
  LYAP_TRY(ensure(X.part, (size_t)4 * RED_BLOCKS * 8));
  LYAP_TRY(prepare_newton<double>(X, (int)n, (int)m, LYAP_FP64));
  double* Lw = nullptr;
  double* sd = nullptr;
  bool indef = false;
  LYAP_TRY(prepare_rhs(X, pb, &Lw, &sd, &indef));
  LYAP_TRY(ensure(X.Zs, (size_t)n * std::max<int64_t>(r, 1) * 8));
  LYAP_TRY((copy_cast<double, double>(Z, n, r, ldz, P<double>(X.Zs), n, 1.0, X.s)));
  LYAP_TRY(ensure(X.ysol, (size_t)(r + 8) * 8));
  if (D) LYAP_CUDA_TRY(cudaMemcpyAsync(X.ysol.p, D, sizeof(double) * r, cudaMemcpyDeviceToDevice, X.s));
  double* sc = P<double>(X.scal);
  LYAP_TRY(ensure(X.gram, (size_t)m * m * 8 + 64));
  LYAP_TRY(gemm<double>('T', 'N', m, m, n, 1.0, Lw, n, Lw, n, 0.0, P<double>(X.gram), m, X.s));
  gram_norm_kernel<<<1, 256, 0, X.s>>>(P<double>(X.gram), (int)m, sd, sc + 26);
  lyap_count_launch();
  LYAP_TRY(sumsq<double>(A, n, n, lda, sc + 23, P<double>(X.part), X.s));
  double h = 0;
  LYAP_TRY(sync_read(X, sc + 26, &h, sizeof(double)));
  h = sqrt(h);
  LYAP_CUDA_TRY(cudaMemcpyAsync(sc + 22, &h, sizeof(double), cudaMemcpyHostToDevice, X.s));
  LYAP_CUDA_TRY(cudaStreamSynchronize(X.s));
  ResOut ro;
  LYAP_TRY(res_fac(X, pb, Lw, sd, P<double>(X.Zs), (int)r, D ? P<double>(X.ysol) : nullptr, D != nullptr, 0.0, false,
                   &ro));
  *res_out = ro.res;
  return LYAP_OK;
}

// kappa_sign(B) in the Frobenius norm, B = [[A, W], [0, -A^T]] (Sec. 4.2).  The FP64 Newton
// iteration on B (Frobenius scaling until delta_k < 1e-2, stopped one step after delta_k <= 1e-8)
// keeps its inverses X_k^{-1} and mu_k; the Frechet derivative L(B, E) is the derivative of that
// iteration, E <- (mu_k E - mu_k^{-1} X_k^{-1} E X_k^{-1}) / 2 (exact in the limit: the fixed
// mu_k sequence converges for B + tE too), its adjoint L(B^T, .) the same with transposed
// inverses; ||L||_F comes from the power method on L^* L.
int lyap_kappa_sign(lyap_ctx_t* C, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl, int64_t m,
                    const double* S, int64_t lds, int power_steps, double* kappa, double* lnorm, int* newton_steps) {
  if (!C || !A || !L || !kappa || n <= 0 || m <= 0 || lda < n || ldl < n || (S && lds < m) || power_steps < 1 ||
      power_steps > 100 || n > 16384)
    return LYAP_ERR_ARG;
  Ctx& X = *C;
  Problem pb{A, (int)n, lda, L, ldl, (int)m, S, lds};
  LYAP_TRY(ensure(X.scal, 4096));
  LYAP_TRY(ensure(X.part, (size_t)4 * RED_BLOCKS * 8));
  double* Lw = nullptr;
  double* sd = nullptr;
  bool indef = false;
  LYAP_TRY(prepare_rhs(X, pb, &Lw, &sd, &indef));
  const int64_t N = 2 * n;
  const size_t NN = (size_t)N * N;
  // workspace: iterate, next iterate, E, two temporaries (5 N^2), W (n^2) and L S (n m); the
  // inverses of the iteration in their own allocations; all freed on return
  double* ws = nullptr;
  if (cudaMalloc(&ws, (5 * NN + (size_t)n * n + (size_t)n * m) * 8) != cudaSuccess) {
    cudaGetLastError();
    lyap_set_error_message("device allocation failed (kappa_sign workspace)", __FILE__, __LINE__);
    return LYAP_ERR_NOMEM;
  }
  std::vector<double*> inv;
  std::vector<double> mus;
  auto run = [&]() -> int {
    double* Xc = ws;
    double* Xn = ws + NN;
    double* E = ws + 2 * NN;
    double* T1 = ws + 3 * NN;
    double* T2 = ws + 4 * NN;
    double* W = ws + 5 * NN;
    double* LS = W + (size_t)n * n;
    double* sc = P<double>(X.scal) + 40;
    double* part = P<double>(X.part);
    LYAP_TRY((copy_cast<double, double>(Lw, n, m, n, LS, n, 1.0, X.s)));
    if (sd) LYAP_TRY(scale_cols<double>(LS, n, m, n, sd, X.s));
    LYAP_TRY(gemm<double>('N', 'T', n, n, m, 1.0, LS, n, Lw, n, 0.0, W, n, X.s));
    const unsigned g = (unsigned)std::min<int64_t>(4096, ceil_div((int64_t)NN, 256));
    sign_block_kernel<<<g, 256, 0, X.s>>>(A, lda, W, (int)n, Xc);
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
    double h[2];
    LYAP_TRY(sumsq<double>(Xc, N, N, N, sc, part, X.s));
    LYAP_TRY(sync_read(X, sc, h, sizeof(double)));
    const double nB = std::sqrt(h[0]);
    bool scaling = true;
    int after = -1;
    for (int k = 0; k < 64; ++k) {
      double* Ik = nullptr;
      if (cudaMalloc(&Ik, NN * 8) != cudaSuccess) {
        cudaGetLastError();
        lyap_set_error_message("device allocation failed (kappa_sign inverses)", __FILE__, __LINE__);
        return LYAP_ERR_NOMEM;
      }
      inv.push_back(Ik);
      LYAP_TRY(lyap_invert(C, Xc, N, N, LYAP_FP64, Ik, N, nullptr, nullptr));
      double mu = 1.0;
      if (scaling) {
        LYAP_TRY(sumsq<double>(Xc, N, N, N, sc, part, X.s));
        LYAP_TRY(sumsq<double>(Ik, N, N, N, sc + 1, part, X.s));
        LYAP_TRY(sync_read(X, sc, h, sizeof(h)));
        mu = std::sqrt(std::sqrt(h[1]) / std::sqrt(h[0]));
        if (!std::isfinite(mu) || !(mu > 0.0)) return LYAP_ERR_NONFINITE;
      }
      mus.push_back(mu);
      axpby_kernel<<<g, 256, 0, X.s>>>((int64_t)NN, 0.5 * mu, Xc, 0.5 / mu, Ik, Xn, T1);
      LYAP_CUDA_TRY(cudaGetLastError());
      lyap_count_launch();
      LYAP_TRY(sumsq<double>(T1, N, N, N, sc, part, X.s));
      LYAP_TRY(sumsq<double>(Xn, N, N, N, sc + 1, part, X.s));
      LYAP_TRY(sync_read(X, sc, h, sizeof(h)));
      std::swap(Xc, Xn);
      const double delta = std::sqrt(h[0] / h[1]);
      if (!std::isfinite(delta)) return LYAP_ERR_NONFINITE;
      if (after >= 0 && k >= after) break;
      if (after < 0 && delta <= 1e-8) after = k + 1;
      if (scaling && delta < 1e-2) scaling = false;
      if (k == 63) {
        lyap_set_error_message("Newton iteration on [[A, W], [0, -A^T]] did not converge", __FILE__, __LINE__);
        return LYAP_ERR_NOCONV;
      }
    }
    LYAP_TRY(sumsq<double>(Xc, N, N, N, sc, part, X.s));
    LYAP_TRY(sync_read(X, sc, h, sizeof(double)));
    const double nS = std::sqrt(h[0]);
    const int K = (int)inv.size();
    // the derivative of the iteration applied to E in place (adjoint: transposed inverses)
    auto apply = [&](bool adj) -> int {
      for (int k = 0; k < K; ++k) {
        const char t = adj ? 'T' : 'N';
        LYAP_TRY(gemm<double>(t, 'N', N, N, N, 1.0, inv[k], N, E, N, 0.0, T1, N, X.s));
        LYAP_TRY(gemm<double>('N', t, N, N, N, 1.0, T1, N, inv[k], N, 0.0, T2, N, X.s));
        axpby_kernel<<<g, 256, 0, X.s>>>((int64_t)NN, 0.5 * mus[k], E, -0.5 / mus[k], T2, E, nullptr);
        LYAP_CUDA_TRY(cudaGetLastError());
        lyap_count_launch();
      }
      return LYAP_OK;
    };
    hash_fill_kernel<<<g, 256, 0, X.s>>>((int64_t)NN, 0x2510021260ull, E);
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
    double gam = 0.0;
    for (int it = 0; it < power_steps; ++it) {
      // E <- E / ||E||_F; gamma = ||L(B, E)||_F; E <- L^*(B, L(B, E))
      LYAP_TRY(sumsq<double>(E, N, N, N, sc, part, X.s));
      LYAP_TRY(sync_read(X, sc, h, sizeof(double)));
      if (!(h[0] > 0.0)) break;
      axpby_kernel<<<g, 256, 0, X.s>>>((int64_t)NN, 1.0 / std::sqrt(h[0]), E, 0.0, E, E, nullptr);
      lyap_count_launch();
      LYAP_TRY(apply(false));
      LYAP_TRY(sumsq<double>(E, N, N, N, sc, part, X.s));
      LYAP_TRY(sync_read(X, sc, h, sizeof(double)));
      gam = std::max(gam, std::sqrt(h[0]));
      LYAP_TRY(apply(true));
    }
    *kappa = gam * nB / nS;
    if (lnorm) *lnorm = gam;
    if (newton_steps) *newton_steps = K;
    return LYAP_OK;
  };
  const int rc = run();
  cudaStreamSynchronize(X.s);
  for (double* p : inv) cudaFree(p);
  cudaFree(ws);
  return rc;
}

int lyap_dgemm(lyap_ctx_t* C, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* Cm, int64_t ldc,
               int method) {
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!C || m < 0 || n < 0 || k < 0 || method < 0 || method > 2) return LYAP_ERR_ARG;
  if ((transa != 'N' && transa != 'n' && !ta) || (transb != 'N' && transb != 'n' && !tb)) return LYAP_ERR_ARG;
  if (m == 0 || n == 0) return LYAP_OK;
  if (!Cm || ldc < m || (k > 0 && (!A || !B || lda < (ta ? k : m) || ldb < (tb ? n : k)))) return LYAP_ERR_ARG;
  const int prev = dgemm_method();
  set_dgemm_method(method);
  int st = gemm<double>(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, C->s);
  set_dgemm_method(prev);
  LYAP_TRY(st);
  LYAP_CUDA_TRY(cudaStreamSynchronize(C->s));
  int tcs = 0;
  LYAP_TRY(tc_status_read(&tcs));
  return tcs;
}

int lyap_trace_loss(lyap_ctx_t* C, const double* Z, int64_t n, int64_t ldz, int64_t r, const double* D,
                    const double* Cm, int64_t ldc, int64_t q, double* loss, double* dC, int64_t lddc) {
  if (!C || !Z || !Cm || !loss || n <= 0 || r < 0 || q <= 0 || ldz < n || ldc < q || (dC && lddc < q))
    return LYAP_ERR_ARG;
  Ctx& X = *C;
  LYAP_TRY(ensure(X.scal, 4096));
  const int64_t rr = std::max<int64_t>(r, 1);
  LYAP_TRY(ensure(X.tl, (size_t)2 * q * rr * 8 + 64));
  double* Tm = P<double>(X.tl);
  double* TD = Tm + (size_t)q * rr;
  double* out = P<double>(X.scal) + 320;
  if (r == 0) {
    LYAP_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), X.s));
    if (dC) LYAP_TRY(set_zero<double>(dC, q, n, lddc, X.s));
  } else {
    LYAP_TRY(gemm<double>('N', 'N', q, r, n, 1.0, Cm, ldc, Z, ldz, 0.0, Tm, q, X.s));
    trace_loss_kernel<<<1, 256, 0, X.s>>>(Tm, (int)q, (int)r, D, TD, out);
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
    if (dC) LYAP_TRY(gemm<double>('N', 'T', q, n, r, 2.0, TD, q, Z, ldz, 0.0, dC, lddc, X.s));
  }
  return sync_read(X, out, loss, sizeof(double));
}

}  // extern "C"
