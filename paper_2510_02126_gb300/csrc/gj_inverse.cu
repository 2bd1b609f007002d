// Blocked Gauss-Jordan inversion with partial pivoting on sm_103a.
//
// One blocked step eliminates a panel of GJ_BS columns [k, k+bb):
//   1. panel kernel (one CTA, or a thread-block cluster whose CTAs share the
//      panel rows through distributed shared memory): for each panel column
//      pick the pivot (largest |a_ij| among rows >= the diagonal, lowest row on
//      ties -- the getrf choice), swap it into place and eliminate the column
//      from every other row (in-place Gauss-Jordan, so the eliminated columns
//      accumulate the inverse).  It also emits the two GEMM operands of the
//      rank-bb update: P' (the panel with the identity subtracted on its
//      diagonal block) and R (the pivot rows, gathered from the old matrix).
//   2. update kernel: Mnew[i, x] = Mold[orig[i], x] + sum_t P'[i, t] R[t, x]
//      for every column x outside the panel (SIMT for FP32/FP64, tcgen05 tensor
//      cores on 16-bit operands for FP16/BF16, see tc_gemm.cu).
// After the last step the working matrix is X = (P A)^{-1}; A^{-1}[:, perm[c]] = X[:, c].
#include "gj_inverse.cuh"

#include <algorithm>
#include <atomic>

namespace lyap {

// implemented in tc_gemm.cu
int gj_update_tc(int prec, int n, int k, int bb, int step, const float* Mcur, float* Mnew,
                 const void* Pp, const void* Rt, const int* orig, const int* exps, cudaStream_t s);

__device__ __forceinline__ void op_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void op_store(double* p, double v) { *p = v; }
__device__ __forceinline__ void op_store(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void op_store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

template <typename OP> struct is16 { static constexpr bool value = false; };
template <> struct is16<__half> { static constexpr bool value = true; };
template <> struct is16<__nv_bfloat16> { static constexpr bool value = true; };

// Register-resident panel, lane = panel column: CTA `rank` of the cluster owns rows
// [rank R, rank R + R), R = NW * RPT (NW warps); warp w holds rows base + w + NW i
// (i < RPT) and lane t holds column t of each of them.  A Gauss-Jordan step is then one
// warp shuffle (the row's pivot-column entry) and one FMA per held row and lane, and
// loads and stores of panel rows are 128-byte coalesced.
//
// One barrier (CTA or cluster) per column: before it every warp publishes its pivot
// candidate for the column (value, row, and the whole row) and the owner of the
// diagonal row g publishes row g; after it every warp reduces the candidates to the
// pivot p and reads the pivot row and row g directly.  The published slots are
// double-buffered by column parity, so the writes of column j+1 never meet the reads of
// column j.  Row interchanges are recorded as the pivot sequence and replayed at the
// end to give each row its source row in the old matrix.
template <typename T>
struct PanelSh {
  T cv[2][32];          // candidate |value| per warp
  int ci[2][32];        // candidate row (global), -1 if none
  T crow[2][32][GJ_BS]; // candidate rows
  T grow[2][GJ_BS];     // row g before the step
  T ccv[2];             // candidate of the whole CTA (cluster panels)
  int cci[2];
  int piv[GJ_BS];       // pivot row of each panel column
  int rsrc[GJ_BS];      // source row (in the old matrix) of pivot row k + t
  float red[32];
  float cmax[2];
};

template <typename T, bool CL>
__device__ __forceinline__ void panel_sync() {
  if constexpr (CL) cluster_sync_all(); else __syncthreads();
}

template <typename T, bool CL>
__device__ float panel_max2(float v, PanelSh<T>& sh, int C, int slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_max(v);
  if (lane == 0) sh.red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    float w = (lane < (int)(blockDim.x >> 5)) ? sh.red[lane] : 0.f;
    w = warp_max(w);
    if (lane == 0) sh.cmax[slot] = w;
  }
  panel_sync<T, CL>();
  float m = 0.f;
  if constexpr (CL) {
    for (int c = 0; c < C; ++c) m = fmaxf(m, dsmem_ld_f32(dsmem_map(&sh.cmax[slot], c)));
  } else {
    m = sh.cmax[slot];
  }
  return m;
}

template <typename T, int RPT>
__device__ __forceinline__ T pick(const T (&v)[RPT], int i) {
  T r = T(0);
#pragma unroll
  for (int u = 0; u < RPT; ++u) r = (u == i) ? v[u] : r;
  return r;
}

// Source row of position r after the interchanges (g_0 <-> piv[0]), ..., applied in
// order: position r ends up holding old row s_0(s_1(... s_{bb-1}(r))).
__device__ __forceinline__ int replay_swaps(int r, int k, int bb, const int* piv) {
  int x = r;
  for (int j = bb - 1; j >= 0; --j) {
    const int g = k + j, p = piv[j];
    x = (x == g) ? p : ((x == p) ? g : x);
  }
  return x;
}

template <typename T, int NW, int RPT, bool CL, typename OP>
__global__ void __launch_bounds__(NW * 32, 1)
gj_panel_kernel(int n, int k, int step, const T* __restrict__ Mcur, T* __restrict__ Mnew,
                OP* __restrict__ Pp, OP* __restrict__ Rt, int* __restrict__ orig_out,
                const int* __restrict__ perm_old, int* __restrict__ perm_new,
                double* __restrict__ logpiv, int* __restrict__ ipiv, int* __restrict__ status,
                int* __restrict__ exps) {
  __shared__ PanelSh<T> sh;
  const int C = CL ? (int)gridDim.x : 1;
  const int rank = CL ? (int)cluster_ctarank() : 0;
  constexpr int R = NW * RPT;
  const int base = rank * R;
  const int bb = min(GJ_BS, n - k);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = base + warp;  // global row of v[0]; v[i] is row row0 + NW i

  T v[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int gr = row0 + NW * i;
    v[i] = (gr < n && lane < bb) ? Mcur[(size_t)gr * n + k + lane] : T(0);
  }
  // per-lane running candidate of this lane's column over the warp's rows >= k
  T bv = T(-1);
  int bi = -1;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int gr = row0 + NW * i;
    const T a = fabs(v[i]);
    if (gr < n && gr >= k && (bi < 0 || a > bv)) { bv = a; bi = i; }
  }

  bool bad = false;
#pragma unroll 1
  for (int j = 0; j < bb; ++j) {
    const int g = k + j, buf = j & 1;
    // (a) publish this warp's candidate for column j and, by its owner, row g
    const T wv = __shfl_sync(0xffffffffu, bv, j);
    const int wi = __shfl_sync(0xffffffffu, bi, j);
    if (wi >= 0) sh.crow[buf][warp][lane] = pick<T, RPT>(v, wi);
    if (lane == 0) {
      sh.cv[buf][warp] = wv;
      sh.ci[buf][warp] = (wi >= 0) ? row0 + NW * wi : -1;
    }
    const int og = g / R, lg = g - og * R;
    if (rank == og && warp == lg % NW) sh.grow[buf][lane] = pick<T, RPT>(v, lg / NW);
    // (b) pivot: every warp reduces all candidates (the same result everywhere).  In a
    // cluster each CTA first reduces its warps' candidates to one (a CTA barrier), so that
    // after the cluster barrier a single round of remote loads (lane c reads CTA c) remains.
    T pv = T(-1);
    int p = -1;
    if constexpr (CL) {
      __syncthreads();
      if (warp == 0) {
        T wv2 = (lane < NW) ? sh.cv[buf][lane] : T(-1);
        int wi2 = (lane < NW) ? sh.ci[buf][lane] : -1;
        warp_argmax(wv2, wi2);
        if (lane == 0) { sh.ccv[buf] = wv2; sh.cci[buf] = wi2; }
      }
      panel_sync<T, CL>();
      if (lane < C) {
        pv = dsmem_ld<T>(dsmem_map(&sh.ccv[buf], lane));
        p = dsmem_ld_s32(dsmem_map(&sh.cci[buf], lane));
        if (p < 0) pv = T(-1);
      }
    } else {
      panel_sync<T, CL>();
      if (lane < NW) { pv = sh.cv[buf][lane]; p = sh.ci[buf][lane]; }
    }
    warp_argmax(pv, p);
    if (p < 0 || !(pv > T(0)) || !isfinite(pv)) {
      if (tid == 0 && rank == 0)
        atomicCAS(status, 0, (p >= 0 && (isnan(pv) || isinf(pv))) ? LYAP_ERR_NONFINITE : LYAP_ERR_SINGULAR);
      bad = true;
      break;  // every thread of every CTA takes the same branch
    }
    const int op = p / R, lp = p - op * R;
    T prow_t;
    if constexpr (CL) prow_t = dsmem_ld<T>(dsmem_map(&sh.crow[buf][lp % NW][lane], op));
    else prow_t = sh.crow[buf][lp % NW][lane];
    const T pj = __shfl_sync(0xffffffffu, prow_t, j);
    const T inv = T(1) / pj;
    // lane j: v <- -f inv (the eliminated column becomes the inverse's column);
    // other lanes: v <- v - f q_t with q_t = prow_t / pj
    const T qq = (lane == j) ? inv : prow_t * inv;
    const T keep = (lane == j) ? T(0) : T(1);
    // (c) row swap + elimination of column j; candidates of column j+1 on the fly
    bv = T(-1);
    bi = -1;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int gr = row0 + NW * i;
      if (gr < n) {  // warp-uniform
        if (gr == g) {
          v[i] = qq;
        } else {
          if (gr == p) {  // receives the displaced row g
            if constexpr (CL) v[i] = dsmem_ld<T>(dsmem_map(&sh.grow[buf][lane], og));
            else v[i] = sh.grow[buf][lane];
          }
          const T f = __shfl_sync(0xffffffffu, v[i], j);
          v[i] = fma(-f, qq, v[i] * keep);
          const T a = fabs(v[i]);
          if (gr > g && (bi < 0 || a > bv)) { bv = a; bi = i; }
        }
      }
    }
    if (tid == 0) {
      sh.piv[j] = p;
      if (rank == 0) {
        logpiv[g] = (double)pj;  // the logarithms are taken after the inversion (pivot_logs)
        if (ipiv) ipiv[g] = p;
      }
    }
  }
  panel_sync<T, CL>();
  if (bad) return;

  // ---- outputs --------------------------------------------------------------
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int gr = row0 + NW * i;
    if (gr < n && lane < bb) Mnew[(size_t)gr * n + k + lane] = v[i];
  }
  for (int r = tid; r < R; r += NW * 32) {
    const int gr = base + r;
    if (gr >= n) continue;
    const int o = replay_swaps(gr, k, bb, sh.piv);
    orig_out[gr] = o;
    perm_new[gr] = perm_old[o];
  }
  if (warp == 0) sh.rsrc[lane] = (lane < bb) ? replay_swaps(k + lane, k, bb, sh.piv) : 0;
  __syncthreads();
  const int x0 = (int)((int64_t)rank * n / C), x1 = (int)((int64_t)(rank + 1) * n / C);
  constexpr int LDO = is16<OP>::value ? GJ_KLD16 : GJ_BS;

  float sP = 1.f, sR = 1.f;
  if constexpr (is16<OP>::value) {
    float mp = 0.f;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int gr = row0 + NW * i;
      if (gr < n && lane < bb) mp = fmaxf(mp, fabsf((float)v[i] - (gr == k + lane ? 1.f : 0.f)));
    }
    float mr = 0.f;
    if (lane < bb) {
      const T* src = Mcur + (size_t)sh.rsrc[lane] * n;
      for (int x = x0 + warp; x < x1; x += NW)
        if (x < k || x >= k + bb) mr = fmaxf(mr, fabsf((float)src[x]));
    }
    mp = panel_max2<T, CL>(mp, sh, C, 0);
    mr = panel_max2<T, CL>(mr, sh, C, 1);
    const int eP = pow2_exponent(mp), eR = pow2_exponent(mr);
    sP = ldexpf(1.f, -eP);
    sR = ldexpf(1.f, -eR);
    if (tid == 0 && rank == 0) { exps[2 * step] = eP; exps[2 * step + 1] = eR; }
  }
  // P' = panel - I on its diagonal block (lane = column: coalesced rows)
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int gr = row0 + NW * i;
    if (gr >= n) continue;
    const T val = (lane < bb) ? v[i] - (gr == k + lane ? T(1) : T(0)) : T(0);
    if constexpr (is16<OP>::value) {
      op_store(&Pp[(size_t)gr * LDO + lane], (float)val * sP);
      op_store(&Pp[(size_t)gr * LDO + 32 + lane], 0.f);
    } else {
      op_store(&Pp[(size_t)gr * LDO + lane], val);
    }
  }
  // R^T[x, t] = pivot row t at column x (lane = t: coalesced rows of R^T)
  const T* srow = Mcur + (size_t)sh.rsrc[lane] * n;
  for (int x = x0 + warp; x < x1; x += NW) {
    const bool use = lane < bb && (x < k || x >= k + bb);
    const T val = use ? srow[x] : T(0);
    if constexpr (is16<OP>::value) {
      op_store(&Rt[(size_t)x * LDO + lane], (float)val * sR);
      op_store(&Rt[(size_t)x * LDO + 32 + lane], 0.f);
    } else {
      op_store(&Rt[(size_t)x * LDO + lane], val);
    }
  }
  if constexpr (CL) cluster_sync_all();  // keep shared memory alive for remote readers
}

// Mnew[i, x] = Mold[orig[i], x] + sum_t Pp[i, t] Rt[x, t] for x outside [k, k+bb).
template <typename T>
__global__ void __launch_bounds__(256)
gj_update_simt(int n, int k, int bb, const T* __restrict__ Mcur, T* __restrict__ Mnew,
               const T* __restrict__ Pp, const T* __restrict__ Rt, const int* __restrict__ orig) {
  __shared__ T As[64][GJ_BS + 1];
  __shared__ T Bs[64][GJ_BS + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int x0 = blockIdx.x * 64, i0 = blockIdx.y * 64;
  for (int e = threadIdx.x; e < 64 * GJ_BS; e += 256) {
    const int r = e / GJ_BS, t = e - r * GJ_BS;
    const int gi = i0 + r, gx = x0 + r;
    As[r][t] = (gi < n) ? Pp[(size_t)gi * GJ_BS + t] : T(0);
    Bs[r][t] = (gx < n) ? Rt[(size_t)gx * GJ_BS + t] : T(0);
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 4
  for (int t = 0; t < GJ_BS; ++t) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[ty * 4 + a][t];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[tx + 16 * b][t];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
    if (i >= n) continue;
    const T* src = Mcur + (size_t)orig[i] * n;
    T* dst = Mnew + (size_t)i * n;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int x = x0 + tx + 16 * b;
      if (x < n && (x < k || x >= k + bb)) dst[x] = src[x] + acc[a][b];
    }
  }
}

// Panel geometry (lane = column, NW warps x RPT rows per CTA, C = ceil(n / (NW RPT))
// CTAs in one cluster, at most 16).  FP32: 16 warps x 4, 8, 16 or 32 rows per CTA, about
// 8 CTAs per cluster.  FP64 (two registers per value, and FP64
// arithmetic slow enough that it must spread over many SMs): 16 warps x 4, 8 or 16 rows,
// the smallest that fits n in 16 CTAs.
struct PanelGeom { int nw, rpt, C; };
static PanelGeom panel_geom(int n, int elt) {
  PanelGeom g;
  if (elt == 4) {
    // about 8 CTAs per cluster: the per-column work shrinks with the rows a warp holds,
    // while barriers of larger clusters cost more (measured at n = 1024 and 2048)
    g.nw = 16;
    g.rpt = (n <= 512) ? 4 : (n <= 1024) ? 8 : (n <= 2048) ? 16 : 32;
  } else {
    g.nw = 16;
    g.rpt = (n <= 16 * 16 * 4) ? 4 : (n <= 16 * 16 * 8) ? 8 : 16;
  }
  g.C = (int)ceil_div(n, (int64_t)g.nw * g.rpt);
  return g;
}

int gj_panel_cluster(int n, int elt) { return panel_geom(n, elt).C; }

template <typename T, int NW, int RPT, bool CL, typename OP>
static int launch_panel(GJWork& W, int k, int step, cudaStream_t s) {
  const int n = W.n;
  const int C = panel_geom(n, sizeof(T)).C;
  if (C > 16 || (!CL && C != 1)) {
    lyap_set_error_message("matrix order too large for the panel cluster", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  auto kern = gj_panel_kernel<T, NW, RPT, CL, OP>;
  static DeviceOnce attr_set;
  if (CL && attr_set.need()) {
    LYAP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    attr_set.set();
  }
  const T* Mcur = (const T*)W.M[W.cur];
  T* Mnew = (T*)W.M[1 - W.cur];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(NW * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (CL) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  LYAP_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, n, k, step, Mcur, Mnew, (OP*)W.Pp, (OP*)W.Rt, W.orig,
                                   (const int*)W.perm[W.cur], W.perm[1 - W.cur], W.logpiv, W.ipiv,
                                   W.status, W.exps));
  lyap_count_launch();
  return LYAP_OK;
}

template <typename T, int NW, int RPT, typename OP>
static int panel_dispatch_g(GJWork& W, int k, int step, cudaStream_t s) {
  if (gj_panel_cluster(W.n, sizeof(T)) > 1) return launch_panel<T, NW, RPT, true, OP>(W, k, step, s);
  return launch_panel<T, NW, RPT, false, OP>(W, k, step, s);
}
template <typename T, typename OP>
static int panel_dispatch(GJWork& W, int k, int step, cudaStream_t s) {

  const PanelGeom g = panel_geom(W.n, sizeof(T));
  if constexpr (sizeof(T) == 4) {
    if (g.rpt == 4) return panel_dispatch_g<T, 16, 4, OP>(W, k, step, s);
    if (g.rpt == 8) return panel_dispatch_g<T, 16, 8, OP>(W, k, step, s);
    if (g.rpt == 16) return panel_dispatch_g<T, 16, 16, OP>(W, k, step, s);
    return panel_dispatch_g<T, 16, 32, OP>(W, k, step, s);
  } else {
    if (g.rpt == 4) return panel_dispatch_g<T, 16, 4, OP>(W, k, step, s);
    if (g.rpt == 8) return launch_panel<T, 16, 8, true, OP>(W, k, step, s);
    return launch_panel<T, 16, 16, true, OP>(W, k, step, s);
  }
}

template <typename T>
static int update_simt(GJWork& W, int k, int bb, cudaStream_t s) {
  const int n = W.n;
  dim3 grid((unsigned)ceil_div(n, 64), (unsigned)ceil_div(n, 64));
  gj_update_simt<T><<<grid, 256, 0, s>>>(n, k, bb, (const T*)W.M[W.cur], (T*)W.M[1 - W.cur],
                                         (const T*)W.Pp, (const T*)W.Rt, W.orig);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}

__global__ void pivot_log_kernel(double* __restrict__ piv, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double l = log(fabs(piv[i]));
    piv[i] = l;
    t += l;
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *out = s;
  }
}

int pivot_logs(GJWork& W, double* out, cudaStream_t s) {
  pivot_log_kernel<<<1, 1024, 0, s>>>(W.logpiv, W.n, out);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}

int gj_invert_run(GJWork& W, int prec, cudaStream_t s) {
  const int n = W.n;
  int step = 0;
  for (int k = 0; k < n; k += GJ_BS, ++step) {
    const int bb = std::min(GJ_BS, n - k);
    switch (prec) {
      case LYAP_FP64:
        LYAP_TRY((panel_dispatch<double, double>(W, k, step, s)));
        LYAP_TRY(update_simt<double>(W, k, bb, s));
        break;
      case LYAP_FP32:
        LYAP_TRY((panel_dispatch<float, float>(W, k, step, s)));
        LYAP_TRY(update_simt<float>(W, k, bb, s));
        break;
      case LYAP_FP16:
        LYAP_TRY((panel_dispatch<float, __half>(W, k, step, s)));
        LYAP_TRY(gj_update_tc(prec, n, k, bb, step, (const float*)W.M[W.cur], (float*)W.M[1 - W.cur],
                              W.Pp, W.Rt, W.orig, W.exps, s));
        break;
      case LYAP_BF16:
        LYAP_TRY((panel_dispatch<float, __nv_bfloat16>(W, k, step, s)));
        LYAP_TRY(gj_update_tc(prec, n, k, bb, step, (const float*)W.M[W.cur], (float*)W.M[1 - W.cur],
                              W.Pp, W.Rt, W.orig, W.exps, s));
        break;
      default:
        return LYAP_ERR_ARG;
    }
    W.cur ^= 1;
  }
  return LYAP_OK;
}

}  // namespace lyap
