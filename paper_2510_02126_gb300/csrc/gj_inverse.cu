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

namespace lyap {

// implemented in tc_gemm.cu
int gj_update_tc(int prec, int n, int k, int bb, int step, const float* Mcur, float* Mnew,
                 const void* Pp, const void* Rt, const int* orig, const int* exps, cudaStream_t s);

template <typename T>
struct PanelShared {
  T wv[32];
  int wi[32];
  T prow[GJ_BS];
  T grow[GJ_BS];
  T prl[GJ_BS];
  int prow_orig, grow_orig, stop;
  int rsrc[GJ_BS];
  float red[32];
  float cmax[2];
};

__device__ __forceinline__ void op_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void op_store(double* p, double v) { *p = v; }
__device__ __forceinline__ void op_store(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void op_store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

template <typename OP> struct is16 { static constexpr bool value = false; };
template <> struct is16<__half> { static constexpr bool value = true; };
template <> struct is16<__nv_bfloat16> { static constexpr bool value = true; };

template <typename T, bool CL>
__device__ __forceinline__ void panel_sync() {
  if constexpr (CL) cluster_sync_all(); else __syncthreads();
}

// Block (cluster) wide max of a non-negative float; every thread gets the result.
template <typename T, bool CL>
__device__ float panel_max(float v, PanelShared<T>& sh, int C, int slot) {
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

template <typename T, bool CL, typename OP>
__global__ void __launch_bounds__(GJ_PANEL_THREADS, 1)
gj_panel_kernel(int n, int k, int step, const T* __restrict__ Mcur, T* __restrict__ Mnew,
                OP* __restrict__ Pp, OP* __restrict__ Rt, int* __restrict__ orig_out,
                const int* __restrict__ perm_old, int* __restrict__ perm_new,
                double* __restrict__ logpiv, int* __restrict__ ipiv, int* __restrict__ status,
                int* __restrict__ exps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PanelShared<T>& sh = *reinterpret_cast<PanelShared<T>*>(smem_raw);
  const size_t head = (sizeof(PanelShared<T>) + 15) & ~size_t(15);
  const int C = CL ? (int)gridDim.x : 1;
  const int rank = CL ? (int)cluster_ctarank() : 0;
  const int R = (n + C - 1) / C;
  T* panel = reinterpret_cast<T*>(smem_raw + head);
  int* orig_s = reinterpret_cast<int*>(smem_raw + head + sizeof(T) * (size_t)R * GJ_BS);
  const int base = rank * R;
  const int Rc = max(0, min(R, n - base));
  const int bb = min(GJ_BS, n - k);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NT = blockDim.x, NW = NT >> 5;

  for (int idx = tid; idx < Rc * GJ_BS; idx += NT) {
    const int r = idx / GJ_BS, t = idx - r * GJ_BS;
    panel[idx] = (t < bb) ? Mcur[(size_t)(base + r) * n + k + t] : T(0);
  }
  for (int r = tid; r < Rc; r += NT) orig_s[r] = base + r;
  if (tid == 0) sh.stop = 0;
  __syncthreads();

  bool bad = false;
  for (int j = 0; j < bb; ++j) {
    const int g = k + j;
    // (a) local pivot candidate
    T bv = T(-1);
    int bi = -1;
    for (int r = tid; r < Rc; r += NT) {
      const int gr = base + r;
      if (gr >= g) {
        const T v = fabs(panel[r * GJ_BS + j]);
        if (bi < 0 || v > bv) { bv = v; bi = gr; }
      }
    }
    warp_argmax(bv, bi);
    if (lane == 0) { sh.wv[warp] = bv; sh.wi[warp] = bi; }
    panel_sync<T, CL>();
    // (b) global pivot: every warp reduces all candidates (identical result everywhere)
    T pv = T(-1);
    int p = -1;
    for (int e = lane; e < C * NW; e += 32) {
      const int cr = e / NW, w = e - cr * NW;
      T cv;
      int ci;
      if constexpr (CL) {
        cv = dsmem_ld<T>(dsmem_map(&sh.wv[w], cr));
        ci = dsmem_ld_s32(dsmem_map(&sh.wi[w], cr));
      } else {
        cv = sh.wv[w];
        ci = sh.wi[w];
      }
      if (ci >= 0 && (p < 0 || cv > pv || (cv == pv && ci < p))) { pv = cv; p = ci; }
    }
    warp_argmax(pv, p);
    if (p < 0 || !(pv > T(0)) || !isfinite((double)pv)) {
      if (tid == 0 && rank == 0)
        atomicCAS(status, 0, (p >= 0 && isnan((double)pv)) || isinf((double)pv) ? LYAP_ERR_NONFINITE
                                                                                : LYAP_ERR_SINGULAR);
      bad = true;
      break;  // every thread of every CTA takes the same branch
    }
    // (c) publish the pivot row and the row it displaces
    const int op = p / R, rp = p - op * R;
    const int og = g / R, rg = g - og * R;
    if (rank == op && tid < GJ_BS) sh.prow[tid] = panel[rp * GJ_BS + tid];
    if (rank == op && tid == 0) sh.prow_orig = orig_s[rp];
    if (rank == og && tid < GJ_BS) sh.grow[tid] = panel[rg * GJ_BS + tid];
    if (rank == og && tid == 0) sh.grow_orig = orig_s[rg];
    panel_sync<T, CL>();
    const T* prow;
    if constexpr (CL) {
      if (warp == 0) sh.prl[lane] = dsmem_ld<T>(dsmem_map(&sh.prow[lane], op));
      __syncthreads();
      prow = sh.prl;
    } else {
      prow = sh.prow;
    }
    const T piv = prow[j];
    const T inv = T(1) / piv;
    // (d) row swap + Gauss-Jordan elimination of column j
    for (int r = tid; r < Rc; r += NT) {
      const int gr = base + r;
      T* row = panel + r * GJ_BS;
      if (gr == g) {
#pragma unroll 8
        for (int t = 0; t < GJ_BS; ++t) row[t] = (t == j) ? inv : prow[t] * inv;
        if (p != g) {
          int po;
          if constexpr (CL) po = dsmem_ld_s32(dsmem_map(&sh.prow_orig, op)); else po = sh.prow_orig;
          orig_s[r] = po;
        }
      } else {
        if (gr == p) {  // p != g here: receives the displaced row g
#pragma unroll 8
          for (int t = 0; t < GJ_BS; ++t) {
            T v;
            if constexpr (CL) v = dsmem_ld<T>(dsmem_map(&sh.grow[t], og)); else v = sh.grow[t];
            row[t] = v;
          }
          int go;
          if constexpr (CL) go = dsmem_ld_s32(dsmem_map(&sh.grow_orig, og)); else go = sh.grow_orig;
          orig_s[r] = go;
        }
        const T f = row[j];
        if (f != T(0)) {
#pragma unroll 8
          for (int t = 0; t < GJ_BS; ++t) {
            if (t != j) row[t] -= f * (prow[t] * inv);
          }
          row[j] = -f * inv;
        }
      }
    }
    if (tid == 0 && rank == 0) {
      logpiv[g] = log(fabs((double)piv));
      if (ipiv) ipiv[g] = p;
    }
  }
  panel_sync<T, CL>();  // all rows final, all orig_s final
  if (bad) return;

  // ---- outputs --------------------------------------------------------------
  for (int idx = tid; idx < Rc * GJ_BS; idx += NT) {
    const int r = idx / GJ_BS, t = idx - r * GJ_BS;
    if (t < bb) Mnew[(size_t)(base + r) * n + k + t] = panel[idx];
  }
  for (int r = tid; r < Rc; r += NT) {
    orig_out[base + r] = orig_s[r];
    perm_new[base + r] = perm_old[orig_s[r]];
  }
  // sources of the pivot rows k..k+bb-1
  if (warp == 0) {
    int src = -1;
    if (lane < bb) {
      const int gr = k + lane, oc = gr / R, rr = gr - oc * R;
      if constexpr (CL) src = dsmem_ld_s32(dsmem_map(&orig_s[rr], oc)); else src = orig_s[rr];
    }
    sh.rsrc[lane] = src;
  }
  __syncthreads();
  const int x0 = (int)((int64_t)rank * n / C), x1 = (int)((int64_t)(rank + 1) * n / C);

  float sP = 1.f, sR = 1.f;
  if constexpr (is16<OP>::value) {
    float mp = 0.f;
    for (int idx = tid; idx < Rc * GJ_BS; idx += NT) {
      const int r = idx / GJ_BS, t = idx - r * GJ_BS;
      if (t < bb) {
        const float v = (float)panel[idx] - ((base + r) == k + t ? 1.f : 0.f);
        mp = fmaxf(mp, fabsf(v));
      }
    }
    float mr = 0.f;
    for (int x = x0 + tid; x < x1; x += NT) {
      if (x >= k && x < k + bb) continue;
      for (int t = 0; t < bb; ++t) mr = fmaxf(mr, fabsf((float)Mcur[(size_t)sh.rsrc[t] * n + x]));
    }
    mp = panel_max<T, CL>(mp, sh, C, 0);
    mr = panel_max<T, CL>(mr, sh, C, 1);
    const int eP = pow2_exponent(mp), eR = pow2_exponent(mr);
    sP = ldexpf(1.f, -eP);
    sR = ldexpf(1.f, -eR);
    if (tid == 0 && rank == 0) { exps[2 * step] = eP; exps[2 * step + 1] = eR; }
  }
  constexpr int LDO = is16<OP>::value ? GJ_KLD16 : GJ_BS;
  for (int idx = tid; idx < Rc * LDO; idx += NT) {
    const int r = idx / LDO, t = idx - r * LDO;
    T v = T(0);
    if (t < bb) v = panel[r * GJ_BS + t] - ((base + r) == k + t ? T(1) : T(0));
    if constexpr (is16<OP>::value) op_store(&Pp[(size_t)(base + r) * LDO + t], (float)v * sP);
    else op_store(&Pp[(size_t)(base + r) * LDO + t], v);
  }
  for (int x = x0 + tid; x < x1; x += NT) {
    const bool inpanel = (x >= k && x < k + bb);
#pragma unroll 4
    for (int t = 0; t < LDO; ++t) {
      T v = T(0);
      if (t < bb && !inpanel) v = Mcur[(size_t)sh.rsrc[t] * n + x];
      if constexpr (is16<OP>::value) op_store(&Rt[(size_t)x * LDO + t], (float)v * sR);
      else op_store(&Rt[(size_t)x * LDO + t], v);
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

int gj_panel_cluster(int n, int elt) {
  const int64_t bytes = (int64_t)n * (GJ_BS * elt + 4);
  int C = (int)ceil_div(bytes, GJ_PANEL_SMEM_BUDGET);
  if (C < 1) C = 1;
  if (C > n) C = n;
  return C;
}

template <typename T, bool CL, typename OP>
static int launch_panel(GJWork& W, int k, int step, cudaStream_t s) {
  const int n = W.n;
  const int C = gj_panel_cluster(n, sizeof(T));
  if (C > 8) {
    lyap_set_error_message("matrix order too large for the panel cluster", __FILE__, __LINE__);
    return LYAP_ERR_ARG;
  }
  const int R = (n + C - 1) / C;
  const size_t head = (sizeof(PanelShared<T>) + 15) & ~size_t(15);
  const size_t smem = head + sizeof(T) * (size_t)R * GJ_BS + sizeof(int) * (size_t)R;
  auto kern = gj_panel_kernel<T, CL, OP>;
  static bool attr_set = false;
  if (!attr_set) {
    LYAP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr_set = true;
  }
  const T* Mcur = (const T*)W.M[W.cur];
  T* Mnew = (T*)W.M[1 - W.cur];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(GJ_PANEL_THREADS);
  cfg.dynamicSmemBytes = smem;
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

template <typename T, typename OP>
static int panel_dispatch(GJWork& W, int k, int step, cudaStream_t s) {
  if (gj_panel_cluster(W.n, sizeof(T)) > 1) return launch_panel<T, true, OP>(W, k, step, s);
  return launch_panel<T, false, OP>(W, k, step, s);
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
