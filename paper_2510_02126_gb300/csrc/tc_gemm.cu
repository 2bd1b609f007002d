// tcgen05 tensor-core GEMM for sm_103a.
//
// D[128 x 128 tile] = A[128 x K] * B[128 x K]^T with 16-bit operands (FP16 or
// BF16) in K-major layout, staged into shared memory by TMA (128-byte swizzle,
// 64 K-elements per stage, a ring of STAGES stages guarded by mbarriers), FP32
// accumulation in tensor memory (TMEM, 128 columns), one thread issuing
// tcgen05.mma, and an epilogue in which each of the 4 warps reads its 32 TMEM
// lanes (tcgen05.ld 32x32b) and applies an operation-specific store:
//   * GJ update:  Mnew[i, x] = Mold[orig[i], x] + 2^(eP+eR) * acc      (x outside the panel)
//   * product:    Y[i, j]    = 2^(eX+eZ[j]) * acc
// Every mbarrier wait is bounded; on timeout the kernel records LYAP_ERR_TIMEOUT,
// releases its TMEM and returns.
#include <cuda.h>

#include "gj_inverse.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#include <atomic>

namespace lyap {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 2;  // 16 KB per operand per stage
// Stages of the TMA ring: the Gauss-Jordan update has K = 64 (one stage suffices, and the
// small footprint lets four CTAs share an SM -- the TMEM limit -- so that one CTA's
// epilogue overlaps another's loads); the factor product streams K = n through four.
__host__ __device__ constexpr int tc_stages(int mode) { return mode == 0 ? 1 : 4; }
__host__ __device__ constexpr int tc_smem(int mode) { return tc_stages(mode) * 2 * TC_TILE_BYTES + 1024 + 256; }
// epilogue staging of the update (per warp 32 x 33 floats) fits in the stage buffers
static_assert(4 * 32 * 33 * 4 <= 2 * TC_TILE_BYTES, "staging area");

// instruction descriptor for the 128 x 128 tiles of this file
__host__ __device__ constexpr uint32_t make_idesc(int fmt) { return make_idesc_mn(fmt, TC_BM, TC_BN); }

struct EpiGJ {
  const float* Mcur;
  float* Mnew;
  const int* orig;
  const int* exps;
  int n, k, bb, step;
};
struct EpiProd {
  float* Y;
  int64_t ldy;
  const int* eX;
  const int* eZ;
  int n, c;
};

template <int MODE>  // 0 = GJ update, 1 = product
__global__ void __launch_bounds__(128, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
               int K, int fmt, EpiGJ eg, EpiProd ep, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;
  constexpr int TC_STAGES = tc_stages(MODE);
  unsigned char* sB = base + TC_STAGES * TC_TILE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + 2 * TC_STAGES * TC_TILE_BYTES);
  uint64_t* done = full + TC_STAGES;
  uint64_t* fin = done + TC_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ int fail_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  const int KB = (K + TC_BK - 1) / TC_BK;

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&done[s], 1);
    }
    mbar_init(fin, 1);
    fail_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, TC_BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (tid == 0) {
    const uint32_t idesc = make_idesc(fmt);
    const int pre = KB < TC_STAGES ? KB : TC_STAGES;
    for (int kb = 0; kb < pre; ++kb) {
      mbar_expect_tx(&full[kb], 2 * TC_TILE_BYTES);
      tma_load_2d(sA + kb * TC_TILE_BYTES, &tmA, kb * TC_BK, m0, &full[kb]);
      tma_load_2d(sB + kb * TC_TILE_BYTES, &tmB, kb * TC_BK, n0, &full[kb]);
    }
    bool ok = true;
    for (int kb = 0; kb < KB && ok; ++kb) {
      const int s = kb % TC_STAGES;
      const unsigned ph = (unsigned)(kb / TC_STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) { ok = false; break; }
      tc_fence_after();
      const uint64_t ad = smem_desc_sw128(sA + s * TC_TILE_BYTES);
      const uint64_t bd = smem_desc_sw128(sB + s * TC_TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        // +32 bytes along K inside the 128-byte swizzle atom = +2 in the encoded address
        tc_mma(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kb > 0 || kk > 0) ? 1 : 0);
      }
      tc_commit(&done[s]);
      const int nk = kb + TC_STAGES;
      if (nk < KB) {
        if (!mbar_wait(&done[s], ph)) { ok = false; break; }
        mbar_expect_tx(&full[s], 2 * TC_TILE_BYTES);
        tma_load_2d(sA + s * TC_TILE_BYTES, &tmA, nk * TC_BK, m0, &full[s]);
        tma_load_2d(sB + s * TC_TILE_BYTES, &tmB, nk * TC_BK, n0, &full[s]);
      }
    }
    if (ok) {
      tc_commit(fin);
    } else {
      atomicCAS(status, 0, LYAP_ERR_TIMEOUT);
      fail_s = 1;
      // let copies in flight land before the CTA exits (bounded)
      for (int s = 0; s < TC_STAGES; ++s) (void)mbar_wait(&done[s], 0);
    }
  }
  __syncthreads();
  bool ok = (fail_s == 0);
  if (ok) ok = mbar_wait(fin, 0);
  if (!ok) atomicCAS(status, 0, LYAP_ERR_TIMEOUT);
  tc_fence_after();

  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    if (MODE == 0) {
      // TMEM rows are thread-private (lane = row), global rows are 4 n bytes apart: each
      // warp stages 32 x 32 blocks through shared memory (the drained stage buffers) so that
      // every global load and store covers 32 consecutive columns of one row
      const float sc = ldexpf(1.f, eg.exps[2 * eg.step] + eg.exps[2 * eg.step + 1]);
      float* stg = reinterpret_cast<float*>(base) + warp * 32 * 33;
      const int rbase = m0 + warp * 32;
      const int my_src = (rbase + lane < eg.n) ? eg.orig[rbase + lane] : 0;
      for (int j0 = 0; j0 < TC_BN; j0 += 32) {
        float v[32];
        tmem_ld16(trow + j0, v);
        tmem_ld16(trow + j0 + 16, v + 16);
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 32; ++t) stg[lane * 33 + t] = v[t];
        __syncwarp();
        const int x = n0 + j0 + lane;
        const bool xok = x < eg.n && (x < eg.k || x >= eg.k + eg.bb);
        // all 32 row loads of the block are issued before any is used (memory-level
        // parallelism: the old rows come from DRAM at large n)
        float old[32];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
          const int src = __shfl_sync(0xffffffffu, my_src, rr);
          old[rr] = (rbase + rr < eg.n && xok) ? __ldcs(eg.Mcur + (size_t)src * eg.n + x) : 0.f;
        }
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
          if (rbase + rr < eg.n && xok) __stcs(eg.Mnew + (size_t)(rbase + rr) * eg.n + x, old[rr] + sc * stg[rr * 33 + lane]);
      }
    } else {
      const int ex = *ep.eX;
      for (int j0 = 0; j0 < TC_BN; j0 += 16) {
        float v[16];
        tmem_ld16(trow + j0, v);
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int j = n0 + j0 + t;
          if (row < ep.n && j < ep.c) ep.Y[(size_t)row + (size_t)j * ep.ldy] = ldexpf(v[t], ex + ep.eZ[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TC_BN);
}

// ---------------------------------------------------------------------------
// host side: tensor maps through the driver entry point (no libcuda link needed)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {  // initialised once, thread-safe
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return nullptr;
  }();
  return fn;
}

// 2-D map over a row-major [rows x cols] 16-bit array with row pitch ld (elements); box 64 x box_rows
int tc_make_map(CUtensorMap* map, const void* ptr, int prec, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    lyap_set_error_message("cuTensorMapEncodeTiled unavailable", __FILE__, __LINE__);
    return LYAP_ERR_CUDA;
  }
  const CUtensorMapDataType dt = (prec == LYAP_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dt, 2, const_cast<void*>(ptr), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    lyap_set_error_message("cuTensorMapEncodeTiled failed", __FILE__, __LINE__);
    return LYAP_ERR_CUDA;
  }
  return LYAP_OK;
}

struct MapCache {
  const void* ptr = nullptr;
  int prec = -1;
  int64_t rows = -1, cols = -1, ld = -1;
  CUtensorMap map;
};
static int cached_map(MapCache* cache, int ncache, const void* ptr, int prec, int64_t rows, int64_t cols, int64_t ld,
                      CUtensorMap* out) {
  for (int i = 0; i < ncache; ++i) {
    MapCache& c = cache[i];
    if (c.ptr == ptr && c.prec == prec && c.rows == rows && c.cols == cols && c.ld == ld) {
      *out = c.map;
      return LYAP_OK;
    }
  }
  static thread_local int victim = 0;
  MapCache& c = cache[victim++ % ncache];
  LYAP_TRY(tc_make_map(&c.map, ptr, prec, rows, cols, ld, TC_BM));
  c.ptr = ptr;
  c.prec = prec;
  c.rows = rows;
  c.cols = cols;
  c.ld = ld;
  *out = c.map;
  return LYAP_OK;
}
// per host thread: contexts used from different threads (batched solves) keep their own
// tensor maps and status word
static thread_local MapCache g_cache[16];

static thread_local int* g_status = nullptr;
int* tc_status_word() {
  int*& p = g_status;
  if (!p) {
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
    // cleared before any kernel (on any stream) can report into it
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return nullptr;
  }
  return p;
}

static int launch_tc(int mode, int prec, const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K,
                     const EpiGJ& eg, const EpiProd& ep, cudaStream_t s) {
  static DeviceOnce attr;
  if (attr.need()) {
    LYAP_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(0)));
    LYAP_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(1)));
    attr.set();
  }
  int* st = tc_status_word();
  if (!st) return LYAP_ERR_NOMEM;
  dim3 grid((unsigned)ceil_div(N, TC_BN), (unsigned)ceil_div(M, TC_BM));
  const int fmt = (prec == LYAP_BF16) ? 1 : 0;
  if (mode == 0) tc_gemm_kernel<0><<<grid, 128, tc_smem(0), s>>>(a, b, M, N, K, fmt, eg, ep, st);
  else tc_gemm_kernel<1><<<grid, 128, tc_smem(1), s>>>(a, b, M, N, K, fmt, eg, ep, st);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}

// Frees the calling thread's status word (a worker thread about to exit, its work finished);
// the next use on this thread allocates a fresh one.
void tc_release_thread_state() {
  if (g_status) {
    cudaFree(g_status);
    g_status = nullptr;
  }
}

int tc_status_read(int* out) {
  int* st = tc_status_word();
  if (!st) return LYAP_ERR_NOMEM;
  LYAP_CUDA_TRY(cudaMemcpy(out, st, sizeof(int), cudaMemcpyDeviceToHost));  // after the caller's stream sync
  if (*out) LYAP_CUDA_TRY(cudaMemset(st, 0, sizeof(int)));                     // reported once
  return LYAP_OK;
}

int gj_update_tc(int prec, int n, int k, int bb, int step, const float* Mcur, float* Mnew, const void* Pp,
                 const void* Rt, const int* orig, const int* exps, cudaStream_t s) {
  CUtensorMap a, b;
  // the operand buffers hold at least TC_BM rows (tc_rows), so the 128-row box never exceeds the map
  const int rows = tc_rows(n);
  LYAP_TRY(cached_map(g_cache, 16, Pp, prec, rows, GJ_KLD16, GJ_KLD16, &a));
  LYAP_TRY(cached_map(g_cache, 16, Rt, prec, rows, GJ_KLD16, GJ_KLD16, &b));
  EpiGJ eg{Mcur, Mnew, orig, exps, n, k, bb, step};
  EpiProd ep{};
  return launch_tc(0, prec, a, b, n, n, GJ_KLD16, eg, ep, s);
}

int tc_product(int prec, int n, int c, const void* Xs, const int* eX, const void* Zh, const int* eZ, float* Y,
               int64_t ldy, cudaStream_t s) {
  if (c <= 0) return LYAP_OK;
  CUtensorMap a, b;
  const int64_t ldk = tc_kpitch(n);  // row pitch of Zh and of the stored inverses
  // maps cover at least one full 128 x 64 box; the padding of both operands is zero (K)
  // or outside the stored output (M, N), see tc_rows / tc_kpitch
  LYAP_TRY(cached_map(g_cache, 16, Xs, prec, tc_rows(n), std::max<int64_t>(n, TC_BK), ldk, &a));
  LYAP_TRY(cached_map(g_cache, 16, Zh, prec, tc_rows(c), std::max<int64_t>(n, TC_BK), ldk, &b));
  EpiGJ eg{};
  EpiProd ep{Y, ldy, eX, eZ, n, c};
  return launch_tc(1, prec, a, b, n, c, n, eg, ep, s);
}

// Zh[j, l] = Z[l, j] * 2^-eZ[j]  (c x ldk row-major, 16-bit), eZ[j] from max_l |Z[l, j]|
template <typename H>
__global__ void factor16_kernel(const float* __restrict__ Z, int n, int c, int64_t ld, H* __restrict__ Zh, int64_t ldk,
                                int* __restrict__ eZ) {
  const int j = blockIdx.x;
  if (j >= c) return;
  const float* z = Z + (size_t)j * ld;
  float m = 0.f;
  for (int l = threadIdx.x; l < n; l += blockDim.x) m = fmaxf(m, fabsf(z[l]));
  __shared__ float red[32];
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
    t = warp_max(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  const int e = pow2_exponent((double)red[0]);
  const float sc = ldexpf(1.f, -e);
  for (int l = threadIdx.x; l < ldk; l += blockDim.x) Zh[(size_t)j * ldk + l] = to_half<H>(l < n ? z[l] * sc : 0.f);
  if (threadIdx.x == 0) eZ[j] = e;
}

int factor_to_16(int prec, const float* Z, int n, int c, int64_t ld, void* Zh, int* eZ, cudaStream_t s) {
  if (c <= 0) return LYAP_OK;
  const int64_t ldk = tc_kpitch(n);
  if (prec == LYAP_BF16) factor16_kernel<__nv_bfloat16><<<c, 256, 0, s>>>(Z, n, c, ld, (__nv_bfloat16*)Zh, ldk, eZ);
  else factor16_kernel<__half><<<c, 256, 0, s>>>(Z, n, c, ld, (__half*)Zh, ldk, eZ);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  return LYAP_OK;
}

}  // namespace lyap
