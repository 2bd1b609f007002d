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

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (unsigned it = 0; it < (1u << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// K-major operand tile of 128 rows x 64 16-bit elements, 128-byte swizzle:
// 8-row swizzle atoms of 1024 bytes stacked along M/N (stride byte offset 1024).
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;                 // start address
  d |= (uint64_t)(16 >> 4) << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset
  d |= 1ull << 46;                              // descriptor version (sm_100 family)
  d |= 2ull << 61;                              // SWIZZLE_128B
  return d;
}
// instruction descriptor: D = F32, A/B = F16 (fmt 0) or BF16 (fmt 1), both K-major, M = 128, N = TC_BN
__host__ __device__ constexpr uint32_t make_idesc(int fmt) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

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
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
          const int src = __shfl_sync(0xffffffffu, my_src, rr);
          if (rbase + rr < eg.n && xok)
            eg.Mnew[(size_t)(rbase + rr) * eg.n + x] = eg.Mcur[(size_t)src * eg.n + x] + sc * stg[rr * 33 + lane];
        }
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

// 2-D map over a row-major [rows x cols] 16-bit array with row pitch ld (elements); box 64 x 128
static int make_map(CUtensorMap* map, const void* ptr, int prec, int64_t rows, int64_t cols, int64_t ld) {
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    lyap_set_error_message("cuTensorMapEncodeTiled unavailable", __FILE__, __LINE__);
    return LYAP_ERR_CUDA;
  }
  const CUtensorMapDataType dt = (prec == LYAP_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
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
  LYAP_TRY(make_map(&c.map, ptr, prec, rows, cols, ld));
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
static int* status_word() {
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
  int* st = status_word();
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
  int* st = status_word();
  if (!st) return LYAP_ERR_NOMEM;
  LYAP_CUDA_TRY(cudaMemcpy(out, st, sizeof(int), cudaMemcpyDeviceToHost));  // after the caller's stream sync
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
