// FP64 products on tcgen05 tensor cores by error-free splitting into FP16 digit slices.
//
// 1. Split (oz_rowexp_kernel, oz_digits_kernel): row i of op(A) gets the exponent e_i with
//    max_l |op(A)_il| < 2^e_i; the scaled row a = op(A)_i. 2^-e_i in (-1, 1) is cut into
//    OZ_SLICES digits, d_s = rint(2^OZ_BETA r_{s-1}), r_s = 2^OZ_BETA r_{s-1} - d_s (every
//    step exact in FP64), stored as FP16 integers in K-major slices (slice s at rows
//    [s Mp, (s+1) Mp) of one tall array).  op(B) is split the same way by columns.
// 2. Product (oz_gemm_kernel): one CTA per 128 x 64 tile of C.  A producer warp streams the
//    digit tiles by TMA through a ring of shared-memory stages and issues tcgen05.mma
//    (kind::f16, FP32 accumulators in TMEM) for every pair (s, t) with s + t <= OZ_SLICES + 1
//    over K chunks of OZ_KCHUNK; each pair's integer product is exact in FP32.  Two TMEM
//    accumulators alternate: while the MMAs of one pair fill one, four epilogue warps drain
//    the other into FP64 registers (scaled by 2^(-OZ_BETA (s + t)), deepest pairs first).
//    The tile is finally scaled by 2^(e_i + f_j), alpha and beta applied, and stored.
// Every mbarrier wait is bounded: on timeout the CTA records LYAP_ERR_TIMEOUT, lets its copies
// land, frees its TMEM and returns.
#include "ozaki.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace lyap {

constexpr int OZ_BM = 128, OZ_BN = 32, OZ_BK = 64, OZ_STAGES = 4;
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;  // 16 KB
constexpr int OZ_B_BYTES = OZ_BN * OZ_BK * 2;  // 4 KB
constexpr int OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES + 1024 + 256;
constexpr int OZ_NPAIRS = OZ_SLICES * (OZ_SLICES + 1) / 2;  // pairs with s + t <= S + 1 (s, t >= 1)
constexpr int OZ_THREADS = 192;                             // 4 epilogue warps, MMA warp, TMA warp
constexpr int64_t OZ_TARGET_CTAS = 148;                      // split K until about one CTA per SM
constexpr int64_t OZ_MAX_SPLIT = 16;
constexpr int OZ_FP32_LEVEL = 5;                             // 0-based s + t summed in FP32 from here
// pairs at levels >= OZ_FP32_LEVEL (they come first in the descending order)
constexpr int OZ_NPAIRS_FP32 = OZ_NPAIRS - OZ_FP32_LEVEL * (OZ_FP32_LEVEL + 1) / 2;
static_assert(OZ_NPAIRS_FP32 == 21, "levels 5, 6, 7 of eight slices");

// ---------------------------------------------------------------------------
// split
// ---------------------------------------------------------------------------
// The split runs in integer arithmetic on the bit patterns (FP64 operations are scarce on
// this GPU and would cost as much as the product).
constexpr int OZ_NO_EXP = (int)0x80808080;  // byte-wise memset sentinel: the row is zero

// frexp exponent of |x| from its bits (|x| < 2^result); OZ_NO_EXP for zero
__device__ __forceinline__ int oz_exponent(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  if (b == 0) return OZ_NO_EXP;
  const int E = (int)(b >> 52);
  return (E == 0 ? 1 : E) - 1022;
}

// e[r] = max over the row of the exponents (max_l |x(r, l)| < 2^e[r]); e must hold OZ_NO_EXP
// on entry.  x(r, l) = X[r + l ld] (tr = 0) or X[l + r ld] (tr = 1).  One 32 x 32 tile per
// CTA, loads coalesced along the contiguous index, one atomicMax per row and tile.
__global__ void __launch_bounds__(256) oz_rowexp_kernel(const double* __restrict__ X, int64_t ld, int tr, int64_t R,
                                                        int64_t K, int* __restrict__ e) {
  __shared__ int m[8][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, l0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  if (tr == 0) {
    // thread tx <-> row r0 + tx (contiguous), columns l0 + ty + 8 k
    const int64_t r = r0 + tx;
    int mx = OZ_NO_EXP;
    for (int k = ty; k < 32; k += 8) {
      const int64_t l = l0 + k;
      if (r < R && l < K) mx = max(mx, oz_exponent(X[r + l * ld]));
    }
    m[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && r < R) {
      for (int u = 1; u < 8; ++u) mx = max(mx, m[u][tx]);
      if (mx != OZ_NO_EXP) atomicMax(&e[r], mx);
    }
  } else {
    // warp ty <-> rows r0 + ty + 8 k, lane tx <-> column l0 + tx (contiguous)
    for (int k = ty; k < 32; k += 8) {
      const int64_t r = r0 + k, l = l0 + tx;
      int v = (r < R && l < K) ? oz_exponent(X[l + r * ld]) : OZ_NO_EXP;
      v = __reduce_max_sync(0xffffffffu, v);
      if (tx == 0 && r < R && v != OZ_NO_EXP) atomicMax(&e[r], v);
    }
  }
}

// digits of the 32 x 32 tile (rows r0.., columns l0..) into the slices (zeros in the padding):
// A = round(|x| 2^(56 - e)) as a 64-bit integer (|A| <= 2^56), then balanced base-2^OZ_BETA
// digits from the top: d = round(A / 2^sh), A -= d 2^sh, sh = 56 - OZ_BETA s.  Exact:
// x = 2^(e - 56) sum_s d_s 2^(56 - OZ_BETA s) up to the bits of x below 2^(e - 56).
__global__ void __launch_bounds__(256) oz_digits_kernel(const double* __restrict__ X, int64_t ld, int tr, int64_t R,
                                                        int64_t K, const int* __restrict__ e, __half* __restrict__ D,
                                                        int64_t Rp, int64_t Kp) {
  static_assert(OZ_BETA * OZ_SLICES == 56, "digits cover 56 bits below the row exponent");
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, l0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    // tr = 0: consecutive tx -> consecutive rows (contiguous); tr = 1: consecutive columns
    if (tr == 0) {
      const int64_t r = r0 + tx, l = l0 + k;
      t[tx][k] = (r < R && l < K) ? X[r + l * ld] : 0.0;
    } else {
      const int64_t r = r0 + k, l = l0 + tx;
      t[k][tx] = (r < R && l < K) ? X[l + r * ld] : 0.0;
    }
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = r0 + k, l = l0 + tx;
    if (r >= Rp || l >= Kp) continue;
    long long A = 0;
    const int er = (r < R) ? e[r] : OZ_NO_EXP;
    const unsigned long long b = (unsigned long long)__double_as_longlong(t[k][tx]);
    const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
    if (er != OZ_NO_EXP && mag != 0) {
      const int E = (int)(mag >> 52);
      const unsigned long long mant = (mag & 0x000FFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
      const int shift = (E ? E : 1) - 1075 + 56 - er;  // |x| = mant 2^((E ? E : 1) - 1075)
      unsigned long long a;
      if (shift >= 0) a = mant << shift;                 // |x| < 2^er: a < 2^56
      else if (shift > -64) a = (mant + (1ull << (-shift - 1))) >> (-shift);
      else a = 0;
      A = (b >> 63) ? -(long long)a : (long long)a;
    }
#pragma unroll
    for (int sl = 0; sl < OZ_SLICES; ++sl) {
      const int sh = 56 - OZ_BETA * (sl + 1);
      long long d;
      if (sh > 0) {
        d = (A + (1ll << (sh - 1))) >> sh;
        A -= d << sh;
      } else {
        d = A;
      }
      D[(size_t)sl * Rp * Kp + (size_t)r * Kp + l] = __int2half_rn((int)d);  // |d| <= 2^OZ_BETA: exact
    }
  }
}

// ---------------------------------------------------------------------------
// product
// ---------------------------------------------------------------------------
struct OzPairs {
  unsigned char s[OZ_NPAIRS], t[OZ_NPAIRS];
};
// (s, t), 0-based, ordered by descending level s + t (the smallest terms are summed first)
static constexpr OzPairs oz_make_pairs() {
  OzPairs p{};
  int k = 0;
  for (int lev = OZ_SLICES - 1; lev >= 0; --lev)
    for (int s = 0; s <= lev; ++s) {
      p.s[k] = (unsigned char)s;
      p.t[k] = (unsigned char)(lev - s);
      ++k;
    }
  return p;
}
__constant__ OzPairs c_oz_pairs = oz_make_pairs();

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
               int64_t Mp, int64_t Np, int nkb_all, int kbs, const int* __restrict__ eA, const int* __restrict__ eB,
               double alpha, double beta, double* __restrict__ C, int64_t ldc, double* __restrict__ part, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + OZ_STAGES * OZ_STAGE_BYTES);
  uint64_t* empty = full + OZ_STAGES;
  uint64_t* accfull = empty + OZ_STAGES;  // [2]
  uint64_t* accempty = accfull + 2;       // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accempty + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * OZ_BM, n0 = blockIdx.x * OZ_BN;
  // split-K: this CTA takes the k-blocks [kb_lo, kb_lo + nkb) of the product
  const int kb_lo = blockIdx.z * kbs;
  const int nkb = max(0, min(nkb_all - kb_lo, kbs));
  const int nchunk = max(1, (nkb + OZ_KCHUNK / OZ_BK - 1) / (OZ_KCHUNK / OZ_BK));
  const int total = (nkb > 0) ? nchunk * OZ_NPAIRS : 0;  // accumulations (pairs x chunks)

  if (tid == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, 2 * OZ_BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp >= 4) {
    // Iteration `it` is one k-block of one accumulation (chunk, pair); chunks are full
    // (OZ_KCHUNK / OZ_BK k-blocks) but the last.  Warp 5 (one lane) streams the digit tiles
    // by TMA into the ring as stages free up; warp 4 (one lane) waits for each stage and
    // issues its MMAs -- the two never wait for each other's latency.
    constexpr int KBC = OZ_KCHUNK / OZ_BK;
    const int per_chunk = KBC * OZ_NPAIRS;
    const int last_len = nkb - (nchunk - 1) * KBC;
    const int total_it = (nkb > 0) ? (nchunk - 1) * per_chunk + last_len * OZ_NPAIRS : 0;
    auto decode = [&](int x, int& pi, int& kb, int& first, int& last) {
      const int c = min(x / per_chunk, nchunk - 1);
      const int off = x - c * per_chunk;
      const int len = (c == nchunk - 1) ? last_len : KBC;
      pi = off / len;
      const int kk = off - pi * len;
      kb = kb_lo + c * KBC + kk;
      first = (kk == 0);
      last = (kk == len - 1);
    };
    if (warp == 5 && lane == 0) {
      // ---------------- TMA producer ----------------
      bool ok = true;
      int issued = 0;
      for (; issued < total_it; ++issued) {
        const int st = issued % OZ_STAGES;
        const unsigned ph = (unsigned)(issued / OZ_STAGES) & 1u;
        if (issued >= OZ_STAGES && !mbar_wait(&empty[st], ph ^ 1u)) { ok = false; break; }
        int pi, kb, f, l;
        decode(issued, pi, kb, f, l);
        unsigned char* sa = base + st * OZ_STAGE_BYTES;
        mbar_expect_tx(&full[st], OZ_STAGE_BYTES);
        tma_load_2d(sa, &tmA, kb * OZ_BK, (int)(c_oz_pairs.s[pi] * Mp + m0), &full[st]);
        tma_load_2d(sa + OZ_A_BYTES, &tmB, kb * OZ_BK, (int)(c_oz_pairs.t[pi] * Np + n0), &full[st]);
      }
      if (!ok) {
        atomicCAS(status, 0, LYAP_ERR_TIMEOUT);
        // let the copies in flight land before the CTA exits (bounded waits)
        for (int x = max(0, issued - OZ_STAGES); x < issued; ++x)
          (void)mbar_wait(&full[x % OZ_STAGES], (unsigned)(x / OZ_STAGES) & 1u);
      }
    } else if (warp == 4 && lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = make_idesc_mn(0, OZ_BM, OZ_BN);
      bool ok = true;
      int a = -1;  // current accumulation
      for (int it = 0; it < total_it; ++it) {
        int pi, kb, first, last;
        decode(it, pi, kb, first, last);
        const int st = it % OZ_STAGES;
        const unsigned ph = (unsigned)(it / OZ_STAGES) & 1u;
        if (first) {
          ++a;
          const int use = a >> 1;
          if (use > 0 && !mbar_wait(&accempty[a & 1], (unsigned)(use - 1) & 1u)) { ok = false; break; }
        }
        if (!mbar_wait(&full[st], ph)) { ok = false; break; }
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)((a & 1) * OZ_BN);
        unsigned char* sa = base + st * OZ_STAGE_BYTES;
        const uint64_t ad = smem_desc_sw128(sa);
        const uint64_t bd = smem_desc_sw128(sa + OZ_A_BYTES);
#pragma unroll
        for (int kk = 0; kk < OZ_BK / 16; ++kk) tc_mma(dcol, ad + 2 * kk, bd + 2 * kk, idesc, (!first || kk > 0) ? 1 : 0);
        tc_commit(&empty[st]);
        if (last) tc_commit(&accfull[a & 1]);
      }
      if (!ok) atomicCAS(status, 0, LYAP_ERR_TIMEOUT);
    }
  } else {
    // ---------------- epilogue warps 0..3: TMEM lanes 32 w .. 32 w + 31 ----------------
    // The pairs of the deepest levels (0-based s + t >= OZ_FP32_LEVEL) are summed in FP32,
    // relative to 2^(-OZ_BETA (OZ_FP32_LEVEL + 2)): their rounding stays below 2^-55 K of the
    // row / column scale, and the FP64 pipe (narrow on this GPU) takes only the leading pairs.
    double acc[OZ_BN];
    float acc32[OZ_BN];
#pragma unroll
    for (int j = 0; j < OZ_BN; ++j) { acc[j] = 0.0; acc32[j] = 0.f; }
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    for (int a = 0; a < total; ++a) {
      const int pi = a % OZ_NPAIRS;
      const int b = a & 1, use = a >> 1;
      const int lev = c_oz_pairs.s[pi] + c_oz_pairs.t[pi];
      if (!mbar_wait(&accfull[b], (unsigned)use & 1u)) { ok = false; break; }
      tc_fence_after();
      if (lev >= OZ_FP32_LEVEL) {
        const float sc = ldexpf(1.f, -OZ_BETA * (lev - OZ_FP32_LEVEL));
#pragma unroll
        for (int j0 = 0; j0 < OZ_BN; j0 += 16) {
          float v[16];
          tmem_ld16(lane_base + (uint32_t)(b * OZ_BN + j0), v);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc32[j0 + u] = fmaf(sc, v[u], acc32[j0 + u]);
        }
      } else {
        if (pi == OZ_NPAIRS_FP32) {  // first FP64 pair of this chunk: fold the FP32 sum in
#pragma unroll
          for (int j = 0; j < OZ_BN; ++j) {
            acc[j] += ldexp((double)acc32[j], -OZ_BETA * (OZ_FP32_LEVEL + 2));
            acc32[j] = 0.f;
          }
        }
        const double sc = ldexp(1.0, -OZ_BETA * (lev + 2));
#pragma unroll
        for (int j0 = 0; j0 < OZ_BN; j0 += 16) {
          float v[16];
          tmem_ld16(lane_base + (uint32_t)(b * OZ_BN + j0), v);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[j0 + u] = fma(sc, (double)v[u], acc[j0 + u]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[b]);
    }
    if (!ok) atomicCAS(status, 0, LYAP_ERR_TIMEOUT);
    const int row = m0 + warp * 32 + lane;
    if (ok && row < M) {
      const int ea = max(eA[row], -1100);  // a zero row (no exponent) has acc = 0
      if (part) {
        // split-K: this split's share of op(A) op(B), summed by oz_reduce_kernel
        double* pz = part + (size_t)blockIdx.z * Mp * Np;
#pragma unroll
        for (int j = 0; j < OZ_BN; ++j) {
          const int col = n0 + j;
          if (col < N) pz[(size_t)row + (size_t)col * Mp] = ldexp(acc[j], ea + max(eB[col], -1100));
        }
      } else {
#pragma unroll
        for (int j = 0; j < OZ_BN; ++j) {
          const int col = n0 + j;
          if (col < N) {
            double* c = C + (size_t)row + (size_t)col * ldc;
            const double v = alpha * ldexp(acc[j], ea + max(eB[col], -1100));
            *c = (beta == 0.0) ? v : fma(beta, *c, v);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * OZ_BN);
}

// C = alpha sum_z part[z] + beta C, the splits summed in a fixed order (same bits every call)
__global__ void oz_reduce_kernel(const double* __restrict__ part, int nsplit, int64_t Mp, int64_t Np, int M, int N,
                                 double alpha, double beta, double* __restrict__ C, int64_t ldc) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / M, row = e - col * M;
    double acc = 0.0;
    for (int z = 0; z < nsplit; ++z) acc += part[(size_t)z * Mp * Np + row + col * Mp];
    double* c = C + row + col * ldc;
    const double v = alpha * acc;
    *c = (beta == 0.0) ? v : fma(beta, *c, v);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
struct OzBufs {
  void* p = nullptr;
  size_t cap = 0;
};
thread_local OzBufs g_oz;

int oz_ensure(size_t bytes) {
  if (g_oz.p && g_oz.cap >= bytes) return LYAP_OK;
  if (g_oz.p) {
    // work queued on any stream may still read the old buffer
    LYAP_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(g_oz.p);
    g_oz.p = nullptr;
    g_oz.cap = 0;
  }
  const size_t want = bytes + bytes / 4 + 4096;
  if (cudaMalloc(&g_oz.p, want) != cudaSuccess) {
    cudaGetLastError();
    lyap_set_error_message("device allocation failed (FP64 tensor-core products)", __FILE__, __LINE__);
    return LYAP_ERR_NOMEM;
  }
  g_oz.cap = want;
  return LYAP_OK;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int oz_split(const double* X, int64_t ld, int tr, int64_t R, int64_t K, int64_t Rp, int64_t Kp, int* e, __half* D,
             cudaStream_t s) {
  LYAP_CUDA_TRY(cudaMemsetAsync(e, 0x80, sizeof(int) * (size_t)Rp, s));  // OZ_NO_EXP
  dim3 g((unsigned)(Kp / 32), (unsigned)(Rp / 32));
  oz_rowexp_kernel<<<g, 256, 0, s>>>(X, ld, tr, R, K, e);
  oz_digits_kernel<<<g, 256, 0, s>>>(X, ld, tr, R, K, e, D, Rp, Kp);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch(2);
  return LYAP_OK;
}
}  // namespace

int ozaki_dgemm(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                const double* B, int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return LYAP_OK;
  if (K <= 0 || alpha == 0.0) {
    if (beta == 0.0) return set_zero<double>(C, M, N, ldc, s);
    return gemm<double>('N', 'N', M, N, 0, 0.0, A, lda, B, ldb, beta, C, ldc, s);
  }
  const int64_t Mp = round_up(M, OZ_BM), Np = round_up(N, OZ_BN), Kp = round_up(K, OZ_BK);
  if (Mp * OZ_SLICES > INT32_MAX || Np * OZ_SLICES > INT32_MAX || Kp > INT32_MAX) return LYAP_ERR_ARG;
  // workspace: digit slices of op(A) (S Mp x Kp) and of op(B)^T (S Np x Kp), exponents
  const size_t bA = (size_t)OZ_SLICES * Mp * Kp * 2, bB = (size_t)OZ_SLICES * Np * Kp * 2;
  const size_t bE = (size_t)(Mp + Np) * 4;
  // split-K when the output has under half a wave of tiles, to about one wave of CTAs with at
  // least 4 k-blocks a split (measured: with half a wave or more the extra pass over the
  // partial products costs more than the idle SMs)
  const int nkb = (int)(Kp / OZ_BK);
  const int64_t tiles = (Mp / OZ_BM) * (Np / OZ_BN);
  int nsplit = 1;
  if (2 * tiles < OZ_TARGET_CTAS) nsplit = (int)std::min<int64_t>({OZ_MAX_SPLIT, nkb / 4, ceil_div(OZ_TARGET_CTAS, tiles)});
  nsplit = std::max(1, nsplit);
  const int kbs = (nkb + nsplit - 1) / nsplit;
  nsplit = (nkb + kbs - 1) / kbs;
  const size_t bP = (nsplit > 1) ? (size_t)nsplit * Mp * Np * 8 : 0;
  LYAP_TRY(oz_ensure(bP + bA + bB + bE + 512));
  double* part = (nsplit > 1) ? static_cast<double*>(g_oz.p) : nullptr;
  char* base = static_cast<char*>(g_oz.p) + bP;
  __half* DA = reinterpret_cast<__half*>(base);
  __half* DB = reinterpret_cast<__half*>(base + bA);
  int* eA = reinterpret_cast<int*>(base + bA + bB);
  int* eB = eA + Mp;
  // op(A) rows: A[i + l lda] ('N') or A[l + i lda] ('T');
  // op(B)^T rows (= columns of op(B)): B[l + j ldb] ('N') or B[j + l ldb] ('T')
  LYAP_TRY(oz_split(A, lda, (ta == 'T' || ta == 't') ? 1 : 0, M, K, Mp, Kp, eA, DA, s));
  LYAP_TRY(oz_split(B, ldb, (tb == 'T' || tb == 't') ? 0 : 1, N, K, Np, Kp, eB, DB, s));
  CUtensorMap mA, mB;
  LYAP_TRY(tc_make_map(&mA, DA, LYAP_FP16, (int64_t)OZ_SLICES * Mp, Kp, Kp, OZ_BM));
  LYAP_TRY(tc_make_map(&mB, DB, LYAP_FP16, (int64_t)OZ_SLICES * Np, Kp, Kp, OZ_BN));
  static DeviceOnce attr;
  if (attr.need()) {
    LYAP_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    attr.set();
  }
  int* st = tc_status_word();
  if (!st) return LYAP_ERR_NOMEM;
  dim3 grid((unsigned)(Np / OZ_BN), (unsigned)(Mp / OZ_BM), (unsigned)nsplit);
  oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM, s>>>(mA, mB, (int)M, (int)N, Mp, Np, nkb, kbs, eA, eB, alpha, beta, C,
                                                   ldc, part, st);
  LYAP_CUDA_TRY(cudaGetLastError());
  lyap_count_launch();
  if (part) {
    oz_reduce_kernel<<<(unsigned)std::min<int64_t>(4096, ceil_div(M * N, 256)), 256, 0, s>>>(part, nsplit, Mp, Np, (int)M,
                                                                                           (int)N, alpha, beta, C, ldc);
    LYAP_CUDA_TRY(cudaGetLastError());
    lyap_count_launch();
  }
  return LYAP_OK;
}

}  // namespace lyap
