// tcgen05 tensor-core GEMMs (sm_103a): TMA-fed 16-bit operands, FP32 accumulators in TMEM.
#pragma once
#include <cuda.h>

#include "lyap_common.cuh"

namespace lyap {

// Layout rules of the 16-bit tensor-core operands.  Every operand buffer holds at least
// 128 rows (one TMA box) and a K pitch of at least 64 elements (one 128-byte swizzle row),
// so that small problems never encode a map smaller than its box.  Rows beyond the
// problem only feed outputs that the epilogues discard; K padding must be zero.
inline int64_t tc_rows(int64_t rows) { return rows < 128 ? 128 : rows; }
inline int64_t tc_kpitch(int64_t k) { const int64_t p = (k + 7) / 8 * 8; return p < 64 ? 64 : p; }

// Gauss-Jordan trailing update on 16-bit operands (prec = LYAP_FP16 / LYAP_BF16):
//   Mnew[i, x] = Mcur[orig[i], x] + 2^(eP+eR) sum_t Pp[i, t] Rt[x, t]   for x outside [k, k+bb)
// Pp, Rt: n x 32 (K-major, 16-bit, scaled by 2^-eP / 2^-eR, exponents in exps[2 step .. 2 step+1]).
int gj_update_tc(int prec, int n, int k, int bb, int step, const float* Mcur, float* Mnew,
                 const void* Pp, const void* Rt, const int* orig, const int* exps, cudaStream_t s);

// Factor product on 16-bit operands:
//   Y[:, j] = 2^(eX + eZ[j]) sum_l Xs[i, l] Zh[j, l]       (i < n, j < c)
// Xs: n x n row-major 16-bit (K-major A operand), *eX its exponent (device int);
// Zh: c x n row-major 16-bit (= the n x c factor, column-major; K-major B operand),
// eZ: per-column exponents (device int[c]); Y: FP32 column-major (ldy).
int tc_product(int prec, int n, int c, const void* Xs, const int* eX, const void* Zh, const int* eZ,
               float* Y, int64_t ldy, cudaStream_t s);

// Convert an FP32 column-major factor (n x c, ld) into the 16-bit operand of
// tc_product with one power-of-two exponent per column.
// Reads (and clears) the status word of the tensor-core kernels (0 or LYAP_ERR_TIMEOUT).
int tc_status_read(int* out);
// Release the calling host thread's status word (call before the thread exits).
void tc_release_thread_state();

int factor_to_16(int prec, const float* Z, int n, int c, int64_t ld, void* Zh, int* eZ, cudaStream_t s);

// The calling host thread's device status word of the tensor-core kernels (nullptr if it
// cannot be allocated); kernels record LYAP_ERR_TIMEOUT there.
int* tc_status_word();
// Encode a TMA map over a row-major [rows x cols] 16-bit array of precision prec with row
// pitch ld (elements), box 64 (K) x box_rows, 128-byte swizzle.
int tc_make_map(CUtensorMap* map, const void* ptr, int prec, int64_t rows, int64_t cols, int64_t ld, int box_rows);

}  // namespace lyap
