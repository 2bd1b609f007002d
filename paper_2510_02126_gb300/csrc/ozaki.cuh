// FP64 matrix products on the FP16 tensor cores by error-free splitting (Ozaki-type scheme):
// the FP64 products of the refinement (A Z, the core matrices T P T^T and Gamma J Gamma^T, the
// Gram matrices, the Ogita-Aishima products) at FP64 accuracy without the FP64 pipe.
#pragma once
#include "dense.cuh"

namespace lyap {

// Slices: every row of op(A) (and every column of op(B)) is scaled by a power of two into
// (-1, 1) and cut into OZ_SLICES digits of OZ_BETA bits (integers, exact in FP16):
// x = 2^e sum_s d_s 2^(-OZ_BETA s) + O(2^(e - OZ_BETA OZ_SLICES)).  A product of two digit
// slices is a sum of at most OZ_KCHUNK integer terms below 2^(2 OZ_BETA), exact in the FP32
// accumulator of the tensor core; the pairs with s + t <= OZ_SLICES + 1 are summed in FP64.
constexpr int OZ_BETA = 7;
constexpr int OZ_SLICES = 8;
constexpr int OZ_KCHUNK = 1024;  // K columns per exact FP32 accumulation (1024 * 2^14 = 2^24)

// C = alpha op(A) op(B) + beta C for FP64 column-major operands (op = 'N' or 'T'), on
// tcgen05 tensor cores.  beta == 0 does not read C.  Workspace is held per host thread.
// The error is that of the truncated digit expansion plus the FP64 summation of the pair
// products: about 2^-50 max_l |op(A)_il| max_l |op(B)_lj| K per entry, the order of an FP64
// product's bound.
int ozaki_dgemm(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                const double* B, int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t s);

// Products at or above this many multiply-adds go to ozaki_dgemm in gemm<double> (smaller
// ones are latency-bound either way and stay on the FP64 SIMT kernel).
constexpr double OZ_MIN_MACS = 3.0e7;

}  // namespace lyap
