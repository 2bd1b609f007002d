// Householder QR kernels: thin QR of tall-skinny factors (Fragments ResFacChol /
// SolUptChol and their LDL^T twins, Sec. 2) and QR with column pivoting for the
// rank truncation of the Newton factor (RankTruncChol, Sec. 3.2).
#pragma once
#include "dense.cuh"

namespace lyap {

struct QRScratch {
  GridBar* bar = nullptr;   // grid barrier (count must be 0 before a launch)
  int* status = nullptr;    // device status word
  void* cand = nullptr;     // per-block candidates (>= 3 * 256 doubles)
  void* norms = nullptr;    // column norms (>= 2 * ncols values of T)
  int* piv = nullptr;       // pivot order (>= ncols)
  void* rdiag = nullptr;    // R diagonal (>= ncols)
  void* work = nullptr;     // transposed copy of the factor (c x n values of T)
  int* rank = nullptr;      // device int: truncation rank
  int* flags = nullptr;     // per-column ready flags of householder_qr (>= min(m, q) ints)
  int num_sms = 0;
};

// Householder QR of F (m x q, column-major, ld) in place: R in the upper triangle,
// reflector vectors below the diagonal (unit leading entry implicit), tau[min(m,q)].
template <typename T>
int householder_qr(T* F, int64_t m, int64_t q, int64_t ld, T* tau, QRScratch& sc, cudaStream_t s);

// Y (m x r, ldy) = Q [C; 0] with Q = H_0 H_1 ... H_{k-1} from householder_qr,
// C (k x r, ldc).  Y may not alias C.
template <typename T>
int apply_q(const T* F, int64_t m, int64_t k, int64_t ldf, const T* tau, const T* C, int64_t ldc,
            int64_t r, T* Y, int64_t ldy, cudaStream_t s);

// RankTruncChol: QR with column pivoting of Z^T (Z is n x c, column-major, ldz),
// stopping at the first r with ||S_r||_F <= tol |r_11|; writes Pi [T C]^T into
// Z[:, 0:r] and r into *sc.rank (device).
template <typename T>
int qrcp_truncate(T* Z, int64_t n, int64_t c, int64_t ldz, double tol, QRScratch& sc, cudaStream_t s);

}  // namespace lyap
