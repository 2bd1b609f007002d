// Blocked Gauss-Jordan inversion with partial pivoting (getrf pivot sequence fused
// with the getri inversion), the dense kernel behind every sign-Newton step
// (Sec. 3.1-3.3: A_k^{-1}, 2 n^3 flops per inversion).
#pragma once
#include "lyap_common.cuh"

namespace lyap {

// Width of one pivoted panel (columns eliminated per blocked step).
constexpr int GJ_BS = 32;
// Row pitch (elements) of the 16-bit panel operands: one 128-byte TMA/UMMA row, upper half zero.
constexpr int GJ_KLD16 = 64;

// Device workspace of one inversion of order n in working type T (row-major).
struct GJWork {
  int n = 0;
  int elt = 0;           // sizeof(T)
  void* M[2] = {nullptr, nullptr};   // ping-pong working matrices (n x n, row-major)
  void* Pp = nullptr;    // panel operand, n x GJ_BS (T or 16-bit)
  void* Rt = nullptr;    // pivot-row operand, n x GJ_BS (T or 16-bit)
  int* orig = nullptr;   // row gather map of the current step (n)
  int* perm[2] = {nullptr, nullptr};  // composed row permutation (n)
  double* logpiv = nullptr;  // pivot of each column (n); log|pivot| after pivot_logs()
  int* ipiv = nullptr;       // pivot row chosen at each column (n)
  int* status = nullptr;     // device status word (0 = ok, else LYAP_ERR_*)
  int* exps = nullptr;       // per-step power-of-two exponents of the 16-bit operands (2 per step)
  float* amax = nullptr;     // scratch for operand max reductions (per step: 2 floats)
  int cur = 0;           // which M / perm holds the current state
};

// Launch the panel + update sequence.  On entry W.M[W.cur] holds the row-major
// matrix to invert.  On exit W.M[W.cur] holds X = (P A)^{-1} and W.perm[W.cur]
// the row permutation P (perm[i] = original row at position i), so that
// A^{-1}[:, perm[c]] = X[:, c].  prec selects the update kernel:
// FP64 -> T=double SIMT, FP32 -> T=float SIMT, FP16/BF16 -> T=float working
// matrix with tcgen05 tensor-core updates on 16-bit operands.
int gj_invert_run(GJWork& W, int prec, cudaStream_t s);

// Replace the recorded pivots by log|pivot| and write their sum to *out (device).
int pivot_logs(GJWork& W, double* out, cudaStream_t s);

// Cluster size used by the panel kernel for order n and element size elt.
int gj_panel_cluster(int n, int elt);

}  // namespace lyap
