// Symmetric eigendecomposition of the small core matrices H = T P T^T and
// K = Gamma J Gamma^T (Fragments ResFacChol / SolUptChol and their LDL^T twins).
#pragma once
#include "dense.cuh"

namespace lyap {

struct EigScratch {
  float* work32 = nullptr;   // 2 q^2 floats (used when the matrix does not fit shared memory)
  double* X = nullptr;       // q^2 each
  double* R = nullptr;
  double* S = nullptr;
  double* HX = nullptr;
  double* E = nullptr;
  double* W = nullptr;       // q^2 (cluster rotations)
  double* lam = nullptr;     // q
  double* pv = nullptr;      // 2 q (power iteration vectors)
  double* red = nullptr;     // >= 16 + RED_BLOCKS doubles
  int* order = nullptr;      // q
  int* coff = nullptr;       // q + 1
  int* cidx = nullptr;       // q
  int* cinfo = nullptr;      // 4
  GridBar* bar = nullptr;    // grid barrier of the cooperative Jacobi
  int* status = nullptr;     // device status word
  int num_sms = 0;
};

// H (q x q, ldh, FP64, symmetric; not modified) = Q diag(w) Q^T, w ascending,
// Q (q x q, ldq).  FP32 parallel cyclic Jacobi, then (refine != 0) FP64
// refinement: Ogita-Aishima steps, Newton-Schulz re-orthonormalisation, and
// re-diagonalisation of every remaining eigenvalue cluster (its block of
// X^T H X, shifted and scaled to unit size, by a batched FP32 Jacobi), repeated
// until the coupling left is below 1e-15 ||H||_2.
int sym_eig(const double* H, int64_t q, int64_t ldh, double* w, double* Q, int64_t ldq, int refine,
            EigScratch& sc, cudaStream_t s);

}  // namespace lyap
