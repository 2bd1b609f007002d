// Symmetric eigendecomposition of the small core matrices H = T P T^T and
// K = Gamma J Gamma^T (Fragments ResFacChol / SolUptChol and their LDL^T twins).
#pragma once
#include "dense.cuh"

namespace lyap {

// largest order of the block Jacobi (its round-robin tables); above it sym_eig runs Jacobi over
// super-blocks whose pairs the block Jacobi diagonalises
constexpr int EIG_MAX_Q = 1280;

struct EigScratch {
  float* work32 = nullptr;   // bjac_work_floats(q) floats (block Jacobi workspace)
  float* big = nullptr;      // eig_big_floats(q) floats (orders above EIG_MAX_Q only)
  double* X = nullptr;       // q^2 each
  double* R = nullptr;
  double* S = nullptr;
  double* HX = nullptr;
  double* E = nullptr;
  double* W = nullptr;       // q^2 (cluster rotations)
  double* lam = nullptr;     // q
  double* pv = nullptr;      // 2 q (power iteration vectors)
  double* red = nullptr;     // >= 16 + RED_BLOCKS + 128 doubles
  int* order = nullptr;      // q
  int* coff = nullptr;       // q + 1
  int* cidx = nullptr;       // q
  int* cinfo = nullptr;      // 4
  GridBar* bar = nullptr;    // grid barrier of the cooperative Jacobi
  int* status = nullptr;     // device status word
  int num_sms = 0;
  // optional phase profiling hooks of the caller: mark(mark_ctx, LYAP_PHASE_*) starts a
  // timed phase; flops[LYAP_PHASE_*] accumulates algorithmic flops (host memory)
  void (*mark)(void*, int) = nullptr;
  void* mark_ctx = nullptr;
  double* flops = nullptr;
  // fast refinement (refine = 2) only: the relative accuracy its result must reach
  // (remaining coupling below target ||H||_2 before it may stop); 0 = the fixed fast rule
  double target = 0.0;
};

// H (q x q, ldh, FP64, symmetric; not modified) = Q diag(w) Q^T, w ascending,
// Q (q x q, ldq).  FP32 Jacobi (two-sided in shared memory for q <= 160, block
// two-sided across the GPU beyond), then FP64 refinement: Ogita-Aishima steps and
// re-diagonalisation of every remaining eigenvalue cluster (its block of X^T H X,
// shifted and scaled to unit size, by the FP32 Jacobi).
// refine: 0 = FP32 result; 1 = FP64-accurate (up to 8 rounds, clusters to 1e-6);
// 2 = FP64, fast (at most 3 rounds, clusters to 1e-3: for the projected update of the
// refinement loop, whose next step corrects what is left).
int sym_eig(const double* H, int64_t q, int64_t ldh, double* w, double* Q, int64_t ldq, int refine,
            EigScratch& sc, cudaStream_t s);

// Floats of EigScratch::work32 that sym_eig needs for order q (block Jacobi for q > 160).
size_t bjac_work_floats(int q);
// Floats of EigScratch::big that sym_eig needs for order q (0 up to EIG_MAX_Q).
size_t eig_big_floats(int64_t q);

}  // namespace lyap
