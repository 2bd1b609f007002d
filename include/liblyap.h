/*
 * liblyap -- mixed-precision iterative refinement for low-rank Lyapunov equations
 *            A X + X A^T + W = 0,  W = L L^T  or  W = L S L^T           (Eq. (1.1), (1.2))
 * on one NVIDIA GB300 GPU (sm_103a), after Benner & Liu, arXiv 2510.02126.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are column-major FP64 unless stated otherwise; `ld*` is the leading
 *    dimension in elements (>= number of rows).
 *  - Pointers named A, L, S, Z, D, Ainv, ... are DEVICE pointers (memory of the
 *    GPU that is current when the context was created).  The caller owns every
 *    buffer it passes; the library never frees or retains them after a call.
 *  - Scalar outputs (rank_out, info, ...) are HOST pointers; they are written
 *    after the call has synchronised its stream.
 *  - All work is queued on the context's stream.  Device outputs are complete
 *    when the entry point returns (every solver entry point synchronises the
 *    stream, because its control flow depends on device-computed scalars).
 *  - Return value: 0 = success, < 0 = error (LYAP_ERR_*), > 0 = warning (the
 *    outputs hold the best result found).  lyap_last_error() gives detail.
 *  - There is no CPU fallback: every arithmetic step runs in this library's
 *    CUDA kernels.  A context on a machine without a usable GPU fails with
 *    LYAP_ERR_CUDA.
 *  - A context is not thread-safe; use one context per host thread / stream.
 */
#ifndef LIBLYAP_H
#define LIBLYAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LYAP_OK 0
#define LYAP_ERR_ARG (-1)        /* invalid argument (size, stride, null pointer, option) */
#define LYAP_ERR_NONFINITE (-2)  /* NaN/Inf in an input or produced by the iteration */
#define LYAP_ERR_SINGULAR (-3)   /* exactly zero pivot in an inversion */
#define LYAP_ERR_NOCONV (-4)     /* sign-Newton reached kmax without meeting its stop test */
#define LYAP_ERR_CAPACITY (-5)   /* output factor capacity too small; *rank_out = rank needed */
#define LYAP_ERR_TIMEOUT (-6)    /* a bounded device wait gave up */
#define LYAP_ERR_CUDA (-7)       /* CUDA runtime/driver error */
#define LYAP_ERR_NOMEM (-8)      /* device workspace allocation failed */
#define LYAP_WARN_STAGNATED 1    /* IR stopped by the stagnation rule, Eq. (4.2) */
#define LYAP_WARN_MAXIT 2        /* IR reached imax without meeting tau_ir */

/* Solver precisions u_s (Table 1.1); u = u_r = u_c = FP64 in this library. */
typedef enum { LYAP_FP64 = 0, LYAP_FP32 = 1, LYAP_FP16 = 2, LYAP_BF16 = 3 } lyap_prec_t;

/* Newton scaling (Sec. 3.1): Frobenius (the paper's choice, Sec. 4), determinantal, none,
 * 2-norm mu = (||A_k^-1||_2 / ||A_k||_2)^1/2 and spectral mu = (rho(A_k^-1) / rho(A_k))^1/2.
 * The last two are estimated on the GPU in FP32: the 2-norms by 12 power steps on M^T M,
 * the spectral radii by the geometric mean of ||M v|| / ||v|| over steps 13..24 of a power
 * iteration on M (a few per cent, which only steers the scaling). */
typedef enum {
  LYAP_SCALE_FROB = 0,
  LYAP_SCALE_DET = 1,
  LYAP_SCALE_NONE = 2,
  LYAP_SCALE_NORM2 = 3,
  LYAP_SCALE_SPECTRAL = 4
} lyap_scaling_t;

typedef struct lyap_ctx lyap_ctx_t;

/*
 * Algorithm parameters.  lyap_opts_default() sets the paper's values (Sec. 4.1):
 * tau_ir = n u, imax = kmax = 50, rho = 0.1, eta_s = 10 u, eta_r = 1e-4,
 * Frobenius scaling switched off once delta_k < 1e-2, stop test
 * ||A_k + I||_1 <= 10 sqrt(n u_s) (Eq. (3.4)), stagnation theta > 0.9 twice (Eq. (4.2)).
 */
typedef struct {
  int u_s;              /* lyap_prec_t: precision of the sign-Newton solver */
  int scaling;          /* lyap_scaling_t */
  double tau_newton;    /* <= 0: 10 sqrt(n u_s) */
  int newton_norm_fro;  /* 0: ||A_k + I||_1 (Eq. (3.4)); 1: ||A_k + I||_F */
  int stop_after;       /* the Newton loop ends at the stop_after-th iterate counted from,
                           and including, the first one meeting the stop test ("two more
                           iterations", Sec. 3.2; 2 reproduces Table 4.1's FP64 counts) */
  int delta_rule;       /* 1: also stop on delta_k > delta_{k-1}/2 once unscaled (Sec. 4) */
  double scale_off;     /* scaling is switched off for good once delta_k < scale_off (1e-2) */
  double rank_tol;      /* <= 0: sqrt(u_s) (Cholesky type) / u_s (LDL^T type), relative */
  double rho;           /* compress Z_k when cols(Z_k) > rho n; 0 = every step */
  int kmax;             /* Newton iteration limit */
  int imax;             /* refinement step limit */
  double tau_ir;        /* <= 0: n * 2^-53; bound on the relative residual of Eq. (4.1) */
  double eta_r;         /* residual truncation, relative to max |lambda(H)| */
  double eta_s;         /* <= 0: 10 * 2^-53; solution truncation, relative to max |sigma(K)| */
  double stag_theta;    /* stagnation ratio (0.9) */
  int stag_count;       /* consecutive stagnating steps that stop IR (2) */
  int project_psd;      /* 1: PSD projection in the solution update (forced off for indefinite S) */
  int profile;          /* 1: record per-phase device times into lyap_info_t.phase_ms (CUDA events) */
  int ckpt_every;       /* 0: the context keeps every inverse A_k^{-1} of the first solve (Sec. 3.4);
                           c > 0: it keeps only the iterates A_0, A_c, A_2c, ... (working
                           precision) and every later solve (corrections, adjoint) recomputes the
                           inverses from them with the recorded mu_k: one inversion per replayed
                           step in exchange for ceil(K / c) instead of K stored n x n matrices */
  int64_t mem_budget;   /* bytes the stored inverse sequence may take (0 = no limit); when kmax
                           stored inverses would exceed it, checkpoints every ckpt_every steps
                           (4 when ckpt_every = 0) are kept instead */
  int fp64_products;    /* FP64 matrix products of the refinement: 0 = library's choice (emulated
                           on the FP16 tensor cores above a size threshold), 1 = FP64 SIMT,
                           2 = always emulated (see lyap_dgemm) */
  int u, u_r, u_c;      /* lyap_prec_t of the working precision, of the residual and of the
                           solution update (Algorithms IR-Chol / IR-LDLT, Table 2.1): the
                           presets u = u_r = u_c = LYAP_FP64 (default) or LYAP_FP32; other
                           combinations return LYAP_ERR_ARG.  With FP32 the residual factors
                           and the updated solution factor are stored rounded to FP32 (their
                           products run in FP64), tau_ir and eta_s default to n u and 10 u of
                           FP32, and the attainable residual is near u = 2^-24 (Table 2.1's
                           u = fp32 rows).  The adjoint accepts FP64 only */
  int inner;            /* lyap_inner_t: inner solver of the refinement (and of lyap_sign_solve) */
  int adi_shifts;       /* low-rank ADI: number of cyclic real shifts (<= 0: 8; at most kmax) */
  int adi_maxit;        /* low-rank ADI: step limit per solve (<= 0: 200) */
  double adi_tol;       /* low-rank ADI and extended Krylov: stop once the residual of the inner
                           solve is <= adi_tol ||L S L^T||_F (<= 0: max(10 u_s, 1e-14)) */
  int eksm_maxit;       /* extended Krylov: block steps per solve (<= 0: 60) */
  int reserved2;
} lyap_opts_t;

/*
 * Inner solvers.  LYAP_INNER_SIGN: the scaled sign-function Newton iteration (Sec. 3).
 * LYAP_INNER_ADI: low-rank ADI (Sec. 5 names ADI-based solvers as alternatives inside the
 * same refinement framework; no counterpart in the paper's experiments) with real cyclic
 * shifts p_j = -b (a/b)^((2j-1)/(2 adi_shifts)), a = 1/||A^-1||_2 and b = ||A||_2 estimated
 * by power iteration: V_j = (A + p_j I)^-1 W_{j-1}, W_j = W_{j-1} - 2 p_j V_j (W_0 = L),
 * Z_j = [Z_{j-1}, sqrt(-2 p_j) V_j] (Cholesky) or [Z_{j-1}, V_j] with weights -2 p_j S
 * (LDL^T), so that the residual of Z_j is W_j S W_j^T.  The shifted inverses are computed
 * once at u_s (the GJ inversion, 16-bit storage) and every correction solve reuses them,
 * as the sign-Newton sequence (Sec. 3.4).  Real shifts suit spectra near the real axis;
 * eigenvalues with |Im| >> |Re| converge slowly.  Checkpointing does not apply (the
 * adi_shifts inverses are always stored).  In lyap_info_t the inner counts (newton_*) and
 * n_inversions count the stored shifted inverses, and mu[j] holds the shift p_j (of the
 * power-of-two prescaled A).
 */
typedef enum { LYAP_INNER_SIGN = 0, LYAP_INNER_ADI = 1, LYAP_INNER_EKSM = 2 } lyap_inner_t;
/*
 * LYAP_INNER_EKSM: the extended Krylov (Galerkin) method, the Krylov alternative Sec. 5
 * names (no counterpart in the paper's experiments): V spans {L, A^-1 L, A L, A^-2 L, ...}
 * in orthonormal blocks of 2m columns (A^-1 computed once at u_s and stored, products with
 * A in the working precision of u_s), the projected equation V^T A V Y + Y V^T A^T V + V^T L S
 * L^T V = 0 is solved by the FP64 sign-Newton solver on an internal context (V^T A V must be
 * stable: A + A^T < 0 guarantees it), X = V Y V^T, and the iteration stops when
 * sqrt(2) ||U_next^T A V Y||_F (its residual norm) is <= adi_tol ||L S L^T||_F, on breakdown
 * of the next block, or after eksm_maxit blocks.  The stored A^-1 serves every correction
 * solve and the adjoint.  n_inversions counts the one stored inverse.
 */

/* Phases reported in lyap_info_t.phase_ms / phase_calls / phase_flops when
 * opts.profile = 1 (LYAP_NUM_PHASES slots; the unused ones stay zero). */
enum {
  LYAP_PHASE_INVERT = 0,   /* n x n inversions (panel + trailing-update kernels) */
  LYAP_PHASE_NEWTON = 1,   /* Newton scalar/epilogue kernels (scaling, A_{k+1}, stop test) */
  LYAP_PHASE_FACTOR = 2,   /* factor products A_k^{-1} Z_k and their scaling */
  LYAP_PHASE_COMPRESS = 3, /* rank truncation inside the Newton iteration */
  LYAP_PHASE_RESFAC = 4,   /* residual factorisation without its eigensolver (A Z, QR, core matrix) */
  LYAP_PHASE_EIG = 5,      /* FP32 Jacobi stage of the symmetric eigensolver */
  LYAP_PHASE_SOLUPT = 6,   /* projected solution update without its eigensolver */
  LYAP_PHASE_OTHER = 7,
  LYAP_PHASE_EIG_REFINE = 8 /* FP64 refinement stage of the symmetric eigensolver */
};
#define LYAP_NUM_PHASES 12

typedef struct {
  int status;           /* same value as returned */
  int rank;             /* columns of the returned factor */
  int ir_steps;         /* refinement steps performed (corrections applied) */
  int newton_calls;     /* calls of the sign-Newton solver (first solve + corrections) */
  int newton_total;     /* total Newton iterations over all calls (varsigma, Table 4.1) */
  int newton_max;       /* maximum Newton iterations in one call (alpha) */
  int n_inversions;     /* distinct n x n inversions computed (stored and replayed, Sec. 3.4) */
  int stagnated;        /* stagnation rule fired */
  int converged;        /* relative residual <= tau_ir */
  int n_res;            /* entries used in res_hist */
  double res_final;     /* relative residual (Eq. (4.1)) of the returned factor */
  double res_hist[64];  /* relative residual before each refinement step */
  double mu[64];        /* Newton scaling parameters mu_0, mu_1, ... */
  int64_t kernel_launches; /* CUDA kernels launched by this call */
  double device_ms;     /* device time of the call (CUDA events on the context stream) */
  double phase_ms[LYAP_NUM_PHASES];    /* per-phase device time (opts.profile = 1), LYAP_PHASE_* */
  int64_t phase_calls[LYAP_NUM_PHASES];/* intervals timed per phase */
  double phase_flops[LYAP_NUM_PHASES]; /* algorithmic flops per phase: 2 n^3 per inversion;
                                          9 q^3 per FP32 Jacobi eigendecomposition (the
                                          symmetric QR count with eigenvectors, Golub-Van Loan);
                                          2 m n k per FP64 GEMM of the refinement */
} lyap_info_t;

/* Fill *o with the paper's defaults (u_s = FP16).  Returns LYAP_OK. */
int lyap_opts_default(lyap_opts_t* o);

/* Create a context bound to the current CUDA device and `stream` (a cudaStream_t,
 * NULL = legacy default stream).  The context owns its device workspace and the
 * stored inverse sequence; both grow on demand and are freed by lyap_ctx_destroy. */
int lyap_ctx_create(lyap_ctx_t** ctx, void* stream);
int lyap_ctx_destroy(lyap_ctx_t* ctx);
/* Rebind the context to another stream (pending work is not synchronised). */
int lyap_ctx_set_stream(lyap_ctx_t* ctx, void* stream);

/*
 * One sign-function Newton solve at precision opts->u_s (Sec. 3.2: the
 * Cholesky-type iteration Eq. (3.2) when S == NULL, the LDL^T-type iteration
 * Eq. (3.3) otherwise), with rank truncation (RankTruncChol / RankTruncLdlt).
 *   A      n x n, lda >= n               (A must be Hurwitz)
 *   L      n x m, ldl >= n
 *   S      m x m symmetric, lds >= m, or NULL (W = L L^T)
 *   Z      n x z_cap output, ldz >= n: X ~= Z Z^T (Cholesky) or Z diag(D) Z^T
 *   D      z_cap output (LDL^T only; ignored when S == NULL; may be NULL then)
 *   *rank_out  columns written to Z (on LYAP_ERR_CAPACITY: columns needed)
 * The computed inverse sequence {A_k^{-1}, mu_k} is kept in the context (Sec. 3.4).
 */
int lyap_sign_solve(lyap_ctx_t* ctx, const double* A, int64_t n, int64_t lda,
                    const double* L, int64_t ldl, int64_t m, const double* S, int64_t lds,
                    const lyap_opts_t* opts, double* Z, int64_t ldz, int64_t z_cap,
                    double* D, int64_t* rank_out, lyap_info_t* info);

/*
 * Mixed-precision iterative refinement: Algorithm IR-Chol (Sec. 2.1) when S == NULL,
 * Algorithm IR-LDLT (Sec. 2.3) otherwise, with the sign-Newton solver at u_s,
 * the residual factorisation (Fragments ResFacChol / ResFacLdlt) and the projected
 * solution update (Fragments SolUptChol / SolUptLdlt) in FP64, and the stopping
 * rules of Sec. 4.1.  Every correction solve replays the stored inverse sequence
 * of the first solve (Sec. 3.4).  Arguments as for lyap_sign_solve.
 */
int lyap_solve_ir(lyap_ctx_t* ctx, const double* A, int64_t n, int64_t lda,
                  const double* L, int64_t ldl, int64_t m, const double* S, int64_t lds,
                  const lyap_opts_t* opts, double* Z, int64_t ldz, int64_t z_cap,
                  double* D, int64_t* rank_out, lyap_info_t* info);

/*
 * Many independent Cholesky-type refinements (Algorithm IR-Chol) in one call, for
 * batches of small equations A_e X_e + X_e A_e^T + L_e L_e^T = 0 of uneven order: the
 * equations run concurrently on `workers` internal contexts (each with its own
 * non-blocking stream and host thread; <= 0 selects 8), largest n first.  Each equation
 * is solved exactly as by lyap_solve_ir with the same opts.
 *   A, L, Z    HOST arrays of nb DEVICE pointers: A[e] (n[e] x n[e]), L[e] (n[e] x m[e]),
 *              Z[e] (n[e] x z_cap[e]); leading dimensions equal n[e]; column-major FP64
 *   n, m, z_cap HOST arrays of nb sizes;  rank_out HOST array of nb ranks
 *   info       optional HOST array of nb lyap_info_t, or NULL
 * The call waits for the context stream first (inputs ready) and returns after every
 * solve has finished.  Returns LYAP_OK, the first negative status of any equation (the
 * others are still solved; lyap_last_error names the equation), or else the first warning.
 */
int lyap_solve_ir_batched(lyap_ctx_t* ctx, int nb, const double* const* A, const int64_t* n,
                          const double* const* L, const int64_t* m, const lyap_opts_t* opts,
                          double* const* Z, const int64_t* z_cap, int64_t* rank_out,
                          lyap_info_t* info, int workers);

/*
 * Adjoint of the solve (no counterpart in the paper; it follows from differentiating
 * Eq. (1.1)): gradients of the loss l = trace(C X C^T), X = Z diag(D) Z^T (D == NULL:
 * X = Z Z^T), the solution of A X + X A^T + L S L^T = 0 (S == NULL: S = I).
 * With Y solving the adjoint equation A^T Y + Y A + C^T C = 0,
 *   dl/dA = 2 Y X (n x n),  dl/dL = 2 Y L S (n x m),  dl/dS = L^T Y L (m x m),  dl/dW = Y.
 * Y = Zy Zy^T is computed by the mixed-precision refinement of lyap_solve_ir (precisions
 * and tolerances from opts).  When the context still holds the inverse sequence of this
 * A (the last lyap_solve_ir / lyap_sign_solve on it, same u_s, recognised by a device
 * fingerprint of A), every Newton solve replays it transposed -- the sign-Newton
 * sequence of A^T is (A_k^{-1})^T with the same mu_k -- and no inversion is computed
 * (info->n_inversions = 0); otherwise the sequence of A^T is computed and stored.
 *   A (n x n, lda), L (n x m, ldl), S (m x m, lds, or NULL), Z (n x r, ldz), D (r or NULL):
 *              the forward problem and its solution factor, DEVICE, column-major FP64
 *   Cm         q x n (ldc >= q), DEVICE: the loss matrix C
 *   dA, dL, dS optional DEVICE outputs (NULL to skip), leading dimensions as named
 *   Zy         optional DEVICE output n x zy_cap (ldzy): the adjoint factor; *rank_y its
 *              column count (required with Zy; LYAP_ERR_CAPACITY if zy_cap is too small)
 *   info       as for lyap_solve_ir, describing the adjoint refinement
 * Returns as lyap_solve_ir (warnings > 0 still produce gradients from the best Zy).
 */
int lyap_adjoint(lyap_ctx_t* ctx, const double* A, int64_t n, int64_t lda,
                 const double* L, int64_t ldl, int64_t m, const double* S, int64_t lds,
                 const double* Z, int64_t ldz, int64_t r, const double* D,
                 const double* Cm, int64_t ldc, int64_t q, const lyap_opts_t* opts,
                 double* dA, int64_t ldda, double* dL, int64_t lddl, double* dS, int64_t ldds,
                 double* Zy, int64_t ldzy, int64_t zy_cap, int64_t* rank_y, lyap_info_t* info);

/*
 * Relative residual of Eq. (4.1),
 *   ||A X + X A^T + W||_F / (||W||_F + 2 ||X||_F ||A||_F),  X = Z Z^T or Z diag(D) Z^T,
 * evaluated in FP64 from the factors without forming n x n matrices (thin QR of
 * [Z, AZ, L] and the Frobenius norm of the small core, as in Fragment ResFacChol).
 * D == NULL means X = Z Z^T; S == NULL means W = L L^T.  *res_out is a host double.
 */
int lyap_residual(lyap_ctx_t* ctx, const double* A, int64_t n, int64_t lda,
                  const double* L, int64_t ldl, int64_t m, const double* S, int64_t lds,
                  const double* Z, int64_t ldz, int64_t r, const double* D, double* res_out);

/*
 * The loss of the differentiable solve and its gradient in C (no counterpart in the
 * paper: the loss l = trace(C X C^T) is the one the adjoint entry point differentiates):
 *   *loss = trace(C X C^T) = sum_j D_j ||C z_j||^2,   dC = dl/dC = 2 C X  (q x n, lddc),
 * X = Z diag(D) Z^T (D == NULL: X = Z Z^T), in FP64 from the factor (C Z, no n x n matrix).
 *   Z (n x r, ldz), D (r or NULL), Cm (q x n, ldc): DEVICE, column-major FP64
 *   loss  HOST double;  dC optional DEVICE output (NULL to skip)
 * Returns LYAP_OK or LYAP_ERR_ARG / LYAP_ERR_CUDA / LYAP_ERR_NOMEM.
 */
int lyap_trace_loss(lyap_ctx_t* ctx, const double* Z, int64_t n, int64_t ldz, int64_t r, const double* D,
                    const double* Cm, int64_t ldc, int64_t q, double* loss, double* dC, int64_t lddc);

/*
 * kappa_sign(B) in the Frobenius norm for B = [[A, W], [0, -A^T]], W = L L^T (S == NULL)
 * or L S L^T: the condition of the matrix sign function that the sign-Newton iteration
 * computes (sign(B) = [[-I, 2X], [0, I]]), the indicator Sec. 4.2 uses for the accuracy of
 * the Newton solver.  An FP64 Newton iteration on B (order 2n, Frobenius scaling) keeps its
 * inverses; the Frechet derivative L(B, E) is the derivative of that iteration and its
 * adjoint uses the transposed inverses; ||L||_F is estimated by power_steps (1..100) steps
 * of the power method on L^* L from a fixed pseudo-random start (a lower bound, typically
 * within a few per cent).  Out (host): *kappa = ||L||_F ||B||_F / ||sign(B)||_F; *lnorm =
 * ||L||_F (may be NULL); *newton_steps = iterations on B (may be NULL).  A, L, S: device,
 * column-major, as lyap_solve_ir.  Workspace: about (K + 5) (2n)^2 doubles (K Newton
 * steps), allocated and freed by the call (LYAP_ERR_NOMEM when it does not fit); n <= 16384.
 * Cost: K inversions of order 2n and 4 K power_steps FP64 products of order 2n.
 */
int lyap_kappa_sign(lyap_ctx_t* ctx, const double* A, int64_t n, int64_t lda, const double* L, int64_t ldl,
                    int64_t m, const double* S, int64_t lds, int power_steps, double* kappa, double* lnorm,
                    int* newton_steps);

/*
 * FP64 matrix product C = alpha op(A) op(B) + beta C (op = 'N' or 'T'; column-major DEVICE
 * operands, beta == 0 does not read C): the products of the FP64 steps of the method -- A Z and
 * the core matrices T P T^T, Gamma J Gamma^T of Fragments ResFacChol / SolUptChol (Sec. 2.1),
 * the Gram matrices of Eq. (4.1), the eigen-refinement products.
 *   method 1: FP64 SIMT arithmetic.
 *   method 2: emulated on the FP16 tensor cores (no counterpart in the paper): every row of
 *             op(A) and column of op(B) is scaled by a power of two and cut into 8 digits of
 *             7 bits; digit products are exact in the FP32 accumulators (K in chunks of 1024)
 *             and the 36 leading pairs are summed in FP64.  Error about 2^-50 K max|a| max|b|
 *             per entry (row / column maxima), the order of an FP64 product's bound.
 *   method 0: 2 for products of at least 3e7 multiply-adds with k >= 128 and at least 48
 *             (output tile of 128 x 32, K range) pairs -- outputs of fewer than 74 tiles split
 *             K into up to 16 ranges of at least 256, summed in a fixed order -- 1 otherwise.
 * Synchronises the context stream; returns LYAP_ERR_TIMEOUT if a bounded device wait gave up.
 */
int lyap_dgemm(lyap_ctx_t* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
               int method);

/*
 * Dense inversion behind every Newton step (Sec. 3.3 cost model: 2 n^3 flops):
 * blocked Gauss-Jordan elimination with partial pivoting -- the getrf pivot
 * sequence (largest |a_ij| in the active column, lowest row on ties) fused with
 * the getri inversion -- at precision `prec` (FP64 / FP32 SIMT, FP16 / BF16
 * operands on tcgen05 tensor cores with FP32 accumulation and an FP32 working matrix).
 *   Ainv   n x n output, ldai >= n (may not alias A)
 *   ipiv   optional DEVICE int32[n]: row chosen as pivot at step j (0-based), or NULL
 *   logabsdet optional HOST double: log|det A| from the pivots, or NULL
 */
int lyap_invert(lyap_ctx_t* ctx, const double* A, int64_t n, int64_t lda, int prec,
                double* Ainv, int64_t ldai, int32_t* ipiv, double* logabsdet);

/*
 * lyap_invert without any device allocation (the paper has no counterpart: this entry
 * point serves callers that may not allocate device memory at all -- code running
 * under a fixed, pre-reserved memory budget, or inside a framework whose allocator
 * must not see foreign cudaMalloc/cudaFree calls).  Same operation, kernels and
 * results as lyap_invert at prec LYAP_FP64 or LYAP_FP32, for n <= LYAP_NOALLOC_MAX_N.
 *   A, Ainv, ipiv  DEVICE pointers as in lyap_invert (ipiv may be NULL)
 *   logabsdet      optional HOST double, or NULL
 *   stream         cudaStream_t to run on (NULL = legacy default stream)
 * Workspace: one static __device__ array of about 4.4 MiB inside this library,
 * sized for n = LYAP_NOALLOC_MAX_N in FP64; its address is looked up once per
 * device, with that device current, on the first call made on that device.  The
 * call synchronizes `stream` to read the status word and log|det|, so it cannot
 * be captured into a CUDA graph.  Calls on the same device share the workspace:
 * they must not overlap (serialize them on one stream or host thread).
 * Errors: LYAP_ERR_ARG for n > LYAP_NOALLOC_MAX_N, another prec, bad sizes or
 * NULL pointers (nothing is launched); otherwise as lyap_invert.
 */
#define LYAP_NOALLOC_MAX_N 512
int lyap_invert_noalloc(const double* A, int64_t n, int64_t lda, int prec, double* Ainv,
                        int64_t ldai, int32_t* ipiv, double* logabsdet, void* stream);

/*
 * RankTruncChol (Sec. 3.2): QR with column pivoting of Z^T, truncated at the first
 * r with ||S_r||_F <= tol * |r_11|, returned as Pi [T C]^T (n x r), overwriting the
 * leading r columns of Z (FP64 arithmetic).  *rank_out receives r.
 */
int lyap_rank_trunc(lyap_ctx_t* ctx, double* Z, int64_t n, int64_t c, int64_t ldz, double tol,
                    int64_t* rank_out);

/*
 * Symmetric eigendecomposition H = Q diag(w) Q^T of a q x q FP64 matrix (the kernel
 * behind Fragments ResFacChol / SolUptChol): H (ldh >= q, overwritten), w (q, ascending),
 * Q (q x q, ldq >= q).  All device pointers.  fp64_refine = 1 refines the eigenpairs
 * to FP64 accuracy; 0 returns the FP32-accurate result.  Up to order 1280 one block
 * Jacobi launch (one CTA per pair of 8-index blocks, all resident: q / 16 CTAs, twice
 * that when the GPU has the SMs); above it Jacobi over super-blocks of at most 512
 * indices whose pairs that kernel diagonalises (FP32 products update the rest), then the
 * same refinement.  Orders above 32768 return LYAP_ERR_ARG before any launch.  Scratch
 * grows to about 18 q^2 floats for q > 1280.
 */
int lyap_sym_eig(lyap_ctx_t* ctx, double* H, int64_t q, int64_t ldh, double* w, double* Q,
                 int64_t ldq, int fp64_refine);

/* Message of the last error raised on the calling host thread (thread-local storage). */
const char* lyap_last_error(void);
/* Human-readable name of a status code. */
const char* lyap_status_string(int status);
/* Library version string. */
const char* lyap_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBLYAP_H */
