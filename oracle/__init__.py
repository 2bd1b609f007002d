"""CPU FP64 oracle for mixed-precision iterative refinement of low-rank Lyapunov equations.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the method of Benner & Liu, "Mixed-precision
iterative refinement for low-rank Lyapunov equations" (arXiv 2510.02126), written
with numpy/scipy library primitives (matrix product, inverse, QR, QR with column
pivoting, symmetric eigendecomposition, complex Schur form, triangular solve).
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline /
reference legs may import it.  The CUDA library never calls it and shares no
code with it; the only code both sides use is the seeded input generator module
``lyapgen``, which holds none of the method's arithmetic.

Functions and the passages they follow:

* ``bartels_stewart``      -- exact solution X of Eq. (1.1) (Schur-based direct method)
* ``newton_chol``          -- Algorithm "sign function Newton, Cholesky type" (Sec. 3.2, Eq. (3.2))
* ``newton_ldlt``          -- Algorithm "sign function Newton, LDL^T type" (Sec. 3.2, Eq. (3.3))
* ``rank_trunc_chol``/``rank_trunc_ldlt`` -- their truncation sub-functions
* ``res_fac_chol``/``sol_upt_chol``       -- Fragments ResFacChol / SolUptChol (Sec. 2.1)
* ``res_fac_ldlt``/``sol_upt_ldlt``       -- Fragments ResFacLdlt / SolUptLdlt (Sec. 2.3)
* ``ir_chol``/``ir_ldlt``                 -- the two IR algorithms (Sec. 2.1, 2.3) with the
  stopping rules of Sec. 4.1 (Eq. (4.2))
* ``residual_eq41``        -- relative residual of Eq. (4.1), explicit n x n formation
* ``adjoint``              -- gradient of trace(C X C^T) (not in the paper; derived from Eq. (1.1))
* ``getrf_pp``             -- LU with partial pivoting (the factorisation behind the inversions)
* ``newton_sequence``      -- the scaled Newton iteration with the scalings of Sec. 3.1
  (Frobenius, determinantal, 2-norm, spectral)
* ``lr_adi_chol``/``lr_adi_ldlt``/``adi_record`` -- low-rank ADI with real cyclic shifts as
  the alternative inner solver (Sec. 5 names ADI-based solvers inside the same refinement
  framework; ``Opts.inner = "adi"`` in ``ir_chol``/``ir_ldlt``)
* ``eksm_chol``/``eksm_ldlt`` -- the extended Krylov (Galerkin) method as the Krylov
  alternative inner solver (``Opts.inner = "eksm"``)
* ``sign_block``/``sign_matrix``/``frechet_sign``/``kappa_sign_fro`` -- sign(B) of
  B = [[A, W], [0, -A^T]], its Frechet derivative and kappa_sign(B) in the Frobenius norm,
  the indicator Sec. 4.2 uses to explain the accuracy of the Newton solver

Pins (tests/test_oracle_*.py) tie every function to something other than itself:
the Kronecker form Eq. (2.1) solved densely, closed forms for diagonal and
sine-basis-diagonalisable A, Schur-known normal A, LAPACK's Lyapunov routine,
the invariants X = X^T, X >= 0, sign(A) = -I, and Table 4.1's FP64 iteration counts.
Parity of intermediate reduced-precision iterates is unpinned (the paper rounds
every scalar operation; this oracle rounds every matrix operation).
"""
from .lyap_oracle import *  # noqa: F401,F403
