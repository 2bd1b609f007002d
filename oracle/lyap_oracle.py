"""Plain CPU FP64 restatement of the paper's method (test infrastructure only).

See the package docstring for the list of functions and the passages they follow.
Every routine here is written for readability: one library primitive per step of
the paper, no blocking, fusion or reordering beyond what the paper states.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np
import scipy.linalg as sla

__all__ = [
    "UNIT", "Opts", "rnd", "bartels_stewart", "getrf_pp", "rank_trunc_chol", "rank_trunc_ldlt",
    "newton_sequence", "NewtonRecord", "IRInfo", "newton_chol", "newton_ldlt", "res_fac_chol", "sol_upt_chol", "res_fac_ldlt", "sol_upt_ldlt",
    "ir_chol", "ir_ldlt", "residual_eq41", "adjoint", "norm_xyx", "lyap_operator_kappa2_normal",
    "sign_block", "sign_matrix", "frechet_sign", "kappa_sign_fro",
    "ADIRecord", "adi_shifts", "adi_record", "lr_adi_chol", "lr_adi_ldlt",
    "EKSMRecord", "eksm_chol", "eksm_ldlt",
]

# Unit roundoffs of Table 1.1 (t significand bits incl. the implicit bit: u = 2^-t).
UNIT = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "fp32": 2.0 ** -24, "fp64": 2.0 ** -53}


def _round_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP64 -> bf16 (8-bit significand, round to nearest even) -> FP64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    out = b.astype(np.uint32).view(np.float32).astype(np.float64)
    # keep NaN/Inf as they are
    bad = ~np.isfinite(f)
    if np.any(bad):
        out = np.where(bad, f.astype(np.float64), out)
    return out


def rnd(x, prec: str):
    """Round every entry of ``x`` to precision ``prec`` and return it as FP64.

    This is the oracle's model of "performed at precision u_s": the result of each
    matrix operation is rounded once (the paper simulates bf16 by rounding each
    scalar operation, Sec. 4; the two agree to first order).
    """
    if prec == "fp64":
        return np.asarray(x, dtype=np.float64)
    if prec == "fp32":
        return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    if prec == "fp16":
        # fp16 has 5 exponent bits (Table 1.1): every matrix is brought into range by an
        # exact power-of-two factor before rounding and scaled back afterwards.
        x = np.asarray(x, dtype=np.float64)
        amax = float(np.max(np.abs(x))) if x.size else 0.0
        if not np.isfinite(amax) or amax == 0.0:
            return x.astype(np.float16).astype(np.float64)
        e = math.floor(math.log2(amax))
        return np.ldexp(np.ldexp(x, -e).astype(np.float16).astype(np.float64), e)
    if prec == "bf16":
        return _round_bf16(x)
    raise ValueError(prec)


@dataclass
class Opts:
    """Algorithm parameters; defaults are the paper's (Sec. 4.1)."""
    u_s: str = "fp64"              # solver precision (Algorithms IR-Chol / IR-LDLT)
    u: str = "fp64"                # working precision = u_r = u_c (Table 2.1: fp64 or fp32); the
                                   # residual factors and the updated solution factor are
                                   # stored (rounded) in u
    scaling: str = "frob"          # "frob" (Sec. 4, chosen), "det", "norm2", "spectral", "none"
                                   # (the scalings listed in Sec. 3.1)
    tau_newton: float = 0.0        # <= 0: 10 sqrt(n u_s)  (Eq. (3.4))
    newton_norm: str = "one"       # "one": ||A_k + I||_1 (Eq. (3.4)); "fro": ||A_k + I||_F
    stop_after: int = 2            # "two more iterations" (Sec. 3.2): the iteration ends at the
                                   # stop_after-th iterate counted from, and including, the first
                                   # one that meets the test; this reading reproduces every FP64
                                   # iteration count of Table 4.1
    delta_rule: bool = True        # Higham's roundoff indicator delta_k > delta_{k-1}/2 (Sec. 4)
    scale_off: float = 1e-2        # stop scaling once delta_k < 1e-2 (Sec. 4)
    rank_tol: float = 0.0          # <= 0: sqrt(u_s) (Chol) / u_s (LDL^T) (Sec. 3.2 sub-functions)
    rho: float = 0.1               # truncate when cols(Z) > rho n; 0 = every step (Sec. 4.1)
    kmax: int = 50
    imax: int = 50
    tau_ir: float = 0.0            # <= 0: n u (u = fp64), on the relative residual Eq. (4.1)
    eta_r: float = 1e-4            # residual truncation, relative to max |lambda| (Sec. 4.1)
    eta_s: float = 0.0             # <= 0: 10 u; solution truncation relative to max sigma
    stag_theta: float = 0.9        # Eq. (4.2)
    stag_count: int = 2
    project_psd: bool = True       # SolUpt projection onto the PSD cone (Sec. 2.1)
    inner: str = "sign"            # inner solver: "sign" (Sec. 3), "adi" (low-rank ADI) or "eksm"
                                   # (extended Krylov): the alternatives Sec. 5 names
    adi_shifts: int = 8            # number of cyclic real shifts
    adi_tol: float = 0.0           # <= 0: max(10 u_s, 1e-14); ||W S W^T||_F <= tol ||L S L^T||_F
    adi_maxit: int = 200
    eksm_maxit: int = 60           # extended Krylov: block steps per solve (tolerance: adi_tol)


def _u(prec: str) -> float:
    return UNIT[prec]


# ---------------------------------------------------------------------------
# Exact solution: Schur-based direct method (Bartels-Stewart), Eq. (1.1)
# ---------------------------------------------------------------------------

def bartels_stewart(A: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Solve A X + X A^T + W = 0 in FP64 by the Schur method.

    A = Q T Q^H (complex Schur form), W~ = Q^H W Q, then T X~ + X~ T^H = -W~ is
    solved one column at a time from the last: column j satisfies
    (T + conj(t_jj) I) x_j = -w~_j - sum_{l>j} conj(t_jl) x_l, an upper triangular
    system.  X = Q X~ Q^H (real part).
    """
    A = np.asarray(A, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    n = A.shape[0]
    T, Q = sla.schur(A, output="complex")
    Wt = Q.conj().T @ W @ Q
    Xt = np.zeros((n, n), dtype=np.complex128)
    I = np.eye(n)
    for j in range(n - 1, -1, -1):
        rhs = -Wt[:, j]
        if j + 1 < n:
            rhs = rhs - Xt[:, j + 1:] @ np.conj(T[j, j + 1:])
        Xt[:, j] = sla.solve_triangular(T + np.conj(T[j, j]) * I, rhs, lower=False)
    X = Q @ Xt @ Q.conj().T
    return X.real.copy()


def lyap_operator_kappa2_normal(eigs: np.ndarray) -> float:
    """2-norm condition number of L(X) = AX + XA^T for NORMAL A with eigenvalues ``eigs``.

    The operator is normal with eigenvalues l_i + l_j, so kappa_2 = max|l_i+l_j| / min|l_i+l_j|.
    """
    s = np.abs(eigs[:, None] + eigs[None, :])
    return float(s.max() / s.min())


# ---------------------------------------------------------------------------
# LU with partial pivoting (the factorisation behind every Newton inversion)
# ---------------------------------------------------------------------------

def getrf_pp(A: np.ndarray):
    """Unblocked right-looking LU with partial pivoting: P A = L U.

    Pivot = first row of maximal |a_ij| in the active column (lowest index on ties).
    Returns (LU packed, perm) with perm[i] = original row now at position i, and the
    list of pivot rows chosen at each step (LAPACK ipiv convention, 0-based).
    """
    U = np.array(A, dtype=np.float64, copy=True)
    n = U.shape[0]
    perm = np.arange(n)
    ipiv = np.zeros(n, dtype=np.int64)
    for j in range(n):
        p = j + int(np.argmax(np.abs(U[j:, j])))
        ipiv[j] = p
        if p != j:
            U[[j, p], :] = U[[p, j], :]
            perm[[j, p]] = perm[[p, j]]
        if U[j, j] == 0.0:
            continue
        U[j + 1:, j] /= U[j, j]
        U[j + 1:, j + 1:] -= np.outer(U[j + 1:, j], U[j, j + 1:])
    return U, perm, ipiv


# ---------------------------------------------------------------------------
# Sign-function Newton iterations, Sec. 3
# ---------------------------------------------------------------------------

def rank_trunc_chol(Z: np.ndarray, tol: float):
    """Sub-function RankTruncChol (Sec. 3.2): QR with column pivoting of Z^T.

    Z^T Pi = Q [[T, C], [0, S]]; the kept rank r is the smallest index whose trailing
    block satisfies ||S||_F <= tol * |r_11|.  Since ||S||_2 <= ||S||_F and
    |r_11| <= ||Z||_2 this implies the paper's ||S||_2 <= tol ||Z||_2.
    Returns Pi [T C]^T (n x r), which satisfies Z Z^T ~= Pi [T C]^T [T C] Pi^T.
    """
    n, c = Z.shape
    if c == 0:
        return Z.copy()
    R, piv = sla.qr(Z.T, mode="r", pivoting=True)
    k = min(c, n)
    R = R[:k, :]
    # ||R[j:, j:]||_F^2 = sum_{i >= j} ||R[i, :]||^2 (R is upper trapezoidal)
    rows = np.sum(R ** 2, axis=1)
    tail = np.sqrt(np.concatenate([np.cumsum(rows[::-1])[::-1], [0.0]]))
    r11 = abs(R[0, 0])
    r = k
    for j in range(1, k + 1):
        if tail[j] <= tol * r11:
            r = j
            break
    Zt = np.zeros((n, r))
    Zt[piv, :] = R[:r, :].T
    return Zt


def rank_trunc_ldlt(Z: np.ndarray, y: np.ndarray, tol: float):
    """Sub-function RankTruncLdlt (Sec. 3.2): thin QR Z = QR, eig of R Y R^T.

    Keeps |lambda_i| > tol * max|lambda| (magnitude, so that indefinite Y keeps its
    negative part); returns (Q V_t, lambda_t).
    """
    if Z.shape[1] == 0:
        return Z.copy(), y.copy()
    Q, R = np.linalg.qr(Z)
    M = (R * y[None, :]) @ R.T
    lam, V = np.linalg.eigh(M)
    lmax = np.max(np.abs(lam))
    keep = np.abs(lam) > tol * lmax
    return Q @ V[:, keep], lam[keep]


@dataclass
class NewtonRecord:
    """The coefficient sequence of one sign-Newton run (depends on A only, Sec. 3.4)."""
    inverses: list = field(default_factory=list)   # A_{k-1}^{-1}, k = 1..K
    mus: list = field(default_factory=list)        # mu_{k-1}
    stop_measure: list = field(default_factory=list)
    deltas: list = field(default_factory=list)
    A_final: np.ndarray | None = None


def newton_sequence(A: np.ndarray, opts: Opts) -> NewtonRecord:
    """The matrix part of the scaled sign-function Newton iteration, Eq. (3.1a).

    A_k = (mu_{k-1} A_{k-1} + mu_{k-1}^{-1} A_{k-1}^{-1}) / 2 with
      Frobenius scaling mu = (||A^{-1}||_F / ||A||_F)^{1/2},
      determinantal scaling mu = |det A|^{-1/n} (evaluated from the LU diagonal in
      logarithms, since the determinant itself over/underflows, Sec. 4),
      2-norm scaling mu = (||A^{-1}||_2 / ||A||_2)^{1/2}, or
      spectral scaling mu = (rho(A^{-1}) / rho(A))^{1/2} (rho: spectral radius); Sec. 3.1.
    Scaling is switched off for good once delta_k = ||A_k - A_{k-1}||_F / ||A_k||_F < 1e-2.
    The stop test is ||A_k + I|| <= tau_N (Eq. (3.4)) or, once scaling is off,
    delta_k > delta_{k-1}/2 (Sec. 4); the iteration ends at the second iterate counted
    from the first one that meets it (``Opts.stop_after``).
    Every matrix result is rounded to u_s.
    """
    n = A.shape[0]
    p = opts.u_s
    tau = opts.tau_newton if opts.tau_newton > 0 else 10.0 * math.sqrt(n * _u(p))
    rec = NewtonRecord()
    Ak = rnd(A, p)
    scaling_on = opts.scaling != "none"
    fired = 0
    delta_prev = None
    prev_unscaled = False
    I = np.eye(n)
    for k in range(1, opts.kmax + 1):
        Xk = rnd(np.linalg.inv(Ak), p)
        if scaling_on and opts.scaling == "frob":
            mu = math.sqrt(np.linalg.norm(Xk, "fro") / np.linalg.norm(Ak, "fro"))
        elif scaling_on and opts.scaling == "det":
            lu, _, _ = getrf_pp(Ak)
            mu = math.exp(-np.sum(np.log(np.abs(np.diag(lu)))) / n)
        elif scaling_on and opts.scaling == "norm2":
            mu = math.sqrt(np.linalg.norm(Xk, 2) / np.linalg.norm(Ak, 2))
        elif scaling_on and opts.scaling == "spectral":
            mu = math.sqrt(np.max(np.abs(np.linalg.eigvals(Xk))) / np.max(np.abs(np.linalg.eigvals(Ak))))
        else:
            mu = 1.0
        Anew = rnd(0.5 * (mu * Ak + Xk / mu), p)
        rec.inverses.append(Xk)
        rec.mus.append(mu)
        delta = np.linalg.norm(Anew - Ak, "fro") / np.linalg.norm(Anew, "fro")
        rec.deltas.append(delta)
        E = Anew + I
        meas = np.linalg.norm(E, 1) if opts.newton_norm == "one" else np.linalg.norm(E, "fro")
        rec.stop_measure.append(meas)
        this_unscaled = (mu == 1.0)
        Ak = Anew
        if fired == 0:
            fire = meas <= tau
            if (opts.delta_rule and this_unscaled and prev_unscaled and delta_prev is not None
                    and delta > delta_prev / 2):
                fire = True
            if fire:
                fired = 1
        else:
            fired += 1
        if fired >= max(opts.stop_after, 1):
            break
        if scaling_on and delta < opts.scale_off:
            scaling_on = False
        delta_prev = delta
        prev_unscaled = this_unscaled
    rec.A_final = Ak
    return rec


def newton_chol(A: np.ndarray, L: np.ndarray, opts: Opts, record: NewtonRecord | None = None):
    """Sign-function Newton iteration for a Cholesky-type factor (Sec. 3.2, Eq. (3.2)).

    Z_k = 2^{-1/2} [mu^{1/2} Z_{k-1}, mu^{-1/2} A_{k-1}^{-1} Z_{k-1}], Z_0 = L, truncated by
    RankTruncChol whenever cols(Z_k) > rho n; returns Z = Z_K / sqrt(2).
    ``record`` replays a stored inverse sequence (Sec. 3.4); it is computed when absent.
    """
    n = A.shape[0]
    p = opts.u_s
    if record is None:
        record = newton_sequence(A, opts)
    tol = opts.rank_tol if opts.rank_tol > 0 else math.sqrt(_u(p))
    Z = rnd(L, p)
    for Xk, mu in zip(record.inverses, record.mus):
        Z = rnd(np.hstack([math.sqrt(mu / 2.0) * Z, (1.0 / math.sqrt(2.0 * mu)) * (Xk @ Z)]), p)
        if Z.shape[1] > opts.rho * n:
            Z = rnd(rank_trunc_chol(Z, tol), p)
    return Z / math.sqrt(2.0), record


def newton_ldlt(A: np.ndarray, L: np.ndarray, y: np.ndarray, opts: Opts,
                record: NewtonRecord | None = None):
    """Sign-function Newton iteration for an LDL^T-type factor (Sec. 3.2, Eq. (3.3)).

    Z_k = [Z_{k-1}, A_{k-1}^{-1} Z_{k-1}], Y_k = blkdiag(mu Y_{k-1}, mu^{-1} Y_{k-1}) / 2,
    Z_0 = L, Y_0 = S = diag(y); RankTruncLdlt when cols(Z_k) > rho n; Y = Y_K / 2.
    """
    n = A.shape[0]
    p = opts.u_s
    if record is None:
        record = newton_sequence(A, opts)
    tol = opts.rank_tol if opts.rank_tol > 0 else _u(p)
    Z = rnd(L, p)
    yk = np.asarray(y, dtype=np.float64).copy()
    for Xk, mu in zip(record.inverses, record.mus):
        Z = rnd(np.hstack([Z, Xk @ Z]), p)
        yk = np.concatenate([0.5 * mu * yk, 0.5 / mu * yk])
        if Z.shape[1] > opts.rho * n:
            Z, yk = rank_trunc_ldlt(Z, yk, tol)
            Z = rnd(Z, p)
    return Z, yk / 2.0, record


# ---------------------------------------------------------------------------
# Low-rank ADI as the inner solver (Sec. 5 names ADI-based solvers as an alternative inside
# the same refinement framework; the iteration is the standard real-shift low-rank ADI)
# ---------------------------------------------------------------------------
@dataclass
class ADIRecord:
    """Shifts and the shifted inverses (A + p_j I)^{-1} rounded to u_s (depend on A only, so
    every correction solve reuses them, as the sign-Newton sequence of Sec. 3.4)."""
    shifts: list = field(default_factory=list)
    inverses: list = field(default_factory=list)


def adi_shifts(a: float, b: float, count: int) -> np.ndarray:
    """Real shifts for a spectrum with |lambda| in [a, b]: the geometric grid
    p_j = -b (a / b)^((2j - 1) / (2 count)), j = 1..count."""
    j = np.arange(1, count + 1)
    return -b * (a / b) ** ((2 * j - 1) / (2.0 * count))


def adi_record(A: np.ndarray, opts: Opts) -> ADIRecord:
    """Shifts from the 2-norm bounds a = 1 / ||A^{-1}||_2, b = ||A||_2 and the inverses."""
    n = A.shape[0]
    a = 1.0 / np.linalg.norm(np.linalg.inv(A), 2)
    b = np.linalg.norm(A, 2)
    rec = ADIRecord()
    for p in adi_shifts(a, b, opts.adi_shifts):
        rec.shifts.append(float(p))
        rec.inverses.append(rnd(np.linalg.inv(rnd(A + p * np.eye(n), opts.u_s)), opts.u_s))
    return rec


def _lr_adi(A, L, y, opts: Opts, rec: ADIRecord | None, ldlt: bool):
    """V_j = (A + p_j I)^{-1} W_{j-1}, W_j = W_{j-1} - 2 p_j V_j (W_0 = L, shifts cyclic);
    Cholesky type: Z_j = [Z_{j-1}, sqrt(-2 p_j) V_j]; LDL^T type: Z_j = [Z_{j-1}, V_j] with
    weights -2 p_j y.  Then A X_j + X_j A^T + L diag(y) L^T = W_j diag(y) W_j^T for
    X_j = Z_j diag(D_j) Z_j^T; the iteration stops once ||W diag(y) W^T||_F <= adi_tol
    ||L diag(y) L^T||_F.  Every matrix result is rounded to u_s; Z is truncated by
    RankTruncChol / RankTruncLdlt whenever cols(Z) > rho n, as in the Newton solver."""
    n = A.shape[0]
    p_ = opts.u_s
    if rec is None:
        rec = adi_record(A, opts)
    tol = opts.adi_tol if opts.adi_tol > 0 else max(10.0 * _u(p_), 1e-14)
    rtol = opts.rank_tol if opts.rank_tol > 0 else (_u(p_) if ldlt else math.sqrt(_u(p_)))
    y0 = np.ones(L.shape[1]) if y is None else np.asarray(y, dtype=np.float64)
    W = rnd(L, p_)
    nrm0 = np.linalg.norm((W * y0) @ W.T, "fro")
    Z = np.zeros((n, 0))
    yZ = np.zeros(0)
    steps = 0
    for it in range(opts.adi_maxit):
        if nrm0 == 0.0 or np.linalg.norm((W * y0) @ W.T, "fro") <= tol * nrm0:
            break
        j = it % len(rec.shifts)
        pj = rec.shifts[j]
        V = rnd(rec.inverses[j] @ W, p_)
        W = rnd(W - 2.0 * pj * V, p_)
        if ldlt:
            Z = np.hstack([Z, V])
            yZ = np.concatenate([yZ, -2.0 * pj * y0])
        else:
            Z = rnd(np.hstack([Z, math.sqrt(-2.0 * pj) * V]), p_)
        steps += 1
        if Z.shape[1] > opts.rho * n:
            if ldlt:
                Z, yZ = rank_trunc_ldlt(Z, yZ, rtol)
                Z = rnd(Z, p_)
            else:
                Z = rnd(rank_trunc_chol(Z, rtol), p_)
    return Z, yZ, W, rec, steps


def lr_adi_chol(A, L, opts: Opts, rec: ADIRecord | None = None):
    """Low-rank ADI for A X + X A^T + L L^T = 0: returns (Z, rec, W, steps), X ~ Z Z^T."""
    Z, _, W, rec, steps = _lr_adi(A, L, None, opts, rec, False)
    return Z, rec, W, steps


def lr_adi_ldlt(A, L, y, opts: Opts, rec: ADIRecord | None = None):
    """Low-rank ADI for A X + X A^T + L diag(y) L^T = 0: returns (Z, yZ, rec, W, steps)."""
    Z, yZ, W, rec, steps = _lr_adi(A, L, y, opts, rec, True)
    return Z, yZ, rec, W, steps


# ---------------------------------------------------------------------------
# Extended Krylov subspace method as the inner solver (the Krylov alternative Sec. 5 names):
# Galerkin projection onto span{L, A^-1 L, A L, A^-2 L, A^2 L, ...}
# ---------------------------------------------------------------------------
@dataclass
class EKSMRecord:
    """A^{-1} rounded to u_s (depends on A only: every correction solve reuses it)."""
    inverses: list = field(default_factory=list)


def _orth(W):
    Q, _ = np.linalg.qr(W)
    return Q


def _eksm(A, L, y, opts: Opts, rec: EKSMRecord | None, ldlt: bool):
    """Block extended Krylov (Galerkin).  U_1 = orth([L, A^{-1} L]); step j takes the two
    halves of the newest block U_j to [A U_j^(1), A^{-1} U_j^(2)], orthogonalises it against
    V_j = [U_1, ..., U_j] (twice) into U_{j+1}.  With T_j = V_j^T A V_j and E = V_j^T L,
    T_j Y + Y T_j^T + E diag(y) E^T = 0 (Bartels-Stewart, FP64) gives X_j = V_j Y V_j^T, whose
    residual has norm sqrt(2) ||U_{j+1}^T A V_j Y||_F (A V_j lies in span V_{j+1}); the
    iteration stops when that is <= tol ||L diag(y) L^T||_F.  Products and the basis are
    rounded to u_s.  Returns (Z, yZ, rec, steps, resnorm) with X_j = Z diag(yZ) Z^T
    (Cholesky type: the eigenvalues of Y below zero are dropped, yZ = 1)."""
    n, m = L.shape
    p_ = opts.u_s
    if rec is None:
        rec = EKSMRecord(inverses=[rnd(np.linalg.inv(rnd(A, p_)), p_)])
    Ai = rec.inverses[0]
    tol = opts.adi_tol if opts.adi_tol > 0 else max(10.0 * _u(p_), 1e-14)
    y0 = np.ones(m) if y is None else np.asarray(y, dtype=np.float64)
    Lr = rnd(L, p_)
    nrm0 = np.linalg.norm((Lr * y0) @ Lr.T, "fro")
    V = rnd(_orth(np.hstack([Lr, rnd(Ai @ Lr, p_)])), p_)
    U = V
    Y = np.zeros((V.shape[1], V.shape[1]))
    Vy = V
    steps, res = 0, math.inf
    for j in range(opts.eksm_maxit):
        W = rnd(np.hstack([A @ U[:, :m], Ai @ U[:, m:]]), p_)
        for _ in range(2):
            W = W - V @ (V.T @ W)
        Un = rnd(_orth(W), p_)
        AV = A @ V
        T = V.T @ AV
        E = V.T @ Lr
        Y = bartels_stewart(T, (E * y0) @ E.T)
        Vy = V
        steps = j + 1
        res = math.sqrt(2.0) * np.linalg.norm((Un.T @ AV) @ Y, "fro")
        if nrm0 == 0.0 or res <= tol * nrm0 or V.shape[1] + Un.shape[1] > n:
            break
        V = np.hstack([V, Un])
        U = Un
    lam, Q = np.linalg.eigh((Y + Y.T) / 2)
    if ldlt:
        keep = np.abs(lam) > 1e-14 * max(np.max(np.abs(lam)), 1e-300)
        return rnd(Vy @ Q[:, keep], p_), lam[keep], rec, steps, res
    keep = lam > 1e-14 * max(np.max(lam), 1e-300)
    return rnd(Vy @ (Q[:, keep] * np.sqrt(lam[keep])), p_), np.ones(int(keep.sum())), rec, steps, res


def eksm_chol(A, L, opts: Opts, rec: EKSMRecord | None = None):
    """Extended Krylov for A X + X A^T + L L^T = 0: returns (Z, rec, steps, resnorm)."""
    Z, _, rec, steps, res = _eksm(A, L, None, opts, rec, False)
    return Z, rec, steps, res


def eksm_ldlt(A, L, y, opts: Opts, rec: EKSMRecord | None = None):
    """Extended Krylov for A X + X A^T + L diag(y) L^T = 0: returns (Z, yZ, rec, steps, resnorm)."""
    return _eksm(A, L, y, opts, rec, True)


# ---------------------------------------------------------------------------
# Residual factorisation and solution update, Sec. 2
# ---------------------------------------------------------------------------

def _sym_eig(H: np.ndarray):
    return np.linalg.eigh(H)


def res_fac_chol(A, L, Z, eta_r):
    """Fragment ResFacChol: R(Z) = F P F^T with F = [Z, AZ, L] (Eq. (2.2) and the product form).

    Thin QR F = U T, H = T P T^T = Q Lambda Q^T; keep lambda >= eta_r max|lambda| for the
    PSD part and lambda <= -eta_r max|lambda| for the NSD part (eta_r relative to
    ||Lambda||_2, as in the truncation bound of Sec. 2.2).
    Returns (L+, L-, ||R||_F) with ||R||_F = ||Lambda||_F before truncation.
    """
    c = Z.shape[1]
    m = L.shape[1]
    F = np.hstack([Z, A @ Z, L])
    U, T = np.linalg.qr(F)
    q = 2 * c + m
    P = np.zeros((q, q))
    P[:c, c:2 * c] = np.eye(c)
    P[c:2 * c, :c] = np.eye(c)
    P[2 * c:, 2 * c:] = np.eye(m)
    H = T @ P @ T.T
    lam, Qh = _sym_eig(H)
    resF = math.sqrt(float(np.sum(lam ** 2)))
    lmax = float(np.max(np.abs(lam))) if lam.size else 0.0
    Jp = lam >= eta_r * lmax
    Jm = lam <= -eta_r * lmax
    if lmax == 0.0:
        Jp[:] = False
        Jm[:] = False
    Lp = (U @ Qh[:, Jp]) * np.sqrt(lam[Jp])[None, :]
    Lm = (U @ Qh[:, Jm]) * np.sqrt(-lam[Jm])[None, :]
    return Lp, Lm, resF


def sol_upt_chol(Z, Zp, Zm, eta_s):
    """Fragment SolUptChol: projected update Z_{i+1} with Z_{i+1} Z_{i+1}^T ~= P_psd(Z Z^T + Z+Z+^T - Z-Z-^T).

    G = [Z, Z+, Z-] = V Gamma, K = Gamma J Gamma^T with J = blkdiag(I, I, -I),
    K = Theta Sigma Theta^T; keep sigma >= eta_s max|sigma|; Z_{i+1} = V Theta_t Sigma_t^{1/2}.
    """
    G = np.hstack([Z, Zp, Zm])
    V, Gam = np.linalg.qr(G)
    J = np.concatenate([np.ones(Z.shape[1] + Zp.shape[1]), -np.ones(Zm.shape[1])])
    K = (Gam * J[None, :]) @ Gam.T
    sig, Th = _sym_eig(K)
    smax = float(np.max(np.abs(sig)))
    keep = sig >= eta_s * smax
    return (V @ Th[:, keep]) * np.sqrt(sig[keep])[None, :]


def res_fac_ldlt(A, L, s, Z, y, eta_r):
    """Fragment ResFacLdlt: R(Z, Y) = F N F^T, N = [[0, Y, 0], [Y, 0, 0], [0, 0, S]] (Sec. 2.3).

    Thin QR F = U T, H = T N T^T = Q Lambda Q^T; keep |lambda| >= eta_r max|lambda|.
    Returns (L^Delta, s^Delta (diagonal of S^Delta), ||R||_F).
    """
    c = Z.shape[1]
    m = L.shape[1]
    F = np.hstack([Z, A @ Z, L])
    U, T = np.linalg.qr(F)
    q = 2 * c + m
    N = np.zeros((q, q))
    N[:c, c:2 * c] = np.diag(y)
    N[c:2 * c, :c] = np.diag(y)
    N[2 * c:, 2 * c:] = np.diag(s)
    H = T @ N @ T.T
    lam, Qh = _sym_eig(H)
    resF = math.sqrt(float(np.sum(lam ** 2)))
    lmax = float(np.max(np.abs(lam))) if lam.size else 0.0
    keep = np.abs(lam) >= eta_r * lmax
    if lmax == 0.0:
        keep[:] = False
    return U @ Qh[:, keep], lam[keep], resF


def sol_upt_ldlt(Z, y, Zd, yd, eta_s, project_psd=True):
    """Fragment SolUptLdlt: G = [Z, Z^Delta] = V Gamma, K = Gamma blkdiag(Y, Y^Delta) Gamma^T.

    Keeps sigma >= eta_s max|sigma| (projection onto the PSD cone), or, for an
    indefinite right-hand side (``project_psd`` False), |sigma| >= eta_s max|sigma|.
    """
    G = np.hstack([Z, Zd])
    V, Gam = np.linalg.qr(G)
    ups = np.concatenate([y, yd])
    K = (Gam * ups[None, :]) @ Gam.T
    sig, Th = _sym_eig(K)
    smax = float(np.max(np.abs(sig)))
    keep = (sig >= eta_s * smax) if project_psd else (np.abs(sig) >= eta_s * smax)
    return V @ Th[:, keep], sig[keep]


def norm_xyx(Z, y=None):
    """||Z Y Z^T||_F from the Gram matrix G = Z^T Z: sum_ij G_ij^2 y_i y_j (y = 1 for Z Z^T)."""
    G = Z.T @ Z
    if y is None:
        return float(np.linalg.norm(G, "fro"))
    return math.sqrt(max(float(np.sum(G * G * np.outer(y, y))), 0.0))


@dataclass
class IRInfo:
    res_hist: list = field(default_factory=list)
    ir_steps: int = 0
    newton_calls: int = 0
    newton_total: int = 0
    newton_max: int = 0
    n_inversions: int = 0
    rank: int = 0
    stagnated: bool = False
    converged: bool = False
    res_final: float = float("nan")


def ir_chol(A, L, opts: Opts):
    """Algorithm IR-Chol (Sec. 2.1) with the sign-Newton solver (Sec. 3; or low-rank ADI,
    ``opts.inner``) and Sec. 4.1 rules.

    The inverse sequence of the first solve is stored and replayed by every
    correction solve (Sec. 3.4): the sequence depends on A only.
    Returns (Z, IRInfo).
    """
    n = A.shape[0]
    tau_ir = opts.tau_ir if opts.tau_ir > 0 else n * UNIT[opts.u]
    eta_s = opts.eta_s if opts.eta_s > 0 else 10.0 * UNIT[opts.u]
    info = IRInfo()
    if opts.inner == "adi":
        def solve(Lr, r):
            return lr_adi_chol(A, Lr, opts, r)[:2]
    elif opts.inner == "eksm":
        def solve(Lr, r):
            return eksm_chol(A, Lr, opts, r)[:2]
    else:
        def solve(Lr, r):
            return newton_chol(A, Lr, opts, r)
    Z, rec = solve(L, None)
    Z = rnd(Z, opts.u)
    K = len(rec.inverses)
    info.n_inversions = K
    info.newton_calls, info.newton_total, info.newton_max = 1, K, K
    W_F = float(np.linalg.norm(L.T @ L, "fro"))
    A_F = float(np.linalg.norm(A, "fro"))
    best = (math.inf, Z)
    stag = 0
    res_prev = None
    for i in range(1, opts.imax + 2):
        Lp, Lm, resF = res_fac_chol(A, L, Z, opts.eta_r)
        res = resF / (W_F + 2.0 * norm_xyx(Z) * A_F)
        info.res_hist.append(res)
        if res < best[0]:
            best = (res, Z)
        if res <= tau_ir:
            info.converged = True
            break
        if res_prev is not None and res / res_prev > opts.stag_theta:
            stag += 1
        else:
            stag = 0
        res_prev = res
        if stag >= opts.stag_count:
            info.stagnated = True
            break
        if i == opts.imax + 1:
            break
        Lp, Lm = rnd(rnd(Lp, opts.u), opts.u_s), rnd(rnd(Lm, opts.u), opts.u_s)
        Zp = solve(Lp, rec)[0] if Lp.shape[1] else np.zeros((n, 0))
        Zm = solve(Lm, rec)[0] if Lm.shape[1] else np.zeros((n, 0))
        info.newton_calls += 1
        info.newton_total += K
        Z = rnd(sol_upt_chol(Z, Zp, Zm, eta_s), opts.u)
        info.ir_steps = i
    info.res_final = best[0]
    info.rank = best[1].shape[1]
    return best[1], info


def ir_ldlt(A, L, S, opts: Opts):
    """Algorithm IR-LDLT (Sec. 2.3) with the sign-Newton solver (Sec. 3; or low-rank ADI,
    ``opts.inner``) and Sec. 4.1 rules.

    S is diagonalised at entry (S = V diag(s) V^T, L <- L V), which is exact, so that
    every inner factor Y is a diagonal vector.  When S is indefinite the PSD
    projection of SolUptLdlt is replaced by magnitude truncation (the solution X is
    then indefinite, outside the paper's assumption that W is PSD).
    Returns (Z, y, IRInfo) with X ~= Z diag(y) Z^T.
    """
    n = A.shape[0]
    s, Vs = np.linalg.eigh(np.asarray(S, dtype=np.float64))
    L = L @ Vs
    project = opts.project_psd and bool(np.all(s >= 0))
    tau_ir = opts.tau_ir if opts.tau_ir > 0 else n * UNIT[opts.u]
    eta_s = opts.eta_s if opts.eta_s > 0 else 10.0 * UNIT[opts.u]
    info = IRInfo()
    if opts.inner == "adi":
        def solve(Lr, yr, r):
            Zr, yZ, r2, _, _ = lr_adi_ldlt(A, Lr, yr, opts, r)
            return Zr, yZ, r2
    elif opts.inner == "eksm":
        def solve(Lr, yr, r):
            Zr, yZ, r2, _, _ = eksm_ldlt(A, Lr, yr, opts, r)
            return Zr, yZ, r2
    else:
        def solve(Lr, yr, r):
            return newton_ldlt(A, Lr, yr, opts, r)
    Z, y, rec = solve(L, s, None)
    Z, y = rnd(Z, opts.u), rnd(y, opts.u)
    K = len(rec.inverses)
    info.n_inversions = K
    info.newton_calls, info.newton_total, info.newton_max = 1, K, K
    W_F = norm_xyx(L, s)
    A_F = float(np.linalg.norm(A, "fro"))
    best = (math.inf, Z, y)
    stag = 0
    res_prev = None
    for i in range(1, opts.imax + 2):
        Ld, sd, resF = res_fac_ldlt(A, L, s, Z, y, opts.eta_r)
        res = resF / (W_F + 2.0 * norm_xyx(Z, y) * A_F)
        info.res_hist.append(res)
        if res < best[0]:
            best = (res, Z, y)
        if res <= tau_ir:
            info.converged = True
            break
        if res_prev is not None and res / res_prev > opts.stag_theta:
            stag += 1
        else:
            stag = 0
        res_prev = res
        if stag >= opts.stag_count:
            info.stagnated = True
            break
        if i == opts.imax + 1:
            break
        Ld, sd = rnd(rnd(Ld, opts.u), opts.u_s), rnd(rnd(sd, opts.u), opts.u_s)
        Zd, yd, _ = solve(Ld, sd, rec)
        info.newton_calls += 1
        info.newton_total += K
        Z, y = sol_upt_ldlt(Z, y, Zd, yd, eta_s, project)
        Z, y = rnd(Z, opts.u), rnd(y, opts.u)
        info.ir_steps = i
    info.res_final = best[0]
    info.rank = best[1].shape[1]
    return best[1], best[2], info


# ---------------------------------------------------------------------------
# Diagnostics
# ---------------------------------------------------------------------------

def residual_eq41(A, Z, W, y=None) -> float:
    """Relative residual of Eq. (4.1), evaluated explicitly in FP64 on n x n matrices."""
    X = Z @ Z.T if y is None else (Z * y[None, :]) @ Z.T
    R = A @ X + X @ A.T + W
    return float(np.linalg.norm(R, "fro") /
                 (np.linalg.norm(W, "fro") + 2.0 * np.linalg.norm(X, "fro") * np.linalg.norm(A, "fro")))


def adjoint(A, L, C, S=None):
    """Gradient of l = trace(C X C^T) where A X + X A^T + L S L^T = 0 (S = I if None).

    With Y solving A^T Y + Y A + C^T C = 0:  dl/dW = Y, dl/dA = 2 Y X,
    dl/dL = 2 Y L S, dl/dS = L^T Y L.  Not in the paper; follows from differentiating
    Eq. (1.1) and the adjoint of the Lyapunov operator.
    Returns dict(X, Y, loss, dA, dL, dS).
    """
    m = L.shape[1]
    S = np.eye(m) if S is None else np.asarray(S, dtype=np.float64)
    W = L @ S @ L.T
    X = bartels_stewart(A, W)
    G = C.T @ C
    Y = bartels_stewart(A.T, G)
    return {"X": X, "Y": Y, "loss": float(np.trace(C @ X @ C.T)),
            "dA": 2.0 * Y @ X, "dL": 2.0 * Y @ L @ S, "dS": L.T @ Y @ L}


# ---------------------------------------------------------------------------------------
# Condition of the matrix sign function at B = [[A, W], [0, -A^T]] (Sec. 4.2: the sign-
# Newton iteration for Eq. (1.1) computes sign(B); kappa_sign(B) in the Frobenius norm
# predicts its accuracy).  Plain definitions for small orders: the eigendecomposition
# B = V diag(lambda) V^{-1} (B diagonalisable, no eigenvalue on the imaginary axis).
# ---------------------------------------------------------------------------------------
def sign_block(A: np.ndarray, W: np.ndarray) -> np.ndarray:
    """B = [[A, W], [0, -A^T]], whose sign is [[-I, 2X], [0, I]] for Hurwitz A (Sec. 3)."""
    n = A.shape[0]
    return np.block([[A, W], [np.zeros((n, n)), -A.T]])


def sign_matrix(B: np.ndarray) -> np.ndarray:
    """sign(B) = V diag(sign(Re lambda_i)) V^{-1}."""
    lam, V = np.linalg.eig(B)
    return np.real(V @ np.diag(np.sign(lam.real)) @ np.linalg.inv(V))


def frechet_sign(B: np.ndarray, E: np.ndarray) -> np.ndarray:
    """Frechet derivative L_sign(B, E) = V (D o (V^{-1} E V)) V^{-1} with the divided
    differences D_ij = (sign lambda_i - sign lambda_j) / (lambda_i - lambda_j), 0 where the
    signs agree (the derivative of a function constant on each half plane)."""
    lam, V = np.linalg.eig(B)
    sg = np.sign(lam.real)
    Vi = np.linalg.inv(V)
    dl = lam[:, None] - lam[None, :]
    same = sg[:, None] == sg[None, :]
    D = np.where(same, 0.0, (sg[:, None] - sg[None, :]) / np.where(same, 1.0, dl))
    return np.real(V @ (D * (Vi @ E @ V)) @ Vi)


def kappa_sign_fro(B: np.ndarray) -> float:
    """kappa_sign(B) = ||L_sign(B)||_F ||B||_F / ||sign(B)||_F, where ||L||_F is the 2-norm of
    the N^2 x N^2 matrix of E -> L_sign(B, E) in vec form (columns L(B, e_i e_j^T))."""
    N = B.shape[0]
    K = np.empty((N * N, N * N))
    for j in range(N):
        for i in range(N):
            E = np.zeros((N, N))
            E[i, j] = 1.0
            K[:, i + j * N] = frechet_sign(B, E).reshape(-1, order="F")
    return float(np.linalg.norm(K, 2) * np.linalg.norm(B, "fro") / np.linalg.norm(sign_matrix(B), "fro"))
