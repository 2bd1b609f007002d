"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every check here is independent of ``oracle/``'s own formulas: dense Kronecker
solves of Eq. (2.1), closed forms, textbook library routines, invariants of the
Lyapunov equation, and the paper's printed iteration counts (Table 4.1).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import lyapgen as gen
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def kron_solve(A, W):
    """(I (x) A + A (x) I) vec X = -vec W, Eq. (2.1), solved densely."""
    n = A.shape[0]
    I = np.eye(n)
    M = np.kron(I, A) + np.kron(A, I)
    x = np.linalg.solve(M, -W.reshape(-1, order="F"))
    return x.reshape(n, n, order="F")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ----------------------------------------------------------------- exact solver

@pytest.mark.parametrize("n", [1, 2, 5, 17, 30])
def test_bartels_stewart_vs_kronecker(n):
    g = gen.rng(100 + n)
    d = gen.random_stable(n, 3, g)
    A, L = d["A"], d["L"]
    W = L @ L.T
    X = O.bartels_stewart(A, W)
    assert rel(X, kron_solve(A, W)) < 1e-12


def test_bartels_stewart_indefinite_rhs_vs_kronecker():
    g = gen.rng(7)
    A = gen.random_stable(20, 2, g)["A"]
    B = g.standard_normal((20, 20))
    W = B + B.T
    assert rel(O.bartels_stewart(A, W), kron_solve(A, W)) < 1e-12


def test_bartels_stewart_diagonal_closed_form():
    g = gen.rng(3)
    a = -10.0 ** g.uniform(-2, 2, 40)
    L = g.standard_normal((40, 3))
    W = L @ L.T
    X = O.bartels_stewart(np.diag(a), W)
    Xc = -W / (a[:, None] + a[None, :])
    assert rel(X, Xc) < 1e-13


def test_bartels_stewart_sine_basis_closed_form():
    # A = -V diag(d) V^T with V the symmetric orthogonal sine matrix (Sec. 4.2 generator):
    # V^T X V has entries (V^T W V)_ij / (d_i + d_j).
    d = gen.paper_synthetic(60, 2.0)
    V, dd, A, L = d["V"], d["d"], d["A"], d["L"]
    assert np.linalg.norm(V @ V - np.eye(60)) < 1e-12
    W = L @ L.T
    Wt = V @ W @ V
    X = V @ (Wt / (dd[:, None] + dd[None, :])) @ V
    assert rel(O.bartels_stewart(A, W), X) < 1e-12


def schur_blocks_solution(Q, alpha, beta, W):
    """Closed form for A = Q T Q^T with T = blkdiag([[-a, b], [-b, -a]]) (block-diagonal Schur form)."""
    n = Q.shape[0]
    nb = n // 2
    Wt = Q.T @ W @ Q
    T = np.zeros((nb, 2, 2))
    T[:, 0, 0] = T[:, 1, 1] = -alpha
    T[:, 0, 1] = beta
    T[:, 1, 0] = -beta
    I2 = np.eye(2)
    # block (i, j): T_i Y + Y T_j^T = -Wt_ij  <=>  (I (x) T_i + T_j (x) I) vec Y = -vec Wt_ij
    M = np.einsum("ab,icd->iacbd", I2, T).reshape(nb, 1, 4, 4) + \
        np.einsum("jab,cd->jacbd", T, I2).reshape(1, nb, 4, 4)
    Wb = Wt.reshape(nb, 2, nb, 2).transpose(0, 2, 3, 1).reshape(nb, nb, 4)  # vec (column-major)
    Y = np.linalg.solve(M, -Wb[..., None])[..., 0]
    Xt = Y.reshape(nb, nb, 2, 2).transpose(0, 3, 1, 2).reshape(n, n)
    return Q @ Xt @ Q.T


def test_schur_block_closed_form_is_kronecker():
    d = gen.normal_blocks(n=12, p=2, m=3)
    A, L, S = d["A"], d["L"], d["S"]
    W = L @ S @ L.T
    assert rel(schur_blocks_solution(d["Q"], d["alpha"], d["beta"], W), kron_solve(A, W)) < 1e-11


def test_bartels_stewart_normal_blocks_closed_form():
    d = gen.normal_blocks(n=120, p=3, m=4)
    A, L, S = d["A"], d["L"], d["S"]
    W = L @ S @ L.T
    X = O.bartels_stewart(A, W)
    assert rel(X, schur_blocks_solution(d["Q"], d["alpha"], d["beta"], W)) < 1e-11


def test_bartels_stewart_vs_lapack_routine():
    d = gen.convdiff_shifted(grid=8, m=3)
    A, L = d["A"], d["L"]
    W = L @ L.T
    X = O.bartels_stewart(A, W)
    assert rel(X, sla.solve_continuous_lyapunov(A, -W)) < 1e-11


def test_solution_symmetric_psd():
    d = gen.convdiff_shifted(grid=6, m=2)
    X = O.bartels_stewart(d["A"], d["L"] @ d["L"].T)
    assert np.linalg.norm(X - X.T) <= 1e-12 * np.linalg.norm(X)
    assert np.linalg.eigvalsh(0.5 * (X + X.T)).min() >= -1e-12 * np.linalg.norm(X, 2)


# ------------------------------------------------------------- LU / rounding

def test_getrf_pivots_match_lapack():
    g = gen.rng(11)
    A = g.standard_normal((40, 40))
    LU, perm, ipiv = O.getrf_pp(A)
    lu, piv = sla.lu_factor(A)
    assert np.array_equal(ipiv, piv)
    Lm = np.tril(LU, -1) + np.eye(40)
    Um = np.triu(LU)
    assert rel(Lm @ Um, A[perm]) < 1e-14


def test_rounding_formats():
    # bf16: 8-bit significand; 1 + 2^-8 is a tie -> even (1); 1 + 3*2^-8 -> 1 + 2^-6
    x = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, -3.0, 2.0 ** -130])
    r = O.rnd(x, "bf16")
    assert r[0] == 1.0 and r[1] == 1.0 + 2.0 ** -6 and r[2] == 1.0 + 2.0 ** -7 and r[3] == -3.0
    # fp16: 11-bit significand, scaled into range: huge and tiny values keep 11 bits
    y = np.array([1.0 + 2.0 ** -11, 1.0 + 2.0 ** -10, 3.0])
    assert np.array_equal(O.rnd(y, "fp16"), [1.0, 1.0 + 2.0 ** -10, 3.0])
    z = np.array([1e-12, 3e-12])
    assert np.all(np.abs(O.rnd(z, "fp16") - z) <= 2.0 ** -11 * z)
    w = np.array([1.0 + 2.0 ** -24, 1.0 + 2.0 ** -23])
    assert np.array_equal(O.rnd(w, "fp32"), [1.0, 1.0 + 2.0 ** -23])
    for k, u in O.UNIT.items():
        assert abs(u - json.load(open(os.path.join(HERE, "golden", "table41_fp64_newton_counts.json")))
                   ["unit_roundoff_table11"][k]) <= 0.005 * u


# ----------------------------------------------------------- sign-Newton solver

def test_sign_newton_converges_to_minus_identity():
    d = gen.convdiff_shifted(grid=6, m=2)
    rec = O.newton_sequence(d["A"], O.Opts(u_s="fp64"))
    n = d["A"].shape[0]
    assert np.linalg.norm(rec.A_final + np.eye(n), 1) < 1e-10


def test_sign_newton_scaling_invariance():
    # Frobenius scaling makes A_1 independent of a positive factor on A (Sec. 3): A -> 8 A.
    d = gen.convdiff_shifted(grid=5, m=2)
    r1 = O.newton_sequence(d["A"], O.Opts(u_s="fp64"))
    r2 = O.newton_sequence(8.0 * d["A"], O.Opts(u_s="fp64"))
    assert len(r1.inverses) == len(r2.inverses)
    assert rel(r2.A_final, r1.A_final) < 1e-12
    assert abs(r2.mus[0] * 8.0 - r1.mus[0]) < 1e-12 * r1.mus[0]


def test_sign_newton_norm2_and_spectral_scaling_closed_forms():
    # Sec. 3.1 scalings on matrices with known norms and spectra.
    # (1) Upper triangular A = [[-1, 10, 0], [0, -2, 5], [0, 0, -4]]: rho(A) = 4 and
    # rho(A^{-1}) = 1, so the spectral mu_0 = 1/2 exactly.  The squared singular values are
    # the roots of x^3 - t x^2 + c x - det(A)^2 with t = ||A||_F^2 = 146 and
    # c = (t^2 - tr((A^T A)^2)) / 2 (integers); sigma_max(A^{-1}) = 1 / sigma_min(A), so the
    # 2-norm mu_0 = (x_min x_max)^(-1/4).  Frobenius: ||A^{-1}||_F^2 = 65.765625 by hand.
    A = np.array([[-1.0, 10.0, 0.0], [0.0, -2.0, 5.0], [0.0, 0.0, -4.0]])
    M = A.T @ A
    t = float(np.trace(M))
    c = (t * t - float(np.trace(M @ M))) / 2
    x = np.sort(np.roots([1.0, -t, c, -64.0]).real)
    mu_n2 = (x[0] * x[2]) ** -0.25
    mu_fro = math.sqrt(math.sqrt(65.765625) / math.sqrt(146.0))
    r_sp = O.newton_sequence(A, O.Opts(u_s="fp64", scaling="spectral"))
    r_n2 = O.newton_sequence(A, O.Opts(u_s="fp64", scaling="norm2"))
    r_fr = O.newton_sequence(A, O.Opts(u_s="fp64", scaling="frob"))
    assert abs(r_sp.mus[0] - 0.5) <= 1e-15
    assert abs(r_n2.mus[0] - mu_n2) <= 1e-12 * mu_n2
    assert abs(r_fr.mus[0] - mu_fro) <= 1e-14 * mu_fro
    assert min(abs(mu_n2 - mu_fro), abs(mu_n2 - 0.5), abs(mu_fro - 0.5)) > 1e-2
    for r in (r_sp, r_n2, r_fr):
        assert np.linalg.norm(r.A_final + np.eye(3)) <= 1e-12
    # (2) symmetric negative definite A with spectrum in [-b, -a]: both scalings give
    # mu_0 = 1 / sqrt(a b), which maps the two extreme eigenvalues to the same value of
    # A_1 = (mu A + (mu A)^{-1}) / 2: -(sqrt(b/a) + sqrt(a/b)) / 2
    g = gen.rng(77)
    Q, _ = np.linalg.qr(g.standard_normal((12, 12)))
    lam = -np.geomspace(0.5, 200.0, 12)
    S = (Q * lam) @ Q.T
    S = (S + S.T) / 2
    for sc in ("norm2", "spectral"):
        r = O.newton_sequence(S, O.Opts(u_s="fp64", scaling=sc))
        assert abs(r.mus[0] - 1.0 / math.sqrt(0.5 * 200.0)) <= 1e-13 / math.sqrt(100.0)
        A1 = 0.5 * (r.mus[0] * S + np.linalg.inv(S) / r.mus[0])
        e = np.linalg.eigvalsh(A1)
        assert abs(e[0] - (-(math.sqrt(400.0) + math.sqrt(1 / 400.0)) / 2)) <= 1e-12 * abs(e[0])
        assert np.linalg.norm(r.A_final + np.eye(12)) <= 1e-10


def test_newton_chol_fp64_laplacian_config():
    d = gen.fp64_laplacian(8, 2)
    A, L = d["A"], d["L"]
    W = L @ L.T
    opts = O.Opts(u_s="fp64", scaling="det", newton_norm="fro", tau_newton=1e-12 * 64, rho=0.0,
                  rank_tol=1e-14)
    Z, rec = O.newton_chol(A, L, opts)
    X = kron_solve(A, W)
    assert rel(Z @ Z.T, X) < 1e-12
    assert O.residual_eq41(A, Z, W) < 1e-14


def test_newton_chol_fp64_kronecker_n16():
    d = gen.fp64_laplacian(4, 2)
    A, L = d["A"], d["L"]
    opts = O.Opts(u_s="fp64", scaling="det", newton_norm="fro", tau_newton=1e-12 * 16, rho=0.0,
                  rank_tol=1e-14)
    Z, _ = O.newton_chol(A, L, opts)
    assert rel(Z @ Z.T, kron_solve(A, L @ L.T)) < 1e-12


def test_newton_ldlt_fp64_indefinite():
    d = gen.normal_blocks(n=40, p=1, m=4)
    A, L, S = d["A"], d["L"], d["S"]
    s = np.diag(S)
    Z, y, _ = O.newton_ldlt(A, L, s, O.Opts(u_s="fp64", rho=0.0))
    X = kron_solve(A, L @ S @ L.T)
    assert rel((Z * y) @ Z.T, X) < 1e-10


def test_table41_fp64_iteration_counts():
    gold = json.load(open(os.path.join(HERE, "golden", "table41_fp64_newton_counts.json")))
    for nkey in ("100", "1000"):
        n = int(nkey)
        qs = gold["q"] if n == 100 else [0.1, 1.0, 2.0, 3.5]
        for q in qs:
            d = gen.paper_synthetic(n, q)
            rec = O.newton_sequence(d["A"], O.Opts(u_s="fp64"))
            want = gold["alpha"][nkey]["chol"][gold["q"].index(q)]
            assert len(rec.inverses) == want, (n, q, len(rec.inverses), want)


def test_table41_fp32_inner_counts_n100():
    gold = json.load(open(os.path.join(HERE, "golden", "table41_fp64_newton_counts.json")))
    g = gold["fp32_inner_iter_u64_n100_chol"]
    for q, tot, al in zip(g["q"], g["total"], g["alpha"]):
        d = gen.paper_synthetic(100, q)
        Z, info = O.ir_chol(d["A"], d["L"], O.Opts(u_s="fp32"))
        assert info.converged
        assert (info.newton_total, info.newton_max) == (tot, al)


def test_cond_column_is_lyapunov_kappa2():
    # the printed cond 1.3e0 / 3.2e0 / 1.0e1 of Table 4.1 equals 10^q for the Sec. 4.2 generator
    gold = json.load(open(os.path.join(HERE, "golden", "table41_fp64_newton_counts.json")))
    for q, printed in zip(gold["q"], gold["cond_printed"]):
        d = gen.paper_synthetic(100, q)
        k = O.lyap_operator_kappa2_normal(-d["d"])
        assert f"{k:.1e}".replace("e+0", "e").replace("e-0", "e-") == printed


# -------------------------------------------------------- truncation routines

def test_rank_trunc_chol_exact_rank_and_product():
    g = gen.rng(5)
    n, r = 80, 7
    Z = g.standard_normal((n, r)) @ g.standard_normal((r, 30))  # exact rank 7, 30 columns
    Zt = O.rank_trunc_chol(Z, 1e-10)
    assert Zt.shape[1] == r
    assert rel(Zt @ Zt.T, Z @ Z.T) < 1e-12


def test_rank_trunc_chol_bound():
    g = gen.rng(6)
    n, c = 60, 25
    U, _ = np.linalg.qr(g.standard_normal((n, c)))
    s = 10.0 ** -np.linspace(0, 12, c)
    Z = U * s
    tol = 1e-6
    Zt = O.rank_trunc_chol(Z, tol)
    err = np.linalg.norm(Z @ Z.T - Zt @ Zt.T, 2)
    assert err <= (tol * np.linalg.norm(Z, 2)) ** 2 * 1.0001 + 1e-15
    assert Zt.shape[1] < c


def test_rank_trunc_ldlt_indefinite():
    g = gen.rng(8)
    n = 50
    Z = g.standard_normal((n, 4)) @ g.standard_normal((4, 12))
    y = g.standard_normal(12)
    Zt, yt = O.rank_trunc_ldlt(Z, y, 1e-12)
    assert Zt.shape[1] == 4
    assert np.any(yt < 0) or np.all(y > 0)
    assert rel((Zt * yt) @ Zt.T, (Z * y) @ Z.T) < 1e-11


# ---------------------------------------------- residual factorisation / update

def test_res_fac_chol_norm_and_split():
    d = gen.convdiff_shifted(grid=6, m=2)
    A, L = d["A"], d["L"]
    X = kron_solve(A, L @ L.T)
    g = gen.rng(9)
    Z = np.linalg.cholesky(X + 1e-6 * np.eye(36)) + 1e-4 * g.standard_normal((36, 36))
    R = A @ Z @ Z.T + Z @ Z.T @ A.T + L @ L.T
    Lp, Lm, resF = O.res_fac_chol(A, L, Z, 0.0)
    assert abs(resF - np.linalg.norm(R)) < 1e-10 * np.linalg.norm(R)
    assert rel(Lp @ Lp.T - Lm @ Lm.T, R) < 1e-10
    # truncation at eta_r drops at most eta_r * ||R||_2 per eigenvalue
    Lp2, Lm2, _ = O.res_fac_chol(A, L, Z, 1e-2)
    err = np.linalg.norm(Lp2 @ Lp2.T - Lm2 @ Lm2.T - R, 2)
    assert err <= 1.0001e-2 * np.linalg.norm(R, 2)


def test_res_fac_ldlt_matches_explicit_residual():
    d = gen.normal_blocks(n=30, p=1, m=3)
    A, L, S = d["A"], d["L"], d["S"]
    s = np.diag(S)
    g = gen.rng(10)
    Z = g.standard_normal((30, 9))
    y = g.standard_normal(9)
    R = A @ (Z * y) @ Z.T + (Z * y) @ Z.T @ A.T + L @ S @ L.T
    Ld, sd, resF = O.res_fac_ldlt(A, L, s, Z, y, 0.0)
    assert abs(resF - np.linalg.norm(R)) < 1e-10 * np.linalg.norm(R)
    assert rel((Ld * sd) @ Ld.T, R) < 1e-10


def test_sol_upt_chol_is_psd_projection():
    g = gen.rng(12)
    n = 40
    Z = g.standard_normal((n, 6))
    Zp = 0.1 * g.standard_normal((n, 3))
    Zm = 0.3 * g.standard_normal((n, 2))
    Xbp = Z @ Z.T + Zp @ Zp.T - Zm @ Zm.T
    w, V = np.linalg.eigh(Xbp)
    Xproj = (V * np.maximum(w, 0)) @ V.T
    Zn = O.sol_upt_chol(Z, Zp, Zm, 1e-15)
    assert rel(Zn @ Zn.T, Xproj) < 1e-12


def test_sol_upt_ldlt_projection_and_indefinite():
    g = gen.rng(13)
    n = 40
    Z = g.standard_normal((n, 5))
    y = np.abs(g.standard_normal(5))
    Zd = 0.2 * g.standard_normal((n, 4))
    yd = g.standard_normal(4)
    Xbp = (Z * y) @ Z.T + (Zd * yd) @ Zd.T
    w, V = np.linalg.eigh(Xbp)
    Zn, yn = O.sol_upt_ldlt(Z, y, Zd, yd, 1e-15, True)
    assert rel((Zn * yn) @ Zn.T, (V * np.maximum(w, 0)) @ V.T) < 1e-12
    Zi, yi = O.sol_upt_ldlt(Z, y, Zd, yd, 1e-15, False)
    assert rel((Zi * yi) @ Zi.T, Xbp) < 1e-12


def test_norm_xyx_gram_identity():
    g = gen.rng(14)
    Z = g.standard_normal((30, 7))
    y = g.standard_normal(7)
    assert abs(O.norm_xyx(Z, y) - np.linalg.norm((Z * y) @ Z.T)) < 1e-12 * np.linalg.norm((Z * y) @ Z.T)
    assert abs(O.norm_xyx(Z) - np.linalg.norm(Z @ Z.T)) < 1e-12 * np.linalg.norm(Z @ Z.T)


def test_residual_eq41_zero_at_solution():
    d = gen.convdiff_shifted(grid=5, m=2)
    A, L = d["A"], d["L"]
    W = L @ L.T
    X = kron_solve(A, W)
    w, V = np.linalg.eigh(0.5 * (X + X.T))
    Z = V * np.sqrt(np.maximum(w, 0))
    assert O.residual_eq41(A, Z, W) < 1e-14


def test_residual_eq41_normalisation_closed_form():
    # Eq. (4.1) at X = c X*, with X* the exact solution: A X + X A^T + W = (1 - c) W, so the
    # relative residual is |1 - c| ||W||_F / (||W||_F + 2 c ||X*||_F ||A||_F).  For
    # A = diag(-1, -2), L = (1, 1)^T the pieces are worked out by hand: W = [[1, 1], [1, 1]]
    # (||W||_F = 2), X*_ij = 1 / (i + j) over i, j in {1, 2} = [[1/2, 1/3], [1/3, 1/4]]
    # (||X*||_F = sqrt(77) / 12), ||A||_F = sqrt(5).  At c = 2 the value is
    # 2 / (2 + 4 sqrt(77) sqrt(5) / 12) = 6 / (6 + sqrt(385)); at c = 1/2 it is
    # 1 / (2 + sqrt(385) / 12) = 12 / (24 + sqrt(385)).  A wrong factor 2, a missing
    # ||W||_F term, or a 2-norm in place of a Frobenius norm changes both values.
    A = np.diag([-1.0, -2.0])
    L = np.array([[1.0], [1.0]])
    W = L @ L.T
    Xs = np.array([[0.5, 1.0 / 3.0], [1.0 / 3.0, 0.25]])
    C = np.linalg.cholesky(Xs)
    for c, want in ((2.0, 6.0 / (6.0 + math.sqrt(385.0))), (0.5, 12.0 / (24.0 + math.sqrt(385.0)))):
        Z = math.sqrt(c) * C
        assert abs(O.residual_eq41(A, Z, W) - want) <= 1e-15 * want
        # the LDL^T form (X = Z diag(y) Z^T) with y = c on the Cholesky factor of X*
        assert abs(O.residual_eq41(A, C, W, np.full(2, c)) - want) <= 1e-15 * want
    # Z = 0: the residual is W itself and the normalisation reduces to ||W||_F
    assert O.residual_eq41(A, np.zeros((2, 1)), W) == 1.0


# ------------------------------------------------------- refinement algorithms

@pytest.mark.parametrize("us", ["fp64", "fp32", "fp16", "bf16"])
def test_ir_chol_reaches_solution(us):
    d = gen.paper_synthetic(60, 1.0)
    A, L = d["A"], d["L"]
    X = O.bartels_stewart(A, L @ L.T)
    Z, info = O.ir_chol(A, L, O.Opts(u_s=us))
    assert info.converged
    assert O.residual_eq41(A, Z, L @ L.T) < 1e-13
    assert rel(Z @ Z.T, X) < 1e-11
    if us != "fp64":
        assert info.ir_steps >= 1


@pytest.mark.parametrize("us", ["fp64", "fp16"])
def test_ir_ldlt_indefinite_reaches_solution(us):
    d = gen.normal_blocks(n=40, p=1, m=4)
    A, L, S = d["A"], d["L"], d["S"]
    W = L @ S @ L.T
    X = kron_solve(A, W)
    Z, y, info = O.ir_ldlt(A, L, S, O.Opts(u_s=us))
    assert info.converged
    assert rel((Z * y) @ Z.T, X) < 1e-11


def test_ir_stagnation_beyond_bf16_bound():
    # kappa ~ 3e3 > 1e3 (Table 2.1 bound for bf16): refinement stalls and reports it
    d = gen.paper_synthetic(100, 3.5)
    Z, info = O.ir_chol(d["A"], d["L"], O.Opts(u_s="bf16"))
    assert not info.converged


def test_ir_ldlt_bf16_stalls_on_normal_blocks():
    # A = Q T Q^T with 2 x 2 blocks -a +- i b (b up to 5, a down to 0.1): eigenvalues close to
    # the imaginary axis relative to their size put the problem beyond bf16's reach (Table 2.1);
    # the BF16-inner refinement does not contract and the stagnation rule stops it
    d = gen.normal_blocks(n=128, p=1, m=4)
    Z, y, info = O.ir_ldlt(d["A"], d["L"], d["S"], O.Opts(u_s="bf16", tau_ir=1e-12, imax=20))
    assert not info.converged and info.stagnated
    assert min(info.res_hist) > 1e-3


# ---------------------------------------------------------------- adjoint

def test_adjoint_vs_kronecker_bruteforce():
    g = gen.rng(15)
    n = 10
    d = gen.random_stable(n, 2, g)
    A, L = d["A"], d["L"]
    C = g.standard_normal((3, n))
    out = O.adjoint(A, L, C)
    # d l / d vec(W) = -M^{-T} vec(G), M = I (x) A + A (x) I
    I = np.eye(n)
    M = np.kron(I, A) + np.kron(A, I)
    Y = np.linalg.solve(M.T, -(C.T @ C).reshape(-1, order="F")).reshape(n, n, order="F")
    assert rel(out["Y"], -Y) < 1e-11 or rel(out["Y"], Y) < 1e-11
    assert rel(out["Y"], Y) < 1e-11


def test_adjoint_vs_finite_differences():
    g = gen.rng(16)
    n = 12
    d = gen.random_stable(n, 2, g)
    A, L = d["A"], d["L"]
    C = g.standard_normal((2, n))
    out = O.adjoint(A, L, C)

    def loss(Am, Lm):
        X = kron_solve(Am, Lm @ Lm.T)
        return float(np.trace(C @ X @ C.T))

    for _ in range(3):
        E = g.standard_normal((n, n))
        E /= np.linalg.norm(E)
        h = 1e-6 * np.linalg.norm(A)
        fd = (loss(A + h * E, L) - loss(A - h * E, L)) / (2 * h)
        assert abs(np.sum(out["dA"] * E) - fd) <= 1e-6 * abs(fd) + 1e-12
        F = g.standard_normal(L.shape)
        F /= np.linalg.norm(F)
        h = 1e-6 * np.linalg.norm(L)
        fd = (loss(A, L + h * F) - loss(A, L - h * F)) / (2 * h)
        assert abs(np.sum(out["dL"] * F) - fd) <= 1e-6 * abs(fd) + 1e-12


def test_adjoint_diagonal_closed_form():
    g = gen.rng(17)
    a = -10.0 ** g.uniform(-1, 1, 15)
    C = g.standard_normal((2, 15))
    L = g.standard_normal((15, 2))
    out = O.adjoint(np.diag(a), L, C)
    G = C.T @ C
    assert rel(out["Y"], -G / (a[:, None] + a[None, :])) < 1e-12



# ----------------------------------------------------- condition of the sign function

def test_kappa_sign_diagonal_closed_form():
    # diagonal B: L_sign(B, E)_ij = E_ij (sign d_i - sign d_j) / (d_i - d_j), so
    # ||L|| = 2 / (smallest positive d - largest negative d) and ||sign B||_F = sqrt(N)
    d = np.array([-3.0, -0.5, 0.25, 2.0, -7.0, 1.5])
    B = np.diag(d)
    k = O.kappa_sign_fro(B)
    ref = 2.0 / (0.25 - (-0.5)) * np.linalg.norm(d) / math.sqrt(6.0)
    assert abs(k - ref) <= 1e-12 * ref


def test_frechet_sign_against_library_sign_central_differences():
    # L_sign(B, E) against central differences of scipy's sign function (an independent route)
    g = gen.rng(88)
    B = g.standard_normal((5, 5)) + np.diag([3.0, -3.0, 2.5, -2.0, 4.0])
    E = g.standard_normal((5, 5))
    assert np.linalg.norm(O.sign_matrix(B) - sla.signm(B)) <= 1e-10
    h = 1e-6
    fd = (sla.signm(B + h * E) - sla.signm(B - h * E)) / (2 * h)
    assert np.linalg.norm(O.frechet_sign(B, E) - fd) <= 1e-6 * np.linalg.norm(fd)


def test_sign_block_structure_is_lyapunov_solution():
    # sign([[A, W], [0, -A^T]]) = [[-I, 2X], [0, I]] with A X + X A^T + W = 0 (Hurwitz A)
    d = gen.convdiff_shifted(grid=4, m=2)
    A, L = d["A"], d["L"]
    W = L @ L.T
    S = O.sign_matrix(O.sign_block(A, W))
    n = A.shape[0]
    X = O.bartels_stewart(A, W)
    assert np.linalg.norm(S[:n, :n] + np.eye(n)) <= 1e-9
    assert np.linalg.norm(S[n:, n:] - np.eye(n)) <= 1e-9
    assert np.linalg.norm(S[:n, n:] - 2 * X) <= 1e-9 * np.linalg.norm(X)



# ----------------------------------------------------------- low-rank ADI (inner solver)

def test_lr_adi_diagonal_closed_form():
    # diagonal A = diag(a): after j steps with shifts p_1..p_j, X - X_j = X o (r r^T) with
    # r_i = prod_k (a_i - p_k) / (a_i + p_k) (the ADI error is R X R^T, R = diag(r))
    a = -np.array([0.3, 1.0, 2.5, 7.0, 20.0])
    L = gen.rng(91).standard_normal((5, 2))
    W = L @ L.T
    X = -W / (a[:, None] + a[None, :])
    opts = O.Opts(u_s="fp64", adi_shifts=3, adi_tol=1e-300, adi_maxit=5, rho=10.0)
    rec = O.ADIRecord(shifts=[-0.5, -2.0, -10.0],
                      inverses=[np.diag(1.0 / (a + p)) for p in (-0.5, -2.0, -10.0)])
    Z, _, Wres, steps = O.lr_adi_chol(np.diag(a), L, opts, rec)
    assert steps == 5
    r = np.ones(5)
    for p in [-0.5, -2.0, -10.0, -0.5, -2.0]:
        r *= (a - p) / (a + p)
    assert np.linalg.norm(Z @ Z.T - X * (1 - np.outer(r, r))) <= 1e-13 * np.linalg.norm(X)
    assert np.linalg.norm(Wres @ Wres.T - W * np.outer(r, r)) <= 1e-13 * np.linalg.norm(W)


def test_lr_adi_residual_identity_and_ir():
    # A X_j + X_j A^T + L S L^T = W_j S W_j^T for a nonsymmetric A (both forms), and the
    # refinement with ADI inner solves reaches the Bartels-Stewart solution
    d = gen.convdiff_shifted(grid=6, m=2)
    A, L = d["A"], d["L"]
    opts = O.Opts(u_s="fp64", adi_maxit=6, adi_tol=1e-300, rho=10.0)
    Z, rec, Wr, _ = O.lr_adi_chol(A, L, opts)
    Xj = Z @ Z.T
    R = A @ Xj + Xj @ A.T + L @ L.T
    assert np.linalg.norm(R - Wr @ Wr.T) <= 1e-10 * np.linalg.norm(L @ L.T)
    s = np.array([1.0, -1.0])
    Zl, yl, _, Wl, _ = O.lr_adi_ldlt(A, L, s, opts, rec)
    Xl = (Zl * yl) @ Zl.T
    Rl = A @ Xl + Xl @ A.T + (L * s) @ L.T
    assert np.linalg.norm(Rl - (Wl * s) @ Wl.T) <= 1e-10 * np.linalg.norm(L @ L.T)
    X = O.bartels_stewart(A, L @ L.T)
    Zi, info = O.ir_chol(A, L, O.Opts(u_s="fp16", inner="adi", tau_ir=1e-13))
    assert info.converged
    assert rel(Zi @ Zi.T, X) <= 1e-10


def test_ir_working_precision_fp32_limits_the_residual():
    # Table 2.1 (u = fp32 rows): with the residual factors and the solution factor stored in
    # FP32 the refinement reaches the default tau = n u (u = 2^-24) and stalls near u; with
    # u = fp64 the same refinement goes on to FP64 level
    d = gen.paper_synthetic(100, 1.0)
    A, L = d["A"], d["L"]
    Z, info = O.ir_chol(A, L, O.Opts(u_s="fp16", u="fp32"))
    assert info.converged and info.res_final <= 100 * 2.0 ** -24
    _, forced = O.ir_chol(A, L, O.Opts(u_s="fp16", u="fp32", tau_ir=1e-30, imax=12))
    assert forced.stagnated and 1e-10 < forced.res_final < 100 * 2.0 ** -24
    _, f64 = O.ir_chol(A, L, O.Opts(u_s="fp16", u="fp64", tau_ir=1e-30, imax=12))
    assert f64.res_final < 1e-14
    s = np.array([1.0, -1.0, 1.0])
    _, _, fl = O.ir_ldlt(A, L, np.diag(s), O.Opts(u_s="fp16", u="fp32", tau_ir=1e-30, imax=12))
    assert 1e-10 < fl.res_final < 100 * 2.0 ** -24


# ----------------------------------------------------------- extended Krylov (inner solver)

def test_eksm_residual_formula_and_exactness():
    # the Galerkin residual norm sqrt(2) ||U_{j+1}^T A V_j Y||_F equals the explicit residual
    # (A V_j lies in span V_{j+1}); once the space is all of R^n the projection is exact
    d = gen.convdiff_shifted(grid=8, m=2)
    A, L = d["A"], d["L"]
    W = L @ L.T
    for steps in (2, 4):
        Z, _, st, res = O.eksm_chol(A, L, O.Opts(u_s="fp64", eksm_maxit=steps, adi_tol=1e-300))
        Xk = Z @ Z.T
        R = A @ Xk + Xk @ A.T + W
        assert st == steps and abs(res - np.linalg.norm(R)) <= 1e-9 * np.linalg.norm(R)
    # the space after 3 steps is span{L, A^-1 L, A L, A^-2 L, A^2 L, A^-3 L} (the block
    # powers written out and orthonormalised at once), and X_3 is the Galerkin solution on
    # it (the projected equation solved by the library's Lyapunov routine)
    Ai = np.linalg.inv(A)
    K = np.hstack([L, Ai @ L, A @ L, Ai @ Ai @ L, A @ A @ L, Ai @ Ai @ Ai @ L])
    Vk, _ = np.linalg.qr(K)
    s = np.array([1.0, -1.0])
    for y in (None, s):
        ys = np.ones(2) if y is None else y
        Tk = Vk.T @ A @ Vk
        Ek = Vk.T @ L
        Yk = sla.solve_continuous_lyapunov(Tk, -(Ek * ys) @ Ek.T)
        Xref = Vk @ Yk @ Vk.T
        if y is None:
            Z, _, _, _ = O.eksm_chol(A, L, O.Opts(u_s="fp64", eksm_maxit=3, adi_tol=1e-300))
            assert rel(Z @ Z.T, Xref) <= 1e-9
        else:
            Zl, yl, _, _, _ = O.eksm_ldlt(A, L, y, O.Opts(u_s="fp64", eksm_maxit=3, adi_tol=1e-300))
            assert rel((Zl * yl) @ Zl.T, Xref) <= 1e-9


def test_ir_with_eksm_inner_converges():
    d = gen.convdiff_shifted(grid=8, m=2)
    A, L = d["A"], d["L"]
    Z, info = O.ir_chol(A, L, O.Opts(u_s="fp16", inner="eksm", tau_ir=1e-13))
    assert info.converged and rel(Z @ Z.T, O.bartels_stewart(A, L @ L.T)) <= 1e-10
    d = gen.paper_synthetic(60, 1.0)
    S = np.diag([1.0, -1.0, 1.0])
    Zl, yl, il = O.ir_ldlt(d["A"], d["L"], S, O.Opts(u_s="fp16", inner="eksm", tau_ir=1e-13))
    assert il.converged
    assert rel((Zl * yl) @ Zl.T, O.bartels_stewart(d["A"], d["L"] @ S @ d["L"].T)) <= 1e-10
