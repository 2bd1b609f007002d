"""Solver-level parity of the CUDA path (C ABI) with the CPU oracle: the
sign-Newton solver (Algorithms Newton-Chol / Newton-LDLT) and the mixed-precision
IR algorithms, checked against the exact solution (Schur method), the relative residual
of Eq. (4.1), and the iteration counts that depend on A only."""
import json
import os

import numpy as np
import pytest

import lyapgen as gen
import oracle as O
from tests.gpu_util import N, T, rel

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def lib():
    from paper_2510_02126_gb300 import lyap
    return lyap


FP64_LAPLACE = dict(u_s="fp64", scaling="det", newton_norm_fro=1, rho=0.0, rank_tol=1e-14)


@pytest.mark.parametrize("grid", [4, 8])
def test_sign_solve_fp64_laplacian(grid):
    d = gen.fp64_laplacian(grid, 2)
    A, L = d["A"], d["L"]
    n = A.shape[0]
    W = L @ L.T
    X = O.bartels_stewart(A, W)
    Z, _, info = lib().sign_solve(T(A), T(L), tau_newton=1e-12 * n, **FP64_LAPLACE)
    Z = N(Z)
    opts = O.Opts(u_s="fp64", scaling="det", newton_norm="fro", tau_newton=1e-12 * n, rho=0.0, rank_tol=1e-14)
    Zo, rec = O.newton_chol(A, L, opts)
    assert info.newton_max == len(rec.inverses)
    assert np.allclose(list(info.mu)[1:info.newton_max], rec.mus[1:], rtol=1e-9)
    assert rel(Z @ Z.T, X) <= 1e-10
    assert O.residual_eq41(A, Z, W) <= 1e-12
    assert abs(Z.shape[1] - Zo.shape[1]) <= 2


def test_table41_fp64_counts_on_gpu():
    gold = json.load(open(os.path.join(HERE, "golden", "table41_fp64_newton_counts.json")))
    for q, alpha in zip(gold["q"], gold["alpha"]["100"]["chol"]):
        d = gen.paper_synthetic(100, q)
        Z, _, info = lib().sign_solve(T(d["A"]), T(d["L"]), u_s="fp64")
        assert info.newton_max == alpha, (q, info.newton_max, alpha)
        X = O.bartels_stewart(d["A"], d["L"] @ d["L"].T)
        assert rel(N(Z) @ N(Z).T, X) <= 1e-10


@pytest.mark.parametrize("u_s,kappa", [("fp64", 1e3), ("fp32", 1e3), ("fp16", 1e2), ("fp16", 1e3), ("bf16", 1e2)])
def test_ir_chol_convdiff(u_s, kappa):
    d = gen.convdiff_shifted(grid=12, m=3, kappa=kappa)
    A, L = d["A"], d["L"]
    W = L @ L.T
    X = O.bartels_stewart(A, W)
    Z, _, info = lib().solve_ir(T(A), T(L), u_s=u_s, tau_ir=1e-12)
    Z = N(Z)
    assert info.converged, info.as_dict()
    assert O.residual_eq41(A, Z, W) <= 1e-12
    assert rel(Z @ Z.T, X) <= 1e-10
    assert abs(info.res_final - O.residual_eq41(A, Z, W)) <= 1e-3 * info.res_final + 1e-16
    # the inverse sequence is computed once and replayed by every correction solve
    assert info.n_inversions == info.newton_max
    assert info.newton_total == info.newton_calls * info.newton_max


@pytest.mark.parametrize("u_s,p", [("fp64", 1), ("fp32", 2), ("fp16", 1), ("fp16", 2)])
def test_ir_ldlt_indefinite(u_s, p):
    d = gen.normal_blocks(n=128, p=p, m=4)
    A, L, S = d["A"], d["L"], d["S"]
    W = L @ S @ L.T
    X = O.bartels_stewart(A, W)
    Z, D, info = lib().solve_ir(T(A), T(L), S=T(S), u_s=u_s, tau_ir=1e-12)
    Z, D = N(Z), N(D)
    assert info.converged, info.as_dict()
    assert O.residual_eq41(A, Z, W, D) <= 1e-12
    assert rel((Z * D) @ Z.T, X) <= 1e-10


def test_ir_ldlt_bf16_normal_blocks_stalls_like_oracle():
    # the input on which BF16 inner solves cannot converge (the oracle's BF16 emulation stalls
    # as well, tests/test_oracle_pins.py): the GPU refinement stops by the stagnation rule with
    # a residual of the oracle's order, far above the FP64 limit
    d = gen.normal_blocks(n=128, p=1, m=4)
    A, L, S = d["A"], d["L"], d["S"]
    Z, D, info = lib().solve_ir(T(A), T(L), S=T(S), u_s="bf16", tau_ir=1e-12, imax=20)
    assert not info.converged and info.status in (lib().WARN_STAGNATED, lib().WARN_MAXIT), info.as_dict()
    Zo, yo, oinfo = O.ir_ldlt(A, L, S, O.Opts(u_s="bf16", tau_ir=1e-12, imax=20))
    assert not oinfo.converged
    assert 0.1 <= info.res_final / oinfo.res_final <= 10.0, (info.res_final, oinfo.res_final)


def test_ir_ldlt_indefinite_n1024_fp32():
    # LDL^T form at n = 1024 (indefinite S, normal blocks, p = 1) with FP32 inner solves,
    # against the Schur-block closed form of the exact solution
    from tests.test_oracle_pins import schur_blocks_solution
    d = gen.normal_blocks(n=1024, p=1, m=8, indefinite=True)
    A, L, S = d["A"], d["L"], d["S"]
    W = L @ S @ L.T
    Z, D, info = lib().solve_ir(T(A), T(L), S=T(S), u_s="fp32", tau_ir=1e-12, imax=20)
    assert info.converged, info.as_dict()
    X = schur_blocks_solution(d["Q"], d["alpha"], d["beta"], W)
    assert rel((N(Z) * N(D)) @ N(Z).T, X) <= 1e-10
    assert O.residual_eq41(A, N(Z), W, N(D)) <= 1e-12


def test_ir_ldlt_bf16_synthetic():
    # bf16 needs a mild problem (Table 4.1: bf16 converges up to cond ~1e2 at n = 100);
    # on the normal-block family with Re(lambda) down to -0.1 the oracle stalls as well
    d = gen.paper_synthetic(100, 1.0)
    A, L = d["A"], d["L"]
    X = O.bartels_stewart(A, L @ L.T)
    Z, D, info = lib().solve_ir(T(A), T(L), S=T(np.eye(3)), u_s="bf16", tau_ir=1e-12)
    assert info.converged, info.as_dict()
    assert rel((N(Z) * N(D)) @ N(Z).T, X) <= 1e-10


def test_ir_ldlt_psd_matches_chol():
    d = gen.paper_synthetic(80, 1.5)
    A, L = d["A"], d["L"]
    X = O.bartels_stewart(A, L @ L.T)
    Z, D, info = lib().solve_ir(T(A), T(L), S=T(np.eye(3)), u_s="fp16", tau_ir=1e-12)
    assert info.converged
    assert np.all(N(D) > 0)
    assert rel((N(Z) * N(D)) @ N(Z).T, X) <= 1e-10


def test_ir_config_convdiff_1024_fp16():
    d = gen.convdiff_shifted()
    A, L = d["A"], d["L"]
    W = L @ L.T
    Z, _, info = lib().solve_ir(T(A), T(L), u_s="fp16", tau_ir=1e-12, imax=50)
    Z = N(Z)
    res = O.residual_eq41(A, Z, W)
    assert info.converged and res <= 1e-12, (res, info.as_dict())
    X = O.bartels_stewart(A, W)
    assert rel(Z @ Z.T, X) <= 1e-10


def test_ir_config_convdiff_1024_bf16():
    # the BF16 variant of the n = 1024 workload: kappa ~ 1e3 is at the Table 2.1 bound of
    # bf16, so the refinement contracts slowly (about x0.5 per step) but reaches 1e-12
    d = gen.convdiff_shifted()
    A, L = d["A"], d["L"]
    W = L @ L.T
    Z, _, info = lib().solve_ir(T(A), T(L), u_s="bf16", tau_ir=1e-12, imax=50)
    Z = N(Z)
    res = O.residual_eq41(A, Z, W)
    assert info.converged and res <= 1e-12, (res, info.as_dict())
    assert info.n_inversions == info.newton_max
    X = O.bartels_stewart(A, W)
    assert rel(Z @ Z.T, X) <= 1e-10


def test_fp64_sign_newton_config_convdiff_1024():
    d = gen.convdiff_shifted()
    A, L = d["A"], d["L"]
    W = L @ L.T
    Z, _, info = lib().sign_solve(T(A), T(L), u_s="fp64")
    rec = O.newton_sequence(A, O.Opts(u_s="fp64"))
    assert info.newton_max == len(rec.inverses)
    assert O.residual_eq41(A, N(Z), W) <= 1e-12


# ---------------------------------------------------------------- edge cases

def test_scalar_equation():
    A = np.array([[-2.0]])
    L = np.array([[3.0]])
    Z, _, info = lib().solve_ir(T(A), T(L), u_s="fp16", tau_ir=1e-14)
    assert abs(N(Z)[0, 0] ** 2 - 9.0 / 4.0) <= 1e-13


def test_single_rhs_column_fp32():
    d = gen.convdiff_shifted(grid=7, m=1)
    A, L = d["A"], d["L"]
    X = O.bartels_stewart(A, L @ L.T)
    Z, _, info = lib().solve_ir(T(A), T(L), u_s="fp32", tau_ir=1e-12)
    assert rel(N(Z) @ N(Z).T, X) <= 1e-10


def test_capacity_error():
    d = gen.convdiff_shifted(grid=6, m=2)
    with pytest.raises(Exception) as ei:
        lib().solve_ir(T(d["A"]), T(d["L"]), u_s="fp64", z_cap=2)
    assert getattr(ei.value, "status", None) == lib().ERR_CAPACITY


def test_mixed_working_precisions_rejected():
    # the presets are u = u_r = u_c = FP64 or FP32 (Table 2.1); mixed settings and 16-bit
    # working precisions are rejected
    d = gen.convdiff_shifted(grid=5, m=2)
    for field in ("u", "u_r", "u_c"):
        o = lib().make_opts("fp16", **{field: lib().FP32})
        with pytest.raises(Exception) as ei:
            lib().solve_ir(T(d["A"]), T(d["L"]), opts=o)
        assert getattr(ei.value, "status", None) == lib().ERR_ARG
    o = lib().make_opts("fp16", u=lib().FP16, u_r=lib().FP16, u_c=lib().FP16)
    with pytest.raises(Exception) as ei:
        lib().solve_ir(T(d["A"]), T(d["L"]), opts=o)
    assert getattr(ei.value, "status", None) == lib().ERR_ARG


@pytest.mark.parametrize("form", ["chol", "ldlt"])
def test_working_precision_fp32_preset(form):
    # u = u_r = u_c = FP32 (Table 2.1, top half): the refinement reaches tau = n u of FP32 and,
    # pushed further, stalls near u, as the oracle with the same storage points does; the
    # FP64 preset goes on to FP64 level on the same input
    d = gen.paper_synthetic(100, 1.0)
    A, L = d["A"], d["L"]
    S = np.diag([1.0, -1.0, 1.0]) if form == "ldlt" else None
    Sg = T(S) if S is not None else None
    f32 = dict(u=lib().FP32, u_r=lib().FP32, u_c=lib().FP32)
    _, _, info = lib().solve_ir(T(A), T(L), S=Sg, opts=lib().make_opts("fp16", **f32))
    assert info.converged and info.res_final <= 100 * 2.0 ** -24, info.as_dict()
    _, _, forced = lib().solve_ir(T(A), T(L), S=Sg, opts=lib().make_opts("fp16", tau_ir=1e-30, imax=12, **f32))
    assert forced.status == lib().WARN_STAGNATED
    assert 1e-10 < forced.res_final < 100 * 2.0 ** -24, forced.as_dict()
    if form == "chol":
        _, ref = O.ir_chol(A, L, O.Opts(u_s="fp16", u="fp32", tau_ir=1e-30, imax=12))
    else:
        _, _, ref = O.ir_ldlt(A, L, S, O.Opts(u_s="fp16", u="fp32", tau_ir=1e-30, imax=12))
    assert ref.res_final / 30 <= forced.res_final <= 30 * ref.res_final, (forced.res_final, ref.res_final)
    _, _, f64 = lib().solve_ir(T(A), T(L), S=Sg, opts=lib().make_opts("fp16", tau_ir=1e-30, imax=12))
    assert f64.res_final < 1e-14


def test_nonfinite_input():
    d = gen.convdiff_shifted(grid=5, m=2)
    A = d["A"].copy()
    A[1, 2] = np.inf
    with pytest.raises(Exception) as ei:
        lib().solve_ir(T(A), T(d["L"]), u_s="fp16")
    assert getattr(ei.value, "status", None) == lib().ERR_NONFINITE


def test_non_hurwitz_does_not_converge():
    # eigenvalues +-i on the imaginary axis: the sign function is undefined
    A = np.kron(np.eye(4), np.array([[0.0, 1.0], [-1.0, 0.0]]))
    L = np.ones((8, 1))
    with pytest.raises(Exception) as ei:
        lib().sign_solve(T(A), T(L), u_s="fp64", kmax=30)
    assert getattr(ei.value, "status", None) in (lib().ERR_NOCONV, lib().ERR_NONFINITE, lib().ERR_SINGULAR)


def test_fp64_sign_newton_ldlt_nearly_full_rank():
    # block-normal A (eigenvalues -a +- ib), indefinite W = L S L^T: the solution has rank
    # close to n, so every compression is an order-n FP64 eigendecomposition (RankTruncLdlt)
    d = gen.normal_blocks(n=512, p=2, m=8, indefinite=True, seed=gen.SEED_BASE + 60)
    A, L, S = d["A"], d["L"], d["S"]
    Z, D, info = lib().sign_solve(T(A), T(L), T(S), u_s="fp64")
    assert info.status == 0
    assert info.res_final <= 1e-13
    X = (N(Z) * N(D)[None, :]) @ N(Z).T
    Xo = O.bartels_stewart(A, L @ S @ L.T)
    assert np.linalg.norm(X - Xo) <= 1e-11 * np.linalg.norm(Xo)


# ------------------------------------------------- Sec. 4.2 synthetic study (Table 4.1)

def _sine_basis_solution(d):
    # A = -V diag(d) V^T with V symmetric orthogonal: V X V = (V W V)_ij / (d_i + d_j)
    V, dd, L = d["V"], d["d"], d["L"]
    Wt = V @ (L @ L.T) @ V
    return V @ (Wt / (dd[:, None] + dd[None, :])) @ V


def test_table41_fp64_counts_n1000_on_gpu():
    gold = json.load(open(os.path.join(HERE, "golden", "table41_fp64_newton_counts.json")))
    for q, alpha in zip(gold["q"], gold["alpha"]["1000"]["chol"]):
        d = gen.paper_synthetic(1000, q)
        Z, _, info = lib().sign_solve(T(d["A"]), T(d["L"]), u_s="fp64")
        assert info.newton_max == alpha, (q, info.newton_max, alpha)
        X = _sine_basis_solution(d)
        assert rel(N(Z) @ N(Z).T, X) <= 1e-10, q


def test_table41_fp32_inner_counts_n100_on_gpu():
    # Table 4.1, Cholesky type, n = 100, u_s = fp32: varsigma(alpha) printed per cond.  FP32
    # is the one inner precision that the GPU computes in the paper's own arithmetic
    # (IEEE single throughout), so the counts must agree, not only the final residual.
    gold = json.load(open(os.path.join(HERE, "golden", "table41_fp64_newton_counts.json")))
    g = gold["fp32_inner_iter_u64_n100_chol"]
    for q, tot, al in zip(g["q"], g["total"], g["alpha"]):
        d = gen.paper_synthetic(100, q)
        Z, _, info = lib().solve_ir(T(d["A"]), T(d["L"]), u_s="fp32")
        assert info.converged, q
        assert (info.newton_total, info.newton_max) == (tot, al), (q, info.newton_total, info.newton_max)
        assert rel(N(Z) @ N(Z).T, _sine_basis_solution(d)) <= 1e-10, q


# ------------------------------------------------------------- stagnation (Eq. (4.2))

def _stagnation_stop(hist, theta=0.9, count=2):
    """Index of the residual at which the rule of Eq. (4.2) stops the refinement (theta
    exceeded `count` times in a row), or None."""
    stag = 0
    for i in range(1, len(hist)):
        stag = stag + 1 if hist[i] / hist[i - 1] > theta else 0
        if stag >= count:
            return i
    return None


def test_ir_stagnation_rule_on_gpu():
    # tau_ir below the FP64 floor: the FP16-inner refinement falls to ~1e-16 and then
    # stalls; the rule of Eq. (4.2) (theta > 0.9 twice in a row) must stop it with
    # LYAP_WARN_STAGNATED at the first place the history allows, returning the best factor.
    lp = lib()
    d = gen.paper_synthetic(100, 1.0)
    A, L = d["A"], d["L"]
    W = L @ L.T
    Z, _, info = lp.solve_ir(T(A), T(L), u_s="fp16", tau_ir=1e-30, imax=50)
    assert info.status == lp.WARN_STAGNATED and info.stagnated and not info.converged, info.as_dict()
    hist = list(info.res_hist[: info.n_res])
    assert _stagnation_stop(hist) == len(hist) - 1, hist
    assert info.res_final == min(hist)
    assert info.res_final <= 1e-14
    assert abs(O.residual_eq41(A, N(Z), W) - info.res_final) <= 1e-2 * info.res_final + 1e-17
    # the oracle stagnates on the same input at the FP64 floor as well; the GPU's best
    # residual is at least as small (its FP16 inner solves accumulate in FP32)
    Zo, oinfo = O.ir_chol(A, L, O.Opts(u_s="fp16", tau_ir=1e-30))
    assert oinfo.stagnated and not oinfo.converged
    assert _stagnation_stop(oinfo.res_hist) == len(oinfo.res_hist) - 1
    assert oinfo.res_final <= 1e-14
    assert info.res_final <= 10.0 * oinfo.res_final, (info.res_final, oinfo.res_final)


def test_ir_ldlt_indefinite_n4096_fp32():
    # the LDL^T family at full size (n = 4096, indefinite S, normal blocks, p = 1), FP32 inner
    # solves: the projected-update eigenproblems reach order ~4096 (Jacobi over super-blocks);
    # the result against the Schur-block closed form and the oracle's Eq. (4.1)
    from tests.test_oracle_pins import schur_blocks_solution
    d = gen.normal_blocks(n=4096, p=1, m=8, indefinite=True)
    A, L, S = d["A"], d["L"], d["S"]
    W = L @ S @ L.T
    Z, D, info = lib().solve_ir(T(A), T(L), S=T(S), u_s="fp32", tau_ir=1e-12, imax=20)
    assert info.converged, info.as_dict()
    X = schur_blocks_solution(d["Q"], d["alpha"], d["beta"], W)
    Zn, Dn = N(Z), N(D)
    assert rel((Zn * Dn) @ Zn.T, X) <= 1e-10
    assert O.residual_eq41(A, Zn, W, Dn) <= 1e-12
    assert abs(info.res_final - O.residual_eq41(A, Zn, W, Dn)) <= 1e-3 * info.res_final


@pytest.mark.parametrize("scaling", ["norm2", "spectral"])
def test_sign_solve_norm2_and_spectral_scaling(scaling):
    # the 2-norm and spectral scalings of Sec. 3.1: the GPU estimates ||.||_2 and rho(.) by
    # power iteration, the oracle takes them exactly.  On the nonsymmetric convection-
    # diffusion matrix (n = 144): mu_k (k >= 1; mu_0 also carries the power-of-two prescale
    # of A_0) within 5% while scaling is on, the Newton count within one step, and the same
    # solution; FP16-inner refinement with this scaling converges to 1e-12
    d = gen.convdiff_shifted(grid=12, m=2)
    A, L = d["A"], d["L"]
    W = L @ L.T
    X = O.bartels_stewart(A, W)
    rec = O.newton_sequence(A, O.Opts(u_s="fp64", scaling=scaling))
    Z, _, info = lib().sign_solve(T(A), T(L), u_s="fp64", scaling=scaling)
    assert abs(info.newton_max - len(rec.mus)) <= 1
    mu = list(info.mu)
    checked = 0
    for k in range(1, min(info.newton_max, len(rec.mus))):
        if rec.mus[k] == 1.0:
            break
        assert abs(mu[k] - rec.mus[k]) <= 0.05 * rec.mus[k], (k, mu[k], rec.mus[k])
        checked += 1
    assert checked >= 1
    assert rel(N(Z) @ N(Z).T, X) <= 1e-10
    Z2, _, info2 = lib().solve_ir(T(A), T(L), u_s="fp16", scaling=scaling, tau_ir=1e-12, imax=30)
    assert info2.converged, info2.as_dict()
    assert rel(N(Z2) @ N(Z2).T, X) <= 1e-10
    assert O.residual_eq41(A, N(Z2), W) <= 1e-12


# ------------------------------------------------ low-rank ADI as the inner solver

def test_adi_single_solve_fp64_matches_bartels_stewart():
    # lyap_sign_solve with inner = ADI at FP64: one low-rank ADI solve to ||W W^T|| <= 1e-14
    d = gen.convdiff_shifted(grid=10, m=2)
    A, L = d["A"], d["L"]
    X = O.bartels_stewart(A, L @ L.T)
    Z, _, info = lib().sign_solve(T(A), T(L), u_s="fp64", inner="adi", adi_shifts=10, rho=0.5)
    assert rel(N(Z) @ N(Z).T, X) <= 1e-10
    # the shifts are recorded in info.mu: negative and ascending (largest magnitude first)
    p = np.array(list(info.mu)[:10])
    assert np.all(p < 0) and np.all(np.diff(p) > 0)


@pytest.mark.parametrize("u_s", ["fp16", "fp32"])
def test_ir_chol_adi_inner_matches_oracle(u_s):
    # IR-Chol with low-rank ADI inner solves (16-bit / FP32 shifted inverses, stored once and
    # reused by every correction): the FP64 refinement reaches 1e-12 and the Bartels-Stewart
    # solution, as the oracle's IR with its ADI solver does on the same input
    d = gen.convdiff_shifted(grid=20, m=3)
    A, L = d["A"], d["L"]
    W = L @ L.T
    X = O.bartels_stewart(A, W)
    Z, _, info = lib().solve_ir(T(A), T(L), u_s=u_s, inner="adi", tau_ir=1e-12, imax=30)
    assert info.converged, info.as_dict()
    assert rel(N(Z) @ N(Z).T, X) <= 1e-10
    assert O.residual_eq41(A, N(Z), W) <= 1e-12
    assert info.n_inversions == 8                      # the shifted inverses, computed once
    Zo, io = O.ir_chol(A, L, O.Opts(u_s=u_s, inner="adi", tau_ir=1e-12, imax=30))
    assert io.converged
    # the GPU's shifted inverses are 16-bit operands with FP32 accumulation, the oracle rounds
    # every matrix result to u_s: the GPU contracts at least as fast (3 against 7 steps at FP16)
    assert info.ir_steps <= io.ir_steps + 1, (info.ir_steps, io.ir_steps)


def test_ir_ldlt_adi_inner_indefinite():
    # IR-LDLT with ADI inner solves on the Sec. 4.2 family (symmetric A, real spectrum) with
    # an indefinite S: against the Bartels-Stewart solution of the indefinite equation
    d = gen.paper_synthetic(120, 1.0)
    A, L = d["A"], d["L"]
    S = np.diag([1.0, -1.0, 1.0])
    W = L @ S @ L.T
    X = O.bartels_stewart(A, W)
    Z, D, info = lib().solve_ir(T(A), T(L), S=T(S), u_s="fp16", inner="adi", tau_ir=1e-12, imax=30)
    assert info.converged, info.as_dict()
    assert rel((N(Z) * N(D)) @ N(Z).T, X) <= 1e-10
    assert O.residual_eq41(A, N(Z), W, N(D)) <= 1e-12


# ------------------------------------------------ extended Krylov as the inner solver

def test_eksm_single_solve_fp64_matches_bartels_stewart():
    # lyap_sign_solve with inner = EKSM at FP64 (Sec. 4.2 family: symmetric negative definite A,
    # so every projected matrix is stable): one Galerkin solve to a residual of 1e-14
    d = gen.paper_synthetic(100, 1.0)
    A, L = d["A"], d["L"]
    X = O.bartels_stewart(A, L @ L.T)
    Z, _, info = lib().sign_solve(T(A), T(L), u_s="fp64", inner="eksm")
    assert rel(N(Z) @ N(Z).T, X) <= 1e-10
    assert info.n_inversions == 1


@pytest.mark.parametrize("form", ["chol", "ldlt"])
def test_ir_eksm_inner_matches_bartels_stewart(form):
    # the refinement with extended Krylov inner solves (A^-1 stored once at FP16 and reused by
    # every correction) reaches 1e-12 and the exact solution, as the oracle's does
    d = gen.paper_synthetic(200, 1.5)
    A, L = d["A"], d["L"]
    S = np.diag([1.0, -1.0, 1.0]) if form == "ldlt" else np.eye(3)
    W = L @ S @ L.T
    X = O.bartels_stewart(A, W)
    Z, D, info = lib().solve_ir(T(A), T(L), S=T(S) if form == "ldlt" else None, u_s="fp16", inner="eksm",
                                tau_ir=1e-12, imax=30)
    assert info.converged, info.as_dict()
    Xg = (N(Z) * N(D)) @ N(Z).T if form == "ldlt" else N(Z) @ N(Z).T
    assert rel(Xg, X) <= 1e-10
    assert info.n_inversions == 1
    if form == "chol":
        _, io = O.ir_chol(A, L, O.Opts(u_s="fp16", inner="eksm", tau_ir=1e-12, imax=30))
    else:
        _, _, io = O.ir_ldlt(A, L, S, O.Opts(u_s="fp16", inner="eksm", tau_ir=1e-12, imax=30))
    assert io.converged
