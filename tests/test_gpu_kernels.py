"""Kernel-level parity of the CUDA path (through the C ABI) against the CPU oracle
and against the mathematics of each kernel: inversion (K1-K3), QR with column
pivoting (K6), symmetric eigendecomposition (K9), residual verifier (K13)."""
import numpy as np
import pytest
import scipy.linalg as sla

import lyapgen as gen
import oracle as O
from tests.gpu_util import N, T, rel

pytestmark = pytest.mark.gpu


def lib():
    from paper_2510_02126_gb300 import lyap
    return lyap


@pytest.mark.parametrize("n", [1, 2, 17, 31, 32, 33, 64, 100, 257, 1024])
def test_invert_fp64_matches_lapack_and_pivots(n):
    g = gen.rng(1000 + n)
    A = g.standard_normal((n, n))
    Ai, ipiv, logdet = lib().invert(T(A), "fp64")
    Ai = N(Ai)
    ref = np.linalg.inv(A)
    assert rel(Ai, ref) < 1e-10 * max(1.0, np.linalg.cond(A) / 1e3)
    # the pivot sequence is the getrf one (largest |a_ij|, lowest row on ties)
    _, _, piv = O.getrf_pp(A)
    assert np.array_equal(N(ipiv).astype(np.int64), piv)
    assert abs(logdet - np.linalg.slogdet(A)[1]) < 1e-9 * max(1.0, abs(logdet))


@pytest.mark.parametrize("prec,u", [("fp32", 2.0 ** -24), ("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
@pytest.mark.parametrize("n", [7, 64, 130, 512, 1024])
def test_invert_low_precision_error_bound(prec, u, n):
    g = gen.rng(2000 + n)
    A = g.standard_normal((n, n)) + 2 * n ** 0.5 * np.eye(n)  # moderately conditioned
    Ai = N(lib().invert(T(A), prec)[0])
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(A @ Ai - np.eye(n)) / np.sqrt(n)
    assert err <= 10 * n ** 0.5 * u * kappa, (err, kappa)


def test_invert_bf16_and_fp16_use_distinct_rounding():
    g = gen.rng(77)
    A = g.standard_normal((256, 256)) + 16 * np.eye(256)
    e16 = np.linalg.norm(A @ N(lib().invert(T(A), "fp16")[0]) - np.eye(256))
    eb = np.linalg.norm(A @ N(lib().invert(T(A), "bf16")[0]) - np.eye(256))
    e32 = np.linalg.norm(A @ N(lib().invert(T(A), "fp32")[0]) - np.eye(256))
    assert e32 < e16 < eb


def test_invert_singular_reports_error():
    A = np.ones((8, 8))
    with pytest.raises(Exception) as ei:
        lib().invert(T(A), "fp64")
    assert getattr(ei.value, "status", None) == lib().ERR_SINGULAR


def test_invert_nonfinite_reports_error():
    A = np.eye(8)
    A[3, 3] = np.nan
    with pytest.raises(Exception) as ei:
        lib().invert(T(A), "fp64")
    assert getattr(ei.value, "status", None) in (lib().ERR_NONFINITE, lib().ERR_SINGULAR)


@pytest.mark.parametrize("n,r,c", [(80, 7, 30), (1024, 40, 200), (64, 1, 3), (33, 33, 33)])
def test_rank_trunc_exact_rank(n, r, c):
    g = gen.rng(n + r + c)
    Z = g.standard_normal((n, r)) @ g.standard_normal((r, c))
    Zt = N(lib().rank_trunc(T(Z), 1e-10))
    assert Zt.shape[1] == min(r, c)
    assert rel(Zt @ Zt.T, Z @ Z.T) < 1e-11


def test_rank_trunc_matches_oracle_rank_and_bound():
    g = gen.rng(5)
    n, c = 300, 60
    U, _ = np.linalg.qr(g.standard_normal((n, c)))
    Z = (U * 10.0 ** -np.linspace(0, 14, c)) @ np.linalg.qr(g.standard_normal((c, c)))[0]
    for tol in (1e-4, 1e-8, 1e-12):
        Zt = N(lib().rank_trunc(T(Z), tol))
        Zo = O.rank_trunc_chol(Z, tol)
        assert abs(Zt.shape[1] - Zo.shape[1]) <= 1
        err = np.linalg.norm(Z @ Z.T - Zt @ Zt.T, 2)
        # truncation bound of RankTruncChol plus the FP64 rounding of the products
        assert err <= 1.01 * (tol * np.linalg.norm(Z, 2)) ** 2 + 50 * n * 2.0 ** -53 * np.linalg.norm(Z, 2) ** 2


@pytest.mark.parametrize("q", [1, 2, 5, 64, 129, 160, 161, 300])
@pytest.mark.parametrize("refine", [False, True])
def test_sym_eig(q, refine):
    g = gen.rng(300 + q)
    B = g.standard_normal((q, q))
    H = (B + B.T) / 2
    H[0, 0] += 3.0
    w, Q = lib().sym_eig(T(H), refine)
    w, Q = N(w), N(Q)
    wref = np.linalg.eigvalsh(H)
    tol = 1e-12 if refine else 2e-5
    nh = np.linalg.norm(H, 2)
    assert np.max(np.abs(w - wref)) <= tol * nh * max(1, q ** 0.5)
    assert np.linalg.norm(H @ Q - Q * w) <= tol * nh * q
    assert np.linalg.norm(Q.T @ Q - np.eye(q)) <= tol * q
    assert np.all(np.diff(w) >= -tol * nh)


def test_residual_verifier_matches_explicit():
    d = gen.convdiff_shifted(grid=10, m=3)
    A, L = d["A"], d["L"]
    g = gen.rng(9)
    Z = g.standard_normal((100, 12))
    res = lib().residual(T(A), T(L), T(Z))
    ref = O.residual_eq41(A, Z, L @ L.T)
    assert abs(res - ref) <= 1e-12 * ref
    S = np.diag([1.0, -1.0, 2.0])
    y = g.standard_normal(12)
    res = lib().residual(T(A), T(L), T(Z), S=T(S), D=T(y))
    ref = O.residual_eq41(A, Z, L @ S @ L.T, y)
    assert abs(res - ref) <= 1e-12 * ref


@pytest.mark.parametrize("kind", ["random", "graded"])
def test_sym_eig_fp64_accuracy_large(kind):
    # block Jacobi (q > 160) + FP64 refinement at q = 1024: FP64-accurate pairs
    q = 1024
    g = gen.rng(900 + (kind == "graded"))
    if kind == "random":
        B = g.standard_normal((q, q))
        H = (B + B.T) / 2
    else:  # eigenvalues 1 .. 1e-16, the spectrum shape of the projected-update cores
        Qm, _ = np.linalg.qr(g.standard_normal((q, q)))
        H = (Qm * 10.0 ** (-16.0 * np.arange(q) / q)) @ Qm.T
    w, Q = lib().sym_eig(T(H), True)
    w, Q = N(w), N(Q)
    nh = np.linalg.norm(H, 2)
    assert np.max(np.abs(w - np.linalg.eigvalsh(H))) <= 1e-13 * nh
    assert np.max(np.abs(Q.T @ Q - np.eye(q))) <= 1e-13
    S = Q.T @ H @ Q
    assert np.linalg.norm(S - np.diag(np.diag(S)), 2) <= 1e-13 * nh


@pytest.mark.parametrize("refine", [False, True])
def test_sym_eig_order_beyond_split_grid(refine):
    # q = 1260: 79 block pairs, so 2 x 79 CTAs exceed the 152 SMs of a GB300 and the block
    # Jacobi runs without a separate eigenvector side (each pair CTA also updates V);
    # below the order limit 1280, with a padded tail (1260 = 78 x 16 + 12)
    q = 1260
    g = gen.rng(1260)
    B = g.standard_normal((q, q))
    H = (B + B.T) / 2
    w, Q = lib().sym_eig(T(H), refine)
    w, Q = N(w), N(Q)
    nh = np.linalg.norm(H, 2)
    tol = 1e-13 if refine else 2e-5
    assert np.max(np.abs(w - np.linalg.eigvalsh(H))) <= tol * nh * (1 if refine else q ** 0.5)
    assert np.max(np.abs(Q.T @ Q - np.eye(q))) <= (1e-13 if refine else 1e-4)
    S = Q.T @ H @ Q
    assert np.linalg.norm(S - np.diag(np.diag(S)), 2) <= tol * nh * (1 if refine else q ** 0.5)


@pytest.mark.parametrize("q,refine", [(1500, False), (1500, True), (4096, False), (4096, True), (8192, True)])
def test_sym_eig_super_block_orders(q, refine):
    # orders above the block Jacobi's 1280: Jacobi over super-blocks of at most 512 indices
    # (uneven at 1500: 4 blocks of 375), each pair diagonalised by the block Jacobi, then the
    # FP64 refinement; checked against LAPACK (eigvalsh) and by the residual and orthogonality
    g = gen.rng(7000 + q)
    B = g.standard_normal((q, q))
    H = (B + B.T) / 2
    H[0, 0] += 3.0
    w, Q = lib().sym_eig(T(H), refine)
    w, Q = N(w), N(Q)
    nh = np.linalg.norm(H, 2)
    wref = np.linalg.eigvalsh(H)
    if refine:
        tol = 1e-13 * max(1.0, (q / 1024) ** 0.5)
        assert np.max(np.abs(w - wref)) <= tol * nh
        assert np.max(np.abs(Q.T @ Q - np.eye(q))) <= tol
        S = Q.T @ (H @ Q)
        assert np.linalg.norm(S - np.diag(np.diag(S))) <= tol * nh * q ** 0.5
    else:
        assert np.max(np.abs(w - wref)) <= 2e-5 * nh * q ** 0.5
        assert np.max(np.abs(Q.T @ Q - np.eye(q))) <= 1e-4
        assert np.linalg.norm(H @ Q - Q * w) <= 2e-5 * nh * q
    assert np.all(np.diff(w) >= 0.0)


def test_sym_eig_super_block_low_rank_graded():
    # q = 2048 with eigenvalues 1 .. 1e-16 and a 600-fold zero eigenvalue (the spectrum shape
    # of the projected-update cores of nearly full-rank solutions): FP64-accurate pairs
    q = 2048
    g = gen.rng(7100)
    Qm, _ = np.linalg.qr(g.standard_normal((q, q)))
    lam = np.concatenate([10.0 ** (-16.0 * np.arange(q - 600) / (q - 600)), np.zeros(600)])
    H = (Qm * lam) @ Qm.T
    H = (H + H.T) / 2
    w, Q = lib().sym_eig(T(H), True)
    w, Q = N(w), N(Q)
    nh = np.linalg.norm(H, 2)
    assert np.max(np.abs(w - np.linalg.eigvalsh(H))) <= 2e-13 * nh
    assert np.max(np.abs(Q.T @ Q - np.eye(q))) <= 2e-13
    S = Q.T @ H @ Q
    assert np.linalg.norm(S - np.diag(np.diag(S)), 2) <= 2e-13 * nh


# ------------------------------------------------ FP64 products on the tensor cores

@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 7, 3), (128, 64, 64), (300, 200, 1100), (1000, 421, 1024),
                                   (130, 129, 2050), (64, 40, 20000)])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_dgemm_tensor_emulation_fp64_accuracy(m, n, k, ta, tb):
    # lyap_dgemm method 2 (FP16 digit slices on tcgen05, FP64 sums) against the exact product's
    # FP64 error bound: |C - AB|_ij <= 4 k u max_l|a_il| max_l|b_lj| + 64 u (|A||B|)_ij
    g = gen.rng(3000 + m + 7 * n + 13 * k)
    A = g.standard_normal((k, m) if ta == "T" else (m, k))
    B = g.standard_normal((n, k) if tb == "T" else (k, n))
    A *= 2.0 ** g.integers(-20, 20, size=(A.shape[0], 1))  # graded rows
    C0 = g.standard_normal((m, n))
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    for alpha, beta in ((1.0, 0.0), (-0.5, 2.0)):
        C = lib().dgemm(T(A), T(B), ta, tb, alpha=alpha, beta=beta, C=T(C0), method="tensor")
        ref = alpha * (opA @ opB) + beta * C0
        u = 2.0 ** -53
        bound = (4 * k * u * np.abs(alpha) * np.max(np.abs(opA), axis=1)[:, None] * np.max(np.abs(opB), axis=0)[None, :]
                 + 64 * u * (np.abs(alpha) * np.abs(opA) @ np.abs(opB) + np.abs(beta * C0)))
        err = np.abs(N(C) - ref)
        assert np.all(err <= bound), (float(np.max(err / bound)))


def test_dgemm_tensor_matches_simt_and_exact_integers():
    # integer matrices whose products are exact in FP64: every method returns them exactly
    g = gen.rng(3100)
    A = g.integers(-1000, 1000, size=(257, 333)).astype(np.float64)
    B = g.integers(-1000, 1000, size=(333, 190)).astype(np.float64)
    ref = A @ B
    for method in ("tensor", "simt", "auto"):
        C = N(lib().dgemm(T(A), T(B), method=method))
        assert np.array_equal(C, ref), method


def test_dgemm_tensor_split_k_exact_and_deterministic():
    # few output tiles and a long K: the product is split over K and the partial products summed
    # in a fixed order; integer data keeps every partial sum exact, and repeated calls agree bitwise
    g = gen.rng(3200)
    for (m, n, k) in ((100, 30, 5000), (260, 33, 3000), (40, 300, 2300)):
        A = g.integers(-1000, 1000, size=(m, k)).astype(np.float64)
        B = g.integers(-1000, 1000, size=(k, n)).astype(np.float64)
        ref = A @ B
        C1 = N(lib().dgemm(T(A), T(B), method="tensor"))
        assert np.array_equal(C1, ref), (m, n, k)
        Ar, Br = g.standard_normal((m, k)), g.standard_normal((k, n))
        R1 = N(lib().dgemm(T(Ar), T(Br), method="tensor"))
        R2 = N(lib().dgemm(T(Ar), T(Br), method="tensor"))
        assert np.array_equal(R1, R2)


def test_dgemm_zero_and_empty():
    A = np.zeros((64, 40))
    B = np.ones((40, 30))
    C = N(lib().dgemm(T(A), T(B), method="tensor"))
    assert np.all(C == 0.0)
    C0 = np.full((64, 30), 3.0)
    C = N(lib().dgemm(T(np.zeros((64, 0))), T(np.zeros((0, 30))), beta=1.0, C=T(C0), method="tensor"))
    assert np.array_equal(C, C0)


# ------------------------------------------------ condition of the sign function

@pytest.mark.parametrize("n,indef", [(6, False), (12, True)])
def test_kappa_sign_matches_oracle(n, indef):
    # lyap_kappa_sign (derivative of the Newton iteration on B, power method on L^* L)
    # against the oracle's exact kappa_sign(B) (Kronecker matrix of the Frechet derivative)
    d = gen.normal_blocks(n=n, p=1, m=2, indefinite=indef, seed=gen.SEED_BASE + 60 + n)
    A, L = d["A"], d["L"]
    S = d["S"] if indef else None
    W = L @ (S if indef else np.eye(2)) @ L.T
    ref = O.kappa_sign_fro(O.sign_block(A, W))
    out = lib().kappa_sign(T(A), T(L), S=T(S) if indef else None, power_steps=20)
    assert 0.95 * ref <= out["kappa"] <= ref * (1 + 1e-6), (out, ref)
    assert out["newton_steps"] >= 3


def test_kappa_sign_scaling_and_similarity_invariance():
    # kappa_sign(B) is invariant under A -> 4 A, L -> 2 L (B -> 4 B: exact in binary, and the
    # Frobenius scaling of the Newton iteration absorbs it) and under an orthogonal change of
    # basis (A -> Q^T A Q, L -> Q^T L); n = 100 convection-diffusion
    d = gen.convdiff_shifted(grid=10, m=2)
    A, L = d["A"], d["L"]
    k0 = lib().kappa_sign(T(A), T(L), power_steps=20)
    k1 = lib().kappa_sign(T(4.0 * A), T(2.0 * L), power_steps=20)
    assert abs(k1["kappa"] - k0["kappa"]) <= 1e-8 * k0["kappa"]
    assert k1["newton_steps"] == k0["newton_steps"]
    Q, _ = np.linalg.qr(gen.rng(61).standard_normal(A.shape))
    k2 = lib().kappa_sign(T(Q.T @ A @ Q), T(Q.T @ L), power_steps=20)
    assert abs(k2["kappa"] - k0["kappa"]) <= 0.02 * k0["kappa"], (k0, k2)
