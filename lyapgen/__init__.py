"""Seeded synthetic inputs for low-rank Lyapunov equations  A X + X A^T + W = 0.

This module is shared by the CPU oracle tests, the CUDA-path tests and the
benchmark.  It builds coefficient matrices and right-hand-side factors only:
it contains none of the solver's arithmetic (no sign iteration, no residual
factorisation, no refinement).  Every generator takes an explicit seed and
draws from ``numpy.random.default_rng(seed)``.

Workload families:

* ``laplacian_2d``/``convdiff_2d`` -- 5-point finite-difference operators on an
  N x N grid with Dirichlet boundary (the shape of the paper's SLICOT-style
  PDE examples, Sec. 4.3, which are not shipped here).
* ``normal_blocks`` -- A = Q T Q^T with Haar Q and 2x2 blocks
  [[-a, b], [-b, -a]], whose Schur form is known by construction.
* ``paper_synthetic`` -- the generator of Sec. 4.2: A = -V diag(logspace(0,q,n)) V^T
  with V the symmetric orthogonal sine matrix.
* ``random_stable`` -- A = -(G G^T/n + 0.1 I) + 0.5 (H - H^T)/sqrt(n).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2510021260


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def sine_basis(n: int) -> np.ndarray:
    """Symmetric orthogonal V_ij = sqrt(2/(n+1)) sin(i j pi/(n+1)), i, j = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return math.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, i) * math.pi / (n + 1))


def tridiag(n: int, sub: float, diag: float, sup: float) -> np.ndarray:
    T = np.zeros((n, n))
    idx = np.arange(n)
    T[idx, idx] = diag
    T[idx[1:], idx[:-1]] = sub
    T[idx[:-1], idx[1:]] = sup
    return T


def laplacian_2d(N: int) -> np.ndarray:
    """A = -(1/h^2) * (5-point Laplacian) on an N x N interior grid, h = 1/(N+1).

    Diagonal -4/h^2, neighbours +1/h^2; symmetric and stable.
    """
    h = 1.0 / (N + 1)
    K1 = tridiag(N, -1.0, 2.0, -1.0) / h**2
    I = np.eye(N)
    return -(np.kron(I, K1) + np.kron(K1, I))


def convdiff_1d_coeffs(N: int, v: float):
    """(sub, diag, sup) of the 1-D operator  -u'' + v u'  with first-order upwind."""
    h = 1.0 / (N + 1)
    return (-1.0 / h**2 - v / h, 2.0 / h**2 + v / h, -1.0 / h**2)


def convdiff_2d(N: int, vx: float, vy: float) -> np.ndarray:
    """K = 5-point diffusion + first-order upwind convection (velocity (vx, vy)), N x N grid."""
    Kx = tridiag(N, *convdiff_1d_coeffs(N, vx))
    Ky = tridiag(N, *convdiff_1d_coeffs(N, vy))
    I = np.eye(N)
    return np.kron(I, Kx) + np.kron(Ky, I)


def convdiff_1d_eigs(N: int, v: float) -> np.ndarray:
    """Eigenvalues of the tridiagonal Toeplitz 1-D upwind operator (closed form)."""
    a, b, c = convdiff_1d_coeffs(N, v)
    k = np.arange(1, N + 1)
    return b - 2.0 * math.sqrt(a * c) * np.cos(k * math.pi / (N + 1))


def fp64_laplacian(grid: int = 8, m: int = 2, seed: int = SEED_BASE + 1):
    """n = grid^2 symmetric stable A (scaled 5-point Laplacian), L n x m N(0,1)."""
    A = laplacian_2d(grid)
    n = A.shape[0]
    L = rng(seed).standard_normal((n, m))
    return {"A": A, "L": L, "name": f"laplacian{grid}x{grid}_m{m}"}


def convdiff_shifted(grid: int = 32, m: int = 4, vel: float = 10.0, kappa: float = 1e3,
                     seed: int = SEED_BASE + 2):
    """A = -K + sigma I on a grid x grid upwind convection-diffusion operator.

    sigma is fixed in closed form so that the eigenvalue ratio of the Lyapunov
    operator, max|l_i + l_j| / min|l_i + l_j| over eigenvalues l of A, equals
    ``kappa`` (the spectrum of K is the Kronecker sum of two tridiagonal Toeplitz
    spectra, so it is known exactly).
    """
    K = convdiff_2d(grid, vel, vel)
    ex = convdiff_1d_eigs(grid, vel)
    lmin = 2.0 * ex.min()
    lmax = 2.0 * ex.max()
    # ratio (lmax - s) / (lmin - s) = kappa
    sigma = (kappa * lmin - lmax) / (kappa - 1.0)
    n = K.shape[0]
    A = -K + sigma * np.eye(n)
    L = rng(seed).standard_normal((n, m))
    return {"A": A, "L": L, "sigma": sigma, "eig_min": -(lmax - sigma), "eig_max": -(lmin - sigma),
            "name": f"convdiff{grid}x{grid}_m{m}_k{kappa:g}"}


def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    G = g.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def normal_blocks(n: int = 4096, p: int = 2, m: int = 8, indefinite: bool = True,
                  seed: int = SEED_BASE + 3, beta_max: float = 5.0):
    """A = Q T Q^T, T = blkdiag([[-a_i, b_i], [-b_i, -a_i]]), a_i log-uniform in [10^-p, 1].

    W = L S L^T with S = diag(+-1) (random signs) when ``indefinite``, else S = I.
    """
    assert n % 2 == 0
    g = rng(seed)
    nb = n // 2
    alpha = 10.0 ** g.uniform(-p, 0.0, nb)
    beta = g.uniform(0.0, beta_max, nb)
    Q = haar_orthogonal(n, g)
    # (Q T) column pairs: [q0, q1] @ [[-a, b], [-b, -a]] = [-a q0 - b q1, b q0 - a q1]
    q0, q1 = Q[:, 0::2], Q[:, 1::2]
    QT = np.empty_like(Q)
    QT[:, 0::2] = -alpha[None, :] * q0 - beta[None, :] * q1
    QT[:, 1::2] = beta[None, :] * q0 - alpha[None, :] * q1
    A = QT @ Q.T
    L = g.standard_normal((n, m))
    if indefinite:
        s = np.where(g.uniform(size=m) < 0.5, -1.0, 1.0)
        if np.all(s > 0):
            s[-1] = -1.0
        if np.all(s < 0):
            s[0] = 1.0
    else:
        s = np.ones(m)
    return {"A": A, "L": L, "S": np.diag(s), "Q": Q, "alpha": alpha, "beta": beta,
            "name": f"normal{n}_p{p}_m{m}"}


def paper_synthetic(n: int, q: float, m: int = 3, seed: int = SEED_BASE + 6):
    """Sec. 4.2 generator: A = -V diag(logspace(0, q, n)) V^T, L n x m N(0,1)."""
    V = sine_basis(n)
    d = np.logspace(0.0, q, n)
    A = -(V * d[None, :]) @ V.T
    L = rng(seed).standard_normal((n, m))
    return {"A": A, "L": L, "V": V, "d": d, "name": f"synthetic{n}_q{q:g}"}


def random_stable(n: int, r: int, g: np.random.Generator):
    G = g.standard_normal((n, n))
    H = g.standard_normal((n, n))
    A = -(G @ G.T / n + 0.1 * np.eye(n)) + 0.5 * (H - H.T) / math.sqrt(n)
    L = g.standard_normal((n, r))
    return {"A": A, "L": L}


def batch_uneven(count: int = 256, nmin: int = 64, nmax: int = 1024, rmax: int = 8,
                 seed: int = SEED_BASE + 5):
    """``count`` independent equations, n log-uniform in [nmin, nmax], r uniform in 1..rmax."""
    g = rng(seed)
    ns = np.rint(np.exp(g.uniform(math.log(nmin), math.log(nmax), count))).astype(int)
    rs = g.integers(1, rmax + 1, count)
    out = []
    for n, r in zip(ns, rs):
        out.append(random_stable(int(n), int(r), g))
    return out


def loss_weights(q: int, n: int, seed: int = SEED_BASE + 4) -> np.ndarray:
    """C (q x n) N(0,1) for the loss trace(C X C^T)."""
    return rng(seed).standard_normal((q, n))
