"""Seeded synthetic inputs for the least-squares workloads.

This module only draws inputs.  It holds none of the solver's arithmetic and
imports neither the CUDA binding nor the oracle, so both sides of every
parity check can take their inputs from here.

Matrices are returned column-major (numpy: Fortran order; torch: an (m, n)
view with stride (1, m)), the layout the C ABI expects.

Workloads (shapes of the paper's rank-deficient test problems, Sec. 4):

* ``lowrank_xy``     -- A = X Y with X (m x r), Y (r x n) i.i.d. N(0,1), exact
                        rank r, plus optional i.i.d. noise.
* ``spectrum_matrix``-- A = Q1 diag(sigma) Q2^T with Haar-random orthogonal
                        factors (QR of a Gaussian matrix with the signs of
                        diag(R) made positive, Mezzadri 2007).
* ``step_spectrum`` / ``geometric_spectrum`` -- the two singular value
                        profiles used with ``spectrum_matrix``.
* ``rhs_consistent`` -- b = A x0 + noise.
* ``replicated_rows``-- the paper's own performance generator (Sec. 4.2): a
                        random diagonally dominant r x n row block replicated
                        with random scale factors to m rows.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Problem:
    """One least-squares problem: A (m x n), B (m x nrhs), tolerance and the
    exact spectral facts known from the construction."""

    A: np.ndarray
    B: np.ndarray
    tol: float
    norm2: float
    rank: int
    nb: int
    q: int
    factors: dict | None = None


def lowrank_xy(m: int, n: int, r: int, seed: int, noise: float = 0.0):
    """A = X Y + noise * N(0,1), X (m x r) and Y (r x n) i.i.d. N(0,1).

    Returns (A, X, Y) with A in Fortran order.
    """
    g = _rng(seed)
    X = g.standard_normal((m, r))
    Y = g.standard_normal((r, n))
    A = np.asfortranarray(X @ Y)
    if noise:
        A += noise * g.standard_normal((m, n))
    return A, X, Y


def norm2_of_product(X: np.ndarray, Y: np.ndarray) -> float:
    """||X Y||_2 from the small triangular factors of X and Y^T."""
    if X.shape[1] == 0:
        return 0.0
    Rx = np.linalg.qr(X, mode="r")
    Ry = np.linalg.qr(Y.T, mode="r")
    return float(np.linalg.svd(Rx @ Ry.T, compute_uv=False)[0])


def haar_orthogonal(m: int, n: int, g: np.random.Generator) -> np.ndarray:
    """First n columns of a Haar-random m x m orthogonal matrix (m >= n)."""
    Q, R = np.linalg.qr(g.standard_normal((m, n)))
    return Q * np.sign(np.diagonal(R))


def step_spectrum(n: int, r: int, top_exp: float, tail: float) -> np.ndarray:
    """sigma_i = 10^(-top_exp * i / r) for i < r, ``tail`` otherwise."""
    s = np.full(n, tail)
    s[:r] = 10.0 ** (-top_exp * np.arange(r) / r)
    return s


def geometric_spectrum(n: int, r: int, low: float, tail: float) -> np.ndarray:
    """sigma decays geometrically from 1 to ``low`` over i < r, then ``tail``."""
    s = np.full(n, tail)
    if r == 1:
        s[0] = 1.0
    elif r > 1:
        s[:r] = low ** (np.arange(r) / (r - 1))
    return s


def spectrum_matrix(m: int, n: int, sigma: np.ndarray, seed: int):
    """A = Q1 diag(sigma) Q2^T (numpy, for sizes a CPU handles quickly).

    Returns (A, Q1, Q2) with Q1 m x n, Q2 n x n.
    """
    g = _rng(seed)
    Q1 = haar_orthogonal(m, n, g)
    Q2 = haar_orthogonal(n, n, g)
    A = np.asfortranarray((Q1 * sigma) @ Q2.T)
    return A, Q1, Q2


def spectrum_matrix_torch(m: int, n: int, sigma, seed: int, device="cuda"):
    """The same construction drawn with torch on ``device`` (large sizes).

    Returns (A, Q1, Q2) as column-major (m, n) torch views in float64.
    """
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    sig = torch.as_tensor(np.asarray(sigma), dtype=torch.float64, device=device)

    def haar(rows, cols):
        G = torch.randn(rows, cols, generator=gen, dtype=torch.float64, device=device)
        Q, R = torch.linalg.qr(G, mode="reduced")
        del G
        Q *= torch.sign(torch.diagonal(R))
        del R
        return Q

    Q1 = haar(m, n)
    Q2 = haar(n, n)
    # column-major A (m x n) is the row-major (n x m) tensor A^T = Q2 diag(s) Q1^T
    At = (Q2 * sig) @ Q1.T
    return At.t(), Q1, Q2


def rhs_consistent(A: np.ndarray, nrhs: int, noise: float, seed: int):
    """B = A X0 + noise * N(0,1), X0 (n x nrhs) i.i.d. N(0,1)."""
    g = _rng(seed)
    m, n = A.shape
    X0 = g.standard_normal((n, nrhs))
    B = np.asfortranarray(A @ X0 + noise * g.standard_normal((m, nrhs)))
    return B, X0


def rhs_gaussian(m: int, nrhs: int, seed: int) -> np.ndarray:
    return np.asfortranarray(_rng(seed).standard_normal((m, nrhs)))


def replicated_rows(m: int, n: int, r: int, seed: int) -> np.ndarray:
    """Sec. 4.2 generator: an r x n random block made diagonally dominant,
    copied with random scale factors until m rows are filled."""
    g = _rng(seed)
    blk = g.uniform(-1.0, 1.0, (r, n))
    d = np.arange(min(r, n))
    blk[d, d] = np.sign(blk[d, d] + 0.5) * (np.abs(blk).sum(axis=1)[: d.size] + 1.0)
    A = np.empty((m, n), order="F")
    for start in range(0, m, r):
        stop = min(m, start + r)
        A[start:stop] = g.uniform(0.5, 2.0) * blk[: stop - start]
    return A


# ---------------------------------------------------------------------------
# Named workloads.  Seeds: inputs 1000 + config, sketch 2000 + config.
# ---------------------------------------------------------------------------
def c1_problem() -> Problem:
    """2000 x 1000, exact rank 400 (X Y) + 1e-14 noise, b ~ N(0,1),
    tol = 1e-10 ||A||_2, nb = 64, q = 1."""
    A, X, Y = lowrank_xy(2000, 1000, 400, seed=1001, noise=1e-14)
    nrm = norm2_of_product(X, Y)
    B = rhs_gaussian(2000, 1, seed=1101)
    return Problem(A, B, 1e-10 * nrm, nrm, 400, 64, 1)


def c2_like(n: int, nrhs: int = 16, nb: int = 128, q: int = 2, seed: int = 1002) -> Problem:
    """Square n x n, rank n/2, sigma_i = 10^(-6 i / (n/2)) then 1e-15;
    b = A x0 + 1e-8 N(0,1); tol = 1e-10 (||A||_2 = 1).  n = 16384 is the
    full-size workload (drawn with ``spectrum_matrix_torch`` there)."""
    r = n // 2
    sigma = step_spectrum(n, r, 6.0, 1e-15)
    A, Q1, Q2 = spectrum_matrix(n, n, sigma, seed)
    B, X0 = rhs_consistent(A, nrhs, 1e-8, seed + 100)
    return Problem(A, B, 1e-10, 1.0, r, nb, q, dict(Q1=Q1, Q2=Q2, sigma=sigma, X0=X0))


def c3_like(m: int, n: int, r: int, nrhs: int = 1, nb: int = 128, q: int = 1,
            seed: int = 1003) -> Problem:
    """m x n, rank r, sigma geometric 1 -> 1e-4 then 1e-14;
    b = A x0 + 1e-8 N(0,1); tol = 1e-6 ||A||_2."""
    sigma = geometric_spectrum(n, r, 1e-4, 1e-14)
    A, Q1, Q2 = spectrum_matrix(m, n, sigma, seed)
    B, X0 = rhs_consistent(A, nrhs, 1e-8, seed + 100)
    return Problem(A, B, 1e-6, 1.0, r, nb, q, dict(Q1=Q1, Q2=Q2, sigma=sigma, X0=X0))


def batched_problems(count: int, seed: int = 1004, m_range=(256, 2048),
                     nrhs_choices=(1, 8, 32)):
    """Independent X Y problems: m ~ U[m_range], n ~ U[128, m],
    r ~ U[ceil(n/4), n], nrhs from ``nrhs_choices``, b ~ N(0,1),
    tol = 1e-10 ||A||_2."""
    g = _rng(seed)
    out = []
    for j in range(count):
        m = int(g.integers(m_range[0], m_range[1] + 1))
        n = int(g.integers(min(128, m), m + 1))
        r = int(g.integers(math.ceil(n / 4), n + 1))
        nrhs = int(g.choice(nrhs_choices))
        A, X, Y = lowrank_xy(m, n, r, seed=seed * (1 << 32) + j)
        nrm = norm2_of_product(X, Y)
        B = rhs_gaussian(m, nrhs, seed=seed * (1 << 32) + j + (1 << 31))
        out.append(Problem(A, B, 1e-10 * nrm, nrm, r, 64, 1))
    return out
