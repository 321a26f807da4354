"""FP64 CPU oracle for the randUTV minimum-norm least-squares solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: it is used by ``tests/``, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  It shares no
code with the CUDA library (``paper_2408_05238_b300/csrc``) and imports
nothing from the package.

What it computes (Chillaron, Quintana-Orti, Vidal, Martinsson,
arXiv 2408.05238, Sec. 3):

* ``randutv``      -- Fig. 2 (randUTV): per block of ``nb`` columns a Gaussian
                      sketch G, the sample Y = (A^T A)^q A^T G, an unpivoted
                      Householder QR of Y giving (W_V, T_V), the right update
                      with I - W_V T_V W_V^T, a Householder QR of the block
                      column giving (W_U, T_U), the left update, and the SVD
                      of the small diagonal block.
* ``compute_rank`` -- Compute_rank of Fig. 4 (count of diagonal entries of T
                      above the threshold; the leading-run reading below).
* ``nullify``      -- Fig. 3 (Nullify_top_right_part_of_T): row blocks of
                      [C D] from the bottom up, one RZ reflector per row.
* ``solve``        -- Fig. 4 (Solve_linear_system): x = V (T_tl^{-1} (U^T b)),
                      with the fast option of the Remark after Fig. 4 (skip
                      Nullify, Eq. (7) x_simple).
* ``refine``       -- iterative refinement of a solution with the solve
                      operator P = V_1 T_11^{-1} U_1^T of Fig. 4:
                      x <- x + P (b - A x), the residual in FP64.
* ``refine_min_norm`` -- two-stage refinement (least squares with the right
                      preconditioner V_1 T_11^{-1}, then the projection onto
                      range(A^T)) whose fixed point is the minimum-norm
                      least-squares solution even when the factors are only
                      approximate.
* ``pinv_solve``   -- Sec. 2.2 truncated-SVD least squares, used as the
                      brute-force pin on small inputs.

Readings of the paper taken here where it is silent or garbled:

* The right update of Fig. 2 is applied to *all* m rows of the trailing
  columns (Fig. 2 prints only the A_BR block; without the rows above,
  A V = U T fails).
* The left update applies (I - W_U T_U W_U^T)^T, i.e. Q^T, to [A12; A22]
  (Fig. 2 prints W_U^* T_U^* W_U).
* The loop runs while k < min(m, n) with block b_i = min(nb, m-k, n-k); the
  sketch for step i has m-k rows and b_i columns.
* Householder vectors follow the LAPACK xLARFG convention:
  beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta, v(0) = 1; a vector
  whose tail is exactly zero gives tau = 0 (identity).  No rescaling of
  tiny norms is done.
* The diagonal-block SVD returns singular values in descending order; the
  signs of the singular vectors are those of LAPACK (numpy.linalg.svd) and
  are free -- x does not depend on them.
* Compute_rank: entry j is nonzero iff |T_jj| > tol (tol absolute); the rank
  r is the length of the leading run of nonzero entries; the count of all
  nonzero entries is returned beside it.
* Nullify processes row blocks of C = T(0:r, 0:r) from the bottom with block
  size nb (the top block holds the remainder); inside a block the rows go
  from the bottom up, one reflector per row acting on column i and columns
  r..n-1 (the xLATRZ order).
* The Gaussian sketch is drawn with Philox4x64-10 (Salmon, Moraes, Dror,
  Shaw, SC'11) keyed by (seed, 0), counter (row/4, column, step, 0), and the
  Box-Muller transform; see ``sketch_matrix``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "philox4x64_10",
    "sketch_matrix",
    "householder",
    "householder_qr",
    "wy_factor",
    "randutv",
    "compute_rank",
    "nullify",
    "solve",
    "refine",
    "refine_min_norm",
    "pinv_solve",
    "pinv_solve_from_factors",
    "normal_equation_residual",
]

# ---------------------------------------------------------------------------
# Philox4x64-10 counter-based generator (Salmon et al., SC'11, Sec. 4.2).
# Round: two 64x64->128-bit products of counter words 0 and 2 with the
# multipliers, outputs permuted and xor-ed with the key; the key is bumped
# by the Weyl constants between rounds.
# ---------------------------------------------------------------------------
_PHILOX_M0 = 0xD2E7470EE14C6C93
_PHILOX_M1 = 0xCA5A826395121157
_PHILOX_W0 = 0x9E3779B97F4A7C15
_PHILOX_W1 = 0xBB67AE8584CAA73B
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a: int, b: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Full 128-bit product of the constant ``a`` and each uint64 of ``b``."""
    a_lo = np.uint64(a & 0xFFFFFFFF)
    a_hi = np.uint64(a >> 32)
    b_lo = b & _LO32
    b_hi = b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _LO32) + (hl & _LO32)
    lo = (ll & _LO32) | ((mid & _LO32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(counter, key):
    """Philox4x64 with 10 rounds.

    ``counter``: sequence of 4 uint64 arrays (broadcastable), ``key``: pair of
    Python ints.  Returns 4 uint64 arrays.
    """
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64).copy() for c in counter)
        c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
        k0 = key[0] & 0xFFFFFFFFFFFFFFFF
        k1 = key[1] & 0xFFFFFFFFFFFFFFFF
        for rnd in range(10):
            if rnd > 0:
                k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFFFFFFFFFF
                k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFFFFFFFFFF
            hi0, lo0 = _mulhilo64(_PHILOX_M0, c0)
            hi1, lo1 = _mulhilo64(_PHILOX_M1, c2)
            c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                              hi0 ^ c3 ^ np.uint64(k1), lo0)
        return c0, c1, c2, c3


def sketch_matrix(seed: int, step: int, rows: int, cols: int) -> np.ndarray:
    """The Gaussian sketch G of Fig. 2 (generate_iid_stdnorm_matrix).

    G is ``rows x cols`` with i.i.d. N(0,1) entries.  Entry (p, j) comes from
    the Philox4x64-10 block with counter (p // 4, j, step, 0) and key
    (seed, 0): its four 64-bit words w0..w3 give two Box-Muller pairs,
    u = ((w >> 11) + 1) 2^-53 in (0, 1] for the radius and
    t = (w >> 11) 2^-53 in [0, 1) for the angle:
        G(4g+0, j) = sqrt(-2 ln u0) cos(2 pi t1)
        G(4g+1, j) = sqrt(-2 ln u0) sin(2 pi t1)
        G(4g+2, j) = sqrt(-2 ln u2) cos(2 pi t3)
        G(4g+3, j) = sqrt(-2 ln u2) sin(2 pi t3)
    """
    if rows <= 0 or cols <= 0:
        return np.zeros((max(rows, 0), max(cols, 0)))
    ngroups = (rows + 3) // 4
    g_idx, j_idx = np.meshgrid(np.arange(ngroups, dtype=np.uint64),
                               np.arange(cols, dtype=np.uint64), indexing="ij")
    w0, w1, w2, w3 = philox4x64_10(
        (g_idx, j_idx, np.uint64(step), np.uint64(0)), (seed, 0))
    s11 = np.uint64(11)
    scale = 2.0 ** -53
    u0 = ((w0 >> s11).astype(np.float64) + 1.0) * scale
    t1 = (w1 >> s11).astype(np.float64) * scale
    u2 = ((w2 >> s11).astype(np.float64) + 1.0) * scale
    t3 = (w3 >> s11).astype(np.float64) * scale
    r0 = np.sqrt(-2.0 * np.log(u0))
    r2 = np.sqrt(-2.0 * np.log(u2))
    two_pi = 2.0 * math.pi
    z = np.stack([r0 * np.cos(two_pi * t1), r0 * np.sin(two_pi * t1),
                  r2 * np.cos(two_pi * t3), r2 * np.sin(two_pi * t3)], axis=1)
    # z has shape (ngroups, 4, cols): row 4g + e of column j is z[g, e, j]
    return z.reshape(4 * ngroups, cols)[:rows].copy()


# ---------------------------------------------------------------------------
# Householder reflectors and unpivoted QR (Golub & Van Loan, Sec. 5.1-5.2),
# compact WY representation (Schreiber & Van Loan 1989).
# ---------------------------------------------------------------------------
def householder(x: np.ndarray):
    """Reflector H = I - tau v v^T with H x = beta e_1 and v(0) = 1.

    LAPACK xLARFG convention: beta = -sign(alpha) ||x||,
    tau = (beta - alpha) / beta; if x(1:) == 0 then tau = 0 and beta = alpha.
    """
    x = np.asarray(x, dtype=np.float64)
    alpha = float(x[0])
    sigma = float(np.linalg.norm(x[1:])) if x.size > 1 else 0.0
    v = np.zeros_like(x)
    v[0] = 1.0
    if sigma == 0.0:
        return v, 0.0, alpha
    beta = -math.copysign(math.hypot(alpha, sigma), alpha)
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return v, tau, beta


def householder_qr(Y: np.ndarray):
    """Unpivoted Householder QR of Y (rows x cols), one column at a time.

    Returns (R, W, tau): R is min(rows, cols) x cols upper trapezoidal,
    W is rows x min(rows, cols) unit lower trapezoidal (the Householder
    vectors, the third output of unpivoted_QR in Fig. 2) and
    Q = H_0 H_1 ... H_{k-1}, H_j = I - tau_j W(:, j) W(:, j)^T, with Y = Q R.
    """
    Y = np.array(Y, dtype=np.float64, copy=True)
    rows, cols = Y.shape
    k = min(rows, cols)
    W = np.zeros((rows, k))
    tau = np.zeros(k)
    for j in range(k):
        v, t, beta = householder(Y[j:, j])
        if j + 1 < cols:
            Y[j:, j + 1:] -= t * np.outer(v, v @ Y[j:, j + 1:])
        Y[j, j] = beta
        Y[j + 1:, j] = 0.0
        W[j:, j] = v
        tau[j] = t
    return np.triu(Y[:k, :]), W, tau


def wy_factor(W: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Upper triangular T with H_0 H_1 ... H_{k-1} = I - W T W^T.

    Forward recurrence: T(j, j) = tau_j and
    T(0:j, j) = -tau_j T(0:j, 0:j) W(:, 0:j)^T W(:, j).
    """
    k = tau.shape[0]
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = tau[j]
        if j > 0:
            T[:j, j] = -tau[j] * (T[:j, :j] @ (W[:, :j].T @ W[:, j]))
    return T


# ---------------------------------------------------------------------------
# randUTV (Fig. 2)
# ---------------------------------------------------------------------------
@dataclass
class UTV:
    """Result of ``randutv``: A V = U T with U, V orthogonal, T upper
    trapezoidal.  ``steps`` records, per step, (k, b, Y, W_V, T_V, W_U, T_U,
    sigma) for step-level checks."""

    U: np.ndarray
    T: np.ndarray
    V: np.ndarray
    steps: list = field(default_factory=list)


def randutv(A: np.ndarray, q: int, nb: int, seed: int, max_steps: int | None = None,
            keep_steps: bool = False) -> UTV:
    """randUTV of Fig. 2 with explicit U and V (they start as identities).

    ``max_steps`` stops after that many steps (used to time a bounded
    sample of a large problem); the result is then only partly triangular.
    """
    T = np.array(A, dtype=np.float64, copy=True)
    m, n = T.shape
    U = np.eye(m)
    V = np.eye(n)
    out = UTV(U, T, V)
    k = 0
    i = 0
    while k < min(m, n):
        if max_steps is not None and i >= max_steps:
            break
        b = min(nb, m - k, n - k)
        # --- Apply transformations from the right.
        G = sketch_matrix(seed, i, m - k, b)
        A_BR = T[k:, k:]
        Y = A_BR.T @ G
        for _ in range(q):
            Y = A_BR.T @ (A_BR @ Y)
        _, W_V, tau_V = householder_qr(Y)
        T_V = wy_factor(W_V, tau_V)
        T[:, k:] -= ((T[:, k:] @ W_V) @ T_V) @ W_V.T      # all m rows
        V[:, k:] -= ((V[:, k:] @ W_V) @ T_V) @ W_V.T
        # --- Apply transformations from the left.
        R11, W_U, tau_U = householder_qr(T[k:, k:k + b])
        T_U = wy_factor(W_U, tau_U)
        T[k:, k:k + b] = 0.0
        T[k:k + b, k:k + b] = R11
        if k + b < n:
            T[k:, k + b:] -= W_U @ (T_U.T @ (W_U.T @ T[k:, k + b:]))
        U[:, k:] -= ((U[:, k:] @ W_U) @ T_U) @ W_U.T
        # --- Small SVD and update of A, U and V.
        U_svd, sigma, V_svd_t = np.linalg.svd(R11)
        V_svd = V_svd_t.T
        T[k:k + b, k:k + b] = np.diag(sigma)
        T[:k, k:k + b] = T[:k, k:k + b] @ V_svd
        T[k:k + b, k + b:] = U_svd.T @ T[k:k + b, k + b:]
        V[:, k:k + b] = V[:, k:k + b] @ V_svd
        U[:, k:k + b] = U[:, k:k + b] @ U_svd
        if keep_steps:
            out.steps.append(dict(k=k, b=b, G=G, Y=Y, W_V=W_V, T_V=T_V, tau_V=tau_V,
                                  W_U=W_U, T_U=T_U, tau_U=tau_U, R11=R11, sigma=sigma))
        k += b
        i += 1
    return out


def compute_rank(T: np.ndarray, tol: float) -> tuple[int, int]:
    """Compute_rank (Fig. 4): returns (r, count).

    An entry of diag(T) is nonzero iff |T_jj| > tol.  r is the length of the
    leading run of nonzero entries (T_11 = T(0:r, 0:r) must be invertible),
    count is the number of all nonzero entries.
    """
    d = np.abs(np.diagonal(T))
    nz = d > tol
    count = int(np.count_nonzero(nz))
    zeros = np.flatnonzero(~nz)
    r = int(zeros[0]) if zeros.size else int(d.size)
    return r, count


# ---------------------------------------------------------------------------
# Nullify_top_right_part_of_T (Fig. 3)
# ---------------------------------------------------------------------------
def _apply_rz_right(M: np.ndarray, rows: slice, i: int, r: int, v: np.ndarray, tau: float):
    """M(rows, J) <- M(rows, J) (I - tau v v^T) with J = {i} U {r, ..., n-1}."""
    if tau == 0.0:
        return
    block = M[rows]
    if block.shape[0] == 0:
        return
    w = block[:, i] * v[0] + block[:, r:] @ v[1:]
    block[:, i] -= tau * w * v[0]
    block[:, r:] -= tau * np.outer(w, v[1:])


def nullify(T: np.ndarray, V: np.ndarray, r: int, nb: int) -> list:
    """Annihilate T_12 = T(0:r, r:n) in place, updating V (Fig. 3).

    [C D] = T(0:r, :) is processed in row blocks C_11 of nb rows from the
    bottom.  Nullify(C_11, D_1) builds one reflector per row, bottom row
    first, acting on column i and on columns r..n-1 and zeroing D(i, :);
    each is applied at once to the rows above it inside the block.  Update
    then applies the block's reflectors, in the same order, to the rows
    above the block (C_01, D_0) and to the columns (E_1, F) of V.
    Returns the list of (i, v, tau).
    """
    m, n = T.shape
    reflectors = []
    if r <= 0 or r >= n:
        return reflectors
    j1 = r
    while j1 > 0:
        j0 = max(0, j1 - nb)
        block = []
        for i in range(j1 - 1, j0 - 1, -1):
            x = np.concatenate(([T[i, i]], T[i, r:]))
            v, tau, beta = householder(x)
            T[i, i] = beta
            T[i, r:] = 0.0
            _apply_rz_right(T, slice(j0, i), i, r, v, tau)
            block.append((i, v, tau))
        for (i, v, tau) in block:                         # Update(C_01, D_0)
            _apply_rz_right(T, slice(0, j0), i, r, v, tau)
        for (i, v, tau) in block:                         # Update(E_1, F)
            _apply_rz_right(V, slice(0, n), i, r, v, tau)
        reflectors.extend(block)
        j1 = j0
    return reflectors


def _back_substitution(R: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Solve R Y = C for upper triangular R, one row at a time from the bottom."""
    r = R.shape[0]
    Y = np.zeros_like(C)
    for i in range(r - 1, -1, -1):
        Y[i] = (C[i] - R[i, i + 1:] @ Y[i + 1:]) / R[i, i]
    return Y


@dataclass
class Solution:
    x: np.ndarray
    rank: int
    rank_count: int
    diag: np.ndarray
    utv: UTV | None = None


def solve(A: np.ndarray, B: np.ndarray, q: int, nb: int, tol: float, seed: int,
          do_nullify: bool = True, keep: bool = False) -> Solution:
    """Solve_linear_system (Fig. 4).

    [U, T, V] = randUTV(A, q, nb); r = Compute_rank(T);
    [T, V] = Nullify_top_right_part_of_T(T, V, r) unless ``do_nullify`` is
    False (the fast option); x = V (T_tl^{-1} (U^T b)) with T_tl = T(0:r, 0:r)
    and the r-vector padded with n - r zeros.
    """
    A = np.asarray(A, dtype=np.float64)
    B2 = np.asarray(B, dtype=np.float64)
    vec = B2.ndim == 1
    if vec:
        B2 = B2[:, None]
    m, n = A.shape
    utv = randutv(A, q, nb, seed)
    diag = np.abs(np.diagonal(utv.T)).copy()
    r, count = compute_rank(utv.T, tol)
    if do_nullify:
        nullify(utv.T, utv.V, r, nb)
    X = np.zeros((n, B2.shape[1]))
    if r > 0:
        c = (utv.U.T @ B2)[:r]
        y = _back_substitution(utv.T[:r, :r], c)
        X = utv.V[:, :r] @ y
    if vec:
        X = X[:, 0]
    return Solution(X, r, count, diag, utv if keep else None)


def refine(A: np.ndarray, B: np.ndarray, sol: Solution, x0: np.ndarray | None = None,
           steps: int = 1) -> np.ndarray:
    """``steps`` refinement steps x <- x + P (b - A x) from x0 (default:
    sol.x), with P = V(:, :r) T(:r, :r)^{-1} U(:, :r)^T taken from the
    factors of ``sol`` (``solve(..., keep=True)``; after Nullify when it ran).
    Since U_1^T A V_1 = T_11 (A V = U T with T upper triangular), P A acts
    as the identity on range(V_1): one step removes any error in that
    subspace, and P b is a fixed point."""
    if sol.utv is None:
        raise ValueError("refine needs solve(..., keep=True)")
    A = np.asarray(A, dtype=np.float64)
    Bm = np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1)
    x = np.array(sol.x if x0 is None else x0, dtype=np.float64).reshape(A.shape[1], -1)
    r = sol.rank
    U, T, V = sol.utv.U, sol.utv.T, sol.utv.V
    for _ in range(steps):
        if r == 0:
            break
        res = Bm - A @ x
        y = _back_substitution(T[:r, :r], (U.T @ res)[:r])
        x = x + V[:, :r] @ y
    return x.reshape(np.shape(sol.x if x0 is None else x0))


def _forward_substitution_transposed(R: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Solve R^T Y = C for upper triangular R (R^T lower triangular), one row
    at a time from the top."""
    r = R.shape[0]
    Y = np.zeros_like(C)
    for i in range(r):
        Y[i] = (C[i] - R[:i, i] @ Y[:i]) / R[i, i]
    return Y


MIN_NORM_GAP = 1e-2


def refine_min_norm(A: np.ndarray, B: np.ndarray, sol: Solution, steps: int = 1) -> np.ndarray:
    """Refinement that also restores the minimum-norm property when the
    factors are only approximate (the TF32 update modes), in two stages of
    ``steps`` iterations each, with the residuals and the products with A in
    FP64 and the factors of ``sol`` (``solve(..., keep=True)``):

    1. least squares: with N = V_1 T_11^{-1}, from x = P b (P = N U_1^T),
           x <- x + N N^T A^T (b - A x).
       In z with x = N z this is z <- z + K^T (b - K z) for K = A N, which
       equals U_1 up to the factors' error times the condition number of
       T_11, so it contracts by about that much per step (not by its
       square); its fixed point has V_1^T A^T r = 0, i.e. r orthogonal to
       range(A V_1) = range(A): a least-squares solution x_ls.
    2. minimum norm: with L = A^T U_1 T_11^{-T} (V_1 up to the same error),
       from x = 0,
           x <- x + L L^T (x_ls - x),
       whose fixed point is the orthogonal projection of x_ls onto
       range(L) = range(A^T): the minimum-norm least-squares solution.
    For exact factors of a rank-r matrix one step of each stage gives the
    pseudoinverse solution.

    The fixed points are the truncated solution only when A is of numerical
    rank r (its singular values beyond the rank enter through A).  So, as
    the library does, the diagonal blocks' singular values (``sol.diag``,
    before Nullify) are checked first: when the largest dropped one exceeds
    MIN_NORM_GAP times the smallest kept one there is no gap at the rank, and
    ``sol.x`` is returned unrefined."""
    if sol.utv is None:
        raise ValueError("refine_min_norm needs solve(..., keep=True)")
    A = np.asarray(A, dtype=np.float64)
    Bm = np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1)
    r = sol.rank
    U, T, V = sol.utv.U, sol.utv.T, sol.utv.V
    if r == 0:
        return np.zeros_like(np.asarray(sol.x, dtype=np.float64))
    if r < sol.diag.size and sol.diag[r:].max() > MIN_NORM_GAP * sol.diag[:r].min():
        return np.array(sol.x, dtype=np.float64)
    T11, U1, V1 = T[:r, :r], U[:, :r], V[:, :r]
    x = np.array(sol.x, dtype=np.float64).reshape(A.shape[1], -1)
    for _ in range(steps):           # stage 1: least squares in range(V_1)
        s = V1.T @ (A.T @ (Bm - A @ x))
        x = x + V1 @ _back_substitution(T11, _forward_substitution_transposed(T11, s))
    x_ls = x
    x = np.zeros_like(x_ls)
    for _ in range(steps):           # stage 2: projection onto range(A^T)
        e = _back_substitution(T11, U1.T @ (A @ (x_ls - x)))
        x = x + A.T @ (U1 @ _forward_substitution_transposed(T11, e))
    return x.reshape(np.shape(sol.x))


# ---------------------------------------------------------------------------
# Pins and measures
# ---------------------------------------------------------------------------
def pinv_solve(A: np.ndarray, B: np.ndarray, r: int) -> np.ndarray:
    """Truncated-SVD least squares (Sec. 2.2): x = V_1 Sigma_11^{-1} U_1^T b."""
    U, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    if r == 0:
        return np.zeros((A.shape[1],) + np.shape(B)[1:])
    return Vt[:r].T @ ((U[:, :r].T @ B) / (s[:r] if np.ndim(B) == 1 else s[:r, None]))


def pinv_solve_from_factors(Q1: np.ndarray, sigma: np.ndarray, Q2: np.ndarray, B: np.ndarray,
                            r: int) -> np.ndarray:
    """Truncated-SVD least squares (Sec. 2.2) for A = Q1 diag(sigma) Q2^T with
    orthonormal Q1, Q2 known: x = Q2(:, :r) diag(1/sigma(:r)) Q1(:, :r)^T b."""
    Bm = np.asarray(B, dtype=np.float64).reshape(Q1.shape[0], -1)
    return Q2[:, :r] @ ((Q1[:, :r].T @ Bm) / np.asarray(sigma)[:r, None])


def normal_equation_residual(A, x, b, norm2_A: float) -> float:
    """||A^T (b - A x)|| / (||A||_2 (||A||_2 ||x|| + ||b||)), columnwise max."""
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(x, dtype=np.float64).reshape(A.shape[1], -1)
    Bm = np.asarray(b, dtype=np.float64).reshape(A.shape[0], -1)
    worst = 0.0
    for j in range(X.shape[1]):
        res = A.T @ (Bm[:, j] - A @ X[:, j])
        den = norm2_A * (norm2_A * np.linalg.norm(X[:, j]) + np.linalg.norm(Bm[:, j]))
        worst = max(worst, float(np.linalg.norm(res) / den) if den > 0 else 0.0)
    return worst
