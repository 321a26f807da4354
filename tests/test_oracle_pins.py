"""Pins for the FP64 oracle: each test ties the oracle to something other than
itself -- a library routine, a closed form, an invariant of the factorization,
the structural example of Fig. 1, or the brute-force pseudoinverse.

CPU only (no GPU marker).
"""

import os

import numpy as np
import pytest
import scipy.stats

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- RNG
@pytest.mark.parametrize("key", [(0, 0), (5, 7), (2**64 - 1, 2**63 + 12345), (2002, 0)])
@pytest.mark.parametrize("ctr", [(1, 0, 0, 0), (17, 3, 9, 0), (2**40, 2**33, 127, 5),
                                 (2**64 - 1, 0, 0, 0)])
def test_philox_matches_numpy_bit_generator(key, ctr):
    """numpy.random.Philox is Philox4x64-10; it increments its 256-bit
    counter before producing a block, so a generator whose counter is c - 1
    yields the block of counter c."""
    before = list(ctr)
    before[0] -= 1  # ctr[0] >= 1 in every case above: no borrow
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(before, dtype=np.uint64))
    want = bg.random_raw(4)
    got = orc.philox4x64_10([np.uint64(c) for c in ctr], key)
    assert [int(g) for g in got] == [int(w) for w in want]


def test_sketch_is_standard_normal():
    G = orc.sketch_matrix(2001, 0, 4000, 64)
    z = G.ravel()
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    # different steps and columns are uncorrelated
    G1 = orc.sketch_matrix(2001, 1, 4000, 64)
    assert abs(np.corrcoef(G[:, 0], G1[:, 0])[0, 1]) < 0.1
    assert abs(np.corrcoef(G[:, 0], G[:, 1])[0, 1]) < 0.1


def test_sketch_layout_is_prefix_stable():
    """Entry (p, j) depends only on (seed, step, p, j): a smaller sketch is a
    leading block of a larger one (ragged row counts included)."""
    big = orc.sketch_matrix(7, 3, 103, 9)
    small = orc.sketch_matrix(7, 3, 50, 5)
    assert np.array_equal(big[:50, :5], small)


# -------------------------------------------------------------- Householder
@pytest.mark.parametrize("x", [np.array([3.0, 4.0]), np.array([-1.0, 2.0, -2.0]),
                               np.array([0.0, 1e-3, 5.0]), np.array([2.5, 0.0, 0.0]),
                               np.array([-2.5, 0.0])])
def test_householder_reflects_to_axis(x):
    v, tau, beta = orc.householder(x)
    H = np.eye(x.size) - tau * np.outer(v, v)
    y = H @ x
    assert np.allclose(y[1:], 0.0, atol=1e-15 * np.linalg.norm(x))
    assert np.isclose(y[0], beta)
    assert np.allclose(H @ H.T, np.eye(x.size), atol=1e-15)
    if np.any(x[1:] != 0):
        assert np.isclose(abs(beta), np.linalg.norm(x))
        assert beta * x[0] <= 0.0  # beta = -sign(alpha) ||x||
    else:
        assert tau == 0.0 and beta == x[0]


@pytest.mark.parametrize("shape", [(40, 12), (12, 12), (7, 11), (300, 64)])
def test_householder_qr_matches_lapack(shape):
    """LAPACK dgeqrf (numpy.linalg.qr mode='raw') uses the same xLARFG
    convention: R and tau agree to rounding."""
    Y = np.random.default_rng(3).standard_normal(shape)
    R, W, tau = orc.householder_qr(Y)
    h, tau_lapack = np.linalg.qr(Y, mode="raw")
    R_lapack = np.triu(h.T[: min(shape), :])
    assert np.allclose(R, R_lapack, rtol=0, atol=1e-13 * np.abs(Y).max())
    assert np.allclose(tau, tau_lapack, atol=1e-14)
    # Q = H_0 ... H_{k-1} reproduces Y and is orthogonal
    Q = np.eye(shape[0])
    for j in range(tau.size):
        Q = Q @ (np.eye(shape[0]) - tau[j] * np.outer(W[:, j], W[:, j]))
    assert np.allclose(Q[:, : R.shape[0]] @ R, Y, atol=1e-13 * np.abs(Y).max())
    assert np.allclose(Q.T @ Q, np.eye(shape[0]), atol=1e-14 * shape[0])


def test_wy_factor_equals_product_of_reflectors():
    Y = np.random.default_rng(4).standard_normal((50, 16))
    _, W, tau = orc.householder_qr(Y)
    T = orc.wy_factor(W, tau)
    P = np.eye(50)
    for j in range(16):
        P = P @ (np.eye(50) - tau[j] * np.outer(W[:, j], W[:, j]))
    assert np.allclose(np.eye(50) - W @ T @ W.T, P, atol=1e-14)
    assert np.allclose(T, np.triu(T))


# ------------------------------------------------------------------ randUTV
def _check_utv(A, res, nb, tol_fact=1e-13):
    m, n = A.shape
    U, T, V = res.U, res.T, res.V
    assert np.linalg.norm(U.T @ U - np.eye(m)) < 1e-14 * m
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 1e-14 * n
    nrm = max(np.linalg.norm(A), 1e-300)
    assert np.linalg.norm(A - U @ T @ V.T) / nrm < tol_fact
    assert np.allclose(np.tril(T, -1), 0.0)
    # each diagonal block is diagonal with nonnegative, descending entries
    k = 0
    while k < min(m, n):
        b = min(nb, m - k, n - k)
        blk = T[k:k + b, k:k + b]
        assert np.allclose(blk - np.diag(np.diagonal(blk)), 0.0)
        d = np.diagonal(blk)
        assert np.all(d >= 0) and np.all(np.diff(d) <= 0)
        k += b


@pytest.mark.parametrize("m,n,nb,q", [(60, 40, 8, 1), (40, 40, 16, 0), (33, 57, 7, 2),
                                      (101, 37, 37, 1), (25, 10, 64, 1)])
def test_randutv_invariants(m, n, nb, q):
    A = np.random.default_rng(m * n).standard_normal((m, n))
    res = orc.randutv(A, q, nb, seed=11)
    _check_utv(A, res, nb)


def test_randutv_rank_deficient_invariants():
    A, _, _ = wl.lowrank_xy(120, 90, 30, seed=5)
    res = orc.randutv(A, 1, 16, seed=12)
    _check_utv(A, res, 16)
    d = np.diagonal(res.T)
    assert np.all(d[:30] > 1e-3 * d[0]) and np.all(d[30:] < 1e-12 * d[0])


def _read_fig1():
    pats, cur = {}, None
    with open(os.path.join(GOLDEN, "fig1_pattern.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("step"):
                cur = int(line.split()[1])
                pats[cur] = []
            else:
                pats[cur].append(line)
    return pats


def test_fig1_sparsity_pattern():
    """Fig. 1: m = 11, n = 8, nb = 3; T after each step has the printed
    zero / nonzero structure."""
    pats = _read_fig1()
    A = np.random.default_rng(1).standard_normal((11, 8))
    for step, rows in pats.items():
        T = orc.randutv(A, 1, 3, seed=3, max_steps=step).T
        for i, row in enumerate(rows):
            for j, ch in enumerate(row):
                if ch == ".":
                    assert abs(T[i, j]) < 1e-13, (step, i, j, T[i, j])
                else:
                    assert abs(T[i, j]) > 1e-10, (step, i, j, T[i, j])


def test_rsvd_identity_first_step():
    """Remark after Fig. 2: U(:,1:nb) T(1:nb,1:nb) V(:,1:nb)^T equals the
    randomized-SVD rank-nb approximation from the same sketch, A P_Y with
    P_Y the projector onto range(Y), Y = (A^T A)^q A^T G."""
    A, _, _ = wl.lowrank_xy(80, 60, 25, seed=8, noise=1e-3)
    nb, q, seed = 10, 1, 21
    res = orc.randutv(A, q, nb, seed=seed, max_steps=1)
    G = orc.sketch_matrix(seed, 0, 80, nb)
    Y = A.T @ G
    for _ in range(q):
        Y = A.T @ (A @ Y)
    Qy = np.linalg.qr(Y)[0]
    approx = res.U[:, :nb] @ res.T[:nb, :nb] @ res.V[:, :nb].T
    assert np.allclose(approx, A @ Qy @ Qy.T, atol=1e-12 * np.linalg.norm(A))


def test_diagonal_tracks_singular_values_with_power_iteration():
    """Sec. 3.1: power iterations make the diagonal of T approximate the
    singular values (median relative error shrinks with q; below 1e-3 at
    q = 2); the first block's diagonal interlaces, T(j,j) <= sigma_j, since it
    holds the singular values of U_1^T A V_1."""
    sigma = wl.step_spectrum(96, 48, 3.0, 1e-15)
    A, _, _ = wl.spectrum_matrix(96, 96, sigma, seed=9)
    med = []
    for q in (0, 1, 2):
        d = np.diagonal(orc.randutv(A, q, 16, seed=4).T)
        med.append(np.median(np.abs(d[:48] - sigma[:48]) / sigma[:48]))
        assert np.all(d[:16] <= sigma[:16] * (1 + 1e-13))
        assert np.all(d[48:] < 1e-13)
    assert med[0] > med[1] > med[2] and med[2] < 1e-3


# ------------------------------------------------------------------- rank
def test_compute_rank_prefix_and_count():
    T = np.diag([5.0, 3.0, 1e-12, 2.0, 1e-13])
    assert orc.compute_rank(T, 1e-10) == (2, 3)
    assert orc.compute_rank(np.diag([1.0, 1e-10]), 1e-10) == (1, 1)  # equal -> zero
    assert orc.compute_rank(np.zeros((3, 2)), 0.0) == (0, 0)
    assert orc.compute_rank(np.eye(4)[:, :3], 0.5) == (3, 3)


# ------------------------------------------------------------------ Nullify
@pytest.mark.parametrize("r,n,nb", [(12, 20, 5), (7, 30, 7), (16, 17, 4), (9, 9, 3)])
def test_nullify_is_an_rz_factorization(r, n, nb):
    """On an upper-trapezoidal [C D] with a dense D: afterwards T(0:r, r:n) = 0,
    C is upper triangular, V is orthogonal and T_before = T_after V^T; the
    min-norm solution of [C D] z = c built from it equals lstsq's."""
    g = np.random.default_rng(r * n)
    T = np.zeros((r + 3, n))
    T[:r, :r] = np.triu(g.standard_normal((r, r))) + 3 * np.eye(r)
    T[:r, r:] = g.standard_normal((r, n - r))
    T0 = T.copy()
    V = np.eye(n)
    orc.nullify(T, V, r, nb)
    assert np.allclose(T[:r, r:], 0.0, atol=1e-14)
    assert np.allclose(np.tril(T[:r, :r], -1), 0.0, atol=1e-14)
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-14 * n)
    assert np.allclose(T @ V.T, T0, atol=1e-13)
    c = g.standard_normal(r)
    z = V[:, :r] @ np.linalg.solve(T[:r, :r], c)
    z_ref = np.linalg.lstsq(T0[:r], c, rcond=None)[0]
    assert np.allclose(z, z_ref, atol=1e-12 * np.linalg.norm(z_ref))


# -------------------------------------------------------------------- solve
@pytest.mark.parametrize("m,n,r,nb,q", [(150, 100, 40, 16, 1), (100, 150, 40, 16, 1),
                                        (200, 200, 120, 32, 0), (90, 60, 60, 13, 2),
                                        (64, 64, 1, 8, 1)])
def test_solution_matches_pseudoinverse(m, n, r, nb, q):
    """Brute force: x equals the truncated-SVD least-squares solution with the
    same rank (Sec. 2.2) on exactly-rank-r matrices."""
    A, X, Y = wl.lowrank_xy(m, n, r, seed=m + n + r, noise=1e-14)
    B = np.random.default_rng(2).standard_normal((m, 3))
    nrm = wl.norm2_of_product(X, Y)
    sol = orc.solve(A, B, q, nb, 1e-10 * nrm, seed=77)
    assert sol.rank == r and sol.rank_count == r
    x_ref = orc.pinv_solve(A, B, r)
    assert np.linalg.norm(sol.x - x_ref) / np.linalg.norm(x_ref) < 1e-12
    assert orc.normal_equation_residual(A, sol.x, B, nrm) < 1e-14


def test_full_column_rank_equals_qr_least_squares():
    """Eq. (6) / Sec. 2.1: with no nullspace x = R^{-1} Q^T b."""
    g = np.random.default_rng(6)
    A = g.standard_normal((120, 45))
    b = g.standard_normal(120)
    sol = orc.solve(A, b, 1, 16, 1e-10 * np.linalg.norm(A, 2), seed=5)
    Q, R = np.linalg.qr(A)
    assert sol.rank == 45
    assert np.allclose(sol.x, np.linalg.solve(R, Q.T @ b), rtol=1e-12, atol=1e-13)


def test_consistent_system_recovers_row_space_solution():
    A, X, Y = wl.lowrank_xy(70, 90, 30, seed=31)
    x0 = A.T @ np.random.default_rng(1).standard_normal(70)   # in range(A^T)
    sol = orc.solve(A, A @ x0, 1, 8, 1e-10 * wl.norm2_of_product(X, Y), seed=3)
    assert np.allclose(sol.x, x0, rtol=1e-11, atol=1e-11 * np.linalg.norm(x0))


def test_zero_matrix_gives_zero():
    sol = orc.solve(np.zeros((30, 20)), np.ones(30), 1, 8, 0.0, seed=1)
    assert sol.rank == 0 and np.all(sol.x == 0)


def test_single_step_and_power_iteration_independence():
    sigma = wl.step_spectrum(80, 50, 4.0, 1e-15)
    A, _, _ = wl.spectrum_matrix(100, 80, sigma, seed=12)
    b = np.random.default_rng(0).standard_normal(100)
    xs = [orc.solve(A, b, q, nb, 1e-10, seed=8).x for q, nb in [(0, 16), (2, 16), (1, 128)]]
    ref = orc.pinv_solve(A, b, 50)
    for x in xs:
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9


def test_nullify_gives_no_larger_norm_than_fast_option():
    """The fast option (Eq. (7)) solves the same truncated system without
    the minimum-norm guarantee: its norm can only be larger or equal, and on
    a gap matrix the two agree."""
    g = np.random.default_rng(13)
    A = g.standard_normal((60, 50)) @ np.diag(np.logspace(0, -12, 50)) @ \
        np.linalg.qr(g.standard_normal((50, 50)))[0]
    b = g.standard_normal(60)
    full = orc.solve(A, b, 0, 8, 1e-8, seed=2)
    fast = orc.solve(A, b, 0, 8, 1e-8, seed=2, do_nullify=False)
    assert full.rank == fast.rank
    assert np.linalg.norm(full.x) <= np.linalg.norm(fast.x) * (1 + 1e-12)
    A2, X, Y = wl.lowrank_xy(80, 60, 20, seed=3, noise=1e-14)
    nrm = wl.norm2_of_product(X, Y)
    a = orc.solve(A2, b[:50].tolist() + [0.0] * 30, 1, 8, 1e-10 * nrm, seed=2)
    f = orc.solve(A2, b[:50].tolist() + [0.0] * 30, 1, 8, 1e-10 * nrm, seed=2, do_nullify=False)
    assert np.linalg.norm(a.x - f.x) / np.linalg.norm(a.x) < 1e-9


def test_solution_orthogonal_to_nullspace():
    A, X, Y = wl.lowrank_xy(90, 70, 25, seed=44, noise=1e-14)
    b = np.random.default_rng(9).standard_normal(90)
    sol = orc.solve(A, b, 1, 16, 1e-10 * wl.norm2_of_product(X, Y), seed=4)
    N0 = np.linalg.svd(A)[2][25:].T  # trailing right singular vectors
    assert np.linalg.norm(N0.T @ sol.x) / np.linalg.norm(sol.x) < 1e-12


def test_pinv_from_factors_equals_svd_pinv():
    """The factor-based pseudoinverse used at full size equals the SVD-based
    one on a matrix built from the same factors."""
    sigma = wl.step_spectrum(120, 60, 6.0, 1e-15)
    A, Q1, Q2 = wl.spectrum_matrix(150, 120, sigma, seed=3)
    B = np.random.default_rng(1).standard_normal((150, 4))
    x1 = orc.pinv_solve_from_factors(Q1, sigma, Q2, B, 60)
    x2 = orc.pinv_solve(A, B, 60)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-9


# -------------------------------------------------------------------- refinement
@pytest.mark.parametrize("nullify", [True, False])
def test_refine_removes_error_in_row_space_in_one_step(nullify):
    """U_1^T A V_1 = T_11 (A V = U T, T upper triangular), so P A = I on
    range(V_1): one refinement step from x + V_1 c returns x for any c."""
    A, X, Y = wl.lowrank_xy(120, 90, 35, seed=21, noise=1e-14)
    b = np.random.default_rng(3).standard_normal(120)
    nrm = wl.norm2_of_product(X, Y)
    sol = orc.solve(A, b, 1, 16, 1e-10 * nrm, seed=5, do_nullify=nullify, keep=True)
    assert sol.rank == 35
    V1 = sol.utv.V[:, :35]
    x_bad = sol.x + V1 @ np.random.default_rng(4).standard_normal(35)
    assert np.linalg.norm(x_bad - sol.x) > 0.1 * np.linalg.norm(sol.x)
    x1 = orc.refine(A, b, sol, x0=x_bad, steps=1)
    assert np.linalg.norm(x1 - sol.x) / np.linalg.norm(sol.x) < 1e-12


def test_refine_fixed_point_and_pseudoinverse():
    """P b is a fixed point: refining the solution changes it only by
    rounding, and the refined x is still the truncated-SVD solution."""
    A, X, Y = wl.lowrank_xy(100, 80, 30, seed=8, noise=1e-14)
    B = np.random.default_rng(5).standard_normal((100, 2))
    nrm = wl.norm2_of_product(X, Y)
    sol = orc.solve(A, B, 1, 16, 1e-10 * nrm, seed=9, keep=True)
    x2 = orc.refine(A, B, sol, steps=2)
    assert np.linalg.norm(x2 - sol.x) / np.linalg.norm(sol.x) < 1e-13
    x_ref = orc.pinv_solve(A, B, 30)
    assert np.linalg.norm(x2 - x_ref) / np.linalg.norm(x_ref) < 1e-12


def test_refine_leaves_nullspace_components():
    """After Nullify T_12 = 0, so P A V_2 = 0: refinement cannot remove a
    nullspace component (the minimum-norm property comes from P b itself)."""
    A, X, Y = wl.lowrank_xy(70, 60, 20, seed=17, noise=1e-14)
    b = np.random.default_rng(6).standard_normal(70)
    sol = orc.solve(A, b, 1, 8, 1e-10 * wl.norm2_of_product(X, Y), seed=2, keep=True)
    V2 = sol.utv.V[:, 20:]
    c = np.random.default_rng(7).standard_normal(40)
    x1 = orc.refine(A, b, sol, x0=sol.x + V2 @ c, steps=1)
    assert np.linalg.norm(x1 - (sol.x + V2 @ c)) < 1e-9 * np.linalg.norm(c)


def _perturbed(sol, angle, rel, seed):
    """A copy of sol's factors spoiled like a TF32 factorization: U and V
    rotated by random orthogonal matrices exp(angle S) (S skew, so range(U_1)
    and range(V_1) tilt by about `angle`) and T_11 perturbed by `rel`
    relative."""
    import copy

    import scipy.linalg

    g = np.random.default_rng(seed)
    bad = copy.deepcopy(sol)
    for name in ("U", "V"):
        F = getattr(sol.utv, name)
        S = g.standard_normal((F.shape[0], F.shape[0]))
        setattr(bad.utv, name, F @ scipy.linalg.expm(angle * (S - S.T) / np.sqrt(F.shape[0])))
    r = sol.rank
    bad.utv.T[:r, :r] = np.triu(sol.utv.T[:r, :r] * (1 + rel * g.standard_normal((r, r))))
    return bad


def test_refine_min_norm_exact_factors_give_pinv_in_one_step():
    """With exact factors P = A^+ and M = A^T P^T P P^T A^T = A^+: one step
    from 0 is the truncated-SVD solution (b with a residual outside range(A))."""
    A, X, Y = wl.lowrank_xy(90, 70, 25, seed=31, noise=0.0)
    B = np.random.default_rng(8).standard_normal((90, 2))
    sol = orc.solve(A, B, 1, 16, 1e-10 * wl.norm2_of_product(X, Y), seed=4, keep=True)
    assert sol.rank == 25
    x1 = orc.refine_min_norm(A, B, sol, steps=1)
    x_ref = orc.pinv_solve(A, B, 25)
    assert np.linalg.norm(x1 - x_ref) / np.linalg.norm(x_ref) < 1e-11


def test_refine_min_norm_recovers_from_approximate_factors():
    """Factors with a 1e-5 tilt of range(U_1) and range(V_1) and 1e-6
    relative error in T_11 (a TF32-accurate factorization): refine converges
    to a solution inside the tilted range(V_1), 1e-5 away from the
    minimum-norm one, and so would x <- x + A^T P^T P (b - A x) (fixed point
    U_1^T r = 0, oblique to range(A)); refine_min_norm converges to the
    pseudoinverse solution (stage 1 makes A^T r = 0, stage 2 projects onto
    range(A^T))."""
    A, X, Y = wl.lowrank_xy(120, 80, 30, seed=13, noise=0.0)
    B = np.random.default_rng(2).standard_normal((120, 2))
    sol = orc.solve(A, B, 1, 16, 1e-10 * wl.norm2_of_product(X, Y), seed=6, keep=True)
    bad = _perturbed(sol, 1e-5, 1e-6, seed=1)
    x_ref = orc.pinv_solve(A, B, 30)
    err = lambda x: np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    x_plain = orc.refine(A, B, bad, x0=np.zeros_like(sol.x), steps=8)
    assert err(x_plain) > 1e-7
    U, T, V, r = bad.utv.U, bad.utv.T, bad.utv.V, bad.rank
    x_obl = np.zeros_like(sol.x)
    for _ in range(8):   # A^T P^T P (b - A x): the trailing P^T A^T left out
        y = orc._back_substitution(T[:r, :r], U[:, :r].T @ (B - A @ x_obl))
        x_obl = x_obl + A.T @ (U[:, :r] @ orc._forward_substitution_transposed(T[:r, :r], y))
    assert err(x_obl) > 1e-7
    errs = [err(orc.refine_min_norm(A, B, bad, steps=k)) for k in (1, 2, 4)]
    assert errs[0] > 1e-9 and errs[1] < errs[0] and errs[2] < 1e-12
    x4 = orc.refine_min_norm(A, B, bad, steps=4)
    assert np.linalg.norm(A.T @ (B - A @ x4)) < 1e-12 * np.linalg.norm(A) ** 2 * np.linalg.norm(x4)
    N0 = np.linalg.svd(A)[2][30:].T
    assert np.linalg.norm(N0.T @ x4) < 1e-12 * np.linalg.norm(x4)


def test_refine_min_norm_contracts_by_kappa_eps_not_its_square():
    """Singular values 1 .. 1e-4 (kappa = 1e4, the 32768 x 16384 workload's
    spectrum) and factors perturbed by 1e-5: kappa eps = 0.1 < 1 but
    kappa^2 eps = 1000 > 1.  A one-stage iteration x <- x + M (b - A x) with
    M = A^T P^T P P^T A^T carries P P^T ~ (A^T A)^+ and diverges; the two
    stages converge to the pseudoinverse solution."""
    p = wl.c3_like(160, 100, 60, nrhs=2, nb=16, q=1)
    sol = orc.solve(p.A, p.B, 1, 16, p.tol, 2001, keep=True)
    assert sol.rank == 60
    bad = _perturbed(sol, 1e-5, 1e-5, seed=3)
    x_ref = orc.pinv_solve_from_factors(p.factors["Q1"], p.factors["sigma"], p.factors["Q2"], p.B, 60)
    err = lambda x: np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    U, T, V, r = bad.utv.U, bad.utv.T, bad.utv.V, bad.rank
    T11 = T[:r, :r]
    Pf = lambda R: V[:, :r] @ orc._back_substitution(T11, U[:, :r].T @ R)
    Pt = lambda S: U[:, :r] @ orc._forward_substitution_transposed(T11, V[:, :r].T @ S)
    x = np.zeros_like(sol.x)
    errs_one = []
    for _ in range(4):
        x = x + p.A.T @ Pt(Pf(Pt(p.A.T @ (p.B - p.A @ x))))
        errs_one.append(err(x))
    assert errs_one[3] > errs_one[2] > errs_one[1] > 1.0     # diverges
    errs = [err(orc.refine_min_norm(p.A, p.B, bad, steps=k)) for k in (1, 2, 8)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-11


def test_refine_min_norm_needs_a_gap_at_the_rank():
    """sigma_i = 0.8^i (no gap) with tol inside the spectrum: A is not of rank
    r, M = A^T P^T P P^T A^T differs from P by about sigma_{r+1} / sigma_r and
    its fixed point from the truncated solution P b.  The largest dropped
    singular value of the diagonal blocks exceeds 1e-2 times the smallest
    kept one, so refine_min_norm returns the solution unrefined."""
    m, n = 60, 40
    Q1 = np.linalg.qr(np.random.default_rng(1).standard_normal((m, m)))[0][:, :n]
    Q2 = np.linalg.qr(np.random.default_rng(2).standard_normal((n, n)))[0]
    A = (Q1 * 0.8 ** np.arange(n)) @ Q2.T
    b = np.random.default_rng(3).standard_normal(m)
    sol = orc.solve(A, b, 0, 8, 1e-3, seed=4, keep=True)
    assert 0 < sol.rank < n
    assert sol.diag[sol.rank:].max() > orc.MIN_NORM_GAP * sol.diag[:sol.rank].min()
    assert np.array_equal(orc.refine_min_norm(A, b, sol, steps=3), sol.x)


# -------------------------------------------------------------------- properties
def test_normal_equation_residual_closed_forms():
    """The normalisation of the normal-equation residual (reading c15),
    ||A^T (b - A x)|| / (||A||_2 (||A||_2 ||x|| + ||b||)) per column, max over
    columns, pinned by values worked out by hand on A = [[3, 0], [0, 1], [0, 0]]
    (||A||_2 = 3):
      column 0: x = (1, 2), b = (1, 1, 5): A x = (3, 2, 0), b - A x = (-2, -1, 5),
                A^T (b - A x) = (-6, -1), norm sqrt(37); ||x|| = sqrt(5),
                ||b|| = 3 sqrt(3)  ->  sqrt(37) / (9 (sqrt(5) + sqrt(3))) = 0.170323...
      column 1: x = 0, b = (0, 4, 0): A^T b = (0, 4), norm 4; ||b|| = 4
                ->  4 / (3 (0 + 4)) = 1/3.
    A dropped or extra ||A||_2, a transposed A, the wrong column or norms
    taken over all columns at once each give another number."""
    A = np.array([[3.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    x0, b0 = np.array([1.0, 2.0]), np.array([1.0, 1.0, 5.0])
    x1, b1 = np.zeros(2), np.array([0.0, 4.0, 0.0])
    assert orc.normal_equation_residual(A, x0, b0, 3.0) == pytest.approx(0.170323153, rel=1e-8)
    assert orc.normal_equation_residual(A, x1, b1, 3.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    X, B = np.stack([x0, x1], axis=1), np.stack([b0, b1], axis=1)
    assert orc.normal_equation_residual(A, X, B, 3.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert orc.normal_equation_residual(A, X[:, ::-1], B[:, ::-1], 3.0) == pytest.approx(1.0 / 3.0,
                                                                                         rel=1e-15)
    # the exact least-squares solution of b = (3, 1, 7): x = (1, 1), A^T r = 0 exactly
    assert orc.normal_equation_residual(A, np.array([1.0, 1.0]), np.array([3.0, 1.0, 7.0]), 3.0) == 0.0
    # invariant under (A, b, ||A||) -> (c A, c b, c ||A||): numerator and
    # denominator both scale with c^2 (an extra or missing ||A|| breaks it)
    for c in (0.25, 8.0):
        assert orc.normal_equation_residual(c * A, x0, c * b0, 3.0 * c) == pytest.approx(0.170323153,
                                                                                          rel=1e-8)


from hypothesis import HealthCheck, given, settings, strategies as st  # noqa: E402


@settings(max_examples=30, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(m=st.integers(1, 36), n=st.integers(1, 36), nb=st.integers(1, 40), q=st.integers(0, 2),
       r=st.integers(0, 36), seed=st.integers(0, 2**31 - 1), nullify=st.booleans())
def test_solve_properties_on_random_small_problems(m, n, nb, q, r, seed, nullify):
    """Over random shapes, block sizes (including nb > min(m, n) and nb = 1),
    power counts and ranks: the factorization invariants hold, the rank is the
    construction's, and with Nullify x is the truncated-SVD solution; without
    it x is still a least-squares solution of the rank-r system."""
    r = min(r, m, n)
    g = np.random.default_rng(seed)
    if r > 0:
        X = g.standard_normal((m, r))
        Y = g.standard_normal((r, n))
        A = X @ Y
    else:
        A = np.zeros((m, n))
    b = g.standard_normal(m)
    s = np.linalg.svd(A, compute_uv=False) if min(m, n) else np.zeros(0)
    smax = s[0] if s.size else 0.0
    if r > 0 and s[r - 1] < 1e-6 * smax:       # nearly dependent draw: rank not well defined
        return
    tol = 1e-9 * smax
    res = orc.randutv(A, q, nb, seed=seed % 1000)
    if min(m, n) > 0:
        _check_utv(A, res, nb, tol_fact=1e-12)
    sol = orc.solve(A, b, q, nb, tol, seed=seed % 1000, do_nullify=nullify)
    assert sol.rank == r and sol.rank_count == r
    if r == 0:
        assert np.all(sol.x == 0)
        return
    x_ref = orc.pinv_solve(A, b, r)
    if nullify:
        assert np.linalg.norm(sol.x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    else:
        # same residual as the minimum-norm solution, norm no smaller
        assert np.linalg.norm(A @ sol.x - A @ x_ref) <= 1e-9 * max(np.linalg.norm(b), 1.0)
        assert np.linalg.norm(sol.x) >= np.linalg.norm(x_ref) * (1 - 1e-9)
