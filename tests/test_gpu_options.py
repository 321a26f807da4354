"""Options of the C ABI beyond the default path: an explicit V (accumulated
during randUTV, Nullify's reflectors included) and iterative refinement
x <- x + P (b - A x).  Parity with the oracle's Fig. 4 solve (rank equal, x
within 1e-9 relative, normal-equation residual <= 1e-13), plus the
invariants an explicit factorization must satisfy: V^T V = I,
(A V)^T (A V) = T^T T (A V = U T with U orthogonal), T(0:r, r:n) = 0 after
Nullify, and the row-space projector V_1 V_1^T equal to the oracle's."""

import numpy as np
import pytest
import torch

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

pytestmark = pytest.mark.gpu

X_TOL = 1e-9
NER_TOL = 1e-13


def dev(x):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    out = torch.empty((x.shape[1], x.shape[0]), dtype=torch.float64, device="cuda").t()
    out.copy_(torch.as_tensor(x))
    return out


def problem(m, n, r, nrhs, seed):
    A, X, Y = wl.lowrank_xy(m, n, r, seed=seed, noise=1e-14)
    B = np.random.default_rng(seed + 1).standard_normal((m, nrhs))
    nrm = wl.norm2_of_product(X, Y)
    return A, B, nrm


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,r,nb,q,nullify", [
    (700, 300, 120, 32, 1, 1),    # tall, Nullify on V
    (300, 520, 110, 64, 1, 1),    # wide
    (400, 257, 77, 37, 0, 0),     # odd block, fast option (V without Nullify)
    (260, 100, 100, 128, 1, 1),   # full column rank: no Nullify, one step
])
def test_explicit_v_solve_and_invariants(lls, precision, m, n, r, nb, q, nullify):
    if precision != 0 and not nullify:
        pytest.skip("the fast option is FP64-only (test_mixed_fast_option_is_refused)")
    A, B, nrm = problem(m, n, r, 3, seed=m + n + r)
    tol = 1e-10 * nrm
    ref = orc.solve(A, B, q, nb, tol, 2001, do_nullify=bool(nullify), keep=True)
    dA, dB = dev(A), dev(B)
    h = lls.lls_create(nb=nb, q=q, seed=2001, nullify=nullify, precision=precision, explicit_v=1)
    h0 = lls.lls_create(nb=nb, q=q, seed=2001, nullify=nullify, precision=precision)
    # In mixed precision the BF16 sample fixes V_1 only to BF16 accuracy, so
    # the factors (and the fast option's x, which keeps T_12) differ from the
    # oracle's FP64 ones; the minimum-norm x and the row space do not.
    exact_factors = precision == 0
    try:
        X, rank, code = lls.lls_solve(h, dA, dB, tol)
        X0, _, _ = lls.lls_solve(h0, dA, dB, tol)
        assert code == 0 and rank == ref.rank == r
        x, x0 = X.cpu().numpy(), X0.cpu().numpy()
        if exact_factors or nullify:
            assert rel(x, ref.x) <= X_TOL
        assert rel(x, x0) <= 1e-12          # same x as the reflector-replay solve
        assert orc.normal_equation_residual(A, x, B, nrm) <= NER_TOL

        fid, frank, _ = lls.lls_factor(h, dA, tol)
        assert frank == r
        T = lls.lls_factor_get(h, fid, lls.LLS_FACTOR_T, m, n).cpu().numpy()
        V = lls.lls_factor_get(h, fid, lls.LLS_FACTOR_V, n, n).cpu().numpy()
        # solves with the resident factor apply V as one product
        Xf = lls.lls_solve_factored(h, fid, dB, n).cpu().numpy()
        assert rel(Xf, x) <= 1e-13
        lls.lls_factor_release(h, fid)
    finally:
        lls.lls_destroy(h)
        lls.lls_destroy(h0)
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13 * np.sqrt(n)
    AV = A @ V
    assert np.linalg.norm(AV.T @ AV - T.T @ T) <= 1e-13 * nrm ** 2 * np.sqrt(n)
    assert np.all(np.tril(T, -1) == 0.0)
    if nullify and r < n:
        assert np.all(T[:r, r:] == 0.0)
    # row-space projector: unique for a gap matrix, sign-free (without
    # Nullify in mixed mode V_1 is the BF16 sample's subspace instead)
    if exact_factors or nullify:
        V1, W1 = V[:, :r], ref.utv.V[:, :r]
        assert np.linalg.norm(V1 @ V1.T - W1 @ W1.T) <= 1e-10
    # |diag(T)| over the rank: the oracle's, up to the signs of the block SVD
    if exact_factors:
        assert rel(np.abs(np.diagonal(T))[:r], np.abs(np.diagonal(ref.utv.T))[:r]) <= 1e-10


def test_mixed_fast_option_is_refused(lls):
    """With the BF16 sample, range(V_1) carries a BF16-sized error, so T_12 is
    far from zero and the fast option (no Nullify, Eq. (7)) would return a
    least-squares x whose norm exceeds the minimum by 1e-4..1e-2 relative
    (Remark after Fig. 4 only holds for an accurate sample).  The library
    refuses that combination (argument 2, the options) instead; with Nullify
    the mixed x is the oracle's minimum-norm x."""
    with pytest.raises(lls.LLSError) as e:
        lls.lls_create(nb=37, q=0, seed=2001, nullify=0, precision=lls.LLS_MIXED_BF16)
    assert e.value.status == lls.LLS_ERR_ARG
    h = lls.lls_create(nb=37, q=0, seed=2001, nullify=1, precision=lls.LLS_MIXED_BF16)
    try:
        with pytest.raises(lls.LLSError) as e:
            lls.lls_set_options(h, nb=37, q=0, seed=2001, nullify=0, precision=lls.LLS_MIXED_BF16)
        assert e.value.status == lls.LLS_ERR_ARG and e.value.arg == 2
        A, B, nrm = problem(400, 257, 77, 2, seed=400 + 257 + 77)
        tol = 1e-10 * nrm
        x_mn = orc.solve(A, B, 0, 37, tol, 2001).x
        X, rank, code = lls.lls_solve(h, dev(A), dev(B), tol)
        assert code == 0 and rank == 77
        assert rel(X.cpu().numpy(), x_mn) <= X_TOL
        assert orc.normal_equation_residual(A, X.cpu().numpy(), B, nrm) <= NER_TOL
    finally:
        lls.lls_destroy(h)


def test_factor_get_errors(lls):
    A, B, nrm = problem(200, 120, 40, 1, seed=5)
    h = lls.lls_create(nb=32, q=1)
    try:
        fid, _, _ = lls.lls_factor(h, dev(A), 1e-10 * nrm)
        out = lls.empty_colmajor(120, 120)
        # V needs explicit_v = 1
        assert lls._lib.lls_factor_get(h, fid, lls.LLS_FACTOR_V, lls._ptr(out), 120) == lls.LLS_ERR_ARG
        assert lls._lib.lls_factor_get(h, fid, 7, lls._ptr(out), 120) == lls.LLS_ERR_ARG
        assert lls._lib.lls_factor_get(h, fid, lls.LLS_FACTOR_T, lls._ptr(out), 100) == lls.LLS_ERR_ARG
        assert lls._lib.lls_factor_get(h, fid + 99, lls.LLS_FACTOR_T, lls._ptr(out), 200) == \
            lls.LLS_ERR_NOT_FOUND
        lls.lls_factor_release(h, fid)
    finally:
        lls.lls_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_refinement_converges_and_keeps_parity(lls, precision):
    """C1 (2000 x 1000, rank 400): P b is a fixed point of the refinement, so
    the corrections are at the rounding level and the first one is below
    refine_tol = 1e-12; x stays at parity with the oracle."""
    p = wl.c1_problem()
    ref = orc.solve(p.A, p.B, p.q, p.nb, p.tol, 2001)
    h = lls.lls_create(nb=p.nb, q=p.q, seed=2001, precision=precision, max_refine=3)
    try:
        X, rank, code = lls.lls_solve(h, dev(p.A), dev(p.B), p.tol)
        steps, corr = lls.lls_refinement_info(h)
    finally:
        lls.lls_destroy(h)
    assert code == 0 and rank == 400
    assert steps == 1 and 0.0 < corr <= 1e-12
    x = X.cpu().numpy()
    assert rel(x, np.reshape(ref.x, x.shape)) <= X_TOL
    assert orc.normal_equation_residual(p.A, x, p.B, p.norm2) <= NER_TOL


def test_refinement_warns_when_tolerance_unreachable(lls):
    """refine_tol = 0 cannot be met by a nonzero correction: the iteration
    stops at the rounding floor (or max_refine) with LLS_WARN_REFINE_NOCONV
    and a valid, refined x."""
    A, B, nrm = problem(600, 400, 150, 2, seed=11)
    tol = 1e-10 * nrm
    ref = orc.solve(A, B, 1, 32, tol, 2001)
    h = lls.lls_create(nb=32, q=1, seed=2001, max_refine=4, refine_tol=0.0)
    try:
        X, rank, code = lls.lls_solve(h, dev(A), dev(B), tol)
        steps, corr = lls.lls_refinement_info(h)
    finally:
        lls.lls_destroy(h)
    assert code == lls.LLS_WARN_REFINE_NOCONV
    assert 2 <= steps <= 4 and 0.0 < corr < 1e-12
    assert rank == 150
    assert rel(X.cpu().numpy(), ref.x) <= X_TOL


def test_refinement_with_resident_factor(lls):
    """A factor made with max_refine > 0 keeps a copy of A and refines later
    solves with it; a factor made with max_refine = 0 holds no copy, so its
    solves are not refined (0 steps).  Both stay at parity with the oracle."""
    A, B, nrm = problem(500, 300, 90, 4, seed=23)
    tol = 1e-10 * nrm
    ref = orc.solve(A, B, 1, 32, tol, 2001)
    dA, dB = dev(A), dev(B)
    h = lls.lls_create(nb=32, q=1, seed=2001, max_refine=2)
    try:
        fid, rank, _ = lls.lls_factor(h, dA, tol)
        X = lls.lls_solve_factored(h, fid, dB, 300)
        steps, corr = lls.lls_refinement_info(h)
        assert steps >= 1 and corr <= 1e-12
        assert rel(X.cpu().numpy(), ref.x) <= X_TOL
        lls.lls_factor_release(h, fid)
        lls.lls_set_options(h, nb=32, q=1, seed=2001, max_refine=0)
        fid0, _, _ = lls.lls_factor(h, dA, tol)
        lls.lls_set_options(h, nb=32, q=1, seed=2001, max_refine=2)
        X0 = lls.lls_solve_factored(h, fid0, dB, 300)
        assert lls.lls_refinement_info(h)[0] == 0      # no copy of A in that factor
        assert rel(X0.cpu().numpy(), ref.x) <= X_TOL
        lls.lls_factor_release(h, fid0)
    finally:
        lls.lls_destroy(h)


def test_batched_with_options_matches_alone(lls):
    """explicit_v and refinement in the worker pool: each problem's x is
    bit-identical to its lls_solve alone with the same options."""
    probs = [problem(m, n, r, k, seed=s) for (m, n, r, k, s) in
             [(500, 300, 100, 2, 1), (300, 450, 80, 1, 2), (640, 640, 200, 3, 3), (256, 128, 128, 1, 4)]]
    opts = dict(nb=64, q=1, seed=2001, explicit_v=1, max_refine=1)
    h = lls.lls_create(**opts)
    try:
        alone = []
        for A, B, nrm in probs:
            X, _, _ = lls.lls_solve(h, dev(A), dev(B), 1e-10 * nrm)
            alone.append(X.cpu().numpy())
        keep, plist = [], []
        for A, B, nrm in probs:
            dA, dB = dev(A), dev(B)
            X = lls.empty_colmajor(A.shape[1], B.shape[1])
            keep += [dA, dB, X]
            plist.append(lls.make_problem(dA, dB, 1e-10 * nrm, X))
        lls.lls_set_workers(h, 3)
        code = lls.lls_solve_batched(h, plist)
        assert code >= 0
        for i, (A, B, nrm) in enumerate(probs):
            assert plist[i].status >= 0
            np.testing.assert_array_equal(keep[3 * i + 2].cpu().numpy(), alone[i])
            ref = orc.solve(A, B, 1, 64, 1e-10 * nrm, 2001)
            assert rel(alone[i], np.reshape(ref.x, alone[i].shape)) <= X_TOL
    finally:
        lls.lls_destroy(h)
