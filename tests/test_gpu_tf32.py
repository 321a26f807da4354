"""TF32 precision modes: the split-operand GEMM on the TF32 tensor cores
(lls_k_gemm_tf32) against plain FP64 products, the transposed triangular
solve, and whole solves against the FP64 oracle.

With 3xTF32 products (hi*hi + hi*lo + lo*hi, FP32 accumulation) the
factorization carries errors of about 2^-21 ||A||, so the solve is at parity
only after the minimum-norm refinement (least squares with the right
preconditioner V_1 T_11^{-1}, then the projection onto range(A^T)), and only
where tol and the kept singular values sit well above that noise
(tol = 1e-6 ||A|| here, as in the 32768 x 16384 workload).
Plain TF32 (hi*hi only, about 2^-11) reveals the rank of a matrix whose
kept singular values stay above about 1e-2 ||A|| and fails on the
geometric spectrum down to 1e-4: that failure is asserted, not hidden."""

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


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ the GEMM
@pytest.mark.parametrize("terms", [3, 1])
@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (130, 70, 200), (300, 129, 1000), (128, 128, 256),
                                   (257, 65, 4097)])
def test_tf32_gemm_error_against_fp64(lls, terms, ta, tb, m, n, k):
    """|C - A B| <= c sum_k |a_ik b_kj| with c = 2e-6 for 3xTF32 (splitting
    2^-22 per operand, FP32 accumulation over at most 1024 terms) and 2e-3
    for plain TF32; rows and columns spread over 16 orders of magnitude."""
    g = np.random.default_rng(m + 3 * n + 7 * k + ta + 2 * tb + 11 * terms)
    A = g.standard_normal((m, k)) * 10.0 ** g.uniform(-8, 8, (m, 1))
    B = g.standard_normal((k, n)) * 10.0 ** g.uniform(-8, 8, (1, n))
    got, st = lls.lls_k_gemm_tf32(ta, tb, dev(A.T if ta else A), dev(B.T if tb else B), terms=terms)
    assert st == 0
    scale = np.abs(A) @ np.abs(B)
    err = np.max(np.abs(host(got) - A @ B) / scale)
    assert err < (2e-6 if terms == 3 else 2e-3), err
    if terms == 1 and k >= 200:
        assert err > 1e-6, err          # plain TF32 really drops the low parts


@pytest.mark.parametrize("terms", [3, 1])
def test_tf32_gemm_integer_inputs_are_exact(lls, terms):
    # |entries| <= 30 fit in 11 bits: hi is exact, the products and their
    # FP32 sums (below 2^24) too, so the layout is checked to the last bit
    g = np.random.default_rng(5)
    A = g.integers(-30, 31, (200, 1500)).astype(np.float64)
    B = g.integers(-30, 31, (1500, 90)).astype(np.float64)
    got, st = lls.lls_k_gemm_tf32(0, 0, dev(A), dev(B), terms=terms)
    assert st == 0
    assert np.array_equal(host(got), A @ B)


def test_tf32_gemm_alpha_beta_unit_lower_gram(lls):
    g = np.random.default_rng(6)
    A, B, C0 = g.standard_normal((150, 300)), g.standard_normal((300, 80)), g.standard_normal((150, 80))
    got, st = lls.lls_k_gemm_tf32(0, 0, dev(A), dev(B), dev(C0), alpha=-0.5, beta=2.0)
    assert st == 0
    assert np.max(np.abs(host(got) - (2.0 * C0 - 0.5 * (A @ B)))) < 2e-6 * np.max(np.abs(A) @ np.abs(B))
    # Gram W^T W of a unit lower W (its planes reused for both operands): the
    # diagonal sums K squares of one sign, so the FP32 accumulation error grows
    # with K instead of averaging out -- up to K 2^-24 relative.  That is why the
    # solver forms its T factors' Gram matrices with the exact-slice GEMM.
    W = g.standard_normal((400, 64))
    Wl = np.tril(W, -1)
    Wl[np.arange(64), np.arange(64)] = 1.0
    Wd = dev(W)
    got, st = lls.lls_k_gemm_tf32(1, 0, Wd, Wd, unit_lower_a=True, unit_lower_b=True)
    assert st == 0
    err = np.abs(host(got) - Wl.T @ Wl) / (np.abs(Wl.T) @ np.abs(Wl))
    assert err.max() < 400 * 2.0 ** -24
    assert np.median(err) < 2e-6


def test_trsm_upper_trans(lls):
    g = np.random.default_rng(7)
    r = 200
    R = np.triu(g.standard_normal((r, r))) + 5 * np.eye(r)
    B = g.standard_normal((r, 3))
    got = host(lls.lls_k_trsm_upper_trans(dev(R), dev(B)))
    assert np.allclose(R.T @ got, B, rtol=0, atol=1e-12 * np.abs(B).max())


# ------------------------------------------------------------------ solves
def solve(lls, A, B, tol, nb, q, precision, max_refine=10, explicit_v=0, seed=2001):
    h = lls.lls_create(nb=nb, q=q, seed=seed, precision=precision, max_refine=max_refine,
                       refine_tol=1e-11, explicit_v=explicit_v)
    try:
        X, rank, code = lls.lls_solve(h, dev(A), dev(B), tol)
        steps, corr = lls.lls_refinement_info(h)
        return host(X), rank, code, steps
    finally:
        lls.lls_destroy(h)


@pytest.mark.parametrize("nb,q,explicit_v", [(32, 1, 0), (64, 2, 0), (128, 1, 0), (48, 1, 1)])
def test_3xtf32_solve_scaled_mixed_workload(lls, nb, q, explicit_v):
    """1024 x 512, rank 384, sigma geometric 1 -> 1e-4 then 1e-14, tol 1e-6:
    the rank is revealed and x matches the oracle after refinement; without
    refinement x carries the TF32 factorization's error."""
    p = wl.c3_like(1024, 512, 384, nrhs=2, nb=nb, q=q)
    ref = orc.solve(p.A, p.B, q, nb, p.tol, 2001)
    assert ref.rank == 384
    x0, rank0, _, _ = solve(lls, p.A, p.B, p.tol, nb, q, lls.LLS_MIXED_BF16_3xTF32, max_refine=0,
                            explicit_v=explicit_v)
    assert rank0 == 384 and rel(x0, ref.x) > 1e-8
    x, rank, code, steps = solve(lls, p.A, p.B, p.tol, nb, q, lls.LLS_MIXED_BF16_3xTF32,
                                 explicit_v=explicit_v)
    assert code == lls.LLS_OK and rank == 384 and steps >= 2
    assert rel(x, ref.x) <= X_TOL
    assert orc.normal_equation_residual(p.A, x, p.B, 1.0) <= NER_TOL


@pytest.mark.parametrize("m,n,r", [(2000, 1000, 400), (300, 520, 110), (257, 129, 129)])
def test_3xtf32_solve_lowrank(lls, m, n, r):
    A, X, Y = wl.lowrank_xy(m, n, r, seed=m + n + r, noise=1e-14)
    B = np.random.default_rng(r).standard_normal((m, 2))
    nrm = wl.norm2_of_product(X, Y)
    tol = 1e-6 * nrm
    ref = orc.solve(A, B, 1, 64, tol, 2001)
    assert ref.rank == r
    x, rank, code, _ = solve(lls, A, B, tol, 64, 1, lls.LLS_MIXED_BF16_3xTF32)
    assert code == lls.LLS_OK and rank == r
    assert rel(x, ref.x) <= X_TOL
    assert orc.normal_equation_residual(A, x, B, nrm) <= NER_TOL


def test_3xtf32_factor_reuse_refines(lls):
    p = wl.c3_like(800, 400, 300, nrhs=1, nb=64, q=1)
    ref = orc.solve(p.A, p.B, 1, 64, p.tol, 2001)
    h = lls.lls_create(nb=64, q=1, seed=2001, precision=lls.LLS_MIXED_BF16_3xTF32, max_refine=10,
                       refine_tol=1e-11)
    try:
        fid, rank, _ = lls.lls_factor(h, dev(p.A), p.tol)
        assert rank == 300
        for _ in range(2):
            X = host(lls.lls_solve_factored(h, fid, dev(p.B), 400))
            assert rel(X, ref.x) <= X_TOL
        steps, _ = lls.lls_refinement_info(h)
        assert steps >= 2
    finally:
        lls.lls_destroy(h)


def test_plain_tf32_solves_a_wide_gap_matrix(lls):
    """Kept singular values above 1e-2 ||A|| and tol = 1e-2 ||A||: the
    2^-11 noise stays below tol, and refinement recovers x."""
    A, X, Y = wl.lowrank_xy(2000, 1000, 400, seed=1001, noise=1e-14)
    B = np.random.default_rng(1101).standard_normal((2000, 1))
    nrm = wl.norm2_of_product(X, Y)
    tol = 1e-2 * nrm
    ref = orc.solve(A, B, 1, 64, tol, 2001)
    assert ref.rank == 400
    x, rank, code, _ = solve(lls, A, B, tol, 64, 1, lls.LLS_MIXED_BF16_TF32, max_refine=16)
    assert rank == 400 and code in (lls.LLS_OK, lls.LLS_WARN_REFINE_NOCONV)
    assert rel(x, ref.x) <= X_TOL


def test_plain_tf32_fails_on_the_geometric_spectrum(lls):
    """sigma down to 1e-4 ||A|| with tol = 1e-6 ||A||: plain TF32 updates
    leave noise of about 1e-4 ||A|| in the trailing matrix, so the rank is
    not the oracle's (3xTF32 and the exact-slice mode reveal it)."""
    p = wl.c3_like(1024, 512, 384, nrhs=1, nb=32, q=1)
    _, rank, _, _ = solve(lls, p.A, p.B, p.tol, 32, 1, lls.LLS_MIXED_BF16_TF32)
    assert rank != 384
