"""Kernel-level parity: each CUDA step launcher against the oracle's routine
for the same step (or a plain FP64 definition), element by element."""

import numpy as np
import pytest
import torch

from oracle import randutv_oracle as orc

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.asfortranarray(x), dtype=torch.float64, device="cuda").t().contiguous().t()


def host(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------ a1 sketch
@pytest.mark.parametrize("seed,step,groups,cols", [(2001, 0, 37, 5), (7, 12, 4096, 3), (2**63 + 5, 127, 1, 1)])
def test_philox_words_bit_exact(lls, seed, step, groups, cols):
    got = host(lls.lls_k_philox(seed, step, groups, cols)).view(np.uint64).reshape(cols, groups, 4)
    g, j = np.meshgrid(np.arange(groups, dtype=np.uint64), np.arange(cols, dtype=np.uint64), indexing="ij")
    want = orc.philox4x64_10((g, j, np.uint64(step), np.uint64(0)), (seed, 0))
    for w in range(4):
        assert np.array_equal(got[:, :, w], want[w].T)


@pytest.mark.parametrize("rows,cols,step", [(2000, 64, 0), (1003, 7, 5), (3, 1, 2), (16384, 128, 1)])
def test_sketch_matches_oracle(lls, rows, cols, step):
    G = host(lls.lls_k_sketch(2002, step, rows, cols))
    ref = orc.sketch_matrix(2002, step, rows, cols)
    # same integer stream; log / cos / sin differ in the last bits between libm and CUDA
    assert np.max(np.abs(G - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


# ------------------------------------------------------------------- GEMM
@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (67, 45, 33), (130, 129, 4000), (64, 64, 16),
                                   (300, 16, 5000), (5000, 3, 128), (129, 9, 777), (128, 16, 20000)])
def test_gemm_all_transposes(lls, ta, tb, m, n, k):
    g = np.random.default_rng(m * 7 + n + k)
    A = g.standard_normal((k, m) if ta else (m, k))
    B = g.standard_normal((n, k) if tb else (k, n))
    C0 = g.standard_normal((m, n))
    got = host(lls.lls_k_gemm(ta, tb, dev(A), dev(B), dev(C0), alpha=-0.5, beta=2.0))
    ref = -0.5 * (A.T if ta else A) @ (B.T if tb else B) + 2.0 * C0
    assert np.allclose(got, ref, rtol=0, atol=1e-13 * np.sqrt(k) * np.abs(ref).max())


def test_gemm_split_k_is_deterministic(lls):
    g = np.random.default_rng(1)
    A = g.standard_normal((20000, 128))
    Gm = g.standard_normal((20000, 96))
    a, b = dev(A), dev(Gm)
    r1 = host(lls.lls_k_gemm(1, 0, a, b))
    r2 = host(lls.lls_k_gemm(1, 0, a, b))
    assert np.array_equal(r1, r2)
    assert np.allclose(r1, A.T @ Gm, rtol=0, atol=1e-12 * np.abs(A.T @ Gm).max())
    # narrow outputs (n <= 16) take their own tile and a deeper split
    Bn = Gm[:, :16]
    n1 = host(lls.lls_k_gemm(1, 0, a, dev(Bn)))
    n2 = host(lls.lls_k_gemm(1, 0, a, dev(Bn)))
    assert np.array_equal(n1, n2)
    assert np.allclose(n1, A.T @ Bn, rtol=0, atol=1e-12 * np.abs(A.T @ Bn).max())


@pytest.mark.parametrize("ta", [0, 1])
def test_gemm_unit_lower_operands(lls, ta):
    g = np.random.default_rng(5)
    W = g.standard_normal((90, 40))          # stored matrix, read as unit lower trapezoidal
    Wl = np.tril(W, -1)
    Wl[np.arange(40), np.arange(40)] = 1.0
    X = g.standard_normal((90 if ta else 40, 17))
    got = host(lls.lls_k_gemm(ta, 0, dev(W), dev(X), unit_lower_a=True))
    ref = (Wl.T if ta else Wl) @ X
    assert np.allclose(got, ref, atol=1e-13 * np.abs(ref).max())
    Y = g.standard_normal((23, 40))
    got = host(lls.lls_k_gemm(0, 1, dev(Y), dev(W), unit_lower_b=True))
    assert np.allclose(got, Y @ Wl.T, atol=1e-13 * np.abs(Y @ Wl.T).max())


# -------------------------------------------------------------- a3/a5 panel QR
# (300, 128), (129, 7), (8, 12): one thread-block cluster; (2000, 64) to
# (30000, 128): the cooperative shared-memory (slab) kernel, odd and ragged
# slabs included; (40000, 128): slabs too tall for shared memory, the
# cooperative global-memory kernel
@pytest.mark.parametrize("m,n", [(2000, 64), (129, 7), (300, 128), (16384, 128), (40000, 128),
                                 (8, 12), (5000, 1), (7001, 128), (2049, 37), (30000, 128)])
def test_panel_qr_matches_oracle(lls, m, n):
    Y = np.random.default_rng(m + n).standard_normal((m, n))
    A, tau, T = lls.lls_k_geqrf(dev(Y))
    A, tau, T = host(A), host(tau), host(T)
    R_ref, W_ref, tau_ref = orc.householder_qr(Y)
    k = min(m, n)
    scale = np.abs(Y).max()
    assert np.allclose(np.triu(A[:k]), R_ref, rtol=0, atol=1e-13 * scale * np.sqrt(m))
    assert np.allclose(tau, tau_ref, rtol=0, atol=1e-13)
    W = np.tril(A[:, :k], -1)
    W[np.arange(k), np.arange(k)] = 1.0
    assert np.allclose(W, W_ref, rtol=0, atol=1e-12)
    assert np.allclose(T, orc.wy_factor(W_ref, tau_ref), rtol=0, atol=1e-12 * max(1, np.abs(T).max()))


@pytest.mark.parametrize("m", [500, 9000])
def test_panel_qr_zero_and_rank_deficient_columns(lls, m):
    """A zero column gives tau = 0 on both sides; after a dependent column the
    trailing rows of R are not unique (the reflector is built from rounding
    noise), so rows before it are compared and the rest is checked for
    validity: Q R = Y with Q = I - W T W^T orthogonal."""
    g = np.random.default_rng(3)
    Y = g.standard_normal((m, 10))
    Y[:, 3] = 0.0
    Y[:, 6] = Y[:, 1] * 2.0
    A, tau, T = lls.lls_k_geqrf(dev(Y))
    A, tau, T = host(A), host(tau), host(T)
    R_ref, _, tau_ref = orc.householder_qr(Y)
    R = np.triu(A[:10])
    assert np.allclose(R[:6], R_ref[:6], atol=1e-12)
    assert np.allclose(tau[:6], tau_ref[:6], atol=1e-13) and tau[3] == 0.0
    assert abs(R[6, 6]) < 1e-12
    W = np.tril(A, -1)[:, :10]
    W[np.arange(10), np.arange(10)] = 1.0
    Q = np.eye(m) - W @ T @ W.T
    assert np.allclose(Q.T @ Q, np.eye(m), atol=1e-13)
    assert np.allclose(Q[:, :10] @ R, Y, atol=1e-12)


# ------------------------------------------------------------------ a7 SVD
@pytest.mark.parametrize("b", [1, 2, 3, 17, 33, 64, 97, 127, 128])
def test_jacobi_svd(lls, b):
    # b < 32: one CTA; 32 <= b <= 64: a cluster of 4 CTAs; b > 64: a cluster of 8
    # (odd b leaves a padding column in the round-robin order)
    g = np.random.default_rng(b)
    R = np.triu(g.standard_normal((b, b))) @ np.diag(np.logspace(0, -10, b))
    sigma, Us, Vs, status = lls.lls_k_jacobi_svd(dev(R))
    sigma, Us, Vs = host(sigma), host(Us), host(Vs)
    assert status == 0
    ref = np.linalg.svd(R, compute_uv=False)
    assert np.all(np.diff(sigma) <= 0)
    assert np.allclose(sigma, ref, rtol=0, atol=1e-14 * ref[0] * b)
    assert np.allclose(Us.T @ Us, np.eye(b), atol=1e-13)
    assert np.allclose(Vs.T @ Vs, np.eye(b), atol=1e-13)
    assert np.allclose(Us @ np.diag(sigma) @ Vs.T, np.triu(R), atol=1e-13 * ref[0])


@pytest.mark.parametrize("b", [12, 70])
def test_jacobi_svd_singular_block_completes_u(lls, b):
    R = np.triu(np.random.default_rng(1).standard_normal((b, b)))
    R[:, [2, 5, 9]] = 0.0
    R[[4, 7], :] = 0.0
    sigma, Us, Vs, status = lls.lls_k_jacobi_svd(dev(R))
    Us, Vs, sigma = host(Us), host(Vs), host(sigma)
    assert status == 0
    assert np.allclose(Us.T @ Us, np.eye(b), atol=1e-13)
    assert np.allclose(Us @ np.diag(sigma) @ Vs.T, R, atol=1e-13 * np.abs(R).max())
    assert np.allclose(sigma, np.linalg.svd(R, compute_uv=False), atol=1e-13)


# -------------------------------------------------------------- a8 rank, a10 TRSM
def test_rank_scan(lls):
    T = np.diag([5.0, 3.0, 1e-12, 2.0, 1e-13, 0.0])
    assert lls.lls_k_rank(dev(T), 1e-10) == (2, 3, 0)
    assert lls.lls_k_rank(dev(np.diag([1.0, 1e-10])), 1e-10) == (1, 1, 0)
    big = np.zeros((3000, 2500))
    big[np.arange(2500), np.arange(2500)] = np.r_[np.ones(2400), np.zeros(100)]
    assert lls.lls_k_rank(dev(big), 0.5) == (2400, 2400, 0)


@pytest.mark.parametrize("r,nrhs", [(1, 1), (63, 3), (200, 16), (1000, 5)])
def test_trsm_upper(lls, r, nrhs):
    g = np.random.default_rng(r)
    R = np.triu(g.standard_normal((r, r))) + r * np.eye(r)
    Rfull = R + np.tril(g.standard_normal((r, r)), -1)   # lower garbage must be ignored
    B = g.standard_normal((r, nrhs))
    got = host(lls.lls_k_trsm_upper(dev(Rfull), dev(B)))
    assert np.allclose(got, np.linalg.solve(R, B), rtol=1e-12, atol=1e-13)
