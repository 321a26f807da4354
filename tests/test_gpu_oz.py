"""FP64 GEMM on the tensor cores by exact BF16 slicing (lls_k_gemm_oz)
against plain FP64 products: integer inputs give exact results, and random
inputs with rows and columns spread over many orders of magnitude agree
with the FP64 product to FP64 rounding relative to the row/column scales."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.asfortranarray(x), dtype=torch.float64, device="cuda").t().contiguous().t()


def host(t):
    return t.detach().cpu().numpy()


def scaled_err(got, ref, A, B):
    # |error| relative to max_k |A_ik| * max_k |B_kj| * K
    ra = np.abs(A).max(axis=1)[:, None]
    cb = np.abs(B).max(axis=0)[None, :]
    K = A.shape[1]
    return np.max(np.abs(got - ref) / (ra * cb * K + 1e-300))


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (130, 70, 200), (300, 129, 1000), (128, 64, 256),
                                   (257, 65, 4097), (1030, 515, 777)])
def test_oz_gemm_matches_fp64(lls, ta, tb, m, n, k):
    g = np.random.default_rng(m + 3 * n + 7 * k + ta + 2 * tb)
    A = g.standard_normal((m, k)) * 10.0 ** g.uniform(-8, 8, (m, 1))
    B = g.standard_normal((k, n)) * 10.0 ** g.uniform(-8, 8, (1, n))
    got, st = lls.lls_k_gemm_oz(ta, tb, dev(A.T if ta else A), dev(B.T if tb else B))
    assert st == 0
    err = scaled_err(host(got), A @ B, A, B)
    assert err < 2e-16, err


def test_oz_gemm_rank_update_many_items(lls):
    """The randUTV update shape C -= P W^T with more 128 x 128 items than
    SMs, so every CTA of the persistent grid runs several items through
    both passes and the operand rings wrap many times."""
    g = np.random.default_rng(12)
    P, W, C0 = g.standard_normal((2304, 128)), g.standard_normal((2200, 128)), g.standard_normal((2304, 2200))
    got, st = lls.lls_k_gemm_oz(0, 1, dev(P), dev(W), dev(C0), alpha=-1.0, beta=1.0)
    assert st == 0
    assert np.max(np.abs(host(got) - (C0 - P @ W.T))) < 1e-12


def test_oz_gemm_alpha_beta(lls):
    g = np.random.default_rng(11)
    A, B, C0 = g.standard_normal((150, 300)), g.standard_normal((300, 80)), g.standard_normal((150, 80))
    got, st = lls.lls_k_gemm_oz(0, 0, dev(A), dev(B), dev(C0), alpha=-0.5, beta=2.0)
    ref = 2.0 * C0 - 0.5 * (A @ B)
    assert st == 0
    assert np.max(np.abs(host(got) - ref)) < 1e-13


def test_oz_gemm_integer_inputs_are_exact(lls):
    g = np.random.default_rng(5)
    A = g.integers(-1000, 1001, (200, 300)).astype(np.float64)
    B = g.integers(-1000, 1001, (300, 90)).astype(np.float64)
    got, st = lls.lls_k_gemm_oz(0, 0, dev(A), dev(B))
    assert st == 0
    assert np.array_equal(host(got), A @ B)


def test_oz_gemm_unit_lower_and_zero_rows(lls):
    g = np.random.default_rng(6)
    W = g.standard_normal((400, 64))
    Wl = np.tril(W, -1)
    Wl[np.arange(64), np.arange(64)] = 1.0
    X = g.standard_normal((400, 33))
    X[:, 5] = 0.0
    got, st = lls.lls_k_gemm_oz(1, 0, dev(W), dev(X), unit_lower_a=True)
    ref = Wl.T @ X
    assert st == 0
    assert scaled_err(host(got), ref, Wl.T, X) < 2e-16
    assert np.all(host(got)[:, 5] == 0.0)
