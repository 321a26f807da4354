"""Out-of-core solve (lls_solve_ooc): the matrix in host memory, at most a
few column panels of it on the device, moved by the latest-in-the-future or
LRU schedule.  Same sketch and arithmetic as the in-core solve, so: rank
equal to the oracle's, x within 1e-9 of the oracle's and within 1e-10 of
lls_solve's, normal-equation residual <= 1e-13."""

import numpy as np
import pytest
import torch

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FAR, LRU = 0, 1


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m,n,r,nb,q,nullify,cache,policy", [
    (150, 100, 40, 16, 1, 1, 3, FAR),     # tall; D starts inside the last block's panel
    (100, 150, 40, 16, 1, 1, 2, LRU),     # wide: a narrow last step inside its panel
    (120, 120, 48, 16, 2, 1, 4, FAR),     # r a multiple of nb; q = 2
    (110, 90, 30, 16, 3, 1, 3, LRU),      # q = 3: two fused sampling passes in a row
    (90, 60, 60, 13, 0, 1, 2, FAR),       # full column rank: no Nullify; q = 0
    (80, 70, 25, 8, 1, 0, 3, LRU),        # the fast option
    (64, 64, 1, 8, 1, 1, 1, FAR),         # rank 1, a cache of one panel
    (300, 200, 64, 32, 1, 1, 100, FAR),   # everything fits
])
def test_ooc_matches_oracle_and_in_core(lls, m, n, r, nb, q, nullify, cache, policy):
    A, X, Y = wl.lowrank_xy(m, n, r, seed=m + 3 * n + r, noise=1e-14)
    B = np.random.default_rng(r).standard_normal((m, 2))
    nrm = wl.norm2_of_product(X, Y)
    tol = 1e-10 * nrm
    ref = orc.solve(A, B, q, nb, tol, 2001, do_nullify=bool(nullify))
    h = lls.lls_create(nb=nb, q=q, seed=2001, nullify=nullify)
    try:
        x, rank, code = lls.lls_solve_ooc(h, A, B, tol, cache, policy)
        dA = torch.as_tensor(np.asfortranarray(A), device="cuda").t().contiguous().t()
        dB = torch.as_tensor(np.asfortranarray(B), device="cuda").t().contiguous().t()
        xi, rank_i, _ = lls.lls_solve(h, dA, dB, tol)
    finally:
        lls.lls_destroy(h)
    assert code == 0 and rank == ref.rank == rank_i == r
    assert rel(x, ref.x) <= 1e-9
    assert rel(x, xi.cpu().numpy()) <= 1e-10
    assert orc.normal_equation_residual(A, x, B, nrm) <= 1e-13


def test_ooc_argument_and_input_errors(lls):
    A, _, _ = wl.lowrank_xy(40, 30, 10, seed=1)
    B = np.ones((40, 1))
    h = lls.lls_create(nb=8, q=1)
    try:
        with pytest.raises(lls.LLSError) as e:
            lls.lls_solve_ooc(h, A, B, 1e-8, 0)
        assert e.value.status == lls.LLS_ERR_ARG and e.value.arg == 13
        with pytest.raises(lls.LLSError) as e:
            lls.lls_solve_ooc(h, A, B, 1e-8, 2, policy=9)
        assert e.value.arg == 14
        bad = A.copy()
        bad[3, 4] = np.nan
        with pytest.raises(lls.LLSError) as e:
            lls.lls_solve_ooc(h, bad, B, 1e-8, 2)
        assert e.value.status == lls.LLS_ERR_NONFINITE
        lls.lls_set_options(h, nb=8, q=1, precision=lls.LLS_MIXED_BF16)
        with pytest.raises(lls.LLSError) as e:
            lls.lls_solve_ooc(h, A, B, 1e-8, 2)
        assert e.value.status == lls.LLS_ERR_ARG and e.value.arg == 1
    finally:
        lls.lls_destroy(h)
