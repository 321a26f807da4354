"""Full-size parity on the bench workloads, in the launch configuration
bench.py times: the 16384^2 matrix (rank 8192, nrhs = 16, nb = 128, q = 2)
in FP64 and mixed precision, and the 32768 x 16384 mixed-precision matrix
(rank 12000, sigma geometric 1 -> 1e-4 then 1e-14, tol 1e-6, nrhs = 1,
nb = 128, q = 1).  The oracle cannot factor these matrices in test time, so
the solution is checked against the truncated-SVD solution built from the
known factors of the construction (the oracle's pinv_solve_from_factors),
with the rank equal to the construction's (a mismatch fails) and the FP64
normal-equation residual <= 1e-13."""

import numpy as np
import pytest
import torch

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 16384


@pytest.fixture(scope="module")
def c2():
    sigma = wl.step_spectrum(N, N // 2, 6.0, 1e-15)
    A, Q1, Q2 = wl.spectrum_matrix_torch(N, N, sigma, seed=1002, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(1102)
    X0 = torch.randn(N, 16, generator=g, dtype=torch.float64, device="cuda")
    noise = torch.randn(N, 16, generator=g, dtype=torch.float64, device="cuda")
    B = (A @ X0 + 1e-8 * noise).t().contiguous().t()
    xref = orc.pinv_solve_from_factors(Q1.cpu().numpy(), sigma, Q2.cpu().numpy(),
                                       B.cpu().numpy(), N // 2)
    del Q1, Q2, X0, noise
    torch.cuda.empty_cache()
    return A, B, xref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c2_full_size(lls, c2, precision):
    A, B, xref = c2
    prec = lls.LLS_MIXED_BF16 if precision == "mixed" else lls.LLS_FP64
    h = lls.lls_create(nb=128, q=2, seed=2002, precision=prec)
    try:
        X, rank, code = lls.lls_solve(h, A, B, 1e-10)
        torch.cuda.synchronize()
    finally:
        lls.lls_destroy(h)
    assert code == 0 and rank == N // 2
    x = X.cpu().numpy()
    assert np.linalg.norm(x - xref) / np.linalg.norm(xref) <= 1e-9
    res = (A.t() @ (B - A @ X)).cpu().numpy()         # ||A||_2 = 1
    ner = max(np.linalg.norm(res[:, j]) / (np.linalg.norm(x[:, j]) + np.linalg.norm(B[:, j].cpu().numpy()))
              for j in range(16))
    assert ner <= 1e-13


M3, N3, R3 = 2 * N, N, 12000


@pytest.fixture(scope="module")
def c3():
    sigma = wl.geometric_spectrum(N3, R3, 1e-4, 1e-14)
    A, Q1, Q2 = wl.spectrum_matrix_torch(M3, N3, sigma, seed=1003, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(1103)
    X0 = torch.randn(N3, 1, generator=g, dtype=torch.float64, device="cuda")
    noise = torch.randn(M3, 1, generator=g, dtype=torch.float64, device="cuda")
    B = (A @ X0 + 1e-8 * noise).t().contiguous().t()
    xref = orc.pinv_solve_from_factors(Q1.cpu().numpy(), sigma, Q2.cpu().numpy(),
                                       B.cpu().numpy(), R3)
    del Q1, Q2, X0, noise
    torch.cuda.empty_cache()
    return A, B, xref


@pytest.mark.parametrize("precision", ["mixed", "3xtf32"])
def test_c3_full_size(lls, c3, precision):
    """Exact-slice updates, and 3xTF32 updates with the minimum-norm
    refinement (at most 10 steps)."""
    A, B, xref = c3
    prec = {"mixed": lls.LLS_MIXED_BF16, "3xtf32": lls.LLS_MIXED_BF16_3xTF32}[precision]
    h = lls.lls_create(nb=128, q=1, seed=2003, precision=prec,
                       max_refine=10 if precision == "3xtf32" else 0, refine_tol=1e-11)
    try:
        X, rank, code = lls.lls_solve(h, A, B, 1e-6)
        torch.cuda.synchronize()
    finally:
        lls.lls_destroy(h)
    assert code == 0 and rank == R3
    x = X.cpu().numpy()
    assert np.linalg.norm(x - xref) / np.linalg.norm(xref) <= 1e-9
    res = (A.t() @ (B - A @ X)).cpu().numpy()         # ||A||_2 = 1
    ner = np.linalg.norm(res) / (np.linalg.norm(x) + np.linalg.norm(B.cpu().numpy()))
    assert ner <= 1e-13
