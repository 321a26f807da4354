"""Full-size parity on the bench workload (16384^2, rank 8192, nrhs = 16,
nb = 128, q = 2), in the launch configuration bench.py times.  The oracle
cannot factor this matrix in test time, so the solution is checked against
the truncated-SVD solution built from the known factors of the construction
(the oracle's pinv_solve_from_factors), with the rank equal to the
construction's and the FP64 normal-equation residual <= 1e-13 -- for the
FP64 path and for the mixed-precision path."""

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
