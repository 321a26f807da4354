"""Mixed precision (sampling products in BF16 on tcgen05 tensor cores):
the tensor-core GEMM against a plain PyTorch FP32 product of the same BF16
inputs, and the whole solve against the FP64 oracle (rank equal, x within
1e-9): the sample only chooses V, T = U^T A V stays FP64."""

import numpy as np
import pytest
import torch

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def bf16_colmajor(K, M, seed, pad=0):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    ld = K + pad
    buf = torch.randn((M, ld), generator=g, device="cuda").to(torch.bfloat16)
    return buf.t()[:K]            # K x M view, column-major with leading dimension ld


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 64, 1000), (16384, 128, 16384),
                                   (1000, 40, 4100), (129, 16, 8), (2049, 96, 777)])
def test_tc_gemm_matches_fp32_reference(lls, M, N, K):
    X = bf16_colmajor(K, M, 1, pad=(8 - K % 8) % 8)
    Z = bf16_colmajor(K, N, 2, pad=(8 - K % 8) % 8)
    D, status = lls.lls_k_gemm_bf16_tn(X, Z)
    torch.cuda.synchronize()
    assert status == 0
    ref = X.float().t() @ Z.float()
    scale = (X.float().abs().t() @ Z.float().abs()).max().item()
    err = (D - ref).abs().max().item()
    assert err <= 1e-5 * scale, (err, scale)


def dev(x):
    return torch.as_tensor(np.asfortranarray(x), dtype=torch.float64, device="cuda").t().contiguous().t()


def solve_mixed(lls, A, B, tol, nb, q, seed):
    h = lls.lls_create(nb=nb, q=q, seed=seed, precision=lls.LLS_MIXED_BF16)
    try:
        X, rank, code = lls.lls_solve(h, dev(A), dev(np.reshape(B, (A.shape[0], -1))), tol)
        return X.cpu().numpy(), rank, code
    finally:
        lls.lls_destroy(h)


@pytest.mark.parametrize("case", ["c1", "c2_1024", "c3_1024", "wide"])
def test_mixed_solve_matches_fp64_oracle(lls, case):
    if case == "c1":
        p = wl.c1_problem()
        A, B, tol, nb, q, nrm, r = p.A, p.B, p.tol, p.nb, p.q, p.norm2, 400
    elif case == "c2_1024":
        p = wl.c2_like(1024)
        A, B, tol, nb, q, nrm, r = p.A, p.B, p.tol, p.nb, p.q, 1.0, 512
    elif case == "c3_1024":
        p = wl.c3_like(1024, 512, 384, nb=64)
        A, B, tol, nb, q, nrm, r = p.A, p.B, p.tol, p.nb, p.q, 1.0, 384
    else:
        A, X, Y = wl.lowrank_xy(300, 700, 120, seed=5, noise=1e-14)
        B = np.random.default_rng(1).standard_normal((300, 2))
        nrm = wl.norm2_of_product(X, Y)
        tol, nb, q, r = 1e-10 * nrm, 32, 1, 120
    x, rank, code = solve_mixed(lls, A, B, tol, nb, q, 2001)
    ref = orc.solve(A, B, q, nb, tol, 2001)
    assert code == 0 and rank == ref.rank == r
    xr = np.reshape(ref.x, x.shape)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-9
    assert orc.normal_equation_residual(A, x, B, nrm) <= 1e-13
