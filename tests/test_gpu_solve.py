"""End-to-end parity of lls_solve (C ABI) with the oracle's Fig. 4 solve:
same sketch seed, rank equal to the oracle's, x within 1e-9 relative, and the
FP64 normal-equation residual <= 1e-13 (||A^T (b - A x)|| / (||A||_2
(||A||_2 ||x|| + ||b||)))."""

import numpy as np
import pytest
import torch

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

pytestmark = pytest.mark.gpu

X_TOL = 1e-9
NER_TOL = 1e-13


def dev(x):
    return torch.as_tensor(np.asfortranarray(x), dtype=torch.float64, device="cuda").t().contiguous().t()


def run(lls, A, B, tol, nb, q, seed, nullify=1, precision=0):
    h = lls.lls_create(nb=nb, q=q, seed=seed, nullify=nullify, precision=precision)
    try:
        X, rank, code = lls.lls_solve(h, dev(A), dev(np.reshape(B, (A.shape[0], -1))), tol)
        return X.cpu().numpy(), rank, code
    finally:
        lls.lls_destroy(h)


def check(lls, A, B, tol, nb, q, seed, norm2, nullify=1, rank_expected=None):
    x, rank, code = run(lls, A, B, tol, nb, q, seed, nullify)
    ref = orc.solve(A, B, q, nb, tol, seed, do_nullify=bool(nullify))
    assert code == 0
    assert rank == ref.rank
    if rank_expected is not None:
        assert rank == rank_expected
    xr = np.reshape(ref.x, x.shape)
    err = np.linalg.norm(x - xr) / max(np.linalg.norm(xr), 1e-300)
    assert err <= X_TOL, err
    assert orc.normal_equation_residual(A, x, B, norm2) <= NER_TOL
    return x, ref


def test_c1_full_size(lls):
    """2000 x 1000, exact rank 400 + 1e-14 noise, nb = 64, q = 1."""
    p = wl.c1_problem()
    check(lls, p.A, p.B, p.tol, p.nb, p.q, 2001, p.norm2, rank_expected=400)


def test_c1_fast_option(lls):
    p = wl.c1_problem()
    x, ref = check(lls, p.A, p.B, p.tol, p.nb, p.q, 2001, p.norm2, nullify=0)
    full = np.reshape(orc.solve(p.A, p.B, p.q, p.nb, p.tol, 2001).x, x.shape)
    assert np.linalg.norm(x - full) / np.linalg.norm(full) < 1e-9


@pytest.mark.parametrize("m,n,r,nb,q,nrhs", [
    (700, 300, 120, 32, 1, 3),     # tall, ragged steps
    (300, 700, 120, 32, 1, 2),     # wide (underdetermined)
    (513, 513, 200, 64, 2, 1),     # square, nb does not divide n
    (260, 100, 100, 128, 1, 4),    # full column rank, one step (nb >= n)
    (400, 257, 77, 37, 0, 1),      # odd block size, q = 0
    (129, 129, 1, 16, 1, 1),       # rank 1
])
def test_shapes_against_oracle(lls, m, n, r, nb, q, nrhs):
    A, X, Y = wl.lowrank_xy(m, n, r, seed=m * n + r, noise=1e-14)
    B = np.random.default_rng(r).standard_normal((m, nrhs))
    nrm = wl.norm2_of_product(X, Y)
    check(lls, A, B, 1e-10 * nrm, nb, q, 2001 + q, nrm, rank_expected=r)


def test_c2_scaled(lls):
    """The 16384^2 construction scaled to n = 1024: Haar factors, sigma from
    1 to 1e-6 over rank n/2 then 1e-15, b = A x0 + 1e-8 noise, nrhs = 16,
    nb = 128, q = 2."""
    p = wl.c2_like(1024)
    check(lls, p.A, p.B, p.tol, p.nb, p.q, 2002, 1.0, rank_expected=512)


def test_c3_scaled_fp64(lls):
    p = wl.c3_like(1024, 512, 384, nb=64)
    check(lls, p.A, p.B, p.tol, p.nb, p.q, 2003, 1.0, rank_expected=384)


def test_zero_matrix_and_empty_shapes(lls):
    x, rank, code = run(lls, np.zeros((50, 30)), np.ones((50, 2)), 0.0, 8, 1, 1)
    assert rank == 0 and code == 0 and np.all(x == 0)
    h = lls.lls_create()
    try:
        for (m, n, k) in [(0, 5, 1), (5, 0, 1), (5, 4, 0)]:
            A = lls.empty_colmajor(m, n)
            B = lls.empty_colmajor(m, k)
            X = torch.full((max(n, 1), max(k, 1)), 7.0, dtype=torch.float64, device="cuda")[:n, :k]
            X = lls.colmajor(X)
            _, rank, code = lls.lls_solve(h, A, B, 0.0, X)
            assert rank == 0 and code == 0
            if m == 0 and n > 0 and k > 0:
                assert torch.all(X == 0)
    finally:
        lls.lls_destroy(h)


def test_nonfinite_input_is_reported(lls):
    A = np.random.default_rng(0).standard_normal((40, 20))
    A[3, 7] = np.nan
    with pytest.raises(lls.LLSError) as e:
        run(lls, A, np.ones(40), 1e-8, 8, 1, 1)
    assert e.value.status == lls.LLS_ERR_NONFINITE
    A[3, 7] = 1.0
    B = np.ones(40)
    B[5] = np.inf
    with pytest.raises(lls.LLSError) as e:
        run(lls, A, B, 1e-8, 8, 1, 1)
    assert e.value.status == lls.LLS_ERR_NONFINITE


def test_argument_errors_name_the_argument(lls):
    h = lls.lls_create()
    try:
        A = lls.empty_colmajor(10, 5)
        B = lls.empty_colmajor(10, 1)
        X = lls.empty_colmajor(5, 1)
        lib = lls._lib
        import ctypes as C
        r = C.c_int64(0)
        code = lib.lls_solve(h, A.data_ptr(), 10, 5, 9, B.data_ptr(), 1, 10, 0.0, X.data_ptr(), 5, C.byref(r))
        assert code == lls.LLS_ERR_ARG
        arg = C.c_int(0)
        lib.lls_last_error(h, C.byref(arg), None, 0)
        assert arg.value == 5          # lda
        code = lib.lls_solve(h, A.data_ptr(), 10, -5, 10, B.data_ptr(), 1, 10, 0.0, X.data_ptr(), 5, C.byref(r))
        assert code == lls.LLS_ERR_ARG
        lib.lls_last_error(h, C.byref(arg), None, 0)
        assert arg.value == 4          # n
    finally:
        lls.lls_destroy(h)


def test_factor_reuse_matches_solve(lls):
    """lls_factor once, lls_solve_factored with two different right-hand
    sides: each equals a fresh lls_solve (the stored-factor variant)."""
    p = wl.c1_problem()
    h = lls.lls_create(nb=64, q=1, seed=2001)
    try:
        fid, rank, _ = lls.lls_factor(h, dev(p.A), p.tol)
        assert rank == 400
        diag, cnt = lls.lls_factor_diag(h, fid, 1000)
        ref = orc.solve(p.A, p.B, 1, 64, p.tol, 2001)
        assert cnt == ref.rank_count
        assert np.allclose(diag[:400], ref.diag[:400], rtol=1e-10)
        for s in (0, 1):
            B = np.random.default_rng(s).standard_normal((2000, 3))
            X = lls.lls_solve_factored(h, fid, dev(B), 1000).cpu().numpy()
            xr = np.reshape(orc.solve(p.A, B, 1, 64, p.tol, 2001).x, X.shape)
            assert np.linalg.norm(X - xr) / np.linalg.norm(xr) < X_TOL
        lls.lls_factor_release(h, fid)
        with pytest.raises(lls.LLSError):
            lls.lls_solve_factored(h, fid, dev(p.B), 1000)
    finally:
        lls.lls_destroy(h)


def test_host_entry_point(lls):
    p = wl.c1_problem()
    h = lls.lls_create(nb=64, q=1, seed=2001)
    try:
        X, rank, code = lls.lls_solve_host(h, p.A, p.B, p.tol)
    finally:
        lls.lls_destroy(h)
    ref = orc.solve(p.A, p.B, 1, 64, p.tol, 2001)
    assert rank == 400
    xr = np.reshape(ref.x, X.shape)
    assert np.linalg.norm(X - xr) / np.linalg.norm(xr) < X_TOL


def test_repeat_solves_are_bit_identical(lls):
    p = wl.c2_like(512, nrhs=2, nb=64)
    a, _, _ = run(lls, p.A, p.B, p.tol, 64, 2, 9)
    b, _, _ = run(lls, p.A, p.B, p.tol, 64, 2, 9)
    assert np.array_equal(a, b)


def test_trace_reports_kernel_families_and_phases(lls):
    from paper_2408_05238_b300 import workloads as wl
    p = wl.c1_problem()
    A = torch.as_tensor(np.asfortranarray(p.A), device="cuda").t().contiguous().t()
    B = torch.as_tensor(np.asfortranarray(p.B), device="cuda").t().contiguous().t()
    h = lls.lls_create(nb=64, q=1, seed=2001)
    try:
        lls.lls_trace_enable(h, True)
        _, rank, _ = lls.lls_solve(h, A, B, p.tol)
        tr = lls.lls_trace_read(h)
    finally:
        lls.lls_destroy(h)
    steps = -(-min(p.A.shape) // 64)
    assert tr["dgemm_kernel"][0] > 0 and tr["panel_qr_kernel"][0] >= 2 * steps
    for ph in ("sample", "qr_y", "right_update", "panel", "left_update"):
        assert tr["phase:" + ph][0] == steps                    # once per step
    for ph in ("block_svd", "rank", "solve"):
        assert tr["phase:" + ph][0] == 1
    assert 0 < rank < p.A.shape[1] and tr["phase:nullify"][0] == 1   # rank 400 of 1000
    fam = sum(v[1] for k, v in tr.items() if not k.startswith("phase:"))
    phases = sum(v[1] for k, v in tr.items() if k.startswith("phase:"))
    assert 0.5 * fam < phases < 2.0 * fam + 0.05             # two views of the same time
