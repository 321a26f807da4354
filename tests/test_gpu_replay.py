"""Replays of the stored reflectors (c = U^T b and x = V z of Fig. 4, and
the refinement's operators) with at most four right-hand sides run as one
cooperative launch per replay (replay_kernel) on factors whose larger side
has at least 4096 rows and whose leading dimension is even (the reflector
chunks are TMA tensor loads); five or more right-hand sides, smaller factors
or an odd leading dimension take the per-step kernels.  The choice depends on
the shape alone, so batched and served solves keep giving the same bits as
solves alone.
Checked here: x against the FP64 oracle for 1..4 right-hand sides and
several block sizes (ragged last step included), agreement with the
per-step path on the same factor, one launch per replay in the trace,
bit-identical repeats, and a grid-barrier timeout reported as
LLS_ERR_TIMEOUT with the handle still usable afterwards (the wait runs out
because the poll limit is lowered to zero: nothing faults or hangs)."""

import numpy as np
import pytest
import torch

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("m,n,r,nb", [(4096, 1000, 400, 64), (4200, 1500, 1100, 128),
                                      (900, 4100, 500, 96), (6000, 200, 200, 48),
                                      (4097, 500, 300, 64), (2000, 1000, 400, 64)])
def test_replay_against_oracle_and_per_step_path(lls, m, n, r, nb):
    A, X, Y = wl.lowrank_xy(m, n, r, seed=m + n + r, noise=1e-14)
    nrm = wl.norm2_of_product(X, Y)
    tol = 1e-10 * nrm
    B = np.random.default_rng(nb).standard_normal((m, 5))
    ref = orc.solve(A, B, 1, nb, tol, 2001)
    assert ref.rank == r
    h = lls.lls_create(nb=nb, q=1, seed=2001)
    try:
        fid, rank, _ = lls.lls_factor(h, dev(A), tol)
        assert rank == r
        x5 = host(lls.lls_solve_factored(h, fid, dev(B), n))        # per-step kernels
        assert rel(x5, ref.x) <= 1e-9
        for nrhs in (1, 2, 3, 4):
            lls.lls_trace_enable(h, True)
            x = host(lls.lls_solve_factored(h, fid, dev(B[:, :nrhs]), n))
            tr = lls.lls_trace_read(h)
            lls.lls_trace_enable(h, False)
            # U^T and V one launch each on a factor with 4096 rows or columns; an
            # odd leading dimension (no TMA map: 16-byte rows) keeps the
            # per-step kernels for that side, and so does a smaller factor
            want = (m % 2 == 0) + (n % 2 == 0) if max(m, n) >= 4096 else 0
            assert tr.get("replay_kernel", (0,))[0] == want
            assert rel(x, ref.x[:, :nrhs]) <= 1e-9
            assert np.max(np.abs(x - x5[:, :nrhs])) <= 1e-12 * np.max(np.abs(x5))
        assert orc.normal_equation_residual(A, x, B[:, :4], nrm) <= 1e-13
    finally:
        lls.lls_destroy(h)


def test_replay_repeats_are_bit_identical(lls):
    A, X, Y = wl.lowrank_xy(4096, 1024, 700, seed=41, noise=1e-14)
    B = np.random.default_rng(42).standard_normal((4096, 3))
    tol = 1e-10 * wl.norm2_of_product(X, Y)
    h = lls.lls_create(nb=128, q=1, seed=2001)
    try:
        fid, _, _ = lls.lls_factor(h, dev(A), tol)
        lls.lls_trace_enable(h, True)
        a = host(lls.lls_solve_factored(h, fid, dev(B), 1024))
        assert lls.lls_trace_read(h)["replay_kernel"][0] == 2
        b = host(lls.lls_solve_factored(h, fid, dev(B), 1024))
        assert np.array_equal(a, b)
    finally:
        lls.lls_destroy(h)


def test_3xtf32_refinement_replays_in_one_launch_each(lls):
    p = wl.c3_like(4096, 1024, 768, nrhs=2, nb=64, q=1)
    ref = orc.solve(p.A, p.B, 1, 64, p.tol, 2001)
    h = lls.lls_create(nb=64, q=1, seed=2001, precision=lls.LLS_MIXED_BF16_3xTF32, max_refine=10,
                       refine_tol=1e-11)
    try:
        lls.lls_trace_enable(h, True)
        X, rank, code = lls.lls_solve(h, dev(p.A), dev(p.B), p.tol)
        tr = lls.lls_trace_read(h)
        steps, _ = lls.lls_refinement_info(h)
    finally:
        lls.lls_destroy(h)
    assert code == lls.LLS_OK and rank == 768
    assert rel(host(X), ref.x) <= 1e-9
    # the solve's two replays, then two per refinement iteration (V^T, V or
    # U^T, U); an iteration whose correction grew is undone and not counted
    launches = tr["replay_kernel"][0]
    assert launches >= 2 + 2 * steps and launches % 2 == 0


def test_replay_barrier_timeout_is_reported_and_the_handle_recovers(lls):
    m, n, r, nb = 4096, 1024, 700, 128
    A, X, Y = wl.lowrank_xy(m, n, r, seed=77, noise=1e-14)
    nrm = wl.norm2_of_product(X, Y)
    tol = 1e-10 * nrm
    B = np.random.default_rng(78).standard_normal((m, 2))
    h = lls.lls_create(nb=nb, q=1, seed=2001)
    try:
        fid, rank, _ = lls.lls_factor(h, dev(A), tol)
        assert rank == r
        lls.lls_debug_barrier_limit(0)
        try:
            with pytest.raises(lls.LLSError) as e:
                lls.lls_solve_factored(h, fid, dev(B), n)
            assert e.value.status == lls.LLS_ERR_TIMEOUT
        finally:
            lls.lls_debug_barrier_limit(-1)
        x = host(lls.lls_solve_factored(h, fid, dev(B), n))
        ref = orc.solve(A, B, 1, nb, tol, 2001)
        assert rel(x, ref.x) <= 1e-9
    finally:
        lls.lls_destroy(h)
