"""Guard-word debug mode (lls_debug_guard): the machinery detects a write just
past either end of a guarded buffer (written with cudaMemset inside the
allocation, so nothing faults), and the solver's kernels leave every guard
intact on small odd shapes in both precision modes, with Nullify, an
explicit V, refinement, factor reuse and the batched worker pool, while
their results stay at parity with the oracle."""

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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_guard_selftest(lls):
    assert lls.lls_debug_guard_selftest() == lls.LLS_OK


@pytest.fixture
def guarded(lls):
    lls.lls_debug_guard(True)
    try:
        yield
    finally:
        lls.lls_debug_guard(False)


CASES = [  # m, n, r, nb, q, nullify, precision, explicit_v, max_refine, nrhs
    (333, 201, 77, 32, 1, 0, 0, 0, 0, 3),
    (201, 333, 77, 48, 0, 1, 0, 1, 1, 2),
    (257, 129, 129, 64, 2, 1, 0, 0, 1, 1),
    (390, 260, 90, 64, 1, 1, 1, 0, 0, 2),
    (260, 390, 100, 37, 1, 1, 1, 1, 1, 1),
    (97, 97, 1, 16, 1, 1, 1, 1, 0, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_solver_leaves_guards_intact(lls, guarded, case):
    m, n, r, nb, q, nullify, precision, explicit_v, max_refine, nrhs = case
    A, X, Y = wl.lowrank_xy(m, n, r, seed=m + 7 * n + r, noise=1e-14)
    B = np.random.default_rng(r).standard_normal((m, nrhs))
    nrm = wl.norm2_of_product(X, Y)
    tol = 1e-10 * nrm
    ref = orc.solve(A, B, q, nb, tol, 2001, do_nullify=bool(nullify))
    h = lls.lls_create(nb=nb, q=q, seed=2001, nullify=nullify, precision=precision,
                       explicit_v=explicit_v, max_refine=max_refine)
    try:
        dA, dB = dev(A), dev(B)
        Xs, rank, code = lls.lls_solve(h, dA, dB, tol)
        assert code >= 0 and rank == ref.rank == r
        assert rel(Xs.cpu().numpy(), np.reshape(ref.x, (n, nrhs))) <= 1e-9
        fid, _, _ = lls.lls_factor(h, dA, tol)
        Xf = lls.lls_solve_factored(h, fid, dB, n)
        assert rel(Xf.cpu().numpy(), Xs.cpu().numpy()) <= 1e-12
        lls.lls_factor_release(h, fid)
    finally:
        lls.lls_destroy(h)
    count, first = lls.lls_debug_guard_report()
    assert count == 0, first


def test_batched_pool_leaves_guards_intact(lls, guarded):
    shapes = [(300, 200, 60, 3), (150, 260, 40, 1), (400, 400, 120, 2), (129, 65, 65, 1)]
    h = lls.lls_create(nb=32, q=1, seed=2001, explicit_v=1, max_refine=1)
    try:
        lls.lls_set_workers(h, 3)
        keep, plist, refs = [], [], []
        for i, (m, n, r, k) in enumerate(shapes):
            A, X, Y = wl.lowrank_xy(m, n, r, seed=100 + i, noise=1e-14)
            B = np.random.default_rng(i).standard_normal((m, k))
            tol = 1e-10 * wl.norm2_of_product(X, Y)
            dA, dB = dev(A), dev(B)
            Xo = lls.empty_colmajor(n, k)
            keep += [dA, dB, Xo]
            plist.append(lls.make_problem(dA, dB, tol, Xo))
            refs.append(orc.solve(A, B, 1, 32, tol, 2001).x)
        assert lls.lls_solve_batched(h, plist) >= 0
        for i, p in enumerate(plist):
            assert p.status >= 0
            assert rel(keep[3 * i + 2].cpu().numpy(), refs[i]) <= 1e-9
    finally:
        lls.lls_destroy(h)
    count, first = lls.lls_debug_guard_report()
    assert count == 0, first
