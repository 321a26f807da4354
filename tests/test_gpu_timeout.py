"""Failure detection without a GPU fault: every wait of the cooperative panel
kernels at their grid barrier is bounded, and a wait that runs out makes the
kernel exit and the call return LLS_ERR_TIMEOUT, with the context and the
handle still usable.  The test lowers the poll limit (lls_debug_barrier_limit)
to zero, so any CTA that does not pass the barrier at once gives up; nothing
faults, traps or hangs.  Panels of 8192 and 16384 rows take the cooperative
shared-memory kernel (smaller ones run on one thread-block cluster, which
has no grid barrier)."""

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


def test_panel_barrier_timeout_is_reported_by_the_step_entry_point(lls):
    Y = np.random.default_rng(11).standard_normal((16384, 128))
    lls.lls_debug_barrier_limit(0)
    try:
        with pytest.raises(lls.LLSError) as e:
            lls.lls_k_geqrf(dev(Y))
        assert e.value.status == lls.LLS_ERR_TIMEOUT
    finally:
        lls.lls_debug_barrier_limit(-1)
    A, tau, _ = lls.lls_k_geqrf(dev(Y))       # the default limit: the same call succeeds
    R_ref, _, tau_ref = orc.householder_qr(Y)
    assert np.allclose(np.triu(A.cpu().numpy()[:128]), R_ref, rtol=0, atol=1e-13 * np.abs(Y).max() * 128)
    assert np.allclose(tau.cpu().numpy(), tau_ref, rtol=0, atol=1e-13)


def test_solve_returns_timeout_and_the_handle_recovers(lls):
    m, n, r, nb, q = 8192, 256, 100, 128, 1
    A, X, Y = wl.lowrank_xy(m, n, r, seed=8192 + 256, noise=1e-14)
    B = np.random.default_rng(5).standard_normal((m, 2))
    nrm = wl.norm2_of_product(X, Y)
    tol = 1e-10 * nrm
    dA, dB = dev(A), dev(B)
    h = lls.lls_create(nb=nb, q=q, seed=2001)
    try:
        lls.lls_debug_barrier_limit(0)
        try:
            with pytest.raises(lls.LLSError) as e:
                lls.lls_solve(h, dA, dB, tol)
            assert e.value.status == lls.LLS_ERR_TIMEOUT
        finally:
            lls.lls_debug_barrier_limit(-1)
        x, rank, code = lls.lls_solve(h, dA, dB, tol)
        assert code == lls.LLS_OK and rank == r
        ref = orc.solve(A, B, q, nb, tol, 2001)
        assert ref.rank == r
        assert rel(x.cpu().numpy(), ref.x) <= 1e-9
        assert orc.normal_equation_residual(A, x.cpu().numpy(), B, nrm) <= 1e-13
    finally:
        lls.lls_destroy(h)
