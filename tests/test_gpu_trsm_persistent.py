"""Triangular solves through the inverses of the 64 x 64 diagonal blocks
(lls_k_trsm_upper_blockinv), the T_11^{-1} and T_11^{-T} of the refinement
of the TF32 modes: with at most four right-hand sides one cooperative launch
with a grid barrier per block, with five to sixteen two launches a block.
Checked against scipy's substitution on well-conditioned upper triangles,
ragged last blocks included, plus a barrier timeout reported as
LLS_ERR_TIMEOUT (the poll limit lowered to zero: nothing faults or hangs)."""

import numpy as np
import pytest
import scipy.linalg as sla
import torch

pytestmark = pytest.mark.gpu


def dev(x):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    out = torch.empty((x.shape[1], x.shape[0]), dtype=torch.float64, device="cuda").t()
    out.copy_(torch.as_tensor(x))
    return out


def upper(r, seed):
    g = np.random.default_rng(seed)
    R = np.triu(g.standard_normal((r, r))) / np.sqrt(max(r, 1))
    R[np.arange(r), np.arange(r)] = g.uniform(1.0, 2.0, r) * g.choice([-1.0, 1.0], r)
    # junk below the diagonal: only the upper triangle may be read
    return R + np.tril(np.full((r, r), np.nan), -1)


@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("r", [1, 63, 64, 65, 200, 1000, 3001])
def test_blockinv_solve_matches_substitution(lls, r, nrhs, trans):
    R = upper(r, r + 7 * nrhs + trans)
    B = np.random.default_rng(r + nrhs).standard_normal((r, nrhs))
    Ru = np.triu(np.nan_to_num(R))
    ref = sla.solve_triangular(Ru, B, lower=False, trans="T" if trans else "N")
    Bd = dev(B)
    lls.lls_k_trsm_upper_blockinv(dev(R), Bd, trans=bool(trans))
    got = Bd.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_blockinv_solve_leading_dimensions(lls):
    r, nrhs = 300, 3
    R = upper(r, 11)
    Rbig = np.zeros((r + 5, r))
    Rbig[:r] = np.nan_to_num(R)
    Rt = dev(Rbig)[:r]                                # ldr = r + 5
    B = np.random.default_rng(12).standard_normal((r, nrhs))
    Bbig = dev(np.vstack([B, np.zeros((9, nrhs))]))   # ldb = r + 9
    lls.lls_k_trsm_upper_blockinv(Rt, Bbig[:r], trans=True)
    ref = sla.solve_triangular(np.triu(np.nan_to_num(R)), B, lower=False, trans="T")
    assert np.max(np.abs(Bbig[:r].cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.all(Bbig[r:].cpu().numpy() == 0.0)      # rows past r untouched


def test_blockinv_barrier_timeout(lls):
    r = 2000
    R = dev(upper(r, 21))
    B = np.random.default_rng(22).standard_normal((r, 2))
    lls.lls_debug_barrier_limit(0)
    try:
        with pytest.raises(lls.LLSError) as e:
            lls.lls_k_trsm_upper_blockinv(R, dev(B))
        assert e.value.status == lls.LLS_ERR_TIMEOUT
    finally:
        lls.lls_debug_barrier_limit(-1)
    Bd = dev(B)
    lls.lls_k_trsm_upper_blockinv(R, Bd)
    ref = sla.solve_triangular(np.triu(np.nan_to_num(R.cpu().numpy())), B, lower=False)
    assert np.max(np.abs(Bd.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
