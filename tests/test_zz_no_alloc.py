"""lls_k_panel_qr_noalloc: the panel QR for callers that cannot allocate
device memory (their memory is owned by another allocator, or they must not
block on cudaMalloc / cudaFree).  Its scratch is a fixed array inside the
library; its results must equal those of lls_k_geqrf, which allocates its
scratch.

Each pair below makes two calls in a row whose panels both use that array,
so the second call starts from the first call's leftovers in it: the
shared-memory (slab) kernel twice at different column counts, the slab
kernel followed by the global-memory kernel (a 40000-row panel's slabs do
not fit in shared memory), and the global-memory kernel followed by a small
panel.  Panels of at most a few thousand rows run on one thread-block
cluster and use no scratch at all.

Collected last on purpose: a failure here leaves every other test run."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.asfortranarray(x), dtype=torch.float64, device="cuda").t().contiguous().t()


@pytest.mark.parametrize("shapes", [((8192, 96), (16384, 128)),
                                    ((16384, 128), (40000, 128)),
                                    ((40000, 128), (300, 128), (129, 7))])
def test_noalloc_panel_qr_matches_allocating_entry_point(lls, shapes):
    for call, (m, n) in enumerate(shapes):
        Y = np.random.default_rng(10 * m + n + call).standard_normal((m, n))
        A_ref, tau_ref, _ = lls.lls_k_geqrf(dev(Y))
        A = dev(Y)
        tau = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        code = lls.lls_k_panel_qr_noalloc(A, tau, status)
        torch.cuda.synchronize()
        assert code == lls.LLS_OK
        assert int(status.item()) == 0
        k = min(m, n)
        got, ref = A.cpu().numpy(), A_ref.cpu().numpy()
        scale = np.abs(Y).max()
        assert np.allclose(np.triu(got[:k]), np.triu(ref[:k]), rtol=0, atol=1e-13 * scale * np.sqrt(m))
        assert np.allclose(np.tril(got, -1), np.tril(ref, -1), rtol=0, atol=1e-12)
        assert np.allclose(tau.cpu().numpy()[:k], tau_ref.cpu().numpy(), rtol=0, atol=1e-13)


def test_noalloc_rejects_too_many_columns(lls):
    A = lls.empty_colmajor(300, 129)
    tau = torch.zeros(129, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lls.lls_k_panel_qr_noalloc(A, tau, status) == lls.LLS_ERR_CAPACITY
