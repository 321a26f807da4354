"""Batched solves and the serving queue: each result is the same alone and in
the mix (bit for bit: every kernel reduces in a fixed order), admission
respects the memory cap, resident factors are reused with new right-hand
sides, and results match the FP64 oracle."""

import ctypes as C
import time

import numpy as np
import pytest
import torch

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.asfortranarray(x), dtype=torch.float64, device="cuda").t().contiguous().t()


def problems(count, seed):
    return wl.batched_problems(count, seed=seed, m_range=(200, 700), nrhs_choices=(1, 3, 8))


def solve_alone(lls, p, nb=64, q=1, seed=2004, precision=0):
    h = lls.lls_create(nb=nb, q=q, seed=seed, precision=precision)
    try:
        X, rank, _ = lls.lls_solve(h, dev(p.A), dev(p.B), p.tol)
        return X.cpu().numpy(), rank
    finally:
        lls.lls_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_alone_and_oracle(lls, precision):
    # precision 1 (BF16 sampling, exact-slice tensor-core updates) also runs
    # kernels whose launch shapes differ between problems on several host
    # threads at once
    ps = problems(24, 7)
    h = lls.lls_create(nb=64, q=1, seed=2004, precision=precision)
    lls.lls_set_workers(h, 6)
    # the worker pool runs lls_solve's own launch sequence (the persistent
    # launch, whose tiles sum in another order, has its own test below)
    lls.lls_set_batched_mode(h, lls.LLS_BATCHED_WORKERS)
    try:
        keep, plist, ranks = [], [], []
        for p in ps:
            A, B = dev(p.A), dev(p.B)
            X = lls.empty_colmajor(p.A.shape[1], p.B.shape[1])
            r = C.c_int64(-1)
            ranks.append(r)
            keep.append((A, B, X))
            plist.append(lls.make_problem(A, B, p.tol, X, rank_out=C.pointer(r)))
        code = lls.lls_solve_batched(h, plist)
        torch.cuda.synchronize()
        assert code == 0
    finally:
        lls.lls_destroy(h)
    for i, p in enumerate(ps):
        assert plist[i].status == 0
        x_alone, r_alone = solve_alone(lls, p, precision=precision)
        assert ranks[i].value == r_alone == p.rank
        assert np.array_equal(keep[i][2].cpu().numpy(), x_alone)
    for p, (_, _, X) in list(zip(ps, keep))[:4]:
        ref = orc.solve(p.A, p.B, 1, 64, p.tol, 2004)
        xr = np.reshape(ref.x, X.shape)
        assert np.linalg.norm(X.cpu().numpy() - xr) / np.linalg.norm(xr) < 1e-9


def wait_all(lls, h, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            s = lls.lls_poll(h, t)
            if s != lls.LLS_PENDING:
                out[t] = s
        assert time.time() - t0 < timeout
        time.sleep(0.002)
    return out


def test_serving_results_same_alone_and_in_the_mix(lls):
    ps = problems(16, 11)
    h = lls.lls_create(nb=64, q=1, seed=2004)
    lls.lls_set_workers(h, 4)
    try:
        held, tickets = [], []
        for p in ps:
            A, B = dev(p.A), dev(p.B)
            X = lls.empty_colmajor(p.A.shape[1], p.B.shape[1])
            held.append((A, B, X))
            tickets.append(lls.lls_submit(h, lls.make_problem(A, B, p.tol, X)))
        st = wait_all(lls, h, tickets)
        assert all(v == 0 for v in st.values())
        torch.cuda.synchronize()
    finally:
        lls.lls_destroy(h)
    for p, (_, _, X) in zip(ps, held):
        x_alone, _ = solve_alone(lls, p)
        assert np.array_equal(X.cpu().numpy(), x_alone)


def test_serving_factor_reuse_and_memory_cap(lls):
    p = wl.c1_problem()
    h = lls.lls_create(nb=64, q=1, seed=2001)
    try:
        A, B = dev(p.A), dev(p.B)
        X = lls.empty_colmajor(1000, 1)
        t = lls.lls_submit(h, lls.make_problem(A, B, p.tol, X, keep_factor=1))
        fid = None
        t0 = time.time()
        while fid is None:
            fid = lls.lls_ticket_factor(h, t)
            assert time.time() - t0 < 60
            time.sleep(0.005)
        assert lls.lls_poll(h, t) == 0
        # new right-hand sides against the resident factor, several at once
        Bs = [np.random.default_rng(s).standard_normal((2000, 2)) for s in range(3)]
        held, tickets = [], []
        for b in Bs:
            Bd, Xd = dev(b), lls.empty_colmajor(1000, 2)
            held.append((Bd, Xd))
            tickets.append(lls.lls_submit(h, lls.make_problem(None, Bd, p.tol, Xd, factor_id=fid)))
        st = wait_all(lls, h, tickets)
        assert all(v == 0 for v in st.values())
        for b, (_, Xd) in zip(Bs, held):
            ref = lls.lls_solve_factored(h, fid, dev(b), 1000)
            assert torch.equal(Xd, ref)
            xr = np.reshape(orc.solve(p.A, b, 1, 64, p.tol, 2001).x, (1000, 2))
            assert np.linalg.norm(Xd.cpu().numpy() - xr) / np.linalg.norm(xr) < 1e-9
        # a cap smaller than one request: rejected at submit; a small cap runs one at a time
        lls.lls_set_memory_cap(h, 1 << 20)
        with pytest.raises(lls.LLSError) as e:
            lls.lls_submit(h, lls.make_problem(A, B, p.tol, X))
        assert e.value.status == lls.LLS_ERR_CAPACITY
        lls.lls_set_memory_cap(h, 40 << 20)
        bufs = [(dev(q.A), dev(q.B), lls.empty_colmajor(q.A.shape[1], q.B.shape[1]), q.tol)
                for q in problems(3, 5)]
        ts = [lls.lls_submit(h, lls.make_problem(a, b, tol, x)) for a, b, x, tol in bufs]
        assert all(v == 0 for v in wait_all(lls, h, ts).values())
    finally:
        lls.lls_destroy(h)


def test_autotune_table_drives_tuned_solves(lls, tmp_path):
    h = lls.lls_create(nb=0, q=1, seed=2004)   # nb = 0: n_b and q from the tuning table
    try:
        assert lls.lls_tuning_lookup(h, 700, 300) == (64, 1)       # no entry yet: defaults
        nb, q = lls.lls_autotune(h, 700, 300, trials=1)
        assert nb in (32, 64, 128) and q in (0, 1, 2)
        assert lls.lls_tuning_lookup(h, 1000, 400) == (nb, q)      # same bucket (1024, 512)
        assert lls.lls_tuning_lookup(h, 2000, 400) == (64, 1)      # other bucket
        path = str(tmp_path / "tune.txt")
        lls.lls_tuning_save(h, path)
        h2 = lls.lls_create(nb=0, q=1, seed=2004)
        try:
            lls.lls_tuning_load(h2, path)
            assert lls.lls_tuning_lookup(h2, 700, 300) == (nb, q)
        finally:
            lls.lls_destroy(h2)
        # a tuned solve equals the explicit choice bit for bit, and the oracle to 1e-9
        p = problems(1, 21)[0]
        A, B = dev(p.A), dev(p.B)
        Xt, rt, _ = lls.lls_solve(h, A, B, p.tol)
        mb, nbk = p.A.shape
        tnb, tq = lls.lls_tuning_lookup(h, mb, nbk)
        he = lls.lls_create(nb=tnb, q=tq, seed=2004)
        try:
            Xe, re_, _ = lls.lls_solve(he, A, B, p.tol)
        finally:
            lls.lls_destroy(he)
        assert rt == re_ == p.rank
        assert torch.equal(Xt, Xe)
        ref = np.reshape(orc.solve(p.A, p.B, tq, tnb, p.tol, 2004).x, Xt.shape)
        assert np.linalg.norm(Xt.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-9
        bad = tmp_path / "bad.txt"
        bad.write_text("1 2 300 1\n")
        with pytest.raises(lls.LLSError):
            lls.lls_tuning_load(h, str(bad))
    finally:
        lls.lls_destroy(h)


def test_tuned_batched_solves_use_the_table(lls, tmp_path):
    # workers of a tuned handle (nb = 0) read the parent's table: a batch
    # solved through the pool equals solves with the table's explicit choice
    ps = problems(6, 31)
    path = tmp_path / "tune.txt"
    rows = ["# test table"]
    for p in ps:
        m, n = p.A.shape
        rows.append(f"{(m - 1).bit_length()} {(n - 1).bit_length()} 32 2")
    path.write_text("\n".join(rows) + "\n")
    h = lls.lls_create(nb=0, q=1, seed=2004)
    lls.lls_set_workers(h, 3)
    lls.lls_set_batched_mode(h, lls.LLS_BATCHED_WORKERS)   # lls_solve's own launches
    lls.lls_tuning_load(h, str(path))
    try:
        held, plist = [], []
        for p in ps:
            A, B = dev(p.A), dev(p.B)
            X = lls.empty_colmajor(p.A.shape[1], p.B.shape[1])
            held.append((A, B, X))
            plist.append(lls.make_problem(A, B, p.tol, X))
        assert lls.lls_solve_batched(h, plist) == 0
        torch.cuda.synchronize()
    finally:
        lls.lls_destroy(h)
    for p, (_, _, X) in zip(ps, held):
        x_explicit, _ = solve_alone(lls, p, nb=32, q=2)
        assert np.array_equal(X.cpu().numpy(), x_explicit)


def test_cancel_withdraws_a_queued_request(lls):
    # one worker and slow requests ahead: the last request is still queued
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    mats = [torch.randn(2048, 4096, generator=g, dtype=torch.float64, device="cuda").t()
            for _ in range(4)]
    h = lls.lls_create(nb=64, q=2, seed=2004)
    lls.lls_set_workers(h, 1)
    try:
        held, tickets = [], []
        for A in mats:
            B = torch.randn(1, 4096, generator=g, dtype=torch.float64, device="cuda").t()
            X = lls.empty_colmajor(2048, 1)
            held.append((A, B, X))
            tickets.append(lls.lls_submit(h, lls.make_problem(A, B, 1e-10, X)))
        assert lls.lls_cancel(h, tickets[3]) == lls.LLS_OK
        assert lls.lls_cancel(h, tickets[3]) == lls.LLS_ERR_NOT_FOUND   # already gone
        st = wait_all(lls, h, tickets[:3])
        assert all(v == 0 for v in st.values())
        with pytest.raises(lls.LLSError) as e:
            lls.lls_poll(h, tickets[3])
        assert e.value.status == lls.LLS_ERR_NOT_FOUND
        assert lls.lls_cancel(h, tickets[0]) == lls.LLS_ERR_NOT_FOUND   # finished and polled
    finally:
        lls.lls_destroy(h)


def test_injected_allocation_failure_is_reported_and_recovered(lls):
    p = problems(1, 41)[0]
    A, B = dev(p.A), dev(p.B)
    x_ref, r_ref = solve_alone(lls, p)
    for after in (0, 3):            # the first, or a later, workspace allocation fails
        h = lls.lls_create(nb=64, q=1, seed=2004)
        try:
            lls.lls_debug_fail_allocation(after)
            with pytest.raises(lls.LLSError) as e:
                lls.lls_solve(h, A, B, p.tol)
            assert e.value.status == lls.LLS_ERR_NOMEM
            lls.lls_debug_fail_allocation(-1)
            X, r, _ = lls.lls_solve(h, A, B, p.tol)     # the same handle recovers
            assert r == r_ref and np.array_equal(X.cpu().numpy(), x_ref)
        finally:
            lls.lls_debug_fail_allocation(-1)
            lls.lls_destroy(h)


@pytest.mark.slow
def test_batched_on_the_full_size_distribution(lls):
    """128 problems of the batched workload's own size distribution (m in
    [256, 2048], n in [128, m], rank in [n/4, n], nrhs in {1, 8, 32}) in one
    lls_solve_batched call on 8 workers: every rank equals the construction's
    and a random subset matches the oracle's solve."""
    ps = wl.batched_problems(128, seed=1004)
    h = lls.lls_create(nb=64, q=1, seed=2004)
    lls.lls_set_workers(h, 8)
    try:
        keep, plist, ranks = [], [], []
        for p in ps:
            A, B = dev(p.A), dev(p.B)
            X = lls.empty_colmajor(p.A.shape[1], p.B.shape[1])
            r = C.c_int64(-1)
            ranks.append(r)
            keep.append((A, B, X))
            plist.append(lls.make_problem(A, B, p.tol, X, rank_out=C.pointer(r)))
        code = lls.lls_solve_batched(h, plist)
        torch.cuda.synchronize()
        assert code == 0
    finally:
        lls.lls_destroy(h)
    assert [pl.status for pl in plist] == [0] * len(ps)
    assert [r.value for r in ranks] == [p.rank for p in ps]
    pick = np.random.default_rng(0).choice([i for i, p in enumerate(ps) if p.A.shape[0] <= 1200],
                                           size=4, replace=False)
    for i in pick:
        p = ps[i]
        ref = orc.solve(p.A, p.B, 1, 64, p.tol, 2004)
        x = keep[i][2].cpu().numpy()
        assert ref.rank == p.rank
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-9
        assert orc.normal_equation_residual(p.A, x, p.B, p.norm2) <= 1e-13


# ------------------------------------------------------------------ one persistent launch
def run_batch(lls, ps, mode, workers=6, nb=64, q=1, seed=2004):
    h = lls.lls_create(nb=nb, q=q, seed=seed)
    lls.lls_set_workers(h, workers)
    lls.lls_set_batched_mode(h, mode)
    keep, plist, ranks = [], [], []
    try:
        for p in ps:
            A, B = dev(p.A), dev(p.B)
            X = lls.empty_colmajor(p.A.shape[1], p.B.shape[1])
            r = C.c_int64(-1)
            ranks.append(r)
            keep.append((A, B, X))
            plist.append(lls.make_problem(A, B, p.tol, X, rank_out=C.pointer(r)))
        code = lls._lib.lls_solve_batched(h, len(plist), (lls.lls_problem * len(plist))(*plist))
        torch.cuda.synchronize()
    finally:
        lls.lls_destroy(h)
    return code, [k[2].cpu().numpy() for k in keep], [r.value for r in ranks]


def mixed_shapes():
    """Uneven problems: tall, wide, a narrow last step, n < nb, full rank, a
    zero matrix (rank 0), q's effect through the construction."""
    ps = problems(14, 31)
    g = np.random.default_rng(3)
    for m, n, r in ((90, 300, 40), (333, 47, 47), (64, 64, 64), (700, 129, 100)):
        A, X, Y = wl.lowrank_xy(m, n, r, seed=m * n + r, noise=1e-14)
        ps.append(wl.Problem(A, g.standard_normal((m, 3)), 1e-10 * wl.norm2_of_product(X, Y),
                             wl.norm2_of_product(X, Y), r, 64, 1))
    Z = np.zeros((120, 80))
    ps.append(wl.Problem(Z, g.standard_normal((120, 2)), 1e-10, 1.0, 0, 64, 1))
    return ps


@pytest.mark.parametrize("nb,q", [(64, 1), (32, 2), (48, 0)])
def test_persistent_batched_matches_oracle(lls, nb, q):
    """All problems factored in one persistent launch: ranks equal the
    construction's, x matches the oracle's Fig. 4 solve."""
    ps = mixed_shapes()
    code, xs, ranks = run_batch(lls, ps, lls.LLS_BATCHED_PERSISTENT, nb=nb, q=q)
    assert code == 0
    for p, x, r in zip(ps, xs, ranks):
        assert r == p.rank
        ref = orc.solve(p.A, p.B, q, nb, p.tol, 2004)
        if ref.rank == 0:
            assert np.all(x == 0.0)
            continue
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-9
        assert orc.normal_equation_residual(p.A, x, p.B, p.norm2) <= 1e-13


def test_persistent_batched_alone_equals_in_batch_and_workers(lls):
    """A problem's result does not depend on what else is in the persistent
    launch (bit for bit: each task sums in a fixed order whatever CTA runs
    it), and agrees with the worker-pool path to rounding."""
    ps = mixed_shapes()
    _, xs, _ = run_batch(lls, ps, lls.LLS_BATCHED_PERSISTENT)
    _, xw, _ = run_batch(lls, ps, lls.LLS_BATCHED_WORKERS)
    for i in (0, 5, len(ps) - 2):
        _, x1, _ = run_batch(lls, [ps[i]], lls.LLS_BATCHED_PERSISTENT)
        np.testing.assert_array_equal(x1[0], xs[i])
    for p, a, b in zip(ps, xs, xw):
        if p.rank:
            assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-11


def test_persistent_batched_reports_bad_problems_and_refusals(lls):
    ps = problems(6, 41)
    bad = wl.Problem(ps[2].A.copy(), ps[2].B, ps[2].tol, ps[2].norm2, ps[2].rank, 64, 1)
    bad.A[3, 1] = np.nan
    code, xs, ranks = run_batch(lls, ps[:2] + [bad] + ps[3:], lls.LLS_BATCHED_PERSISTENT)
    assert code == lls.LLS_ERR_NONFINITE
    for i in (0, 1, 3):
        ref = orc.solve(ps[i].A, ps[i].B, 1, 64, ps[i].tol, 2004)
        assert np.linalg.norm(xs[i] - ref.x) / np.linalg.norm(ref.x) <= 1e-9
    # outside the persistent path (explicit V): refused in PERSISTENT mode
    h = lls.lls_create(nb=64, q=1, seed=2004, explicit_v=1)
    try:
        lls.lls_set_batched_mode(h, lls.LLS_BATCHED_PERSISTENT)
        p = ps[0]
        A, B = dev(p.A), dev(p.B)
        X = lls.empty_colmajor(p.A.shape[1], p.B.shape[1])
        arr = (lls.lls_problem * 1)(lls.make_problem(A, B, p.tol, X))
        assert lls._lib.lls_solve_batched(h, 1, arr) == lls.LLS_ERR_ARG
    finally:
        lls.lls_destroy(h)


def test_persistent_batched_scheduler_wait_runs_out(lls):
    """With the poll limit at zero, a CTA that finds no ready task gives up at
    once: the launch ends with LLS_ERR_TIMEOUT (no hang, no fault) and the
    next batch on a fresh handle solves."""
    ps = problems(8, 51)
    lls.lls_debug_barrier_limit(0)
    try:
        code, _, _ = run_batch(lls, ps, lls.LLS_BATCHED_PERSISTENT)
    finally:
        lls.lls_debug_barrier_limit(-1)
    assert code == lls.LLS_ERR_TIMEOUT
    code, xs, ranks = run_batch(lls, ps, lls.LLS_BATCHED_PERSISTENT)
    assert code == 0 and ranks == [p.rank for p in ps]
