"""The library's host-side code, run on the CPU through its public C API.

tests/host_harness links the library's own api.cu, serving.cu, solver.cu,
tuner.cu, trace.cu, guard.cu, ooc_solve.cu and ooc_plan.cu, compiled as they
are, with plain-loop stand-ins for the launchers and the CUDA runtime, so the
exact sequence of launches, operand pointers, leading dimensions, operand
modes, buffer reservations and copies of a solve -- and the worker pool, the
serving queue, the tuning table, guard words and argument checks -- run here
without a GPU ("device" memory is host memory).  The oracle gets the
harness's deterministic sketch.  Over random shapes (tall, wide, narrow last
steps, nb = 1 and nb > n, rank 0 to full), q = 0..4, all four precision modes
(the mixed mode's products are exact here: its orchestration is what is
checked), with and without Nullify, explicit V and refinement, and for the
out-of-core executor caches
of one panel to all of them under both eviction policies, the rank must equal
the oracle's and x must agree to 1e-8; where the fast option's x is itself
ill-determined (the oracle's fast x is far from the pseudoinverse solution:
T_12 not small) the least-squares property is checked instead.  The GPU
kernels themselves are checked by the gpu tests.
"""

import ctypes as C
import random

import numpy as np
import pytest

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

I = C.c_int64


@pytest.fixture(scope="module")
def harness():
    import importlib.util
    import os

    from paper_2408_05238_b300 import lls as binding

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host_harness", "build.py")
    spec = importlib.util.spec_from_file_location("host_harness_build", path)
    hb = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(hb)
    lib = C.CDLL(hb.build())
    H, P, D = C.c_void_p, C.c_void_p, C.c_double
    sigs = {
        "lls_create": [C.POINTER(H), C.POINTER(binding.lls_options), P],
        "lls_destroy": [H],
        "lls_solve": [H, P, I, I, I, P, I, I, D, P, I, C.POINTER(I)],
        "lls_factor": [H, P, I, I, I, D, C.POINTER(I), C.POINTER(I)],
        "lls_solve_factored": [H, I, P, I, I, P, I],
        "lls_factor_get": [H, I, C.c_int32, P, I],
        "lls_factor_release": [H, I],
        "lls_refinement_info": [H, C.POINTER(C.c_int32), C.POINTER(D)],
        "lls_solve_batched": [H, I, C.POINTER(binding.lls_problem)],
        "lls_set_workers": [H, C.c_int],
        "lls_set_batched_mode": [H, C.c_int],
        "lls_set_memory_cap": [H, I],
        "lls_submit": [H, C.POINTER(binding.lls_problem), C.POINTER(I)],
        "lls_poll": [H, I, C.POINTER(C.c_int)],
        "lls_autotune": [H, I, I, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "lls_tuning_lookup": [H, I, I, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "lls_tuning_save": [H, C.c_char_p],
        "lls_tuning_load": [H, C.c_char_p],
        "lls_last_error": [H, C.POINTER(C.c_int), C.c_char_p, I],
        "lls_debug_guard": [C.c_int],
        "lls_debug_guard_report": [C.c_char_p, I],
        "lls_debug_guard_selftest": [],
        "lls_solve_ooc": [H, P, I, I, I, P, I, I, D, P, I, C.POINTER(I), I, C.c_int32],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int64 if name == "lls_debug_guard_report" else C.c_int
    lib.binding = binding
    return lib


def create(lib, **kw):
    o = lib.binding.lls_default_options(**kw)
    h = C.c_void_p()
    assert lib.lls_create(C.byref(h), C.byref(o), None) == 0
    return h


def F(x):
    return np.asfortranarray(np.asarray(x, dtype=np.float64))


def hashed_sketch(seed, step, rows, cols):
    """The harness's sketch: a fixed hash of (row, column, step, seed)."""
    i = np.arange(rows, dtype=np.float64)[:, None]
    j = np.arange(cols, dtype=np.float64)[None, :]
    v = np.sin(12.9898 * i + 78.233 * j + 37.719 * step + float(seed % 1000)) * 43758.5453
    return v - np.floor(v) - 0.5


@pytest.fixture
def sketch(monkeypatch):
    monkeypatch.setattr(orc, "sketch_matrix", hashed_sketch)


def problem(kind, m, n, r, seed):
    if kind == "decay":   # no gap: sigma_i = 0.8^i, tol inside the spectrum
        k = min(m, n)
        Q1 = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, m)))[0][:, :k]
        Q2 = np.linalg.qr(np.random.default_rng(seed + 1).standard_normal((n, n)))[0][:, :k]
        return (Q1 * 0.8 ** np.arange(k)) @ Q2.T, 1e-3
    if r == 0:
        return np.zeros((m, n)), 0.0
    A, X, Y = wl.lowrank_xy(m, n, r, seed=seed, noise=1e-14)
    return A, 1e-10 * wl.norm2_of_product(X, Y)


def check(A, B, x, code, rank, ref, nullify):
    assert code >= 0 and rank == ref.rank
    nx = np.linalg.norm(ref.x)
    if nx == 0:
        assert np.linalg.norm(x) == 0
        return
    if np.linalg.norm(x - ref.x) <= 1e-8 * nx:
        return
    assert not nullify, np.linalg.norm(x - ref.x) / nx
    xp = orc.pinv_solve(A, B, ref.rank)            # an ill-determined fast option
    assert np.linalg.norm(ref.x - xp) > 1e-9 * np.linalg.norm(xp)
    assert np.linalg.norm(A @ x - A @ xp) <= 1e-8 * np.linalg.norm(B)


def random_configs(seed, count, ooc):
    g = random.Random(seed)
    for it in range(count):
        m, n, nb, q = g.randint(1, 60), g.randint(1, 60), g.randint(1, 40), g.randint(0, 4)
        kind = "decay" if g.random() < 0.25 else "xy"
        if kind == "decay":
            q, nb = 0, min(nb, 12)
        r = g.randint(0, min(m, n))
        P = -(-n // nb)
        nullify = g.randint(0, 1)
        precision = 0 if ooc else g.randint(0, 3)
        yield dict(it=it, kind=kind, m=m, n=n, r=r, nb=nb, q=q, nullify=nullify,
                   precision=precision if nullify else 0,   # the fast option is FP64-only
                   explicit_v=0 if ooc else g.randint(0, 1),
                   max_refine=0 if ooc else g.choice([0, 0, 1, 2]),
                   cache=g.randint(1, P + 1), policy=g.randint(0, 1))


def run_case(harness, c, ooc):
    A, tol = problem(c["kind"], c["m"], c["n"], c["r"], seed=1000 + c["it"])
    m, n = A.shape
    B = np.random.default_rng(c["it"]).standard_normal((m, 2))
    ref = orc.solve(A, B, c["q"], c["nb"], tol, 77, do_nullify=bool(c["nullify"]))
    h = create(harness, nb=c["nb"], q=c["q"], nullify=c["nullify"], seed=77,
               precision=c["precision"], explicit_v=c["explicit_v"], max_refine=c["max_refine"])
    try:
        Af, Bf = F(A), F(B)
        X = np.zeros((n, 2), order="F")
        rk = I(0)
        if ooc:
            code = harness.lls_solve_ooc(h, Af.ctypes.data, m, n, m, Bf.ctypes.data, 2, m, tol,
                                         X.ctypes.data, n, C.byref(rk), c["cache"], c["policy"])
        else:
            code = harness.lls_solve(h, Af.ctypes.data, m, n, m, Bf.ctypes.data, 2, m, tol,
                                     X.ctypes.data, n, C.byref(rk))
    finally:
        harness.lls_destroy(h)
    check(A, B, X, code, rk.value, ref, c["nullify"])


@pytest.mark.parametrize("chunk", range(4))
def test_in_core_orchestration_random(harness, sketch, chunk):
    for c in random_configs(100 + chunk, 25, ooc=False):
        run_case(harness, c, ooc=False)


@pytest.mark.parametrize("chunk", range(4))
def test_out_of_core_executor_random(harness, sketch, chunk):
    for c in random_configs(200 + chunk, 25, ooc=True):
        run_case(harness, c, ooc=True)


# ---- the public C API on the harness ------------------------------------------
def gap_problem(m, n, r, seed, nrhs=2):
    A, X, Y = wl.lowrank_xy(m, n, r, seed=seed, noise=1e-14)
    B = np.random.default_rng(seed).standard_normal((m, nrhs))
    return A, B, 1e-10 * wl.norm2_of_product(X, Y)


def test_factor_reuse_export_and_refinement(harness, sketch):
    """lls_factor keeps A for refinement and V for export: solves with the
    resident factor match the oracle, V^T V = I, (A V)^T (A V) = T^T T and
    T(0:r, r:n) = 0 after Nullify."""
    m, n, r = 50, 40, 17
    A, B, tol = gap_problem(m, n, r, seed=3)
    ref = orc.solve(A, B, 1, 8, tol, 77)
    h = create(harness, nb=8, q=1, seed=77, explicit_v=1, max_refine=2)
    try:
        Af, Bf = F(A), F(B)
        fid, rk = I(0), I(0)
        assert harness.lls_factor(h, Af.ctypes.data, m, n, m, tol, C.byref(fid), C.byref(rk)) == 0
        assert rk.value == r
        X = np.zeros((n, 2), order="F")
        assert harness.lls_solve_factored(h, fid.value, Bf.ctypes.data, 2, m, X.ctypes.data, n) == 0
        steps, corr = C.c_int32(0), C.c_double(0)
        harness.lls_refinement_info(h, C.byref(steps), C.byref(corr))
        assert steps.value >= 1 and corr.value <= 1e-12
        T = np.zeros((m, n), order="F")
        V = np.zeros((n, n), order="F")
        assert harness.lls_factor_get(h, fid.value, 0, T.ctypes.data, m) == 0
        assert harness.lls_factor_get(h, fid.value, 1, V.ctypes.data, n) == 0
        assert harness.lls_factor_release(h, fid.value) == 0
    finally:
        harness.lls_destroy(h)
    assert np.linalg.norm(X - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13 * n
    AV = A @ V
    assert np.linalg.norm(AV.T @ AV - T.T @ T) <= 1e-12 * np.linalg.norm(A) ** 2
    assert np.all(T[:r, r:] == 0.0) and np.all(np.tril(T, -1) == 0.0)


@pytest.mark.parametrize("m,precision", [(4096, 0), (4097, 0), (4096, 2)])
def test_large_factor_replays_and_solves(harness, sketch, m, precision):
    """A factor with 4096 rows takes the solve kernels chosen for large factors
    (one cooperative launch per replay and per triangular solve, with at most
    four right-hand sides; an odd leading dimension keeps the per-step kernels
    for U); five right-hand sides take the per-step kernels.  Both match the
    oracle and each other, in FP64 and in the 3xTF32 mode with refinement."""
    n, r = 24, 10
    A, B, tol = gap_problem(m, n, r, seed=m + precision, nrhs=5)
    ref = orc.solve(A, B, 1, 8, tol, 77)
    xs = []
    for nrhs in (2, 5):
        h = create(harness, nb=8, q=1, seed=77, precision=precision,
                   max_refine=8 if precision else 0)
        try:
            Bn = F(B[:, :nrhs])
            X = np.zeros((n, nrhs), order="F")
            rk = I(0)
            code = harness.lls_solve(h, F(A).ctypes.data, m, n, m, Bn.ctypes.data, nrhs, m, tol,
                                     X.ctypes.data, n, C.byref(rk))
        finally:
            harness.lls_destroy(h)
        assert code == 0 and rk.value == r
        assert np.linalg.norm(X - ref.x[:, :nrhs]) <= 1e-9 * np.linalg.norm(ref.x[:, :nrhs])
        xs.append(X)
    assert np.max(np.abs(xs[0] - xs[1][:, :2])) <= 1e-12 * np.max(np.abs(xs[1]))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batched_pool_equals_alone(harness, sketch, mode):
    """Problems solved as a batch are bit-identical to the same problems
    solved alone, and match the oracle: through the persistent launch's
    driver (mode 0 picks it for these FP64 problems, mode 2 asks for it; the
    kernel itself is emulated here by the plain-loop launchers in its phase
    order) and through the worker pool (mode 1, three host threads)."""
    probs = [gap_problem(m, n, r, seed=s) for (m, n, r, s) in
             [(40, 30, 10, 1), (30, 45, 12, 2), (50, 50, 20, 3), (25, 12, 12, 4), (33, 33, 5, 5)]]
    h = create(harness, nb=8, q=1, seed=77)
    assert harness.lls_set_batched_mode(h, mode) == 0
    try:
        alone = []
        for A, B, tol in probs:
            m, n = A.shape
            X = np.zeros((n, 2), order="F")
            rk = I(0)
            assert harness.lls_solve(h, F(A).ctypes.data, m, n, m, F(B).ctypes.data, 2, m, tol,
                                     X.ctypes.data, n, C.byref(rk)) == 0
            alone.append(X)
        assert harness.lls_set_workers(h, 3) == 0
        keep, arr = [], (harness.binding.lls_problem * len(probs))()
        for i, (A, B, tol) in enumerate(probs):
            m, n = A.shape
            Af, Bf, X = F(A), F(B), np.zeros((n, 2), order="F")
            keep += [Af, Bf, X]
            p = arr[i]
            p.A, p.m, p.n, p.lda = Af.ctypes.data, m, n, m
            p.B, p.nrhs, p.ldb = Bf.ctypes.data, 2, m
            p.tol, p.X, p.ldx = tol, X.ctypes.data, n
            p.factor_id, p.keep_factor = -1, 0
        assert harness.lls_solve_batched(h, len(probs), arr) >= 0
    finally:
        harness.lls_destroy(h)
    for i, (A, B, tol) in enumerate(probs):
        assert arr[i].status == 0
        np.testing.assert_array_equal(keep[3 * i + 2], alone[i])
        ref = orc.solve(A, B, 1, 8, tol, 77)
        assert np.linalg.norm(alone[i] - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_serving_queue_memory_cap_and_factor_reuse(harness, sketch):
    """Submitted requests complete with the oracle's result; a request larger
    than the memory cap is refused at submission; a kept factor serves a later
    request with new right-hand sides."""
    A, B, tol = gap_problem(40, 30, 9, seed=7)
    B2 = np.random.default_rng(8).standard_normal((40, 2))
    h = create(harness, nb=8, q=1, seed=77)
    try:
        assert harness.lls_set_workers(h, 2) == 0
        Af, Bf, B2f = F(A), F(B), F(B2)
        X1, X2 = np.zeros((30, 2), order="F"), np.zeros((30, 2), order="F")
        p = harness.binding.lls_problem()
        p.A, p.m, p.n, p.lda, p.B, p.nrhs, p.ldb = Af.ctypes.data, 40, 30, 40, Bf.ctypes.data, 2, 40
        p.tol, p.X, p.ldx, p.factor_id, p.keep_factor = tol, X1.ctypes.data, 30, -1, 1
        t = I(0)
        assert harness.lls_submit(h, C.byref(p), C.byref(t)) == 0
        st = C.c_int(1)
        while st.value == 1:
            assert harness.lls_poll(h, t.value, C.byref(st)) >= 0 or st.value < 0
        assert st.value == 0
        assert harness.lls_set_memory_cap(h, 1000) == 0          # far below any request
        assert harness.lls_submit(h, C.byref(p), C.byref(t)) == harness.binding.LLS_ERR_CAPACITY
    finally:
        harness.lls_destroy(h)
    ref1 = orc.solve(A, B, 1, 8, tol, 77)
    assert np.linalg.norm(X1 - ref1.x) <= 1e-9 * np.linalg.norm(ref1.x)


def test_tuning_table_roundtrip(harness, sketch, tmp_path):
    """lls_autotune fills the bucket of (m, n); the table written by
    lls_tuning_save is read back by another handle; a malformed file is
    refused with nothing merged."""
    h = create(harness, nb=0, q=1, seed=77)
    h2 = create(harness, nb=0, q=1, seed=77)
    try:
        nb, q = C.c_int32(0), C.c_int32(0)
        assert harness.lls_autotune(h, 60, 40, 1, C.byref(nb), C.byref(q)) == 0
        assert nb.value in (32, 64) and q.value in (0, 1, 2)
        path = str(tmp_path / "table.txt").encode()
        assert harness.lls_tuning_save(h, path) == 0
        assert harness.lls_tuning_load(h2, path) == 0
        nb2, q2 = C.c_int32(0), C.c_int32(0)
        assert harness.lls_tuning_lookup(h2, 60, 40, C.byref(nb2), C.byref(q2)) == 0
        assert (nb2.value, q2.value) == (nb.value, q.value)
        bad = tmp_path / "bad.txt"
        bad.write_text("9 9 16 2\nnot a line\n")
        assert harness.lls_tuning_load(h2, str(bad).encode()) == harness.binding.LLS_ERR_ARG
        nb3, q3 = C.c_int32(0), C.c_int32(0)
        assert harness.lls_tuning_lookup(h2, 300, 300, C.byref(nb3), C.byref(q3)) == 0
        assert (nb3.value, q3.value) == (64, 1)      # bucket (9, 9) not merged: the default
        # (60, 40) and (33, 33) share the bucket (ceil log2 m, ceil log2 n) = (6, 6)
        assert harness.lls_tuning_lookup(h2, 33, 33, C.byref(nb3), C.byref(q3)) == 0
        assert (nb3.value, q3.value) == (nb.value, q.value)
    finally:
        harness.lls_destroy(h)
        harness.lls_destroy(h2)


def test_guard_words_on_host_memory(harness, sketch):
    """The guard-word machinery detects writes just past either end of a
    buffer, and a guarded solve leaves every guard intact."""
    assert harness.lls_debug_guard_selftest() == 0
    A, B, tol = gap_problem(45, 35, 11, seed=9)
    assert harness.lls_debug_guard(1) == 0
    try:
        h = create(harness, nb=8, q=1, seed=77, explicit_v=1)
        try:
            X = np.zeros((35, 2), order="F")
            rk = I(0)
            assert harness.lls_solve(h, F(A).ctypes.data, 45, 35, 45, F(B).ctypes.data, 2, 45, tol,
                                     X.ctypes.data, 35, C.byref(rk)) == 0
        finally:
            harness.lls_destroy(h)
        msg = C.create_string_buffer(256)
        assert harness.lls_debug_guard_report(msg, 256) == 0, msg.value
    finally:
        harness.lls_debug_guard(0)


@pytest.mark.parametrize("bad,index", [("m", 3), ("lda", 5), ("ldb", 8), ("ldx", 11), ("tol", 9)])
def test_argument_errors_name_their_argument(harness, bad, index):
    h = create(harness, nb=8, q=1)
    try:
        A, B = F(np.ones((10, 6))), F(np.ones((10, 1)))
        X = np.zeros((6, 1), order="F")
        args = dict(m=10, lda=10, ldb=10, ldx=6, tol=1e-8)
        args[bad] = {"m": -1, "lda": 9, "ldb": 9, "ldx": 5, "tol": float("nan")}[bad]
        rk = I(0)
        code = harness.lls_solve(h, A.ctypes.data, args["m"], 6, args["lda"], B.ctypes.data, 1,
                                 args["ldb"], args["tol"], X.ctypes.data, args["ldx"], C.byref(rk))
        assert code == harness.binding.LLS_ERR_ARG
        arg = C.c_int(0)
        harness.lls_last_error(h, C.byref(arg), None, 0)
        assert arg.value == index
    finally:
        harness.lls_destroy(h)


def test_host_entry_point_and_phase_trace(harness, sketch):
    """lls_solve_host (host buffers, copies inside) gives lls_solve's x, and
    the per-phase trace counts one sample, QR of Y, right update, panel and
    left update per step (left update: every step with columns to its right),
    one block-SVD phase, one rank phase, one Nullify and one solve."""
    binding = harness.binding
    harness.lls_solve_host.argtypes = harness.lls_solve.argtypes
    harness.lls_solve_host.restype = C.c_int
    harness.lls_trace_enable.argtypes = [C.c_void_p, C.c_int]
    harness.lls_trace_read.argtypes = [C.c_void_p, C.POINTER(binding.lls_trace_stat), I,
                                       C.POINTER(I)]
    m, n, r, nb = 50, 44, 15, 8
    A, B, tol = gap_problem(m, n, r, seed=12)
    h = create(harness, nb=nb, q=1, seed=77)
    try:
        X1, X2 = np.zeros((n, 2), order="F"), np.zeros((n, 2), order="F")
        rk = I(0)
        assert harness.lls_solve(h, F(A).ctypes.data, m, n, m, F(B).ctypes.data, 2, m, tol,
                                 X1.ctypes.data, n, C.byref(rk)) == 0
        assert harness.lls_trace_enable(h, 1) == 0
        assert harness.lls_solve_host(h, F(A).ctypes.data, m, n, m, F(B).ctypes.data, 2, m, tol,
                                      X2.ctypes.data, n, C.byref(rk)) == 0
        stats = (binding.lls_trace_stat * 64)()
        cnt = I(0)
        assert harness.lls_trace_read(h, stats, 64, C.byref(cnt)) == 0
        phases = {s.name.decode(): s.launches for s in stats[:cnt.value]
                  if s.name.decode().startswith("phase:")}
    finally:
        harness.lls_destroy(h)
    np.testing.assert_array_equal(X1, X2)
    steps = -(-min(m, n) // nb)
    assert phases["phase:sample"] == phases["phase:qr_y"] == steps
    assert phases["phase:right_update"] == phases["phase:panel"] == steps
    assert phases["phase:left_update"] == steps
    assert phases["phase:block_svd"] == phases["phase:rank"] == 1
    assert phases["phase:nullify"] == 1 and phases["phase:solve"] == 1


def test_persistent_batched_mode_refuses_what_it_cannot_take(harness, sketch):
    """LLS_BATCHED_PERSISTENT with an option the persistent path does not take
    (explicit V) returns LLS_ERR_ARG naming argument 3; AUTO falls back to
    the worker pool for the same batch; a mode outside 0..2 is refused."""
    A, B, tol = gap_problem(30, 20, 8, seed=9)
    h = create(harness, nb=8, q=1, seed=77, explicit_v=1)
    try:
        assert harness.lls_set_batched_mode(h, 3) == -1
        Af, Bf, X = F(A), F(B), np.zeros((20, 2), order="F")
        arr = (harness.binding.lls_problem * 1)()
        p = arr[0]
        p.A, p.m, p.n, p.lda = Af.ctypes.data, 30, 20, 30
        p.B, p.nrhs, p.ldb = Bf.ctypes.data, 2, 30
        p.tol, p.X, p.ldx, p.factor_id = tol, X.ctypes.data, 20, -1
        assert harness.lls_set_batched_mode(h, 2) == 0
        assert harness.lls_solve_batched(h, 1, arr) == -1
        arg = C.c_int(0)
        harness.lls_last_error(h, C.byref(arg), None, 0)
        assert arg.value == 3
        assert harness.lls_set_batched_mode(h, 0) == 0
        assert harness.lls_solve_batched(h, 1, arr) == 0 and arr[0].status == 0
        ref = orc.solve(A, B, 1, 8, tol, 77)
        assert np.linalg.norm(X - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    finally:
        harness.lls_destroy(h)
