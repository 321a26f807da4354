"""The solver's host-side orchestration, run on the CPU.

tests/host_harness links the library's own solver.cu, ooc_solve.cu and
ooc_plan.cu with plain-loop stand-ins for the launchers and the CUDA runtime,
so the exact sequence of launches, operand pointers, leading dimensions,
operand modes, buffer reservations and copies of a solve runs here without a
GPU.  The oracle gets the harness's deterministic sketch, and over random
shapes (tall, wide, narrow last steps, nb = 1 and nb > n, rank 0 to full),
q = 0..4, with and without Nullify, explicit V and refinement, and for the
out-of-core executor caches of one panel to all of them under both eviction
policies, the rank must equal the oracle's and x must agree to 1e-8.  Where
the fast option's x is itself ill-determined (the oracle's fast x is far
from the pseudoinverse solution: T_12 not small), the least-squares property
is checked instead.  The GPU kernels themselves are checked by the gpu tests.
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

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host_harness", "build.py")
    spec = importlib.util.spec_from_file_location("host_harness_build", path)
    hb = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(hb)
    lib = C.CDLL(hb.build())
    lib.harness_handle.restype = C.c_void_p
    lib.harness_handle.argtypes = [C.c_int, C.c_int, C.c_int, C.c_ulonglong]
    lib.harness_solve.argtypes = [C.c_void_p, C.c_void_p, I, I, I, C.c_void_p, I, I, C.c_double,
                                  C.c_void_p, I, C.POINTER(I), C.c_int, C.c_int]
    lib.lls_solve_ooc.argtypes = [C.c_void_p, C.c_void_p, I, I, I, C.c_void_p, I, I, C.c_double,
                                  C.c_void_p, I, C.POINTER(I), I, C.c_int32]
    return lib


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
        yield dict(it=it, kind=kind, m=m, n=n, r=r, nb=nb, q=q, nullify=g.randint(0, 1),
                   explicit_v=0 if ooc else g.randint(0, 1),
                   max_refine=0 if ooc else g.choice([0, 0, 1, 2]),
                   cache=g.randint(1, P + 1), policy=g.randint(0, 1))


def run_case(harness, c, ooc):
    A, tol = problem(c["kind"], c["m"], c["n"], c["r"], seed=1000 + c["it"])
    m, n = A.shape
    B = np.random.default_rng(c["it"]).standard_normal((m, 2))
    ref = orc.solve(A, B, c["q"], c["nb"], tol, 77, do_nullify=bool(c["nullify"]))
    h = harness.harness_handle(c["nb"], c["q"], c["nullify"], 77)
    Af, Bf = np.asfortranarray(A), np.asfortranarray(B)
    X = np.zeros((n, 2), order="F")
    rk = I(0)
    if ooc:
        code = harness.lls_solve_ooc(h, Af.ctypes.data, m, n, m, Bf.ctypes.data, 2, m, tol,
                                     X.ctypes.data, n, C.byref(rk), c["cache"], c["policy"])
    else:
        code = harness.harness_solve(h, Af.ctypes.data, m, n, m, Bf.ctypes.data, 2, m, tol,
                                     X.ctypes.data, n, C.byref(rk), c["explicit_v"],
                                     c["max_refine"])
    check(A, B, X, code, rk.value, ref, c["nullify"])


@pytest.mark.parametrize("chunk", range(4))
def test_in_core_orchestration_random(harness, sketch, chunk):
    for c in random_configs(100 + chunk, 25, ooc=False):
        run_case(harness, c, ooc=False)


@pytest.mark.parametrize("chunk", range(4))
def test_out_of_core_executor_random(harness, sketch, chunk):
    for c in random_configs(200 + chunk, 25, ooc=True):
        run_case(harness, c, ooc=True)
