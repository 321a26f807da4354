"""The C-ABI library loads and exports every entry point its headers declare;
host-side argument checks that run before any CUDA call (CPU only)."""

import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_05238_b300 import build

    build.build()
    from paper_2408_05238_b300 import lls

    return lls


def declared_functions():
    names = set()
    for hdr in ("lls.h", "lls_kernels.h"):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lls_\w+)\s*\(", text, flags=re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lls_\w+)", out))
    missing = names - exported
    assert not missing, missing
    for n in names:
        assert getattr(lib._lib, n) is not None


def test_status_strings(lib):
    for code in (0, 1, 2, 3, -1, -2, -3, -4, -5, -6, -7, -8):
        s = lib.status_string(code)
        assert s and s != "unknown status"
    assert lib.status_string(12345) == "unknown status"


def test_default_options(lib):
    o = lib.lls_default_options()
    assert (o.nb, o.q, o.precision, o.nullify, o.seed) == (64, 1, 0, 1, 2001)
    assert (o.explicit_v, o.max_refine, o.refine_tol) == (0, 0, 1e-12)
    assert list(o.reserved) == [0, 0]
    # the ctypes mirror has the C struct's size (4 int32, uint64, 2 int32, double, 2 int32)
    assert C.sizeof(lib.lls_options) == 48
    assert lib._lib.lls_default_options(None) == lib.LLS_ERR_ARG


def test_null_handle_and_bad_create(lib):
    assert lib._lib.lls_create(None, None, None) == lib.LLS_ERR_ARG
    assert lib._lib.lls_destroy(None) == lib.LLS_ERR_ARG
    assert lib._lib.lls_solve(None, None, 0, 0, 1, None, 0, 1, 0.0, None, 1, None) == lib.LLS_ERR_ARG
    h = C.c_void_p()
    for nb in (-1, 129):   # nb = 0 is valid: n_b and q from the tuning table
        bad = lib.lls_default_options(nb=nb)
        assert lib._lib.lls_create(C.byref(h), C.byref(bad), None) == lib.LLS_ERR_ARG
    bad = lib.lls_default_options(q=9)
    assert lib._lib.lls_create(C.byref(h), C.byref(bad), None) == lib.LLS_ERR_ARG


@pytest.mark.parametrize("field,value", [("explicit_v", 2), ("explicit_v", -1), ("max_refine", -1),
                                         ("max_refine", 17), ("refine_tol", -1e-3),
                                         ("refine_tol", float("nan")), ("refine_tol", float("inf")),
                                         ("nullify", 2), ("precision", 7)])
def test_bad_options_rejected_before_any_cuda_call(lib, field, value):
    h = C.c_void_p()
    bad = lib.lls_default_options(**{field: value})
    assert lib._lib.lls_create(C.byref(h), C.byref(bad), None) == lib.LLS_ERR_ARG
    bad = lib.lls_default_options()
    bad.reserved[1] = 1
    assert lib._lib.lls_create(C.byref(h), C.byref(bad), None) == lib.LLS_ERR_ARG


def test_fast_option_with_a_bf16_sample_is_refused(lib):
    """nullify = 0 keeps T_12, which a BF16 sample leaves at BF16 size: the
    fast option is accepted with the FP64 sample only (argument 2)."""
    h = C.c_void_p()
    bad = lib.lls_default_options(nullify=0, precision=lib.LLS_MIXED_BF16)
    assert lib._lib.lls_create(C.byref(h), C.byref(bad), None) == lib.LLS_ERR_ARG


def test_barrier_limit_hook_accepts_and_restores(lib):
    assert lib._lib.lls_debug_barrier_limit(0) == lib.LLS_OK
    assert lib._lib.lls_debug_barrier_limit(-1) == lib.LLS_OK


def test_new_entry_points_reject_null_handle(lib):
    assert lib._lib.lls_factor_get(None, 0, 0, None, 1) == lib.LLS_ERR_ARG
    assert lib._lib.lls_refinement_info(None, None, None) == lib.LLS_ERR_ARG


def test_kernel_entry_points_reject_bad_sizes(lib):
    L = lib._lib
    assert L.lls_k_gemm(0, 0, 0, 0, -1, 1, 1, 1.0, None, 1, None, 1, 0.0, None, 1, None) == lib.LLS_ERR_ARG
    assert L.lls_k_gemm(0, 0, 0, 0, 4, 4, 4, 1.0, None, 3, None, 4, 0.0, None, 4, None) == lib.LLS_ERR_ARG
    assert L.lls_k_sketch(1, 0, 10, 2, None, 5, None) == lib.LLS_ERR_ARG
    assert L.lls_k_philox(1, -1, 2, 2, None, None) == lib.LLS_ERR_ARG
    assert L.lls_k_geqrf(10, 3, None, 5, None, None, 3, None) == lib.LLS_ERR_ARG
    assert L.lls_k_trsm_upper_blockinv(10, 17, None, 10, None, 10, 0, None) == lib.LLS_ERR_ARG
    assert L.lls_k_trsm_upper_blockinv(10, 2, None, 10, None, 10, 1, None) == lib.LLS_ERR_ARG
    assert L.lls_k_jacobi_svd(129, None, 129, None, None, 129, None, 129, None, None) == lib.LLS_ERR_ARG
    assert L.lls_k_trsm_upper(5, 1, None, 4, None, 5, None) == lib.LLS_ERR_ARG
    assert L.lls_k_rank(-1, None, 1, 0.0, None, None) == lib.LLS_ERR_ARG
    # zero-size problems are valid no-ops
    assert L.lls_k_geqrf(0, 3, None, 1, None, None, 1, None) == lib.LLS_OK
    assert L.lls_k_jacobi_svd(0, None, 1, None, None, 1, None, 1, None, None) == lib.LLS_OK
