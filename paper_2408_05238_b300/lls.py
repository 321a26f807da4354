"""ctypes binding of ``liblls.so`` (include/lls.h, include/lls_kernels.h).

Argument marshalling only: every numerical step runs in the CUDA library.
Device matrices are torch float64 CUDA tensors in column-major layout, i.e.
an (m, n) tensor with stride (1, ld) -- ``colmajor`` makes one.  If the
library has not been built, importing this module raises: there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblls.so")

LLS_OK = 0
LLS_PENDING = 1
LLS_WARN_RANK_NONPREFIX = 2
LLS_WARN_REFINE_NOCONV = 3
LLS_ERR_ARG = -1
LLS_ERR_NOMEM = -2
LLS_ERR_CUDA = -3
LLS_ERR_NONFINITE = -4
LLS_ERR_SVD_NOCONV = -5
LLS_ERR_TIMEOUT = -6
LLS_ERR_NOT_FOUND = -7
LLS_ERR_CAPACITY = -8
LLS_FP64 = 0
LLS_MIXED_BF16 = 1
LLS_MIXED_BF16_3xTF32 = 2
LLS_MIXED_BF16_TF32 = 3
LLS_FACTOR_T = 0
LLS_FACTOR_V = 1
LLS_BATCHED_AUTO = 0
LLS_BATCHED_WORKERS = 1
LLS_BATCHED_PERSISTENT = 2
LLS_OOC_FARTHEST = 0
LLS_OOC_LRU = 1


class lls_options(C.Structure):
    _fields_ = [("nb", C.c_int32), ("q", C.c_int32), ("precision", C.c_int32),
                ("nullify", C.c_int32), ("seed", C.c_uint64), ("explicit_v", C.c_int32),
                ("max_refine", C.c_int32), ("refine_tol", C.c_double),
                ("reserved", C.c_int32 * 2)]


class lls_problem(C.Structure):
    _fields_ = [("A", C.c_void_p), ("m", C.c_int64), ("n", C.c_int64), ("lda", C.c_int64),
                ("B", C.c_void_p), ("nrhs", C.c_int64), ("ldb", C.c_int64),
                ("tol", C.c_double), ("X", C.c_void_p), ("ldx", C.c_int64),
                ("rank_out", C.POINTER(C.c_int64)), ("factor_id", C.c_int64),
                ("keep_factor", C.c_int32), ("status", C.c_int32)]


class lls_trace_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("seconds", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


class lls_ooc_stats(C.Structure):
    _fields_ = [("panels", C.c_int64), ("passes", C.c_int64), ("accesses", C.c_int64),
                ("hits", C.c_int64), ("loads", C.c_int64), ("stores", C.c_int64),
                ("load_bytes", C.c_double), ("store_bytes", C.c_double),
                ("side_bytes", C.c_double)]


class lls_ooc_action(C.Structure):
    _fields_ = [("kind", C.c_int32), ("write", C.c_int32), ("step", C.c_int64),
                ("pass_", C.c_int64), ("panel", C.c_int64), ("slot", C.c_int64), ("evict", C.c_int64),
                ("store", C.c_int32), ("load", C.c_int32)]


class LLSError(RuntimeError):
    def __init__(self, status: int, arg: int = 0, msg: str = ""):
        self.status, self.arg, self.msg = status, arg, msg
        super().__init__(f"lls status {status} ({status_string(status)}), arg {arg}: {msg}")


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_2408_05238_b300.build` (no CPU fallback exists)")
_lib = C.CDLL(LIB_PATH)

_H = C.c_void_p
_P = C.c_void_p
_I = C.c_int64
_D = C.c_double


def _sig(name, args, res=C.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("lls_default_options", [C.POINTER(lls_options)])
_sig("lls_create", [C.POINTER(_H), C.POINTER(lls_options), _P])
_sig("lls_destroy", [_H])
_sig("lls_set_options", [_H, C.POINTER(lls_options)])
_sig("lls_solve", [_H, _P, _I, _I, _I, _P, _I, _I, _D, _P, _I, C.POINTER(_I)])
_sig("lls_solve_host", [_H, _P, _I, _I, _I, _P, _I, _I, _D, _P, _I, C.POINTER(_I)])
_sig("lls_factor", [_H, _P, _I, _I, _I, _D, C.POINTER(_I), C.POINTER(_I)])
_sig("lls_solve_factored", [_H, _I, _P, _I, _I, _P, _I])
_sig("lls_factor_release", [_H, _I])
_sig("lls_factor_diag", [_H, _I, _P, _I, C.POINTER(_I)])
_sig("lls_factor_get", [_H, _I, C.c_int32, _P, _I])
_sig("lls_refinement_info", [_H, C.POINTER(C.c_int32), C.POINTER(_D)])
_sig("lls_solve_batched", [_H, _I, C.POINTER(lls_problem)])
_sig("lls_submit", [_H, C.POINTER(lls_problem), C.POINTER(_I)])
_sig("lls_poll", [_H, _I, C.POINTER(C.c_int)])
_sig("lls_set_memory_cap", [_H, _I])
_sig("lls_ticket_factor", [_H, _I, C.POINTER(_I)])
_sig("lls_set_workers", [_H, C.c_int])
_sig("lls_set_batched_mode", [_H, C.c_int])
_sig("lls_cancel", [_H, _I])
_sig("lls_debug_fail_allocation", [_I])
_sig("lls_debug_barrier_limit", [_I])
_sig("lls_debug_guard", [C.c_int])
_sig("lls_debug_guard_report", [C.c_char_p, _I], C.c_int64)
_sig("lls_debug_guard_selftest", [])
_sig("lls_autotune", [_H, _I, _I, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)])
_sig("lls_tuning_lookup", [_H, _I, _I, C.POINTER(C.c_int32), C.POINTER(C.c_int32)])
_sig("lls_tuning_save", [_H, C.c_char_p])
_sig("lls_tuning_load", [_H, C.c_char_p])
_sig("lls_status_string", [C.c_int], C.c_char_p)
_sig("lls_last_error", [_H, C.POINTER(C.c_int), C.c_char_p, _I])
_sig("lls_trace_enable", [_H, C.c_int])
_sig("lls_trace_read", [_H, C.POINTER(lls_trace_stat), _I, C.POINTER(_I)])
_sig("lls_launch_count", [], C.c_int64)
_sig("lls_ooc_plan", [_I, _I, C.c_int32, C.c_int32, _I, C.c_int32, _I, C.c_int32,
                      C.POINTER(lls_ooc_stats)])
_sig("lls_ooc_schedule", [_I, _I, C.c_int32, C.c_int32, _I, C.c_int32, _I, C.c_int32,
                          C.c_int32, C.POINTER(lls_ooc_action), _I, C.POINTER(_I)])
_sig("lls_solve_ooc", [_H, _P, _I, _I, _I, _P, _I, _I, _D, _P, _I, C.POINTER(_I), _I, C.c_int32])
_sig("lls_ooc_simulate", [C.POINTER(_I), C.POINTER(C.c_int8), _I, _I, _I, _I, _I, C.c_int32,
                          C.POINTER(lls_ooc_stats)])
_sig("lls_alloc_count", [], C.c_int64)
_sig("lls_k_philox", [C.c_uint64, _I, _I, _I, _P, _P])
_sig("lls_k_sketch", [C.c_uint64, _I, _I, _I, _P, _I, _P])
_sig("lls_k_gemm", [C.c_int, C.c_int, C.c_int, C.c_int, _I, _I, _I, _D, _P, _I, _P, _I, _D, _P,
                    _I, _P])
_sig("lls_k_geqrf", [_I, _I, _P, _I, _P, _P, _I, _P])
_sig("lls_k_jacobi_svd", [_I, _P, _I, _P, _P, _I, _P, _I, _P, _P])
_sig("lls_k_trsm_upper", [_I, _I, _P, _I, _P, _I, _P])
_sig("lls_k_rank", [_I, _P, _I, _D, _P, _P])
_sig("lls_k_gemm_bf16_tn", [_I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _P])
_sig("lls_k_gemm_oz", [C.c_int, C.c_int, C.c_int, C.c_int, _I, _I, _I, _D, _P, _I, _P, _I, _D,
                       _P, _I, _P, _P])
_sig("lls_k_panel_qr_noalloc", [_I, _I, _P, _I, _P, _P, _P])
_sig("lls_k_gemm_tf32", [C.c_int, C.c_int, C.c_int, C.c_int, _I, _I, _I, _D, _P, _I, _P, _I, _D,
                         _P, _I, C.c_int, _P, _P])
_sig("lls_k_trsm_upper_trans", [_I, _I, _P, _I, _P, _I, _P])
_sig("lls_k_trsm_upper_blockinv", [_I, _I, _P, _I, _P, _I, _I, _P])

EXPORTED = [n for n in dir(_lib) if n.startswith("lls_")]


def status_string(status: int) -> str:
    return _lib.lls_status_string(int(status)).decode()


# --------------------------------------------------------------------------- helpers
def colmajor(t: torch.Tensor) -> torch.Tensor:
    """Column-major (m, n) copy/view of a 2-D tensor (stride (1, m))."""
    if t.dim() == 1:
        t = t[:, None]
    if t.stride(0) == 1 and (t.shape[1] <= 1 or t.stride(1) >= max(1, t.shape[0])):
        return t
    return t.t().contiguous().t()


def empty_colmajor(m: int, n: int, device="cuda", dtype=torch.float64) -> torch.Tensor:
    return torch.empty((n, max(m, 1)), device=device, dtype=dtype).t()[:m]


def _ld(t: torch.Tensor) -> int:
    return max(1, t.stride(1) if t.shape[1] > 1 else t.shape[0])


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check(h, code: int):
    if code < 0:
        arg = C.c_int(0)
        buf = C.create_string_buffer(512)
        if h is not None:
            _lib.lls_last_error(h, C.byref(arg), buf, 512)
        raise LLSError(code, arg.value, buf.value.decode(errors="replace"))
    return code


# --------------------------------------------------------------------------- handle API
def lls_default_options(**kw) -> lls_options:
    o = lls_options()
    _lib.lls_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def lls_create(options: lls_options | None = None, stream=None, **kw):
    """Handle on torch's current device, borrowing ``stream`` (default: the
    current torch stream)."""
    o = options if options is not None else lls_default_options(**kw)
    h = _H()
    _check(None, _lib.lls_create(C.byref(h), C.byref(o), _stream(stream)))
    return h


def lls_destroy(h):
    _check(None, _lib.lls_destroy(h))


def lls_set_options(h, options: lls_options | None = None, **kw):
    o = options if options is not None else lls_default_options(**kw)
    _check(h, _lib.lls_set_options(h, C.byref(o)))


def lls_solve(h, A: torch.Tensor, B: torch.Tensor, tol: float, X: torch.Tensor | None = None):
    """X = argmin ||A X - B|| with minimum norm; returns (X, rank, status)."""
    m, n = A.shape
    Bm = B if B.dim() == 2 else B[:, None]
    nrhs = Bm.shape[1]
    if X is None:
        X = empty_colmajor(n, nrhs, device=A.device)
    rank = _I(0)
    code = _check(h, _lib.lls_solve(h, _ptr(A), m, n, _ld(A), _ptr(Bm), nrhs, _ld(Bm), float(tol),
                                    _ptr(X), _ld(X), C.byref(rank)))
    return X, rank.value, code


def lls_solve_host(h, A, B, tol: float, X=None):
    """Host-memory variant (numpy or CPU torch, column-major float64)."""
    import numpy as np

    A = np.asfortranarray(A, dtype=np.float64)
    B2 = np.asfortranarray(B if np.ndim(B) == 2 else np.reshape(B, (-1, 1)), dtype=np.float64)
    m, n = A.shape
    nrhs = B2.shape[1]
    if X is None:
        X = np.zeros((n, nrhs), order="F")
    rank = _I(0)
    code = _check(h, _lib.lls_solve_host(h, A.ctypes.data, m, n, max(1, m), B2.ctypes.data, nrhs,
                                         max(1, m), float(tol), X.ctypes.data, max(1, n),
                                         C.byref(rank)))
    return X, rank.value, code


def lls_solve_host_ptr(h, A_ptr: int, m: int, n: int, B_ptr: int, nrhs: int, tol: float,
                       X_ptr: int):
    """Host-pointer variant for pinned buffers (column-major, ld = rows)."""
    rank = _I(0)
    code = _check(h, _lib.lls_solve_host(h, C.c_void_p(A_ptr), m, n, max(1, m), C.c_void_p(B_ptr),
                                         nrhs, max(1, m), float(tol), C.c_void_p(X_ptr), max(1, n),
                                         C.byref(rank)))
    return rank.value, code


def lls_factor(h, A: torch.Tensor, tol: float):
    m, n = A.shape
    fid, rank = _I(0), _I(0)
    code = _check(h, _lib.lls_factor(h, _ptr(A), m, n, _ld(A), float(tol), C.byref(fid),
                                     C.byref(rank)))
    return fid.value, rank.value, code


def lls_solve_factored(h, factor_id: int, B: torch.Tensor, n: int, X=None):
    Bm = B if B.dim() == 2 else B[:, None]
    nrhs = Bm.shape[1]
    if X is None:
        X = empty_colmajor(n, nrhs, device=B.device)
    _check(h, _lib.lls_solve_factored(h, factor_id, _ptr(Bm), nrhs, _ld(Bm), _ptr(X), _ld(X)))
    return X


def lls_factor_release(h, factor_id: int):
    _check(h, _lib.lls_factor_release(h, factor_id))


def lls_factor_diag(h, factor_id: int, length: int):
    import numpy as np

    d = np.zeros(max(length, 1))
    cnt = _I(0)
    _check(h, _lib.lls_factor_diag(h, factor_id, d.ctypes.data, length, C.byref(cnt)))
    return d[:length], cnt.value


def lls_factor_get(h, factor_id: int, which: int, rows: int, cols: int) -> torch.Tensor:
    """T (which = LLS_FACTOR_T, rows x cols = m x n) or V (LLS_FACTOR_V, n x n)
    of a resident factor as a new column-major CUDA tensor."""
    out = empty_colmajor(rows, cols)
    _check(h, _lib.lls_factor_get(h, factor_id, int(which), _ptr(out), max(1, rows)))
    return out


def lls_refinement_info(h) -> tuple[int, float]:
    """(steps, last correction) of the last solve's iterative refinement."""
    steps, corr = C.c_int32(0), _D(0.0)
    _check(h, _lib.lls_refinement_info(h, C.byref(steps), C.byref(corr)))
    return steps.value, corr.value


def make_problem(A, B, tol, X, factor_id=-1, keep_factor=0, rank_out=None) -> lls_problem:
    p = lls_problem()
    m, n = (A.shape if A is not None else (B.shape[0], X.shape[0]))
    Bm = B if B.dim() == 2 else B[:, None]
    p.A = A.data_ptr() if A is not None else None
    p.m, p.n = m, n
    p.lda = _ld(A) if A is not None else max(1, m)
    p.B, p.nrhs, p.ldb = Bm.data_ptr(), Bm.shape[1], _ld(Bm)
    p.tol = float(tol)
    p.X, p.ldx = X.data_ptr(), _ld(X)
    p.rank_out = rank_out if rank_out is not None else C.POINTER(_I)()
    p.factor_id, p.keep_factor, p.status = factor_id, keep_factor, 0
    return p


def lls_solve_batched(h, problems: list[lls_problem]) -> int:
    arr = (lls_problem * len(problems))(*problems)
    code = _lib.lls_solve_batched(h, len(problems), arr)
    for i, p in enumerate(problems):
        p.status = arr[i].status
        p.factor_id = arr[i].factor_id
    if code < 0:
        _check(h, code)
    return code


def lls_submit(h, problem: lls_problem) -> int:
    t = _I(0)
    _check(h, _lib.lls_submit(h, C.byref(problem), C.byref(t)))
    return t.value


def lls_poll(h, ticket: int) -> int:
    s = C.c_int(0)
    _check(h, _lib.lls_poll(h, ticket, C.byref(s)))
    return s.value


def lls_set_memory_cap(h, nbytes: int):
    _check(h, _lib.lls_set_memory_cap(h, int(nbytes)))


def lls_ticket_factor(h, ticket: int):
    """Factor id of a finished keep_factor request, or None while pending."""
    f = _I(-1)
    code = _check(h, _lib.lls_ticket_factor(h, ticket, C.byref(f)))
    return None if code == LLS_PENDING else f.value


def lls_set_workers(h, workers: int):
    _check(h, _lib.lls_set_workers(h, int(workers)))


def lls_set_batched_mode(h, mode: int):
    _check(h, _lib.lls_set_batched_mode(h, int(mode)))


def lls_cancel(h, ticket: int) -> int:
    """Withdraw a request that has not started (LLS_OK) or LLS_ERR_NOT_FOUND."""
    return int(_lib.lls_cancel(h, ticket))


def lls_debug_fail_allocation(after: int):
    """Testing hook: the (after + 1)-th workspace allocation fails; -1 = off."""
    _check(None, _lib.lls_debug_fail_allocation(after))


def lls_ooc_plan(m: int, n: int, nb: int, q: int, rank: int, nullify: int, cache_panels: int,
                 policy: int = LLS_OOC_FARTHEST) -> dict:
    """Host<->device panel traffic of an out-of-core solve (lls_ooc_plan)."""
    st = lls_ooc_stats()
    _check(None, _lib.lls_ooc_plan(m, n, nb, q, rank, nullify, cache_panels, policy, C.byref(st)))
    return {k: getattr(st, k) for k, _ in lls_ooc_stats._fields_}


OOC_KINDS = ["sample_atg", "sample_ay", "sample_atw_ay", "sample_atw", "product_twv", "update",
             "svd", "null_gather", "null_read", "null_write", "solve_utb", "solve_trsm", "flush"]


def lls_ooc_schedule(m: int, n: int, nb: int, q: int, rank: int, nullify: int, cache_panels: int,
                     policy: int = LLS_OOC_FARTHEST, phase: int = 0) -> list[dict]:
    """The planned access list with cache slots, loads and write-backs."""
    cnt = _I(0)
    _check(None, _lib.lls_ooc_schedule(m, n, nb, q, rank, nullify, cache_panels, policy, phase,
                                       None, 0, C.byref(cnt)))
    arr = (lls_ooc_action * max(cnt.value, 1))()
    _check(None, _lib.lls_ooc_schedule(m, n, nb, q, rank, nullify, cache_panels, policy, phase,
                                       arr, cnt.value, C.byref(cnt)))
    names = [f for f, _ in lls_ooc_action._fields_]
    out = []
    for a in arr[:cnt.value]:
        d = {f: getattr(a, f) for f in names}
        d["kind"] = OOC_KINDS[d["kind"]]
        out.append(d)
    return out


def lls_solve_ooc(h, A, B, tol: float, cache_panels: int, policy: int = LLS_OOC_FARTHEST):
    """Out-of-core solve of host arrays (numpy, float64): returns (X, rank, status)."""
    import numpy as np

    A = np.asfortranarray(A, dtype=np.float64)
    B2 = np.asfortranarray(B if np.ndim(B) == 2 else np.reshape(B, (-1, 1)), dtype=np.float64)
    m, n = A.shape
    nrhs = B2.shape[1]
    X = np.zeros((n, nrhs), order="F")
    rank = _I(0)
    code = _check(h, _lib.lls_solve_ooc(h, A.ctypes.data, m, n, max(1, m), B2.ctypes.data, nrhs,
                                        max(1, m), float(tol), X.ctypes.data, max(1, n),
                                        C.byref(rank), int(cache_panels), int(policy)))
    return X, rank.value, code


def lls_ooc_simulate(panels, writes=None, num_panels: int | None = None, rows: int = 1,
                     cols: int = 1, cache_panels: int = 1, policy: int = LLS_OOC_FARTHEST) -> dict:
    """The planner's cache over an arbitrary panel access list (lls_ooc_simulate)."""
    n = len(panels)
    pa = (_I * max(n, 1))(*panels)
    wa = (C.c_int8 * max(n, 1))(*([1 if w else 0 for w in writes] if writes is not None else []))
    if num_panels is None:
        num_panels = (max(panels) + 1) if n else 1
    st = lls_ooc_stats()
    _check(None, _lib.lls_ooc_simulate(pa, wa if writes is not None else None, n, num_panels, rows,
                                       cols, cache_panels, policy, C.byref(st)))
    return {k: getattr(st, k) for k, _ in lls_ooc_stats._fields_}


def lls_debug_barrier_limit(polls: int):
    """Grid-barrier poll limit of the cooperative panel kernels (< 0: default)."""
    _kcheck(_lib.lls_debug_barrier_limit(int(polls)))


def lls_debug_guard(on: bool):
    """Guard words around every buffer allocated from now on, checked after
    every launch (debug mode)."""
    _check(None, _lib.lls_debug_guard(1 if on else 0))


def lls_debug_guard_report() -> tuple[int, str]:
    """(violations since the mode was turned on, the first one's description)."""
    buf = C.create_string_buffer(512)
    n = _lib.lls_debug_guard_report(buf, 512)
    return int(n), buf.value.decode(errors="replace")


def lls_debug_guard_selftest() -> int:
    return int(_lib.lls_debug_guard_selftest())


def lls_autotune(h, m: int, n: int, trials: int = 2) -> tuple[int, int]:
    """Time n_b x q candidates on a synthetic m x n matrix; returns the (n_b, q)
    stored for the (m, n) bucket (lls_autotune)."""
    nb, q = C.c_int32(0), C.c_int32(0)
    _check(h, _lib.lls_autotune(h, m, n, int(trials), C.byref(nb), C.byref(q)))
    return nb.value, q.value


def lls_tuning_lookup(h, m: int, n: int) -> tuple[int, int]:
    nb, q = C.c_int32(0), C.c_int32(0)
    _check(h, _lib.lls_tuning_lookup(h, m, n, C.byref(nb), C.byref(q)))
    return nb.value, q.value


def lls_tuning_save(h, path: str):
    _check(h, _lib.lls_tuning_save(h, os.fsencode(path)))


def lls_tuning_load(h, path: str):
    _check(h, _lib.lls_tuning_load(h, os.fsencode(path)))


def lls_trace_enable(h, on: bool = True):
    _check(h, _lib.lls_trace_enable(h, int(on)))


def lls_trace_read(h) -> dict:
    """{kernel family: (launches, seconds, flops, bytes)} since tracing was enabled."""
    arr = (lls_trace_stat * 32)()
    cnt = _I(0)
    _check(h, _lib.lls_trace_read(h, arr, 32, C.byref(cnt)))
    return {arr[i].name.decode(): (arr[i].launches, arr[i].seconds, arr[i].flops, arr[i].bytes)
            for i in range(min(cnt.value, 32))}


def lls_launch_count() -> int:
    return int(_lib.lls_launch_count())


def lls_alloc_count() -> int:
    return int(_lib.lls_alloc_count())


# --------------------------------------------------------------------------- step-level API
def _kcheck(code):
    if code != LLS_OK:
        raise LLSError(code)


def lls_k_philox(seed: int, step: int, groups: int, cols: int) -> torch.Tensor:
    out = torch.zeros(groups * cols * 4, dtype=torch.int64, device="cuda")
    _kcheck(_lib.lls_k_philox(seed, step, groups, cols, _ptr(out), _stream()))
    return out


def lls_k_sketch(seed: int, step: int, rows: int, cols: int) -> torch.Tensor:
    G = empty_colmajor(rows, cols)
    _kcheck(_lib.lls_k_sketch(seed, step, rows, cols, _ptr(G), max(1, rows), _stream()))
    return G


def lls_k_gemm(transa, transb, A, B, C_=None, alpha=1.0, beta=0.0, unit_lower_a=False,
               unit_lower_b=False):
    m = A.shape[1] if transa else A.shape[0]
    k = A.shape[0] if transa else A.shape[1]
    n = B.shape[0] if transb else B.shape[1]
    if C_ is None:
        C_ = torch.zeros((n, max(m, 1)), dtype=torch.float64, device=A.device).t()[:m]
    _kcheck(_lib.lls_k_gemm(int(transa), int(transb), int(unit_lower_a), int(unit_lower_b), m, n,
                            k, float(alpha), _ptr(A), _ld(A), _ptr(B), _ld(B), float(beta),
                            _ptr(C_), _ld(C_), _stream()))
    return C_


def lls_k_geqrf(A: torch.Tensor):
    """In-place Householder QR; returns (A, tau, T)."""
    m, n = A.shape
    k = min(m, n)
    tau = torch.zeros(max(k, 1), dtype=torch.float64, device=A.device)
    T = empty_colmajor(max(k, 1), max(k, 1))
    _kcheck(_lib.lls_k_geqrf(m, n, _ptr(A), _ld(A), _ptr(tau), _ptr(T), max(1, k), _stream()))
    return A, tau[:k], T[:k, :k]


def lls_k_jacobi_svd(R: torch.Tensor):
    b = R.shape[0]
    sigma = torch.zeros(max(b, 1), dtype=torch.float64, device=R.device)
    Us = empty_colmajor(b, b)
    Vs = empty_colmajor(b, b)
    st = torch.zeros(1, dtype=torch.int32, device=R.device)
    _kcheck(_lib.lls_k_jacobi_svd(b, _ptr(R), _ld(R), _ptr(sigma), _ptr(Us), max(1, b), _ptr(Vs),
                                  max(1, b), _ptr(st), _stream()))
    return sigma[:b], Us, Vs, int(st.item())


def lls_k_trsm_upper(R: torch.Tensor, B: torch.Tensor):
    r = R.shape[0]
    _kcheck(_lib.lls_k_trsm_upper(r, B.shape[1], _ptr(R), _ld(R), _ptr(B), _ld(B), _stream()))
    return B


def lls_k_trsm_upper_trans(R: torch.Tensor, B: torch.Tensor):
    r = R.shape[0]
    _kcheck(_lib.lls_k_trsm_upper_trans(r, B.shape[1], _ptr(R), _ld(R), _ptr(B), _ld(B),
                                        _stream()))
    return B


def lls_k_trsm_upper_blockinv(R: torch.Tensor, B: torch.Tensor, trans: bool = False):
    r = R.shape[0]
    _kcheck(_lib.lls_k_trsm_upper_blockinv(r, B.shape[1], _ptr(R), _ld(R), _ptr(B), _ld(B),
                                           int(trans), _stream()))
    return B


def lls_k_rank(T: torch.Tensor, tol: float):
    out = torch.zeros(3, dtype=torch.int64, device=T.device)
    length = min(T.shape)
    _kcheck(_lib.lls_k_rank(length, _ptr(T), _ld(T), float(tol), _ptr(out), _stream()))
    return tuple(int(v) for v in out.cpu())


def lls_k_gemm_bf16_tn(X: torch.Tensor, Z: torch.Tensor):
    """D = X^T Z (FP32) with X (K x M) and Z (K x N) column-major bf16."""
    K, M = X.shape
    N = Z.shape[1]
    D = torch.zeros((N, max(M, 1)), dtype=torch.float32, device=X.device).t()[:M]
    status = torch.zeros(1, dtype=torch.int32, device=X.device)
    _kcheck(_lib.lls_k_gemm_bf16_tn(M, N, K, _ptr(X), _ld(X), _ptr(Z), _ld(Z), _ptr(D), max(1, M),
                                    _ptr(status), _stream()))
    return D, int(status.item())


def lls_k_gemm_oz(transa, transb, A, B, C_=None, alpha=1.0, beta=0.0, unit_lower_a=False,
                  unit_lower_b=False):
    """FP64 GEMM on the tensor cores by exact BF16 slicing (lls_k_gemm_oz)."""
    m = A.shape[1] if transa else A.shape[0]
    k = A.shape[0] if transa else A.shape[1]
    n = B.shape[0] if transb else B.shape[1]
    if C_ is None:
        C_ = torch.zeros((n, max(m, 1)), dtype=torch.float64, device=A.device).t()[:m]
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _kcheck(_lib.lls_k_gemm_oz(int(transa), int(transb), int(unit_lower_a), int(unit_lower_b), m,
                               n, k, float(alpha), _ptr(A), _ld(A), _ptr(B), _ld(B), float(beta),
                               _ptr(C_), _ld(C_), _ptr(status), _stream()))
    return C_, int(status.item())


def lls_k_gemm_tf32(transa, transb, A, B, C_=None, alpha=1.0, beta=0.0, unit_lower_a=False,
                    unit_lower_b=False, terms=3):
    """FP64-operand GEMM on the TF32 tensor cores with split operands
    (lls_k_gemm_tf32; terms = 3: 3xTF32, 1: plain TF32)."""
    m = A.shape[1] if transa else A.shape[0]
    k = A.shape[0] if transa else A.shape[1]
    n = B.shape[0] if transb else B.shape[1]
    if C_ is None:
        C_ = torch.zeros((n, max(m, 1)), dtype=torch.float64, device=A.device).t()[:m]
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _kcheck(_lib.lls_k_gemm_tf32(int(transa), int(transb), int(unit_lower_a), int(unit_lower_b), m,
                                 n, k, float(alpha), _ptr(A), _ld(A), _ptr(B), _ld(B), float(beta),
                                 _ptr(C_), _ld(C_), int(terms), _ptr(status), _stream()))
    return C_, int(status.item())


def lls_k_panel_qr_noalloc(A: torch.Tensor, tau: torch.Tensor, status: torch.Tensor) -> int:
    """Panel QR of A in place using the library's fixed scratch (no device
    allocation inside the call); returns the status code of the call."""
    m, n = A.shape
    return int(_lib.lls_k_panel_qr_noalloc(m, n, _ptr(A), _ld(A), _ptr(tau), _ptr(status),
                                           _stream()))
