"""The out-of-core schedule (lls_ooc_schedule) carries a whole solve.

A streamed randUTV solve is run here in numpy, following the library's
schedule action by action: a "host store" holds every column panel, a
"device cache" holds min(cache, panels) slots, panels move only through the
schedule's loads and write-backs, and every step of the method touches panel
data only through the slot the schedule names for that access.  The
arithmetic of each step is the oracle's (its sketch, Householder QR, compact
WY factors and SVD), so the result must match the in-core oracle: T after the
block-SVD pass to rounding, the rank exactly, and x to 1e-9.  A schedule that
forgot a load, a write-back or a needed visit, or ordered two passes wrongly,
fails this test.
"""

import numpy as np
import pytest
import scipy.linalg

from oracle import randutv_oracle as orc
from paper_2408_05238_b300 import workloads as wl

FAR, LRU = 0, 1


@pytest.fixture(scope="module")
def lls():
    from paper_2408_05238_b300 import build

    build.build()
    from paper_2408_05238_b300 import lls as binding

    return binding


class StreamedSolve:
    """Executes a schedule on a host store and a slot cache (numpy)."""

    def __init__(self, A, B, nb, q, tol, seed, nullify, cache, policy, lls):
        self.m, self.n = A.shape
        self.nb, self.q, self.seed, self.tol, self.nullify = nb, q, seed, tol, nullify
        self.B = np.array(B, dtype=np.float64).reshape(self.m, -1)
        m, n = self.m, self.n
        self.P = -(-n // nb)
        self.steps = -(-min(m, n) // nb)
        self.host = [np.array(A[:, self.c0(j):self.c1(j)], dtype=np.float64) for j in range(self.P)]
        self.slots = {}
        self.resident = {}          # panel -> slot, for the T snapshot only
        self.cache, self.policy, self.lls = cache, policy, lls
        # side state that a device executor keeps outside the panel cache
        self.WV, self.TV, self.WU, self.TU, self.R11 = {}, {}, {}, {}, {}
        self.sigma, self.Us, self.Vs = {}, {}, {}
        self.rz = []
        self.pass_key = None
        self.rank_for_plan = self.r = None

    # panel geometry ---------------------------------------------------------
    def c0(self, j):
        return j * self.nb

    def c1(self, j):
        return min(self.n, (j + 1) * self.nb)

    def kb(self, i):
        k = i * self.nb
        return k, min(self.nb, self.m - k, self.n - k)

    def snapshot(self):
        """The current T: host store overlaid with the resident slots."""
        cols = [self.host[j].copy() for j in range(self.P)]
        for j, s in self.resident.items():
            cols[j] = self.slots[s].copy()
        return np.concatenate(cols, axis=1)

    # driver -----------------------------------------------------------------
    def run(self, phases=(0,)):
        sched = []
        for ph in phases:
            part = self.lls.lls_ooc_schedule(self.m, self.n, self.nb, self.q, self.rank_for_plan,
                                             self.nullify, self.cache, self.policy, ph)
            if ph == 1:   # ends with every modified panel written back: the cache starts empty
                part.append({"kind": "drop"})
            sched += part
        self.max_slot = max([a.get("slot", -1) for a in sched], default=-1)
        self.T_after_svd = None
        for a in sched:
            if a["kind"] == "drop":
                self.slots, self.resident = {}, {}
                continue
            if self.pass_key and self.pass_key[0] == "svd" and a["kind"] != "svd":
                self.T_after_svd = self.snapshot()
            if a["evict"] >= 0 and a["kind"] != "flush":
                if a["store"]:
                    self.host[a["evict"]] = self.slots[a["slot"]].copy()
                self.slots[a["slot"]] = None
                del self.resident[a["evict"]]
            if a["kind"] == "flush":
                self.host[a["panel"]] = self.slots[a["slot"]].copy()
                continue
            if a["load"]:
                assert self.slots.get(a["slot"]) is None, "load into an occupied slot"
                self.slots[a["slot"]] = self.host[a["panel"]].copy()
                self.resident[a["panel"]] = a["slot"]
            assert self.resident.get(a["panel"]) == a["slot"], "panel not in its slot"
            key = (a["kind"], a["pass_"])
            first = key != self.pass_key
            self.pass_key = key
            before = None if a["write"] else self.slots[a["slot"]].copy()
            getattr(self, "op_" + a["kind"])(a["step"], a["panel"], self.slots[a["slot"]], first)
            if before is not None:   # an access planned as a read must not modify the panel
                assert np.array_equal(before, self.slots[a["slot"]]), a
        if self.T_after_svd is None:
            self.T_after_svd = self.snapshot()
        return sched

    # sampling and the P pass (step i, panel j >= i; A_j = T(k:m, panel j)) ----
    def y_rows(self, i, j):
        k, _ = self.kb(i)
        return slice(self.c0(j) - k, self.c1(j) - k)

    def op_sample_atg(self, i, j, X, first):
        k, b = self.kb(i)
        if first:
            self.G = orc.sketch_matrix(self.seed, i, self.m - k, b)
            self.Y = np.zeros((self.n - k, b))
        self.Y[self.y_rows(i, j)] = X[k:].T @ self.G

    def op_sample_ay(self, i, j, X, first):
        k, b = self.kb(i)
        if first:
            self.W = np.zeros((self.m - k, b))
        self.W += X[k:] @ self.Y[self.y_rows(i, j)]

    def op_sample_atw_ay(self, i, j, X, first):
        k, b = self.kb(i)
        if first:
            self.W_prev, self.W = self.W, np.zeros((self.m - k, b))
        rows = self.y_rows(i, j)
        self.Y[rows] = X[k:].T @ self.W_prev
        self.W += X[k:] @ self.Y[rows]

    def op_sample_atw(self, i, j, X, first):
        k, _ = self.kb(i)
        self.Y[self.y_rows(i, j)] = X[k:].T @ self.W

    def op_product_twv(self, i, j, X, first):
        k, b = self.kb(i)
        if first:
            _, self.WV[i], tau = orc.householder_qr(self.Y)
            self.TV[i] = orc.wy_factor(self.WV[i], tau)
            self.Pm = np.zeros((self.m, b))
        self.Pm += X @ self.WV[i][self.y_rows(i, j)]

    # update pass: right update; panel QR (j = i) or left update; next A_j^T G
    def left_update(self, i, Xs):
        W, Tu = self.WU[i], self.TU[i]
        Xs -= W @ (Tu.T @ (W.T @ Xs))

    def op_update(self, i, j, X, first):
        k, b = self.kb(i)
        nxt = i + 1 < self.steps
        if first:
            self.P2 = self.Pm @ self.TV[i]
            if nxt:
                k2, b2 = self.kb(i + 1)
                self.G = orc.sketch_matrix(self.seed, i + 1, self.m - k2, b2)
                self.Ynext = np.zeros((self.n - k2, b2))
        X -= self.P2 @ self.WV[i][self.y_rows(i, j)].T            # all m rows
        if j == i:
            R11, W, tau = orc.householder_qr(X[k:, :b])
            self.WU[i], self.TU[i], self.R11[i] = W, orc.wy_factor(W, tau), R11
            # R above the diagonal, W_U's vectors below it (the device layout)
            X[k:, :b] = np.tril(W, -1)
            X[k:k + b, :b] += R11
            if X.shape[1] > b:                                    # a narrow last step
                self.left_update(i, X[k:, b:])
        else:
            self.left_update(i, X[k:])
        if nxt and j >= i + 1:
            k2, _ = self.kb(i + 1)
            self.Ynext[self.y_rows(i + 1, j)] = X[k2:].T @ self.G
        if nxt and j == self.P - 1:
            self.Y = self.Ynext

    # block SVDs and their updates (one pass over every panel) ----------------
    def op_svd(self, _, j, X, first):
        if first:
            for i in range(self.steps):
                U, s, Vt = np.linalg.svd(self.R11[i])
                self.Us[i], self.sigma[i], self.Vs[i] = U, s, Vt.T
            self.rank, self.rank_count = orc.compute_rank(
                np.diag(np.concatenate([self.sigma[i] for i in range(self.steps)])), self.tol)
        if j < self.steps:
            k, b = self.kb(j)
            X[:k, :b] = X[:k, :b] @ self.Vs[j]
            X[k:k + b, :b] = np.tril(X[k:k + b, :b], -1) + np.diag(self.sigma[j])
            if X.shape[1] > b:
                X[k:k + b, b:] = self.Us[j].T @ X[k:k + b, b:]
        for i in range(min(j, self.steps)):
            k, b = self.kb(i)
            X[k:k + b] = self.Us[i].T @ X[k:k + b]

    # Nullify, panel-aligned row blocks p from the bottom ---------------------
    def block(self, p):
        j0 = p * self.nb
        return j0, min(self.r, j0 + self.nb)

    def d_cols(self, j):
        """Columns of panel j that belong to D = T(0:r, r:n): local slice and D columns."""
        lo = max(self.c0(j), self.r)
        return slice(lo - self.c0(j), self.c1(j) - self.c0(j)), slice(lo - self.r, self.c1(j) - self.r)

    def op_null_gather(self, p, j, X, first):
        j0, j1 = self.block(p)
        if first:
            self.D1 = np.zeros((j1 - j0, self.n - self.r))
        loc, dc = self.d_cols(j)
        self.D1[:, dc] = X[j0:j1, loc]

    def op_null_read(self, p, j, X, first):
        j0, j1 = self.block(p)
        bsz = j1 - j0
        if first:
            assert j == p
            C11 = np.triu(X[j0:j1, :bsz])            # W_U's vectors sit below it
            M = np.vstack([C11[::-1, ::-1].T, self.D1[::-1, :].T])
            R, Wz, tau = orc.householder_qr(M)
            assert np.array_equal(Wz[:bsz], np.eye(bsz))
            self.cur = dict(j0=j0, bsz=bsz, R=R, Wbot=Wz[bsz:], Tz=orc.wy_factor(Wz, tau))
            self.rz.append(self.cur)
            self.Pacc = X[:j0, :bsz][:, ::-1].copy()  # [C_01 reversed] W_top, W_top = I
        if j >= self.r // self.nb:                    # D's part of this panel
            loc, dc = self.d_cols(j)
            self.Pacc += X[:j0, loc] @ self.cur["Wbot"][dc]

    def op_null_write(self, p, j, X, first):
        j0, j1 = self.block(p)
        bsz = j1 - j0
        if first:
            self.P2 = self.Pacc @ self.cur["Tz"]
            if p > 0:
                self.D1_next = np.zeros((self.nb, self.n - self.r))
        if j >= self.r // self.nb:
            loc, dc = self.d_cols(j)
            X[:j0, loc] -= self.P2 @ self.cur["Wbot"][dc].T
            X[j0:j1, loc] = 0.0
            if p > 0:
                self.D1_next[:, dc] = X[j0 - self.nb:j0, loc]
        if j == p:
            C01rev = X[:j0, :bsz][:, ::-1] - self.P2
            X[:j0, :bsz] = C01rev[:, ::-1]
            X[j0:j1, :bsz] = np.triu(self.cur["R"][::-1, ::-1].T) + np.tril(X[j0:j1, :bsz], -1)
            if p > 0:
                self.D1 = self.D1_next

    # solve: U^T b, then T_11^{-1} by panels from the right -------------------
    def op_solve_utb(self, _, i, X, first):
        if first:
            self.c = self.B.copy()
        k, b = self.kb(i)
        W = np.tril(X[k:, :b], -1)
        W[np.arange(b), np.arange(b)] = 1.0
        self.c[k:] -= W @ (self.TU[i].T @ (W.T @ self.c[k:]))
        self.c[k:k + b] = self.Us[i].T @ self.c[k:k + b]

    def op_solve_trsm(self, _, p, X, first):
        if first:
            self.y = self.c[:self.r].copy()
        c0, c1 = self.c0(p), min(self.c1(p), self.r)
        self.y[c0:c1] = scipy.linalg.solve_triangular(np.triu(X[c0:c1, :c1 - c0]), self.y[c0:c1])
        self.y[:c0] -= X[:c0, :c1 - c0] @ self.y[c0:c1]

    def solution(self):
        """x = V Z [y; 0]: Nullify's reflectors (last block first), then V."""
        z = np.zeros((self.n, self.B.shape[1]))
        if self.r == 0:
            return z
        z[:self.r] = self.y
        for blk in reversed(self.rz):
            j0, bsz, Wb, Tz = blk["j0"], blk["bsz"], blk["Wbot"], blk["Tz"]
            zc = z[j0:j0 + bsz][::-1].copy()
            p2 = Tz @ (zc + Wb.T @ z[self.r:])
            zc -= p2
            z[self.r:] -= Wb @ p2
            z[j0:j0 + bsz] = zc[::-1]
        for i in reversed(range(self.steps)):
            k, b = self.kb(i)
            z[k:k + b] = self.Vs[i] @ z[k:k + b]
            z[k:] -= self.WV[i] @ (self.TV[i] @ (self.WV[i].T @ z[k:]))
        return z


CASES = [  # input, m, n, r, nb, q, nullify, cache panels, policy
    ("xy", 150, 100, 40, 16, 1, 1, 3, FAR),     # tall; D starts inside the last block's panel
    ("xy", 100, 150, 40, 16, 1, 1, 2, LRU),     # wide: a narrow last step inside its panel
    ("xy", 120, 120, 48, 16, 2, 1, 4, FAR),     # r a multiple of nb; q = 2
    ("xy", 110, 90, 30, 16, 3, 1, 3, LRU),      # q = 3: two fused sampling passes in a row
    ("xy", 90, 110, 30, 16, 4, 1, 2, FAR),      # q = 4
    ("xy", 90, 60, 60, 13, 0, 1, 2, FAR),       # full column rank: no Nullify; q = 0
    ("xy", 80, 70, 25, 8, 1, 0, 3, LRU),        # the fast option
    ("xy", 64, 64, 1, 8, 1, 1, 1, FAR),         # rank 1, a cache of one panel
    ("xy", 200, 130, 50, 32, 1, 1, 100, FAR),   # everything fits
    # no gap (sigma_i = 0.8^i) and q = 0: T_12 is far from zero, so Nullify
    # changes T and x by much more than rounding
    ("decay", 90, 60, None, 8, 0, 1, 3, FAR),
    ("decay", 90, 60, None, 8, 0, 0, 3, LRU),
]


def make_input(kind, m, n, r, seed):
    if kind == "xy":
        A, X, Y = wl.lowrank_xy(m, n, r, seed=seed, noise=1e-14)
        return A, 1e-10 * wl.norm2_of_product(X, Y)
    sigma = 0.8 ** np.arange(n)
    A, _, _ = wl.spectrum_matrix(m, n, sigma, seed=seed)
    return A, 1e-3


@pytest.mark.parametrize("phases", [(0,), (1, 2)], ids=["whole", "two-phase"])
@pytest.mark.parametrize("kind,m,n,r,nb,q,nullify,cache,policy", CASES)
def test_streamed_solve_follows_schedule_and_matches_oracle(lls, kind, m, n, r, nb, q, nullify,
                                                             cache, policy, phases):
    A, tol = make_input(kind, m, n, r, seed=m + 3 * n + (r or 0))
    B = np.random.default_rng(n).standard_normal((m, 2))
    seed = 77
    ref = orc.solve(A, B, q, nb, tol, seed, do_nullify=bool(nullify), keep=True)
    utv = orc.randutv(A, q, nb, seed)
    if r is not None:
        assert ref.rank == r
    r = ref.rank
    if kind == "decay":   # Nullify must matter here for the check to mean something
        assert 0 < r < n
        assert np.linalg.norm(np.triu(utv.T)[:r, r:]) > 1e-6 * np.linalg.norm(utv.T)

    ss = StreamedSolve(A, B, nb, q, tol, seed, nullify, cache, policy, lls)
    ss.rank_for_plan = ss.r = r
    sched = ss.run(phases)
    assert ss.rank == r and ss.rank_count == ref.rank_count
    # T after the block-SVD pass: the oracle's randUTV T
    T = np.triu(ss.T_after_svd)
    assert np.linalg.norm(T - utv.T) <= 1e-12 * np.linalg.norm(utv.T)
    # T at the end (after Nullify, all panels written back): the oracle's
    T_end = np.triu(np.concatenate(ss.host, axis=1))
    assert np.linalg.norm(T_end - ref.utv.T) <= 1e-11 * np.linalg.norm(ref.utv.T)
    x = ss.solution()
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    plan = lls.lls_ooc_plan(m, n, nb, q, r, nullify, cache, policy)
    assert ss.max_slot < min(cache, plan["panels"])
    if phases == (0,):   # the schedule's traffic is the plan's
        assert sum(a["load"] for a in sched) == plan["loads"]
        assert sum(a["store"] for a in sched) == plan["stores"]
        assert sum(a["kind"] != "flush" for a in sched) == plan["accesses"]


def test_schedule_api_errors(lls):
    import ctypes as C

    cnt = C.c_int64(0)
    L = lls._lib
    assert L.lls_ooc_schedule(10, 10, 4, 1, 5, 1, 2, 0, 0, None, 0, None) == lls.LLS_ERR_ARG
    assert L.lls_ooc_schedule(10, 10, 4, 1, 11, 1, 2, 0, 0, None, 0, C.byref(cnt)) == \
        lls.LLS_ERR_ARG
    assert L.lls_ooc_schedule(10, 10, 4, 1, 5, 1, 2, 0, 3, None, 0, C.byref(cnt)) == \
        lls.LLS_ERR_ARG
    assert L.lls_ooc_schedule(10, 10, 4, 1, 5, 1, 2, 0, 0, None, 0, C.byref(cnt)) == lls.LLS_OK
    assert cnt.value > 0
    small = (lls.lls_ooc_action * 1)()
    assert L.lls_ooc_schedule(10, 10, 4, 1, 5, 1, 2, 0, 0, small, 1, C.byref(cnt)) == \
        lls.LLS_ERR_CAPACITY
    # phase 1 ends with nothing modified left on the device
    acts = lls.lls_ooc_schedule(60, 40, 8, 1, 20, 1, 2, 0, 1)
    dirty = set()
    for a in acts:
        if a["store"]:
            dirty.discard(a["evict"])
        if a["kind"] != "flush" and a["write"]:
            dirty.add(a["panel"])
    assert not dirty
