"""Out-of-core planning (lls_ooc_plan, lls_ooc_simulate): host code only, so
these run on the CPU.  The cache is pinned against facts that do not come
from its own code: hand-checkable page-reference strings with their known
fault counts for Belady's MIN ("latest in the future") and LRU, an
exhaustive search for the fewest loads on short random lists, an
independent LRU written here with an ordered dict, closed forms of the
plan's pass and access counts, and the theorems MIN <= LRU and "no more
loads with a larger cache" for both policies."""

import functools
import random
from collections import OrderedDict

import pytest

FAR, LRU = 0, 1


@pytest.fixture(scope="module")
def lls():
    from paper_2408_05238_b300 import build

    build.build()
    from paper_2408_05238_b300 import lls as binding

    return binding


def brute_force_min_loads(seq, cache):
    """Fewest loads over every eviction choice (depth-first search with memo)."""

    @functools.lru_cache(maxsize=None)
    def best(t, resident):
        if t == len(seq):
            return 0
        p = seq[t]
        if p in resident:
            return best(t + 1, resident)
        if len(resident) < cache:
            return 1 + best(t + 1, tuple(sorted(resident + (p,))))
        return 1 + min(best(t + 1, tuple(sorted(tuple(x for x in resident if x != v) + (p,))))
                       for v in resident)

    return best(0, ())


def lru_reference(seq, writes, cache):
    """Loads and write-backs of an LRU cache, written independently."""
    od = OrderedDict()   # panel -> dirty
    loads = stores = 0
    for p, w in zip(seq, writes):
        if p in od:
            od.move_to_end(p)
        else:
            if len(od) == cache:
                _, dirty = od.popitem(last=False)
                stores += dirty
            od[p] = False
            loads += 1
        od[p] = od[p] or bool(w)
    stores += sum(od.values())
    return loads, stores


def test_textbook_reference_strings(lls):
    # Classic page-reference strings whose fault counts are worked by hand in
    # operating-systems courses: with 3 frames, MIN 9 and LRU 12 faults; and
    # Belady's anomaly string, MIN 7 / LRU 10 with 3 frames, LRU 8 with 4.
    s1 = [7, 0, 1, 2, 0, 3, 0, 4, 2, 3, 0, 3, 2, 1, 2, 0, 1, 7, 0, 1]
    assert lls.lls_ooc_simulate(s1, cache_panels=3, policy=FAR)["loads"] == 9
    assert lls.lls_ooc_simulate(s1, cache_panels=3, policy=LRU)["loads"] == 12
    s2 = [1, 2, 3, 4, 1, 2, 5, 1, 2, 3, 4, 5]
    assert lls.lls_ooc_simulate(s2, cache_panels=3, policy=FAR)["loads"] == 7
    assert lls.lls_ooc_simulate(s2, cache_panels=3, policy=LRU)["loads"] == 10
    assert lls.lls_ooc_simulate(s2, cache_panels=4, policy=LRU)["loads"] == 8
    assert brute_force_min_loads(tuple(s1), 3) == 9
    assert brute_force_min_loads(tuple(s2), 3) == 7


@pytest.mark.parametrize("seed", range(40))
def test_farthest_is_optimal_and_lru_matches_reference(lls, seed):
    g = random.Random(seed)
    P = g.randint(1, 5)
    seq = [g.randrange(P) for _ in range(g.randint(0, 12))]
    writes = [g.random() < 0.3 for _ in seq]
    cache = g.randint(1, 4)
    far = lls.lls_ooc_simulate(seq, writes, num_panels=P, rows=10, cols=3, cache_panels=cache,
                               policy=FAR)
    lru = lls.lls_ooc_simulate(seq, writes, num_panels=P, rows=10, cols=3, cache_panels=cache,
                               policy=LRU)
    assert far["loads"] == brute_force_min_loads(tuple(seq), cache)
    assert (lru["loads"], lru["stores"]) == lru_reference(seq, writes, cache)
    for st in (far, lru):
        assert st["loads"] + st["hits"] == st["accesses"] == len(seq)
        assert st["load_bytes"] == 8 * 10 * 3 * st["loads"]
        assert st["store_bytes"] == 8 * 10 * 3 * st["stores"]
        # every modified panel is written back exactly once per residency
        assert st["stores"] <= sum(writes)


def test_write_backs_by_hand(lls):
    # cache of 1: 0w (load 0) | 1 (evict dirty 0: store, load 1) | 0 (load) |
    # 0w | end (flush dirty 0): 3 loads, 2 stores
    st = lls.lls_ooc_simulate([0, 1, 0, 0], [1, 0, 0, 1], num_panels=2, cache_panels=1, policy=LRU)
    assert (st["loads"], st["stores"], st["hits"]) == (3, 2, 1)


def plan_counts(m, n, nb, q, r, nullify):
    """Passes and panel visits of the plan, counted from its definition."""
    P = -(-n // nb)
    s = -(-min(m, n) // nb)
    passes = accesses = 0
    for i in range(s):
        per_step = (1 if i == 0 else 0) + (q + 1 if q >= 1 else 0) + 1 + 1
        passes += per_step
        accesses += per_step * (P - i)
    if s:
        passes += 1
        accesses += P
        if nullify and 0 < r < n:
            pr, top = r // nb, (r - 1) // nb
            passes += 1 + 2 * (top + 1)             # gather, then read + write per block
            accesses += P - pr
            for p in range(top + 1):                # the block's panel + D's other panels
                accesses += 2 * (1 + P - max(pr, p + 1))
        if r > 0:
            passes += 2
            accesses += s + (r - 1) // nb + 1
    return P, passes, accesses


CASES = [(2000, 1000, 64, 1, 400, 1), (1024, 1024, 128, 2, 512, 1), (300, 700, 64, 0, 200, 1),
         (700, 300, 32, 1, 300, 1), (512, 512, 100, 1, 0, 1), (640, 512, 64, 2, 257, 0),
         (64, 64, 128, 1, 10, 1)]


@pytest.mark.parametrize("m,n,nb,q,r,nullify", CASES)
def test_plan_pass_and_access_counts(lls, m, n, nb, q, r, nullify):
    P, passes, accesses = plan_counts(m, n, nb, q, r, nullify)
    st = lls.lls_ooc_plan(m, n, nb, q, r, nullify, 3, FAR)
    assert (st["panels"], st["passes"], st["accesses"]) == (P, passes, accesses)


@pytest.mark.parametrize("m,n,nb,q,r,nullify", CASES)
def test_plan_cache_theorems(lls, m, n, nb, q, r, nullify):
    P = -(-n // nb)
    prev = {FAR: None, LRU: None}
    for cache in range(1, P + 2):
        far = lls.lls_ooc_plan(m, n, nb, q, r, nullify, cache, FAR)
        lru = lls.lls_ooc_plan(m, n, nb, q, r, nullify, cache, LRU)
        assert far["loads"] <= lru["loads"]                 # MIN is optimal
        for pol, st in ((FAR, far), (LRU, lru)):
            if prev[pol] is not None:
                assert st["loads"] <= prev[pol]             # stack algorithms: no anomaly
            prev[pol] = st["loads"]
        if cache >= P:                                      # everything fits: compulsory only
            for st in (far, lru):
                assert st["loads"] == P and st["stores"] == P
                assert st["load_bytes"] == 8.0 * m * n == st["store_bytes"]


def test_plan_side_bytes_closed_form(lls):
    m, n, nb, r = 1000, 600, 64, 250
    st = lls.lls_ooc_plan(m, n, nb, 1, r, 1, 4, FAR)
    wv = sum(2 * 8 * (n - k) * min(nb, m - k, n - k) for k in range(0, min(m, n), nb))
    rz = sum(2 * 8 * (min(r, j0 + nb) - j0 + n - r) * (min(r, j0 + nb) - j0)
             for j0 in range(0, r, nb))
    assert st["side_bytes"] == wv + rz
    assert lls.lls_ooc_plan(m, n, nb, 1, r, 0, 4, FAR)["side_bytes"] == wv


def test_empty_and_invalid(lls):
    st = lls.lls_ooc_plan(0, 100, 32, 1, 0, 1, 2, FAR)
    assert st["accesses"] == 0 and st["loads"] == 0 and st["stores"] == 0
    L = lls._lib
    out = lls.lls_ooc_stats()
    import ctypes as C
    for args in [(-1, 10, 4, 1, 0, 1, 2, 0), (10, 10, 0, 1, 0, 1, 2, 0), (10, 10, 4, 5, 0, 1, 2, 0),
                 (10, 10, 4, 1, 11, 1, 2, 0), (10, 10, 4, 1, 0, 2, 2, 0), (10, 10, 4, 1, 0, 1, 0, 0),
                 (10, 10, 4, 1, 0, 1, 2, 7)]:
        assert L.lls_ooc_plan(*args, C.byref(out)) == lls.LLS_ERR_ARG
    assert L.lls_ooc_plan(10, 10, 4, 1, 0, 1, 2, 0, None) == lls.LLS_ERR_ARG
    with pytest.raises(lls.LLSError):
        lls.lls_ooc_simulate([0, 3], num_panels=2)
