"""The algorithmic flop model used for TFLOP/s figures (host logic, CPU)."""

import pytest

from paper_2408_05238_b300 import perf_model as pm


def test_randutv_flops_closed_form():
    """For m = n and nb | n the per-step sum equals (10 + 4q) S plus the
    right update's rows above, minus the left update's b x b corner, with
    S = sum m' n' b."""
    m = n = 1024
    nb, q = 64, 2
    S = sum((m - k) * (n - k) * nb for k in range(0, n, nb))
    right_extra = sum(4.0 * k * (n - k) * nb for k in range(0, n, nb))
    left_fix = sum(4.0 * (m - k) * nb * nb for k in range(0, n, nb))
    assert pm.randutv_flops(m, n, nb, q) == pytest.approx((10 + 4 * q) * S + right_extra - left_fix)


def test_c2_flops_match_closed_form_estimate():
    """16384^2, nb = 128, q = 2: (10 + 4q) S + 2n^3/3 with S ~ mn^2/2 - n^3/6 gives
    about 29.3 TFLOP for the factorization."""
    f = pm.randutv_flops(16384, 16384, 128, 2)
    assert 29.0e12 < f < 29.6e12


def test_nullify_flops_approx():
    n, r, nb = 4096, 2048, 128
    assert pm.nullify_flops(n, r, nb) == pytest.approx(2.0 * r * r * (n - r), rel=0.1)
    assert pm.nullify_flops(n, 0, nb) == 0.0 and pm.nullify_flops(n, n, nb) == 0.0


def test_steps_cover_min_dimension():
    for m, n, nb in [(100, 37, 8), (37, 100, 8), (64, 64, 64), (5, 5, 7)]:
        ks = list(pm.steps(m, n, nb))
        assert sum(b for _, b in ks) == min(m, n)


def test_c3_flops_match_closed_form_estimate():
    """32768 x 16384, nb = 128, q = 1: the same closed form gives about 54.2 TFLOP."""
    f = pm.randutv_flops(32768, 16384, 128, 1)
    assert 53.7e12 < f < 54.7e12


def test_bench_workload_shapes():
    """The bench's single-matrix workloads: C2 square with rank n/2, C3 2n x n
    with rank 12000 n / 16384."""
    import argparse
    import bench

    c2 = argparse.Namespace(workload="c2", n=16384)
    c3 = argparse.Namespace(workload="c3", n=16384)
    assert bench.dense_shape(c2) == (16384, 16384, 8192, 1e-10)
    assert bench.dense_shape(c3) == (32768, 16384, 12000, 1e-6)
    assert bench.dense_shape(argparse.Namespace(workload="c3", n=1024))[:3] == (2048, 1024, 750)


def test_bench_replica_throughput():
    import bench

    solves, tf = bench.replica_throughput(30.0e12, 2, 4, 60.0)
    assert solves == 8 and tf == pytest.approx(4.0)
