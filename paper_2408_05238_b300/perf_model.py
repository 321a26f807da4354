"""Algorithmic work of the randUTV least-squares solve (for throughput and
roofline figures; never a dense-SVD-equivalent count).

Per randUTV step i with k = i nb, m' = m - k, n' = n - k, b = min(nb, m', n'):
  sampling      (2 + 4q) m' n' b      Y = (A^T A)^q A^T G
  right update  4 m n' b              all m rows (T W_V, then the rank-b update)
  left update   4 m' (n' - b) b       W_U^T T, then the rank-b update
The O(b^2 (m + n)) panel, T-factor and diagonal-block SVD terms are left out.
Nullify (Fig. 3) with rank r adds 4 j0 (n - r) bsz per row block of bsz rows
starting at j0 (about 2 r^2 (n - r)); the solve adds, per right-hand side,
4 m' b per step for U^T b, r^2 for the triangular solve, 4 n' b per step for
V y and 4 (n - r) r for the Nullify reflectors.
"""

from __future__ import annotations


def steps(m: int, n: int, nb: int):
    k = 0
    while k < min(m, n):
        b = min(nb, m - k, n - k)
        yield k, b
        k += b


def step_flops(m: int, n: int, k: int, b: int, q: int) -> float:
    mp, np_ = m - k, n - k
    return (2 + 4 * q) * mp * np_ * b + 4.0 * m * np_ * b + 4.0 * mp * (np_ - b) * b


def randutv_flops(m: int, n: int, nb: int, q: int) -> float:
    return sum(step_flops(m, n, k, b, q) for k, b in steps(m, n, nb))


def nullify_flops(n: int, r: int, nb: int) -> float:
    if r <= 0 or r >= n:
        return 0.0
    total, j1 = 0.0, r
    while j1 > 0:
        j0 = max(0, j1 - nb)
        total += 4.0 * j0 * (n - r) * (j1 - j0)
        j1 = j0
    return total


def solve_flops(m: int, n: int, nb: int, r: int, nrhs: int, nullified: bool) -> float:
    total = 0.0
    for k, b in steps(m, n, nb):
        total += 4.0 * (m - k) * b + 4.0 * (n - k) * b
    total += float(r) * r
    if nullified and 0 < r < n:
        total += 4.0 * (n - r) * r
    return total * nrhs


def lls_flops(m: int, n: int, nb: int, q: int, r: int, nrhs: int, nullify: bool = True) -> float:
    """Flops of one lls_solve: randUTV + Nullify + solve."""
    f = randutv_flops(m, n, nb, q) + solve_flops(m, n, nb, r, nrhs, nullify)
    if nullify:
        f += nullify_flops(n, r, nb)
    return f
