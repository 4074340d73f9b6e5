"""Seeded synthetic inputs shared by the oracle side and the GPU side.

This module holds workload definitions and random number generation only --
none of the method's arithmetic.  Both the tests (oracle and GPU paths) and
the benchmark draw their inputs from here, so that the two sides always see
identical data.

Workloads (matrix, batch, distributions) follow the configurations this
project measures; workload ``i`` (1-based) uses numpy PCG64 seed ``i - 1``.
"""
from __future__ import annotations

import numpy as np

# Dilation/pattern matrices of the measured workloads.
M_SMALL_2D = [[64, 16], [-16, 64]]                          # det 4352, cycles (16, 272)
M_BATCHED_2D = [[4096, 1024], [0, 4096]]                    # det 2^24, cycles (1024, 16384)
M_AUTOGRAD_3D = [[256, 64, 0], [0, 256, 32], [0, 0, 256]]   # det 2^24, cycles (32, 64, 8192)
M_AUTOGRAD_TINY = [[4, 1, 0], [0, 4, 1], [0, 0, 4]]         # det 64, one cycle of 64
M_WAVELET_2D = [[1024, 1024], [-1024, 1024]]                # 2^10 [[1,1],[-1,1]], det 2^21
J_DIAG_A = [[1, 1], [-1, 1]]
J_DIAG_B = [[1, -1], [1, 1]]
# the dilation set of Section 6.2 (J_x, J_y, J_d) and the pattern it is applied to
DIRECTIONAL_J = {"J_x": [[2, 0], [0, 1]], "J_y": [[1, 0], [0, 2]], "J_d": [[1, -1], [1, 1]]}
M_DIRECTIONAL = [[512, 0], [0, 512]]

WORKLOADS = {
    "small_2d": dict(M=M_SMALL_2D, batch=1, seed=0),
    "batched_2d": dict(M=M_BATCHED_2D, batch=8, seed=1),
    "autograd_3d": dict(M=M_AUTOGRAD_3D, batch=4, seed=2),
    "wavelet_2d": dict(M=M_WAVELET_2D, batch=16, seed=3, levels=12),
    "uneven_mix": dict(n_patterns=4096, seed=4, even_det=False),
    "directional": dict(M=M_DIRECTIONAL, batch=16, seed=5),
    "table1": dict(n=2048, batch=8, seed=6),
}

SAMPLE_SEED = 12345


def wavelet_dilations(levels: int):
    """Dilations J_1, J_2, ... alternating [[1,1],[-1,1]] and [[1,-1],[1,1]]."""
    return [J_DIAG_A if l % 2 == 0 else J_DIAG_B for l in range(levels)]


def complex_normal(batch: int, n: int, seed: int, dtype=np.complex64) -> np.ndarray:
    """[batch, n] complex values whose real and imaginary parts are i.i.d. N(0,1)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((batch, n))
    im = rng.standard_normal((batch, n))
    return (re + 1j * im).astype(dtype)


def complex_normal_flat(n: int, seed: int) -> np.ndarray:
    """[n] complex64 values, real and imaginary parts i.i.d. N(0,1), drawn in
    single precision (interleaved re, im) -- the concatenated signals of a
    pattern batch."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(2 * n, dtype=np.float32).view(np.complex64)


def uniform01(shape, seed: int, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.random(shape).astype(dtype)


def sample_slots(m: int, n: int = 4096, seed: int = SAMPLE_SEED) -> np.ndarray:
    """n distinct slot indices in [0, m), sorted (all of them when n >= m)."""
    if n >= m:
        return np.arange(m, dtype=np.int64)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(m, size=n, replace=False).astype(np.int64))


def random_upper_triangular(rng, d: int, lo: int, hi: int):
    """Upper-triangular integer matrix, diagonal uniform in [lo, hi],
    entry (r, c), r < c, uniform in [0, M_rr)."""
    M = [[0] * d for _ in range(d)]
    for r in range(d):
        M[r][r] = int(rng.integers(lo, hi + 1))
    for r in range(d):
        for c in range(r + 1, d):
            M[r][c] = int(rng.integers(0, M[r][r]))
    return M


def uneven_mix(n_patterns: int = 4096, seed: int = 4, max_det: int = 1 << 20,
               lo: int = 16, hi: int = 512, even_det: bool = False):
    """Patterns of the uneven serving-style mix: d uniform in {2, 3}, upper
    triangular, diagonals uniform in [lo, hi], off-diagonals in [0, diag),
    resampled until the determinant (product of the diagonal) is <= max_det
    (and even, if ``even_det``: a dilation of determinant 2 needs it)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n_patterns:
        d = int(rng.integers(2, 4))
        M = random_upper_triangular(rng, d, lo, hi)
        prod = 1
        for r in range(d):
            prod *= M[r][r]
        if prod <= max_det and (prod % 2 == 0 or not even_det):
            out.append(M)
    return out


def prime_dilation(M, p: int):
    """A dilation J with |det J| = p (a prime dividing det M) and J^{-1} M
    integral (workload construction, not part of the method).
    J Z^d = {x : v . x = 0 mod p} for a non-zero v in GF(p)^d with
    v^T M = 0 mod p (one exists: M mod p is singular), scaled so that its last
    non-zero entry v_r is 1.  The columns e_j - v_j e_r (j != r) and p e_r
    span that lattice: J = I + e_r w^T, w_j = -v_j (j != r), w_r = p - 1."""
    d = len(M)
    rows = [[int(M[i][j]) % p for i in range(d)] for j in range(d)]  # rows of M^T mod p
    piv_cols, rank = [], 0
    for c in range(d):
        q = next((r for r in range(rank, d) if rows[r][c]), None)
        if q is None:
            continue
        rows[rank], rows[q] = rows[q], rows[rank]
        inv = pow(rows[rank][c], p - 2, p)
        rows[rank] = [(x * inv) % p for x in rows[rank]]
        for r in range(d):
            if r != rank and rows[r][c]:
                f = rows[r][c]
                rows[r] = [(a - f * b) % p for a, b in zip(rows[r], rows[rank])]
        piv_cols.append(c)
        rank += 1
    free = [c for c in range(d) if c not in piv_cols]
    if not free:
        raise ValueError(f"{p} does not divide det M: no dilation of determinant {p} divides M")
    v = [0] * d
    v[free[0]] = 1
    for i, c in enumerate(piv_cols):
        v[c] = (-rows[i][free[0]]) % p
    r = max(i for i in range(d) if v[i])
    inv = pow(v[r], p - 2, p)
    v = [(x * inv) % p for x in v]
    J = [[int(i == j) for j in range(d)] for i in range(d)]
    for j in range(d):
        J[r][j] = p if j == r else -v[j]
    return J


def parity_dilation(M):
    """A dilation J with |det J| = 2 and J^{-1} M integral: prime_dilation(M, 2)."""
    return prime_dilation(M, 2)


def smallest_prime_factor(n: int) -> int:
    n = abs(int(n))
    f = 2
    while f * f <= n:
        if n % f == 0:
            return f
        f += 1
    return n


def mix_dilation(M):
    """The dilation of the uneven mix: determinant 2 when det M is even, else
    the smallest (odd) prime p dividing det M."""
    D = 1
    for r in range(len(M)):
        D *= int(M[r][r])  # upper triangular
    return prime_dilation(M, smallest_prime_factor(D))


def random_regular_matrix(rng, d: int, amax: int, max_det: int):
    """A random integer matrix with 0 < |det| <= max_det (rejection sampling)."""
    while True:
        M = [[int(rng.integers(-amax, amax + 1)) for _ in range(d)] for _ in range(d)]
        D = int(round(np.linalg.det(np.array(M, dtype=np.float64))))
        if 0 < abs(D) <= max_det:
            return M
