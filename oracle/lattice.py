"""Exact-integer lattice algebra for the oracle (test infrastructure only).

This module belongs to the CPU oracle.  Only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import it; the GPU library never does,
and it shares no code with the library's own host planner.

Everything here works on Python integers (arbitrary precision) and
``fractions.Fraction``, so every result is exact.

Paper notation (Section 2.2):
  * congruence  h = k mod M  <=>  k - h in M Z^d
  * Lambda(M) = M^{-1} Z^d, pattern P(M) = a complete residue system of
    Lambda(M) mod Z^d, generating group G(M) = M P(M) (integer residues
    mod M Z^d), frequency set G(M^T).
  * Smith normal form M = Q E R, E = diag(eps_1 | ... | eps_d),
    |det Q| = |det R| = 1 (eq. (SNF)).
  * Pattern normal form: upper-triangular matrices that generate the same
    lattice (eq. (FFTexampleMatrix), Section 6.1).

Layout convention shared with the library (a contract, not shared code):
the integer box  x_{r} [0, H_rr)  of the column-style upper-triangular Hermite
normal form H of M (H Z^d = M Z^d) is a complete residue system of Z^d / M Z^d.
Slots are numbered row-major over that box, last coordinate fastest.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

__all__ = [
    "det", "adjugate", "inverse", "transpose", "matmul", "matvec", "identity",
    "hnf", "box_shape", "box_points", "box_reduce", "slot_of", "point_of",
    "snf", "elementary_divisors", "centered_rep_coords",
]


def identity(d):
    return [[int(i == j) for j in range(d)] for i in range(d)]


def transpose(A):
    return [list(r) for r in zip(*A)]


def matmul(A, B):
    return [[sum(A[i][k] * B[k][j] for k in range(len(B))) for j in range(len(B[0]))]
            for i in range(len(A))]


def matvec(A, x):
    return [sum(A[i][j] * x[j] for j in range(len(x))) for i in range(len(A))]


def det(M):
    """Exact determinant by Bareiss fraction-free elimination."""
    d = len(M)
    A = [list(map(int, r)) for r in M]
    sign, prev = 1, 1
    for k in range(d - 1):
        if A[k][k] == 0:
            piv = next((r for r in range(k + 1, d) if A[r][k] != 0), None)
            if piv is None:
                return 0
            A[k], A[piv] = A[piv], A[k]
            sign = -sign
        for i in range(k + 1, d):
            for j in range(k + 1, d):
                A[i][j] = (A[i][j] * A[k][k] - A[i][k] * A[k][j]) // prev
        prev = A[k][k]
    return sign * A[d - 1][d - 1]


def adjugate(M):
    """Classical adjoint: adj(M) M = M adj(M) = det(M) I (cofactor expansion)."""
    d = len(M)
    if d == 1:
        return [[1]]
    out = [[0] * d for _ in range(d)]
    for i in range(d):
        for j in range(d):
            minor = [[M[r][c] for c in range(d) if c != i] for r in range(d) if r != j]
            out[i][j] = (-1) ** (i + j) * det(minor)
    return out


def inverse(M):
    """Exact rational inverse M^{-1} = adj(M) / det(M)."""
    D = det(M)
    if D == 0:
        raise ValueError("singular matrix")
    A = adjugate(M)
    return [[Fraction(x, D) for x in row] for row in A]


def hnf(M):
    """Column-style Hermite normal form H = M U (U unimodular).

    H is upper triangular with H_rr > 0 and 0 <= H_rc < H_rr for c > r, and
    H Z^d = M Z^d.  It is unique, which makes it a safe layout contract: the
    library computes it with its own code and the two must agree exactly.
    Upper-triangular lattice bases are the pattern normal form of Section 6.1.
    """
    d = len(M)
    A = [list(map(int, r)) for r in M]
    if det(A) == 0:
        raise ValueError("singular matrix")

    def colop(dst, src, q):  # column dst -= q * column src
        for i in range(d):
            A[i][dst] -= q * A[i][src]

    for r in range(d - 1, -1, -1):
        # Euclid on row r over columns 0..r until only one entry is non-zero.
        while True:
            nz = [c for c in range(r + 1) if A[r][c] != 0]
            piv = min(nz, key=lambda c: abs(A[r][c]))
            for c in nz:
                if c != piv:
                    colop(c, piv, A[r][c] // A[r][piv])
            if all(A[r][c] == 0 for c in range(r + 1) if c != piv):
                break
        for i in range(d):
            A[i][piv], A[i][r] = A[i][r], A[i][piv]
        if A[r][r] < 0:
            for i in range(d):
                A[i][r] = -A[i][r]
    # Reduce entries right of the diagonal, bottom row first, so that a
    # reduction never disturbs a row that is already reduced.
    for r in range(d - 1, -1, -1):
        for c in range(r + 1, d):
            colop(c, r, A[r][c] // A[r][r])
    return A


def box_shape(M):
    """Shape of the residue box of Z^d / M Z^d (the diagonal of hnf(M))."""
    H = hnf(M)
    return [H[i][i] for i in range(len(H))]


def box_points(H):
    """All integer points of the box x_r [0, H_rr), row-major (last fastest)."""
    return itertools.product(*[range(H[i][i]) for i in range(len(H))])


def box_reduce(H, y):
    """Representative of y mod H Z^d inside the box (back-substitution)."""
    y = list(y)
    d = len(H)
    for r in range(d - 1, -1, -1):
        q = y[r] // H[r][r]
        if q:
            for i in range(r + 1):
                y[i] -= q * H[i][r]
    return tuple(y)


def slot_of(H, y):
    s = 0
    for r in range(len(H)):
        s = s * H[r][r] + y[r]
    return s


def point_of(H, s):
    d = len(H)
    y = [0] * d
    for r in range(d - 1, -1, -1):
        s, y[r] = divmod(s, H[r][r])
    return tuple(y)


def snf(M):
    """Smith normal form M = Q E R (eq. (SNF), Section 2.2).

    Returns (Q, E, R) with integer Q, R of determinant +-1 and
    E = diag(eps_1, ..., eps_d), eps_j > 0, eps_j | eps_{j+1}.
    Computed by elementary row/column operations: U M V = E, Q = U^{-1},
    R = V^{-1}.
    """
    d = len(M)
    A = [list(map(int, r)) for r in M]
    if det(A) == 0:
        raise ValueError("singular matrix")
    U = identity(d)
    V = identity(d)

    def rowop(i, j, q):
        A[i] = [A[i][k] - q * A[j][k] for k in range(d)]
        U[i] = [U[i][k] - q * U[j][k] for k in range(d)]

    def colop(i, j, q):
        for r in range(d):
            A[r][i] -= q * A[r][j]
            V[r][i] -= q * V[r][j]

    def rowswap(i, j):
        A[i], A[j] = A[j], A[i]
        U[i], U[j] = U[j], U[i]

    def colswap(i, j):
        for r in range(d):
            A[r][i], A[r][j] = A[r][j], A[r][i]
            V[r][i], V[r][j] = V[r][j], V[r][i]

    for t in range(d):
        while True:
            cand = [(abs(A[i][j]), i, j) for i in range(t, d) for j in range(t, d) if A[i][j]]
            _, i, j = min(cand)
            rowswap(t, i)
            colswap(t, j)
            clean = True
            for i in range(t + 1, d):
                rowop(i, t, A[i][t] // A[t][t])
                clean &= A[i][t] == 0
            for j in range(t + 1, d):
                colop(j, t, A[t][j] // A[t][t])
                clean &= A[t][j] == 0
            if not clean:
                continue
            bad = [(i, j) for i in range(t + 1, d) for j in range(t + 1, d) if A[i][j] % A[t][t]]
            if bad:
                rowop(t, bad[0][0], -1)  # bring a non-divisible entry into row t
                continue
            break
        if A[t][t] < 0:
            A[t] = [-x for x in A[t]]
            U[t] = [-x for x in U[t]]
    Q = [[int(x) for x in row] for row in inverse(U)]
    R = [[int(x) for x in row] for row in inverse(V)]
    return Q, A, R


def elementary_divisors(M):
    _, E, _ = snf(M)
    return [E[i][i] for i in range(len(E))]


def centered_rep_coords(M, h):
    """Coordinates u = M^{-T} k of the representative k of h mod M^T Z^d that
    lies in M^T [-1/2, 1/2)^d (the centred frequency set of Ex. 1 and Section 6.2).
    Returns u as Fractions; k = M^T u."""
    t = matvec(inverse(transpose(M)), list(h))
    return [x - math.floor(x + Fraction(1, 2)) for x in t]
