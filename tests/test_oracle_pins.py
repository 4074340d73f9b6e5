"""Pins for the CPU oracle: every check compares it with something other than
itself -- the textbook DFT (numpy, a library call), brute force with exact
rational phases, closed-form identities of the paper, or printed values
(Table 1, Example 1).  CPU only."""
import cmath
import itertools
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import lattice as L
import seeded_inputs as SI

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_c(m, batch=1, seed=0):
    return SI.complex_normal(batch, m, seed, dtype=np.complex128)


def _gauss_jordan_inverse(M):
    """Rational inverse by Gauss-Jordan elimination (independent of the
    adjugate route the oracle takes)."""
    d = len(M)
    A = [[Fraction(x) for x in r] + [Fraction(int(i == j)) for j in range(d)] for i, r in enumerate(M)]
    for c in range(d):
        p = next(r for r in range(c, d) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [x / piv for x in A[c]]
        for r in range(d):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [A[r][k] - f * A[c][k] for k in range(2 * d)]
    return [r[d:] for r in A]


def _box(M):
    return list(itertools.product(*[range(n) for n in L.box_shape(M)]))


# ---------------------------------------------------------------- transform
@pytest.mark.parametrize("shape", [(12,), (4, 8), (6, 10), (2, 3, 5), (8, 4, 2)])
def test_diagonal_matrix_gives_textbook_dft(shape):
    """M = diag(n_1..n_d): eq. (Fouriermatrix) reduces to the d-dimensional DFT."""
    M = [[shape[i] if i == j else 0 for j in range(len(shape))] for i in range(len(shape))]
    m = int(np.prod(shape))
    c = _rand_c(m, 2, seed=7)
    ref = np.fft.fftn(c.reshape((2,) + shape), axes=range(1, len(shape) + 1), norm="ortho")
    got = oracle.pattern_fft(M, c)
    assert np.allclose(got, ref.reshape(2, m), atol=1e-12)
    back = np.fft.ifftn(ref, axes=range(1, len(shape) + 1), norm="ortho").reshape(2, m)
    assert np.allclose(oracle.pattern_fft(M, ref.reshape(2, m), inverse=True), back, atol=1e-12)


@pytest.mark.parametrize("M", [[[4, -3], [4, 5]], [[3, 1], [-2, 5]], [[2, 7], [1, 1]],
                               [[0, 3], [2, 1]], [[2, 1, 0], [0, 3, 1], [1, 0, 2]],
                               [[1, 2, 0], [-1, 1, 3], [2, 0, 1]]])
def test_brute_force_exact_rational_phase(M):
    """Direct sum with k^T M^{-1} y formed exactly in rationals (Gauss-Jordan)."""
    Minv = _gauss_jordan_inverse(M)
    m = abs(L.det(M))
    ys = _box(M)
    ks = _box(L.transpose(M))
    assert len(ys) == len(ks) == m
    c = _rand_c(m, seed=3)[0]
    ref = np.zeros(m, complex)
    for a, k in enumerate(ks):
        acc = 0j
        for b, y in enumerate(ys):
            ph = sum(k[i] * Minv[i][j] * y[j] for i in range(len(k)) for j in range(len(k)))
            frac = ph - math.floor(ph)
            acc += c[b] * cmath.exp(-2j * math.pi * float(frac))
        ref[a] = acc / math.sqrt(m)
    assert np.allclose(oracle.pattern_fft(M, c), ref, atol=1e-12)
    # inverse: sum over k with the conjugate phase, output on the G(M) box
    back = np.zeros(m, complex)
    for b, y in enumerate(ys):
        acc = 0j
        for a, k in enumerate(ks):
            ph = sum(k[i] * Minv[i][j] * y[j] for i in range(len(k)) for j in range(len(k)))
            acc += ref[a] * cmath.exp(2j * math.pi * float(ph - math.floor(ph)))
        back[b] = acc / math.sqrt(m)
    assert np.allclose(oracle.pattern_fft(M, ref, inverse=True), back, atol=1e-12)
    assert np.allclose(back, c, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_parseval_and_inverse_identity(seed):
    rng = np.random.default_rng(100 + seed)
    d = 2 + seed % 2
    M = SI.random_regular_matrix(rng, d, 6, 600)
    m = abs(L.det(M))
    c = _rand_c(m, 3, seed)
    ch = oracle.pattern_fft(M, c)
    assert np.allclose(np.linalg.norm(ch, axis=1), np.linalg.norm(c, axis=1), rtol=1e-13)
    assert np.allclose(oracle.pattern_fft(M, ch, inverse=True), c, atol=1e-12)


@pytest.mark.parametrize("M", [[[5, -2], [3, 7]], [[6, 2], [0, 9]], [[4, 1], [0, 4]],
                               [[3, 1, 2], [0, 4, 1], [0, 0, 2]], [[2, 1, 0], [1, 3, 1], [0, 1, 4]]])
def test_transposed_pattern_gives_the_transposed_matrix(M):
    """Eq. (Fouriermatrix): entry (k, y) of F(M) is m^{-1/2} exp(-2 pi i k^T M^{-1} y),
    k in G(M^T), y indexing P(M); the same expression read for M^T is entry (y, k) of
    F(M^T) with the roles of the two boxes exchanged.  So F(M^T) = F(M)^T in box
    order, and the inverse of M is the conjugated forward transform of M^T."""
    Mt = L.transpose(M)
    m = abs(L.det(M))
    F = oracle.pattern_fft(M, np.eye(m, dtype=complex)).T    # column j = F(M) e_j
    Ft = oracle.pattern_fft(Mt, np.eye(m, dtype=complex)).T
    assert np.allclose(Ft, F.T, atol=1e-12)
    c = _rand_c(m, 2, 7)
    assert np.allclose(np.conj(oracle.pattern_fft(Mt, np.conj(c))), oracle.pattern_fft(M, c, inverse=True),
                       atol=1e-12)


@pytest.mark.parametrize("M", [SI.M_SMALL_2D, [[6, 2], [-2, 6]], [[4, 0], [0, 2]],
                               SI.M_AUTOGRAD_TINY, [[3, 1, 2], [0, 2, 1], [1, 0, 4]],
                               [[8, 2], [2, -4]], [[8, 8], [-8, 8]]])
def test_kronecker_form_in_smith_coordinates(M):
    """Thm 1: in the orderings of eq. (orderings) the transform is the tensor
    product of 1-D DFTs.  lambda = Q^{-1} y mod eps, mu = R^{-T} k mod eps."""
    Q, E, R = L.snf(M)
    d = len(M)
    eps = [E[i][i] for i in range(d)]
    m = abs(L.det(M))
    Qi = [[int(x) for x in r] for r in L.inverse(Q)]
    RiT = [[int(x) for x in r] for r in L.transpose(L.inverse(R))]
    c = _rand_c(m, seed=11)[0]
    X = np.zeros(eps, complex)
    for s, y in enumerate(_box(M)):
        lam = tuple(v % e for v, e in zip(L.matvec(Qi, list(y)), eps))
        X[lam] = c[s]
    Y = np.fft.fftn(X, norm="ortho")
    ref = np.array([Y[tuple(v % e for v, e in zip(L.matvec(RiT, list(k)), eps))]
                    for k in _box(L.transpose(M))])
    assert np.allclose(oracle.pattern_fft(M, c), ref, atol=1e-12)


def test_sampled_slots_match_full_output():
    M = [[40, 7], [0, 36]]
    m = abs(L.det(M))
    c = _rand_c(m, 2, seed=5)
    full = oracle.pattern_fft(M, c)
    slots = SI.sample_slots(m, 97, seed=1)
    assert np.allclose(oracle.pattern_fft(M, c, out_slots=slots), full[:, slots], atol=1e-13)


# ------------------------------------------------------- lattice / SNF pins
@pytest.mark.parametrize("seed", range(40))
def test_smith_form_properties(seed):
    rng = np.random.default_rng(seed)
    d = 1 + seed % 4
    M = SI.random_regular_matrix(rng, d, 9, 10**6)
    Q, E, R = L.snf(M)
    assert L.matmul(L.matmul(Q, E), R) == M
    assert abs(L.det(Q)) == 1 and abs(L.det(R)) == 1
    eps = [E[i][i] for i in range(d)]
    assert all(E[i][j] == 0 for i in range(d) for j in range(d) if i != j)
    assert all(e > 0 for e in eps)
    assert all(eps[j + 1] % eps[j] == 0 for j in range(d - 1))
    assert math.prod(eps) == abs(L.det(M))


def test_table1_cycle_lengths():
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLD, "table1_cycles.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 12
    for i, *cycles in rows:
        eps = L.elementary_divisors([[2048, i], [0, 2048]])
        assert [e for e in eps if e > 1] == cycles


def test_example1_smith_diagonal():
    vals = {l.split()[0]: list(map(int, l.split()[1:])) for l in open(os.path.join(GOLD, "example1.txt"))
            if l.strip() and not l.startswith("#")}
    M = [vals["M"][:2], vals["M"][2:]]
    F1 = [vals["F1"][:2], vals["F1"][2:]]
    F2 = [vals["F2"][:2], vals["F2"][2:]]
    assert L.matmul(F1, F2) == M
    assert L.elementary_divisors(M) == vals["E"]


@pytest.mark.parametrize("M", [SI.M_SMALL_2D, SI.M_BATCHED_2D, SI.M_AUTOGRAD_3D, [[4, -3], [4, 5]],
                               [[3, 1, 2], [0, 2, 1], [1, 0, 4]]])
def test_lemma1_biorthogonality(M):
    """<h_j, y_i> = delta_ij / eps_i for h_j = R^T e_j and y_i = R^{-1} e_i / eps_i."""
    Q, E, R = L.snf(M)
    d = len(M)
    Ri = L.inverse(R)
    for i in range(d):
        for j in range(d):
            hj = [R[j][r] for r in range(d)]
            yi = [Ri[r][i] / E[i][i] for r in range(d)]
            ip = sum(a * b for a, b in zip(hj, yi))
            assert ip == (Fraction(1, E[i][i]) if i == j else 0)


@pytest.mark.parametrize("seed", range(12))
def test_hnf_box_is_complete_residue_system(seed):
    rng = np.random.default_rng(50 + seed)
    d = 1 + seed % 3
    M = SI.random_regular_matrix(rng, d, 5, 200)
    H = L.hnf(M)
    U = L.matmul(L.inverse(M), H)
    assert all(x.denominator == 1 for r in U for x in r) and abs(L.det([[int(x) for x in r] for r in U])) == 1
    assert all(H[r][c] == 0 for r in range(d) for c in range(r))
    assert all(0 <= H[r][c] < H[r][r] for r in range(d) for c in range(r + 1, d))
    Minv = L.inverse(M)
    pts = _box(M)
    assert len(pts) == abs(L.det(M))
    keys = set()
    for y in pts:  # class key: fractional part of M^{-1} y
        t = L.matvec(Minv, list(y))
        keys.add(tuple(x - math.floor(x) for x in t))
    assert len(keys) == len(pts)
    for y in [(5, -3, 7)[:d], (-11, 4, 2)[:d]]:
        z = L.box_reduce(H, y)
        diff = L.matvec(Minv, [a - b for a, b in zip(y, z)])
        assert all(x.denominator == 1 for x in diff)


# --------------------------------------------------------- wavelet pins
def _closed_cube_reps(M, bound=None):
    """All k in Z^d with M^{-T} k in [-1/2, 1/2]^d."""
    MT = L.transpose(M)
    MiT = L.inverse(MT)
    d = len(M)
    bound = bound or sum(abs(x) for r in M for x in r)
    out = []
    for k in itertools.product(range(-bound, bound + 1), repeat=d):
        t = L.matvec(MiT, list(k))
        if all(abs(x) <= Fraction(1, 2) for x in t):
            out.append(k)
    return out


def _dirichlet_coeff(M, k):
    """c_k(phi_M) of the Dirichlet kernel (Section 6.2)."""
    t = L.matvec(L.inverse(L.transpose(M)), list(k))
    if any(abs(x) > Fraction(1, 2) for x in t):
        return 0.0
    r = sum(abs(x) == Fraction(1, 2) for x in t)
    return 2.0 ** (-r / 2) / math.sqrt(abs(L.det(M)))


CASES = [([[8, 8], [-8, 8]], SI.J_DIAG_A), ([[8, 0], [0, 8]], SI.J_DIAG_B),
         ([[8, 0], [0, 8]], [[2, 0], [0, 1]]), ([[8, 0], [0, 8]], [[1, 0], [0, 2]]),
         ([[6, 2], [-2, 6]], SI.J_DIAG_A), ([[4, 4], [-4, 4]], SI.J_DIAG_A),
         ([[4, 1, 0], [0, 4, 1], [0, 0, 4]], [[1, 0, 0], [0, 1, 0], [0, 0, 2]])]


@pytest.mark.parametrize("M,J", CASES)
def test_dirichlet_kernel_class_norm(M, J):
    """Orthonormal translates of phi_M: the |c_k|^2 of each class of
    G(M^T) add up to 1/m (the boundary weights 2^{-r} make this exact)."""
    m = abs(L.det(M))
    G = L.hnf(L.transpose(M))
    acc = {}
    for k in _closed_cube_reps(M):
        key = L.box_reduce(G, k)
        acc[key] = acc.get(key, 0.0) + _dirichlet_coeff(M, k) ** 2
    assert len(acc) == m
    assert all(abs(v - 1.0 / m) < 1e-14 for v in acc.values())


@pytest.mark.parametrize("M,J", CASES)
def test_dirichlet_two_scale_relation(M, J):
    """c_k(phi_N) = A_h c_k(phi_M) for every k with M^{-T}k in the closed cube
    (Section 6.2), with A from the oracle's scaling symbol."""
    N = oracle.exact_N(M, J)
    ks = _closed_cube_reps(M)
    A = oracle.scaling_symbol(M, J, np.array(ks), oracle.DIRICHLET)
    for k, a in zip(ks, A):
        assert abs(_dirichlet_coeff(N, k) - a * _dirichlet_coeff(M, k)) < 1e-14


def _split_roundtrip(M, J, symbol, eta, batch=2, seed=0):
    m = abs(L.det(M))
    c = _rand_c(m, batch, seed)
    d1, d2 = oracle.wavelet_level(M, J, symbol, eta, c_hat=c)
    back = oracle.wavelet_level(M, J, symbol, eta, d1=d1, d2=d2, mode="reconstruct")
    return c, d1, d2, back


@pytest.mark.parametrize("M,J", CASES)
@pytest.mark.parametrize("symbol", [oracle.DIRICHLET, oracle.DLVP])
def test_split_perfect_reconstruction(M, J, symbol):
    c, d1, d2, back = _split_roundtrip(M, J, symbol, 0.125)
    assert np.allclose(back, c, atol=1e-12)


@pytest.mark.parametrize("M,J", CASES)
def test_dirichlet_split_is_orthogonal(M, J):
    c, d1, d2, back = _split_roundtrip(M, J, oracle.DIRICHLET, 0.0)
    # norm preservation
    assert np.allclose(np.linalg.norm(d1, axis=1) ** 2 + np.linalg.norm(d2, axis=1) ** 2,
                       np.linalg.norm(c, axis=1) ** 2, rtol=1e-13)
    # V_N^{phi_N} and V_N^{psi_N} are orthogonal: synthesised parts are orthogonal
    z = np.zeros_like(d1)
    v = oracle.wavelet_level(M, J, oracle.DIRICHLET, d1=d1, d2=z, mode="reconstruct")
    w = oracle.wavelet_level(M, J, oracle.DIRICHLET, d1=z, d2=d2, mode="reconstruct")
    assert abs(np.vdot(v, w)) < 1e-12 * np.linalg.norm(c) ** 2
    assert np.allclose(v + w, c, atol=1e-12)


@pytest.mark.parametrize("M,J", CASES[:4])
@pytest.mark.parametrize("symbol", [oracle.DIRICHLET, oracle.DLVP])
def test_split_adjoint_dot_product(M, J, symbol):
    m = abs(L.det(M))
    c = _rand_c(m, 1, 1)
    e1 = _rand_c(m // 2, 1, 2)
    e2 = _rand_c(m // 2, 1, 3)
    d1, d2 = oracle.wavelet_level(M, J, symbol, 0.125, c_hat=c)
    ct = oracle.wavelet_level(M, J, symbol, 0.125, d1=e1, d2=e2, mode="adjoint")
    assert abs(np.vdot(e1, d1) + np.vdot(e2, d2) - np.vdot(ct, c)) < 1e-12 * m


@pytest.mark.parametrize("M,J", CASES)
def test_dlvp_partition_of_unity_and_dirichlet_limit(M, J):
    """w(N^{-T} h0) + w(N^{-T} h1) = 1 on every fibre; as eta -> 0 the symbol
    equals the Dirichlet one wherever the fibre has no boundary point."""
    N = oracle.exact_N(M, J)
    HN = L.hnf(L.transpose(N))
    HM = L.hnf(L.transpose(M))
    l1 = oracle.nonzero_class_JT(J)
    NTl1 = L.matvec(L.transpose(N), l1)
    hs0, hs1 = [], []
    for g in L.box_points(HN):
        hs0.append(L.box_reduce(HM, g))
        hs1.append(L.box_reduce(HM, [a + b for a, b in zip(g, NTl1)]))
    r2 = math.sqrt(abs(L.det(J)))
    for eta in (0.125, 0.3):
        w0 = oracle.scaling_symbol(M, J, np.array(hs0), oracle.DLVP, eta) / r2
        w1 = oracle.scaling_symbol(M, J, np.array(hs1), oracle.DLVP, eta) / r2
        assert np.allclose(w0 + w1, 1.0, atol=1e-14)
        assert (w0 >= 0).all() and (w1 >= 0).all()
    tiny = 1e-9
    a0 = oracle.scaling_symbol(M, J, np.array(hs0), oracle.DLVP, tiny)
    a1 = oracle.scaling_symbol(M, J, np.array(hs1), oracle.DLVP, tiny)
    D0 = oracle.scaling_symbol(M, J, np.array(hs0), oracle.DIRICHLET)
    D1 = oracle.scaling_symbol(M, J, np.array(hs1), oracle.DIRICHLET)
    clean = (np.isin(D0, [0.0, math.sqrt(2)])) & (np.isin(D1, [0.0, math.sqrt(2)]))
    assert clean.sum() > 0
    assert np.allclose(a0[clean], D0[clean], atol=1e-6) and np.allclose(a1[clean], D1[clean], atol=1e-6)


def _containment(J):
    """[-1/2,1/2]^d inside J^T[-1/2,1/2]^d: every row of J^{-T} has l1 norm <= 1."""
    JiT = L.inverse(L.transpose(J))
    return all(sum(abs(x) for x in row) <= 1 for row in JiT)


def _fibres(M, J):
    N = oracle.exact_N(M, J)
    HN, HM = L.hnf(L.transpose(N)), L.hnf(L.transpose(M))
    NTl1 = L.matvec(L.transpose(N), oracle.nonzero_class_JT(J))
    h0 = [L.box_reduce(HM, g) for g in L.box_points(HN)]
    h1 = [L.box_reduce(HM, [a + b for a, b in zip(g, NTl1)]) for g in L.box_points(HN)]
    return np.array(h0), np.array(h1)


# Dilations of determinant 2 without the containment (parity dilations of the
# uneven mix, J = I + e_r w^T): the paper's case formula is not a valid symbol there.
NO_CONTAINMENT = [([[3, 1], [1, 3]], [[1, 0], [-1, 2]]),
                  ([[10, 1, 7], [0, 9, 1], [0, 0, 32]], [[1, 0, 0], [-1, 2, 0], [0, 0, 1]]),
                  ([[6, 1, 1], [0, 5, 1], [0, 0, 4]], [[1, 0, 0], [0, 1, 0], [-1, -1, 2]])]


@pytest.mark.parametrize("M,J", CASES + [([[6, 2, 0], [0, 6, 2], [0, 0, 4]], [[2, 0, 0], [0, 1, 0], [0, 0, 1]]),
                                         ([[5, 1, 2], [0, 6, 2], [0, 0, 4]], [[1, 0, 0], [0, 2, 0], [0, 0, 1]])])
def test_periodised_dirichlet_equals_case_formula(M, J):
    """Where phi_N lies in V_M ([-1/2,1/2]^d inside J^T[-1/2,1/2]^d, true for
    the dilations of Section 6.2), the periodised Dirichlet symbol is the
    paper's case formula on every class of G(M^T)."""
    assert _containment(J)
    hs = np.array(list(L.box_points(L.hnf(L.transpose(M)))))
    a = oracle.scaling_symbol(M, J, hs, oracle.DIRICHLET)
    b = oracle.scaling_symbol(M, J, hs, oracle.DIRICHLET_CASE)
    assert np.allclose(a, b, atol=1e-15)


@pytest.mark.parametrize("M,J", NO_CONTAINMENT)
def test_case_formula_fails_without_containment(M, J):
    """Without the containment the case formula read literally breaks perfect
    reconstruction (|A(h0)|^2 + |A(h1)|^2 != 2 on some fibre), which is why the
    oracle uses the periodised form: it sums to 2 on every fibre and gives an
    orthogonal, norm-preserving split."""
    assert not _containment(J)
    h0, h1 = _fibres(M, J)
    c0 = oracle.scaling_symbol(M, J, h0, oracle.DIRICHLET_CASE)
    c1 = oracle.scaling_symbol(M, J, h1, oracle.DIRICHLET_CASE)
    assert not np.allclose(c0 ** 2 + c1 ** 2, 2.0)
    a0 = oracle.scaling_symbol(M, J, h0, oracle.DIRICHLET)
    a1 = oracle.scaling_symbol(M, J, h1, oracle.DIRICHLET)
    assert np.allclose(a0 ** 2 + a1 ** 2, 2.0, atol=1e-14)
    c, d1, d2, back = _split_roundtrip(M, J, oracle.DIRICHLET, 0.0)
    assert np.allclose(back, c, atol=1e-12)
    assert np.allclose(np.linalg.norm(d1, axis=1) ** 2 + np.linalg.norm(d2, axis=1) ** 2,
                       np.linalg.norm(c, axis=1) ** 2, rtol=1e-13)


@pytest.mark.parametrize("symbol", [oracle.DIRICHLET, oracle.DLVP])
def test_twelve_level_cascade_reconstructs(symbol):
    M0 = [[64, 64], [-64, 64]]  # same shape family as the measured workload, det 2^13
    Js = SI.wavelet_dilations(12)
    m = abs(L.det(M0))
    c = _rand_c(m, 2, 9)
    s, w = oracle.wavelet_cascade(M0, Js, c, symbol, 0.125)
    assert s.shape[1] == 2 and [x.shape[1] for x in w] == [m >> (l + 1) for l in range(12)]
    back = oracle.wavelet_cascade_inverse(M0, Js, s, w, symbol, 0.125)
    assert np.allclose(back, c, atol=1e-11)
    if symbol == oracle.DIRICHLET:
        tot = np.linalg.norm(s) ** 2 + sum(np.linalg.norm(x) ** 2 for x in w)
        assert abs(tot - np.linalg.norm(c) ** 2) < 1e-10 * tot


def test_cascade_matrices_follow_the_dilation_chain():
    """N_{2k-1} = 2^{11-k} I and N_{2k} = 2^{10-k} [[1,1],[-1,1]] for the 12-level workload."""
    M = SI.M_WAVELET_2D
    for lev, J in enumerate(SI.wavelet_dilations(12), start=1):
        M = oracle.exact_N(M, J)
        k = (lev + 1) // 2
        if lev % 2:
            assert M == [[2 ** (11 - k), 0], [0, 2 ** (11 - k)]]
        else:
            s = 2 ** (10 - k)
            assert M == [[s, s], [-s, s]]


@pytest.mark.parametrize("seed", range(10))
def test_theorem3_dimension_step(seed):
    """For |det J| = 2 (d_J = 1) the number of cycles grows by 0 or 1."""
    rng = np.random.default_rng(seed)
    J = [SI.J_DIAG_A, SI.J_DIAG_B, [[2, 0], [0, 1]], [[1, 0], [0, 2]]][seed % 4]
    N = SI.random_regular_matrix(rng, 2, 7, 400)
    M = L.matmul(J, N)
    dM = sum(e > 1 for e in L.elementary_divisors(M))
    dN = sum(e > 1 for e in L.elementary_divisors(N))
    assert dM - dN in (0, 1)


# ------------------------------------------- general split step (|det J| = p)
GENERAL = [([[6, 1], [0, 9]], [[1, 0], [0, 3]]),            # p = 3, coordinate dilation
           ([[10, 5], [5, 15]], [[1, 1], [-1, 4]]),         # p = 5, not triangular
           ([[8, 4], [0, 12]], [[2, 0], [0, 1]]),           # p = 2
           ([[4, 1, 0], [0, 6, 2], [0, 0, 7]], [[1, 0, 0], [0, 1, 0], [0, 0, 7]]),  # p = 7, d = 3
           ([[12, 4], [4, 12]], [[1, 1], [-1, 3]])]         # p = 4 (cyclic G(J^T))


@pytest.mark.parametrize("M,J", GENERAL)
def test_general_fibres_partition_the_classes(M, J):
    """The fibres of step 4: every class of G(M^T) lies in exactly one fibre,
    and h_t - g lies in N^T Z^d with the p members pairwise different mod M^T Z^d."""
    N = oracle.exact_N(M, J)
    S, p, n = oracle._general_fibres(M, J)
    m = abs(L.det(M))
    assert p == abs(L.det(J)) and n * p == m
    assert sorted(S.reshape(-1).tolist()) == list(range(m))
    HM, HN = L.hnf(L.transpose(M)), L.hnf(L.transpose(N))
    NTinv = L.inverse(L.transpose(N))
    for gs in range(0, n, max(1, n // 17)):
        g = L.point_of(HN, gs)
        for t in range(p):
            h = L.point_of(HM, int(S[gs, t]))
            assert all(x.denominator == 1 for x in L.matvec(NTinv, [a - b for a, b in zip(h, g)]))


def _dft_symbols(M, J):
    """A unitary symbol system: b_j(h_t) = exp(-2 pi i j t / p) on the fibre
    position t of every class (the columns of the p-point DFT)."""
    S, p, n = oracle._general_fibres(M, J)
    sym = np.zeros((p, n * p), dtype=np.complex128)
    for t in range(p):
        for j in range(p):
            sym[j, S[:, t]] = np.exp(-2j * np.pi * j * t / p)
    return sym


@pytest.mark.parametrize("M,J", GENERAL)
def test_general_split_unitary_symbols(M, J):
    """With a unitary symbol system the split preserves the norm and the
    adjoint undoes it; with b_0 = sqrt(p) on one fibre member and 0 elsewhere
    the first part picks that member."""
    m = abs(L.det(M))
    c = _rand_c(m, 2, 11)
    sym = _dft_symbols(M, J)
    parts = oracle.split_general(M, J, sym, c)
    assert np.allclose((np.abs(parts) ** 2).sum(axis=(0, 2)), (np.abs(c) ** 2).sum(axis=1), rtol=1e-13)
    assert np.allclose(oracle.merge_general(M, J, sym, parts), c, atol=1e-12)
    S, p, n = oracle._general_fibres(M, J)
    pick = np.zeros((1, m), dtype=np.complex128)
    pick[0, S[:, 0]] = np.sqrt(p)
    assert np.allclose(oracle.split_general(M, J, pick, c)[0], c[:, S[:, 0]], atol=1e-13)


@pytest.mark.parametrize("M,J", [([[8, 8], [-8, 8]], SI.J_DIAG_A), ([[6, 2], [-2, 6]], SI.J_DIAG_A),
                                 ([[8, 0], [0, 8]], [[2, 0], [0, 1]])])
def test_general_split_reduces_to_dirichlet_level(M, J):
    """p = 2 with the Dirichlet symbol system (scaling A, wavelet
    B(h) = A(h + N^T l) exp(-2 pi i h^T M^{-1} (J z))) gives the split of the
    dedicated C routine."""
    m = abs(L.det(M))
    HM = L.hnf(L.transpose(M))
    hs = np.array(list(L.box_points(HM)))
    N = oracle.exact_N(M, J)
    l1 = oracle.nonzero_class_JT(J)
    NTl1 = L.matvec(L.transpose(N), l1)
    A = oracle.scaling_symbol(M, J, hs, oracle.DIRICHLET)
    shifted = np.array([L.box_reduce(HM, [a + b for a, b in zip(h, NTl1)]) for h in hs.tolist()])
    A1 = oracle.scaling_symbol(M, J, shifted, oracle.DIRICHLET)
    u = oracle.wavelet_shift(J)
    Minv = L.inverse(M)
    ph = np.array([float(sum(Fraction(int(h[i])) * sum(Minv[i][k] * u[k] for k in range(len(u)))
                             for i in range(len(u))) % 1) for h in hs])
    B = A1 * np.exp(-2j * np.pi * ph)
    c = _rand_c(m, 2, 5)
    parts = oracle.split_general(M, J, np.stack([A, B]), c)
    d1, d2 = oracle.wavelet_level(M, J, oracle.DIRICHLET, c_hat=c)
    assert np.allclose(parts[0], d1, atol=1e-12) and np.allclose(parts[1], d2, atol=1e-12)


# ------------------------------------------------- wavelet shift z (Section 6.2)
def _wavelet_shift_golden():
    rows = []
    with open(os.path.join(GOLD, "wavelet_shift.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            t = line.split()
            J = [[int(t[1]), int(t[2])], [int(t[3]), int(t[4])]]
            z = [Fraction(t[5]), Fraction(t[6])]
            u = [int(t[7]), int(t[8])]
            rows.append((t[0], J, z, u))
    return rows


SHIFT_ROWS = _wavelet_shift_golden()


@pytest.mark.parametrize("name,J,z,u", SHIFT_ROWS, ids=[r[0] for r in SHIFT_ROWS])
def test_wavelet_shift_is_the_centred_pattern_point(name, J, z, u):
    """The oracle's z is the non-zero point of Lambda(J) cap [-1/2, 1/2)^d
    (Section 6.2), and u = J z."""
    # the golden z is a non-zero pattern point of J in the half-open centred cube
    Jz = [sum(J[i][k] * z[k] for k in range(2)) for i in range(2)]
    assert all(x.denominator == 1 for x in Jz) and [int(x) for x in Jz] == u
    assert any(x != 0 for x in z) and all(Fraction(-1, 2) <= x < Fraction(1, 2) for x in z)
    assert oracle.wavelet_shift(J) == u


WAVELET_DELTA_CASES = [([[8, 8], [-8, 8]], "J_diag_a"), ([[8, 0], [0, 8]], "J_diag_b"),
                       ([[8, 0], [0, 8]], "J_x"), ([[8, 0], [0, 8]], "J_y"),
                       ([[6, 2], [-2, 6]], "J_diag_a")]


@pytest.mark.parametrize("M,name", WAVELET_DELTA_CASES)
def test_wavelet_part_of_a_delta_matches_the_symbol_definition(M, name):
    """For the input c_hat = e_h (one class h of G(M^T)) step 4 leaves
    d2[g] = 2^{-1/2} conj(B(h)), g the class of h in G(N^T), with the wavelet
    symbol of Section 6.2, B(h) = A(h + N^T l) exp(-2 pi i h^T N^{-1} z),
    l the non-zero class of G(J^T).  The phase is evaluated here from the
    golden z with exact rationals (N^{-1} by Gauss-Jordan elimination); the
    oracle reaches it through u = J z and adj(M)."""
    J, z = next((r[1], r[2]) for r in SHIFT_ROWS if r[0] == name)
    m = abs(L.det(M))
    N = oracle.exact_N(M, J)
    Ninv = _gauss_jordan_inverse(N)
    HM, HN = L.hnf(L.transpose(M)), L.hnf(L.transpose(N))
    # a vector outside J^T Z^d: the non-zero class of G(J^T), found by brute force
    JTinv = _gauss_jordan_inverse(L.transpose(J))
    lvec = next(v for v in ([1, 0], [0, 1]) if any(
        x.denominator != 1 for x in [sum(JTinv[i][k] * v[k] for k in range(2)) for i in range(2)]))
    NTl = [sum(N[k][i] * lvec[k] for k in range(2)) for i in range(2)]
    hs = [list(h) for h in L.box_points(HM)]
    c = np.eye(m, dtype=np.complex128)  # row s: the delta at slot s
    d1, d2 = oracle.wavelet_level(M, J, oracle.DIRICHLET, c_hat=c)
    shifted = np.array([L.box_reduce(HM, [a + b for a, b in zip(h, NTl)]) for h in hs])
    A_shift = oracle.scaling_symbol(M, J, shifted, oracle.DIRICHLET)
    for s, h in enumerate(hs):
        Nz = [sum(Ninv[i][k] * z[k] for k in range(2)) for i in range(2)]
        t = sum(Fraction(h[i]) * Nz[i] for i in range(2))  # h^T N^{-1} z
        t -= math.floor(t)
        B = A_shift[s] * cmath.exp(-2j * math.pi * float(t))
        g = L.slot_of(HN, L.box_reduce(HN, h))
        assert abs(d2[s, g] - np.conj(B) / math.sqrt(2)) < 1e-13, (h, d2[s, g], B)
        others = np.delete(d2[s], g)
        assert np.abs(others).max(initial=0.0) == 0.0


# ------------------------------------------- dilations of prime determinant p
P_CASES = [([[9, 0], [0, 9]], [[3, 0], [0, 1]]), ([[9, 3], [0, 9]], [[1, 0], [0, 3]]),
           ([[15, 5], [0, 10]], [[1, 0], [0, 5]]), ([[9, 6], [9, 15]], [[1, 0], [-2, 3]]),
           ([[6, 1, 2], [0, 7, 3], [0, 0, 14]], [[1, 0, 0], [0, 1, 0], [0, 0, 7]]),
           ([[10, 0, 0], [0, 10, 0], [0, 0, 5]], [[5, 0, 0], [0, 1, 0], [0, 0, 1]])]


def _p_fibres(M, J):
    return oracle._general_fibres(M, J)


@pytest.mark.parametrize("M,J", P_CASES)
def test_prime_dilation_scaling_weights_sum_to_p(M, J):
    """sum over each fibre of |A|^2 = p for the periodised Dirichlet symbol:
    the p members of a fibre cover every Z^d shift of N^{-T} g once, and the
    box indicator (1/2 on the boundary) is a partition of unity."""
    S, p, n = _p_fibres(M, J)
    HM = L.hnf(L.transpose(M))
    hs = np.array([L.point_of(HM, s) for s in range(n * p)])
    A = oracle.scaling_symbol(M, J, hs, oracle.DIRICHLET)
    assert np.allclose((A[S] ** 2).sum(axis=1), p, atol=1e-13)
    assert (A >= 0).all()


def test_prime_dilation_two_scale_relation():
    """c_k(phi_N) = A_h c_k(phi_M) (Section 6.2) for J = diag(3, 1) on
    M = 9 I, where [-1/2,1/2]^2 lies inside J^T [-1/2,1/2]^2."""
    M, J = [[9, 0], [0, 9]], [[3, 0], [0, 1]]
    N = oracle.exact_N(M, J)
    ks = _closed_cube_reps(M)
    A = oracle.scaling_symbol(M, J, np.array(ks), oracle.DIRICHLET)
    for k, a in zip(ks, A):
        assert abs(_dirichlet_coeff(N, k) - a * _dirichlet_coeff(M, k)) < 1e-14


@pytest.mark.parametrize("u", [[1, 0, 0], [0, 1, 0], [0.6, 0.8, 0], [0.5, 0.5, 0.5, 0.5], [0, 0, 0, 0, 1],
                               [np.sqrt(0.5), 0, np.sqrt(0.5)]])
def test_householder_completion(u):
    """U is real orthogonal and symmetric with first row u; for p = 2 its
    second row is (u_1, -u_0)."""
    U = oracle.householder_completion(np.array(u, dtype=float))
    p = len(u)
    assert np.allclose(U @ U.T, np.eye(p), atol=1e-14)
    assert np.allclose(U, U.T, atol=1e-14)
    assert np.allclose(U[0], u, atol=1e-14)
    if p == 2:
        assert np.allclose(U[1], [u[1], -u[0]], atol=1e-14)


@pytest.mark.parametrize("M,J", P_CASES)
def test_prime_dilation_split_is_unitary(M, J):
    """The p-band system is unitary on every fibre: perfect reconstruction,
    norm preservation, orthogonal synthesised bands, band 0 = the scaling
    part (analysis with conj(A))."""
    S, p, n = _p_fibres(M, J)
    m = n * p
    sym = oracle.dirichlet_p_symbols(M, J)
    for gs in range(n):
        B = sym[:, S[gs]] / np.sqrt(p)
        assert np.allclose(B @ B.conj().T, np.eye(p), atol=1e-12)
    c = _rand_c(m, 2, 9)
    parts = oracle.wavelet_level_p(M, J, c_hat=c)
    assert np.allclose(np.linalg.norm(parts, axis=(0, 2)), np.linalg.norm(c, axis=1), rtol=1e-13)
    back = oracle.wavelet_level_p(M, J, parts=parts, mode="reconstruct")
    assert np.allclose(back, c, atol=1e-12)
    synth = []
    for j in range(p):
        z = np.zeros_like(parts)
        z[j] = parts[j]
        synth.append(oracle.wavelet_level_p(M, J, parts=z, mode="reconstruct"))
    for i in range(p):
        for j in range(i + 1, p):
            assert abs(np.vdot(synth[i], synth[j])) < 1e-12 * np.linalg.norm(c) ** 2
    A = oracle.scaling_symbol(M, J, np.array([L.point_of(L.hnf(L.transpose(M)), s) for s in range(m)]),
                              oracle.DIRICHLET)
    assert np.allclose(parts[0], (c[:, S] * A[S][None]).sum(axis=2) / np.sqrt(p), atol=1e-12)


@pytest.mark.parametrize("M,J", [([[8, 8], [-8, 8]], SI.J_DIAG_A), ([[6, 2], [-2, 6]], SI.J_DIAG_A),
                                 ([[8, 0], [0, 8]], [[2, 0], [0, 1]]), ([[3, 1], [1, 3]], [[1, 0], [-1, 2]])])
def test_prime_dilation_system_reduces_to_the_p2_split(M, J):
    """For p = 2 the p-band system is the scaling / wavelet pair of Section
    6.2 (the dedicated two-band routine)."""
    c = _rand_c(abs(L.det(M)), 2, 4)
    parts = oracle.wavelet_level_p(M, J, c_hat=c)
    d1, d2 = oracle.wavelet_level(M, J, oracle.DIRICHLET, c_hat=c)
    assert np.allclose(parts[0], d1, atol=1e-12) and np.allclose(parts[1], d2, atol=1e-12)


@pytest.mark.parametrize("M,J", P_CASES)
def test_pattern_generator_pairs_to_one_over_p(M, J):
    """u = J z with z in Lambda(J) cap [-1/2, 1/2)^d and l^T z = 1/p mod 1."""
    p = abs(L.det(J))
    l = oracle.cyclic_generator_JT(J)
    u = oracle.pattern_generator_J(J, l)
    z = L.matvec(L.inverse(J), u)
    assert all(Fraction(-1, 2) <= x < Fraction(1, 2) for x in z)
    assert (sum(Fraction(a) * b for a, b in zip(l, z)) - Fraction(1, p)).denominator == 1


@pytest.mark.parametrize("M,J", P_CASES[:4])
def test_bands_at_sampled_fibres_equal_the_full_split(M, J):
    """wavelet_bands_at (the sampled form the large-size GPU checks use) gives
    the full split's values at the chosen fibres."""
    m, p = abs(L.det(M)), abs(L.det(J))
    c = _rand_c(m, 2, 12)
    full = oracle.wavelet_level_p(M, J, c_hat=c)
    g = np.array([0, 1, m // p - 1])
    assert np.allclose(oracle.wavelet_bands_at(M, J, c, g), full[:, :, g], atol=1e-13)
