"""CPU FP64 oracle for the pattern FFT and the wavelet split step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The GPU
library under ``paper_1107_5415_gb300`` never imports it and shares no code
with it; the two meet only through the seeded input generators and the layout
contract (row-major slots over the box of the Hermite normal form).

What it computes (each function cites the passage it follows):
  * ``pattern_fft``      : eq. (Fouriermatrix), Section 2.2 -- the plain direct
                           sum with exact integer phase numerators mod m.
  * ``wavelet_level``    : Section 5.3 step 4 with the Dirichlet symbols of
                           Section 6.2 (and the de la Vallee Poussin reading, see
                           ``pattern_oracle.c``; PARITY UNPINNED for its values).
  * ``wavelet_cascade``  : the dyadic repetition of Section 5.3 (input of the
                           next level = scaling part of this one).
  * ``split_general``    : Section 5.3 step 4 for any |det J| = p with cyclic
                           G(J^T), symbols given by the caller (and its adjoint
                           ``merge_general``).
  * ``lattice``          : exact integer HNF / SNF / box enumeration.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

from . import lattice as L

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pattern_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DIRICHLET = 0        # periodised Dirichlet symbol (equals the case formula where it is valid)
DLVP = 1             # de la Vallee Poussin reading, blend width eta
DIRICHLET_CASE = 2   # the case formula of Section 6.2 read literally (pins only)


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP).  Returns the path of the .so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            i64p = P(ctypes.c_int64)
            dp = P(ctypes.c_double)
            lib.po_transform.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, i64p, i64p, i64p,
                                         ctypes.c_int64, dp, dp, i64p, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_int]
            lib.po_wavelet_level.argtypes = [ctypes.c_int, i64p, i64p, i64p, ctypes.c_int64, i64p, i64p,
                                             ctypes.c_int64, i64p, i64p, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int64, ctypes.c_int, dp, dp, dp, ctypes.c_int]
            lib.po_scaling_symbol.argtypes = [ctypes.c_int, i64p, ctypes.c_int64, i64p, i64p,
                                              ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_int64, i64p, dp]
            _lib = lib
    return _lib


def _i64(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def layout(M):
    """(input box shape, output box shape, m) for the regular integer matrix M."""
    return L.box_shape(M), L.box_shape(L.transpose(M)), abs(L.det(M))


def pattern_fft(M, c, inverse=False, out_slots=None, nthreads=0):
    """Direct-sum Fourier transform on the pattern P(M) (eq. (Fouriermatrix)).

    c : complex array [batch, m] (or [m]) in input-box slot order (box of hnf(M)).
    Returns complex128 [batch, nk] for the output slots ``out_slots`` of the
    box of hnf(M^T) (all m slots when None).  Unitary scaling m^{-1/2} both ways;
    ``inverse`` conjugates the phase (the inverse maps G(M^T) slots back to
    G(M) slots, so then the roles of the two boxes swap: pass M^T's layout in
    via ``inverse=True`` and the same M).
    """
    M = [list(map(int, r)) for r in M]
    d = len(M)
    D = L.det(M)
    if D == 0:
        raise ValueError("singular M")
    m = abs(D)
    sdet = 1 if D > 0 else -1
    c = np.asarray(c)
    squeeze = c.ndim == 1
    c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.complex128)
    batch = c.shape[0]
    if c.shape[1] != m:
        raise ValueError("signal length must be |det M|")
    if not inverse:
        A = L.adjugate(M)
        ext_in, ext_out = L.box_shape(M), L.box_shape(L.transpose(M))
        adj_rows = A
    else:
        # inverse: sum over k in G(M^T) of c[k] exp(+2 pi i k^T M^{-1} y), output y in G(M).
        # k^T adj(M) y = y^T adj(M)^T k, so the roles are those of the forward sum with adj(M)^T.
        A = L.adjugate(M)
        ext_in, ext_out = L.box_shape(L.transpose(M)), L.box_shape(M)
        adj_rows = L.transpose(A)
    if out_slots is None:
        nk = m
        kp = None
    else:
        ks, kp = _i64(out_slots)
        nk = len(ks)
    out = np.empty((batch, nk), dtype=np.complex128)
    adj_a, adj_p = _i64(np.array(adj_rows).reshape(-1))
    ei, eip = _i64(ext_in)
    eo, eop = _i64(ext_out)
    rc = _load().po_transform(d, m, sdet, adj_p, eip, eop, batch, _f64(c), _f64(out), kp, nk,
                              1 if inverse else 0, int(nthreads))
    if rc != 0:
        raise ValueError("po_transform rejected its arguments")
    return out[0] if squeeze else out


def exact_N(M, J):
    """N = J^{-1} M (Section 2.2, decomposition M = J N); must be integral."""
    N = L.matmul(L.inverse(J), M)
    if any(x.denominator != 1 for r in N for x in r):
        raise ValueError("J^{-1} M is not integral")
    return [[int(x) for x in r] for r in N]


def nonzero_class_JT(J):
    """A representative l1 of the non-zero class of G(J^T) = Z^d / J^T Z^d (|det J| = 2)."""
    JT = L.transpose(J)
    inv = L.inverse(JT)
    d = len(J)
    for i in range(d):
        e = [int(i == j) for j in range(d)]
        if any(x.denominator != 1 for x in L.matvec(inv, e)):
            return e
    raise ValueError("J^T is unimodular")


def wavelet_shift(J):
    """u = J z for the non-zero z of P(J) = Lambda(J) cap [-1/2, 1/2)^d (|det J| = 2).

    The wavelet phase exp(-2 pi i h^T N^{-1} z) of Section 6.2 depends on this
    choice of representative; the centred one follows the pattern choice
    Lambda(M) cap [-1/2,1/2)^d made in Section 6.2.
    """
    d = len(J)
    inv = L.inverse(J)
    H = L.hnf(J)
    for y in L.box_points(H):
        z = L.matvec(inv, list(y))
        zc = [x - (x + Fraction(1, 2)).__floor__() for x in z]
        if any(x != 0 for x in zc):
            u = L.matvec(J, zc)
            return [int(x) for x in u]
    raise ValueError("J is unimodular")


def _level_args(M, J):
    d = len(M)
    N = exact_N(M, J)
    if abs(L.det(J)) != 2:
        raise ValueError("the oracle's split handles |det J| = 2")
    HM = L.hnf(L.transpose(M))
    HN = L.hnf(L.transpose(N))
    adjMT = L.adjugate(L.transpose(M))
    adjJT = L.adjugate(L.transpose(J))
    l1 = nonzero_class_JT(J)
    NTl1 = L.matvec(L.transpose(N), l1)
    u = wavelet_shift(J)
    return N, HM, HN, adjMT, adjJT, NTl1, u


def wavelet_level(M, J, symbol=DIRICHLET, eta=0.125, *, c_hat=None, d1=None, d2=None,
                  mode="decompose", nthreads=0):
    """One level of the split (Section 5.3, step 4) or its inverse / adjoint.

    decompose   : c_hat [batch, |det M|] on G(M^T)  ->  (d1, d2) [batch, |det N|] on G(N^T)
    reconstruct : (d1, d2) -> c_hat (exact inverse of decompose)
    adjoint     : (d1, d2) -> c_hat (conjugate transpose of decompose)
    """
    M = [list(map(int, r)) for r in M]
    J = [list(map(int, r)) for r in J]
    d = len(M)
    N, HM, HN, adjMT, adjJT, NTl1, u = _level_args(M, J)
    mM, mN = abs(L.det(M)), abs(L.det(N))
    modes = {"decompose": 0, "reconstruct": 1, "adjoint": 2}
    md = modes[mode]
    if md == 0:
        c_hat = np.ascontiguousarray(np.atleast_2d(c_hat), dtype=np.complex128)
        batch = c_hat.shape[0]
        d1 = np.zeros((batch, mN), np.complex128)
        d2 = np.zeros((batch, mN), np.complex128)
    else:
        d1 = np.ascontiguousarray(np.atleast_2d(d1), dtype=np.complex128)
        d2 = np.ascontiguousarray(np.atleast_2d(d2), dtype=np.complex128)
        batch = d1.shape[0]
        c_hat = np.zeros((batch, mM), np.complex128)
    a = [_i64(np.array(x).reshape(-1)) for x in (HM, HN, adjMT, J, adjJT, NTl1, u)]
    rc = _load().po_wavelet_level(d, a[0][1], a[1][1], a[2][1], L.det(M), a[3][1], a[4][1], L.det(J),
                                  a[5][1], a[6][1], int(symbol), float(eta), batch, md,
                                  _f64(c_hat), _f64(d1), _f64(d2), int(nthreads))
    if rc != 0:
        raise ValueError("po_wavelet_level rejected its arguments")
    return (d1, d2) if md == 0 else c_hat


def wavelet_cascade(M0, Js, c_hat, symbol=DIRICHLET, eta=0.125, nthreads=0):
    """Multi-level decomposition: level l+1 splits the scaling part of level l.

    Returns (scaling, [wavelet_1, ..., wavelet_L]) with wavelet_l on G(N_l^T)
    and scaling on G(N_L^T).
    """
    M = [list(map(int, r)) for r in M0]
    cur = np.atleast_2d(c_hat)
    wav = []
    for J in Js:
        d1, d2 = wavelet_level(M, J, symbol, eta, c_hat=cur, nthreads=nthreads)
        wav.append(d2)
        cur = d1
        M = exact_N(M, J)
    return cur, wav


def wavelet_cascade_inverse(M0, Js, scaling, wavelets, symbol=DIRICHLET, eta=0.125,
                            mode="reconstruct", nthreads=0):
    """Inverse (or adjoint) of ``wavelet_cascade``, levels in reverse order."""
    Ms = [[list(map(int, r)) for r in M0]]
    for J in Js:
        Ms.append(exact_N(Ms[-1], J))
    cur = np.atleast_2d(scaling)
    for lev in range(len(Js) - 1, -1, -1):
        cur = wavelet_level(Ms[lev], Js[lev], symbol, eta, d1=cur, d2=wavelets[lev], mode=mode,
                            nthreads=nthreads)
    return cur


def scaling_symbol(M, J, hs, symbol=DIRICHLET, eta=0.125):
    """Values A(h) of the scaling symbol for integer frequency vectors hs [n, d]."""
    M = [list(map(int, r)) for r in M]
    J = [list(map(int, r)) for r in J]
    d = len(M)
    hs, hp = _i64(np.asarray(hs).reshape(-1, d))
    out = np.empty(len(hs), np.float64)
    adjMT = _i64(np.array(L.adjugate(L.transpose(M))).reshape(-1))
    Ja = _i64(np.array(J).reshape(-1))
    adjJT = _i64(np.array(L.adjugate(L.transpose(J))).reshape(-1))
    _load().po_scaling_symbol(d, adjMT[1], L.det(M), Ja[1], adjJT[1], L.det(J), int(symbol), float(eta),
                              len(hs), hp, _f64(out))
    return out


def cyclic_generator_JT(J):
    """A generator l of G(J^T) = Z^d / J^T Z^d when that group is cyclic
    (one elementary divisor of J above 1): with J^T = Q E R (Smith form), the
    class of Q e_d generates Z^d / Q E Z^d = Z^d / J^T Z^d."""
    JT = L.transpose(J)
    Q, E, R = L.snf(JT)
    d = len(J)
    if sum(1 for i in range(d) if abs(E[i][i]) > 1) > 1:
        raise ValueError("G(J^T) is not cyclic")
    return [Q[i][d - 1] for i in range(d)]


def _general_fibres(M, J):
    """Slots (box of H(M^T)) of the fibres h_t = g + t N^T l, t < p, for every
    slot g of the box of H(N^T); Section 5.3 step 4 sums over these."""
    N = exact_N(M, J)
    p = abs(L.det(J))
    HM, HN = L.hnf(L.transpose(M)), L.hnf(L.transpose(N))
    shift = L.matvec(L.transpose(N), cyclic_generator_JT(J))
    n = abs(L.det(N))
    S = np.empty((n, p), dtype=np.int64)
    for gs in range(n):
        g = L.point_of(HN, gs)
        for t in range(p):
            S[gs, t] = L.slot_of(HM, L.box_reduce(HM, [a + t * b for a, b in zip(g, shift)]))
    return S, p, n


def split_general(M, J, symbols, c_hat):
    """d_j[g] = p^{-1/2} sum_t conj(b_j(h_t)) c(h_t) (Section 5.3 step 4, with
    the conjugated analysis symbols of this project's reading), for symbols
    b_j given on the box of H(M^T): symbols [p, m], c_hat [batch, m] ->
    parts [p, batch, m / p]."""
    S, p, n = _general_fibres(M, J)
    sym = np.asarray(symbols, dtype=np.complex128)
    c = np.atleast_2d(np.asarray(c_hat, dtype=np.complex128))
    return np.einsum("jnt,bnt->jbn", np.conj(sym[:, S]), c[:, S]) / np.sqrt(p)


def merge_general(M, J, symbols, parts):
    """Adjoint of ``split_general``: c(h_t) = p^{-1/2} sum_j b_j(h_t) d_j[g]."""
    S, p, n = _general_fibres(M, J)
    sym = np.asarray(symbols, dtype=np.complex128)
    dp = np.asarray(parts, dtype=np.complex128)
    batch = dp.shape[1]
    c = np.zeros((batch, n * p), dtype=np.complex128)
    vals = np.einsum("jnt,jbn->bnt", sym[:, S], dp) / np.sqrt(p)
    for t in range(p):
        c[:, S[:, t]] = vals[:, :, t]
    return c


# ----------------------------------------------------------------------------
# Dilations of any prime |det J| = p (Section 5.3, step 4 with p bands)
# ----------------------------------------------------------------------------
def pattern_generator_J(J, l):
    """u = J z for the generator z of the cyclic pattern P(J) = Lambda(J) cap
    [-1/2, 1/2)^d dual to the generator l of G(J^T): l^T z = 1/p (mod 1),
    p = |det J|.  For p = 2 this is the non-zero point of ``wavelet_shift``."""
    p = abs(L.det(J))
    inv = L.inverse(J)
    for y in L.box_points(L.hnf(J)):
        z = L.matvec(inv, list(y))
        frac = sum(Fraction(a) * b for a, b in zip(l, z))
        if (frac - Fraction(1, p)).denominator == 1:
            zc = [x - (x + Fraction(1, 2)).__floor__() for x in z]
            return [int(x) for x in L.matvec(J, zc)]
    raise ValueError("no pattern point of J pairs with l to 1/p")


def householder_completion(u):
    """Real orthogonal, symmetric p x p matrix with first row (and column) u,
    for a unit vector u with u_0 >= 0: U = 2 v v^T / (v^T v) - I, v = u + e_0
    (the negated reflection that exchanges e_0 and -u; v^T v = 2 + 2 u_0 > 0,
    so U is defined for every such u, and for p = 2 its second row is
    (u_1, -u_0))."""
    u = np.asarray(u, dtype=np.float64)
    p = len(u)
    v = u.copy()
    v[0] += 1.0
    return 2.0 * np.outer(v, v) / float(v @ v) - np.eye(p)


def band_generator_JT(J):
    """The generator l = e_i of G(J^T) that labels the members of a fibre in
    the band system: the first unit vector outside J^T Z^d (for |det J| = 2
    the class of ``nonzero_class_JT``)."""
    return nonzero_class_JT(J)


def band_fibre_slots(M, J, gslots):
    """Slots (box of H(M^T)) of the members h_t = g + t N^T l, t < p, of the
    fibres of the given slots g of the box of H(N^T), l = band_generator_JT(J)."""
    N = exact_N(M, J)
    p = abs(L.det(J))
    HM, HN = L.hnf(L.transpose(M)), L.hnf(L.transpose(N))
    shift = L.matvec(L.transpose(N), band_generator_JT(J))
    out = np.empty((len(gslots), p), dtype=np.int64)
    for i, gs in enumerate(gslots):
        g = L.point_of(HN, int(gs))
        for t in range(p):
            out[i, t] = L.slot_of(HM, L.box_reduce(HM, [a + t * b for a, b in zip(g, shift)]))
    return out


def _band_system_at(M, J, gslots):
    """Members and symbols of the fibres of the slots gslots of the box of
    H(N^T): (S [n, p] member slots, b [n, p(band), p(member)] values of
    b_j(h_t)); see ``dirichlet_p_symbols``."""
    M = [list(map(int, r)) for r in M]
    J = [list(map(int, r)) for r in J]
    N = exact_N(M, J)
    p = abs(L.det(J))
    m = abs(L.det(M))
    gslots = np.asarray(list(gslots), dtype=np.int64)
    S = band_fibre_slots(M, J, gslots)
    HM = L.hnf(L.transpose(M))
    hs = np.array([L.point_of(HM, int(s)) for s in S.reshape(-1)], dtype=np.int64).reshape(len(gslots) * p, -1)
    A = scaling_symbol(M, J, hs, DIRICHLET).reshape(len(gslots), p)
    l = band_generator_JT(J)
    u = pattern_generator_J(J, l)
    adj = L.adjugate(M)
    D = L.det(M)
    sgn = 1 if D > 0 else -1
    # exact phase numerator of g^T M^{-1} u = sgn g^T adj(M) u / m
    au = [sum(adj[r][c] * u[c] for c in range(len(u))) for r in range(len(u))]
    HN = L.hnf(L.transpose(N))
    b = np.zeros((len(gslots), p, p), dtype=np.complex128)
    for i, gs in enumerate(gslots):
        g = L.point_of(HN, int(gs))
        num = (sgn * sum(x * y for x, y in zip(g, au))) % m
        e = np.exp(-2j * np.pi * num / m)
        U = householder_completion(A[i] / np.sqrt(p))
        b[i] = np.sqrt(p) * U * (e ** np.arange(p))[:, None]
    return S, b


def dirichlet_p_symbols(M, J):
    """Symbol system of a dilation J of prime determinant p = |det J| (this
    project's reading of Section 5.3 step 4 for p bands):

    * scaling symbol A(h) = sqrt(p w(N^{-T} h)), the periodised Dirichlet
      weight of Section 6.2 (``scaling_symbol``), so sum_fibre |A|^2 = p;
    * on the fibre h_t = g + t N^T l (t < p) of g in the box of H(N^T), l the
      first unit vector outside J^T Z^d, with u_t = A(h_t) / sqrt(p) and U
      the completion of u (``householder_completion``), the band symbols
      b_j(h_t) = sqrt(p) U[j, t] e(g)^j, j < p, with
      e(g) = exp(-2 pi i g^T N^{-1} z) for the centred generator z of P(J)
      with l^T z = 1/p.

    b_0 = A, and (b_j(h_t) / sqrt(p))_{j,t} is unitary on every fibre; for
    p = 2 the system is the scaling / wavelet pair of Section 6.2.
    Returns symbols [p, |det M|] on the box of H(M^T)."""
    p = abs(L.det(J))
    m = abs(L.det(M))
    S, b = _band_system_at(M, J, range(m // p))
    sym = np.zeros((p, m), dtype=np.complex128)
    for i in range(len(S)):
        sym[:, S[i]] = b[i]
    return sym


def wavelet_bands_at(M, J, c_hat, gslots):
    """The bands of ``wavelet_level_p`` at the slots gslots of the box of
    H(N^T) only: d_j[g] = p^{-1/2} sum_t conj(b_j(h_t)) c(h_t) over the
    fibre of each g.  c_hat [batch, |det M|] -> [p, batch, len(gslots)]."""
    p = abs(L.det(J))
    S, b = _band_system_at(M, J, gslots)
    c = np.atleast_2d(np.asarray(c_hat, dtype=np.complex128))
    return np.einsum("gjt,bgt->jbg", np.conj(b), c[:, S]) / np.sqrt(p)


def wavelet_level_p(M, J, c_hat=None, parts=None, mode="decompose"):
    """One split level by a dilation of prime determinant p with the symbol
    system of ``dirichlet_p_symbols``: Section 5.3 step 4 (``split_general``),
    and its inverse, which is the adjoint (``merge_general``) because the
    system is unitary on every fibre.
    decompose: c_hat [batch, m] -> parts [p, batch, m / p];
    reconstruct: parts -> c_hat."""
    sym = dirichlet_p_symbols(M, J)
    if mode == "decompose":
        return split_general(M, J, sym, c_hat)
    return merge_general(M, J, sym, parts)
