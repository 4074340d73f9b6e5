"""Host checks of the index arithmetic of the compile-time specialised passes
(complex64 column pencils of 2^6 .. 2^13 with T = min(16, 8192 / L) columns per
CTA, bulk-copy rows of 2^13 and 2^14), for every thread and element the
kernels touch:

* the shared tile places row i of column c at phys(i) + c,
  phys(i) = (i + floor(i / 32)) T; the kernels split phys(b + r D) into a
  per-thread base phys(b) and a constant phys(r D) -- exact for every row set
  the stages, the tail stage, the epilogue and (for P >= 32) the sheared walk
  touch, with the wrap of the walk taking off phys(L);
* the tile is a bijection of (row, column) onto addresses inside the
  allocation of T L + T L / 32 elements;
* the row pass's arithmetic walk of the workspace permutation
  pos(mu) = ((mu mod 2^lg) << ls) | ((floor(mu / 2^lg) inv) mod 2^ls) with
  block padding equals the per-element formula for every lg <= log2 P.

Plain integer arithmetic, no GPU."""
import itertools

import numpy as np
import pytest

R = 32


def phys(i, logt):
    return (i + (i >> 5)) << logt


def col_shapes():
    for logl in range(6, 14):
        yield logl, min(4, 13 - logl)


def stage_row_sets(logl):
    """(name, base rows per thread p, constant offsets) of the stage exchanges."""
    L, P = 1 << logl, (1 << logl) // R
    nmain = logl // 5
    tail = 1 << (logl - 5 * nmain)
    p = np.arange(P)
    sets = [("read", p, np.arange(R) * P)]  # rows p + P r (stage reads, epilogue)
    if tail > 1:
        nq = R // tail
        offs = np.array([q * P * tail + r for q in range(nq) for r in range(tail)])
        sets.append(("tail", p * tail, offs))
    Ns = tail
    for s in range(nmain - 1):
        k = p & (Ns - 1)
        sets.append((f"write{s}", (p - k) * R + k, np.arange(R) * Ns))
        Ns *= R
    return sets


@pytest.mark.parametrize("logl,logt", list(col_shapes()))
def test_column_tile_offsets_are_affine(logl, logt):
    L, T = 1 << logl, 1 << logt
    for name, base, offs in stage_row_sets(logl):
        rows = base[:, None] + offs[None, :]
        assert rows.min() >= 0 and rows.max() < L, name
        direct = phys(rows, logt)
        split = phys(base, logt)[:, None] + phys(offs, logt)[None, :]
        assert (direct == split).all(), name
    # every row appears exactly once per column in the reads and the writes
    P = L // R
    rows = (np.arange(P)[:, None] + P * np.arange(R)[None, :]).ravel()
    assert np.array_equal(np.sort(rows), np.arange(L))


@pytest.mark.parametrize("logl,logt", list(col_shapes()))
def test_column_walk_offsets(logl, logt):
    L, P = 1 << logl, (1 << logl) // R
    i0 = np.arange(L)[:, None]
    j = np.arange(R)[None, :]
    i = i0 + j * P
    direct = phys(np.where(i >= L, i - L, i), logt)
    if P >= 32:
        split = phys(i0, logt) + phys(j * P, logt) - np.where(i >= L, phys(L, logt), 0)
        assert (direct == split).all()
    # the walk of one thread visits each row of its column once
    assert all(len(set(((k + j * P) % L).ravel())) == R for k in range(0, L, max(1, L // 64)))


@pytest.mark.parametrize("logl,logt", list(col_shapes()) + [(13, 0), (14, 0)])
def test_tile_is_a_bijection_inside_the_allocation(logl, logt):
    L, T = 1 << logl, 1 << logt
    rows, cols = np.meshgrid(np.arange(L), np.arange(T), indexing="ij")
    addr = phys(rows, logt) + cols
    nel = T * L
    assert addr.max() < nel + (nel >> 5)
    assert len(np.unique(addr)) == nel


def col_pos(mu, lg, ls, inv):
    return ((mu & ((1 << lg) - 1)) << ls) | (((mu >> lg) * inv) & ((1 << ls) - 1))


@pytest.mark.parametrize("logl", [13, 14])
def test_row_permutation_walk(logl):
    L, P, LP = 1 << logl, (1 << logl) // R, logl - 5
    p = np.arange(P)[:, None]
    k = np.arange(R)[None, :]
    mu = p + P * k
    rng = np.random.default_rng(logl)
    for lg in range(0, LP + 1):
        ls = logl - lg
        for inv in itertools.chain([1], rng.integers(0, 1 << ls, 6) | 1):
            inv = int(inv)
            pos = col_pos(mu, lg, ls, inv)
            assert np.array_equal(np.sort(pos.ravel()), np.arange(L))  # a permutation
            for pad in (0, 2, 16):
                direct = pos + (pos >> ls) * pad
                lo = p & ((1 << lg) - 1)
                hp = (lo << ls) + lo * pad
                bp = (p >> lg) * inv
                cstep = inv << (LP - lg)
                walk = hp + ((bp + k * cstep) & ((1 << ls) - 1))
                assert (walk == direct).all(), (lg, inv, pad)
                assert (bp + k * cstep).max() < 2 ** 31


def _wavefronts(elems):
    """Shared-memory wavefronts of one warp's 64-bit accesses: per bank, the
    number of distinct 8-byte elements touching it; the maximum over banks."""
    banks = {}
    for e in set(int(x) for x in elems):
        for b in (2 * e % 32, (2 * e + 1) % 32):
            banks.setdefault(b, set()).add(e)
    return max(len(v) for v in banks.values())


@pytest.mark.parametrize("logl,logt", [(10, 3), (11, 2), (12, 1), (9, 4), (8, 4)])
def test_column_tile_bank_spread(logl, logt):
    """With one padding row per 32 rows, a warp's stage reads and the epilogue
    writes take the minimum two wavefronts, and its sheared-walk reads at most
    three for every shear tried (the element-wise padding needed up to eight)."""
    L, T = 1 << logl, 1 << logt
    P = L // R
    nthr = P * T
    worst_walk = 0
    for alpha in (0, 1, 2, 3, 4, 5, 7, 12, 37, 100, L // 2 + 1, L - 1):
        for w in range(0, nthr // 32, max(1, nthr // 32 // 4)):
            th = np.arange(32) + 32 * w
            tc, p = th & (T - 1), th >> logt
            for r in range(0, R, 7):
                if alpha == 0:
                    assert _wavefronts(phys(p + P * r, logt) + tc) == 2
                i = (p + (tc * alpha) % L + r * P) % L
                worst_walk = max(worst_walk, _wavefronts(phys(i, logt) + tc))
    assert worst_walk <= 3
