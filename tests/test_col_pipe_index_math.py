"""Host model of the persistent pipelined column pass (pencils of 2^10
complex64 points, 8 columns per tile, 256 threads: thread (c, p) holds rows
p + 32 k of column c).

The model replays every shared-memory access of the kernel for one tile:

* the dense tile read (forward) or the walk-layout gather (inverse), the
  radix-32 stage, the exchange in two rounds through the padded half tile X
  (both directions; round h moves register half h xor bit 4 of p) and the
  twiddled second stage give each column's
  1024-point DFT
  (numpy), v[r] of thread (c, p) = frequency p + 32 r;
* in the two output rounds each slot of X is written once, and the walker
  (c, p) reads at step j exactly the frequency i_j = (p + c alpha + 32 j)
  mod 1024 of column c -- the order of the sheared walk -- for every shear
  alpha;
* every warp access (dense reads, exchange writes and reads, X writes and
  reads) costs the minimum of two wavefronts.

Plain integer arithmetic and numpy, no GPU."""
import numpy as np
import pytest

from test_row_pipe_index_math import wavefronts

L, T, P, R = 1024, 8, 32, 32


def ct_phys(i):
    return (i + (i >> 5)) << 3


def masked_wavefronts(words, active):
    """wavefronts() for a predicated access: inactive lanes take no bank slot."""
    total = 0
    for half in (slice(0, 16), slice(16, 32)):
        per_bank = {}
        for w, on in zip(words[half], active[half]):
            if on:
                for b in (w % 32, (w + 1) % 32):
                    per_bank.setdefault(b, set()).add(w // 2)
        total += max((len(x) for x in per_bank.values()), default=0)
    return total


def check_banks(idx):
    """idx[thread] -> element index of one access; threads tid = p * 8 + c."""
    for w in range(256 // 32):
        assert wavefronts(2 * idx[32 * w:32 * w + 32]) == 2


def model(tile, alpha, check=True):
    tid = np.arange(256)
    c, p = tid & 7, tid >> 3
    v = np.empty((256, R), complex)
    for k in range(R):
        idx = (p + P * k) * T + c
        v[:, k] = tile.reshape(-1)[idx]
        if check:
            check_banks(idx)
    v = np.fft.fft(v, axis=1)  # stage 0 (Ns = 1): output r at position 32 p + r
    # exchange in two rounds through the padded half tile X: round h moves
    # register half H = h xor bit 4 of p; bit 9 of the position is dropped
    XS = ct_phys(L // 2)
    for h in range(2):
        X = np.full(XS, np.nan + 0j)
        H = h ^ ((p >> 4) & 1)
        regs = 16 * H[:, None] + np.arange(16)[None, :]
        widx = ct_phys(32 * (p & 15))[:, None] + ct_phys(regs) + c[:, None]
        pos_w = 32 * p[:, None] + regs
        assert (((pos_w >> 9) ^ (pos_w >> 4)) & 1 == h).all()
        assert (widx == ct_phys(pos_w & 511) + c[:, None]).all()
        assert len(np.unique(widx)) == widx.size and widx.max() < XS
        X[widx] = v[tid[:, None], regs]
        ridx = ct_phys(p)[:, None] + ct_phys(32 * np.arange(16))[None, :] + c[:, None]
        pos_r = p[:, None] + 32 * regs
        assert (((pos_r >> 9) ^ (pos_r >> 4)) & 1 == h).all()
        assert (ridx == ct_phys(pos_r & 511) + c[:, None]).all()
        v[tid[:, None], regs] = X[ridx]
        if check:
            for j in range(16):
                check_banks(widx[:, j])
                check_banks(ridx[:, j])
    assert not np.isnan(v).any()
    v *= np.exp(-2j * np.pi * np.outer(p, np.arange(R)) / L)
    v = np.fft.fft(v, axis=1)  # v[r] = frequency p + 32 r
    # two output rounds
    off = (c * alpha) % L
    i0 = p + off
    i0 = np.where(i0 >= L, i0 - L, i0)
    pw = (p - off) & (P - 1)
    i0w = pw + off
    i0w = np.where(i0w >= L, i0w - L, i0w)
    m0h = i0w >> 5
    sw = i0 & (P - 1)
    got = np.empty((256, R), complex)
    for h in range(2):
        X = np.full(16 * P * T, np.nan + 0j)
        written = np.zeros(16 * P * T, bool)
        for r in range(R):
            t = (r - m0h - 16 * h) & 31
            sel = t < 16
            idx = (t * P + p) * T + c
            assert not written[idx[sel]].any()
            written[idx[sel]] = True
            X[idx[sel]] = v[sel, r]
            if check:
                # predicated lanes: only the active ones take bank slots
                for w in range(8):
                    assert masked_wavefronts(2 * idx[32 * w:32 * w + 32], sel[32 * w:32 * w + 32]) <= 2
        assert written.all()
        for t in range(16):
            idx = (t * P + sw) * T + c
            got[:, 16 * h + t] = X[idx]
            if check:
                check_banks(idx)
    return v, got, i0


@pytest.mark.parametrize("alpha", [0, 1, 5, 96, 513, 1023])
def test_pipelined_column_tile(alpha):
    rng = np.random.default_rng(alpha)
    tile = rng.standard_normal((L, T)) + 1j * rng.standard_normal((L, T))
    v, got, i0 = model(tile, alpha, check=alpha in (1, 513))
    ref = np.fft.fft(tile, axis=0)  # [frequency, column]
    tid = np.arange(256)
    c, p = tid & 7, tid >> 3
    for r in range(R):
        assert np.allclose(v[:, r], ref[p + P * r, c], atol=1e-9 * np.abs(ref).max())
    for j in range(R):
        i_j = (i0 + 32 * j) % L
        assert np.allclose(got[:, j], ref[i_j, c], atol=1e-9 * np.abs(ref).max())


def test_forward_loads_cover_the_tile_aligned():
    """16-byte pieces: thread tid, piece i covers row (tid + 256 i) >> 2,
    columns 2 ((tid + 256 i) & 3) + {0, 1}; every element of the tile once."""
    seen = np.zeros((L, T), int)
    for i in range(16):
        cpiece = np.arange(256) + 256 * i
        row, part = cpiece >> 2, cpiece & 3
        for e in range(2):
            np.add.at(seen, (row, 2 * part + e), 1)
        assert ((row * T + part * 2) * 8 % 16 == 0).all()
    assert (seen == 1).all()


def test_shared_memory_layout_fits_two_ctas_per_sm():
    S = L * T
    X = max(ct_phys(L // 2), 16 * P * T)
    Es = 2 * T * 4 * 4 // 8  # two tiles' column points, 4 int32 each, in 8-byte elements
    stw_n = 166
    per_cta = (ct_phys(L) + X + Es + stw_n) * 8
    assert ct_phys(L) >= S and Es == 32 and per_cta <= 110 * 1024 and 2 * (per_cta + 1024) <= 228 * 1024


@pytest.mark.parametrize("alpha", [0, 3, 96, 513])
def test_inverse_gather_in_walk_layout(alpha):
    """Inverse direction: walker (c, p) gathers step j = 16 h + t of its walk
    (row (i_0 + 32 j) mod 1024 of column c) into W[j][p][c] in S (two halves
    of 16 steps, issued together); thread (c, p) then finds its register k
    (row p + 32 k) at step j = (k - m0h) mod 32 of walker pw = (p - c alpha)
    mod 32 -- every register once, every access conflict free, and the walk
    layout fits the tile buffer."""
    tid = np.arange(256)
    c, p = tid & 7, tid >> 3
    off = (c * alpha) % L
    i0 = (p + off) % L
    W = np.full(ct_phys(L), -1, np.int64)  # S holds the padded tile's worth of elements
    for h in range(2):
        for t in range(16):
            j = 16 * h + t
            rows = (i0 + 32 * j) % L
            idx = h * 16 * P * T + t * P * T + p * T + c  # S + h 16 NT + t NT + p T + c
            assert (W[idx] == -1).all()
            W[idx] = rows * T + c  # the tile element gathered
            if alpha in (3, 513):
                check_banks(idx)
    pw = (p - off) & (P - 1)
    m0h = ((pw + off) % L) >> 5
    for k in range(R):
        j = (k - m0h) & 31
        idx = j * P * T + pw * T + c
        assert (W[idx] == (p + P * k) * T + c).all()
        if alpha in (3, 513):
            check_banks(idx)
