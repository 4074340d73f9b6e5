"""Host model of the persistent pipelined row pass (rows of 2^14 complex64
points: radix 16 x 32 x 32 Stockham stages on 512 threads, exchanges and
output in two rounds of 2^13 elements through a padded buffer X).

The model replays, for every thread and register, the element each kernel
step reads or writes, with numpy's FFT for the butterflies:

* the row computed through the kernel's loads, two-round exchanges and
  stage twiddles equals the 2^14-point DFT (numpy), in the register order
  the output stage assumes (v[r] of thread p = frequency p + 512 r);
* in every exchange round each slot of X is written once and read once, and
  every index stays inside the buffer of 2^13 + 2^9 elements;
* the forward output (workspace order, column permutation PI with block
  staging) puts every element at its position, for several permutations;
* the padding spreads every warp access of X over the banks: at most two
  wavefronts per 32 eight-byte accesses (the minimum).

Plain integer arithmetic and numpy, no GPU."""
import numpy as np
import pytest

P, L, HALF = 512, 1 << 14, 1 << 13
XSIZE = HALF + (HALF >> 4)


def xphys(i):
    return i + (i >> 4)


def wavefronts(addr_words):
    """Shared-memory wavefronts of one warp of 8-byte accesses (word addresses
    of 32 lanes): two half-warps, each costing the largest number of distinct
    8-byte slots that meet in one bank."""
    total = 0
    for half in (addr_words[:16], addr_words[16:]):
        per_bank = {}
        for w in half:
            for b in (w % 32, (w + 1) % 32):
                per_bank.setdefault(b, set()).add(w // 2)
        total += max(len(s) for s in per_bank.values())
    return total


class XBuffer:
    """X with a per-round check: every slot written at most once, every read
    of a slot written in the same round."""

    def __init__(self):
        self.data = np.zeros(XSIZE, complex)
        self.new_round()

    def new_round(self):
        self.written = np.zeros(XSIZE, bool)

    def write(self, idx, val):
        assert idx.min() >= 0 and idx.max() < XSIZE
        flat = idx.reshape(-1)
        assert len(np.unique(flat)) == len(flat)
        assert not self.written[flat].any()
        self.written[flat] = True
        self.data[idx] = val

    def read(self, idx):
        assert self.written[idx].all()
        return self.data[idx]


def kernel_model(x, check_banks=False):
    p = np.arange(P)
    v = np.empty((P, 32), complex)
    for q in range(2):
        for r in range(16):
            v[:, 16 * q + r] = x[p + P * (q + 2 * r)]
    X = XBuffer()
    banks = []
    # tail stage and exchange 1
    for q in range(2):
        v[:, 16 * q:16 * q + 16] = np.fft.fft(v[:, 16 * q:16 * q + 16], axis=1)
        X.new_round()
        widx = np.stack([xphys((p << 4) | r) for r in range(16)], axis=1)
        X.write(widx, v[:, 16 * q:16 * q + 16])
        ridx = np.stack([xphys((r << 9) | p) for r in range(16)], axis=1)
        v[:, 16 * q:16 * q + 16] = X.read(ridx)
        banks += [widx, ridx]
    # stage 0 (Ns = 16)
    k = p & 15
    v *= np.exp(-2j * np.pi * np.outer(k, np.arange(32)) / 512)
    v = np.fft.fft(v, axis=1)
    # exchange 2: round h, register half H = h xor bit 8 of p
    for h in range(2):
        X.new_round()
        H = h ^ ((p >> 8) & 1)
        base = (((p >> 4) & 15) << 9) | (p & 15)
        regs = 16 * H[:, None] + np.arange(16)[None, :]
        widx = xphys(base[:, None] | (regs << 4))
        X.write(widx, v[p[:, None], regs])
        ridx = xphys((np.arange(16)[None, :] << 9) | p[:, None])
        v[p[:, None], regs] = X.read(ridx)
        banks += [widx, ridx]
    # stage 1 (Ns = 512)
    v *= np.exp(-2j * np.pi * np.outer(p, np.arange(32)) / L)
    v = np.fft.fft(v, axis=1)
    out = np.empty(L, complex)
    out[p[:, None] + P * np.arange(32)[None, :]] = v
    if check_banks:
        for idx in banks:
            for w in range(P // 32):
                lanes = idx[32 * w:32 * w + 32]
                for j in range(lanes.shape[1]):
                    assert wavefronts(2 * lanes[:, j]) == 2
    return v, out


def test_pipelined_row_is_the_dft():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    _, out = kernel_model(x, check_banks=True)
    ref = np.fft.fft(x)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-12


def ws_pos(p, k, lg, inv):
    """Arithmetic walk of the workspace permutation (lg <= 9)."""
    ls = 14 - lg
    lo = p & ((1 << lg) - 1)
    return (lo << ls) + ((((p >> lg) * inv) + k * (inv << (9 - lg))) & ((1 << ls) - 1))


def pi_formula(mu, lg, inv):
    ls = 14 - lg
    return ((mu & ((1 << lg) - 1)) << ls) | (((mu >> lg) * inv) & ((1 << ls) - 1))


@pytest.mark.parametrize("lg,inv", [(0, 1), (0, 12345), (2, 4095), (4, 31), (6, 1), (1, 8191)])
def test_forward_output_rounds_place_every_position(lg, inv):
    ls = 14 - lg
    assert inv % 2 == 1
    pad = (max(16, 128 >> lg) // 8) if lg > 0 else 0
    p = np.arange(P)
    vals = (p[:, None] * 32 + np.arange(32)[None, :]).astype(np.int64)  # element id p + 512 k <-> value
    ws = np.full(L, -1, np.int64)
    for h in range(2):
        X = np.full(XSIZE, -1, np.int64)
        for k in range(32):
            pos = ws_pos(p, k, lg, inv)
            assert (pos == pi_formula(p + P * k, lg, inv)).all()
            sel = (pos >> 13) == h
            if not sel.any():
                continue
            q = pos[sel] & (HALF - 1)
            idx = q + (q >> ls) * pad if pad else q
            assert idx.max() < XSIZE and (X[idx] == -1).all()
            X[idx] = vals[sel, k]
        nbh = (HALF >> ls) if pad else 1
        sph = HALF // nbh
        for c in range(nbh):
            ws[h * HALF + c * sph:h * HALF + (c + 1) * sph] = X[c * (sph + pad):c * (sph + pad) + sph]
            assert ((c * (sph + pad)) * 8) % 16 == 0 and (sph * 8) % 16 == 0
    # every position holds the element (value id p * 32 + k <-> element p + 512 k)
    # whose permuted position it is
    elem = (ws // 32) + P * (ws % 32)
    assert (np.sort(ws) == np.arange(L)).all()
    assert (pi_formula(elem, lg, inv) == np.arange(L)).all()


def test_inverse_output_rounds_split_runs():
    """Element-order output: round h sends the part of every run inside
    [2^13 h, 2^13 (h + 1)); pieces stay 16-byte aligned when runs are."""
    runs = [(0, 4096, 4096), (4096, 0, 4096), (8192, 12288, 4096), (12288, 8192, 4096)]
    runs += [(0, 100, 10000), (10000, 20000, 6384)]
    for x0, y0, z in runs:
        for h in range(2):
            lo, hi = max(x0, h * HALF), min(x0 + z, (h + 1) * HALF)
            if hi > lo:
                assert 0 <= lo - h * HALF and hi - h * HALF <= HALF
                assert (lo - x0) % 2 == 0 and (lo - h * HALF) % 2 == 0 and (hi - lo) % 2 == 0


def test_single_round_exchange1_fits_s_and_x():
    """Exchange 1 in one round (X1S): positions (q << 13) | (p << 4) | r
    written and (r << 9) | p read through the padded region that starts at S
    and runs into X; a bijection inside the 2^14 + 2^10 slots, with two
    wavefronts per warp access."""
    p = np.arange(P)
    w = np.stack([xphys((q << 13) | (p << 4) | r) for q in range(2) for r in range(16)], axis=1)
    rd = np.stack([xphys((r << 9) | p) for r in range(32)], axis=1)
    for idx in (w, rd):
        flat = idx.reshape(-1)
        assert len(np.unique(flat)) == L and flat.max() < L + (L >> 4)
        for wp in range(P // 32):
            for j in range(idx.shape[1]):
                assert wavefronts(2 * idx[32 * wp:32 * wp + 32, j]) == 2
    assert set(w.reshape(-1)) == set(rd.reshape(-1))
    # S holds 2^14 elements plus staging pads, X starts at a multiple of 16
    # elements after it and holds 2^13 + 2^9: the region fits for any pad
    for s_el in (L, L + 64 * 2, L + 4 * 4):
        x_off = (s_el + 15) & ~15
        assert L + (L >> 4) <= x_off + XSIZE


@pytest.mark.parametrize("lg", [0, 1, 2, 3])
def test_direct_forward_output_is_the_permutation(lg):
    """Forward output from registers when the permutation multiplier is 1:
    element p + 512 k goes to ((p mod 2^lg) << ls) + (p >> lg) + k 2^(9 - lg);
    lanes of a warp form runs of 2^(5 - lg) consecutive positions."""
    ls = 14 - lg
    p = np.arange(P)
    for k in range(32):
        pos = ((p & ((1 << lg) - 1)) << ls) + (p >> lg) + k * (P >> lg)
        assert (pos == pi_formula(p + P * k, lg, 1)).all()
        for wp in range(P // 32):
            lanes = np.sort(pos[32 * wp:32 * wp + 32])
            runs = np.split(lanes, np.where(np.diff(lanes) != 1)[0] + 1)
            assert min(len(r) for r in runs) >= 1 << (5 - lg)


@pytest.mark.parametrize("lrun", [5, 9, 12, 14])
def test_direct_inverse_output_finds_the_run(lrun):
    """Box rows of uniform runs of 2^lrun elements (run j covers elements
    [j 2^lrun, (j + 1) 2^lrun)): element e is stored at y_j + (e mod 2^lrun),
    j = e >> lrun, and a warp's 32 consecutive elements stay in one run."""
    rng = np.random.default_rng(lrun)
    nr = L >> lrun
    y = rng.permutation(nr) * (1 << lrun) + 7
    e = np.arange(L)
    slot = y[e >> lrun] + (e & ((1 << lrun) - 1))
    assert len(np.unique(slot)) == L
    for wp in range(L // 32):
        j = e[32 * wp:32 * wp + 32] >> lrun
        assert (j == j[0]).all()
