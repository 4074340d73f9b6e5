"""Host model of the register-resident column pass over two pencil axes
(fft_fast2.cuh), without a GPU.

The pass runs the 1-D Stockham DFT of length L = n0 n1 that the
register-resident kernels use (a tail stage of radix t = L / 32^s first,
then s radix-32 stages) on a pencil whose rows are r = i0 n1 + i1, with two
changes made by the planner and the output indexing:

* the stage tables: from span Ns = n0 on, the twiddle of k at span Ns is
  that of floor(k / n0) at span Ns / n0 (entries of a table of order nD,
  index ((k' 2^b) mod (Ns' R)) (nD / (Ns' R)), powers composed from the
  binary digits of r as main_twiddle does);
* the output at position f0 + n0 f1 is written to row f0 n1 + f1.

The model checks that this is the 2-D DFT of the pencil (numpy fft2) for
every pair of axis lengths the planner accepts (n0 a product of the first
stages' radices), that the planner's axis order accepts exactly those pairs,
and that a pair with the boundary inside a stage is not the 2-D DFT."""
import numpy as np
import pytest

R = 32


def stages(L):
    lg = L.bit_length() - 1
    nmain = lg // 5
    return 1 << (lg - 5 * nmain), nmain


def fast2_axes(top, low):
    """The planner's acceptance rule (fft_plan.cu, fast2_axes)."""
    if top < 2 or low < 2 or top & (top - 1) or low & (low - 1):
        return False
    L = top * low
    if L < 64 or L > 16384:
        return False
    t, nmain = stages(L)
    return top in [t * 32 ** j for j in range(nmain)]


def table(L, n0, nD):
    """Stage tables as the planner builds them: per main stage s, for k < Ns
    and b < 5, the entry index into exp(-2 pi i t / nD)."""
    t, nmain = stages(L)
    out, Ns = [], t
    for _ in range(nmain):
        two = Ns >= n0
        NsR = (Ns // n0 if two else Ns) * R
        out.append([[((k // n0 if two else k) << b) % NsR * (nD // NsR) for b in range(5)] for k in range(Ns)])
        Ns *= R
    return out


def pencil_dft(x, n0, nD):
    L = len(x)
    t, nmain = stages(L)
    tw = np.exp(-2j * np.pi * np.arange(nD) / nD)
    tabs = table(L, n0, nD)
    # tail stage (Ns = 1, no twiddles), then the main stages
    for radix, tab in [(t, None)] + [(R, tb) for tb in tabs]:
        if radix == 1:
            continue
        Ns = 1 if tab is None else len(tab)
        P = L // radix
        y = np.empty_like(x)
        for j in range(P):
            k = j % Ns
            v = x[j + P * np.arange(radix)]
            if tab is not None and k:
                pw = tw[tab[k]]
                f = np.array([np.prod([pw[b] for b in range(5) if (r >> b) & 1]) for r in range(radix)])
                v = v * f
            v = np.fft.fft(v)
            y[(j - k) * radix + k + Ns * np.arange(radix)] = v
        x = y
    return x


def row_of(pos, n0, n1):
    return (pos % n0) * n1 + pos // n0


PAIRS = [(t, low) for t in (2, 4, 8, 16, 32, 64, 128, 256) for low in (2, 4, 8, 16, 32, 64, 128, 256, 512)
         if fast2_axes(t, low) and t * low <= 4096]


@pytest.mark.parametrize("n0,n1", PAIRS)
def test_two_axis_pass_is_the_2d_dft(n0, n1):
    rng = np.random.default_rng(n0 * 1000 + n1)
    L = n0 * n1
    nD = max(L, 8192)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    y = pencil_dft(x.copy(), n0, nD)
    out = np.empty_like(y)
    out[row_of(np.arange(L), n0, n1)] = y
    assert np.allclose(out, np.fft.fft2(x.reshape(n0, n1)).reshape(-1), atol=1e-9 * np.sqrt(L))


def test_acceptance_is_a_stage_boundary():
    for L in (64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384):
        t, nmain = stages(L)
        bounds = {t * 32 ** j for j in range(nmain)} - {1}
        got = {top for top in (1 << k for k in range(1, L.bit_length())) if top < L and fast2_axes(top, L // top)}
        assert got == bounds
    # config 3's pencil (cycles 32 and 64): only the order 64 x 32 starts on a boundary
    assert not fast2_axes(32, 64) and fast2_axes(64, 32)


def test_boundary_inside_a_stage_is_not_the_2d_dft():
    n0, n1 = 32, 64  # L = 2048 = 2 x 32 x 32: the boundary 32 falls inside the second stage
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n0 * n1) + 1j * rng.standard_normal(n0 * n1)
    y = pencil_dft(x.copy(), n0, 8192)
    out = np.empty_like(y)
    out[row_of(np.arange(n0 * n1), n0, n1)] = y
    assert not np.allclose(out, np.fft.fft2(x.reshape(n0, n1)).reshape(-1), atol=1e-6)
