"""GPU parity of the passes specialised at compile time -- the column pass
on (L, T) (complex64, L = 2^6 .. 2^13, T = min(16, 8192 / L), d = 2 and 3)
and the bulk-copy row pass on rows of 2^13 and 2^14 -- against the FP64
oracle, forward and inverse, through the C ABI.

Each pattern is built to have the Smith form diag(L, n) (d = 2) or
diag(1, L, n) (d = 3), so that its column pass is a single power-of-two
pencil axis of length L: the case the specialised kernels take over.  The
patterns carry shears, so the sheared walk wraps for most columns."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import rel_l2

pytestmark = pytest.mark.gpu


def _mm(A, B):
    return [[sum(A[i][k] * B[k][j] for k in range(len(B))) for j in range(len(B[0]))] for i in range(len(A))]


def _pattern(d, lg):
    """(M, expected nontrivial Smith diagonal) with column pencil length 2^lg."""
    if d == 2:
        if lg <= 11:
            return [[2 ** (lg + 1), 3 * 2 ** lg], [0, 2 ** (lg + 1)]], [2 ** lg, 2 ** (lg + 2)]
        return [[2 ** lg, 2 ** (lg + 1)], [0, 2 ** lg]], [2 ** lg, 2 ** lg]
    K = lg if lg >= 11 else lg + 2
    U = [[1, 1, 0], [0, 1, 1], [0, 0, 1]]
    V = [[1, 0, 0], [2, 1, 0], [1, 3, 1]]
    return _mm(_mm(U, [[1, 0, 0], [0, 2 ** lg, 0], [0, 0, 2 ** K]]), V), [2 ** lg, 2 ** K]


CASES = [(d, lg) for d in (2, 3) for lg in range(6, 14)]


@pytest.mark.parametrize("d,lg", CASES, ids=[f"d{d}-L{2 ** lg}" for d, lg in CASES])
def test_specialised_column_pass(d, lg):
    M, n = _pattern(d, lg)
    m = abs(L.det(M))
    plan = pf.PatternFFT(M, 2)
    assert [int(e) for e in plan.eps if e > 1] == n
    c = SI.complex_normal(2, m, seed=100 + 10 * d + lg)
    x = torch.from_numpy(c).cuda()
    y = plan.forward(x)
    yh = y.cpu().numpy()
    if m <= 1 << 16:
        assert rel_l2(yh, oracle.pattern_fft(M, c)) <= 1e-5
    else:
        slots = SI.sample_slots(m, 256 if m <= 1 << 22 else 64, seed=lg)
        assert rel_l2(yh[1:2, slots], oracle.pattern_fft(M, c[1:2], out_slots=slots)) <= 1e-5
    assert np.allclose(np.linalg.norm(yh, axis=1), np.linalg.norm(c, axis=1), rtol=1e-5)
    back = plan.inverse(y)
    plan.check_device_status()
    bh = back.cpu().numpy()
    assert rel_l2(bh, c) <= 1e-5
    slots = SI.sample_slots(m, 64, seed=lg + 1)
    ref = oracle.pattern_fft(M, yh[0:1].astype(np.complex128), inverse=True, out_slots=slots)
    assert rel_l2(bh[0:1, slots], ref) <= 1e-5


# Row passes of 2^13 and 2^14 elements (one row per CTA, bulk-copy staging):
# the compile-time specialised row kernel, with workspace permutations whose
# low-bit block count 2^lg is small (arithmetic walk) or the whole row (the
# diagonal pattern, where the fastest output coordinate misses the long cycle).
ROWS = [
    [[2, 0], [0, 16384]],                    # (2, 16384)
    [[8, 4], [0, 4096]],                     # (4, 8192), sheared
    [[64, 24], [0, 2048]],                   # (8, 16384)
    [[4096, 3072], [0, 4096]],               # (1024, 16384): the benchmark's family
    [[16384, 0], [0, 2]],                    # (2, 16384), long cycle along the slow axis
    _mm(_mm([[1, 1, 0], [0, 1, 1], [0, 0, 1]], [[1, 0, 0], [0, 2, 0], [0, 0, 16384]]),
        [[1, 0, 0], [2, 1, 0], [1, 3, 1]]),  # (1, 2, 16384) in d = 3
    _mm(_mm([[1, 1, 0], [0, 1, 1], [0, 0, 1]], [[1, 0, 0], [0, 16, 0], [0, 0, 8192]]),
        [[1, 0, 0], [2, 1, 0], [1, 3, 1]]),  # (1, 16, 8192) in d = 3
    [[8192, 2048], [0, 64]],                 # (64, 8192)
]


@pytest.mark.parametrize("M", ROWS, ids=[str(i) for i in range(len(ROWS))])
def test_specialised_row_pass(M):
    m = abs(L.det(M))
    plan = pf.PatternFFT(M, 2)
    c = SI.complex_normal(2, m, seed=200 + m % 89)
    x = torch.from_numpy(c).cuda()
    y = plan.forward(x)
    yh = y.cpu().numpy()
    if m <= 1 << 16:
        assert rel_l2(yh, oracle.pattern_fft(M, c)) <= 1e-5
    else:
        slots = SI.sample_slots(m, 256, seed=m % 13)
        assert rel_l2(yh[0:1, slots], oracle.pattern_fft(M, c[0:1], out_slots=slots)) <= 1e-5
    back = plan.inverse(y)
    plan.check_device_status()
    bh = back.cpu().numpy()
    assert rel_l2(bh, c) <= 1e-5
    slots = SI.sample_slots(m, 128, seed=m % 11)
    ref = oracle.pattern_fft(M, yh[1:2].astype(np.complex128), inverse=True, out_slots=slots)
    assert rel_l2(bh[1:2, slots], ref) <= 1e-5
