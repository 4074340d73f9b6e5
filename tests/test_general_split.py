"""GPU parity of the general split step (Section 5.3, step 4) for |det J| = p
with cyclic G(J^T) and caller symbols (pwt_split_general / pwt_merge_general)
against the oracle's fibre sums."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import TOL, rel_l2

pytestmark = pytest.mark.gpu

CASES = [([[6, 1], [0, 9]], [[1, 0], [0, 3]]),
         ([[10, 5], [5, 15]], [[1, 1], [-1, 4]]),
         ([[8, 4], [0, 12]], [[2, 0], [0, 1]]),
         ([[4, 1, 0], [0, 6, 2], [0, 0, 7]], [[1, 0, 0], [0, 1, 0], [0, 0, 7]]),
         ([[12, 4], [4, 12]], [[1, 1], [-1, 3]]),
         ([[130, 13], [0, 169]], [[13, 0], [0, 1]]),                   # p = 13
         ([[96, 32], [0, 256]], [[1, 0], [0, 16]])]                    # p = 16, 24576 points


def _gpu(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_general_split_and_merge_vs_oracle(case, dtype):
    M, J = CASES[case]
    m, p = abs(L.det(M)), abs(L.det(J))
    sym = SI.complex_normal(p, m, 40 + case, dtype=np.complex128)
    c = SI.complex_normal(2, m, 50 + case, dtype=np.complex128)
    tol = TOL["c64" if dtype == torch.complex64 else "c128"]
    parts = pf.split_general(M, J, _gpu(sym, dtype), _gpu(c, dtype)).cpu().numpy()
    ref = oracle.split_general(M, J, sym, c)
    assert rel_l2(parts.reshape(p * 2, -1), ref.reshape(p * 2, -1)) <= tol
    back = pf.merge_general(M, J, _gpu(sym, dtype), _gpu(ref, dtype)).cpu().numpy()
    assert rel_l2(back, oracle.merge_general(M, J, sym, ref)) <= tol


@pytest.mark.parametrize("case", [0, 1, 3, 6])
def test_general_split_unitary_round_trip(case):
    """The p-point DFT symbol system is unitary on every fibre: merge(split(c)) = c."""
    M, J = CASES[case]
    m = abs(L.det(M))
    S, p, n = oracle._general_fibres(M, J)
    sym = np.zeros((p, m), dtype=np.complex128)
    for t in range(p):
        for j in range(p):
            sym[j, S[:, t]] = np.exp(-2j * np.pi * j * t / p)
    c = SI.complex_normal(3, m, 60 + case)
    sg = _gpu(sym, torch.complex64)
    parts = pf.split_general(M, J, sg, _gpu(c, torch.complex64))
    back = pf.merge_general(M, J, sg, parts).cpu().numpy()
    assert rel_l2(back, c) <= 1e-5


def test_general_split_errors():
    x = torch.zeros(1, 16, dtype=torch.complex64, device="cuda")
    s4 = torch.zeros(4, 16, dtype=torch.complex64, device="cuda")
    with pytest.raises(pf.PfftError) as e:   # G(J^T) = Z_2 x Z_2 is not cyclic
        pf.split_general([[4, 0], [0, 4]], [[2, 0], [0, 2]], s4, x)
    assert e.value.status == 5
    s3 = torch.zeros(3, 16, dtype=torch.complex64, device="cuda")
    with pytest.raises(pf.PfftError) as e:   # J^{-1} M not integral
        pf.split_general([[4, 0], [0, 4]], [[3, 0], [0, 1]], s3, x)
    assert e.value.status in (3, 4, 5)
    big = torch.zeros(17, 34, dtype=torch.complex64, device="cuda")
    with pytest.raises(pf.PfftError) as e:   # p = 17 > 16
        pf.split_general([[17, 0], [0, 2]], [[17, 0], [0, 1]], big, torch.zeros(1, 34, dtype=torch.complex64,
                                                                               device="cuda"))
    assert e.value.status == 5


# Built-in band system (symbols NULL): dilations of prime determinant p
# (the harness's prime dilation for the p dividing det M), against the
# oracle's Householder-completed Dirichlet system.
BUILTIN = [([[9, 0], [0, 9]], [[3, 0], [0, 1]]),
           ([[9, 6], [9, 15]], [[1, 0], [-2, 3]]),
           ([[15, 5], [0, 10]], [[1, 0], [0, 5]]),
           ([[6, 1, 2], [0, 7, 3], [0, 0, 14]], [[1, 0, 0], [0, 1, 0], [0, 0, 7]]),
           ([[31, 7], [0, 62]], SI.prime_dilation([[31, 7], [0, 62]], 31)),
           ([[127, 3], [0, 254]], SI.prime_dilation([[127, 3], [0, 254]], 127)),
           ([[8, 8], [-8, 8]], SI.J_DIAG_A)]


@pytest.mark.parametrize("case", range(len(BUILTIN)))
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_builtin_band_system_vs_oracle(case, dtype):
    M, J = BUILTIN[case]
    m, p = abs(L.det(M)), abs(L.det(J))
    c = SI.complex_normal(2, m, 70 + case, dtype=np.complex128)
    tol = TOL["c64" if dtype == torch.complex64 else "c128"]
    parts = pf.split_general(M, J, None, _gpu(c, dtype)).cpu().numpy()
    ref = oracle.wavelet_level_p(M, J, c_hat=c)
    for j in range(p):
        assert rel_l2(parts[j], ref[j]) <= tol or np.linalg.norm(ref[j]) < 1e-12 * np.linalg.norm(c), j
    assert rel_l2(parts.transpose(1, 0, 2).reshape(2, -1), ref.transpose(1, 0, 2).reshape(2, -1)) <= tol
    back = pf.merge_general(M, J, None, _gpu(ref, dtype)).cpu().numpy()
    assert rel_l2(back, c) <= tol


def test_builtin_band_system_p2_equals_the_dirichlet_split():
    """For p = 2 the built-in system is the split of pwt_decompose (Dirichlet)."""
    M, J = [[64, 64], [-64, 64]], SI.J_DIAG_A
    c = _gpu(SI.complex_normal(3, 8192, 77), torch.complex64)
    parts = pf.split_general(M, J, None, c)
    plan = pf.WaveletSplit(M, [J], pf.PWT_DIRICHLET, 0.125, 3)
    s, w = plan.decompose(c)
    assert rel_l2(parts[0].cpu().numpy(), s.cpu().numpy()) <= 1e-6
    assert rel_l2(parts[1].cpu().numpy(), w[0].cpu().numpy()) <= 1e-6
