"""GPU parity of the Smith-coordinate layout (PFFT_FLAG_LAYOUT_SNF, the
reordering-free order of Section 4): input indexed by lambda, output by mu,
row-major over the cycles.  Checked two ways: against the oracle's transform
of diag(eps) (the d-dimensional DFT that Theorem 1 gives in Smith
coordinates), and against the oracle's box-layout transform of M carried
through the lambda / mu maps (whose phase identity is pinned in
test_fft_parity.py)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import rel_l2

pytestmark = pytest.mark.gpu

CASES = [SI.M_SMALL_2D, [[4, -3], [4, 5]], [[6, 2, 0], [0, 6, 3], [0, 0, 6]], [[9, 0, 3], [0, 12, 2], [0, 0, 10]],
         [[4, 1], [0, 8192]], [[509, 0], [0, 67]], [[8, 2], [2, -4]]]


def _maps(M):
    box = pf.PatternFFT(M, 1)
    n = [int(e) for e in box.eps if e > 1]
    lam = box.index_map(pf.PFFT_MAP_INPUT_SNF)
    mu = box.index_map(pf.PFFT_MAP_OUTPUT_SNF)
    return box, n, np.ravel_multi_index(tuple(lam.T), n), np.ravel_multi_index(tuple(mu.T), n)


@pytest.mark.parametrize("M", CASES, ids=[str(i) for i in range(len(CASES))])
def test_snf_layout_full(M):
    box, n, fl, fm = _maps(M)
    eps = [int(e) for e in box.eps]
    m = box.m
    snf = pf.PatternFFT(M, 2, layout="snf")
    assert [int(e) for e in snf.in_box] == eps and [int(e) for e in snf.out_box] == eps
    c = SI.complex_normal(2, m, m % 83)
    x = np.empty_like(c)
    x[:, fl] = c
    y = snf.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_l2(y, oracle.pattern_fft(np.diag(eps).tolist(), x)) <= 1e-5
    ref_box = oracle.pattern_fft(M, c)
    expect = np.empty_like(ref_box)
    expect[:, fm] = ref_box
    assert rel_l2(y, expect) <= 1e-5
    back = snf.inverse(torch.from_numpy(y).cuda()).cpu().numpy()
    assert rel_l2(back, x) <= 1e-5


def test_snf_layout_batched_workload_sampled():
    w = SI.WORKLOADS["batched_2d"]
    M = w["M"]
    box, n, fl, fm = _maps(M)
    eps = [int(e) for e in box.eps]
    m = box.m
    snf = pf.PatternFFT(M, 2, layout="snf")
    c = SI.complex_normal(2, m, w["seed"])
    x = np.empty_like(c)
    x[:, fl] = c
    y = snf.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    slots = SI.sample_slots(m, 2048)
    assert rel_l2(y[:1, slots], oracle.pattern_fft(np.diag(eps).tolist(), x[:1], out_slots=slots)) <= 1e-5
    inv = np.empty(m, dtype=np.int64)
    inv[fm] = np.arange(m)                      # mu-slot -> box slot k
    ks = inv[slots]
    assert rel_l2(y[:1, slots], oracle.pattern_fft(M, c[:1], out_slots=ks)) <= 1e-5


@pytest.mark.parametrize("M,Js", [([[8, 8], [-8, 8]], [SI.J_DIAG_A, SI.J_DIAG_B]),
                                  ([[12, 4], [0, 10]], [[[2, 0], [0, 1]], [[1, 0], [0, 2]]]),
                                  ([[10, 1, 7], [0, 9, 1], [0, 0, 32]], [[[1, 0, 0], [-1, 2, 0], [0, 0, 1]]]),
                                  ([[32, 32], [-32, 32]], SI.wavelet_dilations(3))])
@pytest.mark.parametrize("sym", [pf.PWT_DIRICHLET, pf.PWT_DLVP])
def test_transform_then_split_in_smith_coordinates(M, Js, sym):
    """The pipeline without reordering: transform in the Smith-coordinate
    layout, split reading that order (PWT_FLAG_INPUT_SNF); against the
    oracle's transform and split in the box layout; reconstruction returns the
    Smith-ordered coefficients."""
    box, n, fl, fm = _maps(M)
    m = box.m
    c = SI.complex_normal(2, m, 7)
    x = np.empty_like(c)
    x[:, fl] = c
    chat_snf = pf.PatternFFT(M, 2, layout="snf").forward(torch.from_numpy(x).cuda())
    split = pf.WaveletSplit(M, Js, sym, 0.125, 2, input_layout="snf")
    sc, wv = split.decompose(chat_snf)
    osym = oracle.DIRICHLET if sym == pf.PWT_DIRICHLET else oracle.DLVP
    s_ref, w_ref = oracle.wavelet_cascade(M, Js, oracle.pattern_fft(M, c), osym, 0.125)
    assert rel_l2(sc.cpu().numpy(), s_ref) <= 1e-5
    for a, b in zip(wv, w_ref):
        assert rel_l2(a.cpu().numpy(), b) <= 1e-5
    back = split.reconstruct(sc, wv).cpu().numpy()
    assert rel_l2(back, chat_snf.cpu().numpy()) <= 1e-5
