"""GPU parity of pattern batches -- many patterns of uneven size transformed
and split one level in grouped launches (pfft_batch_*) -- against the FP64
oracle, through the C ABI.

Small mixes are compared on every output of every pattern.  The uneven
serving-style mix (4096 patterns, about 2^28.7 points) in the benchmark's
launch configuration is compared on sampled frequencies of every pattern
(direct FP64 sums) and on sampled fibres of the split (the oracle's split of
a coefficient vector holding the oracle's values on those fibres), plus
Parseval and the Dirichlet norm identity per pattern at full size."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import rel_l2

pytestmark = pytest.mark.gpu

EXTRA = [[[37, 5], [0, 74]], [[509, 7], [0, 4]], [[2, 1], [0, 1]], [[11, 2, 3], [0, 13, 4], [0, 0, 2]],
         [[64, 0], [0, 64]]]


def _small_mix(seed):
    return SI.uneven_mix(40, seed=seed, max_det=4096, lo=2, hi=40, even_det=True) + EXTRA


def _np(t):
    return t.cpu().numpy()


def _split_ref_at(M, J, c, gslots, symbol, eta=0.125):
    """Oracle (d1, d2) at the slots gslots of the box of H(N^T): the oracle's
    transform on the two members of each fibre (direct sums), then the
    oracle's split of the coefficient vector that holds only those values."""
    N = oracle.exact_N(M, J)
    HM, HN = L.hnf(L.transpose(M)), L.hnf(L.transpose(N))
    NTl1 = L.matvec(L.transpose(N), oracle.nonzero_class_JT(J))
    slots = set()
    for g in gslots:
        y = L.point_of(HN, int(g))
        slots.add(L.slot_of(HM, L.box_reduce(HM, y)))
        slots.add(L.slot_of(HM, L.box_reduce(HM, [a + b for a, b in zip(y, NTl1)])))
    slots = np.array(sorted(slots))
    sparse = np.zeros((1, abs(L.det(M))), np.complex128)
    sparse[0, slots] = oracle.pattern_fft(M, c[None, :], out_slots=slots)[0]
    d1, d2 = oracle.wavelet_level(M, J, symbol, eta, c_hat=sparse)
    return d1[0, gslots], d2[0, gslots]


@pytest.mark.parametrize("symbol", [pf.PWT_DIRICHLET, pf.PWT_DLVP])
def test_small_mix_full(symbol):
    Ms = _small_mix(40 + symbol)
    Js = [SI.parity_dilation(M) for M in Ms]
    B = pf.PatternBatch(Ms, Js, symbol, 0.125)
    x = SI.complex_normal_flat(B.total, 41)
    chat, sc, wv = (_np(t) for t in B.forward(torch.from_numpy(x).cuda()))
    for i, (M, J) in enumerate(zip(Ms, Js)):
        o, m = int(B.offsets[i]), int(B.m[i])
        ref = oracle.pattern_fft(M, x[None, o:o + m])
        assert rel_l2(chat[o:o + m], ref[0]) <= 1e-5, (i, M)
        d1, d2 = oracle.wavelet_level(M, J, symbol, 0.125, c_hat=ref)
        h = slice(o // 2, (o + m) // 2)
        assert rel_l2(sc[h], d1[0]) <= 1e-5, (i, M)
        assert rel_l2(wv[h], d2[0]) <= 1e-5, (i, M)


def test_radix8_schedule_full():
    """The schedule with radix-8 power-of-two stages (one the autotuner may
    pick), every output of a small mix with large power-of-two factors."""
    Ms = _small_mix(80) + [[[256, 3], [0, 64]], [[128, 0, 0], [0, 8, 1], [0, 0, 4]]]
    Js = [SI.parity_dilation(M) for M in Ms]
    B = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, flags=pf.PFFT_BATCH_RADIX8)
    assert B.schedule()[3] == 8
    x = SI.complex_normal_flat(B.total, 81)
    chat, sc, wv = (_np(t) for t in B.forward(torch.from_numpy(x).cuda()))
    for i, (M, J) in enumerate(zip(Ms, Js)):
        o, m = int(B.offsets[i]), int(B.m[i])
        ref = oracle.pattern_fft(M, x[None, o:o + m])
        assert rel_l2(chat[o:o + m], ref[0]) <= 1e-5, (i, M)
        d1, d2 = oracle.wavelet_level(M, J, pf.PWT_DIRICHLET, c_hat=ref)
        assert rel_l2(sc[o // 2:(o + m) // 2], d1[0]) <= 1e-5
        assert rel_l2(wv[o // 2:(o + m) // 2], d2[0]) <= 1e-5


def test_small_mix_complex128():
    Ms = _small_mix(50)
    Js = [SI.parity_dilation(M) for M in Ms]
    B = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, dtype=torch.complex128)
    x = SI.complex_normal_flat(B.total, 51).astype(np.complex128)
    chat, sc, wv = (_np(t) for t in B.forward(torch.from_numpy(x).cuda()))
    for i, (M, J) in enumerate(zip(Ms, Js)):
        o, m = int(B.offsets[i]), int(B.m[i])
        ref = oracle.pattern_fft(M, x[None, o:o + m])
        assert rel_l2(chat[o:o + m], ref[0]) <= 1e-12, (i, M)
        d1, d2 = oracle.wavelet_level(M, J, pf.PWT_DIRICHLET, c_hat=ref)
        assert rel_l2(sc[o // 2:(o + m) // 2], d1[0]) <= 1e-12
        assert rel_l2(wv[o // 2:(o + m) // 2], d2[0]) <= 1e-12


def test_transform_only_batch_with_identity_pattern():
    """Without dilations: any patterns, odd determinants and m = 1 included."""
    Ms = SI.uneven_mix(24, seed=60, max_det=2048, lo=2, hi=33) + [[[1, 0], [0, 1]], [[3]], [[5, 2], [1, 3]]]
    B = pf.PatternBatch(Ms)
    x = SI.complex_normal_flat(B.total, 61)
    chat = _np(B.forward(torch.from_numpy(x).cuda()))
    for i, M in enumerate(Ms):
        o, m = int(B.offsets[i]), int(B.m[i])
        assert rel_l2(chat[o:o + m], oracle.pattern_fft(M, x[None, o:o + m])[0]) <= 1e-5, (i, M)


def test_graph_direct_and_autotuned_schedules_agree():
    """Graph replay, direct launches and an autotuned schedule compute the
    same values; a new output buffer rebuilds the graph."""
    Ms = _small_mix(70)
    Js = [SI.parity_dilation(M) for M in Ms]
    x = torch.from_numpy(SI.complex_normal_flat(sum(abs(L.det(M)) for M in Ms), 71)).cuda()
    Bg = pf.PatternBatch(Ms, Js)
    Bd = pf.PatternBatch(Ms, Js, flags=pf.PFFT_BATCH_NO_GRAPH)
    Bt = pf.PatternBatch(Ms, Js, flags=pf.PFFT_BATCH_AUTOTUNE)
    a = Bg.forward(x)
    b = Bd.forward(x)
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    a2 = Bg.forward(x)  # replay of the same graph
    for u, v in zip(a, a2):
        assert torch.equal(u, v)
    out = torch.empty_like(a[0])
    Bg.forward(x, c_hat=out)  # new pointer: the graph is rebuilt
    assert torch.equal(out, a[0])
    c = Bt.forward(x)
    for u, v in zip(a, c):
        assert rel_l2(_np(u), _np(v)) <= 1e-6
    rb, cb, order, radix = Bt.schedule()
    assert rb in (2048, 4096, 8192, 16384) and cb in (2048, 4096, 8192, 16384) and order in (0, 1)
    assert radix in (8, 16)


def test_batch_errors():
    Ms = [[[4, 1], [0, 6]], [[6, 0], [0, 2]]]
    Js = [SI.parity_dilation(M) for M in Ms]
    B = pf.PatternBatch(Ms, Js)
    x = torch.zeros(B.total, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    h = torch.zeros(B.total // 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_batch_forward(B._h, x.data_ptr(), y.data_ptr(), h.data_ptr(), None, 0)
    assert e.value.status == 1
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_batch_forward(B._h, x.data_ptr(), x.data_ptr(), None, None, 0)
    assert e.value.status == 1
    T = pf.PatternBatch(Ms)
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_batch_forward(T._h, x.data_ptr(), y.data_ptr(), h.data_ptr(), h.data_ptr(), 0)
    assert e.value.status == 1  # no dilations: no split
    with pytest.raises(pf.PfftError) as e:
        pf.PatternBatch([[[3, 0], [0, 4]]], [[[2, 0], [0, 1]]])
    assert e.value.status == 4  # J^{-1} M not integral
    with pytest.raises(pf.PfftError) as e:
        pf.PatternBatch([[[4, 0], [0, 2]], [[1031, 0], [0, 2]]])
    assert e.value.status == 5  # prime factor beyond the direct-stage limit
    with pytest.raises(ValueError):
        B.forward(x.cpu())


def _bands_of(B, i, sc, wv):
    """[p, n] bands of pattern i of a batch (band 0: the scaling part)."""
    p, n = int(B.p[i]), int(B.m[i]) // int(B.p[i])
    s0, w0 = int(B.sc_off[i]), int(B.wv_off[i])
    return np.concatenate([sc[None, s0:s0 + n], wv[w0:w0 + (p - 1) * n].reshape(p - 1, n)])


def _bands_ref_at(M, J, c, gslots):
    """Oracle bands at the slots gslots of the box of H(N^T) (prime |det J|):
    the oracle's transform on the p members of each fibre, then its p-band
    split of the coefficient vector holding only those values."""
    members = oracle.band_fibre_slots(M, J, gslots)
    slots = np.unique(members.reshape(-1))
    sparse = np.zeros((1, abs(L.det(M))), np.complex128)
    sparse[0, slots] = oracle.pattern_fft(M, c[None, :], out_slots=slots)[0]
    return oracle.wavelet_bands_at(M, J, sparse, gslots)[:, 0]


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_small_mix_mixed_determinants_full(dtype):
    """Patterns of even and odd determinant, each split by its mix dilation
    (determinant 2, or the smallest odd prime of det M: the built-in band
    system), every output of every pattern against the oracle."""
    Ms = SI.uneven_mix(40, seed=90, max_det=4096, lo=2, hi=40, even_det=False) + \
        [[[37, 5], [0, 74]], [[3, 1], [0, 9]], [[7, 2, 1], [0, 5, 3], [0, 0, 3]], [[31, 7], [0, 31]]]
    Js = [SI.mix_dilation(M) for M in Ms]
    B = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, dtype=dtype)
    assert sorted(set(int(p) for p in B.p)) != [2]
    c128 = dtype == torch.complex128
    tol = 1e-12 if c128 else 1e-5
    x = SI.complex_normal_flat(B.total, 91).astype(np.complex128 if c128 else np.complex64)
    chat, sc, wv = (_np(t) for t in B.forward(torch.from_numpy(x).cuda()))
    assert len(sc) == B.sc_total and len(wv) == B.wv_total
    for i, (M, J) in enumerate(zip(Ms, Js)):
        o, m = int(B.offsets[i]), int(B.m[i])
        ref = oracle.pattern_fft(M, x[None, o:o + m])
        assert rel_l2(chat[o:o + m], ref[0]) <= tol, (i, M)
        bands = _bands_of(B, i, sc, wv)
        if B.p[i] == 2:
            d1, d2 = oracle.wavelet_level(M, J, pf.PWT_DIRICHLET, c_hat=ref)
            want = np.stack([d1[0], d2[0]])
        else:
            want = oracle.wavelet_level_p(M, J, c_hat=ref)[:, 0]
        assert rel_l2(bands.reshape(1, -1), want.reshape(1, -1)) <= tol, (i, M, int(B.p[i]))


def test_odd_determinant_needs_the_dirichlet_bands():
    with pytest.raises(pf.PfftError) as e:
        pf.PatternBatch([[[9, 0], [0, 3]]], [[[3, 0], [0, 1]]], pf.PWT_DLVP, 0.125)
    assert e.value.status == 5


def test_uneven_mix_full_size_sampled():
    """The uneven serving-style mix in the benchmark's configuration
    (4096 patterns drawn as the rules state, odd determinants included;
    each split by its mix dilation; autotuned schedule, graph replay,
    Dirichlet symbol)."""
    w = SI.WORKLOADS["uneven_mix"]
    Ms = SI.uneven_mix(w["n_patterns"], seed=w["seed"], even_det=w["even_det"])
    Js = [SI.mix_dilation(M) for M in Ms]
    B = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, flags=pf.PFFT_BATCH_AUTOTUNE)
    assert (B.p % 2 == 1).sum() > 0
    x = SI.complex_normal_flat(B.total, w["seed"])
    chat, sc, wv = (_np(t) for t in B.forward(torch.from_numpy(x).cuda()))
    off, ms = B.offsets, B.m
    # Parseval and the norm identity of the unitary split, every pattern
    e_x = np.add.reduceat(np.abs(x.astype(np.complex128)) ** 2, off)
    e_c = np.add.reduceat(np.abs(chat.astype(np.complex128)) ** 2, off)
    e_s = np.add.reduceat(np.abs(sc.astype(np.complex128)) ** 2, B.sc_off)
    e_w = np.zeros(len(Ms))
    a_w = np.abs(wv.astype(np.complex128)) ** 2
    for i in range(len(Ms)):
        n = int(ms[i]) // int(B.p[i])
        e_w[i] = a_w[int(B.wv_off[i]):int(B.wv_off[i]) + (int(B.p[i]) - 1) * n].sum()
    assert np.allclose(e_c, e_x, rtol=1e-5)
    assert np.allclose(e_s + e_w, e_c, rtol=1e-5)
    rng = np.random.default_rng(SI.SAMPLE_SEED)
    worst = 0.0
    for i, M in enumerate(Ms):
        o, m = int(off[i]), int(ms[i])
        slots = np.sort(rng.choice(m, 8, replace=False))
        ref = oracle.pattern_fft(M, x[None, o:o + m], out_slots=slots)[0]
        worst = max(worst, rel_l2(chat[o + slots], ref))
        p = int(B.p[i])
        if i % 8 == 0 or (p > 2 and i % 2 == 0):
            g = np.sort(rng.choice(m // p, 2, replace=False))
            bands = _bands_of(B, i, sc, wv)[:, g]
            if p == 2:
                d1, d2 = _split_ref_at(M, Js[i], x[o:o + m], g, pf.PWT_DIRICHLET)
                want = np.stack([d1, d2])
            else:
                want = _bands_ref_at(M, Js[i], x[o:o + m], g)
            worst = max(worst, rel_l2(bands.reshape(1, -1), want.reshape(1, -1)))
    assert worst <= 1e-5, worst
