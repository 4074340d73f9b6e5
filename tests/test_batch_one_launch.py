"""GPU tests of the single-launch batch (PFFT_BATCH_ONE_LAUNCH): every row
tile, column tile and split unit of a pattern batch in one kernel launch whose
CTAs take work units from a device queue, a column tile waiting (bounded) for
its pattern's row tiles and a split unit for its pattern's coefficients.

The launch runs the same tile and split arithmetic as the grouped launches
with 512 threads per CTA for every tile (a grouped launch uses its bucket's
largest thread count), so outputs agree with theirs up to the rounding of the
stage twiddle powers, which each thread forms for its own butterflies
(measured rel-L2 1e-8 in complex64; the grouped path is checked against the
FP64 oracle in test_batch_parity.py); a small batch is also compared with the
oracle directly.  The bounded wait is made to run out with
a spin limit of 0 (a column tile that finds its pattern's rows unfinished
gives up at once), which must be reported as PFFT_ERR_TIMEOUT and leave the
batch usable."""
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
         [[64, 0], [0, 64]], [[15, 5], [0, 21]]]


def _mix(seed, even):
    return SI.uneven_mix(40, seed=seed, max_det=4096, lo=2, hi=40, even_det=even) + EXTRA


def _run(B, x):
    out = B.forward(x)
    torch.cuda.synchronize()
    return out


def _close(r, g):
    tol = 1e-6 if r.dtype == torch.complex64 else 1e-13
    return (torch.linalg.vector_norm(r - g) / torch.linalg.vector_norm(r)).item() <= tol


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("flags", [0, pf.PFFT_BATCH_NO_GRAPH])
def test_one_launch_equals_grouped_launches(dtype, flags):
    Ms = _mix(90, even=False)
    Js = [SI.mix_dilation(M) if abs(L.det(M)) > 1 else None for M in Ms]
    Ms = [M for M, J in zip(Ms, Js) if J is not None]
    Js = [J for J in Js if J is not None]
    A = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, 0.125, dtype=dtype, flags=flags)
    Q = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, 0.125, dtype=dtype, flags=flags | pf.PFFT_BATCH_ONE_LAUNCH)
    x = torch.from_numpy(SI.complex_normal_flat(A.total, 91)).to(dtype).cuda()
    ref = _run(A, x)
    for _ in range(2):  # twice: the queue's counters start from zero on every call
        got = _run(Q, x)
        for r, g in zip(ref, got):
            assert _close(r, g)
        Q.check_device_status()
    # transform only (no split units in the queue)
    assert _close(A.forward(x, split=False), Q.forward(x, split=False))


def test_one_launch_against_the_oracle():
    Ms = [[[64, 16], [-16, 64]], [[37, 5], [0, 74]], [[6, 1, 2], [0, 7, 3], [0, 0, 14]], [[128, 0], [0, 96]]]
    Js = [SI.mix_dilation(M) for M in Ms]
    B = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, 0.125, flags=pf.PFFT_BATCH_ONE_LAUNCH)
    x = SI.complex_normal_flat(B.total, 92)
    chat = B.forward(torch.from_numpy(x).cuda(), split=False).cpu().numpy()
    for i, M in enumerate(Ms):
        o, m = int(B.offsets[i]), int(B.m[i])
        ref = oracle.pattern_fft(M, x[None, o:o + m].astype(np.complex128))[0]
        assert rel_l2(chat[o:o + m], ref) <= 1e-5


def test_one_launch_uneven_mix_equals_grouped_launches():
    """The 4096-pattern uneven mix (odd determinants split by their smallest
    prime) in one launch: every output equal to the grouped launches' up to
    rounding."""
    w = SI.WORKLOADS["uneven_mix"]
    Ms = SI.uneven_mix(w["n_patterns"], seed=w["seed"], even_det=w["even_det"])
    Js = [SI.mix_dilation(M) for M in Ms]
    A = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET)
    Q = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, flags=pf.PFFT_BATCH_ONE_LAUNCH)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w["seed"])
    x = torch.randn(A.total, dtype=torch.complex64, device="cuda", generator=gen)
    ref = _run(A, x)
    got = _run(Q, x)
    Q.check_device_status()
    for r, g in zip(ref, got):
        assert _close(r, g)
    A.close()
    Q.close()


def test_one_launch_bounded_wait_runs_out_then_recovers():
    """Spin limit 0: a column tile dispensed while its pattern's last row tile
    still runs gives up at once, records PFFT_ERR_TIMEOUT and stops the rest
    of the launch; with the default limit the same batch is correct again."""
    Ms = [[[512, 0], [0, 256]]]  # one pattern: 16 row tiles, then 16 column tiles, all resident at once
    Q = pf.PatternBatch(Ms, None, flags=pf.PFFT_BATCH_ONE_LAUNCH | pf.PFFT_BATCH_NO_GRAPH)
    A = pf.PatternBatch(Ms, None)
    x = torch.from_numpy(SI.complex_normal_flat(Q.total, 93)).cuda()
    ref = A.forward(x)
    Q.set_wait_limit(0)
    timed_out = 0
    for _ in range(8):
        Q.forward(x)
        try:
            Q.check_device_status()
        except pf.PfftError as e:
            assert e.status == 8  # PFFT_ERR_TIMEOUT
            timed_out += 1
    assert timed_out > 0
    Q.set_wait_limit(-1)
    got = Q.forward(x)
    Q.check_device_status()
    assert _close(ref, got)


def test_wait_limit_needs_a_single_launch_batch():
    B = pf.PatternBatch([[[16, 0], [0, 16]]], None)
    with pytest.raises(pf.PfftError) as e:
        B.set_wait_limit(0)
    assert e.value.status == 5  # PFFT_ERR_UNSUPPORTED
    B.check_device_status()  # no status word: PFFT_OK
