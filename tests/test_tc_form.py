"""GPU parity of the split-precision tensor-core form (PFFT_FLAG_TC_SPLIT):
radix-16 / 32 stages as fp16 hi + lo DFT-matrix products with fp32
accumulation, against the FP64 oracle at the complex64 bar (rel-L2 <= 1e-5).
The measured errors are printed (run with -s to see them)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import rel_l2

pytestmark = pytest.mark.gpu

SMALL = [
    [[16, 0], [0, 16]],                    # 2-D DFT 16 x 16: radix-16 stages on the tensor cores
    [[32, 0], [0, 64]],                    # (32, 64): radix 32 in both passes
    SI.M_SMALL_2D,                         # (16, 272): radix 16 with a direct radix 17
    [[64, 0], [0, 96]],                    # (32, 192): radix 32, 2 and 3
    [[4, 1], [0, 8192]],                   # one cycle of 32768, split 2 x 16384
    [[4, 1, 0], [0, 4, 1], [0, 0, 4]],     # one cycle of 64 in d = 3
    [[6, 2], [-2, 6]],                     # (2, 20): no radix-16 / 32 stage
]


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("M", SMALL, ids=[str(i) for i in range(len(SMALL))])
def test_tc_small_patterns_full(M):
    m = abs(L.det(M))
    plan = pf.PatternFFT(M, 2, tc_split=True)
    c = SI.complex_normal(2, m, seed=m % 89)
    ref = oracle.pattern_fft(M, c)
    got = plan.forward(_gpu(c)).cpu().numpy()
    err = rel_l2(got, ref)
    back = plan.inverse(_gpu(ref.astype(np.complex64))).cpu().numpy()
    err_b = rel_l2(back, oracle.pattern_fft(M, ref, inverse=True))
    print(f"tc {M}: forward rel-L2 {err:.2e}, inverse {err_b:.2e}")
    assert err <= 1e-5 and err_b <= 1e-5


@pytest.mark.parametrize("name", ["batched_2d", "autograd_3d"])
def test_tc_workloads_sampled(name):
    """The batched 2-D and the 3-D workloads in the tensor-core form: 4096
    sampled frequencies by the direct FP64 sum, and the round trip."""
    w = SI.WORKLOADS[name]
    M, batch = w["M"], w["batch"]
    m = abs(L.det(M))
    plan = pf.PatternFFT(M, batch, tc_split=True)
    c = SI.complex_normal(batch, m, w["seed"])
    y = plan.forward(_gpu(c))
    yh = y.cpu().numpy()
    slots = SI.sample_slots(m, 4096)
    err = rel_l2(yh[:1, slots], oracle.pattern_fft(M, c[:1], out_slots=slots))
    back = plan.inverse(y).cpu().numpy()
    err_rt = rel_l2(back, c)
    plain = pf.PatternFFT(M, batch).forward(_gpu(c)).cpu().numpy()
    print(f"tc {name}: sampled forward rel-L2 {err:.2e}, round trip {err_rt:.2e}, "
          f"vs plain fp32 {rel_l2(yh, plain):.2e}")
    assert err <= 1e-5 and err_rt <= 1e-5


def test_tc_rejects_complex128():
    with pytest.raises(pf.PfftError) as e:
        pf.PatternFFT([[16, 0], [0, 16]], 1, torch.complex128, tc_split=True)
    assert e.value.status == 5


@pytest.mark.parametrize("scale", [1e-3, 1e3, 1e-30, 1e30])
@pytest.mark.parametrize("M", [[[32, 0], [0, 64]], [[4, 1], [0, 8192]]], ids=["32x64", "split32768"])
def test_tc_accuracy_is_scale_free(M, scale):
    """Inputs scaled far from unit size (small enough for fp16 subnormals, or
    beyond the fp16 range) keep the complex64 bar against the oracle: each
    butterfly is rescaled by a power of two around the split."""
    m = abs(L.det(M))
    plan = pf.PatternFFT(M, 1, tc_split=True)
    c = SI.complex_normal(1, m, seed=5).astype(np.complex128) * scale
    slots = SI.sample_slots(m, min(m, 2048))
    ref = oracle.pattern_fft(M, c, out_slots=slots)
    got = plan.forward(_gpu(c.astype(np.complex64))).cpu().numpy()
    err = rel_l2(got[:, slots], ref)
    print(f"tc {M} x {scale:g}: rel-L2 {err:.2e}")
    assert err <= 1e-5
