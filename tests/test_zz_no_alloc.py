"""The allocation-free decomposition entry point (pwt_decompose_noalloc).

It exists for callers that cannot call cudaMalloc (device-memory budgets or
pools that forbid allocations, code that must not fail on an allocation in
the middle of its work).  It keeps its inter-level scratch in a fixed device
array instead of a plan workspace.  This file is collected last on purpose.
The tests call it through the C ABI twice in a row (the second call runs on
the scratch the first one left behind) and compare each result with the
plan-based pwt_decompose and with the FP64 oracle's cascade, within the
complex64 tolerance of the suite; they also run its 64-bit index path and
the exact edge of its scratch bound."""
import numpy as np
import pytest
import torch

import oracle
import paper_1107_5415_gb300 as pf
from paper_1107_5415_gb300 import _capi
import seeded_inputs as SI
from parity_util import TOL, rel_l2

pytestmark = pytest.mark.gpu

# (|det M| / 2) * batch may reach this many complex64 values when levels > 1
SCRATCH_HALF = 1 << 20


def _noalloc(M, Js, sym, batch, c, like_s, like_w):
    s = torch.empty_like(like_s)
    w = [torch.empty_like(x) for x in like_w]
    stream = torch.cuda.current_stream().cuda_stream
    _capi.pwt_decompose_noalloc(M, Js, sym, 0.125, batch, c.data_ptr(), s.data_ptr(),
                                [x.data_ptr() for x in w], stream)
    torch.cuda.synchronize()
    return s, w


def _check_twice(M, Js, sym, batch, seeds, with_oracle):
    plan = pf.WaveletSplit(M, Js, sym, 0.125, batch)
    for call, seed in enumerate(seeds):
        c_np = SI.complex_normal(batch, plan.sizes[0], seed)
        c = torch.from_numpy(c_np).cuda()
        s_ref, w_ref = plan.decompose(c)
        s, w = _noalloc(M, Js, sym, batch, c, s_ref, w_ref)
        assert rel_l2(s.cpu().numpy(), s_ref.cpu().numpy()) <= TOL["c64"], call
        for a, b in zip(w, w_ref):
            assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= TOL["c64"], call
        if with_oracle:
            so, wo = oracle.wavelet_cascade(M, Js, c_np.astype(np.complex128), sym, 0.125)
            assert rel_l2(s.cpu().numpy(), so) <= TOL["c64"], call
            for a, b in zip(w, wo):
                assert rel_l2(a.cpu().numpy(), b) <= TOL["c64"], call


@pytest.mark.parametrize("sym", [pf.PWT_DIRICHLET, pf.PWT_DLVP])
def test_noalloc_matches_plan_and_oracle_twice(sym):
    _check_twice([[64, 64], [-64, 64]], SI.wavelet_dilations(6), sym, 3, (11, 12), with_oracle=True)


@pytest.mark.parametrize("sym", [pf.PWT_DIRICHLET, pf.PWT_DLVP])
def test_noalloc_wide_index_path(sym):
    """Entries near 2^23 make the symbol numerators exceed the int32 range, so
    the first level takes the kernel's 64-bit index arithmetic."""
    M = [[1 << 23, (1 << 23) - 64], [1, 1]]
    Js = [[[2, 0], [0, 1]]] * 5
    _check_twice(M, Js, sym, 3, (21, 22), with_oracle=True)


def test_noalloc_at_the_scratch_bound():
    """(|det M| / 2) * batch equal to the bound runs; one more signal is
    rejected with PFFT_ERR_OVERFLOW and nothing is queued."""
    M, Js = [[64, 64], [-64, 64]], SI.wavelet_dilations(4)
    batch = SCRATCH_HALF // 4096  # |det M| / 2 = 4096
    _check_twice(M, Js, pf.PWT_DIRICHLET, batch, (31, 32), with_oracle=False)
    over = batch + 1
    c = torch.zeros(over, 8192, dtype=torch.complex64, device="cuda")
    s = torch.zeros(over, 512, dtype=torch.complex64, device="cuda")
    w = [torch.zeros(over, 8192 >> (l + 1), dtype=torch.complex64, device="cuda") for l in range(4)]
    with pytest.raises(pf.PfftError) as e:
        _capi.pwt_decompose_noalloc(M, Js, pf.PWT_DIRICHLET, 0.125, over, c.data_ptr(), s.data_ptr(),
                                    [x.data_ptr() for x in w], 0)
    assert e.value.status == 3  # PFFT_ERR_OVERFLOW


def test_noalloc_rejects_sizes_beyond_its_scratch():
    M, Js = SI.M_WAVELET_2D, SI.wavelet_dilations(2)   # (2^21 / 2) * 4 > 2^20
    c = torch.zeros(4, 1 << 21, dtype=torch.complex64, device="cuda")
    s = torch.zeros(4, 1 << 19, dtype=torch.complex64, device="cuda")
    w = [torch.zeros(4, 1 << 20, dtype=torch.complex64, device="cuda"), s]
    with pytest.raises(pf.PfftError) as e:
        _capi.pwt_decompose_noalloc(M, Js, pf.PWT_DIRICHLET, 0.125, 4, c.data_ptr(), s.data_ptr(),
                                    [x.data_ptr() for x in w], 0)
    assert e.value.status == 3  # PFFT_ERR_OVERFLOW
