"""The allocation-free decomposition entry point (pwt_decompose_noalloc).

It exists for callers that cannot call cudaMalloc (device-memory budgets or
pools that forbid allocations, code that must not fail on an allocation in
the middle of its work).  It keeps its inter-level scratch in a fixed device
array instead of a plan workspace.  This file is collected last on purpose.
The test calls it through the C ABI twice in a row (the second call runs on
the scratch the first one left behind) and compares each result with the
plan-based pwt_decompose within the complex64 tolerance of the suite."""
import numpy as np
import pytest
import torch

import paper_1107_5415_gb300 as pf
from paper_1107_5415_gb300 import _capi
import seeded_inputs as SI
from parity_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sym", [pf.PWT_DIRICHLET, pf.PWT_DLVP])
def test_noalloc_matches_plan_twice(sym):
    M, Js, batch = [[64, 64], [-64, 64]], SI.wavelet_dilations(6), 3
    plan = pf.WaveletSplit(M, Js, sym, 0.125, batch)
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((11, 12)):
        c = torch.from_numpy(SI.complex_normal(batch, plan.sizes[0], seed)).cuda()
        s_ref, w_ref = plan.decompose(c)
        s = torch.empty_like(s_ref)
        w = [torch.empty_like(x) for x in w_ref]
        _capi.pwt_decompose_noalloc(M, Js, sym, 0.125, batch, c.data_ptr(), s.data_ptr(),
                                    [x.data_ptr() for x in w], stream)
        torch.cuda.synchronize()
        assert rel_l2(s.cpu().numpy(), s_ref.cpu().numpy()) <= 1e-5, call
        for a, b in zip(w, w_ref):
            assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 1e-5, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    M, Js = SI.M_WAVELET_2D, SI.wavelet_dilations(2)   # (2^21 / 2) * 4 > 2^20
    c = torch.zeros(4, 1 << 21, dtype=torch.complex64, device="cuda")
    s = torch.zeros(4, 1 << 19, dtype=torch.complex64, device="cuda")
    w = [torch.zeros(4, 1 << 20, dtype=torch.complex64, device="cuda"), s]
    with pytest.raises(pf.PfftError) as e:
        _capi.pwt_decompose_noalloc(M, Js, pf.PWT_DIRICHLET, 0.125, 4, c.data_ptr(), s.data_ptr(),
                                    [x.data_ptr() for x in w], 0)
    assert e.value.status == 3  # PFFT_ERR_OVERFLOW
