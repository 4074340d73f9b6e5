"""Step 5 of the fast wavelet decomposition (Section 5.3): after the split
cascade, the inverse pattern FFT on G(N_l^T) of every part gives its
time-domain coefficients.  The chain runs on the 12-level workload
(M_0 = 2^10 [[1,1],[-1,1]], batch 16, coefficients (1 + |h|^2)^{-1} times
complex normal values) through the C ABI: pwt_decompose, then pfft_inverse
with a plan for each N_l, in the plain fp32 form and in the split-precision
tensor-core form.  Reference: the oracle's cascade followed by the oracle's
inverse direct sum (all slots for the small levels, 256 sampled slots of two
signals for the large ones)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import TOL, rel_l2
from test_wavelet_parity import _centred_weight

pytestmark = pytest.mark.gpu

SYM = {"dirichlet": (pf.PWT_DIRICHLET, oracle.DIRICHLET), "dlvp": (pf.PWT_DLVP, oracle.DLVP)}
FULL_MAX = 4096  # levels up to this size are checked on every slot


@pytest.mark.parametrize("form,sym", [("fp32", "dirichlet"), ("fp32", "dlvp"), ("tc_split", "dirichlet")])
def test_split_cascade_then_step5_inverse_ffts(form, sym):
    w = SI.WORKLOADS["wavelet_2d"]
    M, batch, levels = w["M"], w["batch"], w["levels"]
    Js = SI.wavelet_dilations(levels)
    gsym, osym = SYM[sym]
    m = abs(L.det(M))
    c = (SI.complex_normal(batch, m, w["seed"], dtype=np.complex128) * _centred_weight(M)[None, :])
    split = pf.WaveletSplit(M, Js, gsym, 0.125, batch)
    s, wav = split.decompose(torch.from_numpy(c.astype(np.complex64)).cuda())
    s_ref, w_ref = oracle.wavelet_cascade(M, Js, c, osym, 0.125)
    Ns, cur = [], M
    for J in Js:
        cur = oracle.exact_N(cur, J)
        Ns.append(cur)
    parts = list(zip(Ns, wav, w_ref)) + [(Ns[-1], s, s_ref)]
    worst = 0.0
    for N, got_hat, ref_hat in parts:
        n = abs(L.det(N))
        plan = pf.PatternFFT(N, batch, tc_split=(form == "tc_split"))
        got = plan.inverse(got_hat).cpu().numpy()
        plan.close()
        if n <= FULL_MAX:
            err = rel_l2(got, oracle.pattern_fft(N, ref_hat, inverse=True))
        else:
            rows = [0, batch - 1]
            slots = SI.sample_slots(n, 256)
            ref = oracle.pattern_fft(N, ref_hat[rows], inverse=True, out_slots=slots)
            err = rel_l2(got[rows][:, slots], ref)
        worst = max(worst, err)
        assert err <= TOL["c64"], (N, err)
    print(f"step 5 ({form}, {sym}): worst rel-L2 over the 13 parts {worst:.2e}")
