"""The bounded mbarrier wait of the bulk-copy row pass and the device status
word (through the C ABI).

The row pass waits for its rows' asynchronous copies with an iteration limit.
A limit of zero makes that wait give up at once: the kernel must record
PFFT_ERR_TIMEOUT in the plan's status word, wait (with the default limit) for
its own copies and return, leaving the GPU usable.  The status is read and
cleared by pfft_last_device_status, and the next call with the default limit
must be correct again.  Nothing here faults or hangs: the copies are valid
and land; only the first wait is cut short."""
import numpy as np
import pytest
import torch

import oracle
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import TOL, rel_l2

pytestmark = pytest.mark.gpu

PFFT_ERR_TIMEOUT = 8


@pytest.mark.parametrize("dtype,M", [(torch.complex64, [[16, 0], [0, 8192]]),      # rows of 2^13
                                     (torch.complex64, [[4, 0], [0, 16384]]),      # rows of 2^14
                                     (torch.complex128, [[16, 0], [0, 8192]])])    # generic bulk-copy rows
def test_bounded_wait_runs_out_then_recovers(dtype, M):
    c128 = dtype == torch.complex128
    plan = pf.PatternFFT(M, 2, dtype=dtype)
    np_dt = np.complex128 if c128 else np.complex64
    c = SI.complex_normal(2, plan.m, 41, dtype=np_dt)
    x = torch.from_numpy(c).cuda()
    slots = SI.sample_slots(plan.m, 256)
    ref_f = oracle.pattern_fft(M, c.astype(np.complex128), out_slots=slots)
    tol = TOL["c128" if c128 else "c64"]
    for direction in ("forward", "inverse"):
        pf.pfft_set_wait_limit(plan._h, 0)
        getattr(plan, direction)(x)
        with pytest.raises(pf.PfftError) as e:
            plan.check_device_status()
        assert e.value.status == PFFT_ERR_TIMEOUT, direction
        plan.check_device_status()  # read-and-clear: the word is zero again
        pf.pfft_set_wait_limit(plan._h, -1)
    y = plan.forward(x)
    plan.check_device_status()
    assert rel_l2(y.cpu().numpy()[:, slots], ref_f) <= tol
    z = plan.inverse(y)
    plan.check_device_status()
    assert rel_l2(z.cpu().numpy(), c) <= 10 * tol


def test_wait_limit_needs_a_bulk_copy_row_pass():
    plan = pf.PatternFFT(SI.M_SMALL_2D, 1)  # radix-17 cycles: no bulk-copy staging
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_set_wait_limit(plan._h, 0)
    assert e.value.status == 5  # PFFT_ERR_UNSUPPORTED
