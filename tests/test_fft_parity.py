"""GPU parity of the pattern FFT against the FP64 oracle (through the C ABI).

Bar: bit-exact index maps; relative L2 error <= 1e-5 (complex64) or 1e-12
(complex128).  Small patterns are compared on every output; the batched
2^24-point workload in the benchmark's launch configuration is compared on
4096 seeded random frequencies evaluated by the oracle's direct sum."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import TOL, rel_l2

pytestmark = pytest.mark.gpu

SMALL = [
    SI.M_SMALL_2D,                          # cycles (16, 272): radix 17
    [[4, -3], [4, 5]],                      # Example 1: one cycle of 32
    [[6, 2], [-2, 6]],                      # (2, 20): radix 5
    [[8, 2], [2, -4]],                      # negative determinant, (2, 18)
    [[12]],                                 # d = 1
    [[7, 0], [0, 5]],                       # cyclic 35 (gcd 1)
    [[16, 0], [0, 16]],                     # plain 2-D DFT
    [[4, 1, 0], [0, 4, 1], [0, 0, 4]],      # one cycle of 64 in d = 3
    [[6, 2, 0], [0, 6, 3], [0, 0, 6]],      # three cycles
    [[3, 1, 2], [0, 2, 1], [1, 0, 4]],      # non-triangular 3-D
    [[1, 0], [0, 1]],                       # m = 1
    [[2, 1], [1, 1]],                       # unimodular, m = 1
    [[9, 0, 3], [0, 12, 2], [0, 0, 10]],    # fast axis is not a maximal generator
    [[64, 0], [0, 96]],                     # (32, 192): radix 3 with powers of two
    [[4, 1], [0, 8192]],                    # one cycle of 32768: split four-step (2 x 16384)
    [[17, 0], [0, 2048]],                   # one cycle of 34816 = 17 * 2^11: split, mixed radix
    [[2, 1, 0], [0, 2, 1], [0, 0, 8192]],   # one cycle of 32768 in d = 3
    [[37, 0], [0, 41]],                     # cyclic 1517: two direct prime stages, the second twiddled
    [[74, 0], [0, 148]],                    # (74, 148): direct radix 37 in both passes
    [[11, 3, 5], [0, 13, 2], [0, 0, 4]],    # 572 = 4 * 11 * 13 in d = 3
    [[509, 0], [0, 67]],                    # cyclic 34103 = 509 * 67: split, direct stages in both passes
    [[23, 7], [0, 46]],                     # (23, 46): odd column tile count
    [[32, 0, 16], [0, 16, 6], [0, 0, 4]],   # (2, 32, 32): register-resident column pass over two axes
    [[32, 0, 16], [0, 8, 4], [0, 0, 16]],   # (4, 32, 32): the same, tail radix 4
    [[64, 0, 48], [0, 16, 8], [0, 0, 16]],  # (8, 32, 64): the same, tail radix 8
]


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _plan_or_skip(M, batch, dtype):
    try:
        return pf.PatternFFT(M, batch, dtype)
    except pf.PfftError as e:
        if e.status == 5:  # PFFT_ERR_UNSUPPORTED: documented limits
            pytest.skip(f"outside the kernels' limits: {e}")
        raise


@pytest.mark.parametrize("M", SMALL, ids=[str(i) for i in range(len(SMALL))])
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_small_patterns_full(M, dtype):
    m = abs(L.det(M))
    batch = 3
    plan = _plan_or_skip(M, batch, dtype)
    npdt = np.complex64 if dtype == torch.complex64 else np.complex128
    c = SI.complex_normal(batch, m, seed=m % 97, dtype=npdt)
    ref = oracle.pattern_fft(M, c)
    got = plan.forward(_gpu(c)).cpu().numpy()
    tol = TOL["c64" if dtype == torch.complex64 else "c128"]
    assert rel_l2(got, ref) <= tol
    back_ref = oracle.pattern_fft(M, ref, inverse=True)
    back = plan.inverse(_gpu(ref.astype(npdt))).cpu().numpy()
    assert rel_l2(back, back_ref) <= tol


def test_small_2d_workload_seed0():
    w = SI.WORKLOADS["small_2d"]
    M, batch = w["M"], w["batch"]
    m = abs(L.det(M))
    c = SI.complex_normal(batch, m, w["seed"])
    plan = pf.PatternFFT(M, batch)
    got = plan.forward(_gpu(c))
    ref = oracle.pattern_fft(M, c)
    assert rel_l2(got.cpu().numpy(), ref) <= 1e-5
    back = plan.inverse(got).cpu().numpy()
    assert rel_l2(back, oracle.pattern_fft(M, ref, inverse=True)) <= 1e-5
    assert rel_l2(back, c) <= 1e-5


@pytest.mark.parametrize("M", [SI.M_SMALL_2D, [[6, 2], [-2, 6]], [[8, 2], [2, -4]], [[4, 1, 0], [0, 4, 1], [0, 0, 4]],
                               [[6, 2, 0], [0, 6, 3], [0, 0, 6]], [[3, 1, 2], [0, 2, 1], [1, 0, 4]],
                               [[9, 0, 3], [0, 12, 2], [0, 0, 10]], SI.M_BATCHED_2D, SI.M_AUTOGRAD_3D])
def test_index_maps_bit_exact(M):
    """The maps the kernels evaluate on the device are bijections onto the
    boxes of the layout contract, agree with the host maps, and turn the
    phase k^T M^{-1} y into sum_j lambda_j mu_j / n_j exactly (Theorem 1)."""
    plan = pf.PatternFFT(M, 1)
    m, d = plan.m, plan.d
    Hbox = np.array(list(L.box_points(L.hnf(M)))) if m <= 1 << 16 else None
    yin = plan.index_map(pf.PFFT_MAP_INPUT_BOX)
    kout = plan.index_map(pf.PFFT_MAP_OUTPUT_BOX)
    if Hbox is not None:
        assert (yin == Hbox).all()
        assert (kout == np.array(list(L.box_points(L.hnf(L.transpose(M)))))).all()
    if plan.dM == 0:
        return
    lam = plan.index_map(pf.PFFT_MAP_INPUT_SNF)
    mu = plan.index_map(pf.PFFT_MAP_OUTPUT_SNF)
    n = [int(e) for e in plan.eps if e > 1]
    flat = lambda v: np.ravel_multi_index(tuple(v.T), n)
    dev_in = plan.device_index_map(pf.PFFT_MAP_INPUT_BOX).cpu().numpy()
    dev_out = plan.device_index_map(pf.PFFT_MAP_OUTPUT_BOX).cpu().numpy()
    slots = np.arange(m)
    assert (np.sort(dev_in) == slots).all() and (np.sort(dev_out) == slots).all()
    assert (dev_in[flat(lam)] == slots).all()
    assert (dev_out[flat(mu)] == slots).all()
    # exact phase identity on random pairs, against the adjugate numerator
    A = np.array(L.adjugate(M), dtype=object)
    sd = 1 if L.det(M) > 0 else -1
    rng = np.random.default_rng(0)
    for _ in range(300):
        a, b = int(rng.integers(m)), int(rng.integers(m))
        k, y = [int(x) for x in kout[a]], [int(x) for x in yin[b]]
        num = sd * sum(k[i] * int(A[i][j]) * y[j] for i in range(d) for j in range(d)) % m
        s = sum(int(lam[b][j]) * int(mu[a][j]) * (m // n[j]) for j in range(len(n))) % m
        assert num == s


def test_batched_2d_sampled_frequencies():
    """Benchmark workload (M = [[4096,1024],[0,4096]], batch 8) in the launch
    configuration the benchmark times; 4096 sampled frequencies of signal 0
    and 512 of signal 7 by the direct FP64 sum; inverse on 1024 sampled slots."""
    w = SI.WORKLOADS["batched_2d"]
    M, batch = w["M"], w["batch"]
    m = abs(L.det(M))
    plan = pf.PatternFFT(M, batch)
    c = SI.complex_normal(batch, m, w["seed"])
    x = _gpu(c)
    y = plan.forward(x)
    yh = y.cpu().numpy()
    for item, ns in ((0, 4096), (batch - 1, 512)):
        slots = SI.sample_slots(m, ns)
        ref = oracle.pattern_fft(M, c[item:item + 1], out_slots=slots)
        assert rel_l2(yh[item:item + 1, slots], ref) <= 1e-5
    # Parseval per signal (holds at every size)
    assert np.allclose(np.linalg.norm(yh, axis=1), np.linalg.norm(c, axis=1), rtol=1e-5)
    back = plan.inverse(y)
    plan.check_device_status()  # no bounded wait timed out
    slots = SI.sample_slots(m, 1024, seed=7)
    ref = oracle.pattern_fft(M, yh[2:3].astype(np.complex128), inverse=True, out_slots=slots)
    assert rel_l2(back.cpu().numpy()[2:3, slots], ref) <= 1e-5
    assert rel_l2(back.cpu().numpy(), c) <= 1e-5


@pytest.mark.parametrize("M,batch", [(SI.M_BATCHED_2D, 2), ([[64, 16], [-16, 64]], 4), ([[5, -2], [3, 7]], 3),
                                     ([[32, 5, 7], [0, 64, 9], [0, 0, 8192]], 1), (SI.M_AUTOGRAD_3D, 1)])
def test_inverse_equals_conjugated_forward_of_the_transpose(M, batch):
    """F(M^T) = F(M)^T in box order (eq. (Fouriermatrix) read for M^T), so the
    inverse of M equals the conjugated forward transform of M^T: two plans whose
    passes walk different boxes and cycles must agree to rounding."""
    A = pf.PatternFFT(M, batch)
    B = pf.PatternFFT(L.transpose(M), batch)
    assert A.m == B.m
    y = _gpu(SI.complex_normal(batch, A.m, 21))
    back = A.inverse(y)
    alt = torch.conj(B.forward(torch.conj(y).resolve_conj())).resolve_conj()
    A.check_device_status()
    B.check_device_status()
    assert (torch.linalg.vector_norm(back - alt) / torch.linalg.vector_norm(back)).item() <= 1e-5


@pytest.mark.parametrize("M", [[[32, 64, 0], [0, 64, 64], [0, 0, 64]], [[64, 0, 0], [0, 32, 0], [0, 0, 128]]])
def test_two_axis_column_pass_with_swapped_axes_sampled(M):
    """Cycles (32, 64, n): the register-resident column pass over the pencil of
    32 x 64 runs with the longer axis first (its stages start with radix 2 x 32);
    sampled frequencies, the round trip and the device index maps."""
    plan = pf.PatternFFT(M, 2)
    m = plan.m
    c = SI.complex_normal(2, m, 17)
    y = plan.forward(_gpu(c)).cpu().numpy()
    slots = SI.sample_slots(m, 512, seed=5)
    assert rel_l2(y[1:2, slots], oracle.pattern_fft(M, c[1:2], out_slots=slots)) <= 1e-5
    assert rel_l2(plan.inverse(_gpu(y)).cpu().numpy(), c) <= 1e-5
    lam = plan.index_map(pf.PFFT_MAP_INPUT_SNF)
    n = [int(e) for e in plan.eps if e > 1]
    dev_in = plan.device_index_map(pf.PFFT_MAP_INPUT_BOX).cpu().numpy()
    assert (dev_in[np.ravel_multi_index(tuple(lam.T), n)] == np.arange(m)).all()


def test_autograd_3d_sampled_frequencies():
    w = SI.WORKLOADS["autograd_3d"]
    M, batch = w["M"], w["batch"]
    m = abs(L.det(M))
    plan = pf.PatternFFT(M, batch)
    c = SI.complex_normal(batch, m, w["seed"])
    y = plan.forward(_gpu(c)).cpu().numpy()
    slots = SI.sample_slots(m, 2048)
    ref = oracle.pattern_fft(M, c[1:2], out_slots=slots)
    assert rel_l2(y[1:2, slots], ref) <= 1e-5
    back = plan.inverse(_gpu(y)).cpu().numpy()
    assert rel_l2(back, c) <= 1e-5


def test_gpu_argument_errors():
    plan = pf.PatternFFT(SI.M_SMALL_2D, 1)
    x = torch.zeros(1, plan.m, dtype=torch.complex64, device="cuda")
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_forward(plan._h, x.data_ptr(), x.data_ptr(), 0)
    assert e.value.status == 1
    with pytest.raises(ValueError):
        plan.forward(x.to(torch.complex128))
    with pytest.raises(ValueError):
        plan.forward(x.cpu())


def test_streams_and_repeat_calls_are_deterministic():
    plan = pf.PatternFFT(SI.M_AUTOGRAD_3D, 1)
    c = _gpu(SI.complex_normal(1, plan.m, 5))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = plan.forward(c)
        b = plan.forward(c)
    s.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("i", [1, 2, 16, 1024, 0])
def test_table1_shapes_sampled(i):
    """The pattern family of Table 1 (Section 6.1): M = [[2048, i], [0, 2048]],
    m = 2^22, cycles (i, 2^22 / i); cycles longer than one row tile are split."""
    M = [[2048, i], [0, 2048]]
    m = 1 << 22
    plan = pf.PatternFFT(M, 2)
    c = SI.complex_normal(2, m, 20 + i)
    y = plan.forward(_gpu(c)).cpu().numpy()
    slots = SI.sample_slots(m, 512, seed=i)
    assert rel_l2(y[1:2, slots], oracle.pattern_fft(M, c[1:2], out_slots=slots)) <= 1e-5
    back = plan.inverse(_gpu(y)).cpu().numpy()
    assert rel_l2(back, c) <= 1e-5
    assert np.allclose(np.linalg.norm(y, axis=1), np.linalg.norm(c, axis=1), rtol=1e-5)


@pytest.mark.parametrize("M", SMALL, ids=[str(i) for i in range(len(SMALL))])
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_transposed_route_full(M, dtype):
    """PFFT_FLAG_TRANSPOSED: both directions through the plan of M^T (its
    adjoint passes without conjugations, its forward passes with conjugated
    input and output), compared with the oracle on every output."""
    m = abs(L.det(M))
    batch = 3
    try:
        plan = pf.PatternFFT(M, batch, dtype, route="transposed")
    except pf.PfftError as e:
        if e.status == 5:
            pytest.skip(f"no transposed route: {e}")
        raise
    assert plan.route == (True, True)
    npdt = np.complex64 if dtype == torch.complex64 else np.complex128
    c = SI.complex_normal(batch, m, seed=m % 89, dtype=npdt)
    ref = oracle.pattern_fft(M, c)
    tol = TOL["c64" if dtype == torch.complex64 else "c128"]
    assert rel_l2(plan.forward(_gpu(c)).cpu().numpy(), ref) <= tol
    back = plan.inverse(_gpu(ref.astype(npdt))).cpu().numpy()
    assert rel_l2(back, oracle.pattern_fft(M, ref, inverse=True)) <= tol
    plan.check_device_status()


@pytest.mark.parametrize("M,batch", [([[2048, 2], [0, 2048]], 2), ([[2048, 16], [0, 2048]], 2),
                                     ([[2048, 1], [0, 2048]], 2), (SI.M_BATCHED_2D, 2),
                                     ([[32, 5, 7], [0, 64, 9], [0, 0, 8192]], 1)])
def test_autotuned_route_sampled(M, batch):
    """PFFT_FLAG_AUTOTUNE at full size: whichever route each direction took,
    sampled frequencies against the oracle's direct sum and the round trip."""
    plan = pf.PatternFFT(M, batch, route="auto")
    m = plan.m
    c = SI.complex_normal(batch, m, 31)
    y = plan.forward(_gpu(c)).cpu().numpy()
    slots = SI.sample_slots(m, 512, seed=3)
    assert rel_l2(y[batch - 1:batch, slots], oracle.pattern_fft(M, c[batch - 1:batch], out_slots=slots)) <= 1e-5
    back = plan.inverse(_gpu(y)).cpu().numpy()
    assert rel_l2(back, c) <= 1e-5
    plan.check_device_status()
    assert all(isinstance(r, bool) for r in plan.route)


def test_long_cycle_fp64_full():
    """A cycle longer than the complex128 row tile (8192), full oracle."""
    M = [[4, 1], [0, 4096]]  # one cycle of 16384
    plan = pf.PatternFFT(M, 1, torch.complex128)
    c = SI.complex_normal(1, plan.m, 5, np.complex128)
    y = plan.forward(_gpu(c)).cpu().numpy()
    assert rel_l2(y, oracle.pattern_fft(M, c)) <= 1e-12
    assert rel_l2(plan.inverse(_gpu(y)).cpu().numpy(), c) <= 1e-12


def test_largest_direct_primes_sampled():
    """One cycle of 1021 * 1019 (the largest supported prime radices), split
    four-step; 512 sampled frequencies and the round trip."""
    M = [[1021, 0], [0, 1019]]
    plan = pf.PatternFFT(M, 1)
    c = SI.complex_normal(1, plan.m, 31)
    y = plan.forward(_gpu(c)).cpu().numpy()
    slots = SI.sample_slots(plan.m, 512, seed=3)
    assert rel_l2(y[:, slots], oracle.pattern_fft(M, c, out_slots=slots)) <= 1e-5
    assert rel_l2(plan.inverse(_gpu(y)).cpu().numpy(), c) <= 1e-5


def test_prime_beyond_direct_limit_is_rejected():
    with pytest.raises(pf.PfftError) as e:
        pf.PatternFFT([[1031, 0], [0, 2]], 1)
    assert e.value.status == 5
