"""GPU parity of the wavelet split (Section 5.3 step 4, symbols of Section
6.2) against the FP64 oracle, through the C ABI, including the 12-level
cascade on M_0 = 2^10 [[1,1],[-1,1]] with batch 16 at full size."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import rel_l2

pytestmark = pytest.mark.gpu

SYM = {"dirichlet": (pf.PWT_DIRICHLET, oracle.DIRICHLET), "dlvp": (pf.PWT_DLVP, oracle.DLVP)}

CASES = [([[8, 8], [-8, 8]], [SI.J_DIAG_A]), ([[8, 0], [0, 8]], [[[2, 0], [0, 1]]]),
         ([[8, 0], [0, 8]], [[[1, 0], [0, 2]]]), ([[6, 2], [-2, 6]], [SI.J_DIAG_A]),
         ([[16, 16], [-16, 16]], SI.wavelet_dilations(5)),
         ([[12, 4], [0, 10]], [[[2, 0], [0, 1]], [[1, 0], [0, 2]]]),
         ([[4, 1, 0], [0, 4, 1], [0, 0, 4]], [[[1, 0, 0], [0, 1, 0], [0, 0, 2]]]),
         ([[8, 2, 0], [0, 4, 2], [0, 0, 6]], [[[2, 0, 0], [0, 1, 0], [0, 0, 1]], [[1, 0, 0], [0, 2, 0], [0, 0, 1]]]),
         # dilations whose symbol cube does not contain [-1/2, 1/2]^d (parity dilations)
         ([[3, 1], [1, 3]], [[[1, 0], [-1, 2]]]),
         ([[10, 1, 7], [0, 9, 1], [0, 0, 32]], [[[1, 0, 0], [-1, 2, 0], [0, 0, 1]]]),
         ([[6, 1, 1], [0, 5, 1], [0, 0, 4]], [[[1, 0, 0], [0, 1, 0], [-1, -1, 2]]])]


def _gpu(x, dt=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("sym", ["dirichlet", "dlvp"])
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_small_cascades_vs_oracle(case, sym, dtype):
    M, Js = CASES[case]
    gsym, osym = SYM[sym]
    batch = 2
    m = abs(L.det(M))
    plan = pf.WaveletSplit(M, Js, gsym, 0.125, batch, dtype)
    c = SI.complex_normal(batch, m, 3, dtype=np.complex128)
    s_ref, w_ref = oracle.wavelet_cascade(M, Js, c, osym, 0.125)
    s, w = plan.decompose(_gpu(c, dtype))
    tol = 1e-5 if dtype == torch.complex64 else 1e-12
    assert rel_l2(s.cpu().numpy(), s_ref) <= tol
    for a, b in zip(w, w_ref):
        assert rel_l2(a.cpu().numpy(), b) <= tol
    back = plan.reconstruct(s, w).cpu().numpy()
    assert rel_l2(back, c) <= tol
    back_ref = oracle.wavelet_cascade_inverse(M, Js, s_ref, w_ref, osym, 0.125, mode="adjoint")
    adj = plan.adjoint(_gpu(s_ref, dtype), [_gpu(x, dtype) for x in w_ref]).cpu().numpy()
    assert rel_l2(adj, back_ref) <= tol


def _centred_weight(M):
    """(1 + |h|^2)^{-1} for the centred representative h of every output slot."""
    G = L.hnf(L.transpose(M))
    d = len(M)
    ext = [G[i][i] for i in range(d)]
    grids = np.meshgrid(*[np.arange(e, dtype=np.int64) for e in ext], indexing="ij")
    h = np.stack([g.reshape(-1) for g in grids], axis=1)                # box points
    D = L.det(M)
    A = np.array(L.adjugate(L.transpose(M)), dtype=np.int64)            # M^{-T} = adj(M^T) / det
    p = (h @ A.T) * (1 if D > 0 else -1)
    q = abs(D)
    u = p - q * np.floor_divide(2 * p + q, 2 * q)                       # centred numerators
    k = (u @ np.array(M, dtype=np.int64)) // q                          # k = M^T u  (row form)
    assert ((u @ np.array(M, dtype=np.int64)) % q == 0).all()
    return 1.0 / (1.0 + (k.astype(np.float64) ** 2).sum(axis=1))


@pytest.mark.parametrize("sym", ["dirichlet", "dlvp"])
def test_twelve_level_workload_full_size(sym):
    w = SI.WORKLOADS["wavelet_2d"]
    M, batch, levels = w["M"], w["batch"], w["levels"]
    Js = SI.wavelet_dilations(levels)
    gsym, osym = SYM[sym]
    m = abs(L.det(M))
    c = SI.complex_normal(batch, m, w["seed"], dtype=np.complex128) * _centred_weight(M)[None, :]
    plan = pf.WaveletSplit(M, Js, gsym, 0.125, batch)
    s, wav = plan.decompose(_gpu(c))
    s_ref, w_ref = oracle.wavelet_cascade(M, Js, c, osym, 0.125)
    assert rel_l2(s.cpu().numpy(), s_ref) <= 1e-5
    for a, b in zip(wav, w_ref):
        assert rel_l2(a.cpu().numpy(), b) <= 1e-5
    back = plan.reconstruct(s, wav).cpu().numpy()
    assert rel_l2(back, c) <= 1e-5
    if sym == "dirichlet":
        tot = np.linalg.norm(s.cpu().numpy(), axis=1) ** 2 + sum(
            np.linalg.norm(x.cpu().numpy(), axis=1) ** 2 for x in wav)
        assert np.allclose(tot, np.linalg.norm(c, axis=1) ** 2, rtol=1e-5)


def test_adjoint_dot_product_on_gpu():
    M, Js = [[32, 32], [-32, 32]], SI.wavelet_dilations(4)
    for gsym in (pf.PWT_DIRICHLET, pf.PWT_DLVP):
        plan = pf.WaveletSplit(M, Js, gsym, 0.125, 1, torch.complex128)
        c = _gpu(SI.complex_normal(1, plan.sizes[0], 1, np.complex128), torch.complex128)
        s, w = plan.decompose(c)
        e_s = _gpu(SI.complex_normal(1, plan.sizes[-1], 2, np.complex128), torch.complex128)
        e_w = [_gpu(SI.complex_normal(1, n, 3 + i, np.complex128), torch.complex128)
               for i, n in enumerate(plan.sizes[1:])]
        ct = plan.adjoint(e_s, e_w)
        lhs = torch.vdot(e_s.flatten(), s.flatten()) + sum(torch.vdot(a.flatten(), b.flatten())
                                                          for a, b in zip(e_w, w))
        rhs = torch.vdot(ct.flatten(), c.flatten())
        assert abs(complex(lhs - rhs)) < 1e-10 * plan.sizes[0]


def test_wavelet_argument_errors():
    with pytest.raises(pf.PfftError) as e:
        pf.WaveletSplit([[3, 0], [0, 4]], [[[2, 0], [0, 1]]])
    assert e.value.status == 4
    with pytest.raises(pf.PfftError) as e:
        pf.WaveletSplit([[8, 0], [0, 8]], [[[3, 0], [0, 1]]])
    assert e.value.status == 5


@pytest.mark.parametrize("name", list(SI.DIRECTIONAL_J))
@pytest.mark.parametrize("sym", ["dirichlet", "dlvp"])
def test_directional_dilations_one_level(name, sym):
    """One split level of M = 512 I by each dilation of the set of Section 6.2
    (J_x, J_y, J_d), on seeded coefficients, every output against the oracle;
    perfect reconstruction on the GPU."""
    w = SI.WORKLOADS["directional"]
    M, J = w["M"], SI.DIRECTIONAL_J[name]
    gsym, osym = SYM[sym]
    plan = pf.WaveletSplit(M, [J], gsym, 0.125, 2)
    c = SI.complex_normal(2, plan.sizes[0], w["seed"])
    s_gpu, w_gpu = plan.decompose(_gpu(c))
    d1, d2 = oracle.wavelet_level(M, J, osym, 0.125, c_hat=c)
    assert rel_l2(s_gpu.cpu().numpy(), d1) <= 1e-5
    assert rel_l2(w_gpu[0].cpu().numpy(), d2) <= 1e-5
    back = plan.reconstruct(s_gpu, w_gpu).cpu().numpy()
    assert rel_l2(back, c) <= 1e-5
