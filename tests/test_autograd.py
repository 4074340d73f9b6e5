"""Hand-written adjoints behind torch.autograd: the transform's backward runs
the inverse kernels (F(M) is unitary), the split's backward runs the adjoint
kernel.  Checked against FP64 central finite differences on a tiny pattern
and against the oracle's analytic gradient."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lattice as L
import paper_1107_5415_gb300 as pf
import seeded_inputs as SI
from parity_util import rel_l2

pytestmark = pytest.mark.gpu


def _loss(plan, c, w):
    y = pf.pattern_fft(c, plan)
    return ((w * y).abs() ** 2).sum()


def test_finite_differences_tiny_pattern():
    M = SI.M_AUTOGRAD_TINY
    plan = pf.PatternFFT(M, 1, torch.complex128)
    m = plan.m
    c0 = torch.from_numpy(SI.complex_normal(1, m, 2, np.complex128)).cuda()
    w = torch.from_numpy(SI.uniform01((1, m), 2)).cuda()
    c = c0.clone().requires_grad_(True)
    _loss(plan, c, w).backward()
    g = c.grad.cpu().numpy()
    h = 1e-6
    fd = np.zeros(m, np.complex128)
    with torch.no_grad():
        for i in range(m):
            for part, unit in ((0, 1.0), (1, 1j)):
                e = torch.zeros_like(c0)
                e[0, i] = unit * h
                lp = _loss(plan, c0 + e, w).item()
                lm = _loss(plan, c0 - e, w).item()
                d = (lp - lm) / (2 * h)
                fd[i] += d if part == 0 else 1j * d
    assert np.max(np.abs(fd - g[0])) < 1e-6 * np.max(np.abs(g))
    # analytic gradient of the oracle: 2 F^H (w^2 . F c)
    y = oracle.pattern_fft(M, c0.cpu().numpy())
    ref = 2 * oracle.pattern_fft(M, (w.cpu().numpy() ** 2) * y, inverse=True)
    assert rel_l2(g, ref) <= 1e-12


def test_autograd_3d_workload_sampled_gradient():
    wl = SI.WORKLOADS["autograd_3d"]
    M, batch = wl["M"], wl["batch"]
    plan = pf.PatternFFT(M, batch)
    m = plan.m
    c = torch.from_numpy(SI.complex_normal(batch, m, wl["seed"])).cuda().requires_grad_(True)
    w = torch.from_numpy(SI.uniform01((batch, m), wl["seed"], np.float32)).cuda()
    y = pf.pattern_fft(c, plan)
    ((w * y).abs() ** 2).sum().backward()
    g = c.grad.cpu().numpy()
    # oracle: 2 F^H (w^2 . y) on 1024 sampled slots of signal 0, with y checked first
    yh = y.detach().cpu().numpy()
    slots = SI.sample_slots(m, 512)
    assert rel_l2(yh[0:1, slots], oracle.pattern_fft(M, c.detach().cpu().numpy()[0:1], out_slots=slots)) <= 1e-5
    rhs = 2 * (w.cpu().numpy()[0:1].astype(np.float64) ** 2) * yh[0:1].astype(np.complex128)
    ref = oracle.pattern_fft(M, rhs, inverse=True, out_slots=slots)
    assert rel_l2(g[0:1, slots], ref) <= 1e-5
    # adjoint dot-product identity <F c, u> = <c, F^H u> on every signal
    u = torch.from_numpy(SI.complex_normal(batch, m, 99)).cuda()
    lhs = (plan.forward(c.detach()).conj() * u).sum(dim=1)
    rhs = (c.detach().conj() * plan.inverse(u)).sum(dim=1)
    assert torch.allclose(lhs, rhs, rtol=1e-4, atol=1e-2)


def test_wavelet_split_gradient():
    M, Js = [[16, 16], [-16, 16]], SI.wavelet_dilations(3)
    plan = pf.WaveletSplit(M, Js, pf.PWT_DLVP, 0.125, 1, torch.complex128)
    c = torch.from_numpy(SI.complex_normal(1, plan.sizes[0], 4, np.complex128)).cuda().requires_grad_(True)
    s, w = pf.wavelet_decompose(c, plan)
    loss = (s.abs() ** 2).sum() + 0.5 * sum((x.abs() ** 2).sum() for x in w)
    loss.backward()
    # finite differences on a few coordinates
    h = 1e-6
    c0 = c.detach()
    for i in (0, 7, 100, 255):
        for unit in (1.0, 1j):
            e = torch.zeros_like(c0)
            e[0, i] = unit * h
            def L_(x):
                s_, w_ = plan.decompose(x)
                return ((s_.abs() ** 2).sum() + 0.5 * sum((y.abs() ** 2).sum() for y in w_)).item()
            fd = (L_(c0 + e) - L_(c0 - e)) / (2 * h)
            got = c.grad[0, i].real.item() if unit == 1.0 else c.grad[0, i].imag.item()
            assert abs(fd - got) < 1e-6 * (1 + abs(fd))
