#!/usr/bin/env python3
"""Benchmark of the pattern FFT hot path on GB300.

A step is one forward and one inverse pattern FFT (both passes of each, with
the gather / scatter between the Hermite boxes and the Smith coordinates
fused in) over one batch of the batched 2-D workload: M = [[4096, 1024],
[0, 4096]] (|det M| = 2^24, cycles (1024, 16384)), batch 8, complex64 inputs
with i.i.d. N(0,1) parts, resident in HBM.  Each buffer is 1 GiB, larger than
the 126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

The value is transform points per second (each forward or inverse transform
of m points counts m points) summed over all GPUs; for N > 1 every GPU runs
an independent replica (the workload has no exchange step) and the time is
the maximum over ranks.  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import seeded_inputs as SI  # noqa: E402

METRIC = "pattern-FFT points/s & % of HBM roofline vs plain FP32 form at rel-L2≤1e-5"
WORKLOAD = "batched_2d"
BYTES_PER_POINT_PASS = 16  # complex64: 8 B read + 8 B write per point and pass
KERNELS = ("row_pass", "col_pass")
WAVELET = "wavelet_2d"


def workload_desc(batch=None):
    w = SI.WORKLOADS[WORKLOAD]
    b = batch or w["batch"]
    return {"workload": "batched 2-D pattern FFT, forward + inverse", "M": w["M"], "m": 1 << 24,
            "batch": b, "cycles": [1024, 16384], "input": "complex64, re/im i.i.d. N(0,1), seed 1",
            "l2": f"inputs larger than L2 ({b * 128} MiB per buffer), no flush"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# sources that define each measured kernel and its launch configuration
KERNEL_SOURCES = {
    "row_pass": ["fft_row_pipe.cuh", "fft_tma.cu", "fft_tma.cuh", "fft_fast_ct.cuh", "fft_fast.cuh",
                 "device_common.cuh", "fft_plan.hpp"],
    "col_pass": ["fft_col_pipe.cuh", "fft_fast_ct.cu", "fft_fast_ct.cuh", "fft_fast.cuh", "device_common.cuh",
                 "fft_plan.hpp"],
}


def source_hash(kernel):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1107_5415_gb300", "csrc", name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get(kernel)
    if not ent or ent.get("source_hash") != source_hash(kernel):
        return None
    return ent.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def aggregate(ms_local: float, points_local: float, world: int):
    """Whole-job numbers: time = max over ranks, points = sum over ranks."""
    if world == 1:
        return ms_local, points_local
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    p = torch.tensor([points_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_sample_rate(target_s: float, threads: int | None = None):
    """Oracle (direct FP64 sum) on a bounded sample of the workload: S output
    frequencies of one signal.  Returns (points/s, seconds, S, threads)."""
    import oracle
    w = SI.WORKLOADS[WORKLOAD]
    M = w["M"]
    m = 1 << 24
    c = SI.complex_normal(1, m, w["seed"], dtype=np.complex128)
    nthreads = threads or os.cpu_count() or 1
    probe = SI.sample_slots(m, max(2 * nthreads, 16), seed=3)
    t0 = time.perf_counter()
    oracle.pattern_fft(M, c, out_slots=probe, nthreads=nthreads)
    per = (time.perf_counter() - t0) / len(probe)
    S = int(max(len(probe), min(1 << 16, target_s / max(per, 1e-9))))
    S = max(nthreads, (S // nthreads) * nthreads)
    slots = SI.sample_slots(m, S, seed=5)
    t0 = time.perf_counter()
    oracle.pattern_fft(M, c, out_slots=slots, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return S / dt, dt, S, nthreads


def smith_fftn(M, c):
    """A library CPU transform for context beside the oracle: the exact Smith
    gather lambda = Q^{-1} y mod eps of every box point of H(M), numpy's
    fftn over diag(eps) (Theorem 1, unitary), and the gather of the output box
    of H(M^T) at mu = R^{-T} k mod eps.  One signal c in box order."""
    from oracle import lattice as L
    d = len(M)
    Q, E, R = L.snf(M)
    eps = [E[i][i] for i in range(d)]
    Qi = np.array(L.inverse(Q), dtype=np.int64)
    RiT = np.array(L.transpose(L.inverse(R)), dtype=np.int64)
    mod = np.array(eps, dtype=np.int64)[:, None]
    y = np.indices(L.box_shape(M), dtype=np.int64).reshape(d, -1)
    lam = (Qi @ y) % mod
    X = np.zeros(eps, dtype=np.complex128)
    X[tuple(lam)] = c
    del y, lam
    Y = np.fft.fftn(X, norm="ortho")
    k = np.indices(L.box_shape(L.transpose(M)), dtype=np.int64).reshape(d, -1)
    return Y[tuple((RiT @ k) % mod)]


def fast_cpu_rate():
    """smith_fftn on one signal of the workload: (points/s, seconds)."""
    w = SI.WORKLOADS[WORKLOAD]
    c = SI.complex_normal(1, 1 << 24, w["seed"], dtype=np.complex128)[0]
    t0 = time.perf_counter()
    smith_fftn(w["M"], c)
    dt = time.perf_counter() - t0
    return c.size / dt, dt


def bench_wavelet(pf, torch, peaks_hbm, steps=20, warmup=3):
    """12-level split cascade on M_0 = 2^10 [[1,1],[-1,1]] (2^21 points), batch 16,
    Dirichlet and de la Vallee Poussin symbols, coefficients resident in HBM.
    Reports input points per second of the whole cascade and the roofline of
    its dominant kernel (the first split level: 8 B read + 8 B written per
    input point, from a one-level plan timed with CUDA events)."""
    w = SI.WORKLOADS[WAVELET]
    M, batch, levels = w["M"], w["batch"], w["levels"]
    out = {"workload": "12-level wavelet split cascade, M0 = 2^10 [[1,1],[-1,1]], J alternating "
                       "[[1,1],[-1,1]] / [[1,-1],[1,1]], batch 16, complex64", "m": 1 << 21, "batch": batch}
    stream = torch.cuda.current_stream()
    for sym, name in ((pf.PWT_DIRICHLET, "dirichlet"), (pf.PWT_DLVP, "dlvp")):
        for L in (levels, 1):
            plan = pf.WaveletSplit(M, SI.wavelet_dilations(L), sym, 0.125, batch)
            c = torch.from_numpy(SI.complex_normal(batch, plan.sizes[0], w["seed"])).cuda()
            for _ in range(warmup):
                plan.decompose(c)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                plan.decompose(c)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            pts = plan.sizes[0] * batch
            if L == levels:
                # compulsory bytes of the fused cascade: each group of three levels reads its
                # input once and writes every part once (16 B per input point of the group)
                alg, n_in = 0, pts
                for _ in range(0, levels, 3):
                    alg += 16 * n_in
                    n_in //= 8
                out[name] = {"value": pts / (ms * 1e-3), "unit": "points/s", "ms": ms,
                             "cascade_alg_bytes": alg, "cascade_gbs": alg / (ms * 1e-3) / 1e9,
                             "cascade_frac": alg / (ms * 1e-3) / 1e9 / peaks_hbm}
            else:
                gbs = 16 * pts / (ms * 1e-3) / 1e9
                out[name]["level1_kernel"] = {"avg_ms": ms, "achieved_gbs": gbs, "frac": gbs / peaks_hbm,
                                              "alg_bytes_per_launch": 16 * pts}
            plan.close()
    out["step5"] = bench_step5(pf, torch, steps=steps, warmup=warmup)
    return out


def _next_pattern(M, J):
    """N = J^{-1} M for |det J| = 2 (exact: adj(J) M / det J)."""
    M = np.asarray(M, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    det = int(round(np.linalg.det(J)))
    adj = np.array([[J[1, 1], -J[0, 1]], [-J[1, 0], J[0, 0]]], dtype=np.int64)
    P = adj @ M
    assert (P % det == 0).all()
    return (P // det).tolist()


def bench_step5(pf, torch, steps=20, warmup=3):
    """Section 5.3 step 5 on the 12-level workload (Dirichlet symbol): the
    split cascade alone, and the cascade followed by the inverse pattern FFT
    of each of its 13 parts on G(N_l^T) (12 wavelet parts, one scaling part),
    with the step-5 transforms in the plain fp32 form and in the
    split-precision tensor-core form.  Input points of the cascade per second;
    the tensor-core result is compared with the fp32 one over all parts (each
    form's error against the FP64 oracle is checked by the tests)."""
    w = SI.WORKLOADS[WAVELET]
    M, batch, levels = w["M"], w["batch"], w["levels"]
    Js = SI.wavelet_dilations(levels)
    split = pf.WaveletSplit(M, Js, pf.PWT_DIRICHLET, 0.125, batch)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w["seed"])
    c = torch.randn(batch, split.sizes[0], dtype=torch.complex64, device="cuda", generator=gen)
    sc, wv = split.decompose(c)
    Ns, cur = [], M
    for J in Js:
        cur = _next_pattern(cur, J)
        Ns.append(cur)
    parts = list(zip(Ns, wv)) + [(Ns[-1], sc)]
    pts = split.sizes[0] * batch
    out = {"workload": "12-level cascade (Dirichlet) + inverse pattern FFT of every part (Section 5.3 step 5)"}
    ms_split = _time_ms(torch, lambda: split.decompose(c), steps, warmup)
    out["split_only"] = {"ms": ms_split, "value": pts / (ms_split * 1e-3), "unit": "points/s"}
    results = {}
    for form in ("fp32", "tc_split"):
        plans = [pf.PatternFFT(N, batch, tc_split=(form == "tc_split")) for N, _ in parts]
        outs = [torch.empty_like(x) for _, x in parts]

        def chain():
            s_, w_ = split.decompose(c)
            for p_, x_, o_ in zip(plans, w_ + [s_], outs):
                p_.inverse(x_, o_)

        ms = _time_ms(torch, chain, steps, warmup)
        results[form] = torch.cat([o.flatten() for o in outs])
        out[form] = {"ms": ms, "value": pts / (ms * 1e-3), "unit": "points/s",
                     "step5_ms": ms - ms_split}
        for p_ in plans:
            p_.close()
    num = torch.linalg.vector_norm(results["tc_split"] - results["fp32"]).item()
    out["tc_split"]["rel_l2_vs_fp32"] = num / torch.linalg.vector_norm(results["fp32"]).item()
    out["tc_split"]["speedup_vs_fp32"] = out["fp32"]["ms"] / out["tc_split"]["ms"]
    split.close()
    return out


def bench_tc(pf, torch, x, y_fp32, ms_fp32, peaks_hbm, steps=50, warmup=5):
    """The same step (forward + inverse of the batched 2-D workload) in the
    split-precision tensor-core form: the radix-32 stages as fp16 hi + lo
    DFT-matrix products on the tensor cores (tcgen05) with fp32 accumulation.  Reports
    its speed against the plain fp32 form measured above and its agreement
    with it (the error against the FP64 oracle is checked by the tests)."""
    w = SI.WORKLOADS[WORKLOAD]
    plan = pf.PatternFFT(w["M"], x.shape[0], tc_split=True)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.forward(x, y)
        plan.inverse(y, z)
    torch.cuda.synchronize()
    plan.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.forward(x, y)
        plan.inverse(y, z)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = plan.profile_read()
    plan.close()
    pts = 2.0 * x.numel()
    num = torch.linalg.vector_norm((y - y_fp32).flatten()).item()
    den = torch.linalg.vector_norm(y_fp32.flatten()).item()
    rt = (torch.linalg.vector_norm((z - x).flatten()) / torch.linalg.vector_norm(x.flatten())).item()
    kernels = {k: {"launches": int(v[0]), "avg_ms": v[1] / max(v[0], 1),
                   "achieved_gbs": BYTES_PER_POINT_PASS * x.numel() / (v[1] / max(v[0], 1) * 1e-3) / 1e9}
               for k, v in prof.items() if v[0]}
    return {"form": "split fp16 (hi + lo) radix-32 stages on tcgen05 (radix-16 tail in fp32), fp32 accumulation",
            "value": pts / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms,
            "speedup_vs_plain_fp32": ms_fp32 / ms, "rel_l2_vs_plain_fp32": num / den,
            "round_trip_rel_l2": rt, "kernels": kernels,
            "compulsory_frac": BYTES_PER_POINT_PASS * pts / (ms * 1e-3) / 1e9 / peaks_hbm}


TABLE1_I = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 0]
# Table 1 (Section 6.1), context only: serial times (s) of the paper's implementation
# (Mathematica 8 Fourier, Intel Core 2 Quad at 2 GHz, 4 GB), per i, and its 1-D FFT of
# the same 2^22 points (0.260816 s)
TABLE1_PAPER_SERIAL_S = {1: 0.266664, 2: 0.471722, 4: 0.468220, 8: 0.457126, 16: 0.457321, 32: 0.469080,
                         64: 0.466902, 128: 0.572192, 256: 0.920226, 512: 1.144126, 1024: 0.949403,
                         0: 0.907286}
TABLE1_PAPER_1D_S = 0.260816


def _time_ms(torch, fn, steps, warmup):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_table1(pf, torch, peaks_hbm, steps=20, warmup=3):
    """The pattern family of Table 1 (Section 6.1): M = [[2048, i], [0, 2048]]
    for every divisor i of 2048 (i = 0 last), 2^22 points, forward transforms
    of 8 signals per launch (256 MiB, larger than L2).  The factor is the
    time against the 1-D transform of 2^22 points by this library
    (M = [[2^22]]), the comparison the table's factor column makes; the
    library 1-D FFT of torch (cuFFT) is listed as context.  Each row is timed
    with the direct route and with the route chosen at plan time
    (PFFT_FLAG_AUTOTUNE: the forward transform of M may run as the adjoint
    passes of M^T)."""
    w = SI.WORKLOADS["table1"]
    n, batch = w["n"], w["batch"]
    m = n * n
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w["seed"])
    x = torch.randn(batch, m, dtype=torch.complex64, device="cuda", generator=gen) * math.sqrt(2.0)
    y = torch.empty_like(x)

    def run(M, route="direct"):
        plan = pf.PatternFFT(M, batch, route=route)
        ms = _time_ms(torch, lambda: plan.forward(x, y), steps, warmup)
        via = plan.route[0]
        plan.close()
        return ms, via

    ms_1d, _ = run([[m]])
    ms_cufft = _time_ms(torch, lambda: torch.fft.fft(x, dim=1, norm="ortho"), steps, warmup)
    rows = []
    for i in TABLE1_I:
        ms, _ = run([[n, i], [0, n]])
        ms_auto, via = run([[n, i], [0, n]], "auto")
        rows.append({"i": i, "ms_per_transform": ms / batch, "factor_vs_1d": ms / ms_1d,
                     "achieved_gbs_2pass": 2 * 16 * batch * m / (ms * 1e-3) / 1e9,
                     "autotuned_ms_per_transform": ms_auto / batch, "autotuned_via_transpose": via,
                     "autotuned_achieved_gbs_2pass": 2 * 16 * batch * m / (ms_auto * 1e-3) / 1e9,
                     "paper_serial_s": TABLE1_PAPER_SERIAL_S[i],
                     "paper_factor": TABLE1_PAPER_SERIAL_S[i] / TABLE1_PAPER_1D_S})
    return {"workload": "Table 1 family M = [[2048, i], [0, 2048]], 2^22 points, 8 signals per launch",
            "paper_context": "paper: Mathematica 8 on an Intel Core 2 Quad at 2 GHz, serial; 1-D FFT of 2^22 "
                             "points 0.260816 s",
            "one_d_ms_per_transform": ms_1d / batch, "cufft_1d_ms_per_transform": ms_cufft / batch,
            "rows": rows}


def bench_autograd3d(pf, torch, peaks_hbm, steps=20, warmup=3):
    """The 3-D workload with autograd: M = [[256,64,0],[0,256,32],[0,0,256]]
    (cycles 32, 64, 8192), batch 4, complex64.  Times the forward and the
    inverse transform (two passes each, 16 B per point and pass compulsory)
    and one gradient step of loss = sum |w * F c|^2 with real weights w (the
    forward transform, the loss, and the backward pass through the inverse
    kernels)."""
    w = SI.WORKLOADS["autograd_3d"]
    M, batch = w["M"], w["batch"]
    plan = pf.PatternFFT(M, batch)
    m = plan.m
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w["seed"])
    x = torch.randn(batch, m, dtype=torch.complex64, device="cuda", generator=gen)
    wt = torch.rand(batch, m, device="cuda", generator=gen)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    fwd = _time_ms(torch, lambda: plan.forward(x, y), steps, warmup)
    inv = _time_ms(torch, lambda: plan.inverse(y, z), steps, warmup)
    xg = x.clone().requires_grad_(True)

    def grad_step():
        xg.grad = None
        loss = (wt * pf.pattern_fft(xg, plan).abs() ** 2).sum()
        loss.backward()

    step = _time_ms(torch, grad_step, steps, warmup)
    pts = batch * m
    comp = lambda ms: 2 * 16 * pts / (ms * 1e-3) / 1e9
    out = {"workload": "3-D pattern FFT, M = [[256,64,0],[0,256,32],[0,0,256]], batch 4, complex64",
           "forward_ms": fwd, "inverse_ms": inv, "grad_step_ms": step,
           "forward_points_per_s": pts / (fwd * 1e-3),
           "forward_compulsory_gbs": comp(fwd), "forward_compulsory_frac": comp(fwd) / peaks_hbm,
           "inverse_compulsory_frac": comp(inv) / peaks_hbm}
    plan.close()
    return out


def bench_directional(pf, torch, peaks_hbm, steps=20, warmup=3):
    """One split level of M = 512 I by each dilation of Section 6.2's set
    {J_x, J_y, J_d} (Dirichlet symbol), 16 signals of anisotropic synthetic
    coefficients c_h = (1 + h_1^2 + 16 h_2^2)^{-1} z_h (h centred, z complex
    N(0,1) seeded); per dilation the time and the share of the energy that
    lands in the wavelet part."""
    w = SI.WORKLOADS["directional"]
    M, batch = w["M"], w["batch"]
    n = M[0][0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w["seed"])
    h = torch.arange(n, device="cuda", dtype=torch.float32)
    h = torch.where(h >= n // 2, h - n, h)
    wt = 1.0 / (1.0 + h[:, None] ** 2 + 16.0 * h[None, :] ** 2)
    c = (torch.randn(batch, n * n, dtype=torch.complex64, device="cuda", generator=gen) * math.sqrt(2.0)
         * wt.reshape(1, -1))
    e_c = torch.linalg.vector_norm(c).item() ** 2
    out = {"workload": "one split level, M = 512 I, J in {J_x, J_y, J_d}, batch 16, anisotropic coefficients"}
    for name, J in SI.DIRECTIONAL_J.items():
        plan = pf.WaveletSplit(M, [J], pf.PWT_DIRICHLET, 0.125, batch)
        sc, wv = plan.decompose(c)
        ms = _time_ms(torch, lambda: plan.decompose(c), steps, warmup)
        e_w = torch.linalg.vector_norm(wv[0]).item() ** 2
        out[name] = {"J": J, "ms": ms, "wavelet_energy_share": e_w / e_c,
                     "achieved_gbs": 16 * batch * n * n / (ms * 1e-3) / 1e9}
        plan.close()
    return out


def bench_snf_layout(pf, torch, x, ms_box, steps=50, warmup=5):
    """The same step in the Smith-coordinate layout (PFFT_FLAG_LAYOUT_SNF):
    the transform without the gather from and the scatter to the Hermite
    boxes (the order the paper computes in); its time against the box layout
    shows what the reordering costs."""
    w = SI.WORKLOADS[WORKLOAD]
    plan = pf.PatternFFT(w["M"], x.shape[0], layout="snf")
    y = torch.empty_like(x)
    z = torch.empty_like(x)

    def step():
        plan.forward(x, y)
        plan.inverse(y, z)

    ms = _time_ms(torch, step, steps, warmup)
    plan.close()
    return {"value": 2.0 * x.numel() / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms,
            "box_layout_ms_per_step": ms_box, "box_over_snf": ms_box / ms}


def bench_mix(pf, torch, peaks_hbm, steps=10, warmup=3, n_patterns=None):
    """Uneven serving-style mix: 4096 seeded patterns (d in {2, 3}, upper
    triangular, diagonals in [16, 512], det <= 2^20), forward transform + one
    Dirichlet split level per pattern (a dilation of determinant 2 when det M
    is even, else of the smallest odd prime of det M with the built-in band
    system), replayed as one CUDA graph with the autotuned schedule.  Inputs:
    seeded complex normal values drawn on the device."""
    w = SI.WORKLOADS["uneven_mix"]
    Ms = SI.uneven_mix(w["n_patterns"], seed=w["seed"], even_det=w["even_det"])[:n_patterns or w["n_patterns"]]
    Js = [SI.mix_dilation(M) for M in Ms]
    t0 = time.perf_counter()
    B = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, flags=pf.PFFT_BATCH_AUTOTUNE)
    t_plan = time.perf_counter() - t0
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w["seed"])
    x = torch.randn(B.total, dtype=torch.complex64, device="cuda", generator=gen) * math.sqrt(2.0)
    chat = torch.empty_like(x)
    sc = torch.empty(B.sc_total, dtype=torch.complex64, device="cuda")
    wv = torch.empty(B.wv_total, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    odd = int((B.p % 2 == 1).sum())
    out = {"workload": f"uneven mix: {B.n} patterns ({odd} of odd determinant, split by an odd prime), "
                       "forward FFT + one split level each", "patterns": B.n,
           "points": int(B.total), "plan_s": t_plan, "schedule": dict(zip(("row_budget", "col_budget", "order", "max_radix"),
                                                                           B.schedule()))}
    for split, name in ((True, "fft_split"), (False, "fft_only")):
        for _ in range(warmup):
            B.forward(x, chat, sc, wv, split=split)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            B.forward(x, chat, sc, wv, split=split)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        alg = (32 if split else 16) * B.total  # compulsory bytes: FFT 8 + 8, split 8 + 4 + 4 per point
        out[name] = {"value": B.total / (ms * 1e-3), "unit": "points/s", "ms": ms,
                     "compulsory_gbs": alg / (ms * 1e-3) / 1e9, "compulsory_frac": alg / (ms * 1e-3) / 1e9 / peaks_hbm}
    B.close()
    # the same batch in one launch (device work queue, bounded dependency waits)
    t0 = time.perf_counter()
    Q = pf.PatternBatch(Ms, Js, pf.PWT_DIRICHLET, flags=pf.PFFT_BATCH_AUTOTUNE | pf.PFFT_BATCH_ONE_LAUNCH)
    out["one_launch_plan_s"] = time.perf_counter() - t0
    for split, name in ((True, "fft_split_one_launch"), (False, "fft_only_one_launch")):
        for _ in range(warmup):
            Q.forward(x, chat, sc, wv, split=split)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            Q.forward(x, chat, sc, wv, split=split)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"value": Q.total / (ms * 1e-3), "unit": "points/s", "ms": ms, "launches_per_step": 1}
    Q.check_device_status()
    Q.close()
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    target = float(os.environ.get("PFFT_REF_STEP_S", "2.0"))
    times, rates = [], []
    S = threads = None
    for i in range(args.warmup + args.steps):
        rate, dt, S, threads = oracle_sample_rate(target)
        if i >= args.warmup:
            times.append(dt)
            rates.append(rate)
    value = float(np.median(rates))
    sample = (f"direct FP64 sum (oracle) for {S} seeded output frequencies of one of the 8 signals "
              f"of the workload, per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.median(times)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_desc(),
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import torch
    import paper_1107_5415_gb300 as pf
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = SI.WORKLOADS[WORKLOAD]
    M, batch = w["M"], args.batch or w["batch"]
    plan = pf.PatternFFT(M, batch)
    m = plan.m
    host = torch.from_numpy(SI.complex_normal(batch, m, w["seed"] + 1000 * rank))
    x = host.to(dev)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def step():
        plan.forward(x, y)
        plan.inverse(y, z)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    plan.profile(True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    prof = plan.profile_read()
    plan.profile(False)
    barrier(world)
    torch.cuda.synchronize()
    points_local = 2.0 * m * batch  # forward + inverse transform points per step
    ms_max, points = aggregate(ms, points_local, world)
    value = points / (ms_max * 1e-3)

    peaks_hbm = float(measured_peaks()[0]["hbm_gbs"])
    tc = None
    if not args.no_tc:
        plan.forward(x, y)
        tc = bench_tc(pf, torch, x, y, ms, peaks_hbm)
    snf_layout = None if args.no_tc else bench_snf_layout(pf, torch, x, ms)
    wavelet = None if args.no_wavelet else bench_wavelet(pf, torch, peaks_hbm=peaks_hbm)
    mix = None if args.no_mix else bench_mix(pf, torch, peaks_hbm=peaks_hbm, n_patterns=args.mix_patterns)
    table1 = None if args.no_table1 else bench_table1(pf, torch, peaks_hbm)
    autograd3d = None if args.no_table1 else bench_autograd3d(pf, torch, peaks_hbm)
    directional = None if args.no_directional else bench_directional(pf, torch, peaks_hbm)
    if args.no_e2e:
        e2e_value, e2e_ms = None, None
        plan.close()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "points/s", "ms_per_step": ms_max,
                              "kernels": prof, "tc_split": tc, "snf_layout": snf_layout, "wavelet": wavelet,
                              "uneven_mix": mix,
                              "table1": table1, "autograd_3d": autograd3d, "directional": directional,
                              "note": "profiling run (no e2e)"}), flush=True)
        return 0
    # end to end through the public API with host buffers (pinned), per step:
    # H2D of the input, forward + inverse, D2H of the result.  The steps are
    # pipelined as a serving loop would run them: uploads, transforms and
    # downloads on three streams with double buffers, so that step k's
    # transforms overlap step k+1's upload and step k-1's download.
    hin = host.pin_memory()
    houts = [torch.empty_like(hin).pin_memory() for _ in range(2)]
    xs = [x, torch.empty_like(x)]
    zs = [z, torch.empty_like(z)]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for e in ev_cmp + ev_out:
        e.record(stream)

    def e2e_steps_run(n):
        for k in range(n):
            i = k % 2
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_cmp[i])           # step k-2 has finished reading xs[i]
                xs[i].copy_(hin, non_blocking=True)
                ev_in[i].record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_in[i])
                s_cmp.wait_event(ev_out[i])          # step k-2's download of zs[i] is done
                plan.forward(xs[i], y, stream=s_cmp)
                plan.inverse(y, zs[i], stream=s_cmp)
                ev_cmp[i].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_cmp[i])
                houts[i].copy_(zs[i], non_blocking=True)
                ev_out[i].record(s_out)

    e2e_steps = max(3, min(args.steps, 20))
    e2e_steps_run(2)
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s_in.wait_event(ev_out[0])
    s_in.wait_event(ev_out[1])
    e0.record(s_in)
    e2e_steps_run(e2e_steps)
    s_in.wait_event(ev_out[0])
    s_in.wait_event(ev_out[1])
    e1.record(s_in)
    torch.cuda.synchronize()
    e2e_ms, _ = aggregate(e0.elapsed_time(e1) / e2e_steps, points_local, world)
    e2e_value = points / (e2e_ms * 1e-3)

    # roofline of the dominant kernel: algorithmic bytes per launch / mean duration
    peaks, peak_kind = measured_peaks()
    dom = max(KERNELS, key=lambda k: prof.get(k, (0, 0.0))[1])
    launches, tot_ms = prof[dom]
    avg_s = tot_ms / launches * 1e-3
    alg_bytes = BYTES_PER_POINT_PASS * m * batch
    achieved = alg_bytes / avg_s / 1e9
    peak = float(peaks["hbm_gbs"])
    traffic = recorded_traffic(dom)
    kernels = {k: {"launches": int(v[0]), "avg_ms": v[1] / max(v[0], 1),
                   "achieved_gbs": BYTES_PER_POINT_PASS * m * batch / (v[1] / max(v[0], 1) * 1e-3) / 1e9}
               for k, v in prof.items() if v[0]}

    line = None
    if rank == 0:
        cpu = cpu_fast = None
        if world == 1 and not args.no_cpu_baseline:
            rate, dt, S, threads = oracle_sample_rate(float(os.environ.get("PFFT_CPU_BASELINE_S", "15")))
            cpu = {"value": rate, "unit": "points/s", "cores": threads, "kind": "oracle",
                   "sample": f"direct FP64 sum for {S} seeded output frequencies of one signal "
                             f"({dt:.1f} s on the host cores)",
                   "extrapolated_full_step_s": points / rate,
                   "extrapolated_note": "one whole step (forward + inverse, all signals) by the "
                                        "direct sum at the sampled rate: extrapolated, not measured"}
            try:
                frate, fdt = fast_cpu_rate()
                cpu_fast = {"value": frate, "unit": "points/s", "cores": 1,
                            "kind": "numpy.fft.fftn after the exact Smith-coordinate gather (Theorem 1); "
                                    "a library transform for context, not the oracle",
                            "sample": f"one forward transform of one 2^24-point signal ({fdt:.1f} s)"}
            except Exception as e:  # context only: never fail the bench line on it
                cpu_fast = {"error": f"{type(e).__name__}: {e}"[:200]}
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_desc(),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs", "alg_bytes_per_launch": alg_bytes},
            "compulsory_frac": (BYTES_PER_POINT_PASS * points_local / (ms * 1e-3) / 1e9) / peak,
            "kernels": kernels,
            "cpu_baseline": cpu,
            "cpu_fast_baseline": cpu_fast,
            "tc_split": tc,
            "snf_layout": snf_layout,
            "wavelet": wavelet,
            "uneven_mix": mix,
            "table1": table1,
            "autograd_3d": autograd3d,
            "directional": directional,
            "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": int(x.numel() * 8),
                    "d2h_bytes_per_step": int(z.numel() * 8),
                    "ms_per_step": e2e_ms, "h2d_gbs": x.numel() * 8 / (e2e_ms * 1e-3) / 1e9,
                    "note": "pinned host buffers; uploads, transforms and downloads pipelined on three streams"},
            "gpu_launches": 4 * args.steps,
            "clocks": clk.summary(),
            "impl": "native",
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-wavelet", action="store_true", help="skip the wavelet cascade measurement")
    ap.add_argument("--no-mix", action="store_true", help="skip the uneven pattern-mix measurement")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core form measurement")
    ap.add_argument("--mix-patterns", type=int, default=0,
                    help="first N patterns of the uneven mix only (profiling runs; default all 4096)")
    ap.add_argument("--no-table1", action="store_true",
                    help="skip the Table 1 pattern sweep and the 3-D autograd workload")
    ap.add_argument("--no-directional", action="store_true", help="skip the directional dilation comparison")
    ap.add_argument("--batch", type=int, default=0, help="override the workload batch (profiling runs)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    return run_reference(args) if args.impl == "reference" else run_native(args)


if __name__ == "__main__":
    sys.exit(main())
