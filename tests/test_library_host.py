"""CPU tests of the C-ABI library: it builds, loads and exports every entry
point declared in include/pfft.h, and its exact host planner agrees with the
oracle's independent lattice code.  No compute calls (no GPU here)."""
import os
import re
import subprocess

import numpy as np
import pytest
import torch

import oracle
import paper_1107_5415_gb300 as pf
from paper_1107_5415_gb300 import _capi
from oracle import lattice as L
import seeded_inputs as SI

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pfft.h")).read()
    return sorted(set(re.findall(r"^\s*(?:pfft_status|const char\*)\s+((?:pfft|pwt)_\w+)\(", src, re.M)))


def test_header_declarations_match_binding():
    assert _declared() == _capi.declared_symbols()


def test_library_exports_every_declared_symbol():
    path = pf.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T ((?:pfft|pwt)_\w+)$", out, re.M))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    lib = _capi.lib()
    for s in _declared():
        assert hasattr(lib, s)


@pytest.mark.parametrize("seed", range(25))
def test_hnf_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    d = 1 + seed % 4
    M = SI.random_regular_matrix(rng, d, 40, 10**7)
    assert pf.pfft_hermite_normal_form(M).tolist() == L.hnf(M)


@pytest.mark.parametrize("seed", range(25))
def test_smith_form_properties(seed):
    rng = np.random.default_rng(1000 + seed)
    d = 1 + seed % 4
    M = SI.random_regular_matrix(rng, d, 40, 10**7)
    Q, eps, R = pf.pfft_smith_normal_form(M)
    Q, R, eps = Q.tolist(), R.tolist(), [int(e) for e in eps]
    E = [[eps[i] if i == j else 0 for j in range(d)] for i in range(d)]
    assert L.matmul(L.matmul(Q, E), R) == [list(map(int, r)) for r in M]
    assert abs(L.det(Q)) == 1 and abs(L.det(R)) == 1
    assert all(eps[j + 1] % eps[j] == 0 for j in range(d - 1))
    assert eps == L.elementary_divisors(M)


def test_table1_cycles_from_library():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_cycles.txt")
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        i, *cycles = map(int, line.split())
        _, eps, _ = pf.pfft_smith_normal_form([[2048, i], [0, 2048]])
        assert [int(e) for e in eps if e > 1] == cycles


@pytest.mark.parametrize("M", [SI.M_SMALL_2D, SI.M_BATCHED_2D, SI.M_AUTOGRAD_3D, SI.M_WAVELET_2D])
def test_workload_boxes(M):
    H = pf.pfft_hermite_normal_form(M)
    G = pf.pfft_hermite_normal_form(np.asarray(M).T)
    assert np.prod(np.diag(H)) == np.prod(np.diag(G)) == abs(L.det(M))


def test_host_errors():
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_hermite_normal_form([[1, 2], [2, 4]])
    assert e.value.status == 2  # PFFT_ERR_SINGULAR
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_smith_normal_form([[1 << 25, 0], [0, 1]])
    assert e.value.status == 3  # PFFT_ERR_OVERFLOW
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_hermite_normal_form(np.eye(5, dtype=np.int64))
    assert e.value.status == 1  # PFFT_ERR_ARG


def test_noalloc_binding_needs_one_wavelet_pointer_per_level():
    """The C side reads wavelets[l] for every level: a short list is refused
    before the call."""
    with pytest.raises(ValueError):
        _capi.pwt_decompose_noalloc(SI.M_WAVELET_2D, SI.wavelet_dilations(3), pf.PWT_DIRICHLET, 0.125, 1,
                                    1, 2, [3, 4], 0)


def test_dense_large_entries_overflow_cleanly():
    """A dense 4 x 4 matrix with entries near the 2^24 cap has |det| near 2^94
    and 3 x 3 minors near 2^70: the planner's exact determinant must report
    PFFT_ERR_OVERFLOW, not a wrapped i128 value."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        M = rng.integers(-(1 << 24) + 1, 1 << 24, size=(4, 4))
        assert abs(L.det(M.tolist())) >= 1 << 63
        with pytest.raises(pf.PfftError) as e:
            pf.pfft_hermite_normal_form(M)
        assert e.value.status == 3  # PFFT_ERR_OVERFLOW


def test_large_entries_small_determinant_exact():
    """Entries near 2^22 whose products cancel down to |det M| = 3: the
    determinant and the Hermite form stay exact (oracle's Python integers)."""
    rng = np.random.default_rng(7)
    done = 0
    while done < 5:
        A = [[1 if i == j else (int(rng.integers(-2**11, 2**11)) if i > j else 0) for j in range(4)] for i in range(4)]
        B = [[1 if i == j else (int(rng.integers(-2**11, 2**11)) if i < j else 0) for j in range(4)] for i in range(4)]
        D = [[int(i == j) * (3 if i == 3 else 1) for j in range(4)] for i in range(4)]
        M = L.matmul(L.matmul(B, D), A)
        if max(abs(x) for r in M for x in r) >= 1 << 24:
            continue
        assert pf.pfft_hermite_normal_form(M).tolist() == L.hnf(M)
        done += 1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU path")
def test_plan_without_gpu_fails_loudly():
    with pytest.raises(pf.PfftError) as e:
        pf.PatternFFT(SI.M_SMALL_2D, 1)
    assert e.value.status == 7  # PFFT_ERR_CUDA: no CPU fallback
    with pytest.raises(pf.PfftError):
        pf.WaveletSplit(SI.M_WAVELET_2D, SI.wavelet_dilations(2))


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU path")
def test_batch_without_gpu_fails_loudly():
    with pytest.raises(pf.PfftError) as e:
        pf.PatternBatch([SI.M_SMALL_2D, [[4, 1], [0, 6]]])
    assert e.value.status == 7


def test_batch_argument_errors():
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_batch_create([2 * np.eye(5, dtype=np.int64)])
    assert e.value.status == 1  # d = 5
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_batch_create([[[2, 0], [0, 2]]], [[[2, 0], [0, 1]]], symbol=7)
    assert e.value.status == 1  # unknown symbol
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_batch_create([[[2, 0], [0, 2]]], [[[2, 0], [0, 1]]], symbol=pf.PWT_DLVP, eta=1.5)
    assert e.value.status == 1  # blend width outside (0, 1)
    with pytest.raises(ValueError):
        pf.pfft_batch_create([[[2, 0], [0, 2]]], [[[2, 0], [0, 1]], [[2, 0], [0, 1]]])


def test_general_split_host_errors():
    """Argument and lattice checks of the general split run on the host before
    anything is queued (the device pointers are never touched here)."""
    fake = 1 << 20  # never dereferenced: every call below fails on the host
    cases = [([[4, 0], [0, 4]], [[2, 0], [0, 2]], 5),    # G(J^T) = Z_2 x Z_2 is not cyclic
             ([[4, 0], [0, 4]], [[3, 0], [0, 1]], 4),    # J^{-1} M not integral
             ([[17, 0], [0, 2]], [[17, 0], [0, 1]], 5),  # p = 17 > 16
             ([[4, 0], [0, 4]], [[0, 0], [0, 1]], 2)]    # singular J
    for M, J, code in cases:
        with pytest.raises(pf.PfftError) as e:
            pf.pwt_split_general(M, J, 1, pf.PFFT_C64, fake, fake + 64, fake + 128, 0)
        assert e.value.status == code, (M, J)
    with pytest.raises(pf.PfftError) as e:
        pf.pwt_merge_general([[4, 0], [0, 4]], [[2, 0], [0, 1]], 1, pf.PFFT_C64, fake, fake, fake, 0)
    assert e.value.status == 1  # parts and c_hat must differ


@pytest.mark.parametrize("seed", range(6))
def test_parity_dilation_divides_pattern(seed):
    """The workload helper that picks a dilation for each pattern of the
    uneven mix: |det J| = 2 and J^{-1} M integral, for triangular and general
    matrices of even determinant; odd determinants are refused."""
    rng = np.random.default_rng(seed)
    for _ in range(40):
        d = int(rng.integers(1, 5))
        M = SI.random_regular_matrix(rng, d, 9, 1 << 16)
        if L.det(M) % 2:
            with pytest.raises(ValueError):
                SI.parity_dilation(M)
            continue
        J = SI.parity_dilation(M)
        assert abs(L.det(J)) == 2
        oracle.exact_N(M, J)  # raises unless J^{-1} M is integral


@pytest.mark.parametrize("seed", range(4))
def test_prime_dilation_divides_pattern(seed):
    """The dilation of any prime p dividing det M: |det J| = p and J^{-1} M
    integral; primes not dividing det M are refused."""
    rng = np.random.default_rng(100 + seed)
    for _ in range(30):
        d = int(rng.integers(1, 5))
        M = SI.random_regular_matrix(rng, d, 9, 1 << 16)
        D = abs(L.det(M))
        for p in (2, 3, 5, 7, 11, 13):
            if D % p:
                with pytest.raises(ValueError):
                    SI.prime_dilation(M, p)
                continue
            J = SI.prime_dilation(M, p)
            assert abs(L.det(J)) == p
            oracle.exact_N(M, J)


def test_mix_dilations_of_the_uneven_mix():
    """Every pattern of the uneven mix (drawn without the even filter) gets a
    dilation of determinant 2 or of the smallest odd prime of its
    determinant, with J^{-1} M integral."""
    w = SI.WORKLOADS["uneven_mix"]
    Ms = SI.uneven_mix(w["n_patterns"], seed=w["seed"], even_det=w["even_det"])
    odd = 0
    for M in Ms:
        D = abs(L.det(M))
        J = SI.mix_dilation(M)
        p = abs(L.det(J))
        assert p == SI.smallest_prime_factor(D)
        odd += p > 2
        if p > 2:
            assert D % 2 == 1
    assert odd > 0.15 * len(Ms)


def test_plan_argument_errors():
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_plan_create([[2, 1], [4, 2]], 1)
    assert e.value.status == 2
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_plan_create([[2, 0], [0, 2]], 0)
    assert e.value.status == 1
    with pytest.raises(pf.PfftError) as e:
        pf.pwt_plan_create([[3, 0], [0, 4]], [[[2, 0], [0, 1]]], 0, 0.0, 1)
    assert e.value.status == 4  # not integral (checked before the device)


def test_header_constants_match_binding():
    """Every PFFT_* / PWT_* enumerator of include/pfft.h has the same value in
    the ctypes binding (flags, dtypes, maps, symbols, batch flags)."""
    src = open(os.path.join(ROOT, "include", "pfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, val = (x.strip() for x in item.partition("="))
            nxt = int(val.rstrip("uU"), 0) if val else nxt
            consts[name] = nxt
            nxt += 1
    checked = 0
    for name, val in consts.items():
        if hasattr(_capi, name):
            assert getattr(_capi, name) == val, name
            checked += 1
    assert checked >= 15
    for name in ("PFFT_FLAG_TC_SPLIT", "PFFT_FLAG_LAYOUT_SNF", "PFFT_FLAG_AUTOTUNE", "PFFT_FLAG_TRANSPOSED",
                 "PFFT_BATCH_ONE_LAUNCH"):
        assert name in consts and hasattr(_capi, name)


def test_unknown_plan_flags_are_rejected_on_the_host():
    with pytest.raises(pf.PfftError) as e:
        pf.pfft_plan_create([[4, 0], [0, 4]], 1, flags=16)
    assert e.value.status == 1  # PFFT_ERR_ARG before any device work
    with pytest.raises(ValueError):
        pf.PatternFFT([[4, 0], [0, 4]], 1, route="sideways")
