"""Host checks of the tcgen05 operand layout of the split-precision stages
(fft_tc.cuh), without a GPU: a small host program compiled from the header
prints the K-major offsets, the shared-memory and instruction descriptors and
the tensor-memory column counts, and the checks below hold them to the
layout the PTX ISA documents for tcgen05.mma (kind::f16, no swizzle):

* an 8 x 8 fp16 core matrix is 128 contiguous bytes, its rows 16 bytes
  apart;
* with the canonical K-major layout the core matrix of row group g and
  column group c starts at g * SBO + c * LBO (LBO: leading byte offset
  between core matrices adjacent along K; SBO: stride byte offset between
  8-row groups), and the offsets form a bijection onto the operand;
* the shared-memory descriptor holds start >> 4 in bits 0-13, LBO >> 4 in
  16-29, SBO >> 4 in 32-45 and the fixed value 1 in bits 46-48;
* the instruction descriptor of an fp32 accumulator with fp16 A and B,
  both K-major, holds D format 1 in bits 4-5, N >> 3 in bits 17-22 and
  M >> 4 in bits 24-28;
* every stage's 128-butterfly chunks fit the tensor-memory columns of the
  pass (2R fp32 columns per chunk) within 512 columns."""
import os
import subprocess

import pytest

from paper_1107_5415_gb300 import build_lib as B

PROG = r'''
#include <cstdio>
#include "fft_tc.cuh"
using namespace pfft;
int main() {
  for (int K : {32, 64}) {
    for (int r = 0; r < 128; ++r)
      for (int k = 0; k < K; ++k) std::printf("off %d %d %d %u\n", K, r, k, tc_kmajor_off(r, k, K));
    std::printf("chunk %d %d\n", K, tc_chunk_bytes(K / 2));
    std::printf("idesc %d %u\n", K, tc_instr_desc(128, K));
  }
  std::printf("sdesc %llu\n", (unsigned long long)tc_smem_desc(0x12340u, 128u, 1024u));
  for (int pts : {64, 96, 1024, 3200, 6144, 8192, 12288, 16384})
    std::printf("cols %d %d %d %d\n", pts, tc_tmem_cols(pts, true, false), tc_tmem_cols(pts, false, true),
                tc_tmem_cols(pts, true, true));
  return 0;
}
'''


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    d = tmp_path_factory.mktemp("tc")
    src, exe = d / "tc_dump.cu", d / "tc_dump"
    src.write_text(PROG)
    try:
        subprocess.run([B.nvcc(), "-std=c++17", "-I", B.CSRC, "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True,
                       capture_output=True, text=True, timeout=300)
    except (OSError, subprocess.CalledProcessError) as e:
        pytest.skip(f"no host build of the tcgen05 header: {e}")
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    rec = {"off": {}, "chunk": {}, "idesc": {}, "cols": {}}
    for line in out.splitlines():
        f = line.split()
        if f[0] == "off":
            rec["off"][(int(f[1]), int(f[2]), int(f[3]))] = int(f[4])
        elif f[0] in ("chunk", "idesc"):
            rec[f[0]][int(f[1])] = int(f[2])
        elif f[0] == "sdesc":
            rec["sdesc"] = int(f[1])
        elif f[0] == "cols":
            rec["cols"][int(f[1])] = tuple(int(x) for x in f[2:])
    return rec


@pytest.mark.parametrize("K", [32, 64])
def test_kmajor_layout_is_the_canonical_no_swizzle_layout(dump, K):
    off = {(r, k): v for (KK, r, k), v in dump["off"].items() if KK == K}
    lbo, sbo = 128, K * 16  # the values the stage passes to its descriptors
    seen = set()
    for (r, k), v in off.items():
        assert v % 2 == 0 and 0 <= v < 128 * K * 2
        # core matrix (r // 8, k // 8) at (r // 8) SBO + (k // 8) LBO; row r % 8 at 16 bytes, element k % 8 at 2
        assert v == (r // 8) * sbo + (k // 8) * lbo + (r % 8) * 16 + (k % 8) * 2
        seen.add(v // 2)
    assert len(seen) == 128 * K  # a bijection onto the operand's fp16 slots
    # each core matrix is 128 contiguous bytes
    for g in range(16):
        for c in range(K // 8):
            block = sorted(off[(8 * g + i, 8 * c + j)] for i in range(8) for j in range(8))
            assert block == list(range(block[0], block[0] + 128, 2))
    # the hi and lo halves of a 128-butterfly chunk (R = K / 2 points per butterfly)
    assert dump["chunk"][K] == 2 * 128 * K * 2


def test_shared_memory_descriptor_fields(dump):
    d = dump["sdesc"]
    assert d & 0x3FFF == 0x12340 >> 4
    assert (d >> 16) & 0x3FFF == 128 >> 4
    assert (d >> 32) & 0x3FFF == 1024 >> 4
    assert (d >> 46) & 0x7 == 1
    assert (d >> 49) & 0x7 == 0 and (d >> 52) & 1 == 0 and (d >> 61) & 0x7 == 0  # base offset 0, no swizzle


@pytest.mark.parametrize("K", [32, 64])
def test_instruction_descriptor_fields(dump, K):
    i = dump["idesc"][K]
    assert i & 0x3 == 0 and (i >> 2) & 1 == 0 and (i >> 3) & 1 == 0  # dense, no saturation
    assert (i >> 4) & 0x3 == 1  # fp32 accumulator
    assert (i >> 7) & 0x7 == 0 and (i >> 10) & 0x7 == 0  # A and B fp16
    assert (i >> 13) & 0x3 == 0 and (i >> 15) & 0x3 == 0  # no negation, both K-major
    assert (i >> 17) & 0x3F == K // 8  # N = 2R = K
    assert (i >> 24) & 0x1F == 128 // 16  # M = 128
    assert (i >> 30) & 0x3 == 0


def test_tensor_memory_columns_hold_every_chunk(dump):
    for pts, (c32, c16, both) in dump["cols"].items():
        for R, c in ((32, c32), (16, c16)):
            need = -(-(pts // R) // 128) * 2 * R  # chunks x 2R columns
            assert c >= need and c >= 32 and c & (c - 1) == 0 and c <= 512
        assert both == max(c32, c16)
