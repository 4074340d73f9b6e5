// Split-precision tensor-core stages of radix 16 and 32 (complex64 only).
//
// A Stockham stage of radix R is, per butterfly, the dense product
// y = F x' with F[s][r] = omega_R^{s r} and x' the twiddled inputs.  In real
// arithmetic this is the 2R x 2R matrix [[Fr, -Fi], [Fi, Fr]] applied to
// [Re x'; Im x'], and the butterflies of a tile are its columns: a GEMM with
// M = K = 2R and N = the butterflies, run with mma.sync m16n8k16 (one warp,
// eight butterflies per N-tile).  Both operands are split into fp16 halves,
// a = a_hi + a_lo with a_hi = fp16(a) and a_lo = fp16(a - a_hi), and the
// product is accumulated in fp32 as a_hi b_hi + a_hi b_lo + a_lo b_hi, which
// keeps about 22 significant bits (the dropped a_lo b_lo term is below the
// fp32 rounding of the sums).  Each butterfly is scaled by a power of two
// before the split so that its largest input lies in [2^10, 2^11) (the four
// lanes holding its inputs agree on the factor through two shuffles), and its
// outputs are scaled back after the accumulation: both steps are exact in
// fp32, so the fp16 halves neither overflow nor fall into the subnormal range
// for data of any magnitude from 2^-116 up to the fp32 range.
//
// The A operand (the DFT matrix) is the same for every butterfly: each CTA
// writes its fragments, hi and lo, to shared memory once, in the register
// order of the m16n8k16 A fragment, so that a lane fetches its four
// registers of a tile with one 16-byte load.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fft_plan.hpp"

namespace pfft {

template <int R>
__host__ __device__ constexpr int tc_tiles() {
  return (2 * R / 16) * (2 * R / 16);
}
// 32-bit words of the hi and lo fragment tables of radix R
template <int R>
__host__ __device__ constexpr int tc_words() {
  return 2 * tc_tiles<R>() * 32 * 4;
}

// Two fp32 values -> packed fp16 pairs (hi, lo); the first value in the low half.
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
  const __half l0 = __float2half_rn(x0 - __half2float(h0));
  const __half l1 = __float2half_rn(x1 - __half2float(h1));
  hi = uint32_t(__half_as_ushort(h0)) | (uint32_t(__half_as_ushort(h1)) << 16);
  lo = uint32_t(__half_as_ushort(l0)) | (uint32_t(__half_as_ushort(l1)) << 16);
}

__device__ __forceinline__ void mma_f16_16816(float* d, const uint4& a, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// Fragment tables of the real DFT matrix of radix R: words [hl][tile][lane][4]
// (hl = 0: hi, 1: lo; tile = mt * KT + kt).  Register q of lane (g, t) of a
// tile holds rows 16 mt + g (+8 if q odd) and columns 16 kt + 2t, +1 (+8 if q >= 2).
template <int R>
__device__ void tc_build_tables(uint32_t* tab, const float2* __restrict__ tw, int tw_n) {
  constexpr int KT = 2 * R / 16;
  constexpr int n = tc_tiles<R>() * 32 * 4;
  const int wstride = tw_n / R;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int tile = e >> 7, lane = (e >> 2) & 31, reg = e & 3;
    const int mt = tile / KT, kt = tile - (tile / KT) * KT;
    const int g = lane >> 2, t = lane & 3;
    const int row = 16 * mt + g + ((reg & 1) ? 8 : 0);
    const int col = 16 * kt + 2 * t + ((reg & 2) ? 8 : 0);
    float v[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = col + c;
      const int s = row % R, r = cc % R;
      const float2 f = __ldg(tw + ((s * r) % R) * wstride);  // omega_R^{s r} = Fr + i Fi
      const bool yi = row >= R, xi = cc >= R;
      v[c] = (yi == xi) ? f.x : (xi ? -f.y : f.y);
    }
    uint32_t hi, lo;
    split_h2(v[0], v[1], hi, lo);
    tab[e] = hi;
    tab[n + e] = lo;
  }
}

// One Stockham stage of radix R (16 or 32) on the tensor cores; the same
// index walk as run_stage (fft_kernels.cuh).  Warp w takes the N-tiles
// (groups of eight consecutive butterflies) w, w + nwarps, ...; at most
// G = 128 / R per warp, which holds when the block has >= T L / 32 threads.
// All reads of the stage happen before the barrier, all writes after it.
template <int R, bool COLS, bool PAD>
__device__ __noinline__ void run_tc_stage(float2* sm, const PassArgs& a, const StageDesc& s,
                                          const float2* __restrict__ tw, const uint32_t* tab) {
  constexpr int MT = 2 * R / 16, KT = MT, HALF = MT / 2;
  constexpr int G = 128 / R;
  constexpr int NR = 2 * R / 8;  // inputs r of one butterfly held by a lane
  const int per_pencil = a.L / R;
  const int nbf = a.T * per_pencil;
  const int ngrp = (nbf + 7) >> 3;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int escale = COLS ? a.T : 1;
  const int step = s.sigma * escale;
  const int istep = s.aR * step;
  const uint4* ahi = reinterpret_cast<const uint4*>(tab);
  const uint4* alo = ahi + tc_tiles<R>() * 32;
  auto locate = [&](int b, int& ebase, int& k, int& j) {
    int tt, rest;
    if (COLS) {
      rest = a.divT.div(b);
      tt = b - rest * a.T;
    } else {
      tt = b / per_pencil;
      rest = b - tt * per_pencil;
    }
    const int o = s.div_aR.div(rest);
    j = rest - o * s.aR;
    const int hi = s.div_sigma.div(o);
    const int base = hi * s.a * s.sigma + (o - hi * s.sigma);
    k = j - s.div_Ns.div(j) * s.Ns;
    ebase = COLS ? base * a.T + tt : tt * a.L + base;
  };
  float acc[G][MT][4];
  int ex_of[G];
#pragma unroll
  for (int u = 0; u < G; ++u) {
    ex_of[u] = 0;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[u][mt][c] = 0.f;
    const int grp = warp + u * nw;
    if (grp >= ngrp) continue;  // warp-uniform
    float xr[NR], xi[NR];
    const int bf = grp * 8 + g;
    if (bf < nbf) {
      int ebase, k, j;
      locate(bf, ebase, k, j);
      const int i0 = ebase + j * step;
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const int r = (q >> 2) * 16 + 2 * t + (q & 1) + ((q & 2) ? 8 : 0);
        float2 x = sm[phys<PAD>(i0 + r * istep)];
        if (s.Ns > 1) x = cmul(x, __ldg(tw + (k * r) * s.twstep));  // k r < Ns R: no reduction
        xr[q] = x.x;
        xi[q] = x.y;
      }
    } else {
#pragma unroll
      for (int q = 0; q < NR; ++q) xr[q] = xi[q] = 0.f;
    }
    // power-of-two scale of this butterfly (lanes 4 g .. 4 g + 3 hold its inputs)
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < NR; ++q) mx = fmaxf(mx, fmaxf(fabsf(xr[q]), fabsf(xi[q])));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    int ex = mx > 0.f ? 10 - ilogbf(mx) : 0;
    ex = ex > 126 ? 126 : (ex < -126 ? -126 : ex);  // 2^ex and 2^-ex both normal
    ex_of[u] = ex;
    const float up = __int_as_float((127 + ex) << 23);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      xr[q] *= up;
      xi[q] *= up;
    }
    uint32_t bh[KT][2], bl[KT][2];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      const int qb = (kt % HALF) * 4;
      const float* src = kt < HALF ? xr : xi;
      split_h2(src[qb + 0], src[qb + 1], bh[kt][0], bl[kt][0]);
      split_h2(src[qb + 2], src[qb + 3], bh[kt][1], bl[kt][1]);
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        const uint4 ah = ahi[(mt * KT + kt) * 32 + lane];
        const uint4 al = alo[(mt * KT + kt) * 32 + lane];
        mma_f16_16816(acc[u][mt], ah, bh[kt][0], bh[kt][1]);
        mma_f16_16816(acc[u][mt], ah, bl[kt][0], bl[kt][1]);
        mma_f16_16816(acc[u][mt], al, bh[kt][0], bh[kt][1]);
      }
  }
  __syncthreads();
  const int ostep = s.Ns * step;
#pragma unroll
  for (int u = 0; u < G; ++u) {
    const int grp = warp + u * nw;
    if (grp >= ngrp) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {  // D columns 2t, 2t + 1
      const int bf = grp * 8 + 2 * t + c;
      // undo the scale of butterfly 2t + c (held by lane 4 (2t + c))
      const int ex = __shfl_sync(0xffffffffu, ex_of[u], (2 * t + c) * 4);
      const float down = __int_as_float((127 - ex) << 23);
      if (bf >= nbf) continue;
      int ebase, k, j;
      locate(bf, ebase, k, j);
      const int ob = ebase + ((j - k) * R + k) * step;
#pragma unroll
      for (int mt = 0; mt < HALF; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // D rows g, g + 8
          const int so = 16 * mt + g + 8 * h;
          sm[phys<PAD>(ob + so * ostep)] =
              make_float2(acc[u][mt][2 * h + c] * down, acc[u][mt + HALF][2 * h + c] * down);
        }
    }
  }
  __syncthreads();
}

}  // namespace pfft
