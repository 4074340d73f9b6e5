// Persistent, pipelined column pass for pencils of 2^10 complex64 points,
// eight columns per tile (the pencils of the other cycles in eq.
// (KroneckerFFT), here one cycle of length 1024).
//
// Two CTAs of 256 threads per SM walk the tiles g = blockIdx.x, + gridDim.x,
// ...; each keeps the next tile's copies in flight while it transforms the
// current one.  Thread (c, p), c < 8, p < 32, holds rows p + 32 k of column
// c (two radix-32 Stockham stages, as col_fast_ct_kernel).  Shared memory:
//
//   S (66 KiB)  the tile: filled with cp.async (16-byte pieces of the
//               workspace rows in the forward direction, the sheared gather
//               from the output box in the inverse one) in a dense
//               [row][column] layout, read into registers, then reused as
//               the padded exchange tile of the two stages; after the
//               exchange the copies of the next tile are issued into it;
//   X (32 KiB)  the sheared output of the forward direction, in two rounds
//               of 16 walk steps;
//   stw         the stage twiddles.
//
// Sheared output in two rounds.  The walk of thread (c, p) visits rows
// i_j = (i_0 + 32 j) mod 1024, i_0 = p + c alpha mod 1024, and stores row
// i_j of column c to consecutive output slots across the eight columns (the
// shear alpha).  Row i = 32 m + s is held by thread (c, s) in register m; at
// step j the walker (c, p) reads residue s = i_0 mod 32 and register
// (m_0 + j) mod 32, m_0 = floor(i_0 / 32).  Round h takes the steps
// j = 16 h + t, t < 16: the holder (c, s) writes its register r to X[t][s][c]
// when t = (r - m_0' - 16 h) mod 32 < 16, m_0' the m_0 of its walker, and the
// walker reads X[t][s][c] at step 16 h + t.  Word address 512 t + 16 s + 2 c
// puts the sixteen lanes of a half warp on distinct bank pairs whatever t
// each lane has, so X needs no padding.
#pragma once
#include <cuda_runtime.h>

#include "fft_fast_ct.cuh"

namespace pfft {

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}

// FWD: the forward column pass (workspace -> box, scaled); else the inverse
// (box -> workspace, conjugated input).
template <int DIM, bool FWD>
__global__ void __launch_bounds__(256, 2) col_pipe_kernel(PassArgs a) {
  using C = float2;
  constexpr int R = 32, LOGL = kCPipeLogL, L = 1 << LOGL, LOGT = 3, T = 1 << LOGT, P = L / R;
  constexpr int TS = DIM <= 2 ? 2 : 4;
  constexpr int NT = T * P;  // threads
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw);
  C* X = S + a.cpipe_x_off;
  const int tid = threadIdx.x;
  const int tcol = tid & (T - 1), p = tid >> LOGT;
  const int ntile = a.nD >> LOGT;
  const int total = ntile * a.batch;
  const C* __restrict__ in_all = static_cast<const C*>(a.in);
  C* __restrict__ out_all = static_cast<C*>(a.out);
  C* stw = stage_table(S, a);

  // the sheared walk of this thread: rows i0 + 32 j (mod L), box point step cP
  const int off = int((int64_t(tcol) * a.alpha[0]) % L);
  int i0 = p + off;
  if (i0 >= L) i0 -= L;

  auto issue = [&](int g) {
    const int b = g / ntile, p0 = (g - b * ntile) << LOGT;
    const C* in = in_all + (int64_t)b * a.m;
    if constexpr (FWD) {
#pragma unroll
      for (int i = 0; i < (L * T / 2) / NT; ++i) {  // 16-byte pieces, dense [row][column]
        const int c = tid + NT * i;
        const int row = c >> 2, part = c & 3;
        cp_async16(S + row * T + part * 2, in + (size_t)row * a.nD + p0 + part * 2);
      }
    } else {
      int z[4], et[4], cP[4];
      load_point<TS>(a.Etab, p0 + tcol, et);
      load_point<TS>(a.Ctab, i0, z);
      load_point<TS>(a.Ctab, P, cP);
      box_add_t<DIM>(a.boxG, z, et);
      int i = i0;
#pragma unroll 4
      for (int j = 0; j < R; ++j) {
        cp_async8(S + i * T + tcol, in + box_slot_t<DIM>(a.boxG, z));
        box_add_t<DIM>(a.boxG, z, cP);
        i += P;
        if (i >= L) i -= L;
      }
    }
  };

  if (blockIdx.x < total) issue(blockIdx.x);
  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();  // the tile (and, once, the stage table) has landed
    const int b = g / ntile, p0 = (g - b * ntile) << LOGT;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = S[(p + P * k) * T + tcol];
    if constexpr (!FWD) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = cconj(v[k]);
    }
    __syncthreads();  // dense reads done: S becomes the exchange tile
    // stage 0 (Ns = 1), exchange through the padded tile
    dft_pow2<C, R>(v);
    {
      C* wb = S + ct_phys<LOGT>(p * R) + tcol;
#pragma unroll
      for (int r = 0; r < R; ++r) wb[ct_phys<LOGT>(r)] = v[r];
    }
    __syncthreads();
    {
      const C* rb = S + ct_phys<LOGT>(p) + tcol;
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = rb[ct_phys<LOGT>(r * P)];
    }
    __syncthreads();  // S is free: the next tile may land in it
    if (g + gridDim.x < total) issue(g + gridDim.x);
    // stage 1 (Ns = 32): v[r] = frequency p + 32 r
    if (p) main_twiddle<C, R>(v, stw + a.stw_off[1] + p * 5);
    dft_pow2<C, R>(v);

    if constexpr (FWD) {
      // sheared store in two rounds of 16 walk steps through X
      const int pw = (p - off) & (P - 1);  // the walker of this thread's residue
      int i0w = pw + off;
      if (i0w >= L) i0w -= L;
      const int m0h = i0w >> 5;
      const int sw = i0 & (P - 1);
      int z[4], et[4], cP[4];
      load_point<TS>(a.Etab, p0 + tcol, et);
      load_point<TS>(a.Ctab, i0, z);
      load_point<TS>(a.Ctab, P, cP);
      box_add_t<DIM>(a.boxG, z, et);
      C* out = out_all + (int64_t)b * a.m;
      const float sc = float(a.scale);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h) __syncthreads();  // round 0's reads of X are done
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int t = (r - m0h - 16 * h) & 31;
          if (t < 16) X[(t * P + p) * T + tcol] = v[r];
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < 16; ++t) {
          const C x = X[(t * P + sw) * T + tcol];
          out[box_slot_t<DIM>(a.boxG, z)] = cmake<C>(x.x * sc, x.y * sc);
          box_add_t<DIM>(a.boxG, z, cP);
        }
      }
    } else {
      C* out = out_all + (int64_t)b * a.m + p0 + tcol;
#pragma unroll
      for (int k = 0; k < R; ++k) out[(size_t)(p + P * k) * a.nD] = v[k];
    }
  }
}

}  // namespace pfft
