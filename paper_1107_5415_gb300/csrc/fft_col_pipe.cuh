// Persistent, pipelined column pass for pencils of 2^10 complex64 points,
// eight columns per tile (the pencils of the other cycles in eq.
// (KroneckerFFT), here one cycle of length 1024).
//
// Two CTAs of 256 threads per SM walk the tiles g = blockIdx.x, + gridDim.x,
// ...; each keeps the next tile's copies in flight while it transforms the
// current one.  Thread (c, p), c < 8, p < 32, holds rows p + 32 k of column
// c (two radix-32 Stockham stages, as col_fast_ct_kernel).  Shared memory:
//
//   S (66 KiB)  the tile: forward, filled with cp.async in 16-byte pieces of
//               the workspace rows (dense [row][column]); inverse, the
//               sheared gather from the box in walk layout (8-byte pieces).
//               As soon as the threads have read it the copies of the next
//               tile are issued into it;
//   X (33 KiB)  the exchange between the two stages in two rounds of half a
//               tile, and (forward) the sheared output in two rounds;
//   Es          the column points of the walk (forward);
//   stw         the stage twiddles.
//
// Exchange in two rounds.  Stage 0 writes position 32 p + r, stage 1 reads
// p + 32 r' (10-bit positions per column).  Splitting by bit 9 xor bit 4
// makes thread p write and read the register half H = h xor bit 4 of p in
// round h (warp-uniform), and dropping bit 9 maps each round one-to-one onto
// 512 rows of the half tile.
//
// The inverse direction's gather leans on the L2: while it computes tile n
// it gathers tile n + 1 into S and prefetches into L2 the lines that tile
// n + 2 will gather (the start and the end of each row's run of 8 slots).
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

__device__ __forceinline__ void prefetch_l2(const void* gmem) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(gmem));
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}

// Exchange round with register half H (compile time): stage-0 outputs of
// positions 32 p + r and stage-1 inputs of positions p + 32 r, r in
// [16 H, 16 H + 16), at the 9-bit position (bit 9 dropped) in the padded
// half tile, one padding row per 32 rows.
template <int H>
__device__ __forceinline__ void cpipe_x_write(const float2* v, float2* X, int p, int tcol) {
  float2* wb = X + ct_phys<3>(32 * (p & 15)) + tcol;
#pragma unroll
  for (int i = 0; i < 16; ++i) wb[ct_phys<3>(16 * H + i)] = v[16 * H + i];
}
template <int H>
__device__ __forceinline__ void cpipe_x_read(float2* v, const float2* X, int p, int tcol) {
  const float2* rb = X + ct_phys<3>(p) + tcol;
#pragma unroll
  for (int i = 0; i < 16; ++i) v[16 * H + i] = rb[ct_phys<3>(32 * i)];
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

  // The sheared walk of thread (c, p) visits rows i0 + 32 j (mod L).  Row
  // p + 32 k of column c (register k of this thread) is visited by the walker
  // (c, pw), pw = (p - c alpha) mod 32, at step (k - m0h) mod 32, m0h =
  // floor(i_0 / 32) of that walker; this thread as a walker reads residue sw.
  const int off = int((int64_t(tcol) * a.alpha[0]) % L);
  int i0 = p + off;
  if (i0 >= L) i0 -= L;
  const int pw = (p - off) & (P - 1);
  int i0w = pw + off;
  if (i0w >= L) i0w -= L;
  const int m0h = i0w >> 5;
  const int sw = i0 & (P - 1);

  // The walk needs the box points of its start (a row of the column cycle,
  // times its generator; L1-resident table entries), of its step 32 g and
  // the point E(p0 + c) of its column.  The column points of a tile are
  // copied into Es (double-buffered by the parity of the CTA's tile count)
  // ahead of their use: with the tile's own copies (forward), one tile
  // earlier still (inverse, whose gather for tile n + 1 runs during tile n).
  int* Es = reinterpret_cast<int*>(S + a.cpipe_e_off);  // [2][T][TS]
  auto copy_points = [&](int g, int slot) {
    if (tid < T) {
      const int b = g / ntile, p0 = (g - b * ntile) << LOGT;
      if constexpr (TS == 2)
        cp_async8(Es + (slot * T + tid) * TS, a.Etab + (size_t)(p0 + tid) * TS);
      else
        cp_async16(Es + (slot * T + tid) * TS, a.Etab + (size_t)(p0 + tid) * TS);
    }
  };
  auto col_point = [&](int slot, int* et) {
#pragma unroll
    for (int r = 0; r < 4; ++r) et[r] = r < TS ? Es[(slot * T + tcol) * TS + r] : 0;
  };

  // forward: the workspace tile in 16-byte pieces, dense [row][column]
  auto issue_fwd = [&](int g, int n) {
    const int b = g / ntile, p0 = (g - b * ntile) << LOGT;
    const C* in = in_all + (int64_t)b * a.m;
#pragma unroll
    for (int i = 0; i < (L * T / 2) / NT; ++i) {
      const int c = tid + NT * i;
      const int row = c >> 2, part = c & 3;
      cp_async16(S + row * T + part * 2, in + (size_t)row * a.nD + p0 + part * 2);
    }
    copy_points(g, n & 1);
  };
  // inverse: walk steps [16 h, 16 h + 16) of the sheared gather, in walk
  // layout W[j][p][c] in S (word address 512 j + 16 p + 2 c: conflict free)
  auto issue_inv = [&](int g, int h, int n) {
    const int b = g / ntile;
    const C* in = in_all + (int64_t)b * a.m;
    int z[4], cP[4], et[4];
    col_point(n & 1, et);
    int ih = i0 + (h << (LOGL - 1));
    if (ih >= L) ih -= L;
    load_point<TS>(a.Ctab, ih, z);
    load_point<TS>(a.Ctab, P, cP);
    box_add_t<DIM>(a.boxG, z, et);
    C* dst = S + h * 16 * NT + p * T + tcol;
#pragma unroll 4
    for (int t = 0; t < 16; ++t) {
      cp_async8(dst + t * NT, in + box_slot_t<DIM>(a.boxG, z));
      box_add_t<DIM>(a.boxG, z, cP);
    }
  };

  // inverse: the rows of the column cycle whose runs the L2 prefetch visits
  // (the same for every tile)
  int pfp[FWD ? 1 : L / NT][4];
  if constexpr (!FWD) {
#pragma unroll
    for (int q = 0; q < L / NT; ++q) load_point<TS>(a.Ctab, tid + NT * q, pfp[q]);
  }

  if (blockIdx.x < total) {
    if constexpr (FWD) {
      issue_fwd(blockIdx.x, 0);
    } else {
      copy_points(blockIdx.x, 0);
      cp_async_wait_all();
      __syncthreads();
      issue_inv(blockIdx.x, 0, 0);
      issue_inv(blockIdx.x, 1, 0);
      if (blockIdx.x + gridDim.x < total) copy_points(blockIdx.x + gridDim.x, 1);
    }
  }
  int n = 0;  // this CTA's tile count
  for (int g = blockIdx.x; g < total; g += gridDim.x, ++n) {
    const int gn = g + gridDim.x;
    cp_async_wait_all();
    __syncthreads();  // the tile (and, once, the stage table) has landed
    const int b = g / ntile, p0 = (g - b * ntile) << LOGT;
    C v[R];
    if constexpr (FWD) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = S[(p + P * k) * T + tcol];
      __syncthreads();  // S is read: the next tile may land in it
      if (gn < total) issue_fwd(gn, n + 1);
    } else {
      // register k from walk step j = (k - m0h) mod 32 of walker pw (conjugated input)
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int j = (k - m0h) & (R - 1);
        v[k] = cconj(S[j * NT + pw * T + tcol]);
      }
      __syncthreads();  // S is read: the next tile's gather may land in it
      if (gn < total) {
        issue_inv(gn, 0, n + 1);
        issue_inv(gn, 1, n + 1);
        const int gnn = gn + gridDim.x;
        if (gnn < total) {
          copy_points(gnn, n & 1);  // for the gather after next
          // pull the lines of the gather after next into L2: row i of column
          // p0 starts a run of T consecutive slots (the shear), four rows per thread
          const int b2 = gnn / ntile, p2 = (gnn - b2 * ntile) << LOGT;
          const C* in2 = in_all + (int64_t)b2 * a.m;
          int e2[4];
          load_point<TS>(a.Etab, p2, e2);
#pragma unroll
          for (int q = 0; q < L / NT; ++q) {
            int y[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) y[r] = pfp[q][r];
            box_add_t<DIM>(a.boxG, y, e2);
            const int y0 = box_slot_t<DIM>(a.boxG, y);
            prefetch_l2(in2 + y0);
            prefetch_l2(in2 + min(y0 + T - 1, a.m - 1));  // the run's end, inside the signal
          }
        }
      }
    }
    // stage 0 (Ns = 1), exchange in two rounds through X: round h moves
    // register half H = h xor bit 4 of p (positions 32 p + r written,
    // p + 32 r' read, split by bit 9 xor bit 4 of the position; bit 9 dropped)
    dft_pow2<C, R>(v);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h) __syncthreads();  // round 0's reads of X are done
      if ((h ^ (p >> 4)) & 1)
        cpipe_x_write<1>(v, X, p, tcol);
      else
        cpipe_x_write<0>(v, X, p, tcol);
      __syncthreads();
      if ((h ^ (p >> 4)) & 1)
        cpipe_x_read<1>(v, X, p, tcol);
      else
        cpipe_x_read<0>(v, X, p, tcol);
    }
    // stage 1 (Ns = 32): v[r] = frequency p + 32 r
    if (p) main_twiddle<C, R>(v, stw + a.stw_off[1] + p * 5);
    dft_pow2<C, R>(v);

    if constexpr (FWD) {
      // sheared store in two rounds of 16 walk steps through X
      int z[4], cP[4], ec[4];
      load_point<TS>(a.Ctab, i0, z);
      load_point<TS>(a.Ctab, P, cP);
      col_point(n & 1, ec);
      box_add_t<DIM>(a.boxG, z, ec);
      C* out = out_all + (int64_t)b * a.m;
      const float sc = float(a.scale);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        __syncthreads();  // the previous reads of X are done
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int t = (r - m0h - 16 * h) & 31;
          if (t < 16) X[(t * P + p) * T + tcol] = v[r];
        }
        __syncthreads();
#pragma unroll 2
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
