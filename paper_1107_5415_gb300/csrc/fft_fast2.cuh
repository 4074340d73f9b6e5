// Register-resident column pass over two pencil axes (complex64).
//
// The pencil of a column holds the rows r = i0 n1 + i1 of two cycles of
// lengths n0 x n1 (powers of two; i0 the slower axis), and the pass computes
// their 2-D DFT (eq. (KroneckerFFT): one DFT per cycle).  It runs as the 1-D
// Stockham DFT of length L = n0 n1 of fast_pencil_dft (tail stage, then
// radix-32 stages) with two changes, both in the plan's stage tables and the
// output indexing rather than in the butterflies:
//
//   * the planner orders the axes so that the first stages' radices
//     multiply to n0; those stages then transform i0 alone, and from span
//     Ns = n0 on the stage table holds, for k < Ns, the twiddle of floor(k /
//     n0) at span Ns / n0, which removes exactly the factors that couple the
//     two axes in the 1-D algorithm;
//   * the DFT leaves frequency (f0, f1) at position f0 + n0 f1, which the
//     pass writes to row f0 n1 + f1.
//
// Loads and stores are those of col_fast_kernel: workspace rows coalesced
// across the T columns of the tile, box rows in a sheared walk through shared
// memory, here with one shear per axis (shear_index).
#pragma once
#include <cuda_runtime.h>

#include "fft_fast.cuh"
#include "fft_kernels.cuh"

namespace pfft {

template <typename C, int R, int DIM>
__global__ void __launch_bounds__(kMaxThreads, 1) col_fast2_kernel(PassArgs a) {
  constexpr int TS = DIM <= 2 ? 2 : 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* stw = stage_table(sm, a);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)blockIdx.y * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)blockIdx.y * a.m;
  const int T = a.T;
  const int P = a.L / R;
  const int tcol = threadIdx.x & (T - 1);
  const int p = threadIdx.x >> a.logT;
  const int p0 = blockIdx.x * T;
  const int LB = a.LB;
  const int nthr = blockDim.x;
  const int n0 = a.sub_n[0];
  int l0 = 0, l1 = 0;
  while ((1 << l0) < n0) ++l0;
  while ((1 << l1) < a.sub_n[1]) ++l1;
  // row of the DFT output at position f0 + n0 f1
  auto row_of = [&](int pos) { return ((pos & (n0 - 1)) << l1) | (pos >> l0); };
  int et[4], ct[4];
  load_point<TS>(a.Etab, p0 + tcol, et);
  // the sheared walk of column tcol: axis offsets tcol * alpha_s mod n_s
  int off[kMaxSub];
#pragma unroll
  for (int s = 0; s < kMaxSub; ++s)
    off[s] = (s < a.nsub) ? int((int64_t(tcol) * a.alpha[s]) % a.sub_n[s]) : 0;
  C v[R];
  if (a.load_mode == MAP_WS) {
    const C* src = in + p0 + tcol;
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = __ldg(src + (p + P * k) * a.nD);
    if (a.conj_in) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = cconj(v[k]);
    }
    cp_async_wait_all();
    __syncthreads();
  } else {
#pragma unroll 4
    for (int w = threadIdx.x; w < LB * T; w += nthr) {
      const int i = shear_index(a, w >> a.logT, off);
      load_point<TS>(a.Ctab, i, ct);
      C x = __ldg(in + box_sum_slot_t<DIM>(a.boxG, ct, et));
      sm[fphys(i * T + tcol)] = a.conj_in ? cconj(x) : x;
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = sm[fphys((p + P * k) * T + tcol)];
    __syncthreads();
  }
  fast_pencil_dft<C, R, true>(v, sm, stw, a, p, tcol, T, a.L);
  using Rl = decltype(C::x);
  const Rl sc = Rl(a.scale);
  if (a.store_mode == MAP_WS) {
    C* dst = out + p0 + tcol;
#pragma unroll
    for (int k = 0; k < R; ++k) dst[row_of(p + P * k) * a.nD] = v[k];
  } else {
    __syncthreads();  // the last stage's shared-memory reads are done
#pragma unroll
    for (int k = 0; k < R; ++k) sm[fphys(row_of(p + P * k) * T + tcol)] = v[k];
    __syncthreads();
#pragma unroll 4
    for (int w = threadIdx.x; w < LB * T; w += nthr) {
      const int i = shear_index(a, w >> a.logT, off);
      C x = sm[fphys(i * T + tcol)];
      if (a.conj_out) x = cconj(x);
      load_point<TS>(a.Ctab, i, ct);
      out[box_sum_slot_t<DIM>(a.boxG, ct, et)] = cscale(x, sc);
    }
  }
}

}  // namespace pfft
