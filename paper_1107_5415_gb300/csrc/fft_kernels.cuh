// Transform kernel templates for sm_103a: the row pass and the column pass of the
// Kronecker factorisation in Smith coordinates (Theorem 1, eq. (KroneckerFFT)),
// each a batched Stockham autosort DFT held in shared memory, with the
// bit-exact gather / scatter between the Hermite boxes and the Smith
// coordinates fused into the global loads and stores.
#pragma once
#include <cuda_runtime.h>

#include "fft_plan.hpp"

namespace pfft {

// Shared-memory index with one padding element per 16, which keeps the
// stride-R writes of the first radix stages free of bank conflicts.
__device__ __forceinline__ int phys(int x) { return x + (x >> 4); }

// One Stockham stage of radix R over every pencil of the tile.  Element
// (pencil t, index i) lives at i*T + t (column pass, COLS) or t*L + i (row
// pass).  Butterfly j of the axis reads i = base + (j + r a/R) sigma and,
// after the twiddles exp(-2 pi i k r / (Ns R)) (k = j mod Ns) and the
// length-R DFT, writes i = base + ((j - k) R + k + r Ns) sigma.
template <typename C, int R, int NB, bool COLS>
__device__ __forceinline__ void run_stage(C* sm, const PassArgs& a, const StageDesc& s,
                                          const C* __restrict__ tw) {
  const int per_pencil = a.L / R;
  const int total = a.T * per_pencil;
  const int escale = COLS ? a.T : 1;
  C v[NB][R];
  int obase[NB];
  int ostep = s.Ns * s.sigma * escale;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    obase[q] = -1;
    if (b < total) {
      int t, rest;
      if (COLS) {
        rest = a.divT.div(b);
        t = b - rest * a.T;
      } else {
        t = b / per_pencil;
        rest = b - t * per_pencil;
      }
      const int o = s.div_aR.div(rest);
      const int j = rest - o * s.aR;
      const int hi = s.div_sigma.div(o);
      const int base = hi * s.a * s.sigma + (o - hi * s.sigma);
      const int k = j - s.div_Ns.div(j) * s.Ns;
      const int ebase = COLS ? base * a.T + t : t * a.L + base;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = sm[phys(ebase + (j + r * s.aR) * s.sigma * escale)];
      if (s.Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], tw[k * r * s.twstep]);
      }
      obase[q] = ebase + ((j - k) * R + k) * s.sigma * escale;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    if (obase[q] >= 0) {
      dft<C, R>(v[q], tw, a.nD);
#pragma unroll
      for (int r = 0; r < R; ++r) sm[phys(obase[q] + r * ostep)] = v[q][r];
    }
  }
  __syncthreads();
}

// The stages are grouped by radix in the fixed order of kRadixOrder (the
// planner sorts them so): the radices of one axis may run in any order in a
// Stockham DFT and different axes commute, and one loop per radix keeps the
// register allocation of each butterfly size separate (mixing sizes inside
// one loop body makes the allocator spill).  POW2 kernels carry only the
// power-of-two regions.
template <typename C, int EPT, bool COLS, bool POW2>
__device__ void run_all_stages(C* sm, const PassArgs& a, const C* __restrict__ tw) {
  int i = 0;
#define PFFT_REGION(RR, IDX)                                                     \
  _Pragma("unroll 1") for (int q = 0; q < a.cnt[IDX]; ++q, ++i)                  \
      run_stage<C, RR, (EPT / RR > 0 ? EPT / RR : 1), COLS>(sm, a, a.st[i], tw);
  PFFT_REGION(16, 0)
  PFFT_REGION(8, 1)
  PFFT_REGION(4, 2)
  PFFT_REGION(2, 3)
  if constexpr (!POW2) {
    PFFT_REGION(3, 4)
    PFFT_REGION(5, 5)
    PFFT_REGION(7, 6)
    PFFT_REGION(11, 7)
    PFFT_REGION(13, 8)
    PFFT_REGION(17, 9)
    PFFT_REGION(19, 10)
    PFFT_REGION(23, 11)
    PFFT_REGION(29, 12)
    PFFT_REGION(31, 13)
  }
#undef PFFT_REGION
}

template <typename C>
__device__ __forceinline__ C maybe_conj(C v, int c) {
  return c ? cconj(v) : v;
}

// Row pass: T rows of length nD per CTA, smem layout [t][e].
template <typename C, int EPT, bool POW2>
__global__ void __launch_bounds__(kMaxThreads, 1) row_pass_kernel(PassArgs a) {
  extern __shared__ unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)blockIdx.y * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)blockIdx.y * a.m;
  const int r0 = blockIdx.x * a.T;
  const int n = a.T * a.nD;
  const int d = a.d;

  for (int w = threadIdx.x; w < n; w += blockDim.x) {
    const int t = a.divnD.div(w);
    const int e = w - t * a.nD;
    const int row = r0 + t;
    if (row >= a.LB) continue;
    C v;
    int sidx;
    if (a.load_mode == MAP_BOX_H) {
      v = in[box_sum_slot(a.boxH, a.Atab + row * d, a.Btab + e * d)];
      sidx = e;
    } else if (a.load_mode == MAP_WS) {
      v = in[row * a.nD + e];
      sidx = a.PIinv[e];
    } else {
      v = in[box_sum_slot(a.boxG, a.Ctab + row * d, a.Etab + e * d)];
      sidx = a.PIinv[e];
    }
    sm[phys(t * a.nD + sidx)] = maybe_conj(v, a.conj_in);
  }
  __syncthreads();
  run_all_stages<C, EPT, false, POW2>(sm, a, tw);
  using Rl = decltype(C::x);
  const Rl sc = Rl(a.scale);
  for (int w = threadIdx.x; w < n; w += blockDim.x) {
    const int t = a.divnD.div(w);
    const int e = w - t * a.nD;
    const int row = r0 + t;
    if (row >= a.LB) continue;
    if (a.store_mode == MAP_WS) {
      out[row * a.nD + e] = sm[phys(t * a.nD + a.PIinv[e])];
    } else if (a.store_mode == MAP_BOX_H) {
      C v = maybe_conj(sm[phys(t * a.nD + e)], a.conj_out);
      out[box_sum_slot(a.boxH, a.Atab + row * d, a.Btab + e * d)] = cscale(v, sc);
    } else {
      C v = maybe_conj(sm[phys(t * a.nD + a.PIinv[e])], a.conj_out);
      out[box_sum_slot(a.boxG, a.Ctab + row * d, a.Etab + e * d)] = cscale(v, sc);
    }
  }
}

// Pencil-internal index of the sheared walk: unflatten j over the
// non-trivial cycles before the last one, add the per-thread offset, wrap.
__device__ __forceinline__ int shear_index(const PassArgs& a, int j, const int* off) {
  int c[kMaxSub];
#pragma unroll
  for (int s = kMaxSub - 1; s >= 0; --s) {
    if (s < a.nsub) {
      const int q = a.sub_div[s].div(j);
      c[s] = j - q * a.sub_n[s] + off[s];
      if (c[s] >= a.sub_n[s]) c[s] -= a.sub_n[s];
      j = q;
    }
  }
  int i = 0;
#pragma unroll
  for (int s = 0; s < kMaxSub; ++s)
    if (s < a.nsub) i = i * a.sub_n[s] + c[s];
  return i;
}

// Column pass: all LB rows of T adjacent workspace columns per CTA, smem
// layout [i][t].  The DFT runs over the (D-1) cycles inside the pencil.
template <typename C, int EPT, bool POW2>
__global__ void __launch_bounds__(kMaxThreads, 1) col_pass_kernel(PassArgs a) {
  extern __shared__ unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)blockIdx.y * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)blockIdx.y * a.m;
  const int p0 = blockIdx.x * a.T;
  const int n = a.T * a.LB;
  const int d = a.d;
  // blockDim.x is a multiple of T, so each thread keeps one column.
  const int tcol = a.divT.mod(threadIdx.x);
  int off[kMaxSub];
#pragma unroll
  for (int s = 0; s < kMaxSub; ++s)
    off[s] = (s < a.nsub) ? int((int64_t(tcol) * a.alpha[s]) % a.sub_n[s]) : 0;
  const int* etab = a.Etab + (p0 + tcol) * d;

  if (a.load_mode == MAP_WS) {
    for (int w = threadIdx.x; w < n; w += blockDim.x) {
      const int i = a.divT.div(w);
      sm[phys(i * a.T + tcol)] = maybe_conj(in[i * a.nD + p0 + tcol], a.conj_in);
    }
  } else {
    for (int w = threadIdx.x; w < n; w += blockDim.x) {
      const int i = shear_index(a, a.divT.div(w), off);
      C v = in[box_sum_slot(a.boxG, a.Ctab + i * d, etab)];
      sm[phys(i * a.T + tcol)] = maybe_conj(v, a.conj_in);
    }
  }
  __syncthreads();
  run_all_stages<C, EPT, true, POW2>(sm, a, tw);
  using Rl = decltype(C::x);
  const Rl sc = Rl(a.scale);
  if (a.store_mode == MAP_WS) {
    for (int w = threadIdx.x; w < n; w += blockDim.x) {
      const int i = a.divT.div(w);
      out[i * a.nD + p0 + tcol] = sm[phys(i * a.T + tcol)];
    }
  } else {
    for (int w = threadIdx.x; w < n; w += blockDim.x) {
      const int i = shear_index(a, a.divT.div(w), off);
      C v = maybe_conj(sm[phys(i * a.T + tcol)], a.conj_out);
      out[box_sum_slot(a.boxG, a.Ctab + i * d, etab)] = cscale(v, sc);
    }
  }
}

template <typename C, int EPT, bool POW2>
inline int launch_typed(const PassArgs& a, cudaStream_t s) {
  dim3 grid(a.groups, a.batch), block(a.nthreads);
  if (a.cols) {
    auto k = col_pass_kernel<C, EPT, POW2>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes) != cudaSuccess)
      return -1;
    k<<<grid, block, a.smem_bytes, s>>>(a);
  } else {
    auto k = row_pass_kernel<C, EPT, POW2>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes) != cudaSuccess)
      return -1;
    k<<<grid, block, a.smem_bytes, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}


}  // namespace pfft
