// Column pass of the register-resident power-of-two kernels, specialised at
// compile time on the pencil length L = 2^LOGL and the columns per CTA
// T = 2^LOGT (complex64, radix 32).
//
// Same computation as col_fast_kernel (fft_fast.cuh): thread (tcol, p) owns
// rows p + P k (k < 32, P = L / 32) of column tcol, runs the Stockham stages
// in registers with shared-memory exchanges between them, and the sheared
// box store (forward) or gather (inverse) goes through the shared tile in the
// walk i_j = (p + off + j P) mod L, off = tcol alpha mod L.  What changes is
// the index arithmetic:
//
//   * row i of column c of the tile sits at phys(i) + c with
//     phys(i) = (i + floor(i / 32)) T: one padding row after every 32 rows
//     (for T = 1 the padding of fphys).  Both the Stockham exchanges and the
//     sheared walk of a warp then hit every bank pair at most about twice,
//     where the element-wise padding of fphys left the walk up to four-way
//     conflicted for some shears.  Every row set a thread touches in the
//     stages is b + r D with (b mod 32) + (r D mod 32) < 32, so that
//     phys(b + r D) = phys(b) + phys(r D): a per-thread base and a constant
//     offset per unrolled r, with no per-element integer work (the walk too
//     when P >= 32);
//   * the box points of the walk advance by one box addition per element,
//     z_{j+1} = reduce(z_j + c_P) with c_P the box point of P g (g the
//     generator of the column cycle), instead of a table load and a sum per
//     element: i_j g + e advances by P g whatever the wrap of i_j.
#pragma once
#include <cuda_runtime.h>

#include "fft_fast.cuh"
#include "fft_plan.hpp"

namespace pfft {

template <int LOGT>
__host__ __device__ __forceinline__ constexpr int ct_phys(int i) {
  return (i + (i >> 5)) << LOGT;
}

// y <- reduce(y + c) for box points y, c of the box B (the reduction of
// box_sum_slot_t, keeping the point).
template <int DIM>
__device__ __forceinline__ void box_add_t(const BoxDesc& B, int* y, const int* c) {
  if constexpr (DIM == 2) {
    int y1 = y[1] + c[1];
    const int c1 = y1 >= B.H[1][1];
    y1 -= c1 * B.H[1][1];
    int y0 = y[0] + c[0] - c1 * B.H[0][1];
    y0 += (y0 < 0) * B.H[0][0];
    y0 -= (y0 >= B.H[0][0]) * B.H[0][0];
    y[0] = y0;
    y[1] = y1;
  } else {
    int y2 = y[2] + c[2];
    const int c2 = y2 >= B.H[2][2];
    y2 -= c2 * B.H[2][2];
    int y1 = y[1] + c[1] - c2 * B.H[1][2];
    int y0 = y[0] + c[0] - c2 * B.H[0][2];
    const int c1 = (y1 >= B.H[1][1]) - (y1 < 0);
    y1 -= c1 * B.H[1][1];
    y0 -= c1 * B.H[0][1];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      y0 += (y0 < 0) * B.H[0][0];
      y0 -= (y0 >= B.H[0][0]) * B.H[0][0];
    }
    y[0] = y0;
    y[1] = y1;
    y[2] = y2;
  }
}

template <int DIM>
__device__ __forceinline__ int box_slot_t(const BoxDesc& B, const int* y) {
  if constexpr (DIM == 2)
    return y[0] * B.stride[0] + y[1];
  else
    return y[0] * B.stride[0] + y[1] * B.stride[1] + y[2];
}

// All stages of one pencil (rows p + P k of column tcol) with compile-time
// spans; on entry v holds rows p + P k, on exit frequencies p + P k.
template <typename C, int LOGL, int LOGT>
__device__ __forceinline__ void fast_pencil_ct(C* v, C* smc, const C* stw, const PassArgs& a, int p) {
  constexpr int R = 32, LR = 5;
  constexpr int L = 1 << LOGL, P = L / R;
  constexpr int NMAIN = LOGL / LR, TAIL = 1 << (LOGL - NMAIN * LR);
  static_assert(NMAIN >= 1 && NMAIN <= 2, "pencil length out of the specialised range");
  if constexpr (TAIL > 1) {
    // tail stage (Ns = 1): butterfly q combines registers q + r NQ, writes rows (p + P q) TAIL + r
    constexpr int NQ = R / TAIL;
    C* wb = smc + ct_phys<LOGT>(p * TAIL);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      C u[TAIL];
#pragma unroll
      for (int r = 0; r < TAIL; ++r) u[r] = v[q + r * NQ];
      dft_pow2<C, TAIL>(u);
#pragma unroll
      for (int r = 0; r < TAIL; ++r) wb[ct_phys<LOGT>(q * P * TAIL + r)] = u[r];
    }
    __syncthreads();
  }
  const C* rb = smc + ct_phys<LOGT>(p);
#pragma unroll
  for (int s = 0; s < NMAIN; ++s) {
    const int Ns = TAIL << (LR * s);  // a constant once unrolled
    if (s > 0 || TAIL > 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = rb[ct_phys<LOGT>(r * P)];
      __syncthreads();
    }
    const int k = p & (Ns - 1);
    if (k) main_twiddle<C, R>(v, stw + a.stw_off[s] + k * LR);
    dft_pow2<C, R>(v);
    if (s + 1 < NMAIN) {
      C* wb = smc + ct_phys<LOGT>((p - k) * R + k);
#pragma unroll
      for (int r = 0; r < R; ++r) wb[ct_phys<LOGT>(r * Ns)] = v[r];
      __syncthreads();
    }
  }
}

template <int LOGL, int LOGT>
__host__ __device__ constexpr int ct_threads() {
  return (1 << (LOGL + LOGT)) / 32;
}

template <typename C, int DIM, int LOGL, int LOGT>
__global__ void __launch_bounds__(ct_threads<LOGL, LOGT>(), 512 / ct_threads<LOGL, LOGT>())
    col_fast_ct_kernel(PassArgs a) {
  constexpr int R = 32;
  constexpr int L = 1 << LOGL, T = 1 << LOGT, P = L / R;
  constexpr int TS = DIM <= 2 ? 2 : 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* stw = stage_table(sm, a);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)blockIdx.y * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)blockIdx.y * a.m;
  const int tcol = threadIdx.x & (T - 1);
  const int p = threadIdx.x >> LOGT;
  const int p0 = blockIdx.x * T;
  C* smc = sm + tcol;
  const bool walk_in = a.load_mode != MAP_WS, walk_out = a.store_mode != MAP_WS;
  // the sheared walk of this thread: rows i0 + j P (mod L), box points z_j of i_j g + e
  int i0 = 0, z[4] = {0, 0, 0, 0}, cP[4] = {0, 0, 0, 0};
  if (walk_in || walk_out) {
    int et[4], ct[4];
    load_point<TS>(a.Etab, p0 + tcol, et);
    const int off = int((int64_t(tcol) * a.alpha[0]) % L);
    i0 = p + off;
    if (i0 >= L) i0 -= L;
    load_point<TS>(a.Ctab, i0, ct);
    load_point<TS>(a.Ctab, P, cP);
#pragma unroll
    for (int r = 0; r < 4; ++r) z[r] = ct[r];
    box_add_t<DIM>(a.boxG, z, et);
  }
  // shared-memory position of walk row i0 + j P (mod L), column tcol
  constexpr int WRAP = ct_phys<LOGT>(L);
  auto walk_addr = [&](int j) {
    if constexpr (P >= 32) {
      return ct_phys<LOGT>(i0) + ct_phys<LOGT>(j * P) - (i0 + j * P >= L ? WRAP : 0);
    } else {
      const int i = i0 + j * P;
      return ct_phys<LOGT>(i >= L ? i - L : i);
    }
  };
  C v[R];
  if (!walk_in) {
    const C* src = in + p0 + tcol + p * a.nD;
    const int stride = P * a.nD;
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = __ldg(src + k * stride);
    if (a.conj_in) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = cconj(v[k]);
    }
    cp_async_wait_all();
    __syncthreads();
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      C x = __ldg(in + box_slot_t<DIM>(a.boxG, z));
      if (a.conj_in) x = cconj(x);
      smc[walk_addr(j)] = x;
      if (j + 1 < R) box_add_t<DIM>(a.boxG, z, cP);
    }
    cp_async_wait_all();
    __syncthreads();
    const C* rb = smc + ct_phys<LOGT>(p);
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = rb[ct_phys<LOGT>(k * P)];
    __syncthreads();
  }
  fast_pencil_ct<C, LOGL, LOGT>(v, smc, stw, a, p);
  if (!walk_out) {
    C* dst = out + p0 + tcol + p * a.nD;
    const int stride = P * a.nD;
#pragma unroll
    for (int k = 0; k < R; ++k) dst[k * stride] = v[k];
  } else {
    using Rl = decltype(C::x);
    const Rl sx = Rl(a.scale), sy = a.conj_out ? -sx : sx;
    __syncthreads();  // the last stage's shared-memory reads are done
    C* wb = smc + ct_phys<LOGT>(p);
#pragma unroll
    for (int k = 0; k < R; ++k) wb[ct_phys<LOGT>(k * P)] = v[k];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const C x = smc[walk_addr(j)];
      out[box_slot_t<DIM>(a.boxG, z)] = cmake<C>(x.x * sx, x.y * sy);
      if (j + 1 < R) box_add_t<DIM>(a.boxG, z, cP);
    }
  }
}

}  // namespace pfft
