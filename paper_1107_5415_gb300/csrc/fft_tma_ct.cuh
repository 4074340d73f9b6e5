// Row pass with bulk-copy staging (fft_tma.cuh), specialised at compile time
// on the row length L = 2^LOGL (complex64, radix 32, one row per CTA of
// L / 32 threads).
//
// The staging, the bounded mbarrier waits and the bulk stores are those of
// row_tma_kernel; the stages run with compile-time spans (fast_pencil_ct with
// T = 1: row element j at j + floor(j / 32), the padding of fphys), and the
// workspace positions of a thread's elements mu = p + P k are walked
// arithmetically.  With the permutation
//     pos(mu) = ((mu mod 2^lg) << ls) | ((floor(mu / 2^lg) inv) mod 2^ls)
// and lg <= log2 P, mu mod 2^lg = p mod 2^lg for every k and
// floor(mu / 2^lg) = floor(p / 2^lg) + k P / 2^lg, so the staging address of
// element k is  hp + ((bp + k cstep) mod 2^ls)  with per-thread hp, bp
// (the block padding of the staging adds (p mod 2^lg) pad to hp).  Other
// permutations take col_pos per element.
#pragma once
#include <cuda_runtime.h>

#include "fft_fast_ct.cuh"
#include "fft_tma.cuh"

namespace pfft {

template <typename C, int LOGL>
__global__ void __launch_bounds__((1 << LOGL) / 32, (1 << 14) >> LOGL) row_tma_ct_kernel(PassArgs a) {
  constexpr int R = 32, L = 1 << LOGL, P = L / R, LP = LOGL - 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + a.bar_smem_off);
  C* stw = stage_table(sm, a);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)blockIdx.y * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)blockIdx.y * a.m;
  const int p = threadIdx.x;
  const int row = blockIdx.x;
  const int4* runs = reinterpret_cast<const int4*>(a.runs) + (size_t)row * a.nruns;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, uint32_t(L) * uint32_t(sizeof(C)));
  __syncthreads();
  const int nblk = a.stg_pad ? (1 << a.pi_lg) : 1;
  const int span = L / nblk;
  if (a.load_mode == MAP_BOX_H) {
    if (threadIdx.x < a.nruns) {
      const int4 r = __ldg(runs + threadIdx.x);
      if (r.z > 0) bulk_g2s(sm + r.x, in + r.y, uint32_t(r.z) * uint32_t(sizeof(C)), bar);
    }
  } else if (threadIdx.x < nblk) {
    const int c = threadIdx.x;
    bulk_g2s(sm + c * (span + a.stg_pad), in + (size_t)row * a.nD + c * span, uint32_t(span) * uint32_t(sizeof(C)),
             bar);
  }
  // staging addresses of workspace positions pos(p + P k)
  const bool ws_walk = a.pi_arith && a.pi_lg <= LP;
  int hp = 0, bp = 0, cstep = 0, m2 = 0;
  if (ws_walk) {
    const int lg = a.pi_lg, ls = a.pi_lspan;
    const int lo = p & ((1 << lg) - 1);
    hp = (lo << ls) + lo * a.stg_pad;
    bp = (p >> lg) * a.pi_inv;
    cstep = a.pi_inv << (LP - lg);
    m2 = (1 << ls) - 1;
  }
  auto ws_addr = [&](int k) {
    if (ws_walk) return hp + ((bp + k * cstep) & m2);
    const int pos = col_pos(a, p + P * k);
    return a.stg_pad ? pos + (pos >> a.pi_lspan) * a.stg_pad : pos;
  };
  if (!mbar_wait_bounded(bar, 0, a.spin_limit)) {
    if (threadIdx.x == 0) atomicExch(a.status, kStatusTimeout);
    mbar_wait_bounded(bar, 0);  // let this CTA's own copies land before leaving
    cp_async_wait_all();
    return;
  }
  C v[R];
  if (a.load_mode == MAP_BOX_H) {
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = sm[p + P * k];
  } else {
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = sm[ws_addr(k)];
  }
  if (a.conj_in) {
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = cconj(v[k]);
  }
  if (a.fs_na > 1 && a.load_mode == MAP_WS) {
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = cmul(v[k], fs_twiddle<C>(a, row, p + P * k));
  }
  cp_async_wait_all();
  __syncthreads();  // staging reads done: the exchange may overwrite it
  fast_pencil_ct<C, LOGL, 0>(v, sm, stw, a, p);
  using Rl = decltype(C::x);
  if (a.store_mode == MAP_WS) {
    if (a.fs_na > 1) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = cmul(v[k], fs_twiddle<C>(a, row, p + P * k));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) sm[ws_addr(k)] = v[k];
  } else {
    const Rl sx = Rl(a.scale), sy = a.conj_out ? -sx : sx;
#pragma unroll
    for (int k = 0; k < R; ++k) sm[p + P * k] = cmake<C>(v[k].x * sx, v[k].y * sy);
  }
  fence_async_smem();
  __syncthreads();
  if (a.store_mode == MAP_WS) {
    if (threadIdx.x < nblk) {
      const int c = threadIdx.x;
      bulk_s2g(out + (size_t)row * a.nD + c * span, sm + c * (span + a.stg_pad), uint32_t(span) * uint32_t(sizeof(C)));
      bulk_commit();
      bulk_wait_read_all();
    }
  } else if (threadIdx.x < a.nruns) {
    const int4 r = __ldg(runs + threadIdx.x);
    if (r.z > 0) {
      bulk_s2g(out + r.y, sm + r.x, uint32_t(r.z) * uint32_t(sizeof(C)));
      bulk_commit();
      bulk_wait_read_all();
    }
  }
}

}  // namespace pfft
