// Row pass with bulk-copy (TMA) staging, for power-of-two rows held by one CTA.
//
// The input row is a union of runs: element ranges of the Smith coordinate
// lambda_D whose box slots are consecutive (the planner finds them exactly,
// per row, and uses this kernel only when every run starts and ends on a
// 16-byte boundary).  A few threads issue one cp.async.bulk per run into a
// dense shared staging buffer, completing on an mbarrier; the workspace side
// of the pass is a single contiguous bulk copy.  Threads then take their
// elements p + P k from shared memory, run the register-resident stages of
// fft_fast.cuh, write their outputs back to the staging buffer (in workspace
// position order, or element order for the box scatter) and a bulk store
// sends the row out.  No thread computes a global address per element.
//
// Every wait on the mbarrier is bounded; on timeout the kernel records
// PFFT_ERR_TIMEOUT in the plan's device status word, waits (bounded) for its
// own copies and returns.
#pragma once
#include <cuda_runtime.h>

#include "fft_fast.cuh"

namespace pfft {

constexpr int kStatusTimeout = 8;  // PFFT_ERR_TIMEOUT

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t limit = kSpinLimit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

template <typename C, int R>
__global__ void __launch_bounds__(kMaxThreads, 1) row_tma_kernel(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + a.bar_smem_off);
  C* stw = stage_table(sm, a);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)blockIdx.y * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)blockIdx.y * a.m;
  const int L = a.L;
  const int P = L / R;
  const int p = threadIdx.x;
  const int row = blockIdx.x;
  const int4* runs = reinterpret_cast<const int4*>(a.runs) + (size_t)row * a.nruns;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  // ---- stage the row in shared memory (dense, element or position order)
  if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, uint32_t(L) * uint32_t(sizeof(C)));
  __syncthreads();
  // workspace-order staging: block c of 2^pi_lg holds positions [c span, (c+1) span)
  const int nblk = a.stg_pad ? (1 << a.pi_lg) : 1;
  const int span = L / nblk;
  auto spos = [&](int pos) { return a.stg_pad ? pos + (pos >> a.pi_lspan) * a.stg_pad : pos; };
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
    for (int k = 0; k < R; ++k) v[k] = sm[spos(col_pos(a, p + P * k))];
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
  fast_pencil_dft<C, R, false>(v, sm, stw, a, p, 0, 1, L);
  // ---- write the row back through the staging buffer
  using Rl = decltype(C::x);
  if (a.store_mode == MAP_WS) {
    if (a.fs_na > 1) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = cmul(v[k], fs_twiddle<C>(a, row, p + P * k));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) sm[spos(col_pos(a, p + P * k))] = v[k];
  } else {
    const Rl sc = Rl(a.scale);
#pragma unroll
    for (int k = 0; k < R; ++k) sm[p + P * k] = cscale(a.conj_out ? cconj(v[k]) : v[k], sc);
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
