// Grouped launches of a pattern batch: one launch runs the same pass for many
// patterns of different size.  Each CTA finds its pattern in a prefix table of
// first-CTA indices, copies that pattern's pass descriptor into shared memory
// and runs the generic (shared-memory Stockham) pass body of fft_kernels.cuh
// or the split butterfly of wavelet_kernels.cuh on its tile.
#include <cuda_runtime.h>

#include "batch.hpp"
#include "fft_kernels.cuh"
#include "wavelet_kernels.cuh"

namespace pfft {

// Largest k with cta0[k] <= b (cta0 ascending, cta0[0] = 0).
__device__ __forceinline__ int find_item(const int* __restrict__ cta0, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(cta0 + mid) <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ void copy_to_smem(T* dst, const T* src) {
  static_assert(sizeof(T) % 16 == 0, "descriptor size must be a multiple of 16 bytes");
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < int(sizeof(T) / 16); i += blockDim.x) d[i] = __ldg(s + i);
}

template <typename C, int EPT, bool COLS, int MINB>
__global__ void __launch_bounds__(kMaxThreads, MINB) grouped_pass_kernel(GroupArgs g) {
  __shared__ PassArgs a;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int it = find_item(g.cta0, g.n, blockIdx.x);
  copy_to_smem(&a, g.items + it);
  __syncthreads();
  if (threadIdx.x == 0) {
    a.in = static_cast<const char*>(g.base[a.in_sel]) + reinterpret_cast<uintptr_t>(a.in);
    a.out = static_cast<char*>(const_cast<void*>(g.base[a.out_sel])) + reinterpret_cast<uintptr_t>(a.out);
  }
  __syncthreads();
  const int tile = blockIdx.x - __ldg(g.cta0 + it);
  C* sm = reinterpret_cast<C*>(smem_raw);
  if constexpr (COLS) {
    if (a.pad)
      col_pass_body<C, EPT, false, true, false>(a, tile, 0, sm);
    else
      col_pass_body<C, EPT, false, false, false>(a, tile, 0, sm);
  } else {
    if (a.pad)
      row_pass_body<C, EPT, false, true, false>(a, tile, 0, sm);
    else
      row_pass_body<C, EPT, false, false, false>(a, tile, 0, sm);
  }
}

template <typename C>
__global__ void __launch_bounds__(kSplitThreads) grouped_split_kernel(const SplitItem* __restrict__ items,
                                                                      const int* __restrict__ cta0, int n,
                                                                      const C* __restrict__ chat,
                                                                      C* __restrict__ sc, C* __restrict__ wv) {
  __shared__ SplitItem it;
  const int k = find_item(cta0, n, blockIdx.x);
  copy_to_smem(&it, items + k);
  __syncthreads();
  const int g0 = (blockIdx.x - __ldg(cta0 + k)) * (kSplitThreads * kSplitPerThread) + threadIdx.x;
  const C* cin = chat + it.in_off;
  C* d1 = sc + it.sc_off;
  C* d2 = wv + it.wv_off;
#pragma unroll
  for (int f = 0; f < kSplitPerThread; ++f) {
    const int gs = g0 + f * kSplitThreads;
    if (gs >= it.L.mN) break;
    if (it.L.small)
      split_fibre<C, 0, true, true>(it.L, gs, 1, cin, nullptr, nullptr, nullptr, d1, d2);
    else
      split_fibre<C, 0, true, false>(it.L, gs, 1, cin, nullptr, nullptr, nullptr, d1, d2);
  }
}

template <typename C>
__global__ void __launch_bounds__(kSplitThreads) grouped_prime_kernel(const PrimeItem* __restrict__ items,
                                                                      const int* __restrict__ cta0, int n,
                                                                      const C* __restrict__ chat,
                                                                      C* __restrict__ sc, C* __restrict__ wv) {
  __shared__ PrimeItem it;
  const int k = find_item(cta0, n, blockIdx.x);
  copy_to_smem(&it, items + k);
  __syncthreads();
  const long long w = (long long)(blockIdx.x - __ldg(cta0 + k)) * kSplitThreads + threadIdx.x;
  const long long mN = it.P.mN;
  if (w >= mN * it.P.nch) return;
  const int ch = int(w / mN), gs = int(w - ch * mN);
  prime_split_item<C, 0>(it.P, gs, ch * kPrimeChunk, chat + it.in_off, nullptr, nullptr, nullptr,
                         sc + it.sc_off + gs, wv + it.wv_off + gs, mN);
}

namespace {
template <typename K>
int allow_smem(K* k) {
  // the static descriptor copy shares the 227 KB with the dynamic tile
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kGroupedMaxDynSmem) == cudaSuccess
             ? 0
             : -1;
}
}  // namespace

int prepare_grouped(int dtype) {
  if (dtype == 0) {
    static const int ok = allow_smem(grouped_pass_kernel<float2, kGroupedEptC64, false, 2>) |
                          allow_smem(grouped_pass_kernel<float2, kGroupedEptC64, true, 2>);
    return ok;
  }
  static const int ok = allow_smem(grouped_pass_kernel<double2, 16, false, 1>) |
                        allow_smem(grouped_pass_kernel<double2, 16, true, 1>);
  return ok;
}

int launch_grouped_pass(const GroupArgs& g, int cols, int dtype, int nctas, int threads, int smem,
                        cudaStream_t s) {
  if (nctas <= 0) return 0;
  if (smem > kGroupedMaxDynSmem || threads > kMaxThreads) return -1;
  if (dtype == 0) {
    if (cols)
      grouped_pass_kernel<float2, kGroupedEptC64, true, 2><<<nctas, threads, smem, s>>>(g);
    else
      grouped_pass_kernel<float2, kGroupedEptC64, false, 2><<<nctas, threads, smem, s>>>(g);
  } else {
    if (cols)
      grouped_pass_kernel<double2, 16, true, 1><<<nctas, threads, smem, s>>>(g);
    else
      grouped_pass_kernel<double2, 16, false, 1><<<nctas, threads, smem, s>>>(g);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_grouped_split(const SplitItem* items, const int* cta0, int n, int nctas, const void* chat, void* sc,
                         void* wv, int dtype, cudaStream_t s) {
  if (nctas <= 0) return 0;
  if (dtype == 0)
    grouped_split_kernel<float2><<<nctas, kSplitThreads, 0, s>>>(
        items, cta0, n, static_cast<const float2*>(chat), static_cast<float2*>(sc), static_cast<float2*>(wv));
  else
    grouped_split_kernel<double2><<<nctas, kSplitThreads, 0, s>>>(
        items, cta0, n, static_cast<const double2*>(chat), static_cast<double2*>(sc), static_cast<double2*>(wv));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pfft

namespace pfft {
int launch_grouped_prime_split(const PrimeItem* items, const int* cta0, int n, int nctas, const void* chat,
                               void* sc, void* wv, int dtype, cudaStream_t s) {
  if (nctas <= 0) return 0;
  if (dtype == 0)
    grouped_prime_kernel<float2><<<nctas, kSplitThreads, 0, s>>>(
        items, cta0, n, static_cast<const float2*>(chat), static_cast<float2*>(sc), static_cast<float2*>(wv));
  else
    grouped_prime_kernel<double2><<<nctas, kSplitThreads, 0, s>>>(
        items, cta0, n, static_cast<const double2*>(chat), static_cast<double2*>(sc), static_cast<double2*>(wv));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
}  // namespace pfft
