// Grouped launches of a pattern batch: one launch runs the same pass for many
// patterns of different size.  Each CTA reads its pattern and tile from a
// per-CTA map stored after the launch's prefix table of first-CTA indices,
// copies that pattern's pass descriptor into shared memory and runs the
// generic (shared-memory Stockham) pass body of fft_kernels.cuh or the split
// butterfly of wavelet_kernels.cuh on its tile.  The single-launch queue
// kernel finds the pattern of a work unit by a search of its prefix table.
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

// Item k and tile t of CTA b (CTAs cta0[k] .. cta0[k+1]-1 run item k): the
// pair stored for b after the prefix table (n + 1 ints, padded to an even
// count), one load instead of a search.
__device__ __forceinline__ int2 cta_item(const int* __restrict__ cta0, int n, int b) {
  return __ldg(reinterpret_cast<const int2*>(cta0 + ((n + 2) & ~1)) + b);
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
  const int2 kt = cta_item(g.cta0, g.n, blockIdx.x);
  copy_to_smem(&a, g.items + kt.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    a.in = static_cast<const char*>(g.base[a.in_sel]) + reinterpret_cast<uintptr_t>(a.in);
    a.out = static_cast<char*>(const_cast<void*>(g.base[a.out_sel])) + reinterpret_cast<uintptr_t>(a.out);
  }
  __syncthreads();
  const int tile = kt.y;
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
  const int2 kt = cta_item(cta0, n, blockIdx.x);
  copy_to_smem(&it, items + kt.x);
  __syncthreads();
  const int g0 = kt.y * (kSplitThreads * kSplitPerThread) + threadIdx.x;
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
  const int2 kt = cta_item(cta0, n, blockIdx.x);
  copy_to_smem(&it, items + kt.x);
  __syncthreads();
  const long long w = (long long)kt.y * kSplitThreads + threadIdx.x;
  const long long mN = it.P.mN;
  if (w >= mN * it.P.nch) return;
  const int ch = int(w / mN), gs = int(w - ch * mN);
  prime_split_item<C, 0>(it.P, gs, ch * kPrimeChunk, chat + it.in_off, nullptr, nullptr, nullptr,
                         sc + it.sc_off + gs, wv + it.wv_off + gs, mN);
}

// Bounded wait (thread 0) until *done reaches need: spin_limit tries and about
// one second of the global timer, or the abort flag.  Returns 1 when ready.
__device__ __forceinline__ int queue_wait(const int* done, int need, const int* abort_flag, unsigned limit) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (unsigned i = 0;; ++i) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(done) : "memory");
    if (v >= need) return 1;
    if (i >= limit || *reinterpret_cast<const volatile int*>(abort_flag)) return 0;
    if ((i & 63) == 63) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) return 0;
    }
    __nanosleep(128);
  }
}

// The units of the single-launch queue.
template <typename C, int EPT>
__device__ __forceinline__ void queue_row(const PassArgs& a, int tile, C* sm) {
  if (a.pad)
    row_pass_body<C, EPT, false, true, false>(a, tile, 0, sm);
  else
    row_pass_body<C, EPT, false, false, false>(a, tile, 0, sm);
}
// the workspace was written by other CTAs of the launch: coherent loads
template <typename C, int EPT>
__device__ __forceinline__ void queue_col(const PassArgs& a, int tile, C* sm) {
  if (a.pad)
    col_pass_body<C, EPT, false, true, false, true>(a, tile, 0, sm);
  else
    col_pass_body<C, EPT, false, false, false, true>(a, tile, 0, sm);
}
template <typename C>
__device__ __noinline__ void queue_split(const SplitItem& si, int local, const QueueArgs& g) {
  const C* cin = static_cast<const C*>(g.base[2]) + si.in_off;
  C* d1 = static_cast<C*>(g.sc) + si.sc_off;
  C* d2 = static_cast<C*>(g.wv) + si.wv_off;
  const int g0 = local * kQueueSplitFibres + threadIdx.x;
  for (int f = 0; f < kSplitPerThread; ++f) {
    const int gs = g0 + f * kMaxThreads;
    if (gs >= si.L.mN || threadIdx.x >= kMaxThreads) break;
    if (si.L.small)
      split_fibre<C, 0, true, true, true>(si.L, gs, 1, cin, nullptr, nullptr, nullptr, d1, d2);
    else
      split_fibre<C, 0, true, false, true>(si.L, gs, 1, cin, nullptr, nullptr, nullptr, d1, d2);
  }
}
template <typename C>
__device__ __noinline__ void queue_prime(const PrimeItem& pi, int local, const QueueArgs& g) {
  const long long w = (long long)local * kMaxThreads + threadIdx.x;
  const long long mN = pi.P.mN;
  if (w >= mN * pi.P.nch) return;
  const int ch = int(w / mN), gs = int(w - ch * mN);
  prime_split_item<C, 0, true>(pi.P, gs, ch * kPrimeChunk, static_cast<const C*>(g.base[2]) + pi.in_off, nullptr,
                               nullptr, nullptr, static_cast<C*>(g.sc) + pi.sc_off + gs,
                               static_cast<C*>(g.wv) + pi.wv_off + gs, mN);
}

// One unit of the launch: find its item, wait (bounded) for its dependency,
// run it and, for a pass tile, count it done.
template <typename C, int EPT>
__device__ __forceinline__ void queue_unit(const QueueArgs& g, int u, C* sm) {
  __shared__ PassArgs it_a;
  __shared__ SplitItem it_s;
  __shared__ PrimeItem it_p;
  __shared__ int s_ok;
  int* const abort_flag = g.counters + 1;
  int* const rows_done = g.counters + 2;
  int* const cols_done = rows_done + g.npat;
  const int U1 = g.u_rows, U2 = U1 + g.u_cols, U3 = U2 + g.u_splits;
  // the unit's item, its pattern and its dependency
  int k, local, pat;
  const int* done = nullptr;
  int need = 0;
  if (u < U1) {
    k = find_item(g.row_u0, g.nrow, u);
    local = u - __ldg(g.row_u0 + k);
    pat = __ldg(g.row_pat + k);
  } else if (u < U2) {
    k = find_item(g.col_u0, g.ncol, u - U1);
    local = u - U1 - __ldg(g.col_u0 + k);
    pat = __ldg(g.col_pat + k);
    done = rows_done + pat;
    need = __ldg(g.need_rows + pat);
  } else {
    if (u < U3) {
      k = find_item(g.split_u0, g.nsplit, u - U2);
      local = u - U2 - __ldg(g.split_u0 + k);
      pat = __ldg(g.split_pat + k);
    } else {
      k = find_item(g.prime_u0, g.nprime, u - U3);
      local = u - U3 - __ldg(g.prime_u0 + k);
      pat = __ldg(g.prime_pat + k);
    }
    const int nc = __ldg(g.need_cols + pat);
    done = nc ? cols_done + pat : rows_done + pat;
    need = nc ? nc : __ldg(g.need_rows + pat);
  }
  if (threadIdx.x == 0) {
    int ok = 1;
    if (done && !queue_wait(done, need, abort_flag, g.spin_limit)) {
      ok = 0;
      atomicExch(g.status, 8);  // PFFT_ERR_TIMEOUT
      atomicExch(abort_flag, 1);
    }
    s_ok = ok;
  }
  // the descriptor of the unit's item
  if (u < U1)
    copy_to_smem(&it_a, g.rows + k);
  else if (u < U2)
    copy_to_smem(&it_a, g.cols + k);
  else if (u < U3)
    copy_to_smem(&it_s, g.splits + k);
  else
    copy_to_smem(&it_p, g.primes + k);
  __syncthreads();
  if (!s_ok) return;  // block-uniform
  if (u < U2) {
    if (threadIdx.x == 0) {
      it_a.in = static_cast<const char*>(g.base[it_a.in_sel]) + reinterpret_cast<uintptr_t>(it_a.in);
      it_a.out = static_cast<char*>(const_cast<void*>(g.base[it_a.out_sel])) + reinterpret_cast<uintptr_t>(it_a.out);
    }
    __syncthreads();
    if (u < U1)
      queue_row<C, EPT>(it_a, local, sm);
    else
      queue_col<C, EPT>(it_a, local, sm);
    __syncthreads();  // every output of the tile is written
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd((u < U1 ? rows_done : cols_done) + pat, 1);
    }
  } else if (u < U3) {
    queue_split<C>(it_s, local, g);
  } else {
    queue_prime<C>(it_p, local, g);
  }
}

// The whole batch in one launch: each CTA takes the next unit of the queue
// (in the order the CTAs start, so a unit's dependencies are held by CTAs
// that started earlier and run to completion).  One unit per CTA: a loop of
// units around the generic pass bodies made the compiler keep their per-thread
// values live across iterations (kilobytes of spills per thread).
template <typename C, int EPT, int MINB>
__global__ void __launch_bounds__(kMaxThreads, MINB) batch_queue_kernel(QueueArgs g) {
  __shared__ int s_unit;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  if (threadIdx.x == 0) s_unit = atomicAdd(g.counters, 1);
  __syncthreads();
  const int u = s_unit;
  if (u >= g.u_rows + g.u_cols + g.u_splits + g.u_primes) return;
  if (*reinterpret_cast<volatile int*>(g.counters + 1)) return;  // aborted after a timed-out wait
  queue_unit<C, EPT>(g, u, reinterpret_cast<C*>(sm));
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

namespace pfft {
int prepare_queue(int dtype) {
  if (dtype == 0) {
    static const int ok = allow_smem(batch_queue_kernel<float2, kGroupedEptC64, 2>);
    return ok;
  }
  static const int ok = allow_smem(batch_queue_kernel<double2, 16, 1>);
  return ok;
}

int launch_batch_queue(const QueueArgs& g, int dtype, int nunits, int smem, cudaStream_t s) {
  if (nunits <= 0) return 0;
  if (smem > kGroupedMaxDynSmem) return -1;
  if (dtype == 0)
    batch_queue_kernel<float2, kGroupedEptC64, 2><<<nunits, kMaxThreads, smem, s>>>(g);
  else
    batch_queue_kernel<double2, 16, 1><<<nunits, kMaxThreads, smem, s>>>(g);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
}  // namespace pfft
