// Instantiation of the bulk-copy staged row pass (fft_tma.cuh), with the
// compile-time specialised complex64 rows of 2^13 and 2^14 elements
// (fft_tma_ct.cuh) where they apply.
#include "fft_kernels.cuh"
#include "fft_tma.cuh"
#include "fft_tma_ct.cuh"
#include "fft_row_pipe.cuh"

namespace pfft {

template <typename C, int R>
static int launch_tma_t(const PassArgs& a, cudaStream_t s) {
  static const int ok = configure_kernel(reinterpret_cast<const void*>(row_tma_kernel<C, R>));
  if (ok != 0) return -1;
  dim3 grid(a.groups, a.batch), block(a.nthreads);
  row_tma_kernel<C, R><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LOGL>
static int launch_tma_ct(const PassArgs& a, cudaStream_t s) {
  static const int ok = configure_kernel(reinterpret_cast<const void*>(row_tma_ct_kernel<float2, LOGL>));
  if (ok != 0) return -1;
  dim3 grid(a.groups, a.batch), block((1 << LOGL) / 32);
  row_tma_ct_kernel<float2, LOGL><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

#ifndef PFFT_PIPE_X1S
#define PFFT_PIPE_X1S 1
#endif

template <bool FWD, bool DIRECT>
static int launch_pipe_t(const PassArgs& a, cudaStream_t s) {
  constexpr bool X1S = PFFT_PIPE_X1S != 0;
  static const int ok = configure_kernel(reinterpret_cast<const void*>(row_pipe_kernel<FWD, DIRECT, X1S>));
  if (ok != 0) return -1;
  const int total = a.LB * a.batch;
  dim3 grid(total < a.pipe_grid ? total : a.pipe_grid), block(1 << (kPipeLogL - 5));
  row_pipe_kernel<FWD, DIRECT, X1S><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The pipelined row pass serves the two-pass directions: forward (box ->
// workspace, no conjugation, unit scale) and inverse (workspace -> box,
// conjugated output, scaled).
static int launch_pipe(const PassArgs& a, cudaStream_t s) {
  if (a.load_mode == MAP_BOX_H && a.store_mode == MAP_WS && !a.conj_in && !a.conj_out && a.scale == 1.0)
    return (a.pipe_direct & 1) ? launch_pipe_t<true, true>(a, s) : launch_pipe_t<true, false>(a, s);
  if (a.load_mode == MAP_WS && a.store_mode == MAP_BOX_H && !a.conj_in && a.conj_out)
    return (a.pipe_direct & 2) ? launch_pipe_t<false, true>(a, s) : launch_pipe_t<false, false>(a, s);
  return -1;
}

int launch_tma(const PassArgs& a, int dtype, cudaStream_t s) {
  if (a.pipe && dtype == 0) return launch_pipe(a, s);
  if (dtype == 0 && a.T == 1 && a.nthreads == a.L / 32) {
    if (a.L == 1 << 14) return launch_tma_ct<14>(a, s);
    if (a.L == 1 << 13) return launch_tma_ct<13>(a, s);
  }
  return dtype == 0 ? launch_tma_t<float2, 32>(a, s) : launch_tma_t<double2, 16>(a, s);
}

}  // namespace pfft
