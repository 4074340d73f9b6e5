// Instantiation of the bulk-copy staged row pass (fft_tma.cuh).
#include "fft_kernels.cuh"
#include "fft_tma.cuh"

namespace pfft {

template <typename C, int R>
static int launch_tma_t(const PassArgs& a, cudaStream_t s) {
  static const int ok = configure_kernel(reinterpret_cast<const void*>(row_tma_kernel<C, R>));
  if (ok != 0) return -1;
  dim3 grid(a.groups, a.batch), block(a.nthreads);
  row_tma_kernel<C, R><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_tma(const PassArgs& a, int dtype, cudaStream_t s) {
  return dtype == 0 ? launch_tma_t<float2, 32>(a, s) : launch_tma_t<double2, 16>(a, s);
}

}  // namespace pfft
