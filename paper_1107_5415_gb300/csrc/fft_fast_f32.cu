// Instantiation of the register-resident power-of-two passes (float2).
#include "fft_fast.cuh"
#include "fft_kernels.cuh"

namespace pfft {

int launch_col_ct_f32(const PassArgs& a, cudaStream_t s);  // fft_fast_ct.cu

template <int DIM, bool TC>
static int launch_dim(const PassArgs& a, cudaStream_t s) {
  static const int row_ok = configure_kernel(reinterpret_cast<const void*>(row_fast_kernel<float2, 32, DIM, TC>));
  static const int col_ok = configure_kernel(reinterpret_cast<const void*>(col_fast_kernel<float2, 32, DIM, TC>));
  if (row_ok != 0 || col_ok != 0) return -1;
  dim3 grid(a.groups, a.batch), block(a.nthreads);
  if (a.cols)
    col_fast_kernel<float2, 32, DIM, TC><<<grid, block, a.smem_bytes, s>>>(a);
  else
    row_fast_kernel<float2, 32, DIM, TC><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int DIM>
static int launch_dim(const PassArgs& a, cudaStream_t s) {
  return a.tc ? launch_dim<DIM, true>(a, s) : launch_dim<DIM, false>(a, s);
}

int launch_fast_f32(const PassArgs& a, cudaStream_t s) {
  if (a.cols && !a.tc) {
    const int rc = launch_col_ct_f32(a, s);
    if (rc != -2) return rc;
  }
  switch (a.d) {
    case 1: return launch_dim<1>(a, s);
    case 2: return launch_dim<2>(a, s);
    default: return launch_dim<3>(a, s);
  }
}

}  // namespace pfft
