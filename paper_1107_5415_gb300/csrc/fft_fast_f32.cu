// Instantiation of the register-resident power-of-two passes (float2).
#include "fft_fast.cuh"
#include "fft_fast2.cuh"
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

// Column pass over two pencil axes (fft_fast2.cuh).
template <int DIM>
static int launch_fast2(const PassArgs& a, cudaStream_t s) {
  static const int ok = configure_kernel(reinterpret_cast<const void*>(col_fast2_kernel<float2, 32, DIM>));
  if (ok != 0) return -1;
  dim3 grid(a.groups, a.batch), block(a.nthreads);
  col_fast2_kernel<float2, 32, DIM><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_fast_f32(const PassArgs& a, cudaStream_t s) {
  if (a.cols && a.nsub == 2)  // two axes without a four-step split: three cycles, d = 3
    return a.d == 3 ? launch_fast2<3>(a, s) : -1;
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
