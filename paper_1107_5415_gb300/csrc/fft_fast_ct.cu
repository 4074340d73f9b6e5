// Instantiations of the compile-time specialised column pass (complex64):
// pencil lengths L = 2^6 .. 2^13 with the planner's column count
// T = min(16, 8192 / L), for d = 2 and 3.
#include "fft_col_pipe.cuh"
#include "fft_fast_ct.cuh"
#include "fft_kernels.cuh"

namespace pfft {

template <int DIM, int LOGL, int LOGT>
static int launch_ct(const PassArgs& a, cudaStream_t s) {
  static const int ok = configure_kernel(reinterpret_cast<const void*>(col_fast_ct_kernel<float2, DIM, LOGL, LOGT>));
  if (ok != 0) return -1;
  dim3 grid(a.groups, a.batch), block(ct_threads<LOGL, LOGT>());
  col_fast_ct_kernel<float2, DIM, LOGL, LOGT><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int DIM>
static int launch_ct_dim(const PassArgs& a, cudaStream_t s) {
  switch (a.L) {
    case 1 << 6: return a.T == 16 ? launch_ct<DIM, 6, 4>(a, s) : -2;
    case 1 << 7: return a.T == 16 ? launch_ct<DIM, 7, 4>(a, s) : -2;
    case 1 << 8: return a.T == 16 ? launch_ct<DIM, 8, 4>(a, s) : -2;
    case 1 << 9: return a.T == 16 ? launch_ct<DIM, 9, 4>(a, s) : -2;
    case 1 << 10: return a.T == 8 ? launch_ct<DIM, 10, 3>(a, s) : -2;
    case 1 << 11: return a.T == 4 ? launch_ct<DIM, 11, 2>(a, s) : -2;
    case 1 << 12: return a.T == 2 ? launch_ct<DIM, 12, 1>(a, s) : -2;
    case 1 << 13: return a.T == 1 ? launch_ct<DIM, 13, 0>(a, s) : -2;
    default: return -2;
  }
}

template <int DIM, bool FWD>
static int launch_cpipe_t(const PassArgs& a, cudaStream_t s) {
  static const int ok = configure_kernel(reinterpret_cast<const void*>(col_pipe_kernel<DIM, FWD>));
  if (ok != 0) return -1;
  const int total = (a.nD / 8) * a.batch;
  dim3 grid(total < a.cpipe_grid ? total : a.cpipe_grid), block(256);
  col_pipe_kernel<DIM, FWD><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The pipelined column pass serves the two-pass directions: forward
// (workspace -> box, scaled) and inverse (box -> workspace, conjugated input).
static int launch_cpipe(const PassArgs& a, cudaStream_t s) {
  const bool fwd = a.load_mode == MAP_WS && a.store_mode == MAP_BOX_G && !a.conj_in && !a.conj_out;
  const bool inv = a.load_mode == MAP_BOX_G && a.store_mode == MAP_WS && a.conj_in && !a.conj_out && a.scale == 1.0;
  if (a.d == 2) return fwd ? launch_cpipe_t<2, true>(a, s) : inv ? launch_cpipe_t<2, false>(a, s) : -2;
  if (a.d == 3) return fwd ? launch_cpipe_t<3, true>(a, s) : inv ? launch_cpipe_t<3, false>(a, s) : -2;
  return -2;
}

// Launches the specialised column pass when one matches (L, T, d); returns
// -2 when none does, so that the caller runs the generic kernel.
int launch_col_ct_f32(const PassArgs& a, cudaStream_t s) {
  if (!a.cols || a.LB != a.L || a.nthreads != a.T * a.L / 32) return -2;
  if (a.cpipe) {
    const int rc = launch_cpipe(a, s);
    if (rc != -2) return rc;
  }
  switch (a.d) {
    case 2: return launch_ct_dim<2>(a, s);
    case 3: return launch_ct_dim<3>(a, s);
    default: return -2;
  }
}

}  // namespace pfft
