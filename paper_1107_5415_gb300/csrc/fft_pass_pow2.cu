// Instantiation of the power-of-two shared-memory transform passes
// (fft_kernels.cuh); the register-resident ones are in fft_fast_f32.cu and
// fft_fast_f64.cu.
#include "fft_kernels.cuh"

namespace pfft {

int launch_fast_f32(const PassArgs& a, cudaStream_t s);
int launch_fast_f64(const PassArgs& a, cudaStream_t s);
int launch_tma(const PassArgs& a, int dtype, cudaStream_t s);

int launch_pass_pow2(const PassArgs& a, int dtype, cudaStream_t s) {
  if (a.tma && !a.cols) return launch_tma(a, dtype, s);
  if (a.fast) return dtype == 0 ? launch_fast_f32(a, s) : launch_fast_f64(a, s);
  if (dtype != 0) return launch_typed<double2, 16, true>(a, s);
  return a.ept == 16 ? launch_typed<float2, 16, true, 2>(a, s) : launch_typed<float2, 32, true>(a, s);
}

}  // namespace pfft
