// Dispatch of the power-of-two transform passes: the bulk-copy row pass
// (fft_tma.cu), the register-resident passes (fft_fast_f32.cu,
// fft_fast_f64.cu) and the shared-memory ones, instantiated per element type
// and width in fft_pass_pow2_*.cu so that they compile in parallel.
#include "fft_plan.hpp"

namespace pfft {

int launch_fast_f32(const PassArgs& a, cudaStream_t s);
int launch_fast_f64(const PassArgs& a, cudaStream_t s);
int launch_tma(const PassArgs& a, int dtype, cudaStream_t s);
int launch_pow2_c128(const PassArgs& a, cudaStream_t s);     // fft_pass_pow2_c128.cu
int launch_pow2_c64_e16(const PassArgs& a, cudaStream_t s);  // fft_pass_pow2_c64.cu
int launch_pow2_c64_e32(const PassArgs& a, cudaStream_t s);  // fft_pass_pow2_c64_e32.cu

int launch_pass_pow2(const PassArgs& a, int dtype, cudaStream_t s) {
  if (a.tma && !a.cols) return launch_tma(a, dtype, s);
  if (a.fast) return dtype == 0 ? launch_fast_f32(a, s) : launch_fast_f64(a, s);
  if (dtype != 0) return launch_pow2_c128(a, s);
  return a.ept == 16 ? launch_pow2_c64_e16(a, s) : launch_pow2_c64_e32(a, s);
}

}  // namespace pfft
