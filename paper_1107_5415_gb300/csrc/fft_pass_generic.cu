// Dispatch of the transform passes with odd prime radices; the kernels are
// instantiated one element type and width per translation unit
// (fft_pass_generic_*.cu) so that they compile in parallel.
#include "fft_plan.hpp"

namespace pfft {

int launch_generic_c128(const PassArgs& a, cudaStream_t s);     // fft_pass_generic_c128.cu
int launch_generic_c64_e16(const PassArgs& a, cudaStream_t s);  // fft_pass_generic_c64_e16.cu
int launch_generic_c64_e32(const PassArgs& a, cudaStream_t s);  // fft_pass_generic_c64_e32{,u}.cu

int launch_pass_generic(const PassArgs& a, int dtype, cudaStream_t s) {
  if (dtype != 0) return launch_generic_c128(a, s);
  return a.ept == 16 ? launch_generic_c64_e16(a, s) : launch_generic_c64_e32(a, s);
}

}  // namespace pfft
