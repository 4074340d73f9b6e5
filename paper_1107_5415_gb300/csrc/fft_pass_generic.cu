// Instantiation of the transform passes with odd prime radices.
#include "fft_kernels.cuh"

namespace pfft {
int launch_pass_generic(const PassArgs& a, int dtype, cudaStream_t s) {
  return dtype == 0 ? launch_typed<float2, 32, false>(a, s) : launch_typed<double2, 16, false>(a, s);
}
}  // namespace pfft
