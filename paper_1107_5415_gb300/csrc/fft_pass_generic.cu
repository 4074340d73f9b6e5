// Instantiation of the transform passes with odd prime radices.
#include "fft_kernels.cuh"

namespace pfft {
int launch_pass_generic(const PassArgs& a, int dtype, cudaStream_t s) {
  if (dtype != 0) return launch_typed<double2, 16, false>(a, s);
  return a.ept == 16 ? launch_typed<float2, 16, false, 2>(a, s) : launch_typed<float2, 32, false>(a, s);
}
}  // namespace pfft
