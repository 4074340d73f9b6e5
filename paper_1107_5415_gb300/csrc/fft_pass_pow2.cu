// Instantiation of the transform passes whose stages are all powers of two.
#include "fft_kernels.cuh"

namespace pfft {
int launch_pass_pow2(const PassArgs& a, int dtype, cudaStream_t s) {
  return dtype == 0 ? launch_typed<float2, 32, true>(a, s) : launch_typed<double2, 16, true>(a, s);
}
}  // namespace pfft
