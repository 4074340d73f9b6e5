// Odd-prime-radix transform passes, complex64 with 32 points per thread, the
// unpadded tile used with direct prime stages.
#include "fft_kernels.cuh"

namespace pfft {
int launch_generic_c64_e32_unpadded(const PassArgs& a, cudaStream_t s) {
  return launch_typed_pad<float2, 32, false, false, 1>(a, s);
}
}  // namespace pfft
