// Odd-prime-radix transform passes, complex64 with 32 points per thread, the
// padded tile (no direct prime stage); the unpadded one is in
// fft_pass_generic_c64_e32u.cu.
#include "fft_kernels.cuh"

namespace pfft {
int launch_generic_c64_e32_unpadded(const PassArgs& a, cudaStream_t s);
int launch_generic_c64_e32(const PassArgs& a, cudaStream_t s) {
  if (!a.pad) return launch_generic_c64_e32_unpadded(a, s);
  return launch_typed_pad<float2, 32, false, true, 1>(a, s);
}
}  // namespace pfft
