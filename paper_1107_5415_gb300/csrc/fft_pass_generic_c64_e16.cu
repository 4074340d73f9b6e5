// Odd-prime-radix transform passes, complex64 with 16 points per thread (two CTAs per SM).
#include "fft_kernels.cuh"

namespace pfft {
int launch_generic_c64_e16(const PassArgs& a, cudaStream_t s) { return launch_typed<float2, 16, false, 2>(a, s); }
}  // namespace pfft
