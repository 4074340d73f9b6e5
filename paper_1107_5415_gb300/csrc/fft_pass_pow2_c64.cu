// Power-of-two shared-memory transform passes, complex64 with 16 points per
// thread (two CTAs per SM); 32 points per thread in fft_pass_pow2_c64_e32.cu.
#include "fft_kernels.cuh"

namespace pfft {
int launch_pow2_c64_e16(const PassArgs& a, cudaStream_t s) { return launch_typed<float2, 16, true, 2>(a, s); }
}  // namespace pfft
