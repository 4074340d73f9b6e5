// Power-of-two shared-memory transform passes, complex64 with 32 points per thread.
#include "fft_kernels.cuh"

namespace pfft {
int launch_pow2_c64_e32(const PassArgs& a, cudaStream_t s) { return launch_typed<float2, 32, true>(a, s); }
}  // namespace pfft
