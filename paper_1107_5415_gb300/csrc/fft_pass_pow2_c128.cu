// Power-of-two shared-memory transform passes, complex128 (16 points per thread).
#include "fft_kernels.cuh"

namespace pfft {
int launch_pow2_c128(const PassArgs& a, cudaStream_t s) { return launch_typed<double2, 16, true>(a, s); }
}  // namespace pfft
