// Transform support kernels: pass dispatch, twiddle table, index probe.
#include <cuda_runtime.h>

#include "fft_plan.hpp"

namespace pfft {

int launch_pass_pow2(const PassArgs& a, int dtype, cudaStream_t s);
int launch_pass_generic(const PassArgs& a, int dtype, cudaStream_t s);

int launch_pass(const PassArgs& a, int dtype, cudaStream_t s) {
  return a.pow2 ? launch_pass_pow2(a, dtype, s) : launch_pass_generic(a, dtype, s);
}

// Twiddle table omega_{nD}^t = exp(-2 pi i t / nD), t in [0, nD): exact
// integer t, FP64 sincospi, rounded to the working precision.
template <typename C>
__global__ void twiddle_kernel(C* tw, int nD) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nD) return;
  double s, c;
  sincospi(2.0 * double(t) / double(nD), &s, &c);
  tw[t] = cmake<C>(decltype(C::x)(c), decltype(C::x)(-s));
}

int launch_twiddles(void* tw, int nD, int dtype, cudaStream_t s) {
  const int blk = 256, grd = (nD + blk - 1) / blk;
  if (dtype == 0)
    twiddle_kernel<float2><<<grd, blk, 0, s>>>(static_cast<float2*>(tw), nD);
  else
    twiddle_kernel<double2><<<grd, blk, 0, s>>>(static_cast<double2*>(tw), nD);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// dst[i] = tw[idx[i]]: the stage tables of the register-resident passes.
template <typename C>
__global__ void twiddle_gather_kernel(C* dst, const C* tw, const int* idx, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = tw[idx[i]];
}

int launch_twiddle_gather(void* dst, const void* tw, const int* idx, int n, int dtype, cudaStream_t s) {
  const int blk = 256, grd = (n + blk - 1) / blk;
  if (dtype == 0)
    twiddle_gather_kernel<float2><<<grd, blk, 0, s>>>(static_cast<float2*>(dst), static_cast<const float2*>(tw),
                                                      idx, n);
  else
    twiddle_gather_kernel<double2><<<grd, blk, 0, s>>>(static_cast<double2*>(dst),
                                                       static_cast<const double2*>(tw), idx, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Two-level table of exp(-2 pi i t / q): lo[t] for t < 2048, hi[t] = value at
// t << 11 (exact integer arguments, FP64 sincospi, rounded to the working type).
template <typename C>
__global__ void fs_phase_kernel(C* lo, C* hi, long long q, int nhi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  using Rl = decltype(C::x);
  double s, c;
  if (t < 2048) {
    sincospi(2.0 * double(t % q) / double(q), &s, &c);
    lo[t] = cmake<C>(Rl(c), Rl(-s));
  }
  if (t < nhi) {
    sincospi(2.0 * double(((long long)t << 11) % q) / double(q), &s, &c);
    hi[t] = cmake<C>(Rl(c), Rl(-s));
  }
}

int launch_phase_tables(void* tab, int64_t q, int nhi, int dtype, cudaStream_t s) {
  const int n = nhi > 2048 ? nhi : 2048;
  const int blk = 256, grd = (n + blk - 1) / blk;
  if (dtype == 0)
    fs_phase_kernel<float2><<<grd, blk, 0, s>>>(static_cast<float2*>(tab), static_cast<float2*>(tab) + 2048, q, nhi);
  else
    fs_phase_kernel<double2><<<grd, blk, 0, s>>>(static_cast<double2*>(tab), static_cast<double2*>(tab) + 2048, q,
                                                 nhi);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Index probe: for every Smith coordinate vector (row-major, flattened as
// row * nD + element), the box slot the transform kernels read (input map,
// which = 0) or write (output map, which = 1), evaluated with the same
// device code as the passes.  For the output map the element index is the
// Smith coordinate mu_D (converted to its workspace position).
__global__ void index_probe_kernel(PassArgs a, const int* __restrict__ PI, int which, int64_t* out) {
  const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= a.m) return;
  const int row = int(w / a.nD), e = int(w - int64_t(row) * a.nD);
  int slot;
  if (which == 0)
    slot = box_sum_slot(a.boxH, a.Atab + row * a.ts, a.Btab + e * a.ts);
  else
    slot = box_sum_slot(a.boxG, a.Ctab + row * a.ts, a.Etab + PI[e] * a.ts);
  // Smith coordinates of (row, e), flattened row-major over the cycles: with a
  // split last cycle lambda_D = lambda_a + n_a lambda_b (input) and
  // mu_D = mu_b + n_b mu_a (output), lambda_a / mu_a the fastest row index.
  int64_t smith = w;
  if (a.nsub == 2 && a.fs_na == 1 && a.sub_n[0] > a.sub_n[1]) {
    // rows over (lambda_2, lambda_1): the planner put the longer axis first
    // for the two-axis column pass (cycles are otherwise ascending)
    const int l2 = row / a.sub_n[1], l1 = row - l2 * a.sub_n[1];
    smith = (int64_t(l1) * a.sub_n[0] + l2) * a.nD + e;
  }
  if (a.fs_na > 1) {
    const int ra = row % a.fs_na, rest = row / a.fs_na;
    const int64_t n = int64_t(a.fs_na) * a.nD;
    smith = rest * n + (which == 0 ? ra + int64_t(a.fs_na) * e : e + int64_t(a.nD) * ra);
  }
  out[smith] = slot;
}

int launch_index_probe(const PassArgs& rowp, const PassArgs& colp, int which, int64_t* out,
                       cudaStream_t s) {
  (void)colp;
  const int blk = 256;
  const int grd = int((int64_t(rowp.m) + blk - 1) / blk);
  index_probe_kernel<<<grd, blk, 0, s>>>(rowp, rowp.PIinv + rowp.nD, which, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pfft
