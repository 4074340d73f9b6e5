// General split step (Section 5.3, step 4) for dilations of any determinant p
// whose group G(J^T) = Z^d / J^T Z^d is cyclic, with symbols supplied by the
// caller, and its adjoint.
//
// M = J N.  The fibre of g in G(N^T) is {h_t = g + t N^T l : t < p}, l a
// generator of G(J^T); step 4 computes, for every symbol b_j (j < p),
//     d_j[g] = p^{-1/2} sum_t conj(b_j(h_t)) c(h_t)
// (analysis with conjugated symbols, the reading used for |det J| = 2), and
// the adjoint puts c(h_t) = p^{-1/2} sum_j b_j(h_t) d_j[g].  When the p x p
// matrix (b_j(h_t)) / sqrt(p) is unitary on every fibre the adjoint is the
// inverse.  One thread per fibre: it walks h_t by adding the box point of
// N^T l and reducing into the box of H(M^T), keeps the p slots, and reads
// each coefficient and symbol value once.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/pfft.h"
#include "device_common.cuh"
#include "lattice.hpp"

namespace pfft {

constexpr int kGeneralMaxP = 16;

struct GeneralDesc {
  int d, p;
  int mM, mN;
  BoxDesc HM;
  int HNext[4];
  FastDiv divHN[4];
  int shift[4];  // box(H(M^T)) point of N^T l
};

template <typename C, int MODE>
__global__ void __launch_bounds__(256) split_general_kernel(GeneralDesc G, int batch, const C* __restrict__ sym,
                                                            const C* __restrict__ cin, C* __restrict__ cout,
                                                            const C* __restrict__ din, C* __restrict__ dout) {
  using Rl = decltype(C::x);
  const int b = blockIdx.y;
  const int p = G.p;
  const Rl rs = Rl(1) / sqrt(Rl(p));
  for (int gs = blockIdx.x * blockDim.x + threadIdx.x; gs < G.mN; gs += gridDim.x * blockDim.x) {
    int h[4] = {0, 0, 0, 0};
    int s = gs;
    for (int r = G.d - 1; r >= 0; --r) {
      const int q = G.divHN[r].div(s);
      h[r] = s - q * G.HNext[r];
      s = q;
    }
    int slot[kGeneralMaxP];
#pragma unroll
    for (int t = 0; t < kGeneralMaxP; ++t) {
      if (t >= p) break;
      int sl = 0;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (r < G.d) sl += h[r] * G.HM.stride[r];
      slot[t] = sl;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (r < G.d) h[r] += G.shift[r];
      box_fix(G.HM, h);
    }
    if (MODE == 0) {
      C c[kGeneralMaxP];
#pragma unroll
      for (int t = 0; t < kGeneralMaxP; ++t)
        if (t < p) c[t] = cin[(long long)b * G.mM + slot[t]];
      for (int j = 0; j < p; ++j) {
        C acc = cmake<C>(0, 0);
#pragma unroll
        for (int t = 0; t < kGeneralMaxP; ++t)
          if (t < p) acc = cadd(acc, cmul(cconj(__ldg(sym + (long long)j * G.mM + slot[t])), c[t]));
        dout[((long long)j * batch + b) * G.mN + gs] = cscale(acc, rs);
      }
    } else {
      C dv[kGeneralMaxP];
#pragma unroll
      for (int j = 0; j < kGeneralMaxP; ++j)
        if (j < p) dv[j] = din[((long long)j * batch + b) * G.mN + gs];
#pragma unroll
      for (int t = 0; t < kGeneralMaxP; ++t) {
        if (t >= p) break;
        C acc = cmake<C>(0, 0);
#pragma unroll
        for (int j = 0; j < kGeneralMaxP; ++j)
          if (j < p) acc = cadd(acc, cmul(__ldg(sym + (long long)j * G.mM + slot[t]), dv[j]));
        cout[(long long)b * G.mM + slot[t]] = cscale(acc, rs);
      }
    }
  }
}

}  // namespace pfft

using namespace pfft;

// Host setup (exact integers): N = J^{-1} M, the boxes, a generator l of the
// cyclic G(J^T) (from J^T = Q E R: the class of Q e_d) and the box point of N^T l.
static pfft_status general_setup(int d, const int64_t* Mv, const int64_t* Jv, GeneralDesc& G) {
  if (d < 1 || d > 4) return PFFT_ERR_ARG;
  std::memset(&G, 0, sizeof(G));
  IMat M(d), J(d);
  for (int i = 0; i < d * d; ++i) {
    if (Mv[i] >= (int64_t(1) << 24) || Mv[i] <= -(int64_t(1) << 24) || Jv[i] >= (int64_t(1) << 24) ||
        Jv[i] <= -(int64_t(1) << 24))
      return PFFT_ERR_OVERFLOW;
    M.a[i] = Mv[i];
    J.a[i] = Jv[i];
  }
  const i64 detM = determinant(M), detJ = determinant(J);
  if (detM == 0 || detJ == 0) return PFFT_ERR_SINGULAR;
  const i64 m = detM < 0 ? -detM : detM, p = detJ < 0 ? -detJ : detJ;
  if (m >= (i64(1) << 30)) return PFFT_ERR_OVERFLOW;  // box sums stay below 2^31
  if (p < 2 || p > kGeneralMaxP) return PFFT_ERR_UNSUPPORTED;
  IMat N = matmul(adjugate(J), M);
  for (auto& x : N.a) {
    if (x % detJ != 0) return PFFT_ERR_NOT_INTEGRAL;
    x /= detJ;
  }
  IMat Q, R, U, V;
  std::vector<i64> eps;
  smith_normal_form(J.transpose(), Q, eps, R, U, V);
  int nontrivial = 0;
  for (i64 e : eps)
    if (e > 1) ++nontrivial;
  if (nontrivial != 1) return PFFT_ERR_UNSUPPORTED;  // G(J^T) not cyclic
  IMat HM = hermite_normal_form(M.transpose());
  IMat HN = hermite_normal_form(N.transpose());
  G.d = d;
  G.p = int(p);
  G.mM = int(m);
  G.mN = int(m / p);
  G.HM.d = d;
  int stride = 1;
  for (int r = d - 1; r >= 0; --r) {
    for (int c = 0; c < d; ++c) G.HM.H[r][c] = int(HM(r, c));
    G.HM.stride[r] = stride;
    stride *= int(HM(r, r));
    G.HNext[r] = int(HN(r, r));
    G.divHN[r].init(uint32_t(HN(r, r)));
    if (HN(r, r) > HM(r, r)) return PFFT_ERR_OVERFLOW;  // cannot happen for M = J N
  }
  std::vector<i64> l(d), sh(d, 0);
  for (int i = 0; i < d; ++i) l[i] = Q(i, d - 1);
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k) sh[i] += N(k, i) * l[k];  // N^T l
  box_reduce(HM, sh.data());
  for (int i = 0; i < d; ++i) G.shift[i] = int(sh[i]);
  return PFFT_OK;
}

static pfft_status general_run(int mode, int d, const int64_t* M, const int64_t* J, int64_t batch, int dtype,
                               const void* symbols, const void* src, void* dst, void* stream) {
  if (!M || !J || !symbols || !src || !dst || src == dst || batch < 1 || batch > 65535 ||
      (dtype != PFFT_C64 && dtype != PFFT_C128))
    return PFFT_ERR_ARG;
  GeneralDesc G;
  pfft_status st;
  try {
    st = general_setup(d, M, J, G);
  } catch (const LatticeError& e) {
    st = pfft_status(e.code);
  }
  if (st != PFFT_OK) return st;
  if (int64_t(G.mM) * batch >= (int64_t(1) << 40)) return PFFT_ERR_OVERFLOW;
  const int blk = 256;
  long long gx = (G.mN + blk - 1) / blk;
  const long long cap = (152LL * 16 + batch - 1) / batch;
  if (gx > cap) gx = cap;
  dim3 grid(unsigned(gx < 1 ? 1 : gx), unsigned(batch));
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == PFFT_C64) {
    using C = float2;
    if (mode == 0)
      split_general_kernel<C, 0><<<grid, blk, 0, s>>>(G, int(batch), static_cast<const C*>(symbols),
                                                       static_cast<const C*>(src), nullptr, nullptr,
                                                       static_cast<C*>(dst));
    else
      split_general_kernel<C, 1><<<grid, blk, 0, s>>>(G, int(batch), static_cast<const C*>(symbols), nullptr,
                                                       static_cast<C*>(dst), static_cast<const C*>(src), nullptr);
  } else {
    using C = double2;
    if (mode == 0)
      split_general_kernel<C, 0><<<grid, blk, 0, s>>>(G, int(batch), static_cast<const C*>(symbols),
                                                       static_cast<const C*>(src), nullptr, nullptr,
                                                       static_cast<C*>(dst));
    else
      split_general_kernel<C, 1><<<grid, blk, 0, s>>>(G, int(batch), static_cast<const C*>(symbols), nullptr,
                                                       static_cast<C*>(dst), static_cast<const C*>(src), nullptr);
  }
  return cudaGetLastError() == cudaSuccess ? PFFT_OK : PFFT_ERR_CUDA;
}

extern "C" pfft_status pwt_split_general(int d, const int64_t* M, const int64_t* J, int64_t batch, int dtype,
                                         const void* symbols, const void* c_hat, void* parts, void* stream) {
  return general_run(0, d, M, J, batch, dtype, symbols, c_hat, parts, stream);
}

extern "C" pfft_status pwt_merge_general(int d, const int64_t* M, const int64_t* J, int64_t batch, int dtype,
                                         const void* symbols, const void* parts, void* c_hat, void* stream) {
  return general_run(1, d, M, J, batch, dtype, symbols, parts, c_hat, stream);
}
