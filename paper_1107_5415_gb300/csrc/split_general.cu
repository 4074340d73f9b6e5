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
#include "split_prime.cuh"

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

// Built-in band system (split_prime.cuh): one work item per fibre and chunk
// of band outputs, blockIdx.y the signal.  parts: [p][batch][mN].
template <typename C, int MODE>
__global__ void __launch_bounds__(256) split_prime_kernel(PrimeDesc P, int batch, const C* __restrict__ cin,
                                                          C* __restrict__ cout, const C* __restrict__ din,
                                                          C* __restrict__ dout) {
  const int b = blockIdx.y;
  const long long items = (long long)P.mN * P.nch;
  const long long dstride = (long long)batch * P.mN;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < items;
       w += (long long)gridDim.x * blockDim.x) {
    const int ch = int(w / P.mN), gs = int(w - (long long)ch * P.mN);
    const long long off = (long long)b * P.mN + gs;
    prime_split_item<C, MODE>(P, gs, ch * kPrimeChunk, MODE == 0 ? cin + (long long)b * P.mM : nullptr,
                              MODE == 0 ? nullptr : cout + (long long)b * P.mM, MODE == 0 ? nullptr : din + off,
                              MODE == 0 ? nullptr : din + off + dstride, MODE == 0 ? dout + off : nullptr,
                              MODE == 0 ? dout + off + dstride : nullptr, dstride);
  }
}

}  // namespace pfft

using namespace pfft;

// Host setup of the built-in band system (exact integers): the general
// fibre description, the numerators of N^{-T} h, the functional v of
// J^T Z^d (last row of Q^{-1}, J^T = Q E R, so that v . l = 1 for the
// generator l = Q e_d), and the phase vector adj(M) (J z) for the centred
// generator z of P(J) with l^T z = 1/p, found among the p points of P(J).
pfft_status pfft::describe_prime_level(int d, const int64_t* Mv, const int64_t* Jv, PrimeDesc* out) {
  if (!Mv || !Jv || !out || d < 1 || d > 4) return PFFT_ERR_ARG;
  PrimeDesc P;
  std::memset(&P, 0, sizeof(P));
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
  if (m >= (i64(1) << 30)) return PFFT_ERR_OVERFLOW;
  if (p < 2 || p > (i64(1) << 20)) return PFFT_ERR_UNSUPPORTED;
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
  if (nontrivial != 1 || eps[d - 1] != p) return PFFT_ERR_UNSUPPORTED;  // G(J^T) not cyclic
  for (i64 f = 2; f * f <= p; ++f)
    if (p % f == 0) return PFFT_ERR_UNSUPPORTED;  // the built-in band system takes prime p
  IMat Qi;
  if (!inverse_unimodular(Q, Qi)) return PFFT_ERR_OVERFLOW;
  // v: the functional with kernel J^T Z^d (last row of Q^{-1}, mod p); the
  // band generator l = e_i for the first i with v_i != 0 (the first unit
  // vector outside J^T Z^d), and v scaled so that v . l = 1
  std::vector<i64> l(d, 0), v(d);
  for (int i = 0; i < d; ++i) v[i] = posmod(Qi(d - 1, i), p);
  int istar = -1;
  for (int i = 0; i < d && istar < 0; ++i)
    if (v[i] != 0) istar = i;
  if (istar < 0) return PFFT_ERR_OVERFLOW;
  l[istar] = 1;
  {
    // v_i* ^ (p - 2) mod p: the inverse of v_i* (p prime)
    i64 inv = 1, b = v[istar], e = p - 2;
    while (e > 0) {
      if (e & 1) inv = i64((i128)inv * b % p);
      b = i64((i128)b * b % p);
      e >>= 1;
    }
    for (int i = 0; i < d; ++i) v[i] = i64((i128)v[i] * inv % p);
  }
  IMat HM = hermite_normal_form(M.transpose());
  IMat HN = hermite_normal_form(N.transpose());
  P.d = d;
  P.p = int(p);
  P.mM = int(m);
  P.mN = int(m / p);
  P.HM.d = d;
  int stride = 1;
  for (int r = d - 1; r >= 0; --r) {
    for (int c = 0; c < d; ++c) P.HM.H[r][c] = int(HM(r, c));
    P.HM.stride[r] = stride;
    stride *= int(HM(r, r));
    P.HNext[r] = int(HN(r, r));
    P.divHN[r].init(uint32_t(HN(r, r)));
  }
  std::vector<i64> sh(d, 0);
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k) sh[i] += N(k, i) * l[k];  // N^T l
  box_reduce(HM, sh.data());
  for (int i = 0; i < d; ++i) {
    P.shift[i] = int(sh[i]);
    P.v[i] = v[i];
  }
  // numerators of N^{-T} h = J^T M^{-T} h over q: sign(det M) J^T adj(M^T)
  const int sM = detM < 0 ? -1 : 1;
  IMat K = matmul(J.transpose(), adjugate(M.transpose()));
  i128 bound = 0;
  for (int r = 0; r < d; ++r) {
    i128 row = 0;
    for (int c = 0; c < d; ++c) {
      P.K[r * d + c] = sM * K(r, c);
      row += (i128)(K(r, c) < 0 ? -K(r, c) : K(r, c)) * HN(c, c);
    }
    if (row > bound) bound = row;
  }
  if (bound >= ((i128)1 << 60)) return PFFT_ERR_OVERFLOW;
  P.q = m;
  // the centred generator z of P(J) with l^T z = 1/p: z = adj(J) y / det J for
  // the points y of the box of H(J); u = J z
  IMat HJ = hermite_normal_form(J);
  IMat adjJ = adjugate(J);
  std::vector<i64> u(d, 0);
  bool found = false;
  std::vector<i64> y(d, 0);
  for (i64 cnt = 0; cnt < p && !found; ++cnt) {
    i64 rest = cnt;
    for (int r = d - 1; r >= 0; --r) {
      y[r] = rest % HJ(r, r);
      rest /= HJ(r, r);
    }
    // z numerators over |det J| (sign folded in): zn = sign(det J) adj(J) y
    std::vector<i128> zn(d, 0);
    for (int i = 0; i < d; ++i)
      for (int c = 0; c < d; ++c) zn[i] += (i128)adjJ(i, c) * y[c];
    if (detJ < 0)
      for (auto& x : zn) x = -x;
    i128 lz = 0;
    for (int i = 0; i < d; ++i) lz += (i128)l[i] * zn[i];  // l^T z = lz / p
    i128 lzm = lz % p;
    if (lzm < 0) lzm += p;
    if (lzm != 1) continue;
    // centre each coordinate into [-1/2, 1/2): numerator in [-p/2, p/2)
    for (int i = 0; i < d; ++i) {
      i128 r = zn[i] % p;
      if (r < 0) r += p;
      if (2 * r >= p) r -= p;
      zn[i] = r;
    }
    for (int i = 0; i < d; ++i) {
      i128 acc = 0;
      for (int c = 0; c < d; ++c) acc += (i128)J(i, c) * zn[c];
      if (acc % p != 0) return PFFT_ERR_OVERFLOW;
      u[i] = i64(acc / p);
    }
    found = true;
  }
  if (!found) return PFFT_ERR_OVERFLOW;
  IMat adjM = adjugate(M);
  for (int i = 0; i < d; ++i) {
    i128 acc = 0;
    for (int c = 0; c < d; ++c) acc += (i128)adjM(i, c) * u[c];
    i64 r = i64(acc % m);
    if (r < 0) r += m;
    P.phw[i] = sM > 0 ? r : (m - r) % m;
  }
  P.nch = int((p + kPrimeChunk - 1) / kPrimeChunk);
  *out = P;
  return PFFT_OK;
}

static pfft_status prime_run(int mode, int d, const int64_t* M, const int64_t* J, int64_t batch, int dtype,
                             const void* src, void* dst, void* stream) {
  PrimeDesc P;
  pfft_status st;
  try {
    st = describe_prime_level(d, M, J, &P);
  } catch (const LatticeError& e) {
    st = pfft_status(e.code);
  }
  if (st != PFFT_OK) return st;
  if (int64_t(P.mM) * batch >= (int64_t(1) << 40)) return PFFT_ERR_OVERFLOW;
  const int blk = 256;
  long long gx = ((long long)P.mN * P.nch + blk - 1) / blk;
  const long long cap = (152LL * 16 + batch - 1) / batch;
  if (gx > cap) gx = cap;
  dim3 grid(unsigned(gx < 1 ? 1 : gx), unsigned(batch));
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == PFFT_C64) {
    using C = float2;
    if (mode == 0)
      split_prime_kernel<C, 0><<<grid, blk, 0, s>>>(P, int(batch), static_cast<const C*>(src), nullptr, nullptr,
                                                     static_cast<C*>(dst));
    else
      split_prime_kernel<C, 1><<<grid, blk, 0, s>>>(P, int(batch), nullptr, static_cast<C*>(dst),
                                                     static_cast<const C*>(src), nullptr);
  } else {
    using C = double2;
    if (mode == 0)
      split_prime_kernel<C, 0><<<grid, blk, 0, s>>>(P, int(batch), static_cast<const C*>(src), nullptr, nullptr,
                                                     static_cast<C*>(dst));
    else
      split_prime_kernel<C, 1><<<grid, blk, 0, s>>>(P, int(batch), nullptr, static_cast<C*>(dst),
                                                     static_cast<const C*>(src), nullptr);
  }
  return cudaGetLastError() == cudaSuccess ? PFFT_OK : PFFT_ERR_CUDA;
}

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
  if (!M || !J || !src || !dst || src == dst || batch < 1 || batch > 65535 ||
      (dtype != PFFT_C64 && dtype != PFFT_C128))
    return PFFT_ERR_ARG;
  if (!symbols) return prime_run(mode, d, M, J, batch, dtype, src, dst, stream);
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
