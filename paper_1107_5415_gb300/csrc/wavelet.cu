// Fast wavelet split step (Section 5.3, step 4) with the Dirichlet symbols of
// Section 6.2, its exact inverse and its adjoint: plans (host, exact integer
// setup) and the sm_103a kernel.
//
// One level, M = J N with |det J| = 2.  G(M^T) -> G(N^T) is onto with kernel
// N^T G(J^T), so the fibre of g in G(N^T) is {h0, h1} = {g, g + N^T l1}, l1
// the non-zero class of G(J^T).  The kernel walks the slots g of the box of
// H(N^T) (coalesced writes); g already lies in the box of H(M^T) because the
// diagonal of H(M^T) dominates that of H(N^T) (M^T Z^d is a sublattice of
// N^T Z^d), and h1 is g plus a fixed box point, reduced with at most one
// column step per coordinate.
//
// Scaling symbol, evaluated in the periodised form
//     A(h) = sqrt(|det J| w(N^{-T} h)),   w(t) = sum_{n in J^T Z^d} prod_j B(t_j + n_j),
// with B the indicator of [-1/2, 1/2] taking 1/2 on the boundary (Dirichlet,
// equal to the case formula of Section 6.2), or, for the de la Vallee Poussin
// reading, A(h) = sqrt|det J| w(N^{-T} h) with B(s) = clamp(((1+eta)/2-|s|)/eta, 0, 1).
// Because J^T Z^d has index 2 it is the kernel of n -> v.n mod 2 for one
// parity vector v, and both B's are partitions of unity over integer shifts,
//     w(t) = (1 + prod_j U_j(t_j)) / 2,   U_j(t) = sum_n B(t + n) (-1)^(v_j n),
// so each coordinate needs at most three candidate shifts and no product over
// lattice points.  On the fibre partner (t shifted by the class not in
// J^T Z^d) the product changes sign: w(h1) = 1 - w(h0).  N^{-T} h is formed
// from exact integer numerators K h over |det M|, K = sign(det M) J^T adj(M^T),
// reduced mod 2 |det M| (U_j has period 2).  Wavelet symbol B(h) = A(h + N^T l1)
// exp(-2 pi i h^T N^{-1} z), with h^T N^{-1} z = h^T M^{-1} (J z) read from a
// two-level table of exp(-2 pi i t / |det M|) built in FP64; on the partner
// the phase changes sign (l1^T z = 1/2 mod 1).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <new>
#include <vector>

#include "../../include/pfft.h"
#include "device_common.cuh"
#include "wavelet_kernels.cuh"
#include "lattice.hpp"
#include "plan_common.hpp"
#include "plan_internal.hpp"

namespace pfft {

template <typename C>
__global__ void phase_table_kernel(C* lo, C* hi, long long q, int nhi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  using Rl = decltype(C::x);
  double s, c;
  if (t < (1 << kLoBits)) {
    sincospi(2.0 * double(t % q) / double(q), &s, &c);
    lo[t] = cmake<C>(Rl(c), Rl(-s));
  }
  if (t < nhi) {
    const long long a = ((long long)t << kLoBits) % q;
    sincospi(2.0 * double(a) / double(q), &s, &c);
    hi[t] = cmake<C>(Rl(c), Rl(-s));
  }
}

template <typename C, bool SMALL>
static void launch_split_t(const LevelDesc& L, int batch, int mode, const void* cin, void* cout,
                           const void* d1in, const void* d2in, void* d1out, void* d2out, cudaStream_t s) {
  const int blk = 256;
  unsigned gx, gy;
  int chunk;
  split_grid(L.mN, batch, gx, gy, chunk);
  dim3 grid(gx, gy);
  auto c = [](const void* p) { return static_cast<const C*>(p); };
  auto m = [](void* p) { return static_cast<C*>(p); };
  if (mode == 0)
    split_kernel<C, 0, true, SMALL><<<grid, blk, 0, s>>>(L, batch, chunk, c(cin), nullptr, nullptr, nullptr,
                                                          m(d1out), m(d2out));
  else if (mode == 1)
    split_kernel<C, 1, true, SMALL><<<grid, blk, 0, s>>>(L, batch, chunk, nullptr, m(cout), c(d1in), c(d2in),
                                                          nullptr, nullptr);
  else
    split_kernel<C, 2, true, SMALL><<<grid, blk, 0, s>>>(L, batch, chunk, nullptr, m(cout), c(d1in), c(d2in),
                                                          nullptr, nullptr);
}

template <typename C>
static int launch_split(const LevelDesc& L, int batch, int mode, const void* cin, void* cout, const void* d1in,
                        const void* d2in, void* d1out, void* d2out, cudaStream_t s) {
  if (L.small)
    launch_split_t<C, true>(L, batch, mode, cin, cout, d1in, d2in, d1out, d2out, s);
  else
    launch_split_t<C, false>(L, batch, mode, cin, cout, d1in, d2in, d1out, d2out, s);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pfft

using namespace pfft;

struct pwt_plan_s {
  int d = 0, levels = 0, symbol = 0, dtype = 0;
  int64_t batch = 0;
  double eta = 0;
  std::vector<IMat> Ms;       // M_1 .. M_{levels+1} (M_{l+1} = N_l)
  std::vector<i64> sizes;     // |det M_l|
  std::vector<IMat> boxes;    // H(M_l^T)
  std::vector<LevelDesc> lv;  // device descriptors
  LevelDesc* dlv = nullptr;   // the same in device memory (fused launches)
  void* symtab = nullptr;     // per-fibre symbols of the levels that fused launches take
  void* tables = nullptr;     // phase tables of all levels
  void* ws[2] = {nullptr, nullptr};
  Profiler prof;
};

static size_t cbytes(int dtype) { return dtype == PFFT_C64 ? 8 : 16; }

static void release(pwt_plan_s* P) {
  if (!P) return;
  if (P->tables) cudaFree(P->tables);
  if (P->dlv) cudaFree(P->dlv);
  if (P->symtab) cudaFree(P->symtab);
  for (auto p : P->ws)
    if (p) cudaFree(p);
  delete P;
}

// The non-zero class of G(J^T) = Z^d / J^T Z^d: a unit vector outside J^T Z^d.
static bool nonzero_class(const IMat& J, std::vector<i64>& l1) {
  const int d = J.d;
  IMat A = adjugate(J.transpose());
  const i64 D = determinant(J);
  const i64 aD = D < 0 ? -D : D;
  for (int i = 0; i < d; ++i) {
    // e_i in J^T Z^d  <=>  adj(J^T) e_i = 0 mod |det J|
    bool inside = true;
    for (int r = 0; r < d; ++r)
      if (posmod(A(r, i), aD) != 0) inside = false;
    if (!inside) {
      l1.assign(d, 0);
      l1[i] = 1;
      return true;
    }
  }
  return false;
}

// u = J z for the non-zero z of P(J) = Lambda(J) cap [-1/2, 1/2)^d.
static bool wavelet_shift(const IMat& J, std::vector<i64>& u) {
  const int d = J.d;
  const i64 D = determinant(J);
  const i64 aD = D < 0 ? -D : D;
  const int sD = D < 0 ? -1 : 1;
  IMat A = adjugate(J);
  IMat H = hermite_normal_form(J);
  // enumerate the box of H(J) (the classes of G(J)); z = J^{-1} y, centred
  std::vector<i64> y(d, 0);
  for (i64 s = 0; s < aD; ++s) {
    box_point(H, s, y.data());
    std::vector<i64> num(d);  // z = num / aD
    bool zero = true;
    for (int i = 0; i < d; ++i) {
      i128 t = 0;
      for (int k = 0; k < d; ++k) t += (i128)A(i, k) * y[k];
      t *= sD;
      // centre into [-1/2, 1/2): num - aD * floor((2 num + aD) / (2 aD))
      i64 v = i64(t);
      v -= aD * floordiv(2 * v + aD, 2 * aD);
      num[i] = v;
      if (v != 0) zero = false;
    }
    if (zero) continue;
    u.assign(d, 0);
    for (int i = 0; i < d; ++i) {
      i128 t = 0;
      for (int k = 0; k < d; ++k) t += (i128)J(i, k) * num[k];
      if (t % aD != 0) return false;
      u[i] = i64(t / aD);
    }
    return true;
  }
  return false;
}

static pfft_status plan_levels(pwt_plan_s& P, const int64_t* Mv, const int64_t* Jv) {
  const int d = P.d;
  IMat M(d);
  for (int i = 0; i < d * d; ++i) {
    if (Mv[i] >= (int64_t(1) << 24) || Mv[i] <= -(int64_t(1) << 24)) return PFFT_ERR_OVERFLOW;
    M.a[i] = Mv[i];
  }
  i64 det = determinant(M);
  if (det == 0) return PFFT_ERR_SINGULAR;
  if ((det < 0 ? -det : det) >= (i64(1) << 31)) return PFFT_ERR_OVERFLOW;
  P.Ms.push_back(M);
  for (int l = 0; l < P.levels; ++l) {
    IMat J(d);
    for (int i = 0; i < d * d; ++i) J.a[i] = Jv[size_t(l) * d * d + i];
    const i64 dJ = determinant(J);
    if (dJ == 0) return PFFT_ERR_SINGULAR;
    if (dJ != 2 && dJ != -2) return PFFT_ERR_UNSUPPORTED;
    const IMat& Mc = P.Ms.back();
    // N = J^{-1} M = adj(J) M / det J, must be integral
    IMat N = matmul(adjugate(J), Mc);
    for (auto& x : N.a) {
      if (x % dJ != 0) return PFFT_ERR_NOT_INTEGRAL;
      x /= dJ;
    }
    const i64 detM = determinant(Mc);
    const i64 q = detM < 0 ? -detM : detM;
    LevelDesc L;
    std::memset(&L, 0, sizeof(L));
    L.d = d;
    IMat HM = hermite_normal_form(Mc.transpose());
    IMat HN = hermite_normal_form(N.transpose());
    L.mM = int(q);
    L.mN = int(q / 2);
    L.HM.d = d;
    int stride = 1;
    for (int r = d - 1; r >= 0; --r) {
      for (int c = 0; c < d; ++c) L.HM.H[r][c] = int(HM(r, c));
      L.HM.stride[r] = stride;
      stride *= int(HM(r, r));
      L.HNext[r] = int(HN(r, r));
      L.divHN[r].init(uint32_t(HN(r, r)));
      if (HN(r, r) > HM(r, r)) return PFFT_ERR_OVERFLOW;  // cannot happen for M = J N
    }
    std::vector<i64> l1, u;
    if (!nonzero_class(J, l1) || !wavelet_shift(J, u)) return PFFT_ERR_UNSUPPORTED;
    std::vector<i64> sh(d, 0);
    for (int i = 0; i < d; ++i)
      for (int k = 0; k < d; ++k) sh[i] += N(k, i) * l1[k];  // N^T l1
    box_reduce(HM, sh.data());
    for (int i = 0; i < d; ++i) L.shift1[i] = int(sh[i]);
    IMat adjMT = adjugate(Mc.transpose());
    IMat adjM = adjugate(Mc);
    IMat adjJT = adjugate(J.transpose());
    for (int i = 0; i < d * d; ++i) {
      L.adjMT[i] = adjMT.a[i];
      L.J[i] = int(J.a[i]);
      L.adjJT[i] = adjJT.a[i];
    }
    L.q = q;
    L.sM = detM < 0 ? -1 : 1;
    L.aJ = 2;
    for (int i = 0; i < d; ++i) {
      i128 t = 0;
      for (int k = 0; k < d; ++k) t += (i128)adjM(i, k) * u[k];
      t %= q;  // only needed mod q
      L.phw[i] = (long long)t;
    }
    // overflow guards for the device's int64 arithmetic: |adj(M^T)_ij| h_j summed
    // over d terms must stay below 2^62 for every box point h
    for (int i = 0; i < d; ++i) {
      i128 bound = 0;
      for (int k = 0; k < d; ++k) {
        const i64 a = adjMT(i, k) < 0 ? -adjMT(i, k) : adjMT(i, k);
        bound += (i128)a * HM(k, k);
      }
      if (bound >= ((i128)1 << 60)) return PFFT_ERR_OVERFLOW;
    }
    L.symbol = P.symbol;
    L.eta = P.eta;
    {
      // K = sign(det M) J^T adj(M^T): numerators of N^{-T} h over q
      IMat JT = J.transpose();
      IMat K = matmul(JT, adjMT);
      const int sM = detM < 0 ? -1 : 1;
      i128 bound = 0;
      for (int r = 0; r < d; ++r) {
        i128 row = 0;
        for (int c = 0; c < d; ++c) {
          L.K[r * d + c] = sM * K(r, c);
          const i64 a = K(r, c) < 0 ? -K(r, c) : K(r, c);
          row += (i128)a * HM(c, c);
        }
        if (row > bound) bound = row;
      }
      if (bound >= ((i128)1 << 60)) return PFFT_ERR_OVERFLOW;
      const i128 twoq = 2 * (i128)q;
      // phase vector sign(det M) adj(M) (J z) reduced mod q into (-q, q)
      i128 pbound = 0;
      for (int i = 0; i < d; ++i) {
        const i64 v = (L.sM < 0 ? -1 : 1) * (L.phw[i] % q);
        L.ph32[i] = int(v);
        pbound += (i128)(v < 0 ? -v : v) * HM(i, i);
      }
      L.small = (bound < ((i128)1 << 29) && twoq < ((i128)1 << 29) && pbound < ((i128)1 << 29)) ? 1 : 0;
      if (L.small) {
        for (int k = 0; k < d * d; ++k) L.K32[k] = int(L.K[k]);
        L.div2q.init(uint32_t(2 * q));
        L.off2q = int(((bound / twoq) + 1) * twoq);
        L.divq.init(uint32_t(q));
        L.offq = int(((pbound / q) + 1) * q);
      }
      // parity vector: v . n = 0 mod 2 exactly on J^T Z^d (its columns span it)
      bool found = false;
      for (int v = 1; v < (1 << d) && !found; ++v) {
        bool ok = true;
        for (int c = 0; c < d && ok; ++c) {
          i64 s2 = 0;
          for (int r = 0; r < d; ++r) s2 += ((v >> r) & 1) * JT(r, c);
          if (posmod(s2, 2) != 0) ok = false;
        }
        if (ok) {
          for (int r = 0; r < d; ++r) L.vpar[r] = (v >> r) & 1;
          found = true;
        }
      }
      if (!found) return PFFT_ERR_UNSUPPORTED;
    }
    P.lv.push_back(L);
    P.boxes.push_back(HM);
    P.sizes.push_back(q);
    P.Ms.push_back(N);
  }
  {
    IMat HL = hermite_normal_form(P.Ms.back().transpose());
    P.boxes.push_back(HL);
    const i64 dl = determinant(P.Ms.back());
    P.sizes.push_back(dl < 0 ? -dl : dl);
  }
  return PFFT_OK;
}

// Smith-coordinate order of the first level's coefficients: the mu basis of
// the transform planner for M (the order a PFFT_FLAG_LAYOUT_SNF plan of M
// writes), and mu of N^T l1.
static pfft_status set_snf_input(LevelDesc& L, int d, const int64_t* Mv, const int64_t* Jv) {
  pfft_plan_s T;
  pfft_status st = plan_host(T, d, Mv);
  if (st != PFFT_OK) return st;
  if (T.D > 4) return PFFT_ERR_UNSUPPORTED;
  IMat M(d), J(d);
  for (int i = 0; i < d * d; ++i) {
    M.a[i] = Mv[i];
    J.a[i] = Jv[i];
  }
  const i64 dJ = determinant(J);
  IMat N = matmul(adjugate(J), M);
  for (auto& x : N.a) x /= dJ;  // integral (checked by plan_levels)
  std::vector<i64> l1;
  if (!nonzero_class(J, l1)) return PFFT_ERR_UNSUPPORTED;
  L.snf_D = T.D;
  int str = 1;
  for (int j = T.D - 1; j >= 0; --j) {
    L.snf_n[j] = T.n[j];
    L.snf_str[j] = str;
    str *= T.n[j];
    i128 acc = 0;
    for (int c = 0; c < d; ++c) {
      L.snf_mu[j][c] = posmod(T.MU[j][c], T.n[j]);
      i64 v = 0;  // (N^T l1)_c
      for (int k = 0; k < d; ++k) v += N(k, c) * l1[k];
      acc += (i128)L.snf_mu[j][c] * v;
    }
    L.snf_l1[j] = int(posmod(i64(acc % T.n[j]), T.n[j]));
  }
  return PFFT_OK;
}

static pfft_status plan_device(pwt_plan_s& P) {
  const size_t cb = cbytes(P.dtype);
  size_t total = 0;
  std::vector<size_t> offs;
  for (auto& L : P.lv) {
    const int nhi = int((L.q + (1LL << kLoBits) - 1) >> kLoBits);
    offs.push_back(total);
    total += size_t((1 << kLoBits) + nhi) * cb;
  }
  if (int e_ = device_alloc((void**)&P.tables, total)) return pfft_status(e_);
  for (size_t l = 0; l < P.lv.size(); ++l) {
    LevelDesc& L = P.lv[l];
    const int nhi = int((L.q + (1LL << kLoBits) - 1) >> kLoBits);
    char* base = static_cast<char*>(P.tables) + offs[l];
    L.tab_lo = base;
    L.tab_hi = base + size_t(1 << kLoBits) * cb;
    const int n = std::max(1 << kLoBits, nhi);
    const int blk = 256, grd = (n + blk - 1) / blk;
    if (P.dtype == PFFT_C64)
      phase_table_kernel<float2><<<grd, blk>>>((float2*)L.tab_lo, (float2*)L.tab_hi, L.q, nhi);
    else
      phase_table_kernel<double2><<<grd, blk>>>((double2*)L.tab_lo, (double2*)L.tab_hi, L.q, nhi);
    if (cudaGetLastError() != cudaSuccess) return PFFT_ERR_CUDA;
  }
  // per-fibre symbol tables for the fused launches (complex64, int32 index
  // paths; for batches of four signals or more, where reading a fibre's
  // symbols costs less than evaluating them in every chunk of signals)
  if (P.dtype == PFFT_C64 && P.levels > 1 && P.batch >= 4) {
    size_t n = 0;
    for (auto& L : P.lv)
      if (L.small) n += size_t(L.mN);
    if (n) {
      if (int e_ = device_alloc(&P.symtab, n * sizeof(float4))) return pfft_status(e_);
      float4* t = static_cast<float4*>(P.symtab);
      for (auto& L : P.lv) {
        if (!L.small) continue;
        if (launch_symbol_table(L, t) != 0) return PFFT_ERR_CUDA;
        t += L.mN;
      }
    }
  }
  if (int e_ = device_alloc((void**)&P.dlv, sizeof(LevelDesc) * P.lv.size())) return pfft_status(e_);
  if (cudaMemcpy(P.dlv, P.lv.data(), sizeof(LevelDesc) * P.lv.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return PFFT_ERR_CUDA;
  if (P.levels > 1) {
    const size_t half = size_t(P.sizes[0] / 2) * P.batch * cb;
    for (int i = 0; i < 2; ++i)
      if (int e_ = device_alloc((void**)&P.ws[i], half)) return pfft_status(e_);
  }
  return cudaDeviceSynchronize() == cudaSuccess ? PFFT_OK : PFFT_ERR_CUDA;
}

extern "C" pfft_status pwt_plan_create(pwt_plan* out, int d, const int64_t* M, int levels,
                                       const int64_t* J, int symbol, double eta, int64_t batch,
                                       int dtype, unsigned flags) {
  if (!out || !M || !J || d < 1 || d > 4 || levels < 1 || levels > 64 || batch < 1 ||
      batch > (int64_t(1) << 20) || (dtype != PFFT_C64 && dtype != PFFT_C128) ||
      (flags & ~unsigned(PWT_FLAG_INPUT_SNF)) ||
      (symbol != PWT_DIRICHLET && symbol != PWT_DLVP) ||
      (symbol == PWT_DLVP && !(eta > 0.0 && eta < 1.0)))
    return PFFT_ERR_ARG;
  *out = nullptr;
  pwt_plan_s* P = new (std::nothrow) pwt_plan_s;
  if (!P) return PFFT_ERR_OOM;
  P->d = d;
  P->levels = levels;
  P->symbol = symbol;
  P->eta = eta;
  P->batch = batch;
  P->dtype = dtype;
  pfft_status st;
  try {
    st = plan_levels(*P, M, J);
    if (st == PFFT_OK && P->sizes[0] * batch >= (int64_t(1) << 40)) st = PFFT_ERR_OVERFLOW;
    if (st == PFFT_OK && (flags & PWT_FLAG_INPUT_SNF)) st = set_snf_input(P->lv[0], d, M, J);
    if (st == PFFT_OK) st = plan_device(*P);
  } catch (const LatticeError& e) {
    st = pfft_status(e.code);
  }
  if (st != PFFT_OK) {
    release(P);
    return st;
  }
  *out = P;
  return PFFT_OK;
}

extern "C" pfft_status pwt_plan_destroy(pwt_plan p) {
  if (!p) return PFFT_ERR_ARG;
  release(p);
  return PFFT_OK;
}

extern "C" pfft_status pwt_plan_info(pwt_plan p, int level, int64_t* n, int64_t* box) {
  if (!p || level < 0 || level > p->levels) return PFFT_ERR_ARG;
  if (n) *n = p->sizes[level];
  if (box)
    for (int i = 0; i < p->d; ++i) box[i] = p->boxes[level](i, i);
  return PFFT_OK;
}

static int run_level(pwt_plan_s* P, int l, int mode, const void* cin, void* cout, const void* d1in,
                     const void* d2in, void* d1out, void* d2out, cudaStream_t s) {
  P->prof.begin(0, s);
  int rc = P->dtype == PFFT_C64
               ? launch_split<float2>(P->lv[l], int(P->batch), mode, cin, cout, d1in, d2in, d1out, d2out, s)
               : launch_split<double2>(P->lv[l], int(P->batch), mode, cin, cout, d1in, d2in, d1out, d2out, s);
  P->prof.end(0, s);
  return rc;
}

// Levels l, l + 1, ... that one fused launch takes (fused_split_kernel):
// complex64, int32 index paths, the first level's input in box order; 1 when
// the level runs alone.
static int fuse_count(const pwt_plan_s* P, int l) {
  if (P->dtype != PFFT_C64 || P->lv[l].snf_D) return 1;
  int F = 0;
  while (F < kFuseMax && l + F < P->levels && P->lv[l + F].small) ++F;
  return F < 2 ? 1 : F;
}

template <int F>
static int launch_fused_t(pwt_plan_s* P, int l, const void* cin, void* sout, void* const* wavelets,
                          cudaStream_t s) {
  constexpr int smem = fused_smem_bytes<float2, F>();
  static const bool ok = cudaFuncSetAttribute(reinterpret_cast<const void*>(fused_split_kernel<float2, F>),
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
  if (!ok) return -1;
  // fibres of the last level over CTAs of kFuseThreads threads, about
  // kFuseWaves resident waves; the signals split into chunks only when the
  // fibres are too few
  const long long mN = P->lv[l + F - 1].mN, cap = 152LL * kFuseWaves;
  long long x = (mN + kFuseThreads - 1) / kFuseThreads;
  if (x > cap) x = cap;
  long long y = (cap + x - 1) / x;
  if (y > P->batch) y = P->batch;
  const int chunk = int((P->batch + y - 1) / y);
  const unsigned gy = unsigned((P->batch + chunk - 1) / chunk);
  float2* w[3] = {nullptr, nullptr, nullptr};
  for (int k = 0; k < F; ++k) w[k] = static_cast<float2*>(wavelets[l + k]);
  fused_split_kernel<float2, F><<<dim3(unsigned(x), gy), kFuseThreads, smem, s>>>(
      P->dlv + l, int(P->batch), chunk, static_cast<const float2*>(cin), static_cast<float2*>(sout), w[0], w[1],
      w[2]);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

static int launch_fused(pwt_plan_s* P, int l, int F, const void* cin, void* sout, void* const* wavelets,
                        cudaStream_t s) {
  P->prof.begin(0, s);
  const int rc = F == 3 ? launch_fused_t<3>(P, l, cin, sout, wavelets, s)
                        : launch_fused_t<2>(P, l, cin, sout, wavelets, s);
  P->prof.end(0, s);
  return rc;
}

extern "C" pfft_status pwt_decompose(pwt_plan p, const void* c_hat, void* scaling, void* const* wavelets,
                                     void* stream) {
  if (!p || !c_hat || !scaling || !wavelets) return PFFT_ERR_ARG;
  for (int l = 0; l < p->levels; ++l)
    if (!wavelets[l]) return PFFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const void* cur = c_hat;
  int g = 0;  // launches so far: their scaling parts alternate between the two workspaces
  for (int l = 0; l < p->levels; ++g) {
    const int F = fuse_count(p, l);
    void* d1 = (l + F == p->levels) ? scaling : p->ws[g & 1];
    const int rc = F > 1 ? launch_fused(p, l, F, cur, d1, wavelets, s)
                         : run_level(p, l, 0, cur, nullptr, nullptr, nullptr, d1, wavelets[l], s);
    if (rc != 0) return PFFT_ERR_CUDA;
    cur = d1;
    l += F;
  }
  return PFFT_OK;
}

static pfft_status synthesise(pwt_plan p, const void* scaling, const void* const* wavelets, void* c_hat,
                              void* stream, int mode) {
  if (!p || !c_hat || !scaling || !wavelets) return PFFT_ERR_ARG;
  for (int l = 0; l < p->levels; ++l)
    if (!wavelets[l]) return PFFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const void* cur = scaling;
  for (int l = p->levels - 1; l >= 0; --l) {
    void* dst = (l == 0) ? c_hat : p->ws[l & 1];
    if (run_level(p, l, mode, nullptr, dst, cur, wavelets[l], nullptr, nullptr, s) != 0) return PFFT_ERR_CUDA;
    cur = dst;
  }
  return PFFT_OK;
}

extern "C" pfft_status pwt_reconstruct(pwt_plan p, const void* scaling, const void* const* wavelets,
                                       void* c_hat, void* stream) {
  return synthesise(p, scaling, wavelets, c_hat, stream, 1);
}

extern "C" pfft_status pwt_adjoint(pwt_plan p, const void* scaling, const void* const* wavelets,
                                   void* c_hat, void* stream) {
  return synthesise(p, scaling, wavelets, c_hat, stream, 2);
}

// Two-level phase table of a level descriptor (lo: 2^kLoBits entries, then
// hi: ceil(q / 2^kLoBits)) at `tab`, sized by split_table_elems; queued on the
// legacy stream.
size_t pfft::split_table_elems(const LevelDesc& L) {
  return size_t(1 << kLoBits) + size_t((L.q + (1LL << kLoBits) - 1) >> kLoBits);
}

int pfft::launch_symbol_table(LevelDesc& L, void* tab) {
  if (!L.small || !L.tab_lo) return -1;
  const int grd = int(std::min<long long>((L.mN + 255) / 256, 152LL * 8));
  symbol_table_kernel<float2><<<grd, 256>>>(L, static_cast<float4*>(tab));
  if (cudaGetLastError() != cudaSuccess) return -1;
  L.symtab = tab;
  return 0;
}

int pfft::launch_split_tables(LevelDesc& L, void* tab, int dtype) {
  const int nhi = int((L.q + (1LL << kLoBits) - 1) >> kLoBits);
  const size_t cb = dtype == PFFT_C64 ? 8 : 16;
  L.tab_lo = tab;
  L.tab_hi = static_cast<char*>(tab) + size_t(1 << kLoBits) * cb;
  const int n = std::max(1 << kLoBits, nhi);
  const int blk = 256, grd = (n + blk - 1) / blk;
  if (dtype == PFFT_C64)
    phase_table_kernel<float2><<<grd, blk>>>((float2*)L.tab_lo, (float2*)L.tab_hi, L.q, nhi);
  else
    phase_table_kernel<double2><<<grd, blk>>>((double2*)L.tab_lo, (double2*)L.tab_hi, L.q, nhi);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Descriptor of one split level of M by J (host only; batch plans add the
// phase tables with launch_split_tables).
pfft_status pfft::describe_split_level(int d, const int64_t* M, const int64_t* J, int symbol, double eta,
                                       LevelDesc* out) {
  if (!M || !J || !out || d < 1 || d > 4 || (symbol != PWT_DIRICHLET && symbol != PWT_DLVP) ||
      (symbol == PWT_DLVP && !(eta > 0.0 && eta < 1.0)))
    return PFFT_ERR_ARG;
  pwt_plan_s P;
  P.d = d;
  P.levels = 1;
  P.symbol = symbol;
  P.eta = eta;
  P.batch = 1;
  P.dtype = PFFT_C64;
  pfft_status st;
  try {
    st = plan_levels(P, M, J);
  } catch (const LatticeError& e) {
    st = pfft_status(e.code);
  }
  if (st == PFFT_OK) *out = P.lv[0];
  return st;
}

// ---------------------------------------------------------------------------
// Decomposition without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code running under an external
// memory budget or pool that forbids new device allocations, callers that
// must not risk an allocation failure (or its implicit synchronisation) in
// the middle of their work, and drivers that only own the buffers they pass
// in.  For them the cascade keeps the scaling parts between levels in the
// fixed array below instead of a plan-owned workspace, takes its per-level
// parameters as kernel arguments and evaluates the wavelet phases in the
// kernel instead of reading plan tables.  The array lives in every GPU that
// loads this library until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchElems = size_t(1) << 21;  // complex64 elements: 16 MiB
__device__ __align__(256) float2 g_pwt_noalloc_scratch[kNoAllocScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
float2* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device pointer).
pfft_status noalloc_scratch(float2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PFFT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pwt_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PFFT_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<float2*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return PFFT_OK;
}
}  // namespace

extern "C" pfft_status pwt_decompose_noalloc(int d, const int64_t* M, int levels, const int64_t* J, int symbol,
                                             double eta, int64_t batch, const void* c_hat, void* scaling,
                                             void* const* wavelets, void* stream) {
  if (!M || !J || !c_hat || !scaling || !wavelets || d < 1 || d > 4 || levels < 1 || levels > 64 || batch < 1 ||
      batch > (int64_t(1) << 20) || (symbol != PWT_DIRICHLET && symbol != PWT_DLVP) ||
      (symbol == PWT_DLVP && !(eta > 0.0 && eta < 1.0)))
    return PFFT_ERR_ARG;
  for (int l = 0; l < levels; ++l)
    if (!wavelets[l]) return PFFT_ERR_ARG;
  pwt_plan_s P;  // host-side description only: plan_device is not called
  P.d = d;
  P.levels = levels;
  P.symbol = symbol;
  P.eta = eta;
  P.batch = batch;
  P.dtype = PFFT_C64;
  pfft_status st;
  try {
    st = plan_levels(P, M, J);
  } catch (const LatticeError& e) {
    st = pfft_status(e.code);
  }
  if (st != PFFT_OK) return st;
  if (P.sizes[0] * batch >= (int64_t(1) << 40)) return PFFT_ERR_OVERFLOW;  // as pwt_plan_create
  // two ping-pong halves of the scratch hold the scaling parts of levels < L
  const size_t half = kNoAllocScratchElems / 2;
  if (levels > 1 && size_t(P.sizes[0] / 2) * size_t(batch) > half) return PFFT_ERR_OVERFLOW;
  float2* scratch = nullptr;
  if (levels > 1) {
    st = noalloc_scratch(&scratch);
    if (st != PFFT_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const void* cur = c_hat;
  for (int l = 0; l < levels; ++l) {
    void* d1 = (l == levels - 1) ? scaling : static_cast<void*>(scratch + (l & 1) * half);
    const LevelDesc& L = P.lv[l];
    unsigned gx, gy;
    int chunk;
    split_grid(L.mN, int(batch), gx, gy, chunk);
    dim3 grid(gx, gy);
    const float2* src = static_cast<const float2*>(cur);
    float2* o1 = static_cast<float2*>(d1);
    float2* o2 = static_cast<float2*>(wavelets[l]);
    if (L.small)
      split_kernel<float2, 0, false, true><<<grid, 256, 0, s>>>(L, int(batch), chunk, src, nullptr, nullptr, nullptr, o1,
                                                                o2);
    else
      split_kernel<float2, 0, false, false><<<grid, 256, 0, s>>>(L, int(batch), chunk, src, nullptr, nullptr, nullptr, o1,
                                                                  o2);
    if (cudaGetLastError() != cudaSuccess) return PFFT_ERR_CUDA;
    cur = d1;
  }
  return PFFT_OK;
}
