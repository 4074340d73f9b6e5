// Split step (Section 5.3, step 4) by a dilation J whose group G(J^T) is
// cyclic of order p = |det J|, with a built-in unitary band system: the
// periodised Dirichlet scaling symbol of Section 6.2 for any p and p - 1
// band symbols completing it on every fibre.
//
// Fibres.  With l a generator of G(J^T) and v the functional with
// n in J^T Z^d <=> v . n = 0 (mod p) and v . l = 1, the fibre of g in G(N^T)
// is h_t = g + t N^T l (t < p).  Let tau = N^{-T} g.  The Dirichlet weight of
// member t is
//     w_t = sum over k in Z^d with v . k = t (mod p) of prod_j B(tau_j + k_j),
// B the indicator of [-1/2, 1/2] with 1/2 on the boundary: the shifts t l +
// J^T Z^d of the periodisation over J^T Z^d run through the residues of v . k.
// Only k with |tau_j + k_j| <= 1/2 contribute, so at most 2^d members of a
// fibre carry weight, and they are found without visiting the others.
//
// Band system.  u_t = sqrt(w_t) is a unit vector (the weights of a fibre sum
// to 1).  U = 2 V V^T / (V^T V) - I with V = u + e_0 is real, orthogonal and
// symmetric with first row u (V^T V = 2 + 2 u_0 > 0).  The symbols are
// b_j(h_t) = sqrt(p) U[j][t] e^j, e = exp(-2 pi i g^T N^{-1} z), z the
// generator of the pattern P(J) (centred) with l^T z = 1/p: b_0 = A =
// sqrt(p w) is the scaling symbol, and for p = 2 (b_0, b_1) is the scaling /
// wavelet pair of Section 6.2.  The analysis of step 4 with conjugated
// symbols is then
//     d_j[g] = conj(e^j) x_j,   x = U c = 2 V (V . c) / (V^T V) - c,
// and, (b_j(h_t) / sqrt(p)) being unitary, its inverse (the adjoint) is
// c = U y with y_j = e^j d_j[g].  O(p + 2^d) work per fibre.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/pfft.h"
#include "device_common.cuh"

namespace pfft {

constexpr int kPrimeChunk = 16;  // band outputs per work item
constexpr int kPrimeMaxW = 16;   // members with non-zero weight (2^d, d <= 4)

struct alignas(16) PrimeDesc {
  int d, p;
  int mM, mN;              // points of G(M^T) and of G(N^T)
  BoxDesc HM;              // box of H(M^T)
  int HNext[4];            // extents of the box of H(N^T)
  FastDiv divHN[4];
  int shift[4];            // box(H(M^T)) point of N^T l
  long long K[16];         // sign(det M) J^T adj(M^T): N^{-T} h = K h / q
  long long q;             // |det M|
  long long v[4];          // n in J^T Z^d <=> v . n = 0 mod p; v . l = 1
  long long phw[4];        // sign(det M) adj(M) (J z) mod q: phase numerator of g is g . phw
  int nch;                 // chunks of kPrimeChunk band outputs per fibre
};

// Box point g + t s reduced into the box of H (coordinates of g, s in the
// box, 0 <= t < 2^20): last coordinate first, exact in 64 bits.
__device__ __forceinline__ void prime_member(const BoxDesc& H, const int* g, const int* s, int t, int* y) {
  long long w[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) w[r] = r < H.d ? (long long)g[r] + (long long)t * s[r] : 0;
#pragma unroll
  for (int r = 3; r >= 0; --r) {
    if (r < H.d) {
      const long long h = H.H[r][r];
      long long qd = w[r] / h;
      if (w[r] - qd * h < 0) --qd;
      if (qd != 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i <= r) w[i] -= qd * H.H[i][r];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) y[r] = int(w[r]);
}

__device__ __forceinline__ int prime_slot(const BoxDesc& H, const int* y) {
  int s = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (r < H.d) s += y[r] * H.stride[r];
  return s;
}

// Members of the fibre of g with non-zero weight: tm[i], u_i = sqrt(w_i);
// returns their count (distinct members, weights merged).
template <typename Rl>
__device__ __forceinline__ int prime_weights(const PrimeDesc& P, const int* g, int* tm, Rl* um) {
  const int d = P.d;
  const long long q = P.q;
  long long k0[4];
  int two[4];
  Rl wh[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    k0[j] = 0;
    two[j] = 0;
    wh[j] = Rl(1);
    if (j < d) {
      long long a = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < d) a += P.K[j * d + i] * (long long)g[i];
      long long r = a % q;
      if (r < 0) r += q;
      const long long kk = (r - a) / q;  // a + kk q = r in [0, q)
      if (2 * r < q) {
        k0[j] = kk;
      } else if (2 * r > q) {
        k0[j] = kk - 1;
      } else {  // on the boundary: k = kk and kk - 1, weight 1/2 each
        k0[j] = kk - 1;
        two[j] = 1;
        wh[j] = Rl(0.5);
      }
    }
  }
  int n = 0;
  const int ncomb = 1 << (two[0] + two[1] + two[2] + two[3]);
  for (int c = 0; c < ncomb; ++c) {
    long long t = 0;
    Rl w = Rl(1);
    int bit = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j < d) {
        long long k = k0[j];
        if (two[j]) {
          k += (c >> bit) & 1;
          ++bit;
        }
        w *= wh[j];
        long long km = k % P.p;
        if (km < 0) km += P.p;
        t += (P.v[j] % P.p) * km;
      }
    }
    const int tt = int(t % P.p);
    int i = 0;
    while (i < n && tm[i] != tt) ++i;
    if (i == n) {
      tm[n] = tt;
      um[n] = Rl(0);
      ++n;
    }
    um[i] += w;
  }
  for (int i = 0; i < n; ++i) um[i] = sqrt(um[i]);
  return n;
}

// exp(-2 pi i t / q), 0 <= t < q, in the working precision from the exactly
// reduced numerator.
template <typename C>
__device__ __forceinline__ C prime_phase(long long t, long long q) {
  using Rl = decltype(C::x);
  if constexpr (std::is_same<Rl, double>::value) {
    double sn, cs;
    sincospi(2.0 * (double(t) / double(q)), &sn, &cs);
    return cmake<C>(cs, -sn);
  } else {
    float sn, cs;
    sincospif(2.0f * (float(t) / float(q)), &sn, &cs);
    return cmake<C>(cs, -sn);
  }
}

// One work item: fibre gs of G(N^T), band outputs [j0, j0 + kPrimeChunk) of
// one signal: coefficients cin / cout (the signal's base), band 0 (the
// scaling part) at d0 and band j >= 1 at dw + (j - 1) dstride (pointers at
// fibre gs).  MODE 0: analysis c -> bands; MODE 1: synthesis bands -> c.
template <typename C, int MODE, bool COH = false>
__device__ __forceinline__ void prime_split_item(const PrimeDesc& P, int gs, int j0, const C* __restrict__ cin,
                                                 C* __restrict__ cout, const C* __restrict__ din0,
                                                 const C* __restrict__ dinw, C* __restrict__ dout0,
                                                 C* __restrict__ doutw, long long dstride) {
  using Rl = decltype(C::x);
  int g[4] = {0, 0, 0, 0};
  {
    int s = gs;
    for (int r = P.d - 1; r >= 0; --r) {
      const int qd = P.divHN[r].div(s);
      g[r] = s - qd * P.HNext[r];
      s = qd;
    }
  }
  int tm[kPrimeMaxW];
  Rl um[kPrimeMaxW];
  const int nw = prime_weights<Rl>(P, g, tm, um);
  Rl u0 = Rl(0);
  for (int i = 0; i < nw; ++i)
    if (tm[i] == 0) u0 = um[i];
  const Rl coef = Rl(2) / (Rl(2) + Rl(2) * u0);  // 2 / (V^T V)
  long long num = 0;                            // phase numerator of g
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (r < P.d) num += ((long long)g[r] * P.phw[r]) % P.q;
  num %= P.q;
  if (num < 0) num += P.q;
  // sigma = V . c (analysis) or V . y (synthesis): member 0 and the weighted members
  C sig = cmake<C>(0, 0);
  {
    int y[4];
    prime_member(P.HM, g, P.shift, 0, y);
    C x0 = MODE == 0 ? load_c<COH>(cin + prime_slot(P.HM, y)) : din0[0];
    sig = x0;  // the e_0 part of V
    for (int i = 0; i < nw; ++i) {
      const int t = tm[i];
      C xt;
      if (MODE == 0) {
        prime_member(P.HM, g, P.shift, t, y);
        xt = load_c<COH>(cin + prime_slot(P.HM, y));
      } else {
        const C dt = t == 0 ? din0[0] : dinw[(long long)(t - 1) * dstride];
        xt = cmul(dt, prime_phase<C>((long long)t * num % P.q, P.q));
      }
      sig = cadd(sig, cscale(xt, um[i]));
    }
  }
  const int j1 = min(j0 + kPrimeChunk, P.p);
  int y[4];
  prime_member(P.HM, g, P.shift, j0, y);
  for (int j = j0; j < j1; ++j) {
    Rl vj = Rl(j == 0);
    for (int i = 0; i < nw; ++i)
      if (tm[i] == j) vj += um[i];
    const int sl = prime_slot(P.HM, y);
    const C e = prime_phase<C>((long long)j * num % P.q, P.q);
    if (MODE == 0) {
      const C xj = csub(cscale(sig, coef * vj), load_c<COH>(cin + sl));
      (j == 0 ? dout0 : doutw + (long long)(j - 1) * dstride)[0] = cmul(cconj(e), xj);
    } else {
      const C yj = cmul((j == 0 ? din0 : dinw + (long long)(j - 1) * dstride)[0], e);
      cout[sl] = csub(cscale(sig, coef * vj), yj);
    }
    if (j + 1 < j1) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (r < P.d) y[r] += P.shift[r];
      box_fix(P.HM, y);
    }
  }
}

// Host (split_general.cu): the descriptor of one split level of M by J with the
// built-in band system (G(J^T) cyclic, 2 <= |det J| <= 2^20, |det M| < 2^30).
pfft_status describe_prime_level(int d, const int64_t* M, const int64_t* J, PrimeDesc* out);

}  // namespace pfft
