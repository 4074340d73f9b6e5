// Device side of the wavelet split step (Section 5.3, step 4): the level
// descriptor, the periodised symbol weights, the wavelet phase and the
// per-fibre butterfly, shared by the plan-based launches (wavelet.cu) and the
// grouped launches of pattern batches (batch_kernels.cu).  The derivation of
// the symbol evaluation is given at the top of wavelet.cu.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/pfft.h"
#include "device_common.cuh"

namespace pfft {

constexpr int kLoBits = 11;

struct LevelDesc {
  int d;
  int mN;                // points of G(N^T)
  int mM;                // points of G(M^T)
  BoxDesc HM;            // box of H(M^T)
  int HNext[4];          // extents of the box of H(N^T)
  FastDiv divHN[4];
  int shift1[4];         // box(H(M^T)) point of N^T l1
  long long adjMT[16];   // adj(M^T)
  long long q;           // |det M|
  int sM;                // sign det M
  int J[16];
  long long adjJT[16];
  int aJ;                // |det J|
  long long phw[4];      // adj(M) (J z): phase numerator of h is sM * h . phw mod q
  int symbol;
  double eta;
  long long K[16];       // sign(det M) J^T adj(M^T): N^{-T} h = K h / q
  int K32[16];           // the same in int32 when `small`
  int small;             // |K h| < 2^30 for every box point h: int32 arithmetic
  int vpar[4];           // parity vector of J^T Z^d
  FastDiv div2q;         // division by 2q (int32 path)
  int off2q;             // multiple of 2q that makes K h non-negative (int32 path)
  int ph32[4];           // sign(det M) adj(M) (J z) mod q (int32 path)
  FastDiv divq;          // division by q (int32 path)
  int offq;              // multiple of q that makes ph32 . h non-negative
  const void* tab_lo;    // exp(-2 pi i t / q), t < 2^kLoBits
  const void* tab_hi;    // exp(-2 pi i (t << kLoBits) / q)
  // per-fibre symbols of the fused launches, by slot of G(N^T): float4
  // (A(h0), A(h1), conjugate phase) for complex64, or null (evaluated in place)
  const void* symtab;
  // Smith-coordinate order of the coefficients on G(M^T) (first level of a
  // plan created with PWT_FLAG_INPUT_SNF): the slot of h is the row-major
  // index of mu(h) = (MU_j . h mod n_j) over the snf_D non-trivial cycles,
  // and mu(h + N^T l1) = mu(h) + mu_l1 (mu is additive on G(M^T)).
  int snf_D;             // 0: box order of H(M^T)
  int snf_n[4];
  int snf_str[4];
  long long snf_mu[4][4];  // MU_j (reduced mod n_j), one row per cycle
  int snf_l1[4];           // mu(N^T l1)
};

// Periodised weight w(N^{-T} h) of the point h (see the header comment);
// the fibre partner has weight 1 - w.
template <typename Rl, bool SMALL>
__device__ __forceinline__ Rl fibre_weight(const LevelDesc& L, const int* h) {
  using I = typename std::conditional<SMALL, int, long long>::type;
  const int d = L.d;
  const I q = I(L.q);
  Rl prod = Rl(1);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j >= d) break;
    I t;  // numerator of (N^{-T} h)_j mod 2, in [0, 2q)
    if constexpr (SMALL) {
      int acc = L.off2q;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < d) acc += L.K32[j * d + i] * h[i];
      t = L.div2q.mod(acc);
    } else {
      long long acc = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < d) acc += L.K[j * d + i] * (long long)h[i];
      t = acc % (2 * q);
      if (t < 0) t += 2 * q;
    }
    Rl U = Rl(0);
#pragma unroll
    for (int n = 0; n >= -2; --n) {  // shifts with |t/q + n| possibly < 1
      const I sn = t + I(n) * q;
      const I an = sn < 0 ? -sn : sn;
      Rl b;
      if (L.symbol == PWT_DIRICHLET) {
        b = (2 * an < q) ? Rl(1) : (2 * an == q) ? Rl(0.5) : Rl(0);
      } else {
        const Rl eta = Rl(L.eta);
        b = (Rl(0.5) * (Rl(1) + eta) - Rl(an) / Rl(q)) / eta;
        b = b < Rl(0) ? Rl(0) : (b > Rl(1) ? Rl(1) : b);
      }
      U += ((L.vpar[j] & n) & 1) ? -b : b;
    }
    prod *= U;
  }
  return Rl(0.5) * (Rl(1) + prod);
}

template <typename C, bool TAB = true, bool SMALL = false>
__device__ __forceinline__ C wavelet_phase(const LevelDesc& L, const int* h) {
  long long t = 0;
  if constexpr (SMALL) {
    int acc = L.offq;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < L.d) acc += L.ph32[i] * h[i];
    t = L.divq.mod(acc);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)  // each product < 2^62; reduce term by term
      if (i < L.d) t += ((long long)h[i] * L.phw[i]) % L.q;
    t = (L.sM * t) % L.q;
    if (t < 0) t += L.q;
  }
  if constexpr (!TAB) {
    // no tables: sincospi, in the working precision, of the exactly reduced
    // fraction t / q
    using Rl = decltype(C::x);
    if constexpr (std::is_same<Rl, double>::value) {
      double sn, cs;
      sincospi(2.0 * (double(t) / double(L.q)), &sn, &cs);
      return cmake<C>(cs, -sn);
    } else {
      float sn, cs;
      sincospif(2.0f * (float(t) / float(L.q)), &sn, &cs);
      return cmake<C>(cs, -sn);
    }
  }
  const C* lo = static_cast<const C*>(L.tab_lo);
  const C* hi = static_cast<const C*>(L.tab_hi);
  return cmul(hi[t >> kLoBits], lo[t & ((1 << kLoBits) - 1)]);
}

// mode 0: decompose c -> (d1, d2); 1: reconstruct; 2: adjoint, for the
// fibre of slot gs of the box of H(N^T) in each of `batch` signals (signal b
// at c + b mM, d + b mN).  The symbols depend on the fibre only: they are
// evaluated once and applied to every signal.
template <typename C, int MODE, bool TAB, bool SMALL, bool COH = false>
__device__ __forceinline__ void split_fibre(const LevelDesc& L, int gs, int batch, const C* __restrict__ cin,
                                            C* __restrict__ cout, const C* __restrict__ d1in,
                                            const C* __restrict__ d2in, C* __restrict__ d1out,
                                            C* __restrict__ d2out) {
  using Rl = decltype(C::x);
  int g[4] = {0, 0, 0, 0}, h1[4] = {0, 0, 0, 0};
  int s = gs;
  for (int r = L.d - 1; r >= 0; --r) {
    const int qd = L.divHN[r].div(s);
    g[r] = s - qd * L.HNext[r];
    s = qd;
  }
  int slot0 = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (r < L.d) {
      h1[r] = g[r] + L.shift1[r];
      slot0 += g[r] * L.HM.stride[r];
    }
  }
  box_fix(L.HM, h1);
  int slot1 = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (r < L.d) slot1 += h1[r] * L.HM.stride[r];
  if (L.snf_D) {  // coefficients on G(M^T) in Smith-coordinate order
    slot0 = slot1 = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j >= L.snf_D) break;
      long long acc = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < L.d) acc += L.snf_mu[j][c] * g[c];
      const int mu0 = int(acc % L.snf_n[j]);
      int mu1 = mu0 + L.snf_l1[j];
      if (mu1 >= L.snf_n[j]) mu1 -= L.snf_n[j];
      slot0 += mu0 * L.snf_str[j];
      slot1 += mu1 * L.snf_str[j];
    }
  }
  Rl A0, A1;
  C e0;
  bool tabulated = false;
  if constexpr (sizeof(Rl) == 4) {
    if (L.symtab) {  // the plan's per-fibre symbols: A(h0), A(h1), conj(e(h0))
      const float4 t = __ldg(static_cast<const float4*>(L.symtab) + gs);
      A0 = t.x;
      A1 = t.y;
      e0 = cmake<C>(t.z, -t.w);
      tabulated = true;
    }
  }
  if (!tabulated) {
    const Rl w0 = fibre_weight<Rl, SMALL>(L, g);
    const Rl w1 = Rl(1) - w0;
    if (L.symbol == PWT_DIRICHLET) {
      A0 = sqrt(Rl(2) * w0);
      A1 = sqrt(Rl(2) * w1);
    } else {
      A0 = Rl(1.41421356237309504880) * w0;
      A1 = Rl(1.41421356237309504880) * w1;
    }
    e0 = wavelet_phase<C, TAB, SMALL>(L, g);
  }
  // B(h0) = A(h1) e(h0), B(h1) = A(h0) e(h1), e(h1) = -e(h0)
  const Rl r2 = Rl(0.70710678118654752440);
  const long long mM = L.mM, mN = L.mN;
  if (MODE == 0) {
    const C ce = cconj(e0);
#pragma unroll 4
    for (int b = 0; b < batch; ++b) {
      const C c0 = load_c<COH>(cin + b * mM + slot0), c1 = load_c<COH>(cin + b * mM + slot1);
      d1out[b * mN + gs] = cscale(cadd(cscale(c0, A0), cscale(c1, A1)), r2);
      // conj(B0) c0 + conj(B1) c1 = conj(e0) (A1 c0 - A0 c1)
      d2out[b * mN + gs] = cscale(cmul(ce, csub(cscale(c0, A1), cscale(c1, A0))), r2);
    }
  } else {
    const Rl S = A0 * A0 + A1 * A1;
    const Rl fac = (MODE == 1) ? Rl(1.41421356237309504880) / S : r2;
#pragma unroll 4
    for (int b = 0; b < batch; ++b) {
      const C a = d1in[b * mN + gs], bb = d2in[b * mN + gs];
      const C eb = cmul(e0, bb);
      cout[b * mM + slot0] = cscale(cadd(cscale(a, A0), cscale(eb, A1)), fac);
      cout[b * mM + slot1] = cscale(csub(cscale(a, A1), cscale(eb, A0)), fac);
    }
  }
}

// One thread per fibre g (grid-stride over the slots of the box of H(N^T));
// blockIdx.y takes the signals [y chunk, (y + 1) chunk) of the batch in turn
// (one chunk holds the whole batch unless the level has few fibres).
template <typename C, int MODE, bool TAB = true, bool SMALL = false>
__global__ void __launch_bounds__(256) split_kernel(LevelDesc L, int batch, int chunk, const C* __restrict__ cin,
                                                    C* __restrict__ cout, const C* __restrict__ d1in,
                                                    const C* __restrict__ d2in, C* __restrict__ d1out,
                                                    C* __restrict__ d2out) {
  const int b0 = blockIdx.y * chunk;
  const int nb = min(chunk, batch - b0);
  if (nb <= 0) return;
  const long long oM = (long long)b0 * L.mM, oN = (long long)b0 * L.mN;
  for (int gs = blockIdx.x * blockDim.x + threadIdx.x; gs < L.mN; gs += gridDim.x * blockDim.x)
    split_fibre<C, MODE, TAB, SMALL>(L, gs, nb, MODE == 0 ? cin + oM : nullptr, MODE == 0 ? nullptr : cout + oM,
                                     MODE == 0 ? nullptr : d1in + oN, MODE == 0 ? nullptr : d2in + oN,
                                     MODE == 0 ? d1out + oN : nullptr, MODE == 0 ? d2out + oN : nullptr);
}

// Symbols of the fibre at box point g: A(h0), A(h1) and the conjugate
// wavelet phase (the analysis applies conj(e)).
template <typename C>
__device__ __forceinline__ void fibre_symbols(const LevelDesc& L, const int* g, decltype(C::x)& a0,
                                              decltype(C::x)& a1, C& ph) {
  using Rl = decltype(C::x);
  const Rl w = fibre_weight<Rl, true>(L, g);
  if (L.symbol == PWT_DIRICHLET) {
    a0 = sqrt(Rl(2) * w);
    a1 = sqrt(Rl(2) * (Rl(1) - w));
  } else {
    a0 = Rl(1.41421356237309504880) * w;
    a1 = Rl(1.41421356237309504880) * (Rl(1) - w);
  }
  ph = cconj(wavelet_phase<C, true, true>(L, g));
}

// The symbol table of one level (int32 index path): one float4 per fibre,
// by its slot in the box of H(N^T).
template <typename C>
__global__ void __launch_bounds__(256) symbol_table_kernel(LevelDesc L, float4* __restrict__ tab) {
  for (int gs = blockIdx.x * blockDim.x + threadIdx.x; gs < L.mN; gs += gridDim.x * blockDim.x) {
    int g[4] = {0, 0, 0, 0};
    int s = gs;
    for (int r = L.d - 1; r >= 0; --r) {
      const int qd = L.divHN[r].div(s);
      g[r] = s - qd * L.HNext[r];
      s = qd;
    }
    float a0, a1;
    C ph;
    fibre_symbols<C>(L, g, a0, a1, ph);
    tab[gs] = make_float4(a0, a1, ph.x, ph.y);
  }
}

// ---- Several levels in one launch (the repetition of steps 2-4 at the end
// of Section 5.3).  After F levels, a fibre g of G(N_F^T) (the last level's
// output) draws on 2^F coefficients of the first level's input: its two
// members are fibres of level F - 1, theirs of level F - 2, and so on.  One
// thread takes g, reads those 2^F inputs once per signal, runs the 2^F - 1
// butterflies of the tree level by level and writes every wavelet part once
// and the last scaling part; the scaling parts of the inner levels never
// leave registers.  The symbols depend on the fibres only: each thread
// takes them once per g (top-down, so that only the box points of the
// current level are live) from the plan's per-fibre symbol table (or
// evaluates them) into its column of shared-memory tables and applies them
// to every signal of its chunk, two signals at a time so that the loads of
// both are in flight together.
constexpr int kFuseThreads = 128;
constexpr int kFuseMax = 3;   // levels per launch (4 needs more registers than pays off)
constexpr int kFuseWaves = 8; // resident waves of CTAs for the fibres

// Dynamic shared memory of fused_split_kernel<C, F>: per thread and fibre of
// the tree (2^F - 1) the symbols (A(h0), A(h1), conjugate phase) and the
// output slot, per member of the first level (2^F) the input slot.
template <typename C, int F>
__host__ __device__ constexpr int fused_smem_bytes() {
  return kFuseThreads * (((1 << F) - 1) * (4 * int(sizeof(decltype(C::x))) + 4) + (1 << F) * 4);
}

// F levels of the analysis (mode 0) starting at the level whose descriptor is
// lvg[0]: inputs cin (the first level's coefficients), wavelet parts of level
// k at w_k, the last scaling part at sout; signals [y chunk, (y + 1) chunk).
// Every level of the group has the int32 index path (`small`).
template <typename C, int F>
__global__ void __launch_bounds__(kFuseThreads, 4)
    fused_split_kernel(const LevelDesc* __restrict__ lvg, int batch, int chunk, const C* __restrict__ cin,
                       C* __restrict__ sout, C* __restrict__ w0, C* __restrict__ w1, C* __restrict__ w2) {
  using Rl = decltype(C::x);
  constexpr int NT = kFuseThreads;
  constexpr int NL = 1 << (F - 1);   // fibres of the first level per thread
  constexpr int FIB = (1 << F) - 1;  // fibres of the tree
  constexpr int SG = 2;              // signals per iteration
  __shared__ LevelDesc lv[F];
  extern __shared__ __align__(16) unsigned char fsm[];
  // per-thread tables, thread index fastest: symbols [FIB][4][NT] (A0, A1,
  // phase), output slots [FIB][NT], input slots [2^F][NT]
  Rl* sym = reinterpret_cast<Rl*>(fsm);
  int* osl = reinterpret_cast<int*>(fsm + size_t(FIB) * NT * 4 * sizeof(Rl));
  int* isl = osl + FIB * NT;
  static_assert(sizeof(LevelDesc) % 4 == 0, "level descriptors are copied as 32-bit words");
  for (int i = threadIdx.x; i < int(F * sizeof(LevelDesc) / 4); i += blockDim.x)
    reinterpret_cast<int*>(lv)[i] = __ldg(reinterpret_cast<const int*>(lvg) + i);
  __syncthreads();
  const int b0 = blockIdx.y * chunk;
  const int nb = min(chunk, batch - b0);
  if (nb <= 0) return;
  const LevelDesc& Lt = lv[F - 1];
  C* const wout[3] = {w0, w1, w2};
  const int tid = threadIdx.x;
  // fibre i of level k has the flat index 2^(F-1-k) - 1 + i in the tables
  for (int gs = blockIdx.x * NT + tid; gs < Lt.mN; gs += gridDim.x * NT) {
    int cur[NL][4];
    {
      int s = gs;
#pragma unroll
      for (int r = 3; r >= 0; --r) {
        cur[0][r] = 0;
        if (r < Lt.d) {
          const int qd = Lt.divHN[r].div(s);
          cur[0][r] = s - qd * Lt.HNext[r];
          s = qd;
        }
      }
    }
#pragma unroll
    for (int k = F - 1; k >= 0; --k) {
      const LevelDesc& L = lv[k];
#pragma unroll
      for (int i = 0; i < (1 << (F - 1 - k)); ++i) {
        const int f = (1 << (F - 1 - k)) - 1 + i;
        int sl = 0, str = 1;
#pragma unroll
        for (int r = 3; r >= 0; --r)
          if (r < L.d) {
            sl += cur[i][r] * str;
            str *= L.HNext[r];
          }
        osl[f * NT + tid] = sl;
        Rl a0, a1;
        C ph;
        if constexpr (sizeof(Rl) == 4) {
          if (L.symtab) {
            const float4 t = __ldg(static_cast<const float4*>(L.symtab) + sl);
            a0 = t.x;
            a1 = t.y;
            ph = cmake<C>(t.z, t.w);
          } else {
            fibre_symbols<C>(L, cur[i], a0, a1, ph);
          }
        } else {
          fibre_symbols<C>(L, cur[i], a0, a1, ph);
        }
        sym[(4 * f + 0) * NT + tid] = a0;
        sym[(4 * f + 1) * NT + tid] = a1;
        sym[(4 * f + 2) * NT + tid] = ph.x;
        sym[(4 * f + 3) * NT + tid] = ph.y;
      }
      // the members of this level's fibres: the fibres of level k - 1 (for
      // k = 0, the input slots); highest first, so that cur[i] is read
      // before cur[2 i], cur[2 i + 1] overwrite it
#pragma unroll
      for (int i = (1 << (F - 1 - k)) - 1; i >= 0; --i) {
        int h1[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) h1[r] = cur[i][r] + (r < L.d ? L.shift1[r] : 0);
        box_fix(L.HM, h1);
        if (k == 0) {
          int s0 = 0, s1 = 0;
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (r < L.d) {
              s0 += cur[i][r] * L.HM.stride[r];
              s1 += h1[r] * L.HM.stride[r];
            }
          isl[(2 * i) * NT + tid] = s0;
          isl[(2 * i + 1) * NT + tid] = s1;
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            cur[2 * i + 1][r] = h1[r];
            cur[2 * i][r] = cur[i][r];
          }
        }
      }
    }
    const Rl r2 = Rl(0.70710678118654752440);
    for (int bb = 0; bb < nb; bb += SG) {
      C v[SG][2 * NL];
#pragma unroll
      for (int j = 0; j < SG; ++j)
        if (j == 0 || bb + j < nb) {
#pragma unroll
          for (int i = 0; i < 2 * NL; ++i)
            v[j][i] = cin[(long long)(b0 + bb + j) * lv[0].mM + isl[i * NT + tid]];
        }
#pragma unroll
      for (int k = 0; k < F; ++k) {
#pragma unroll
        for (int i = 0; i < (1 << (F - 1 - k)); ++i) {
          const int f = (1 << (F - 1 - k)) - 1 + i;
          const Rl a0 = sym[(4 * f + 0) * NT + tid], a1 = sym[(4 * f + 1) * NT + tid];
          const C ph = cmake<C>(sym[(4 * f + 2) * NT + tid], sym[(4 * f + 3) * NT + tid]);
          const int os = osl[f * NT + tid];
#pragma unroll
          for (int j = 0; j < SG; ++j)
            if (j == 0 || bb + j < nb) {
              const C c0 = v[j][2 * i], c1 = v[j][2 * i + 1];
              const C d1 = cscale(cadd(cscale(c0, a0), cscale(c1, a1)), r2);
              const C d2 = cscale(cmul(ph, csub(cscale(c0, a1), cscale(c1, a0))), r2);
              wout[k][(long long)(b0 + bb + j) * lv[k].mN + os] = d2;
              v[j][i] = d1;
            }
        }
      }
#pragma unroll
      for (int j = 0; j < SG; ++j)
        if (j == 0 || bb + j < nb) sout[(long long)(b0 + bb + j) * Lt.mN + gs] = v[j][0];
    }
  }
}

// Launch shape of split_kernel: enough fibre CTAs for about 8 resident waves,
// and the signals split into chunks only when the fibres alone are too few.
inline void split_grid(long long mN, int batch, unsigned& gx, unsigned& gy, int& chunk) {
  long long x = (mN + 255) / 256;
  if (x > 152LL * 8) x = 152LL * 8;
  if (x < 1) x = 1;
  long long y = (152LL * 8 + x - 1) / x;
  if (y > batch) y = batch;
  if (y < 1) y = 1;
  chunk = int((batch + y - 1) / y);
  gy = unsigned((batch + chunk - 1) / chunk);
  gx = unsigned(x);
}

// Host (wavelet.cu): elements of the two-level phase table of a level, and its
// construction at `tab` (sets tab_lo / tab_hi; 0 on success).
size_t split_table_elems(const LevelDesc& L);
int launch_split_tables(LevelDesc& L, void* tab, int dtype);
// The per-fibre symbol table of a complex64 level with the int32 index path
// (L.small, phase tables built): L.mN float4 at `tab`, set as L.symtab
// (0 on success).
int launch_symbol_table(LevelDesc& L, void* tab);

// Host: the descriptor of one split level of M by J (wavelet.cu).
pfft_status describe_split_level(int d, const int64_t* M, const int64_t* J, int symbol, double eta,
                                 LevelDesc* out);

}  // namespace pfft
