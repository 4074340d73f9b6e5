// Transform kernel templates for sm_103a: the row pass and the column pass of the
// Kronecker factorisation in Smith coordinates (Theorem 1, eq. (KroneckerFFT)),
// each a batched Stockham autosort DFT held in shared memory, with the
// bit-exact gather / scatter between the Hermite boxes and the Smith
// coordinates fused into the global loads and stores.
#pragma once
#include <cuda_runtime.h>

#include "fft_plan.hpp"

namespace pfft {

// Shared-memory index with one padding element per 16, which keeps the
// stride-R writes of the first radix stages free of bank conflicts.  Passes
// with direct prime stages run unpadded (PAD = false): those stages read
// consecutive addresses across a warp anyway and walk their inputs with
// pointer increments.
template <bool PAD>
__device__ __forceinline__ int phys(int x) { return PAD ? x + (x >> 4) : x; }

}  // namespace pfft
#include "fft_tc.cuh"
namespace pfft {

// Multiply v[r] by w^r, w = tw[base], r = 1..R-1.  The powers w^(2^b) come
// from the table and w^r is their product over the set bits of r, so every
// factor carries at most log2(R) - 1 rounded multiplications.
template <typename C, int R>
__device__ __forceinline__ void apply_twiddles(C* v, const C* __restrict__ tw, int base) {
  constexpr int NB = (R > 16) ? 5 : (R > 8) ? 4 : (R > 4) ? 3 : (R > 2) ? 2 : 1;
  C pw[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) pw[b] = __ldg(tw + (base << b));
#pragma unroll
  for (int r = 1; r < R; ++r) {
    C f;
    bool first = true;
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (r & (1 << b)) {
        f = first ? pw[b] : cmul(f, pw[b]);
        first = false;
      }
    v[r] = cmul(v[r], f);
  }
}

// One Stockham stage of radix R over every pencil of the tile.  Element
// (pencil t, index i) lives at i*T + t (column pass, COLS) or t*L + i (row
// pass).  Butterfly j of the axis reads i = base + (j + r a/R) sigma and,
// after the twiddles exp(-2 pi i k r / (Ns R)) (k = j mod Ns) and the
// length-R DFT, writes i = base + ((j - k) R + k + r Ns) sigma.
template <typename C, int R, int NB, bool COLS, bool PAD>
__device__ __forceinline__ void run_stage(C* sm, const PassArgs& a, const StageDesc& s,
                                          const C* __restrict__ tw) {
  const int per_pencil = a.L / R;
  const int total = a.T * per_pencil;
  const int escale = COLS ? a.T : 1;
  C v[NB][R];
  int obase[NB];
  int ostep = s.Ns * s.sigma * escale;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    obase[q] = -1;
    if (b < total) {
      int t, rest;
      if (COLS) {
        rest = a.divT.div(b);
        t = b - rest * a.T;
      } else {
        t = b / per_pencil;
        rest = b - t * per_pencil;
      }
      const int o = s.div_aR.div(rest);
      const int j = rest - o * s.aR;
      const int hi = s.div_sigma.div(o);
      const int base = hi * s.a * s.sigma + (o - hi * s.sigma);
      const int k = j - s.div_Ns.div(j) * s.Ns;
      const int ebase = COLS ? base * a.T + t : t * a.L + base;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = sm[phys<PAD>(ebase + (j + r * s.aR) * s.sigma * escale)];
      if (s.Ns > 1) apply_twiddles<C, R>(v[q], tw, k * s.twstep);
      obase[q] = ebase + ((j - k) * R + k) * s.sigma * escale;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    if (obase[q] >= 0) {
      dft<C, R>(v[q], tw, a.tw_n);
#pragma unroll
      for (int r = 0; r < R; ++r) sm[phys<PAD>(obase[q] + r * ostep)] = v[q][r];
    }
  }
  __syncthreads();
}

// One stage of a prime radix R >= 11, evaluated directly, in the order of a
// primitive root g of R.  With x'_r = x_r exp(-2 pi i r k / (Ns R))
// (k = j mod Ns; none when Ns = 1), h = (R - 1) / 2 and r_m = g^m mod R, so
// that R - r_m = r_{m+h}, a pre-pass forms
//     a_m = x'_{r_m} + x'_{R - r_m},   b_m = x'_{r_m} - x'_{R - r_m},   m < h,
// and stores them at slots 1 + m and 1 + h + m of the butterfly (slot 0 keeps
// x_0).  For an output q = r_n (n < h), r_m q = g^{m+n}, so with the table
// P[t] = omega_R^{g^t} = c_t - i s_t (t < R - 1)
//     y_q     = x_0 + sum_m (a_m c_{m+n} - i b_m s_{m+n}),
//     y_{R-q} = x_0 + sum_m (a_m c_{m+n} + i b_m s_{m+n}),
// because omega_R^{(R - r) q} is the conjugate of omega_R^{r q}; y_0 is x_0 plus
// the sum of the a_m.  A work item takes Q consecutive outputs n of one
// butterfly: per step m it reads a_m and b_m once (consecutive addresses
// across the lanes, which take consecutive butterflies) and Q table entries
// P[m + n] (broadcasts) for 4Q FMAs, with no index arithmetic.  Every read of
// a phase happens before the barrier that precedes its writes.
template <bool COLS>
__device__ __forceinline__ void direct_locate(const PassArgs& a, const StageDesc& s, int b, int& ebase, int& k,
                                              int& j) {
  const int per_pencil = a.L / s.R;
  int t, rest;
  if (COLS) {
    rest = a.divT.div(b);
    t = b - rest * a.T;
  } else {
    t = b / per_pencil;
    rest = b - t * per_pencil;
  }
  const int o = s.div_aR.div(rest);
  j = rest - o * s.aR;
  const int hi = s.div_sigma.div(o);
  const int base = hi * s.a * s.sigma + (o - hi * s.sigma);
  k = j - s.div_Ns.div(j) * s.Ns;
  ebase = COLS ? base * a.T + t : t * a.L + base;
}

// y_0 and the output pairs of a direct stage whose a_m, b_m are in place.
template <typename C, int NQ, int Q, bool COLS, bool PAD>
__device__ __noinline__ void direct_pairs(C* sm, const PassArgs& a, const StageDesc& s, const C* P, const int* gp) {
  using Rl = decltype(C::x);
  const int R = s.R;
  const int h = (R - 1) / 2;
  const int nbfly = a.T * (a.L / R);
  const int step = s.sigma * (COLS ? a.T : 1);
  const int istep = s.aR * step;
  const int nthr = blockDim.x;
  const int nblk = (h + Q - 1) / Q;
  auto locate = [&](int b, int& ebase, int& k, int& j) { direct_locate<COLS>(a, s, b, ebase, k, j); };
  C y0s[kDirectZero];
  int z0[kDirectZero];
#pragma unroll
  for (int u = 0; u < kDirectZero; ++u) {
    const int b = threadIdx.x + u * nthr;
    z0[u] = -1;
    if (b < nbfly) {
      int ebase, k, j;
      locate(b, ebase, k, j);
      const int i0 = ebase + j * step;
      C acc0 = sm[phys<PAD>(i0)];
      for (int m = 0; m < h; ++m) acc0 = cadd(acc0, sm[phys<PAD>(i0 + (1 + m) * istep)]);
      y0s[u] = acc0;
      z0[u] = ebase + ((j - k) * R + k) * step;
    }
  }
  Rl acc[NQ][Q][4];
  int ob[NQ], n0[NQ];
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    const int w = threadIdx.x + u * nthr;
    ob[u] = -1;
    n0[u] = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) acc[u][i][0] = acc[u][i][1] = acc[u][i][2] = acc[u][i][3] = Rl(0);
    if (w < nbfly * nblk) {
      const int blk = w / nbfly;
      const int b = w - blk * nbfly;
      int ebase, k, j;
      locate(b, ebase, k, j);
      const int i0 = ebase + j * step;
      const C x0 = sm[phys<PAD>(i0)];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        acc[u][i][0] = x0.x;
        acc[u][i][2] = x0.y;
      }
      const C* pt = P + blk * Q;
      if constexpr (PAD) {
        for (int m = 0; m < h; ++m) {
          const C av = sm[phys<PAD>(i0 + (1 + m) * istep)];
          const C bv = sm[phys<PAD>(i0 + (1 + h + m) * istep)];
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const C wv = pt[m + i];
            acc[u][i][0] = fma(av.x, wv.x, acc[u][i][0]);
            acc[u][i][1] = fma(bv.y, wv.y, acc[u][i][1]);
            acc[u][i][2] = fma(av.y, wv.x, acc[u][i][2]);
            acc[u][i][3] = fma(bv.x, wv.y, acc[u][i][3]);
          }
        }
      } else {
        const C* pa = sm + i0 + istep;
        const C* pb = sm + i0 + (1 + h) * istep;
#pragma unroll 2
        for (int m = 0; m < h; ++m) {
          const C av = *pa, bv = *pb;
          pa += istep;
          pb += istep;
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const C wv = pt[m + i];  // (c, -s) of g^{m + n}
            acc[u][i][0] = fma(av.x, wv.x, acc[u][i][0]);
            acc[u][i][1] = fma(bv.y, wv.y, acc[u][i][1]);  // -sum b.im s
            acc[u][i][2] = fma(av.y, wv.x, acc[u][i][2]);
            acc[u][i][3] = fma(bv.x, wv.y, acc[u][i][3]);  // -sum b.re s
          }
        }
      }
      ob[u] = ebase + ((j - k) * R + k) * step;
      n0[u] = blk * Q;
    }
  }
  __syncthreads();
  const int ostep = s.Ns * step;
#pragma unroll
  for (int u = 0; u < kDirectZero; ++u)
    if (z0[u] >= 0) sm[phys<PAD>(z0[u])] = y0s[u];
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    if (ob[u] < 0) continue;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int n = n0[u] + i;
      if (n >= h) break;
      const int q = gp[n];
      sm[phys<PAD>(ob[u] + q * ostep)] = cmake<C>(acc[u][i][0] - acc[u][i][1], acc[u][i][2] + acc[u][i][3]);
      sm[phys<PAD>(ob[u] + (R - q) * ostep)] = cmake<C>(acc[u][i][0] + acc[u][i][1], acc[u][i][2] - acc[u][i][3]);
    }
  }
  __syncthreads();
}

template <typename C, int EPT, bool COLS, bool PAD>
__device__ __noinline__ void run_direct_stage(C* sm, const PassArgs& a, const StageDesc& s,
                                              const C* __restrict__ tw) {
  constexpr int NA = kDirectPre<EPT>;
  const int R = s.R;
  const int h = (R - 1) / 2;
  const int per_pencil = a.L / R;
  const int nbfly = a.T * per_pencil;
  const int nthr = blockDim.x;
  const int escale = COLS ? a.T : 1;
  const int step = s.sigma * escale;
  const int istep = s.aR * step;  // element distance of consecutive slots
  // tables after the tile: P[t] = omega_R^{g^t} (R - 1 complex), then g^t mod R (R - 1 int)
  C* P = sm + a.dir_off;
  int* gp = reinterpret_cast<int*>(P + (R - 1));
  const int wstride = a.tw_n / R;
  for (int e = threadIdx.x; e < R - 1; e += nthr) {
    int pw = 1, base = s.gen, x = e;  // g^e mod R by squaring (R <= 1021: products < 2^20)
    while (x) {
      if (x & 1) pw = pw * base % R;
      base = base * base % R;
      x >>= 1;
    }
    gp[e] = pw;
    P[e] = __ldg(tw + pw * wstride);
  }
  __syncthreads();
  auto locate = [&](int b, int& ebase, int& k, int& j) { direct_locate<COLS>(a, s, b, ebase, k, j); };
  // ---- pre-pass: read x_{r_m}, x_{R - r_m} (twiddled), then store a_m, b_m in m order
  {
    C av[NA], bv[NA];
    int dst[NA];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int w = threadIdx.x + u * nthr;
      dst[u] = -1;
      if (w < nbfly * h) {
        const int m = w / nbfly;
        const int b = w - m * nbfly;
        int ebase, k, j;
        locate(b, ebase, k, j);
        const int i0 = ebase + j * step;
        const int r = gp[m];
        C x0 = sm[phys<PAD>(i0 + r * istep)];
        C x1 = sm[phys<PAD>(i0 + (R - r) * istep)];
        if (s.Ns > 1) {  // r k < Ns R: no reduction
          x0 = cmul(x0, __ldg(tw + (r * k) * s.twstep));
          x1 = cmul(x1, __ldg(tw + ((R - r) * k) * s.twstep));
        }
        av[u] = cadd(x0, x1);
        bv[u] = csub(x0, x1);
        dst[u] = i0 + (1 + m) * istep;
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      if (dst[u] >= 0) {
        sm[phys<PAD>(dst[u])] = av[u];
        sm[phys<PAD>(dst[u] + h * istep)] = bv[u];
      }
    }
    __syncthreads();
  }
  // ---- y_0 = x_0 + sum_m a_m and the output pairs
  if (R >= kDirectQ4MinRadix)
    direct_pairs<C, kDirectQ4Items<EPT>, 4, COLS, PAD>(sm, a, s, P, gp);
  else
    direct_pairs<C, kDirectQ2Items<EPT>, 2, COLS, PAD>(sm, a, s, P, gp);
}

// The stages are grouped by radix in the fixed order of kRadixOrder (the
// planner sorts them so): the radices of one axis may run in any order in a
// Stockham DFT and different axes commute, and one loop per radix keeps the
// register allocation of each butterfly size separate (mixing sizes inside
// one loop body makes the allocator spill).  POW2 kernels carry only the
// power-of-two regions.
template <typename C, int EPT, bool COLS, bool POW2, bool PAD, bool TCK>
__device__ void run_all_stages(C* sm, const PassArgs& a, const C* __restrict__ tw) {
  int i = 0;
  constexpr bool kC64 = sizeof(C) == 8 && TCK;  // TCK = false: no tensor-core code in the kernel
  if constexpr (!POW2) {
    _Pragma("unroll 1") for (int q = 0; q < a.cnt[kDirectRegion]; ++q, ++i)
        run_direct_stage<C, EPT, COLS, PAD>(sm, a, a.st[i], tw);
  }
#define PFFT_REGION(RR, IDX)                                                     \
  _Pragma("unroll 1") for (int q = 0; q < a.cnt[IDX]; ++q, ++i)                  \
      run_stage<C, RR, (EPT / RR > 0 ? EPT / RR : 1), COLS, PAD>(sm, a, a.st[i], tw);
  bool tc16 = false;
#if defined(__CUDA_ARCH__)
  if constexpr (kC64) {
    if (a.tc) {
      // W tables, mbarrier and tensor memory (fft_tc.cuh), then the radix-32
      // and radix-16 stages on the tensor cores
      TcCtx cx;
      cx.base = reinterpret_cast<unsigned char*>(sm);
      cx.lay = tc_layout(a.tc_off, a.cnt[kTC32Region] > 0, a.cnt[0] > 0, a.T * a.L / 16);
      cx.phase = 0;
      cx.ok = 1;
      const int cols = tc_tmem_cols(a.T * a.L, a.cnt[kTC32Region] > 0, a.cnt[0] > 0);
      const float2* twf = reinterpret_cast<const float2*>(tw);
      if (a.cnt[kTC32Region]) tc_build_w<32>(cx.base + cx.lay.w32, twf, a.tw_n);
      if (a.cnt[0]) tc_build_w<16>(cx.base + cx.lay.w16, twf, a.tw_n);
      uint32_t* tslot = reinterpret_cast<uint32_t*>(cx.base + cx.lay.taddr);
      if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem_u32(cx.base + cx.lay.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      }
      if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc_smem_u32(tslot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // W tables -> tensor-core reads
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      cx.tmem = *tslot;
      float2* smf = reinterpret_cast<float2*>(sm);
      _Pragma("unroll 1") for (int q = 0; q < a.cnt[kTC32Region]; ++q, ++i)
          run_tc_stage<32, COLS, PAD>(smf, a, a.st[i], twf, cx);
      _Pragma("unroll 1") for (int q = 0; q < a.cnt[0]; ++q, ++i)
          run_tc_stage<16, COLS, PAD>(smf, a, a.st[i], twf, cx);
      tc16 = true;
      // every stage ends with tcgen05.fence::before_thread_sync and a barrier
      if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(cx.tmem), "r"(cols) : "memory");
      }
    }
  }
#endif
  if (!tc16) {
    PFFT_REGION(16, 0)
  }
  PFFT_REGION(8, 1)
  PFFT_REGION(4, 2)
  PFFT_REGION(2, 3)
  if constexpr (!POW2) {
    PFFT_REGION(3, 4)
    PFFT_REGION(5, 5)
    PFFT_REGION(7, 6)
  }
#undef PFFT_REGION
}


// Row pass: T rows of length nD per CTA, smem layout [t][e].  Each thread
// owns at most EPT elements of the tile: all of its global loads are issued
// before the first shared-memory write (and all shared reads before the
// first global store), so the loads of a thread are in flight together.
//
// The body takes the tile (blockIdx.x of a plain launch) and the signal index
// (blockIdx.y) as arguments so that the grouped launches of many patterns
// (batch_kernels.cu) run the same code on a per-CTA copy of the arguments.
template <typename C, int EPT, bool POW2, bool PAD, bool TCK = true>
__device__ __forceinline__ void row_pass_body(const PassArgs& a, int tile, int sig, C* sm) {
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)sig * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)sig * a.m;
  const int r0 = tile * a.T;
  const int n = a.T * a.nD;
  const int d = a.d;
  const int nthr = blockDim.x;
  constexpr int CH = EPT / 2;  // loads in flight per thread per chunk
#pragma unroll
  for (int k0 = 0; k0 < EPT; k0 += CH) {
  C v[CH];
  int sidx[CH];
#pragma unroll
  for (int kk = 0; kk < CH; ++kk) {
    const int k = kk;
    const int w = threadIdx.x + (k0 + k) * nthr;
    sidx[k] = -1;
    if (w < n) {
      const int t = a.divnD.div(w);
      const int e = w - t * a.nD;
      const int row = r0 + t;
      if (row < a.LB) {
        if (a.load_mode == MAP_BOX_H) {
          v[k] = __ldg(in + box_sum_slot(a.boxH, a.Atab + row * a.ts, a.Btab + e * a.ts));
          sidx[k] = t * a.nD + e;
        } else if (a.load_mode == MAP_WS) {
          const int mu = __ldg(a.PIinv + e);
          v[k] = __ldg(in + row * a.nD + e);
          if (a.fs_na > 1) v[k] = cmul(maybe_conj(v[k], a.conj_in), fs_twiddle<C>(a, row, mu));
          else v[k] = maybe_conj(v[k], a.conj_in);
          sidx[k] = t * a.nD + mu;
        } else {
          v[k] = __ldg(in + box_sum_slot(a.boxG, a.Ctab + row * a.ts, a.Etab + e * a.ts));
          sidx[k] = t * a.nD + __ldg(a.PIinv + e);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < CH; ++k)
    if (sidx[k] >= 0) sm[phys<PAD>(sidx[k])] = (a.load_mode == MAP_WS) ? v[k] : maybe_conj(v[k], a.conj_in);
  }
  __syncthreads();
  run_all_stages<C, EPT, false, POW2, PAD, TCK>(sm, a, tw);
  using Rl = decltype(C::x);
  const Rl sc = Rl(a.scale);
#pragma unroll
  for (int k0 = 0; k0 < EPT; k0 += CH) {
  C v[CH];
  int gidx[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    const int w = threadIdx.x + (k0 + k) * nthr;
    gidx[k] = -1;
    if (w < n) {
      const int t = a.divnD.div(w);
      const int e = w - t * a.nD;
      const int row = r0 + t;
      if (row < a.LB) {
        if (a.store_mode == MAP_WS) {
          const int mu = __ldg(a.PIinv + e);
          v[k] = sm[phys<PAD>(t * a.nD + mu)];
          if (a.fs_na > 1) v[k] = cmul(v[k], fs_twiddle<C>(a, row, mu));
          gidx[k] = row * a.nD + e;
        } else if (a.store_mode == MAP_BOX_H) {
          v[k] = cscale(maybe_conj(sm[phys<PAD>(t * a.nD + e)], a.conj_out), sc);
          gidx[k] = box_sum_slot(a.boxH, a.Atab + row * a.ts, a.Btab + e * a.ts);
        } else {
          v[k] = cscale(maybe_conj(sm[phys<PAD>(t * a.nD + __ldg(a.PIinv + e))], a.conj_out), sc);
          gidx[k] = box_sum_slot(a.boxG, a.Ctab + row * a.ts, a.Etab + e * a.ts);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < CH; ++k)
    if (gidx[k] >= 0) out[gidx[k]] = v[k];
  }
}

// Pencil-internal index of the sheared walk: unflatten j over the
// non-trivial cycles before the last one, add the per-thread offset, wrap.
__device__ __forceinline__ int shear_index(const PassArgs& a, int j, const int* off) {
  int c[kMaxSub];
#pragma unroll
  for (int s = kMaxSub - 1; s >= 0; --s) {
    if (s < a.nsub) {
      const int q = a.sub_div[s].div(j);
      c[s] = j - q * a.sub_n[s] + off[s];
      if (c[s] >= a.sub_n[s]) c[s] -= a.sub_n[s];
      j = q;
    }
  }
  int i = 0;
#pragma unroll
  for (int s = 0; s < kMaxSub; ++s)
    if (s < a.nsub) i = i * a.sub_n[s] + c[s];
  return i;
}

// Column pass: all LB rows of T adjacent workspace columns per CTA, smem
// layout [i][t].  The DFT runs over the (D-1) cycles inside the pencil.
// Loads and stores are batched per thread as in the row pass.
template <typename C, int EPT, bool POW2, bool PAD, bool TCK = true, bool COH = false>
__device__ __forceinline__ void col_pass_body(const PassArgs& a, int tile, int sig, C* sm) {
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)sig * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)sig * a.m;
  const int p0 = tile * a.T;
  const int n = a.T * a.LB;
  const int d = a.d;
  const int nthr = blockDim.x;
  // blockDim.x is a multiple of T, so each thread keeps one column.
  const int tcol = a.divT.mod(threadIdx.x);
  // the last CTA may hold fewer than T columns (T need not divide nD)
  const int nvalid = min(a.T, a.nD - p0);
  const int n_ok = tcol < nvalid ? n : 0;
  int off[kMaxSub];
#pragma unroll
  for (int s = 0; s < kMaxSub; ++s)
    off[s] = (s < a.nsub) ? int((int64_t(tcol) * a.alpha[s]) % a.sub_n[s]) : 0;
  int et[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) et[r] = (r < d && n_ok) ? __ldg(a.Etab + (p0 + tcol) * a.ts + r) : 0;
  constexpr int CH = EPT / 2;  // loads in flight per thread per chunk
  const bool ws_in = a.load_mode == MAP_WS;
#pragma unroll
  for (int k0 = 0; k0 < EPT; k0 += CH) {
  C v[CH];
  int sidx[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    const int w = threadIdx.x + (k0 + k) * nthr;
    sidx[k] = -1;
    if (w < n_ok) {
      const int j = a.divT.div(w);
      if (ws_in) {
        v[k] = COH ? __ldcg(in + j * a.nD + p0 + tcol) : __ldg(in + j * a.nD + p0 + tcol);
        sidx[k] = j * a.T + tcol;
      } else {
        const int i = shear_index(a, j, off);
        v[k] = __ldg(in + box_sum_slot(a.boxG, a.Ctab + i * a.ts, et));
        sidx[k] = i * a.T + tcol;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < CH; ++k)
    if (sidx[k] >= 0) sm[phys<PAD>(sidx[k])] = maybe_conj(v[k], a.conj_in);
  }
  __syncthreads();
  run_all_stages<C, EPT, true, POW2, PAD, TCK>(sm, a, tw);
  using Rl = decltype(C::x);
  const Rl sc = Rl(a.scale);
  const bool ws_out = a.store_mode == MAP_WS;
#pragma unroll
  for (int k0 = 0; k0 < EPT; k0 += CH) {
  C v[CH];
  int gidx[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    const int w = threadIdx.x + (k0 + k) * nthr;
    gidx[k] = -1;
    if (w < n_ok) {
      const int j = a.divT.div(w);
      if (ws_out) {
        v[k] = sm[phys<PAD>(j * a.T + tcol)];
        gidx[k] = j * a.nD + p0 + tcol;
      } else {
        const int i = shear_index(a, j, off);
        v[k] = cscale(maybe_conj(sm[phys<PAD>(i * a.T + tcol)], a.conj_out), sc);
        gidx[k] = box_sum_slot(a.boxG, a.Ctab + i * a.ts, et);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < CH; ++k)
    if (gidx[k] >= 0) out[gidx[k]] = v[k];
  }
}

// MINB: resident CTAs per SM the register allocation is fitted to (2 for the
// 16-points-per-thread build, whose tiles hold at most 8192 points).  Only the
// 32-points-per-thread build carries the tensor-core stages.
template <typename C, int EPT, bool POW2, bool PAD, int MINB = 1>
__global__ void __launch_bounds__(kMaxThreads, MINB) row_pass_kernel(PassArgs a) {
  extern __shared__ unsigned char smem_raw[];
  row_pass_body<C, EPT, POW2, PAD, EPT == 32>(a, blockIdx.x, blockIdx.y, reinterpret_cast<C*>(smem_raw));
}

template <typename C, int EPT, bool POW2, bool PAD, int MINB = 1>
__global__ void __launch_bounds__(kMaxThreads, MINB) col_pass_kernel(PassArgs a) {
  extern __shared__ unsigned char smem_raw[];
  col_pass_body<C, EPT, POW2, PAD, EPT == 32>(a, blockIdx.x, blockIdx.y, reinterpret_cast<C*>(smem_raw));
}

// Allow the largest dynamic shared-memory size and prefer the maximum shared
// carveout (more resident CTAs per SM).
inline int configure_kernel(const void* k) {
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
    return -1;
  if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess) return -1;
  return 0;
}

template <typename C, int EPT, bool POW2, bool PAD, int MINB>
inline int launch_typed_pad(const PassArgs& a, cudaStream_t s) {
  dim3 grid(a.groups, a.batch), block(a.nthreads);
  static const int row_ok =
      configure_kernel(reinterpret_cast<const void*>(row_pass_kernel<C, EPT, POW2, PAD, MINB>));
  static const int col_ok =
      configure_kernel(reinterpret_cast<const void*>(col_pass_kernel<C, EPT, POW2, PAD, MINB>));
  if (row_ok != 0 || col_ok != 0) return -1;
  if (a.cols)
    col_pass_kernel<C, EPT, POW2, PAD, MINB><<<grid, block, a.smem_bytes, s>>>(a);
  else
    row_pass_kernel<C, EPT, POW2, PAD, MINB><<<grid, block, a.smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename C, int EPT, bool POW2, int MINB = 1>
inline int launch_typed(const PassArgs& a, cudaStream_t s) {
  if constexpr (POW2) return launch_typed_pad<C, EPT, true, true, MINB>(a, s);  // no direct stages
  return a.pad ? launch_typed_pad<C, EPT, POW2, true, MINB>(a, s) : launch_typed_pad<C, EPT, POW2, false, MINB>(a, s);
}

}  // namespace pfft
