// Split-precision tensor-core stages of radix 16 and 32 (complex64 only), on
// the fifth-generation tensor cores (tcgen05.mma, accumulators in tensor
// memory).
//
// A Stockham stage of radix R is, per butterfly, the dense product
// y = F x' with F[s][r] = omega_R^{s r} and x' the twiddled inputs.  In real
// arithmetic [Re y; Im y] = W [Re x'; Im x'] with the 2R x 2R matrix
// W = [[Fr, -Fi], [Fi, Fr]].  The butterflies of a stage, 128 at a time, are
// the rows of the operand A (M = 128, K = 2R: row m holds [Re x'; Im x'] of
// butterfly m), W^T is the operand B (K x N, N = 2R), and D = A B holds the
// outputs of butterfly m in row m, which is lane m of the tensor memory.
//
// Both operands are split into fp16 halves, a = a_hi + a_lo with
// a_hi = fp16(a) and a_lo = fp16(a - a_hi), and the three products
// A_hi B_hi + A_hi B_lo + A_lo B_hi are chained into one fp32 accumulator
// (kind::f16), which keeps about 22 significant bits (the dropped
// A_lo B_lo term is below the fp32 rounding of the sums).  Each butterfly is
// scaled by a power of two before the split so that its largest input lies
// in [2^10, 2^11), and its outputs are scaled back after the accumulation:
// both steps are exact in fp32, so the fp16 halves neither overflow nor fall
// into the subnormal range for data of any magnitude from 2^-116 up to the
// fp32 range.  One thread holds whole butterflies (32 / R of them), so the
// scale needs no lane exchange.
//
// Per stage: every thread gathers and twiddles its butterflies from the tile;
// after a barrier it writes their hi and lo rows over the tile (the staging
// takes the tile's 8 bytes per point: 2R fp16 values twice per butterfly of
// R points), in the canonical K-major layout without swizzle (core matrices
// of 8 rows x 16 bytes, adjacent along K, 8-row groups 2R x 16 bytes apart).
// One thread issues the 3 x 2R / 16 MMAs of every 128-butterfly chunk, each
// chunk into its own 2R tensor-memory columns, and commits them to an
// mbarrier; after the bounded wait every warp reads its lane quarter of D
// with tcgen05.ld, undoes the scale and writes the outputs into the tile.
// W's hi and lo halves are staged once per CTA in shared memory.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_plan.hpp"

namespace pfft {

// Shared-memory tile index of the generic passes (fft_kernels.cuh).
template <bool PAD>
__device__ __forceinline__ int phys(int x);

// Byte offset of element (row, k) of a K-major fp16 operand with K columns:
// core matrices of 8 rows x 16 bytes, the core matrices of one 8-row group
// adjacent along K (128 bytes apart), 8-row groups K x 16 bytes apart.
__host__ __device__ constexpr uint32_t tc_kmajor_off(int row, int k, int K) {
  return uint32_t((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
// Bytes of one operand half (hi or lo): rows x K fp16.
__host__ __device__ constexpr int tc_half_bytes(int rows, int K) { return rows * K * 2; }
// Shared-memory bytes of W (hi and lo) for radix R.
__host__ __device__ constexpr int tc_w_bytes(int R) { return 2 * tc_half_bytes(2 * R, 2 * R); }
// Staging bytes of one 128-butterfly chunk (hi and lo rows of A).
__host__ __device__ constexpr int tc_chunk_bytes(int R) { return 2 * tc_half_bytes(128, 2 * R); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between core matrices adjacent along K), stride-dimension byte
// offset (between 8-row groups), all in 16-byte units; bits 46-48 hold the
// fixed value 0b001; base offset 0, no swizzle.
__host__ __device__ constexpr uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}
// Instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1), A
// and B fp16 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N / 8 in
// bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_instr_desc(int M, int N) {
  return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Shared-memory layout of the tensor-core context (planner and kernel):
// [W32 hi | W32 lo] [W16 hi | W16 lo] [scale exponents, int8, one per
// butterfly] [mbarrier] [tensor-memory address]
struct TcLayout {
  int w32, w16, ex, bar, taddr, end;
};
__host__ __device__ inline TcLayout tc_layout(int base, bool has32, bool has16, int max_bfly) {
  TcLayout t;
  t.w32 = base;
  t.w16 = t.w32 + (has32 ? tc_w_bytes(32) : 0);
  t.ex = t.w16 + (has16 ? tc_w_bytes(16) : 0);
  t.bar = (t.ex + max_bfly + 15) & ~15;
  t.taddr = t.bar + 8;
  t.end = t.bar + 16;
  return t;
}
// Tensor-memory columns of a pass: a stage of radix R keeps 2R fp32 columns
// per 128-butterfly chunk (T L / R butterflies); the largest of the pass's
// tensor-core stages, as a power of two >= 32.
__host__ __device__ inline int tc_tmem_cols(int points, bool has32, bool has16) {
  int need = 0;
  if (has32) need = ((points / 32 + 127) / 128) * 64;
  if (has16) need = need > ((points / 16 + 127) / 128) * 32 ? need : ((points / 16 + 127) / 128) * 32;
  int c = 32;
  while (c < need) c <<= 1;
  return c;
}

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool tc_mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t tc_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}
// Bounded wait: at most `limit` tries and about one second.
__device__ __forceinline__ bool tc_mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit) {
  const uint64_t t0 = tc_globaltimer();
  for (uint32_t i = 0; i < limit; ++i) {
    if (tc_mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && tc_globaltimer() - t0 > 1000000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// One D += A B (or D = A B when acc == 0), M = 128, operands in shared memory.
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}
// 16 consecutive fp32 columns of this thread's lane (warp-wide).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Two fp32 values -> packed fp16 pairs (hi, lo); the first value in the low half.
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);  // packed conversions, round to nearest
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// W of radix R, hi and lo, as the K-major operand B (row n = output n of
// [Re y; Im y], column k = input k of [Re x; Im x]).
template <int R>
__device__ void tc_build_w(unsigned char* wsm, const float2* __restrict__ tw, int tw_n) {
  constexpr int K = 2 * R;
  const int wstride = tw_n / R;
  for (int e = threadIdx.x; e < K * K / 2; e += blockDim.x) {
    const int n = e / (K / 2), k = 2 * (e - n * (K / 2));
    float v[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int kk = k + c;
      const int s = n % R, r = kk % R;
      const float2 f = __ldg(tw + ((s * r) % R) * wstride);  // omega_R^{s r} = Fr + i Fi
      const bool yi = n >= R, xi = kk >= R;
      v[c] = (yi == xi) ? f.x : (xi ? -f.y : f.y);
    }
    uint32_t hi, lo;
    split_h2(v[0], v[1], hi, lo);
    const uint32_t off = tc_kmajor_off(n, k, K);
    *reinterpret_cast<uint32_t*>(wsm + off) = hi;
    *reinterpret_cast<uint32_t*>(wsm + tc_half_bytes(K, K) + off) = lo;
  }
}

// Per-pass tensor-core state: shared-memory layout, the tensor-memory base
// and the mbarrier phase.
struct TcCtx {
  unsigned char* base;  // dynamic shared memory
  TcLayout lay;
  uint32_t tmem;        // tensor-memory address of column 0, lane 0
  uint32_t phase;
  int ok;               // 0 once a wait has timed out (later stages skip the tensor cores)
};

// One Stockham stage of radix R (16 or 32) on the tensor cores; the same index
// walk as run_stage (fft_kernels.cuh).  Thread t takes butterflies t, t + n,
// ... (at most 32 / R); the planner's thread count guarantees it.  All reads
// of the tile happen before the first barrier, all writes of outputs after
// the MMAs have completed.
template <int R, bool COLS, bool PAD>
__device__ __noinline__ void run_tc_stage(float2* sm, const PassArgs& a, const StageDesc& s,
                                          const float2* __restrict__ tw, TcCtx& cx) {
  constexpr int K = 2 * R;
  constexpr int NB = 32 / R;
  constexpr int CHB = tc_chunk_bytes(R);
  const int per_pencil = a.L / R;
  const int nbf = a.T * per_pencil;
  const int nthr = blockDim.x;
  const int escale = COLS ? a.T : 1;
  const int step = s.sigma * escale;
  const int istep = s.aR * step;
  signed char* exs = reinterpret_cast<signed char*>(cx.base + cx.lay.ex);
  auto locate = [&](int b, int& ebase, int& k, int& j) {
    int tt, rest;
    if (COLS) {
      rest = a.divT.div(b);
      tt = b - rest * a.T;
    } else {
      tt = b / per_pencil;
      rest = b - tt * per_pencil;
    }
    const int o = s.div_aR.div(rest);
    j = rest - o * s.aR;
    const int hi = s.div_sigma.div(o);
    const int base = hi * s.a * s.sigma + (o - hi * s.sigma);
    k = j - s.div_Ns.div(j) * s.Ns;
    ebase = COLS ? base * a.T + tt : tt * a.L + base;
  };
  // ---- gather, twiddle, scale
  float x[NB][K];
  int ex[NB];
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int bf = threadIdx.x + u * nthr;
    ex[u] = 0;
    if (bf < nbf) {
      int ebase, k, j;
      locate(bf, ebase, k, j);
      const int i0 = ebase + j * step;
      float mx = 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 v = sm[phys<PAD>(i0 + r * istep)];
        if (s.Ns > 1 && r > 0) v = cmul(v, __ldg(tw + (k * r) * s.twstep));  // k r < Ns R: no reduction
        x[u][r] = v.x;
        x[u][R + r] = v.y;
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
      int e = mx > 0.f ? 10 - ilogbf(mx) : 0;
      e = e > 126 ? 126 : (e < -126 ? -126 : e);  // 2^e and 2^-e both normal
      ex[u] = e;
      const float up = __int_as_float((127 + e) << 23);
#pragma unroll
      for (int i = 0; i < K; ++i) x[u][i] *= up;
    }
  }
  __syncthreads();  // every read of the tile is done: the staging may overwrite it
  // ---- hi / lo rows of A over the tile
  unsigned char* stg = reinterpret_cast<unsigned char*>(sm);
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int bf = threadIdx.x + u * nthr;
    if (bf < nbf) {
      unsigned char* ch = stg + (bf >> 7) * CHB;
      const int m = bf & 127;
      exs[bf] = static_cast<signed char>(ex[u]);
#pragma unroll
      for (int kg = 0; kg < K / 8; ++kg) {
        uint4 h, l;
        split_h2(x[u][8 * kg + 0], x[u][8 * kg + 1], h.x, l.x);
        split_h2(x[u][8 * kg + 2], x[u][8 * kg + 3], h.y, l.y);
        split_h2(x[u][8 * kg + 4], x[u][8 * kg + 5], h.z, l.z);
        split_h2(x[u][8 * kg + 6], x[u][8 * kg + 7], h.w, l.w);
        const uint32_t off = tc_kmajor_off(m, 8 * kg, K);
        *reinterpret_cast<uint4*>(ch + off) = h;
        *reinterpret_cast<uint4*>(ch + tc_half_bytes(128, K) + off) = l;
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic-proxy writes -> tensor-core reads
  __syncthreads();
  const int nch = (nbf + 127) >> 7;
  const uint32_t bar = tc_smem_u32(cx.base + cx.lay.bar);
  if (threadIdx.x == 0 && cx.ok) {
    tc_fence_after();
    constexpr uint32_t idesc = tc_instr_desc(128, K);
    const uint32_t wb = tc_smem_u32(cx.base + (R == 32 ? cx.lay.w32 : cx.lay.w16));
    const uint32_t sb = tc_smem_u32(stg);
    for (int c = 0; c < nch; ++c) {
      const uint32_t ahi = sb + c * CHB, alo = ahi + tc_half_bytes(128, K);
      const uint32_t dt = cx.tmem + uint32_t(c * K);
#pragma unroll
      for (int kk = 0; kk < K / 16; ++kk) {
        const uint64_t dah = tc_smem_desc(ahi + kk * 256, 128, K * 16);
        const uint64_t dal = tc_smem_desc(alo + kk * 256, 128, K * 16);
        const uint64_t dbh = tc_smem_desc(wb + kk * 256, 128, K * 16);
        const uint64_t dbl = tc_smem_desc(wb + tc_half_bytes(K, K) + kk * 256, 128, K * 16);
        tc_mma(dt, dah, dbh, idesc, kk > 0 ? 1u : 0u);
        tc_mma(dt, dah, dbl, idesc, 1u);
        tc_mma(dt, dal, dbh, idesc, 1u);
      }
    }
    tc_commit(bar);
  }
  // ---- wait for the products (bounded), then read D back
  bool done = cx.ok != 0;
  if (done) {
    done = tc_mbar_wait_bounded(bar, cx.phase, a.spin_limit);
    if (!done) {
      if (threadIdx.x == 0) atomicExch(a.status, 8);  // PFFT_ERR_TIMEOUT
      tc_mbar_wait_bounded(bar, cx.phase, kSpinLimit);  // let the products in flight finish
    }
    cx.phase ^= 1u;
  }
  done = __syncthreads_and(done ? 1 : 0) != 0;
  if (!done) cx.ok = 0;
  tc_fence_after();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = nthr >> 5;
  const int q = warp & 3;
  const int ostep = s.Ns * step;
  for (int c = warp >> 2; c < nch; c += nw >> 2) {
    const uint32_t ta = cx.tmem + (uint32_t(32 * q) << 16) + uint32_t(c * K);
    const int bf = c * 128 + 32 * q + lane;
    const bool mine = bf < nbf && done;
    int ob = 0;
    float down = 0.f;
    if (mine) {
      int ebase, k, j;
      locate(bf, ebase, k, j);
      ob = ebase + ((j - k) * R + k) * step;
      down = __int_as_float((127 - int(exs[bf])) << 23);
    }
    // outputs 16 h .. 16 h + 15: real parts in columns 16 h.., imaginary parts in R + 16 h..
#pragma unroll
    for (int h = 0; h < R / 16; ++h) {
      uint32_t re[16], im[16];
      tc_ld16(ta + 16 * h, re);
      tc_ld16(ta + R + 16 * h, im);
      tc_wait_ld();
      if (mine) {
#pragma unroll
        for (int so = 0; so < 16; ++so)
          sm[phys<PAD>(ob + (16 * h + so) * ostep)] =
              make_float2(__uint_as_float(re[so]) * down, __uint_as_float(im[so]) * down);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
}
// ---- The same product inside the register-resident passes (fft_fast.cuh):
// every thread holds one radix-32 butterfly in registers, so it scales,
// splits and stages its own row of A (row = thread index, over the tile,
// whose reads are complete), and reads its own row of D back (warp w reads
// lanes 32 (w mod 4) .. of chunk w / 4: rows 32 w .. 32 w + 31, i.e. its own
// threads).  The block size is a multiple of 128.  Each 128-thread chunk
// runs on its own: its four warps stage their rows and meet at a named
// barrier, one of them issues the chunk's MMAs and commits them to the
// chunk's mbarrier, and the four warps wait for that one only, so the
// products of one chunk overlap the staging of the others.
constexpr int kTcMaxChunks = 4;  // 512 threads
struct TcRegs {
  unsigned char* stg;  // the tile (staging)
  uint32_t w32;        // shared address of W (hi, lo), radix 32
  uint32_t bar;        // shared address of the chunks' mbarriers (8 bytes each)
  uint32_t tmem;       // tensor-memory base
  uint32_t phase;
  int ok;
};

// Shared-memory bytes the register-resident passes add for the tensor cores
// (after their own footprint): W of radix 32 (hi, lo), the chunks' mbarriers
// and the tensor-memory address.
__host__ __device__ constexpr int tc_regs_extra_bytes() { return tc_w_bytes(32) + 8 * kTcMaxChunks + 16; }

// Set-up at the start of a register-resident pass (all threads): W, the
// mbarrier, the tensor memory (one 64-column accumulator per 128 threads).
__device__ __forceinline__ void tc_regs_begin(TcRegs& cx, unsigned char* smem, int tc_off, const float2* tw,
                                              int tw_n) {
  unsigned char* w = smem + tc_off;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(w + tc_w_bytes(32) + 8 * kTcMaxChunks);
  tc_build_w<32>(w, tw, tw_n);
  if (threadIdx.x < kTcMaxChunks) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem_u32(w + tc_w_bytes(32) + 8 * threadIdx.x))
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const int cols = tc_tmem_cols(int(blockDim.x) * 32, true, false);
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc_smem_u32(tslot)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cx.stg = smem;
  cx.w32 = tc_smem_u32(w);
  cx.bar = tc_smem_u32(w + tc_w_bytes(32));
  cx.tmem = *tslot;
  cx.phase = 0;
  cx.ok = 1;
}

__device__ __forceinline__ void tc_regs_end(const TcRegs& cx) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    const int cols = tc_tmem_cols(int(blockDim.x) * 32, true, false);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(cx.tmem), "r"(cols) : "memory");
  }
}

// v[r] <- sum_s omega_32^{r s} v[s] for the thread's butterfly, on the tensor
// cores.  Entry: every thread's reads of the tile are complete (a barrier
// separates them from this call).  Exit: the tile is free again.
__device__ __forceinline__ void tc_dft32_regs(float2* v, TcRegs& cx, const PassArgs& a) {
  constexpr int R = 32, K = 64;
  constexpr int CHB = tc_chunk_bytes(R);
  float mx = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) mx = fmaxf(mx, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
  int e = mx > 0.f ? 10 - ilogbf(mx) : 0;
  e = e > 126 ? 126 : (e < -126 ? -126 : e);
  const float up = __int_as_float((127 + e) << 23);
  {
    unsigned char* ch = cx.stg + (threadIdx.x >> 7) * CHB;
    const int m = threadIdx.x & 127;
#pragma unroll
    for (int kg = 0; kg < K / 8; ++kg) {
      // inputs 8 kg .. 8 kg + 7 of [Re x; Im x]
      float f[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int kk = 8 * kg + i;
        f[i] = (kk < R ? v[kk].x : v[kk - R].y) * up;
      }
      uint4 h, l;
      split_h2(f[0], f[1], h.x, l.x);
      split_h2(f[2], f[3], h.y, l.y);
      split_h2(f[4], f[5], h.z, l.z);
      split_h2(f[6], f[7], h.w, l.w);
      const uint32_t off = tc_kmajor_off(m, 8 * kg, K);
      *reinterpret_cast<uint4*>(ch + off) = h;
      *reinterpret_cast<uint4*>(ch + tc_half_bytes(128, K) + off) = l;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  const int c = threadIdx.x >> 7;
  asm volatile("bar.sync %0, 128;\n" ::"r"(1 + c) : "memory");  // the chunk's rows are staged
  const uint32_t bar = cx.bar + 8 * c;
  if ((threadIdx.x & 127) == 0 && cx.ok) {
    tc_fence_after();
    constexpr uint32_t idesc = tc_instr_desc(128, K);
    const uint32_t ahi = tc_smem_u32(cx.stg) + c * CHB, alo = ahi + tc_half_bytes(128, K);
    const uint32_t dt = cx.tmem + uint32_t(c * K);
#pragma unroll
    for (int kk = 0; kk < K / 16; ++kk) {
      const uint64_t dah = tc_smem_desc(ahi + kk * 256, 128, K * 16);
      const uint64_t dal = tc_smem_desc(alo + kk * 256, 128, K * 16);
      const uint64_t dbh = tc_smem_desc(cx.w32 + kk * 256, 128, K * 16);
      const uint64_t dbl = tc_smem_desc(cx.w32 + tc_half_bytes(K, K) + kk * 256, 128, K * 16);
      tc_mma(dt, dah, dbh, idesc, kk > 0 ? 1u : 0u);
      tc_mma(dt, dah, dbl, idesc, 1u);
      tc_mma(dt, dal, dbh, idesc, 1u);
    }
    tc_commit(bar);
  }
  bool done = cx.ok != 0;
  if (done) {
    done = tc_mbar_wait_bounded(bar, cx.phase, a.spin_limit);
    if (!done) {
      if ((threadIdx.x & 127) == 0) atomicExch(a.status, 8);  // PFFT_ERR_TIMEOUT
      tc_mbar_wait_bounded(bar, cx.phase, kSpinLimit);
    }
  }
  tc_fence_after();
  {
    const int warp = threadIdx.x >> 5;
    const uint32_t ta = cx.tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t((warp >> 2) * K);
    const float down = __int_as_float((127 - e) << 23);
#pragma unroll
    for (int h = 0; h < R / 16; ++h) {
      uint32_t re[16], im[16];
      tc_ld16(ta + 16 * h, re);
      tc_ld16(ta + R + 16 * h, im);
      tc_wait_ld();
#pragma unroll
      for (int so = 0; so < 16; ++so)
        v[16 * h + so] = make_float2(__uint_as_float(re[so]) * down, __uint_as_float(im[so]) * down);
    }
  }
  tc_fence_before();
  if (cx.ok) cx.phase ^= 1u;
  if (!__syncthreads_and(done ? 1 : 0)) cx.ok = 0;  // every chunk's products are complete
}
}  // namespace pfft
