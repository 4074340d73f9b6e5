// Persistent, pipelined row pass for rows of 2^14 complex64 elements.
//
// The row pass of a 2^14-point cycle (eq. (KroneckerFFT): the blockwise
// transforms along the longest cycle) holds one row in the registers of 512
// threads (32 elements each; radix 16 x 32 x 32 Stockham stages).  A CTA
// that stages the whole row in shared memory for its exchanges can keep no
// second row in flight, so its load, compute and store phases serialise.
// Here one CTA per SM walks rows g = blockIdx.x, + gridDim.x, ... and keeps
// the next row's bulk copies in flight while it transforms the current one:
//
//   S  (128 KiB)  the input row, filled by cp.async.bulk on an mbarrier;
//                 released as soon as the threads have read their elements,
//                 after which the copies of the next row are issued into it;
//   X  (68 KiB)   the exchange buffer of the stages and the staging buffer
//                 of the output, used in two rounds of 2^13 elements each;
//   stw           the stage twiddles, copied once per CTA.
//
// Exchanges in two rounds.  Stockham positions are 14-bit numbers.  The tail
// stage (radix 16, Ns = 1) writes position (q << 13) | (p << 4) | r from its
// butterfly q in {0, 1}, and stage 0 reads (r' << 9) | p: a round per value
// of bit 13 moves exactly register half q of every thread if the elements
// are loaded so that butterfly q sits in registers 16 q .. 16 q + 15.  Stage
// 0 (Ns = 16) writes ((p >> 4) << 9) | (r << 4) | (p mod 16) and stage 1
// reads (r' << 9) | p; splitting by bit 8 xor bit 13 makes thread p write and
// read the register half H = h xor bit 8 of p in round h (warp-uniform),
// and dropping bit 13 maps each round one-to-one onto 2^13 slots of X.
//
// Output in two rounds.  The inverse direction writes the box in element
// order: round h holds elements [2^13 h, 2^13 (h + 1)), registers
// 16 h .. 16 h + 15, sent by one bulk copy per run piece.  The forward
// direction writes the workspace row in position order (the column
// permutation PI): each element goes to X in the round of bit 13 of its
// position (a predicated store) and the round's half row leaves in one bulk
// copy per staging block.
//
// Every wait on the mbarrier is bounded.  The threads agree on its outcome
// (__syncthreads_and); on a timeout the kernel records PFFT_ERR_TIMEOUT,
// waits (bounded) for its own copies in flight and returns.
#pragma once
#include <cuda_runtime.h>

#include "fft_fast_ct.cuh"
#include "fft_tma.cuh"

namespace pfft {

// X slot of exchange index i: one padding element per 16, so that the
// stride-16 writes of the tail stage spread over all banks.
__device__ __forceinline__ int xphys(int i) { return i + (i >> 4); }

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Exchange 2 for register half H (compile time): write the stage-0 outputs,
// barrier, read the stage-1 inputs.
template <int H>
__device__ __forceinline__ void pipe_x2_write(const float2* v, float2* X, int p) {
  const int base = (((p >> 4) & 15) << 9) | (p & 15);
#pragma unroll
  for (int i = 0; i < 16; ++i) X[xphys(base | ((16 * H + i) << 4))] = v[16 * H + i];
}
template <int H>
__device__ __forceinline__ void pipe_x2_read(float2* v, const float2* X, int p) {
#pragma unroll
  for (int i = 0; i < 16; ++i) v[16 * H + i] = X[xphys((i << 9) | p)];
}

// FWD: the forward row pass (box runs -> workspace row); else the inverse
// (workspace row -> box runs, conjugated and scaled).
// DIRECT: the output leaves from the registers with plain stores (workspace
// rows whose permutation keeps lanes in runs, box rows made of uniform runs);
// else it is staged through X in two rounds of bulk copies.
// X1S: exchange 1 in one round through S and X together, the next row's
// copies issued after it; else in two rounds through X, the copies issued
// as soon as the row has been read from S.
template <bool FWD, bool DIRECT, bool X1S>
__global__ void __launch_bounds__(512, 1) row_pipe_kernel(PassArgs a) {
  using C = float2;
  constexpr int R = 32, L = 1 << kPipeLogL, P = L / R, LP = kPipeLogL - 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw);
  C* X = S + a.pipe_x_off;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + a.bar_smem_off);
  const int p = threadIdx.x;
  const int total = a.LB * a.batch;
  const int nblk = a.stg_pad ? (1 << a.pi_lg) : 1;
  const int span = L / nblk;
  const C* __restrict__ in_all = static_cast<const C*>(a.in);
  C* __restrict__ out_all = static_cast<C*>(a.out);

  // bulk copies of row g into S (issuing threads only; the expected bytes
  // are announced by thread 0 before the barrier that precedes this)
  auto issue_load = [&](int g) {
    const int b = g / a.LB, row = g - b * a.LB;
    const C* in = in_all + (int64_t)b * a.m;
    if constexpr (FWD) {
      if (p < a.nruns) {
        const int4 r = __ldg(reinterpret_cast<const int4*>(a.runs) + (size_t)row * a.nruns + p);
        if (r.z > 0) bulk_g2s(S + r.x, in + r.y, uint32_t(r.z) * uint32_t(sizeof(C)), bar);
      }
    } else if (p < nblk) {
      bulk_g2s(S + p * (span + a.stg_pad), in + (size_t)row * a.nD + p * span, uint32_t(span) * uint32_t(sizeof(C)),
               bar);
    }
  };

  if (p == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  C* stw = stage_table(S, a);
  cp_async_wait_all();
  __syncthreads();
  if (blockIdx.x < total) {
    if (p == 0) mbar_arrive_expect_tx(bar, uint32_t(L) * uint32_t(sizeof(C)));
    __syncthreads();
    issue_load(blockIdx.x);
  }

  // workspace position of this thread's element p + P k (see fft_tma_ct.cuh);
  // evaluated where it is used, so that nothing of it stays live across the stages
  auto ws_pos = [&](int k) {
    if (a.pi_arith && a.pi_lg <= LP) {
      const int lg = a.pi_lg, ls = a.pi_lspan;
      const int lo = p & ((1 << lg) - 1);
      return (lo << ls) + ((((p >> lg) * a.pi_inv) + k * (a.pi_inv << (LP - lg))) & ((1 << ls) - 1));
    }
    return col_pos(a, p + P * k);
  };
  auto stg = [&](int pos) { return a.stg_pad ? pos + (pos >> a.pi_lspan) * a.stg_pad : pos; };
  auto issuer = [&]() { return FWD ? (p < (a.stg_pad ? (kPipeHalf >> a.pi_lspan) : 1)) : (p < a.nruns); };
  uint32_t phase = 0;

  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    const bool ok = mbar_wait_bounded(bar, phase, a.spin_limit);
    if (!__syncthreads_and(ok)) {
      if (p == 0) atomicExch(a.status, kStatusTimeout);
      mbar_wait_bounded(bar, phase);  // let this CTA's copies land before leaving
      bulk_wait_all();
      return;
    }
    phase ^= 1u;
    const int gn = g + gridDim.x;
    if (p == 0 && gn < total) mbar_arrive_expect_tx(bar, uint32_t(L) * uint32_t(sizeof(C)));
    const int b = g / a.LB, row = g - b * a.LB;

    // ---- S -> registers: v[16 q + r] = element p + P (q + 2 r)
    C v[R];
    if constexpr (FWD) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 16; ++r) v[16 * q + r] = S[p + P * (q + 2 * r)];
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 16; ++r) v[16 * q + r] = S[stg(ws_pos(q + 2 * r))];
    }
    if (!FWD && a.fs_na > 1) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 16; ++r) v[16 * q + r] = cmul(v[16 * q + r], fs_twiddle<C>(a, row, p + P * (q + 2 * r)));
    }
    if (!DIRECT && issuer()) bulk_wait_read_all();  // the previous row's output has left X
    __syncthreads();  // S is read
    if constexpr (X1S) {
      // ---- tail stage (radix 16) and exchange 1 in one round through S and X
      dft16(v);
      dft16(v + 16);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 16; ++r) S[xphys((q << 13) | (p << 4) | r)] = v[16 * q + r];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = S[xphys((r << 9) | p)];
      __syncthreads();  // S is free: the next row may land in it
      if (gn < total) issue_load(gn);
    } else {
      if (gn < total) issue_load(gn);
      // ---- tail stage (radix 16) and exchange 1, one round per butterfly
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        dft16(v + 16 * q);
#pragma unroll
        for (int r = 0; r < 16; ++r) X[xphys((p << 4) | r)] = v[16 * q + r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) v[16 * q + r] = X[xphys((r << 9) | p)];
        __syncthreads();
      }
    }
    // ---- stage 0 (Ns = 16) and exchange 2
    {
      const int k = p & 15;
      if (k) main_twiddle<C, R>(v, stw + a.stw_off[0] + k * 5);
      dft_pow2<C, R>(v);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if ((h ^ (p >> 8)) & 1)
          pipe_x2_write<1>(v, X, p);
        else
          pipe_x2_write<0>(v, X, p);
        __syncthreads();
        if ((h ^ (p >> 8)) & 1)
          pipe_x2_read<1>(v, X, p);
        else
          pipe_x2_read<0>(v, X, p);
        __syncthreads();
      }
    }
    // ---- stage 1 (Ns = 512): v[r] = frequency p + P r
    if (p) main_twiddle<C, R>(v, stw + a.stw_off[1] + p * 5);
    dft_pow2<C, R>(v);

    // ---- output
    if constexpr (FWD && DIRECT) {
      // workspace position ((p mod 2^lg) << ls) + (p >> lg) + k 2^(9 - lg)
      // (permutation multiplier 1): lanes write runs of 2^(5 - lg) elements
      if (a.fs_na > 1) {
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = cmul(v[k], fs_twiddle<C>(a, row, p + P * k));
      }
      const int lg = a.pi_lg;
      C* out = out_all + (int64_t)b * a.m + (size_t)row * a.nD + ((p & ((1 << lg) - 1)) << a.pi_lspan) + (p >> lg);
      const int cst = P >> lg;
#pragma unroll
      for (int k = 0; k < R; ++k) out[k * cst] = v[k];
    } else if constexpr (!FWD && DIRECT) {
      // box rows of uniform runs of 2^lrun elements: element e lies in run e >> lrun
      C* out = out_all + (int64_t)b * a.m;
      const int4* runs = reinterpret_cast<const int4*>(a.runs) + (size_t)row * a.nruns;
      const int lrun = a.pipe_lrun, mrun = (1 << lrun) - 1;
      const float sx = float(a.scale), sy = -sx;  // conjugate and scale
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = p + P * r;
        const C x = v[r];
        out[__ldg(&runs[e >> lrun].y) + (e & mrun)] = cmake<C>(x.x * sx, x.y * sy);
      }
    } else if constexpr (FWD) {
      // ---- output in two rounds through X
      if (a.fs_na > 1) {
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = cmul(v[k], fs_twiddle<C>(a, row, p + P * k));
      }
      C* out = out_all + (int64_t)b * a.m + (size_t)row * a.nD;
      const int nbh = a.stg_pad ? (kPipeHalf >> a.pi_lspan) : 1;
      const int sph = kPipeHalf / nbh;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h) {
          if (issuer()) bulk_wait_read_all();
          __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const int pos = ws_pos(k);
          if ((pos >> 13) == h) X[stg(pos & (kPipeHalf - 1))] = v[k];
        }
        fence_async_smem();
        __syncthreads();
        if (p < nbh) {
          bulk_s2g(out + h * kPipeHalf + p * sph, X + p * (sph + a.stg_pad), uint32_t(sph) * uint32_t(sizeof(C)));
          bulk_commit();
        }
      }
    } else {
      C* out = out_all + (int64_t)b * a.m;
      const float sx = float(a.scale), sy = -sx;  // conjugate and scale
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h) {
          if (issuer()) bulk_wait_read_all();
          __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const C x = v[16 * h + r];
          X[p + P * r] = cmake<C>(x.x * sx, x.y * sy);
        }
        fence_async_smem();
        __syncthreads();
        if (p < a.nruns) {
          const int4 run = __ldg(reinterpret_cast<const int4*>(a.runs) + (size_t)row * a.nruns + p);
          const int lo = max(run.x, h * kPipeHalf), hi = min(run.x + run.z, (h + 1) * kPipeHalf);
          if (hi > lo) bulk_s2g(out + run.y + (lo - run.x), X + (lo - h * kPipeHalf), uint32_t(hi - lo) * uint32_t(sizeof(C)));
          bulk_commit();
        }
      }
    }
  }
  if constexpr (!DIRECT) bulk_wait_all();  // every output copy of this CTA is complete
}

}  // namespace pfft
