// Register-resident transform passes for power-of-two pencils (sm_103a).
//
// Same passes as fft_kernels.cuh (row pass: length-nD DFT with the box gather
// or scatter fused; column pass: length-LB DFT over one non-trivial cycle with
// the sheared box scatter / gather fused), specialised for pencil lengths
// L = 2^l >= R, where R = 32 (complex64) or 16 (complex128) is the radix of
// the main stages:
//
//   * every thread owns the R elements p + P k (k < R) of one pencil,
//     P = L / R.  A Stockham stage of radix R reads exactly the elements
//     p + P r of butterfly p, and the last stage (Ns = P) writes them back, so
//     the first stage takes its inputs straight from the global loads and the
//     last stage hands its outputs straight to the global stores;
//   * L = Rt R^s: one "tail" stage of radix Rt in {1, 2, 4, 8, 16} runs
//     first (Ns = 1, no twiddles), then s main stages;
//   * shared memory is used only between stages (padding of one element per
//     32 keeps the stride-R writes of the early stages conflict free).
#pragma once
#include <cuda_runtime.h>

#include "fft_plan.hpp"
#include "fft_tc.cuh"

namespace pfft {

__device__ __forceinline__ int fphys(int x) { return x + (x >> 5); }

// Length 32 as 16 x 2: n = 2 n1 + n2, k = k1 + 16 k2.
template <typename C>
__device__ __forceinline__ void dft32(C* x) {
  C e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = x[2 * i];
    o[i] = x[2 * i + 1];
  }
  dft16(e);
  dft16(o);
  using Rl = decltype(C::x);
  // cos and sin of 2 pi k / 32, k = 0..15
  const Rl cs[16] = {Rl(1.0), Rl(0.98078528040323044913), Rl(0.92387953251128675613),
                     Rl(0.83146961230254523708), Rl(0.70710678118654752440), Rl(0.55557023301960222474),
                     Rl(0.38268343236508977173), Rl(0.19509032201612826785), Rl(0.0),
                     Rl(-0.19509032201612826785), Rl(-0.38268343236508977173), Rl(-0.55557023301960222474),
                     Rl(-0.70710678118654752440), Rl(-0.83146961230254523708), Rl(-0.92387953251128675613),
                     Rl(-0.98078528040323044913)};
  const Rl sn[16] = {Rl(0.0), Rl(0.19509032201612826785), Rl(0.38268343236508977173),
                     Rl(0.55557023301960222474), Rl(0.70710678118654752440), Rl(0.83146961230254523708),
                     Rl(0.92387953251128675613), Rl(0.98078528040323044913), Rl(1.0),
                     Rl(0.98078528040323044913), Rl(0.92387953251128675613), Rl(0.83146961230254523708),
                     Rl(0.70710678118654752440), Rl(0.55557023301960222474), Rl(0.38268343236508977173),
                     Rl(0.19509032201612826785)};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    C t = o[k];
    if (k) t = cmul(t, cmake<C>(cs[k], -sn[k]));
    x[k] = cadd(e[k], t);
    x[k + 16] = csub(e[k], t);
  }
}

template <typename C, int R>
__device__ __forceinline__ void dft_pow2(C* x) {
  if constexpr (R == 2) {
    dft2(x[0], x[1]);
  } else if constexpr (R == 4) {
    dft4(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 8) {
    dft8(x);
  } else if constexpr (R == 16) {
    dft16(x);
  } else {
    dft32(x);
  }
}

// Tail stage (radix RT, Ns = 1) on the thread's R registers: butterfly q
// (q < R / RT) combines registers q + r (R / RT) and writes the Stockham
// outputs (p + P q) RT + r of its pencil to shared memory.
template <typename C, int R, int RT, bool COLS>
__device__ __forceinline__ void tail_stage(C* v, C* sm, int p, int P, int pencil_base, int escale) {
  constexpr int NQ = R / RT;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    C u[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) u[r] = v[q + r * NQ];
    dft_pow2<C, RT>(u);
    const int j = p + P * q;
#pragma unroll
    for (int r = 0; r < RT; ++r) sm[fphys(pencil_base + (j * RT + r) * escale)] = u[r];
  }
}

// Twiddles of a main stage of radix R and span Ns: v[r] *= w^r, w = exp(-2 pi i k / (Ns R)),
// k = p mod Ns.  The stage table (shared memory) holds w^(2^b) for b < NB;
// w^r = w^(r - 2^hb) w^(2^hb) with hb the highest set bit of r reuses the
// lower powers, so each factor carries at most log2(R) - 1 rounded products.
template <typename C, int R>
__device__ __forceinline__ void main_twiddle(C* v, const C* stw) {
  constexpr int NB = (R == 32) ? 5 : (R == 16) ? 4 : (R == 8) ? 3 : (R == 4) ? 2 : 1;
  C pw[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) pw[b] = stw[b];
  C f[R];
#pragma unroll
  for (int r = 1; r < R; ++r) {
    int hb = 0;
    while ((2 << hb) <= r) ++hb;
    const int rest = r - (1 << hb);
    f[r] = rest ? cmul(f[rest], pw[hb]) : pw[hb];
  }
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = cmul(v[r], f[r]);
}

// All stages of one pencil on the thread's registers v[R].  On entry v holds
// elements p + P k; on exit v holds output frequencies p + P k.
// TC (complex64, radix 32): the main stages' butterflies on the tensor cores
// (fft_tc.cuh, tc_dft32_regs); the tail stage stays in registers.
template <typename C, int R, bool COLS, bool TC = false>
__device__ __forceinline__ void fast_pencil_dft(C* v, C* sm, const C* stw, const PassArgs& a, int p,
                                                int pencil_base, int escale, int L, TcRegs* tcx = nullptr) {
  const int P = L / R;
  int Ns = 1;
  bool in_regs = true;
  if (a.fast_tail > 1) {
    switch (a.fast_tail) {
      case 2: tail_stage<C, R, 2, COLS>(v, sm, p, P, pencil_base, escale); break;
      case 4: tail_stage<C, R, 4, COLS>(v, sm, p, P, pencil_base, escale); break;
      case 8: tail_stage<C, R, 8, COLS>(v, sm, p, P, pencil_base, escale); break;
      default: tail_stage<C, R, 16, COLS>(v, sm, p, P, pencil_base, escale); break;
    }
    Ns = a.fast_tail;
    in_regs = false;
    __syncthreads();
  }
#pragma unroll 1
  for (int s = 0; s < a.fast_nmain; ++s) {
    if (!in_regs) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = sm[fphys(pencil_base + (p + P * r) * escale)];
      __syncthreads();
    }
    const int k = p & (Ns - 1);
    constexpr int NB = (R == 32) ? 5 : 4;
    if (k) main_twiddle<C, R>(v, stw + a.stw_off[s] + k * NB);
    if constexpr (TC) {
      if (in_regs) __syncthreads();  // the tile may hold the input gather's staging
      tc_dft32_regs(v, *tcx, a);
    } else {
      dft_pow2<C, R>(v);
    }
    if (s + 1 < a.fast_nmain) {
      const int ob = (p - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[fphys(pencil_base + (ob + r * Ns) * escale)] = v[r];
      __syncthreads();
      in_regs = false;
    }
    Ns *= R;
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Start the copy of the stage twiddle table into shared memory (completed
// by cp_async_wait_all + a barrier before the first main stage).
template <typename C>
__device__ __forceinline__ C* stage_table(C* sm, const PassArgs& a) {
  C* stw = sm + a.stw_smem_off;
  const int chunks = a.stw_n * int(sizeof(C)) / 16;
  const char* src = static_cast<const char*>(a.stw_g);
  for (int i = threadIdx.x; i < chunks; i += blockDim.x)
    cp_async16(reinterpret_cast<char*>(stw) + 16 * i, src + 16 * i);
  return stw;
}

// Column position of mu_D (the permutation PI of the workspace).
__device__ __forceinline__ int col_pos(const PassArgs& a, int mu) {
  if (a.pi_arith) {
    const int span = 1 << a.pi_lspan;
    return ((mu & ((1 << a.pi_lg) - 1)) << a.pi_lspan) | (((mu >> a.pi_lg) * a.pi_inv) & (span - 1));
  }
  return __ldg(a.PI + mu);
}

// Box point of lambda_D g_D (the gather table Btab), from the small table bz
// when the last generator is the fastest input coordinate.
template <int DIM, int TS>
__device__ __forceinline__ void gather_point(const PassArgs& a, int e, int* bt) {
  if (a.bz_arith) {
    const int q = e >> a.bz_lh;
#pragma unroll
    for (int r = 0; r < 3; ++r) bt[r] = (r < DIM - 1) ? a.bz[q][r] : 0;
    bt[DIM - 1] = e & ((1 << a.bz_lh) - 1);
    bt[3] = 0;
  } else {
    load_point<TS>(a.Btab, e, bt);
  }
}

// Row pass, power-of-two nD.  Thread (t, p): pencil (row) t, elements
// p + P k.  Consecutive threads hold consecutive elements of a row.
template <typename C, int R, int DIM, bool TC = false>
__global__ void __launch_bounds__(kMaxThreads, 1) row_fast_kernel(PassArgs a) {
  constexpr int TS = DIM <= 2 ? 2 : 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* stw = stage_table(sm, a);
  TcRegs tcx;
  if constexpr (TC) tc_regs_begin(tcx, smem_raw, a.tc_off, reinterpret_cast<const float2*>(a.tw), a.tw_n);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)blockIdx.y * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)blockIdx.y * a.m;
  const int L = a.L;
  const int P = L / R;
  const int t = threadIdx.x / P;
  const int p = threadIdx.x - t * P;
  const int row = int(blockIdx.x) * a.T + t;
  const bool live = row < a.LB;
  const int rowc = live ? row : 0;
  C v[R];
  int at[4], bt[4];
  if (a.load_mode == MAP_BOX_H) {
    load_point<TS>(a.Atab, rowc, at);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      gather_point<DIM, TS>(a, p + P * k, bt);
      v[k] = __ldg(in + box_sum_slot_t<DIM>(a.boxH, at, bt));
    }
  } else if (a.load_mode == MAP_WS) {
    const C* src = in + rowc * a.nD;
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = __ldg(src + col_pos(a, p + P * k));
  } else {
    load_point<TS>(a.Ctab, rowc, at);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      load_point<TS>(a.Etab, col_pos(a, p + P * k), bt);
      v[k] = __ldg(in + box_sum_slot_t<DIM>(a.boxG, at, bt));
    }
  }
  if (a.conj_in) {
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = cconj(v[k]);
  }
  if (a.fs_na > 1 && a.load_mode == MAP_WS) {
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = cmul(v[k], fs_twiddle<C>(a, rowc, p + P * k));
  }
  cp_async_wait_all();
  __syncthreads();
  fast_pencil_dft<C, R, false, TC>(v, sm, stw, a, p, t * L, 1, L, &tcx);
  if constexpr (TC) tc_regs_end(tcx);
  if (!live) return;
  using Rl = decltype(C::x);
  const Rl sc = Rl(a.scale);
  if (a.store_mode == MAP_WS) {
    C* dst = out + row * a.nD;
    if (a.fs_na > 1) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = cmul(v[k], fs_twiddle<C>(a, row, p + P * k));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) dst[col_pos(a, p + P * k)] = v[k];
  } else {
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = cscale(a.conj_out ? cconj(v[k]) : v[k], sc);
    if (a.store_mode == MAP_BOX_H) {
      load_point<TS>(a.Atab, row, at);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        gather_point<DIM, TS>(a, p + P * k, bt);
        out[box_sum_slot_t<DIM>(a.boxH, at, bt)] = v[k];
      }
    } else {
      load_point<TS>(a.Ctab, row, at);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        load_point<TS>(a.Etab, col_pos(a, p + P * k), bt);
        out[box_sum_slot_t<DIM>(a.boxG, at, bt)] = v[k];
      }
    }
  }
}

// Column pass, one non-trivial cycle before the last (a single pencil axis of
// length LB, a power of two).  Thread (t, p), t fastest: column p0 + t, rows
// p + P k.  Workspace loads are coalesced in t; the sheared box store (or
// load, inverse) goes through shared memory in the walk of fft_kernels.cuh.
template <typename C, int R, int DIM, bool TC = false>
__global__ void __launch_bounds__(kMaxThreads, 1) col_fast_kernel(PassArgs a) {
  constexpr int TS = DIM <= 2 ? 2 : 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* stw = stage_table(sm, a);
  TcRegs tcx;
  if constexpr (TC) tc_regs_begin(tcx, smem_raw, a.tc_off, reinterpret_cast<const float2*>(a.tw), a.tw_n);
  const C* __restrict__ in = static_cast<const C*>(a.in) + (int64_t)blockIdx.y * a.m;
  C* __restrict__ out = static_cast<C*>(a.out) + (int64_t)blockIdx.y * a.m;
  const int T = a.T;
  const int P = a.L / R;
  const int tcol = threadIdx.x & (T - 1);
  const int p = threadIdx.x >> a.logT;
  const int p0 = blockIdx.x * T;
  const int LB = a.LB;
  int et[4], ct[4];
  load_point<TS>(a.Etab, p0 + tcol, et);
  // the sheared walk: thread (tcol, .) visits rows (j + tcol * alpha) mod LB
  const int off = int((int64_t(tcol) * a.alpha[0]) % LB);
  const int nthr = blockDim.x;
  C v[R];
  if (a.load_mode == MAP_WS) {
    const C* src = in + p0 + tcol;
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = __ldg(src + (p + P * k) * a.nD);
    if (a.conj_in) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = cconj(v[k]);
    }
    cp_async_wait_all();
    __syncthreads();
  } else {
    // gather in the sheared walk into shared memory, then pick up p + P k
#pragma unroll 4
    for (int w = threadIdx.x; w < LB * T; w += nthr) {
      int i = (w >> a.logT) + off;
      if (i >= LB) i -= LB;
      load_point<TS>(a.Ctab, i, ct);
      C x = __ldg(in + box_sum_slot_t<DIM>(a.boxG, ct, et));
      sm[fphys(i * T + tcol)] = a.conj_in ? cconj(x) : x;
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = sm[fphys((p + P * k) * T + tcol)];
    __syncthreads();
  }
  fast_pencil_dft<C, R, true, TC>(v, sm, stw, a, p, tcol, T, a.L, &tcx);
  if constexpr (TC) tc_regs_end(tcx);
  using Rl = decltype(C::x);
  const Rl sc = Rl(a.scale);
  if (a.store_mode == MAP_WS) {
    C* dst = out + p0 + tcol;
#pragma unroll
    for (int k = 0; k < R; ++k) dst[(p + P * k) * a.nD] = v[k];
  } else {
    __syncthreads();  // the last stage's shared-memory reads are done
#pragma unroll
    for (int k = 0; k < R; ++k) sm[fphys((p + P * k) * T + tcol)] = v[k];
    __syncthreads();
#pragma unroll 4
    for (int w = threadIdx.x; w < LB * T; w += nthr) {
      int i = (w >> a.logT) + off;
      if (i >= LB) i -= LB;
      C x = sm[fphys(i * T + tcol)];
      if (a.conj_out) x = cconj(x);
      load_point<TS>(a.Ctab, i, ct);
      out[box_sum_slot_t<DIM>(a.boxG, ct, et)] = cscale(x, sc);
    }
  }
}

}  // namespace pfft
