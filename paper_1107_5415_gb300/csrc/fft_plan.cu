// Host planner and C entry points for the pattern FFT (setup is host-side,
// exact integers; every transform step runs in the kernels of fft_kernels.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pfft.h"
#include "fft_plan.hpp"
#include "fft_tc.cuh"
#include "lattice.hpp"
#include "plan_common.hpp"
#include "plan_internal.hpp"

using namespace pfft;

namespace {

// Radices for a cycle length: primes from 11 up first (direct stages, up to
// kMaxDirectRadix), then 16s, the rest of the power of two and 3, 5, 7 -- the
// execution order of the stage regions.  Returns false if a prime factor is
// not supported.
// max2: the largest power-of-two radix (16, or 8 for the schedules the batch
// autotuner may pick instead).
bool factor_radices(int n, std::vector<int>& out, bool tc = false, int max2 = 16) {
  out.clear();
  for (int p = kMinDirectRadix; p <= kMaxDirectRadix && p <= n; p += 2) {
    bool prime = true;
    for (int q = 3; q * q <= p; q += 2)
      if (p % q == 0) {
        prime = false;
        break;
      }
    if (!prime) continue;
    while (n % p == 0) {
      out.push_back(p);
      n /= p;
    }
  }
  int p2 = 0;
  while (n % 2 == 0) {
    n /= 2;
    ++p2;
  }
  while (tc && p2 >= 5) {  // tensor-core passes: radix-32 stages first
    out.push_back(32);
    p2 -= 5;
  }
  while (max2 >= 16 && p2 >= 4) {
    out.push_back(16);
    p2 -= 4;
  }
  while (p2 >= 3) {
    out.push_back(8);
    p2 -= 3;
  }
  if (p2 == 2) out.push_back(4);
  if (p2 == 1) out.push_back(2);
  static const int primes[] = {3, 5, 7};
  for (int p : primes)
    while (n % p == 0) {
      out.push_back(p);
      n /= p;
    }
  return n == 1;
}

void set_box(BoxDesc& B, const IMat& H) {
  std::memset(&B, 0, sizeof(B));
  B.d = H.d;
  for (int i = 0; i < H.d; ++i)
    for (int j = 0; j < H.d; ++j) B.H[i][j] = int(H(i, j));
  int s = 1;
  for (int r = H.d - 1; r >= 0; --r) {
    B.stride[r] = s;
    s *= int(H(r, r));
  }
}

// Stages of a Stockham DFT along one pencil axis of length a and stride
// sigma, in the radix order of kRadixOrder (Ns accumulates in that order);
// twiddles come from a table of order nD (a multiple of a).
// Smallest primitive root of the prime p (g^((p-1)/f) != 1 for every prime f | p - 1).
int primitive_root(int p) {
  std::vector<int> fs;
  int n = p - 1;
  for (int f = 2; f * f <= n; ++f)
    if (n % f == 0) {
      fs.push_back(f);
      while (n % f == 0) n /= f;
    }
  if (n > 1) fs.push_back(n);
  auto powmod = [p](int b, int e) {
    long long r = 1, x = b;
    while (e) {
      if (e & 1) r = r * x % p;
      x = x * x % p;
      e >>= 1;
    }
    return int(r);
  };
  for (int g = 2; g < p; ++g) {
    bool ok = true;
    for (int f : fs)
      if (powmod(g, (p - 1) / f) == 1) {
        ok = false;
        break;
      }
    if (ok) return g;
  }
  return 0;
}

bool axis_stages(std::vector<StageDesc>& out, int a, int sigma, int nD, bool tc, int max2) {
  std::vector<int> rad;
  if (!factor_radices(a, rad, tc, max2)) return false;
  int Ns = 1;
  for (int R : rad) {
    StageDesc s;
    std::memset(&s, 0, sizeof(s));
    s.R = R;
    s.a = a;
    s.aR = a / R;
    s.sigma = sigma;
    s.Ns = Ns;
    s.twstep = nD / (Ns * R);
    s.gen = R >= kMinDirectRadix ? primitive_root(R) : 0;
    s.div_aR.init(uint32_t(s.aR));
    s.div_sigma.init(uint32_t(sigma));
    s.div_Ns.init(uint32_t(Ns));
    out.push_back(s);
    Ns *= R;
  }
  return true;
}

int radix_region(int R) {
  for (int i = 0; i < kDirectRegion; ++i)
    if (kRadixOrder[i] == R) return i;
  if (R == 32) return kTC32Region;
  return R >= kMinDirectRadix && R <= kMaxDirectRadix ? kDirectRegion : -1;
}

// Execution order of the regions: direct prime stages first, then radix 32.
int region_rank(int R) {
  const int reg = radix_region(R);
  return reg == kDirectRegion ? -2 : reg == kTC32Region ? -1 : reg;
}

// Merge the stages of all axes, grouped by radix region (stable, so each
// axis keeps its own order), and fill the per-region counts.
bool set_stages(PassArgs& p, std::vector<StageDesc> all) {
  std::stable_sort(all.begin(), all.end(), [](const StageDesc& x, const StageDesc& y) {
    return region_rank(x.R) < region_rank(y.R);
  });
  if (all.size() > size_t(kMaxStages)) return false;
  p.nstages = int(all.size());
  std::memset(p.cnt, 0, sizeof(p.cnt));
  p.pow2 = 1;
  for (size_t i = 0; i < all.size(); ++i) {
    const int reg = radix_region(all[i].R);
    if (reg < 0) return false;
    p.st[i] = all[i];
    p.cnt[reg] += 1;
    if (reg > 3 && reg != kTC32Region) p.pow2 = 0;  // radix 32 (tensor-core plans) is a power of two
  }
  return true;
}

// Threads needed so that every stage fits its per-thread register budget.
int threads_for(const PassArgs& p, int ept) {
  int need = (p.T * p.L + ept - 1) / ept;
  for (int i = 0; i < p.nstages; ++i) {
    const int R = p.st[i].R;
    if (radix_region(R) == kDirectRegion) {  // the phases of run_direct_stage
      const int nbfly = p.T * (p.L / R), h = (R - 1) / 2;
      const int Q = R >= kDirectQ4MinRadix ? 4 : 2;
      const int cap_main = ept / 8 + (Q == 4 ? 1 : 2);  // kDirectQ4Items / kDirectQ2Items
      const int items = nbfly * ((h + Q - 1) / Q);
      need = std::max(need, (nbfly * h + ept / 2 - 1) / (ept / 2));  // kDirectPre
      need = std::max(need, (items + cap_main - 1) / cap_main);
      need = std::max(need, (nbfly + kDirectZero - 1) / kDirectZero);
      continue;
    }
    const int nb = std::max(1, ept / R);
    const int bfly = p.T * p.L / R;
    need = std::max(need, (bfly + nb - 1) / nb);
  }
  need = ((need + 31) / 32) * 32;
  return need;
}

size_t elem_bytes(int dtype) { return dtype == PFFT_C64 ? 8 : 16; }

// Whether one pencil of length L fits a CTA of the shared-memory kernels:
// at most `row_max` elements and kMaxThreads threads for its stages.
bool tile_fits(int L, int row_max, int ept) {
  if (L > row_max) return false;
  std::vector<int> rad;
  if (!factor_radices(L, rad)) return false;
  PassArgs p;
  std::memset(&p, 0, sizeof(p));
  p.T = 1;
  p.L = L;
  p.nstages = int(rad.size());
  if (p.nstages > kMaxStages) return false;
  for (int i = 0; i < p.nstages; ++i) p.st[i].R = rad[i];
  return threads_for(p, ept) <= kMaxThreads;
}

// Register-resident column pass over two pencil axes (fft_fast2.cuh): the
// 2-D DFT of sizes top x low (top the slower axis of the row index) is the
// 1-D Stockham DFT of length L = top low without the twiddles that couple the
// axes, provided the first stages' radices multiply to top -- a radix-32
// complex64 pass of L = t 32^s (tail t first) has those products t 32^j,
// j < s.  Box layout, complex64, no split-precision stages, no four-step
// split, both axes powers of two.
bool fast2_axes(const pfft_plan_s& P, int top, int low) {
  if (P.dtype != PFFT_C64 || P.tc || P.generic_only || P.fs_na != 1 || P.pen.size() != 2) return false;
  if (top < 2 || low < 2 || (top & (top - 1)) || (low & (low - 1))) return false;
  const int L = top * low;
  if (L < 64 || L > 16384) return false;
  int lg = 0;
  while ((1 << lg) < L) ++lg;
  const int nmain = lg / 5;
  int b = 1 << (lg - 5 * nmain);
  for (int j = 0; j < nmain; ++j, b *= 32)
    if (b == top) return true;
  return false;
}

pfft_status configure_pass(PassArgs& p, const pfft_plan_s& P, bool cols, int T) {
  const int ept = P.dtype == PFFT_C64 ? P.ept_c64 : 16;
  p.cols = cols;
  p.nD = P.nD;
  p.LB = P.LB;
  p.m = int(P.m);
  p.d = P.d;
  p.batch = int(P.batch);
  p.T = T;
  std::vector<StageDesc> stg;
  if (!cols) {
    p.L = P.nD;
    if (!axis_stages(stg, P.nD, 1, P.nD, P.tc, P.max2)) return PFFT_ERR_UNSUPPORTED;
    p.groups = (P.LB + T - 1) / T;
  } else {
    p.L = P.LB;
    int sigma = 1;
    for (int s = int(P.pen.size()) - 1; s >= 0; --s) {  // pencil axes, last fastest
      if (!axis_stages(stg, P.pen[s], sigma, p.tw_n, P.tc, P.max2)) return PFFT_ERR_UNSUPPORTED;
      sigma *= P.pen[s];
    }
    p.groups = (P.nD + T - 1) / T;
  }
  if (!set_stages(p, stg)) return PFFT_ERR_UNSUPPORTED;
  p.divT.init(uint32_t(T));
  p.divnD.init(uint32_t(P.nD));
  p.logT = 0;
  while ((1 << p.logT) < T) ++p.logT;
  // register-resident power-of-two kernels (fft_fast.cuh)
  {
    const int Rm = P.dtype == PFFT_C64 ? 32 : 16;
    const int L = p.L;
    const bool pow2L = L >= Rm && (L & (L - 1)) == 0 && (T & (T - 1)) == 0;
    // split-precision plans use them too, their radix-32 main stages on the tensor cores
    const bool tc_fast = P.tc && P.dtype == PFFT_C64 && p.tw_n % 32 == 0;
    // (a column tile of the register-resident pass holds T whole columns: T divides nD)
    p.fast = ((!P.generic_only || tc_fast) && p.tw_n == P.nD && p.pow2 && pow2L && P.d <= 3 && (!cols || P.pen.size() == 1 || fast2_axes(P, P.pen[0], P.pen[1])) && (!cols || P.nD % T == 0) && T * L <= (P.dtype == PFFT_C64 ? 16384 : 8192)) ? 1 : 0;
    if (p.fast) {
      int lg = 0, lr = 0;
      while ((1 << lg) < L) ++lg;
      while ((1 << lr) < Rm) ++lr;
      p.fast_nmain = lg / lr;
      p.fast_tail = 1 << (lg - p.fast_nmain * lr);
      p.nthreads = T * L / Rm;
      // stage twiddle table: for main stage s (span Ns), w^(2^b) for k < Ns, b < log2 R
      int off = 0, Ns = p.fast_tail;
      for (int s = 0; s < p.fast_nmain; ++s) {
        p.stw_off[s] = off;
        off += Ns * lr;
        Ns *= Rm;
      }
      p.stw_n = (off + 1) & ~1;
      const int nel = T * L;
      p.stw_smem_off = (nel + (nel >> 5) + 1) & ~1;
      p.smem_bytes = int(size_t(p.stw_smem_off + p.stw_n) * elem_bytes(P.dtype));
      bool ok = true;
      if (P.tc) {  // W (radix 32), mbarrier and tensor-memory address after the stage table (fft_tc.cuh)
        p.tc = 1;
        p.tc_off = (p.smem_bytes + 15) & ~15;
        p.smem_bytes = p.tc_off + tc_regs_extra_bytes();
        ok = p.nthreads % 128 == 0 && p.fast_nmain >= 1;
      }
      if (ok && p.nthreads <= kMaxThreads && p.smem_bytes <= 227 * 1024 && p.fast_nmain <= 4) return PFFT_OK;
      p.fast = 0;
      p.tc = 0;
    }
  }
  // generic kernels: 16 points per thread (64 registers, two CTAs per SM)
  // when the tile fits 512 threads, else 32; the tensor-core stages need 32
  p.ept = ept;
  if (P.dtype == PFFT_C64 && !P.tc && ept == 32 && threads_for(p, 16) <= kMaxThreads) p.ept = 16;
  p.nthreads = threads_for(p, p.ept);
  if (cols && T > 32) p.nthreads = (p.nthreads + T - 1) / T * T;  // each thread keeps one column
  if (p.nthreads > kMaxThreads) return PFFT_ERR_UNSUPPORTED;
  const int nel = T * p.L;
  int rmax = 0;  // omega_R table of the direct stages, after the tile
  for (int i = 0; i < p.nstages; ++i)
    if (radix_region(p.st[i].R) == kDirectRegion) rmax = std::max(rmax, p.st[i].R);
  p.pad = rmax ? 0 : 1;
  p.dir_off = p.pad ? (nel - 1) + ((nel - 1) >> 4) + 1 : nel;
  // direct-stage tables: omega_R^{g^t} (R - 1 complex) and g^t (R - 1 int), with slack
  p.smem_bytes = int(size_t(p.dir_off + 2 * rmax) * elem_bytes(P.dtype));
  p.tc = P.tc ? 1 : 0;
  p.tc_off = (p.smem_bytes + 15) & ~15;
  if (p.tc) {  // tensor-core stages (fft_tc.cuh), in the 32-points-per-thread kernels only
    if (p.ept != 32) return PFFT_ERR_UNSUPPORTED;
    // the hi / lo rows of a stage's 128-butterfly chunks overwrite the tile
    for (int i = 0; i < p.nstages; ++i) {
      const int R = p.st[i].R;
      if (R != 16 && R != 32) continue;
      const int nch = (T * p.L / R + 127) / 128;
      p.tc_off = std::max(p.tc_off, nch * tc_chunk_bytes(R));
    }
    p.tc_off = (p.tc_off + 15) & ~15;
    p.smem_bytes = tc_layout(p.tc_off, p.cnt[kTC32Region] > 0, p.cnt[0] > 0, T * p.L / 16).end;
    // every warp of a lane quarter reads its rows of the accumulator: whole warp quadruples
    p.nthreads = (p.nthreads + 127) / 128 * 128;
    if (p.nthreads > kMaxThreads || tc_tmem_cols(T * p.L, p.cnt[kTC32Region] > 0, p.cnt[0] > 0) > 256)
      return PFFT_ERR_UNSUPPORTED;
  }
  if (p.smem_bytes > 227 * 1024) return PFFT_ERR_UNSUPPORTED;
  return PFFT_OK;
}

// Choose the pencils-per-CTA count: the largest power of two (<= cap) whose
// tile fits `budget` elements and the thread limit.
pfft_status choose_and_configure(PassArgs& p, const pfft_plan_s& P, bool cols, int cap, int budget) {
  const int L = cols ? P.LB : P.nD;
  const int limit = cols ? P.nD : P.LB;
  int T = 1;
  while (T * 2 <= cap && T * 2 <= limit && T * 2 * L <= budget) T *= 2;
  for (;;) {
    pfft_status st = configure_pass(p, P, cols, T);
    if (st == PFFT_OK) return st;
    if (T == 1) return st;
    T /= 2;
  }
}

}  // namespace

// ----------------------------------------------------------------- planning
pfft_status pfft::plan_host(pfft_plan_s& P, int d, const int64_t* Mv) {
  if (d < 1 || d > 4) return PFFT_ERR_ARG;
  P.d = d;
  P.M = IMat(d);
  for (int i = 0; i < d * d; ++i) {
    if (Mv[i] >= (int64_t(1) << 24) || Mv[i] <= -(int64_t(1) << 24)) return PFFT_ERR_OVERFLOW;
    P.M.a[i] = Mv[i];
  }
  const i64 det = determinant(P.M);
  if (det == 0) return PFFT_ERR_SINGULAR;
  P.m = det < 0 ? -det : det;
  if (P.m >= (i64(1) << 31)) return PFFT_ERR_OVERFLOW;
  P.H = hermite_normal_form(P.M);
  P.G = hermite_normal_form(P.M.transpose());
  IMat Q, R, U, V;
  smith_normal_form(P.M, Q, P.eps, R, U, V);
  // lambda = Q^{-1} y = U y mod eps ;  mu = R^{-T} k = V^T k mod eps
  std::vector<std::vector<i64>> LAM(d, std::vector<i64>(d)), MU(d, std::vector<i64>(d));
  for (int j = 0; j < d; ++j)
    for (int c = 0; c < d; ++c) {
      LAM[j][c] = posmod(U(j, c), P.eps[j]);
      MU[j][c] = posmod(V(c, j), P.eps[j]);
    }
  // Remark 2: any biorthogonal pair of bases works.  If the fastest input
  // coordinate e_f generates a cycle of maximal length, re-base so that it is
  // the generator of the last cycle; then the row pass reads contiguous runs.
  {
    const int f = d - 1;
    const i64 E = P.eps[d - 1];
    int j0 = -1;
    for (int j = d - 1; j >= 0; --j)
      if (P.eps[j] == E && gcd64(LAM[j][f], E) == 1) {
        j0 = j;
        break;
      }
    if (j0 >= 0 && E > 1) {
      std::vector<i64> v(d);
      for (int j = 0; j < d; ++j) v[j] = LAM[j][f] % P.eps[j];
      const i64 u = modinv(v[j0], E);
      auto L2 = LAM, M2 = MU;
      for (int c = 0; c < d; ++c) L2[j0][c] = posmod(i64((i128)u * LAM[j0][c] % E), E);
      for (int j = 0; j < d; ++j) {
        if (j == j0) continue;
        for (int c = 0; c < d; ++c) {
          i128 t = (i128)LAM[j][c] - (i128)v[j] * u % P.eps[j] * LAM[j0][c];
          L2[j][c] = posmod(i64(t % P.eps[j]), P.eps[j]);
        }
      }
      for (int c = 0; c < d; ++c) {
        i128 s = 0;
        for (int i = 0; i < d; ++i) s += (i128)v[i] * (E / P.eps[i]) % E * MU[i][c];
        M2[j0][c] = posmod(i64(s % E), E);
      }
      std::swap(L2[j0], L2[d - 1]);
      std::swap(M2[j0], M2[d - 1]);
      LAM = L2;
      MU = M2;
    }
  }
  P.D = 0;
  P.n.clear();
  P.LAM.clear();
  P.MU.clear();
  for (int j = 0; j < d; ++j)
    if (P.eps[j] > 1) {
      P.n.push_back(int(P.eps[j]));
      P.LAM.push_back(LAM[j]);
      P.MU.push_back(MU[j]);
      ++P.D;
    }
  if (P.D > 3) return PFFT_ERR_UNSUPPORTED;
  P.fs_N = P.D ? P.n[P.D - 1] : 1;
  P.fs_na = 1;
  P.nD = int(P.fs_N);
  P.pen.assign(P.n.begin(), P.n.end() - (P.D ? 1 : 0));
  // A last cycle longer than one row tile is split four-step style,
  // n = n_a n_b with lambda = lambda_a + n_a lambda_b: the row pass runs the
  // length-n_b DFTs (twiddle exp(-2 pi i lambda_a mu_b / n) between the passes)
  // and lambda_a becomes one more pencil axis of the column pass.
  const int row_max = P.dtype == PFFT_C64 ? 16384 : 8192;
  const int ept = P.dtype == PFFT_C64 ? P.ept_c64 : 16;
  if (P.fs_N > 1 && !tile_fits(int(std::min<i64>(P.fs_N, row_max + 1)), row_max, ept)) {
    const i64 other = P.m / P.fs_N;
    int best = 0;
    for (i64 nb = std::min<i64>(row_max, P.fs_N - 1); nb >= 2; --nb) {
      if (P.fs_N % nb) continue;
      const i64 na = P.fs_N / nb;
      if (other * na > row_max || !tile_fits(int(nb), row_max, ept) || !tile_fits(int(other * na), row_max, ept))
        continue;
      best = int(nb);
      break;
    }
    if (!best) return PFFT_ERR_UNSUPPORTED;
    P.nD = best;
    P.fs_na = int(P.fs_N / best);
    P.pen.push_back(P.fs_na);
  }
  if (P.pen.size() > size_t(kMaxSub)) return PFFT_ERR_UNSUPPORTED;
  P.LB = int(P.m / P.nD);
  return PFFT_OK;
}

namespace {
// g_j = M MU_j^T / n_j  (in box(H));  h_j = M^T LAM_j^T / n_j  (in box(G)).
std::vector<i64> generator(const IMat& A, const std::vector<i64>& row, i64 nj, const IMat& box) {
  const int d = A.d;
  std::vector<i64> g(d);
  for (int i = 0; i < d; ++i) {
    i128 s = 0;
    for (int c = 0; c < d; ++c) s += (i128)A(i, c) * row[c];
    if (s % nj != 0) throw LatticeError{PFFT_ERR_OVERFLOW, "generator is not integral"};
    g[i] = i64(s / nj);
  }
  box_reduce(box, g.data());
  return g;
}

std::vector<i64> combo(const std::vector<std::vector<i64>>& gens, const std::vector<i64>& coef,
                       const IMat& box) {
  const int d = box.d;
  std::vector<i64> y(d, 0);
  for (size_t j = 0; j < gens.size(); ++j)
    for (int r = 0; r < d; ++r) y[r] += coef[j] * gens[j][r];  // < 2^62: coef, gens < 2^31
  box_reduce(box, y.data());
  return y;
}
}  // namespace

pfft_status pfft::plan_device(pfft_plan_s& P) {
  const int d = P.d, D = P.D;
  if (cudaGetDevice(&P.device) != cudaSuccess) return PFFT_ERR_CUDA;
  if (D == 0) return PFFT_OK;  // m == 1: the transform is the identity
  // generators of the cycles
  std::vector<std::vector<i64>> g(D), h(D);
  for (int j = 0; j < D; ++j) {
    g[j] = generator(P.M, P.MU[j], P.n[j], P.H);
    h[j] = generator(P.M.transpose(), P.LAM[j], P.n[j], P.G);
  }
  // biorthogonality check (Lemma 1 / Remark 2), exact
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      i128 a = 0, b = 0;
      for (int c = 0; c < d; ++c) {
        a += (i128)P.LAM[i][c] * g[j][c];
        b += (i128)P.MU[i][c] * h[j][c];
      }
      const i64 want = (i == j) ? 1 : 0;
      if (posmod(i64(a % P.n[i]), P.n[i]) != want || posmod(i64(b % P.n[i]), P.n[i]) != want)
        return PFFT_ERR_OVERFLOW;
    }
  const int nD = P.nD, LB = P.LB;
  const int na = P.fs_na;
  const int npen = int(P.pen.size());
  // two pencil axes of which only the faster one starts a register-resident
  // column pass (fast2_axes): make it the slower axis of the row index (the
  // rows then run over (lambda_2, lambda_1); the tables below follow)
  const bool swap2 = npen == 2 && na == 1 && !fast2_axes(P, P.pen[0], P.pen[1]) && fast2_axes(P, P.pen[1], P.pen[0]);
  if (swap2) std::swap(P.pen[0], P.pen[1]);
  // Row (A, B) and column (C, E) generator lists of the logical LB x nD array:
  //   row index  = flatten(lambda_1..lambda_{D-1}[, lambda_a]),  element = lambda_b
  //   col index  = flatten(mu_1..mu_{D-1}[, mu_a]),              position of mu_b
  // with lambda_D = lambda_a + n_a lambda_b and mu_D = mu_b + n_b mu_a when the
  // last cycle is split (n_a > 1); otherwise lambda_b = lambda_D, mu_b = mu_D.
  std::vector<std::vector<i64>> genA(g.begin(), g.end() - 1), genC(h.begin(), h.end() - 1);
  if (swap2) {
    std::swap(genA[0], genA[1]);
    std::swap(genC[0], genC[1]);
  }
  std::vector<i64> gB = g[D - 1], hE = h[D - 1];
  if (na > 1) {
    genA.push_back(g[D - 1]);
    std::vector<i64> hb(d), gb(d);
    for (int k = 0; k < d; ++k) {
      hb[k] = h[D - 1][k] * nD;  // n_b h_D (|h| < 2^31, n_b <= 2^14)
      gb[k] = g[D - 1][k] * na;  // n_a g_D
    }
    box_reduce(P.G, hb.data());
    box_reduce(P.H, gb.data());
    genC.push_back(hb);
    gB = gb;
  }
  // column permutation PI for the column pass (see fft_plan.hpp)
  std::vector<int> PI(nD), PIinv(nD);
  std::vector<int> alpha(3, 0);
  {
    const i64 cf = posmod(P.MU[D - 1][d - 1], P.fs_N);  // mu_D of the fastest output coordinate
    i64 beta = cf % nD;
    for (int j = 0; j + 1 < D; ++j) alpha[j] = int(posmod(P.MU[j][d - 1], P.n[j]));
    if (na > 1) alpha[npen - 1] = int((cf / nD) % na);
    if (swap2) std::swap(alpha[0], alpha[1]);
    const i64 gg = beta == 0 ? nD : gcd64(beta, nD);
    const i64 span = nD / gg;
    const i64 inv = span > 1 ? modinv(beta / gg, span) : 0;
    for (i64 mu = 0; mu < nD; ++mu) {
      const i64 pos = (mu % gg) * span + ((mu / gg) * inv) % span;
      PI[mu] = int(pos);
      PIinv[pos] = int(mu);
    }
  }
  // index tables
  const int ts = d <= 2 ? 2 : 4;  // int32 per entry, so that one vector load fetches a point
  std::vector<int> tab(size_t(2 * LB + 2 * nD) * ts + 2 * nD, 0);
  int* Atab = tab.data();
  int* Btab = Atab + size_t(LB) * ts;
  int* Ctab = Btab + size_t(nD) * ts;
  int* Etab = Ctab + size_t(LB) * ts;
  int* PIi = Etab + size_t(nD) * ts;
  int* PIf = PIi + nD;
  std::vector<i64> coef(npen);
  for (int r = 0; r < LB; ++r) {
    int x = r;
    for (int j = npen - 1; j >= 0; --j) {
      coef[j] = x % P.pen[j];
      x /= P.pen[j];
    }
    auto a = combo(genA, coef, P.H);
    auto c = combo(genC, coef, P.G);
    for (int k = 0; k < d; ++k) {
      Atab[size_t(r) * ts + k] = int(a[k]);
      Ctab[size_t(r) * ts + k] = int(c[k]);
    }
  }
  for (int e = 0; e < nD; ++e) {
    auto b = combo({gB}, {e}, P.H);
    auto c = combo({hE}, {PIinv[e]}, P.G);
    for (int k = 0; k < d; ++k) {
      Btab[size_t(e) * ts + k] = int(b[k]);
      Etab[size_t(e) * ts + k] = int(c[k]);
    }
    PIi[e] = PIinv[e];
    PIf[e] = PI[e];
  }
  if (int e_ = P.alloc((void**)&P.dtab, tab.size() * sizeof(int))) return pfft_status(e_);
  if (cudaMemcpy(P.dtab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return PFFT_ERR_CUDA;
  const size_t eb = elem_bytes(P.dtype);
  if (int e_ = P.alloc((void**)&P.tw, size_t(nD) * eb)) return pfft_status(e_);
  if (int e_ = P.alloc((void**)&P.status, sizeof(int))) return pfft_status(e_);
  cudaMemset(P.status, 0, sizeof(int));
  if (launch_twiddles(P.tw, nD, P.dtype, 0) != 0) return PFFT_ERR_CUDA;
  // The column pass transforms the pencil axes; their twiddles come from the
  // nD table when every axis divides nD (always, unless the last cycle is
  // split four-step: n_a need not divide n_b), else from a table of order
  // lcm(axes) <= LB.
  int col_n = nD;
  {
    i64 l = 1;
    for (int a : P.pen) l = l / gcd64(l, a) * a;
    if (npen >= 1 && nD % l != 0) {
      col_n = int(l);
      if (int e_ = P.alloc(&P.tw_col, size_t(col_n) * eb)) return pfft_status(e_);
      if (launch_twiddles(P.tw_col, col_n, P.dtype, 0) != 0) return PFFT_ERR_CUDA;
    }
  }
  if (npen >= 1 && P.own_workspace)
    if (int e_ = P.alloc(&P.ws, size_t(P.m) * P.batch * eb)) return pfft_status(e_);
  if (na > 1) {  // exp(-2 pi i t / n) for t < n, as lo[t & 2047] * hi[t >> 11]
    const int nhi = int((P.fs_N + 2047) >> 11);
    if (int e_ = P.alloc(&P.fs_tab, size_t(2048 + nhi) * eb)) return pfft_status(e_);
    if (launch_phase_tables(P.fs_tab, P.fs_N, nhi, P.dtype, 0) != 0) return PFFT_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return PFFT_ERR_CUDA;

  // pass descriptors (data pointers and modes are filled per call)
  // arithmetic forms of PI and of the gather table (power-of-two cycles)
  PassArgs arith;
  std::memset(&arith, 0, sizeof(arith));
  {
    const i64 beta = posmod(P.MU[D - 1][d - 1], nD);
    const i64 gg = beta == 0 ? nD : gcd64(beta, nD);
    const i64 span = nD / gg;
    auto lg2 = [](i64 v) { int l = 0; while ((i64(1) << l) < v) ++l; return (i64(1) << l) == v ? l : -1; };
    if (lg2(gg) >= 0 && lg2(span) >= 0) {
      arith.pi_arith = 1;
      arith.pi_lg = lg2(gg);
      arith.pi_lspan = lg2(span);
      arith.pi_inv = int(span > 1 ? modinv(beta / gg, span) : 0);
    }
    // Btab[e] = (Z[e / H_ff], e mod H_ff) when g_D = e_f (the last input coordinate) and H_ff | nD
    const i64 Hff = P.H(d - 1, d - 1);
    bool unit = true;
    std::vector<i64> ef(d, 0);
    ef[d - 1] = 1;
    {
      std::vector<i64> gD = g[D - 1];
      std::vector<i64> e1 = ef;
      box_reduce(P.H, e1.data());
      unit = (gD == e1);
    }
    const int lh = int(lg2(Hff));
    if (unit && lh >= 0 && nD % Hff == 0 && nD / Hff <= 64 && d <= 3) {
      arith.bz_arith = 1;
      arith.bz_lh = lh;
      for (i64 q = 0; q < nD / Hff; ++q) {
        const int* b = Btab + size_t(q * Hff) * ts;
        for (int r = 0; r + 1 < d; ++r) arith.bz[q][r] = b[r];
        if (b[d - 1] != 0) arith.bz_arith = 0;
      }
      for (int e = 0; e < nD && arith.bz_arith; ++e) {  // exact check against the table
        const int* b = Btab + size_t(e) * ts;
        for (int r = 0; r + 1 < d; ++r)
          if (b[r] != arith.bz[e >> lh][r]) arith.bz_arith = 0;
        if (b[d - 1] != (e & ((1 << lh) - 1))) arith.bz_arith = 0;
      }
    }
    if (arith.pi_arith)
      for (int mu = 0; mu < nD; ++mu) {  // exact check against the table
        const int span_i = 1 << arith.pi_lspan;
        const int pos = ((mu & ((1 << arith.pi_lg) - 1)) << arith.pi_lspan) |
                        (((mu >> arith.pi_lg) * arith.pi_inv) & (span_i - 1));
        if (pos != PI[mu]) {
          arith.pi_arith = 0;
          break;
        }
      }
  }
  const int budget = P.dtype == PFFT_C64 ? 8192 : 4096;
  for (PassArgs* p : {&P.rowp, &P.colp}) {
    std::memset(p, 0, sizeof(PassArgs));
    p->Atab = Atab - tab.data() + P.dtab;
    p->Btab = Btab - tab.data() + P.dtab;
    p->Ctab = Ctab - tab.data() + P.dtab;
    p->Etab = Etab - tab.data() + P.dtab;
    p->PIinv = PIi - tab.data() + P.dtab;
    p->PI = PIf - tab.data() + P.dtab;
    const bool colt = (p == &P.colp) && P.tw_col;
    p->tw = colt ? P.tw_col : P.tw;
    p->tw_n = colt ? col_n : nD;
    p->ts = ts;
    p->status = P.status;
    p->spin_limit = kSpinLimit;
    set_box(p->boxH, P.H);
    set_box(p->boxG, P.G);
    p->pi_arith = arith.pi_arith;
    p->pi_lg = arith.pi_lg;
    p->pi_lspan = arith.pi_lspan;
    p->pi_inv = arith.pi_inv;
    p->bz_arith = arith.bz_arith;
    p->bz_lh = arith.bz_lh;
    std::memcpy(p->bz, arith.bz, sizeof(arith.bz));
    p->nsub = npen;
    for (int s = 0; s < npen; ++s) {
      p->sub_n[s] = P.pen[s];
      p->sub_div[s].init(uint32_t(P.pen[s]));
      p->alpha[s] = alpha[s];
    }
    p->fs_na = na;
    p->fs_div.init(uint32_t(na));
    p->fs_lo = P.fs_tab;
    p->fs_hi = P.fs_tab ? static_cast<const char*>(P.fs_tab) + size_t(2048) * eb : nullptr;
  }
  pfft_status st = choose_and_configure(P.rowp, P, false, 64, std::max(budget, nD));
  if (st != PFFT_OK) return st;
  if (npen >= 1) {
    // generic column tiles may hold many short columns (split last cycles)
    st = choose_and_configure(P.colp, P, true, P.generic_only ? 512 : 16, std::max(budget, LB));
    if (st != PFFT_OK) return st;
  }
  // stage twiddle tables of the register-resident passes, gathered on the
  // device from the FP64-built table: entry (s, k, b) = omega_{Ns R}^(k 2^b)
  std::vector<int> idx;
  std::vector<PassArgs*> fastp;
  for (PassArgs* p : {&P.rowp, &P.colp})
    if (p->fast && (p == &P.rowp || npen >= 1)) fastp.push_back(p);
  std::vector<size_t> base;
  for (PassArgs* p : fastp) {
    const int Rm = P.dtype == PFFT_C64 ? 32 : 16;
    const int lr = Rm == 32 ? 5 : 4;
    base.push_back(idx.size());
    // two pencil axes (fft_fast2.cuh): from span top on, the twiddle of k at
    // span Ns is that of floor(k / top) at span Ns / top (the axes uncoupled)
    const int top = (p == &P.colp && p->nsub == 2) ? p->sub_n[0] : 0;
    int Ns = p->fast_tail;
    for (int s = 0; s < p->fast_nmain; ++s) {
      const bool two = top && Ns >= top;
      const int NsR = (two ? Ns / top : Ns) * Rm;
      for (int k = 0; k < Ns; ++k) {
        const int kk = two ? k / top : k;
        for (int b = 0; b < lr; ++b) idx.push_back(int(((int64_t(kk) << b) % NsR) * (nD / NsR)));
      }
      Ns *= Rm;
    }
    while (idx.size() - base.back() < size_t(p->stw_n)) idx.push_back(0);
  }
  // runs of consecutive box slots along each row, for bulk-copy staging
  if (P.rowp.fast && !P.tc && P.rowp.T == 1 && npen >= 1 && (P.m * elem_bytes(P.dtype)) % 16 == 0) {
    std::vector<std::array<int, 4>> runs;
    int maxr = 0;
    bool ok = true;
    std::vector<std::vector<std::array<int, 4>>> per(LB);
    std::vector<i64> y(d);
    auto slot_of = [&](int r, int e) {
      for (int k = 0; k < d; ++k) y[k] = i64(Atab[size_t(r) * ts + k]) + Btab[size_t(e) * ts + k];
      box_reduce(P.H, y.data());
      return box_slot(P.H, y.data());
    };
    const int align = int(16 / elem_bytes(P.dtype));  // elements per 16 bytes
    for (int r = 0; r < LB && ok; ++r) {
      i64 start = slot_of(r, 0), prev = start;
      int e0 = 0;
      for (int e = 1; e <= nD && ok; ++e) {
        const i64 s = e < nD ? slot_of(r, e) : -2;
        if (s != prev + 1) {
          const int len = e - e0;
          if (e0 % align || start % align || len % align) ok = false;
          per[r].push_back({e0, int(start), len, 0});
          e0 = e;
          start = s;
        }
        prev = s;
      }
      maxr = std::max<int>(maxr, int(per[r].size()));
      if (maxr > 64 || maxr > P.rowp.nthreads) ok = false;
    }
    if (ok) {
      std::vector<int> flat(size_t(LB) * maxr * 4, 0);
      for (int r = 0; r < LB; ++r)
        for (size_t j = 0; j < per[r].size(); ++j)
          for (int k = 0; k < 4; ++k) flat[(size_t(r) * maxr + j) * 4 + k] = per[r][j][k];
      if (int e_ = P.alloc((void**)&P.runs, flat.size() * sizeof(int))) return pfft_status(e_);
      cudaMemcpy(P.runs, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice);
      P.rowp.tma = 1;
      // padded workspace-order staging (fft_tma.cuh): 2^lg blocks of one
      // span each, offset so that blocks start 32 / 2^lg banks apart (16-byte
      // multiples for the bulk copies)
      P.rowp.stg_pad = 0;
      if (P.rowp.pi_arith && P.rowp.pi_lg > 0 && P.rowp.pi_lg <= 6 && P.rowp.pi_lspan >= 2) {
        const int esz = int(elem_bytes(P.dtype));
        const int pad = std::max(16, 128 >> P.rowp.pi_lg) / esz;  // elements
        const int nel = P.rowp.T * P.rowp.L;
        const int stage_end = nel + (1 << P.rowp.pi_lg) * pad;
        if (stage_end <= P.rowp.stw_smem_off) P.rowp.stg_pad = pad;  // fits before the stage table
      }
      P.rowp.runs = P.runs;
      P.rowp.nruns = maxr;
      P.rowp.bar_smem_off = (P.rowp.smem_bytes + 15) & ~15;
      P.rowp.smem_bytes = P.rowp.bar_smem_off + 16;
      // rows of 2^14 complex64 elements: the persistent pipelined row pass,
      // shared memory [S: the row + staging pads | X: exchange | stage table | mbarrier]
      if (P.dtype == PFFT_C64 && P.rowp.L == (1 << kPipeLogL) && P.rowp.nthreads == 512 &&
          P.rowp.fast_tail == 16 && P.rowp.fast_nmain == 2) {
        const int nblk = P.rowp.stg_pad ? (1 << P.rowp.pi_lg) : 1;
        const int s_el = P.rowp.L + nblk * P.rowp.stg_pad;
        const int x_off = (s_el + 15) & ~15;
        const int stw_off = (x_off + kPipeX + 15) & ~15;
        const int bar_off = ((stw_off + P.rowp.stw_n) * 8 + 15) & ~15;
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P.device) != cudaSuccess || nsm < 1)
          return PFFT_ERR_CUDA;
        if (bar_off + 16 <= 227 * 1024) {
          // outputs stored from registers: the workspace when the permutation
          // multiplier is 1 and lanes form runs of >= 4 elements (32 B); the
          // box when every row is made of runs of one power-of-two length >= 32
          int direct = 0, lrun = 0;
          if (P.rowp.pi_arith && P.rowp.pi_inv == 1 && P.rowp.pi_lg <= 3) direct |= 1;
          for (int l = 5; l <= kPipeLogL && !(direct & 2); ++l) {
            bool uni = maxr == (1 << (kPipeLogL - l));
            for (int r = 0; r < LB && uni; ++r) {
              uni = per[r].size() == size_t(maxr);
              for (size_t j = 0; j < per[r].size() && uni; ++j)
                uni = per[r][j][0] == int(j) << l && per[r][j][2] == 1 << l;
            }
            if (uni) {
              direct |= 2;
              lrun = l;
            }
          }
          P.rowp.pipe_direct = direct;
          P.rowp.pipe_lrun = lrun;
          P.rowp.pipe = 1;
          P.rowp.pipe_x_off = x_off;
          P.rowp.pipe_grid = nsm;
          P.rowp.stw_smem_off = stw_off;
          P.rowp.bar_smem_off = bar_off;
          P.rowp.smem_bytes = bar_off + 16;
        }
      }
    }
  }
  // pencils of 2^10 complex64 points, 8 per tile: the persistent pipelined column pass
  if (npen == 1 && P.dtype == PFFT_C64 && !P.tc && P.colp.fast && P.colp.L == (1 << kCPipeLogL) && P.colp.T == 8 &&
      P.colp.LB == P.colp.L && P.colp.nthreads == 256 && P.colp.fast_tail == 1 && P.colp.fast_nmain == 2 &&
      (d == 2 || d == 3) && P.nD % 8 == 0) {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P.device) != cudaSuccess || nsm < 1)
      return PFFT_ERR_CUDA;
    const int e_off = kCPipeS + kCPipeX;  // 2 x 8 column points of up to 4 int32: 32 elements
    const int stw_off = e_off + 32;
    const int bytes = (stw_off + P.colp.stw_n) * 8;
    if (bytes <= 110 * 1024) {
      P.colp.cpipe = 1;
      P.colp.cpipe_x_off = kCPipeS;
      P.colp.cpipe_e_off = e_off;
      P.colp.cpipe_grid = 2 * nsm;
      P.colp.stw_smem_off = stw_off;
      P.colp.smem_bytes = bytes;
    }
  }
  if (!idx.empty()) {
    int* didx = nullptr;
    if (int e_ = device_alloc((void**)&didx, idx.size() * sizeof(int))) return pfft_status(e_);
    if (int e_ = P.alloc(&P.stw, idx.size() * eb)) {
      cudaFree(didx);
      return pfft_status(e_);
    }
    cudaMemcpy(didx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
    const int rc = launch_twiddle_gather(P.stw, P.tw, didx, int(idx.size()), P.dtype, 0);
    const cudaError_t ce = cudaDeviceSynchronize();
    cudaFree(didx);
    if (rc != 0 || ce != cudaSuccess) return PFFT_ERR_CUDA;
    for (size_t i = 0; i < fastp.size(); ++i)
      fastp[i]->stw_g = static_cast<const char*>(P.stw) + base[i] * eb;
  }
  return PFFT_OK;
}

pfft_status pfft::plan_retile(pfft_plan_s& P, int row_budget, int col_budget, int max2) {
  if (!P.generic_only || P.D == 0 || (max2 != 16 && max2 != 8)) return PFFT_ERR_ARG;
  P.max2 = max2;
  pfft_status st = choose_and_configure(P.rowp, P, false, 64, std::max(row_budget, P.nD));
  if (st != PFFT_OK || P.pen.empty()) return st;
  return choose_and_configure(P.colp, P, true, 512, std::max(col_budget, P.LB));
}

void pfft::plan_release(pfft_plan_s* P) {
  if (!P) return;
  if (P->tr) {
    P->tr->ws = nullptr;  // this plan's workspace
    plan_release(P->tr);
  }
  if (!P->arena) {
    for (void* p : {(void*)P->dtab, P->tw, P->tw_col, P->ws, P->stw, P->fs_tab, (void*)P->runs, (void*)P->status})
      if (p) cudaFree(p);
  }
  delete P;
}
static void release(pfft_plan_s* P) { plan_release(P); }
static pfft_status plan_route(pfft_plan_s& P, int d, const int64_t* M, unsigned flags);

extern "C" pfft_status pfft_plan_create(pfft_plan* out, int d, const int64_t* M, int64_t batch,
                                        int dtype, unsigned flags) {
  if (!out || !M || batch < 1 || batch > 65535 || (dtype != PFFT_C64 && dtype != PFFT_C128) ||
      (flags & ~unsigned(PFFT_FLAG_TC_SPLIT | PFFT_FLAG_LAYOUT_SNF | PFFT_FLAG_AUTOTUNE | PFFT_FLAG_TRANSPOSED)) ||
      d < 1 || d > 4)
    return PFFT_ERR_ARG;
  if ((flags & PFFT_FLAG_TC_SPLIT) && dtype != PFFT_C64) return PFFT_ERR_UNSUPPORTED;
  *out = nullptr;
  pfft_plan_s* P = new (std::nothrow) pfft_plan_s;
  if (!P) return PFFT_ERR_OOM;
  P->batch = batch;
  P->dtype = dtype;
  if (flags & PFFT_FLAG_TC_SPLIT) {
    P->tc = true;
    P->generic_only = true;
  }
  pfft_status st;
  try {
    if (flags & PFFT_FLAG_LAYOUT_SNF) {
      // Smith-coordinate layout: by Theorem 1 the transform of M in Smith
      // coordinates is the plain d-dimensional DFT of sizes eps_1 .. eps_d,
      // i.e. the transform of diag(eps) in the box layout, whose box order is
      // the row-major order of lambda (input) and mu (output).
      IMat A(d), Q, R, U, V;
      std::vector<i64> eps;
      for (int i = 0; i < d * d; ++i) {
        if (M[i] >= (int64_t(1) << 24) || M[i] <= -(int64_t(1) << 24)) throw LatticeError{PFFT_ERR_OVERFLOW, "entry"};
        A.a[i] = M[i];
      }
      if (determinant(A) == 0) throw LatticeError{PFFT_ERR_SINGULAR, "singular"};
      smith_normal_form(A, Q, eps, R, U, V);
      std::vector<int64_t> D(size_t(d) * d, 0);
      for (int i = 0; i < d; ++i) D[size_t(i) * d + i] = eps[i];
      st = plan_host(*P, d, D.data());
    } else {
      st = plan_host(*P, d, M);
    }
    if (st == PFFT_OK && P->m * batch >= (int64_t(1) << 40)) st = PFFT_ERR_OVERFLOW;
    if (st == PFFT_OK) st = plan_device(*P);
  } catch (const LatticeError& e) {
    st = pfft_status(e.code);
  }
  if (st == PFFT_OK && (flags & (PFFT_FLAG_AUTOTUNE | PFFT_FLAG_TRANSPOSED))) st = plan_route(*P, d, M, flags);
  if (st != PFFT_OK) {
    release(P);
    return st;
  }
  *out = P;
  return PFFT_OK;
}

extern "C" pfft_status pfft_plan_destroy(pfft_plan p) {
  if (!p) return PFFT_ERR_ARG;
  release(p);
  return PFFT_OK;
}

extern "C" pfft_status pfft_plan_route(pfft_plan p, int* fwd, int* inv) {
  if (!p) return PFFT_ERR_ARG;
  if (fwd) *fwd = p->tr && p->tr_fwd ? 1 : 0;
  if (inv) *inv = p->tr && p->tr_inv ? 1 : 0;
  return PFFT_OK;
}

extern "C" pfft_status pfft_plan_info(pfft_plan p, int64_t* m, int* dM, int64_t* eps, int64_t* in_box,
                                      int64_t* out_box) {
  if (!p) return PFFT_ERR_ARG;
  if (m) *m = p->m;
  if (dM) *dM = p->D;
  for (int i = 0; i < p->d; ++i) {
    if (eps) eps[i] = p->eps[i];
    if (in_box) in_box[i] = p->H(i, i);
    if (out_box) out_box[i] = p->G(i, i);
  }
  return PFFT_OK;
}

extern "C" pfft_status pfft_index_map(pfft_plan p, int which, int64_t* coords) {
  if (!p || !coords) return PFFT_ERR_ARG;
  const int d = p->d;
  std::vector<i64> v(d);
  for (i64 s = 0; s < p->m; ++s) {
    switch (which) {
      case PFFT_MAP_INPUT_BOX:
        box_point(p->H, s, coords + s * d);
        break;
      case PFFT_MAP_OUTPUT_BOX:
        box_point(p->G, s, coords + s * d);
        break;
      case PFFT_MAP_INPUT_SNF:
      case PFFT_MAP_OUTPUT_SNF: {
        const bool in = which == PFFT_MAP_INPUT_SNF;
        box_point(in ? p->H : p->G, s, v.data());
        for (int j = 0; j < p->D; ++j) {
          i128 acc = 0;
          for (int c = 0; c < d; ++c) acc += (i128)(in ? p->LAM[j][c] : p->MU[j][c]) * v[c];
          coords[s * p->D + j] = posmod(i64(acc % p->n[j]), p->n[j]);
        }
        break;
      }
      default:
        return PFFT_ERR_ARG;
    }
  }
  return PFFT_OK;
}

extern "C" pfft_status pfft_device_index_map(pfft_plan p, int which, int64_t* slots, void* stream) {
  if (!p || !slots || (which != PFFT_MAP_INPUT_BOX && which != PFFT_MAP_OUTPUT_BOX)) return PFFT_ERR_ARG;
  if (p->D == 0) {
    int64_t zero = 0;
    return cudaMemcpyAsync(slots, &zero, sizeof(zero), cudaMemcpyHostToDevice, (cudaStream_t)stream) ==
                   cudaSuccess
               ? PFFT_OK
               : PFFT_ERR_CUDA;
  }
  PassArgs a = p->rowp;
  return launch_index_probe(a, a, which == PFFT_MAP_INPUT_BOX ? 0 : 1, slots, (cudaStream_t)stream) == 0
             ? PFFT_OK
             : PFFT_ERR_CUDA;
}

static pfft_status run_pass(pfft_plan_s* P, PassArgs a, int load, int store, int cin, int cout,
                            double scale, const void* in, void* out, cudaStream_t s, int which) {
  a.load_mode = load;
  a.store_mode = store;
  a.conj_in = cin;
  a.conj_out = cout;
  a.scale = scale;
  a.in = in;
  a.out = out;
  P->prof.begin(which, s);
  if (launch_pass(a, P->dtype, s) != 0) return PFFT_ERR_CUDA;
  P->prof.end(which, s);
  return PFFT_OK;
}

// The transform of p through the plan t = p->tr of M^T (see pfft_plan_s::tr):
// forward = t's adjoint passes without conjugations, inverse = t's forward
// passes with conjugated input and output.  Kernel time is recorded under p.
static pfft_status transform_transposed(pfft_plan p, const void* in, void* out, cudaStream_t s, bool inverse) {
  pfft_plan_s* t = p->tr;
  const double scale = 1.0 / std::sqrt(double(p->m));
  const int c = inverse ? 1 : 0;
  if (t->pen.empty()) {
    return run_pass(p, t->rowp, inverse ? MAP_BOX_H : MAP_BOX_G, inverse ? MAP_BOX_G : MAP_BOX_H, c, c, scale, in,
                    out, s, 0);
  }
  if (inverse) {
    pfft_status st = run_pass(p, t->rowp, MAP_BOX_H, MAP_WS, 1, 0, 1.0, in, t->ws, s, 0);
    if (st != PFFT_OK) return st;
    return run_pass(p, t->colp, MAP_WS, MAP_BOX_G, 0, 1, scale, t->ws, out, s, 1);
  }
  pfft_status st = run_pass(p, t->colp, MAP_BOX_G, MAP_WS, 0, 0, 1.0, in, t->ws, s, 1);
  if (st != PFFT_OK) return st;
  return run_pass(p, t->rowp, MAP_WS, MAP_BOX_H, 0, 0, scale, t->ws, out, s, 0);
}

static pfft_status transform_route(pfft_plan p, const void* in, void* out, cudaStream_t s, bool inverse,
                                   bool via_tr) {
  const double scale = 1.0 / std::sqrt(double(p->m));
  if (p->D == 0) {
    const size_t bytes = size_t(p->batch) * elem_bytes(p->dtype);
    return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? PFFT_OK
                                                                                       : PFFT_ERR_CUDA;
  }
  if (via_tr) return transform_transposed(p, in, out, s, inverse);
  const int ci = inverse ? 1 : 0;
  if (p->pen.empty()) {
    return run_pass(p, p->rowp, inverse ? MAP_BOX_G : MAP_BOX_H, inverse ? MAP_BOX_H : MAP_BOX_G, ci, ci,
                    scale, in, out, s, 0);
  }
  if (!inverse) {
    pfft_status st = run_pass(p, p->rowp, MAP_BOX_H, MAP_WS, 0, 0, 1.0, in, p->ws, s, 0);
    if (st != PFFT_OK) return st;
    return run_pass(p, p->colp, MAP_WS, MAP_BOX_G, 0, 0, scale, p->ws, out, s, 1);
  }
  pfft_status st = run_pass(p, p->colp, MAP_BOX_G, MAP_WS, 1, 0, 1.0, in, p->ws, s, 1);
  if (st != PFFT_OK) return st;
  return run_pass(p, p->rowp, MAP_WS, MAP_BOX_H, 0, 1, scale, p->ws, out, s, 0);
}

static pfft_status transform(pfft_plan p, const void* in, void* out, void* stream, bool inverse) {
  if (!p || !in || !out || in == out) return PFFT_ERR_ARG;
  const bool via_tr = p->tr && (inverse ? p->tr_inv : p->tr_fwd);
  return transform_route(p, in, out, (cudaStream_t)stream, inverse, via_tr);
}

// Mean time (ms) of one direction by one route over `reps` calls on stream s;
// negative when a call fails.
static float time_route(pfft_plan_s* p, bool inverse, bool via_tr, const void* in, void* out, cudaStream_t s,
                        int reps) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return -1.0f;
  }
  float ms = -1.0f;
  bool ok = transform_route(p, in, out, s, inverse, via_tr) == PFFT_OK;  // warm-up
  ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
  for (int r = 0; ok && r < reps; ++r) ok = transform_route(p, in, out, s, inverse, via_tr) == PFFT_OK;
  ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
       cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return -1.0f;
  }
  return ms / float(reps);
}

// PFFT_FLAG_TRANSPOSED / PFFT_FLAG_AUTOTUNE: plan M^T beside M (same batch and
// precision, this plan's workspace and status word) and route the directions
// through it, always (TRANSPOSED) or where it measures faster (AUTOTUNE: each
// direction timed both ways on zeroed scratch buffers; the transposed route
// must win by 3%).  Plans of the Smith layout or the split-precision form,
// and transposed plans whose row pass is the pipelined kernel (which runs
// only with the conjugations of its own directions), keep the direct route:
// PFFT_ERR_UNSUPPORTED under TRANSPOSED, silently under AUTOTUNE.
static pfft_status plan_route(pfft_plan_s& P, int d, const int64_t* M, unsigned flags) {
  const bool force = (flags & PFFT_FLAG_TRANSPOSED) != 0;
  const pfft_status no = force ? PFFT_ERR_UNSUPPORTED : PFFT_OK;
  if (P.tc || (flags & PFFT_FLAG_LAYOUT_SNF) || P.D == 0) return no;
  std::vector<int64_t> Mt(size_t(d) * d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Mt[size_t(i) * d + j] = M[size_t(j) * d + i];
  pfft_plan_s* T = new (std::nothrow) pfft_plan_s;
  if (!T) return PFFT_ERR_OOM;
  T->batch = P.batch;
  T->dtype = P.dtype;
  T->own_workspace = false;
  pfft_status st;
  try {
    st = plan_host(*T, d, Mt.data());
    if (st == PFFT_OK) st = plan_device(*T);
  } catch (const LatticeError& e) {
    st = pfft_status(e.code);
  }
  if (st == PFFT_OK && (T->rowp.pipe || T->pen.size() != P.pen.size())) st = PFFT_ERR_UNSUPPORTED;
  if (st != PFFT_OK) {
    plan_release(T);
    return force ? st : PFFT_OK;
  }
  T->ws = P.ws;
  T->rowp.status = T->colp.status = P.status;
  P.tr = T;
  if (force) {
    P.tr_fwd = P.tr_inv = true;
    return PFFT_OK;
  }
  // AUTOTUNE: time both routes of each direction
  const size_t bytes = size_t(P.m) * size_t(P.batch) * elem_bytes(P.dtype);
  void *a = nullptr, *b = nullptr;
  cudaStream_t s = nullptr;
  bool ok = cudaMalloc(&a, bytes) == cudaSuccess && cudaMalloc(&b, bytes) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMemsetAsync(a, 0, bytes, s) == cudaSuccess;
  if (ok) {
    const int reps = 3;
    for (int inv = 0; inv < 2; ++inv) {
      const float direct = time_route(&P, inv != 0, false, a, b, s, reps);
      const float via = time_route(&P, inv != 0, true, a, b, s, reps);
      const bool use = direct > 0.0f && via > 0.0f && via < 0.97f * direct;
      (inv ? P.tr_inv : P.tr_fwd) = use;
    }
    cudaStreamSynchronize(s);
  }
  cudaGetLastError();
  if (s) cudaStreamDestroy(s);
  if (a) cudaFree(a);
  if (b) cudaFree(b);
  if (!P.tr_fwd && !P.tr_inv) {
    T->ws = nullptr;
    plan_release(T);
    P.tr = nullptr;
  }
  return PFFT_OK;
}

extern "C" pfft_status pfft_forward(pfft_plan p, const void* in, void* out, void* stream) {
  return transform(p, in, out, stream, false);
}

extern "C" pfft_status pfft_inverse(pfft_plan p, const void* in, void* out, void* stream) {
  return transform(p, in, out, stream, true);
}

static const char* kPassNames[] = {"row_pass", "col_pass"};

extern "C" pfft_status pfft_profile_enable(pfft_plan p, int enable) {
  if (!p) return PFFT_ERR_ARG;
  return p->prof.enable(enable != 0, 2, kPassNames) ? PFFT_OK : PFFT_ERR_CUDA;
}

extern "C" pfft_status pfft_profile_read(pfft_plan p, const char** names, int64_t* launches, double* ms,
                                         int cap, int* n) {
  if (!p) return PFFT_ERR_ARG;
  return p->prof.read(names, launches, ms, cap, n) ? PFFT_OK : PFFT_ERR_CUDA;
}

extern "C" pfft_status pfft_set_wait_limit(pfft_plan p, int64_t spins) {
  if (!p) return PFFT_ERR_ARG;
  if (!p->rowp.tma) return PFFT_ERR_UNSUPPORTED;
  const uint32_t lim = spins < 0 ? kSpinLimit : uint32_t(std::min<int64_t>(spins, int64_t(UINT32_MAX)));
  p->rowp.spin_limit = lim;
  if (p->tr) p->tr->rowp.spin_limit = lim;
  return PFFT_OK;
}

extern "C" pfft_status pfft_last_device_status(pfft_plan p, void* stream) {
  if (!p) return PFFT_ERR_ARG;
  if (!p->status) return PFFT_OK;
  int v = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&v, p->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PFFT_ERR_CUDA;
  if (v != 0) cudaMemsetAsync(p->status, 0, sizeof(int), s);
  return pfft_status(v);
}
