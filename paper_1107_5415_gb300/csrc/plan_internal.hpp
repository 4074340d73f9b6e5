// The transform plan (host planner state and device tables), shared by the
// single-pattern entry points (fft_plan.cu) and the many-pattern batch
// (batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/pfft.h"
#include "fft_plan.hpp"
#include "lattice.hpp"
#include "plan_common.hpp"

struct pfft_plan_s {
  int d = 0;
  int64_t batch = 0;
  int dtype = 0;
  pfft::IMat M, H, G;
  pfft::i64 m = 0;
  std::vector<pfft::i64> eps;                 // all d elementary divisors
  int D = 0;                                  // non-trivial cycles
  std::vector<int> n;                         // their lengths, ascending
  std::vector<std::vector<pfft::i64>> LAM;    // D rows: lambda_j(y) = LAM_j . y mod n_j
  std::vector<std::vector<pfft::i64>> MU;     // D rows: mu_j(k) = MU_j . k mod n_j
  int nD = 1, LB = 1;       // row length and number of rows of the logical LB x nD array
  std::vector<int> pen;     // column-pass pencil axes (row-major), product LB
  int fs_na = 1;            // four-step split of a long last cycle: n = fs_na * nD
  pfft::i64 fs_N = 1;       // the full length of the last cycle
  void* fs_tab = nullptr;   // exp(-2 pi i t / fs_N), two-level table
  // options (set before plan_device)
  pfft::Arena* arena = nullptr;  // sub-allocate device tables here (batch plans)
  bool generic_only = false;     // shared-memory Stockham kernels only (grouped launches)
  bool own_workspace = true;     // allocate the LB x nD workspace
  bool tc = false;               // split-precision tensor-core radix-16 / 32 stages
  int ept_c64 = 32;              // complex64 points per thread of the generic kernels
  int max2 = 16;                 // largest power-of-two radix of the generic kernels (16 or 8)
  // device state
  int device = 0;
  int* dtab = nullptr;
  void* tw = nullptr;
  void* tw_col = nullptr;  // column-pass table when its axes do not divide nD (split last cycle)
  void* ws = nullptr;
  void* stw = nullptr;  // stage twiddle tables of the register-resident passes
  int* runs = nullptr;  // bulk-copy runs of the row pass
  int* status = nullptr;  // device status word
  pfft::PassArgs rowp{}, colp{};
  pfft::Profiler prof;
  // Transposed route.  Entry (k, y) of F(M) is entry (y, k) of F(M^T) in box
  // order (eq. (Fouriermatrix) read for M^T), so the forward transform of M
  // is the adjoint passes of M^T without their conjugations and the inverse
  // of M is the forward passes of M^T with conjugated input and output.  tr
  // is the plan of M^T (sharing this plan's workspace and status word);
  // tr_fwd / tr_inv: the direction runs through it.
  pfft_plan_s* tr = nullptr;
  bool tr_fwd = false, tr_inv = false;

  int alloc(void** p, size_t bytes) { return arena ? arena->alloc(p, bytes) : pfft::device_alloc(p, bytes); }
};

namespace pfft {
// Exact integer planning (HNF, SNF, cycle split); no device work.
pfft_status plan_host(pfft_plan_s& P, int d, const int64_t* M);
// Device tables and pass descriptors.
pfft_status plan_device(pfft_plan_s& P);
// Re-choose the tiles of both passes (pencils per CTA) under the given
// element budgets and the largest power-of-two radix (16 or 8); generic
// kernels only.  Tables are unchanged.
pfft_status plan_retile(pfft_plan_s& P, int row_budget, int col_budget, int max2);
void plan_release(pfft_plan_s* P);
}  // namespace pfft
