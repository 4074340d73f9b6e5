// Descriptors of the grouped launches of a pattern batch (batch.cu host side,
// batch_kernels.cu device side).
#pragma once
#include <cuda_runtime.h>

#include "fft_plan.hpp"
#include "split_prime.cuh"
#include "wavelet_kernels.cuh"

namespace pfft {

constexpr int kSplitThreads = 256;
constexpr int kGroupedEptC64 = 16;  // complex64 points per thread of the grouped pass kernels
constexpr int kSplitPerThread = 4;  // fibres per thread of a grouped split CTA
// Dynamic shared memory of a grouped pass CTA: the 227 KB per CTA less room
// for the static copy of its pass descriptor.
constexpr int kGroupedMaxDynSmem = 227 * 1024 - 4096;

// One grouped pass launch: items[k] is the descriptor of the k-th pattern of
// the launch, whose tiles are CTAs cta0[k] .. cta0[k+1]-1; after the n + 1
// entries of cta0 (padded to an even count) the (item, tile) pair of every
// CTA.  The in / out fields of an item hold byte offsets into base[in_sel] /
// base[out_sel].
struct GroupArgs {
  const PassArgs* items;
  const int* cta0;
  int n;
  const void* base[3];  // 0: the caller's input, 1: the batch workspace, 2: the caller's output
};

// One split level of one pattern with |det J| = 2; offsets in elements into
// the concatenated c_hat (in_off), scaling parts (sc_off) and wavelet parts
// (wv_off).
struct alignas(16) SplitItem {
  LevelDesc L;
  long long in_off, sc_off, wv_off;
};

// One split level of one pattern with |det J| = p > 2 (built-in band
// system, split_prime.cuh): band 0 at scaling + sc_off, band j >= 1 at
// wavelet + wv_off + (j - 1) |det N|.
struct alignas(16) PrimeItem {
  PrimeDesc P;
  long long in_off, sc_off, wv_off;
};

// The whole batch in one launch (batch_queue_kernel): one queue of work
// units in dependency order -- every row-pass tile, then every column-pass
// tile, then the split units -- handed to the CTAs by a counter in the order
// they start.  A column tile of pattern i starts once all row tiles of
// pattern i are done, a split unit once the pattern's coefficients are
// complete; the waits are bounded (spin_limit tries and about one second),
// after which the kernel records PFFT_ERR_TIMEOUT, raises the abort flag and
// the CTAs still to run return at once.  Units of the split phases take
// kQueueSplitFibres fibres (|det J| = 2) or kMaxThreads work items
// (|det J| > 2).
constexpr int kQueueSplitFibres = kMaxThreads * kSplitPerThread;
struct QueueArgs {
  const PassArgs* rows;          // row-pass items, costliest first
  const int* row_u0;             // first unit of each row item (prefix, n + 1 entries)
  const int* row_pat;            // pattern of each row item
  int nrow;
  const PassArgs* cols;
  const int* col_u0;
  const int* col_pat;
  int ncol;
  const SplitItem* splits;
  const int* split_u0;
  const int* split_pat;
  int nsplit;
  const PrimeItem* primes;
  const int* prime_u0;
  const int* prime_pat;
  int nprime;
  int u_rows, u_cols, u_splits, u_primes;  // units per phase (split phases 0 without a split)
  const int* need_rows;  // per pattern: row tiles
  const int* need_cols;  // per pattern: column tiles (0: the row pass writes the coefficients)
  int* counters;         // [0] next unit, [1] abort, then rows done [npat], columns done [npat]
  int npat;
  int* status;           // device status word (PFFT_ERR_TIMEOUT)
  unsigned spin_limit;
  const void* base[3];   // the caller's input, the batch workspace, the caller's output (c_hat)
  void* sc;
  void* wv;
};
// Raise the shared-memory limit of the queue kernel (once per process; call
// before any stream capture).
int prepare_queue(int dtype);
int launch_batch_queue(const QueueArgs& g, int dtype, int nunits, int smem, cudaStream_t s);

// Raise the dynamic shared-memory limit of the grouped kernels (once per
// process; call before any stream capture).
int prepare_grouped(int dtype);
int launch_grouped_pass(const GroupArgs& g, int cols, int dtype, int nctas, int threads, int smem,
                        cudaStream_t s);
// The split levels of the patterns with |det J| = 2 (cta0 and the CTA map as
// in GroupArgs).
int launch_grouped_split(const SplitItem* items, const int* cta0, int n, int nctas, const void* chat, void* sc,
                         void* wv, int dtype, cudaStream_t s);
// The split levels of the patterns with |det J| > 2: items[k]'s work items
// (fibre, chunk of kPrimeChunk bands) start at CTA cta0[k], kSplitThreads
// items per CTA (cta0 and the CTA map as in GroupArgs).
int launch_grouped_prime_split(const PrimeItem* items, const int* cta0, int n, int nctas, const void* chat,
                               void* sc, void* wv, int dtype, cudaStream_t s);

}  // namespace pfft
