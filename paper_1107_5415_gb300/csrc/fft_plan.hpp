// Plan structures shared by the host planner and the transform kernels.
//
// The transform runs in Smith coordinates (Theorem 1): with the non-trivial
// elementary divisors n_1 | ... | n_D (D = d_M <= 3), the data is viewed as a
// logical LB x nD array, nD = n_D the longest cycle and LB = n_1 ... n_{D-1}
// the product of the others (eq. (KroneckerFFT): "blockwise" transforms of
// length n_D, then the transforms over the remaining cycles on interleaved
// data).  Two kernels implement the two halves:
//
//   row pass    one CTA holds T full rows (length nD) in shared memory and
//               runs the length-nD DFT; the gather from the input box (or the
//               scatter to it, inverse direction) is fused into its load
//               (store).
//   column pass one CTA holds all LB rows of T columns and runs the
//               (D-1)-dimensional DFT over the other cycles; the scatter to
//               the output box (gather from it, inverse) is fused into its
//               store (load).
//
// Between them the data sits in a workspace laid out [LB][nD] whose columns
// are permuted (PI) so that the columns one column-pass CTA needs are
// adjacent, and the same CTA's output-box writes come in contiguous runs.
#pragma once
#include <stdint.h>

#include "device_common.cuh"

namespace pfft {

enum MapMode { MAP_WS = 0, MAP_BOX_H = 1, MAP_BOX_G = 2 };

constexpr int kMaxStages = 16;
// Default iteration limit of the bounded mbarrier waits of the bulk-copy
// row passes (far above the time a row's copies take to land).
constexpr uint32_t kSpinLimit = 1u << 22;
// Persistent pipelined row pass (fft_row_pipe.cuh): row length 2^kPipeLogL,
// exchanged and stored in two rounds of kPipeHalf elements through a buffer
// of kPipeX elements (one padding element per 16).
constexpr int kPipeLogL = 14;
constexpr int kPipeHalf = 1 << (kPipeLogL - 1);
constexpr int kPipeX = kPipeHalf + (kPipeHalf >> 4);
// Persistent pipelined column pass (fft_col_pipe.cuh): pencils of
// 2^kCPipeLogL complex64 points, 8 columns per tile; shared memory holds the
// tile (kCPipeS elements: room for one padding row per 32 rows) and the
// two-round exchange and output buffer (kCPipeX: half a padded tile).
constexpr int kCPipeLogL = 10;
constexpr int kCPipeS = ((1 << kCPipeLogL) + (1 << (kCPipeLogL - 5))) * 8;  // padded tile
constexpr int kCPipeX = ((1 << (kCPipeLogL - 1)) + (1 << (kCPipeLogL - 6))) * 8;
constexpr int kMaxSub = 3;
constexpr int kMaxThreads = 512;
constexpr int kRadixOrder[7] = {16, 8, 4, 2, 3, 5, 7};
// Stages of a prime radix from 11 up are evaluated directly from shared
// memory (run_direct_stage; a register butterfly of that size spills); they
// run before all others, so the first one of each axis needs no twiddles.
constexpr int kDirectRegion = 7;
// Radix-32 stages exist only in split-precision tensor-core passes (fft_tc.cuh);
// there the radix-16 stages run on the tensor cores too.
constexpr int kTC32Region = 8;
constexpr int kMinDirectRadix = 11;
constexpr int kMaxDirectRadix = 1021;
// Work items a thread holds in the phases of a direct stage (run_direct_stage),
// for tiles of at most EPT points per thread: pre-pass pairs (h R' per
// butterfly, h = (R - 1) / 2: at most EPT / 2), output items of 4 outputs
// (R >= kDirectQ4MinRadix) or 2 outputs, and butterflies for y_0 (at most
// EPT / 11 + 1).  The planner's thread count guarantees them.
constexpr int kDirectQ4MinRadix = 37;
constexpr int kDirectZero = 3;
template <int EPT>
constexpr int kDirectPre = EPT / 2;
template <int EPT>
constexpr int kDirectQ4Items = EPT / 8 + 1;
template <int EPT>
constexpr int kDirectQ2Items = EPT / 8 + 2;

// One radix stage of a Stockham autosort DFT along one axis of a pencil.
struct StageDesc {
  int R;       // radix
  int a;       // length of the axis
  int aR;      // a / R
  int sigma;   // stride of the axis inside the pencil (elements)
  int Ns;      // product of the radices of the earlier stages on this axis
  int twstep;  // tw_n / (Ns * R): index step into the pass's omega_{tw_n} table
  int gen;     // direct stages: a primitive root of the prime R
  FastDiv div_aR, div_sigma, div_Ns;
};

struct alignas(16) PassArgs {
  // geometry
  int L;        // pencil length (row pass: nD; column pass: LB)
  int T;        // pencils per CTA
  int nD, LB, m, d;
  int ts;       // int32 per table entry: 2 (d <= 2) or 4 (d = 3, 4)
  int cols;     // 1: column pass, 0: row pass
  int nstages;
  int cnt[9];  // stages per radix, in the order of kRadixOrder; [7]: direct prime stages; [8]: radix 32
  int tc;       // 1: radix-16 / 32 stages on the tensor cores in split fp16 (complex64)
  int tc_off;   // byte offset of the tensor-core fragment tables in shared memory
  int dir_off;  // shared-memory element offset of the omega_R table of a direct stage
  int pad;      // 1: padded shared-memory tile (x + x / 16); 0 when the pass has direct stages
  int ept;      // points per thread of the generic kernels (16 or 32 for complex64, 16 for complex128)
  int pow2;     // all radices are powers of two
  int fast;       // 1: use the register-resident power-of-two kernels (fft_fast.cuh)
  int fast_tail;  // radix of the first stage (1 = none)
  int fast_nmain; // number of main-radix stages
  int logT;
  // arithmetic column permutation (power-of-two nD):
  // PI[mu] = ((mu & (g - 1)) << pi_lspan) | (((mu >> pi_lg) * pi_inv) & (span - 1))
  int pi_arith, pi_lg, pi_lspan, pi_inv;
  // arithmetic gather table: Btab[e] = (bz[e >> bz_lh][0..d-2], e & (2^bz_lh - 1))
  int bz_arith, bz_lh;
  int bz[64][3];
  // four-step split of a long last cycle (n = fs_na * nD): the row pass
  // multiplies (row, element) by exp(-2 pi i lambda_a mu_b / n), lambda_a =
  // row mod fs_na, after its DFT (forward) or before it (inverse)
  int fs_na;
  FastDiv fs_div;
  const void* fs_lo;  // exp(-2 pi i t / n), t < 2048
  const void* fs_hi;  // exp(-2 pi i (t << 11) / n)
  int stw_off[4];  // offset of each main stage's twiddles in the stage table
  int stw_n;       // stage table length (complex, even)
  int stw_smem_off;  // its place in shared memory (elements)
  const void* stw_g;  // stage table in global memory
  // bulk-copy staging of the row pass (fft_tma.cuh)
  int tma;            // 1: use row_tma_kernel
  const int* runs;    // [LB][nruns] int4 (element offset, box slot, length, 0)
  int nruns;
  int bar_smem_off;   // byte offset of the mbarrier in shared memory
  int* status;        // device status word (PFFT_ERR_TIMEOUT on a timed-out wait)
  uint32_t spin_limit;  // iterations of the first mbarrier wait before it gives up
  // persistent pipelined row pass (fft_row_pipe.cuh): rows of 2^14 complex64
  int pipe;            // 1: use row_pipe_kernel
  int pipe_x_off;      // element offset of its exchange buffer in shared memory
  int pipe_grid;       // CTAs of its launch (one per SM)
  int pipe_direct;     // 1: output stored from registers (see fft_row_pipe.cuh)
  int pipe_lrun;       // log2 of the uniform run length of the box rows (0: runs not uniform)
  int cpipe;           // 1: use col_pipe_kernel (fft_col_pipe.cuh)
  int cpipe_x_off;     // element offset of its exchange / output buffer in shared memory
  int cpipe_e_off;     // element offset of its column-point buffer (2 x 8 x 4 int32)
  int cpipe_grid;      // CTAs of its launch (two per SM)
  // workspace-order staging of the TMA row pass in 2^pi_lg blocks of 2^pi_lspan
  // positions, each followed by stg_pad elements (0: one dense block), so that
  // the permuted accesses of lanes with equal mu >> pi_lg hit different banks
  int stg_pad;
  StageDesc st[kMaxStages];
  FastDiv divT, divnD;
  int nthreads;
  int smem_bytes;
  int groups;   // CTAs per signal
  int batch;
  // data
  int load_mode, store_mode;
  int conj_in, conj_out;
  double scale;
  const void* in;
  void* out;
  // grouped launches: in / out hold byte offsets into the launch's base
  // pointer number in_sel / out_sel (see batch_kernels.cu)
  int in_sel, out_sel;
  // tables (device, d int32 per entry)
  const int* Atab;   // [LB]  box(H) point of sum_{j<D} lambda_j g_j
  const int* Btab;   // [nD]  box(H) point of lambda_D g_D
  const int* Ctab;   // [LB]  box(G) point of sum_{j<D} mu_j h_j
  const int* Etab;   // [nD]  box(G) point of PIinv[pos] h_D   (indexed by position)
  const int* PIinv;  // [nD]  column position -> mu_D (or lambda_D)
  const int* PI;     // [nD]  mu_D -> column position
  const void* tw;    // [tw_n] omega_{tw_n}^t = exp(-2 pi i t / tw_n)
  int tw_n;          // order of tw: nD (row pass); a common multiple of the pencil axes (column pass)
  BoxDesc boxH, boxG;
  // shear of the column pass: a run of consecutive output slots along the
  // fastest output coordinate visits (mu_<D + t alpha, position + t).
  int nsub;
  int sub_n[kMaxSub];
  FastDiv sub_div[kMaxSub];
  int alpha[kMaxSub];
};

// Four-step twiddle exp(-2 pi i lambda_a mu_b / n) of a split last cycle:
// lambda_a = row mod n_a (the fastest pencil axis), mu_b = element.
template <typename C>
__device__ __forceinline__ C fs_twiddle(const PassArgs& a, int row, int e) {
  const int la = row - a.fs_div.div(row) * a.fs_na;
  const int t = la * e;  // < n_a n_b = n < 2^31
  const C* lo = static_cast<const C*>(a.fs_lo);
  const C* hi = static_cast<const C*>(a.fs_hi);
  return cmul(__ldg(hi + (t >> 11)), __ldg(lo + (t & 2047)));
}

template <typename C>
__device__ __forceinline__ C maybe_conj(C v, int c) {
  return c ? cconj(v) : v;
}

// Host-side launcher (fft_kernels.cu).
int launch_pass(const PassArgs& a, int dtype, cudaStream_t s);
int launch_twiddles(void* tw, int nD, int dtype, cudaStream_t s);
int launch_twiddle_gather(void* dst, const void* tw, const int* idx, int n, int dtype, cudaStream_t s);
int launch_phase_tables(void* tab, int64_t q, int nhi, int dtype, cudaStream_t s);
int launch_index_probe(const PassArgs& rowp, const PassArgs& colp, int which, int64_t* out,
                       cudaStream_t s);

}  // namespace pfft
