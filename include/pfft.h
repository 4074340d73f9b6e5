/*
 * pfft.h -- C ABI of the GB300 pattern FFT / fast wavelet split library.
 *
 * The library computes the Fourier transform on the pattern P(M) of a regular
 * integer matrix M (eq. (Fouriermatrix), Section 2.2),
 *
 *     c_hat[k] = m^{-1/2} sum_{y in G(M)} c[y] exp(-2 pi i k^T M^{-1} y),  k in G(M^T),
 *
 * m = |det M|, through the Kronecker factorisation in Smith coordinates
 * (Theorem 1, Section 4.1; eq. (KroneckerFFT), Section 4.2), and the fast
 * wavelet decomposition step built on it (Section 5.3, step 4): the split of
 * Fourier coefficients on G(M^T) into scaling and wavelet parts on G(N^T),
 * M = J N, |det J| = 2, with the Dirichlet symbols of Section 6.2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Layout ("box layout").  For an integer matrix A let H(A) be its column-style
 *  Hermite normal form (H = A U, U unimodular, H upper triangular, H_rr > 0,
 *  0 <= H_rc < H_rr for c > r; the pattern normal form of Section 6.1).  The
 *  integer box  x_r [0, H_rr)  is a complete residue system of Z^d / A Z^d.
 *  A signal on G(M) (equivalently on the pattern points M^{-1} y of P(M)) is
 *  stored with y in the box of H(M); Fourier coefficients on G(M^T) are
 *  stored with k in the box of H(M^T).  Slots are numbered row-major over the
 *  box (last coordinate fastest).  pfft_index_map returns the coordinates.
 *
 *  Data.  Complex interleaved (re, im): PFFT_C64 = 2 x float, PFFT_C128 =
 *  2 x double.  Buffers are DEVICE pointers owned by the caller, contiguous,
 *  batch outermost ([batch][m]).  All transform calls are asynchronous and
 *  stream-ordered on the given cudaStream_t (passed as void*, NULL = legacy
 *  default stream); nothing on the hot path synchronises with the host.
 *  Input and output must not overlap.
 *
 *  Ownership.  Plans own their device tables and workspace, released by the
 *  matching *_destroy.  A plan may be used from one stream at a time (the
 *  workspace is shared by all calls on the plan).
 *
 *  Errors.  Every entry point returns a pfft_status.  Argument, planning and
 *  capacity errors are detected on the host and returned synchronously before
 *  any work is queued.  Errors raised by the CUDA runtime while queueing are
 *  returned as PFFT_ERR_CUDA.  There is no CPU fallback: without a usable GPU
 *  the plan constructors return PFFT_ERR_CUDA.
 *
 *  Limits.  1 <= d <= 4, |M_ij| < 2^24, 1 <= |det M| < 2^31.  The transform
 *  kernels handle at most three non-trivial Smith cycles.  With the tile
 *  size S = 16384 (PFFT_C64) or 8192 (PFFT_C128): the product P of all
 *  cycles but the last must be <= S; the last cycle n either fits (n <= S)
 *  or splits as n = n_a n_b with n_b <= S and P n_a <= S (four-step split
 *  inside the two passes).  Cycle lengths may contain any prime factor up to
 *  1021 (primes from 11 up are evaluated as direct sums: O(p) work per point
 *  for a factor p).  Anything else is rejected with PFFT_ERR_UNSUPPORTED at
 *  plan time.
 */
#ifndef PFFT_H
#define PFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfft_plan_s* pfft_plan;
typedef struct pwt_plan_s* pwt_plan;
typedef struct pfft_batch_s* pfft_batch;

typedef enum {
  PFFT_OK = 0,
  PFFT_ERR_ARG = 1,          /* NULL pointer, bad d / batch / dtype / flag / level */
  PFFT_ERR_SINGULAR = 2,     /* det M == 0 (or det J == 0) */
  PFFT_ERR_OVERFLOW = 3,     /* entries or determinant beyond the stated limits */
  PFFT_ERR_NOT_INTEGRAL = 4, /* J^{-1} M is not an integer matrix */
  PFFT_ERR_UNSUPPORTED = 5,  /* valid input outside what the kernels handle */
  PFFT_ERR_OOM = 6,          /* device allocation failed */
  PFFT_ERR_CUDA = 7,         /* CUDA runtime error (incl. no device) */
  PFFT_ERR_TIMEOUT = 8,      /* reserved: a bounded device wait gave up */
  PFFT_ERR_DEVICE_CHECK = 9  /* reserved: a device-side check failed */
} pfft_status;

enum { PFFT_C64 = 0, PFFT_C128 = 1 };

/* Flags of pfft_plan_create. */
enum {
  /* Split-precision tensor-core form (PFFT_C64 only): the radix-32 stages
   * (and, in passes that do not fit the register-resident kernels, the
   * radix-16 stages) run as dense DFT-matrix products on the tensor cores
   * (tcgen05, fp16 operands, fp32 accumulation in tensor memory), each
   * operand split into hi + lo fp16 halves (three products per K step),
   * which recovers fp32-level accuracy.  The form uses neither the bulk-copy
   * nor the pipelined passes.  Each
   * butterfly is scaled by a power of two before the split and back after
   * the product (exact), so the accuracy holds for data of any magnitude
   * within the fp32 range.  Without the flag every stage runs in plain fp32
   * on the CUDA cores. */
  PFFT_FLAG_TC_SPLIT = 1u,
  /* Smith-coordinate layout (the reordering-free order of Section 4): the
   * input is indexed by lambda = (lambda_1 .. lambda_d), lambda_j in
   * [0, eps_j), row-major, and the output by mu the same way, where
   * lambda(y) and mu(k) are the coordinates that pfft_index_map returns with
   * PFFT_MAP_INPUT_SNF / PFFT_MAP_OUTPUT_SNF for a box-layout plan of the same
   * M (cycles of length 1 contribute no index).  The transform is then the
   * d-dimensional DFT of sizes eps_1 .. eps_d (Theorem 1) without any
   * gather or scatter; the box extents reported by pfft_plan_info are the
   * eps_j.  Requires eps_d < 2^24. */
  PFFT_FLAG_LAYOUT_SNF = 2u,
  /* Route each direction by measurement at plan time.  Read for M^T, eq.
   * (Fouriermatrix) gives F(M^T) = F(M)^T with the two boxes exchanged, so
   * the forward transform of M can run as the adjoint passes of M^T without
   * their conjugations and the inverse of M as the forward passes of M^T
   * with conjugated input and output; the passes of M^T walk other boxes and
   * cycles and can be faster.  pfft_plan_create then also plans M^T, times
   * each direction both ways (a few calls each, on two zeroed scratch
   * buffers of |det M| * batch values allocated for the timing and freed
   * after it, on a private stream) and keeps the plan of M^T, which shares
   * this plan's workspace, only for a direction where it is at least 3%
   * faster.  No effect with PFFT_FLAG_TC_SPLIT or PFFT_FLAG_LAYOUT_SNF, or
   * when the transposed plan's row pass is the pipelined kernel (which runs
   * only with the conjugations of its own directions). */
  PFFT_FLAG_AUTOTUNE = 4u,
  /* Run both directions through the plan of M^T (see PFFT_FLAG_AUTOTUNE)
   * without timing.  PFFT_ERR_UNSUPPORTED in the cases where AUTOTUNE has
   * no effect. */
  PFFT_FLAG_TRANSPOSED = 8u
};

/* Which index map pfft_index_map returns. */
enum {
  PFFT_MAP_INPUT_BOX = 0,   /* per input slot: y (d coordinates) in the box of H(M)     */
  PFFT_MAP_OUTPUT_BOX = 1,  /* per output slot: k (d coordinates) in the box of H(M^T)  */
  PFFT_MAP_INPUT_SNF = 2,   /* per input slot: Smith coordinates lambda (d_M values)    */
  PFFT_MAP_OUTPUT_SNF = 3   /* per output slot: Smith coordinates mu (d_M values)       */
};

/* Human-readable name of a status code (static string). */
const char* pfft_status_string(pfft_status s);

/* ---------------------------------------------------------------------------
 * Host-only planner queries (exact integer arithmetic, no GPU needed).
 * ------------------------------------------------------------------------- */

/* Hermite normal form H of the d x d row-major integer matrix M (Section 6.1,
 * eq. (FFTexampleMatrix): the upper-triangular normal form of a pattern).
 * H (d*d, row-major) is written by the callee; caller-owned host memory. */
pfft_status pfft_hermite_normal_form(int d, const int64_t* M, int64_t* H);

/* Smith normal form M = Q E R (eq. (SNF), Section 2.2): Q, R unimodular,
 * E = diag(eps), eps_j | eps_{j+1}.  Q, R: d*d row-major; eps: d values.
 * Host memory owned by the caller. */
pfft_status pfft_smith_normal_form(int d, const int64_t* M, int64_t* Q, int64_t* eps, int64_t* R);

/* ---------------------------------------------------------------------------
 * Pattern FFT plans.
 * ------------------------------------------------------------------------- */

/* Plan the transform on P(M) for `batch` signals of |det M| points each.
 * M: d*d row-major host array.  dtype: PFFT_C64 or PFFT_C128.  flags: any of
 * PFFT_FLAG_TC_SPLIT (PFFT_C64 only, else PFFT_ERR_UNSUPPORTED),
 * PFFT_FLAG_LAYOUT_SNF, PFFT_FLAG_AUTOTUNE and PFFT_FLAG_TRANSPOSED.
 * Computes H(M), H(M^T), the Smith form and the basis of Theorem 1
 * (Section 3, eqs. (basisPM), (basisGM); Remark 2 allows any biorthogonal
 * pair, and the planner picks the one whose longest cycle runs along the
 * fastest input coordinate), uploads the index tables, builds the twiddle
 * table on the device (exact integer phase, FP64 sincospi, rounded to the
 * working precision) and allocates the workspace (|det M| * batch complex
 * values).  Synchronises the current device once (setup only). */
pfft_status pfft_plan_create(pfft_plan* out, int d, const int64_t* M, int64_t batch, int dtype,
                             unsigned flags);

/* Sizes of a plan.  Any output pointer may be NULL.
 *   m       : |det M|
 *   dM      : number of Smith cycles longer than one (d_M of Section 2.2)
 *   eps     : d elementary divisors, ascending
 *   in_box  : d extents of the input box (diagonal of H(M))
 *   out_box : d extents of the output box (diagonal of H(M^T)) */
pfft_status pfft_plan_info(pfft_plan p, int64_t* m, int* dM, int64_t* eps, int64_t* in_box,
                           int64_t* out_box);

/* Route of each direction (PFFT_FLAG_AUTOTUNE / PFFT_FLAG_TRANSPOSED): *fwd,
 * *inv = 1 when the forward / inverse transform runs through the plan of
 * M^T, else 0.  Either pointer may be NULL.  Host only. */
pfft_status pfft_plan_route(pfft_plan p, int* fwd, int* inv);

/* Host copy of an index map (see PFFT_MAP_*).  coords: caller-owned host
 * array of m*d int64 (box maps) or m*dM int64 (Smith maps), slot-major. */
pfft_status pfft_index_map(pfft_plan p, int which, int64_t* coords);

/* The same maps as the device kernels evaluate them: for every Smith
 * coordinate vector (row-major over the non-trivial cycles) the box slot the
 * kernels read (which = PFFT_MAP_INPUT_BOX) or write (PFFT_MAP_OUTPUT_BOX).
 * slots: caller-owned DEVICE array of m int64.  Asynchronous on `stream`. */
pfft_status pfft_device_index_map(pfft_plan p, int which, int64_t* slots, void* stream);

/* Forward transform (eq. (Fouriermatrix)): in on the box of H(M), out on the
 * box of H(M^T), both [batch][m] complex device arrays; unitary scaling. */
pfft_status pfft_forward(pfft_plan p, const void* in, void* out, void* stream);

/* Inverse transform = adjoint (F(M) is unitary): in on the box of H(M^T),
 * out on the box of H(M). */
pfft_status pfft_inverse(pfft_plan p, const void* in, void* out, void* stream);

pfft_status pfft_plan_destroy(pfft_plan p);

/* Device status of a plan: synchronises `stream`, returns the status word the
 * kernels set (PFFT_ERR_TIMEOUT when a bounded wait on an asynchronous copy
 * gave up; PFFT_OK otherwise) and clears it. */
pfft_status pfft_last_device_status(pfft_plan p, void* stream);

/* Iteration limit of the first bounded wait of the bulk-copy row pass (the
 * wait for a row's asynchronous copies to land in shared memory).
 * spins >= 0 sets it (values above 2^32 - 1 are clamped), spins < 0
 * restores the default of 2^22 iterations.  With 0 the wait gives up at
 * once, which exercises the timeout path: the kernel records
 * PFFT_ERR_TIMEOUT in the plan's status word (pfft_last_device_status),
 * waits with the default limit for its own copies, and returns without
 * transforming, so the output of such a call is undefined.  Host-side
 * setting, applies to later calls.  Returns PFFT_ERR_UNSUPPORTED for a plan
 * whose row pass does not stage through bulk copies (no such wait). */
pfft_status pfft_set_wait_limit(pfft_plan p, int64_t spins);

/* Per-kernel timing of a plan's launches (CUDA events recorded on the
 * launching stream around each kernel).  enable != 0 starts recording and
 * clears the totals.  pfft_profile_read writes up to `cap` entries: kernel
 * name (static string), launch count and summed milliseconds; it
 * synchronises with the recorded events.  Returns the entry count in *n. */
pfft_status pfft_profile_enable(pfft_plan p, int enable);
pfft_status pfft_profile_read(pfft_plan p, const char** names, int64_t* launches, double* ms,
                              int cap, int* n);

/* ---------------------------------------------------------------------------
 * Wavelet split plans (Section 5.3; Dirichlet symbols of Section 6.2).
 * ------------------------------------------------------------------------- */

enum { PWT_DIRICHLET = 0, PWT_DLVP = 1 };

/* Flags of pwt_plan_create. */
enum {
  /* The coefficients on G(M^T) of the first level (the input of
   * pwt_decompose, the output of pwt_reconstruct / pwt_adjoint) are in the
   * Smith-coordinate order that a pfft plan of the same M created with
   * PFFT_FLAG_LAYOUT_SNF writes (mu row-major over the cycles), so that a
   * transform -> split pipeline runs without any reordering (the split in
   * Smith coordinates of Section 5.3, Lemma 2).  All other parts keep the box
   * layout. */
  PWT_FLAG_INPUT_SNF = 1u
};

/* Plan `levels` split steps: level l (1-based) splits coefficients on
 * G(M_l^T) (M_1 = M) into a scaling part and a wavelet part on G(N_l^T),
 * N_l = J_l^{-1} M_l, and level l+1 splits the scaling part (M_{l+1} = N_l).
 *   J      : levels*d*d row-major host array of dilations, |det J_l| = 2
 *   symbol : PWT_DIRICHLET (Section 6.2) or PWT_DLVP (de la Vallee Poussin
 *            reading: sqrt|det J| times the periodised trapezoid of blend
 *            width eta, 0 < eta < 1; not defined in the paper)
 *   batch, dtype as for pfft_plan_create; flags: 0 or PWT_FLAG_INPUT_SNF.
 * Device memory owned by the plan: two workspaces of |det M| / 2 * batch
 * elements (more than one level), the phase tables, and, for complex64 plans
 * of four or more signals, the per-fibre symbols of every level (16 bytes
 * per point of G(N_l^T), about 16 |det M| bytes in all), which decompose
 * reads when it runs up to three levels in one launch.
 * Returns PFFT_ERR_NOT_INTEGRAL if some J_l^{-1} M_l is not integral. */
pfft_status pwt_plan_create(pwt_plan* out, int d, const int64_t* M, int levels, const int64_t* J,
                            int symbol, double eta, int64_t batch, int dtype, unsigned flags);

/* Size and output box of level l (1 <= l <= levels): n_l = |det N_l| and the
 * d extents of the box of H(N_l^T).  Level 0 returns the input (M_1). */
pfft_status pwt_plan_info(pwt_plan p, int level, int64_t* n, int64_t* box);

/* Decompose: c_hat [batch][|det M|] on G(M^T)  ->  wavelets[l-1] [batch][n_l]
 * on G(N_l^T) for every level and scaling [batch][n_levels] on
 * G(N_levels^T).  Per level and fibre {h0, h1} of g in G(N^T):
 *   d1[g] = 2^{-1/2} (conj A(h0) c[h0] + conj A(h1) c[h1])
 *   d2[g] = 2^{-1/2} (conj B(h0) c[h0] + conj B(h1) c[h1]),
 * B(h) = A(h + N^T l) exp(-2 pi i h^T N^{-1} z) (Section 6.2), z the non-zero
 * element of Lambda(J) cap [-1/2, 1/2)^d.  Device pointers; `wavelets` is a
 * HOST array of `levels` device pointers. */
pfft_status pwt_decompose(pwt_plan p, const void* c_hat, void* scaling, void* const* wavelets,
                          void* stream);

/* Exact inverse of pwt_decompose (perfect reconstruction): per fibre
 * c[h] = sqrt(2) (A(h) d1[g] + B(h) d2[g]) / (|A(h0)|^2 + |A(h1)|^2). */
pfft_status pwt_reconstruct(pwt_plan p, const void* scaling, const void* const* wavelets,
                            void* c_hat, void* stream);

/* Adjoint (conjugate transpose) of pwt_decompose: c[h] = 2^{-1/2} (A d1 + B d2)
 * per level; equals pwt_reconstruct for the Dirichlet symbol. */
pfft_status pwt_adjoint(pwt_plan p, const void* scaling, const void* const* wavelets, void* c_hat,
                        void* stream);

pfft_status pwt_plan_destroy(pwt_plan p);

/* General split step (Section 5.3, step 4) for a dilation J of any
 * determinant p = |det J| whose group G(J^T) = Z^d / J^T Z^d is cyclic (one
 * elementary divisor of J above 1).  M = J N must hold with N integral.  For
 * every g in G(N^T) (box of H(N^T)) and its fibre h_t = g + t N^T l (t < p,
 * l a generator of G(J^T)):
 *     parts[j][b][g] = p^{-1/2} sum_t conj(b_j(h_t)) c_hat[b][h_t],  j < p.
 * Symbols b_j:
 *   symbols != NULL: supplied by the caller (step 1 of the algorithm
 *     computes them from the generating functions), device [p][|det M|] on
 *     the box of H(M^T), p <= 16;
 *   symbols == NULL: the built-in unitary band system (p prime, up to
 *     2^20; the paper defines Dirichlet symbols for |det J| = 2 only):
 *     b_0 = the periodised Dirichlet scaling symbol A = sqrt(p w(N^{-T} h))
 *     of Section 6.2, and on each fibre, labelled by the generator l = the
 *     first unit vector outside J^T Z^d, b_j(h_t) = sqrt(p) U[j][t] e^j with
 *     U the real orthogonal completion U = 2 V V^T / (V^T V) - I,
 *     V = A / sqrt(p) + e_0, and e = exp(-2 pi i g^T N^{-1} z), z the
 *     centred generator of P(J) with l^T z = 1/p.  For p = 2 this is the
 *     pair of pwt_decompose with PWT_DIRICHLET; pwt_merge_general inverts it.
 * c_hat: device [batch][|det M|]; parts: device [p][batch][|det M| / p].
 * Plan-free: the exact setup runs on the host per call, the kernel is queued
 * on `stream`.  Errors: PFFT_ERR_NOT_INTEGRAL (J^{-1} M), PFFT_ERR_UNSUPPORTED
 * (p above the limit or G(J^T) not cyclic), PFFT_ERR_OVERFLOW
 * (|det M| >= 2^30), and the argument errors of pfft_plan_create. */
pfft_status pwt_split_general(int d, const int64_t* M, const int64_t* J, int64_t batch, int dtype,
                              const void* symbols, const void* c_hat, void* parts, void* stream);

/* Adjoint of pwt_split_general: c_hat[b][h_t] = p^{-1/2} sum_j b_j(h_t)
 * parts[j][b][g] (symbols as for pwt_split_general, NULL for the built-in
 * system).  It inverts pwt_split_general when the matrix (b_j(h_t) /
 * sqrt(p))_{j,t} is unitary on every fibre, as the built-in system is. */
pfft_status pwt_merge_general(int d, const int64_t* M, const int64_t* J, int64_t batch, int dtype,
                              const void* symbols, const void* parts, void* c_hat, void* stream);

/* ---------------------------------------------------------------------------
 * Batches of many patterns of uneven size (serving-style mixes).
 *
 * One object holds n patterns M_0 .. M_{n-1} (each with its own d_i) and
 * optionally one dilation J_i per pattern (J_i^{-1} M_i integral, G(J_i^T)
 * cyclic of order p_i = |det J_i|: 2, or a prime up to 2^20).  pfft_batch_forward
 * computes, for every pattern, the transform of pfft_forward and, when
 * dilations were given, one split level (Section 5.3, step 4): for p_i = 2
 * the split of pwt_decompose with the batch's symbol, for p_i > 2 the
 * built-in band system of pwt_split_general (symbols NULL; PWT_DIRICHLET
 * only, else PFFT_ERR_UNSUPPORTED).  All patterns run together: grouped
 * launches (the row pass of every pattern, the column pass, the split
 * levels), each CTA finding its pattern in a device table, with patterns
 * grouped by shared-memory footprint into concurrent launches, replayed as
 * one CUDA graph.
 *
 * Data: the signals are concatenated, pattern i occupying elements
 * [off_i, off_i + m_i) of `in` and `c_hat`, off_i = m_0 + ... + m_{i-1},
 * m_i = |det M_i|, each in the box layout of its own plan.  With n_i =
 * m_i / p_i, the scaling part of pattern i occupies [s_i, s_i + n_i) of
 * `scaling` and its p_i - 1 band parts occupy [w_i + (j - 1) n_i,
 * w_i + j n_i), j = 1 .. p_i - 1, of `wavelet`, where s_i = n_0 + ... +
 * n_{i-1} and w_i = (p_0 - 1) n_0 + ... + (p_{i-1} - 1) n_{i-1}
 * (pfft_batch_split_layout returns them; when every p_i = 2,
 * s_i = w_i = off_i / 2).  One signal per pattern (batch 1).
 * ------------------------------------------------------------------------- */
enum {
  PFFT_BATCH_NO_GRAPH = 1u, /* queue the grouped launches directly instead of replaying a graph */
  PFFT_BATCH_AUTOTUNE = 2u, /* time candidate tile / radix schedules at creation and keep the fastest */
  PFFT_BATCH_RADIX8 = 4u,   /* start from radix-8 power-of-two stages instead of radix 16 */
  /* the whole batch -- every row-pass tile, every column-pass tile, every
   * split unit -- in ONE kernel launch whose CTAs take work units from a
   * device queue in dependency order; a column tile waits (bounded) until
   * its pattern's row tiles are done, a split unit until the pattern's
   * coefficients are.  Results equal the grouped launches' up to rounding
   * (every tile runs with 512 threads, which changes how the stage twiddle
   * powers are formed).  All units share the largest tile's shared memory
   * (fewer CTAs per SM when one pattern needs a large tile). */
  PFFT_BATCH_ONE_LAUNCH = 8u
};

/* n >= 1 patterns; d: host array of n dimensions (1..4); M: host array, the
 * d_i x d_i row-major matrices one after the other; J: NULL (transforms
 * only) or dilations in the same layout; symbol / eta as for
 * pwt_plan_create (ignored when J is NULL); flags: PFFT_BATCH_* bits.
 * Every pattern is subject to the limits of pfft_plan_create; the first
 * failing pattern's status is returned and nothing is kept.  Autotuning runs
 * the batch on scratch buffers it allocates and frees, synchronising the
 * device. */
pfft_status pfft_batch_create(pfft_batch* out, int n, const int* d, const int64_t* M, const int64_t* J,
                              int symbol, double eta, int dtype, unsigned flags);

/* m: host array of n (|det M_i|) or NULL; total: sum of m_i or NULL. */
pfft_status pfft_batch_info(pfft_batch b, int64_t* m, int64_t* total);

/* Split layout of a batch with dilations: per pattern p_i = |det J_i| and the
 * element offsets s_i, w_i of its scaling and band parts (see above), and
 * the element counts of the scaling and wavelet buffers.  Host arrays of n
 * values or NULL; without dilations every value is 0. */
pfft_status pfft_batch_split_layout(pfft_batch b, int* p, int64_t* scaling_off, int64_t* wavelet_off,
                                    int64_t* scaling_total, int64_t* wavelet_total);

/* The chosen schedule: element budgets of the row- and column-pass tiles, the
 * launch order (1: largest work first, 0: pattern order) and the largest
 * power-of-two radix of the stages (16 or 8).  NULLs allowed. */
pfft_status pfft_batch_schedule(pfft_batch b, int* row_budget, int* col_budget, int* order, int* max_radix);

/* in -> c_hat for every pattern; if the batch has dilations and scaling and
 * wavelet are non-NULL, also c_hat -> (scaling, wavelet).  Device pointers,
 * layout above (scaling / wavelet hold the totals of pfft_batch_split_layout).  The graph is built on the first call and rebuilt when any
 * of the four pointers changes; a batch may be used from one stream at a
 * time (its workspace is shared). */
pfft_status pfft_batch_forward(pfft_batch b, const void* in, void* c_hat, void* scaling, void* wavelet,
                               void* stream);

/* PFFT_BATCH_ONE_LAUNCH batches: the number of tries of every dependency
 * wait before it gives up (also bounded by about one second); spins < 0
 * restores the default (2^22).  A wait that gives up records
 * PFFT_ERR_TIMEOUT in the batch's device status word and makes the rest of
 * the launch return without work (outputs incomplete).  Returns
 * PFFT_ERR_UNSUPPORTED for other batches.  Takes effect on the next
 * pfft_batch_forward. */
pfft_status pfft_batch_set_wait_limit(pfft_batch b, int64_t spins);

/* Reads and clears the batch's device status word on `stream` (synchronising
 * it): PFFT_OK, or PFFT_ERR_TIMEOUT after a wait of a PFFT_BATCH_ONE_LAUNCH
 * launch gave up.  PFFT_OK for batches without that flag. */
pfft_status pfft_batch_device_status(pfft_batch b, void* stream);

pfft_status pfft_batch_destroy(pfft_batch b);

/* The same decomposition as pwt_decompose for PFFT_C64 data, but without a
 * plan and without allocating any device memory (the paper has no
 * counterpart; this serves callers that cannot call cudaMalloc, e.g. code
 * that runs under a device-memory budget or pool that forbids allocations,
 * or that must not hit an allocation failure mid-run).  Arguments are those
 * of pwt_plan_create and pwt_decompose; all pointers are caller-owned and
 * `wavelets` is a host array of `levels` device pointers.
 *   Scratch: the scaling parts between levels live in one fixed array of
 *   2^21 complex64 values (16 MiB) that every GPU loading this library holds
 *   until the process exits; (|det M| / 2) * batch must not exceed 2^20 when
 *   levels > 1, else PFFT_ERR_OVERFLOW is returned and nothing runs.
 *   The first call on a device looks the array up (cudaGetSymbolAddress), so
 *   make that first call before any stream capture.  Every call on a device
 *   shares the array: calls whose work overlaps on the GPU (other streams,
 *   other host threads) race and must be serialised by the caller.  Nothing
 *   in the array needs clearing: each call writes every element before it
 *   reads it.  Phases are evaluated in single precision in the kernel
 *   (equal to pwt_decompose within the complex64 tolerance). */
pfft_status pwt_decompose_noalloc(int d, const int64_t* M, int levels, const int64_t* J, int symbol,
                                  double eta, int64_t batch, const void* c_hat, void* scaling,
                                  void* const* wavelets, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PFFT_H */
