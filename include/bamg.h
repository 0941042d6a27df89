/*
 * bamg.h - C ABI of the blocked smoothed-aggregation AMG reuse phase on one GPU.
 *
 * The library implements the two recurring phases of a smoothed-aggregation
 * AMG solve whose hierarchy is reused across solves (arxiv 2606.24748,
 * Sec. 3.1): the numeric Galerkin recompute A_c = P^T A P on rectangular-block
 * matrices, and the V-cycle under CG whose smoother is point-block Jacobi
 * (Sec. 4.1) under Chebyshev acceleration.  Operators are assembled through
 * blocked COO (Sec. 3.4, Sec. 5).
 *
 * Conventions shared by every entry point
 *  - Pointers named "device" point to CUDA device memory of the device that
 *    was current when the context was created; they are borrowed for the call
 *    only (the call is stream ordered: the caller keeps them alive until the
 *    stream reaches the work).  Pointers named "host" are read before return.
 *  - Block values are row-major bs_r x bs_c blocks (element (r, c) at
 *    r * bs_c + c).  Vectors are dof-ordered: dof = block * bs + component.
 *  - Every call returns a bamg_status; on failure bamg_last_error() holds a
 *    one-line description.  No C++ exception crosses this ABI and no kernel
 *    traps: errors detected on the device (non-finite values, exhausted
 *    waits) are recorded in a device error word and returned by the next call
 *    that synchronizes (bamg_ctx_sync, bamg_cg_solve).
 *  - The library allocates its own device memory (matrices, plans, the
 *    hierarchy and work vectors) during the setup calls: bsr_create,
 *    coo_preallocate, ptap_symbolic, mg_setup.  The recurring calls
 *    (coo_set_values, ptap_numeric, mg_update, vcycle, cg_solve, spmv, spmm)
 *    allocate nothing.
 *  - Indices are int32 block indices; counts are int64.
 */
#ifndef BAMG_H
#define BAMG_H

#include <stdint.h>

#if defined(__GNUC__)
#define BAMG_API __attribute__((visibility("default")))
#else
#define BAMG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BAMG_OK = 0,
  BAMG_ERR_INVALID = 1,        /* bad argument or size; nothing was launched */
  BAMG_ERR_OOM = 2,            /* device allocation failed */
  BAMG_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  BAMG_ERR_STATE = 4,          /* object used before the call that prepares it */
  BAMG_ERR_NAN = 5,            /* a non-finite value was produced */
  BAMG_ERR_BREAKDOWN = 6,      /* CG breakdown (p^T A p <= 0) or a non-SPD block */
  BAMG_ERR_NOT_CONVERGED = 7,  /* CG reached maxit */
  BAMG_ERR_TIMEOUT = 8         /* a bounded device wait ran out */
} bamg_status;

typedef enum { BAMG_FP64 = 0, BAMG_FP32 = 1 } bamg_prec;

typedef struct bamg_ctx bamg_ctx;
typedef struct bamg_bsr bamg_bsr;
typedef struct bamg_ptap bamg_ptap;
typedef struct bamg_mg bamg_mg;

/* ---------------------------------------------------------------- context */

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t, borrowed, e.g. torch.cuda.current_stream().cuda_stream;
 * NULL = the legacy default stream).  All work of objects made from this
 * context is issued on that stream. */
BAMG_API bamg_status bamg_ctx_create(void* cuda_stream, bamg_ctx** out);
BAMG_API bamg_status bamg_ctx_destroy(bamg_ctx* ctx);
/* Message of the last failed call on this context ("" if none).  Owned by
 * the context, valid until the next call. */
BAMG_API const char* bamg_last_error(const bamg_ctx* ctx);
/* Wait for the context's stream, then turn the device error word into a
 * status (and clear it). */
BAMG_API bamg_status bamg_ctx_sync(bamg_ctx* ctx);
/* Bounded device waits (a CTA polling a counter that other CTAs of the same
 * launch advance, e.g. inside the coarsest-level factorisation) give up
 * after `polls` polls, record BAMG_ERR_TIMEOUT in the device error word and
 * go on, so that no kernel waits forever; the status reaches the host at
 * the next call that reads the error word (bamg_ctx_sync, bamg_cg_solve).
 * Default 2^22 polls (about 0.4 s).  0 gives up at the first wait without
 * polling, which exercises the timeout path deterministically (the results
 * of that call are then not valid).  BAMG_ERR_INVALID for polls < 0. */
BAMG_API bamg_status bamg_ctx_set_wait_limit(bamg_ctx* ctx, int64_t polls);

/* Kernel timing for benchmarks.  While enabled, the library brackets the
 * launches of the kernels listed in bamg_prof_slot with CUDA events on the
 * context's stream (inside CUDA graphs as external event-record nodes) and
 * accumulates their device time.  Enabling resets the totals.  _read waits
 * for the stream, then returns the total milliseconds and launch count of a
 * slot (kernels that only returned early are not counted). */
typedef enum {
  BAMG_PROF_CHEB_STEP_L0 = 0,   /* fused Chebyshev step on the finest level */
  BAMG_PROF_CHEB_RINIT_L0 = 1,  /* fused residual + first direction, finest level */
  BAMG_PROF_PTAP_STAGE1_L0 = 2, /* Galerkin stage Z = A P, finest level */
  BAMG_PROF_PTAP_STAGE2_L0 = 3, /* Galerkin stage A_c = P^T Z, finest level */
  BAMG_PROF_CG_AP = 4,          /* CG product q = A p */
  BAMG_PROF_COO = 5,            /* blocked COO numeric assembly */
  BAMG_PROF_COARSE_FACTOR = 6,  /* whole coarsest-level factorisation */
  BAMG_PROF_SMOOTH_COARSE = 7,  /* pre- or post-smoothing of a level below the finest */
  BAMG_PROF_TRANSFER = 8,       /* one restriction or prolongation */
  BAMG_PROF_COARSE_SOLVE = 9,   /* coarsest-level solve inside a cycle */
  BAMG_PROF_L0_VECTOR = 10,     /* finest-level smoother start, final update, precision casts */
  BAMG_PROF_CG_XR = 11,         /* CG x, r update and residual norm */
  BAMG_PROF_CG_VECTOR = 12,     /* CG step-length dots and direction update */
  BAMG_PROF_REFRESH = 13,       /* smoother refresh of a level (inverses, eigen-estimate) */
  BAMG_PROF_CHEB_PRE_L0 = 14,   /* the finest level's pre-smoothing steps alone: a sample of slot 0
                                   with one bracket per cycle instead of two.  While it is enabled
                                   those steps are timed here and not in slot 0.  bamg_ctx_profile
                                   does not enable it; bamg_ctx_profile_slots does. */
  BAMG_PROF_COUNT = 15
} bamg_prof_slot;
/* enable != 0: every slot but BAMG_PROF_CHEB_PRE_L0; 0 disables. */
BAMG_API bamg_status bamg_ctx_profile(bamg_ctx* ctx, int enable);
/* Enable timing for the slots in `mask` only (bit s = slot s; 0 disables).
 * Every bracketed launch loses its programmatic overlap with its neighbours
 * and each pair costs two event records, so a timed run that needs one
 * kernel's duration should bracket that kernel alone. */
BAMG_API bamg_status bamg_ctx_profile_slots(bamg_ctx* ctx, unsigned mask);
BAMG_API bamg_status bamg_ctx_profile_read(bamg_ctx* ctx, int slot, double* total_ms, int64_t* launches);
/* Number of kernels this library has launched in this process (kernels run
 * through CUDA graphs included, counted per graph launch). */
BAMG_API uint64_t bamg_kernel_launches(void);
/* Measured FMA throughput of the FP64 (precision = BAMG_FP64) or FP32
 * (BAMG_FP32) pipe on the context's device, in TFLOP/s (2 flop per FMA),
 * written to *tflops (host).  A benchmark aid, not a step of the method: it
 * gives the rooflines of the ALU-bound kernels a measured denominator
 * (Sec. 4.2 ties SpMV to memory traffic; on this part the FP64 FMA pipe
 * binds first).  Independent FMA chains on every SM at full occupancy, one
 * timed launch of about 0.1 s after a warm-up.  Allocates a few KB on the
 * context's stream and waits for it.  BAMG_ERR_INVALID for another
 * precision or a null pointer. */
BAMG_API bamg_status bamg_probe_fma_rate(bamg_ctx* ctx, int precision, double* tflops);
/* Device memory of the library on the context's device: every library
 * allocation is stream-ordered from the device's default memory pool, so the
 * pool's bytes in use and their high-water mark (since the last reset) are the
 * library's own.  Either output may be NULL; reset_peak != 0 restarts the
 * high-water mark at the current use after reading it. */
BAMG_API bamg_status bamg_device_memory(bamg_ctx* ctx, uint64_t* in_use, uint64_t* peak, int reset_peak);

/* ------------------------------------------------------- block matrices */

/* Rectangular-block sparse matrix (Sec. 2.3: independent row and column block
 * sizes; 3x3 fine operator, 3x6 prolongator, 6x6 coarse operators), nbr x nbc
 * blocks of bs_r x bs_c, 1 <= bs_r, bs_c <= 8.  Empty until a pattern is set
 * by bamg_bsr_coo_preallocate or produced by bamg_ptap_symbolic. */
BAMG_API bamg_status bamg_bsr_create(bamg_ctx* ctx, int bs_r, int bs_c, int64_t nbr, int64_t nbc,
                            bamg_bsr** out);
BAMG_API bamg_status bamg_bsr_destroy(bamg_bsr* A);

/* Blocked COO preallocation (Sec. 3.4, Sec. 5): declare the block
 * coordinates of n contributions, bi[k] in [0, nbr), bj[k] in [0, nbc)
 * (device int32 arrays of length n).  Duplicates are allowed and are summed
 * by set_values; a contribution with bi[k] < 0 or bj[k] < 0 is ignored.
 * Builds the block pattern (rows sorted by column) and the cached
 * duplicate-summation plan.  BAMG_ERR_INVALID if an index is >= nbr / nbc
 * (checked on the device before the pattern is built). */
BAMG_API bamg_status bamg_bsr_coo_preallocate(bamg_bsr* A, int64_t n, const int32_t* bi,
                                     const int32_t* bj);
/* Numeric blocked COO assembly (Sec. 5): v is a device array of n row-major
 * bs_r*bs_c blocks in the order given to preallocate.  add = 0: each stored
 * block becomes the sum of its contributions; add = 1: the sum is added.
 * Deterministic (fixed summation order).  Increments the matrix version. */
BAMG_API bamg_status bamg_bsr_coo_set_values(bamg_bsr* A, const double* v, int add);
/* Element-by-element assembly of the same COO stream: every contribution is
 * added straight into its block with an FP64 atomic (the baseline the
 * blocked COO path of Sec. 5 replaces; kept for measurement).  Same arguments
 * and result as bamg_bsr_coo_set_values up to the order of the additions,
 * which atomics do not fix: sums may differ in the last bits and from run to
 * run.  No NaN check.  The first call builds a per-entry slot map (4 bytes per
 * COO entry, owned by the matrix). */
BAMG_API bamg_status bamg_bsr_coo_scatter_values(bamg_bsr* A, const double* v, int add);

/* Sizes and version (any pointer may be NULL). */
BAMG_API bamg_status bamg_bsr_info(const bamg_bsr* A, int* bs_r, int* bs_c, int64_t* nbr, int64_t* nbc,
                          int64_t* nnzb, uint64_t* version);
/* Sliced storage of A (Sec. 4.2's blocked layout, padded to 32-row slices):
 * *stored_slots = block slots held (nnzb plus the padding of every slice to
 * its longest row); *rows_sorted = 1 when the rows sit in the slices by
 * decreasing length within windows of 1,024 rows.  Operators from COO
 * preallocation and Galerkin products are sorted when that removes at least
 * a tenth of the slots (uneven rows, e.g. Q2's vertex and mid-edge nodes);
 * prolongators always.  Vectors are indexed by row either way.  Either
 * pointer may be NULL.  BAMG_ERR_STATE without a pattern. */
BAMG_API bamg_status bamg_bsr_storage(const bamg_bsr* A, int64_t* stored_slots, int* rows_sorted);
/* Copy the block pattern out: rowptr (nbr + 1) and colidx (nnzb), device. */
BAMG_API bamg_status bamg_bsr_get_pattern(const bamg_bsr* A, int32_t* rowptr, int32_t* colidx);
/* Copy the values out in pattern order: nnzb row-major blocks, device. */
BAMG_API bamg_status bamg_bsr_get_values(const bamg_bsr* A, double* vals);
/* Declare A symmetric (A = A^T); Galerkin products with A then compute the
 * upper block triangle and mirror it.  The caller guarantees symmetry. */
BAMG_API bamg_status bamg_bsr_set_symmetric(bamg_bsr* A, int symmetric);

/* Blocked SpMV (Sec. 4.2): y = A x (transpose = 0, x has nbc*bs_c entries,
 * y nbr*bs_r), device vectors of the given precision.  BAMG_FP32 computes
 * with a float copy of the values, refreshed when the version changed.
 * transpose = 1 is not supported (BAMG_ERR_INVALID): transposes are formed
 * explicitly (the hierarchy caches R = P^T). */
BAMG_API bamg_status bamg_bsr_spmv(bamg_bsr* A, const void* x, void* y, bamg_prec prec, int transpose);
/* Multi-right-hand-side blocked product Y = A X for k right-hand sides
 * (1 <= k <= 32), right-hand-side-minor layout: X[dof * k + j]. */
BAMG_API bamg_status bamg_bsr_spmm(bamg_bsr* A, const void* X, void* Y, int k, bamg_prec prec);

/* Thread mapping of this matrix's row kernels ("lanes"): a power of two in
 * 1..32 = lanes per block row (1 = one row per lane for long matrices, more
 * lanes for few, long rows); or, for 6x3 and 6x6 blocks only, the component
 * split: -VS = VS warps (1, 2 or 4) per output component of a 32-row slice,
 * each taking every VS-th block of the rows (no cross-lane sums, no idle
 * lanes; the FP64 pipe's two FMA per clock per SM make those count), or
 * -32 * VR (VR = 1, 2, 4) = one CTA per row, VR warps per component with
 * their lanes over the row's blocks (for few, very long rows; used by the
 * transfer and product kernels, the smoother kernels treat it as -1); for
 * 6x3 blocks only (the finest restriction), -(256 + VB) with VB = 2, 4, 8,
 * 16 or 32 = the block split: VB warps per 32-row slice, each summing every
 * output component over every VB-th block of its lane's row, so that each
 * block's column index and gathered x are loaded once per lane; 0 in
 * _set_lanes means -4.  _autotune times the product for every choice from a
 * flushed L2 on the context's stream and keeps the fastest (a choice must
 * beat the best one before it by 3%, against timing noise), for the FP64
 * values and, when present, the FP32 copy (allocates work vectors; returns
 * the FP64 choice and its time in ms, either may be NULL).  Results do not
 * depend on the choice beyond summation order.  _set_lanes applies to both
 * copies. */
BAMG_API bamg_status bamg_bsr_autotune(bamg_bsr* A, int* lanes, float* ms);
BAMG_API bamg_status bamg_bsr_set_lanes(bamg_bsr* A, int lanes);
BAMG_API bamg_status bamg_bsr_get_lanes(const bamg_bsr* A, int* lanes);
/* The same for one copy: prec = BAMG_FP64 (the values) or BAMG_FP32 (the
 * float copy of the mixed cycle).  The autotuner and the hierarchy's smoother
 * timing choose the two separately; _get_lanes and _set_lanes above read the
 * FP64 choice and write both.  Same codes and checks; BAMG_ERR_INVALID for
 * another precision. */
BAMG_API bamg_status bamg_bsr_set_lanes_prec(bamg_bsr* A, int prec, int lanes);
BAMG_API bamg_status bamg_bsr_get_lanes_prec(const bamg_bsr* A, int prec, int* lanes);

/* ---- Block operator inspection and the aggregation graph (Sec. 2.2, 3.2, 6) */

/* Frobenius norm of every stored block (Sec. 3.2: the block norm is the
 * coupling weight), in block-CSR order (block rows in order, columns
 * ascending), into the device array out (nnzb doubles).  3x3, 3x6, 6x3 and
 * 6x6 blocks; needs current FP64 values (BAMG_ERR_STATE after an FP32-only
 * product). */
BAMG_API bamg_status bamg_bsr_block_norms(bamg_bsr* A, double* out);
typedef enum { BAMG_NORM_FROBENIUS = 0, BAMG_NORM_INFINITY = 1 } bamg_norm_type;
/* Norm of the whole matrix taken over its blocks: Frobenius, or the largest
 * absolute scalar row sum.  *out is a host double; waits for the stream. */
BAMG_API bamg_status bamg_bsr_norm(bamg_bsr* A, int type, double* out);
/* Strength-of-connection graph of a square block operator (Sec. 2.2 with the
 * block norm of Sec. 3.2).  With s the sum of a block's squared entries
 * (row-major, each product and sum rounded apart), j is a strong neighbour of
 * block row i when j != i, s_ij > 0 and s_ij^2 >= (eps^4 s_ii) s_jj, which is
 * ||A_ij||_F >= eps sqrt(||A_ii||_F ||A_jj||_F) decided without a square root.
 * Output: CSR graph in caller-owned device arrays, rowptr (nbr + 1 ints) and
 * col (col_capacity ints; neighbours in ascending order); *nedges (host) gets
 * the edge count.  BAMG_ERR_INVALID if col_capacity < edges (nnzb always
 * suffices) or eps < 0.  Waits for the stream once (the edge count). */
BAMG_API bamg_status bamg_strength_graph(bamg_bsr* A, double eps, int* rowptr, int* col, int64_t col_capacity,
                                         int64_t* nedges);
/* Device MIS coarsening (Sec. 6) of a symmetric CSR graph of n vertices
 * (device arrays rowptr, col).  Vertex weights are splitmix64(i, seed) with
 * ties broken by i; Luby rounds (enter when beating every non-excluded
 * neighbour, then exclude the neighbours of entered vertices) reach the greedy
 * maximal independent set in descending (weight, i) order.  Aggregates: one
 * per set vertex, numbered in vertex order; every other vertex joins its
 * neighbour in the set of largest (weight, j).  agg: device array of n ints
 * (caller-owned); *n_agg and *rounds (host) get the aggregate and round
 * counts.  Waits for the stream after every round.  A graph that is not
 * symmetric can leave a vertex without a set neighbour: BAMG_ERR_INVALID. */
BAMG_API bamg_status bamg_mis_aggregate(bamg_ctx* ctx, int64_t n, const int* rowptr, const int* col, uint64_t seed,
                                        int* agg, int64_t* n_agg, int* rounds);

/* Residual norm ||b - A x||_2 for a square operator with 3x3 or 6x6 blocks,
 * written to *norm (device double) on A's context stream; x, b are device
 * FP64 vectors.  This entry point allocates no device memory at all, for
 * callers that cannot call cudaMalloc: components of a larger application
 * whose device memory is all pre-reserved by that application's own pool, so
 * that a further cudaMalloc would fail or break the pool's accounting.  (It
 * still launches a kernel and issues a memset, so it is no use from a CUDA
 * host callback, where no CUDA call is allowed.)  The paper has no
 * counterpart; it is an operational addition.
 *  - Scratch: the reduction's partial sums live in a file-scope device array
 *    of 4096 doubles (32 KB) plus one counter, which every GPU that loads the
 *    library holds until the process exits.  One partial per 128 thread
 *    slots: a matrix needs (block rows rounded up to 32) x (lanes per row)
 *    <= 4096 x 128 = 524,288 slots (e.g. 524,288 block rows at one lane per
 *    row); larger ones return BAMG_ERR_INVALID with the sizes in the message.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the array and leaves its last contents there; the
 *    counter is cleared at the start of each call.  Calls that overlap on the
 *    GPU (different streams, or several in flight) race on the scratch. */
BAMG_API bamg_status bamg_bsr_residual_norm_noalloc(const bamg_bsr* A, const double* x, const double* b,
                                                    double* norm);

/* ------------------------------------------------- row-sharded operator */

/* Partition plan of a square block pattern over `nparts` contiguous ranges
 * of block rows (Sec. 3.3): part p owns rows [row_starts[p],
 * row_starts[p+1]).  Its rows keep their blocks with columns renumbered
 * locally: the owned columns first (column - row_starts[p]), then the ghost
 * columns (owned by other parts) in ascending global order, which groups
 * them by owner.  Host arrays only (rowptr nbr + 1, colidx, row_starts
 * nparts + 1 with row_starts[0] = 0, row_starts[nparts] = nbr,
 * non-decreasing); no CUDA call, so it runs without a GPU.  The getters copy
 * into caller-owned host arrays sized by bamg_halo_part_info. */
typedef struct bamg_halo bamg_halo;
BAMG_API bamg_status bamg_halo_create(int64_t nbr, const int32_t* rowptr, const int32_t* colidx, int nparts,
                                      const int64_t* row_starts, bamg_halo** out);
BAMG_API bamg_status bamg_halo_destroy(bamg_halo* halo);
BAMG_API bamg_status bamg_halo_part_info(const bamg_halo* halo, int part, int64_t* n_owned, int64_t* n_ghost,
                                         int64_t* nnzb);
/* Local pattern of a part: rowptr (n_owned + 1), colidx (nnzb, local
 * numbering, ascending per row) and block_src (nnzb: the global block index,
 * position in the global colidx, of each local block). */
BAMG_API bamg_status bamg_halo_part_pattern(const bamg_halo* halo, int part, int32_t* rowptr, int32_t* colidx,
                                            int64_t* block_src);
/* Ghost columns of a part (global, ascending) and the part owning each. */
BAMG_API bamg_status bamg_halo_part_ghosts(const bamg_halo* halo, int part, int64_t* ghost, int32_t* owner);
/* The halo message from part `from` to part `to`: the `from`-local row
 * indices whose entries `to` needs, in the order of `to`'s ghost list
 * (*count rows; local_rows may be NULL to query the count). */
BAMG_API bamg_status bamg_halo_sends(const bamg_halo* halo, int from, int to, int64_t* count, int64_t* local_rows);

/* All parts of one partition of A (and of the Galerkin product with P) on
 * the context's GPU, run one after another (Sec. 3.3, Sec. 3.5, Sec. 4.8).
 * Part p keeps A_ext = its rows in a square matrix of owned + ghost rows
 * (ghost rows empty, local columns as bamg_halo) and P_ext = [P_own; P_oth],
 * the rows of P for its owned and ghost nodes.  Creates Ac (caller-owned,
 * bamg_bsr_destroy) with the union of the parts' product patterns, which is
 * the structural pattern of P^T A P.  A, P: FP64 values; square A with
 * square blocks; P with A's block rows (3x3 -> 3x6, 6x6 -> 6x6 or 3x3 -> 3x3). */
typedef struct bamg_sharded bamg_sharded;
BAMG_API bamg_status bamg_sharded_create(bamg_bsr* A, bamg_bsr* P, int nparts, const int64_t* row_starts,
                                         bamg_sharded** out, bamg_bsr** Ac);
/* y = A x through the parts: each gathers its halo (ghost entries of x) and
 * multiplies its rows; FP64 device vectors of the global size.  The parts'
 * copies of A are refreshed when A's version changed. */
BAMG_API bamg_status bamg_sharded_spmv(bamg_sharded* sh, const double* x, double* y);
/* Numeric Galerkin product through the parts: each computes
 * C_p = P_ext^T A_ext P_ext with its cached plan; P_oth is gathered only when
 * P's version changed since the last call (state gate, Sec. 3.5); then
 * A_c = sum of the C_p, block by block in part order (the off-process
 * reduce).  A, P must be the matrices the object was built for and Ac the
 * matrix it created (BAMG_ERR_STATE otherwise). */
BAMG_API bamg_status bamg_sharded_ptap(bamg_sharded* sh, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac);
/* Communication profile of the partition, as a multi-GPU run would move it:
 * halo entries per SpMV, P_oth blocks (once per P version) and the blocks of
 * C_p in coarse rows owned by another part (per recompute; a coarse row
 * belongs to the part owning the first fine row that touches it). */
typedef struct {
  int64_t ghost_rows;           /* sum over parts of ghost block rows */
  int64_t halo_bytes_per_spmv;  /* ghost_rows x bs x 8 */
  int64_t poth_blocks;          /* rows of P gathered from other parts, in blocks */
  int64_t poth_bytes;           /* poth_blocks x (bs x bs_p x 8 + 4) */
  int64_t poth_gathers;         /* gathers done so far (P versions seen) */
  int64_t reduce_blocks;        /* off-process C_p blocks per recompute */
  int64_t reduce_bytes_per_ptap;/* reduce_blocks x (bs_p^2 x 8 + 4) */
  int64_t max_owned_rows;       /* the largest part */
} bamg_shard_stats;
BAMG_API bamg_status bamg_sharded_stats(const bamg_sharded* sh, bamg_shard_stats* out);
BAMG_API bamg_status bamg_sharded_destroy(bamg_sharded* sh);

/* ----------------------------------------------------- Galerkin product */

/* Symbolic Galerkin product (Sec. 3.1, Sec. 3.5): A (n x n blocks of
 * bs x bs) and P (n x nc blocks of bs x bs_p) must have patterns.  Creates the
 * coarse matrix Ac (nc x nc blocks of bs_p x bs_p) with the structural
 * pattern of P^T A P (every stored block counts, no value-based pruning) and
 * a plan holding the intermediate pattern and the gather lists that the
 * numeric phase reuses.  Ac is owned by the caller (bamg_bsr_destroy). */
BAMG_API bamg_status bamg_ptap_symbolic(bamg_bsr* A, bamg_bsr* P, bamg_ptap** plan, bamg_bsr** Ac);
/* State gate of a plan (Sec. 3.5): how many times the numeric phase rebuilt
 * its block-ordered copy of P, which it does only when P's version differs
 * from the one cached (host output). */
BAMG_API bamg_status bamg_ptap_get_refreshes(const bamg_ptap* plan, uint64_t* p_refreshes);
/* Numeric Galerkin recompute with the reused pattern (Sec. 3.1 "hot PtAP",
 * Sec. 3.5): Ac = P^T A P in FP64.  The plan caches a gather-friendly copy of
 * P and rebuilds it only when P's version changed (state gate, Sec. 3.5).
 * Increments Ac's version.  BAMG_ERR_STATE if A, P or Ac are not the
 * matrices (patterns) the plan was built for. */
BAMG_API bamg_status bamg_ptap_numeric(bamg_ptap* plan, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac);
/* Same product in the given precision; BAMG_FP32 writes only the float copy
 * of Ac (used by FP32 V-cycles). */
BAMG_API bamg_status bamg_ptap_numeric_prec(bamg_ptap* plan, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac,
                                   bamg_prec prec);
BAMG_API bamg_status bamg_ptap_destroy(bamg_ptap* plan);

/* ------------------------------------------------------------ multigrid */

typedef struct {
  int max_levels;           /* depth limit, >= 1 (default 10) */
  int64_t max_coarse_dofs;  /* coarsen while a level has more dofs (default 2100) */
  int grid[3];              /* fine node grid for geometric aggregates, x fastest;
                               required (> 0) by bamg_mg_setup */
  int cheb_degree;          /* Chebyshev steps per smoothing (default 2) */
  double cheb_lower;        /* interval [lower, upper] * lambda_max (0.1, 1.1) */
  double cheb_upper;
  int power_its;            /* power iterations of the eigen-estimate (15) */
  int precision;            /* bamg_prec of the V-cycle: FP64, or FP32 = mixed form
                               (FP32 operators, smoother and vectors; FP64 CG,
                               eigen-estimates and coarsest solve) */
  int autotune;             /* 1 (default): bamg_bsr_autotune every level's
                               operator, prolongator and restriction at setup,
                               then time each coarse level's own smoothing pass
                               to pick its warps per component */
  int coarse_solver;        /* coarsest-level exact solve: 0 (default) = banded
                               block-tridiagonal Cholesky when the level's
                               half-bandwidth splits it into >= 3 chunks, else
                               dense; 1 = always dense; 2 = banded whenever
                               it splits into >= 2 chunks */
  int aggregation;          /* BAMG_AGG_GEOMETRIC (default): 3x3x3 node cubes
                               on opts.grid; BAMG_AGG_MIS: on every level, MIS
                               aggregates of the block strength graph (see
                               bamg_mg_setup) */
  double mis_eps;           /* strength threshold eps of BAMG_AGG_MIS (0.02) */
  uint64_t mis_seed;        /* vertex-weight seed of level l: mis_seed + l (1) */
} bamg_mg_opts;
typedef enum { BAMG_AGG_GEOMETRIC = 0, BAMG_AGG_MIS = 1 } bamg_aggregation;

typedef struct {
  int iterations;     /* CG iterations taken */
  int converged;      /* 1 if ||r|| <= rtol ||b|| */
  double rnorm;       /* final recursive residual norm */
  double bnorm;       /* ||b|| */
  double true_rnorm;  /* ||b - A x|| recomputed at exit */
} bamg_cg_info;

BAMG_API void bamg_mg_opts_default(bamg_mg_opts* opts);

/* Cold setup (Sec. 2.2, Sec. 3.2): A is the assembled fine operator (3x3
 * blocks); coords (host, nbr x 3 doubles) and dirichlet (host, nbr bytes,
 * 1 = clamped node) give the rigid-body near-null space.  Aggregates are
 * cubes of 3x3x3 nodes of opts->grid (a remainder joins the last aggregate),
 * or, with opts->aggregation = BAMG_AGG_MIS (Sec. 3.2, Sec. 6), on every level
 * the device MIS aggregates of the block strength graph (bamg_strength_graph
 * with opts->mis_eps, bamg_mis_aggregate with seed mis_seed + level), where a
 * vertex without strong neighbours (a clamped node) joins no aggregate (its
 * prolongator row is empty) and an aggregate whose near-null block is rank
 * deficient (fewer than three non-collinear fine nodes) is dissolved, each of
 * its vertices joining the surviving aggregate of a strong neighbour whose
 * root has the largest (weight, root), survivors renumbered in root order;
 * the tentative prolongator is the per-aggregate QR of the rigid-body modes,
 * the prolongator is smoothed by one damped-Jacobi step with
 * omega = 4 / (3 lambda_max(D^-1 A)), coarse operators are Galerkin
 * products; then bamg_mg_update runs once.  A stays owned by the caller and
 * must outlive the hierarchy. */
BAMG_API bamg_status bamg_mg_setup(bamg_ctx* ctx, bamg_bsr* A, const double* coords,
                          const uint8_t* dirichlet, const bamg_mg_opts* opts, bamg_mg** out);
/* Numeric re-setup for a new operator with the same pattern (same mesh):
 * reuses aggregates, tentative prolongators and every symbolic plan, and
 * recomputes the prolongator damping, the smoothed prolongators and the
 * Galerkin products from the current values of A, then runs the update.
 * Equivalent to a fresh bamg_mg_setup of the same operator. */
BAMG_API bamg_status bamg_mg_resetup(bamg_mg* mg);
/* Hot reuse step (Sec. 3.1): with the prolongators fixed, recompute every
 * Galerkin product from the current values of A, then the smoother data
 * (block-diagonal inverses, eigen-estimates) and the coarsest factor. */
BAMG_API bamg_status bamg_mg_update(bamg_mg* mg);
/* One V-cycle x = M b from x = 0 (Sec. 2.1): FP64 device vectors of the fine
 * size, in either precision form. */
BAMG_API bamg_status bamg_vcycle(bamg_mg* mg, const double* b, double* x);
/* Preconditioned CG (Sec. 4.1) on the fine operator, x0 = 0, stops when the
 * unpreconditioned residual ||r|| <= rtol ||b||.  FP64 device vectors.
 * Synchronizes once at exit to fill info (may be NULL).  Returns
 * BAMG_ERR_NOT_CONVERGED after maxit iterations, BAMG_ERR_BREAKDOWN if
 * p^T A p <= 0. */
BAMG_API bamg_status bamg_cg_solve(bamg_mg* mg, const double* b, double* x, double rtol, int maxit,
                          bamg_cg_info* info);
/* Many right-hand sides at once (blocked SpMM form of the cycle and of CG).
 * B and X are device FP64 arrays of k fine vectors stored RHS-minor: entry
 * (dof d, vector j) at B[d * k + j], 1 <= k <= 32.  Internally the columns are
 * padded to a power of two >= 4; the work arrays (about 6 fine vectors per
 * column plus each level's cycle vectors) are allocated on the first call
 * for a column count and kept with the hierarchy.
 *
 * bamg_mg_vcycle_multi: X = M B, one V-cycle per column from x = 0.  Per
 * column the arithmetic and its order are those of bamg_vcycle with one lane
 * per block row on every operator (bamg_bsr_set_lanes(.., 1)), so the
 * results then agree bit for bit; with other lane counts they differ only by
 * summation order.
 *
 * bamg_cg_solve_multi: k independent preconditioned CG recurrences (the
 * iterates of bamg_cg_solve on each column, up to the summation order of the
 * dot products) that share every pass over the operators: own step lengths,
 * stopping test ||b_j - A x_j|| <= rtol ||b_j|| and iteration count per
 * column; a column that stops is frozen while the others continue.  info
 * (host, k entries, may be NULL) receives each column's result.  Returns
 * BAMG_ERR_BREAKDOWN or BAMG_ERR_NOT_CONVERGED if any column did so (the
 * message names the first). */
BAMG_API bamg_status bamg_mg_vcycle_multi(bamg_mg* mg, const double* B, double* X, int k);
BAMG_API bamg_status bamg_cg_solve_multi(bamg_mg* mg, const double* B, double* X, int k, double rtol, int maxit,
                                         bamg_cg_info* info);
/* Per-block-row smoother weights of a level (device float array of the
 * level's block-row count, borrowed) scaling each row of the Chebyshev
 * update, i.e. the smoother is preconditioned by W D^-1; w = NULL restores
 * the plain smoother.  The eigen-estimate of W D^-1 A is refreshed by the
 * next bamg_mg_update. */
BAMG_API bamg_status bamg_mg_set_smoother_weights(bamg_mg* mg, int level, const float* w);
/* Thread mapping for every operator of the hierarchy (A, P and R = P^T of
 * each level, both precisions), replacing the autotuner's choices, so that
 * results no longer depend on timing: lanes = a power of two in 1..32 lanes
 * per block row, or 0 = component split for the 6x3 / 6x6-block operators
 * and one lane per row for the others (see bamg_bsr_set_lanes). */
BAMG_API bamg_status bamg_mg_set_lanes(bamg_mg* mg, int lanes);
/* Inspection: number of levels; a level's operator and prolongator (P is
 * NULL on the coarsest level); its eigen-estimate and prolongator damping
 * factor; its block-diagonal inverse (device, nbr row-major bs x bs blocks). */
BAMG_API bamg_status bamg_mg_num_levels(const bamg_mg* mg, int* n);
BAMG_API bamg_status bamg_mg_get_level(const bamg_mg* mg, int level, bamg_bsr** A, bamg_bsr** P);
/* The cached restriction R = P^T of a level (NULL on the coarsest level);
 * owned by the hierarchy, refreshed when P changes. */
BAMG_API bamg_status bamg_mg_get_restriction(const bamg_mg* mg, int level, bamg_bsr** R);
/* Aggregate of every block row of a non-coarsest level (the column of its
 * tentative-prolongator block), -1 for a row in no aggregate: nbr ints
 * into a caller-owned device array, on the context's stream. */
BAMG_API bamg_status bamg_mg_get_aggregates(const bamg_mg* mg, int level, int32_t* agg);
/* State gate (Sec. 3.5): how many times the level's prolongator-side caches
 * were rebuilt since setup: the block-ordered copy of P inside the level's
 * Galerkin plan (*p_refreshes) and R = P^T (*r_refreshes).  Both are
 * rebuilt only when P's version changed (cold setup or bamg_mg_resetup),
 * never by bamg_mg_update.  Host outputs; either may be NULL. */
BAMG_API bamg_status bamg_mg_get_gate_counts(const bamg_mg* mg, int level, uint64_t* p_refreshes,
                                             uint64_t* r_refreshes);
BAMG_API bamg_status bamg_mg_get_level_scalars(const bamg_mg* mg, int level, double* lambda_max,
                                      double* omega);
BAMG_API bamg_status bamg_mg_get_dinv(const bamg_mg* mg, int level, double* dinv);
BAMG_API bamg_status bamg_mg_destroy(bamg_mg* mg);

/* ------------------------------------------------- batch of problems */

/* A batch of independent problems, each with its own hierarchy, solved by
 * PCG in one graph launch (not in the paper: a serving-style extension).
 * The graph runs every problem's solve start, then a device-controlled
 * while loop whose body is one CG iteration of every problem still running
 * (a kernel at the end of each iteration sets the loop condition, bounded
 * at maxit iterations), then every problem's x and true residual; no
 * host round trip happens inside a solve.  Problems run as concurrent
 * branches of the graph, dealt largest-first to n_branches branches.  Each
 * problem executes exactly the kernels of bamg_cg_solve, so its result and
 * iteration count are those of a standalone solve.
 *
 * bamg_batch_create: mgs (host array of n hierarchies, borrowed; each set up
 * and updated) must each have their own context, since a context's
 * reduction buffers serve one solve at a time (BAMG_ERR_INVALID otherwise).
 * The batch launches on ctx's stream.  Branches default to n.
 * bamg_batch_cg_solve: b and x are host arrays of n device pointers (FP64
 * fine vectors; x entries may be NULL, x itself may be NULL).  The graph is
 * built on the first call and rebuilt when the pointers, rtol or maxit
 * change.  info (host, n entries, may be NULL), loops (may be NULL): loop
 * iterations run.  Returns BAMG_ERR_BREAKDOWN / BAMG_ERR_NOT_CONVERGED if
 * any problem did so (the message names the first).
 * bamg_batch_autotune: times one solve with 1, 2, 4, ... n branches (median
 * of three after a warm-up) and keeps the fastest; *best_ms (may be NULL)
 * receives its time.  Runs solves, so it overwrites the x vectors. */
typedef struct bamg_batch bamg_batch;
BAMG_API bamg_status bamg_batch_create(bamg_ctx* ctx, int n, bamg_mg* const* mgs, bamg_batch** out);
BAMG_API bamg_status bamg_batch_destroy(bamg_batch* bt);
BAMG_API bamg_status bamg_batch_set_branches(bamg_batch* bt, int n_branches);
BAMG_API bamg_status bamg_batch_get_branches(const bamg_batch* bt, int* n_branches);
BAMG_API bamg_status bamg_batch_cg_solve(bamg_batch* bt, const double* const* b, double* const* x, double rtol,
                                         int maxit, bamg_cg_info* info, int* loops);
BAMG_API bamg_status bamg_batch_autotune(bamg_batch* bt, const double* const* b, double* const* x, double rtol,
                                         int maxit, float* best_ms);

/* --------------------------------------------- learned smoother weights */

/* Per-block-row smoother weights predicted by a small MLP (not in the paper;
 * a learned extension of the point-block Jacobi / Chebyshev smoother): 8
 * features of each block row -> 64 -> 64 -> 1 (ReLU), weight
 * w = 0.5 + 1.5 sigmoid(z).  Parameters, inputs and hidden activations are
 * rounded to bfloat16, products accumulated in FP32 (FP32 master parameters,
 * Adam).  Parameter layout (floats): W1[8][64], b1[64], W2[64][64], b2[64],
 * w3[64], b3.  X is n x 8 row-major floats, t and w are n floats (device).
 * Training is deterministic (fixed-order gradient reductions). */
typedef struct bamg_mlp bamg_mlp;
BAMG_API bamg_status bamg_mlp_num_params(int* n);
/* He-uniform initial weights from splitmix64(seed); biases zero. */
BAMG_API bamg_status bamg_mlp_create(bamg_ctx* ctx, uint64_t seed, bamg_mlp** out);
BAMG_API bamg_status bamg_mlp_destroy(bamg_mlp* mlp);
BAMG_API bamg_status bamg_mlp_get_params(const bamg_mlp* mlp, float* params);
/* Replaces the parameters and resets the optimiser state. */
BAMG_API bamg_status bamg_mlp_set_params(bamg_mlp* mlp, const float* params);
BAMG_API bamg_status bamg_mlp_forward(bamg_mlp* mlp, const float* X, int64_t n, float* w);
/* Gradient of mean((w - t)^2) into grad (device, num_params floats; may be
 * NULL) and the loss into *loss (device float, may be NULL); w_tmp is an n-float
 * work array.  Grows the activation buffers on demand (allocates). */
BAMG_API bamg_status bamg_mlp_gradient(bamg_mlp* mlp, const float* X, const float* t, int64_t n, float* w_tmp,
                                       float* grad, float* loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr on the
 * batch (X, t); *loss (device, may be NULL) receives the batch loss before the step. */
BAMG_API bamg_status bamg_mlp_train_step(bamg_mlp* mlp, const float* X, const float* t, int64_t n, float* w_tmp,
                                         float lr, float* loss);
/* One epoch of mini-batch training (Adam after every batch, as
 * bamg_mlp_train_step): batch k takes rows perm[k * batch .. ] of X (n x 8)
 * and t (n), perm a device array of n int64 row indices (a permutation, or
 * any rows to train on, each < the rows of X), so the rows are gathered
 * inside the kernel.  *loss_sum (device double, caller-owned) is increased
 * by the epoch's summed squared error (divide by n for the mean).  Runs on
 * the context's stream without waiting for it. */
BAMG_API bamg_status bamg_mlp_train_epoch(bamg_mlp* mlp, const float* X, const float* t, const int64_t* perm,
                                          int64_t n, int64_t batch, float lr, double* loss_sum);
/* Features of the block rows of a non-coarsest level (n_l x 8, device):
 * log||A_ii||, sum_{j!=i}||A_ij||/||A_ii||, log(max/min nonzero block norm),
 * blocks/27, clamped-row flag, log sum_j||D_i^-1 A_ij||, level, 1. */
BAMG_API bamg_status bamg_mg_block_features(bamg_mg* mg, int level, float* X);
/* Training targets from the plain FP64 cycle: for the k right-hand sides B
 * (device, k consecutive fine vectors) the residual r after pre-smoothing on
 * every non-coarsest level gives, per block row, clip(sum <r_i, q_i> /
 * sum ||q_i||^2, 0.5, 2) with q = A D^-1 r; written level after level into
 * targets (device floats).  Allocates work arrays. */
BAMG_API bamg_status bamg_mg_smoother_targets(bamg_mg* mg, const double* B, int k, float* targets);
/* With an MLP attached, every bamg_mg_update predicts the weights of every
 * non-coarsest level from its features and estimates the Chebyshev interval
 * for W D^-1 A; a non-finite prediction falls back to weight 1.  NULL
 * detaches (plain smoother).  bamg_mg_set_smoother_weights also takes effect
 * at the next update. */
BAMG_API bamg_status bamg_mg_attach_mlp(bamg_mg* mg, bamg_mlp* mlp);
/* Stationary iteration x_{k+1} = x_k + M (b - A x_k) from x_0 = 0 for `its`
 * steps; rnorms (host, its + 1 doubles) receives ||b - A x_k||. */
BAMG_API bamg_status bamg_mg_stationary(bamg_mg* mg, const double* b, double* x, int its, double* rnorms);

#ifdef __cplusplus
}
#endif

#endif /* BAMG_H */
