// Internal declarations of libbamg: object layouts, the sliced block storage,
// status plumbing and the kernel launchers shared between translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "bamg.h"

namespace bamg {

// Rows per slice of the sliced block storage: one warp, one row per lane.
constexpr int kSlice = 32;
// Threads per CTA of the row kernels (4 slices).
constexpr int kRowThreads = 128;
// CTAs of the fixed-grid reductions (a multiple of the 152 SMs of a GB300).
constexpr int kRedBlocks = 608;
constexpr int kRedGridMax = 8192;  // CTAs of a reducing row kernel (one partial slot each)

// Grid of a one-wave reducing row kernel with 256-thread CTAs (deal_range):
// the SMs times the CTAs of `kernel` resident on one, all of
// them even when the rows would fit in fewer (the deal spreads the tasks
// over every CTA), but no more CTAs than warp tasks.
template <typename K>
inline unsigned deal_grid(K kernel, int sm_count, int64_t threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t cap = std::min<int64_t>((int64_t)sm_count * per_sm, kRedGridMax);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((threads + 31) / 32, cap));
}
constexpr int kRedThreads = 256;

struct Status {
  bamg_status code = BAMG_OK;
  std::string msg;
  bool ok() const { return code == BAMG_OK; }
};

// Kernel launch count (launches captured into a graph are counted when the
// graph is launched, by its kernel-node count).
extern std::atomic<unsigned long long> g_launches;
extern thread_local bool g_capturing;
inline void count_launch() {
  if (!g_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}

struct ProfPair {
  cudaEvent_t a = nullptr, b = nullptr;
  int slot = 0;
  int pos = 0;    // CG iteration position (graph-owned pairs)
  int count = 1;  // launches of the slot's kernel between a and b
};

struct Prof {
  bool on = false;
  unsigned mask = ~0u;  // slots that are timed while on
  uint64_t epoch = 0;
  std::vector<ProfPair> eager;
  size_t eager_used = 0;
  std::vector<ProfPair>* sink = nullptr;  // graph-owned pairs (created before capture)
  size_t sink_used = 0;
  int pos = 0;
  double ms[BAMG_PROF_COUNT] = {};
  int64_t n[BAMG_PROF_COUNT] = {};
};

}  // namespace bamg

#define BAMG_COUNT_LAUNCH ::bamg::count_launch()

struct bamg_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 0;
  std::string err;
  int* d_err = nullptr;            // device error word (first error code wins)
  double* d_partials = nullptr;    // kRedGridMax partial sums x 4 lanes
  unsigned* d_counters = nullptr;  // last-block counters (16 slots)
  int64_t wait_limit = int64_t(1) << 22;  // polls of a bounded device wait before it gives up
  bamg::Prof prof;
};

// Rectangular-block sparse matrix.  The pattern is kept in block-CSR form
// (rows sorted by column) and, for the kernels, in a sliced form: rows are
// grouped in slices of 32, each slice is padded to its longest row, and slot
// t of row lane l in slice s is chunk (slice_ptr[s] + t), lane l, i.e. slot
// index 32 * chunk + l.  Values live only in the sliced form, element e of a
// slot at vals[32 * B * chunk + 32 * e + l] (B = bs_r * bs_c), so the 32 rows
// of a slice read every element with one coalesced access.  Padding slots
// hold zero values and a valid column.
struct bamg_bsr {
  bamg_ctx* ctx = nullptr;
  int br = 0, bc = 0;
  int64_t nbr = 0, nbc = 0, nnzb = 0;
  bool has_pattern = false;
  bool symmetric = false;
  uint64_t version = 0;
  // block-CSR pattern (device + host copies)
  int* rowptr = nullptr;
  int* colidx = nullptr;
  std::vector<int> h_rowptr, h_colidx;
  // sliced form
  int64_t nslices = 0, nchunks = 0;
  int* slice_ptr = nullptr;  // nslices + 1, in chunks
  int* sell_col = nullptr;   // 32 * nchunks
  int* slot_of = nullptr;    // nnzb: CSR block -> slot
  int* diag_slot = nullptr;  // nbr (square blocks only, -1 if no diagonal block)
  int* slot_row = nullptr;   // sorted slices: block row of each of the 32 * nslices row positions
                             // (-1 = padding); null when row position = row
  bool all_diag = false;     // every block row has its diagonal block
  int vec = 1;               // lanes per block row of the FP64 row kernels (1..32, power of 2)
  int vec32 = 1;             // the same for kernels reading the FP32 copy
  int split = 0;             // 6-row blocks: 0 = lanes per row; 1, 2 or 4 = component split with
  int split32 = 0;           //   that many warps per component of a slice; 32, 64, 128 = one CTA per
                             //   row, split / 32 warps per component (FP64 / FP32 kernels)
  bool vec_tuned = false;
  std::vector<int> h_slice_ptr, h_slot_of;
  double* vals = nullptr;    // 32 * nchunks * B
  float* vals32 = nullptr;   // float copy in the same layout
  uint64_t vals32_version = ~0ull;
  bool vals64_stale = false; // an FP32 Galerkin product wrote only vals32
  uint64_t pattern_id = 0;   // changes whenever the pattern is rebuilt
  // blocked COO plan
  int64_t coo_n = 0;
  int* coo_perm = nullptr;   // contributions in (row, col, input order) order
  int* coo_seg = nullptr;    // nnzb + 1 offsets into coo_perm
  int* coo_slot = nullptr;   // per input entry: its block's slot, -1 if ignored (element-by-element path)
  int* coo_soff = nullptr;   // 32 * nchunks + 1: per storage slot (slice order), offset into coo_sperm
  int* coo_sperm = nullptr;  // the contributions of each slot, slots in slice order, each in input order
  int64_t block_elems() const { return (int64_t)br * bc; }
  int64_t nslots() const { return nchunks * bamg::kSlice; }
};

// Galerkin product plan (Sec. 3.1, Sec. 3.5).  Stage 1 forms the intermediate
// Z = A P block by block, stage 2 forms A_c = P^T Z; both gather, for each
// output block, a fixed list of input block pairs (built once by the symbolic
// phase), so the numeric phase has no atomics and a fixed summation order.
// Output blocks are processed in order of decreasing list length so the
// lane groups of a warp carry equal work.
struct bamg_ptap {
  bamg_ctx* ctx = nullptr;
  const bamg_bsr* A = nullptr;
  const bamg_bsr* P = nullptr;
  bamg_bsr* Ac = nullptr;
  uint64_t a_pid = 0, p_pid = 0, ac_pid = 0;
  int bs = 0, bsp = 0;
  bool symmetric = false;
  // intermediate pattern Z = A P (host)
  int64_t nz = 0;
  std::vector<int> h_zrowptr, h_zcol;
  // stage 1: items (Z blocks), their gather lists of (A slot, P block)
  int64_t n1 = 0, e1 = 0;
  int *s1_z = nullptr, *s1_off = nullptr, *s1_a = nullptr, *s1_p = nullptr;
  // stage 2: items (A_c blocks, upper triangle if symmetric), lists of (P block, Z block)
  int64_t n2 = 0, e2 = 0;
  int *s2_slot = nullptr, *s2_tslot = nullptr, *s2_off = nullptr, *s2_p = nullptr, *s2_z = nullptr;
  // work buffers and the state-gated prolongator-side cache (P in block order)
  double* Z = nullptr;
  float* Z32 = nullptr;
  double* Pblk = nullptr;
  float* Pblk32 = nullptr;
  uint64_t pblk_version = ~0ull, pblk32_version = ~0ull;
  uint64_t pblk_refreshes = 0;
  int prof_stage1 = -1, prof_stage2 = -1;  // profiling slots of the two stages (-1: none)
};

namespace bamg {

// Per-level device scalars (doubles): eigen-estimate, Chebyshev coefficients.
enum LevelScalar : int {
  kLam = 0,        // lambda_max estimate of D^-1 A
  kInvTheta = 1,   // 1 / theta
  kCheb = 2,       // (c1_k, c2_k) pairs for k = 0..degree-2 from here
  kScalarsPerLevel = 32
};

// Dense Cholesky data of the coarsest level: the factor's inverse W = L^-1
// (row-major, lower) and its transpose (row-major, upper), padded to a
// multiple of the 32-wide tiles with an identity block.
struct CoarseDense {
  int64_t n = 0, npad = 0;
  double* M = nullptr;   // npad x npad work array (factor, then W)
  double* Wt = nullptr;  // npad x npad transpose of W
  double* b64 = nullptr; // FP64 staging vectors (mixed form)
  double* x64 = nullptr;
  int* rows = nullptr;   // block row of every stored block of the coarsest operator
  double* dinv_tiles = nullptr;  // inverses of the 32x32 diagonal tiles of L
  bool factored = false;
  // Banded form (nc > 0): the padded matrix (npad = nc * s) split into chunks
  // of s rows is block tridiagonal, factored from both ends toward the middle
  // chunk t = nc / 2; per chunk k, s x s row-major:
  //   D[k]   A_kk, then its Schur complement, then the chunk's Cholesky factor
  //   Sub[k] A_{k+1,k};  Sup[k] A_{k,k+1}
  //   Bb[k]  B_k = A_{k+1,k} W_k^T (k < t) or C_k = A_{k-1,k} W_k^T (k > t)
  //   Wb[k]  W_k = inverse of the chunk's factor;  Wtb[k] its transpose
  //   Mb[k] = W_k B_{k-1} (1 <= k <= t);  Mtb[k] = W_k C_{k+1} (t <= k <= nc-2)
  //   Nb[k] = W_k^T B_k^T (k < t);        Ntb[k] = W_k^T C_k^T (k > t)
  int nc = 0, s = 0;
  double *D = nullptr, *Sub = nullptr, *Sup = nullptr, *Wb = nullptr, *Wtb = nullptr, *Bb = nullptr,
         *Mb = nullptr, *Nb = nullptr, *Mtb = nullptr, *Ntb = nullptr;
  double* gpart = nullptr;   // split-K partial tiles of the chunk products
  unsigned* gctr = nullptr;  // per-tile arrival counts of the split (zero between launches)
};

struct Level {
  bamg_bsr* A = nullptr;     // operator (level 0 is borrowed from the caller)
  bool own_A = false;
  bamg_bsr* P = nullptr;     // prolongator from the next level
  bamg_bsr* R = nullptr;     // R = P^T (cached, rebuilt when P's version changes)
  int* rmap = nullptr;       // R block -> P block (pattern order)
  uint64_t r_version = ~0ull;
  uint64_t r_refreshes = 0;  // rebuilds of R (state gate)
  bamg_ptap* plan = nullptr; // Galerkin plan A, P -> next level's A
  int bs = 0;
  int64_t n = 0;             // block rows
  double omega = 0.0;        // prolongator damping used at setup
  double* dinv = nullptr;    // block-diagonal inverse, slice-interleaved
  float* dinv32 = nullptr;
  float* weights = nullptr;  // per-block-row smoother weights (borrowed or learned_w), or null
  float* feat = nullptr;     // block features (learned weights)
  float* learned_w = nullptr;
  // prolongator smoothing data, kept for bamg_mg_resetup
  bamg_bsr* Pt = nullptr;    // tentative prolongator (geometry only)
  bamg_ptap* ap = nullptr;   // plan of A P~ (stage 1 only)
  int* zrow = nullptr;       // block row of each block of A P~
  int* agg = nullptr;        // aggregate of each node
  double* q = nullptr;       // P~ blocks, node-major
  // vectors (FP64 and FP32 forms): right-hand side, iterate, residual, directions
  double *b = nullptr, *x = nullptr, *r = nullptr, *d0 = nullptr, *d1 = nullptr;
  float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *d032 = nullptr, *d132 = nullptr;
};

struct CgState {
  double bnorm2, rtol2, rz, pq, alpha, beta, rnorm2, pad;
  int its, maxit, done, converged, breakdown, loops, pad2[2];  // loops: bodies run by the device loop
};

// Many right-hand sides at once: at most kMaxRhs vectors, stored RHS-minor
// and padded to kp = a power of two >= 4 columns.
constexpr int kMaxRhs = 32;

// Per-column state of k simultaneous PCG recurrences.
struct CgMultiState {
  double bnorm2[kMaxRhs], rnorm2[kMaxRhs], rz[kMaxRhs], alpha[kMaxRhs], beta[kMaxRhs], pq[kMaxRhs];
  double true_r2[kMaxRhs];
  double rtol2;
  int its[kMaxRhs], done[kMaxRhs], converged[kMaxRhs], breakdown[kMaxRhs];
  int maxit, k, kp, all_done;
};

// Work area of the multi-right-hand-side V-cycle and CG (allocated on first
// use for a column count, grown on demand).
struct MultiLevel {
  void *b = nullptr, *x = nullptr, *r = nullptr, *d0 = nullptr, *d1 = nullptr;
};
struct MultiWork {
  int kp = 0;
  std::vector<MultiLevel> lv;
  double* coarse_y = nullptr;  // 2 x npad x kp, FP64 (coarsest-solve work)
  double *cx = nullptr, *cr = nullptr, *cz = nullptr, *cp = nullptr, *cq = nullptr, *czold = nullptr;
  bool own_rz = false;         // cr / cz allocated (mixed form) or aliased to level 0 (FP64)
  CgMultiState* st = nullptr;
  CgMultiState* host = nullptr;  // pinned
  double* partials = nullptr;    // grid x 64
  unsigned* counters = nullptr;  // 8
  cudaGraphExec_t graph = nullptr;  // one CG iteration for graph_kp columns
  uint64_t graph_kernels = 0;
  int graph_kp = 0;
};

}  // namespace bamg

struct bamg_mlp;

struct bamg_mg {
  bamg_ctx* ctx = nullptr;
  bamg_mlp* mlp = nullptr;           // attached weight predictor (borrowed), or null
  bamg_mg_opts opts{};
  std::vector<bamg::Level> levels;
  double* scal = nullptr;            // levels x kScalarsPerLevel device scalars
  int scal_blocks_minus1 = 0;        // index of the spare block of scalars
  bamg::CoarseDense coarse;
  // CG work vectors (fine level, FP64) and state
  double *cx = nullptr, *cr = nullptr, *cp = nullptr, *cq = nullptr, *cz = nullptr, *czold = nullptr;
  bamg::CgState* cg = nullptr;
  bamg::CgState* cg_host = nullptr;  // pinned
  std::vector<cudaGraphExec_t> cg_graphs;  // one, or one per iteration position when profiling
  std::vector<std::vector<bamg::ProfPair>> cg_pairs;
  std::vector<size_t> cg_pairs_used;
  uint64_t cg_graph_epoch = ~0ull;
  uint64_t cg_graph_kernels = 0;
  // unprofiled solves: one graph whose while node runs the iterations on the
  // device (no host round trip until the solve ends)
  cudaGraphExec_t cg_loop = nullptr;
  uint64_t cg_loop_body_kernels = 0;
  double* power_w[2] = {nullptr, nullptr};
  bamg::MultiWork* multi = nullptr;  // multi-right-hand-side work area
  // second stream of the reuse update: the coarsest factorisation runs on it,
  // forked after the last Galerkin product, joined before the update returns
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // mixed form: the finest level's (FP64) smoother refresh runs on a third
  // stream under the FP32 Galerkin products
  cudaStream_t side0 = nullptr;
  cudaEvent_t ev_join0 = nullptr;
};

namespace bamg {

// ------------------------------------------------------------ status helpers
Status make_status(bamg_status code, const char* fmt, ...);
bamg_status fail(bamg_ctx* ctx, const Status& s);
Status cuda_status(cudaError_t e, const char* what);
#define BAMG_CUDA(call)                                          \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return ::bamg::cuda_status(e_, #call); \
  } while (0)
#define BAMG_TRY(expr)                   \
  do {                                   \
    ::bamg::Status s_ = (expr);          \
    if (!s_.ok()) return s_;             \
  } while (0)

template <typename T>
Status dalloc(T** p, int64_t n, cudaStream_t st) {
  *p = nullptr;
  if (n <= 0) return Status{};
  cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * (size_t)n, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return make_status(BAMG_ERR_OOM, "device allocation of %lld bytes failed: %s",
                       (long long)(sizeof(T) * (size_t)n), cudaGetErrorString(e));
  }
  return Status{};
}
template <typename T>
void dfree(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
}
template <typename T>
Status upload(T** dst, const std::vector<T>& src, cudaStream_t st) {
  BAMG_TRY(dalloc(dst, (int64_t)src.size(), st));
  if (!src.empty())
    BAMG_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st));
  return Status{};
}
template <typename T>
Status download(std::vector<T>& dst, const T* src, int64_t n, cudaStream_t st) {
  dst.resize((size_t)n);
  if (n > 0) BAMG_CUDA(cudaMemcpyAsync(dst.data(), src, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, st));
  BAMG_CUDA(cudaStreamSynchronize(st));
  return Status{};
}

// Device error codes written into ctx->d_err.
enum DevErr : int { kDevOk = 0, kDevNaN = 1, kDevBreakdown = 2, kDevTimeout = 3, kDevIndex = 4 };
Status check_device_error(bamg_ctx* ctx);  // synchronizes the stream

// Profiling marks (no-ops when profiling is off).  Return / take an index.
// Brackets `count` consecutive launches of the slot's kernel (back-to-back
// launches of one kernel share a bracket: each bracket costs the kernels it
// encloses their programmatic overlap with their neighbours).
int prof_begin(bamg_ctx* ctx, int slot, cudaStream_t st, int count = 1);
void prof_end(bamg_ctx* ctx, int idx, cudaStream_t st);
void prof_harvest(bamg_ctx* ctx, std::vector<ProfPair>& pairs, size_t count, int active_ap, int active_vc);

// ------------------------------------------------------------ pattern helpers
// Build the sliced form (and device/host CSR copies) from a host CSR pattern;
// allocates zeroed values.  Used by COO preallocation and the Galerkin symbolic.
// sort_rows: place the rows in the slices by decreasing length within
// windows of 1,024 rows (sliced ELL with sorting), so that rows of equal
// length share slices and little padding is stored; kernels then map each
// row position to its row through slot_row.
// Row order of the sliced storage: identity, rows sorted by decreasing length
// within windows of 1,024 rows (slot_row maps positions to rows), or sorted
// only where that removes at least a tenth of the stored slots.
constexpr int kSortNever = 0, kSortAlways = 1, kSortAuto = 2;
Status bsr_set_pattern(bamg_bsr* A, std::vector<int>&& rowptr, std::vector<int>&& colidx, int sort_rows = kSortNever);
Status bsr_ensure_fp32(bamg_bsr* A);   // refresh vals32 if the version changed
void bsr_release(bamg_bsr* A);

// Galerkin plan construction; with want_ac = false only stage 1 (Z = A P) is
// planned (used by prolongator smoothing).
Status ptap_build(bamg_bsr* A, bamg_bsr* P, bool want_ac, bamg_ptap** plan, bamg_bsr** Ac);
Status ptap_run(bamg_ptap* plan, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac, bamg_prec prec, bool stage2);
void ptap_release(bamg_ptap* plan);
// Copy sliced values to block (pattern) order.
Status launch_gather_blocks(const bamg_bsr* A, const double* vals, double* out, cudaStream_t st);

// Hierarchy internals shared by the setup, cycle and coarse-solver units.
Status mg_refresh_level(bamg_mg* mg, int l, cudaStream_t st);        // Dinv, eigen-estimate, Chebyshev coefficients
Status mg_refresh_restriction(bamg_mg* mg, int l, cudaStream_t st);  // state-gated R = P^T
Status coarse_factor(bamg_mg* mg, cudaStream_t st);                      // dense Cholesky + inverse of the coarsest level
template <typename T>
Status coarse_apply(bamg_mg* mg, const T* b, T* x, const int* done, cudaStream_t st);
// The same solve for kp vectors stored RHS-minor (b, x: n x kp); work holds
// 2 * npad * kp doubles.
template <typename T>
Status coarse_apply_multi(bamg_mg* mg, int kp, const T* b, T* x, double* work, const int* done, cudaStream_t st);
template <typename T>
// levels[0].b(32) -> levels[0].x(32); with b64 / x64 (finest level of 3x3
// blocks, degree >= 2) the FP64 input is read and the FP64 result written by
// the finest level's first and last kernels.
Status vcycle_on(bamg_mg* mg, const int* done, cudaStream_t st, const double* b64 = nullptr, double* x64 = nullptr);
Status power_lambda(bamg_mg* mg, int l, bool scalar_diag, double* out_scalar_slot, cudaStream_t st);
void mg_release_graphs(bamg_mg* mg);
void mg_release_multi(bamg_mg* mg);               // multi-right-hand-side work area
Status mg_learned_weights(bamg_mg* mg, int l, cudaStream_t st);  // features -> MLP -> level weights
Status mg_smooth_down_fp64(bamg_mg* mg, int l, cudaStream_t st);  // FP64 pre-smoothing of level l (b -> x, r)
Status mg_restrict_fp64(bamg_mg* mg, int l, cudaStream_t st);     // levels[l+1].b = R_l r_l
Status mg_precond(bamg_mg* mg, const double* r, double* z, cudaStream_t st);  // one V-cycle
Status mg_tune_smoothers(bamg_mg* mg);
// Block strength graph (see bamg_strength_graph) into device rowptr / col.
Status strength_graph(bamg_bsr* A, double eps, int* rowptr, int* col, int64_t cap, int64_t* nedges);
// Device MIS aggregation of a CSR graph (see bamg_mis_aggregate); root_vertex
// (device, optional) receives the root vertex of every aggregate.
Status mis_aggregate(bamg_ctx* ctx, int64_t n, const int* rp, const int* col, uint64_t seed, int* agg,
                     int64_t* n_agg, int* rounds, int* root_vertex);  // warps per component of the coarse smoothers, by timing them
// The phases of one PCG solve on stream st (the batch solver captures them):
// setup, r = b, z = M r, p = z; one iteration (every kernel returns at once
// when the solve is done); x = the iterate, ||b - A x||^2 into *true_r2.
Status cg_prologue(bamg_mg* mg, const double* b, double rtol, int maxit, cudaStream_t st);
Status cg_step(bamg_mg* mg, cudaStream_t st);
Status cg_epilogue(bamg_mg* mg, const double* b, double* x, double* true_r2, cudaStream_t st);

// ------------------------------------------------------------ kernel launchers
// y = A x (row-block product) in precision T (double or float); x, y device.
template <typename T>
Status launch_spmv(const bamg_bsr* A, const T* vals, const T* x, T* y, cudaStream_t st);
template <typename T>
Status launch_spmm(const bamg_bsr* A, const T* vals, const T* X, T* Y, int k, cudaStream_t st);
// Convert a sliced value array to float.
Status launch_to_fp32(const double* src, float* dst, int64_t n, cudaStream_t st);
// Lanes-per-row choice: a size heuristic, and the measured choice (times the
// FP64 product for every width and keeps the fastest).
int default_vec(const bamg_bsr* A);
Status bsr_autotune(bamg_bsr* A, float* best_ms);
inline int64_t row_threads(const bamg_bsr* A) { return A->nslices * kSlice * (int64_t)A->vec; }
template <typename T>
inline int lanes_for(const bamg_bsr* A) {
  return sizeof(T) == 4 ? A->vec32 : A->vec;
}
template <typename T>
inline int split_for(const bamg_bsr* A) {
  return sizeof(T) == 4 ? A->split32 : A->split;
}
// Split codes 32, 64 and 128: the row form (one CTA per row, split / 32 warps
// per output component).
constexpr int kSplitRows = 32;
#define BAMG_DISPATCH_ROWS(s, ...)                          \
  switch (s) {                                             \
    case 128: { constexpr int VR = 4; __VA_ARGS__; } break; \
    case 64: { constexpr int VR = 2; __VA_ARGS__; } break;  \
    default: { constexpr int VR = 1; __VA_ARGS__; } break;  \
  }
// Split codes 256 + VB (VB = 2, 4, 8, 16, 32): the all-component block
// split (row_blocks_split) for 6x3 blocks (the finest restriction), VB warps
// per slice.
constexpr int kSplitBlocks = 256;
inline bool is_block_split(int s) {
  return s == kSplitBlocks + 2 || s == kSplitBlocks + 4 || s == kSplitBlocks + 8 || s == kSplitBlocks + 16 ||
         s == kSplitBlocks + 32;
}
#define BAMG_DISPATCH_VB(s, ...)                            \
  switch (s) {                                             \
    case kSplitBlocks + 32: { constexpr int VB = 32; __VA_ARGS__; } break; \
    case kSplitBlocks + 16: { constexpr int VB = 16; __VA_ARGS__; } break; \
    case kSplitBlocks + 8: { constexpr int VB = 8; __VA_ARGS__; } break; \
    case kSplitBlocks + 4: { constexpr int VB = 4; __VA_ARGS__; } break; \
    default: { constexpr int VB = 2; __VA_ARGS__; } break;  \
  }
// Run `body` with the compile-time warps per component VS matching s (1, 2 or 4).
#define BAMG_DISPATCH_VS(s, ...)                            \
  switch (s) {                                             \
    case 4: { constexpr int VS = 4; __VA_ARGS__; } break;   \
    case 2: { constexpr int VS = 2; __VA_ARGS__; } break;   \
    default: { constexpr int VS = 1; __VA_ARGS__; } break;  \
  }
template <typename T>
inline int64_t row_threads_for(const bamg_bsr* A) {
  return A->nslices * kSlice * (int64_t)lanes_for<T>(A);
}

}  // namespace bamg
