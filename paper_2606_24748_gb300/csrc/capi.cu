// C ABI: contexts, block matrices, errors, blocked SpMV / SpMM entry points.
#include <algorithm>
#include <cstdarg>
#include <new>

#include "device.cuh"
#include "internal.h"

namespace bamg {

std::atomic<unsigned long long> g_launches{0};
thread_local bool g_capturing = false;

static ProfPair* prof_slot_pair(bamg_ctx* ctx, int* idx) {
  Prof& p = ctx->prof;
  if (p.sink) {  // no event creation while a stream is being captured
    if (p.sink_used >= p.sink->size()) return nullptr;
    *idx = (int)p.sink_used++;
    return &(*p.sink)[*idx];
  }
  if (p.eager_used >= p.eager.size()) {
    ProfPair q;
    if (cudaEventCreate(&q.a) != cudaSuccess || cudaEventCreate(&q.b) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    p.eager.push_back(q);
  }
  *idx = (int)p.eager_used++;
  return &p.eager[*idx];
}

static cudaError_t record(cudaEvent_t e, cudaStream_t st) {
  return g_capturing ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
}

int prof_begin(bamg_ctx* ctx, int slot, cudaStream_t st, int count) {
  if (!ctx || !ctx->prof.on || slot < 0 || !((ctx->prof.mask >> slot) & 1u)) return -1;
  int idx = -1;
  ProfPair* q = prof_slot_pair(ctx, &idx);
  if (!q) return -1;
  q->slot = slot;
  q->pos = ctx->prof.pos;
  q->count = count;
  if (record(q->a, st) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return idx;
}

void prof_end(bamg_ctx* ctx, int idx, cudaStream_t st) {
  if (idx < 0 || !ctx->prof.on) return;
  Prof& p = ctx->prof;
  std::vector<ProfPair>& v = p.sink ? *p.sink : p.eager;
  if (record(v[idx].b, st) != cudaSuccess) cudaGetLastError();
}

// Accumulate the first `count` pairs.  Graph-owned pairs carry the CG
// iteration position: the A p product ran in positions < active_ap, the
// preconditioner in positions < active_vc (later launches returned at once).
void prof_harvest(bamg_ctx* ctx, std::vector<ProfPair>& pairs, size_t count, int active_ap, int active_vc) {
  Prof& p = ctx->prof;
  for (size_t i = 0; i < count && i < pairs.size(); ++i) {
    const ProfPair& q = pairs[i];
    if (active_ap >= 0) {
      const int lim = (q.slot == BAMG_PROF_CG_AP || q.slot == BAMG_PROF_CG_XR) ? active_ap : active_vc;
      if (q.pos >= lim) continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      p.ms[q.slot] += ms;
      p.n[q.slot] += q.count;
    } else {
      cudaGetLastError();
    }
  }
}

Status make_status(bamg_status code, const char* fmt, ...) {
  Status s;
  s.code = code;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  s.msg = buf;
  return s;
}

Status cuda_status(cudaError_t e, const char* what) {
  cudaGetLastError();
  return make_status(e == cudaErrorMemoryAllocation ? BAMG_ERR_OOM : BAMG_ERR_CUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

bamg_status fail(bamg_ctx* ctx, const Status& s) {
  if (ctx) ctx->err = s.msg;
  return s.code;
}

Status check_device_error(bamg_ctx* ctx) {
  int h = 0;
  BAMG_CUDA(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  BAMG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (h == kDevOk) return Status{};
  BAMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  switch (h) {
    case kDevNaN: return make_status(BAMG_ERR_NAN, "a non-finite value was produced on the device");
    case kDevBreakdown: return make_status(BAMG_ERR_BREAKDOWN, "breakdown: a matrix that must be SPD is not");
    case kDevTimeout: return make_status(BAMG_ERR_TIMEOUT, "a bounded device wait ran out");
    case kDevIndex: return make_status(BAMG_ERR_INVALID, "an index was out of range");
    default: return make_status(BAMG_ERR_CUDA, "unknown device error %d", h);
  }
}

void bsr_release(bamg_bsr* A) {
  cudaStream_t st = A->ctx->stream;
  dfree(A->rowptr, st);
  dfree(A->colidx, st);
  dfree(A->slice_ptr, st);
  dfree(A->sell_col, st);
  dfree(A->slot_of, st);
  dfree(A->diag_slot, st);
  dfree(A->slot_row, st);
  dfree(A->vals, st);
  dfree(A->vals32, st);
  dfree(A->coo_perm, st);
  dfree(A->coo_seg, st);
  dfree(A->coo_slot, st);
  dfree(A->coo_soff, st);
  dfree(A->coo_sperm, st);
  A->has_pattern = false;
  A->nnzb = 0;
  A->nslices = A->nchunks = 0;
  A->coo_n = 0;
  A->h_rowptr.clear();
  A->h_colidx.clear();
  A->h_slice_ptr.clear();
  A->h_slot_of.clear();
}

Status bsr_set_pattern(bamg_bsr* A, std::vector<int>&& rowptr, std::vector<int>&& colidx, int sort_rows) {
  cudaStream_t st = A->ctx->stream;
  const int64_t nbr = A->nbr;
  if ((int64_t)rowptr.size() != nbr + 1) return make_status(BAMG_ERR_INVALID, "rowptr size");
  A->nnzb = rowptr[nbr];
  A->nslices = (nbr + kSlice - 1) / kSlice;
  // row of each row position (identity, or sorted by decreasing length within
  // windows of 1,024 rows; padding positions past nbr stay at the end)
  std::vector<int> order((size_t)A->nslices * kSlice);
  for (size_t r = 0; r < order.size(); ++r) order[r] = (int64_t)r < nbr ? (int)r : -1;
  auto len = [&](int i) { return i < 0 ? -1 : rowptr[i + 1] - rowptr[i]; };
  auto stored_chunks = [&](const std::vector<int>& ord) {
    int64_t c = 0;
    for (int64_t s = 0; s < A->nslices; ++s) {
      int w = 0;
      for (int64_t r = s * kSlice; r < (s + 1) * kSlice; ++r) w = std::max(w, len(ord[r]));
      c += w;
    }
    return c;
  };
  if (sort_rows != kSortNever) {
    std::vector<int> sorted = order;
    constexpr size_t kWindow = 1024;
    for (size_t w0 = 0; w0 < sorted.size(); w0 += kWindow) {
      const size_t w1 = std::min(sorted.size(), w0 + kWindow);
      std::stable_sort(sorted.begin() + w0, sorted.begin() + w1, [&](int a, int b) { return len(a) > len(b); });
    }
    // auto: only where the sort removes a tenth of the stored slots or more
    // (rows of very uneven length, e.g. Q2 vertex and mid-edge nodes); evenly
    // filled slices keep the identity order and its contiguous vectors
    if (sort_rows == kSortAlways || 10 * stored_chunks(sorted) <= 9 * stored_chunks(order)) {
      order = std::move(sorted);
    } else {
      sort_rows = kSortNever;
    }
  }
  std::vector<int> sp(A->nslices + 1, 0);
  for (int64_t s = 0; s < A->nslices; ++s) {
    int w = 0;
    for (int64_t r = s * kSlice; r < (s + 1) * kSlice; ++r) w = std::max(w, len(order[r]));
    sp[s + 1] = sp[s] + w;
  }
  A->nchunks = sp[A->nslices];
  if (A->nchunks * (int64_t)kSlice >= (int64_t)INT32_MAX)
    return make_status(BAMG_ERR_INVALID, "matrix too large for int32 slots");
  std::vector<int> scol((size_t)A->nchunks * kSlice, 0);
  std::vector<int> slot_of((size_t)A->nnzb);
  std::vector<int> diag(A->br == A->bc ? (size_t)nbr : 0, -1);
  for (int64_t r = 0; r < (int64_t)order.size(); ++r) {
    const int i = order[r];
    if (i < 0) continue;
    const int64_t s = r / kSlice, l = r % kSlice;
    const int n_i = rowptr[i + 1] - rowptr[i];
    const int w = sp[s + 1] - sp[s];
    const int pad_col = n_i > 0 ? colidx[rowptr[i + 1] - 1] : 0;
    for (int t = 0; t < w; ++t) {
      const int64_t slot = (int64_t)(sp[s] + t) * kSlice + l;
      if (t < n_i) {
        const int k = rowptr[i] + t;
        scol[slot] = colidx[k];
        slot_of[k] = (int)slot;
        if (!diag.empty() && colidx[k] == i) diag[i] = (int)slot;
      } else {
        scol[slot] = pad_col;
      }
    }
  }
  A->h_rowptr = std::move(rowptr);
  A->h_colidx = std::move(colidx);
  A->h_slice_ptr = sp;
  A->h_slot_of = slot_of;
  dfree(A->rowptr, st);
  dfree(A->colidx, st);
  dfree(A->slice_ptr, st);
  dfree(A->sell_col, st);
  dfree(A->slot_of, st);
  dfree(A->diag_slot, st);
  dfree(A->slot_row, st);
  dfree(A->vals, st);
  dfree(A->vals32, st);
  if (sort_rows != kSortNever) BAMG_TRY(upload(&A->slot_row, order, st));
  BAMG_TRY(upload(&A->rowptr, A->h_rowptr, st));
  BAMG_TRY(upload(&A->colidx, A->h_colidx, st));
  BAMG_TRY(upload(&A->slice_ptr, sp, st));
  BAMG_TRY(upload(&A->sell_col, scol, st));
  BAMG_TRY(upload(&A->slot_of, slot_of, st));
  if (!diag.empty()) BAMG_TRY(upload(&A->diag_slot, diag, st));
  A->all_diag = !diag.empty() && std::find(diag.begin(), diag.end(), -1) == diag.end();
  const int64_t nv = A->nslots() * A->block_elems();
  BAMG_TRY(dalloc(&A->vals, nv, st));
  if (nv > 0) BAMG_CUDA(cudaMemsetAsync(A->vals, 0, sizeof(double) * nv, st));
  A->vals32_version = ~0ull;
  A->vals64_stale = false;
  A->has_pattern = true;
  A->vec = A->vec32 = default_vec(A);
  A->vec_tuned = false;
  A->version++;
  static uint64_t next_pattern_id = 0;
  A->pattern_id = ++next_pattern_id;
  // keep the host vectors alive until the uploads have been read
  BAMG_CUDA(cudaStreamSynchronize(st));
  return Status{};
}

Status bsr_ensure_fp32(bamg_bsr* A) {
  if (!A->has_pattern) return make_status(BAMG_ERR_STATE, "matrix has no pattern");
  if (A->vals32 && A->vals32_version == A->version) return Status{};
  if (A->vals64_stale) return make_status(BAMG_ERR_STATE, "float copy lost while FP64 values are stale");
  const int64_t nv = A->nslots() * A->block_elems();
  if (!A->vals32) BAMG_TRY(dalloc(&A->vals32, nv, A->ctx->stream));
  BAMG_TRY(launch_to_fp32(A->vals, A->vals32, nv, A->ctx->stream));
  A->vals32_version = A->version;
  return Status{};
}

__global__ void k_to_fp32(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (float)s[i];
}

Status launch_to_fp32(const double* src, float* dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return Status{};
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  { k_to_fp32<<<(unsigned)blocks, 256, 0, st>>>(src, dst, n); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

__global__ void k_get_values_any(const int* __restrict__ slot_of, const double* __restrict__ vals,
                                 double* __restrict__ out, int64_t nnzb, int B) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * B) return;
  const int64_t k = t / B;
  const int e = (int)(t % B);
  const int64_t slot = slot_of[k];
  out[t] = vals[(slot >> 5) * (32LL * B) + 32LL * e + (slot & 31)];
}

Status launch_gather_blocks(const bamg_bsr* A, const double* vals, double* out, cudaStream_t st) {
  const int B = (int)A->block_elems();
  const int64_t n = A->nnzb * B;
  if (n == 0) return Status{};
  { k_get_values_any<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A->slot_of, vals, out, A->nnzb, B); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_ctx_create(void* cuda_stream, bamg_ctx** out) {
  if (!out) return BAMG_ERR_INVALID;
  *out = nullptr;
  bamg_ctx* c = new (std::nothrow) bamg_ctx();
  if (!c) return BAMG_ERR_OOM;
  c->stream = (cudaStream_t)cuda_stream;
  auto body = [&]() -> Status {
    BAMG_CUDA(cudaGetDevice(&c->device));
    BAMG_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    BAMG_TRY(dalloc(&c->d_err, 1, c->stream));
    BAMG_TRY(dalloc(&c->d_partials, kRedGridMax * 4, c->stream));
    BAMG_TRY(dalloc(&c->d_counters, 64, c->stream));
    BAMG_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    BAMG_CUDA(cudaMemsetAsync(c->d_counters, 0, 64 * sizeof(unsigned), c->stream));
    BAMG_CUDA(cudaStreamSynchronize(c->stream));
    return Status{};
  };
  Status s = body();
  if (!s.ok()) {
    fprintf(stderr, "bamg_ctx_create: %s\n", s.msg.c_str());
    delete c;
    return s.code;
  }
  *out = c;
  return BAMG_OK;
}

bamg_status bamg_ctx_destroy(bamg_ctx* c) {
  if (!c) return BAMG_OK;
  for (auto& q : c->prof.eager) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  dfree(c->d_err, c->stream);
  dfree(c->d_partials, c->stream);
  dfree(c->d_counters, c->stream);
  cudaStreamSynchronize(c->stream);
  delete c;
  return BAMG_OK;
}

const char* bamg_last_error(const bamg_ctx* c) { return c ? c->err.c_str() : "null context"; }

bamg_status bamg_ctx_set_wait_limit(bamg_ctx* c, int64_t polls) {
  if (!c || polls < 0) return BAMG_ERR_INVALID;
  c->wait_limit = polls;
  return BAMG_OK;
}

bamg_status bamg_ctx_profile(bamg_ctx* c, int enable) {
  return bamg_ctx_profile_slots(c, enable ? ~(1u << BAMG_PROF_CHEB_PRE_L0) : 0u);
}

bamg_status bamg_ctx_profile_slots(bamg_ctx* c, unsigned mask) {
  if (!c) return BAMG_ERR_INVALID;
  Prof& p = c->prof;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, cuda_status(cudaGetLastError(), "profile"));
  // graphs captured under another mask hold other event nodes: re-capture
  // only when the mask changes (re-enabling the same slots just resets)
  if ((mask != 0) != p.on || mask != p.mask) p.epoch++;
  p.on = mask != 0;
  p.mask = mask;
  p.eager_used = 0;
  for (int k = 0; k < BAMG_PROF_COUNT; ++k) {
    p.ms[k] = 0.0;
    p.n[k] = 0;
  }
  return BAMG_OK;
}

bamg_status bamg_ctx_profile_read(bamg_ctx* c, int slot, double* total_ms, int64_t* launches) {
  if (!c || slot < 0 || slot >= BAMG_PROF_COUNT) return BAMG_ERR_INVALID;
  Prof& p = c->prof;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, cuda_status(cudaGetLastError(), "profile"));
  prof_harvest(c, p.eager, p.eager_used, -1, -1);
  p.eager_used = 0;
  if (total_ms) *total_ms = p.ms[slot];
  if (launches) *launches = p.n[slot];
  return BAMG_OK;
}

uint64_t bamg_kernel_launches(void) { return g_launches.load(); }

bamg_status bamg_device_memory(bamg_ctx* c, uint64_t* in_use, uint64_t* peak, int reset_peak) {
  if (!c) return BAMG_ERR_INVALID;
  cudaMemPool_t pool;
  uint64_t used = 0, high = 0;  // the attributes are 64-bit counts
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high) != cudaSuccess)
    return fail(c, cuda_status(cudaGetLastError(), "memory pool attributes"));
  if (in_use) *in_use = (uint64_t)used;
  if (peak) *peak = (uint64_t)high;
  if (reset_peak) {
    uint64_t zero = 0;  // the pool restarts the mark at the current use
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess)
      return fail(c, cuda_status(cudaGetLastError(), "memory pool reset"));
  }
  return BAMG_OK;
}

bamg_status bamg_ctx_sync(bamg_ctx* c) {
  if (!c) return BAMG_ERR_INVALID;
  Status s = check_device_error(c);
  return s.ok() ? BAMG_OK : fail(c, s);
}

bamg_status bamg_bsr_create(bamg_ctx* ctx, int bs_r, int bs_c, int64_t nbr, int64_t nbc, bamg_bsr** out) {
  if (!ctx || !out) return BAMG_ERR_INVALID;
  *out = nullptr;
  if (bs_r < 1 || bs_r > 8 || bs_c < 1 || bs_c > 8 || nbr < 0 || nbc < 0 || nbr >= INT32_MAX ||
      nbc >= INT32_MAX)
    return fail(ctx, make_status(BAMG_ERR_INVALID, "bamg_bsr_create: bad sizes bs=%dx%d n=%lldx%lld", bs_r,
                                 bs_c, (long long)nbr, (long long)nbc));
  bamg_bsr* A = new (std::nothrow) bamg_bsr();
  if (!A) return BAMG_ERR_OOM;
  A->ctx = ctx;
  A->br = bs_r;
  A->bc = bs_c;
  A->nbr = nbr;
  A->nbc = nbc;
  *out = A;
  return BAMG_OK;
}

bamg_status bamg_bsr_destroy(bamg_bsr* A) {
  if (!A) return BAMG_OK;
  bsr_release(A);
  delete A;
  return BAMG_OK;
}

bamg_status bamg_bsr_info(const bamg_bsr* A, int* bs_r, int* bs_c, int64_t* nbr, int64_t* nbc, int64_t* nnzb,
                          uint64_t* version) {
  if (!A) return BAMG_ERR_INVALID;
  if (bs_r) *bs_r = A->br;
  if (bs_c) *bs_c = A->bc;
  if (nbr) *nbr = A->nbr;
  if (nbc) *nbc = A->nbc;
  if (nnzb) *nnzb = A->nnzb;
  if (version) *version = A->version;
  return BAMG_OK;
}

bamg_status bamg_bsr_storage(const bamg_bsr* A, int64_t* stored_slots, int* rows_sorted) {
  if (!A) return BAMG_ERR_INVALID;
  if (!A->has_pattern) return BAMG_ERR_STATE;
  if (stored_slots) *stored_slots = A->nchunks * (int64_t)kSlice;
  if (rows_sorted) *rows_sorted = A->slot_row ? 1 : 0;
  return BAMG_OK;
}

bamg_status bamg_bsr_get_pattern(const bamg_bsr* A, int32_t* rowptr, int32_t* colidx) {
  if (!A) return BAMG_ERR_INVALID;
  bamg_ctx* ctx = A->ctx;
  if (!A->has_pattern) return fail(ctx, make_status(BAMG_ERR_STATE, "matrix has no pattern"));
  auto body = [&]() -> Status {
    if (rowptr)
      BAMG_CUDA(cudaMemcpyAsync(rowptr, A->rowptr, sizeof(int) * (A->nbr + 1), cudaMemcpyDeviceToDevice, ctx->stream));
    if (colidx && A->nnzb)
      BAMG_CUDA(cudaMemcpyAsync(colidx, A->colidx, sizeof(int) * A->nnzb, cudaMemcpyDeviceToDevice, ctx->stream));
    return Status{};
  };
  Status s = body();
  return s.ok() ? BAMG_OK : fail(ctx, s);
}

bamg_status bamg_bsr_get_values(const bamg_bsr* A, double* vals) {
  if (!A || !vals) return BAMG_ERR_INVALID;
  bamg_ctx* ctx = A->ctx;
  if (!A->has_pattern) return fail(ctx, make_status(BAMG_ERR_STATE, "matrix has no pattern"));
  if (A->vals64_stale)
    return fail(ctx, make_status(BAMG_ERR_STATE, "the matrix holds only FP32 values (FP32 Galerkin product)"));
  Status s = launch_gather_blocks(A, A->vals, vals, ctx->stream);
  return s.ok() ? BAMG_OK : fail(ctx, s);
}

bamg_status bamg_bsr_set_symmetric(bamg_bsr* A, int symmetric) {
  if (!A) return BAMG_ERR_INVALID;
  if (symmetric && (A->br != A->bc || A->nbr != A->nbc))
    return fail(A->ctx, make_status(BAMG_ERR_INVALID, "only square matrices can be symmetric"));
  A->symmetric = symmetric != 0;
  return BAMG_OK;
}

bamg_status bamg_bsr_autotune(bamg_bsr* A, int* lanes, float* ms) {
  if (!A) return BAMG_ERR_INVALID;
  Status s = bsr_autotune(A, ms);
  if (!s.ok()) return fail(A->ctx, s);
  if (lanes) *lanes = A->split ? -A->split : A->vec;
  return BAMG_OK;
}

// Lanes code -> lanes per row (widths only) and split code (0 for a width),
// checked against A's blocks.
static Status parse_lanes(const bamg_bsr* A, int lanes, int* vec, int* split) {
  if (lanes <= 0) {
    const int vs = lanes == 0 ? 4 : -lanes;
    const bool block_split = is_block_split(vs);
    if (vs != 1 && vs != 2 && vs != 4 && vs != 32 && vs != 64 && vs != 128 && !block_split)
      return make_status(BAMG_ERR_INVALID,
                         "split lanes must be -1, -2, -4, -32, -64, -128, -258, -260, -264, -272 or -288");
    if (A->br != 6 || (A->bc != 3 && A->bc != 6))
      return make_status(BAMG_ERR_INVALID, "the component-split form needs 6x3 or 6x6 blocks");
    if (block_split && A->bc != 3) return make_status(BAMG_ERR_INVALID, "the block split needs 6x3 blocks");
    *split = vs;
    return Status{};
  }
  if (lanes > 32 || (lanes & (lanes - 1)))
    return make_status(BAMG_ERR_INVALID, "lanes must be -4, -2, -1, 0 or a power of two in [1, 32]");
  *vec = lanes;
  *split = 0;
  return Status{};
}

// A split code leaves the copy's lanes per row as they were (the kernels
// without a split form keep using them); a width clears the split.
bamg_status bamg_bsr_set_lanes(bamg_bsr* A, int lanes) {
  if (!A) return BAMG_ERR_INVALID;
  int vec = 0, split = 0;
  const Status s = parse_lanes(A, lanes, &vec, &split);
  if (!s.ok()) return fail(A->ctx, s);
  if (!split) A->vec = A->vec32 = vec;
  A->split = A->split32 = split;
  return BAMG_OK;
}

bamg_status bamg_bsr_get_lanes(const bamg_bsr* A, int* lanes) {
  if (!A || !lanes) return BAMG_ERR_INVALID;
  *lanes = A->split ? -A->split : A->vec;
  return BAMG_OK;
}

bamg_status bamg_bsr_set_lanes_prec(bamg_bsr* A, int prec, int lanes) {
  if (!A || (prec != BAMG_FP64 && prec != BAMG_FP32)) return BAMG_ERR_INVALID;
  int& vec = prec == BAMG_FP64 ? A->vec : A->vec32;
  int& split = prec == BAMG_FP64 ? A->split : A->split32;
  int v = 0, sp = 0;
  const Status s = parse_lanes(A, lanes, &v, &sp);
  if (!s.ok()) return fail(A->ctx, s);
  if (!sp) vec = v;
  split = sp;
  return BAMG_OK;
}

bamg_status bamg_bsr_get_lanes_prec(const bamg_bsr* A, int prec, int* lanes) {
  if (!A || !lanes || (prec != BAMG_FP64 && prec != BAMG_FP32)) return BAMG_ERR_INVALID;
  *lanes = prec == BAMG_FP64 ? (A->split ? -A->split : A->vec) : (A->split32 ? -A->split32 : A->vec32);
  return BAMG_OK;
}

bamg_status bamg_bsr_spmv(bamg_bsr* A, const void* x, void* y, bamg_prec prec, int transpose) {
  if (!A) return BAMG_ERR_INVALID;
  bamg_ctx* ctx = A->ctx;
  if (transpose)
    return fail(ctx, make_status(BAMG_ERR_INVALID, "transposed SpMV is not supported; form R = P^T"));
  if (!A->has_pattern) return fail(ctx, make_status(BAMG_ERR_STATE, "matrix has no pattern"));
  if ((!x && A->nbc) || (!y && A->nbr)) return fail(ctx, make_status(BAMG_ERR_INVALID, "null vector"));
  Status s;
  if (prec == BAMG_FP64) {
    s = launch_spmv<double>(A, A->vals, (const double*)x, (double*)y, ctx->stream);
  } else if (prec == BAMG_FP32) {
    s = bsr_ensure_fp32(A);
    if (s.ok()) s = launch_spmv<float>(A, A->vals32, (const float*)x, (float*)y, ctx->stream);
  } else {
    s = make_status(BAMG_ERR_INVALID, "bad precision %d", (int)prec);
  }
  return s.ok() ? BAMG_OK : fail(ctx, s);
}

bamg_status bamg_bsr_spmm(bamg_bsr* A, const void* X, void* Y, int k, bamg_prec prec) {
  if (!A) return BAMG_ERR_INVALID;
  bamg_ctx* ctx = A->ctx;
  if (!A->has_pattern) return fail(ctx, make_status(BAMG_ERR_STATE, "matrix has no pattern"));
  if (k < 1 || k > 32) return fail(ctx, make_status(BAMG_ERR_INVALID, "k must be in [1, 32]"));
  if ((!X && A->nbc) || (!Y && A->nbr)) return fail(ctx, make_status(BAMG_ERR_INVALID, "null vector"));
  Status s;
  if (prec == BAMG_FP64) {
    s = launch_spmm<double>(A, A->vals, (const double*)X, (double*)Y, k, ctx->stream);
  } else if (prec == BAMG_FP32) {
    s = bsr_ensure_fp32(A);
    if (s.ok()) s = launch_spmm<float>(A, A->vals32, (const float*)X, (float*)Y, k, ctx->stream);
  } else {
    s = make_status(BAMG_ERR_INVALID, "bad precision %d", (int)prec);
  }
  return s.ok() ? BAMG_OK : fail(ctx, s);
}

}  // extern "C"
