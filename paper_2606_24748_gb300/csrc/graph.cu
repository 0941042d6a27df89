// Block operator inspection, strength-of-connection graph and device MIS
// aggregation (Sec. 2.2, Sec. 3.2, Sec. 6).
//
// The strength test is the scalar one of Sec. 2.2, |a_ij| >= eps sqrt(a_ii
// a_jj), taken on whole blocks with the Frobenius norm as the weight (Sec.
// 3.2: one graph edge per stored block).  It is decided on squares: with s
// the sum of a block's squared entries (row-major order, each product and
// sum rounded on its own), j is strong for i when j != i, s_ij > 0 and
// s_ij * s_ij >= (eps^4 * s_ii) * s_jj.  No square root and no fused
// operation enters the decision, so it is exactly reproducible.
//
// The coarsener (Sec. 6) is Luby's maximal independent set with fixed
// weights w_i = splitmix64(i, seed), ties broken by i: in a round every
// undecided vertex whose (w, i) beats all its not-excluded neighbours enters
// the set, then every undecided neighbour of a set vertex is excluded.  The
// rounds reach the greedy set in descending (w, i) order whatever the
// schedule.  Aggregates: one per set vertex (root), numbered in vertex order;
// every other vertex joins its neighbour root of largest (w, j).
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <climits>
#include <cstring>

#include "device.cuh"
#include "internal.h"

namespace bamg {

// Sum of squared entries of CSR block k, products and sums rounded apart.
template <typename TM, int B>
__device__ __forceinline__ double block_sumsq(const TM* __restrict__ vals, int64_t slot) {
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < B; ++e) {
    const double v = (double)vals[vidx<B>(slot, e)];
    s = __dadd_rn(s, __dmul_rn(v, v));
  }
  return s;
}

template <int B>
__global__ void k_block_sumsq(int64_t nnzb, const int* __restrict__ slot_of, const double* __restrict__ vals,
                              double* __restrict__ out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nnzb) out[k] = block_sumsq<double, B>(vals, slot_of[k]);
}

__global__ void k_sqrt_inplace(int64_t n, double* __restrict__ v) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) v[k] = sqrt(v[k]);
}

// Largest absolute scalar row sum (as the bits of a non-negative double:
// their integer order is the numeric order, so atomicMax is exact).
template <int BR, int BC>
__global__ void k_row_abs_max(int64_t nbr, const int* __restrict__ rowptr, const int* __restrict__ slot_of,
                              const double* __restrict__ vals, unsigned long long* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  double best = 0.0;
  for (int a = 0; a < BR; ++a) {
    double t = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      for (int c = 0; c < BC; ++c) t += fabs(vals[vidx<BR * BC>(slot_of[k], a * BC + c)]);
    best = fmax(best, t);
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

// s_ii of every block row (its diagonal block in CSR order).
__global__ void k_diag_sumsq(int64_t nbr, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                             const double* __restrict__ ssq, double* __restrict__ dsq) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  double d = 0.0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
    if (colidx[k] == i) d = ssq[k];
  dsq[i] = d;
}

__device__ __forceinline__ bool strong_block(int64_t i, int j, double sij, const double* __restrict__ dsq,
                                             double eps4) {
  return j != i && sij > 0.0 && __dmul_rn(sij, sij) >= __dmul_rn(__dmul_rn(eps4, dsq[i]), dsq[j]);
}

// Pass 1 counts the strong neighbours of each row, pass 2 writes them.
__global__ void k_strength_rows(int64_t nbr, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                const double* __restrict__ ssq, const double* __restrict__ dsq, double eps4,
                                const int* __restrict__ grow, int* __restrict__ count, int* __restrict__ gcol) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  int c = 0;
  const int o = gcol ? grow[i] : 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const int j = colidx[k];
    if (strong_block(i, j, ssq[k], dsq, eps4)) {
      if (gcol) gcol[o + c] = j;
      ++c;
    }
  }
  if (!gcol) count[i] = c;
}

// splitmix64 (Steele, Lea and Flood 2014): output d of the generator seeded
// with `seed` is mix(seed + (d + 1) gamma).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long d, unsigned long long seed) {
  unsigned long long z = seed + (d + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool beats(unsigned long long wa, int a, unsigned long long wb, int b) {
  return wa > wb || (wa == wb && a > b);
}

enum : int8_t { kUndecided = 0, kIn = 1, kOut = 2 };

// A round's entries.  A neighbour that entered in this very round still
// counts as a competitor (state != out): entries of earlier rounds have no
// undecided neighbours left, so this reads the state at the round's start.
__global__ void k_mis_enter(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                            unsigned long long seed, int8_t* __restrict__ st) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || st[i] != kUndecided) return;
  const unsigned long long wi = splitmix64((unsigned long long)i, seed);
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    if (st[j] != kOut && beats(splitmix64((unsigned long long)j, seed), j, wi, (int)i)) return;
  }
  st[i] = kIn;
}

__global__ void k_mis_exclude(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                              int8_t* __restrict__ st, unsigned* __restrict__ undecided) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || st[i] != kUndecided) return;
  for (int k = rp[i]; k < rp[i + 1]; ++k)
    if (st[col[k]] == kIn) {
      st[i] = kOut;
      return;
    }
  atomicAdd(undecided, 1u);
}

// root_vertex[a] = the set vertex numbered a
__global__ void k_root_vertex(int64_t n, const int8_t* __restrict__ st, const int* __restrict__ root_id,
                              int* __restrict__ root_vertex) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && st[i] == kIn) root_vertex[root_id[i]] = (int)i;
}

__global__ void k_root_flags(int64_t n, const int8_t* __restrict__ st, int* __restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) flag[i] = st[i] == kIn ? 1 : 0;
}

__global__ void k_mis_assign(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                             unsigned long long seed, const int8_t* __restrict__ st, const int* __restrict__ root_id,
                             int* __restrict__ agg, int* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (st[i] == kIn) {
    agg[i] = root_id[i];
    return;
  }
  int best = -1;
  unsigned long long wb = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    if (st[j] != kIn) continue;
    const unsigned long long wj = splitmix64((unsigned long long)j, seed);
    if (best < 0 || beats(wj, j, wb, best)) {
      best = j;
      wb = wj;
    }
  }
  if (best < 0) {  // cannot happen for a maximal set of a symmetric graph
    set_err(err, kDevIndex);
    agg[i] = -1;
    return;
  }
  agg[i] = root_id[best];
}

static unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

// out[0 .. n] = exclusive prefix sum of in[0 .. n) (out[n] = total).
static Status exclusive_scan(const int* in, int* out, int64_t n, cudaStream_t st) {
  size_t bytes = 0;
  BAMG_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)n + 1, st));
  char* tmp = nullptr;
  BAMG_TRY(dalloc(&tmp, (int64_t)std::max<size_t>(bytes, 1), st));
  const cudaError_t e = cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, (int)n + 1, st);
  dfree(tmp, st);
  BAMG_CUDA(e);
  return Status{};
}

static Status block_sumsq_all(const bamg_bsr* A, double* out, cudaStream_t st) {
  if (A->vals64_stale) return make_status(BAMG_ERR_STATE, "the FP64 values are stale (FP32-only product)");
  const unsigned g = grid_of(A->nnzb);
  switch (A->br * 8 + A->bc) {
    case 3 * 8 + 3: { k_block_sumsq<9><<<g, 256, 0, st>>>(A->nnzb, A->slot_of, A->vals, out); BAMG_COUNT_LAUNCH; } break;
    case 6 * 8 + 6: { k_block_sumsq<36><<<g, 256, 0, st>>>(A->nnzb, A->slot_of, A->vals, out); BAMG_COUNT_LAUNCH; } break;
    case 3 * 8 + 6:
    case 6 * 8 + 3: { k_block_sumsq<18><<<g, 256, 0, st>>>(A->nnzb, A->slot_of, A->vals, out); BAMG_COUNT_LAUNCH; } break;
    default: return make_status(BAMG_ERR_INVALID, "block norms support 3x3, 3x6, 6x3 and 6x6 blocks");
  }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

Status strength_graph(bamg_bsr* A, double eps, int* grow, int* gcol, int64_t cap, int64_t* nedges) {
  if (!A->has_pattern) return make_status(BAMG_ERR_STATE, "the matrix has no pattern");
  if (A->br != A->bc || A->nbr != A->nbc) return make_status(BAMG_ERR_INVALID, "the strength graph needs a square operator");
  if (!(eps >= 0.0)) return make_status(BAMG_ERR_INVALID, "eps must be >= 0");
  cudaStream_t st = A->ctx->stream;
  const int64_t n = A->nbr;
  double *ssq = nullptr, *dsq = nullptr;
  int* count = nullptr;
  Status s = dalloc(&ssq, std::max<int64_t>(A->nnzb, 1), st);
  if (s.ok()) s = dalloc(&dsq, std::max<int64_t>(n, 1), st);
  if (s.ok()) s = dalloc(&count, n + 1, st);
  if (s.ok()) s = block_sumsq_all(A, ssq, st);
  const double eps2 = eps * eps, eps4 = eps2 * eps2;
  if (s.ok() && n > 0) {
    k_diag_sumsq<<<grid_of(n), 256, 0, st>>>(n, A->rowptr, A->colidx, ssq, dsq);
    BAMG_COUNT_LAUNCH;
    k_strength_rows<<<grid_of(n), 256, 0, st>>>(n, A->rowptr, A->colidx, ssq, dsq, eps4, nullptr, count, nullptr);
    BAMG_COUNT_LAUNCH;
    if (cudaGetLastError() != cudaSuccess) s = make_status(BAMG_ERR_CUDA, "strength count");
  }
  if (s.ok()) s = exclusive_scan(count, grow, n, st);
  int total = 0;
  if (s.ok() && cudaMemcpyAsync(&total, grow + n, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    s = make_status(BAMG_ERR_CUDA, "edge count");
  if (s.ok() && cudaStreamSynchronize(st) != cudaSuccess) s = make_status(BAMG_ERR_CUDA, "edge count");
  if (s.ok() && total > cap) s = make_status(BAMG_ERR_INVALID, "col holds %lld entries, the graph has %d edges", (long long)cap, total);
  if (s.ok() && n > 0) {
    k_strength_rows<<<grid_of(n), 256, 0, st>>>(n, A->rowptr, A->colidx, ssq, dsq, eps4, grow, nullptr, gcol);
    BAMG_COUNT_LAUNCH;
    if (cudaGetLastError() != cudaSuccess) s = make_status(BAMG_ERR_CUDA, "strength fill");
  }
  dfree(ssq, st);
  dfree(dsq, st);
  dfree(count, st);
  if (s.ok() && nedges) *nedges = total;
  return s;
}

// root_vertex (device, optional, capacity n): the root vertex of every aggregate.
Status mis_aggregate(bamg_ctx* ctx, int64_t n, const int* rp, const int* col, uint64_t seed, int* agg,
                     int64_t* n_agg, int* rounds, int* root_vertex) {
  if (n < 0 || n > INT_MAX - 1) return make_status(BAMG_ERR_INVALID, "vertex count out of range");
  cudaStream_t st = ctx->stream;
  int8_t* state = nullptr;
  int *flag = nullptr, *root_id = nullptr;
  unsigned* undecided = nullptr;
  Status s = dalloc(&state, std::max<int64_t>(n, 1), st);
  if (s.ok()) s = dalloc(&flag, n + 1, st);
  if (s.ok()) s = dalloc(&root_id, n + 1, st);
  if (s.ok()) s = dalloc(&undecided, 1, st);
  if (s.ok() && cudaMemsetAsync(state, 0, (size_t)std::max<int64_t>(n, 1), st) != cudaSuccess)
    s = make_status(BAMG_ERR_CUDA, "state");
  int r = 0;
  unsigned left = n > 0 ? 1u : 0u;
  // every round moves the undecided vertex of largest (w, i) into the set, so
  // at most n rounds; the bound only guards against a malformed graph
  while (s.ok() && left > 0 && r <= n) {
    ++r;
    k_mis_enter<<<grid_of(n), 256, 0, st>>>(n, rp, col, (unsigned long long)seed, state);
    BAMG_COUNT_LAUNCH;
    cudaMemsetAsync(undecided, 0, sizeof(unsigned), st);
    k_mis_exclude<<<grid_of(n), 256, 0, st>>>(n, rp, col, state, undecided);
    BAMG_COUNT_LAUNCH;
    if (cudaMemcpyAsync(&left, undecided, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = make_status(BAMG_ERR_CUDA, "MIS round");
  }
  if (s.ok() && left > 0) s = make_status(BAMG_ERR_INVALID, "MIS did not settle: the graph is not symmetric");
  int roots = 0;
  if (s.ok() && n > 0) {
    k_root_flags<<<grid_of(n), 256, 0, st>>>(n, state, flag);
    BAMG_COUNT_LAUNCH;
    s = exclusive_scan(flag, root_id, n, st);
    if (s.ok()) {
      k_mis_assign<<<grid_of(n), 256, 0, st>>>(n, rp, col, (unsigned long long)seed, state, root_id, agg, ctx->d_err);
      BAMG_COUNT_LAUNCH;
      if (root_vertex) {
        k_root_vertex<<<grid_of(n), 256, 0, st>>>(n, state, root_id, root_vertex);
        BAMG_COUNT_LAUNCH;
      }
      if (cudaMemcpyAsync(&roots, root_id + n, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = make_status(BAMG_ERR_CUDA, "root count");
    }
  }
  if (s.ok()) s = check_device_error(ctx);
  dfree(state, st);
  dfree(flag, st);
  dfree(root_id, st);
  dfree(undecided, st);
  if (s.ok()) {
    if (n_agg) *n_agg = roots;
    if (rounds) *rounds = r;
  }
  return s;
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_bsr_block_norms(bamg_bsr* A, double* out) {
  if (!A || (!out && A->nnzb > 0)) return BAMG_ERR_INVALID;
  if (!A->has_pattern) return fail(A->ctx, make_status(BAMG_ERR_STATE, "the matrix has no pattern"));
  cudaStream_t st = A->ctx->stream;
  Status s = block_sumsq_all(A, out, st);
  if (s.ok() && A->nnzb > 0) {
    k_sqrt_inplace<<<grid_of(A->nnzb), 256, 0, st>>>(A->nnzb, out);
    BAMG_COUNT_LAUNCH;
  }
  return s.ok() ? BAMG_OK : fail(A->ctx, s);
}

bamg_status bamg_bsr_norm(bamg_bsr* A, int type, double* out) {
  if (!A || !out || (type != BAMG_NORM_FROBENIUS && type != BAMG_NORM_INFINITY)) return BAMG_ERR_INVALID;
  if (!A->has_pattern) return fail(A->ctx, make_status(BAMG_ERR_STATE, "the matrix has no pattern"));
  cudaStream_t st = A->ctx->stream;
  auto body = [&]() -> Status {
    if (A->vals64_stale) return make_status(BAMG_ERR_STATE, "the FP64 values are stale (FP32-only product)");
    if (type == BAMG_NORM_FROBENIUS) {
      double* ssq = nullptr;
      BAMG_TRY(dalloc(&ssq, std::max<int64_t>(A->nnzb, 1), st));
      Status s = block_sumsq_all(A, ssq, st);
      std::vector<double> h((size_t)A->nnzb);
      if (s.ok() && A->nnzb > 0 &&
          cudaMemcpyAsync(h.data(), ssq, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = make_status(BAMG_ERR_CUDA, "norm");
      if (s.ok() && cudaStreamSynchronize(st) != cudaSuccess) s = make_status(BAMG_ERR_CUDA, "norm");
      dfree(ssq, st);
      BAMG_TRY(s);
      double t = 0.0;  // block order, on the host: one fixed order
      for (double v : h) t += v;
      *out = sqrt(t);
      return Status{};
    }
    unsigned long long* m = nullptr;
    BAMG_TRY(dalloc(&m, 1, st));
    Status s;
    if (cudaMemsetAsync(m, 0, sizeof(unsigned long long), st) != cudaSuccess) s = make_status(BAMG_ERR_CUDA, "norm");
    const unsigned g = grid_of(A->nbr);
    if (s.ok() && A->nbr > 0) {
      switch (A->br * 8 + A->bc) {
        case 3 * 8 + 3: k_row_abs_max<3, 3><<<g, 256, 0, st>>>(A->nbr, A->rowptr, A->slot_of, A->vals, m); break;
        case 6 * 8 + 6: k_row_abs_max<6, 6><<<g, 256, 0, st>>>(A->nbr, A->rowptr, A->slot_of, A->vals, m); break;
        case 3 * 8 + 6: k_row_abs_max<3, 6><<<g, 256, 0, st>>>(A->nbr, A->rowptr, A->slot_of, A->vals, m); break;
        case 6 * 8 + 3: k_row_abs_max<6, 3><<<g, 256, 0, st>>>(A->nbr, A->rowptr, A->slot_of, A->vals, m); break;
        default: s = make_status(BAMG_ERR_INVALID, "norms support 3x3, 3x6, 6x3 and 6x6 blocks");
      }
      if (s.ok()) BAMG_COUNT_LAUNCH;
    }
    unsigned long long h = 0;
    if (s.ok() && (cudaMemcpyAsync(&h, m, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                   cudaStreamSynchronize(st) != cudaSuccess))
      s = make_status(BAMG_ERR_CUDA, "norm");
    dfree(m, st);
    BAMG_TRY(s);
    std::memcpy(out, &h, sizeof(double));  // the bits of a non-negative double
    return Status{};
  };
  Status s = body();
  return s.ok() ? BAMG_OK : fail(A->ctx, s);
}

bamg_status bamg_strength_graph(bamg_bsr* A, double eps, int* rowptr, int* col, int64_t col_capacity,
                                int64_t* nedges) {
  if (!A || !rowptr || (!col && col_capacity > 0) || col_capacity < 0) return BAMG_ERR_INVALID;
  Status s = strength_graph(A, eps, rowptr, col, col_capacity, nedges);
  return s.ok() ? BAMG_OK : fail(A->ctx, s);
}

bamg_status bamg_mis_aggregate(bamg_ctx* ctx, int64_t n, const int* rowptr, const int* col, uint64_t seed, int* agg,
                               int64_t* n_agg, int* rounds) {
  if (!ctx || n < 0 || (n > 0 && (!rowptr || !agg))) return BAMG_ERR_INVALID;
  Status s = mis_aggregate(ctx, n, rowptr, col, seed, agg, n_agg, rounds, nullptr);
  return s.ok() ? BAMG_OK : fail(ctx, s);
}

}  // extern "C"
