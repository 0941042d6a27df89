// Blocked SpMV and multi-right-hand-side SpMM on the sliced block storage
// (Sec. 4.2: one column index per block; FP64 or FP32 values).
#include <algorithm>

#include "bsplit.cuh"
#include "device.cuh"
#include "internal.h"

namespace bamg {

template <int BR, int BC, int V, typename T>
__global__ void __launch_bounds__(kRowThreads) k_spmv(const int* __restrict__ slice_ptr,
                                                      const int* __restrict__ col, const T* __restrict__ vals,
                                                      const int* __restrict__ srow, const T* __restrict__ x,
                                                      T* __restrict__ y, int64_t nbr, int64_t nthreads) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  int64_t pos;
  int sub;
  row_of_thread<V>(t, pos, sub);
  T acc[BR];
  row_product<BR, BC, V, T, T, T>(slice_ptr, col, vals, x, pos, sub, acc);
  const int64_t row = srow ? (int64_t)srow[pos] : pos;  // row position -> block row (sorted slices)
  if (sub == 0 && row >= 0 && row < nbr) {
#pragma unroll
    for (int r = 0; r < BR; ++r) y[row * BR + r] = acc[r];
  }
}

// Component-split form for 6-row blocks (CTA = one slice, BR * VS warps).
template <int BR, int BC, int VS, typename T>
__global__ void __launch_bounds__(768) k_spmv_split(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                                    const T* __restrict__ vals, const int* __restrict__ srow,
                                                    const T* __restrict__ x, T* __restrict__ y, int64_t nbr) {
  const int64_t s = blockIdx.x;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31, a = wp % BR, sub = wp / BR;
  const T acc = row_component<BR, BC, VS, T, T, T>(slice_ptr, col, vals, x, s, lane, a, sub);
  const int64_t i = srow ? (int64_t)srow[s * 32 + lane] : s * 32 + lane;
  if (sub == 0 && i >= 0 && i < nbr) y[i * BR + a] = acc;
}

// All-component block split (6x3 blocks: the finest restriction): CTA = one
// slice, VB warps (see row_blocks_split).
template <int BR, int BC, int VB, typename T>
__global__ void __launch_bounds__(32 * VB) k_spmv_bsplit(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                                          const T* __restrict__ vals, const int* __restrict__ srow,
                                                          const T* __restrict__ x, T* __restrict__ y, int64_t nbr) {
  const int64_t s = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T out[blocks_split_outs<BR, VB>()];
  row_blocks_split<BR, BC, VB, T, T, T>(slice_ptr, col, vals, x, s, lane, w, out);
  const int64_t i = row_at(srow, s * 32 + lane);
  if (i < 0 || i >= nbr) return;
#pragma unroll
  for (int k = 0; k < blocks_split_outs<BR, VB>(); ++k)
    if (w + k * VB < BR) y[i * BR + w + k * VB] = out[k];
}

// Row form (rectangular 6-row-block matrices with few, long rows).
template <int BR, int BC, int VR, typename T>
__global__ void __launch_bounds__(32 * BR * VR) k_spmv_rows(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                                            const T* __restrict__ vals, const int* __restrict__ srow,
                                                            const T* __restrict__ x, T* __restrict__ y, int64_t nbr) {
  const int64_t pos = blockIdx.x;
  const T acc = row_component_lanes<BR, BC, VR, T, T, T>(slice_ptr, col, vals, x, pos);
  const int64_t i = srow ? (int64_t)srow[pos] : pos;
  const int a = threadIdx.x;
  if (a < BR && i >= 0 && i < nbr) y[i * BR + a] = acc;
}

// Any block shape up to 8x8 (shapes without a specialisation).
template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_spmv_any(const int* __restrict__ slice_ptr,
                                                          const int* __restrict__ col, const T* __restrict__ vals,
                                                          const int* __restrict__ srow, const T* __restrict__ x,
                                                          T* __restrict__ y, int64_t nbr, int64_t nrows_pad, int br,
                                                          int bc) {
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= nrows_pad) return;
  const int64_t s = pos >> 5;
  const int lane = (int)(pos & 31);
  const int64_t row = srow ? (int64_t)srow[pos] : pos;
  const int B = br * bc;
  T acc[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) acc[r] = T(0);
  for (int c = slice_ptr[s]; c < slice_ptr[s + 1]; ++c) {
    const int64_t slot = (int64_t)c * 32 + lane;
    const int j = col[slot];
    const T* v = vals + (int64_t)c * 32 * B + lane;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (r < br) {
        for (int q = 0; q < bc; ++q) acc[r] = fma(v[32 * (r * bc + q)], x[(int64_t)j * bc + q], acc[r]);
      }
    }
  }
  if (row >= 0 && row < nbr) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (r < br) y[row * br + r] = acc[r];
  }
}

// Y = A X with k right-hand sides, X[dof * k + j].  Thread = (block row, j):
// the threads of a row share each block value load (broadcast) and read k
// consecutive X entries per block column.
template <int BR, int BC, typename T>
__global__ void __launch_bounds__(256) k_spmm(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                              const T* __restrict__ vals, const int* __restrict__ srow,
                                              const T* __restrict__ X, T* __restrict__ Y, int64_t nbr, int k) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t pos = t / k;
  const int j = (int)(t - pos * k);
  if (pos >= nbr) return;
  const int64_t row = srow ? (int64_t)srow[pos] : pos;
  const int64_t s = pos >> 5;
  const int lane = (int)(pos & 31);
  T acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = T(0);
  const int c0 = __ldg(slice_ptr + s), c1 = __ldg(slice_ptr + s + 1);
  for (int c = c0; c < c1; ++c) {
    const int cj = __ldg(col + (int64_t)c * 32 + lane);
    const T* v = vals + (int64_t)c * (32 * BR * BC) + lane;
    T xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = __ldg(X + ((int64_t)cj * BC + q) * k + j);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[r] = fma(__ldg(v + 32 * (r * BC + q)), xv[q], acc[r]);
  }
#pragma unroll
  for (int r = 0; r < BR; ++r) Y[(row * BR + r) * k + j] = acc[r];
}

// The same product with four right-hand sides per thread (k a multiple of 4,
// X and Y aligned to four elements): each block value is loaded once for four
// vectors.
template <int BR, int BC, typename T>
__global__ void __launch_bounds__(256) k_spmm4(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                               const T* __restrict__ vals, const int* __restrict__ srow,
                                               const T* __restrict__ X, T* __restrict__ Y, int64_t nbr, int k) {
  const int G = k >> 2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t pos = t / G;
  if (pos >= nbr) return;
  const int64_t row = srow ? (int64_t)srow[pos] : pos;
  const int c0 = (int)(t - pos * G) * 4;
  T acc[BR][4];
  row_product4<BR, BC, T>(slice_ptr, col, vals, X, k, pos, c0, acc);
#pragma unroll
  for (int r = 0; r < BR; ++r) st4(Y + (row * BR + r) * k + c0, acc[r]);
}

static bool can_split(const bamg_bsr* A) { return A->br == 6 && (A->bc == 3 || A->bc == 6); }

// vec = lanes per row (1..32), or -VS for the component-split form with VS
// warps per component.
template <typename T>
static Status launch_spmv_v(const bamg_bsr* A, int vec, const T* vals, const T* x, T* y, cudaStream_t st) {
  if (vec <= -kSplitBlocks) {
    if (A->nslices == 0) return Status{};
    if (A->br != 6 || A->bc != 3) return make_status(BAMG_ERR_INVALID, "the block split needs 6x3 blocks");
    BAMG_DISPATCH_VB(-vec, {
      k_spmv_bsplit<6, 3, VB, T><<<(unsigned)A->nslices, 32 * VB, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, x, y,
                                                                           A->nbr);
      BAMG_COUNT_LAUNCH; })
    BAMG_CUDA(cudaGetLastError());
    return Status{};
  }
  if (vec <= -kSplitRows) {
    if (A->nslices == 0) return Status{};
    const unsigned g = (unsigned)(A->nslices * kSlice);
    BAMG_DISPATCH_ROWS(-vec, {
      if (A->bc == 6)
        k_spmv_rows<6, 6, VR, T><<<g, 192 * VR, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, x, y, A->nbr);
      else
        k_spmv_rows<6, 3, VR, T><<<g, 192 * VR, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, x, y, A->nbr);
      BAMG_COUNT_LAUNCH; })
    BAMG_CUDA(cudaGetLastError());
    return Status{};
  }
  if (vec < 0) {
    if (A->nslices == 0) return Status{};
    BAMG_DISPATCH_VS(-vec, {
      if (A->bc == 6)
        k_spmv_split<6, 6, VS, T><<<(unsigned)A->nslices, 192 * VS, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, x, y,
                                                                            A->nbr);
      else
        k_spmv_split<6, 3, VS, T><<<(unsigned)A->nslices, 192 * VS, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, x, y,
                                                                            A->nbr);
      BAMG_COUNT_LAUNCH; })
    BAMG_CUDA(cudaGetLastError());
    return Status{};
  }
  const int64_t nt = A->nslices * kSlice * (int64_t)vec;
  if (nt == 0) return Status{};
  const unsigned blocks = (unsigned)((nt + kRowThreads - 1) / kRowThreads);
#define BAMG_SPMV_CASE(R, C)                                                                                  \
  if (A->br == R && A->bc == C) {                                                                             \
    BAMG_DISPATCH_V(vec, { k_spmv<R, C, V, T><<<blocks, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, x, y, \
                                                                           A->nbr, nt); BAMG_COUNT_LAUNCH; }) \
    BAMG_CUDA(cudaGetLastError());                                                                            \
    return Status{};                                                                                          \
  }
  BAMG_SPMV_CASE(3, 3)
  BAMG_SPMV_CASE(6, 6)
  BAMG_SPMV_CASE(3, 6)
  BAMG_SPMV_CASE(6, 3)
#undef BAMG_SPMV_CASE
  const int64_t rows = A->nslices * kSlice;
  { k_spmv_any<T><<<(unsigned)((rows + kRowThreads - 1) / kRowThreads), kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, x, y, A->nbr, rows, A->br, A->bc); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <typename T>
Status launch_spmv(const bamg_bsr* A, const T* vals, const T* x, T* y, cudaStream_t st) {
  return launch_spmv_v<T>(A, split_for<T>(A) && can_split(A) ? -split_for<T>(A) : lanes_for<T>(A), vals, x, y, st);
}

int default_vec(const bamg_bsr* A) {
  // enough threads to cover the GPU (152 SMs x ~1k threads), no more lanes
  // than the average row has blocks, at most a warp
  const int64_t target = 152 * 1024;
  const double avg = A->nbr > 0 ? (double)A->nnzb / (double)A->nbr : 1.0;
  int v = 1;
  while (v < 32 && A->nbr * v < target && 2 * v <= avg) v *= 2;
  return v;
}

// Measured choice of the lanes per row (tile / warp mapping): time the
// product y = A x for each width on the context's stream (two warm-up
// launches, median of five) and keep the fastest, separately for the FP64
// values and, when the matrix has one, the FP32 copy.  Inside a V-cycle a
// coarse matrix is read after the fine level has streamed through L2, so
// every timed launch starts from a flushed L2 (a 192 MB buffer is written
// first, untimed); timing warm-cache repeats would favour one lane per row
// for matrices that fit in L2.  Cold path (setup); allocates work buffers.
template <typename T>
static Status tune_lanes(bamg_bsr* A, const T* vals, int* out_vec, int* out_split, float* out_ms) {
  cudaStream_t st = A->ctx->stream;
  T *x = nullptr, *y = nullptr;
  const int64_t nx = std::max<int64_t>(1, A->nbc * A->bc), ny = std::max<int64_t>(1, A->nbr * A->br);
  BAMG_TRY(dalloc(&x, nx, st));
  BAMG_TRY(dalloc(&y, ny, st));
  BAMG_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * nx, st));
  cudaEvent_t e0, e1;
  BAMG_CUDA(cudaEventCreate(&e0));
  BAMG_CUDA(cudaEventCreate(&e1));
  const size_t flush_bytes = (size_t)192 << 20;
  void* flush = nullptr;
  BAMG_TRY(dalloc((char**)&flush, (int64_t)flush_bytes, st));
  float best = 1e30f;
  int bestv = *out_vec;
  int best_split = 0;
  Status s;
  // widths 1, 2, ..., 32, then (6-row blocks) the component-split form with
  // 1, 2 and 4 warps per component, coded as -1, -2, -4
  // and, for rectangular ones (the restriction), the row form with 1, 2 and
  // 4 warps per component (-32, -64, -128); for 6x3 blocks also the
  // all-component block split with 8, 16 and 32 warps (-264, -272, -288)
  static const int kChoices[] = {1, 2, 4, 8, 16, 32, -1, -2, -4, -32, -64, -128,
                                 -(kSplitBlocks + 8), -(kSplitBlocks + 16), -(kSplitBlocks + 32)};
  const int n_choices = !can_split(A) ? 6 : (A->br == 6 && A->bc == 3) ? 15 : (A->nbr != A->nbc || A->br != A->bc ? 12 : 9);
  for (int ci = 0; ci < n_choices; ++ci) {
    const int lv = kChoices[ci];
    for (int w = 0; w < 2 && s.ok(); ++w) s = launch_spmv_v<T>(A, lv, vals, x, y, st);
    if (!s.ok()) break;
    float t[5];
    for (int rep = 0; rep < 5; ++rep) {
      cudaMemsetAsync(flush, rep, flush_bytes, st);
      cudaEventRecord(e0, st);
      s = launch_spmv_v<T>(A, lv, vals, x, y, st);
      cudaEventRecord(e1, st);
      if (!s.ok()) break;
      cudaEventSynchronize(e1);
      if (cudaEventElapsedTime(&t[rep], e0, e1) != cudaSuccess) {
        cudaGetLastError();
        t[rep] = 1e30f;
      }
    }
    if (!s.ok()) break;
    std::sort(t, t + 5);
    if (t[2] < best * 0.97f) {
      best = t[2];
      if (lv < 0) {
        best_split = -lv;
      } else {
        best_split = 0;
        bestv = lv;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  dfree(x, st);
  dfree(y, st);
  dfree(flush, st);
  if (!s.ok()) return s;
  *out_vec = bestv;
  *out_split = best_split;
  if (out_ms) *out_ms = best;
  return Status{};
}

Status bsr_autotune(bamg_bsr* A, float* best_ms) {
  if (!A->has_pattern) return make_status(BAMG_ERR_STATE, "autotune needs a pattern");
  const bool special = (A->br == 3 || A->br == 6) && (A->bc == 3 || A->bc == 6);
  if (!special) return Status{};
  if (!A->vals64_stale) BAMG_TRY(tune_lanes<double>(A, A->vals, &A->vec, &A->split, best_ms));
  if (A->vals32) BAMG_TRY(tune_lanes<float>(A, A->vals32, &A->vec32, &A->split32, A->vals64_stale ? best_ms : nullptr));
  A->vec_tuned = true;
  return Status{};
}

template <typename T>
Status launch_spmm(const bamg_bsr* A, const T* vals, const T* X, T* Y, int k, cudaStream_t st) {
  const int64_t nt = A->nbr * (int64_t)k;
  if (nt == 0) return Status{};
  const bool four = k % 4 == 0 && ((uintptr_t)X % (4 * sizeof(T))) == 0 && ((uintptr_t)Y % (4 * sizeof(T))) == 0;
  const unsigned blocks = (unsigned)(((four ? nt / 4 : nt) + 255) / 256);
#define BAMG_SPMM_CASE(R, C)                                                                   \
  if (A->br == R && A->bc == C) {                                                              \
    if (four)                                                                                  \
      { k_spmm4<R, C, T><<<blocks, 256, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, X, Y, A->nbr, k); BAMG_COUNT_LAUNCH; } \
    else                                                                                       \
      { k_spmm<R, C, T><<<blocks, 256, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, X, Y, A->nbr, k); BAMG_COUNT_LAUNCH; } \
    BAMG_CUDA(cudaGetLastError());                                                             \
    return Status{};                                                                           \
  }
  BAMG_SPMM_CASE(3, 3)
  BAMG_SPMM_CASE(6, 6)
  BAMG_SPMM_CASE(3, 6)
  BAMG_SPMM_CASE(6, 3)
#undef BAMG_SPMM_CASE
  return make_status(BAMG_ERR_INVALID, "spmm supports 3x3, 6x6, 3x6 and 6x3 blocks");
}

template Status launch_spmv<double>(const bamg_bsr*, const double*, const double*, double*, cudaStream_t);
template Status launch_spmv<float>(const bamg_bsr*, const float*, const float*, float*, cudaStream_t);
template Status launch_spmm<double>(const bamg_bsr*, const double*, const double*, double*, int, cudaStream_t);
template Status launch_spmm<float>(const bamg_bsr*, const float*, const float*, float*, int, cudaStream_t);

}  // namespace bamg
