// Blocked SpMV and multi-right-hand-side SpMM on the sliced block storage
// (Sec. 4.2: one column index per block; FP64 or FP32 values).
#include "device.cuh"
#include "internal.h"

namespace bamg {

template <int BR, int BC, typename T>
__global__ void __launch_bounds__(kRowThreads) k_spmv(const int* __restrict__ slice_ptr,
                                                      const int* __restrict__ col, const T* __restrict__ vals,
                                                      const T* __restrict__ x, T* __restrict__ y, int64_t nbr,
                                                      int64_t nrows_pad) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= nrows_pad) return;
  T acc[BR];
  row_product<BR, BC, T, T, T>(slice_ptr, col, vals, x, row, acc);
  if (row < nbr) {
#pragma unroll
    for (int r = 0; r < BR; ++r) y[row * BR + r] = acc[r];
  }
}

// Any block shape up to 8x8 (shapes without a specialisation).
template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_spmv_any(const int* __restrict__ slice_ptr,
                                                          const int* __restrict__ col, const T* __restrict__ vals,
                                                          const T* __restrict__ x, T* __restrict__ y, int64_t nbr,
                                                          int64_t nrows_pad, int br, int bc) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= nrows_pad) return;
  const int64_t s = row >> 5;
  const int lane = (int)(row & 31);
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
  if (row < nbr) {
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
                                              const T* __restrict__ vals, const T* __restrict__ X,
                                              T* __restrict__ Y, int64_t nbr, int k) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = t / k;
  const int j = (int)(t - row * k);
  if (row >= nbr) return;
  const int64_t s = row >> 5;
  const int lane = (int)(row & 31);
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

template <typename T>
Status launch_spmv(const bamg_bsr* A, const T* vals, const T* x, T* y, cudaStream_t st) {
  const int64_t rows = A->nslices * kSlice;
  if (rows == 0) return Status{};
  const unsigned blocks = (unsigned)((rows + kRowThreads - 1) / kRowThreads);
#define BAMG_SPMV_CASE(R, C)                                                                                     \
  if (A->br == R && A->bc == C) {                                                                                \
    k_spmv<R, C, T><<<blocks, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, vals, x, y, A->nbr, rows);        \
    BAMG_CUDA(cudaGetLastError());                                                                               \
    return Status{};                                                                                             \
  }
  BAMG_SPMV_CASE(3, 3)
  BAMG_SPMV_CASE(6, 6)
  BAMG_SPMV_CASE(3, 6)
  BAMG_SPMV_CASE(6, 3)
#undef BAMG_SPMV_CASE
  k_spmv_any<T><<<blocks, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, vals, x, y, A->nbr, rows, A->br, A->bc);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <typename T>
Status launch_spmm(const bamg_bsr* A, const T* vals, const T* X, T* Y, int k, cudaStream_t st) {
  const int64_t nt = A->nbr * (int64_t)k;
  if (nt == 0) return Status{};
  const unsigned blocks = (unsigned)((nt + 255) / 256);
#define BAMG_SPMM_CASE(R, C)                                                                   \
  if (A->br == R && A->bc == C) {                                                              \
    k_spmm<R, C, T><<<blocks, 256, 0, st>>>(A->slice_ptr, A->sell_col, vals, X, Y, A->nbr, k); \
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
