// Device-side building blocks shared by the kernels: sliced-storage addressing,
// the one-thread-per-block-row product, and deterministic reductions.
#pragma once

#include "internal.h"

namespace bamg {

// Address of element e of slot `slot` in a sliced value array of B-element blocks.
template <int B>
__device__ __forceinline__ int64_t vidx(int64_t slot, int e) {
  return (slot >> 5) * (32LL * B) + 32LL * e + (slot & 31);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-row product acc[r] = sum over the row's blocks of A_blk[r][:] . x_blk,
// computed by V lanes per row (V divides 32).  With V = 1 a row is one lane
// and the 32 rows of a slice share the slice's chunk range, so the loop is
// uniform across the warp and every value / column load is one coalesced
// access with no cross-lane reduction.  Matrices with few, long rows (the
// restriction R = P^T, coarse levels) use V > 1: the V lanes of a row take
// every V-th chunk and the partial sums are combined with a fixed xor
// shuffle tree, after which every lane of the group holds the row sums.
// Matrix values and columns are streamed (evict-first); x is gathered
// through the read-only path, where neighbouring rows hit the same lines.
// `row` is the thread's row; `sub` its lane within the row's group.
template <int BR, int BC, int V, typename TM, typename TA, typename TX>
__device__ __forceinline__ void row_product(const int* __restrict__ slice_ptr,
                                            const int* __restrict__ col,
                                            const TM* __restrict__ vals,
                                            const TX* __restrict__ x, int64_t row, int sub,
                                            TA (&acc)[BR]) {
  const int64_t s = row >> 5;
  const int lane = (int)(row & 31);
  const int c0 = __ldg(slice_ptr + s), c1 = __ldg(slice_ptr + s + 1);
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = TA(0);
#pragma unroll 2
  for (int c = c0 + sub; c < c1; c += V) {
    const int64_t slot = (int64_t)c * 32 + lane;
    const int j = __ldcs(col + slot);
    const TM* v = vals + (int64_t)c * (32 * BR * BC) + lane;
    TA xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = (TA)__ldg(x + (int64_t)j * BC + q);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[r] = fma((TA)__ldcs(v + 32 * (r * BC + q)), xv[q], acc[r]);
  }
  if (V > 1) {
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int o = V / 2; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  }
}

// Thread -> (row, sub-lane) for V lanes per row.
template <int V>
__device__ __forceinline__ void row_of_thread(int64_t t, int64_t& row, int& sub) {
  row = t / V;
  sub = (int)(t - row * V);
}

// Run `body` with the compile-time lane count matching v (1..32).
#define BAMG_DISPATCH_V(v, ...)                \
  switch (v) {                                 \
    case 32: { constexpr int V = 32; __VA_ARGS__; } break; \
    case 16: { constexpr int V = 16; __VA_ARGS__; } break; \
    case 8: { constexpr int V = 8; __VA_ARGS__; } break;   \
    case 4: { constexpr int V = 4; __VA_ARGS__; } break;   \
    case 2: { constexpr int V = 2; __VA_ARGS__; } break;   \
    default: { constexpr int V = 1; __VA_ARGS__; } break;  \
  }

// Deterministic grid reduction of NV doubles: every CTA reduces its threads'
// values with a fixed shuffle tree, writes its partials, and the last CTA to
// arrive (atomic ticket) sums the partials in CTA order with a fixed tree.
// Returns true in the last CTA; out[] is valid in its thread 0.  The counter
// is reset by the last CTA.  blockDim.x must be a multiple of 32, <= 1024.
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double* __restrict__ partials,
                            unsigned* __restrict__ counter, double (&out)[NV]) {
  __shared__ double sm[32][NV];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double w = warp_sum(v[k]);
    if (lane == 0) sm[warp][k] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double w = warp_sum(lane < nw ? sm[lane][k] : 0.0);
      if (lane == 0) partials[(int64_t)blockIdx.x * NV + k] = w;
    }
    if (lane == 0) {
      __threadfence();
      unsigned t = atomicAdd(counter, 1u);
      is_last = (t == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partials + (int64_t)b * NV + k);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double w = warp_sum(acc[k]);
    if (lane == 0) sm[warp][k] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double w = warp_sum(lane < nw ? sm[lane][k] : 0.0);
      if (lane == 0) out[k] = w;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

__device__ __forceinline__ void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

}  // namespace bamg
