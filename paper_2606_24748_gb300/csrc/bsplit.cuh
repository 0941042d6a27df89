// All-component block split of the 6x3 block-row product (the restriction
// from the finest level), shared by the SpMV and the cycle's transfer.
#pragma once

#include "internal.h"

namespace bamg {

// All-component block split for 6-row blocks: a CTA of VB warps takes one
// 32-row slice; warp w adds, for every output component of its lane's row,
// the products over every VB-th chunk of the slice, starting at w.  Each
// chunk's column index and x entries are then loaded once per lane, where
// the component split loads them once per component warp (six times).  The
// VB partial rows meet in shared memory (one barrier); warp w then adds up
// components w, w + VB, ... in warp order, so that every component is summed
// exactly as row_component with VS = VB sums it, and returns them in out[]
// (out[k] = component w + k * VB, when that is below BR).  Every thread of
// the CTA must call this.
template <int BR, int VB>
constexpr int blocks_split_outs() { return (BR + VB - 1) / VB; }
template <int BR, int BC, int VB, typename TM, typename TA, typename TX>
__device__ __forceinline__ void row_blocks_split(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                                 const TM* __restrict__ vals, const TX* __restrict__ x, int64_t s,
                                                 int lane, int w, TA (&out)[blocks_split_outs<BR, VB>()]) {
  static_assert(VB >= 2, "the block split takes two or more warps");
  const int c0 = __ldg(slice_ptr + s), c1 = __ldg(slice_ptr + s + 1);
  TA acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = TA(0);
  for (int c = c0 + w; c < c1; c += VB) {
    const int j = __ldg(col + (int64_t)c * 32 + lane);
    const TM* v = vals + (int64_t)c * (32 * BR * BC) + lane;
    // the block's values are all requested before the gather of x, so that
    // their loads are in flight together
    TM blk[BR * BC];
#pragma unroll
    for (int e = 0; e < BR * BC; ++e) blk[e] = __ldcs(v + 32 * e);
    TA xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = (TA)__ldg(x + (int64_t)j * BC + q);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[r] = fma((TA)blk[r * BC + q], xv[q], acc[r]);
  }
  __shared__ TA part[VB][BR][32];
#pragma unroll
  for (int r = 0; r < BR; ++r) part[w][r][lane] = acc[r];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < blocks_split_outs<BR, VB>(); ++k) {
    const int a = w + k * VB;
    TA sum = TA(0);
    if (a < BR) {
      sum = part[0][a][lane];
#pragma unroll 8
      for (int t = 1; t < VB; ++t) sum += part[t][a][lane];
    }
    out[k] = sum;
  }
}

}  // namespace bamg
