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

// Component-split block-row product for matrices with 6-row blocks (the
// restriction, coarse operators).  A CTA of BR * VS warps takes one 32-row
// slice: warp (a, sub) adds the products for output component a (lane = row
// within the slice) over every VS-th chunk of the slice, starting at sub.
// Each block adds BC products to one accumulator, so no lane is idle and no
// partial sums are combined across lanes: with FP64 at two FMA per clock per
// SM, the lanes-per-row form spends as many instructions on its reduction
// and its one-lane epilogue as on the products of a short row.  The VS
// partial sums of a component are added in shared memory in sub order
// (one barrier); the result is valid in the sub = 0 warps.  Every thread of
// the CTA must call this.  The warps read the same column indices and x
// entries (cached); every value is read once, coalesced.
template <int BR, int BC, int VS, typename TM, typename TA, typename TX>
__device__ __forceinline__ TA row_component(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                            const TM* __restrict__ vals, const TX* __restrict__ x, int64_t s,
                                            int lane, int a, int sub) {
  const int c0 = __ldg(slice_ptr + s), c1 = __ldg(slice_ptr + s + 1);
  TA acc = TA(0);
  for (int c = c0 + sub; c < c1; c += VS) {
    const int j = __ldg(col + (int64_t)c * 32 + lane);
    const TM* v = vals + (int64_t)c * (32 * BR * BC) + 32 * (a * BC) + lane;
    TA xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = (TA)__ldg(x + (int64_t)j * BC + q);
#pragma unroll
    for (int q = 0; q < BC; ++q) acc = fma((TA)__ldcs(v + 32 * q), xv[q], acc);
  }
  if (VS > 1) {
    __shared__ TA part[VS][BR][32];
    part[sub][a][lane] = acc;
    __syncthreads();
    if (sub == 0) {
#pragma unroll
      for (int t = 1; t < VS; ++t) acc += part[t][a][lane];
    }
  }
  return acc;
}

// Row form of the component split, for matrices with few, very long rows
// (the restriction to the coarsest levels): a CTA of BR * VS warps takes one
// row position; warp (a, sub) sums output component a over every VS-th group
// of 32 chunks of the row, one chunk per lane, then one shuffle tree.  With
// VS > 1 the VS partial sums meet in shared memory; thread a < BR returns
// component a's total (the other threads return 0).
template <int BR, int BC, int VS, typename TM, typename TA, typename TX>
__device__ __forceinline__ TA row_component_lanes(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                                  const TM* __restrict__ vals, const TX* __restrict__ x,
                                                  int64_t pos) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = w / VS, sub = w % VS;
  const int64_t s = pos >> 5;
  const int l = (int)(pos & 31);
  const int c0 = __ldg(slice_ptr + s), c1 = __ldg(slice_ptr + s + 1);
  TA acc = TA(0);
  for (int c = c0 + sub * 32 + lane; c < c1; c += 32 * VS) {
    const int j = __ldg(col + (int64_t)c * 32 + l);
    const TM* v = vals + (int64_t)c * (32 * BR * BC) + 32 * (a * BC) + l;
#pragma unroll
    for (int q = 0; q < BC; ++q) acc = fma((TA)__ldg(v + 32 * q), (TA)__ldg(x + (int64_t)j * BC + q), acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ TA part[BR * VS];
  if (lane == 0) part[w] = acc;
  __syncthreads();
  TA total = TA(0);
  if (threadIdx.x < BR) {
#pragma unroll
    for (int t = 0; t < VS; ++t) total += part[threadIdx.x * VS + t];
  }
  return total;
}

// Thread -> (row, sub-lane) for V lanes per row.
template <int V>
__device__ __forceinline__ void row_of_thread(int64_t t, int64_t& row, int& sub) {
  row = t / V;
  sub = (int)(t - row * V);
}

// Block row stored at row position pos.  Slices sorted by row length carry
// the map (srow; -1 at the padding positions past the last row); otherwise
// the position is the row.  Vectors and block-diagonal inverses stay indexed
// by row in either case.
__device__ __forceinline__ int64_t row_at(const int* __restrict__ srow, int64_t pos) {
  return srow ? (int64_t)__ldg(srow + pos) : pos;
}

// Balanced deal of warp tasks (32 consecutive virtual threads) for the
// one-wave reducing row kernels: CTA c takes a contiguous run of tasks, the
// runs differing in length by at most one, and its warps take every W-th
// task of the run.  With a grid of SMs x resident CTAs every SM then gets the
// same number of rows to within one task per CTA (numbering threads straight
// through leaves some SMs a whole CTA short for the entire kernel), and
// neighbouring rows stay in one CTA, where they share gathered x in L1.
// Loop: for (g = t0 + warp; g < t1; g += W) after deal_range(ntasks, t0, t1).
__device__ __forceinline__ void deal_range(int64_t ntasks, int64_t& t0, int64_t& t1) {
  const int64_t G = gridDim.x, c = blockIdx.x, q = ntasks / G, rem = ntasks - q * G;
  t0 = c * q + (c < rem ? c : rem);
  t1 = t0 + q + (c < rem ? 1 : 0);
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

// Deterministic grid reduction of NV doubles: every CTA sums its threads'
// values in a fixed order, writes its partials, and the last CTA to arrive
// (atomic ticket) sums the partials in CTA order the same way.  Returns true
// in the last CTA; out[] is valid in its thread 0.  The counter is reset by
// the last CTA.  blockDim.x must be a multiple of 32, <= 1024.
// An FP64 add costs a warp 64 cycles of an SM sub-partition here, so the CTA
// sum goes through shared memory: lane l of warp 0 adds the values 32 apart
// (nw - 1 adds), then one shuffle tree (5 adds): 12 FP64 warp instructions
// for 256 threads instead of a shuffle tree per warp (45).
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double* __restrict__ partials,
                            unsigned* __restrict__ counter, double (&out)[NV]) {
  __shared__ double buf[NV][1024];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) buf[k][threadIdx.x] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double w = buf[k][lane];
      for (int i = 1; i < nw; ++i) w += buf[k][lane + 32 * i];
      w = warp_sum(w);
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
#pragma unroll
  for (int k = 0; k < NV; ++k) buf[k][threadIdx.x] = acc[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double w = buf[k][lane];
      for (int i = 1; i < nw; ++i) w += buf[k][lane + 32 * i];
      w = warp_sum(w);
      if (lane == 0) out[k] = w;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Four consecutive values (the right-hand sides one thread of a multi-vector
// kernel owns); p must be aligned to 4 elements.  ld4 reads through the
// read-only path (arrays the kernel does not write), ld4w plainly.
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4w(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4w(const float* p, float (&v)[4]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
}

// Block-row product for four right-hand sides at once: X holds kp vectors
// RHS-minor (entry (dof d, vector j) at X[d * kp + j]) and the thread takes
// vectors c0..c0+3 of block row `row`.  Each block value is loaded once and
// used for the four vectors; the kp / 4 threads of a row read the same value
// (one broadcast).  Per vector, the summation order is that of row_product
// with one lane per row.
template <int BR, int BC, typename T>
__device__ __forceinline__ void row_product4(const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                             const T* __restrict__ vals, const T* __restrict__ X, int kp,
                                             int64_t row, int c0, T (&acc)[BR][4]) {
  const int64_t s = row >> 5;
  const int lane = (int)(row & 31);
  const int a0 = __ldg(slice_ptr + s), a1 = __ldg(slice_ptr + s + 1);
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[r][e] = T(0);
  for (int c = a0; c < a1; ++c) {
    const int j = __ldg(col + (int64_t)c * 32 + lane);
    const T* v = vals + (int64_t)c * (32 * BR * BC) + lane;
    T xv[BC][4];
#pragma unroll
    for (int q = 0; q < BC; ++q) ld4(X + ((int64_t)j * BC + q) * kp + c0, xv[q]);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) {
        const T a = __ldg(v + 32 * (r * BC + q));
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[r][e] = fma(a, xv[q][e], acc[r][e]);
      }
  }
}

// Deterministic grid reduction of ns = G * NV sums at once: thread t adds
// v[e] to sum (t mod G) * NV + e.  G is a power of two <= 32, ns <= 64 and
// blockDim.x = 256 (a multiple of ns); the grid-stride loops that feed it keep
// a thread on one residue mod G.  Fixed shuffle trees inside each warp, warps
// summed in order, per-CTA partials summed by the last CTA to arrive (atomic
// ticket) in a fixed order.  Returns true in the last CTA, where out_sm
// (shared, ns doubles) then holds the sums for every thread of the CTA.
template <int NV>
__device__ bool grid_reduce_groups(const double (&v)[NV], int G, double* __restrict__ partials,
                                   unsigned* __restrict__ counter, double* out_sm) {
  __shared__ double sm[512];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ns = G * NV;
#pragma unroll
  for (int e = 0; e < NV; ++e) {
    double x = v[e];
    for (int o = 16; o >= G; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane < G) sm[warp * ns + lane * NV + e] = x;
  }
  __syncthreads();
  if ((int)threadIdx.x < ns) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += sm[w * ns + threadIdx.x];
    partials[(int64_t)blockIdx.x * ns + threadIdx.x] = a;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  const int step = blockDim.x / ns;
  double a = 0.0;
  for (int b = threadIdx.x / ns; b < (int)gridDim.x; b += step)
    a += __ldcg(partials + (int64_t)b * ns + threadIdx.x % ns);
  sm[threadIdx.x] = a;
  __syncthreads();
  if ((int)threadIdx.x < ns) {
    double t = 0.0;
    for (int k = 0; k < step; ++k) t += sm[k * ns + threadIdx.x];
    out_sm[threadIdx.x] = t;
  }
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
  return true;
}

// Programmatic dependent launch (kernels launched with launch_k): the kernel
// may be launched before the preceding kernel of the stream has finished;
// this waits until that kernel has completed and its memory is visible.  The
// launch of the next kernel is left to the implicit trigger at CTA exit: an
// explicit early trigger let waiting CTAs of the next kernel crowd the SMs
// and made the CG iteration 8% slower.  A no-op for a kernel launched
// without the attribute.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with programmatic stream serialisation allowed (the kernel must
// start with pdl_enter()).  Captured into a CUDA graph, the dependency
// becomes a programmatic edge.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

}  // namespace bamg
