// V-cycle (Sec. 2.1) with Chebyshev / point-block Jacobi smoothing (Sec. 4.1)
// and preconditioned CG (Sec. 4.1), all as fused row kernels on the sliced
// block storage.
//
// Chebyshev (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1,
// preconditioned by the block diagonal D) is run with the residual carried by
// the recurrence: a step with direction d_k does x += d_k, r -= A d_k and
// d_{k+1} = c1_k d_k + c2_k W D^-1 r in one kernel (one SpMV), so after
// pre-smoothing the residual needed for restriction is already there.
// Every kernel takes an optional device flag `done`: when set (CG converged)
// the kernel returns at once, which lets a whole CG iteration be captured in
// one CUDA graph and launched in batches without a host round trip per
// iteration.
#include <algorithm>
#include <type_traits>

#include "bsplit.cuh"
#include "device.cuh"
#include "internal.h"

namespace bamg {

template <int BS, typename T>
__device__ __forceinline__ void dinv_apply(const T* __restrict__ dinv, int64_t i, const T (&r)[BS], T (&z)[BS]) {
  const int64_t base = (i >> 5) * (32LL * BS * BS) + (i & 31);
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    T t = T(0);
#pragma unroll
    for (int c = 0; c < BS; ++c) t = fma(__ldg(dinv + base + 32 * (a * BS + c)), r[c], t);
    z[a] = t;
  }
}

#define BAMG_DONE_RETURN \
  if (done && *done) return;

// r = b; d = w Dinv b / theta; x = 0.  The mixed form's finest level reads
// the FP64 right-hand side itself (TB = double) and keeps its float copy in
// bcopy, in place of a separate conversion launch.
template <int BS, typename T, typename TB = T>
__global__ void __launch_bounds__(kRowThreads) k_cheb_init(int64_t n, const TB* __restrict__ b, T* __restrict__ bcopy,
                                                           T* __restrict__ r, T* __restrict__ d, T* __restrict__ x,
                                                           const T* __restrict__ dinv, const float* __restrict__ w,
                                                           const double* __restrict__ scal, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T bi[BS], z[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    bi[a] = (T)b[i * BS + a];
    if (bcopy) bcopy[i * BS + a] = bi[a];
  }
  dinv_apply<BS, T>(dinv, i, bi, z);
  const T f = (T)(scal[kInvTheta] * (w ? (double)w[i] : 1.0));
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    r[i * BS + a] = bi[a];
    d[i * BS + a] = f * z[a];
    x[i * BS + a] = T(0);
  }
}

// x += d_in; r -= A d_in; if has_next: d_out = c1 d_in + c2 w Dinv r.
// FINAL (the last step of post-smoothing): the next direction is the last
// one; it is added to x here ((x + d_in) + d_out, the order of a separate
// update) instead of being stored.  A separate instance, so that the common
// one keeps its register count.
template <int BS, int V, typename T, bool FINAL = false>
__global__ void __launch_bounds__(kRowThreads) k_cheb_step(const int* __restrict__ sp, const int* __restrict__ col,
                                                           const T* __restrict__ vals, const int* __restrict__ srow,
                                                           int64_t n, int64_t nthreads,
                                                           const T* __restrict__ d_in, T* __restrict__ d_out,
                                                           T* __restrict__ x, T* __restrict__ r,
                                                           const T* __restrict__ dinv, const float* __restrict__ w,
                                                           const double* __restrict__ scal, int k, int has_next,
                                                           double* __restrict__ xout, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  int64_t pos;
  int sub;
  row_of_thread<V>(t, pos, sub);
  T acc[BS];
  row_product<BS, BS, V, T, T, T>(sp, col, vals, d_in, pos, sub, acc);
  const int64_t i = row_at(srow, pos);
  if (sub != 0 || i < 0 || i >= n) return;
  T di[BS], ri[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    di[a] = d_in[i * BS + a];
    ri[a] = r[i * BS + a] - acc[a];
    r[i * BS + a] = ri[a];
    if constexpr (!FINAL) x[i * BS + a] += di[a];
  }
  if (FINAL || has_next) {
    T z[BS];
    dinv_apply<BS, T>(dinv, i, ri, z);
    const T c1 = (T)scal[kCheb + 2 * k];
    const T c2 = (T)(scal[kCheb + 2 * k + 1] * (w ? (double)w[i] : 1.0));
#pragma unroll
    for (int a = 0; a < BS; ++a) {
      const T dn = fma(c1, di[a], c2 * z[a]);
      if constexpr (FINAL) {
        const T xn = (x[i * BS + a] + di[a]) + dn;
        if (xout)  // the mixed form's finest level: the cycle's FP64 result
          xout[i * BS + a] = (double)xn;
        else
          x[i * BS + a] = xn;
      } else {
        d_out[i * BS + a] = dn;
      }
    }
  }
}

// r = b - A x; d = w Dinv r / theta   (x is read by the product: not written here)
template <int BS, int V, typename T>
__global__ void __launch_bounds__(kRowThreads) k_cheb_rinit(const int* __restrict__ sp, const int* __restrict__ col,
                                                            const T* __restrict__ vals, const int* __restrict__ srow,
                                                            int64_t n, int64_t nthreads,
                                                            const T* __restrict__ x, const T* __restrict__ b,
                                                            T* __restrict__ r, T* __restrict__ d,
                                                            const T* __restrict__ dinv, const float* __restrict__ w,
                                                            const double* __restrict__ scal, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  int64_t pos;
  int sub;
  row_of_thread<V>(t, pos, sub);
  T acc[BS];
  row_product<BS, BS, V, T, T, T>(sp, col, vals, x, pos, sub, acc);
  const int64_t i = row_at(srow, pos);
  if (sub != 0 || i < 0 || i >= n) return;
  T ri[BS], z[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    ri[a] = b[i * BS + a] - acc[a];
    r[i * BS + a] = ri[a];
  }
  dinv_apply<BS, T>(dinv, i, ri, z);
  const T f = (T)(scal[kInvTheta] * (w ? (double)w[i] : 1.0));
#pragma unroll
  for (int a = 0; a < BS; ++a) d[i * BS + a] = f * z[a];
}

// Component-split forms of the three row kernels above (6-row blocks): CTA =
// one slice, BS * VS warps (see row_component).  The block-diagonal inverse
// needs every component of the new residual, exchanged through shared memory.
template <int BS, int VS, typename T, bool FINAL = false>
__global__ void __launch_bounds__(768) k_cheb_step_split(const int* __restrict__ sp, const int* __restrict__ col,
                                                         const T* __restrict__ vals, const int* __restrict__ srow,
                                                         int64_t n,
                                                         const T* __restrict__ d_in, T* __restrict__ d_out,
                                                         T* __restrict__ x, T* __restrict__ r,
                                                         const T* __restrict__ dinv, const float* __restrict__ w,
                                                         const double* __restrict__ scal, int k, int has_next,
                                                         const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  __shared__ T rs[BS][32];
  const int64_t s = blockIdx.x;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31, a = wp % BS, sub = wp / BS;
  const int64_t i = row_at(srow, s * 32 + lane);
  const T acc = row_component<BS, BS, VS, T, T, T>(sp, col, vals, d_in, s, lane, a, sub);
  const bool lead = sub == 0 && i >= 0 && i < n;
  T ri = T(0), di = T(0);
  if (lead) {
    di = d_in[i * BS + a];
    ri = r[i * BS + a] - acc;
    r[i * BS + a] = ri;
    if constexpr (!FINAL) x[i * BS + a] += di;
  }
  if (!FINAL && !has_next) return;
  if (sub == 0) rs[a][lane] = ri;
  __syncthreads();
  if (!lead) return;
  const int64_t base = (i >> 5) * (32LL * BS * BS) + (i & 31);
  T z = T(0);
#pragma unroll
  for (int c = 0; c < BS; ++c) z = fma(__ldg(dinv + base + 32 * (a * BS + c)), rs[c][lane], z);
  const T c1 = (T)scal[kCheb + 2 * k];
  const T c2 = (T)(scal[kCheb + 2 * k + 1] * (w ? (double)w[i] : 1.0));
  const T dn = fma(c1, di, c2 * z);
  if constexpr (FINAL)
    x[i * BS + a] = (x[i * BS + a] + di) + dn;  // last post-smoothing step (see k_cheb_step)
  else
    d_out[i * BS + a] = dn;
}

template <int BS, int VS, typename T>
__global__ void __launch_bounds__(768) k_cheb_rinit_split(const int* __restrict__ sp, const int* __restrict__ col,
                                                          const T* __restrict__ vals, const int* __restrict__ srow,
                                                          int64_t n,
                                                          const T* __restrict__ x, const T* __restrict__ b,
                                                          T* __restrict__ r, T* __restrict__ d,
                                                          const T* __restrict__ dinv, const float* __restrict__ w,
                                                          const double* __restrict__ scal, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  __shared__ T rs[BS][32];
  const int64_t s = blockIdx.x;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31, a = wp % BS, sub = wp / BS;
  const int64_t i = row_at(srow, s * 32 + lane);
  const T acc = row_component<BS, BS, VS, T, T, T>(sp, col, vals, x, s, lane, a, sub);
  const bool lead = sub == 0 && i >= 0 && i < n;
  T ri = T(0);
  if (lead) {
    ri = b[i * BS + a] - acc;
    r[i * BS + a] = ri;
  }
  if (sub == 0) rs[a][lane] = ri;
  __syncthreads();
  if (!lead) return;
  const int64_t base = (i >> 5) * (32LL * BS * BS) + (i & 31);
  T z = T(0);
#pragma unroll
  for (int c = 0; c < BS; ++c) z = fma(__ldg(dinv + base + 32 * (a * BS + c)), rs[c][lane], z);
  const T f = (T)(scal[kInvTheta] * (w ? (double)w[i] : 1.0));
  d[i * BS + a] = f * z;
}

template <int BR, int BC, int VS, typename T>
__global__ void __launch_bounds__(768) k_transfer_split(const int* __restrict__ sp, const int* __restrict__ col,
                                                        const T* __restrict__ vals, const int* __restrict__ srow,
                                                        int64_t n, const T* __restrict__ v, T* __restrict__ y,
                                                        int accumulate, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t s = blockIdx.x;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31, a = wp % BR, sub = wp / BR;
  const int64_t i = srow ? (int64_t)srow[s * 32 + lane] : s * 32 + lane;
  const T acc = row_component<BR, BC, VS, T, T, T>(sp, col, vals, v, s, lane, a, sub);
  if (sub == 0 && i >= 0 && i < n) y[i * BR + a] = accumulate ? y[i * BR + a] + acc : acc;
}

// All-component block split (6x3 blocks, the finest restriction): CTA = one
// slice, VB warps (see row_blocks_split).
template <int BR, int BC, int VB, typename T>
__global__ void __launch_bounds__(32 * VB) k_transfer_bsplit(const int* __restrict__ sp, const int* __restrict__ col,
                                                              const T* __restrict__ vals, const int* __restrict__ srow,
                                                              int64_t n, const T* __restrict__ v, T* __restrict__ y,
                                                              int accumulate, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t s = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T out[blocks_split_outs<BR, VB>()];
  row_blocks_split<BR, BC, VB, T, T, T>(sp, col, vals, v, s, lane, w, out);
  const int64_t i = row_at(srow, s * 32 + lane);
  if (i < 0 || i >= n) return;
#pragma unroll
  for (int k = 0; k < blocks_split_outs<BR, VB>(); ++k) {
    const int a = w + k * VB;
    if (a < BR) y[i * BR + a] = accumulate ? y[i * BR + a] + out[k] : out[k];
  }
}

// Row form (see row_component_lanes): CTA = one row position.
template <int BR, int BC, int VR, typename T>
__global__ void __launch_bounds__(32 * BR * VR) k_transfer_rows(const int* __restrict__ sp, const int* __restrict__ col,
                                                                const T* __restrict__ vals, const int* __restrict__ srow,
                                                                int64_t n, const T* __restrict__ v, T* __restrict__ y,
                                                                int accumulate, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t pos = blockIdx.x;
  const T acc = row_component_lanes<BR, BC, VR, T, T, T>(sp, col, vals, v, pos);
  const int64_t i = srow ? (int64_t)srow[pos] : pos;
  const int a = threadIdx.x;
  if (a < BR && i >= 0 && i < n) y[i * BR + a] = accumulate ? y[i * BR + a] + acc : acc;
}

template <typename T>
__global__ void k_axpy_done(int64_t m, const T* __restrict__ d, T* __restrict__ x, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) x[t] += d[t];
}

// y = M v (restriction with R = P^T), or y += M v (prolongation with P)
template <int BR, int BC, int V, typename T>
__global__ void __launch_bounds__(kRowThreads) k_transfer(const int* __restrict__ sp, const int* __restrict__ col,
                                                          const T* __restrict__ vals, const int* __restrict__ srow,
                                                          int64_t n, int64_t nthreads, const T* __restrict__ v,
                                                          T* __restrict__ y, int accumulate, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  int64_t r;
  int sub;
  row_of_thread<V>(t, r, sub);
  T acc[BR];
  row_product<BR, BC, V, T, T, T>(sp, col, vals, v, r, sub, acc);
  const int64_t i = srow ? (int64_t)srow[r] : r;  // row position -> block row (sorted slices)
  if (sub != 0 || i < 0 || i >= n) return;
#pragma unroll
  for (int a = 0; a < BR; ++a) y[i * BR + a] = accumulate ? y[i * BR + a] + acc[a] : acc[a];
}

template <typename TS, typename TD>
__global__ void k_cast_done(int64_t m, const TS* __restrict__ s, TD* __restrict__ d, const int* done) {
  pdl_enter();
  BAMG_DONE_RETURN
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) d[t] = (TD)s[t];
}

// ------------------------------------------------------------------ V-cycle

template <typename T>
struct LevelPtrs {
  T *b, *x, *r, *d0, *d1;
  const T *dinv, *Avals, *Pvals, *Rvals;
};
static LevelPtrs<double> ptrs64(Level& L) {
  return {L.b, L.x, L.r, L.d0, L.d1, L.dinv, L.A->vals, L.P ? L.P->vals : nullptr, L.R ? L.R->vals : nullptr};
}
static LevelPtrs<float> ptrs32(Level& L) {
  return {L.b32, L.x32, L.r32, L.d032, L.d132, L.dinv32, L.A->vals32, L.P ? L.P->vals32 : nullptr,
          L.R ? L.R->vals32 : nullptr};
}
template <typename T>
LevelPtrs<T> level_ptrs(Level& L);
template <>
LevelPtrs<double> level_ptrs<double>(Level& L) { return ptrs64(L); }
template <>
LevelPtrs<float> level_ptrs<float>(Level& L) { return ptrs32(L); }

// CTA size of the fused Chebyshev row kernels.  A level's rows fill about one
// wave of the GPU at the workload sizes (64^3: 8,582 slices for 152 SMs x 64
// warps), so the last CTA of the busier SMs is the kernel's tail: 64-thread
// CTAs (two slices) halve it against 128-thread ones.
constexpr int kChebThreads = 64;

// b64 (mixed form, finest level): the FP64 right-hand side, converted by the
// first kernel; p.b then receives its float copy.
template <int BS, typename T>
static Status smooth_down(bamg_mg* mg, int l, const int* done, cudaStream_t st, const double* b64 = nullptr) {
  Level& L = mg->levels[l];
  auto p = level_ptrs<T>(L);
  const bamg_bsr* A = L.A;
  const int64_t rows = row_threads_for<T>(A);
  const unsigned gr = (unsigned)((rows + kChebThreads - 1) / kChebThreads);
  const unsigned gn = (unsigned)((L.n + kRowThreads - 1) / kRowThreads);
  const double* sc = mg->scal + (int64_t)l * kScalarsPerLevel;
  const int m = mg->opts.cheb_degree;
  const int pw = prof_begin(mg->ctx, l == 0 ? -1 : BAMG_PROF_SMOOTH_COARSE, st);
  const int pi = prof_begin(mg->ctx, l == 0 ? BAMG_PROF_L0_VECTOR : -1, st);
  if (b64) {
    BAMG_CUDA(launch_k(k_cheb_init<BS, T, double>, dim3(gn), dim3(kRowThreads), st, L.n, b64, p.b, p.r, p.d0, p.x,
                       p.dinv, L.weights, sc, done));
  } else {
    BAMG_CUDA(launch_k(k_cheb_init<BS, T>, dim3(gn), dim3(kRowThreads), st, L.n, (const T*)p.b, (T*)nullptr, p.r,
                       p.d0, p.x, p.dinv, L.weights, sc, done));
  }
  BAMG_COUNT_LAUNCH;
  prof_end(mg->ctx, pi, st);
  T* d[2] = {p.d0, p.d1};
  // the m pre-smoothing steps are consecutive launches of one kernel: one
  // bracket, in the sampling slot when that is enabled
  int pm = prof_begin(mg->ctx, l == 0 ? BAMG_PROF_CHEB_PRE_L0 : -1, st, m);
  if (pm < 0) pm = prof_begin(mg->ctx, l == 0 ? BAMG_PROF_CHEB_STEP_L0 : -1, st, m);
  for (int k = 0; k < m; ++k) {
    if (BS == 6 && split_for<T>(A)) {
      BAMG_DISPATCH_VS(split_for<T>(A), {
        BAMG_CUDA(launch_k(k_cheb_step_split<BS, VS, T>, dim3((unsigned)A->nslices), dim3(32 * BS * VS), st, 
            A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, d[k & 1], d[(k + 1) & 1], p.x, p.r, p.dinv, L.weights, sc, k,
            k + 1 < m ? 1 : 0, done));
        BAMG_COUNT_LAUNCH; })
    } else {
      BAMG_DISPATCH_V(lanes_for<T>(A), { BAMG_CUDA(launch_k(k_cheb_step<BS, V, T>, dim3(gr), dim3(kChebThreads), st, A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, rows, d[k & 1],
                                                     d[(k + 1) & 1], p.x, p.r, p.dinv, L.weights, sc, k,
                                                     k + 1 < m ? 1 : 0, (double*)nullptr, done)); BAMG_COUNT_LAUNCH; })
    }
  }
  prof_end(mg->ctx, pm, st);
  prof_end(mg->ctx, pw, st);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

// x64 (mixed form, finest level, degree >= 2): the last step writes the
// cycle's result there in FP64 instead of updating p.x.
template <int BS, typename T>
static Status smooth_up(bamg_mg* mg, int l, const int* done, cudaStream_t st, double* x64 = nullptr) {
  Level& L = mg->levels[l];
  auto p = level_ptrs<T>(L);
  const bamg_bsr* A = L.A;
  const int64_t rows = row_threads_for<T>(A);
  const unsigned gr = (unsigned)((rows + kChebThreads - 1) / kChebThreads);
  const double* sc = mg->scal + (int64_t)l * kScalarsPerLevel;
  const int m = mg->opts.cheb_degree;
  const int split = BS == 6 ? split_for<T>(A) : 0;
  const unsigned gs = (unsigned)A->nslices;
  const int pw = prof_begin(mg->ctx, l == 0 ? -1 : BAMG_PROF_SMOOTH_COARSE, st);
  const int pr = prof_begin(mg->ctx, l == 0 ? BAMG_PROF_CHEB_RINIT_L0 : -1, st);
  if (split) {
    BAMG_DISPATCH_VS(split, {
      BAMG_CUDA(launch_k(k_cheb_rinit_split<BS, VS, T>, dim3(gs), dim3(32 * BS * VS), st, A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, p.x, p.b,
                                                                 p.r, p.d0, p.dinv, L.weights, sc, done));
      BAMG_COUNT_LAUNCH; })
  } else {
    BAMG_DISPATCH_V(lanes_for<T>(A), { BAMG_CUDA(launch_k(k_cheb_rinit<BS, V, T>, dim3(gr), dim3(kChebThreads), st, A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, rows, p.x, p.b, p.r,
                                                    p.d0, p.dinv, L.weights, sc, done)); BAMG_COUNT_LAUNCH; })
  }
  prof_end(mg->ctx, pr, st);
  T* d[2] = {p.d0, p.d1};
  for (int k = 0; k + 1 < m; ++k) {
    const int pm = prof_begin(mg->ctx, l == 0 ? BAMG_PROF_CHEB_STEP_L0 : -1, st);
    const bool last = k + 2 == m;  // the last step adds the final direction to x itself
    if (split) {
      BAMG_DISPATCH_VS(split, {
        auto kern = last ? k_cheb_step_split<BS, VS, T, true> : k_cheb_step_split<BS, VS, T, false>;
        BAMG_CUDA(launch_k(kern, dim3(gs), dim3(32 * BS * VS), st, A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, d[k & 1],
                           d[(k + 1) & 1], p.x, p.r, p.dinv, L.weights, sc, k, 1, done));
        BAMG_COUNT_LAUNCH; })
    } else {
      BAMG_DISPATCH_V(lanes_for<T>(A), {
        auto kern = last ? k_cheb_step<BS, V, T, true> : k_cheb_step<BS, V, T, false>;
        BAMG_CUDA(launch_k(kern, dim3(gr), dim3(kChebThreads), st, A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, rows,
                           d[k & 1], d[(k + 1) & 1], p.x, p.r, p.dinv, L.weights, sc, k, 1, last ? x64 : nullptr,
                           done));
        BAMG_COUNT_LAUNCH; })
    }
    prof_end(mg->ctx, pm, st);
  }
  if (m == 1) {  // degree 1: no step here, the direction from the residual start is the update
    const int64_t mm = L.n * BS;
    const int pa = prof_begin(mg->ctx, l == 0 ? BAMG_PROF_L0_VECTOR : -1, st);
    { BAMG_CUDA(launch_k(k_axpy_done<T>, dim3((unsigned)((mm + 255) / 256)), dim3(256), st, mm, d[0], p.x, done)); BAMG_COUNT_LAUNCH; }
    prof_end(mg->ctx, pa, st);
  }
  prof_end(mg->ctx, pw, st);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <int BR, int BC, typename T>
static Status transfer(const bamg_bsr* M, const T* vals, const T* v, T* y, int accumulate, const int* done,
                       cudaStream_t st) {
  const int64_t rows = row_threads_for<T>(M);
  if (rows == 0) return Status{};
  if constexpr (BR == 6 && BC == 3) {
    if (split_for<T>(M) >= kSplitBlocks) {
      BAMG_DISPATCH_VB(split_for<T>(M), {
        BAMG_CUDA(launch_k(k_transfer_bsplit<BR, BC, VB, T>, dim3((unsigned)M->nslices), dim3(32 * VB), st,
                           M->slice_ptr, M->sell_col, vals, M->slot_row, M->nbr, v, y, accumulate, done));
        BAMG_COUNT_LAUNCH; })
      BAMG_CUDA(cudaGetLastError());
      return Status{};
    }
  }
  if (BR == 6 && split_for<T>(M) >= kSplitRows) {
    BAMG_DISPATCH_ROWS(split_for<T>(M), {
      BAMG_CUDA(launch_k(k_transfer_rows<BR, BC, VR, T>, dim3((unsigned)(M->nslices * kSlice)), dim3(32 * BR * VR), st,
                         M->slice_ptr, M->sell_col, vals, M->slot_row, M->nbr, v, y, accumulate, done));
      BAMG_COUNT_LAUNCH; })
    BAMG_CUDA(cudaGetLastError());
    return Status{};
  }
  if (BR == 6 && split_for<T>(M)) {
    BAMG_DISPATCH_VS(split_for<T>(M), {
      BAMG_CUDA(launch_k(k_transfer_split<BR, BC, VS, T>, dim3((unsigned)M->nslices), dim3(32 * BR * VS), st, M->slice_ptr, M->sell_col, vals,
                                                                                     M->slot_row, M->nbr, v, y, accumulate, done));
      BAMG_COUNT_LAUNCH; })
    BAMG_CUDA(cudaGetLastError());
    return Status{};
  }
  BAMG_DISPATCH_V(lanes_for<T>(M), { BAMG_CUDA(launch_k(k_transfer<BR, BC, V, T>, dim3((unsigned)((rows + kRowThreads - 1) / kRowThreads)), dim3(kRowThreads), st, 
      M->slice_ptr, M->sell_col, vals, M->slot_row, M->nbr, rows, v, y, accumulate, done)); BAMG_COUNT_LAUNCH; })
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

// Restriction (accumulate = 0) or prolongation (1) inside a profiling region.
template <int BR, int BC, typename T>
static Status transfer_prof(bamg_mg* mg, const bamg_bsr* M, const T* vals, const T* v, T* y, int accumulate,
                            const int* done, cudaStream_t st) {
  const int pt = prof_begin(mg->ctx, BAMG_PROF_TRANSFER, st);
  Status s = transfer<BR, BC, T>(M, vals, v, y, accumulate, done, st);
  prof_end(mg->ctx, pt, st);
  return s;
}

// Warps per component of a coarse level's smoother: the lanes autotuner times
// the plain product, and the fused Chebyshev kernels of the same matrix can
// prefer another form.  Time the level's own pre- and post-smoothing with 1,
// 2 and 4 warps per component and keep the fastest; a level the autotuner
// left in the lanes form keeps that form as a candidate too (FP32 products
// of a 64^3 first coarse level chose 16 lanes per row, where the fused
// smoother and the power steps were faster split).  The power steps follow
// the level's choice.  The level's vectors are scratch here.
template <typename T>
static Status tune_smoother_split(bamg_mg* mg, int l) {
  Level& L = mg->levels[l];
  bamg_bsr* A = L.A;
  int& split = std::is_same<T, double>::value ? A->split : A->split32;
  if (L.bs != 6 || A->bc != 6 || split < 0 || split > 4) return Status{};
  cudaStream_t st = mg->ctx->stream;
  cudaEvent_t e0, e1;
  BAMG_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return make_status(BAMG_ERR_CUDA, "event");
  }
  Status s;
  const int keep = split;
  float best = 1e30f;
  int best_vs = keep;
  for (int vs : {0, 1, 2, 4}) {
    if (vs == 0 && keep != 0) continue;  // the lanes form only where the autotuner chose it
    split = vs;
    for (int w = 0; w < 2 && s.ok(); ++w) {
      s = smooth_down<6, T>(mg, l, nullptr, st);
      if (s.ok()) s = smooth_up<6, T>(mg, l, nullptr, st);
    }
    float t[5];
    for (int rep = 0; rep < 5 && s.ok(); ++rep) {
      cudaEventRecord(e0, st);
      s = smooth_down<6, T>(mg, l, nullptr, st);
      if (s.ok()) s = smooth_up<6, T>(mg, l, nullptr, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[rep], e0, e1) != cudaSuccess)
        s = make_status(BAMG_ERR_CUDA, "smoother timing");
    }
    if (!s.ok()) break;
    std::sort(t, t + 5);
    if (t[2] < best) {
      best = t[2];
      best_vs = vs;
    }
  }
  split = s.ok() ? best_vs : keep;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

// Lanes per row of a 3x3-block level's smoother.  The lanes autotuner times
// the plain product; on long rows (Q2: up to 125 blocks) it takes several
// lanes per row, and the fused Chebyshev kernels then leave their per-row
// epilogue (new residual, block-diagonal inverse, update) to one lane in
// several.  Time the level's own pre- and post-smoothing with the product's
// choice and with 1, 2 and 4 lanes, and keep the fastest (the CG product and
// the power steps use the same choice).  The level's vectors are scratch.
template <typename T>
static Status tune_smoother_lanes(bamg_mg* mg, int l) {
  Level& L = mg->levels[l];
  bamg_bsr* A = L.A;
  if (L.bs != 3 || A->bc != 3 || l + 1 >= (int)mg->levels.size()) return Status{};
  int& vec = std::is_same<T, double>::value ? A->vec : A->vec32;
  cudaStream_t st = mg->ctx->stream;
  cudaEvent_t e0, e1;
  BAMG_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return make_status(BAMG_ERR_CUDA, "event");
  }
  Status s;
  const int keep = vec;
  std::vector<int> cand = {keep};  // the product's choice first
  for (int v : {1, 2, 4})
    if (v != keep) cand.push_back(v);
  float best = 1e30f;
  int best_v = keep;
  for (size_t ci = 0; ci < cand.size() && s.ok(); ++ci) {
    const int v = cand[ci];
    vec = v;
    for (int w = 0; w < 2 && s.ok(); ++w) {
      s = smooth_down<3, T>(mg, l, nullptr, st);
      if (s.ok()) s = smooth_up<3, T>(mg, l, nullptr, st);
    }
    float t[5];
    for (int rep = 0; rep < 5 && s.ok(); ++rep) {
      cudaEventRecord(e0, st);
      s = smooth_down<3, T>(mg, l, nullptr, st);
      if (s.ok()) s = smooth_up<3, T>(mg, l, nullptr, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[rep], e0, e1) != cudaSuccess)
        s = make_status(BAMG_ERR_CUDA, "smoother timing");
    }
    if (!s.ok()) break;
    std::sort(t, t + 5);
    // another choice must beat the best so far by 3% (timing noise)
    if (ci == 0 || t[2] < 0.97f * best) {
      best = t[2];
      best_v = v;
    }
  }
  vec = s.ok() ? best_v : keep;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

Status mg_tune_smoothers(bamg_mg* mg) {
  const int nl = (int)mg->levels.size();
  const bool f32 = mg->opts.precision == BAMG_FP32;
  BAMG_TRY(f32 ? tune_smoother_lanes<float>(mg, 0) : tune_smoother_lanes<double>(mg, 0));
  for (int l = 1; l + 1 < nl; ++l) BAMG_TRY(f32 ? tune_smoother_split<float>(mg, l) : tune_smoother_split<double>(mg, l));
  return Status{};
}

template <typename T>
Status vcycle_on(bamg_mg* mg, const int* done, cudaStream_t st, const double* b64, double* x64) {
  const int nl = (int)mg->levels.size();
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = mg->levels[l];
    Level& C = mg->levels[l + 1];
    auto p = level_ptrs<T>(L);
    auto pc = level_ptrs<T>(C);
    if (L.bs == 3) {
      BAMG_TRY((smooth_down<3, T>(mg, l, done, st, l == 0 ? b64 : nullptr)));
      BAMG_TRY((transfer_prof<6, 3, T>(mg, L.R, p.Rvals, p.r, pc.b, 0, done, st)));
    } else {
      BAMG_TRY((smooth_down<6, T>(mg, l, done, st)));
      BAMG_TRY((transfer_prof<6, 6, T>(mg, L.R, p.Rvals, p.r, pc.b, 0, done, st)));
    }
  }
  {
    auto p = level_ptrs<T>(mg->levels[nl - 1]);
    const int pc = prof_begin(mg->ctx, BAMG_PROF_COARSE_SOLVE, st);
    BAMG_TRY(coarse_apply<T>(mg, p.b, p.x, done, st));
    prof_end(mg->ctx, pc, st);
  }
  for (int l = nl - 2; l >= 0; --l) {
    Level& L = mg->levels[l];
    auto p = level_ptrs<T>(L);
    auto pc = level_ptrs<T>(mg->levels[l + 1]);
    if (L.bs == 3) {
      BAMG_TRY((transfer_prof<3, 6, T>(mg, L.P, p.Pvals, pc.x, p.x, 1, done, st)));
      BAMG_TRY((smooth_up<3, T>(mg, l, done, st, l == 0 ? x64 : nullptr)));
    } else {
      BAMG_TRY((transfer_prof<6, 6, T>(mg, L.P, p.Pvals, pc.x, p.x, 1, done, st)));
      BAMG_TRY((smooth_up<6, T>(mg, l, done, st)));
    }
  }
  return Status{};
}

template Status vcycle_on<double>(bamg_mg*, const int*, cudaStream_t, const double*, double*);

Status mg_smooth_down_fp64(bamg_mg* mg, int l, cudaStream_t st) {
  return mg->levels[l].bs == 3 ? smooth_down<3, double>(mg, l, nullptr, st) : smooth_down<6, double>(mg, l, nullptr, st);
}

Status mg_restrict_fp64(bamg_mg* mg, int l, cudaStream_t st) {
  Level& L = mg->levels[l];
  if (L.bs == 3) return transfer<6, 3, double>(L.R, L.R->vals, L.r, mg->levels[l + 1].b, 0, nullptr, st);
  return transfer<6, 6, double>(L.R, L.R->vals, L.r, mg->levels[l + 1].b, 0, nullptr, st);
}
template Status vcycle_on<float>(bamg_mg*, const int*, cudaStream_t, const double*, double*);

// z = M r for FP64 vectors r (read) and z (written); in the mixed form the
// cycle runs on float copies.
static Status precond(bamg_mg* mg, const double* r, double* z, const int* done, cudaStream_t st) {
  Level& L0 = mg->levels[0];
  const int64_t m = L0.n * L0.bs;
  const unsigned g = (unsigned)((m + 255) / 256);
  // the conversions to and from the float cycle ride in its first and last
  // kernels where those are the finest level's Chebyshev kernels (3x3
  // blocks, a coarser level, degree >= 2)
  const bool fold = L0.bs == 3 && mg->levels.size() > 1 && mg->opts.cheb_degree >= 2;
  if (mg->opts.precision == BAMG_FP32 && fold) {
    BAMG_TRY(vcycle_on<float>(mg, done, st, r, z));
  } else if (mg->opts.precision == BAMG_FP32) {
    int pc = prof_begin(mg->ctx, BAMG_PROF_L0_VECTOR, st);
    { BAMG_CUDA(launch_k(k_cast_done<double, float>, dim3(g), dim3(256), st, m, r, L0.b32, done)); BAMG_COUNT_LAUNCH; }
    prof_end(mg->ctx, pc, st);
    BAMG_TRY(vcycle_on<float>(mg, done, st));
    pc = prof_begin(mg->ctx, BAMG_PROF_L0_VECTOR, st);
    { BAMG_CUDA(launch_k(k_cast_done<float, double>, dim3(g), dim3(256), st, m, L0.x32, z, done)); BAMG_COUNT_LAUNCH; }
    prof_end(mg->ctx, pc, st);
  } else {
    if (r != L0.b) { BAMG_CUDA(launch_k(k_cast_done<double, double>, dim3(g), dim3(256), st, m, r, L0.b, done)); BAMG_COUNT_LAUNCH; }
    BAMG_TRY(vcycle_on<double>(mg, done, st));
    if (z != L0.x) { BAMG_CUDA(launch_k(k_cast_done<double, double>, dim3(g), dim3(256), st, m, L0.x, z, done)); BAMG_COUNT_LAUNCH; }
  }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

Status mg_precond(bamg_mg* mg, const double* r, double* z, cudaStream_t st) { return precond(mg, r, z, nullptr, st); }

// ------------------------------------------------------------------ CG

__global__ void k_cg_setup(CgState* s, double rtol, int maxit) {
  pdl_enter();
  s->bnorm2 = 0.0;
  s->rtol2 = rtol * rtol;
  s->rz = s->pq = s->alpha = s->beta = s->rnorm2 = 0.0;
  s->its = 0;
  s->maxit = maxit;
  s->done = s->converged = s->breakdown = 0;
}

// r = b, x = 0, ||b||^2
__global__ void k_cg_init(int64_t m, const double* __restrict__ b, double* __restrict__ r, double* __restrict__ x,
                          CgState* s, double* partials, unsigned* counter) {
  pdl_enter();
  double local[1] = {0.0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[t];
    r[t] = v;
    x[t] = 0.0;
    local[0] = fma(v, v, local[0]);
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) {
    s->bnorm2 = out[0];
    s->rnorm2 = out[0];
    if (!(out[0] > 0.0)) {
      s->done = 1;
      s->converged = 1;
    }
  }
}

// p = z, z_old = z, rz = r.z
__global__ void k_cg_first(int64_t m, const double* __restrict__ r, const double* __restrict__ z,
                           double* __restrict__ p, double* __restrict__ zold, CgState* s, double* partials,
                           unsigned* counter) {
  pdl_enter();
  if (s->done) return;
  double local[1] = {0.0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const double zv = z[t];
    p[t] = zv;
    zold[t] = zv;
    local[0] = fma(r[t], zv, local[0]);
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) s->rz = out[0];
}

// q = A p, alpha = rz / (p.q)
template <int V>
__global__ void __launch_bounds__(256, 8) k_cg_Ap(const int* __restrict__ sp, const int* __restrict__ col,
                                                       const double* __restrict__ vals, const int* __restrict__ srow,
                                                       int64_t n, int64_t nthreads,
                                                       const double* __restrict__ p, double* __restrict__ q,
                                                       CgState* s, double* partials, unsigned* counter) {
  pdl_enter();
  if (s->done) return;
  double local[1] = {0.0};
  const int64_t ntasks = (nthreads + 31) >> 5;
  int64_t t0, t1;
  deal_range(ntasks, t0, t1);
  for (int64_t g = t0 + (threadIdx.x >> 5); g < t1; g += blockDim.x >> 5) {
    const int64_t t = g * 32 + (threadIdx.x & 31);
    if (t >= nthreads) continue;  // rows are whole slices: never taken
    int64_t pos;
    int sub;
    row_of_thread<V>(t, pos, sub);
    double acc[3];
    row_product<3, 3, V, double, double, double>(sp, col, vals, p, pos, sub, acc);
    const int64_t i = row_at(srow, pos);
    if (sub == 0 && i >= 0 && i < n) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        q[i * 3 + a] = acc[a];
        local[0] = fma(p[i * 3 + a], acc[a], local[0]);
      }
    }
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) {
    s->pq = out[0];
    if (!(out[0] > 0.0)) {
      s->breakdown = 1;
      s->done = 1;
    } else {
      s->alpha = s->rz / out[0];
    }
  }
}

// x += alpha p, r -= alpha q, ||r||^2, convergence test
__global__ void k_cg_xr(int64_t m, const double* __restrict__ p, const double* __restrict__ q,
                        double* __restrict__ x, double* __restrict__ r, CgState* s, double* partials,
                        unsigned* counter) {
  pdl_enter();
  if (s->done) return;
  const double alpha = s->alpha;
  double local[1] = {0.0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    x[t] = fma(alpha, p[t], x[t]);
    const double rv = fma(-alpha, q[t], r[t]);
    r[t] = rv;
    local[0] = fma(rv, rv, local[0]);
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) {
    s->rnorm2 = out[0];
    s->its += 1;
    if (!isfinite(out[0])) {
      s->breakdown = 1;
      s->done = 1;
    } else if (out[0] <= s->rtol2 * s->bnorm2) {
      s->converged = 1;
      s->done = 1;
    } else if (s->its >= s->maxit) {
      s->done = 1;
    }
  }
}

// beta = r.(z - z_old) / rz (Polak-Ribiere), rz = r.z
__global__ void k_cg_dots(int64_t m, const double* __restrict__ r, const double* __restrict__ z,
                          const double* __restrict__ zold, CgState* s, double* partials, unsigned* counter) {
  pdl_enter();
  if (s->done) return;
  double local[2] = {0.0, 0.0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const double rv = r[t];
    local[0] = fma(rv, z[t], local[0]);
    local[1] = fma(rv, zold[t], local[1]);
  }
  double out[2];
  if (grid_reduce<2>(local, partials, counter, out) && threadIdx.x == 0) {
    s->beta = (out[0] - out[1]) / s->rz;
    s->rz = out[0];
  }
}

// p = z + beta p, z_old = z
__global__ void k_cg_p(int64_t m, const double* __restrict__ z, double* __restrict__ p, double* __restrict__ zold,
                       const CgState* s) {
  pdl_enter();
  if (s->done) return;
  const double beta = s->beta;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const double zv = z[t];
    p[t] = fma(beta, p[t], zv);
    zold[t] = zv;
  }
}

// ||b - A x||^2 into s->pq (final true residual)
template <int V>
__global__ void __launch_bounds__(256, 8) k_true_residual(const int* __restrict__ sp, const int* __restrict__ col,
                                                               const double* __restrict__ vals,
                                                               const int* __restrict__ srow, int64_t n,
                                                               int64_t nthreads, const double* __restrict__ x,
                                                               const double* __restrict__ b, double* out_norm2,
                                                               double* partials, unsigned* counter) {
  pdl_enter();
  double local[1] = {0.0};
  const int64_t ntasks = (nthreads + 31) >> 5;
  int64_t t0, t1;
  deal_range(ntasks, t0, t1);
  for (int64_t g = t0 + (threadIdx.x >> 5); g < t1; g += blockDim.x >> 5) {
    const int64_t t = g * 32 + (threadIdx.x & 31);
    if (t >= nthreads) continue;  // rows are whole slices: never taken
    int64_t pos;
    int sub;
    row_of_thread<V>(t, pos, sub);
    double acc[3];
    row_product<3, 3, V, double, double, double>(sp, col, vals, x, pos, sub, acc);
    const int64_t i = row_at(srow, pos);
    if (sub == 0 && i >= 0 && i < n) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double t = b[i * 3 + a] - acc[a];
        local[0] = fma(t, t, local[0]);
      }
    }
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) *out_norm2 = out[0];
}

static unsigned vec_grid(int64_t m) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 1216)); }
// One CG iteration after the first preconditioner application.
static Status cg_iteration(bamg_mg* mg, double* r, double* z, cudaStream_t st) {
  bamg_ctx* ctx = mg->ctx;
  Level& L0 = mg->levels[0];
  const bamg_bsr* A = L0.A;
  const int64_t m = L0.n * 3, rows = row_threads(A);
  CgState* s = mg->cg;
  const int* done = &s->done;
  const int pa = prof_begin(ctx, BAMG_PROF_CG_AP, st);
  BAMG_DISPATCH_V(A->vec, { BAMG_CUDA(launch_k(k_cg_Ap<V>, dim3(deal_grid(k_cg_Ap<V>, ctx->sm_count, rows)), dim3(256), st, A->slice_ptr, A->sell_col, A->vals, A->slot_row, L0.n, rows, mg->cp, mg->cq, s,
                                                  ctx->d_partials, ctx->d_counters + 2)); BAMG_COUNT_LAUNCH; })
  prof_end(ctx, pa, st);
  const int px = prof_begin(ctx, BAMG_PROF_CG_XR, st);
  { BAMG_CUDA(launch_k(k_cg_xr, dim3(vec_grid(m)), dim3(256), st, m, mg->cp, mg->cq, mg->cx, r, s, ctx->d_partials, ctx->d_counters + 3)); BAMG_COUNT_LAUNCH; }
  prof_end(ctx, px, st);
  BAMG_TRY(precond(mg, r, z, done, st));
  const int pv = prof_begin(ctx, BAMG_PROF_CG_VECTOR, st);
  { BAMG_CUDA(launch_k(k_cg_dots, dim3(vec_grid(m)), dim3(256), st, m, r, z, mg->czold, s, ctx->d_partials, ctx->d_counters + 4)); BAMG_COUNT_LAUNCH; }
  { BAMG_CUDA(launch_k(k_cg_p, dim3(vec_grid(m)), dim3(256), st, m, z, mg->cp, mg->czold, s)); BAMG_COUNT_LAUNCH; }
  prof_end(ctx, pv, st);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

static void cg_graphs_release(bamg_mg* mg) {
  for (auto g : mg->cg_graphs)
    if (g) cudaGraphExecDestroy(g);
  mg->cg_graphs.clear();
  if (mg->cg_loop) cudaGraphExecDestroy(mg->cg_loop);
  mg->cg_loop = nullptr;
  for (auto& v : mg->cg_pairs)
    for (auto& q : v) {
      cudaEventDestroy(q.a);
      cudaEventDestroy(q.b);
    }
  mg->cg_pairs.clear();
  mg->cg_pairs_used.clear();
}

constexpr int kCgChunk = 4;  // iterations launched between convergence checks

// Condition of the device CG loop, set after the prologue (reset = 1) and at
// the end of every iteration: run another iteration while the solve is
// still going and fewer than maxit iterations have run (a bound that holds
// whatever the state says).
__global__ void k_cg_continue(CgState* s, int reset, cudaGraphConditionalHandle h) {
  const int l = reset ? 0 : s->loops + 1;
  s->loops = l;
  cudaGraphSetConditional(h, (!s->done && l < s->maxit) ? 1u : 0u);
}

static uint64_t graph_kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  uint64_t kn = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
  }
  return kn;
}

// The unprofiled solve's iterations as one graph: the loop decision, then a
// while node whose body is one CG iteration and the next decision.
static Status cg_loop_graph(bamg_mg* mg, double* r, double* z, cudaStream_t cs) {
  const auto mode = cudaStreamCaptureModeThreadLocal;
  cudaGraph_t G = nullptr;
  BAMG_CUDA(cudaGraphCreate(&G, 0));
  Status s;
  auto run = [&]() -> Status {
    cudaGraphConditionalHandle h;
    BAMG_CUDA(cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault));
    BAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, mode));
    k_cg_continue<<<1, 1, 0, cs>>>(mg->cg, 1, h);
    cudaError_t e = cudaGetLastError();
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd);
    std::vector<cudaGraphNode_t> last(deps, deps + nd);
    cudaGraph_t out = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &out);
    if (e != cudaSuccess) return cuda_status(e, "CG loop decision");
    if (ee != cudaSuccess) return cuda_status(ee, "CG loop capture");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond = nullptr;
    BAMG_CUDA(cudaGraphAddNode(&cond, G, last.data(), nullptr, last.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    BAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode));
    Status is = cg_iteration(mg, r, z, cs);
    if (is.ok()) {
      k_cg_continue<<<1, 1, 0, cs>>>(mg->cg, 0, h);
      e = cudaGetLastError();
      if (e != cudaSuccess) is = cuda_status(e, "CG loop decision");
    }
    const cudaError_t be = cudaStreamEndCapture(cs, &out);
    BAMG_TRY(is);
    if (be != cudaSuccess) return cuda_status(be, "CG loop body capture");
    mg->cg_loop_body_kernels = graph_kernel_nodes(body);
    BAMG_CUDA(cudaGraphInstantiate(&mg->cg_loop, G, 0));
    return Status{};
  };
  g_capturing = true;
  s = run();
  g_capturing = false;
  cudaGraphDestroy(G);
  if (!s.ok()) {
    if (mg->cg_loop) cudaGraphExecDestroy(mg->cg_loop);
    mg->cg_loop = nullptr;
  }
  return s;
}

// Capture one CG iteration into a graph; with profiling on, one graph per
// position in a chunk so that each owns its timing events.
static Status cg_graph(bamg_mg* mg, double* r, double* z) {
  bamg_ctx* ctx = mg->ctx;
  if ((!mg->cg_graphs.empty() || mg->cg_loop) && mg->cg_graph_epoch == ctx->prof.epoch) return Status{};
  cg_graphs_release(mg);
  const int ng = ctx->prof.on ? kCgChunk : 1;
  cudaStream_t cs = nullptr;
  BAMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  if (!ctx->prof.on) {
    const Status ls = cg_loop_graph(mg, r, z, cs);
    cudaStreamDestroy(cs);
    mg->cg_graph_epoch = ctx->prof.epoch;
    return ls;
  }
  mg->cg_pairs.resize(ng);
  mg->cg_pairs_used.assign(ng, 0);
  if (ctx->prof.on)
    for (auto& v : mg->cg_pairs) {
      v.resize(64);
      for (auto& q : v) {
        BAMG_CUDA(cudaEventCreate(&q.a));
        BAMG_CUDA(cudaEventCreate(&q.b));
      }
    }
  Status s;
  for (int p = 0; p < ng && s.ok(); ++p) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      s = cuda_status(e, "begin capture");
      break;
    }
    g_capturing = true;
    ctx->prof.sink = &mg->cg_pairs[p];
    ctx->prof.sink_used = 0;
    ctx->prof.pos = p;
    s = cg_iteration(mg, r, z, cs);
    mg->cg_pairs_used[p] = ctx->prof.sink_used;
    ctx->prof.sink = nullptr;
    ctx->prof.pos = 0;
    g_capturing = false;
    e = cudaStreamEndCapture(cs, &g);
    if (s.ok() && e != cudaSuccess) s = cuda_status(e, "end capture");
    if (s.ok()) {
      size_t nn = 0;
      cudaGraphGetNodes(g, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      cudaGraphGetNodes(g, nodes.data(), &nn);
      uint64_t kn = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
      }
      mg->cg_graph_kernels = kn;
      cudaGraphExec_t ex = nullptr;
      e = cudaGraphInstantiate(&ex, g, 0);
      if (e != cudaSuccess)
        s = cuda_status(e, "graph instantiate");
      else
        mg->cg_graphs.push_back(ex);
    }
    if (g) cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cs);
  if (!s.ok()) cg_graphs_release(mg);
  mg->cg_graph_epoch = ctx->prof.epoch;
  return s;
}

void mg_release_graphs(bamg_mg* mg) { cg_graphs_release(mg); }

// CG work vectors r and z: in the FP64 form the cycle reads its right-hand
// side and writes its result in place (level 0's b and x).
static double* cg_r(bamg_mg* mg) { return mg->opts.precision == BAMG_FP64 ? mg->levels[0].b : mg->cr; }
static double* cg_z(bamg_mg* mg) { return mg->opts.precision == BAMG_FP64 ? mg->levels[0].x : mg->cz; }

Status cg_prologue(bamg_mg* mg, const double* b, double rtol, int maxit, cudaStream_t st) {
  bamg_ctx* ctx = mg->ctx;
  const int64_t m = mg->levels[0].n * 3;
  double *r = cg_r(mg), *z = cg_z(mg);
  CgState* s = mg->cg;
  { BAMG_CUDA(launch_k(k_cg_setup, dim3(1), dim3(1), st, s, rtol, maxit)); BAMG_COUNT_LAUNCH; }
  { BAMG_CUDA(launch_k(k_cg_init, dim3(vec_grid(m)), dim3(256), st, m, b, r, mg->cx, s, ctx->d_partials, ctx->d_counters + 5)); BAMG_COUNT_LAUNCH; }
  BAMG_TRY(precond(mg, r, z, &s->done, st));
  { BAMG_CUDA(launch_k(k_cg_first, dim3(vec_grid(m)), dim3(256), st, m, r, z, mg->cp, mg->czold, s, ctx->d_partials, ctx->d_counters + 6)); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

Status cg_step(bamg_mg* mg, cudaStream_t st) { return cg_iteration(mg, cg_r(mg), cg_z(mg), st); }

Status cg_epilogue(bamg_mg* mg, const double* b, double* x, double* true_r2, cudaStream_t st) {
  bamg_ctx* ctx = mg->ctx;
  Level& L0 = mg->levels[0];
  const int64_t m = L0.n * 3;
  if (x) BAMG_CUDA(cudaMemcpyAsync(x, mg->cx, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  const bamg_bsr* A = L0.A;
  const int64_t rows = row_threads(A);
  BAMG_DISPATCH_V(A->vec, { BAMG_CUDA(launch_k(k_true_residual<V>, dim3(deal_grid(k_true_residual<V>, ctx->sm_count, rows)), dim3(256), st, A->slice_ptr, A->sell_col, A->vals, A->slot_row, L0.n, rows, mg->cx, b,
                                                          true_r2, ctx->d_partials, ctx->d_counters + 7)); BAMG_COUNT_LAUNCH; })
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

static Status cg_solve(bamg_mg* mg, const double* b, double* x, double rtol, int maxit, bamg_cg_info* info) {
  bamg_ctx* ctx = mg->ctx;
  cudaStream_t st = ctx->stream;
  CgState* s = mg->cg;
  BAMG_TRY(cg_graph(mg, cg_r(mg), cg_z(mg)));
  BAMG_TRY(cg_prologue(mg, b, rtol, maxit, st));
  const bool device_loop = mg->cg_loop != nullptr;
  if (device_loop) BAMG_CUDA(cudaGraphLaunch(mg->cg_loop, st));
  if (!device_loop) {
    BAMG_CUDA(cudaMemcpyAsync(mg->cg_host, s, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    BAMG_CUDA(cudaStreamSynchronize(st));
  }
  int launched = 0;
  int its_before = device_loop ? 0 : mg->cg_host->its;
  const int ng = (int)mg->cg_graphs.size();
  while (!device_loop && launched < maxit && !mg->cg_host->done) {
    const int c = std::min(kCgChunk, maxit - launched);
    for (int k = 0; k < c; ++k) {
      BAMG_CUDA(cudaGraphLaunch(mg->cg_graphs[k % ng], st));
      g_launches.fetch_add(mg->cg_graph_kernels, std::memory_order_relaxed);
    }
    launched += c;
    BAMG_CUDA(cudaMemcpyAsync(mg->cg_host, s, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    BAMG_CUDA(cudaStreamSynchronize(st));
    if (ng > 1) {
      const int its_now = mg->cg_host->its;
      const int active_ap = its_now - its_before;
      const int active_vc = active_ap - (mg->cg_host->done ? 1 : 0);
      for (int k = 0; k < c; ++k) prof_harvest(ctx, mg->cg_pairs[k], mg->cg_pairs_used[k], active_ap, active_vc);
      its_before = its_now;
    }
  }
  double* tr = mg->scal + (int64_t)mg->levels.size() * kScalarsPerLevel + 8;
  BAMG_TRY(cg_epilogue(mg, b, x, tr, st));
  double tr2 = 0.0;
  BAMG_CUDA(cudaMemcpyAsync(&tr2, tr, sizeof(double), cudaMemcpyDeviceToHost, st));
  BAMG_CUDA(cudaMemcpyAsync(mg->cg_host, s, sizeof(CgState), cudaMemcpyDeviceToHost, st));
  BAMG_TRY(check_device_error(ctx));
  const CgState& h = *mg->cg_host;
  if (device_loop)  // the loop's decisions and its bodies' kernels
    g_launches.fetch_add(1 + (uint64_t)h.loops * mg->cg_loop_body_kernels, std::memory_order_relaxed);
  if (info) {
    info->iterations = h.its;
    info->converged = h.converged;
    info->rnorm = sqrt(h.rnorm2);
    info->bnorm = sqrt(h.bnorm2);
    info->true_rnorm = sqrt(tr2);
  }
  if (h.breakdown) return make_status(BAMG_ERR_BREAKDOWN, "CG breakdown after %d iterations", h.its);
  if (!h.converged) return make_status(BAMG_ERR_NOT_CONVERGED, "CG did not converge in %d iterations", h.its);
  return Status{};
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_vcycle(bamg_mg* mg, const double* b, double* x) {
  if (!mg || !b || !x) return BAMG_ERR_INVALID;
  Status s = precond(mg, b, x, nullptr, mg->ctx->stream);
  return s.ok() ? BAMG_OK : fail(mg->ctx, s);
}

bamg_status bamg_cg_solve(bamg_mg* mg, const double* b, double* x, double rtol, int maxit, bamg_cg_info* info) {
  if (!mg || !b || maxit < 0 || !(rtol >= 0.0)) return BAMG_ERR_INVALID;
  Status s = cg_solve(mg, b, x, rtol, maxit, info);
  return s.ok() ? BAMG_OK : fail(mg->ctx, s);
}

}  // extern "C"
