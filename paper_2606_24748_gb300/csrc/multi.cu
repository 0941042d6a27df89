// Many right-hand sides at once: the V-cycle (Sec. 2.1) and PCG (Sec. 4.1)
// applied to k vectors in one pass over every operator, i.e. with blocked
// SpMM in place of SpMV.
//
// Vectors are stored RHS-minor: entry (dof d, vector j) at X[d * kp + j],
// with kp = the column count rounded up to a power of two >= 4 (padding
// columns are zero and frozen).  A thread owns one block row and four
// consecutive columns, so every block value and column index is loaded once
// for four products and the kp / 4 threads of a row share the load.
//
// The k CG recurrences are independent (own alpha, beta, stopping test and
// iteration count per column); they share only the passes over memory.  Per
// column, the V-cycle's arithmetic is the single-vector cycle's with one lane
// per block row, in the same order, so column j of a multi-vector cycle
// equals the single-vector cycle of column j when every operator runs one
// lane per row.
#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace bamg {

namespace {

#define BAMG_DONE_RETURN \
  if (done && *done) return;

template <int BS, typename T>
__device__ __forceinline__ void dinv_apply4(const T* __restrict__ dinv, int64_t i, const T (&r)[BS][4],
                                            T (&z)[4], int a) {
  const int64_t base = (i >> 5) * (32LL * BS * BS) + (i & 31);
#pragma unroll
  for (int e = 0; e < 4; ++e) z[e] = T(0);
#pragma unroll
  for (int c = 0; c < BS; ++c) {
    const T m = __ldg(dinv + base + 32 * (a * BS + c));
#pragma unroll
    for (int e = 0; e < 4; ++e) z[e] = fma(m, r[c][e], z[e]);
  }
}

// thread -> (block row i, first column c0) for kp = 4 << glog columns
__device__ __forceinline__ bool row_cols(int64_t n, int glog, int64_t& i, int& c0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (n << glog)) return false;
  i = t >> glog;
  c0 = (int)(t & ((1 << glog) - 1)) * 4;
  return true;
}

// r = b; d = w Dinv b / theta; x = 0
template <int BS, typename T>
__global__ void __launch_bounds__(256) k_mcheb_init(int64_t n, int glog, int kp, const T* __restrict__ b,
                                                    T* __restrict__ r, T* __restrict__ d, T* __restrict__ x,
                                                    const T* __restrict__ dinv, const float* __restrict__ w,
                                                    const double* __restrict__ scal, const int* done) {
  BAMG_DONE_RETURN
  int64_t i;
  int c0;
  if (!row_cols(n, glog, i, c0)) return;
  T bi[BS][4];
#pragma unroll
  for (int a = 0; a < BS; ++a) ld4(b + (i * BS + a) * kp + c0, bi[a]);
  const T f = (T)(scal[kInvTheta] * (w ? (double)w[i] : 1.0));
  const T zero[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    T z[4];
    dinv_apply4<BS, T>(dinv, i, bi, z, a);
#pragma unroll
    for (int e = 0; e < 4; ++e) z[e] = f * z[e];
    const int64_t o = (i * BS + a) * kp + c0;
    st4(r + o, bi[a]);
    st4(d + o, z);
    st4(x + o, zero);
  }
}

// x += d_in; r -= A d_in; if has_next: d_out = c1 d_in + c2 w Dinv r
template <int BS, typename T>
__global__ void __launch_bounds__(256) k_mcheb_step(const int* __restrict__ sp, const int* __restrict__ col,
                                                    const T* __restrict__ vals, const int* __restrict__ srow,
                                                    int64_t n, int glog, int kp,
                                                    const T* __restrict__ d_in, T* __restrict__ d_out,
                                                    T* __restrict__ x, T* __restrict__ r,
                                                    const T* __restrict__ dinv, const float* __restrict__ w,
                                                    const double* __restrict__ scal, int k, int has_next,
                                                    const int* done) {
  BAMG_DONE_RETURN
  int64_t pos;
  int c0;
  if (!row_cols(n, glog, pos, c0)) return;
  T acc[BS][4];
  row_product4<BS, BS, T>(sp, col, vals, d_in, kp, pos, c0, acc);
  const int64_t i = row_at(srow, pos);
  T di[BS][4];
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    const int64_t o = (i * BS + a) * kp + c0;
    T rv[4], xv[4];
    ld4(d_in + o, di[a]);
    ld4w(r + o, rv);
    ld4w(x + o, xv);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      acc[a][e] = rv[e] - acc[a][e];
      xv[e] += di[a][e];
    }
    st4(r + o, acc[a]);
    st4(x + o, xv);
  }
  if (has_next) {
    const T c1 = (T)scal[kCheb + 2 * k];
    const T c2 = (T)(scal[kCheb + 2 * k + 1] * (w ? (double)w[i] : 1.0));
#pragma unroll
    for (int a = 0; a < BS; ++a) {
      T z[4];
      dinv_apply4<BS, T>(dinv, i, acc, z, a);
#pragma unroll
      for (int e = 0; e < 4; ++e) z[e] = fma(c1, di[a][e], c2 * z[e]);
      st4(d_out + (i * BS + a) * kp + c0, z);
    }
  }
}

// r = b - A x; d = w Dinv r / theta
template <int BS, typename T>
__global__ void __launch_bounds__(256) k_mcheb_rinit(const int* __restrict__ sp, const int* __restrict__ col,
                                                     const T* __restrict__ vals, const int* __restrict__ srow,
                                                     int64_t n, int glog, int kp,
                                                     const T* __restrict__ x, const T* __restrict__ b,
                                                     T* __restrict__ r, T* __restrict__ d,
                                                     const T* __restrict__ dinv, const float* __restrict__ w,
                                                     const double* __restrict__ scal, const int* done) {
  BAMG_DONE_RETURN
  int64_t pos;
  int c0;
  if (!row_cols(n, glog, pos, c0)) return;
  T acc[BS][4];
  row_product4<BS, BS, T>(sp, col, vals, x, kp, pos, c0, acc);
  const int64_t i = row_at(srow, pos);
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    const int64_t o = (i * BS + a) * kp + c0;
    T bv[4];
    ld4(b + o, bv);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[a][e] = bv[e] - acc[a][e];
    st4(r + o, acc[a]);
  }
  const T f = (T)(scal[kInvTheta] * (w ? (double)w[i] : 1.0));
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    T z[4];
    dinv_apply4<BS, T>(dinv, i, acc, z, a);
#pragma unroll
    for (int e = 0; e < 4; ++e) z[e] = f * z[e];
    st4(d + (i * BS + a) * kp + c0, z);
  }
}

// y = M v, or y += M v
template <int BR, int BC, typename T>
__global__ void __launch_bounds__(256) k_mtransfer(const int* __restrict__ sp, const int* __restrict__ col,
                                                   const T* __restrict__ vals, const int* __restrict__ srow,
                                                   int64_t n, int glog, int kp, const T* __restrict__ v,
                                                   T* __restrict__ y, int accumulate, const int* done) {
  BAMG_DONE_RETURN
  int64_t pos;
  int c0;
  if (!row_cols(n, glog, pos, c0)) return;
  T acc[BR][4];
  row_product4<BR, BC, T>(sp, col, vals, v, kp, pos, c0, acc);
  const int64_t i = srow ? (int64_t)srow[pos] : pos;  // row position -> block row (sorted slices)
#pragma unroll
  for (int a = 0; a < BR; ++a) {
    const int64_t o = (i * BR + a) * kp + c0;
    if (accumulate) {
      T yv[4];
      ld4w(y + o, yv);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][e] = yv[e] + acc[a][e];
    }
    st4(y + o, acc[a]);
  }
}

template <typename T>
__global__ void k_maxpy(int64_t m, const T* __restrict__ d, T* __restrict__ x, const int* done) {
  BAMG_DONE_RETURN
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) x[t] += d[t];
}

template <typename TS, typename TD>
__global__ void k_mcast(int64_t m, const TS* __restrict__ s, TD* __restrict__ d, const int* done) {
  BAMG_DONE_RETURN
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) d[t] = (TD)s[t];
}

// dst[d * kp + j] = src[d * k + j] (j < k), 0 for the padding columns
template <typename TD>
__global__ void k_mpack(int64_t m, int k, int kp, const double* __restrict__ src, TD* __restrict__ dst) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m * kp) return;
  const int64_t d = t / kp;
  const int j = (int)(t - d * kp);
  dst[t] = j < k ? (TD)src[d * k + j] : TD(0);
}

template <typename TS>
__global__ void k_munpack(int64_t m, int k, int kp, const TS* __restrict__ src, double* __restrict__ dst) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m * k) return;
  const int64_t d = t / k;
  const int j = (int)(t - d * k);
  dst[t] = (double)src[d * kp + j];
}

// ----------------------------------------------------------------- CG kernels

__global__ void k_mcg_setup(CgMultiState* s, int k, int kp, double rtol, int maxit) {
  const int c = threadIdx.x;
  if (c < kMaxRhs) {
    s->bnorm2[c] = s->rnorm2[c] = s->rz[c] = s->alpha[c] = s->beta[c] = s->pq[c] = s->true_r2[c] = 0.0;
    s->its[c] = 0;
    s->done[c] = c >= k ? 1 : 0;
    s->converged[c] = 0;
    s->breakdown[c] = 0;
  }
  if (c == 0) {
    s->rtol2 = rtol * rtol;
    s->maxit = maxit;
    s->k = k;
    s->kp = kp;
    s->all_done = 0;
  }
}

// column of this thread in the element-wise kernels (grid stride and block
// size are multiples of kp)
__device__ __forceinline__ int my_col(int kp) { return (int)(threadIdx.x & (kp - 1)); }

__device__ __forceinline__ void update_all_done(CgMultiState* s, int kp) {
  const int c = threadIdx.x;
  const int all = __syncthreads_and(c >= kp || s->done[c]);
  if (c == 0) s->all_done = all;
}

// r = B (packed), x = 0, ||b_j||^2
__global__ void __launch_bounds__(256) k_mcg_init(int64_t m, int k, int kp, const double* __restrict__ B,
                                                  double* __restrict__ r, double* __restrict__ x, CgMultiState* s,
                                                  double* partials, unsigned* counter) {
  __shared__ double out[64];
  const int c = my_col(kp);
  double v[1] = {0.0};
  const int64_t mk = m * kp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < mk; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = t / kp;
    const double bv = c < k ? B[d * k + c] : 0.0;
    r[t] = bv;
    x[t] = 0.0;
    v[0] = fma(bv, bv, v[0]);
  }
  if (!grid_reduce_groups<1>(v, kp, partials, counter, out)) return;
  const int q = threadIdx.x;
  if (q < kp) {
    s->bnorm2[q] = out[q];
    s->rnorm2[q] = out[q];
    if (q < k && !(out[q] > 0.0)) {
      s->done[q] = 1;
      s->converged[q] = 1;
    }
  }
  update_all_done(s, kp);
}

// p = z, z_old = z, rz = r.z
__global__ void __launch_bounds__(256) k_mcg_first(int64_t m, int kp, const double* __restrict__ r,
                                                   const double* __restrict__ z, double* __restrict__ p,
                                                   double* __restrict__ zold, CgMultiState* s, double* partials,
                                                   unsigned* counter) {
  if (s->all_done) return;
  __shared__ double out[64];
  double v[1] = {0.0};
  const int64_t mk = m * kp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < mk; t += (int64_t)gridDim.x * blockDim.x) {
    const double zv = z[t];
    p[t] = zv;
    zold[t] = zv;
    v[0] = fma(r[t], zv, v[0]);
  }
  if (!grid_reduce_groups<1>(v, kp, partials, counter, out)) return;
  if ((int)threadIdx.x < kp) s->rz[threadIdx.x] = out[threadIdx.x];
}

// q = A p, alpha_j = rz_j / (p_j . q_j)
__global__ void __launch_bounds__(256) k_mcg_Ap(const int* __restrict__ sp, const int* __restrict__ col,
                                                const double* __restrict__ vals, const int* __restrict__ srow,
                                                int64_t n, int glog, int kp,
                                                const double* __restrict__ p, double* __restrict__ q,
                                                CgMultiState* s, double* partials, unsigned* counter) {
  if (s->all_done) return;
  __shared__ double out[64];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t nt = n << glog;
  const int c0 = (int)(threadIdx.x & ((1 << glog) - 1)) * 4;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = t >> glog;
    double acc[3][4];
    row_product4<3, 3, double>(sp, col, vals, p, kp, pos, c0, acc);
    const int64_t i = row_at(srow, pos);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int64_t o = (i * 3 + a) * kp + c0;
      double pv[4];
      ld4(p + o, pv);
      st4(q + o, acc[a]);
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = fma(pv[e], acc[a][e], v[e]);
    }
  }
  if (!grid_reduce_groups<4>(v, kp >> 2, partials, counter, out)) return;
  const int c = threadIdx.x;
  if (c < kp && !s->done[c]) {
    s->pq[c] = out[c];
    if (!(out[c] > 0.0)) {
      s->breakdown[c] = 1;
      s->done[c] = 1;
    } else {
      s->alpha[c] = s->rz[c] / out[c];
    }
  }
  update_all_done(s, kp);
}

// x += alpha p, r -= alpha q (active columns), ||r_j||^2, stopping tests
__global__ void __launch_bounds__(256) k_mcg_xr(int64_t m, int kp, const double* __restrict__ p,
                                                const double* __restrict__ q, double* __restrict__ x,
                                                double* __restrict__ r, CgMultiState* s, double* partials,
                                                unsigned* counter) {
  if (s->all_done) return;
  __shared__ double out[64];
  const int c = my_col(kp);
  const bool active = !s->done[c];
  const double alpha = s->alpha[c];
  double v[1] = {0.0};
  const int64_t mk = m * kp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < mk; t += (int64_t)gridDim.x * blockDim.x) {
    double rv = r[t];
    if (active) {
      x[t] = fma(alpha, p[t], x[t]);
      rv = fma(-alpha, q[t], rv);
      r[t] = rv;
    }
    v[0] = fma(rv, rv, v[0]);
  }
  if (!grid_reduce_groups<1>(v, kp, partials, counter, out)) return;
  const int j = threadIdx.x;
  if (j < kp && !s->done[j]) {
    const double rn = out[j];
    s->rnorm2[j] = rn;
    s->its[j] += 1;
    if (!isfinite(rn)) {
      s->breakdown[j] = 1;
      s->done[j] = 1;
    } else if (rn <= s->rtol2 * s->bnorm2[j]) {
      s->converged[j] = 1;
      s->done[j] = 1;
    } else if (s->its[j] >= s->maxit) {
      s->done[j] = 1;
    }
  }
  update_all_done(s, kp);
}

// beta_j = r_j.(z_j - zold_j) / rz_j (Polak-Ribiere), rz_j = r_j.z_j
__global__ void __launch_bounds__(256) k_mcg_dots(int64_t m, int kp, const double* __restrict__ r,
                                                  const double* __restrict__ z, const double* __restrict__ zold,
                                                  CgMultiState* s, double* partials, unsigned* counter) {
  if (s->all_done) return;
  __shared__ double out[64];
  double v[2] = {0.0, 0.0};
  const int64_t mk = m * kp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < mk; t += (int64_t)gridDim.x * blockDim.x) {
    const double rv = r[t];
    v[0] = fma(rv, z[t], v[0]);
    v[1] = fma(rv, zold[t], v[1]);
  }
  if (!grid_reduce_groups<2>(v, kp, partials, counter, out)) return;
  const int j = threadIdx.x;
  if (j < kp && !s->done[j]) {
    s->beta[j] = (out[2 * j] - out[2 * j + 1]) / s->rz[j];
    s->rz[j] = out[2 * j];
  }
}

// p = z + beta p, z_old = z (active columns)
__global__ void __launch_bounds__(256) k_mcg_p(int64_t m, int kp, const double* __restrict__ z,
                                               double* __restrict__ p, double* __restrict__ zold,
                                               const CgMultiState* s) {
  if (s->all_done) return;
  const int c = my_col(kp);
  if (s->done[c]) return;
  const double beta = s->beta[c];
  const int64_t mk = m * kp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < mk; t += (int64_t)gridDim.x * blockDim.x) {
    const double zv = z[t];
    p[t] = fma(beta, p[t], zv);
    zold[t] = zv;
  }
}

// ||b_j - A x_j||^2 (b read from the caller's k-column array)
__global__ void __launch_bounds__(256) k_mcg_true_residual(const int* __restrict__ sp, const int* __restrict__ col,
                                                           const double* __restrict__ vals,
                                                           const int* __restrict__ srow, int64_t n, int glog,
                                                           int kp, int k, const double* __restrict__ x,
                                                           const double* __restrict__ B, CgMultiState* s,
                                                           double* partials, unsigned* counter) {
  __shared__ double out[64];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t nt = n << glog;
  const int c0 = (int)(threadIdx.x & ((1 << glog) - 1)) * 4;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = t >> glog;
    double acc[3][4];
    row_product4<3, 3, double>(sp, col, vals, x, kp, pos, c0, acc);
    const int64_t i = row_at(srow, pos);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = c0 + e;
        const double bv = j < k ? B[(i * 3 + a) * k + j] : 0.0;
        const double d = bv - acc[a][e];
        v[e] = fma(d, d, v[e]);
      }
  }
  if (!grid_reduce_groups<4>(v, kp >> 2, partials, counter, out)) return;
  if ((int)threadIdx.x < kp) s->true_r2[threadIdx.x] = out[threadIdx.x];
}

// ------------------------------------------------------------------ host side

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

unsigned grid_for(int64_t threads, int per_block = 256) {
  return (unsigned)std::max<int64_t>(1, (threads + per_block - 1) / per_block);
}
unsigned stride_grid(int64_t threads) { return (unsigned)std::min<int64_t>(grid_for(threads), 1216); }

template <typename T>
struct MPtrs {
  T *b, *x, *r, *d0, *d1;
  const T *dinv, *Avals, *Pvals, *Rvals;
};
template <typename T>
MPtrs<T> mptrs(Level& L, MultiLevel& W) {
  const bool f = sizeof(T) == 4;
  auto pick = [&](const bamg_bsr* M) -> const T* {
    if (!M) return nullptr;
    return f ? (const T*)(const void*)M->vals32 : (const T*)(const void*)M->vals;
  };
  return {(T*)W.b, (T*)W.x, (T*)W.r, (T*)W.d0, (T*)W.d1,
          f ? (const T*)(const void*)L.dinv32 : (const T*)(const void*)L.dinv, pick(L.A), pick(L.P), pick(L.R)};
}

template <int BS, typename T>
Status msmooth_down(bamg_mg* mg, int l, int kp, const int* done, cudaStream_t st) {
  Level& L = mg->levels[l];
  auto p = mptrs<T>(L, mg->multi->lv[l]);
  const bamg_bsr* A = L.A;
  const int glog = ilog2(kp / 4);
  const unsigned g = grid_for(L.n << glog);
  const double* sc = mg->scal + (int64_t)l * kScalarsPerLevel;
  const int m = mg->opts.cheb_degree;
  { k_mcheb_init<BS, T><<<g, 256, 0, st>>>(L.n, glog, kp, p.b, p.r, p.d0, p.x, p.dinv, L.weights, sc, done); BAMG_COUNT_LAUNCH; }
  T* d[2] = {p.d0, p.d1};
  for (int k = 0; k < m; ++k) {
    k_mcheb_step<BS, T><<<g, 256, 0, st>>>(A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, glog, kp, d[k & 1], d[(k + 1) & 1],
                                           p.x, p.r, p.dinv, L.weights, sc, k, k + 1 < m ? 1 : 0, done);
    BAMG_COUNT_LAUNCH;
  }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <int BS, typename T>
Status msmooth_up(bamg_mg* mg, int l, int kp, const int* done, cudaStream_t st) {
  Level& L = mg->levels[l];
  auto p = mptrs<T>(L, mg->multi->lv[l]);
  const bamg_bsr* A = L.A;
  const int glog = ilog2(kp / 4);
  const unsigned g = grid_for(L.n << glog);
  const double* sc = mg->scal + (int64_t)l * kScalarsPerLevel;
  const int m = mg->opts.cheb_degree;
  { k_mcheb_rinit<BS, T><<<g, 256, 0, st>>>(A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, glog, kp, p.x, p.b, p.r, p.d0,
                                            p.dinv, L.weights, sc, done); BAMG_COUNT_LAUNCH; }
  T* d[2] = {p.d0, p.d1};
  for (int k = 0; k + 1 < m; ++k) {
    k_mcheb_step<BS, T><<<g, 256, 0, st>>>(A->slice_ptr, A->sell_col, p.Avals, A->slot_row, L.n, glog, kp, d[k & 1], d[(k + 1) & 1],
                                           p.x, p.r, p.dinv, L.weights, sc, k, 1, done);
    BAMG_COUNT_LAUNCH;
  }
  const int64_t mm = L.n * BS * kp;
  { k_maxpy<T><<<grid_for(mm), 256, 0, st>>>(mm, d[(m - 1) & 1], p.x, done); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <int BR, int BC, typename T>
Status mtransfer(const bamg_bsr* M, const T* vals, const T* v, T* y, int kp, int accumulate, const int* done,
                 cudaStream_t st) {
  if (M->nbr == 0) return Status{};
  const int glog = ilog2(kp / 4);
  { k_mtransfer<BR, BC, T><<<grid_for(M->nbr << glog), 256, 0, st>>>(M->slice_ptr, M->sell_col, vals, M->slot_row,
                                                                  M->nbr, glog, kp, v, y, accumulate, done); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <typename T>
Status mcoarse(bamg_mg* mg, int kp, const T* b, T* x, const int* done, cudaStream_t st) {
  return coarse_apply_multi<T>(mg, kp, b, x, mg->multi->coarse_y, done, st);
}

// level 0 block right-hand side -> level 0 block iterate
template <typename T>
Status mvcycle(bamg_mg* mg, int kp, const int* done, cudaStream_t st) {
  const int nl = (int)mg->levels.size();
  MultiWork& W = *mg->multi;
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = mg->levels[l];
    auto p = mptrs<T>(L, W.lv[l]);
    auto pc = mptrs<T>(mg->levels[l + 1], W.lv[l + 1]);
    if (L.bs == 3) {
      BAMG_TRY((msmooth_down<3, T>(mg, l, kp, done, st)));
      BAMG_TRY((mtransfer<6, 3, T>(L.R, p.Rvals, p.r, pc.b, kp, 0, done, st)));
    } else {
      BAMG_TRY((msmooth_down<6, T>(mg, l, kp, done, st)));
      BAMG_TRY((mtransfer<6, 6, T>(L.R, p.Rvals, p.r, pc.b, kp, 0, done, st)));
    }
  }
  {
    auto p = mptrs<T>(mg->levels[nl - 1], W.lv[nl - 1]);
    BAMG_TRY(mcoarse<T>(mg, kp, p.b, p.x, done, st));
  }
  for (int l = nl - 2; l >= 0; --l) {
    Level& L = mg->levels[l];
    auto p = mptrs<T>(L, W.lv[l]);
    auto pc = mptrs<T>(mg->levels[l + 1], W.lv[l + 1]);
    if (L.bs == 3) {
      BAMG_TRY((mtransfer<3, 6, T>(L.P, p.Pvals, pc.x, p.x, kp, 1, done, st)));
      BAMG_TRY((msmooth_up<3, T>(mg, l, kp, done, st)));
    } else {
      BAMG_TRY((mtransfer<6, 6, T>(L.P, p.Pvals, pc.x, p.x, kp, 1, done, st)));
      BAMG_TRY((msmooth_up<6, T>(mg, l, kp, done, st)));
    }
  }
  return Status{};
}

bool mixed(const bamg_mg* mg) { return mg->opts.precision == BAMG_FP32; }

// z = M r for kp-column FP64 arrays (r, z may be the level 0 arrays of the
// FP64 form, in which case nothing is copied)
Status mprecond(bamg_mg* mg, int kp, const double* r, double* z, const int* done, cudaStream_t st) {
  MultiWork& W = *mg->multi;
  Level& L0 = mg->levels[0];
  const int64_t m = L0.n * L0.bs * kp;
  const unsigned g = grid_for(m);
  if (mixed(mg)) {
    { k_mcast<double, float><<<g, 256, 0, st>>>(m, r, (float*)W.lv[0].b, done); BAMG_COUNT_LAUNCH; }
    BAMG_TRY(mvcycle<float>(mg, kp, done, st));
    { k_mcast<float, double><<<g, 256, 0, st>>>(m, (const float*)W.lv[0].x, z, done); BAMG_COUNT_LAUNCH; }
  } else {
    if (r != W.lv[0].b) { k_mcast<double, double><<<g, 256, 0, st>>>(m, r, (double*)W.lv[0].b, done); BAMG_COUNT_LAUNCH; }
    BAMG_TRY(mvcycle<double>(mg, kp, done, st));
    if (z != W.lv[0].x) { k_mcast<double, double><<<g, 256, 0, st>>>(m, (const double*)W.lv[0].x, z, done); BAMG_COUNT_LAUNCH; }
  }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

void release_graph(MultiWork& W) {
  if (W.graph) cudaGraphExecDestroy(W.graph);
  W.graph = nullptr;
  W.graph_kernels = 0;
}

void release_arrays(MultiWork& W, cudaStream_t st) {
  release_graph(W);
  for (auto& v : W.lv)
    for (void** p : {&v.b, &v.x, &v.r, &v.d0, &v.d1}) {
      if (*p) cudaFreeAsync(*p, st);
      *p = nullptr;
    }
  W.lv.clear();
  dfree(W.coarse_y, st);
  for (double** p : {&W.cx, &W.cp, &W.cq, &W.czold}) dfree(*p, st);
  if (W.own_rz) {
    dfree(W.cr, st);
    dfree(W.cz, st);
  }
  W.cr = W.cz = nullptr;
  W.own_rz = false;
  W.kp = 0;
}

// Work arrays for kp columns (kept while a call needs no more columns).
Status prepare(bamg_mg* mg, int kp) {
  cudaStream_t st = mg->ctx->stream;
  if (!mg->multi) mg->multi = new MultiWork();
  MultiWork& W = *mg->multi;
  if (!W.st) {
    BAMG_TRY(dalloc(&W.st, 1, st));
    BAMG_CUDA(cudaMallocHost(&W.host, sizeof(CgMultiState)));
    BAMG_TRY(dalloc(&W.partials, 1216 * 64, st));
    BAMG_TRY(dalloc(&W.counters, 8, st));
    BAMG_CUDA(cudaMemsetAsync(W.counters, 0, 8 * sizeof(unsigned), st));
  }
  if (W.kp >= kp) return Status{};
  release_arrays(W, st);
  const bool f32 = mixed(mg);
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const int nl = (int)mg->levels.size();
  W.lv.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const Level& L = mg->levels[l];
    const size_t bytes = (size_t)L.n * L.bs * kp * es;
    MultiLevel& v = W.lv[l];
    const bool coarsest = l == nl - 1;
    for (void** p : {&v.b, &v.x, &v.r, &v.d0, &v.d1}) {
      if (coarsest && (p == &v.r || p == &v.d0 || p == &v.d1)) continue;
      if (bytes == 0) continue;
      cudaError_t e = cudaMallocAsync(p, bytes, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        release_arrays(W, st);
        return make_status(BAMG_ERR_OOM, "multi-vector work arrays (%zu bytes) do not fit", bytes);
      }
    }
  }
  const int64_t m = mg->levels[0].n * 3 * (int64_t)kp;
  BAMG_TRY(dalloc(&W.coarse_y, 2 * mg->coarse.npad * kp, st));
  for (double** p : {&W.cx, &W.cp, &W.cq, &W.czold}) BAMG_TRY(dalloc(p, m, st));
  if (f32) {
    BAMG_TRY(dalloc(&W.cr, m, st));
    BAMG_TRY(dalloc(&W.cz, m, st));
    W.own_rz = true;
  } else {
    W.cr = (double*)W.lv[0].b;
    W.cz = (double*)W.lv[0].x;
    W.own_rz = false;
  }
  for (const MultiLevel& v : W.lv)
    for (const void* p : {v.b, v.x, v.r, v.d0, v.d1})
      if ((uintptr_t)p % 32 != 0) {
        release_arrays(W, st);
        return make_status(BAMG_ERR_CUDA, "work array not aligned to 32 bytes");
      }
  for (const double* p : {W.cx, W.cp, W.cq, W.czold, W.cr, W.cz})
    if ((uintptr_t)p % 32 != 0) {
      release_arrays(W, st);
      return make_status(BAMG_ERR_CUDA, "work array not aligned to 32 bytes");
    }
  W.kp = kp;
  return Status{};
}

int padded_columns(int k) {
  int kp = 4;
  while (kp < k) kp <<= 1;
  return kp;
}

Status check_multi(bamg_mg* mg, int k) {
  if (k < 1 || k > kMaxRhs) return make_status(BAMG_ERR_INVALID, "column count %d outside 1..%d", k, kMaxRhs);
  if (mg->levels.empty() || mg->levels[0].bs != 3)
    return make_status(BAMG_ERR_STATE, "the hierarchy has no 3x3-block fine level");
  if (!mg->coarse.factored) return make_status(BAMG_ERR_STATE, "the hierarchy has not been updated");
  return Status{};
}

Status multi_vcycle(bamg_mg* mg, const double* B, double* X, int k) {
  BAMG_TRY(check_multi(mg, k));
  const int kp = padded_columns(k);
  BAMG_TRY(prepare(mg, kp));
  MultiWork& W = *mg->multi;
  cudaStream_t st = mg->ctx->stream;
  const int64_t m = mg->levels[0].n * 3;
  if (mixed(mg)) {
    { k_mpack<float><<<grid_for(m * kp), 256, 0, st>>>(m, k, kp, B, (float*)W.lv[0].b); BAMG_COUNT_LAUNCH; }
    BAMG_TRY(mvcycle<float>(mg, kp, nullptr, st));
    { k_munpack<float><<<grid_for(m * k), 256, 0, st>>>(m, k, kp, (const float*)W.lv[0].x, X); BAMG_COUNT_LAUNCH; }
  } else {
    { k_mpack<double><<<grid_for(m * kp), 256, 0, st>>>(m, k, kp, B, (double*)W.lv[0].b); BAMG_COUNT_LAUNCH; }
    BAMG_TRY(mvcycle<double>(mg, kp, nullptr, st));
    { k_munpack<double><<<grid_for(m * k), 256, 0, st>>>(m, k, kp, (const double*)W.lv[0].x, X); BAMG_COUNT_LAUNCH; }
  }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

// One multi-vector CG iteration after the first preconditioner application.
Status mcg_iteration(bamg_mg* mg, int kp, cudaStream_t st) {
  MultiWork& W = *mg->multi;
  Level& L0 = mg->levels[0];
  const bamg_bsr* A = L0.A;
  const int64_t m = L0.n * 3;
  const int glog = ilog2(kp / 4);
  CgMultiState* s = W.st;
  const int* done = &s->all_done;
  { k_mcg_Ap<<<stride_grid(L0.n << glog), 256, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, A->slot_row, L0.n, glog, kp, W.cp, W.cq,
                                                       s, W.partials, W.counters + 0); BAMG_COUNT_LAUNCH; }
  { k_mcg_xr<<<stride_grid(m * kp), 256, 0, st>>>(m, kp, W.cp, W.cq, W.cx, W.cr, s, W.partials, W.counters + 1); BAMG_COUNT_LAUNCH; }
  BAMG_TRY(mprecond(mg, kp, W.cr, W.cz, done, st));
  { k_mcg_dots<<<stride_grid(m * kp), 256, 0, st>>>(m, kp, W.cr, W.cz, W.czold, s, W.partials, W.counters + 2); BAMG_COUNT_LAUNCH; }
  { k_mcg_p<<<stride_grid(m * kp), 256, 0, st>>>(m, kp, W.cz, W.cp, W.czold, s); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

// One iteration captured as a graph (rebuilt when the column count changes).
Status mcg_graph(bamg_mg* mg, int kp) {
  MultiWork& W = *mg->multi;
  if (W.graph) return Status{};
  cudaStream_t cs = nullptr;
  BAMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  Status s;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_status(e, "begin capture");
  }
  g_capturing = true;
  s = mcg_iteration(mg, kp, cs);
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
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
      s = cuda_status(e, "graph instantiate");
    } else {
      W.graph = ex;
      W.graph_kernels = kn;
      W.graph_kp = kp;
    }
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  return s;
}

constexpr int kChunk = 4;  // iterations launched between convergence checks

Status multi_cg(bamg_mg* mg, const double* B, double* X, int k, double rtol, int maxit, bamg_cg_info* info) {
  BAMG_TRY(check_multi(mg, k));
  const int kp = padded_columns(k);
  BAMG_TRY(prepare(mg, kp));
  MultiWork& W = *mg->multi;
  if (W.graph && W.graph_kp != kp) release_graph(W);  // the graph bakes in the column count
  bamg_ctx* ctx = mg->ctx;
  cudaStream_t st = ctx->stream;
  Level& L0 = mg->levels[0];
  const bamg_bsr* A = L0.A;
  const int64_t m = L0.n * 3;
  const int glog = ilog2(kp / 4);
  CgMultiState* s = W.st;
  BAMG_TRY(mcg_graph(mg, kp));
  { k_mcg_setup<<<1, 32, 0, st>>>(s, k, kp, rtol, maxit); BAMG_COUNT_LAUNCH; }
  { k_mcg_init<<<stride_grid(m * kp), 256, 0, st>>>(m, k, kp, B, W.cr, W.cx, s, W.partials, W.counters + 3); BAMG_COUNT_LAUNCH; }
  BAMG_TRY(mprecond(mg, kp, W.cr, W.cz, &s->all_done, st));
  { k_mcg_first<<<stride_grid(m * kp), 256, 0, st>>>(m, kp, W.cr, W.cz, W.cp, W.czold, s, W.partials, W.counters + 4); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  BAMG_CUDA(cudaMemcpyAsync(W.host, s, sizeof(CgMultiState), cudaMemcpyDeviceToHost, st));
  BAMG_CUDA(cudaStreamSynchronize(st));
  int launched = 0;
  while (launched < maxit && !W.host->all_done) {
    const int c = std::min(kChunk, maxit - launched);
    for (int q = 0; q < c; ++q) {
      BAMG_CUDA(cudaGraphLaunch(W.graph, st));
      g_launches.fetch_add(W.graph_kernels, std::memory_order_relaxed);
    }
    launched += c;
    BAMG_CUDA(cudaMemcpyAsync(W.host, s, sizeof(CgMultiState), cudaMemcpyDeviceToHost, st));
    BAMG_CUDA(cudaStreamSynchronize(st));
  }
  if (X) { k_munpack<double><<<grid_for(m * k), 256, 0, st>>>(m, k, kp, W.cx, X); BAMG_COUNT_LAUNCH; }
  { k_mcg_true_residual<<<stride_grid(L0.n << glog), 256, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, A->slot_row, L0.n, glog, kp, k,
                                                                  W.cx, B, s, W.partials, W.counters + 5); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaMemcpyAsync(W.host, s, sizeof(CgMultiState), cudaMemcpyDeviceToHost, st));
  BAMG_TRY(check_device_error(ctx));
  const CgMultiState& h = *W.host;
  int not_conv = -1, broke = -1;
  for (int j = 0; j < k; ++j) {
    if (info) {
      info[j].iterations = h.its[j];
      info[j].converged = h.converged[j];
      info[j].rnorm = sqrt(h.rnorm2[j]);
      info[j].bnorm = sqrt(h.bnorm2[j]);
      info[j].true_rnorm = sqrt(h.true_r2[j]);
    }
    if (h.breakdown[j] && broke < 0) broke = j;
    if (!h.converged[j] && not_conv < 0) not_conv = j;
  }
  if (broke >= 0) return make_status(BAMG_ERR_BREAKDOWN, "CG breakdown in column %d after %d iterations", broke, h.its[broke]);
  if (not_conv >= 0)
    return make_status(BAMG_ERR_NOT_CONVERGED, "CG column %d did not converge in %d iterations", not_conv, h.its[not_conv]);
  return Status{};
}

}  // namespace

void mg_release_multi(bamg_mg* mg) {
  if (!mg->multi) return;
  cudaStream_t st = mg->ctx->stream;
  MultiWork& W = *mg->multi;
  release_arrays(W, st);
  dfree(W.st, st);
  dfree(W.partials, st);
  dfree(W.counters, st);
  if (W.host) cudaFreeHost(W.host);
  delete mg->multi;
  mg->multi = nullptr;
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_mg_vcycle_multi(bamg_mg* mg, const double* B, double* X, int k) {
  if (!mg || !B || !X) return BAMG_ERR_INVALID;
  Status s = multi_vcycle(mg, B, X, k);
  return s.ok() ? BAMG_OK : fail(mg->ctx, s);
}

bamg_status bamg_cg_solve_multi(bamg_mg* mg, const double* B, double* X, int k, double rtol, int maxit,
                                bamg_cg_info* info) {
  if (!mg || !B || maxit < 0 || !(rtol >= 0.0)) return BAMG_ERR_INVALID;
  Status s = multi_cg(mg, B, X, k, rtol, maxit, info);
  return s.ok() ? BAMG_OK : fail(mg->ctx, s);
}

}  // extern "C"
