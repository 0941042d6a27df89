// Exact coarsest-level solve.  Dense form: FP64 Cholesky A = L L^T, then the
// explicit inverse factor W = L^-1, so every V-cycle applies x = W^T (W b) as
// two dense triangular matrix-vector products spread over the whole GPU
// instead of two sequential substitutions.  The matrix is padded to a
// multiple of the 32-wide tiles with an identity block (which factors to
// itself).  Banded form (below): block-tridiagonal Cholesky over chunks of
// the band, used when the level's half-bandwidth is small against its size.
//
// Tiled right-looking algorithms, one kernel per tile step:
//   Cholesky   for k: factor tile (k,k); L(i,k) = A(i,k) L(k,k)^-T; A(i,j) -= L(i,k) L(j,k)^T
//   W = L^-1   for i: W(i,k) = L(i,i)^-1 (delta_ik I - S(i,k)), k <= i;  S(r,k) += L(r,i) W(i,k), r > i
#include <cooperative_groups.h>

#include <algorithm>
#include <array>

#include "device.cuh"
#include "internal.h"

namespace bamg {

constexpr int kT = 32;  // tile size
constexpr int kFactorCounters = 32;  // two context counters: quarter updates done, per matrix

template <typename TM, int BS>
__global__ void k_dense_fill(int64_t nnzb, const int* __restrict__ rowptr_rows, const int* __restrict__ colidx,
                             const int* __restrict__ slot_of, const TM* __restrict__ vals, double* __restrict__ M,
                             int64_t ld) {
  constexpr int B = BS * BS;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * B) return;
  const int64_t k = t / B;
  const int e = (int)(t - k * B);
  const int r = e / BS, c = e - r * BS;
  const int64_t I = rowptr_rows[k], J = colidx[k];
  M[(I * BS + r) * ld + J * BS + c] = (double)vals[vidx<B>(slot_of[k], e)];
}

__global__ void k_dense_init(double* __restrict__ M, int64_t n, int64_t npad) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npad * npad) return;
  const int64_t i = t / npad, j = t - i * npad;
  M[t] = (i == j && i >= n) ? 1.0 : 0.0;
}

// Tile GEMM update C -= A B^T (trailing Cholesky update) or C += A B (inverse
// accumulation), 256 threads, 4 outputs each.
template <bool kSyrk>
__device__ __forceinline__ void tile_update(double* __restrict__ C, const double* __restrict__ Ab,
                                            const double* __restrict__ Bb, int64_t ld, double (*As)[kT + 1],
                                            double (*Bs)[kT + 1]) {
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) {
    As[e / kT][e % kT] = Ab[(int64_t)(e / kT) * ld + e % kT];
    Bs[e / kT][e % kT] = Bb[(int64_t)(e / kT) * ld + e % kT];
  }
  __syncthreads();
  const int c = tid % kT, r0 = tid / kT;  // rows r0, r0+8, r0+16, r0+24
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 8
  for (int l = 0; l < kT; ++l) {
    const double b = kSyrk ? Bs[c][l] : Bs[l][c];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(As[r0 + 8 * q][l], b, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double* p = C + (int64_t)(r0 + 8 * q) * ld + c;
    *p = kSyrk ? *p - acc[q] : *p + acc[q];
  }
}

// Rows [r0, r0 + 8) of C -= A A^T for a 32 x 32 tile C and a 32 x 32 tile A
// (one quarter of a diagonal-tile update; 256 threads, one output each).
__device__ __forceinline__ void tile_syrk_rows8(double* __restrict__ C, const double* __restrict__ Ab, int64_t ld,
                                                int r0, double (*As)[kT + 1], double (*Bs)[kT + 1]) {
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) Bs[e / kT][e % kT] = Ab[(int64_t)(e / kT) * ld + e % kT];
  __syncthreads();
  const int r = tid / kT, c = tid % kT;
  double acc = 0.0;
#pragma unroll 8
  for (int l = 0; l < kT; ++l) acc = fma(Bs[r0 + r][l], Bs[c][l], acc);
  C[(int64_t)(r0 + r) * ld + c] -= acc;
}

// 1 / sqrt(d) by Newton's method for the reciprocal square root,
// y <- y + y (1 - d y^2) / 2, from the single-precision estimate; each step
// doubles the correct bits (about 22 -> 44 -> full double precision).
__device__ __forceinline__ double rsqrt_newton(double d) {
  const float f = (float)d;
  double y = (f > 1e-30f && f < 1e30f) ? (double)rsqrtf(f) : 1.0 / sqrt(d);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double e = fma(-d * y, y, 1.0);
    y = fma(0.5 * y, e, y);
  }
  return y;
}

// 1 / d from the hardware's double-precision estimate (PTX rcp.approx.ftz.f64,
// about 20 correct bits) and one third-order step of the iteration for the
// reciprocal: with e = 1 - d y, y (1 + e + e^2) has relative error about e^3.
// Three dependent FP64 operations: at 64 cycles each on this part, the pivot
// chain of a factorisation is the critical path, and a float seed costs two
// conversions more.
__device__ __forceinline__ double rcp_cubic(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// d > 0 and finite, tested on the bits (an FP64 compare is another 64 cycles).
__device__ __forceinline__ bool positive_finite(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0 && b < 0x7ff0000000000000LL;
}

// Lower-triangle entries (i, l), i >= l, of a tile, ordered by l descending:
// the entries right of column j are the first (kT-1-j)(kT-j)/2.  Packed as
// i << 5 | l; built once per CTA.
__device__ void tri_table(unsigned short* tri) {
  for (int p = threadIdx.x; p < kT * (kT + 1) / 2; p += blockDim.x) {
    int l = kT - 1;
    while (l > 0 && (kT - l) * (kT + 1 - l) / 2 <= p) --l;
    tri[p] = (unsigned short)((l + p - (kT - 1 - l) * (kT - l) / 2) << 5 | l);
  }
}

// Cholesky of the diagonal tile (k, k) in shared memory and the inverse of
// the factor (one CTA); L is written back, L^-1 to Linv.  The sweep is the
// square-root-free form A = Lu D Lu^T: column j's pivot d_j = a_jj, then
// a_il -= a_ij a_lj / d_j for l > j, one barrier per column, and every
// thread forms 1 / d_j itself.  Column j is left unscaled (a_ij = Lu_ij d_j),
// so L = Lu D^(1/2) is a_ij / sqrt(d_j) at the end: the square roots leave the
// serial chain.
__device__ void diag_tile(double* __restrict__ M, int64_t ld, int k, double* __restrict__ Linv, int* err,
                          double (*a)[kT + 1], double (*w)[kT + 1], const unsigned short* tri) {
  __shared__ double inv[kT];
  const int tid = threadIdx.x;
  double* base = M + (int64_t)k * kT * ld + (int64_t)k * kT;
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) a[e / kT][e % kT] = __ldcg(base + (int64_t)(e / kT) * ld + e % kT);
  __syncthreads();
  for (int j = 0; j < kT; ++j) {
    double d = a[j][j];
    if (!positive_finite(d)) d = 1.0;  // reported below
    const double r = rcp_cubic(d);
    const int cnt = (kT - 1 - j) * (kT - j) / 2;
    for (int p = tid; p < cnt; p += blockDim.x) {
      const int code = tri[p], i = code >> 5, l = code & 31;
      a[i][l] = fma(-a[i][j] * r, a[l][j], a[i][l]);
    }
    __syncthreads();
  }
  if (tid < kT) {
    double d = a[tid][tid];
    if (!positive_finite(d)) {
      set_err(err, kDevBreakdown);
      d = 1.0;
    }
    inv[tid] = rsqrt_newton(d);
  }
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) {
    const int i = e / kT, l = e % kT;
    if (l <= i) a[i][l] *= inv[l];
  }
  // W = L^-1 by doubling the inverted diagonal blocks: with diagonal blocks
  // W11, W22 of size h already inverted, the block below them is
  // W21 = -W22 L21 W11, formed for every pair at once (two products, 2 h^3
  // multiply-adds per pair) for h = 1, 2, 4, 8, 16.  T = L21 W11 is kept
  // transposed in the (unused) upper triangle of the pair's block.
  if (tid < kT) w[tid][tid] = inv[tid];
  __syncthreads();
  for (int h = 1; h < kT; h *= 2) {
    const int hh = h * h;
    for (int e = tid; e < (kT / 2) * h; e += blockDim.x) {  // (kT / 2h) pairs x h^2 entries
      const int i0 = (e / hh) * 2 * h, m = (e % hh) / h, q = e % h;
      double t = 0.0;
      for (int n = q; n < h; ++n) t = fma(a[i0 + h + m][i0 + n], w[i0 + n][i0 + q], t);
      w[i0 + q][i0 + h + m] = t;
    }
    __syncthreads();
    for (int e = tid; e < (kT / 2) * h; e += blockDim.x) {
      const int i0 = (e / hh) * 2 * h, p = (e % hh) / h, q = e % h;
      double t = 0.0;
      for (int m = 0; m <= p; ++m) t = fma(w[i0 + h + p][i0 + h + m], w[i0 + q][i0 + h + m], t);
      w[i0 + h + p][i0 + q] = -t;
    }
    __syncthreads();
  }
  for (int e = tid; e < kT * kT; e += blockDim.x) {
    const int i = e / kT, l = e % kT;
    base[(int64_t)i * ld + l] = l <= i ? a[i][l] : 0.0;
    Linv[e] = l <= i ? w[i][l] : 0.0;
  }
}

// Rows [r0, r0 + 8) of X = A Linv^T (Cholesky panel), in place over A.
__device__ void panel_rows(double* __restrict__ Xt, int64_t ld, const double* __restrict__ Linv, int r0,
                           double (*a)[kT + 1], double (*w)[kT + 1]) {
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) w[e / kT][e % kT] = Linv[e];
  for (int e = tid; e < 8 * kT; e += blockDim.x) a[e / kT][e % kT] = Xt[(int64_t)(r0 + e / kT) * ld + e % kT];
  __syncthreads();
  const int r = tid / kT, c = tid % kT;  // 8 x 32 outputs
  double t = 0.0;
#pragma unroll 8
  for (int l = 0; l < kT; ++l) t = fma(a[r][l], w[c][l], t);
  Xt[(int64_t)(r0 + r) * ld + c] = t;
}

// Columns [c0, c0 + 8) of W(i,k) = Linv (delta I - S), in place over S.
__device__ void winv_cols(double* __restrict__ St, int64_t ld, const double* __restrict__ Linv, int c0, bool diag,
                          double (*a)[kT + 1], double (*w)[kT + 1]) {
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) w[e / kT][e % kT] = Linv[e];
  for (int e = tid; e < kT * 8; e += blockDim.x) {
    const int r = e / 8, c = e % 8;
    a[r][c] = ((diag && r == c0 + c) ? 1.0 : 0.0) - St[(int64_t)r * ld + c0 + c];
  }
  __syncthreads();
  const int r = tid / 8, c = tid % 8;  // 32 x 8 outputs
  double t = 0.0;
#pragma unroll 8
  for (int l = 0; l < kT; ++l) t = fma(w[r][l], a[l][c], t);
  St[(int64_t)r * ld + c0 + c] = t;
}

// Whole coarsest factorisation in one cooperative launch (256 threads per
// CTA; every CTA runs the same sequence of grid barriers).  One sweep over the
// 32-wide tile columns k computes the Cholesky factor L and W = L^-1 together:
//   phase 1:  L(i,k) = A(i,k) L(k,k)^-T, i > k            (panel, row stripes)
//             W(k,j) = L(k,k)^-1 (delta_kj I - S(k,j)), j <= k   (column stripes)
//   phase 2:  A(i,j) -= L(i,k) L(j,k)^T, k < j <= i         (trailing update)
//             S(r,j) += L(r,k) W(k,j), r > k, j <= k         (S accumulated in W)
//             CTA 0 first updates tile (k+1,k+1), then factors and inverts it
// so each step needs two barriers, and the inverse's updates fill the SMs
// that the shrinking trailing matrix leaves idle.
__global__ void __launch_bounds__(256) k_dense_factor(double* F, double* W, int64_t ld, int nt, double* Dinv,
                                                      int* err, double* F2, double* W2, double* Dinv2,
                                                      unsigned* qctr, int64_t wait_limit) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  __shared__ double a[kT][kT + 1], w[kT][kT + 1];
  __shared__ unsigned short tri[kT * (kT + 1) / 2];
  tri_table(tri);
  // With a second matrix (F2 != null) the two factorisations run side by side
  // on the two halves of the grid, in step with the same barriers.
  const int nm = F2 ? 2 : 1;
  const int G = (int)gridDim.x / nm;
  const int mi = (int)blockIdx.x / G;
  const bool idle = mi >= nm;  // an odd grid's last CTA only takes part in the barriers
  const int b = idle ? (1 << 30) : (int)blockIdx.x - mi * G;
  if (mi == 1) {
    F = F2;
    W = W2;
    Dinv = Dinv2;
  }
  if (b == 0) diag_tile(F, ld, 0, Dinv, err, a, w, tri);
  __threadfence();
  grid.sync();
  for (int k = 0; k < nt; ++k) {
    const double* Lkk_inv = Dinv + (int64_t)k * kT * kT;
    // phase 1
    const int n_panel = (nt - k - 1) * 4, n_winv = (k + 1) * 4;
    for (int item = b; item < n_panel + n_winv; item += G) {
      if (item < n_panel) {
        const int i = k + 1 + item / 4;
        panel_rows(F + (int64_t)i * kT * ld + (int64_t)k * kT, ld, Lkk_inv, (item % 4) * 8, a, w);
      } else {
        const int it = item - n_panel, j = it / 4;
        winv_cols(W + (int64_t)k * kT * ld + (int64_t)j * kT, ld, Lkk_inv, (it % 4) * 8, j == k, a, w);
      }
    }
    __threadfence();
    grid.sync();
    // phase 2: items 0-3 are the four 8-row quarters of the next diagonal
    // tile's update (CTAs 1-4 take them first and count them in qctr), then
    // the rest of the trailing update and the inverse's updates; CTA 0 waits
    // for the quarters and factors that tile meanwhile.
    const int T = nt - k - 1;
    const int n_trail = T * (T + 1) / 2, n_wupd = T * (k + 1);
    const int n_items = T > 0 ? 4 + (n_trail - 1) + n_wupd : 0;
    if (b == 0 && T > 0) {
      const int g = k + 1;
      if (threadIdx.x == 0) {
        // bounded: after wait_limit polls (about 0.4 s at the default of
        // 2^22) record a timeout and go on rather than wait forever; every
        // CTA still reaches the next grid barrier
        const unsigned target = 4u * (unsigned)(k + 1);
        for (int64_t polls = 0;; ++polls) {
          if (polls >= wait_limit) {
            set_err(err, kDevTimeout);
            break;
          }
          if (atomicAdd(qctr + mi, 0u) >= target) break;
          __nanosleep(64);
        }
        __threadfence();
      }
      __syncthreads();
      diag_tile(F, ld, g, Dinv + (int64_t)g * kT * kT, err, a, w, tri);
    }
    for (int item = b - 1; b > 0 && item < n_items; item += G - 1) {
      if (item < 4) {
        const int g = k + 1;
        tile_syrk_rows8(F + (int64_t)g * kT * ld + (int64_t)g * kT, F + (int64_t)g * kT * ld + (int64_t)k * kT, ld,
                        item * 8, a, w);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(qctr + mi, 1u);
        continue;
      }
      const int it0 = item - 4 + 1;  // trailing item 0 is the diagonal tile, done above in quarters
      if (it0 < n_trail) {
        int idx = it0, i = 0;
        while (idx > i) {  // row-major lower triangle (i, j), j <= i
          idx -= i + 1;
          ++i;
        }
        const int gi = k + 1 + i, gj = k + 1 + idx;
        tile_update<true>(F + (int64_t)gi * kT * ld + (int64_t)gj * kT,
                          F + (int64_t)gi * kT * ld + (int64_t)k * kT, F + (int64_t)gj * kT * ld + (int64_t)k * kT,
                          ld, a, w);
      } else {
        const int it = it0 - n_trail;
        const int r = k + 1 + it / (k + 1), j = it % (k + 1);
        tile_update<false>(W + (int64_t)r * kT * ld + (int64_t)j * kT, F + (int64_t)r * kT * ld + (int64_t)k * kT,
                           W + (int64_t)k * kT * ld + (int64_t)j * kT, ld, a, w);
      }
    }
    __threadfence();
    grid.sync();
  }
}

__global__ void k_transpose_dense(const double* __restrict__ S, double* __restrict__ D, int64_t n) {
  __shared__ double t[kT][kT + 1];
  const int64_t bi = blockIdx.y * kT, bj = blockIdx.x * kT;
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) t[e / kT][e % kT] = S[(bi + e / kT) * n + bj + e % kT];
  __syncthreads();
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) D[(bj + e / kT) * n + bi + e % kT] = t[e % kT][e / kT];
}

// y_i = sum_{j<=i} W[i][j] b_j (warp per row); x_j = sum_{i>=j} Wt[j][i] y_i.
template <typename TI, typename TO>
__global__ void k_tri_mv(const double* __restrict__ Wm, int64_t ld, int64_t n, const TI* __restrict__ v,
                         TO* __restrict__ out, int lower, const int* done) {
  pdl_enter();
  if (done && *done) return;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const int64_t j0 = lower ? 0 : row, j1 = lower ? row + 1 : n;
  const double* w = Wm + row * ld;
  double acc = 0.0;
  for (int64_t j = j0 + lane; j < j1; j += 32) acc = fma(w[j], (double)v[j], acc);
  acc = warp_sum(acc);
  if (lane == 0) out[row] = (TO)acc;
}

// The same for KP vectors stored RHS-minor (v[j * KP + c]).
template <int KP, typename TI, typename TO>
__global__ void k_tri_mm(const double* __restrict__ Wm, int64_t ld, int64_t n, const TI* __restrict__ v,
                         TO* __restrict__ out, int lower, const int* done) {
  pdl_enter();
  if (done && *done) return;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const int64_t j0 = lower ? 0 : row, j1 = lower ? row + 1 : n;
  const double* wr = Wm + row * ld;
  double acc[KP];
#pragma unroll
  for (int c = 0; c < KP; ++c) acc[c] = 0.0;
  for (int64_t j = j0 + lane; j < j1; j += 32) {
    const double wv = wr[j];
    const TI* vj = v + j * KP;
#pragma unroll
    for (int c = 0; c < KP; ++c) acc[c] = fma(wv, (double)vj[c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < KP; ++c) acc[c] = warp_sum(acc[c]);
#pragma unroll
  for (int c = 0; c < KP; ++c)
    if (lane == c) out[row * KP + c] = (TO)acc[c];
}

// ------------------------------------------------------------ banded form
//
// With nodes numbered lexicographically the coarsest operator is banded: a
// half-bandwidth of b dofs (27-point block stencil on an m^3 node grid:
// b = 6 (m^2 + m + 2) - 1).  Split into chunks of s >= b rows (a multiple of
// 32) it is block tridiagonal, and its Cholesky factor is block bidiagonal
// with no fill outside the band:
//   S_0 = A_00;  S_k = A_kk - L_{k,k-1} L_{k,k-1}^T
//   L_kk = chol(S_k);  L_{k+1,k} = A_{k+1,k} L_kk^-T
// which costs about nc (s^3 / 6 + 2 s^3) multiply-adds instead of n^3 / 3 for
// the dense factor and its inverse.  The chain of chunk factorisations is
// serial, so it is run from both ends at once ("twisted" block
// factorisation): chunks 0 .. t-1 are eliminated downward as above, chunks
// nc-1 .. t+1 upward,
//   R_{nc-1} = A_{nc-1,nc-1};  R_k = A_kk - C_{k+1} C_{k+1}^T,
//   Lt_k = chol(R_k);  C_k = A_{k-1,k} Lt_k^-T,
// the two sides in lock step (one cooperative launch factors both chunks of
// a round), and the middle chunk t takes both Schur complements:
// S_t = A_tt - B_{t-1} B_{t-1}^T - C_{t+1} C_{t+1}^T.  With W_k the inverse
// of each chunk's factor, M_k = W_k B_{k-1} (top and middle), Mt_k = W_k C_{k+1}
// (bottom and middle), N_k = W_k^T B_k^T (top) and Nt_k = W_k^T C_k^T
// (bottom), the solve is
//   y = blockdiag(W) b;  y_k -= M_k y_{k-1} (top, downward);
//   y_k -= Mt_k y_{k+1} (bottom, upward);  y_t -= M_t y_{t-1} + Mt_t y_{t+1};
//   x = blockdiag(W^T) y;  x_k -= N_k x_{k+1} (top, from t down);
//   x_k -= Nt_k x_{k-1} (bottom, from t up),
// two block-diagonal products and about nc chained rounds in each
// direction, each round one launch for both sides.

// Up to kGemmBatch products C = beta C + alpha A op(B) of s x s row-major
// matrices, op(B) = B or B^T, one per blockIdx.z; one 32 x 32 output tile per
// CTA (256 threads, 4 outputs each); with lower_only, tiles above the
// diagonal are skipped.
constexpr int kGemmBatch = 8;
constexpr int kGemmSplit = 8;  // at most this many K parts per output tile
// tri: which operand is triangular, so that whole zero tiles of the K loop
// are skipped: 0 none, 1 A lower (K tiles <= ti), 2 A upper (>= ti),
// 3 op(B) upper, i.e. B lower and transposed (<= tj).
enum GemmTri : int { kTriNone = 0, kTriALower = 1, kTriAUpper = 2, kTriBtUpper = 3 };
struct GemmBatch {
  double* C[kGemmBatch];
  const double* A[kGemmBatch];
  const double* B[kGemmBatch];
  int tri[kGemmBatch];
};

// Split K (ksplit > 1, blockIdx.z = item * ksplit + part): each part sums
// its share of the K tiles into a partial tile in `part`; the part that
// arrives last at the tile's counter (an atomic count, no waiting) adds the
// partials in part order, writes C and zeroes the counter for the next
// launch.  The order of the sums is fixed, so results are reproducible.  A
// chunk product has 66 to 242 output tiles for 152 SMs; the split fills them.
template <bool kTransB>
__global__ void __launch_bounds__(256) k_chunk_gemm(GemmBatch g, int s, double alpha, double beta, int lower_only,
                                                    int ksplit, double* __restrict__ part, unsigned* __restrict__ ctr) {
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (lower_only && tj > ti) return;
  const int item = (int)blockIdx.z / ksplit, kp = (int)blockIdx.z - item * ksplit;
  double* __restrict__ C = g.C[item];
  const double* __restrict__ A = g.A[item];
  const double* __restrict__ B = g.B[item];
  __shared__ double As[kT][kT + 1], Bs[kT][kT + 1];
  __shared__ unsigned last;
  const int tid = threadIdx.x, c = tid % kT, r0 = tid / kT;
  const int tri = g.tri[item];
  const int kb = tri == kTriAUpper ? ti : 0;
  const int ke = tri == kTriALower ? ti + 1 : (tri == kTriBtUpper ? tj + 1 : s / kT);
  const int len = (ke - kb + ksplit - 1) / ksplit;
  const int k0 = kb + kp * len, k1 = min(ke, k0 + len);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int kt = k0; kt < k1; ++kt) {
    __syncthreads();
    for (int e = tid; e < kT * kT; e += blockDim.x) {
      const int i = e / kT, j = e % kT;
      As[i][j] = A[(int64_t)(ti * kT + i) * s + kt * kT + j];
      Bs[i][j] = kTransB ? B[(int64_t)(tj * kT + i) * s + kt * kT + j] : B[(int64_t)(kt * kT + i) * s + tj * kT + j];
    }
    __syncthreads();
#pragma unroll 8
    for (int l = 0; l < kT; ++l) {
      const double bv = kTransB ? Bs[c][l] : Bs[l][c];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(As[r0 + 8 * q][l], bv, acc[q]);
    }
  }
  if (ksplit > 1) {
    const int ntl = s / kT;
    const int64_t tile = ((int64_t)item * ntl + ti) * ntl + tj;
    double* mine = part + ((int64_t)item * ksplit + kp) * ntl * ntl * (kT * kT) + ((int64_t)ti * ntl + tj) * (kT * kT);
#pragma unroll
    for (int q = 0; q < 4; ++q) mine[(r0 + 8 * q) * kT + c] = acc[q];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(ctr + tile, 1u) == (unsigned)(ksplit - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double t = 0.0;
      for (int pp = 0; pp < ksplit; ++pp) {
        const double* pt = part + ((int64_t)item * ksplit + pp) * ntl * ntl * (kT * kT) + ((int64_t)ti * ntl + tj) * (kT * kT);
        t += __ldcg(pt + (r0 + 8 * q) * kT + c);
      }
      acc[q] = t;
    }
    if (tid == 0) ctr[tile] = 0u;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double* p = C + (int64_t)(ti * kT + r0 + 8 * q) * s + tj * kT + c;
    *p = (beta == 0.0 ? 0.0 : beta * *p) + alpha * acc[q];
  }
}

// Diagonal and subdiagonal chunks from the stored blocks (upper chunks are
// the transposes, not stored); rows past n get an identity diagonal.
template <typename TM, int BS>
__global__ void k_band_fill(int64_t nnzb, const int* __restrict__ rows, const int* __restrict__ colidx,
                            const int* __restrict__ slot_of, const TM* __restrict__ vals, double* __restrict__ D,
                            double* __restrict__ Sub, double* __restrict__ Sup, int s, int* err) {
  constexpr int B = BS * BS;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * B) return;
  const int64_t k = t / B;
  const int e = (int)(t - k * B);
  const int64_t i = (int64_t)rows[k] * BS + e / BS, j = (int64_t)colidx[k] * BS + e % BS;
  const int64_t ci = i / s, cj = j / s, ri = i - ci * s, rj = j - cj * s;
  const double v = (double)vals[vidx<B>(slot_of[k], e)];
  if (ci == cj)
    D[(ci * s + ri) * s + rj] = v;
  else if (ci == cj + 1)
    Sub[(cj * s + ri) * s + rj] = v;
  else if (ci + 1 == cj)
    Sup[(ci * s + ri) * s + rj] = v;
  else if (v != 0.0)
    set_err(err, kDevIndex);  // outside the band the chunks were sized for
}

__global__ void k_band_pad(double* __restrict__ D, int64_t n, int64_t npad, int s) {
  const int64_t i = n + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npad) return;
  const int64_t c = i / s, r = i - c * s;
  D[(c * s + r) * s + r] = 1.0;
}

// Chunk matrix-vector products, kChainSplit warps per row: each warp takes
// every kChainSplit-th group of 32 columns, and the partial sums meet in
// shared memory in warp order.  Every product here is latency-bound (one
// 352 x 352 chunk is 124 K multiply-adds for the whole GPU); splitting the
// row shortens each warp's chain of dependent FP64 adds (64 cycles each) and
// spreads the rows over more SMs.
constexpr int kChainSplit = 4;
constexpr int kChainRows = 8 / kChainSplit;  // rows per 256-thread CTA

// Sum of the kChainSplit warps' totals for KP vectors (acc: each warp's lane
// values); the result is valid in threads sub == 0, lane < KP of each row.
template <int KP>
__device__ __forceinline__ void chain_combine(double (&acc)[KP], double (*part)[KP]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < KP; ++q) acc[q] = warp_sum(acc[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < KP; ++q) part[w][q] = acc[q];
  }
  __syncthreads();
  if (w % kChainSplit == 0 && lane < KP) {
    const int w0 = w;
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kChainSplit; ++k) t += part[w0 + k][lane];
    acc[0] = t;
  }
}

// out[k s + r] = sum_j M_k[r][j] v[k s + j] for every chunk k (rows of v at
// or past nvalid read as 0), KP vectors; tri = 1: M_k lower triangular
// (j <= r), 2: upper (j >= r), 0: full.
template <int KP, typename TI>
__global__ void __launch_bounds__(256) k_chunk_mv(const double* __restrict__ Mats, int s, int64_t rows,
                                                  const TI* __restrict__ v, int64_t nvalid,
                                                  double* __restrict__ out, int tri, const int* done) {
  pdl_enter();
  if (done && *done) return;
  __shared__ double part[8][KP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = w % kChainSplit;
  const int64_t row = (int64_t)blockIdx.x * kChainRows + w / kChainSplit;
  double acc[KP];
#pragma unroll
  for (int c = 0; c < KP; ++c) acc[c] = 0.0;
  if (row < rows) {
    const int64_t k = row / s, r = row - k * s;
    const double* mr = Mats + (k * s + r) * s;
    const int64_t g0 = k * s;
    const int j0 = tri == 2 ? (int)r : 0, j1 = tri == 1 ? (int)r + 1 : s;
    const int jend = (int)std::min<int64_t>(j1, nvalid - g0);
    for (int j = j0 + sub * 32 + lane; j < jend; j += 32 * kChainSplit) {
      const double wv = mr[j];
#pragma unroll
      for (int c = 0; c < KP; ++c) acc[c] = fma(wv, (double)v[(g0 + j) * KP + c], acc[c]);
    }
  }
  chain_combine<KP>(acc, part);
  if (row < rows && sub == 0 && lane < KP) out[row * KP + lane] = acc[0];
}

// One round of the solve chains: up to two jobs (blockIdx.y), each
// y[r] -= M1 z1 + M2 z2 over one chunk (s rows; M2 may be null), KP vectors.
struct ChainRound {
  const double* M1[2];
  const double* z1[2];
  const double* M2[2];
  const double* z2[2];
  double* y[2];
};

template <int KP>
__global__ void __launch_bounds__(256) k_chunk_chain(ChainRound c, int s, const int* done) {
  pdl_enter();
  if (done && *done) return;
  __shared__ double part[8][KP];
  const int job = blockIdx.y;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = w % kChainSplit;
  const int64_t r = (int64_t)blockIdx.x * kChainRows + w / kChainSplit;
  double acc[KP];
#pragma unroll
  for (int q = 0; q < KP; ++q) acc[q] = 0.0;
  if (r < s) {
    for (int term = 0; term < 2; ++term) {
      const double* M = term == 0 ? c.M1[job] : c.M2[job];
      const double* z = term == 0 ? c.z1[job] : c.z2[job];
      if (!M) continue;
      const double* mr = M + r * s;
      for (int j = sub * 32 + lane; j < s; j += 32 * kChainSplit) {
        const double wv = mr[j];
#pragma unroll
        for (int q = 0; q < KP; ++q) acc[q] = fma(wv, z[(int64_t)j * KP + q], acc[q]);
      }
    }
  }
  chain_combine<KP>(acc, part);
  if (r < s && sub == 0 && lane < KP) c.y[job][r * KP + lane] -= acc[0];
}

template <typename TO>
__global__ void k_band_out(int64_t m, const double* __restrict__ x, TO* __restrict__ out, const int* done) {
  pdl_enter();
  if (done && *done) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) out[t] = (TO)x[t];
}

static unsigned chain_grid(int64_t rows) { return (unsigned)std::max<int64_t>(1, (rows + kChainRows - 1) / kChainRows); }

// Half-bandwidth of the coarsest operator in dofs.
static int64_t half_bandwidth(const bamg_bsr* A) {
  int64_t b = 0;
  for (int64_t I = 0; I < A->nbr; ++I)
    for (int k = A->h_rowptr[I]; k < A->h_rowptr[I + 1]; ++k) b = std::max<int64_t>(b, std::llabs(A->h_colidx[k] - I));
  return (b + 1) * A->br - 1;
}

static Status cooperative_factor(bamg_ctx* ctx, cudaStream_t st, double* F, double* W, int64_t ld, int ntl,
                                 double* dt, double* F2 = nullptr, double* W2 = nullptr, double* dt2 = nullptr) {
  int per_sm = 0;
  BAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_factor, 256, 0));
  if (per_sm < 1) return make_status(BAMG_ERR_CUDA, "dense factor kernel cannot be resident");
  // one CTA per SM: a factor step has at most a few tile items per CTA of
  // this grid, and the launch must fit beside the smoother refresh that runs
  // concurrently on the other stream (all its CTAs resident at once)
  const int grid = ctx->sm_count;
  (void)per_sm;
  if (grid / (F2 ? 2 : 1) < 5) return make_status(BAMG_ERR_CUDA, "dense factor needs at least five CTAs per matrix");
  int* err = ctx->d_err;
  unsigned* qctr = ctx->d_counters + kFactorCounters;
  BAMG_CUDA(cudaMemsetAsync(qctr, 0, 2 * sizeof(unsigned), st));
  int64_t wait_limit = ctx->wait_limit;
  void* args[] = {&F, &W, &ld, &ntl, &dt, &err, &F2, &W2, &dt2, &qctr, &wait_limit};
  BAMG_CUDA(cudaLaunchCooperativeKernel((void*)k_dense_factor, grid, 256, args, 0, st));
  BAMG_COUNT_LAUNCH;
  return Status{};
}

struct GemmItem {
  double* C;
  const double* A;
  const double* B;
  int tri;
};

template <bool kTransB>
static Status gemm_batch(const std::vector<GemmItem>& items, int s, double alpha, double beta, int lower_only,
                         const CoarseDense& D, int sm_count, cudaStream_t st) {
  const int ntl = s / kT;
  for (size_t i0 = 0; i0 < items.size(); i0 += kGemmBatch) {
    GemmBatch g = {};
    const int cnt = (int)std::min<size_t>(kGemmBatch, items.size() - i0);
    for (int q = 0; q < cnt; ++q) {
      g.C[q] = items[i0 + q].C;
      g.A[q] = items[i0 + q].A;
      g.B[q] = items[i0 + q].B;
      g.tri[q] = items[i0 + q].tri;
    }
    // about four CTAs per SM: split K when the output tiles alone are fewer
    const int tiles = cnt * (lower_only ? ntl * (ntl + 1) / 2 : ntl * ntl);
    const int ksplit = std::min(kGemmSplit, std::max(1, (4 * sm_count + tiles - 1) / tiles));
    const dim3 grid((unsigned)ntl, (unsigned)ntl, (unsigned)(cnt * ksplit));
    k_chunk_gemm<kTransB><<<grid, 256, 0, st>>>(g, s, alpha, beta, lower_only, ksplit, D.gpart, D.gctr);
    BAMG_COUNT_LAUNCH;
  }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

// Twisted block factorisation of the banded coarsest operator (see above).
static Status band_factor(bamg_mg* mg, cudaStream_t st) {
  bamg_ctx* ctx = mg->ctx;
  Level& C = mg->levels.back();
  CoarseDense& D = mg->coarse;
  const bamg_bsr* A = C.A;
  const int bs = C.bs, s = D.s, nc = D.nc, t = nc / 2;
  const int64_t n = D.n, npad = D.npad, ss = (int64_t)s * s;
  const int ntl = s / kT;
  if (!D.D) {
    for (double** p : {&D.D, &D.Wb, &D.Wtb, &D.Mb, &D.Nb, &D.Mtb, &D.Ntb, &D.Bb}) BAMG_TRY(dalloc(p, nc * ss, st));
    for (double** p : {&D.Sub, &D.Sup}) BAMG_TRY(dalloc(p, std::max(1, nc - 1) * ss, st));
    BAMG_TRY(dalloc(&D.b64, npad, st));
    BAMG_TRY(dalloc(&D.x64, npad, st));
    BAMG_TRY(dalloc(&D.dinv_tiles, 2 * (int64_t)ntl * kT * kT, st));
    BAMG_TRY(dalloc(&D.gpart, (int64_t)kGemmBatch * kGemmSplit * ntl * ntl * kT * kT, st));
    BAMG_TRY(dalloc(&D.gctr, (int64_t)kGemmBatch * ntl * ntl, st));
    BAMG_CUDA(cudaMemsetAsync(D.gctr, 0, sizeof(unsigned) * kGemmBatch * ntl * ntl, st));
  }
  auto Dk = [&](int k) { return D.D + k * ss; };
  auto Wk = [&](int k) { return D.Wb + k * ss; };
  auto Wt = [&](int k) { return D.Wtb + k * ss; };
  auto BC = [&](int k) { return D.Bb + k * ss; };  // B_k (k < t) or C_k (k > t)
  double* dt1 = D.dinv_tiles + (int64_t)ntl * kT * kT;
  const int pm = prof_begin(ctx, BAMG_PROF_COARSE_FACTOR, st);
  BAMG_CUDA(cudaMemsetAsync(D.D, 0, sizeof(double) * nc * ss, st));
  BAMG_CUDA(cudaMemsetAsync(D.Sub, 0, sizeof(double) * std::max(1, nc - 1) * ss, st));
  BAMG_CUDA(cudaMemsetAsync(D.Sup, 0, sizeof(double) * std::max(1, nc - 1) * ss, st));
  BAMG_CUDA(cudaMemsetAsync(D.Wb, 0, sizeof(double) * nc * ss, st));
  if (npad > n) { k_band_pad<<<(unsigned)((npad - n + 255) / 256), 256, 0, st>>>(D.D, n, npad, s); BAMG_COUNT_LAUNCH; }
  const int64_t nt_fill = A->nnzb * bs * bs;
  if (nt_fill > 0) {
    const unsigned b = (unsigned)((nt_fill + 255) / 256);
    const bool f32 = A->vals64_stale;
    if (bs == 6) {
      if (f32) { k_band_fill<float, 6><<<b, 256, 0, st>>>(A->nnzb, D.rows, A->colidx, A->slot_of, A->vals32, D.D, D.Sub, D.Sup, s, ctx->d_err); BAMG_COUNT_LAUNCH; }
      else { k_band_fill<double, 6><<<b, 256, 0, st>>>(A->nnzb, D.rows, A->colidx, A->slot_of, A->vals, D.D, D.Sub, D.Sup, s, ctx->d_err); BAMG_COUNT_LAUNCH; }
    } else {
      if (f32) { k_band_fill<float, 3><<<b, 256, 0, st>>>(A->nnzb, D.rows, A->colidx, A->slot_of, A->vals32, D.D, D.Sub, D.Sup, s, ctx->d_err); BAMG_COUNT_LAUNCH; }
      else { k_band_fill<double, 3><<<b, 256, 0, st>>>(A->nnzb, D.rows, A->colidx, A->slot_of, A->vals, D.D, D.Sub, D.Sup, s, ctx->d_err); BAMG_COUNT_LAUNCH; }
    }
  }
  const dim3 tg((unsigned)ntl, (unsigned)ntl);
  // rounds: top chunk r (r < t) and bottom chunk nc-1-r (> t), side by side
  const int rounds = std::max(t, nc - 1 - t);
  for (int r = 0; r < rounds; ++r) {
    const int kt = r < t ? r : -1;
    const int kb = (nc - 1 - r > t) ? nc - 1 - r : -1;
    std::vector<GemmItem> syrk, panel;
    if (kt > 0) syrk.push_back({Dk(kt), BC(kt - 1), BC(kt - 1), kTriNone});
    if (kb >= 0 && kb < nc - 1) syrk.push_back({Dk(kb), BC(kb + 1), BC(kb + 1), kTriNone});
    if (!syrk.empty()) BAMG_TRY(gemm_batch<true>(syrk, s, -1.0, 1.0, 1, D, ctx->sm_count, st));
    if (kt >= 0 && kb >= 0)
      BAMG_TRY(cooperative_factor(ctx, st, Dk(kt), Wk(kt), s, ntl, D.dinv_tiles, Dk(kb), Wk(kb), dt1));
    else
      BAMG_TRY(cooperative_factor(ctx, st, Dk(kt >= 0 ? kt : kb), Wk(kt >= 0 ? kt : kb), s, ntl, D.dinv_tiles));
    for (int k : {kt, kb})
      if (k >= 0) { k_transpose_dense<<<tg, 256, 0, st>>>(Wk(k), Wt(k), s); BAMG_COUNT_LAUNCH; }
    // B_k = A_{k+1,k} W_k^T, C_k = A_{k-1,k} W_k^T (W_k lower triangular)
    if (kt >= 0) panel.push_back({BC(kt), D.Sub + kt * ss, Wk(kt), kTriBtUpper});
    if (kb >= 0) panel.push_back({BC(kb), D.Sup + (kb - 1) * ss, Wk(kb), kTriBtUpper});
    BAMG_TRY(gemm_batch<true>(panel, s, 1.0, 0.0, 0, D, ctx->sm_count, st));
  }
  // middle chunk: both Schur complements, then its factor
  {
    std::vector<GemmItem> syrk;
    if (t > 0) syrk.push_back({Dk(t), BC(t - 1), BC(t - 1), kTriNone});
    if (t + 1 < nc) syrk.push_back({Dk(t), BC(t + 1), BC(t + 1), kTriNone});
    for (auto& it : syrk) BAMG_TRY(gemm_batch<true>({it}, s, -1.0, 1.0, 1, D, ctx->sm_count, st));  // same output: one at a time
    BAMG_TRY(cooperative_factor(ctx, st, Dk(t), Wk(t), s, ntl, D.dinv_tiles));
    { k_transpose_dense<<<tg, 256, 0, st>>>(Wk(t), Wt(t), s); BAMG_COUNT_LAUNCH; }
  }
  // chain matrices, off the critical path: all in two batched launches
  std::vector<GemmItem> nn, nt;
  for (int k = 1; k <= t; ++k) nn.push_back({D.Mb + k * ss, Wk(k), BC(k - 1), kTriALower});     // M_k = W_k B_{k-1}
  for (int k = t; k + 1 < nc; ++k) nn.push_back({D.Mtb + k * ss, Wk(k), BC(k + 1), kTriALower});  // Mt_k = W_k C_{k+1}
  for (int k = 0; k < t; ++k) nt.push_back({D.Nb + k * ss, Wt(k), BC(k), kTriAUpper});          // N_k = W_k^T B_k^T
  for (int k = t + 1; k < nc; ++k) nt.push_back({D.Ntb + k * ss, Wt(k), BC(k), kTriAUpper});     // Nt_k = W_k^T C_k^T
  BAMG_TRY(gemm_batch<false>(nn, s, 1.0, 0.0, 0, D, ctx->sm_count, st));
  BAMG_TRY(gemm_batch<true>(nt, s, 1.0, 0.0, 0, D, ctx->sm_count, st));
  prof_end(ctx, pm, st);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}
template <int KP>
static Status chain_round(const ChainRound& c, int jobs, int s, const int* done, cudaStream_t st) {
  BAMG_CUDA(launch_k(k_chunk_chain<KP>, dim3(chain_grid(s), (unsigned)jobs), dim3(256), st, c, s, done));
  BAMG_COUNT_LAUNCH;
  return Status{};
}

template <int KP, typename T>
static Status band_apply(bamg_mg* mg, const T* b, T* x, double* y, double* z, const int* done, cudaStream_t st) {
  CoarseDense& D = mg->coarse;
  const int s = D.s, nc = D.nc, t = nc / 2;
  const int64_t ss = (int64_t)s * s, npad = D.npad, cs = (int64_t)s * KP;
  // forward: y = blockdiag(W) b, then the two chains toward the middle chunk
  { BAMG_CUDA(launch_k(k_chunk_mv<KP, T>, dim3(chain_grid(npad)), dim3(256), st, D.Wb, s, npad, b, D.n, y, 1, done)); BAMG_COUNT_LAUNCH; }
  const int fr = std::max(t - 1, nc - 2 - t);
  for (int r = 1; r <= fr; ++r) {
    ChainRound c = {};
    int jobs = 0;
    if (r <= t - 1) {  // top chunk r from r - 1
      c.M1[jobs] = D.Mb + r * ss;
      c.z1[jobs] = y + (r - 1) * cs;
      c.y[jobs++] = y + r * cs;
    }
    const int kb = nc - 1 - r;  // bottom chunk from kb + 1
    if (kb > t) {
      c.M1[jobs] = D.Mtb + kb * ss;
      c.z1[jobs] = y + (kb + 1) * cs;
      c.y[jobs++] = y + kb * cs;
    }
    if (jobs) BAMG_TRY(chain_round<KP>(c, jobs, s, done, st));
  }
  {
    ChainRound c = {};
    c.M1[0] = t > 0 ? D.Mb + t * ss : nullptr;
    c.z1[0] = t > 0 ? y + (t - 1) * cs : nullptr;
    c.M2[0] = t + 1 < nc ? D.Mtb + t * ss : nullptr;
    c.z2[0] = t + 1 < nc ? y + (t + 1) * cs : nullptr;
    c.y[0] = y + t * cs;
    BAMG_TRY(chain_round<KP>(c, 1, s, done, st));
  }
  // backward: z = blockdiag(W^T) y, then outward from the middle chunk
  { BAMG_CUDA(launch_k(k_chunk_mv<KP, double>, dim3(chain_grid(npad)), dim3(256), st, D.Wtb, s, npad, y, npad, z, 2, done)); BAMG_COUNT_LAUNCH; }
  const int br = std::max(t, nc - 1 - t);
  for (int r = 1; r <= br; ++r) {
    ChainRound c = {};
    int jobs = 0;
    const int kt = t - r, kb = t + r;
    if (kt >= 0) {
      c.M1[jobs] = D.Nb + kt * ss;
      c.z1[jobs] = z + (kt + 1) * cs;
      c.y[jobs++] = z + kt * cs;
    }
    if (kb < nc) {
      c.M1[jobs] = D.Ntb + kb * ss;
      c.z1[jobs] = z + (kb - 1) * cs;
      c.y[jobs++] = z + kb * cs;
    }
    if (jobs) BAMG_TRY(chain_round<KP>(c, jobs, s, done, st));
  }
  const int64_t m = D.n * KP;
  { BAMG_CUDA(launch_k(k_band_out<T>, dim3((unsigned)((m + 255) / 256)), dim3(256), st, m, z, x, done)); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

static Status dense_factor(bamg_mg* mg, cudaStream_t st) {
  bamg_ctx* ctx = mg->ctx;
  Level& C = mg->levels.back();
  CoarseDense& D = mg->coarse;
  const int bs = C.bs;
  const int64_t n = D.n, npad = D.npad;
  const int nt = (int)(npad / kT);
  if (!D.M) {
    BAMG_TRY(dalloc(&D.M, npad * npad, st));
    BAMG_TRY(dalloc(&D.Wt, npad * npad, st));
    BAMG_TRY(dalloc(&D.b64, npad, st));
    BAMG_TRY(dalloc(&D.x64, npad, st));
  }
  // The factor L is formed in the Wt buffer (F) and W = L^-1 in M; the final
  // transpose then overwrites the factor with W^T.
  double* F = D.Wt;
  double* W = D.M;
  const int pm = prof_begin(ctx, BAMG_PROF_COARSE_FACTOR, st);
  { k_dense_init<<<(unsigned)((npad * npad + 255) / 256), 256, 0, st>>>(F, n, npad); BAMG_COUNT_LAUNCH; }
  const bamg_bsr* A = C.A;
  const int64_t nt_fill = A->nnzb * bs * bs;
  if (nt_fill > 0) {
    const unsigned b = (unsigned)((nt_fill + 255) / 256);
    if (bs == 6) {
      if (A->vals64_stale)
        { k_dense_fill<float, 6><<<b, 256, 0, st>>>(A->nnzb, D.rows, A->colidx, A->slot_of, A->vals32, F, npad); BAMG_COUNT_LAUNCH; }
      else
        { k_dense_fill<double, 6><<<b, 256, 0, st>>>(A->nnzb, D.rows, A->colidx, A->slot_of, A->vals, F, npad); BAMG_COUNT_LAUNCH; }
    } else {
      if (A->vals64_stale)
        { k_dense_fill<float, 3><<<b, 256, 0, st>>>(A->nnzb, D.rows, A->colidx, A->slot_of, A->vals32, F, npad); BAMG_COUNT_LAUNCH; }
      else
        { k_dense_fill<double, 3><<<b, 256, 0, st>>>(A->nnzb, D.rows, A->colidx, A->slot_of, A->vals, F, npad); BAMG_COUNT_LAUNCH; }
    }
  }
  BAMG_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * npad * npad, st));
  if (!D.dinv_tiles) BAMG_TRY(dalloc(&D.dinv_tiles, (int64_t)nt * kT * kT, st));
  BAMG_TRY(cooperative_factor(ctx, st, F, W, npad, nt, D.dinv_tiles));
  // Wt = W^T (the factor in F is no longer needed)
  dim3 tg((unsigned)nt, (unsigned)nt);
  { k_transpose_dense<<<tg, 256, 0, st>>>(W, F, npad); BAMG_COUNT_LAUNCH; }
  prof_end(ctx, pm, st);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

Status coarse_factor(bamg_mg* mg, cudaStream_t st) {
  Level& C = mg->levels.back();
  CoarseDense& D = mg->coarse;
  const bamg_bsr* A = C.A;
  const int64_t n = C.n * C.bs;
  if (D.n == 0) {  // first factorisation: choose the form
    D.n = n;
    const int64_t b = half_bandwidth(A);
    const int64_t s = ((b + 1 + kT - 1) / kT) * kT;
    const int64_t nc = (n + s - 1) / s;
    const int mode = mg->opts.coarse_solver;
    const bool band = mode != 1 && nc >= (mode == 2 ? 2 : 3);
    if (band) {
      D.s = (int)s;
      D.nc = (int)nc;
      D.npad = nc * s;
    } else {
      D.npad = ((n + kT - 1) / kT) * kT;
      if (D.npad > 16384)
        return make_status(BAMG_ERR_INVALID, "coarsest level too large for a dense solve (%lld)", (long long)n);
    }
    std::vector<int> rows(A->nnzb);
    for (int64_t I = 0; I < A->nbr; ++I)
      for (int k = A->h_rowptr[I]; k < A->h_rowptr[I + 1]; ++k) rows[k] = (int)I;
    BAMG_TRY(upload(&D.rows, rows, st));
    BAMG_CUDA(cudaStreamSynchronize(st));
  }
  BAMG_TRY(D.nc > 0 ? band_factor(mg, st) : dense_factor(mg, st));
  D.factored = true;
  return Status{};
}

template <typename T>
Status coarse_apply(bamg_mg* mg, const T* b, T* x, const int* done, cudaStream_t st) {
  CoarseDense& D = mg->coarse;
  if (D.nc > 0) return band_apply<1, T>(mg, b, x, D.b64, D.x64, done, st);
  const int64_t n = D.n;
  const unsigned g = (unsigned)((n * 32 + 255) / 256);
  { BAMG_CUDA(launch_k(k_tri_mv<T, double>, dim3(g), dim3(256), st, D.M, D.npad, n, b, D.x64, 1, done)); BAMG_COUNT_LAUNCH; }
  { BAMG_CUDA(launch_k(k_tri_mv<double, T>, dim3(g), dim3(256), st, D.Wt, D.npad, n, D.x64, x, 0, done)); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <typename T>
Status coarse_apply_multi(bamg_mg* mg, int kp, const T* b, T* x, double* work, const int* done, cudaStream_t st) {
  CoarseDense& D = mg->coarse;
  const int64_t n = D.n;
  double* y = work;
  double* z = work + D.npad * kp;
#define BAMG_KP_CASE(KP)                                                                                   \
  if (kp == KP) {                                                                                          \
    if (D.nc > 0) return band_apply<KP, T>(mg, b, x, y, z, done, st);                                     \
    const unsigned g = (unsigned)((n * 32 + 255) / 256);                                                   \
    { BAMG_CUDA(launch_k(k_tri_mm<KP, T, double>, dim3(g), dim3(256), st, D.M, D.npad, n, b, y, 1, done)); BAMG_COUNT_LAUNCH; }      \
    { BAMG_CUDA(launch_k(k_tri_mm<KP, double, T>, dim3(g), dim3(256), st, D.Wt, D.npad, n, y, x, 0, done)); BAMG_COUNT_LAUNCH; }     \
    BAMG_CUDA(cudaGetLastError());                                                                         \
    return Status{};                                                                                       \
  }
  BAMG_KP_CASE(4)
  BAMG_KP_CASE(8)
  BAMG_KP_CASE(16)
  BAMG_KP_CASE(32)
#undef BAMG_KP_CASE
  return make_status(BAMG_ERR_INVALID, "unsupported column count %d", kp);
}

template Status coarse_apply<double>(bamg_mg*, const double*, double*, const int*, cudaStream_t);
template Status coarse_apply<float>(bamg_mg*, const float*, float*, const int*, cudaStream_t);
template Status coarse_apply_multi<double>(bamg_mg*, int, const double*, double*, double*, const int*, cudaStream_t);
template Status coarse_apply_multi<float>(bamg_mg*, int, const float*, float*, double*, const int*, cudaStream_t);

}  // namespace bamg
