// Exact coarsest-level solve: dense FP64 Cholesky A = L L^T, then the explicit
// inverse factor W = L^-1, so every V-cycle applies x = W^T (W b) as two
// dense triangular matrix-vector products spread over the whole GPU instead of
// two sequential substitutions.  The matrix is padded to a multiple of the
// 32-wide tiles with an identity block (which factors to itself).
//
// Tiled right-looking algorithms, one kernel per tile step:
//   Cholesky   for k: factor tile (k,k); L(i,k) = A(i,k) L(k,k)^-T; A(i,j) -= L(i,k) L(j,k)^T
//   W = L^-1   for i: W(i,k) = L(i,i)^-1 (delta_ik I - S(i,k)), k <= i;  S(r,k) += L(r,i) W(i,k), r > i
#include <cooperative_groups.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace bamg {

constexpr int kT = 32;  // tile size

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

// Cholesky of the diagonal tile (k, k) in shared memory and the inverse of
// the factor (one CTA); L is written back, L^-1 to Linv.
__device__ void diag_tile(double* __restrict__ M, int64_t ld, int k, double* __restrict__ Linv, int* err,
                          double (*a)[kT + 1], double (*w)[kT + 1]) {
  const int tid = threadIdx.x;
  double* base = M + (int64_t)k * kT * ld + (int64_t)k * kT;
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) a[e / kT][e % kT] = base[(int64_t)(e / kT) * ld + e % kT];
  __syncthreads();
  for (int j = 0; j < kT; ++j) {
    if (tid == 0) {
      double d = a[j][j];
      if (!(d > 0.0)) {
        set_err(err, kDevBreakdown);
        d = 1.0;
      }
      a[j][j] = sqrt(d);
    }
    __syncthreads();
    if (tid > j && tid < kT) a[tid][j] /= a[j][j];
    __syncthreads();
    for (int e = tid; e < kT * kT; e += blockDim.x) {
      const int i = e / kT, l = e % kT;
      if (l > j && i >= l) a[i][l] -= a[i][j] * a[l][j];
    }
    __syncthreads();
  }
  // rows of W = L^-1 one at a time; 8 threads per column split the dot product
  const int c = tid >> 3, part = tid & 7;
  for (int r = 0; r < kT; ++r) {
    double t = 0.0;
    if (c < r)
      for (int l = c + part; l < r; l += 8) t = fma(a[r][l], w[l][c], t);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (part == 0) w[r][c] = (c <= r) ? (((r == c) ? 1.0 : 0.0) - t) / a[r][r] : 0.0;
    __syncthreads();
  }
  for (int e = tid; e < kT * kT; e += blockDim.x) {
    const int i = e / kT, l = e % kT;
    base[(int64_t)i * ld + l] = l <= i ? a[i][l] : 0.0;
    Linv[e] = w[i][l];
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
__global__ void __launch_bounds__(256) k_dense_factor(double* __restrict__ F, double* __restrict__ W, int64_t ld,
                                                      int nt, double* __restrict__ Dinv, int* err) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  __shared__ double a[kT][kT + 1], w[kT][kT + 1];
  const int G = gridDim.x, b = blockIdx.x;
  if (b == 0) diag_tile(F, ld, 0, Dinv, err, a, w);
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
    // phase 2
    const int T = nt - k - 1;
    const int n_trail = T * (T + 1) / 2, n_wupd = T * (k + 1);
    if (b == 0 && T > 0) {
      const int g = k + 1;
      tile_update<true>(F + (int64_t)g * kT * ld + (int64_t)g * kT, F + (int64_t)g * kT * ld + (int64_t)k * kT,
                        F + (int64_t)g * kT * ld + (int64_t)k * kT, ld, a, w);
      __syncthreads();
      __threadfence_block();
      diag_tile(F, ld, g, Dinv + (int64_t)g * kT * kT, err, a, w);
    }
    // item 0 of the trailing update is tile (k+1,k+1), done by CTA 0 above
    for (int item = (b == 0 ? G : b); item < n_trail + n_wupd; item += G) {
      if (item == 0) continue;
      if (item < n_trail) {
        int idx = item, i = 0;
        while (idx > i) {  // row-major lower triangle (i, j), j <= i
          idx -= i + 1;
          ++i;
        }
        const int gi = k + 1 + i, gj = k + 1 + idx;
        tile_update<true>(F + (int64_t)gi * kT * ld + (int64_t)gj * kT,
                          F + (int64_t)gi * kT * ld + (int64_t)k * kT, F + (int64_t)gj * kT * ld + (int64_t)k * kT,
                          ld, a, w);
      } else {
        const int it = item - n_trail;
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

Status coarse_factor(bamg_mg* mg) {
  bamg_ctx* ctx = mg->ctx;
  cudaStream_t st = ctx->stream;
  Level& C = mg->levels.back();
  CoarseDense& D = mg->coarse;
  const int bs = C.bs;
  const int64_t n = C.n * bs;
  const int64_t npad = ((n + kT - 1) / kT) * kT;
  const int nt = (int)(npad / kT);
  if (npad > 16384) return make_status(BAMG_ERR_INVALID, "coarsest level too large for a dense solve (%lld)", (long long)n);
  if (!D.M) {
    D.n = n;
    D.npad = npad;
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
  if (!D.rows) {
    std::vector<int> rows(A->nnzb);
    for (int64_t I = 0; I < A->nbr; ++I)
      for (int k = A->h_rowptr[I]; k < A->h_rowptr[I + 1]; ++k) rows[k] = (int)I;
    BAMG_TRY(upload(&D.rows, rows, st));
    BAMG_CUDA(cudaStreamSynchronize(st));
  }
  const int* d_rows = D.rows;
  const int64_t nt_fill = A->nnzb * bs * bs;
  if (nt_fill > 0) {
    const unsigned b = (unsigned)((nt_fill + 255) / 256);
    if (bs == 6) {
      if (A->vals64_stale)
        { k_dense_fill<float, 6><<<b, 256, 0, st>>>(A->nnzb, d_rows, A->colidx, A->slot_of, A->vals32, F, npad); BAMG_COUNT_LAUNCH; }
      else
        { k_dense_fill<double, 6><<<b, 256, 0, st>>>(A->nnzb, d_rows, A->colidx, A->slot_of, A->vals, F, npad); BAMG_COUNT_LAUNCH; }
    } else {
      if (A->vals64_stale)
        { k_dense_fill<float, 3><<<b, 256, 0, st>>>(A->nnzb, d_rows, A->colidx, A->slot_of, A->vals32, F, npad); BAMG_COUNT_LAUNCH; }
      else
        { k_dense_fill<double, 3><<<b, 256, 0, st>>>(A->nnzb, d_rows, A->colidx, A->slot_of, A->vals, F, npad); BAMG_COUNT_LAUNCH; }
    }
  }
  BAMG_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * npad * npad, st));
  if (!D.dinv_tiles) BAMG_TRY(dalloc(&D.dinv_tiles, (int64_t)nt * kT * kT, st));
  {
    int per_sm = 0;
    BAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_factor, 256, 0));
    const int grid = std::max(1, std::min(per_sm, 2)) * ctx->sm_count;
    int64_t ld = npad;
    int ntl = nt;
    double* dt = D.dinv_tiles;
    int* err = ctx->d_err;
    void* args[] = {&F, &W, &ld, &ntl, &dt, &err};
    if (per_sm < 1) return make_status(BAMG_ERR_CUDA, "dense factor kernel cannot be resident");
    BAMG_CUDA(cudaLaunchCooperativeKernel((void*)k_dense_factor, grid, 256, args, 0, st));
    BAMG_COUNT_LAUNCH;
  }
  // Wt = W^T (the factor in F is no longer needed)
  dim3 tg((unsigned)nt, (unsigned)nt);
  { k_transpose_dense<<<tg, 256, 0, st>>>(W, F, npad); BAMG_COUNT_LAUNCH; }
  prof_end(ctx, pm, st);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <typename T>
Status coarse_apply(bamg_mg* mg, const T* b, T* x, const int* done, cudaStream_t st) {
  CoarseDense& D = mg->coarse;
  const int64_t n = D.n;
  const unsigned g = (unsigned)((n * 32 + 255) / 256);
  { k_tri_mv<T, double><<<g, 256, 0, st>>>(D.M, D.npad, n, b, D.x64, 1, done); BAMG_COUNT_LAUNCH; }
  { k_tri_mv<double, T><<<g, 256, 0, st>>>(D.Wt, D.npad, n, D.x64, x, 0, done); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template Status coarse_apply<double>(bamg_mg*, const double*, double*, const int*, cudaStream_t);
template Status coarse_apply<float>(bamg_mg*, const float*, float*, const int*, cudaStream_t);

}  // namespace bamg
