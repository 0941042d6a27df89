// Exact coarsest-level solve: dense FP64 Cholesky A = L L^T, then the explicit
// inverse factor W = L^-1, so every V-cycle applies x = W^T (W b) as two
// dense triangular matrix-vector products spread over the whole GPU instead of
// two sequential substitutions.  The matrix is padded to a multiple of the
// 32-wide tiles with an identity block (which factors to itself).
//
// Tiled right-looking algorithms, one kernel per tile step:
//   Cholesky   for k: factor tile (k,k); L(i,k) = A(i,k) L(k,k)^-T; A(i,j) -= L(i,k) L(j,k)^T
//   W = L^-1   for i: W(i,k) = L(i,i)^-1 (delta_ik I - S(i,k)), k <= i;  S(r,k) += L(r,i) W(i,k), r > i
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

// Factor the diagonal tile (k, k) in shared memory (unblocked, right-looking).
__global__ void __launch_bounds__(256) k_potrf_tile(double* __restrict__ M, int64_t ld, int k, int* err) {
  __shared__ double a[kT][kT + 1];
  const int tid = threadIdx.x;
  double* base = M + (int64_t)k * kT * ld + (int64_t)k * kT;
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
  for (int e = tid; e < kT * kT; e += blockDim.x) {
    const int i = e / kT, l = e % kT;
    base[(int64_t)i * ld + l] = l <= i ? a[i][l] : 0.0;
  }
}

// L(i,k) = A(i,k) L(k,k)^-T for tiles i = k+1 .. nt-1 (one CTA per tile).
__global__ void __launch_bounds__(128) k_trsm_tiles(double* __restrict__ M, int64_t ld, int k) {
  __shared__ double L[kT][kT + 1], X[kT][kT + 1];
  const int i = k + 1 + blockIdx.x;
  const int tid = threadIdx.x;
  const double* lb = M + (int64_t)k * kT * ld + (int64_t)k * kT;
  double* xb = M + (int64_t)i * kT * ld + (int64_t)k * kT;
  for (int e = tid; e < kT * kT; e += blockDim.x) {
    L[e / kT][e % kT] = lb[(int64_t)(e / kT) * ld + e % kT];
    X[e / kT][e % kT] = xb[(int64_t)(e / kT) * ld + e % kT];
  }
  __syncthreads();
  if (tid < kT) {  // row tid of X solves x L^T = a, i.e. sum_{l<=j} x_l L[j][l] = a_j
    for (int j = 0; j < kT; ++j) {
      double t = X[tid][j];
      for (int l = 0; l < j; ++l) t -= X[tid][l] * L[j][l];
      X[tid][j] = t / L[j][j];
    }
  }
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) xb[(int64_t)(e / kT) * ld + e % kT] = X[e / kT][e % kT];
}

// Tile GEMM update C -= A B^T (trailing Cholesky update) or C += A B (inverse
// accumulation), 256 threads, 4 outputs each.
template <bool kSyrk>
__device__ __forceinline__ void tile_update(double* __restrict__ C, const double* __restrict__ Ab,
                                            const double* __restrict__ Bb, int64_t ld) {
  __shared__ double As[kT][kT + 1], Bs[kT][kT + 1];
  const int tid = threadIdx.x;
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

// A(i,j) -= L(i,k) L(j,k)^T for k < j <= i < nt; blockIdx enumerates (i, j).
__global__ void __launch_bounds__(256) k_syrk_tiles(double* __restrict__ M, int64_t ld, int k, int nt) {
  const int T = nt - k - 1;
  int idx = blockIdx.x, i = 0;
  while (idx > i) {  // row-major lower triangle of a T x T tile grid
    idx -= i + 1;
    ++i;
  }
  const int j = idx;
  const int gi = k + 1 + i, gj = k + 1 + j;
  (void)T;
  tile_update<true>(M + (int64_t)gi * kT * ld + (int64_t)gj * kT, M + (int64_t)gi * kT * ld + (int64_t)k * kT,
                    M + (int64_t)gj * kT * ld + (int64_t)k * kT, ld);
}

// W(i,k) = L(i,i)^-1 (delta_ik I - S(i,k)) for k = 0..i, S accumulated in W.
__global__ void __launch_bounds__(128) k_winv_tiles(const double* __restrict__ Lm, double* __restrict__ W, int64_t ld,
                                                    int i) {
  __shared__ double L[kT][kT + 1], X[kT][kT + 1];
  const int k = blockIdx.x;
  const int tid = threadIdx.x;
  const double* lb = Lm + (int64_t)i * kT * ld + (int64_t)i * kT;
  double* wb = W + (int64_t)i * kT * ld + (int64_t)k * kT;
  for (int e = tid; e < kT * kT; e += blockDim.x) {
    const int r = e / kT, c = e % kT;
    L[r][c] = lb[(int64_t)r * ld + c];
    X[r][c] = ((k == i && r == c) ? 1.0 : 0.0) - wb[(int64_t)r * ld + c];
  }
  __syncthreads();
  if (tid < kT) {  // column tid: forward substitution L x = rhs
    for (int r = 0; r < kT; ++r) {
      double t = X[r][tid];
      for (int l = 0; l < r; ++l) t -= L[r][l] * X[l][tid];
      X[r][tid] = t / L[r][r];
    }
  }
  __syncthreads();
  for (int e = tid; e < kT * kT; e += blockDim.x) wb[(int64_t)(e / kT) * ld + e % kT] = X[e / kT][e % kT];
}

// S(r,k) += L(r,i) W(i,k) for r = i+1..nt-1, k = 0..i; blockIdx = (r - i - 1) * (i + 1) + k.
__global__ void __launch_bounds__(256) k_wupdate_tiles(const double* __restrict__ Lm, double* __restrict__ W,
                                                       int64_t ld, int i) {
  const int r = i + 1 + blockIdx.x / (i + 1);
  const int k = blockIdx.x % (i + 1);
  tile_update<false>(W + (int64_t)r * kT * ld + (int64_t)k * kT, Lm + (int64_t)r * kT * ld + (int64_t)i * kT,
                     W + (int64_t)i * kT * ld + (int64_t)k * kT, ld);
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
  k_dense_init<<<(unsigned)((npad * npad + 255) / 256), 256, 0, st>>>(F, n, npad);
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
        k_dense_fill<float, 6><<<b, 256, 0, st>>>(A->nnzb, d_rows, A->colidx, A->slot_of, A->vals32, F, npad);
      else
        k_dense_fill<double, 6><<<b, 256, 0, st>>>(A->nnzb, d_rows, A->colidx, A->slot_of, A->vals, F, npad);
    } else {
      if (A->vals64_stale)
        k_dense_fill<float, 3><<<b, 256, 0, st>>>(A->nnzb, d_rows, A->colidx, A->slot_of, A->vals32, F, npad);
      else
        k_dense_fill<double, 3><<<b, 256, 0, st>>>(A->nnzb, d_rows, A->colidx, A->slot_of, A->vals, F, npad);
    }
  }
  for (int k = 0; k < nt; ++k) {
    k_potrf_tile<<<1, 256, 0, st>>>(F, npad, k, ctx->d_err);
    if (k + 1 < nt) {
      k_trsm_tiles<<<nt - k - 1, 128, 0, st>>>(F, npad, k);
      const int T = nt - k - 1;
      k_syrk_tiles<<<T * (T + 1) / 2, 256, 0, st>>>(F, npad, k, nt);
    }
  }
  BAMG_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * npad * npad, st));
  for (int i = 0; i < nt; ++i) {
    k_winv_tiles<<<i + 1, 128, 0, st>>>(F, W, npad, i);
    if (i + 1 < nt) k_wupdate_tiles<<<(nt - i - 1) * (i + 1), 256, 0, st>>>(F, W, npad, i);
  }
  // Wt = W^T (the factor in F is no longer needed)
  dim3 tg((unsigned)nt, (unsigned)nt);
  k_transpose_dense<<<tg, 256, 0, st>>>(W, F, npad);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template <typename T>
Status coarse_apply(bamg_mg* mg, const T* b, T* x, const int* done, cudaStream_t st) {
  CoarseDense& D = mg->coarse;
  const int64_t n = D.n;
  const unsigned g = (unsigned)((n * 32 + 255) / 256);
  k_tri_mv<T, double><<<g, 256, 0, st>>>(D.M, D.npad, n, b, D.x64, 1, done);
  k_tri_mv<double, T><<<g, 256, 0, st>>>(D.Wt, D.npad, n, D.x64, x, 0, done);
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

template Status coarse_apply<double>(bamg_mg*, const double*, double*, const int*, cudaStream_t);
template Status coarse_apply<float>(bamg_mg*, const float*, float*, const int*, cudaStream_t);

}  // namespace bamg
