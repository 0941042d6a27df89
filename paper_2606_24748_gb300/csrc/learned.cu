// Learned per-block-row smoother weights: block features, an 8-64-64-1 MLP
// with bfloat16 parameters and activations and FP32 accumulation (forward,
// backward, Adam), training targets from the plain V-cycle, and the hook that
// lets mg_update compute the weights on every update.
//
// MLP: z = w3 . relu(W2^T relu(W1^T x + b1) + b2) + b3, w = 0.5 + 1.5 sigmoid(z);
// inputs, parameters and hidden activations are rounded to bfloat16 (round to
// nearest even), every product is accumulated in FP32, bias added after the
// sum.  Parameters (FP32 master copy): W1[8][64], b1[64], W2[64][64], b2[64],
// w3[64], b3.  Gradients of the mean squared error are reduced over rows with
// a fixed order (per-CTA partial sums in registers, then a second kernel sums
// the CTAs in index order), so training is deterministic.
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"

namespace bamg {

constexpr int kNF = 8, kNH = 64;
constexpr int kOffW1 = 0, kOffB1 = kNF * kNH, kOffW2 = kOffB1 + kNH, kOffB2 = kOffW2 + kNH * kNH,
              kOffW3 = kOffB2 + kNH, kOffB3 = kOffW3 + kNH, kNP = kOffB3 + 1;
constexpr int kBwdRowsPerChunk = 16;
constexpr int kBwdThreads = 256;
constexpr int kBwdMaxCtas = 1216;

}  // namespace bamg

struct bamg_mlp {
  bamg_ctx* ctx = nullptr;
  float* theta = nullptr;    // FP32 master parameters
  float* theta_bf = nullptr; // bfloat16-rounded copy (stored as float)
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  float* partials = nullptr; // kBwdMaxCtas x (kNP + 1)
  __nv_bfloat16* h1 = nullptr;
  __nv_bfloat16* h2 = nullptr;
  int64_t cap_rows = 0;
  int64_t t = 0;             // Adam step count
};

namespace bamg {

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float weight_of(float z) {
  const double s = 1.0 / (1.0 + exp(-(double)z));
  const float w = (float)(0.5 + 1.5 * s);
  return isfinite(w) ? w : 1.0f;  // a non-finite prediction falls back to the plain smoother
}

// One row per thread; parameters in shared memory.  Optionally keeps the
// (bfloat16) hidden activations for the backward pass.
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ pbf, const float* __restrict__ X,
                                                     int64_t n, float* __restrict__ w_out,
                                                     __nv_bfloat16* __restrict__ h1s, __nv_bfloat16* __restrict__ h2s) {
  __shared__ float P[kNP];
  for (int e = threadIdx.x; e < kNP; e += blockDim.x) P[e] = pbf[e];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[kNF];
#pragma unroll
  for (int f = 0; f < kNF; ++f) x[f] = bfr(X[i * kNF + f]);
  float h1[kNH];
#pragma unroll
  for (int j = 0; j < kNH; ++j) {
    float a = 0.f;
#pragma unroll
    for (int f = 0; f < kNF; ++f) a = fmaf(x[f], P[kOffW1 + f * kNH + j], a);
    a += P[kOffB1 + j];
    h1[j] = bfr(fmaxf(a, 0.f));
    if (h1s) h1s[i * kNH + j] = __float2bfloat16_rn(h1[j]);
  }
  float z = 0.f;
  for (int k = 0; k < kNH; ++k) {
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < kNH; ++j) a = fmaf(h1[j], P[kOffW2 + j * kNH + k], a);
    a += P[kOffB2 + k];
    const float h = bfr(fmaxf(a, 0.f));
    if (h2s) h2s[i * kNH + k] = __float2bfloat16_rn(h);
    z = fmaf(h, P[kOffW3 + k], z);
  }
  z += P[kOffB3];
  w_out[i] = weight_of(z);
}

// Gradient of mean((w - t)^2) over n rows; CTA b handles rows
// [b * rows_per_cta, ...) in chunks of 16 and writes its partial sums
// (and the partial squared error at index kNP) to partials[b].
__global__ void __launch_bounds__(kBwdThreads) k_mlp_backward(const float* __restrict__ pbf,
                                                              const float* __restrict__ X,
                                                              const float* __restrict__ tgt, int64_t n,
                                                              int64_t rows_per_cta,
                                                              const __nv_bfloat16* __restrict__ h1s,
                                                              const __nv_bfloat16* __restrict__ h2s,
                                                              float* __restrict__ partials) {
  constexpr int R = kBwdRowsPerChunk;
  __shared__ float W2[kNH * kNH];
  __shared__ float W3[kNH];
  __shared__ float xs[R][kNF];
  __shared__ float h1[R][kNH + 1];
  __shared__ float h2[R][kNH + 1];
  __shared__ float d2[R][kNH + 1];
  __shared__ float d1[R][kNH + 1];
  __shared__ float dz[R];
  __shared__ float sq[R];
  const int tid = threadIdx.x;
  for (int e = tid; e < kNH * kNH; e += blockDim.x) W2[e] = pbf[kOffW2 + e];
  for (int e = tid; e < kNH; e += blockDim.x) W3[e] = pbf[kOffW3 + e];
  const float b3 = pbf[kOffB3];
  float gW2[16], gW1[2], g64 = 0.f, gb3 = 0.f, loss = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) gW2[q] = 0.f;
  gW1[0] = gW1[1] = 0.f;
  const int64_t r0 = blockIdx.x * rows_per_cta;
  const int64_t r1 = (n < r0 + rows_per_cta) ? n : r0 + rows_per_cta;
  for (int64_t c0 = r0; c0 < r1; c0 += R) {
    const int m = (int)((r1 - c0 < R) ? (r1 - c0) : R);
    __syncthreads();
    for (int e = tid; e < R * kNH; e += blockDim.x) {
      const int r = e / kNH, j = e % kNH;
      const bool ok = r < m;
      h1[r][j] = ok ? __bfloat162float(h1s[(c0 + r) * kNH + j]) : 0.f;
      h2[r][j] = ok ? __bfloat162float(h2s[(c0 + r) * kNH + j]) : 0.f;
    }
    for (int e = tid; e < R * kNF; e += blockDim.x) {
      const int r = e / kNF, f = e % kNF;
      xs[r][f] = r < m ? bfr(X[(c0 + r) * kNF + f]) : 0.f;
    }
    __syncthreads();
    if (tid < R) {
      float d = 0.f, s2 = 0.f;
      if (tid < m) {
        float z = 0.f;
        for (int k = 0; k < kNH; ++k) z = fmaf(h2[tid][k], W3[k], z);
        z += b3;
        const double s = 1.0 / (1.0 + exp(-(double)z));
        const double e = 0.5 + 1.5 * s - (double)tgt[c0 + tid];
        d = (float)((2.0 / (double)n) * e * 1.5 * s * (1.0 - s));
        s2 = (float)(e * e);
      }
      dz[tid] = d;
      sq[tid] = s2;
    }
    __syncthreads();
    for (int e = tid; e < R * kNH; e += blockDim.x) {
      const int r = e / kNH, k = e % kNH;
      d2[r][k] = h2[r][k] > 0.f ? dz[r] * W3[k] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < R * kNH; e += blockDim.x) {
      const int r = e / kNH, j = e % kNH;
      float a = 0.f;
      if (h1[r][j] > 0.f)
        for (int k = 0; k < kNH; ++k) a = fmaf(W2[j * kNH + k], d2[r][k], a);
      d1[r][j] = a;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + kBwdThreads * q, j = e / kNH, k = e % kNH;
      float a = gW2[q];
      for (int r = 0; r < R; ++r) a = fmaf(h1[r][j], d2[r][k], a);
      gW2[q] = a;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + kBwdThreads * q, f = e / kNH, j = e % kNH;
      float a = gW1[q];
      for (int r = 0; r < R; ++r) a = fmaf(xs[r][f], d1[r][j], a);
      gW1[q] = a;
    }
    if (tid < kNH) {
      for (int r = 0; r < R; ++r) g64 += d1[r][tid];                 // b1
    } else if (tid < 2 * kNH) {
      for (int r = 0; r < R; ++r) g64 += d2[r][tid - kNH];           // b2
    } else if (tid < 3 * kNH) {
      for (int r = 0; r < R; ++r) g64 = fmaf(dz[r], h2[r][tid - 2 * kNH], g64);  // w3
    } else if (tid == 3 * kNH) {
      for (int r = 0; r < R; ++r) gb3 += dz[r];
    } else if (tid == 3 * kNH + 1) {
      for (int r = 0; r < R; ++r) loss += sq[r];
    }
  }
  float* out = partials + (int64_t)blockIdx.x * (kNP + 1);
#pragma unroll
  for (int q = 0; q < 16; ++q) out[kOffW2 + tid + kBwdThreads * q] = gW2[q];
#pragma unroll
  for (int q = 0; q < 2; ++q) out[kOffW1 + tid + kBwdThreads * q] = gW1[q];
  if (tid < kNH)
    out[kOffB1 + tid] = g64;
  else if (tid < 2 * kNH)
    out[kOffB2 + tid - kNH] = g64;
  else if (tid < 3 * kNH)
    out[kOffW3 + tid - 2 * kNH] = g64;
  else if (tid == 3 * kNH)
    out[kOffB3] = gb3;
  else if (tid == 3 * kNH + 1)
    out[kNP] = loss;
}

// grad[p] = sum over CTAs of partials[b][p] in CTA order; loss = sum / n.
__global__ void k_mlp_reduce(const float* __restrict__ partials, int nb, float* __restrict__ grad,
                             float* __restrict__ loss_out, int64_t n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kNP) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += (double)partials[(int64_t)b * (kNP + 1) + p];
  if (p < kNP)
    grad[p] = (float)s;
  else if (loss_out)
    *loss_out = (float)(s / (double)n);
}

// Adam (Kingma and Ba 2015) on the FP32 master copy, then the bfloat16 copy.
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, float* __restrict__ theta_bf, float lr, float b1, float b2,
                           float eps, int64_t t) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP) return;
  const double gp = g[p];
  const double mp = b1 * (double)m[p] + (1.0 - b1) * gp;
  const double vp = b2 * (double)v[p] + (1.0 - b2) * gp * gp;
  m[p] = (float)mp;
  v[p] = (float)vp;
  const double mh = mp / (1.0 - pow((double)b1, (double)t));
  const double vh = vp / (1.0 - pow((double)b2, (double)t));
  const float th = (float)((double)theta[p] - (double)lr * mh / (sqrt(vh) + (double)eps));
  theta[p] = th;
  theta_bf[p] = bfr(th);
}

__global__ void k_round_params(const float* __restrict__ theta, float* __restrict__ theta_bf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kNP) theta_bf[p] = bfr(theta[p]);
}

// Features of each block row (see the learned-smoother oracle): log ||A_ii||,
// sum_{j!=i} ||A_ij|| / ||A_ii||, log(max/min nonzero block norm), blocks/27,
// clamped-row flag, log sum_j ||D_i^-1 A_ij||, level, 1.
template <int BS, typename TM>
__global__ void k_block_features(const int* __restrict__ rowptr, const int* __restrict__ slice_ptr,
                                 const int* __restrict__ col, const TM* __restrict__ vals,
                                 const double* __restrict__ dinv, int64_t n, float level, float* __restrict__ X) {
  constexpr int B = BS * BS;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t s = i >> 5;
  const int lane = (int)(i & 31);
  const int c0 = slice_ptr[s];
  const int len = rowptr[i + 1] - rowptr[i];
  double D[BS][BS];
  const int64_t db = (i >> 5) * (32LL * B) + lane;
#pragma unroll
  for (int a = 0; a < BS; ++a)
#pragma unroll
    for (int b = 0; b < BS; ++b) D[a][b] = dinv[db + 32 * (a * BS + b)];
  double dnorm = 0.0, offsum = 0.0, mx = 0.0, mn = 1e300, gsum = 0.0;
  bool any_off = false;
  for (int t = 0; t < len; ++t) {
    const int64_t c = c0 + t;
    const int j = col[c * 32 + lane];
    const TM* v = vals + c * (32LL * B) + lane;
    double a[BS][BS];
    double nrm = 0.0;
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int q = 0; q < BS; ++q) {
        a[r][q] = (double)v[32 * (r * BS + q)];
        nrm = fma(a[r][q], a[r][q], nrm);
      }
    nrm = sqrt(nrm);
    if (j == i) {
      dnorm = nrm;
    } else {
      offsum += nrm;
      any_off |= nrm > 0.0;
    }
    if (nrm > 0.0) {
      mx = fmax(mx, nrm);
      mn = fmin(mn, nrm);
    }
    double sn = 0.0;
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int q = 0; q < BS; ++q) {
        double e = 0.0;
#pragma unroll
        for (int k = 0; k < BS; ++k) e = fma(D[r][k], a[k][q], e);
        sn = fma(e, e, sn);
      }
    gsum += sqrt(sn);
  }
  float* o = X + i * kNF;
  o[0] = (float)log(dnorm);
  o[1] = (float)(offsum / dnorm);
  o[2] = (float)(mx > 0.0 ? log(mx / mn) : 0.0);
  o[3] = (float)((double)len / 27.0);
  o[4] = any_off ? 0.f : 1.f;
  o[5] = (float)log(gsum);
  o[6] = level;
  o[7] = 1.f;
}

// u = Dinv r (row-local)
template <int BS>
__global__ void k_apply_dinv(int64_t n, const double* __restrict__ dinv, const double* __restrict__ r,
                             double* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t db = (i >> 5) * (32LL * BS * BS) + (i & 31);
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < BS; ++c) t = fma(dinv[db + 32 * (a * BS + c)], r[i * BS + c], t);
    u[i * BS + a] = t;
  }
}

// q = A u per row; num_i += <r_i, q_i>, den_i += ||q_i||^2
template <int BS, int V>
__global__ void __launch_bounds__(kRowThreads) k_damping_accum(const int* __restrict__ sp, const int* __restrict__ col,
                                                               const double* __restrict__ vals, int64_t n,
                                                               int64_t nthreads, const double* __restrict__ u,
                                                               const double* __restrict__ r, double* __restrict__ num,
                                                               double* __restrict__ den) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  int64_t i;
  int sub;
  row_of_thread<V>(t, i, sub);
  double q[BS];
  row_product<BS, BS, V, double, double, double>(sp, col, vals, u, i, sub, q);
  if (sub != 0 || i >= n) return;
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int k = 0; k < BS; ++k) {
    a = fma(r[i * BS + k], q[k], a);
    b = fma(q[k], q[k], b);
  }
  num[i] += a;
  den[i] += b;
}

__global__ void k_damping_finish(int64_t n, const double* __restrict__ num, const double* __restrict__ den,
                                 float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double w = den[i] > 0.0 ? num[i] / den[i] : 1.0;
  out[i] = (float)fmin(2.0, fmax(0.5, w));
}

// r = b - A x, ||r||^2 (stationary iteration)
__global__ void __launch_bounds__(kRowThreads) k_residual_store(const int* __restrict__ sp, const int* __restrict__ col,
                                                                const double* __restrict__ vals, int64_t n,
                                                                int64_t rows_pad, const double* __restrict__ x,
                                                                const double* __restrict__ b, double* __restrict__ r,
                                                                double* out_norm2, double* partials, unsigned* counter) {
  double local[1] = {0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows_pad; i += stride) {
    double acc[3];
    row_product<3, 3, 1, double, double, double>(sp, col, vals, x, i, 0, acc);
    if (i < n) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double t = b[i * 3 + a] - acc[a];
        r[i * 3 + a] = t;
        local[0] = fma(t, t, local[0]);
      }
    }
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) *out_norm2 = out[0];
}

__global__ void k_axpy(int64_t m, const double* __restrict__ z, double* __restrict__ x) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) x[t] += z[t];
}

static Status mlp_reserve(bamg_mlp* M, int64_t n) {
  if (n <= M->cap_rows) return Status{};
  cudaStream_t st = M->ctx->stream;
  dfree(M->h1, st);
  dfree(M->h2, st);
  BAMG_TRY(dalloc(&M->h1, n * kNH, st));
  BAMG_TRY(dalloc(&M->h2, n * kNH, st));
  M->cap_rows = n;
  return Status{};
}

static Status mlp_forward(bamg_mlp* M, const float* X, int64_t n, float* w, bool keep, cudaStream_t st) {
  if (n <= 0) return Status{};
  if (keep) BAMG_TRY(mlp_reserve(M, n));
  { k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(M->theta_bf, X, n, w, keep ? M->h1 : nullptr,
                                                               keep ? M->h2 : nullptr); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

static Status mlp_gradient(bamg_mlp* M, const float* X, const float* t, int64_t n, float* w_tmp, float* loss,
                           cudaStream_t st) {
  BAMG_TRY(mlp_forward(M, X, n, w_tmp, true, st));
  int64_t per = (n + kBwdMaxCtas - 1) / kBwdMaxCtas;
  per = ((per + kBwdRowsPerChunk - 1) / kBwdRowsPerChunk) * kBwdRowsPerChunk;
  const int nb = (int)((n + per - 1) / per);
  { k_mlp_backward<<<nb, kBwdThreads, 0, st>>>(M->theta_bf, X, t, n, per, M->h1, M->h2, M->partials); BAMG_COUNT_LAUNCH; }
  { k_mlp_reduce<<<(kNP + 1 + 255) / 256, 256, 0, st>>>(M->partials, nb, M->grad, loss, n); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

// Learned weights of every non-coarsest level (features -> MLP), used by
// mg_update when an MLP is attached.
Status mg_learned_weights(bamg_mg* mg, int l, cudaStream_t st) {
  Level& L = mg->levels[l];
  if (!mg->mlp || !L.learned_w) return Status{};
  const bamg_bsr* A = L.A;
  const unsigned g = (unsigned)((L.n + 127) / 128);
  if (L.bs == 3) {
    if (A->vals64_stale)
      { k_block_features<3, float><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals32, L.dinv, L.n, (float)l, L.feat); BAMG_COUNT_LAUNCH; }
    else
      { k_block_features<3, double><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals, L.dinv, L.n, (float)l, L.feat); BAMG_COUNT_LAUNCH; }
  } else {
    if (A->vals64_stale)
      { k_block_features<6, float><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals32, L.dinv, L.n, (float)l, L.feat); BAMG_COUNT_LAUNCH; }
    else
      { k_block_features<6, double><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals, L.dinv, L.n, (float)l, L.feat); BAMG_COUNT_LAUNCH; }
  }
  BAMG_CUDA(cudaGetLastError());
  return mlp_forward(mg->mlp, L.feat, L.n, L.learned_w, false, st);
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_mlp_destroy(bamg_mlp* M);

bamg_status bamg_mlp_num_params(int* n) {
  if (!n) return BAMG_ERR_INVALID;
  *n = kNP;
  return BAMG_OK;
}

bamg_status bamg_mlp_create(bamg_ctx* ctx, uint64_t seed, bamg_mlp** out) {
  if (!ctx || !out) return BAMG_ERR_INVALID;
  *out = nullptr;
  bamg_mlp* M = new bamg_mlp();
  M->ctx = ctx;
  cudaStream_t st = ctx->stream;
  auto body = [&]() -> Status {
    // He-uniform initialisation from splitmix64(seed + index); biases zero
    std::vector<float> th(kNP, 0.f);
    auto u01 = [&](uint64_t d) {
      uint64_t z = seed + (d + 1) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return (double)(z >> 11) * 0x1.0p-53;
    };
    const double a1 = std::sqrt(6.0 / kNF), a2 = std::sqrt(6.0 / kNH);
    for (int e = 0; e < kNF * kNH; ++e) th[kOffW1 + e] = (float)((2 * u01(e) - 1) * a1);
    for (int e = 0; e < kNH * kNH; ++e) th[kOffW2 + e] = (float)((2 * u01(10000 + e) - 1) * a2);
    for (int e = 0; e < kNH; ++e) th[kOffW3 + e] = (float)((2 * u01(20000 + e) - 1) * a2 * 0.1);
    BAMG_TRY(upload(&M->theta, th, st));
    BAMG_TRY(dalloc(&M->theta_bf, kNP, st));
    BAMG_TRY(dalloc(&M->m, kNP, st));
    BAMG_TRY(dalloc(&M->v, kNP, st));
    BAMG_TRY(dalloc(&M->grad, kNP, st));
    BAMG_TRY(dalloc(&M->partials, (int64_t)kBwdMaxCtas * (kNP + 1), st));
    BAMG_CUDA(cudaMemsetAsync(M->m, 0, sizeof(float) * kNP, st));
    BAMG_CUDA(cudaMemsetAsync(M->v, 0, sizeof(float) * kNP, st));
    { k_round_params<<<(kNP + 255) / 256, 256, 0, st>>>(M->theta, M->theta_bf); BAMG_COUNT_LAUNCH; }
    BAMG_CUDA(cudaGetLastError());
    BAMG_CUDA(cudaStreamSynchronize(st));
    return Status{};
  };
  Status s = body();
  if (!s.ok()) {
    bamg_mlp_destroy(M);
    return fail(ctx, s);
  }
  *out = M;
  return BAMG_OK;
}

bamg_status bamg_mlp_destroy(bamg_mlp* M) {
  if (!M) return BAMG_OK;
  cudaStream_t st = M->ctx->stream;
  for (float** p : {&M->theta, &M->theta_bf, &M->m, &M->v, &M->grad, &M->partials}) dfree(*p, st);
  dfree(M->h1, st);
  dfree(M->h2, st);
  cudaStreamSynchronize(st);
  delete M;
  return BAMG_OK;
}

bamg_status bamg_mlp_get_params(const bamg_mlp* M, float* params) {
  if (!M || !params) return BAMG_ERR_INVALID;
  cudaError_t e = cudaMemcpyAsync(params, M->theta, sizeof(float) * kNP, cudaMemcpyDeviceToDevice, M->ctx->stream);
  return e == cudaSuccess ? BAMG_OK : fail(M->ctx, cuda_status(e, "get_params"));
}

bamg_status bamg_mlp_set_params(bamg_mlp* M, const float* params) {
  if (!M || !params) return BAMG_ERR_INVALID;
  cudaStream_t st = M->ctx->stream;
  auto body = [&]() -> Status {
    BAMG_CUDA(cudaMemcpyAsync(M->theta, params, sizeof(float) * kNP, cudaMemcpyDeviceToDevice, st));
    BAMG_CUDA(cudaMemsetAsync(M->m, 0, sizeof(float) * kNP, st));
    BAMG_CUDA(cudaMemsetAsync(M->v, 0, sizeof(float) * kNP, st));
    M->t = 0;
    { k_round_params<<<(kNP + 255) / 256, 256, 0, st>>>(M->theta, M->theta_bf); BAMG_COUNT_LAUNCH; }
    BAMG_CUDA(cudaGetLastError());
    return Status{};
  };
  Status s = body();
  return s.ok() ? BAMG_OK : fail(M->ctx, s);
}

bamg_status bamg_mlp_forward(bamg_mlp* M, const float* X, int64_t n, float* w) {
  if (!M || n < 0 || (n > 0 && (!X || !w))) return BAMG_ERR_INVALID;
  Status s = mlp_forward(M, X, n, w, false, M->ctx->stream);
  return s.ok() ? BAMG_OK : fail(M->ctx, s);
}

bamg_status bamg_mlp_gradient(bamg_mlp* M, const float* X, const float* t, int64_t n, float* w_tmp, float* grad,
                              float* loss) {
  if (!M || n <= 0 || !X || !t || !w_tmp) return BAMG_ERR_INVALID;
  cudaStream_t st = M->ctx->stream;
  Status s = mlp_gradient(M, X, t, n, w_tmp, loss, st);
  if (s.ok() && grad) {
    cudaError_t e = cudaMemcpyAsync(grad, M->grad, sizeof(float) * kNP, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) s = cuda_status(e, "gradient copy");
  }
  return s.ok() ? BAMG_OK : fail(M->ctx, s);
}

bamg_status bamg_mlp_train_step(bamg_mlp* M, const float* X, const float* t, int64_t n, float* w_tmp, float lr,
                                float* loss) {
  if (!M || n <= 0 || !X || !t || !w_tmp || !(lr > 0.f)) return BAMG_ERR_INVALID;
  cudaStream_t st = M->ctx->stream;
  Status s = mlp_gradient(M, X, t, n, w_tmp, loss, st);
  if (s.ok()) {
    M->t++;
    { k_mlp_adam<<<(kNP + 255) / 256, 256, 0, st>>>(M->theta, M->m, M->v, M->grad, M->theta_bf, lr, 0.9f, 0.999f,
                                                    1e-8f, M->t); BAMG_COUNT_LAUNCH; }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "adam");
  }
  return s.ok() ? BAMG_OK : fail(M->ctx, s);
}

bamg_status bamg_mg_block_features(bamg_mg* mg, int level, float* X) {
  if (!mg || !X || level < 0 || level + 1 >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  Level& L = mg->levels[level];
  const bamg_bsr* A = L.A;
  cudaStream_t st = mg->ctx->stream;
  const unsigned g = (unsigned)((L.n + 127) / 128);
  if (L.bs == 3) {
    if (A->vals64_stale)
      { k_block_features<3, float><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals32, L.dinv, L.n, (float)level, X); BAMG_COUNT_LAUNCH; }
    else
      { k_block_features<3, double><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals, L.dinv, L.n, (float)level, X); BAMG_COUNT_LAUNCH; }
  } else {
    if (A->vals64_stale)
      { k_block_features<6, float><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals32, L.dinv, L.n, (float)level, X); BAMG_COUNT_LAUNCH; }
    else
      { k_block_features<6, double><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals, L.dinv, L.n, (float)level, X); BAMG_COUNT_LAUNCH; }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BAMG_OK : fail(mg->ctx, cuda_status(e, "features"));
}

bamg_status bamg_mg_smoother_targets(bamg_mg* mg, const double* Bk, int k, float* targets) {
  if (!mg || !Bk || !targets || k < 1) return BAMG_ERR_INVALID;
  if (mg->opts.precision != BAMG_FP64)
    return fail(mg->ctx, make_status(BAMG_ERR_STATE, "targets are generated with the FP64 plain cycle"));
  bamg_ctx* ctx = mg->ctx;
  cudaStream_t st = ctx->stream;
  const int nl = (int)mg->levels.size();
  auto body = [&]() -> Status {
    std::vector<double*> num(nl, nullptr), den(nl, nullptr);
    Status s;
    for (int l = 0; l + 1 < nl && s.ok(); ++l) {
      const int64_t n = mg->levels[l].n;
      s = dalloc(&num[l], n, st);
      if (s.ok()) s = dalloc(&den[l], n, st);
      if (s.ok()) {
        cudaMemsetAsync(num[l], 0, sizeof(double) * n, st);
        cudaMemsetAsync(den[l], 0, sizeof(double) * n, st);
      }
    }
    const int64_t m0 = mg->levels[0].n * 3;
    for (int r = 0; r < k && s.ok(); ++r) {
      cudaMemcpyAsync(mg->levels[0].b, Bk + (int64_t)r * m0, sizeof(double) * m0, cudaMemcpyDeviceToDevice, st);
      for (int l = 0; l + 1 < nl && s.ok(); ++l) {
        s = mg_smooth_down_fp64(mg, l, st);
        if (!s.ok()) break;
        Level& L = mg->levels[l];
        const bamg_bsr* A = L.A;
        const unsigned g = (unsigned)((L.n + 127) / 128);
        const int64_t rows = row_threads(A);
        const unsigned gr = (unsigned)((rows + kRowThreads - 1) / kRowThreads);
        if (L.bs == 3) {
          { k_apply_dinv<3><<<g, 128, 0, st>>>(L.n, L.dinv, L.r, L.d0); BAMG_COUNT_LAUNCH; }
          BAMG_DISPATCH_V(A->vec, { k_damping_accum<3, V><<<gr, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, L.n, rows, L.d0, L.r, num[l], den[l]); BAMG_COUNT_LAUNCH; })
        } else {
          { k_apply_dinv<6><<<g, 128, 0, st>>>(L.n, L.dinv, L.r, L.d0); BAMG_COUNT_LAUNCH; }
          BAMG_DISPATCH_V(A->vec, { k_damping_accum<6, V><<<gr, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, L.n, rows, L.d0, L.r, num[l], den[l]); BAMG_COUNT_LAUNCH; })
        }
        s = mg_restrict_fp64(mg, l, st);
      }
    }
    int64_t off = 0;
    for (int l = 0; l + 1 < nl && s.ok(); ++l) {
      const int64_t n = mg->levels[l].n;
      { k_damping_finish<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, num[l], den[l], targets + off); BAMG_COUNT_LAUNCH; }
      off += n;
    }
    cudaError_t e = cudaGetLastError();
    if (s.ok() && e != cudaSuccess) s = cuda_status(e, "targets");
    cudaStreamSynchronize(st);
    for (int l = 0; l < nl; ++l) {
      dfree(num[l], st);
      dfree(den[l], st);
    }
    return s;
  };
  Status s = body();
  return s.ok() ? BAMG_OK : fail(ctx, s);
}

bamg_status bamg_mg_attach_mlp(bamg_mg* mg, bamg_mlp* M) {
  if (!mg) return BAMG_ERR_INVALID;
  cudaStream_t st = mg->ctx->stream;
  auto body = [&]() -> Status {
    for (size_t l = 0; l + 1 < mg->levels.size(); ++l) {
      Level& L = mg->levels[l];
      if (M && !L.feat) {
        BAMG_TRY(dalloc(&L.feat, L.n * kNF, st));
        BAMG_TRY(dalloc(&L.learned_w, L.n, st));
      }
      L.weights = M ? L.learned_w : nullptr;
    }
    mg->mlp = M;
    mg_release_graphs(mg);  // the captured iteration holds the weight pointers
    return Status{};
  };
  Status s = body();
  return s.ok() ? BAMG_OK : fail(mg->ctx, s);
}

bamg_status bamg_mg_stationary(bamg_mg* mg, const double* b, double* x, int its, double* rnorms) {
  if (!mg || !b || !x || its < 0 || !rnorms) return BAMG_ERR_INVALID;
  bamg_ctx* ctx = mg->ctx;
  cudaStream_t st = ctx->stream;
  Level& L0 = mg->levels[0];
  const bamg_bsr* A = L0.A;
  const int64_t m = L0.n * 3, rows = A->nslices * kSlice;
  auto body = [&]() -> Status {
    double* norms = nullptr;
    BAMG_TRY(dalloc(&norms, its + 1, st));
    const unsigned gv = (unsigned)((m + 255) / 256);
    const unsigned gr = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + kRowThreads - 1) / kRowThreads, 1216));
    BAMG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * m, st));
    { k_residual_store<<<gr, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, L0.n, rows, x, b, mg->cr, norms, ctx->d_partials, ctx->d_counters + 8); BAMG_COUNT_LAUNCH; }
    Status s;
    for (int k = 0; k < its && s.ok(); ++k) {
      s = mg_precond(mg, mg->cr, mg->cz, st);
      if (!s.ok()) break;
      { k_axpy<<<gv, 256, 0, st>>>(m, mg->cz, x); BAMG_COUNT_LAUNCH; }
      { k_residual_store<<<gr, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, L0.n, rows, x, b, mg->cr, norms + k + 1, ctx->d_partials, ctx->d_counters + 8); BAMG_COUNT_LAUNCH; }
    }
    std::vector<double> h;
    if (s.ok()) s = download(h, norms, its + 1, st);
    dfree(norms, st);
    if (s.ok())
      for (int k = 0; k <= its; ++k) rnorms[k] = std::sqrt(h[k]);
    return s;
  };
  Status s = body();
  return s.ok() ? BAMG_OK : fail(ctx, s);
}

}  // extern "C"
