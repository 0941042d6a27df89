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
constexpr int kBwdMaxCtas = 1216;  // CTAs of the training kernel (one partial-sum slot each)

}  // namespace bamg

struct bamg_mlp {
  bamg_ctx* ctx = nullptr;
  float* theta = nullptr;    // FP32 master parameters
  float* theta_bf = nullptr; // bfloat16-rounded copy (stored as float)
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  float* partials = nullptr; // kBwdMaxCtas x (kNP + 1)
  int64_t t = 0;             // Adam step count
  bool smem_set = false;     // training kernel's shared-memory limit raised
};

namespace bamg {

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float weight_of(float z) {
  const double s = 1.0 / (1.0 + exp(-(double)z));
  const float w = (float)(0.5 + 1.5 * s);
  return isfinite(w) ? w : 1.0f;  // a non-finite prediction falls back to the plain smoother
}

// ------------------------------------------------ tensor-core MLP kernels
//
// Both hidden layers run on the tensor cores as warp-level mma.sync
// m16n8k16 products, BF16 operands and FP32 accumulation.  Fragment layouts
// (PTX ISA, .bf16), with g = lane / 4 and t = lane % 4:
//   A 16x16 row-major:  a0 = (g, 2t..2t+1)  a1 = (g+8, 2t..)  a2 = (g, 2t+8..)  a3 = (g+8, 2t+8..)
//   B 16x8 col-major:   b0 = (2t..2t+1, g)  b1 = (2t+8..2t+9, g)
//   C 16x8 FP32:        c0, c1 = (g, 2t..2t+1)  c2, c3 = (g+8, 2t..2t+1)
// The C tiles of output columns 16q .. 16q+15 (n-tiles 2q and 2q+1) are the
// A fragment of k-tile q of the next product, so a warp's 16 rows go through
// both layers (and back) without leaving registers.  Layer 1 has K = 8: its A
// and B fragments are zero-padded to K = 16.
constexpr int kTcRows = 16;                   // rows of one warp tile
constexpr int kTcWarps = 4;
constexpr int kTcChunk = kTcRows * kTcWarps;  // rows of one CTA step
constexpr int kLd = kNH + 8;                  // padded row of a 64-wide bf16 tile: conflict-free fragment loads
constexpr int kLdX = 24;                      // x tile: 16 columns (8 features, the ones column, zeros) + padding

// Parameters in shared memory: W2 both ways round (B operand of the forward
// product and of the backward product), W1, biases and w3 as floats.
struct __align__(16) TcWeights {
  __nv_bfloat16 w2t[kNH][kLd];  // w2t[k][j] = W2[j][k]
  __nv_bfloat16 w2[kNH][kLd];   // w2[j][k]  = W2[j][k]
  float w1[kNF][kNH];
  float b1[kNH], b2[kNH], w3[kNH];
  float b3, pad[3];
};

struct __align__(16) TcTrainSmem {
  TcWeights W;
  __nv_bfloat16 h1[kTcChunk][kLd];   // hidden layer 1 of the chunk's rows
  __nv_bfloat16 d2[kTcChunk][kLd];   // dL/d(a2)
  __nv_bfloat16 d1[kTcChunk][kLd];   // dL/d(a1)
  __nv_bfloat16 x[kTcChunk][kLdX];   // features, then 1 (valid rows), then zeros
  float red[kTcWarps][2][kNH];       // per-warp column sums (b2, w3 gradients)
  float red2[kTcWarps][2];           // per-warp b3 gradient and squared error
};

__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // lo in the low half (lower column)
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ void sts32(__nv_bfloat16* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four transposed 8x8 bf16 tiles; lane l gives the address of row l % 8 of tile l / 8.
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const __nv_bfloat16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// Parameters (already bf16-exact floats) into shared memory; the caller syncs.
__device__ void tc_load_weights(TcWeights& W, const float* __restrict__ pbf) {
  for (int e = threadIdx.x; e < kNH * kNH; e += blockDim.x) {
    const int j = e / kNH, k = e % kNH;
    const __nv_bfloat16 v = __float2bfloat16_rn(pbf[kOffW2 + e]);
    W.w2[j][k] = v;
    W.w2t[k][j] = v;
  }
  for (int e = threadIdx.x; e < kNF * kNH; e += blockDim.x) W.w1[e / kNH][e % kNH] = pbf[kOffW1 + e];
  for (int e = threadIdx.x; e < kNH; e += blockDim.x) {
    W.b1[e] = pbf[kOffB1 + e];
    W.b2[e] = pbf[kOffB2 + e];
    W.w3[e] = pbf[kOffW3 + e];
  }
  if (threadIdx.x == 0) W.b3 = pbf[kOffB3];
}

// B fragments of layer 1 (n-tile jn, K padded: the second register is zero).
__device__ __forceinline__ void tc_w1_frags(const TcWeights& W, int g, int t, uint32_t (&w1f)[8]) {
#pragma unroll
  for (int jn = 0; jn < 8; ++jn) w1f[jn] = bf2(W.w1[2 * t][8 * jn + g], W.w1[2 * t + 1][8 * jn + g]);
}

// Forward pass of the warp tile of rows r0 .. r0+15 (rows >= rend read as
// zero features).  Returns the packed features, layer 1 as A fragments, the
// bf16-rounded layer 2 in C layout, and z of rows r0+g and r0+g+8 (in every
// lane of the quad).
__device__ __forceinline__ void tc_forward(const TcWeights& W, const uint32_t (&w1f)[8], const float* __restrict__ X,
                                           const int64_t* __restrict__ idx, int64_t r0, int64_t rend, int g, int t,
                                           uint32_t (&xa)[2], uint32_t (&h1a)[4][4], float (&h2)[8][4],
                                           float (&z)[2]) {
  const int64_t ra = r0 + g, rb = r0 + g + 8;
  float2 xv0 = make_float2(0.f, 0.f), xv1 = make_float2(0.f, 0.f);
  if (ra < rend) xv0 = *reinterpret_cast<const float2*>(X + (idx ? idx[ra] : ra) * kNF + 2 * t);
  if (rb < rend) xv1 = *reinterpret_cast<const float2*>(X + (idx ? idx[rb] : rb) * kNF + 2 * t);
  xa[0] = bf2(xv0.x, xv0.y);
  xa[1] = bf2(xv1.x, xv1.y);
  const uint32_t a1[4] = {xa[0], xa[1], 0u, 0u};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int jn = 2 * q + half, c = 8 * jn + 2 * t;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(acc, a1, w1f[jn], 0u);
      h1a[q][2 * half] = bf2(fmaxf(acc[0] + W.b1[c], 0.f), fmaxf(acc[1] + W.b1[c + 1], 0.f));
      h1a[q][2 * half + 1] = bf2(fmaxf(acc[2] + W.b1[c], 0.f), fmaxf(acc[3] + W.b1[c + 1], 0.f));
    }
  }
  float za = 0.f, zb = 0.f;
#pragma unroll
  for (int jn = 0; jn < 8; ++jn) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      mma_bf16(acc, h1a[q], lds32(&W.w2t[8 * jn + g][16 * q + 2 * t]), lds32(&W.w2t[8 * jn + g][16 * q + 8 + 2 * t]));
    const int c = 8 * jn + 2 * t;
    h2[jn][0] = bfr(fmaxf(acc[0] + W.b2[c], 0.f));
    h2[jn][1] = bfr(fmaxf(acc[1] + W.b2[c + 1], 0.f));
    h2[jn][2] = bfr(fmaxf(acc[2] + W.b2[c], 0.f));
    h2[jn][3] = bfr(fmaxf(acc[3] + W.b2[c + 1], 0.f));
    za = fmaf(h2[jn][0], W.w3[c], fmaf(h2[jn][1], W.w3[c + 1], za));
    zb = fmaf(h2[jn][2], W.w3[c], fmaf(h2[jn][3], W.w3[c + 1], zb));
  }
  za += __shfl_xor_sync(0xffffffffu, za, 1);
  za += __shfl_xor_sync(0xffffffffu, za, 2);
  zb += __shfl_xor_sync(0xffffffffu, zb, 1);
  zb += __shfl_xor_sync(0xffffffffu, zb, 2);
  z[0] = za + W.b3;
  z[1] = zb + W.b3;
}

// Inference: every warp takes 16-row tiles in turn.
__global__ void __launch_bounds__(kTcWarps * 32) k_mlp_forward_tc(const float* __restrict__ pbf,
                                                                  const float* __restrict__ X, int64_t n,
                                                                  float* __restrict__ w_out) {
  __shared__ TcWeights W;
  tc_load_weights(W, pbf);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  uint32_t w1f[8];
  tc_w1_frags(W, g, t, w1f);
  for (int64_t r0 = ((int64_t)blockIdx.x * kTcWarps + warp) * kTcRows; r0 < n;
       r0 += (int64_t)gridDim.x * kTcChunk) {
    uint32_t xa[2], h1a[4][4];
    float h2[8][4], z[2];
    tc_forward(W, w1f, X, nullptr, r0, n, g, t, xa, h1a, h2, z);
    if (t == 0) {
      if (r0 + g < n) w_out[r0 + g] = weight_of(z[0]);
      if (r0 + g + 8 < n) w_out[r0 + g + 8] = weight_of(z[1]);
    }
  }
}

// Training: gradient of mean((w - t)^2) over n rows (row r of the batch is
// row idx[r] of X and tgt, or row r without idx).  CTA b takes rows
// [b * rows_per_cta, ...) in chunks of 64 (16 per warp): forward, dz, the
// backward signal d2 = dz w3 (masked by a2 > 0) and d1 = d2 W2^T (masked by
// a1 > 0) in registers; then the chunk's weight gradients h1^T d2 and
// x^T d1 from shared memory (the ones column of x gives the b1 gradient).
// Per-CTA partial sums go to partials[b] (squared error at index kNP).
__global__ void __launch_bounds__(kTcWarps * 32) k_mlp_train_tc(const float* __restrict__ pbf,
                                                                const float* __restrict__ X,
                                                                const float* __restrict__ tgt,
                                                                const int64_t* __restrict__ idx, int64_t n,
                                                                int64_t rows_per_cta, float* __restrict__ w_out,
                                                                float* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char tc_smem[];
  TcTrainSmem& S = *reinterpret_cast<TcTrainSmem*>(tc_smem);
  tc_load_weights(S.W, pbf);
  __syncthreads();
  const TcWeights& W = S.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int mi = lane >> 3, mr = lane & 7;  // ldmatrix: tile and row this lane addresses
  uint32_t w1f[8];
  tc_w1_frags(W, g, t, w1f);
  float gW2[8][4], gW1[2][4], gb2[8][2], gw3[8][2], gb3 = 0.f, sq = 0.f;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
#pragma unroll
    for (int b = 0; b < 4; ++b) gW2[a][b] = 0.f;
    gb2[a][0] = gb2[a][1] = gw3[a][0] = gw3[a][1] = 0.f;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) gW1[0][b] = gW1[1][b] = 0.f;
  const double scale = 2.0 / (double)n;
  const int64_t rbeg = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t rend = n < rbeg + rows_per_cta ? n : rbeg + rows_per_cta;
  const int lr = kTcRows * warp;  // the warp's first row in the chunk
  for (int64_t c0 = rbeg; c0 < rend; c0 += kTcChunk) {
    const int64_t r0 = c0 + lr;
    uint32_t xa[2], h1a[4][4];
    float h2[8][4], z[2];
    tc_forward(W, w1f, X, idx, r0, rend, g, t, xa, h1a, h2, z);
    const bool va = r0 + g < rend, vb = r0 + g + 8 < rend;
    sts32(&S.x[lr + g][2 * t], xa[0]);
    sts32(&S.x[lr + g + 8][2 * t], xa[1]);
    sts32(&S.x[lr + g][8 + 2 * t], (t == 0 && va) ? bf2(1.f, 0.f) : 0u);
    sts32(&S.x[lr + g + 8][8 + 2 * t], (t == 0 && vb) ? bf2(1.f, 0.f) : 0u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sts32(&S.h1[lr + g][16 * q + 2 * t], h1a[q][0]);
      sts32(&S.h1[lr + g + 8][16 * q + 2 * t], h1a[q][1]);
      sts32(&S.h1[lr + g][16 * q + 8 + 2 * t], h1a[q][2]);
      sts32(&S.h1[lr + g + 8][16 * q + 8 + 2 * t], h1a[q][3]);
    }
    // dz of rows g and g+8 (the same in the four lanes of a quad)
    float dz[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t row = r0 + g + 8 * h;
      dz[h] = 0.f;
      if (h == 0 ? va : vb) {
        const double sg = 1.0 / (1.0 + exp(-(double)z[h]));
        const double e = 0.5 + 1.5 * sg - (double)tgt[idx ? idx[row] : row];
        dz[h] = (float)(scale * e * 1.5 * sg * (1.0 - sg));
        if (t == 0) {
          sq += (float)(e * e);
          gb3 += dz[h];
          if (w_out) w_out[row] = weight_of(z[h]);
        }
      }
    }
    // d2 = dz w3 where a2 > 0; column sums for the b2 and w3 gradients
    uint32_t d2a[4][4];
#pragma unroll
    for (int jn = 0; jn < 8; ++jn) {
      const int c = 8 * jn + 2 * t;
      const float e0 = h2[jn][0] > 0.f ? dz[0] * W.w3[c] : 0.f;
      const float e1 = h2[jn][1] > 0.f ? dz[0] * W.w3[c + 1] : 0.f;
      const float e2 = h2[jn][2] > 0.f ? dz[1] * W.w3[c] : 0.f;
      const float e3 = h2[jn][3] > 0.f ? dz[1] * W.w3[c + 1] : 0.f;
      gb2[jn][0] += e0 + e2;
      gb2[jn][1] += e1 + e3;
      gw3[jn][0] = fmaf(dz[0], h2[jn][0], fmaf(dz[1], h2[jn][2], gw3[jn][0]));
      gw3[jn][1] = fmaf(dz[0], h2[jn][1], fmaf(dz[1], h2[jn][3], gw3[jn][1]));
      d2a[jn >> 1][2 * (jn & 1)] = bf2(e0, e1);
      d2a[jn >> 1][2 * (jn & 1) + 1] = bf2(e2, e3);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sts32(&S.d2[lr + g][16 * q + 2 * t], d2a[q][0]);
      sts32(&S.d2[lr + g + 8][16 * q + 2 * t], d2a[q][1]);
      sts32(&S.d2[lr + g][16 * q + 8 + 2 * t], d2a[q][2]);
      sts32(&S.d2[lr + g + 8][16 * q + 8 + 2 * t], d2a[q][3]);
    }
    // d1 = d2 W2^T where a1 > 0
#pragma unroll
    for (int jn = 0; jn < 8; ++jn) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        mma_bf16(acc, d2a[q], lds32(&W.w2[8 * jn + g][16 * q + 2 * t]), lds32(&W.w2[8 * jn + g][16 * q + 8 + 2 * t]));
      const uint32_t ha = h1a[jn >> 1][2 * (jn & 1)], hb = h1a[jn >> 1][2 * (jn & 1) + 1];
      sts32(&S.d1[lr + g][8 * jn + 2 * t], bf2(bf_lo(ha) > 0.f ? acc[0] : 0.f, bf_hi(ha) > 0.f ? acc[1] : 0.f));
      sts32(&S.d1[lr + g + 8][8 * jn + 2 * t], bf2(bf_lo(hb) > 0.f ? acc[2] : 0.f, bf_hi(hb) > 0.f ? acc[3] : 0.f));
    }
    __syncthreads();
    // weight gradients of the chunk: warp w owns rows 16w .. 16w+15 of the
    // W2 gradient (h1^T d2) and columns 16w .. 16w+15 of the W1 gradient (x^T d1)
#pragma unroll
    for (int s = 0; s < kTcWarps; ++s) {
      const int rr = kTcRows * s + (mi >> 1) * 8 + mr;  // A tiles: rows of the k-step, columns by tile
      uint32_t a[4];
      ldsm_x4_t(a, &S.h1[rr][16 * warp + (mi & 1) * 8]);
#pragma unroll
      for (int jp = 0; jp < 4; ++jp) {
        uint32_t b[4];
        ldsm_x4_t(b, &S.d2[kTcRows * s + (mi & 1) * 8 + mr][16 * jp + (mi >> 1) * 8]);
        mma_bf16(gW2[2 * jp], a, b[0], b[1]);
        mma_bf16(gW2[2 * jp + 1], a, b[2], b[3]);
      }
      uint32_t ax[4], bx[4];
      ldsm_x4_t(ax, &S.x[rr][(mi & 1) * 8]);
      ldsm_x4_t(bx, &S.d1[kTcRows * s + (mi & 1) * 8 + mr][16 * warp + (mi >> 1) * 8]);
      mma_bf16(gW1[0], ax, bx[0], bx[1]);
      mma_bf16(gW1[1], ax, bx[2], bx[3]);
    }
    __syncthreads();
  }
  float* out = partials + (int64_t)blockIdx.x * (kNP + 1);
#pragma unroll
  for (int jn = 0; jn < 8; ++jn) {
    const int j0 = 16 * warp + g, k = 8 * jn + 2 * t;
    out[kOffW2 + j0 * kNH + k] = gW2[jn][0];
    out[kOffW2 + j0 * kNH + k + 1] = gW2[jn][1];
    out[kOffW2 + (j0 + 8) * kNH + k] = gW2[jn][2];
    out[kOffW2 + (j0 + 8) * kNH + k + 1] = gW2[jn][3];
  }
#pragma unroll
  for (int nn = 0; nn < 2; ++nn) {
    const int j = 16 * warp + 8 * nn + 2 * t;
    out[kOffW1 + g * kNH + j] = gW1[nn][0];
    out[kOffW1 + g * kNH + j + 1] = gW1[nn][1];
    if (g == 0) {  // row 8 of the padded x^T d1: the ones column
      out[kOffB1 + j] = gW1[nn][2];
      out[kOffB1 + j + 1] = gW1[nn][3];
    }
  }
  // column sums over the warp's rows (lanes of equal t), then over the warps in order
#pragma unroll
  for (int jn = 0; jn < 8; ++jn)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float b2s = gb2[jn][c], w3s = gw3[jn][c];
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        b2s += __shfl_xor_sync(0xffffffffu, b2s, o);
        w3s += __shfl_xor_sync(0xffffffffu, w3s, o);
      }
      if (g == 0) {
        S.red[warp][0][8 * jn + 2 * t + c] = b2s;
        S.red[warp][1][8 * jn + 2 * t + c] = w3s;
      }
    }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if (lane == 0) {
    S.red2[warp][0] = gb3;
    S.red2[warp][1] = sq;
  }
  __syncthreads();
  if (threadIdx.x < kNH) {
    float b2s = 0.f, w3s = 0.f;
    for (int w = 0; w < kTcWarps; ++w) {
      b2s += S.red[w][0][threadIdx.x];
      w3s += S.red[w][1][threadIdx.x];
    }
    out[kOffB2 + threadIdx.x] = b2s;
    out[kOffW3 + threadIdx.x] = w3s;
  } else if (threadIdx.x == kNH) {
    float b3s = 0.f, sqs = 0.f;
    for (int w = 0; w < kTcWarps; ++w) {
      b3s += S.red2[w][0];
      sqs += S.red2[w][1];
    }
    out[kOffB3] = b3s;
    out[kNP] = sqs;
  }
}

// grad[p] = sum over CTAs of partials[b][p] in CTA order; loss = sum / n.
// With loss_sum, the batch's summed squared error is also added to it.
__global__ void k_mlp_reduce(const float* __restrict__ partials, int nb, float* __restrict__ grad,
                             float* __restrict__ loss_out, int64_t n, double* __restrict__ loss_sum) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kNP) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += (double)partials[(int64_t)b * (kNP + 1) + p];
  if (p < kNP) {
    grad[p] = (float)s;
  } else {
    if (loss_out) *loss_out = (float)(s / (double)n);
    if (loss_sum) *loss_sum += s;
  }
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
                                 const int* __restrict__ srow, const double* __restrict__ dinv, int64_t n,
                                 int64_t npos, float level, float* __restrict__ X) {
  constexpr int B = BS * BS;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= npos) return;
  const int64_t i = row_at(srow, pos);
  if (i < 0 || i >= n) return;
  const int64_t s = pos >> 5;
  const int lane = (int)(pos & 31);
  const int c0 = slice_ptr[s];
  const int len = rowptr[i + 1] - rowptr[i];
  double D[BS][BS];
  const int64_t db = (i >> 5) * (32LL * B) + (i & 31);
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
                                                               const double* __restrict__ vals,
                                                               const int* __restrict__ srow, int64_t n,
                                                               int64_t nthreads, const double* __restrict__ u,
                                                               const double* __restrict__ r, double* __restrict__ num,
                                                               double* __restrict__ den) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  int64_t pos;
  int sub;
  row_of_thread<V>(t, pos, sub);
  double q[BS];
  row_product<BS, BS, V, double, double, double>(sp, col, vals, u, pos, sub, q);
  const int64_t i = row_at(srow, pos);
  if (sub != 0 || i < 0 || i >= n) return;
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
                                                                const double* __restrict__ vals,
                                                                const int* __restrict__ srow, int64_t n,
                                                                int64_t rows_pad, const double* __restrict__ x,
                                                                const double* __restrict__ b, double* __restrict__ r,
                                                                double* out_norm2, double* partials, unsigned* counter) {
  double local[1] = {0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < rows_pad; pos += stride) {
    double acc[3];
    row_product<3, 3, 1, double, double, double>(sp, col, vals, x, pos, 0, acc);
    const int64_t i = row_at(srow, pos);
    if (i >= 0 && i < n) {
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

static Status mlp_forward(bamg_mlp* M, const float* X, int64_t n, float* w, cudaStream_t st) {
  if (n <= 0) return Status{};
  const int64_t tiles = (n + kTcChunk - 1) / kTcChunk;
  const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)M->ctx->sm_count * 4));
  { k_mlp_forward_tc<<<nb, kTcWarps * 32, 0, st>>>(M->theta_bf, X, n, w); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

// Rows per CTA of the training kernel: whole 64-row chunks, at least four
// of them (each CTA first stages the parameters), at most two CTAs per SM.
static int64_t train_rows_per_cta(int64_t n, int sm_count) {
  int64_t per = (n + 2 * sm_count - 1) / (2 * (int64_t)sm_count);
  per = std::max<int64_t>(per, 4 * kTcChunk);
  return (per + kTcChunk - 1) / kTcChunk * kTcChunk;
}

static Status mlp_gradient(bamg_mlp* M, const float* X, const float* t, const int64_t* idx, int64_t n,
                           float* w_tmp, float* loss, double* loss_sum, cudaStream_t st) {
  const size_t smem = sizeof(TcTrainSmem);
  if (!M->smem_set) {
    BAMG_CUDA(cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    M->smem_set = true;
  }
  const int64_t per = train_rows_per_cta(n, M->ctx->sm_count);
  const int nb = (int)((n + per - 1) / per);
  if (nb > kBwdMaxCtas) return make_status(BAMG_ERR_INVALID, "too many rows for one training step");
  { k_mlp_train_tc<<<nb, kTcWarps * 32, smem, st>>>(M->theta_bf, X, t, idx, n, per, w_tmp, M->partials); BAMG_COUNT_LAUNCH; }
  { k_mlp_reduce<<<(kNP + 1 + 255) / 256, 256, 0, st>>>(M->partials, nb, M->grad, loss, n, loss_sum); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

static Status mlp_adam(bamg_mlp* M, float lr, cudaStream_t st) {
  M->t++;
  { k_mlp_adam<<<(kNP + 255) / 256, 256, 0, st>>>(M->theta, M->m, M->v, M->grad, M->theta_bf, lr, 0.9f, 0.999f, 1e-8f,
                                                  M->t); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

// Learned weights of every non-coarsest level (features -> MLP), used by
// mg_update when an MLP is attached.
Status mg_learned_weights(bamg_mg* mg, int l, cudaStream_t st) {
  Level& L = mg->levels[l];
  if (!mg->mlp || !L.learned_w) return Status{};
  const bamg_bsr* A = L.A;
  const int64_t npos = A->nslices * kSlice;
  const unsigned g = (unsigned)std::max<int64_t>(1, (npos + 127) / 128);
  if (L.bs == 3) {
    if (A->vals64_stale)
      { k_block_features<3, float><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals32, A->slot_row, L.dinv, L.n, npos, (float)l, L.feat); BAMG_COUNT_LAUNCH; }
    else
      { k_block_features<3, double><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals, A->slot_row, L.dinv, L.n, npos, (float)l, L.feat); BAMG_COUNT_LAUNCH; }
  } else {
    if (A->vals64_stale)
      { k_block_features<6, float><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals32, A->slot_row, L.dinv, L.n, npos, (float)l, L.feat); BAMG_COUNT_LAUNCH; }
    else
      { k_block_features<6, double><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals, A->slot_row, L.dinv, L.n, npos, (float)l, L.feat); BAMG_COUNT_LAUNCH; }
  }
  BAMG_CUDA(cudaGetLastError());
  return mlp_forward(mg->mlp, L.feat, L.n, L.learned_w, st);
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
  Status s = mlp_forward(M, X, n, w, M->ctx->stream);
  return s.ok() ? BAMG_OK : fail(M->ctx, s);
}

bamg_status bamg_mlp_gradient(bamg_mlp* M, const float* X, const float* t, int64_t n, float* w_tmp, float* grad,
                              float* loss) {
  if (!M || n <= 0 || !X || !t || !w_tmp) return BAMG_ERR_INVALID;
  cudaStream_t st = M->ctx->stream;
  Status s = mlp_gradient(M, X, t, nullptr, n, w_tmp, loss, nullptr, st);
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
  Status s = mlp_gradient(M, X, t, nullptr, n, w_tmp, loss, nullptr, st);
  if (s.ok()) s = mlp_adam(M, lr, st);
  return s.ok() ? BAMG_OK : fail(M->ctx, s);
}

bamg_status bamg_mlp_train_epoch(bamg_mlp* M, const float* X, const float* t, const int64_t* perm, int64_t n,
                                 int64_t batch, float lr, double* loss_sum) {
  if (!M || n <= 0 || batch <= 0 || !X || !t || !perm || !(lr > 0.f)) return BAMG_ERR_INVALID;
  cudaStream_t st = M->ctx->stream;
  Status s;
  for (int64_t s0 = 0; s0 < n && s.ok(); s0 += batch) {
    const int64_t m = std::min(batch, n - s0);
    s = mlp_gradient(M, X, t, perm + s0, m, nullptr, nullptr, loss_sum, st);
    if (s.ok()) s = mlp_adam(M, lr, st);
  }
  return s.ok() ? BAMG_OK : fail(M->ctx, s);
}

bamg_status bamg_mg_block_features(bamg_mg* mg, int level, float* X) {
  if (!mg || !X || level < 0 || level + 1 >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  Level& L = mg->levels[level];
  const bamg_bsr* A = L.A;
  cudaStream_t st = mg->ctx->stream;
  const int64_t npos = A->nslices * kSlice;
  const unsigned g = (unsigned)std::max<int64_t>(1, (npos + 127) / 128);
  if (L.bs == 3) {
    if (A->vals64_stale)
      { k_block_features<3, float><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals32, A->slot_row, L.dinv, L.n, npos, (float)level, X); BAMG_COUNT_LAUNCH; }
    else
      { k_block_features<3, double><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals, A->slot_row, L.dinv, L.n, npos, (float)level, X); BAMG_COUNT_LAUNCH; }
  } else {
    if (A->vals64_stale)
      { k_block_features<6, float><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals32, A->slot_row, L.dinv, L.n, npos, (float)level, X); BAMG_COUNT_LAUNCH; }
    else
      { k_block_features<6, double><<<g, 128, 0, st>>>(A->rowptr, A->slice_ptr, A->sell_col, A->vals, A->slot_row, L.dinv, L.n, npos, (float)level, X); BAMG_COUNT_LAUNCH; }
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
          BAMG_DISPATCH_V(A->vec, { k_damping_accum<3, V><<<gr, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, A->slot_row, L.n, rows, L.d0, L.r, num[l], den[l]); BAMG_COUNT_LAUNCH; })
        } else {
          { k_apply_dinv<6><<<g, 128, 0, st>>>(L.n, L.dinv, L.r, L.d0); BAMG_COUNT_LAUNCH; }
          BAMG_DISPATCH_V(A->vec, { k_damping_accum<6, V><<<gr, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, A->slot_row, L.n, rows, L.d0, L.r, num[l], den[l]); BAMG_COUNT_LAUNCH; })
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
    { k_residual_store<<<gr, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, A->slot_row, L0.n, rows, x, b, mg->cr, norms, ctx->d_partials, ctx->d_counters + 8); BAMG_COUNT_LAUNCH; }
    Status s;
    for (int k = 0; k < its && s.ok(); ++k) {
      s = mg_precond(mg, mg->cr, mg->cz, st);
      if (!s.ok()) break;
      { k_axpy<<<gv, 256, 0, st>>>(m, mg->cz, x); BAMG_COUNT_LAUNCH; }
      { k_residual_store<<<gr, kRowThreads, 0, st>>>(A->slice_ptr, A->sell_col, A->vals, A->slot_row, L0.n, rows, x, b, mg->cr, norms + k + 1, ctx->d_partials, ctx->d_counters + 8); BAMG_COUNT_LAUNCH; }
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
