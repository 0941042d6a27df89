// Smoothed-aggregation hierarchy: cold setup (Sec. 2.2, Sec. 3.2), hot reuse
// update (Sec. 3.1), smoother data (point-block Jacobi, Sec. 4.1, under
// Chebyshev acceleration) and the state-gated transpose R = P^T.
#include <algorithm>
#include <cmath>
#include <memory>

#include "device.cuh"
#include "internal.h"

namespace bamg {

// ----------------------------------------------------------------- host setup

// Per direction with m nodes: n_a = max(1, m / 3) aggregates; node i joins
// min(i / 3, n_a - 1) (a remainder of one or two nodes joins the last one).
static void aggregates(const int grid[3], std::vector<int>& agg, int cgrid[3]) {
  std::vector<int> a1[3];
  for (int d = 0; d < 3; ++d) {
    const int m = grid[d];
    const int na = std::max(1, m / 3);
    cgrid[d] = na;
    a1[d].resize(m);
    for (int i = 0; i < m; ++i) a1[d][i] = std::min(i / 3, na - 1);
  }
  const int64_t n = (int64_t)grid[0] * grid[1] * grid[2];
  agg.resize(n);
  for (int64_t v = 0; v < n; ++v) {
    const int ix = (int)(v % grid[0]), iy = (int)((v / grid[0]) % grid[1]), iz = (int)(v / ((int64_t)grid[0] * grid[1]));
    agg[v] = a1[0][ix] + cgrid[0] * (a1[1][iy] + cgrid[1] * a1[2][iz]);
  }
}

// Rigid-body modes of fine nodes relative to their aggregate's centroid:
// columns translations x, y, z, then rotations (-y, x, 0), (0, -z, y), (z, 0, -x);
// clamped nodes and nodes outside every aggregate (agg -1) get zero rows.
// Layout: node-major 3 x 6 row-major.
static std::vector<double> rigid_modes(const double* coords, const uint8_t* dir, const std::vector<int>& agg,
                                       int64_t nagg) {
  const int64_t n = (int64_t)agg.size();
  std::vector<double> cen(nagg * 3, 0.0), cnt(nagg, 0.0), B(n * 18, 0.0);
  for (int64_t v = 0; v < n; ++v) {
    if (agg[v] < 0) continue;
    for (int d = 0; d < 3; ++d) cen[agg[v] * 3 + d] += coords[v * 3 + d];
    cnt[agg[v]] += 1.0;
  }
  for (int64_t a = 0; a < nagg; ++a)
    for (int d = 0; d < 3; ++d) cen[a * 3 + d] /= std::max(cnt[a], 1.0);
  for (int64_t v = 0; v < n; ++v) {
    if ((dir && dir[v]) || agg[v] < 0) continue;
    const double x = coords[v * 3] - cen[agg[v] * 3], y = coords[v * 3 + 1] - cen[agg[v] * 3 + 1],
                 z = coords[v * 3 + 2] - cen[agg[v] * 3 + 2];
    double* b = &B[v * 18];
    b[0 * 6 + 0] = b[1 * 6 + 1] = b[2 * 6 + 2] = 1.0;
    b[0 * 6 + 3] = -y;
    b[1 * 6 + 3] = x;
    b[1 * 6 + 4] = -z;
    b[2 * 6 + 4] = y;
    b[0 * 6 + 5] = z;
    b[2 * 6 + 5] = -x;
  }
  return B;
}

// Thin Householder QR of an m x 6 row-major matrix: Q (m x 6), R (6 x 6 upper)
// with diag(R) > 0.  Returns false if the columns are rank deficient.
static bool thin_qr(int m, const double* Bm, double* Q, double* R) {
  const int k = 6;
  std::vector<double> a(Bm, Bm + (size_t)m * k), v((size_t)m * k, 0.0), beta(k, 0.0);
  double colmax = 0.0;
  for (int j = 0; j < k; ++j) {
    double nrm2 = 0.0;
    for (int i = j; i < m; ++i) nrm2 += a[(size_t)i * k + j] * a[(size_t)i * k + j];
    const double nrm = std::sqrt(nrm2);
    colmax = std::max(colmax, nrm);
    if (nrm <= 1e-12 * std::max(colmax, 1e-300)) return false;
    const double x0 = a[(size_t)j * k + j];
    const double alpha = x0 >= 0 ? -nrm : nrm;  // H x = alpha e_j
    for (int i = 0; i < m; ++i) v[(size_t)i * k + j] = 0.0;
    v[(size_t)j * k + j] = x0 - alpha;
    for (int i = j + 1; i < m; ++i) v[(size_t)i * k + j] = a[(size_t)i * k + j];
    double vv = 0.0;
    for (int i = j; i < m; ++i) vv += v[(size_t)i * k + j] * v[(size_t)i * k + j];
    beta[j] = vv > 0 ? 2.0 / vv : 0.0;
    for (int c = j; c < k; ++c) {
      double s = 0.0;
      for (int i = j; i < m; ++i) s += v[(size_t)i * k + j] * a[(size_t)i * k + c];
      s *= beta[j];
      for (int i = j; i < m; ++i) a[(size_t)i * k + c] -= s * v[(size_t)i * k + j];
    }
  }
  // R = upper part of a; Q = H_0 ... H_5 [I; 0]
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) R[i * k + j] = j >= i ? a[(size_t)i * k + j] : 0.0;
  std::vector<double> q((size_t)m * k, 0.0);
  for (int j = 0; j < k; ++j) q[(size_t)j * k + j] = 1.0;
  for (int j = k - 1; j >= 0; --j) {
    for (int c = 0; c < k; ++c) {
      double s = 0.0;
      for (int i = j; i < m; ++i) s += v[(size_t)i * k + j] * q[(size_t)i * k + c];
      s *= beta[j];
      for (int i = j; i < m; ++i) q[(size_t)i * k + c] -= s * v[(size_t)i * k + j];
    }
  }
  for (int j = 0; j < k; ++j) {
    if (R[j * k + j] < 0) {
      for (int c = j; c < k; ++c) R[j * k + c] = -R[j * k + c];
      for (int i = 0; i < m; ++i) q[(size_t)i * k + j] = -q[(size_t)i * k + j];
    }
  }
  std::copy(q.begin(), q.end(), Q);
  return true;
}

static uint64_t splitmix64_host(uint64_t d, uint64_t seed) {
  uint64_t z = seed + (d + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Stacked near-null rows of the vertices `mem` of level l: at the fine level
// the rigid-body modes about the vertices' centroid (clamped nodes zero), on
// coarse levels the vertices' 6 x 6 blocks of B.  True if they have full
// column rank (the thin QR of the tentative prolongator succeeds).
static bool near_null_full_rank(int l, const std::vector<int>& mem, const double* coords, const uint8_t* dir,
                                const std::vector<double>& B) {
  const int bs = l == 0 ? 3 : 6;
  const int m = (int)mem.size() * bs;
  if (m < 6) return false;
  std::vector<double> Bm((size_t)m * 6, 0.0), Q((size_t)m * 6), R(36);
  if (l == 0) {
    double c[3] = {0, 0, 0};
    for (int v : mem)
      for (int d = 0; d < 3; ++d) c[d] += coords[(int64_t)v * 3 + d];
    for (int d = 0; d < 3; ++d) c[d] /= (double)mem.size();
    for (size_t u = 0; u < mem.size(); ++u) {
      const int64_t v = mem[u];
      if (dir && dir[v]) continue;
      const double x = coords[v * 3] - c[0], y = coords[v * 3 + 1] - c[1], z = coords[v * 3 + 2] - c[2];
      double* b = &Bm[u * 18];
      b[0 * 6 + 0] = b[1 * 6 + 1] = b[2 * 6 + 2] = 1.0;
      b[0 * 6 + 3] = -y;
      b[1 * 6 + 3] = x;
      b[1 * 6 + 4] = -z;
      b[2 * 6 + 4] = y;
      b[0 * 6 + 5] = z;
      b[2 * 6 + 5] = -x;
    }
  } else {
    for (size_t u = 0; u < mem.size(); ++u)
      std::copy(&B[(size_t)mem[u] * 36], &B[(size_t)mem[u] * 36] + 36, &Bm[u * 36]);
  }
  return thin_qr(m, Bm.data(), Q.data(), R.data());
}

// --------------------------------------------------------------- device kernels

__global__ void k_scatter_values(const int* __restrict__ slot_of, const double* __restrict__ src,
                                 double* __restrict__ vals, int64_t nnzb, int B) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * B) return;
  const int64_t k = t / B;
  const int e = (int)(t - k * B);
  const int64_t slot = slot_of[k];
  vals[(slot >> 5) * (32LL * B) + 32LL * e + (slot & 31)] = src[t];
}

// P = P~ - omega D_s^-1 (A P~) on the pattern of Z = A P~ (which contains P~'s).
template <int BS>
__global__ void k_smooth_prolongator(int64_t nz, const int* __restrict__ zrow, const int* __restrict__ zcol,
                                     const double* __restrict__ Z, const int* __restrict__ agg,
                                     const double* __restrict__ Q, const int* __restrict__ diag_slot,
                                     const double* __restrict__ Avals, double omega,
                                     const int* __restrict__ pslot, double* __restrict__ Pvals) {
  constexpr int B = BS * 6;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nz * B) return;
  const int64_t z = t / B;
  const int e = (int)(t - z * B);
  const int r = e / 6;  // row of the 6-column block
  const int i = zrow[z];
  const double d = Avals[vidx<BS * BS>(diag_slot[i], r * BS + r)];
  double v = -omega / d * Z[z * B + e];
  if (zcol[z] == agg[i]) v += Q[(int64_t)i * B + e];
  Pvals[vidx<B>(pslot[z], e)] = v;
}

// R = P^T: block kR of R is the transpose of block rmap[kR] of P.
template <int BS>
__global__ void k_transpose_blocks(int64_t nnzb, const int* __restrict__ rmap, const int* __restrict__ rslot,
                                   const int* __restrict__ pslot, const double* __restrict__ Pvals,
                                   double* __restrict__ Rvals) {
  constexpr int B = BS * 6;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * B) return;
  const int64_t k = t / B;
  const int e = (int)(t - k * B);
  const int u = e / BS, r = e - u * BS;  // R[u][r] = P[r][u]
  Rvals[vidx<B>(rslot[k], e)] = Pvals[vidx<B>(pslot[rmap[k]], r * 6 + u)];
}

// Inverse of each diagonal block by Cholesky (the blocks are SPD), written
// slice-interleaved (element e of row i at (i/32)*32*B + 32*e + i%32).
template <int BS, typename TM>
__global__ void k_block_inverse(int64_t n, const int* __restrict__ diag_slot, const TM* __restrict__ vals,
                                double* __restrict__ dinv, float* __restrict__ dinv32, int* __restrict__ err) {
  constexpr int B = BS * BS;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[BS][BS], L[BS][BS], W[BS][BS];
  const int64_t ds = diag_slot[i];
  bool ok = ds >= 0;
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int c = 0; c < BS; ++c) a[r][c] = ok ? (double)vals[vidx<B>(ds, r * BS + c)] : (r == c ? 1.0 : 0.0);
#pragma unroll
  for (int j = 0; j < BS; ++j) {
    double s = a[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0)) {
      ok = false;
      s = 1.0;
    }
    L[j][j] = sqrt(s);
#pragma unroll
    for (int r = j + 1; r < BS; ++r) {
      double t = a[r][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= L[r][k] * L[j][k];
      L[r][j] = t / L[j][j];
    }
  }
  // W = L^-1 (lower)
#pragma unroll
  for (int c = 0; c < BS; ++c) {
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      if (r < c) {
        W[r][c] = 0.0;
        continue;
      }
      double t = (r == c) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < r; ++k)
        if (k >= c) t -= L[r][k] * W[k][c];
      W[r][c] = t / L[r][r];
    }
  }
  if (!ok && ds >= 0) set_err(err, kDevBreakdown);
  const int64_t base = (i >> 5) * (32LL * B) + (i & 31);
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < BS; ++k)
        if (k >= r && k >= c) t += W[k][r] * W[k][c];
      dinv[base + 32 * (r * BS + c)] = t;
      if (dinv32) dinv32[base + 32 * (r * BS + c)] = (float)t;
    }
}

// splitmix64 (Steele, Lea, Flood 2014): d-th output of the generator seeded
// with 0; start vector v[d] = 2 * (out >> 11) * 2^-53 - 1.
__global__ void k_start_vector(double* __restrict__ v, int64_t n) {
  const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (d >= n) return;
  unsigned long long z = (unsigned long long)(d + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  v[d] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

// One power step w_out = D^-1 A (w_in / ||w_in||) with D the block diagonal
// (dinv) or the scalar diagonal; ||w_out|| goes to *norm_out.
template <int BS, int V, typename TM>
__global__ void __launch_bounds__(256, 8) k_power_step(const int* __restrict__ slice_ptr,
                                                            const int* __restrict__ col, const TM* __restrict__ vals,
                                                            const int* __restrict__ srow,
                                                            const int* __restrict__ diag_slot,
                                                            const double* __restrict__ dinv, int scalar_diag,
                                                            const float* __restrict__ wts,
                                                            const double* __restrict__ w_in,
                                                            double* __restrict__ w_out, const double* norm_in,
                                                            double* norm_out, int64_t n, int64_t nthreads,
                                                            double* partials, unsigned* counter) {
  constexpr int B = BS * BS;
  const double s = norm_in ? 1.0 / *norm_in : 1.0;
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
    double acc[BS];
    row_product<BS, BS, V, TM, double, double>(slice_ptr, col, vals, w_in, pos, sub, acc);
    const int64_t row = row_at(srow, pos);
    if (sub == 0 && row >= 0 && row < n) {
      double z[BS];
      if (scalar_diag) {
        const int64_t ds = diag_slot[row];
#pragma unroll
        for (int r = 0; r < BS; ++r) z[r] = acc[r] * s / (double)vals[vidx<B>(ds, r * BS + r)];
      } else {
        const int64_t base = (row >> 5) * (32LL * B) + (row & 31);
        const double wr = wts ? (double)wts[row] : 1.0;
#pragma unroll
        for (int r = 0; r < BS; ++r) {
          double t = 0.0;
#pragma unroll
          for (int c = 0; c < BS; ++c) t = fma(dinv[base + 32 * (r * BS + c)], acc[c] * s, t);
          z[r] = wr * t;
        }
      }
#pragma unroll
      for (int r = 0; r < BS; ++r) {
        w_out[row * BS + r] = z[r];
        local[0] = fma(z[r], z[r], local[0]);
      }
    }
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) *norm_out = sqrt(out[0]);
}

// The same step (block diagonal only) in the component-split form for 6-row
// blocks: CTA = one slice at a time (grid-stride over slices), BS * VS warps.
template <int BS, int VS, typename TM>
__global__ void __launch_bounds__(768) k_power_step_split(const int* __restrict__ slice_ptr,
                                                          const int* __restrict__ col, const TM* __restrict__ vals,
                                                          const int* __restrict__ srow,
                                                          const double* __restrict__ dinv,
                                                          const float* __restrict__ wts,
                                                          const double* __restrict__ w_in,
                                                          double* __restrict__ w_out, const double* norm_in,
                                                          double* norm_out, int64_t n, int64_t nslices,
                                                          double* partials, unsigned* counter) {
  __shared__ double as[BS][32];
  const double sc = norm_in ? 1.0 / *norm_in : 1.0;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31, a = wp % BS, sub = wp / BS;
  double local[1] = {0.0};
  for (int64_t s = blockIdx.x; s < nslices; s += gridDim.x) {
    const double acc = row_component<BS, BS, VS, TM, double, double>(slice_ptr, col, vals, w_in, s, lane, a, sub);
    __syncthreads();  // the previous slice's readers of `as` are done
    if (sub == 0) as[a][lane] = acc * sc;
    __syncthreads();
    const int64_t i = row_at(srow, s * 32 + lane);
    if (sub == 0 && i >= 0 && i < n) {
      const int64_t base = (i >> 5) * (32LL * BS * BS) + (i & 31);
      double t = 0.0;
#pragma unroll
      for (int c = 0; c < BS; ++c) t = fma(dinv[base + 32 * (a * BS + c)], as[c][lane], t);
      const double z = (wts ? (double)wts[i] : 1.0) * t;
      w_out[i * BS + a] = z;
      local[0] = fma(z, z, local[0]);
    }
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) *norm_out = sqrt(out[0]);
}

// Rayleigh quotient w^T A w / w^T D w; in block mode also the Chebyshev data
// for the interval [lower, upper] * lambda (Saad, Alg. 12.1 coefficients).
template <int BS, int V, typename TM>
__global__ void __launch_bounds__(256) k_rayleigh(const int* __restrict__ slice_ptr,
                                                          const int* __restrict__ col, const TM* __restrict__ vals,
                                                          const int* __restrict__ srow,
                                                          const int* __restrict__ diag_slot, int scalar_diag,
                                                          const float* __restrict__ wts,
                                                          const double* __restrict__ w, int64_t n, int64_t nthreads,
                                                          double* partials, unsigned* counter, double* out_scal,
                                                          double lower, double upper, int degree) {
  constexpr int B = BS * BS;
  double local[2] = {0.0, 0.0};
  const int64_t ntasks = (nthreads + 31) >> 5;
  int64_t t0, t1;
  deal_range(ntasks, t0, t1);
  for (int64_t g = t0 + (threadIdx.x >> 5); g < t1; g += blockDim.x >> 5) {
    const int64_t t = g * 32 + (threadIdx.x & 31);
    if (t >= nthreads) continue;  // rows are whole slices: never taken
    int64_t pos;
    int sub;
    row_of_thread<V>(t, pos, sub);
    double acc[BS];
    row_product<BS, BS, V, TM, double, double>(slice_ptr, col, vals, w, pos, sub, acc);
    const int64_t row = row_at(srow, pos);
    if (sub == 0 && row >= 0 && row < n) {
      const int64_t ds = diag_slot[row];
      double wi[BS];
#pragma unroll
      for (int r = 0; r < BS; ++r) wi[r] = w[row * BS + r];
#pragma unroll
      for (int r = 0; r < BS; ++r) {
        local[0] = fma(wi[r], acc[r], local[0]);
        if (scalar_diag) {
          local[1] = fma(wi[r] * (double)vals[vidx<B>(ds, r * BS + r)], wi[r], local[1]);
        } else {
          double t = 0.0;
#pragma unroll
          for (int c = 0; c < BS; ++c) t = fma((double)vals[vidx<B>(ds, r * BS + c)], wi[c], t);
          // M = D W^-1: the quotient of A v = lam M v for the preconditioner W D^-1
          local[1] = fma(wi[r], wts ? t / (double)wts[row] : t, local[1]);
        }
      }
    }
  }
  double out[2];
  if (grid_reduce<2>(local, partials, counter, out) && threadIdx.x == 0) {
    const double lam = out[0] / out[1];
    out_scal[kLam] = lam;
    if (!scalar_diag) {
      const double lo = lower * lam, hi = upper * lam;
      const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
      double rho = 1.0 / sigma;
      out_scal[kInvTheta] = 1.0 / theta;
      for (int k = 0; k + 1 < degree && kCheb + 2 * k + 1 < kScalarsPerLevel; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        out_scal[kCheb + 2 * k] = rn * rho;
        out_scal[kCheb + 2 * k + 1] = 2.0 * rn / delta;
        rho = rn;
      }
    }
  }
}

template <int BS, typename TM>
static Status power_impl(bamg_mg* mg, const bamg_bsr* A, const TM* vals, const double* dinv, const float* wts,
                         bool scalar_diag, double* out_scal, cudaStream_t st) {
  bamg_ctx* ctx = mg->ctx;
  
  const int64_t n = A->nbr, rows = row_threads_for<TM>(A);
  double* w[2] = {mg->power_w[0], mg->power_w[1]};
  double* norms = mg->scal + (int64_t)mg->levels.size() * kScalarsPerLevel;  // 2 scratch slots
  { k_start_vector<<<(unsigned)((n * BS + 255) / 256), 256, 0, st>>>(w[0], n * BS); BAMG_COUNT_LAUNCH; }
  const int split = (BS == 6 && !scalar_diag) ? split_for<TM>(A) : 0;
  for (int it = 0; it < mg->opts.power_its; ++it) {
    const double* nin = it == 0 ? nullptr : norms + ((it + 1) & 1);
    if (split) {
      const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>(A->nslices, 1216));
      BAMG_DISPATCH_VS(split, {
        k_power_step_split<BS, VS, TM><<<gs, 32 * BS * VS, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, dinv, wts,
                                                                     w[it & 1], w[(it + 1) & 1], nin, norms + (it & 1),
                                                                     n, A->nslices, ctx->d_partials, ctx->d_counters);
        BAMG_COUNT_LAUNCH; })
      continue;
    }
    BAMG_DISPATCH_V(lanes_for<TM>(A), { k_power_step<BS, V, TM><<<deal_grid(k_power_step<BS, V, TM>, ctx->sm_count, rows), 256, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, A->diag_slot, dinv,
                                                    scalar_diag ? 1 : 0, scalar_diag ? nullptr : wts, w[it & 1], w[(it + 1) & 1], nin,
                                                    norms + (it & 1), n, rows, ctx->d_partials, ctx->d_counters); BAMG_COUNT_LAUNCH; })
  }
  BAMG_DISPATCH_V(lanes_for<TM>(A), { k_rayleigh<BS, V, TM><<<deal_grid(k_rayleigh<BS, V, TM>, ctx->sm_count, rows), 256, 0, st>>>(A->slice_ptr, A->sell_col, vals, A->slot_row, A->diag_slot, scalar_diag ? 1 : 0,
                                                scalar_diag ? nullptr : wts, w[mg->opts.power_its & 1], n, rows, ctx->d_partials,
                                                ctx->d_counters + 1, out_scal, mg->opts.cheb_lower,
                                                mg->opts.cheb_upper, mg->opts.cheb_degree); BAMG_COUNT_LAUNCH; })
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

Status power_lambda(bamg_mg* mg, int l, bool scalar_diag, double* out_scal, cudaStream_t st) {
  Level& L = mg->levels[l];
  bamg_bsr* A = L.A;
  // FP64 arithmetic on the FP64 values when they are current (the fine level
  // in both forms); the coarse levels of the mixed form hold only the FP32
  // copy, read and widened.  (The FP32 smoother's operator differs from the
  // FP64 one by single-precision rounding, far inside the interval's margin.)
  const bool f32 = A->vals64_stale;
  if (f32) BAMG_TRY(bsr_ensure_fp32(A));
  const float* wts = L.weights;
  if (L.bs == 3)
    return f32 ? power_impl<3, float>(mg, A, A->vals32, L.dinv, wts, scalar_diag, out_scal, st)
               : power_impl<3, double>(mg, A, A->vals, L.dinv, wts, scalar_diag, out_scal, st);
  if (L.bs == 6)
    return f32 ? power_impl<6, float>(mg, A, A->vals32, L.dinv, wts, scalar_diag, out_scal, st)
               : power_impl<6, double>(mg, A, A->vals, L.dinv, wts, scalar_diag, out_scal, st);
  return make_status(BAMG_ERR_INVALID, "block size %d", L.bs);
}

Status mg_refresh_level(bamg_mg* mg, int l, cudaStream_t st) {
  Level& L = mg->levels[l];
  bamg_ctx* ctx = mg->ctx;
  const bamg_bsr* A = L.A;
  const unsigned b = (unsigned)((L.n + 127) / 128);
  float* d32 = mg->opts.precision == BAMG_FP32 ? L.dinv32 : nullptr;
  if (L.n > 0) {
    if (L.bs == 3) {
      if (A->vals64_stale)
        { k_block_inverse<3, float><<<b, 128, 0, st>>>(L.n, A->diag_slot, A->vals32, L.dinv, d32, ctx->d_err); BAMG_COUNT_LAUNCH; }
      else
        { k_block_inverse<3, double><<<b, 128, 0, st>>>(L.n, A->diag_slot, A->vals, L.dinv, d32, ctx->d_err); BAMG_COUNT_LAUNCH; }
    } else {
      if (A->vals64_stale)
        { k_block_inverse<6, float><<<b, 128, 0, st>>>(L.n, A->diag_slot, A->vals32, L.dinv, d32, ctx->d_err); BAMG_COUNT_LAUNCH; }
      else
        { k_block_inverse<6, double><<<b, 128, 0, st>>>(L.n, A->diag_slot, A->vals, L.dinv, d32, ctx->d_err); BAMG_COUNT_LAUNCH; }
    }
    BAMG_CUDA(cudaGetLastError());
  }
  BAMG_TRY(mg_learned_weights(mg, l, st));
  return power_lambda(mg, l, false, mg->scal + (int64_t)l * kScalarsPerLevel, st);
}

Status mg_refresh_restriction(bamg_mg* mg, int l, cudaStream_t st) {
  Level& L = mg->levels[l];
  if (!L.P || L.r_version == L.P->version) return Status{};
  const int64_t nt = L.R->nnzb * L.R->block_elems();
  if (nt > 0) {
    const unsigned b = (unsigned)((nt + 255) / 256);
    if (L.bs == 3)
      { k_transpose_blocks<3><<<b, 256, 0, st>>>(L.R->nnzb, L.rmap, L.R->slot_of, L.P->slot_of, L.P->vals, L.R->vals); BAMG_COUNT_LAUNCH; }
    else
      { k_transpose_blocks<6><<<b, 256, 0, st>>>(L.R->nnzb, L.rmap, L.R->slot_of, L.P->slot_of, L.P->vals, L.R->vals); BAMG_COUNT_LAUNCH; }
    BAMG_CUDA(cudaGetLastError());
  }
  L.R->version++;
  L.r_version = L.P->version;
  L.r_refreshes++;
  return Status{};
}

static Status bsr_upload_values(bamg_bsr* A, const std::vector<double>& v) {
  cudaStream_t st = A->ctx->stream;
  double* tmp = nullptr;
  BAMG_TRY(upload(&tmp, v, st));
  const int B = (int)A->block_elems();
  const int64_t nt = A->nnzb * B;
  if (nt > 0) { k_scatter_values<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(A->slot_of, tmp, A->vals, A->nnzb, B); BAMG_COUNT_LAUNCH; }
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(st);
  dfree(tmp, st);
  if (e != cudaSuccess) return cuda_status(e, "scatter values");
  A->version++;
  return Status{};
}

static Status alloc_vectors(bamg_mg* mg) {
  cudaStream_t st = mg->ctx->stream;
  const bool f32 = mg->opts.precision == BAMG_FP32;
  for (auto& L : mg->levels) {
    const int64_t m = L.n * L.bs;
    BAMG_TRY(dalloc(&L.b, m, st));
    BAMG_TRY(dalloc(&L.x, m, st));
    BAMG_TRY(dalloc(&L.r, m, st));
    BAMG_TRY(dalloc(&L.d0, m, st));
    BAMG_TRY(dalloc(&L.d1, m, st));
    const int64_t nd = ((L.n + 31) / 32) * 32 * L.bs * L.bs;
    BAMG_TRY(dalloc(&L.dinv, nd, st));
    if (f32) {
      BAMG_TRY(dalloc(&L.b32, m, st));
      BAMG_TRY(dalloc(&L.x32, m, st));
      BAMG_TRY(dalloc(&L.r32, m, st));
      BAMG_TRY(dalloc(&L.d032, m, st));
      BAMG_TRY(dalloc(&L.d132, m, st));
      BAMG_TRY(dalloc(&L.dinv32, nd, st));
    }
  }
  const int64_t m0 = mg->levels[0].n * mg->levels[0].bs;
  BAMG_TRY(dalloc(&mg->power_w[0], mg->levels[0].n * 6, st));
  BAMG_TRY(dalloc(&mg->power_w[1], mg->levels[0].n * 6, st));
  BAMG_TRY(dalloc(&mg->cx, m0, st));
  BAMG_TRY(dalloc(&mg->cr, m0, st));
  BAMG_TRY(dalloc(&mg->cp, m0, st));
  BAMG_TRY(dalloc(&mg->cq, m0, st));
  BAMG_TRY(dalloc(&mg->cz, m0, st));
  BAMG_TRY(dalloc(&mg->czold, m0, st));
  BAMG_TRY(dalloc(&mg->cg, 1, st));
  BAMG_CUDA(cudaMallocHost(&mg->cg_host, sizeof(CgState)));
  const int64_t ns = ((int64_t)mg->levels.size() + 1) * kScalarsPerLevel;
  BAMG_TRY(dalloc(&mg->scal, ns, st));
  mg->scal_blocks_minus1 = (int)mg->levels.size();
  BAMG_CUDA(cudaMemsetAsync(mg->scal, 0, sizeof(double) * ns, st));
  return Status{};
}

static void mg_release(bamg_mg* mg) {
  cudaStream_t st = mg->ctx->stream;
  if (mg->side) {
    cudaStreamSynchronize(mg->side);
    cudaStreamSynchronize(mg->side0);
    cudaStreamDestroy(mg->side);
    cudaStreamDestroy(mg->side0);
    cudaEventDestroy(mg->ev_fork);
    cudaEventDestroy(mg->ev_join);
    cudaEventDestroy(mg->ev_join0);
    mg->side = nullptr;
  }
  mg_release_graphs(mg);
  mg_release_multi(mg);
  for (auto& L : mg->levels) {
    if (L.plan) {
      ptap_release(L.plan);
      delete L.plan;
    }
    if (L.ap) bamg_ptap_destroy(L.ap);
    if (L.Pt) bamg_bsr_destroy(L.Pt);
    dfree(L.zrow, st);
    dfree(L.agg, st);
    dfree(L.q, st);
    if (L.own_A && L.A) bamg_bsr_destroy(L.A);
    if (L.P) bamg_bsr_destroy(L.P);
    if (L.R) bamg_bsr_destroy(L.R);
    dfree(L.rmap, st);
    for (double** p : {&L.b, &L.x, &L.r, &L.d0, &L.d1, &L.dinv}) dfree(*p, st);
    dfree(L.feat, st);
    dfree(L.learned_w, st);
    for (float** p : {&L.b32, &L.x32, &L.r32, &L.d032, &L.d132, &L.dinv32}) dfree(*p, st);
  }
  for (double** p : {&mg->cx, &mg->cr, &mg->cp, &mg->cq, &mg->cz, &mg->czold, &mg->scal, &mg->power_w[0],
                     &mg->power_w[1], &mg->coarse.M, &mg->coarse.Wt, &mg->coarse.b64, &mg->coarse.x64,
                     &mg->coarse.D, &mg->coarse.Sub, &mg->coarse.Sup, &mg->coarse.Wb, &mg->coarse.Wtb,
                     &mg->coarse.Bb, &mg->coarse.Mb, &mg->coarse.Nb, &mg->coarse.Mtb, &mg->coarse.Ntb, &mg->coarse.gpart})
    dfree(*p, st);
  dfree(mg->coarse.rows, st);
  dfree(mg->coarse.dinv_tiles, st);
  dfree(mg->coarse.gctr, st);
  dfree(mg->cg, st);
  if (mg->cg_host) cudaFreeHost(mg->cg_host);
  cudaStreamSynchronize(st);
}

// Prolongator smoothing of level l from the current values of its operator
// (Sec. 2.2): omega = 4 / (3 lambda_max(D_s^-1 A)), P = P~ - omega D_s^-1 A P~.
static Status smooth_level(bamg_mg* mg, int l) {
  bamg_ctx* ctx = mg->ctx;
  cudaStream_t st = ctx->stream;
  Level& L = mg->levels[l];
  const int bs = L.bs;
  // scratch slot in the last (spare) block of scalars
  double* lam_slot = mg->scal + (int64_t)mg->scal_blocks_minus1 * kScalarsPerLevel + 4;
  BAMG_TRY(power_lambda(mg, l, true, lam_slot, st));
  double lam_s = 0.0;
  BAMG_CUDA(cudaMemcpyAsync(&lam_s, lam_slot + kLam, sizeof(double), cudaMemcpyDeviceToHost, st));
  BAMG_CUDA(cudaStreamSynchronize(st));
  if (!(lam_s > 0.0) || !std::isfinite(lam_s))
    return make_status(BAMG_ERR_BREAKDOWN, "level %d: eigen-estimate %g is not positive", l, lam_s);
  L.omega = 4.0 / (3.0 * lam_s);
  BAMG_TRY(ptap_run(L.ap, L.A, L.Pt, nullptr, BAMG_FP64, false));
  bamg_bsr* P = L.P;
  const int64_t nt = P->nnzb * bs * 6;
  if (nt > 0) {
    const unsigned b = (unsigned)((nt + 255) / 256);
    if (bs == 3)
      { k_smooth_prolongator<3><<<b, 256, 0, st>>>(P->nnzb, L.zrow, P->colidx, L.ap->Z, L.agg, L.q, L.A->diag_slot,
                                                 L.A->vals, L.omega, P->slot_of, P->vals); BAMG_COUNT_LAUNCH; }
    else
      { k_smooth_prolongator<6><<<b, 256, 0, st>>>(P->nnzb, L.zrow, P->colidx, L.ap->Z, L.agg, L.q, L.A->diag_slot,
                                                 L.A->vals, L.omega, P->slot_of, P->vals); BAMG_COUNT_LAUNCH; }
    BAMG_CUDA(cudaGetLastError());
  }
  P->version++;
  P->vals64_stale = false;
  return Status{};
}

// Aggregates of level l from the device strength graph and MIS (Sec. 3.2,
// Sec. 6), then the two host rules: vertices without strong neighbours join
// no aggregate, and rank-deficient aggregates are dissolved into their
// neighbours' surviving aggregates (the vertex's strong neighbour whose
// aggregate root has the largest (weight, root)); survivors are renumbered
// in root order.
static Status mis_level_aggregates(bamg_mg* mg, int l, const double* coords, const uint8_t* dir,
                                   const std::vector<double>& B, std::vector<int>& agg, int64_t& nagg) {
  bamg_ctx* ctx = mg->ctx;
  cudaStream_t st = ctx->stream;
  Level& L = mg->levels[l];
  const int64_t n = L.n;
  const uint64_t seed = mg->opts.mis_seed + (uint64_t)l;
  int *rp = nullptr, *col = nullptr, *dagg = nullptr, *droot = nullptr;
  std::vector<int> hrp, hcol, hroot;
  int64_t ne = 0, na = 0;
  int rounds = 0;
  Status s = dalloc(&rp, n + 1, st);
  if (s.ok()) s = dalloc(&col, std::max<int64_t>(L.A->nnzb, 1), st);
  if (s.ok()) s = dalloc(&dagg, std::max<int64_t>(n, 1), st);
  if (s.ok()) s = dalloc(&droot, std::max<int64_t>(n, 1), st);
  if (s.ok()) s = strength_graph(L.A, mg->opts.mis_eps, rp, col, L.A->nnzb, &ne);
  if (s.ok()) s = mis_aggregate(ctx, n, rp, col, seed, dagg, &na, &rounds, droot);
  if (s.ok()) s = download(hrp, rp, n + 1, st);
  if (s.ok()) s = download(hcol, col, ne, st);
  if (s.ok()) s = download(agg, dagg, n, st);
  if (s.ok()) s = download(hroot, droot, na, st);
  dfree(rp, st);
  dfree(col, st);
  dfree(dagg, st);
  dfree(droot, st);
  if (!s.ok()) return s;
  std::vector<std::vector<int>> mem(na);
  for (int64_t v = 0; v < n; ++v) {
    if (hrp[v + 1] == hrp[v]) agg[v] = -1;  // no strong neighbour
    if (agg[v] >= 0) mem[agg[v]].push_back((int)v);
  }
  std::vector<char> dissolved(na, 0);
  for (int64_t a = 0; a < na; ++a)
    dissolved[a] = !mem[a].empty() && !near_null_full_rank(l, mem[a], coords, dir, B);
  auto better = [&](int a, int b) {  // root of aggregate a beats root of aggregate b in (weight, root)
    const uint64_t wa = splitmix64_host((uint64_t)hroot[a], seed), wb = splitmix64_host((uint64_t)hroot[b], seed);
    return wa > wb || (wa == wb && hroot[a] > hroot[b]);
  };
  std::vector<int> out(agg);
  for (int64_t v = 0; v < n; ++v) {
    if (agg[v] < 0 || !dissolved[agg[v]]) continue;
    int best = -1;
    for (int k = hrp[v]; k < hrp[v + 1]; ++k) {
      const int a = agg[hcol[k]];
      if (a >= 0 && !dissolved[a] && (best < 0 || better(a, best))) best = a;
    }
    out[v] = best;
  }
  std::vector<int> renum(na, -1);
  nagg = 0;
  for (int64_t a = 0; a < na; ++a)
    if (!mem[a].empty() && !dissolved[a]) renum[a] = (int)nagg++;
  for (int64_t v = 0; v < n; ++v) agg[v] = out[v] >= 0 ? renum[out[v]] : -1;
  if (nagg == 0) return make_status(BAMG_ERR_INVALID, "level %d: no aggregate survives", l);
  return Status{};
}

static Status mg_setup_impl(bamg_mg* mg, bamg_bsr* A, const double* coords, const uint8_t* dir) {
  bamg_ctx* ctx = mg->ctx;
  cudaStream_t st = ctx->stream;
  const bamg_mg_opts& o = mg->opts;
  Level L0;
  L0.A = A;
  L0.bs = A->br;
  L0.n = A->nbr;
  mg->levels.push_back(L0);
  int grid[3] = {o.grid[0], o.grid[1], o.grid[2]};
  std::vector<double> B;  // near-null blocks of the current level's nodes (bs x 6)
  // Scratch device storage for the scalar eigen-estimate (before alloc_vectors).
  // power-iteration vectors: coarse levels have at most 6 dofs per fine node
  BAMG_TRY(dalloc(&mg->power_w[0], A->nbr * 6, st));
  BAMG_TRY(dalloc(&mg->power_w[1], A->nbr * 6, st));
  BAMG_TRY(dalloc(&mg->scal, (int64_t)(o.max_levels + 1) * kScalarsPerLevel, st));
  mg->scal_blocks_minus1 = o.max_levels;
  while (mg->levels.back().n * mg->levels.back().bs > o.max_coarse_dofs && (int)mg->levels.size() < o.max_levels) {
    const int l = (int)mg->levels.size() - 1;
    Level& L = mg->levels[l];
    std::vector<int> agg;
    int cgrid[3] = {0, 0, 0};
    int64_t nagg = 0;
    const int bs = L.bs;
    if (o.aggregation == BAMG_AGG_MIS) {
      BAMG_TRY(mis_level_aggregates(mg, l, coords, dir, B, agg, nagg));
    } else {
      aggregates(grid, agg, cgrid);
      nagg = (int64_t)cgrid[0] * cgrid[1] * cgrid[2];
    }
    if (l == 0) B = rigid_modes(coords, dir, agg, nagg);
    // tentative prolongator by per-aggregate QR (nodes outside every aggregate get no block)
    std::vector<int64_t> start(nagg + 1, 0);
    for (int64_t v = 0; v < L.n; ++v)
      if (agg[v] >= 0) start[agg[v] + 1]++;
    for (int64_t a = 0; a < nagg; ++a) start[a + 1] += start[a];
    std::vector<int64_t> members(start[nagg]);
    {
      std::vector<int64_t> fill(start.begin(), start.end() - 1);
      for (int64_t v = 0; v < L.n; ++v)
        if (agg[v] >= 0) members[fill[agg[v]]++] = v;
    }
    std::vector<double> Q((size_t)L.n * bs * 6, 0.0), Bc((size_t)nagg * 36, 0.0);
    for (int64_t a = 0; a < nagg; ++a) {
      const int cnt = (int)(start[a + 1] - start[a]);
      const int m = cnt * bs;
      if (m < 6) return make_status(BAMG_ERR_INVALID, "aggregate %lld has fewer than 6 dofs", (long long)a);
      std::vector<double> Bm((size_t)m * 6), Qa((size_t)m * 6), Ra(36);
      for (int u = 0; u < cnt; ++u)
        std::copy(&B[(size_t)members[start[a] + u] * bs * 6], &B[(size_t)members[start[a] + u] * bs * 6] + bs * 6,
                  &Bm[(size_t)u * bs * 6]);
      if (!thin_qr(m, Bm.data(), Qa.data(), Ra.data()))
        return make_status(BAMG_ERR_INVALID, "aggregate %lld: near-null space is rank deficient", (long long)a);
      for (int u = 0; u < cnt; ++u) {
        const int64_t v = members[start[a] + u];
        for (int rr = 0; rr < bs; ++rr) {
          bool zero_row = true;
          for (int c = 0; c < 6; ++c) zero_row &= Bm[((size_t)u * bs + rr) * 6 + c] == 0.0;
          for (int c = 0; c < 6; ++c)
            Q[((size_t)v * bs + rr) * 6 + c] = zero_row ? 0.0 : Qa[((size_t)u * bs + rr) * 6 + c];
        }
      }
      std::copy(Ra.begin(), Ra.end(), &Bc[(size_t)a * 36]);
    }
    // P~ : one block per node in its aggregate's column
    bamg_bsr* Pt = nullptr;
    if (bamg_bsr_create(ctx, bs, 6, L.n, nagg, &Pt) != BAMG_OK) return make_status(BAMG_ERR_OOM, "P~");
    std::unique_ptr<bamg_bsr, bamg_status (*)(bamg_bsr*)> Pt_guard(Pt, bamg_bsr_destroy);
    {
      std::vector<int> rp(L.n + 1, 0), ci;
      std::vector<double> Qb;
      for (int64_t v = 0; v < L.n; ++v) {
        if (agg[v] >= 0) {
          ci.push_back(agg[v]);
          Qb.insert(Qb.end(), &Q[(size_t)v * bs * 6], &Q[(size_t)v * bs * 6] + bs * 6);
        }
        rp[v + 1] = (int)ci.size();
      }
      BAMG_TRY(bsr_set_pattern(Pt, std::move(rp), std::move(ci)));
      BAMG_TRY(bsr_upload_values(Pt, Qb));
    }
    // P = P~ - omega D_s^-1 A P~ on the pattern of A P~ (values by smooth_level)
    bamg_ptap* ap = nullptr;
    BAMG_TRY(ptap_build(L.A, Pt, false, &ap, nullptr));
    L.ap = ap;
    L.Pt = Pt;
    Pt_guard.release();
    bamg_bsr* P = nullptr;
    if (bamg_bsr_create(ctx, bs, 6, L.n, nagg, &P) != BAMG_OK) return make_status(BAMG_ERR_OOM, "P");
    L.P = P;
    {
      std::vector<int> zr = ap->h_zrowptr, zc = ap->h_zcol;
      std::vector<int> zrow(zc.size());
      for (int64_t i = 0; i < L.n; ++i)
        for (int z = zr[i]; z < zr[i + 1]; ++z) zrow[z] = (int)i;
      BAMG_TRY(bsr_set_pattern(P, std::move(zr), std::move(zc), kSortAlways));  // rows of 1..8 blocks: sorted slices
      BAMG_TRY(upload(&L.zrow, zrow, st));
      BAMG_TRY(upload(&L.agg, agg, st));
      BAMG_TRY(upload(&L.q, Q, st));
      BAMG_CUDA(cudaStreamSynchronize(st));
    }
    BAMG_TRY(smooth_level(mg, l));
    // R = P^T pattern and block map (values filled by the state-gated refresh)
    {
      const auto &pr = P->h_rowptr, &pc = P->h_colidx;
      std::vector<int> rr(nagg + 1, 0), rc(pc.size()), rmap(pc.size());
      for (int c : pc) rr[c + 1]++;
      for (int64_t a = 0; a < nagg; ++a) rr[a + 1] += rr[a];
      std::vector<int> fill(rr.begin(), rr.end() - 1);
      for (int64_t i = 0; i < L.n; ++i)
        for (int t = pr[i]; t < pr[i + 1]; ++t) {
          const int a = pc[t];
          rc[fill[a]] = (int)i;
          rmap[fill[a]] = t;
          fill[a]++;
        }
      bamg_bsr* R = nullptr;
      if (bamg_bsr_create(ctx, 6, bs, nagg, L.n, &R) != BAMG_OK) return make_status(BAMG_ERR_OOM, "R");
      L.R = R;
      BAMG_TRY(upload(&L.rmap, rmap, st));
      BAMG_TRY(bsr_set_pattern(R, std::move(rr), std::move(rc)));
    }
    // Galerkin plan and coarse operator (owned by the next level from here on)
    bamg_bsr* Ac = nullptr;
    BAMG_TRY(ptap_build(L.A, P, true, &L.plan, &Ac));
    bamg_ptap* plan = L.plan;
    if (l == 0) {
      plan->prof_stage1 = BAMG_PROF_PTAP_STAGE1_L0;
      plan->prof_stage2 = BAMG_PROF_PTAP_STAGE2_L0;
    }
    Level C;
    C.A = Ac;
    C.own_A = true;
    C.bs = 6;
    C.n = nagg;
    mg->levels.push_back(C);  // invalidates L
    if (!Ac->all_diag) return make_status(BAMG_ERR_INVALID, "coarse operator lacks a diagonal block");
    // the next level's prolongator smoothing needs this level's Galerkin values
    BAMG_TRY(ptap_run(plan, mg->levels[l].A, P, Ac, BAMG_FP64, true));
    for (int d = 0; d < 3; ++d) grid[d] = cgrid[d];
    B = std::move(Bc);
  }
  dfree(mg->power_w[0], st);
  dfree(mg->power_w[1], st);
  dfree(mg->scal, st);
  BAMG_TRY(alloc_vectors(mg));
  return Status{};
}

// The coarsest factorisation needs only the last Galerkin product and is a
// chain of small dependent steps that leaves most of the GPU idle, while the
// smoother refresh (block inverses, power iterations) keeps the FP64 pipes
// busy and never reads the coarsest operator: the factor runs on a second
// stream between the last product and the end of the update.
static Status update_streams(bamg_mg* mg) {
  if (mg->side) return Status{};
  BAMG_CUDA(cudaStreamCreateWithFlags(&mg->side, cudaStreamNonBlocking));
  BAMG_CUDA(cudaStreamCreateWithFlags(&mg->side0, cudaStreamNonBlocking));
  BAMG_CUDA(cudaEventCreateWithFlags(&mg->ev_fork, cudaEventDisableTiming));
  BAMG_CUDA(cudaEventCreateWithFlags(&mg->ev_join, cudaEventDisableTiming));
  BAMG_CUDA(cudaEventCreateWithFlags(&mg->ev_join0, cudaEventDisableTiming));
  return Status{};
}

static Status refresh_one(bamg_mg* mg, int l, cudaStream_t st) {
  BAMG_TRY(mg_refresh_restriction(mg, l, st));
  const int pr = prof_begin(mg->ctx, BAMG_PROF_REFRESH, st);
  Status s = mg_refresh_level(mg, l, st);
  prof_end(mg->ctx, pr, st);
  return s;
}

// Streams of one reuse update:
//   main:  Galerkin products, level by level; then the smoother refresh;
//   side:  the coarsest factorisation, from the last product on;
//   side0: (mixed form only) the finest level's refresh from the start: it
//          reads only the fine operator, its power iteration is FP64-bound
//          while the FP32 Galerkin products are memory-bound, so the two
//          overlap.  (In the FP64 form both are FP64-bound and the refresh
//          stays on the main stream, beside the factor.)
// The refreshes share scratch (power-iteration vectors, reduction partials),
// so the next level's refresh waits for side0.  Every path joins the side
// streams into the caller's stream before returning.
Status mg_update_impl(bamg_mg* mg) {
  const int nl = (int)mg->levels.size();
  const bamg_prec pp = mg->opts.precision == BAMG_FP32 ? BAMG_FP32 : BAMG_FP64;
  cudaStream_t st = mg->ctx->stream;
  BAMG_TRY(update_streams(mg));
  const bool early0 = pp == BAMG_FP32 && nl > 1;
  Status r0;
  if (early0) {
    BAMG_CUDA(cudaEventRecord(mg->ev_fork, st));
    BAMG_CUDA(cudaStreamWaitEvent(mg->side0, mg->ev_fork, 0));
    r0 = refresh_one(mg, 0, mg->side0);
    BAMG_CUDA(cudaEventRecord(mg->ev_join0, mg->side0));
  }
  Status ps;
  for (int l = 0; l + 1 < nl && ps.ok(); ++l) {
    Level& L = mg->levels[l];
    ps = ptap_run(L.plan, L.A, L.P, mg->levels[l + 1].A, pp, true);
  }
  if (!ps.ok()) {
    if (early0) cudaStreamWaitEvent(st, mg->ev_join0, 0);
    return ps;
  }
  BAMG_CUDA(cudaEventRecord(mg->ev_fork, st));
  BAMG_CUDA(cudaStreamWaitEvent(mg->side, mg->ev_fork, 0));
  const Status fs = coarse_factor(mg, mg->side);
  BAMG_CUDA(cudaEventRecord(mg->ev_join, mg->side));
  auto refresh = [&]() -> Status {
    if (early0) {
      BAMG_CUDA(cudaStreamWaitEvent(st, mg->ev_join0, 0));
      BAMG_TRY(r0);
    }
    BAMG_TRY(fs);
    for (int l = early0 ? 1 : 0; l + 1 < nl; ++l) BAMG_TRY(refresh_one(mg, l, st));
    if (pp == BAMG_FP32) {
      BAMG_TRY(bsr_ensure_fp32(mg->levels[0].A));
      for (int l = 0; l + 1 < nl; ++l) {
        BAMG_TRY(bsr_ensure_fp32(mg->levels[l].P));
        BAMG_TRY(bsr_ensure_fp32(mg->levels[l].R));
      }
    }
    return Status{};
  };
  const Status rs = refresh();
  if (early0) cudaStreamWaitEvent(st, mg->ev_join0, 0);
  // joined on every path: the caller's stream never runs ahead of the factor
  BAMG_CUDA(cudaStreamWaitEvent(st, mg->ev_join, 0));
  return rs;
}

}  // namespace bamg

using namespace bamg;

extern "C" {

void bamg_mg_opts_default(bamg_mg_opts* o) {
  if (!o) return;
  o->max_levels = 10;
  o->max_coarse_dofs = 2100;
  o->grid[0] = o->grid[1] = o->grid[2] = 0;
  o->cheb_degree = 2;
  o->cheb_lower = 0.1;
  o->cheb_upper = 1.1;
  o->power_its = 15;
  o->precision = BAMG_FP64;
  o->autotune = 1;
  o->coarse_solver = 0;
  o->aggregation = BAMG_AGG_GEOMETRIC;
  o->mis_eps = 0.02;
  o->mis_seed = 1;
}

bamg_status bamg_mg_setup(bamg_ctx* ctx, bamg_bsr* A, const double* coords, const uint8_t* dirichlet,
                          const bamg_mg_opts* opts, bamg_mg** out) {
  if (!ctx || !A || !out || !coords) return BAMG_ERR_INVALID;
  *out = nullptr;
  bamg_mg_opts o;
  if (opts)
    o = *opts;
  else
    bamg_mg_opts_default(&o);
  if (!A->has_pattern || A->br != 3 || A->bc != 3 || A->nbr != A->nbc)
    return fail(ctx, make_status(BAMG_ERR_INVALID, "mg_setup needs an assembled square 3x3-block operator"));
  if (o.aggregation != BAMG_AGG_GEOMETRIC && o.aggregation != BAMG_AGG_MIS)
    return fail(ctx, make_status(BAMG_ERR_INVALID, "unknown aggregation %d", o.aggregation));
  if (o.aggregation == BAMG_AGG_MIS && !(o.mis_eps >= 0))
    return fail(ctx, make_status(BAMG_ERR_INVALID, "mis_eps must be >= 0"));
  if (o.aggregation == BAMG_AGG_GEOMETRIC &&
      ((int64_t)o.grid[0] * o.grid[1] * o.grid[2] != A->nbr || o.grid[0] <= 0))
    return fail(ctx, make_status(BAMG_ERR_INVALID, "opts.grid %dx%dx%d does not match %lld block rows", o.grid[0],
                                 o.grid[1], o.grid[2], (long long)A->nbr));
  if (o.max_levels < 1 || o.max_levels > 16 || o.cheb_degree < 1 || o.cheb_degree > 12 || o.power_its < 1 ||
      !(o.cheb_lower > 0) || !(o.cheb_upper > o.cheb_lower) ||
      (o.precision != BAMG_FP64 && o.precision != BAMG_FP32))
    return fail(ctx, make_status(BAMG_ERR_INVALID, "bad multigrid options"));
  if (!A->all_diag) return fail(ctx, make_status(BAMG_ERR_INVALID, "every block row needs its diagonal block"));
  A->symmetric = true;  // elasticity operators are symmetric: Galerkin products mirror the upper triangle
  bamg_mg* mg = new bamg_mg();
  mg->ctx = ctx;
  mg->opts = o;
  Status s = mg_setup_impl(mg, A, coords, dirichlet);
  if (s.ok()) s = mg_update_impl(mg);
  if (s.ok() && o.autotune) {
    for (auto& L : mg->levels) {
      if (s.ok()) s = bsr_autotune(L.A, nullptr);
      if (s.ok() && L.P) s = bsr_autotune(L.P, nullptr);
      if (s.ok() && L.R) s = bsr_autotune(L.R, nullptr);
    }
    if (s.ok()) s = mg_tune_smoothers(mg);
  }
  if (s.ok()) s = check_device_error(ctx);
  if (!s.ok()) {
    mg_release(mg);
    delete mg;
    return fail(ctx, s);
  }
  *out = mg;
  return BAMG_OK;
}

bamg_status bamg_mg_resetup(bamg_mg* mg) {
  if (!mg) return BAMG_ERR_INVALID;
  auto body = [&]() -> Status {
    const int nl = (int)mg->levels.size();
    for (int l = 0; l + 1 < nl; ++l) {
      BAMG_TRY(smooth_level(mg, l));
      BAMG_TRY(ptap_run(mg->levels[l].plan, mg->levels[l].A, mg->levels[l].P, mg->levels[l + 1].A, BAMG_FP64, true));
    }
    BAMG_TRY(mg_update_impl(mg));
    return check_device_error(mg->ctx);
  };
  Status s = body();
  return s.ok() ? BAMG_OK : fail(mg->ctx, s);
}

bamg_status bamg_mg_update(bamg_mg* mg) {
  if (!mg) return BAMG_ERR_INVALID;
  Status s = mg_update_impl(mg);
  return s.ok() ? BAMG_OK : fail(mg->ctx, s);
}

bamg_status bamg_mg_set_smoother_weights(bamg_mg* mg, int level, const float* w) {
  if (!mg || level < 0 || level >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  mg->levels[level].weights = const_cast<float*>(w);
  mg_release_graphs(mg);  // the captured iteration holds the old pointer
  return BAMG_OK;
}

bamg_status bamg_mg_set_lanes(bamg_mg* mg, int lanes) {
  if (!mg) return BAMG_ERR_INVALID;
  if (lanes < 0 || lanes > 32 || (lanes & (lanes - 1)))
    return fail(mg->ctx, make_status(BAMG_ERR_INVALID, "lanes must be 0 or a power of two in [1, 32]"));
  for (auto& L : mg->levels)
    for (bamg_bsr* M : {L.A, L.P, L.R})
      if (M) {
        const bool split = lanes == 0 && M->br == 6 && (M->bc == 3 || M->bc == 6);
        M->vec = M->vec32 = lanes == 0 ? 1 : lanes;
        M->split = M->split32 = split ? 4 : 0;
      }
  mg_release_graphs(mg);  // captured iterations hold the old launch shapes
  return BAMG_OK;
}

bamg_status bamg_mg_num_levels(const bamg_mg* mg, int* n) {
  if (!mg || !n) return BAMG_ERR_INVALID;
  *n = (int)mg->levels.size();
  return BAMG_OK;
}

bamg_status bamg_mg_get_level(const bamg_mg* mg, int level, bamg_bsr** A, bamg_bsr** P) {
  if (!mg || level < 0 || level >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  if (A) *A = mg->levels[level].A;
  if (P) *P = mg->levels[level].P;
  return BAMG_OK;
}

bamg_status bamg_mg_get_restriction(const bamg_mg* mg, int level, bamg_bsr** R) {
  if (!mg || !R || level < 0 || level >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  *R = mg->levels[level].R;
  return BAMG_OK;
}

bamg_status bamg_mg_get_aggregates(const bamg_mg* mg, int level, int32_t* agg) {
  if (!mg || !agg || level < 0 || level + 1 >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  const Level& L = mg->levels[level];
  if (L.n > 0 && cudaMemcpyAsync(agg, L.agg, sizeof(int) * L.n, cudaMemcpyDeviceToDevice, mg->ctx->stream) != cudaSuccess)
    return fail(mg->ctx, cuda_status(cudaGetLastError(), "aggregates"));
  return BAMG_OK;
}

bamg_status bamg_mg_get_gate_counts(const bamg_mg* mg, int level, uint64_t* p_refreshes, uint64_t* r_refreshes) {
  if (!mg || level < 0 || level >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  const Level& L = mg->levels[level];
  if (p_refreshes) *p_refreshes = L.plan ? L.plan->pblk_refreshes : 0;
  if (r_refreshes) *r_refreshes = L.r_refreshes;
  return BAMG_OK;
}

bamg_status bamg_mg_get_level_scalars(const bamg_mg* mg, int level, double* lam, double* omega) {
  if (!mg || level < 0 || level >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  const Level& L = mg->levels[level];
  if (omega) *omega = L.omega;
  if (lam) {
    *lam = 0.0;
    if (level + 1 < (int)mg->levels.size()) {
      cudaError_t e = cudaMemcpyAsync(lam, mg->scal + (int64_t)level * kScalarsPerLevel + kLam, sizeof(double),
                                      cudaMemcpyDeviceToHost, mg->ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(mg->ctx->stream);
      if (e != cudaSuccess) return fail(mg->ctx, cuda_status(e, "get_level_scalars"));
    }
  }
  return BAMG_OK;
}

__global__ void k_dinv_rowmajor(int64_t n, int B, const double* __restrict__ dinv, double* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * B) return;
  const int64_t i = t / B;
  const int e = (int)(t - i * B);
  out[t] = dinv[(i >> 5) * 32LL * B + 32LL * e + (i & 31)];
}

bamg_status bamg_mg_get_dinv(const bamg_mg* mg, int level, double* out) {
  if (!mg || !out || level < 0 || level + 1 >= (int)mg->levels.size()) return BAMG_ERR_INVALID;
  const Level& L = mg->levels[level];
  const int B = L.bs * L.bs;
  const int64_t nt = L.n * B;
  if (nt > 0) { k_dinv_rowmajor<<<(unsigned)((nt + 255) / 256), 256, 0, mg->ctx->stream>>>(L.n, B, L.dinv, out); BAMG_COUNT_LAUNCH; }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BAMG_OK : fail(mg->ctx, cuda_status(e, "get_dinv"));
}

bamg_status bamg_mg_destroy(bamg_mg* mg) {
  if (!mg) return BAMG_OK;
  mg_release(mg);
  delete mg;
  return BAMG_OK;
}

}  // extern "C"
