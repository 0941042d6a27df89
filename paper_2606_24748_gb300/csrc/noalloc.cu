// Residual norm ||b - A x||_2 of a square 3x3- or 6x6-block operator with no
// device allocation: the partial sums of the reduction live in a file-scope
// device array instead of the context's work buffers.  For callers that
// cannot call cudaMalloc: code inside a framework whose device memory is
// entirely pre-reserved by its own pool.
#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace bamg {

// One partial sum per CTA: at most kNoallocPartials CTAs of kRowThreads
// threads, i.e. (block rows rounded up to 32) x (lanes per row) <=
// kNoallocPartials * kRowThreads.  32 KB, held by every GPU that loads the
// library until the process exits.
constexpr int kNoallocPartials = 4096;
static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];
static __device__ __align__(256) unsigned g_noalloc_counter[1];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static double* g_partials_addr[kMaxDevices];
static unsigned* g_counter_addr[kMaxDevices];

// Device addresses of the scratch on the current device, looked up once per
// device (host code cannot use the array names as device addresses).
static Status scratch_addresses(double** partials, unsigned** counter) {
  int dev = 0;
  BAMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return make_status(BAMG_ERR_INVALID, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    void* c = nullptr;
    BAMG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
    BAMG_CUDA(cudaGetSymbolAddress(&c, g_noalloc_counter));
    g_partials_addr[dev] = (double*)p;
    g_counter_addr[dev] = (unsigned*)c;
  }
  *partials = g_partials_addr[dev];
  *counter = g_counter_addr[dev];
  return Status{};
}

// Same product and reduction tree as the residual of the CG exit, one pass
// over the rows with one partial per CTA.
template <int BS, int V>
__global__ void __launch_bounds__(kRowThreads) k_residual_norm_noalloc(const int* __restrict__ sp,
                                                                       const int* __restrict__ col,
                                                                       const double* __restrict__ vals,
                                                                       const int* __restrict__ srow, int64_t n,
                                                                       int64_t nthreads, const double* __restrict__ x,
                                                                       const double* __restrict__ b, double* norm,
                                                                       double* partials, unsigned* counter) {
  double local[1] = {0.0};
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nthreads) {
    int64_t pos;
    int sub;
    row_of_thread<V>(t, pos, sub);
    double acc[BS];
    row_product<BS, BS, V, double, double, double>(sp, col, vals, x, pos, sub, acc);
    const int64_t i = row_at(srow, pos);
    if (sub == 0 && i >= 0 && i < n) {
#pragma unroll
      for (int a = 0; a < BS; ++a) {
        const double r = b[i * BS + a] - acc[a];
        local[0] = fma(r, r, local[0]);
      }
    }
  }
  double out[1];
  if (grid_reduce<1>(local, partials, counter, out) && threadIdx.x == 0) *norm = sqrt(out[0]);
}

static Status residual_norm_noalloc(const bamg_bsr* A, const double* x, const double* b, double* norm) {
  if (!A->has_pattern) return make_status(BAMG_ERR_STATE, "matrix has no pattern");
  if (A->br != A->bc || A->nbr != A->nbc || (A->br != 3 && A->br != 6))
    return make_status(BAMG_ERR_INVALID, "residual norm needs a square operator with 3x3 or 6x6 blocks");
  if (A->vals64_stale) return make_status(BAMG_ERR_STATE, "the matrix holds only FP32 values");
  if (!norm || (A->nbr > 0 && (!x || !b))) return make_status(BAMG_ERR_INVALID, "null pointer");
  const int64_t nthreads = row_threads(A);
  const int64_t blocks = std::max<int64_t>(1, (nthreads + kRowThreads - 1) / kRowThreads);
  if (blocks > kNoallocPartials)
    return make_status(BAMG_ERR_INVALID,
                       "residual norm without allocation: %lld block rows x %d lanes need %lld partial sums, "
                       "at most %d are available (%lld thread slots)",
                       (long long)A->nbr, A->vec, (long long)blocks, kNoallocPartials,
                       (long long)kNoallocPartials * kRowThreads);
  double* partials = nullptr;
  unsigned* counter = nullptr;
  BAMG_TRY(scratch_addresses(&partials, &counter));
  cudaStream_t st = A->ctx->stream;
  BAMG_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
  if (A->br == 3) {
    BAMG_DISPATCH_V(A->vec, { k_residual_norm_noalloc<3, V><<<(unsigned)blocks, kRowThreads, 0, st>>>(
                                  A->slice_ptr, A->sell_col, A->vals, A->slot_row, A->nbr, nthreads, x, b, norm, partials,
                                  counter); BAMG_COUNT_LAUNCH; })
  } else {
    BAMG_DISPATCH_V(A->vec, { k_residual_norm_noalloc<6, V><<<(unsigned)blocks, kRowThreads, 0, st>>>(
                                  A->slice_ptr, A->sell_col, A->vals, A->slot_row, A->nbr, nthreads, x, b, norm, partials,
                                  counter); BAMG_COUNT_LAUNCH; })
  }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_bsr_residual_norm_noalloc(const bamg_bsr* A, const double* x, const double* b, double* norm) {
  if (!A) return BAMG_ERR_INVALID;
  Status s = residual_norm_noalloc(A, x, b, norm);
  return s.ok() ? BAMG_OK : fail(A->ctx, s);
}

}  // extern "C"
