// Measured peak of the FP64 and FP32 FMA pipes: the denominator of the
// rooflines of ALU-bound kernels.  GB300 has no separate FP64 tensor path
// worth using for these kernels, and its FP64 FMA rate is a small fraction of
// its FP32 rate, so the FP64 kernels of the V-cycle and the Galerkin product
// are bounded by this pipe rather than by HBM.
//
// The probe keeps 8 independent FMA chains per thread over a full-occupancy
// grid on every SM, so that neither dependent-operation latency nor issue
// slots limit it, and times one launch of about 0.1 s with CUDA events.
#include "device.cuh"
#include "internal.h"

namespace bamg {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int64_t iters, T seed, T* out) {
  T a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = seed + (T)(k + 1) * (T)1e-3 * (T)(threadIdx.x & 7);
  // x <- x * m + c with |m| < 1 converges to c / (1 - m): values stay finite
  const T m = (T)0.9999, c = (T)1e-4;
  for (int64_t i = 0; i < iters; i += kProbeUnroll) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], m, c);
    }
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  // never true for the finite values above; keeps the chains live
  if (s == (T)-1.0) out[blockIdx.x] = s;
}

template <typename T>
static Status fma_probe(bamg_ctx* c, double* tflops) {
  int per_sm = 0;
  BAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, 256, 0));
  per_sm = std::max(1, per_sm);
  const unsigned grid = (unsigned)(c->sm_count * per_sm);
  T* out = nullptr;
  BAMG_CUDA(cudaMallocAsync((void**)&out, sizeof(T) * grid, c->stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Status s;
  float ms = 0.f;
  int64_t iters = 1024;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    s = cuda_status(cudaGetLastError(), "probe events");
  } else {
    k_fma_probe<T><<<grid, 256, 0, c->stream>>>(iters, (T)1, out);  // warm-up
    BAMG_COUNT_LAUNCH;
    // grow the launch until it runs for at least 0.1 s (each step at most 4x)
    for (int round = 0; round < 24 && s.ok(); ++round) {
      cudaEventRecord(e0, c->stream);
      k_fma_probe<T><<<grid, 256, 0, c->stream>>>(iters, (T)1, out);
      BAMG_COUNT_LAUNCH;
      cudaEventRecord(e1, c->stream);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        s = cuda_status(e, "probe launch");
        break;
      }
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms >= 100.f) break;
      const double grow = ms > 1.f ? std::min(4.0, 110.0 / ms) : 4.0;
      iters = ((int64_t)(iters * grow) + kProbeUnroll - 1) / kProbeUnroll * kProbeUnroll;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, c->stream);
  if (!s.ok()) return s;
  BAMG_CUDA(cudaGetLastError());
  const double flops = 2.0 * kProbeChains * (double)iters * grid * 256.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return Status{};
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_probe_fma_rate(bamg_ctx* ctx, int precision, double* tflops) {
  if (!ctx || !tflops || (precision != BAMG_FP64 && precision != BAMG_FP32)) return BAMG_ERR_INVALID;
  Status s = precision == BAMG_FP64 ? fma_probe<double>(ctx, tflops) : fma_probe<float>(ctx, tflops);
  return s.ok() ? BAMG_OK : fail(ctx, s);
}

}  // extern "C"
