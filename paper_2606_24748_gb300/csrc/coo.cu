// Blocked COO assembly (Sec. 3.4, Sec. 5): block coordinates declared once,
// duplicates summed by a cached plan, one gather-sum kernel per numeric
// assembly writing straight into the sliced block storage.
#include <cub/device/device_radix_sort.cuh>

#include "device.cuh"
#include "internal.h"

namespace bamg {

__global__ void k_coo_keys(const int32_t* __restrict__ bi, const int32_t* __restrict__ bj, int64_t n,
                           int64_t nbr, int64_t nbc, unsigned long long* __restrict__ keys,
                           int* __restrict__ idx, int* __restrict__ bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = bi[k], j = bj[k];
    unsigned long long key = ~0ull;
    if (i >= 0 && j >= 0) {
      if (i >= nbr || j >= nbc) {
        atomicExch(bad, 1);
      } else {
        key = ((unsigned long long)(unsigned)i << 32) | (unsigned)j;
      }
    }
    keys[k] = key;
    idx[k] = (int)k;
  }
}

// out block k (pattern order), element e: sum of its contributions in sorted
// (input) order; written into the sliced storage (and its float copy).
template <int B>
__global__ void k_coo_sum(const int* __restrict__ seg, const int* __restrict__ perm,
                          const double* __restrict__ v, const int* __restrict__ slot_of, int64_t nnzb,
                          double* __restrict__ vals, float* __restrict__ vals32, int add,
                          int* __restrict__ err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * B) return;
  const int64_t k = t / B;
  const int e = (int)(t - k * B);
  const int s0 = seg[k], s1 = seg[k + 1];
  // FP64 adds run at two per clock per SM: start from the first contribution
  // instead of zero, and test for NaN / Inf on the exponent bits (integer
  // pipe) rather than with FP64 comparisons.
  // contributions four at a time: their permutation entries, then their
  // values, are loaded before any is added (independent loads in flight);
  // the sum still runs in stream order
  double sum = s1 > s0 ? __ldg(v + (int64_t)__ldg(perm + s0) * B + e) : 0.0;
  int s = s0 + 1;
  for (; s + 3 < s1; s += 4) {
    const int p0 = __ldg(perm + s), p1 = __ldg(perm + s + 1), p2 = __ldg(perm + s + 2), p3 = __ldg(perm + s + 3);
    const double v0 = __ldg(v + (int64_t)p0 * B + e), v1 = __ldg(v + (int64_t)p1 * B + e);
    const double v2 = __ldg(v + (int64_t)p2 * B + e), v3 = __ldg(v + (int64_t)p3 * B + e);
    sum += v0;
    sum += v1;
    sum += v2;
    sum += v3;
  }
  if (s + 1 < s1) {
    const int p0 = __ldg(perm + s), p1 = __ldg(perm + s + 1);
    const double v0 = __ldg(v + (int64_t)p0 * B + e), v1 = __ldg(v + (int64_t)p1 * B + e);
    sum += v0;
    sum += v1;
    s += 2;
  }
  if (s < s1) sum += __ldg(v + (int64_t)__ldg(perm + s) * B + e);
  const int64_t a = vidx<B>(slot_of[k], e);
  if (add) sum += vals[a];
  if ((__double_as_longlong(sum) & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) set_err(err, kDevNaN);
  vals[a] = sum;
  if (vals32) vals32[a] = (float)sum;
}

// The same sum with one thread per storage slot (slice order) and all B
// elements of its block: every store of a warp then writes 32 consecutive
// slots of one element (coalesced), and each contribution is read as one run
// of B values.  The slot's contributions are contiguous in sperm (slots in
// slice order, each slot's in input order), so the sum order is that of
// k_coo_sum.  Padding slots have none and are left alone.
template <int B>
__global__ void __launch_bounds__(128) k_coo_sum_slots(const int* __restrict__ soff, const int* __restrict__ sperm,
                                                       const double* __restrict__ v, int64_t nslots,
                                                       double* __restrict__ vals, float* __restrict__ vals32,
                                                       int add, int* __restrict__ err) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nslots) return;
  const int c0 = soff[s], c1 = soff[s + 1];
  if (c0 == c1 && !add) return;
  double acc[B];
  const int64_t base = (s >> 5) * (32LL * B) + (s & 31);
  if (c0 < c1) {
    const double* p0 = v + (int64_t)__ldg(sperm + c0) * B;
#pragma unroll
    for (int e = 0; e < B; ++e) acc[e] = __ldg(p0 + e);
    for (int c = c0 + 1; c < c1; ++c) {
      const double* p = v + (int64_t)__ldg(sperm + c) * B;
#pragma unroll
      for (int e = 0; e < B; ++e) acc[e] += __ldg(p + e);
    }
  } else {
#pragma unroll
    for (int e = 0; e < B; ++e) acc[e] = 0.0;
  }
  bool bad = false;
#pragma unroll
  for (int e = 0; e < B; ++e) {
    double sum = acc[e];
    if (add) sum += vals[base + 32 * e];
    bad |= (__double_as_longlong(sum) & 0x7FF0000000000000ll) == 0x7FF0000000000000ll;
    vals[base + 32 * e] = sum;
    if (vals32) vals32[base + 32 * e] = (float)sum;
  }
  if (bad) set_err(err, kDevNaN);
}

__global__ void k_coo_sum_any(const int* __restrict__ seg, const int* __restrict__ perm,
                              const double* __restrict__ v, const int* __restrict__ slot_of, int64_t nnzb,
                              int B, double* __restrict__ vals, float* __restrict__ vals32, int add,
                              int* __restrict__ err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * B) return;
  const int64_t k = t / B;
  const int e = (int)(t - k * B);
  double sum = 0.0;
  for (int s = seg[k]; s < seg[k + 1]; ++s) sum += __ldg(v + (int64_t)perm[s] * B + e);
  const int64_t slot = slot_of[k];
  const int64_t a = (slot >> 5) * (32LL * B) + 32LL * e + (slot & 31);
  if (add) sum += vals[a];
  if (!isfinite(sum)) set_err(err, kDevNaN);
  vals[a] = sum;
  if (vals32) vals32[a] = (float)sum;
}

static Status coo_preallocate(bamg_bsr* A, int64_t n, const int32_t* bi, const int32_t* bj) {
  cudaStream_t st = A->ctx->stream;
  if (n < 0 || n >= INT32_MAX) return make_status(BAMG_ERR_INVALID, "coo count %lld out of range", (long long)n);
  if (n > 0 && (!bi || !bj)) return make_status(BAMG_ERR_INVALID, "null coordinate array");
  bsr_release(A);
  unsigned long long *keys = nullptr, *keys_s = nullptr;
  int *idx = nullptr, *idx_s = nullptr, *bad = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  auto cleanup = [&]() {
    dfree(keys, st);
    dfree(keys_s, st);
    dfree(idx, st);
    dfree(bad, st);
    dfree(tmp, st);
  };
  auto body = [&]() -> Status {
    std::vector<int> rowptr(A->nbr + 1, 0), colidx, seg(1, 0);
    if (n == 0) {
      A->coo_n = 0;
      BAMG_TRY(bsr_set_pattern(A, std::move(rowptr), std::move(colidx), kSortAuto));
      return upload(&A->coo_seg, seg, st);
    }
    BAMG_TRY(dalloc(&keys, n, st));
    BAMG_TRY(dalloc(&keys_s, n, st));
    BAMG_TRY(dalloc(&idx, n, st));
    BAMG_TRY(dalloc(&idx_s, n, st));
    BAMG_TRY(dalloc(&bad, 1, st));
    BAMG_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32);
    { k_coo_keys<<<blocks, 256, 0, st>>>(bi, bj, n, A->nbr, A->nbc, keys, idx, bad); BAMG_COUNT_LAUNCH; }
    BAMG_CUDA(cudaGetLastError());
    int hbad = 0;
    BAMG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    BAMG_CUDA(cudaStreamSynchronize(st));
    if (hbad) return make_status(BAMG_ERR_INVALID, "coo block index out of range (nbr=%lld nbc=%lld)",
                                 (long long)A->nbr, (long long)A->nbc);
    // stable radix sort: equal coordinates keep their input order
    BAMG_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys_s, idx, idx_s, (int)n, 0, 64, st));
    BAMG_TRY(dalloc((char**)&tmp, (int64_t)tmp_bytes, st));
    BAMG_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys, keys_s, idx, idx_s, (int)n, 0, 64, st));
    std::vector<unsigned long long> hk;
    BAMG_TRY(download(hk, keys_s, n, st));
    int64_t kept = 0;
    for (int64_t k = 0; k < n; ++k) {
      const unsigned long long key = hk[k];
      if (key == ~0ull) break;
      if (k == 0 || key != hk[k - 1]) {
        const int i = (int)(key >> 32);
        colidx.push_back((int)(key & 0xffffffffu));
        rowptr[i + 1]++;
        if (k > 0) seg.push_back((int)k);
      }
      kept = k + 1;
    }
    if (kept > 0) seg.push_back((int)kept);
    for (int64_t i = 0; i < A->nbr; ++i) rowptr[i + 1] += rowptr[i];
    A->coo_n = n;
    BAMG_TRY(bsr_set_pattern(A, std::move(rowptr), std::move(colidx), kSortAuto));
    BAMG_TRY(upload(&A->coo_seg, seg, st));
    A->coo_perm = idx_s;
    idx_s = nullptr;
    // the same plan in storage-slot order (slots in slice order)
    {
      std::vector<int> hperm;
      BAMG_TRY(download(hperm, A->coo_perm, kept, st));
      const int64_t nslots = A->nchunks * (int64_t)kSlice;
      std::vector<int> kof(nslots, -1), soff(nslots + 1, 0), sperm;
      sperm.reserve((size_t)kept);
      for (int64_t k = 0; k < A->nnzb; ++k) kof[A->h_slot_of[k]] = (int)k;
      for (int64_t t = 0; t < nslots; ++t) {
        const int k = kof[t];
        if (k >= 0) sperm.insert(sperm.end(), hperm.begin() + seg[k], hperm.begin() + seg[k + 1]);
        soff[t + 1] = (int)sperm.size();
      }
      BAMG_TRY(upload(&A->coo_soff, soff, st));
      BAMG_TRY(upload(&A->coo_sperm, sperm, st));
    }
    BAMG_CUDA(cudaStreamSynchronize(st));
    return Status{};
  };
  Status s = body();
  cleanup();
  dfree(idx_s, st);
  return s;
}

static Status coo_set_values(bamg_bsr* A, const double* v, int add) {
  if (!A->has_pattern || !A->coo_seg) return make_status(BAMG_ERR_STATE, "coo_set_values before coo_preallocate");
  if (A->coo_n > 0 && !v) return make_status(BAMG_ERR_INVALID, "null value array");
  cudaStream_t st = A->ctx->stream;
  const int B = (int)A->block_elems();
  const int64_t nt = A->nnzb * B;
  // keep an existing float copy current in the same pass
  float* v32 = (A->vals32 && A->vals32_version == A->version) ? A->vals32 : nullptr;
  if (nt > 0) {
    const unsigned blocks = (unsigned)((nt + 255) / 256);
    const int pm = prof_begin(A->ctx, BAMG_PROF_COO, st);
    const int64_t nslots = A->nchunks * (int64_t)kSlice;
    const unsigned sblocks = (unsigned)((nslots + 127) / 128);
    if (B == 9 && A->coo_soff)
      { k_coo_sum_slots<9><<<sblocks, 128, 0, st>>>(A->coo_soff, A->coo_sperm, v, nslots, A->vals, v32, add,
                                                  A->ctx->d_err); BAMG_COUNT_LAUNCH; }
    else if (B == 9)
      { k_coo_sum<9><<<blocks, 256, 0, st>>>(A->coo_seg, A->coo_perm, v, A->slot_of, A->nnzb, A->vals, v32, add,
                                           A->ctx->d_err); BAMG_COUNT_LAUNCH; }
    else if (B == 36)
      { k_coo_sum<36><<<blocks, 256, 0, st>>>(A->coo_seg, A->coo_perm, v, A->slot_of, A->nnzb, A->vals, v32, add,
                                            A->ctx->d_err); BAMG_COUNT_LAUNCH; }
    else if (B == 18)
      { k_coo_sum<18><<<blocks, 256, 0, st>>>(A->coo_seg, A->coo_perm, v, A->slot_of, A->nnzb, A->vals, v32, add,
                                            A->ctx->d_err); BAMG_COUNT_LAUNCH; }
    else
      { k_coo_sum_any<<<blocks, 256, 0, st>>>(A->coo_seg, A->coo_perm, v, A->slot_of, A->nnzb, B, A->vals, v32, add,
                                            A->ctx->d_err); BAMG_COUNT_LAUNCH; }
    prof_end(A->ctx, pm, st);
    BAMG_CUDA(cudaGetLastError());
  }
  A->version++;
  if (v32) A->vals32_version = A->version;
  return Status{};
}

// Element-by-element assembly, the baseline blocked COO is measured against
// (Sec. 5): every contribution is added straight into its block with an FP64
// atomic.  The slot of each input entry comes from the COO plan.
__global__ void k_coo_entry_slot(const int* __restrict__ seg, const int* __restrict__ perm,
                                 const int* __restrict__ slot_of, int64_t nnzb, int* __restrict__ entry_slot) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nnzb) return;
  const int slot = slot_of[k];
  for (int s = seg[k]; s < seg[k + 1]; ++s) entry_slot[perm[s]] = slot;
}

template <int B>
__global__ void k_coo_scatter(int64_t n, const int* __restrict__ entry_slot, const double* __restrict__ v,
                              double* __restrict__ vals) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * B) return;
  const int64_t k = t / B;
  const int e = (int)(t - k * B);
  const int slot = entry_slot[k];
  if (slot >= 0) atomicAdd(vals + vidx<B>(slot, e), __ldg(v + t));
}

static Status coo_scatter_values(bamg_bsr* A, const double* v, int add) {
  if (!A->has_pattern || !A->coo_seg) return make_status(BAMG_ERR_STATE, "coo_scatter_values before coo_preallocate");
  if (A->coo_n > 0 && !v) return make_status(BAMG_ERR_INVALID, "null value array");
  const int B = (int)A->block_elems();
  if (B != 9 && B != 18 && B != 36) return make_status(BAMG_ERR_INVALID, "element-by-element assembly supports 3x3, 3x6, 6x3 and 6x6 blocks");
  cudaStream_t st = A->ctx->stream;
  if (!A->coo_slot && A->coo_n > 0) {
    BAMG_TRY(dalloc(&A->coo_slot, A->coo_n, st));
    BAMG_CUDA(cudaMemsetAsync(A->coo_slot, 0xFF, sizeof(int) * (size_t)A->coo_n, st));  // -1: ignored entries
    if (A->nnzb > 0) {
      k_coo_entry_slot<<<(unsigned)((A->nnzb + 255) / 256), 256, 0, st>>>(A->coo_seg, A->coo_perm, A->slot_of, A->nnzb,
                                                                          A->coo_slot);
      BAMG_COUNT_LAUNCH;
    }
  }
  if (!add) BAMG_CUDA(cudaMemsetAsync(A->vals, 0, sizeof(double) * (size_t)(A->nslots() * B), st));
  const int64_t nt = A->coo_n * B;
  if (nt > 0) {
    const unsigned blocks = (unsigned)((nt + 255) / 256);
    if (B == 9) k_coo_scatter<9><<<blocks, 256, 0, st>>>(A->coo_n, A->coo_slot, v, A->vals);
    else if (B == 18) k_coo_scatter<18><<<blocks, 256, 0, st>>>(A->coo_n, A->coo_slot, v, A->vals);
    else k_coo_scatter<36><<<blocks, 256, 0, st>>>(A->coo_n, A->coo_slot, v, A->vals);
    BAMG_COUNT_LAUNCH;
  }
  BAMG_CUDA(cudaGetLastError());
  A->version++;  // the float copy, if any, is now behind and is refreshed on its next use
  A->vals64_stale = false;
  return Status{};
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_bsr_coo_scatter_values(bamg_bsr* A, const double* v, int add) {
  if (!A) return BAMG_ERR_INVALID;
  Status s = coo_scatter_values(A, v, add);
  return s.ok() ? BAMG_OK : fail(A->ctx, s);
}

bamg_status bamg_bsr_coo_preallocate(bamg_bsr* A, int64_t n, const int32_t* bi, const int32_t* bj) {
  if (!A) return BAMG_ERR_INVALID;
  Status s = coo_preallocate(A, n, bi, bj);
  return s.ok() ? BAMG_OK : fail(A->ctx, s);
}

bamg_status bamg_bsr_coo_set_values(bamg_bsr* A, const double* v, int add) {
  if (!A) return BAMG_ERR_INVALID;
  Status s = coo_set_values(A, v, add);
  return s.ok() ? BAMG_OK : fail(A->ctx, s);
}

}  // extern "C"
