// Galerkin product A_c = P^T A P on rectangular-block matrices (Sec. 2.2,
// Sec. 3.1): symbolic phase once (host), numeric phase reused (device).
//
// Numeric design.  Stage 1 computes the intermediate Z = A P, one output block
// per lane group (bs_p lanes, one per output column): each lane accumulates
// its column over the block pairs (A_ik, P_kJ) in the output's gather list.
// Stage 2 computes A_c = P^T Z the same way over the pairs (P_iI, Z_iJ).
// Lists are fixed by the symbolic phase, so results are deterministic and no
// atomics are used.  With FP64 arithmetic at 2 FMA/clock/SM the kernels are
// bound by the FP64 pipe, not by memory; the gather lists keep every FMA
// useful (no padding to dense local blocks) and the work-sorted item order
// keeps the lane groups of a warp busy for the same number of steps.
#include <algorithm>
#include <numeric>

#include "device.cuh"
#include "internal.h"

namespace bamg {

template <int BS, int BSP, typename T>
__global__ void __launch_bounds__(256) k_ptap_stage1(int64_t n1, const int* __restrict__ item_z,
                                                     const int* __restrict__ off, const int* __restrict__ ea,
                                                     const int* __restrict__ ep, const T* __restrict__ Avals,
                                                     const T* __restrict__ Pblk, T* __restrict__ Z) {
  constexpr int G = 32 / BSP;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int g = lane / BSP, c = lane - g * BSP;
  if (g >= G) return;
  const int64_t item = warp * G + g;
  if (item >= n1) return;
  T acc[BS];
#pragma unroll
  for (int r = 0; r < BS; ++r) acc[r] = T(0);
  const int s0 = __ldg(off + item), s1 = __ldg(off + item + 1);
  for (int s = s0; s < s1; ++s) {
    const int64_t aslot = __ldg(ea + s);
    const int64_t pb = __ldg(ep + s);
    T p[BS];
#pragma unroll
    for (int q = 0; q < BS; ++q) p[q] = __ldg(Pblk + pb * (BS * BSP) + q * BSP + c);
    const T* a = Avals + (aslot >> 5) * (32LL * BS * BS) + (aslot & 31);
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int q = 0; q < BS; ++q) acc[r] = fma(__ldg(a + 32 * (r * BS + q)), p[q], acc[r]);
  }
  const int64_t z = __ldg(item_z + item);
#pragma unroll
  for (int r = 0; r < BS; ++r) Z[z * (BS * BSP) + r * BSP + c] = acc[r];
}

template <int BS, int BSP, typename T>
__global__ void __launch_bounds__(256) k_ptap_stage2(int64_t n2, const int* __restrict__ item_slot,
                                                     const int* __restrict__ item_tslot,
                                                     const int* __restrict__ off, const int* __restrict__ ep,
                                                     const int* __restrict__ ez, const T* __restrict__ Pblk,
                                                     const T* __restrict__ Z, T* __restrict__ Ac) {
  constexpr int G = 32 / BSP;
  constexpr int BC = BSP * BSP;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int g = lane / BSP, c = lane - g * BSP;
  if (g >= G) return;
  const int64_t item = warp * G + g;
  if (item >= n2) return;
  T acc[BSP];
#pragma unroll
  for (int u = 0; u < BSP; ++u) acc[u] = T(0);
  const int s0 = __ldg(off + item), s1 = __ldg(off + item + 1);
  for (int s = s0; s < s1; ++s) {
    const int64_t pb = __ldg(ep + s);
    const int64_t z = __ldg(ez + s);
    T zc[BS];
#pragma unroll
    for (int r = 0; r < BS; ++r) zc[r] = __ldg(Z + z * (BS * BSP) + r * BSP + c);
    const T* p = Pblk + pb * (BS * BSP);
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int u = 0; u < BSP; ++u) acc[u] = fma(__ldg(p + r * BSP + u), zc[r], acc[u]);
  }
  const int64_t slot = __ldg(item_slot + item);
  T* o = Ac + (slot >> 5) * (32LL * BC) + (slot & 31);
#pragma unroll
  for (int u = 0; u < BSP; ++u) o[32 * (u * BSP + c)] = acc[u];
  const int64_t ts = __ldg(item_tslot + item);
  if (ts >= 0) {
    T* t = Ac + (ts >> 5) * (32LL * BC) + (ts & 31);
#pragma unroll
    for (int u = 0; u < BSP; ++u) t[32 * (c * BSP + u)] = acc[u];
  }
}

// Stable order of items by decreasing list length (counting sort).
static std::vector<int> order_by_work(const std::vector<int>& off) {
  const int64_t n = (int64_t)off.size() - 1;
  int maxlen = 0;
  for (int64_t i = 0; i < n; ++i) maxlen = std::max(maxlen, off[i + 1] - off[i]);
  std::vector<int64_t> start(maxlen + 2, 0);
  for (int64_t i = 0; i < n; ++i) start[maxlen - (off[i + 1] - off[i]) + 1]++;
  for (int l = 0; l <= maxlen; ++l) start[l + 1] += start[l];
  std::vector<int> order((size_t)n);
  for (int64_t i = 0; i < n; ++i) order[start[maxlen - (off[i + 1] - off[i])]++] = (int)i;
  return order;
}

// Reorder CSR-like lists (off, a, b) into item order.
static void permute_lists(const std::vector<int>& order, const std::vector<int>& off, const std::vector<int>& a,
                          const std::vector<int>& b, std::vector<int>& noff, std::vector<int>& na,
                          std::vector<int>& nb) {
  const size_t n = order.size();
  noff.assign(n + 1, 0);
  na.resize(a.size());
  nb.resize(b.size());
  for (size_t t = 0; t < n; ++t) {
    const int i = order[t];
    const int len = off[i + 1] - off[i];
    noff[t + 1] = noff[t] + len;
    std::copy(a.begin() + off[i], a.begin() + off[i + 1], na.begin() + noff[t]);
    std::copy(b.begin() + off[i], b.begin() + off[i + 1], nb.begin() + noff[t]);
  }
}

void ptap_release(bamg_ptap* p) {
  if (!p) return;
  cudaStream_t st = p->ctx->stream;
  dfree(p->s1_z, st);
  dfree(p->s1_off, st);
  dfree(p->s1_a, st);
  dfree(p->s1_p, st);
  dfree(p->s2_slot, st);
  dfree(p->s2_tslot, st);
  dfree(p->s2_off, st);
  dfree(p->s2_p, st);
  dfree(p->s2_z, st);
  dfree(p->Z, st);
  dfree(p->Z32, st);
  dfree(p->Pblk, st);
  dfree(p->Pblk32, st);
}

Status ptap_build(bamg_bsr* A, bamg_bsr* P, bool want_ac, bamg_ptap** plan_out, bamg_bsr** Ac_out) {
  *plan_out = nullptr;
  if (Ac_out) *Ac_out = nullptr;
  if (!A->has_pattern || !P->has_pattern) return make_status(BAMG_ERR_STATE, "Galerkin operands need patterns");
  if (A->br != A->bc || A->nbr != A->nbc)
    return make_status(BAMG_ERR_INVALID, "A must be square with square blocks");
  if (P->nbr != A->nbr || P->br != A->br)
    return make_status(BAMG_ERR_INVALID, "P rows (%lld x bs %d) do not match A (%lld x bs %d)", (long long)P->nbr,
                       P->br, (long long)A->nbr, A->br);
  const int bs = A->br, bsp = P->bc;
  const bool supported = (bs == 3 && bsp == 6) || (bs == 6 && bsp == 6) || (bs == 3 && bsp == 3);
  if (!supported) return make_status(BAMG_ERR_INVALID, "Galerkin block sizes %d -> %d not supported", bs, bsp);
  bamg_ctx* ctx = A->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t n = A->nbr, nc = P->nbc;
  const auto &ar = A->h_rowptr, &ac = A->h_colidx, &aslot = A->h_slot_of;
  const auto &pr = P->h_rowptr, &pc = P->h_colidx;

  bamg_ptap* pl = new bamg_ptap();
  pl->ctx = ctx;
  pl->A = A;
  pl->P = P;
  pl->bs = bs;
  pl->bsp = bsp;
  pl->a_pid = A->pattern_id;
  pl->p_pid = P->pattern_id;
  pl->symmetric = A->symmetric;
  Status s = [&]() -> Status {
    // ---- Z = A P pattern and stage-1 lists (pairs in A-row order, then P-row order)
    std::vector<int>& zr = pl->h_zrowptr;
    std::vector<int>& zc = pl->h_zcol;
    zr.assign(n + 1, 0);
    std::vector<int> mark(nc, -1), pos(nc, -1), rowJ;
    std::vector<int> off1(1, 0), la, lp, cnt;
    for (int64_t i = 0; i < n; ++i) {
      rowJ.clear();
      for (int q = ar[i]; q < ar[i + 1]; ++q) {
        const int k = ac[q];
        for (int t = pr[k]; t < pr[k + 1]; ++t) {
          const int J = pc[t];
          if (mark[J] != (int)i) {
            mark[J] = (int)i;
            rowJ.push_back(J);
          }
        }
      }
      std::sort(rowJ.begin(), rowJ.end());
      const int z0 = (int)zc.size();
      for (size_t u = 0; u < rowJ.size(); ++u) {
        pos[rowJ[u]] = z0 + (int)u;
        zc.push_back(rowJ[u]);
      }
      zr[i + 1] = (int)zc.size();
      cnt.assign(rowJ.size(), 0);
      for (int q = ar[i]; q < ar[i + 1]; ++q)
        for (int t = pr[ac[q]]; t < pr[ac[q] + 1]; ++t) cnt[pos[pc[t]] - z0]++;
      const size_t base = la.size();
      std::vector<int> fill(rowJ.size());
      size_t acc = base;
      for (size_t u = 0; u < rowJ.size(); ++u) {
        fill[u] = (int)acc;
        acc += cnt[u];
        off1.push_back((int)acc);
      }
      la.resize(acc);
      lp.resize(acc);
      for (int q = ar[i]; q < ar[i + 1]; ++q) {
        const int k = ac[q];
        for (int t = pr[k]; t < pr[k + 1]; ++t) {
          const int u = pos[pc[t]] - z0;
          la[fill[u]] = aslot[q];
          lp[fill[u]] = t;
          fill[u]++;
        }
      }
      if (la.size() >= (size_t)INT32_MAX) return make_status(BAMG_ERR_INVALID, "Galerkin product too large");
    }
    pl->nz = (int64_t)zc.size();
    pl->n1 = pl->nz;
    pl->e1 = (int64_t)la.size();
    {
      std::vector<int> order = order_by_work(off1), noff, na, np;
      permute_lists(order, off1, la, lp, noff, na, np);
      BAMG_TRY(upload(&pl->s1_z, order, st));
      BAMG_TRY(upload(&pl->s1_off, noff, st));
      BAMG_TRY(upload(&pl->s1_a, na, st));
      BAMG_TRY(upload(&pl->s1_p, np, st));
      BAMG_CUDA(cudaStreamSynchronize(st));
    }
    BAMG_TRY(dalloc(&pl->Z, pl->nz * bs * bsp, st));
    if (!want_ac) return Status{};

    // ---- A_c pattern and stage-2 lists: rows I over R_I = {(i, t): P(i, I) = t}
    std::vector<int> rr(nc + 1, 0), ri, rt;
    for (int64_t t = 0; t < (int64_t)pc.size(); ++t) rr[pc[t] + 1]++;
    for (int64_t I = 0; I < nc; ++I) rr[I + 1] += rr[I];
    ri.resize(pc.size());
    rt.resize(pc.size());
    {
      std::vector<int> fill(rr.begin(), rr.end() - 1);
      for (int64_t i = 0; i < n; ++i)
        for (int t = pr[i]; t < pr[i + 1]; ++t) {
          const int I = pc[t];
          ri[fill[I]] = (int)i;
          rt[fill[I]] = t;
          fill[I]++;
        }
    }
    std::vector<int> cr(nc + 1, 0), ccol;
    std::vector<int> off2, l2p, l2z, item_ac;
    std::fill(mark.begin(), mark.end(), -1);
    std::vector<std::vector<std::pair<int, int>>> rowlists;
    for (int64_t I = 0; I < nc; ++I) {
      rowJ.clear();
      for (int u = rr[I]; u < rr[I + 1]; ++u) {
        const int i = ri[u];
        for (int z = zr[i]; z < zr[i + 1]; ++z) {
          const int J = zc[z];
          if (mark[J] != (int)I) {
            mark[J] = (int)I;
            rowJ.push_back(J);
          }
        }
      }
      std::sort(rowJ.begin(), rowJ.end());
      const int c0 = (int)ccol.size();
      for (size_t u = 0; u < rowJ.size(); ++u) {
        pos[rowJ[u]] = (int)u;
        ccol.push_back(rowJ[u]);
      }
      cr[I + 1] = (int)ccol.size();
      rowlists.assign(rowJ.size(), {});
      for (int u = rr[I]; u < rr[I + 1]; ++u) {
        const int i = ri[u], t = rt[u];
        for (int z = zr[i]; z < zr[i + 1]; ++z) {
          const int J = zc[z];
          if (pl->symmetric && J < I) continue;
          rowlists[pos[J]].push_back({t, z});
        }
      }
      for (size_t u = 0; u < rowJ.size(); ++u) {
        if (pl->symmetric && rowJ[u] < I) continue;
        item_ac.push_back(c0 + (int)u);
        off2.push_back((int)l2p.size());
        for (auto& e : rowlists[u]) {
          l2p.push_back(e.first);
          l2z.push_back(e.second);
        }
      }
      if (l2p.size() >= (size_t)INT32_MAX) return make_status(BAMG_ERR_INVALID, "Galerkin product too large");
    }
    off2.push_back((int)l2p.size());
    bamg_bsr* Ac = nullptr;
    if (bamg_bsr_create(ctx, bsp, bsp, nc, nc, &Ac) != BAMG_OK) return make_status(BAMG_ERR_OOM, "create A_c");
    *Ac_out = Ac;
    pl->Ac = Ac;
    Ac->symmetric = pl->symmetric;
    std::vector<int> crow_copy = cr, ccol_copy = ccol;
    BAMG_TRY(bsr_set_pattern(Ac, std::move(crow_copy), std::move(ccol_copy), kSortAuto));
    pl->ac_pid = Ac->pattern_id;
    const auto& cslot = Ac->h_slot_of;
    const auto& crp = Ac->h_rowptr;
    const auto& ccl = Ac->h_colidx;
    std::vector<int> islot(item_ac.size()), itslot(item_ac.size(), -1);
    std::vector<int> Irow(ccl.size());
    for (int64_t I = 0; I < nc; ++I)
      for (int k = crp[I]; k < crp[I + 1]; ++k) Irow[k] = (int)I;
    for (size_t it = 0; it < item_ac.size(); ++it) {
      const int k = item_ac[it];
      islot[it] = cslot[k];
      const int I = Irow[k], J = ccl[k];
      if (pl->symmetric && J != I) {
        auto b = ccl.begin() + crp[J], e = ccl.begin() + crp[J + 1];
        auto f = std::lower_bound(b, e, I);
        if (f == e || *f != I) return make_status(BAMG_ERR_INVALID, "symmetric A_c pattern is not symmetric");
        itslot[it] = cslot[crp[J] + (int)(f - b)];
      }
    }
    pl->n2 = (int64_t)item_ac.size();
    pl->e2 = (int64_t)l2p.size();
    std::vector<int> order = order_by_work(off2), noff, np, nz;
    permute_lists(order, off2, l2p, l2z, noff, np, nz);
    std::vector<int> os(order.size()), ots(order.size());
    for (size_t t = 0; t < order.size(); ++t) {
      os[t] = islot[order[t]];
      ots[t] = itslot[order[t]];
    }
    BAMG_TRY(upload(&pl->s2_slot, os, st));
    BAMG_TRY(upload(&pl->s2_tslot, ots, st));
    BAMG_TRY(upload(&pl->s2_off, noff, st));
    BAMG_TRY(upload(&pl->s2_p, np, st));
    BAMG_TRY(upload(&pl->s2_z, nz, st));
    BAMG_CUDA(cudaStreamSynchronize(st));
    return Status{};
  }();
  if (!s.ok()) {
    ptap_release(pl);
    if (Ac_out && *Ac_out) {
      bamg_bsr_destroy(*Ac_out);
      *Ac_out = nullptr;
    }
    delete pl;
    return s;
  }
  *plan_out = pl;
  return Status{};
}

template <typename T>
static Status run_stages(bamg_ptap* pl, const T* Avals, const T* Pblk, T* Z, T* Acvals, bool stage2) {
  cudaStream_t st = pl->ctx->stream;
  const int G = 32 / pl->bsp;
  auto blocks_for = [&](int64_t items) { return (unsigned)((items + (int64_t)G * 8 - 1) / ((int64_t)G * 8)); };
  if (pl->n1 > 0) {
    const unsigned b = blocks_for(pl->n1);
    const int pm = prof_begin(pl->ctx, pl->prof_stage1, st);
    if (pl->bs == 3 && pl->bsp == 6)
      { k_ptap_stage1<3, 6, T><<<b, 256, 0, st>>>(pl->n1, pl->s1_z, pl->s1_off, pl->s1_a, pl->s1_p, Avals, Pblk, Z); BAMG_COUNT_LAUNCH; }
    else if (pl->bs == 6 && pl->bsp == 6)
      { k_ptap_stage1<6, 6, T><<<b, 256, 0, st>>>(pl->n1, pl->s1_z, pl->s1_off, pl->s1_a, pl->s1_p, Avals, Pblk, Z); BAMG_COUNT_LAUNCH; }
    else
      { k_ptap_stage1<3, 3, T><<<b, 256, 0, st>>>(pl->n1, pl->s1_z, pl->s1_off, pl->s1_a, pl->s1_p, Avals, Pblk, Z); BAMG_COUNT_LAUNCH; }
    prof_end(pl->ctx, pm, st);
    BAMG_CUDA(cudaGetLastError());
  }
  if (stage2 && pl->n2 > 0) {
    const unsigned b = blocks_for(pl->n2);
    const int pm = prof_begin(pl->ctx, pl->prof_stage2, st);
    if (pl->bs == 3 && pl->bsp == 6)
      { k_ptap_stage2<3, 6, T><<<b, 256, 0, st>>>(pl->n2, pl->s2_slot, pl->s2_tslot, pl->s2_off, pl->s2_p, pl->s2_z,
                                                Pblk, Z, Acvals); BAMG_COUNT_LAUNCH; }
    else if (pl->bs == 6 && pl->bsp == 6)
      { k_ptap_stage2<6, 6, T><<<b, 256, 0, st>>>(pl->n2, pl->s2_slot, pl->s2_tslot, pl->s2_off, pl->s2_p, pl->s2_z,
                                                Pblk, Z, Acvals); BAMG_COUNT_LAUNCH; }
    else
      { k_ptap_stage2<3, 3, T><<<b, 256, 0, st>>>(pl->n2, pl->s2_slot, pl->s2_tslot, pl->s2_off, pl->s2_p, pl->s2_z,
                                                Pblk, Z, Acvals); BAMG_COUNT_LAUNCH; }
    prof_end(pl->ctx, pm, st);
    BAMG_CUDA(cudaGetLastError());
  }
  return Status{};
}

// State gate (Sec. 3.5): the block-ordered copy of P is rebuilt only when P's
// version differs from the cached one.
static Status refresh_pblk(bamg_ptap* pl, bamg_bsr* P, bool fp32) {
  cudaStream_t st = pl->ctx->stream;
  const int64_t ne = P->nnzb * P->block_elems();
  if (pl->pblk_version != P->version) {
    if (P->vals64_stale) return make_status(BAMG_ERR_STATE, "P holds only FP32 values");
    if (!pl->Pblk) BAMG_TRY(dalloc(&pl->Pblk, ne, st));
    BAMG_TRY(launch_gather_blocks(P, P->vals, pl->Pblk, st));
    pl->pblk_version = P->version;
    pl->pblk_refreshes++;
  }
  if (fp32 && pl->pblk32_version != P->version) {
    if (!pl->Pblk32) BAMG_TRY(dalloc(&pl->Pblk32, ne, st));
    BAMG_TRY(launch_to_fp32(pl->Pblk, pl->Pblk32, ne, st));
    pl->pblk32_version = P->version;
  }
  return Status{};
}

Status ptap_run(bamg_ptap* pl, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac, bamg_prec prec, bool stage2) {
  if (A != pl->A || P != pl->P || (stage2 && Ac != pl->Ac) || A->pattern_id != pl->a_pid ||
      P->pattern_id != pl->p_pid || (stage2 && Ac->pattern_id != pl->ac_pid))
    return make_status(BAMG_ERR_STATE, "Galerkin plan used with matrices it was not built for");
  if (stage2 && !pl->Ac) return make_status(BAMG_ERR_STATE, "plan has no coarse stage");
  cudaStream_t st = pl->ctx->stream;
  if (prec == BAMG_FP64) {
    if (A->vals64_stale) return make_status(BAMG_ERR_STATE, "A holds only FP32 values; use BAMG_FP32");
    BAMG_TRY(refresh_pblk(pl, P, false));
    BAMG_TRY(run_stages<double>(pl, A->vals, pl->Pblk, pl->Z, stage2 ? Ac->vals : nullptr, stage2));
    if (stage2) {
      Ac->version++;
      Ac->vals64_stale = false;
    }
  } else if (prec == BAMG_FP32) {
    BAMG_TRY(bsr_ensure_fp32(A));
    BAMG_TRY(refresh_pblk(pl, P, true));
    if (!pl->Z32) BAMG_TRY(dalloc(&pl->Z32, pl->nz * pl->bs * pl->bsp, st));
    if (stage2 && !Ac->vals32) BAMG_TRY(dalloc(&Ac->vals32, Ac->nslots() * Ac->block_elems(), st));
    if (stage2 && Ac->vals32 && Ac->vals32_version == ~0ull)
      BAMG_CUDA(cudaMemsetAsync(Ac->vals32, 0, sizeof(float) * Ac->nslots() * Ac->block_elems(), st));
    BAMG_TRY(run_stages<float>(pl, A->vals32, pl->Pblk32, pl->Z32, stage2 ? Ac->vals32 : nullptr, stage2));
    if (stage2) {
      Ac->version++;
      Ac->vals32_version = Ac->version;
      Ac->vals64_stale = true;
    }
  } else {
    return make_status(BAMG_ERR_INVALID, "bad precision");
  }
  return Status{};
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_ptap_symbolic(bamg_bsr* A, bamg_bsr* P, bamg_ptap** plan, bamg_bsr** Ac) {
  if (!A || !P || !plan || !Ac) return BAMG_ERR_INVALID;
  Status s = ptap_build(A, P, true, plan, Ac);
  return s.ok() ? BAMG_OK : fail(A->ctx, s);
}

bamg_status bamg_ptap_numeric(bamg_ptap* plan, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac) {
  if (!plan || !A || !P || !Ac) return BAMG_ERR_INVALID;
  Status s = ptap_run(plan, A, P, Ac, BAMG_FP64, true);
  return s.ok() ? BAMG_OK : fail(plan->ctx, s);
}

bamg_status bamg_ptap_numeric_prec(bamg_ptap* plan, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac, bamg_prec prec) {
  if (!plan || !A || !P || !Ac) return BAMG_ERR_INVALID;
  Status s = ptap_run(plan, A, P, Ac, prec, true);
  return s.ok() ? BAMG_OK : fail(plan->ctx, s);
}

bamg_status bamg_ptap_get_refreshes(const bamg_ptap* plan, uint64_t* p_refreshes) {
  if (!plan || !p_refreshes) return BAMG_ERR_INVALID;
  *p_refreshes = plan->pblk_refreshes;
  return BAMG_OK;
}

bamg_status bamg_ptap_destroy(bamg_ptap* plan) {
  if (!plan) return BAMG_OK;
  ptap_release(plan);
  delete plan;
  return BAMG_OK;
}

}  // extern "C"
