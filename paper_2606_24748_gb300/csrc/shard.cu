// Row-sharded operator (Sec. 3.3, Sec. 3.5, Sec. 4.8): the fine operator's
// block rows are split into contiguous ranges, one per part.  A part holds
// its rows with columns renumbered locally: its own columns first, then the
// ghost columns (owned by other parts) in ascending global order, so the
// ghosts arrive grouped by owner.
//
//  - SpMV: a part gathers its ghost entries of x (the halo), then multiplies
//    its rows by [x_own; x_ghost].
//  - Galerkin product: a part needs the rows of P for its ghost columns
//    (P_oth), gathered once and kept until P's version changes (the state
//    gate of Sec. 3.5).  With A_ext = the part's rows in a square matrix of
//    size owned + ghosts whose ghost rows are empty, and
//    P_ext = [P_own; P_oth], the part's contribution is
//    C_p = P_ext^T A_ext P_ext = P_own^T (A_p P_ext), and A_c = sum_p C_p:
//    the contributions to coarse rows another part owns are the
//    off-process reduce.
//
// The partition plan (bamg_halo) is host-only: it lists, for every part, the
// local pattern, the ghosts and their owners, and what each part sends to
// each other part.  The device object (bamg_sharded) runs every part of one
// partition on the context's GPU, one after another, with the exchanges as
// device gathers; the plan's lists are the messages a multi-GPU run would send.
#include <algorithm>
#include <numeric>

#include "device.cuh"
#include "internal.h"

struct bamg_halo {
  int nparts = 0;
  int64_t nbr = 0;
  std::vector<int64_t> starts;  // nparts + 1
  struct Part {
    int64_t n = 0;                         // owned rows
    std::vector<int> rowptr, col;          // local pattern (columns: owned, then ghosts)
    std::vector<int64_t> src;              // global block index of each local block
    std::vector<int64_t> ghost;            // ghost global columns, ascending
    std::vector<int> owner;                // part owning each ghost
  };
  std::vector<Part> parts;
  // sends[p * nparts + q]: local rows of part p that part q needs, in q's ghost order
  std::vector<std::vector<int64_t>> sends;
};

namespace bamg {

static int owner_of(const std::vector<int64_t>& starts, int64_t c) {
  return (int)(std::upper_bound(starts.begin(), starts.end(), c) - starts.begin()) - 1;
}

static Status halo_build(int64_t nbr, const int* rowptr, const int* colidx, int nparts, const int64_t* row_starts,
                         bamg_halo* H) {
  if (nparts < 1 || !row_starts || row_starts[0] != 0 || row_starts[nparts] != nbr)
    return make_status(BAMG_ERR_INVALID, "row_starts must run from 0 to the number of block rows");
  for (int p = 0; p < nparts; ++p)
    if (row_starts[p + 1] < row_starts[p]) return make_status(BAMG_ERR_INVALID, "row_starts must not decrease");
  H->nparts = nparts;
  H->nbr = nbr;
  H->starts.assign(row_starts, row_starts + nparts + 1);
  H->parts.assign(nparts, {});
  H->sends.assign((size_t)nparts * nparts, {});
  for (int p = 0; p < nparts; ++p) {
    bamg_halo::Part& P = H->parts[p];
    const int64_t r0 = row_starts[p], r1 = row_starts[p + 1];
    P.n = r1 - r0;
    for (int64_t i = r0; i < r1; ++i)
      for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        const int64_t c = colidx[q];
        if (c < 0 || c >= nbr) return make_status(BAMG_ERR_INVALID, "column %lld out of range", (long long)c);
        if (c < r0 || c >= r1) P.ghost.push_back(c);
      }
    std::sort(P.ghost.begin(), P.ghost.end());
    P.ghost.erase(std::unique(P.ghost.begin(), P.ghost.end()), P.ghost.end());
    P.owner.resize(P.ghost.size());
    for (size_t k = 0; k < P.ghost.size(); ++k) P.owner[k] = owner_of(H->starts, P.ghost[k]);
    auto local = [&](int64_t c) -> int {
      if (c >= r0 && c < r1) return (int)(c - r0);
      return (int)(P.n + (std::lower_bound(P.ghost.begin(), P.ghost.end(), c) - P.ghost.begin()));
    };
    P.rowptr.assign(P.n + 1, 0);
    std::vector<std::pair<int, int64_t>> row;
    for (int64_t i = r0; i < r1; ++i) {
      row.clear();
      for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) row.push_back({local(colidx[q]), (int64_t)q});
      std::sort(row.begin(), row.end());
      for (auto& e : row) {
        P.col.push_back(e.first);
        P.src.push_back(e.second);
      }
      P.rowptr[i - r0 + 1] = (int)P.col.size();
    }
    for (size_t k = 0; k < P.ghost.size(); ++k)
      H->sends[(size_t)P.owner[k] * nparts + p].push_back(P.ghost[k] - row_starts[P.owner[k]]);
  }
  return Status{};
}

// ------------------------------------------------------------ device side

// dst block b <- src block src_block[b] (sliced layouts of both matrices)
template <typename T>
__global__ void k_copy_blocks(int64_t nb, int B, const int64_t* __restrict__ src_block,
                              const int* __restrict__ src_slot_of, const T* __restrict__ src,
                              const int* __restrict__ dst_slot_of, T* __restrict__ dst) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nb * B) return;
  const int64_t b = t / B;
  const int e = (int)(t % B);
  const int64_t ss = src_slot_of[src_block[b]], ds = dst_slot_of[b];
  dst[(ds >> 5) * 32 * B + 32 * e + (ds & 31)] = src[(ss >> 5) * 32 * B + 32 * e + (ss & 31)];
}

// x_ext = [x rows r0 .. r0+n-1; x rows ghost[0 .. g-1]]  (bs values per row)
__global__ void k_halo_gather(int64_t n, int64_t g, int bs, int64_t r0, const int64_t* __restrict__ ghost,
                              const double* __restrict__ x, double* __restrict__ xe) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (n + g) * bs) return;
  const int64_t i = t / bs;
  const int c = (int)(t % bs);
  const int64_t src = i < n ? r0 + i : ghost[i - n];
  xe[t] = x[src * bs + c];
}

// Off-process reduce: block b of A_c = sum of its contributions k in
// [off[b], off[b+1]), each block cslot[k] of part cpart[k]'s C_p, in part
// order (deterministic).
__global__ void k_reduce_blocks(int64_t nb, int B, const int* __restrict__ off, const int* __restrict__ cpart,
                                const int* __restrict__ cslot, const double* const* __restrict__ cvals,
                                const int* __restrict__ ac_slot_of, double* __restrict__ acv) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nb * B) return;
  const int64_t b = t / B;
  const int e = (int)(t % B);
  double s = 0.0;
  for (int k = off[b]; k < off[b + 1]; ++k) {
    const int64_t cs = cslot[k];
    s += cvals[cpart[k]][(cs >> 5) * 32 * B + 32 * e + (cs & 31)];
  }
  const int64_t as = ac_slot_of[b];
  acv[(as >> 5) * 32 * B + 32 * e + (as & 31)] = s;
}

}  // namespace bamg

struct bamg_sharded {
  bamg_ctx* ctx = nullptr;
  bamg_halo H;
  const bamg_bsr* A = nullptr;   // the global operators the partition was built for
  const bamg_bsr* P = nullptr;
  uint64_t a_pid = 0, p_pid = 0, ac_pid = 0;
  struct Part {
    int64_t n = 0, g = 0, r0 = 0;
    bamg_bsr* Aext = nullptr;      // square, owned + ghost rows (ghost rows empty)
    bamg_bsr* Pext = nullptr;      // [P_own; P_oth]
    bamg_bsr* C = nullptr;         // P_ext^T A_ext P_ext
    bamg_ptap* plan = nullptr;
    int64_t* a_src = nullptr;      // global A block of each A_ext block
    int64_t* p_src = nullptr;      // global P block of each P_ext block
    int64_t* ghost = nullptr;      // ghost global rows
    double* xe = nullptr;          // [x_own; x_ghost]
    double* ye = nullptr;          // A_ext x_ext
    int64_t poth_blocks = 0;       // P_ext blocks in ghost rows
    int64_t reduce_blocks = 0;     // C_p blocks in coarse rows owned by another part
  };
  std::vector<Part> parts;
  uint64_t pext_version = ~0ull;
  uint64_t aext_version = ~0ull;     // A's version the parts' values were copied at
  uint64_t poth_gathers = 0;
  // reduce lists (CSR over A_c blocks)
  int *r_off = nullptr, *r_part = nullptr, *r_slot = nullptr;
  const double** r_vals = nullptr;   // device array of the parts' C_p value pointers
  int64_t nac = 0;
};

namespace bamg {

static void sharded_release(bamg_sharded* S) {
  cudaStream_t st = S->ctx->stream;
  for (auto& p : S->parts) {
    if (p.plan) {
      ptap_release(p.plan);
      delete p.plan;
    }
    if (p.C) bamg_bsr_destroy(p.C);
    if (p.Aext) bamg_bsr_destroy(p.Aext);
    if (p.Pext) bamg_bsr_destroy(p.Pext);
    dfree(p.a_src, st);
    dfree(p.p_src, st);
    dfree(p.ghost, st);
    dfree(p.xe, st);
    dfree(p.ye, st);
  }
  dfree(S->r_off, st);
  dfree(S->r_part, st);
  dfree(S->r_slot, st);
  dfree(S->r_vals, st);
  cudaStreamSynchronize(st);
}

static Status make_bsr(bamg_ctx* ctx, int br, int bc, int64_t nbr, int64_t nbc, std::vector<int>&& rp,
                       std::vector<int>&& ci, bamg_bsr** out) {
  if (bamg_bsr_create(ctx, br, bc, nbr, nbc, out) != BAMG_OK) return make_status(BAMG_ERR_OOM, "part matrix");
  return bsr_set_pattern(*out, std::move(rp), std::move(ci));
}

static Status sharded_build(bamg_sharded* S, bamg_bsr* A, bamg_bsr* P, int nparts, const int64_t* row_starts,
                            bamg_bsr** Ac_out) {
  bamg_ctx* ctx = A->ctx;
  cudaStream_t st = ctx->stream;
  if (!A->has_pattern || !P->has_pattern) return make_status(BAMG_ERR_STATE, "A and P need patterns");
  if (A->br != A->bc || A->nbr != A->nbc || P->nbr != A->nbr || P->br != A->br)
    return make_status(BAMG_ERR_INVALID, "A must be square and P must have A's block rows");
  BAMG_TRY(halo_build(A->nbr, A->h_rowptr.data(), A->h_colidx.data(), nparts, row_starts, &S->H));
  S->A = A;
  S->P = P;
  S->a_pid = A->pattern_id;
  S->p_pid = P->pattern_id;
  const int bs = A->br, bsp = P->bc;
  const int64_t nc = P->nbc;
  const auto &pr = P->h_rowptr, &pc = P->h_colidx;
  // coarse row owner: the part owning the first fine row with a block in that column
  std::vector<int> cowner(nc, -1);
  for (int64_t i = 0; i < P->nbr; ++i)
    for (int q = pr[i]; q < pr[i + 1]; ++q)
      if (cowner[pc[q]] < 0) cowner[pc[q]] = owner_of(S->H.starts, i);
  S->parts.assign(nparts, {});
  std::vector<std::vector<std::pair<int, int>>> ac_rows(nc);  // union pattern (col, -)
  for (int p = 0; p < nparts; ++p) {
    const bamg_halo::Part& hp = S->H.parts[p];
    bamg_sharded::Part& sp = S->parts[p];
    sp.n = hp.n;
    sp.g = (int64_t)hp.ghost.size();
    sp.r0 = S->H.starts[p];
    if (sp.n == 0) continue;
    const int64_t ne = sp.n + sp.g;
    // A_ext: the part's rows, then g empty rows
    std::vector<int> arp(hp.rowptr), aci(hp.col);
    arp.resize(ne + 1, arp.back());
    BAMG_TRY(make_bsr(ctx, bs, bs, ne, ne, std::move(arp), std::move(aci), &sp.Aext));
    // P_ext: P's owned rows, then its ghost rows
    std::vector<int> prp(1, 0), pci;
    std::vector<int64_t> psrc;
    auto add_row = [&](int64_t i) {
      for (int q = pr[i]; q < pr[i + 1]; ++q) {
        pci.push_back(pc[q]);
        psrc.push_back(q);
      }
      prp.push_back((int)pci.size());
    };
    for (int64_t i = 0; i < sp.n; ++i) add_row(sp.r0 + i);
    const int64_t own_blocks = (int64_t)pci.size();
    for (int64_t k = 0; k < sp.g; ++k) add_row(hp.ghost[k]);
    sp.poth_blocks = (int64_t)pci.size() - own_blocks;
    BAMG_TRY(make_bsr(ctx, bs, bsp, ne, nc, std::move(prp), std::move(pci), &sp.Pext));
    BAMG_TRY(upload(&sp.a_src, hp.src, st));
    BAMG_TRY(upload(&sp.p_src, psrc, st));
    BAMG_TRY(upload(&sp.ghost, hp.ghost, st));
    BAMG_TRY(dalloc(&sp.xe, ne * bs, st));
    BAMG_TRY(dalloc(&sp.ye, ne * bs, st));
    BAMG_TRY(ptap_build(sp.Aext, sp.Pext, true, &sp.plan, &sp.C));
    const bamg_bsr* C = sp.C;
    for (int64_t I = 0; I < nc; ++I)
      for (int q = C->h_rowptr[I]; q < C->h_rowptr[I + 1]; ++q) {
        ac_rows[I].push_back({C->h_colidx[q], p});
        if (cowner[I] != p) sp.reduce_blocks++;
      }
  }
  // A_c: the union of the parts' patterns, and each block's contributions in part order
  std::vector<int> rp(nc + 1, 0), ci, off(1, 0), cpart, cslot;
  for (int64_t I = 0; I < nc; ++I) {
    auto& row = ac_rows[I];
    std::sort(row.begin(), row.end());
    for (size_t k = 0; k < row.size(); ++k) {
      if (k == 0 || row[k].first != row[k - 1].first) {
        ci.push_back(row[k].first);
        off.push_back(off.back());
      }
      const int p = row[k].second;
      const bamg_bsr* C = S->parts[p].C;
      const int* b = std::lower_bound(C->h_colidx.data() + C->h_rowptr[I], C->h_colidx.data() + C->h_rowptr[I + 1],
                                      row[k].first);
      cpart.push_back(p);
      cslot.push_back(C->h_slot_of[b - C->h_colidx.data()]);
      off.back()++;
    }
    rp[I + 1] = (int)ci.size();
  }
  S->nac = (int64_t)ci.size();
  bamg_bsr* Ac = nullptr;
  BAMG_TRY(make_bsr(ctx, bsp, bsp, nc, nc, std::move(rp), std::move(ci), &Ac));
  *Ac_out = Ac;
  S->ac_pid = Ac->pattern_id;
  std::vector<const double*> cv(nparts, nullptr);
  for (int p = 0; p < nparts; ++p) cv[p] = S->parts[p].C ? S->parts[p].C->vals : nullptr;
  BAMG_TRY(upload(&S->r_off, off, st));
  BAMG_TRY(upload(&S->r_part, cpart, st));
  BAMG_TRY(upload(&S->r_slot, cslot, st));
  BAMG_TRY(upload(&S->r_vals, cv, st));
  BAMG_CUDA(cudaStreamSynchronize(st));
  return Status{};
}

static Status sharded_check(const bamg_sharded* S, const bamg_bsr* A, const bamg_bsr* P) {
  if (A != S->A || A->pattern_id != S->a_pid || (P && (P != S->P || P->pattern_id != S->p_pid)))
    return make_status(BAMG_ERR_STATE, "sharded operator used with matrices it was not built for");
  if (A->vals64_stale || (P && P->vals64_stale)) return make_status(BAMG_ERR_STATE, "FP64 values needed");
  return Status{};
}

// Each part's rows of A, copied when A's version changed (in a multi-GPU
// run every rank assembles its own rows; here they come from the global A).
static Status sharded_refresh_a(bamg_sharded* S, const bamg_bsr* A, cudaStream_t st) {
  if (S->aext_version == A->version) return Status{};
  const int B = A->br * A->bc;
  for (auto& sp : S->parts) {
    if (sp.n == 0) continue;
    const int64_t nb = sp.Aext->nnzb;
    if (nb > 0) { k_copy_blocks<double><<<(unsigned)((nb * B + 255) / 256), 256, 0, st>>>(nb, B, sp.a_src, A->slot_of, A->vals, sp.Aext->slot_of, sp.Aext->vals); BAMG_COUNT_LAUNCH; }
    sp.Aext->version++;
  }
  BAMG_CUDA(cudaGetLastError());
  S->aext_version = A->version;
  return Status{};
}

static Status sharded_spmv(bamg_sharded* S, const double* x, double* y) {
  cudaStream_t st = S->ctx->stream;
  const bamg_bsr* A = S->A;
  BAMG_TRY(sharded_check(S, A, nullptr));
  BAMG_TRY(sharded_refresh_a(S, A, st));
  const int bs = A->br;
  for (auto& sp : S->parts) {
    if (sp.n == 0) continue;
    const int64_t ne = sp.n + sp.g;
    { k_halo_gather<<<(unsigned)((ne * bs + 255) / 256), 256, 0, st>>>(sp.n, sp.g, bs, sp.r0, sp.ghost, x, sp.xe); BAMG_COUNT_LAUNCH; }
    BAMG_TRY(launch_spmv<double>(sp.Aext, sp.Aext->vals, sp.xe, sp.ye, st));
    BAMG_CUDA(cudaMemcpyAsync(y + sp.r0 * bs, sp.ye, sizeof(double) * sp.n * bs, cudaMemcpyDeviceToDevice, st));
  }
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

static Status sharded_ptap(bamg_sharded* S, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac) {
  cudaStream_t st = S->ctx->stream;
  BAMG_TRY(sharded_check(S, A, P));
  if (Ac->pattern_id != S->ac_pid) return make_status(BAMG_ERR_STATE, "A_c is not the sharded product's matrix");
  const int Bp = P->br * P->bc, Bc = Ac->br * Ac->bc;
  BAMG_TRY(sharded_refresh_a(S, A, st));
  const bool gather_p = S->pext_version != P->version;  // state gate: P_oth only when P changed
  for (auto& sp : S->parts) {
    if (sp.n == 0) continue;
    if (gather_p) {
      const int64_t np = sp.Pext->nnzb;
      if (np > 0) { k_copy_blocks<double><<<(unsigned)((np * Bp + 255) / 256), 256, 0, st>>>(np, Bp, sp.p_src, P->slot_of, P->vals, sp.Pext->slot_of, sp.Pext->vals); BAMG_COUNT_LAUNCH; }
      sp.Pext->version++;
    }
    BAMG_TRY(ptap_run(sp.plan, sp.Aext, sp.Pext, sp.C, BAMG_FP64, true));
  }
  if (gather_p) {
    S->pext_version = P->version;
    S->poth_gathers++;
  }
  if (S->nac > 0) { k_reduce_blocks<<<(unsigned)((S->nac * Bc + 255) / 256), 256, 0, st>>>(S->nac, Bc, S->r_off, S->r_part, S->r_slot, S->r_vals, Ac->slot_of, Ac->vals); BAMG_COUNT_LAUNCH; }
  Ac->version++;
  Ac->vals64_stale = false;
  BAMG_CUDA(cudaGetLastError());
  return Status{};
}

}  // namespace bamg

using namespace bamg;

extern "C" {

bamg_status bamg_halo_create(int64_t nbr, const int32_t* rowptr, const int32_t* colidx, int nparts,
                             const int64_t* row_starts, bamg_halo** out) {
  if (!out || nbr < 0 || (nbr > 0 && (!rowptr || !colidx))) return BAMG_ERR_INVALID;
  *out = nullptr;
  bamg_halo* H = new (std::nothrow) bamg_halo();
  if (!H) return BAMG_ERR_OOM;
  Status s = halo_build(nbr, rowptr, colidx, nparts, row_starts, H);
  if (!s.ok()) {
    delete H;
    return s.code;
  }
  *out = H;
  return BAMG_OK;
}

bamg_status bamg_halo_destroy(bamg_halo* H) {
  delete H;
  return BAMG_OK;
}

bamg_status bamg_halo_part_info(const bamg_halo* H, int p, int64_t* n_owned, int64_t* n_ghost, int64_t* nnzb) {
  if (!H || p < 0 || p >= H->nparts) return BAMG_ERR_INVALID;
  const auto& P = H->parts[p];
  if (n_owned) *n_owned = P.n;
  if (n_ghost) *n_ghost = (int64_t)P.ghost.size();
  if (nnzb) *nnzb = (int64_t)P.col.size();
  return BAMG_OK;
}

bamg_status bamg_halo_part_pattern(const bamg_halo* H, int p, int32_t* rowptr, int32_t* colidx, int64_t* block_src) {
  if (!H || p < 0 || p >= H->nparts) return BAMG_ERR_INVALID;
  const auto& P = H->parts[p];
  if (rowptr) std::copy(P.rowptr.begin(), P.rowptr.end(), rowptr);
  if (colidx) std::copy(P.col.begin(), P.col.end(), colidx);
  if (block_src) std::copy(P.src.begin(), P.src.end(), block_src);
  return BAMG_OK;
}

bamg_status bamg_halo_part_ghosts(const bamg_halo* H, int p, int64_t* ghost, int32_t* owner) {
  if (!H || p < 0 || p >= H->nparts) return BAMG_ERR_INVALID;
  const auto& P = H->parts[p];
  if (ghost) std::copy(P.ghost.begin(), P.ghost.end(), ghost);
  if (owner) std::copy(P.owner.begin(), P.owner.end(), owner);
  return BAMG_OK;
}

bamg_status bamg_halo_sends(const bamg_halo* H, int from, int to, int64_t* count, int64_t* local_rows) {
  if (!H || from < 0 || to < 0 || from >= H->nparts || to >= H->nparts) return BAMG_ERR_INVALID;
  const auto& v = H->sends[(size_t)from * H->nparts + to];
  if (count) *count = (int64_t)v.size();
  if (local_rows) std::copy(v.begin(), v.end(), local_rows);
  return BAMG_OK;
}

bamg_status bamg_sharded_create(bamg_bsr* A, bamg_bsr* P, int nparts, const int64_t* row_starts,
                                bamg_sharded** out, bamg_bsr** Ac) {
  if (!A || !P || !out || !Ac) return BAMG_ERR_INVALID;
  *out = nullptr;
  *Ac = nullptr;
  bamg_sharded* S = new (std::nothrow) bamg_sharded();
  if (!S) return BAMG_ERR_OOM;
  S->ctx = A->ctx;
  Status s = sharded_build(S, A, P, nparts, row_starts, Ac);
  if (!s.ok()) {
    if (*Ac) bamg_bsr_destroy(*Ac);
    *Ac = nullptr;
    sharded_release(S);
    delete S;
    return fail(A->ctx, s);
  }
  *out = S;
  return BAMG_OK;
}

bamg_status bamg_sharded_spmv(bamg_sharded* S, const double* x, double* y) {
  if (!S || !x || !y) return BAMG_ERR_INVALID;
  Status s = sharded_spmv(S, x, y);
  return s.ok() ? BAMG_OK : fail(S->ctx, s);
}

bamg_status bamg_sharded_ptap(bamg_sharded* S, bamg_bsr* A, bamg_bsr* P, bamg_bsr* Ac) {
  if (!S || !A || !P || !Ac) return BAMG_ERR_INVALID;
  Status s = sharded_ptap(S, A, P, Ac);
  return s.ok() ? BAMG_OK : fail(S->ctx, s);
}

bamg_status bamg_sharded_stats(const bamg_sharded* S, bamg_shard_stats* o) {
  if (!S || !o) return BAMG_ERR_INVALID;
  *o = bamg_shard_stats{};
  const int bs = S->A->br, bsp = S->P->bc;
  for (const auto& sp : S->parts) {
    o->ghost_rows += sp.g;
    o->poth_blocks += sp.poth_blocks;
    o->reduce_blocks += sp.reduce_blocks;
    o->max_owned_rows = std::max<int64_t>(o->max_owned_rows, sp.n);
  }
  o->halo_bytes_per_spmv = o->ghost_rows * bs * 8;
  o->poth_bytes = o->poth_blocks * (bs * bsp * 8 + 4);
  o->reduce_bytes_per_ptap = o->reduce_blocks * (bsp * bsp * 8 + 4);
  o->poth_gathers = (int64_t)S->poth_gathers;
  return BAMG_OK;
}

bamg_status bamg_sharded_destroy(bamg_sharded* S) {
  if (!S) return BAMG_OK;
  sharded_release(S);
  delete S;
  return BAMG_OK;
}

}  // extern "C"
