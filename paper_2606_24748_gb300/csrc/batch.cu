// A batch of independent problems (each with its own hierarchy) solved by
// PCG in one graph launch.
//
// The graph holds, for every problem, the prologue of its solve (r = b,
// z = M r, p = z), then one while-loop node whose body is one CG iteration of
// every problem, then the epilogue (x and the true residual).  Inside the
// body each problem's iteration sits in a conditional IF node whose
// condition a one-thread kernel sets from the problem's own state, so a
// problem that has converged launches nothing for the rest of the loop.  A one-warp
// kernel at the end of the prologue and of each loop body decides on the
// device whether another iteration is needed (some problem is still running)
// and sets the loop's condition, so the whole batch runs without a host round
// trip; a loop counter bounds the loop at maxit iterations whatever the
// problems' states.  Problems are dealt largest-first to a number of
// concurrent branches (streams at capture time); the count is a schedule
// choice that bamg_batch_autotune makes by timing.  Each problem runs exactly
// the kernels of bamg_cg_solve with its own context's reduction buffers, so
// its result is that of a standalone solve.
#include <algorithm>
#include <numeric>

#include "device.cuh"
#include "internal.h"

using namespace bamg;

struct bamg_batch {
  bamg_ctx* ctx = nullptr;
  std::vector<bamg_mg*> mgs;
  std::vector<std::vector<int>> branches;  // problems per concurrent branch
  std::vector<cudaStream_t> streams;
  cudaStream_t origin = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const double*> gb;
  std::vector<double*> gx;
  double grtol = -1.0;
  int gmaxit = -1;
  uint64_t outer_kernels = 0, body_kernels = 0;
  std::vector<uint64_t> step_kernels;       // kernels of one CG iteration of each problem
  std::vector<cudaStream_t> inner;          // capture streams of the IF bodies, one per branch
  CgState** d_states = nullptr;
  CgState* d_gather = nullptr;
  int* d_loops = nullptr;
  double* d_true = nullptr;
  CgState* h_states = nullptr;  // pinned
  double* h_true = nullptr;     // pinned
  int* h_loops = nullptr;       // pinned
};

namespace bamg {
namespace {

// Sets the loop condition: 1 while some problem is still iterating and the
// loop has run fewer than max_loops bodies.  reset = 1 at the end of the
// prologue (loop counter to 0).
__global__ void k_batch_continue(CgState* const* states, int n, int* loops, int max_loops, int reset,
                                 cudaGraphConditionalHandle h) {
  int active = 0;
  for (int p = threadIdx.x; p < n; p += 32) active |= states[p]->done ? 0 : 1;
  active = __any_sync(0xffffffffu, active);
  if (threadIdx.x == 0) {
    const int l = reset ? 0 : *loops + 1;
    *loops = l;
    cudaGraphSetConditional(h, (active && l < max_loops) ? 1u : 0u);
  }
}

// Condition of a problem's IF node in the loop body: still iterating.
__global__ void k_batch_if(const CgState* s, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, s->done ? 0u : 1u);
}

__global__ void k_batch_gather(CgState* const* states, int n, CgState* out) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) out[p] = *states[p];
}

int64_t fine_dofs(const bamg_mg* mg) { return mg->levels[0].n * 3; }

// Largest problem first, each to the branch with the fewest dofs so far.
void deal(bamg_batch* bt, int n_branches) {
  const int n = (int)bt->mgs.size();
  n_branches = std::max(1, std::min(n_branches, n));
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return fine_dofs(bt->mgs[a]) > fine_dofs(bt->mgs[b]); });
  bt->branches.assign(n_branches, {});
  std::vector<int64_t> load(n_branches, 0);
  for (int p : order) {
    const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    bt->branches[s].push_back(p);
    load[s] += fine_dofs(bt->mgs[p]);
  }
}

template <class F>
Status fork_join(bamg_batch* bt, std::vector<cudaEvent_t>& events, F per_problem) {
  cudaEvent_t fork = nullptr;
  BAMG_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  events.push_back(fork);
  BAMG_CUDA(cudaEventRecord(fork, bt->origin));
  for (size_t s = 0; s < bt->branches.size(); ++s) {
    cudaStream_t st = bt->streams[s];
    BAMG_CUDA(cudaStreamWaitEvent(st, fork, 0));
    for (int p : bt->branches[s]) BAMG_TRY(per_problem(p, st));
    cudaEvent_t join = nullptr;
    BAMG_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    events.push_back(join);
    BAMG_CUDA(cudaEventRecord(join, st));
    BAMG_CUDA(cudaStreamWaitEvent(bt->origin, join, 0));
  }
  return Status{};
}

uint64_t kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  uint64_t k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

void release_exec(bamg_batch* bt) {
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  bt->exec = nullptr;
  bt->gb.clear();
  bt->gx.clear();
}

// Ends a capture that failed part-way, so the streams leave capture mode.
void abandon_capture(cudaStream_t st) {
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(st, &g);
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();
}

Status build(bamg_batch* bt, const double* const* b, double* const* x, double rtol, int maxit) {
  release_exec(bt);
  const int n = (int)bt->mgs.size();
  cudaGraph_t G = nullptr;
  BAMG_CUDA(cudaGraphCreate(&G, 0));
  std::vector<cudaEvent_t> events;
  Status s;
  cudaGraphConditionalHandle h;
  cudaGraph_t body = nullptr;
  cudaGraphNode_t cond = nullptr;
  const auto mode = cudaStreamCaptureModeThreadLocal;
  auto run = [&]() -> Status {
    BAMG_CUDA(cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault));
    // prologue of every problem, then the first loop decision
    BAMG_CUDA(cudaStreamBeginCaptureToGraph(bt->origin, G, nullptr, nullptr, 0, mode));
    g_capturing = true;
    BAMG_TRY(fork_join(bt, events, [&](int p, cudaStream_t st) { return cg_prologue(bt->mgs[p], b[p], rtol, maxit, st); }));
    k_batch_continue<<<1, 32, 0, bt->origin>>>(bt->d_states, n, bt->d_loops, maxit, 1, h);
    BAMG_CUDA(cudaGetLastError());
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    BAMG_CUDA(cudaStreamGetCaptureInfo(bt->origin, &cst, nullptr, nullptr, &deps, nullptr, &nd));
    std::vector<cudaGraphNode_t> last(deps, deps + nd);
    cudaGraph_t out = nullptr;
    BAMG_CUDA(cudaStreamEndCapture(bt->origin, &out));
    // the loop
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    BAMG_CUDA(cudaGraphAddNode(&cond, G, last.data(), nullptr, last.size(), &cp));
    body = cp.conditional.phGraph_out[0];
    std::vector<cudaGraphConditionalHandle> hp(n);
    for (int p = 0; p < n; ++p) BAMG_CUDA(cudaGraphConditionalHandleCreate(&hp[p], body, 0, 0));
    bt->step_kernels.assign(n, 0);
    BAMG_CUDA(cudaStreamBeginCaptureToGraph(bt->origin, body, nullptr, nullptr, 0, mode));
    BAMG_TRY(fork_join(bt, events, [&](int p, cudaStream_t st) -> Status {
      // condition kernel, then an IF node after it on this branch, whose
      // body is the problem's iteration captured on the branch's inner stream
      k_batch_if<<<1, 1, 0, st>>>(bt->mgs[p]->cg, hp[p]);
      BAMG_CUDA(cudaGetLastError());
      cudaStreamCaptureStatus bst;
      cudaGraph_t bg = nullptr;
      const cudaGraphNode_t* bdeps = nullptr;
      size_t bnd = 0;
      BAMG_CUDA(cudaStreamGetCaptureInfo(st, &bst, nullptr, &bg, &bdeps, nullptr, &bnd));
      cudaGraphNodeParams ip = {};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = hp[p];
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t ifn = nullptr;
      BAMG_CUDA(cudaGraphAddNode(&ifn, bg, bdeps, nullptr, bnd, &ip));
      BAMG_CUDA(cudaStreamUpdateCaptureDependencies(st, &ifn, nullptr, 1, cudaStreamSetCaptureDependencies));
      cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
      size_t bi = 0;
      while (bi < bt->streams.size() && bt->streams[bi] != st) ++bi;
      cudaStream_t in = bt->inner[bi];
      BAMG_CUDA(cudaStreamBeginCaptureToGraph(in, ifbody, nullptr, nullptr, 0, mode));
      Status cs = cg_step(bt->mgs[p], in);
      cudaGraph_t done_g = nullptr;
      cudaError_t ee = cudaStreamEndCapture(in, &done_g);
      BAMG_TRY(cs);
      if (ee != cudaSuccess) return cuda_status(ee, "IF body capture");
      bt->step_kernels[p] = kernel_nodes(ifbody);
      return Status{};
    }));
    k_batch_continue<<<1, 32, 0, bt->origin>>>(bt->d_states, n, bt->d_loops, maxit, 0, h);
    BAMG_CUDA(cudaGetLastError());
    BAMG_CUDA(cudaStreamEndCapture(bt->origin, &out));
    // epilogue
    BAMG_CUDA(cudaStreamBeginCaptureToGraph(bt->origin, G, &cond, nullptr, 1, mode));
    BAMG_TRY(fork_join(bt, events, [&](int p, cudaStream_t st) {
      return cg_epilogue(bt->mgs[p], b[p], x ? x[p] : nullptr, bt->d_true + p, st);
    }));
    BAMG_CUDA(cudaStreamEndCapture(bt->origin, &out));
    return Status{};
  };
  s = run();
  g_capturing = false;
  if (!s.ok()) abandon_capture(bt->origin);
  if (s.ok()) {
    bt->outer_kernels = kernel_nodes(G);
    bt->body_kernels = kernel_nodes(body);
    cudaError_t e = cudaGraphInstantiate(&bt->exec, G, 0);
    if (e != cudaSuccess) s = cuda_status(e, "batch graph instantiate");
  }
  cudaGraphDestroy(G);
  for (auto ev : events) cudaEventDestroy(ev);
  if (!s.ok()) {
    release_exec(bt);
    return s;
  }
  bt->gb.assign(b, b + n);
  bt->gx.assign(n, nullptr);
  if (x) bt->gx.assign(x, x + n);
  bt->grtol = rtol;
  bt->gmaxit = maxit;
  return Status{};
}

bool same_call(const bamg_batch* bt, const double* const* b, double* const* x, double rtol, int maxit) {
  if (!bt->exec || bt->grtol != rtol || bt->gmaxit != maxit) return false;
  for (size_t p = 0; p < bt->mgs.size(); ++p)
    if (bt->gb[p] != b[p] || bt->gx[p] != (x ? x[p] : nullptr)) return false;
  return true;
}

Status solve(bamg_batch* bt, const double* const* b, double* const* x, double rtol, int maxit, bamg_cg_info* info,
             int* loops_out) {
  const int n = (int)bt->mgs.size();
  for (int p = 0; p < n; ++p)
    if (!b[p]) return make_status(BAMG_ERR_INVALID, "right-hand side %d is null", p);
  if (!same_call(bt, b, x, rtol, maxit)) BAMG_TRY(build(bt, b, x, rtol, maxit));
  cudaStream_t st = bt->ctx->stream;
  BAMG_CUDA(cudaGraphLaunch(bt->exec, st));
  { k_batch_gather<<<1, 128, 0, st>>>(bt->d_states, n, bt->d_gather); BAMG_COUNT_LAUNCH; }
  BAMG_CUDA(cudaMemcpyAsync(bt->h_states, bt->d_gather, sizeof(CgState) * n, cudaMemcpyDeviceToHost, st));
  BAMG_CUDA(cudaMemcpyAsync(bt->h_true, bt->d_true, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  BAMG_CUDA(cudaMemcpyAsync(bt->h_loops, bt->d_loops, sizeof(int), cudaMemcpyDeviceToHost, st));
  BAMG_CUDA(cudaStreamSynchronize(st));
  // top-level kernels of the body ran once per loop; each problem's
  // iteration kernels only in the iterations it was still running
  uint64_t launched = bt->outer_kernels + bt->body_kernels * (uint64_t)*bt->h_loops;
  for (int p = 0; p < n; ++p) launched += bt->step_kernels[p] * (uint64_t)bt->h_states[p].its;
  g_launches.fetch_add(launched, std::memory_order_relaxed);
  for (bamg_mg* mg : bt->mgs) BAMG_TRY(check_device_error(mg->ctx));
  if (loops_out) *loops_out = *bt->h_loops;
  int broke = -1, not_conv = -1;
  for (int p = 0; p < n; ++p) {
    const CgState& h = bt->h_states[p];
    if (info) {
      info[p].iterations = h.its;
      info[p].converged = h.converged;
      info[p].rnorm = sqrt(h.rnorm2);
      info[p].bnorm = sqrt(h.bnorm2);
      info[p].true_rnorm = sqrt(bt->h_true[p]);
    }
    if (h.breakdown && broke < 0) broke = p;
    if (!h.converged && not_conv < 0) not_conv = p;
  }
  if (broke >= 0) return make_status(BAMG_ERR_BREAKDOWN, "CG breakdown in problem %d", broke);
  if (not_conv >= 0)
    return make_status(BAMG_ERR_NOT_CONVERGED, "problem %d did not converge in %d iterations", not_conv,
                       bt->h_states[not_conv].its);
  return Status{};
}

Status set_branches(bamg_batch* bt, int n_branches) {
  deal(bt, n_branches);
  while (bt->streams.size() < bt->branches.size()) {
    cudaStream_t s = nullptr, s2 = nullptr;
    BAMG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    bt->streams.push_back(s);
    BAMG_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    bt->inner.push_back(s2);
  }
  release_exec(bt);
  return Status{};
}

void destroy(bamg_batch* bt) {
  release_exec(bt);
  cudaStream_t st = bt->ctx->stream;
  cudaStreamSynchronize(st);
  for (auto s : bt->streams) cudaStreamDestroy(s);
  for (auto s : bt->inner) cudaStreamDestroy(s);
  if (bt->origin) cudaStreamDestroy(bt->origin);
  dfree(bt->d_states, st);
  dfree(bt->d_gather, st);
  dfree(bt->d_loops, st);
  dfree(bt->d_true, st);
  if (bt->h_states) cudaFreeHost(bt->h_states);
  if (bt->h_true) cudaFreeHost(bt->h_true);
  if (bt->h_loops) cudaFreeHost(bt->h_loops);
  cudaStreamSynchronize(st);
}

Status create(bamg_ctx* ctx, int n, bamg_mg* const* mgs, bamg_batch* bt) {
  bt->ctx = ctx;
  bt->mgs.assign(mgs, mgs + n);
  for (int p = 0; p < n; ++p) {
    bamg_mg* mg = mgs[p];
    if (!mg) return make_status(BAMG_ERR_INVALID, "hierarchy %d is null", p);
    if (mg->levels.empty() || mg->levels[0].bs != 3 || !mg->coarse.factored)
      return make_status(BAMG_ERR_STATE, "hierarchy %d is not set up", p);
    for (int q = 0; q < p; ++q)
      if (mgs[q] == mg || mgs[q]->ctx == mg->ctx)
        return make_status(BAMG_ERR_INVALID, "hierarchies %d and %d share a context (each needs its own)", q, p);
  }
  cudaStream_t st = ctx->stream;
  std::vector<CgState*> states(n);
  for (int p = 0; p < n; ++p) states[p] = mgs[p]->cg;
  BAMG_TRY(upload(&bt->d_states, states, st));
  BAMG_TRY(dalloc(&bt->d_gather, n, st));
  BAMG_TRY(dalloc(&bt->d_loops, 1, st));
  BAMG_TRY(dalloc(&bt->d_true, n, st));
  BAMG_CUDA(cudaMemsetAsync(bt->d_loops, 0, sizeof(int), st));
  BAMG_CUDA(cudaMallocHost(&bt->h_states, sizeof(CgState) * n));
  BAMG_CUDA(cudaMallocHost(&bt->h_true, sizeof(double) * n));
  BAMG_CUDA(cudaMallocHost(&bt->h_loops, sizeof(int)));
  BAMG_CUDA(cudaStreamCreateWithFlags(&bt->origin, cudaStreamNonBlocking));
  BAMG_CUDA(cudaStreamSynchronize(st));
  return set_branches(bt, n);
}

}  // namespace
}  // namespace bamg

extern "C" {

bamg_status bamg_batch_create(bamg_ctx* ctx, int n, bamg_mg* const* mgs, bamg_batch** out) {
  if (!ctx || !mgs || !out || n < 1) return BAMG_ERR_INVALID;
  *out = nullptr;
  auto* bt = new bamg_batch();
  Status s = create(ctx, n, mgs, bt);
  if (!s.ok()) {
    destroy(bt);
    delete bt;
    return fail(ctx, s);
  }
  *out = bt;
  return BAMG_OK;
}

bamg_status bamg_batch_destroy(bamg_batch* bt) {
  if (!bt) return BAMG_OK;
  destroy(bt);
  delete bt;
  return BAMG_OK;
}

bamg_status bamg_batch_set_branches(bamg_batch* bt, int n_branches) {
  if (!bt || n_branches < 1) return BAMG_ERR_INVALID;
  Status s = set_branches(bt, n_branches);
  return s.ok() ? BAMG_OK : fail(bt->ctx, s);
}

bamg_status bamg_batch_get_branches(const bamg_batch* bt, int* n_branches) {
  if (!bt || !n_branches) return BAMG_ERR_INVALID;
  *n_branches = (int)bt->branches.size();
  return BAMG_OK;
}

bamg_status bamg_batch_cg_solve(bamg_batch* bt, const double* const* b, double* const* x, double rtol, int maxit,
                                bamg_cg_info* info, int* loops) {
  if (!bt || !b || maxit < 0 || !(rtol >= 0.0)) return BAMG_ERR_INVALID;
  Status s = solve(bt, b, x, rtol, maxit, info, loops);
  return s.ok() ? BAMG_OK : fail(bt->ctx, s);
}

bamg_status bamg_batch_autotune(bamg_batch* bt, const double* const* b, double* const* x, double rtol, int maxit,
                                float* best_ms) {
  if (!bt || !b || maxit < 0 || !(rtol >= 0.0)) return BAMG_ERR_INVALID;
  auto body = [&]() -> Status {
    const int n = (int)bt->mgs.size();
    cudaStream_t st = bt->ctx->stream;
    cudaEvent_t e0, e1;
    BAMG_CUDA(cudaEventCreate(&e0));
    BAMG_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_b = n;
    Status s;
    for (int nb = 1;; nb *= 2) {
      const int c = std::min(nb, n);
      s = set_branches(bt, c);
      if (s.ok()) s = solve(bt, b, x, rtol, maxit, nullptr, nullptr);  // builds, warms up
      if (s.code == BAMG_ERR_NOT_CONVERGED) s = Status{};
      if (!s.ok()) break;
      float t[3];
      for (int r = 0; r < 3 && s.ok(); ++r) {
        cudaEventRecord(e0, st);
        s = solve(bt, b, x, rtol, maxit, nullptr, nullptr);
        if (s.code == BAMG_ERR_NOT_CONVERGED) s = Status{};
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        if (cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess) t[r] = 1e30f;
      }
      if (!s.ok()) break;
      std::sort(t, t + 3);
      if (t[1] < best) {
        best = t[1];
        best_b = c;
      }
      if (c == n) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!s.ok()) return s;
    if (best_ms) *best_ms = best;
    return set_branches(bt, best_b);
  };
  Status s = body();
  return s.ok() ? BAMG_OK : fail(bt->ctx, s);
}

}  // extern "C"
