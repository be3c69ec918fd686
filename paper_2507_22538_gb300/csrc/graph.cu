// Algorithm 1 as one CUDA graph (mdp_solve with opts->graph set and the GMRES
// inner solver).  The stream-driven mdp_solve waits on the host for every Bellman
// residual (Algorithm 1 step 3), for the set-up of every policy evaluation and for
// the solver state after every GMRES restart cycle; on small problems these round
// trips and the launches behind them take most of the time.  Here the whole loop
// runs on the device:
//
//   init
//   WHILE (outer)                         Algorithm 1, one policy evaluation per pass
//     Bellman sweep; check                steps 2-3: TV, pi, ||TV - V||_inf; stop tests
//     IF (go)                             set by the check
//       policy rows; restart residual     step 4 and the first GMRES residual
//       WHILE (inner)                     one GMRES(m) restart cycle per pass
//         steps 0-3; IF (go 1) steps 4-7; IF (go 2) steps 8-11; ...
//         update; restart residual
//       end of the evaluation             k += 1
//
// The Arnoldi steps of a cycle come in chunks of kChunkSteps.  Chunk q > 0 runs
// under an IF with its own condition, which the control kernel after chunk q - 1
// sets while the cycle goes on; the one after chunk 0 (which always runs) first
// clears the conditions of chunks 2 and up.  The steps after a cycle's stop are
// therefore skipped instead of launched as no-ops.
// Small control kernels set the conditions (cudaGraphSetConditional) from the
// residual and the solver's device flags.  The other nodes are the kernels the
// stream-driven solve launches, with the same launch shapes, so both give the
// same iterates bit for bit.  The instantiated graph is kept in the handle and
// rebuilt only when something it bakes in changes (vectors, gamma, options,
// the Bellman launch shape).
#include <algorithm>
#include <cstring>
#include <vector>

#include "krylov_dev.cuh"

namespace mdp {

// launch sequences of krylov.cu (same kernels as the stream-driven GMRES)
mdp_status gmres_residual_launch(mdp_s* h, bool mixed, double gamma, const double* theta, cudaStream_t st);
mdp_status gmres_steps_launch(mdp_s* h, bool mixed, double gamma, int j0, int j1, int refine, cudaStream_t st);
mdp_status gmres_tail_launch(mdp_s* h, bool mixed, double gamma, double* theta, cudaStream_t st);
void gmres_count_work(mdp_s* h, bool mixed, int64_t solves, int64_t cycles, int64_t steps, int64_t tri);

// Add a captured segment to `parent` as a child-graph node after `deps` (the
// segment graph is consumed).
mdp_status graph_add_segment(cudaGraph_t parent, const cudaGraphNode_t* deps, size_t ndeps, cudaGraph_t seg,
                             cudaGraphNode_t* node) {
  const cudaError_t e = cudaGraphAddChildGraphNode(node, parent, deps, ndeps, seg);
  cudaGraphDestroy(seg);  // the node holds its own copy
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddChildGraphNode");
  return MDP_OK;
}

// Add a conditional node (IF or WHILE on handle c) to `parent` after `deps`;
// *body receives the graph of its body.
mdp_status graph_add_conditional(cudaGraph_t parent, const cudaGraphNode_t* deps, size_t ndeps,
                                 cudaGraphConditionalHandle c, cudaGraphConditionalNodeType type,
                                 cudaGraphNode_t* node, cudaGraph_t* body) {
  // zero-filled storage: the parameter union has no default constructor
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
  cudaGraphNodeParams* p = reinterpret_cast<cudaGraphNodeParams*>(raw);
  p->type = cudaGraphNodeTypeConditional;
  p->conditional.handle = c;
  p->conditional.type = type;
  p->conditional.size = 1;
  MDP_CUDA(cudaGraphAddNode(node, parent, deps, nullptr, ndeps, p));
  *body = p->conditional.phGraph_out[0];
  return MDP_OK;
}

namespace {

constexpr int kChunkSteps = 4;              // Arnoldi steps per IF-guarded chunk of a cycle
constexpr int kMaxChunks = (kMaxBasis + kChunkSteps - 1) / kChunkSteps;
constexpr int kSegments = 3 + kMaxChunks + 2;  // init, sweep, go, chunks, tail, end

// Device record of one graph-driven solve.
struct GraphSolveState {
  double res;             // ||TV - V||_inf of the last sweep
  long long inner_total;  // inner iterations of the completed evaluations
  long long solves;       // GMRES solves started
  long long cycles;       // restart cycles that ran at least one Arnoldi step
  long long steps;        // Arnoldi steps
  long long tri;          // sum over those cycles of n (n - 1) / 2, n = steps of the cycle
  int k;                  // policy evaluations completed
  int status;             // MDP_OK, MDP_NOT_CONVERGED or MDP_ERR_NUMERIC
  int converged;
  int sweeps;
  int it_prev;            // K->it after the previous restart residual
  int numeric_inner;      // a non-finite value stopped GMRES
  int passes;             // passes of the inner WHILE body in the current evaluation
  int guard;              // a loop guard ended the solve (never expected: see the control kernels)
  long long launches;     // kernels that ran: every segment's control kernel adds its segment's count
};

// The solve record and the kernels per captured segment (filled by the host after
// the graph is built; each segment ends with its control kernel).
struct GraphDevice {
  GraphSolveState G;
  int seg_kernels[kSegments];
};

__global__ void gs_init_kernel(GraphDevice* D, int seg) {
  if (threadIdx.x != 0) return;
  D->G = GraphSolveState{};
  D->G.launches = D->seg_kernels[seg];
}

// Algorithm 1 step 3 after the sweep: the stop tests in the order of mdp_solve;
// when the loop goes on, the solver state of the next GMRES solve (what
// init_state writes from the host: zeros, tol = alpha * res, the caps).
__global__ void __launch_bounds__(256) gs_outer_check_kernel(const unsigned long long* __restrict__ resmax,
                                                             GraphDevice* D, int seg, KrylovState* K, double atol,
                                                             double alpha, int max_iter_pi, int max_iter_ksp, int m,
                                                             int pstride, cudaGraphConditionalHandle c_outer,
                                                             cudaGraphConditionalHandle c_go) {
  GraphSolveState* G = &D->G;
  const double res = __longlong_as_double((long long)*resmax);
  // k grows by one per evaluation, so at most max_iter_pi + 1 sweeps run; the guard
  // on the sweep count bounds the outer loop even if that ever failed
  const bool guard = (long long)G->sweeps > (long long)max_iter_pi + 1;  // 64-bit: max_iter_pi may be INT_MAX
  const bool go = isfinite(res) && !(res <= atol) && G->k < max_iter_pi && !guard;
  if (go) {
    unsigned long long* words = reinterpret_cast<unsigned long long*>(K);
    for (size_t i = threadIdx.x; i < sizeof(KrylovState) / sizeof(unsigned long long); i += blockDim.x) words[i] = 0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  G->launches += D->seg_kernels[seg];
  G->sweeps += 1;
  G->res = res;
  if (guard)
    G->guard = 1;
  else if (!isfinite(res))
    G->status = MDP_ERR_NUMERIC;
  else if (res <= atol)
    G->converged = 1;
  else if (G->k >= max_iter_pi)
    G->status = MDP_NOT_CONVERGED;
  if (go) {
    K->tol = alpha * res;
    K->maxit = max_iter_ksp;
    K->m = m;
    K->pstride = pstride;
    G->it_prev = 0;
    G->passes = 0;
    G->solves += 1;
  }
  cudaGraphSetConditional(c_go, go ? 1u : 0u);
  if (!go) cudaGraphSetConditional(c_outer, 0u);
}

// After a restart residual: count the cycle that just ended and go on while the
// GMRES solve is not over.  Every cycle runs at least one Arnoldi step (the
// restart residual clears the cycle's stop flag) and the solve ends at max_it
// steps, so at most max_it + 1 passes run; the guard bounds the loop regardless.
__global__ void gs_inner_cond_kernel(KrylovState* K, GraphDevice* D, int seg, int in_loop, long long max_passes,
                                     cudaGraphConditionalHandle c_inner) {
  if (threadIdx.x != 0) return;
  GraphSolveState* G = &D->G;
  G->launches += D->seg_kernels[seg];
  if (in_loop && (long long)(++G->passes) > max_passes) {
    G->guard = 1;
    K->flags |= kSolveDone | kNumeric;
  }
  const long long n = K->it - G->it_prev;
  if (n > 0) {
    G->cycles += 1;
    G->steps += n;
    G->tri += n * (n - 1) / 2;
  }
  G->it_prev = K->it;
  cudaGraphSetConditional(c_inner, (K->flags & kSolveDone) ? 0u : 1u);
}

struct ChunkHandles {
  cudaGraphConditionalHandle go[kMaxChunks];  // go[q] guards chunk q (q >= 1)
};

// After chunk q of Arnoldi steps: chunk q + 1 runs only while the cycle goes on.
__global__ void gs_chunk_cond_kernel(const KrylovState* K, GraphDevice* D, int seg, ChunkHandles hs, int q,
                                     int nchunks) {
  if (threadIdx.x != 0) return;
  D->G.launches += D->seg_kernels[seg];
  if (q == 0)
    for (int i = 2; i < nchunks; ++i) cudaGraphSetConditional(hs.go[i], 0u);
  if (q + 1 < nchunks) cudaGraphSetConditional(hs.go[q + 1], (K->flags & (kCycleStop | kSolveDone)) ? 0u : 1u);
}

// End of one policy evaluation (Algorithm 1 steps 12-13): V_{k+1} = theta is
// already in V; k += 1.  A non-finite value inside GMRES ends the solve as the
// stream-driven mdp_solve does (no increment).
__global__ void gs_outer_end_kernel(const KrylovState* K, GraphDevice* D, int seg, cudaGraphConditionalHandle c_outer) {
  if (threadIdx.x != 0) return;
  GraphSolveState* G = &D->G;
  G->launches += D->seg_kernels[seg];
  if (K->flags & kNumeric) {
    G->status = MDP_ERR_NUMERIC;
    G->numeric_inner = 1;
    cudaGraphSetConditional(c_outer, 0u);
    return;
  }
  G->inner_total += K->it;
  G->k += 1;
}

// What the graph bakes in.
struct GraphKey {
  const void* V;
  const void* pi;
  const void* basis;
  const void* basis32;
  double gamma, atol, alpha;
  int max_pi, max_ksp, m, refine, precision, tile, blocks, rpl, v256, pstore, lowp, lp_ts, lp_blocks;
};

struct GraphCache {
  GraphKey key{};
  bool valid = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;  // private stream the segments are captured on
  GraphDevice* D = nullptr;
  int seg_kernels[kSegments] = {};  // host copy of the kernels per segment
};

bool same_key(const GraphKey& a, const GraphKey& b) { return std::memcmp(&a, &b, sizeof(GraphKey)) == 0; }

void drop_graph(GraphCache* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->exec = nullptr;
  c->graph = nullptr;
  c->valid = false;
}

// Capture what `f` launches on the private stream into a new graph; *kernels
// receives the number of kernels it launched.
template <typename F>
mdp_status capture(mdp_s* h, cudaStream_t cs, cudaGraph_t* out, int* kernels, F f) {
  *out = nullptr;
  const int64_t l0 = h->launches;
  MDP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const mdp_status s = f();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  *kernels = (int)(h->launches - l0);
  h->launches = l0;
  if (s != MDP_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  *out = g;
  return MDP_OK;
}

// Add the nodes of one graph-driven solve on handle h to `graph`: an init node with
// no dependencies, then the outer WHILE.  The conditional handles are made on `graph`;
// c->seg_kernels receives the kernels per segment (for the device record, uploaded
// by the caller before the launch).
mdp_status add_solve_nodes(mdp_s* h, GraphCache* c, cudaGraph_t graph, const mdp_solve_opts* o, double* V,
                           int32_t* pi, bool mixed, bool lowp) {
  cudaStream_t cs = c->cap;
  KrylovState* K = (KrylovState*)h->kstate;
  GraphDevice* D = c->D;
  const double gamma = o->gamma;
  const int m = o->gmres_restart;
  const int nchunks = (m + kChunkSteps - 1) / kChunkSteps;
  enum { kSegInit = 0, kSegSweep = 1, kSegGo = 2, kSegChunk0 = 3 };
  const int seg_tail = kSegChunk0 + nchunks, seg_end = seg_tail + 1;
  int* nk = c->seg_kernels;
  std::memset(nk, 0, sizeof(c->seg_kernels));
  cudaGraphConditionalHandle c_outer, c_go, c_inner;
  MDP_CUDA(cudaGraphConditionalHandleCreate(&c_outer, graph, 1u, cudaGraphCondAssignDefault));
  MDP_CUDA(cudaGraphConditionalHandleCreate(&c_go, graph, 0u, cudaGraphCondAssignDefault));
  MDP_CUDA(cudaGraphConditionalHandleCreate(&c_inner, graph, 0u, cudaGraphCondAssignDefault));
  ChunkHandles hs;
  std::memset(&hs, 0, sizeof(hs));
  for (int q = 1; q < nchunks; ++q)
    MDP_CUDA(cudaGraphConditionalHandleCreate(&hs.go[q], graph, 0u, cudaGraphCondAssignDefault));
  auto control_done = [&]() -> mdp_status {
    h->launches++;
    MDP_CUDA(cudaGetLastError());
    return MDP_OK;
  };

  cudaGraph_t seg = nullptr;
  cudaGraphNode_t n_init, n_outer;
  MDP_TRY(capture(h, cs, &seg, &nk[kSegInit], [&]() -> mdp_status {
    gs_init_kernel<<<1, 32, 0, cs>>>(D, kSegInit);
    return control_done();
  }));
  MDP_TRY(graph_add_segment(graph, nullptr, 0, seg, &n_init));
  cudaGraph_t outer_body = nullptr;
  MDP_TRY(graph_add_conditional(graph, &n_init, 1, c_outer, cudaGraphCondTypeWhile, &n_outer, &outer_body));

  // outer body: the sweep and the stop tests, then IF (go) the evaluation
  cudaGraphNode_t n_sweep, n_if;
  MDP_TRY(capture(h, cs, &seg, &nk[kSegSweep], [&]() -> mdp_status {
    MDP_TRY(launch_sweep(h, lowp, gamma, V, h->TV, pi, cs));
    gs_outer_check_kernel<<<1, 256, 0, cs>>>(h->resmax, D, kSegSweep, K, o->atol_pi, o->alpha, o->max_iter_pi,
                                            o->max_iter_ksp, m, h->partial_stride, c_outer, c_go);
    return control_done();
  }));
  MDP_TRY(graph_add_segment(outer_body, nullptr, 0, seg, &n_sweep));
  cudaGraph_t go_body = nullptr;
  MDP_TRY(graph_add_conditional(outer_body, &n_sweep, 1, c_go, cudaGraphCondTypeIf, &n_if, &go_body));

  // evaluation: policy rows, the first restart residual, WHILE (inner) cycles, the end
  cudaGraphNode_t n_go, n_inner, n_end;
  MDP_TRY(capture(h, cs, &seg, &nk[kSegGo], [&]() -> mdp_status {
    MDP_TRY(extract_policy(h, pi, mixed, cs));
    MDP_TRY(gmres_residual_launch(h, mixed, gamma, V, cs));
    gs_inner_cond_kernel<<<1, 32, 0, cs>>>(K, D, kSegGo, 0, (long long)o->max_iter_ksp + 1, c_inner);
    return control_done();
  }));
  MDP_TRY(graph_add_segment(go_body, nullptr, 0, seg, &n_go));
  cudaGraph_t inner_body = nullptr;
  MDP_TRY(graph_add_conditional(go_body, &n_go, 1, c_inner, cudaGraphCondTypeWhile, &n_inner, &inner_body));

  // one restart cycle: chunk 0, then chunks 1.. each under its own IF, in sequence
  cudaGraphNode_t prev = nullptr;  // the last node of the cycle so far in inner_body
  for (int q = 0; q < nchunks; ++q) {
    const int j0 = q * kChunkSteps, j1 = std::min(m, j0 + kChunkSteps);
    MDP_TRY(capture(h, cs, &seg, &nk[kSegChunk0 + q], [&]() -> mdp_status {
      MDP_TRY(gmres_steps_launch(h, mixed, gamma, j0, j1, o->gmres_refine, cs));
      gs_chunk_cond_kernel<<<1, 32, 0, cs>>>(K, D, kSegChunk0 + q, hs, q, nchunks);
      return control_done();
    }));
    if (q == 0) {
      MDP_TRY(graph_add_segment(inner_body, nullptr, 0, seg, &prev));
    } else {
      cudaGraphNode_t n_if_chunk, n_chunk;
      cudaGraph_t chunk_body = nullptr;
      const mdp_status s_if = graph_add_conditional(inner_body, &prev, 1, hs.go[q], cudaGraphCondTypeIf, &n_if_chunk,
                                              &chunk_body);
      if (s_if != MDP_OK) {
        cudaGraphDestroy(seg);
        return s_if;
      }
      MDP_TRY(graph_add_segment(chunk_body, nullptr, 0, seg, &n_chunk));
      prev = n_if_chunk;
    }
  }
  cudaGraphNode_t n_tail;
  MDP_TRY(capture(h, cs, &seg, &nk[seg_tail], [&]() -> mdp_status {
    MDP_TRY(gmres_tail_launch(h, mixed, gamma, V, cs));
    gs_inner_cond_kernel<<<1, 32, 0, cs>>>(K, D, seg_tail, 1, (long long)o->max_iter_ksp + 1, c_inner);
    return control_done();
  }));
  MDP_TRY(graph_add_segment(inner_body, &prev, 1, seg, &n_tail));
  MDP_TRY(capture(h, cs, &seg, &nk[seg_end], [&]() -> mdp_status {
    gs_outer_end_kernel<<<1, 32, 0, cs>>>(K, D, seg_end, c_outer);
    return control_done();
  }));
  MDP_TRY(graph_add_segment(go_body, &n_inner, 1, seg, &n_end));

  return MDP_OK;
}

mdp_status build_graph(mdp_s* h, GraphCache* c, const mdp_solve_opts* o, double* V, int32_t* pi, bool mixed,
                       cudaStream_t st) {
  MDP_CUDA(cudaGraphCreate(&c->graph, 0));
  MDP_TRY(add_solve_nodes(h, c, c->graph, o, V, pi, mixed, o->lowp_sweep != 0));
  MDP_CUDA(cudaGraphInstantiate(&c->exec, c->graph, 0));
  // the kernels per segment, read by the control kernels
  MDP_CUDA(cudaMemcpyAsync(c->D->seg_kernels, c->seg_kernels, sizeof(c->seg_kernels), cudaMemcpyHostToDevice, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  return MDP_OK;
}

// The handle's graph record: capture stream and device solve record, made on first use.
mdp_status graph_cache(mdp_s* h, cudaStream_t st, GraphCache** out) {
  GraphCache* c = (GraphCache*)h->gcache;
  if (!c) {
    c = new GraphCache();
    h->gcache = c;
    MDP_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  }
  if (!c->D) {
    if (cudaMallocAsync((void**)&c->D, sizeof(GraphDevice), st) != cudaSuccess) {
      cudaGetLastError();
      c->D = nullptr;
      return fail(MDP_ERR_OOM, "device allocation failed: graph solve state");
    }
  }
  *out = c;
  return MDP_OK;
}

// Fill the iteration fields of *local from a solve record; the status of the solve.
mdp_status graph_outcome(mdp_s* h, bool mixed, const GraphSolveState& g, mdp_solve_stats* local) {
  local->outer_iters = g.k;
  local->converged = g.converged;
  local->inner_iters_total = g.inner_total;
  local->final_residual = g.res;
  local->bellman_sweeps = g.sweeps;
  h->launches += g.launches;
  gmres_count_work(h, mixed, g.solves, g.cycles, g.steps, g.tri);
  if (g.guard) return fail(MDP_ERR_CUDA, "internal: a loop guard of the graph-driven solve ended it");
  if (g.status == MDP_ERR_NUMERIC)
    return fail(MDP_ERR_NUMERIC, g.numeric_inner ? "non-finite residual in GMRES" : "non-finite Bellman residual");
  if (g.status == MDP_NOT_CONVERGED)
    return fail(MDP_NOT_CONVERGED, "max_iter_pi policy evaluations without reaching atol_pi");
  return MDP_OK;
}

// Pinned host copies of the solve records of a batch; one per host thread, grown on demand.
struct PinnedRecords {
  GraphSolveState* p = nullptr;
  int cap = 0;
  ~PinnedRecords() {
    if (p) cudaFreeHost(p);
  }
  GraphSolveState* get(int n) {
    if (n <= cap) return p;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    const int want = std::max(n, 64);
    if (cudaMallocHost((void**)&p, sizeof(GraphSolveState) * want) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return nullptr;
    }
    cap = want;
    return p;
  }
};
thread_local PinnedRecords t_records;

}  // namespace

// mdp_solve_batch with every member's opts.graph set: one CUDA graph that holds each
// problem's graph-driven solve (the nodes mdp_solve's graph has) as an independent
// branch.  Every branch decides its own loops on the device, so the problems run at
// their own pace and their kernels overlap on the GPU where the launch leaves room;
// each one computes exactly what its stand-alone solve computes.  The graph is built,
// launched once and destroyed by this call.  A handle's own cached graph reads the
// device record the batch reuses, so it is dropped (and rebuilt by its next graph-
// driven mdp_solve).  Buffers are ensured by the caller; fills local[] and status[].
mdp_status graph_solve_batch(int n, mdp_s* const* hs, const mdp_solve_opts* const* os, double* const* V,
                             int32_t* const* pi, mdp_solve_stats* local, mdp_status* status, int64_t* launches,
                             cudaStream_t st) {
  std::vector<GraphCache*> cs(n, nullptr);
  for (int i = 0; i < n; ++i) {
    MDP_TRY(graph_cache(hs[i], st, &cs[i]));
    drop_graph(cs[i]);
  }
  GraphSolveState* rec = t_records.get(n);
  if (!rec) return fail(MDP_ERR_OOM, "pinned host allocation failed");
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto body = [&]() -> mdp_status {
    MDP_CUDA(cudaGraphCreate(&graph, 0));
    for (int i = 0; i < n; ++i)
      MDP_TRY(add_solve_nodes(hs[i], cs[i], graph, os[i], V[i], pi[i], os[i]->precision == MDP_PREC_MIXED, false));
    MDP_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    for (int i = 0; i < n; ++i)
      MDP_CUDA(cudaMemcpyAsync(cs[i]->D->seg_kernels, cs[i]->seg_kernels, sizeof(cs[i]->seg_kernels),
                               cudaMemcpyHostToDevice, st));
    MDP_CUDA(cudaGraphLaunch(exec, st));
    for (int i = 0; i < n; ++i)
      MDP_CUDA(cudaMemcpyAsync(rec + i, &cs[i]->D->G, sizeof(GraphSolveState), cudaMemcpyDeviceToHost, st));
    MDP_CUDA(cudaStreamSynchronize(st));
    return MDP_OK;
  };
  const mdp_status s = body();
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (s != MDP_OK) return s;
  int64_t total = 0;
  bool guard = false;
  for (int i = 0; i < n; ++i) {
    const mdp_status si = graph_outcome(hs[i], os[i]->precision == MDP_PREC_MIXED, rec[i], local + i);
    guard = guard || rec[i].guard;
    status[i] = (si == MDP_OK || si == MDP_NOT_CONVERGED || si == MDP_ERR_NUMERIC) ? si : MDP_OK;
    total += rec[i].launches;
  }
  *launches = total;
  if (guard) return fail(MDP_ERR_CUDA, "internal: a loop guard of the graph-driven batch ended it");
  return MDP_OK;
}

void graph_cache_free(mdp_s* h) {
  GraphCache* c = (GraphCache*)h->gcache;
  if (!c) return;
  drop_graph(c);
  if (c->D) cudaFreeAsync(c->D, 0);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
  h->gcache = nullptr;
}

// mdp_solve with the GMRES inner solver as one graph launch (arguments checked by
// mdp_solve; stream already bound).  Fills *local like the stream-driven loop.
mdp_status graph_solve(mdp_s* h, const mdp_solve_opts* o, double* V, int32_t* pi, mdp_solve_stats* local,
                       cudaStream_t st) {
  const bool mixed = (o->precision == MDP_PREC_MIXED);
  MDP_TRY(mixed ? ensure_mixed(h, o->gmres_restart + 1) : ensure_basis(h, o->gmres_restart + 1));
  GraphCache* c = nullptr;
  MDP_TRY(graph_cache(h, st, &c));
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  key.V = V;
  key.pi = pi;
  key.basis = mixed ? nullptr : (const void*)h->basis;
  key.basis32 = mixed ? (const void*)h->basis32 : nullptr;
  key.gamma = o->gamma;
  key.atol = o->atol_pi;
  key.alpha = o->alpha;
  key.max_pi = o->max_iter_pi;
  key.max_ksp = o->max_iter_ksp;
  key.m = o->gmres_restart;
  key.refine = o->gmres_refine;
  key.precision = o->precision;
  key.tile = h->bell_tile_states;
  key.blocks = h->bell_blocks;
  key.rpl = h->bell_rpl;
  key.v256 = h->bell_v256;
  key.pstore = h->pstore;
  key.lowp = (o->lowp_sweep && lowp_available(h)) ? 1 : 0;
  key.lp_ts = h->lp_ts;
  key.lp_blocks = h->lp_blocks;
  if (!c->valid || !same_key(c->key, key)) {
    drop_graph(c);
    const mdp_status s = build_graph(h, c, o, V, pi, mixed, st);
    if (s != MDP_OK) {
      drop_graph(c);
      return s;
    }
    c->key = key;
    c->valid = true;
  }
  double* pin = tls_pinned();
  if (!pin) return fail(MDP_ERR_OOM, "pinned host allocation failed");
  MDP_CUDA(cudaGraphLaunch(c->exec, st));
  GraphSolveState* out = reinterpret_cast<GraphSolveState*>(pin + 8);
  static_assert(sizeof(GraphSolveState) <= 48 * sizeof(double), "pinned scratch");
  MDP_CUDA(cudaMemcpyAsync(out, &c->D->G, sizeof(GraphSolveState), cudaMemcpyDeviceToHost, st));
  MDP_CUDA(cudaEventRecord(h->done, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  return graph_outcome(h, mixed, *out, local);
}

}  // namespace mdp
