// Batched inexact policy iteration: Algorithm 1 on many independent MDPs of
// different S, A, k and gamma, advanced in lockstep so that every kernel launch
// covers all problems still running.
//
// Each launch carries a table of per-problem descriptors and, per pass, the
// prefix sums of the problems' block counts: block b finds its problem by binary
// search and runs the single-problem body (bellman_dev.cuh, layout_dev.cuh,
// krylov_dev.cuh) as block b - start of nb = count blocks.  A problem gets the
// same block count as in its stand-alone launch, so its grid reductions add the
// same partial sums in the same order: every problem's iterates, policy, inner
// iteration counts and status are bit for bit those of mdp_solve on it alone.
//
// Host round trips: one residual read per outer iteration (all problems at
// once) and one header read per GMRES cycle (all problems at once), instead of
// one per problem.  Problems that stop (converged, capped, failed) leave the
// tables at the next outer iteration; inside a cycle, problems whose cycle or
// solve ended return at once from the passes queued after.
//
// With opts.graph set on every member the batch runs instead as one CUDA graph
// whose independent branches are the members' graph-driven solves (graph.cu):
// no host round trip until all have stopped, each problem at its own pace.  A
// lockstep graph (all problems in every node, stopped ones returning at once)
// measured slower on uneven mid-size batches: the longest solve then drags every
// other problem's empty blocks through each of its launches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "bellman_dev.cuh"
#include "krylov_dev.cuh"
#include "layout_dev.cuh"

namespace mdp {

struct BatchProblem {
  // stacked matrix (sliced) and costs
  const double* sval;
  const int32_t* scol;
  const int64_t* soff;
  const int32_t* slen;
  const double* g;
  // policy rows (per-state sliced) and g_pi
  double* pval;
  int32_t* pcol;
  const int64_t* poff;
  int32_t* plen;
  double* gpi;
  // iterate, greedy step output, Krylov workspace
  double* V;
  double* TV;
  int32_t* pi;
  double* basis;
  double* w;
  double* partials;
  unsigned long long* resmax;
  KrylovState* K;
  // binary32 cycle of the mixed solver (null for FP64 problems)
  float* basis32;
  float* w32;
  float* pval32;      // binary32 policy values (pstore == kStoreF32)
  uint16_t* pval16;   // binary16 / bfloat16 policy values (otherwise)
  int64_t S;
  double gamma;
  double tol;  // inner stop: alpha * ||r(V_k)||_inf
  int32_t A, skmax, suniform, pkmax, puniform, tile_states, pstride, maxit, m, mixed, pstore, pad;
};

struct BatchReport {
  double res;   // Bellman residual bits as a double, or the last GMRES residual 2-norm
  int32_t it;   // GMRES iterations
  int32_t flags;
};

// The pass kinds with their own block ranges.  FP64 passes give mixed problems no
// blocks and the binary32 passes (suffix F) give FP64 problems none.
enum : int { kRangeBellman = 0, kRangeExtract, kRangeResidual, kRangeUpdate, kRangeDots0,
             kRangeProject0 = kRangeDots0 + 8, kRangeResidualF = kRangeProject0 + 8, kRangeMatvecF, kRangeUpdateF,
             kRangeDotsF0, kRangeProjectF0 = kRangeDotsF0 + 8, kRanges = kRangeProjectF0 + 8 };

// Largest i with start[i] <= b: the problem whose range holds block b (problems
// with an empty range share their start with the next one and are skipped).
__device__ __forceinline__ int find_problem(const int32_t* __restrict__ start, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

#define BATCH_PROLOGUE                                      \
  const int i = find_problem(start, n, (int)blockIdx.x);    \
  const int bid = (int)blockIdx.x - __ldg(start + i);       \
  const int nb = __ldg(start + i + 1) - __ldg(start + i);   \
  const BatchProblem& p = P[i];

__global__ void __launch_bounds__(kBellThreads, kBellMinBlocks) bb_bellman_kernel(const BatchProblem* __restrict__ P,
                                                                   const int32_t* __restrict__ start, int n) {
  BATCH_PROLOGUE
  if (p.suniform)
    bellman_body<true>(bid, nb, p.sval, p.scol, p.soff, p.slen, p.skmax, p.g, p.V, p.S, p.A, p.tile_states, p.gamma,
                       p.TV, p.pi, p.resmax);
  else
    bellman_body<false>(bid, nb, p.sval, p.scol, p.soff, p.slen, 0, p.g, p.V, p.S, p.A, p.tile_states, p.gamma, p.TV,
                        p.pi, p.resmax);
}

__global__ void bb_extract_kernel(const BatchProblem* __restrict__ P, const int32_t* __restrict__ start, int n) {
  BATCH_PROLOGUE
  if (p.suniform)
    extract_policy_body<true>(bid, nb, p.sval, p.scol, p.soff, p.slen, p.skmax, p.g, p.pi, p.S, p.A, p.pval, p.pcol,
                              p.poff, p.plen, p.gpi, p.pval32, p.pval16, p.pstore, nullptr, nullptr);
  else
    extract_policy_body<false>(bid, nb, p.sval, p.scol, p.soff, p.slen, p.skmax, p.g, p.pi, p.S, p.A, p.pval, p.pcol,
                               p.poff, p.plen, p.gpi, p.pval32, p.pval16, p.pstore, nullptr, nullptr);
}

__global__ void __launch_bounds__(kVecThreads) bb_residual_kernel(const BatchProblem* __restrict__ P,
                                                                   const int32_t* __restrict__ start, int n) {
  BATCH_PROLOGUE
  if (p.puniform)
    gm_residual_body<true, double>(bid, nb, p.pval, p.pcol, p.poff, p.plen, p.pkmax, p.S, p.gamma, p.V, p.gpi, p.basis,
                                   p.partials, p.K);
  else
    gm_residual_body<false, double>(bid, nb, p.pval, p.pcol, p.poff, p.plen, 0, p.S, p.gamma, p.V, p.gpi, p.basis,
                                    p.partials, p.K);
}

// The binary64 mat-vec fused with the Gram-Schmidt dots, as the single-problem solver runs it.
template <int NB>
__global__ void __launch_bounds__(kVecThreads, mvd_min_blocks(NB)) bb_matvec_dots_kernel(const BatchProblem* __restrict__ P,
                                                                       const int32_t* __restrict__ start, int n,
                                                                       int j) {
  BATCH_PROLOGUE
  if (p.puniform)
    gm_matvec_dots_body<true, NB>(bid, nb, p.pval, p.pcol, p.poff, p.plen, p.pkmax, p.S, p.gamma, p.basis, j, p.w,
                                  p.partials, p.K);
  else
    gm_matvec_dots_body<false, NB>(bid, nb, p.pval, p.pcol, p.poff, p.plen, 0, p.S, p.gamma, p.basis, j, p.w,
                                   p.partials, p.K);
}

template <int NB>
__global__ void __launch_bounds__(kVecThreads, kProjectMinBlocks) bb_project_kernel(const BatchProblem* __restrict__ P,
                                                                  const int32_t* __restrict__ start, int n, int j) {
  BATCH_PROLOGUE
  gm_project_body<NB, kPlain, double, true>(bid, nb, p.S, p.basis, j, p.w, p.partials, p.K);
}

__global__ void __launch_bounds__(kVecThreads) bb_update_kernel(const BatchProblem* __restrict__ P,
                                                                 const int32_t* __restrict__ start, int n) {
  BATCH_PROLOGUE
  gm_update_body<double>(bid, nb, p.S, p.basis, p.V, p.K);
}

static_assert(sizeof(KrylovState) % 8 == 0, "the batched init zeroes the solver state in 8-byte words");

// The binary32 cycle of the mixed solver: FP64 restart residual into a binary32
// basis, mat-vec on the narrow policy values, binary32 Gram-Schmidt, update of
// the FP64 iterate.
__global__ void __launch_bounds__(kVecThreads) bb_residual_f_kernel(const BatchProblem* __restrict__ P,
                                                                     const int32_t* __restrict__ start, int n) {
  BATCH_PROLOGUE
  if (p.puniform)
    gm_residual_body<true, float>(bid, nb, p.pval, p.pcol, p.poff, p.plen, p.pkmax, p.S, p.gamma, p.V, p.gpi,
                                  p.basis32, p.partials, p.K);
  else
    gm_residual_body<false, float>(bid, nb, p.pval, p.pcol, p.poff, p.plen, 0, p.S, p.gamma, p.V, p.gpi, p.basis32,
                                   p.partials, p.K);
}

template <bool U>
__device__ __forceinline__ void matvec_f(int bid, int nb, const BatchProblem& p, int j) {
  const int k = U ? p.pkmax : 0;
  if (p.pstore == kStoreF16)
    gm_matvec_body<U, __half, float>(bid, nb, (const __half*)p.pval16, p.pcol, p.poff, p.plen, k, p.S, p.gamma,
                                     p.basis32, j, p.w32, p.K);
  else if (p.pstore == kStoreBF16)
    gm_matvec_body<U, __nv_bfloat16, float>(bid, nb, (const __nv_bfloat16*)p.pval16, p.pcol, p.poff, p.plen, k, p.S,
                                            p.gamma, p.basis32, j, p.w32, p.K);
  else
    gm_matvec_body<U, float, float>(bid, nb, p.pval32, p.pcol, p.poff, p.plen, k, p.S, p.gamma, p.basis32, j, p.w32,
                                    p.K);
}

__global__ void __launch_bounds__(kVecThreads) bb_matvec_f_kernel(const BatchProblem* __restrict__ P,
                                                                   const int32_t* __restrict__ start, int n, int j) {
  BATCH_PROLOGUE
  if (p.puniform)
    matvec_f<true>(bid, nb, p, j);
  else
    matvec_f<false>(bid, nb, p, j);
}

template <int NB>
__global__ void __launch_bounds__(kVecThreads) bb_dots_f_kernel(const BatchProblem* __restrict__ P,
                                                                 const int32_t* __restrict__ start, int n, int j) {
  BATCH_PROLOGUE
  gm_dots_body<NB, float, true>(bid, nb, p.S, p.basis32, j, p.w32, p.partials, p.K);
}

template <int NB>
__global__ void __launch_bounds__(kVecThreads, kProjectMinBlocks) bb_project_f_kernel(const BatchProblem* __restrict__ P,
                                                                    const int32_t* __restrict__ start, int n, int j) {
  BATCH_PROLOGUE
  gm_project_body<NB, kPlain, float, true>(bid, nb, p.S, p.basis32, j, p.w32, p.partials, p.K);
}

__global__ void __launch_bounds__(kVecThreads) bb_update_f_kernel(const BatchProblem* __restrict__ P,
                                                                   const int32_t* __restrict__ start, int n) {
  BATCH_PROLOGUE
  gm_update_body<float>(bid, nb, p.S, p.basis32, p.V, p.K);
}

// One block per problem: the solver state zeroed, then tol, maxit, m and the
// partial-sum stride set (the state init_state gives a stand-alone solve).
__global__ void bb_init_kernel(const BatchProblem* __restrict__ P, int n) {
  const BatchProblem& p = P[blockIdx.x];
  unsigned long long* words = reinterpret_cast<unsigned long long*>(p.K);
  for (size_t t = threadIdx.x; t < sizeof(KrylovState) / 8; t += blockDim.x) words[t] = 0ull;
  __syncthreads();
  if (threadIdx.x == 0) {
    p.K->tol = p.tol;
    p.K->maxit = p.maxit;
    p.K->m = p.m;
    p.K->pstride = p.pstride;
  }
}

__global__ void bb_zero_resmax_kernel(const BatchProblem* __restrict__ P, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) *P[i].resmax = 0ull;
}

__global__ void bb_report_kernel(const BatchProblem* __restrict__ P, int n, int krylov, BatchReport* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    BatchReport r;
    if (krylov) {
      r.res = P[i].K->res2;
      r.it = P[i].K->it;
      r.flags = P[i].K->flags;
    } else {
      r.res = __longlong_as_double((long long)*P[i].resmax);
      r.it = 0;
      r.flags = 0;
    }
    out[i] = r;
  }
}

// ---- host side -------------------------------------------------------------------

namespace {

// Pinned staging for the descriptor table, the block ranges and the reports;
// one per host thread, grown on demand.
struct PinnedArena {
  char* p = nullptr;
  size_t cap = 0;
  ~PinnedArena() {
    if (p) cudaFreeHost(p);
  }
  char* get(size_t bytes) {
    if (bytes <= cap) return p;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max<size_t>(bytes, 1 << 16);
    if (cudaMallocHost((void**)&p, want) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return nullptr;
    }
    cap = want;
    return p;
  }
};
thread_local PinnedArena t_arena;

struct Item {
  mdp_s* h;
  const mdp_solve_opts* o;
  double* V;
  int32_t* pi;
  int k = 0;
  bool active = true;
  bool inner_failed = false;
  bool mixed = false;  // MDP_PREC_MIXED: binary32 Arnoldi cycles, FP64 restarts
  double res = 0.0;
  mdp_status status = MDP_OK;
  mdp_solve_stats stats{};
};

constexpr int kNB[8] = {4, 8, 12, 16, 20, 24, 28, 32};  // Gram-Schmidt widths (FP64 and binary32)

// Device and pinned buffers of one batched call.
struct BatchBuffers {
  BatchProblem* desc = nullptr;  // [n]
  int32_t* ranges = nullptr;     // [kRanges][n + 1]
  BatchReport* rep = nullptr;    // [n]
  int n = 0;
  cudaStream_t st = nullptr;
  char* pin = nullptr;
  BatchProblem* pin_desc() const { return reinterpret_cast<BatchProblem*>(pin); }
  int32_t* pin_ranges() const { return reinterpret_cast<int32_t*>(pin + sizeof(BatchProblem) * n); }
  BatchReport* pin_rep() const {
    return reinterpret_cast<BatchReport*>(pin + sizeof(BatchProblem) * n + sizeof(int32_t) * kRanges * (n + 1));
  }
  static size_t pinned_bytes(int n) {
    return sizeof(BatchProblem) * n + sizeof(int32_t) * kRanges * (n + 1) + sizeof(BatchReport) * n + 64;
  }
  const int32_t* range(int kind) const { return ranges + (size_t)kind * (n + 1); }
  ~BatchBuffers() {
    if (desc) cudaFreeAsync(desc, st);
    if (ranges) cudaFreeAsync(ranges, st);
    if (rep) cudaFreeAsync(rep, st);
  }
};

BatchProblem describe(const Item& it) {
  mdp_s* h = it.h;
  BatchProblem p{};
  p.sval = h->P.val;
  p.scol = h->P.col;
  p.soff = h->P.off;
  p.slen = h->P.len;
  p.g = h->g;
  p.pval = h->Ppi.val;
  p.pcol = h->Ppi.col;
  p.poff = h->Ppi.off;
  p.plen = h->Ppi.len;
  p.gpi = h->gpi;
  p.V = it.V;
  p.TV = h->TV;
  p.pi = it.pi;
  p.basis = h->basis;
  p.w = h->w;
  p.partials = h->partials;
  p.resmax = h->resmax;
  p.K = (KrylovState*)h->kstate;
  p.S = h->S;
  p.gamma = it.o->gamma;
  p.tol = it.o->alpha * it.res;
  p.A = h->A;
  p.skmax = h->P.kmax;
  p.suniform = h->P.uniform ? 1 : 0;
  p.pkmax = h->Ppi.kmax;
  p.puniform = h->Ppi.uniform ? 1 : 0;
  p.tile_states = h->bell_tile_states;
  p.pstride = h->partial_stride;
  p.maxit = it.o->max_iter_ksp;
  p.m = it.o->gmres_restart;
  p.mixed = it.mixed ? 1 : 0;
  p.pstore = h->pstore;
  if (it.mixed) {
    p.basis32 = h->basis32;
    p.w32 = h->w32;
    p.pval32 = h->pstore == kStoreF32 ? h->pval32 : nullptr;
    p.pval16 = h->pstore != kStoreF32 ? h->pval16 : nullptr;
  }
  return p;
}

int blocks_for(const Item& it, int kind) {
  mdp_s* h = it.h;
  if (kind == kRangeBellman) return h->bell_blocks;
  if (kind == kRangeExtract) return extract_blocks(h);
  const bool f = kind >= kRangeResidualF;  // a binary32 pass
  if (f != it.mixed) return 0;
  switch (kind) {
    case kRangeResidual: case kRangeResidualF: return gmres_grid(h, kPassResidual, 0, f);
    case kRangeMatvecF: return gmres_grid(h, kPassMatvec, 0, f);
    case kRangeUpdate: case kRangeUpdateF: return gmres_grid(h, kPassUpdate, 0, f);
    default: break;
  }
  if (kind < kRangeProject0) return gmres_grid(h, kPassDots, kNB[kind - kRangeDots0], false);
  if (kind < kRangeResidualF) return gmres_grid(h, kPassProject, kNB[kind - kRangeProject0], false);
  if (kind < kRangeProjectF0) return gmres_grid(h, kPassDots, kNB[kind - kRangeDotsF0], true);
  return gmres_grid(h, kPassProject, kNB[kind - kRangeProjectF0], true);
}

// Upload the descriptors and block ranges of the problems in `act`.
mdp_status upload(BatchBuffers& B, std::vector<Item>& items, const std::vector<int>& act, size_t* bell_smem) {
  const int na = (int)act.size();
  // the previous upload and report copies have completed: the host waited on the stream since
  BatchProblem* pd = B.pin_desc();
  int32_t* pr = B.pin_ranges();
  size_t smem = 0;
  for (int a = 0; a < na; ++a) {
    pd[a] = describe(items[act[a]]);
    smem = std::max(smem, bellman_smem_bytes(items[act[a]].h));
  }
  for (int kind = 0; kind < kRanges; ++kind) {
    int32_t* r = pr + (size_t)kind * (B.n + 1);
    int64_t acc = 0;
    for (int a = 0; a < na; ++a) {
      r[a] = (int32_t)acc;
      acc += blocks_for(items[act[a]], kind);
    }
    if (acc > INT32_MAX) return fail(MDP_ERR_INVALID_ARG, "batch too large: more than 2^31 blocks in one launch");
    r[na] = (int32_t)acc;
  }
  MDP_CUDA(cudaMemcpyAsync(B.desc, pd, sizeof(BatchProblem) * na, cudaMemcpyHostToDevice, B.st));
  MDP_CUDA(cudaMemcpyAsync(B.ranges, pr, sizeof(int32_t) * kRanges * (B.n + 1), cudaMemcpyHostToDevice, B.st));
  *bell_smem = smem;
  return MDP_OK;
}

int total_blocks(const BatchBuffers& B, int kind, int na) { return B.pin_ranges()[(size_t)kind * (B.n + 1) + na]; }

mdp_status report(BatchBuffers& B, int na, int krylov, int64_t* launches) {
  bb_report_kernel<<<(na + 255) / 256, 256, 0, B.st>>>(B.desc, na, krylov, B.rep);
  ++*launches;
  MDP_CUDA(cudaGetLastError());
  MDP_CUDA(cudaMemcpyAsync(B.pin_rep(), B.rep, sizeof(BatchReport) * na, cudaMemcpyDeviceToHost, B.st));
  MDP_CUDA(cudaStreamSynchronize(B.st));
  return MDP_OK;
}

#define BB_LAUNCH(kern, kind, ...)                                                                      \
  do {                                                                                                  \
    const int nblk_ = total_blocks(B, kind, na);                                                        \
    if (nblk_ > 0) {                                                                                    \
      kern<<<nblk_, kVecThreads, 0, B.st>>>(B.desc, B.range(kind), na, ##__VA_ARGS__);                  \
      ++launches;                                                                                       \
      MDP_CUDA(cudaGetLastError());                                                                     \
    }                                                                                                   \
  } while (0)

mdp_status arnoldi_batch(BatchBuffers& B, int na, int j, int64_t& launches) {
  switch ((j + 4) / 4) {  // the binary64 problems: mat-vec with the dots, then the projection
    case 1: BB_LAUNCH(bb_matvec_dots_kernel<4>, kRangeDots0 + 0, j); BB_LAUNCH(bb_project_kernel<4>, kRangeProject0 + 0, j); break;
    case 2: BB_LAUNCH(bb_matvec_dots_kernel<8>, kRangeDots0 + 1, j); BB_LAUNCH(bb_project_kernel<8>, kRangeProject0 + 1, j); break;
    case 3: BB_LAUNCH(bb_matvec_dots_kernel<12>, kRangeDots0 + 2, j); BB_LAUNCH(bb_project_kernel<12>, kRangeProject0 + 2, j); break;
    case 4: BB_LAUNCH(bb_matvec_dots_kernel<16>, kRangeDots0 + 3, j); BB_LAUNCH(bb_project_kernel<16>, kRangeProject0 + 3, j); break;
    case 5: BB_LAUNCH(bb_matvec_dots_kernel<20>, kRangeDots0 + 4, j); BB_LAUNCH(bb_project_kernel<20>, kRangeProject0 + 4, j); break;
    case 6: BB_LAUNCH(bb_matvec_dots_kernel<24>, kRangeDots0 + 5, j); BB_LAUNCH(bb_project_kernel<24>, kRangeProject0 + 5, j); break;
    case 7: BB_LAUNCH(bb_matvec_dots_kernel<28>, kRangeDots0 + 6, j); BB_LAUNCH(bb_project_kernel<28>, kRangeProject0 + 6, j); break;
    default: BB_LAUNCH(bb_matvec_dots_kernel<32>, kRangeDots0 + 7, j); BB_LAUNCH(bb_project_kernel<32>, kRangeProject0 + 7, j); break;
  }
  // the mixed problems' binary32 step at the widths of the single-problem mixed solver
  BB_LAUNCH(bb_matvec_f_kernel, kRangeMatvecF, j);
  switch ((j + 4) / 4) {
    case 1: BB_LAUNCH(bb_dots_f_kernel<4>, kRangeDotsF0 + 0, j); BB_LAUNCH(bb_project_f_kernel<4>, kRangeProjectF0 + 0, j); break;
    case 2: BB_LAUNCH(bb_dots_f_kernel<8>, kRangeDotsF0 + 1, j); BB_LAUNCH(bb_project_f_kernel<8>, kRangeProjectF0 + 1, j); break;
    case 3: BB_LAUNCH(bb_dots_f_kernel<12>, kRangeDotsF0 + 2, j); BB_LAUNCH(bb_project_f_kernel<12>, kRangeProjectF0 + 2, j); break;
    case 4: BB_LAUNCH(bb_dots_f_kernel<16>, kRangeDotsF0 + 3, j); BB_LAUNCH(bb_project_f_kernel<16>, kRangeProjectF0 + 3, j); break;
    case 5: BB_LAUNCH(bb_dots_f_kernel<20>, kRangeDotsF0 + 4, j); BB_LAUNCH(bb_project_f_kernel<20>, kRangeProjectF0 + 4, j); break;
    case 6: BB_LAUNCH(bb_dots_f_kernel<24>, kRangeDotsF0 + 5, j); BB_LAUNCH(bb_project_f_kernel<24>, kRangeProjectF0 + 5, j); break;
    case 7: BB_LAUNCH(bb_dots_f_kernel<28>, kRangeDotsF0 + 6, j); BB_LAUNCH(bb_project_f_kernel<28>, kRangeProjectF0 + 6, j); break;
    default: BB_LAUNCH(bb_dots_f_kernel<32>, kRangeDotsF0 + 7, j); BB_LAUNCH(bb_project_f_kernel<32>, kRangeProjectF0 + 7, j); break;
  }
  return MDP_OK;
}

// GMRES(m) on every problem of the table at once (the single-problem driver's
// cycle structure: queue a whole cycle, then read every problem's header).
mdp_status gmres_batch(BatchBuffers& B, std::vector<Item>& items, const std::vector<int>& act, int64_t& launches) {
  const int na = (int)act.size();
  bb_init_kernel<<<na, 256, 0, B.st>>>(B.desc, na);
  ++launches;
  MDP_CUDA(cudaGetLastError());
  BB_LAUNCH(bb_residual_kernel, kRangeResidual);
  BB_LAUNCH(bb_residual_f_kernel, kRangeResidualF);
  for (;;) {
    MDP_TRY(report(B, na, 1, &launches));
    int steps = 0;
    for (int a = 0; a < na; ++a) {
      const BatchReport& r = B.pin_rep()[a];
      if (r.flags & kSolveDone) continue;
      const Item& it = items[act[a]];
      steps = std::max(steps, std::min(it.o->gmres_restart, it.o->max_iter_ksp - r.it));
    }
    if (steps == 0) break;
    for (int j = 0; j < steps; ++j) MDP_TRY(arnoldi_batch(B, na, j, launches));
    BB_LAUNCH(bb_update_kernel, kRangeUpdate);
    BB_LAUNCH(bb_update_f_kernel, kRangeUpdateF);
    BB_LAUNCH(bb_residual_kernel, kRangeResidual);
    BB_LAUNCH(bb_residual_f_kernel, kRangeResidualF);
  }
  for (int a = 0; a < na; ++a) {
    Item& it = items[act[a]];
    const BatchReport& r = B.pin_rep()[a];
    if (r.flags & kNumeric) {  // as mdp_solve: the failed evaluation's iterations are not counted
      it.status = MDP_ERR_NUMERIC;
      it.inner_failed = true;
    } else {
      it.stats.inner_iters_total += r.it;
    }
  }
  return MDP_OK;
}

}  // namespace

}  // namespace mdp

using namespace mdp;

extern "C" {

mdp_status mdp_solve_batch(int32_t n, const mdp_handle* handles, const mdp_solve_opts* opts, double* const* V,
                           int32_t* const* pi, mdp_solve_stats* stats, mdp_status* status, void* stream) {
  NvtxRange range("mdp_solve_batch");
  const auto t0 = std::chrono::steady_clock::now();
  if (n < 1 || !handles || !opts || !V || !pi || !status) return fail(MDP_ERR_INVALID_ARG, "null argument or n < 1");
  for (int i = 0; i < n; ++i)  // argument errors are reported before any CUDA call
    if (!handles[i] || !V[i] || !pi[i]) return fail(MDP_ERR_INVALID_ARG, "null handle or vector in the batch");
  cudaStream_t st = (cudaStream_t)stream;
  int device = -1;
  MDP_CUDA(cudaGetDevice(&device));
  std::vector<Item> items(n);
  for (int i = 0; i < n; ++i) {
    mdp_s* h = handles[i];
    const mdp_solve_opts* o = opts + i;
    if (!h || !V[i] || !pi[i]) return fail(MDP_ERR_INVALID_ARG, "null handle or vector in the batch");
    if (h->device != device) return fail(MDP_ERR_INVALID_ARG, "every handle of a batch must live on the current device");
    for (int q = 0; q < i; ++q)
      if (handles[q] == h) return fail(MDP_ERR_INVALID_ARG, "a handle appears twice in the batch");
    if (!(o->gamma > 0.0 && o->gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
    if (!(o->atol_pi > 0.0) || !(o->alpha > 0.0 && o->alpha < 1.0))
      return fail(MDP_ERR_INVALID_ARG, "need atol_pi > 0 and 0 < alpha < 1");
    if (o->max_iter_pi < 0 || o->max_iter_ksp < 0) return fail(MDP_ERR_INVALID_ARG, "negative iteration cap");
    if (o->inner != MDP_GMRES || o->gmres_refine != MDP_REFINE_NEVER ||
        (o->precision != MDP_PREC_F64 && o->precision != MDP_PREC_MIXED))
      return fail(MDP_ERR_INVALID_ARG,
                  "mdp_solve_batch runs GMRES (FP64 or mixed) with classical Gram-Schmidt (MDP_REFINE_NEVER) only");
    if (o->gmres_restart < 1 || o->gmres_restart > kMaxBasis)
      return fail(MDP_ERR_INVALID_ARG, "GMRES restart must be in 1..32");
    items[i].h = h;
    items[i].o = o;
    items[i].V = V[i];
    items[i].pi = pi[i];
    items[i].mixed = (o->precision == MDP_PREC_MIXED);
  }
  // order after each handle's earlier calls; allocations of this call go on `st`
  for (int i = 0; i < n; ++i) {
    MDP_TRY(bind_stream(items[i].h, st));
    if (items[i].mixed)
      MDP_TRY(ensure_mixed(items[i].h, items[i].o->gmres_restart + 1));
    else
      MDP_TRY(ensure_basis(items[i].h, items[i].o->gmres_restart + 1));
  }
  bool all_graph = true;
  for (int i = 0; i < n; ++i) all_graph = all_graph && opts[i].graph != 0;
  BatchBuffers B;
  B.n = n;
  B.st = st;
  if (!all_graph) {  // the lockstep tables (the graph-driven batch needs none)
    B.pin = t_arena.get(BatchBuffers::pinned_bytes(n));
    if (!B.pin) return fail(MDP_ERR_OOM, "pinned host allocation failed");
    if (cudaMallocAsync((void**)&B.desc, sizeof(BatchProblem) * n, st) != cudaSuccess ||
        cudaMallocAsync((void**)&B.ranges, sizeof(int32_t) * kRanges * (n + 1), st) != cudaSuccess ||
        cudaMallocAsync((void**)&B.rep, sizeof(BatchReport) * n, st) != cudaSuccess) {
      cudaGetLastError();
      return fail(MDP_ERR_OOM, "device allocation failed: batch tables");
    }
  }
  int64_t launches = 0;
  auto run = [&]() -> mdp_status {
    std::vector<int> act;
    for (;;) {
      act.clear();
      for (int i = 0; i < n; ++i)
        if (items[i].active) act.push_back(i);
      if (act.empty()) break;
      int na = (int)act.size();
      // Algorithm 1 steps 2-3 for every running problem, one residual read for all
      size_t smem = 0;
      MDP_TRY(upload(B, items, act, &smem));
      MDP_TRY(raise_dyn_smem((const void*)bb_bellman_kernel, smem));
      bb_zero_resmax_kernel<<<(na + 255) / 256, 256, 0, st>>>(B.desc, na);
      ++launches;
      MDP_CUDA(cudaGetLastError());
      bb_bellman_kernel<<<total_blocks(B, kRangeBellman, na), kBellThreads, smem, st>>>(B.desc, B.range(kRangeBellman),
                                                                                        na);
      ++launches;
      MDP_CUDA(cudaGetLastError());
      MDP_TRY(report(B, na, 0, &launches));
      std::vector<int> go;
      for (int a = 0; a < na; ++a) {
        Item& it = items[act[a]];
        const double res = B.pin_rep()[a].res;
        it.stats.bellman_sweeps++;
        it.stats.final_residual = res;
        it.res = res;
        if (!std::isfinite(res)) {
          it.status = MDP_ERR_NUMERIC;
          it.active = false;
        } else if (res <= it.o->atol_pi) {
          it.stats.converged = 1;
          it.active = false;
        } else if (it.k >= it.o->max_iter_pi) {
          it.status = MDP_NOT_CONVERGED;
          it.active = false;
        } else {
          go.push_back(act[a]);
        }
      }
      if (go.empty()) break;
      act.swap(go);
      na = (int)act.size();
      // step 4 and steps 5-12 for the problems that go on
      MDP_TRY(upload(B, items, act, &smem));
      bb_extract_kernel<<<total_blocks(B, kRangeExtract, na), 256, 0, st>>>(B.desc, B.range(kRangeExtract), na);
      ++launches;
      MDP_CUDA(cudaGetLastError());
      MDP_TRY(gmres_batch(B, items, act, launches));
      for (int i : act) {
        Item& it = items[i];
        if (it.inner_failed) {
          it.active = false;
        } else {
          it.k++;
        }
      }
    }
    return MDP_OK;
  };
  // opts.graph on every member: one CUDA graph with each problem's graph-driven solve as
  // an independent branch (graph.cu), instead of the lockstep launches
  auto run_branches = [&]() -> mdp_status {
    std::vector<mdp_s*> hs(n);
    std::vector<const mdp_solve_opts*> os(n);
    std::vector<mdp_solve_stats> local(n);
    std::vector<mdp_status> sts(n, MDP_OK);
    for (int i = 0; i < n; ++i) {
      hs[i] = items[i].h;
      os[i] = items[i].o;
    }
    const mdp_status s = graph_solve_batch(n, hs.data(), os.data(), V, pi, local.data(), sts.data(), &launches, st);
    for (int i = 0; i < n; ++i) {
      Item& it = items[i];
      it.k = local[i].outer_iters;
      it.stats.converged = local[i].converged;
      it.stats.inner_iters_total = local[i].inner_iters_total;
      it.stats.final_residual = local[i].final_residual;
      it.stats.bellman_sweeps = local[i].bellman_sweeps;
      it.status = sts[i];
    }
    return s;
  };
  const mdp_status ran = all_graph ? run_branches() : run();
  // every handle's later calls wait for this one, also after a failure part way
  for (int i = 0; i < n; ++i) MDP_CUDA(cudaEventRecord(items[i].h->done, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  if (ran != MDP_OK) return ran;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < n; ++i) {
    Item& it = items[i];
    it.stats.outer_iters = it.k;
    it.stats.kernel_launches = launches;
    it.stats.policy_value_bytes = !it.mixed ? 8 : (it.h->pstore == kStoreF32 ? 4 : 2);
    it.stats.seconds = secs;
    status[i] = it.status;
    if (stats) stats[i] = it.stats;
  }
  return MDP_OK;
}

}  // extern "C"
