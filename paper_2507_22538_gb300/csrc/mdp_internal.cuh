// Internal declarations of libmdp: the handle, error plumbing and kernel launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "../../include/mdp.h"
#include "sell.cuh"

namespace mdp {

constexpr int kMaxBasis = 32;    // GMRES basis vectors held per thread in registers (restart <= 32)
constexpr int kPartialRows = 40;    // per-block partial sums (up to kMaxBasis + 1 values), transposed
constexpr int kGroup = 32;          // blocks per first-level group of a grid reduction
constexpr int kMaxGroups = 64;      // second-level sums per value: grids of up to 2048 blocks
constexpr int kMaxBlocksPerSm = 8;  // 256-thread blocks: 2048 threads per SM
// Largest grid of a reducing kernel: the two-level tail holds kMaxGroups group sums
// of kGroup blocks each.  Grids are clamped to it (a part with more than 256 SMs
// runs fewer blocks per SM instead of overrunning the group rows).
constexpr int kMaxReduceBlocks = kGroup * kMaxGroups;
constexpr int kMatvecTimingStride = 8;  // record_timing times the mat-vec of steps j = 0, 8, 16, ... of a cycle
enum : int { kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2 };
constexpr int kScalarSlots = 512;

// Per-thread message of the last failure.
void set_error(const std::string& msg);
mdp_status fail(mdp_status st, const std::string& msg);
mdp_status cuda_fail(cudaError_t e, const char* what);

// An NVTX range over a scope: the library's calls and the phases of Algorithm 1
// show up by name in Nsight Systems and can select kernels in Nsight Compute
// (--nvtx --nvtx-include).  Without an attached tool a range costs a branch.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define MDP_TRY(x)                 \
  do {                             \
    mdp_status st_ = (x);          \
    if (st_ != MDP_OK) return st_; \
  } while (0)

#define MDP_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return ::mdp::cuda_fail(e_, #call); \
  } while (0)

// Programmatic dependent launch (sm_90 and later).  A kernel launched with launch_pdl
// may be scheduled while the previous kernel on its stream is still finishing, so its
// launch and block scheduling overlap that kernel's tail (the last block's grid
// reduction).  Every such kernel calls pdl_begin() before touching memory:
// griddepcontrol.wait returns once the previous kernel has completed and its writes
// are visible, so results and stream order are unchanged; launch_dependents then
// lets the next kernel start launching.  Both are no-ops in a launch without the
// attribute.  A probe of back-to-back dependent reducing kernels at 10^6 states
// measured about 2 us less per kernel boundary.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args) {
  static_assert(sizeof...(KArgs) == sizeof...(Args), "kernel argument count");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Sliced-ELL (slice height 32) copy of a row-major matrix: slice q holds rows
// 32q..32q+31, each padded to the slice's width w.  The first w & ~3 entries of
// a row are stored in chunks of 4 consecutive entries (chunk c of lane l at
// off[q] + 128 c + 4 l), the remaining w & 3 column-major (entry j of lane l at
// off[q] + 32 j + l).  A warp streaming 32 rows still reads whole contiguous
// lines, and one row's entries come 4 to a 32-byte sector, which is what a
// gather of single rows (the policy rows of Algorithm 1 step 4) pays for.
// When every row has the same length k, `uniform` is set, off[q] = 32*k*q and
// len[] is unused.
struct Sell {
  int64_t rows = 0;
  int64_t nslices = 0;
  int32_t kmax = 0;
  bool uniform = false;
  int64_t* off = nullptr;   // [nslices + 1] (non-uniform only)
  int32_t* len = nullptr;   // [rows]        (non-uniform only)
  double* val = nullptr;    // [off[nslices]]
  int32_t* col = nullptr;
  int64_t nstored = 0;      // off[nslices]
};

}  // namespace mdp

struct mdp_s {
  int device = 0;
  int sm_count = 0;
  int64_t S = 0;
  int32_t A = 0;
  int64_t R = 0;    // S * A rows of Eq. 5
  int64_t nnz = 0;

  mdp::Sell P;      // all S*A rows, row s*A + a
  mdp::Sell Ppi;    // one row per state (the policy's rows), rebuilt per policy
  double* g = nullptr;      // [R]
  double* gpi = nullptr;    // [S]

  // Bellman launch shape
  int bell_tile_states = 32;
  int bell_threads = 256;
  int bell_blocks = 0;
  int bell_max_per_sm = 0;   // resident blocks per SM the tile allows (occupancy calculator)
  int bell_per_sm_cap = 0;   // blocks per SM the grid uses, chosen by mdp_tune (0: bell_max_per_sm)
  int bell_rpl = 1;          // rows of the stacked matrix per lane and warp step (1 or 2), chosen by mdp_tune
  int bell_v256 = 0;         // 1: binary64 values of a chunk in one 32-byte load (chosen by mdp_tune)

  // vector-kernel launch shape (thread per state)
  int vec_threads = 256;
  int vec_blocks = 0;  // reductions over states (bounded so the last block's final sum stays short)
  int mv_blocks = 0;   // policy mat-vec without reduction (as many resident warps as fit)

  // workspace
  double* TV = nullptr;      // [S]
  int32_t* piw = nullptr;    // [S] policy workspace
  double* w = nullptr;       // [S]
  double* tmp = nullptr;     // [S]
  double* basis = nullptr;   // [(restart + 1) * S]
  int basis_cap = 0;         // vectors allocated in basis
  // mixed-precision inner solver: FP32 copies of the policy rows' values, FP32 basis and w
  float* pval32 = nullptr;   // [Ppi.nstored]
  // narrowest exact storage of the probabilities, found at creation: 0 = binary32,
  // 1 = binary16, 2 = bfloat16 (the mixed solver's policy rows then use it)
  int pstore = 0;
  uint16_t* pval16 = nullptr;  // [Ppi.nstored], binary16 or bfloat16 bits
  // every column of P within 32767 of its row's first column (found at creation): the
  // mixed solver's policy rows then also keep column - base as int16, base = the row's
  // first column
  bool col16 = false;
  int16_t* pcol16 = nullptr;   // [Ppi.nstored]
  int32_t* pcolbase = nullptr; // [S]
  float* basis32 = nullptr;  // [(restart + 1) * S]
  int basis32_cap = 0;
  float* w32 = nullptr;      // [S]
  double* tfq = nullptr;     // TFQMR vectors [8 * S] (the first also holds the Jacobi diagonal)
  double* partials = nullptr;  // [kPartialRows * (partial_stride + kMaxGroups)]: row i holds value i of every
                               // block, then the second-level group sums (krylov_dev.cuh grid_finish)
  int partial_stride = 0;      // sm_count * kMaxBlocksPerSm, the largest grid of a reducing kernel
  void* kstate = nullptr;      // device state of the inner solver (krylov.cu)
  double* sc = nullptr;      // device scalars [kScalarSlots]
  unsigned long long* resmax = nullptr;  // device max of |TV - V| bits
  cudaStream_t stream = nullptr;         // stream of mdp_create: device memory is allocated on it
  // certified low-precision sweep (bellman_lowp.cu), set up on first use when the
  // probabilities are exact in binary16 / bfloat16
  uint16_t* P16 = nullptr;               // [P.nstored] 16-bit copy of P.val (same sliced layout)
  int16_t* P16col = nullptr;             // [P.nstored] with col16: column - P16base[row] as int16
  int32_t* P16base = nullptr;            // [R] with col16: each row's first column
  float* g32 = nullptr;                  // [R] binary32 costs
  float* vf32 = nullptr;                 // [S] binary32 copy of the sweep's V
  unsigned long long* lp_rows = nullptr; // rows re-evaluated in binary64 (running count)
  int lp_blocks = 0;                     // grid of the low-precision sweep
  int lp_ts = 0;                         // its states per tile (0: not shaped yet)
  int lp_ts_tuned = 0;                   // the tile mdp_tune chose for it (0: follow the Bellman tile)

  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  cudaEvent_t done = nullptr;  // recorded after the work of every call; mdp_destroy waits on it
  void* gcache = nullptr;      // instantiated graph of the graph-driven mdp_solve (graph.cu)
  // record_timing: events around the Arnoldi mat-vec of every GMRES step (created on first use)
  int timing = 0;
  cudaEvent_t mv_ev[2 * mdp::kMaxBasis] = {};
  double mv_ms = 0.0, mv_bytes = 0.0, mv_flops = 0.0;
  int64_t mv_timed = 0;
  // and after the projection of the same steps (FP64 single-pass steps, whose mat-vec also forms the dots)
  cudaEvent_t gs_ev[mdp::kMaxBasis] = {};
  bool gs_on = false;
  double gs_ms = 0.0, gs_flops = 0.0;
  int64_t gs_timed = 0;
  int64_t launches = 0;
  // algorithmic work counters of the inner solver (see mdp_solve_stats)
  int64_t matvecs = 0, vreads = 0, vwrites = 0;
  double inner_bytes = 0.0;
};

namespace mdp {

// Pinned host scratch of the calling thread (64 doubles), for small stream-ordered
// copies of scalars; allocated once per host thread.
double* tls_pinned();

// layout.cu
// Raise (never lower) a kernel's dynamic shared memory cap on the current device to `bytes`.
mdp_status raise_dyn_smem(const void* func, size_t bytes);
mdp_status extract_policy(mdp_s* h, const int32_t* pi, bool want32, cudaStream_t st);  // fill Ppi, gpi from pi

// bellman.cu
mdp_status configure_bellman(mdp_s* h);  // threads and grid of the Bellman sweep
mdp_status launch_bellman(mdp_s* h, double gamma, const double* V, double* TV, int32_t* pi, cudaStream_t st);

// bellman_lowp.cu: the certified low-precision sweep (bit for bit the results of launch_bellman)
bool lowp_available(const mdp_s* h);          // probabilities exact in binary16 / bfloat16
mdp_status prepare_lowp(mdp_s* h, cudaStream_t st);
mdp_status launch_bellman_lowp(mdp_s* h, double gamma, const double* V, double* TV, int32_t* pi, cudaStream_t st);
// the low-precision sweep when asked for and available, else the binary64 one
mdp_status launch_sweep(mdp_s* h, bool lowp, double gamma, const double* V, double* TV, int32_t* pi,
                        cudaStream_t st);

// krylov.cu
mdp_status launch_policy_apply(mdp_s* h, double gamma, const double* x, double* y, cudaStream_t st);
mdp_status inner_solve(mdp_s* h, double gamma, double* theta, int inner, int restart, int refine, int precision,
                       double omega, double tol, int max_it, int* iters, double* res2, cudaStream_t st);
// Order a call on stream `st` after the handle's earlier calls (its `done`
// event) and make `st` the stream of the handle's later allocations.
mdp_status bind_stream(mdp_s* h, cudaStream_t st);

// Launch shapes of the single-problem passes, reused by the batched solver.
enum GmresPass { kPassResidual, kPassMatvec, kPassUpdate, kPassDots, kPassProject };
int gmres_grid(mdp_s* h, GmresPass pass, int NB, bool mixed);
int extract_blocks(const mdp_s* h);
size_t bellman_smem_bytes(const mdp_s* h);
mdp_status ensure_basis(mdp_s* h, int nvec);
mdp_status ensure_mixed(mdp_s* h, int nvec);  // FP32 policy values, basis and w for the mixed solver
mdp_status ensure_tfqmr(mdp_s* h);            // TFQMR / Jacobi work vectors
size_t krylov_state_bytes();

// graph.cu: Algorithm 1 with the GMRES inner solver as one CUDA graph launch (fills the
// iteration fields of *stats; returns MDP_OK, MDP_NOT_CONVERGED, MDP_ERR_NUMERIC or an error)
mdp_status graph_solve(mdp_s* h, const mdp_solve_opts* o, double* V, int32_t* pi, mdp_solve_stats* stats,
                       cudaStream_t st);
void graph_cache_free(mdp_s* h);
// mdp_solve_batch with opts.graph on every member: one graph, each problem's graph-driven
// solve an independent branch (handles distinct, buffers ensured; fills local[], status[])
mdp_status graph_solve_batch(int n, mdp_s* const* hs, const mdp_solve_opts* const* os, double* const* V,
                             int32_t* const* pi, mdp_solve_stats* local, mdp_status* status, int64_t* launches,
                             cudaStream_t st);
// Building blocks of the captured graphs (graph.cu; also used by the batched graph solve).
mdp_status graph_add_segment(cudaGraph_t parent, const cudaGraphNode_t* deps, size_t ndeps, cudaGraph_t seg,
                             cudaGraphNode_t* node);
mdp_status graph_add_conditional(cudaGraph_t parent, const cudaGraphNode_t* deps, size_t ndeps,
                                 cudaGraphConditionalHandle c, cudaGraphConditionalNodeType type,
                                 cudaGraphNode_t* node, cudaGraph_t* body);

}  // namespace mdp
