// Algorithm 1 for small MDPs inside one thread-block cluster per problem
// (mdp_solve_small_batch): the Bellman sweep (Eq. 3-4), the stop tests, the policy's
// rows (step 4) and restarted GMRES (steps 5-12, classical Gram-Schmidt, Givens
// rotations) run from start to finish in one kernel, and a batch of problems is one
// launch with no host round trip until every problem has stopped.
//
// Why: a grid-wide solve of a 1000-state problem is about 280 kernels of a few
// microseconds each, bound by launch and reduction-tail latency, not by the work.
// Here every synchronisation is a block barrier or a hardware cluster barrier.
//
// Layout of the work: the cluster's c blocks own consecutive ranges of states; the
// stacked matrix (sliced layout of the handle), g, V and the GMRES basis stay in
// global memory (L2-resident at these sizes).  A reduction forms one partial per
// block in a fixed order, publishes it in the block's shared memory, and after a
// cluster barrier every block adds the c partials in rank order, so all blocks hold
// identical sums and take identical decisions (stop tests, Givens rotations, back
// substitution) without further communication.  Partial slots are double-buffered:
// a slot is written again only after the next barrier, when every block has read it.
//
// No block waits on anything but its own block barrier and the cluster barrier, so
// nothing can spin.  Results are deterministic for a given cluster size, which is a
// function of the problem's size alone (so a problem gives the same bits alone and
// in any batch).
#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <unordered_set>
#include <vector>

#include "mdp_internal.cuh"

namespace cg = cooperative_groups;

namespace mdp {
namespace {

constexpr int kBsThreads = 512;           // threads per block
constexpr int kBsWarps = kBsThreads / 32;
constexpr int kBsMaxCluster = 8;          // portable cluster size
constexpr int kBsStatesPerBlock = 512;    // cluster size: enough blocks for about this many states each
constexpr int64_t kBsMaxStates = 65536;
constexpr int kBsSmemCap = 200 * 1024;    // dynamic shared memory for a block's share of the basis and w

struct BsProblem {
  const double* val;
  const int32_t* col;
  const int64_t* off;
  const int32_t* len;
  const double* g;
  double* V;
  int32_t* pi;
  double* basis;  // [(m + 1) * S]
  double* w;      // [S]
  int64_t S;
  int A;
  int k;          // row length when uniform, else 0
  int uniform;
  int m;          // GMRES restart
  int max_pi, max_ksp;
  double gamma, tol, alpha;
};

struct BsResult {
  int outer;
  int sweeps;
  long long inner;
  double res;
  int status;  // mdp_status
  int pad;
};

// Dot of stacked row r (= s * A + a) with x, as the Bellman sweep and the
// policy mat-vec compute it (sell_row_dot over the row's slice position).
__device__ __forceinline__ double bs_row_dot(const BsProblem& P, int64_t r, const double* __restrict__ x) {
  const int64_t q = r / kSlice;
  const int lane = (int)(r % kSlice);
  const int n = P.uniform ? P.k : P.len[r];
  const int w = P.uniform ? P.k : (int)((P.off[q + 1] - P.off[q]) / kSlice);
  const int64_t base = P.uniform ? q * kSlice * (int64_t)P.k : P.off[q];
  return sell_row_dot(P.val, P.col, base, w, lane, n, x);
}

__device__ __forceinline__ double bs_nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

// Shared state of one block.
struct BsShared {
  double part[2][kMaxBasis + 1];   // this block's published partials (double-buffered)
  double warp_red[kBsWarps];
  double h[kMaxBasis + 1];         // reduced values of the current reduction
  double hc[kMaxBasis + 1];        // Hessenberg column of the current step (h_i = v_i . w)
  double coef[kMaxBasis + 1];      // its projection coefficients on the stored u_i
  double H[(kMaxBasis + 1) * kMaxBasis];
  double cs[kMaxBasis], sn[kMaxBasis], e[kMaxBasis + 1], sigma[kMaxBasis + 1], y[kMaxBasis];
  double res, tol_in, beta;
  int flags, jdone, it;
};

enum : int { kBsStop = 1, kBsNumeric = 2 };

}  // namespace
}  // namespace mdp

namespace mdp {
namespace {

// Sum (or NaN-propagating max) over the cluster of nv values that every block has
// written into sh.part[buf][0..nv); the result lands in sh.h[0..nv) of every block.
// The cluster barrier also orders each block's earlier global writes (the caller
// fences them) before every block's later reads.
template <bool MAX>
__device__ __forceinline__ void cluster_combine(cg::cluster_group& cl, BsShared& sh, int buf, int nv) {
  cl.sync();
  if ((int)threadIdx.x < nv) {
    const int c = (int)cl.num_blocks();
    double t = 0.0;
    for (int r = 0; r < c; ++r) {
      const BsShared* o = cl.map_shared_rank(&sh, r);
      const double v = o->part[buf][threadIdx.x];
      t = MAX ? bs_nan_max(t, v) : t + v;
    }
    sh.h[threadIdx.x] = t;
  }
  __syncthreads();
}

// One value per thread: block sum (or max) in a fixed order, then the cluster's.
template <bool MAX>
__device__ __forceinline__ double cluster_reduce1(cg::cluster_group& cl, BsShared& sh, int& buf, double v) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = MAX ? bs_nan_max(v, u) : v + u;
  }
  if (lane == 0) sh.warp_red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBsWarps; ++w) t = MAX ? bs_nan_max(t, sh.warp_red[w]) : t + sh.warp_red[w];
    sh.part[buf][0] = t;
  }
  cluster_combine<MAX>(cl, sh, buf, 1);
  const double r = sh.h[0];
  __syncthreads();  // sh.h is reused by the next reduction
  buf ^= 1;
  return r;
}

// Arnoldi bookkeeping of step j once h_0..h_j (sh.h) and hn are known: column j of
// the Hessenberg matrix, the earlier rotations applied to it, the new rotation, the
// rotated right-hand side and the stop flags (one thread per block; every block
// computes the same values from the same sums).
__device__ void bs_finish_step(BsShared& sh, int j, double hn, int m, int maxit) {
  double* H = sh.H;
  for (int i = 0; i <= j; ++i) H[i * kMaxBasis + j] = sh.hc[i];
  H[(j + 1) * kMaxBasis + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * kMaxBasis + j], b = H[(i + 1) * kMaxBasis + j];
    H[i * kMaxBasis + j] = sh.cs[i] * a + sh.sn[i] * b;
    H[(i + 1) * kMaxBasis + j] = -sh.sn[i] * a + sh.cs[i] * b;
  }
  const double a = H[j * kMaxBasis + j], b = H[(j + 1) * kMaxBasis + j];
  const double d = hypot(a, b);
  sh.cs[j] = a / d;
  sh.sn[j] = b / d;
  H[j * kMaxBasis + j] = d;
  H[(j + 1) * kMaxBasis + j] = 0.0;
  sh.e[j + 1] = -sh.sn[j] * sh.e[j];
  sh.e[j] = sh.cs[j] * sh.e[j];
  sh.sigma[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
  sh.it += 1;
  sh.jdone = j + 1;
  int f = 0;
  if (!isfinite(hn) || !(d > 0.0) || !isfinite(d)) f |= kBsNumeric | kBsStop;
  if (fabs(sh.e[j + 1]) < sh.tol_in || sh.it >= maxit || hn == 0.0 || j + 1 == m) f |= kBsStop;
  sh.flags = f;
}

}  // namespace
}  // namespace mdp

namespace mdp {
namespace {

// Algorithm 1 on problem blockIdx.x / cluster size, by the blocks of one cluster.
// MINB: blocks per SM the register budget is sized for (1 with the basis in shared
// memory, one block per SM anyway; 2 for the global-memory variant of large batches).
template <int MINB>
__global__ void __launch_bounds__(kBsThreads, MINB) block_solve_kernel(const BsProblem* __restrict__ probs,
                                                                       BsResult* __restrict__ results, int smem_bytes) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ BsShared sh;
  extern __shared__ double bs_dyn[];
  const int c = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const BsProblem P = probs[blockIdx.x / c];
  const int64_t S = P.S;
  const int A = P.A, m = P.m;
  const double gamma = P.gamma;
  // this block's states: a contiguous share of [0, S)
  const int64_t per = (S + c - 1) / c;
  const int64_t s_lo = min(S, (int64_t)rank * per), s_hi = min(S, s_lo + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* __restrict__ V = P.V;
  int32_t* __restrict__ pi = P.pi;
  double* __restrict__ U = P.basis;  // global basis: the mat-vec gathers u_j from it
  // The block's own states of the basis and of w: in shared memory when (m + 2) vectors
  // of its share fit (every access of the dots, projection and update is local), else
  // the global arrays.  Same values and order either way, so the same results.
  const bool local = (int64_t)(m + 2) * per * (int64_t)sizeof(double) <= (int64_t)smem_bytes;
  double* const Ul = local ? bs_dyn : U;                  // u_i of state s at Ul[i * ust + s - uoff]
  const int64_t ust = local ? per : S, uoff = local ? s_lo : 0;
  double* const w = local ? bs_dyn + (int64_t)(m + 1) * per - s_lo : P.w;  // w[s] for s in [s_lo, s_hi)
  int buf = 0;
  int k = 0, sweeps = 0, status = MDP_OK;
  long long inner = 0;
  double res = 0.0;
  for (;;) {
    // Algorithm 1 steps 2-3: Q = g + gamma P V, TV = min_a Q, pi = lowest argmin, ||TV - V||_inf
    double dmax = 0.0;
    for (int64_t s = s_lo + threadIdx.x; s < s_hi; s += kBsThreads) {
      double best = 0.0;
      int ba = 0;
      bool bad = false;
      for (int a = 0; a < A; ++a) {
        const int64_t r = s * A + a;
        const double q = fma(gamma, bs_row_dot(P, r, V), P.g[r]);
        bad |= (q != q);
        if (a == 0) {
          best = q;
        } else if (q < best) {
          best = q;
          ba = a;
        }
      }
      if (bad) best = __longlong_as_double(0x7ff8000000000000LL);
      pi[s] = ba;
      dmax = bs_nan_max(dmax, fabs(best - V[s]));
    }
    res = cluster_reduce1<true>(cl, sh, buf, dmax);
    ++sweeps;
    if (!isfinite(res)) {
      status = MDP_ERR_NUMERIC;
      break;
    }
    if (res <= P.tol) break;
    if (k >= P.max_pi) {
      status = MDP_NOT_CONVERGED;
      break;
    }
    // steps 4-12: GMRES(m) on (I - gamma P_pi) theta = g_pi from theta = V, to
    // ||g_pi - J theta||_2 < alpha * res or max_ksp iterations
    if (threadIdx.x == 0) {
      sh.tol_in = P.alpha * res;
      sh.it = 0;
    }
    __syncthreads();
    const double tol_in = sh.tol_in;
    int it = 0;
    bool numeric = false;
    for (;;) {
      // true residual u_0 = g_pi - J theta, beta = ||u_0||
      double nr = 0.0;
      for (int64_t s = s_lo + threadIdx.x; s < s_hi; s += kBsThreads) {
        const int64_t r = s * A + pi[s];
        const double x = P.g[r] - (V[s] - gamma * bs_row_dot(P, r, V));
        U[s] = x;
        if (local) Ul[s - uoff] = x;
        nr = fma(x, x, nr);
      }
      __threadfence();
      const double beta = sqrt(cluster_reduce1<false>(cl, sh, buf, nr));
      if (!isfinite(beta)) {
        numeric = true;
        break;
      }
      if (beta < tol_in || it >= P.max_ksp) break;
      if (threadIdx.x == 0) {
        sh.sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
        sh.e[0] = beta;
        for (int i = 1; i <= kMaxBasis; ++i) sh.e[i] = 0.0;
        sh.it = it;
        sh.flags = 0;
      }
      __syncthreads();
      int j = 0;
      for (;; ++j) {
        // w = J v_j = sigma_j (u_j - gamma P_pi u_j)
        const double sj = sh.sigma[j];
        const double* uj = U + (int64_t)j * S;
        const double* ujl = Ul + (int64_t)j * ust - uoff;
        for (int64_t s = s_lo + threadIdx.x; s < s_hi; s += kBsThreads)
          w[s] = sj * (ujl[s] - gamma * bs_row_dot(P, s * A + pi[s], uj));
        __syncthreads();
        // h_i = v_i . w = sigma_i (u_i . w), i <= j: warp per vector, lanes over states
        for (int i = warp; i <= j; i += kBsWarps) {
          const double* ui = Ul + (int64_t)i * ust - uoff;
          double d = 0.0;
          for (int64_t s = s_lo + lane; s < s_hi; s += 32) d = fma(ui[s], w[s], d);
          for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
          if (lane == 0) sh.part[buf][i] = d;
        }
        cluster_combine<false>(cl, sh, buf, j + 1);
        buf ^= 1;
        if ((int)threadIdx.x <= j) {
          const double h = sh.sigma[threadIdx.x] * sh.h[threadIdx.x];
          sh.hc[threadIdx.x] = h;
          sh.coef[threadIdx.x] = h * sh.sigma[threadIdx.x];
        }
        __syncthreads();
        // u_{j+1} = w - sum_i coef_i u_i, and ||u_{j+1}||^2
        double* un = U + (int64_t)(j + 1) * S;
        double* unl = Ul + (int64_t)(j + 1) * ust - uoff;
        double nn = 0.0;
        for (int64_t s = s_lo + threadIdx.x; s < s_hi; s += kBsThreads) {
          double x = w[s];
          const double* b = Ul + (s - uoff);
          int i = 0;
          for (; i + 4 <= j + 1; i += 4) {
            const double b0 = b[(int64_t)i * ust], b1 = b[(int64_t)(i + 1) * ust];
            const double b2 = b[(int64_t)(i + 2) * ust], b3 = b[(int64_t)(i + 3) * ust];
            x = fma(-sh.coef[i], b0, x);
            x = fma(-sh.coef[i + 1], b1, x);
            x = fma(-sh.coef[i + 2], b2, x);
            x = fma(-sh.coef[i + 3], b3, x);
          }
          for (; i <= j; ++i) x = fma(-sh.coef[i], b[(int64_t)i * ust], x);
          un[s] = x;
          if (local) unl[s] = x;
          nn = fma(x, x, nn);
        }
        __threadfence();
        const double hn = sqrt(cluster_reduce1<false>(cl, sh, buf, nn));
        if (threadIdx.x == 0) bs_finish_step(sh, j, hn, m, P.max_ksp);
        __syncthreads();
        if (sh.flags & kBsStop) break;
      }
      it = sh.it;
      numeric = (sh.flags & kBsNumeric) != 0;
      if (numeric) break;
      // theta += sum_{i < jdone} y_i v_i with R y = e (every block solves it alike)
      const int n = sh.jdone;
      if (threadIdx.x == 0) {
        for (int i = n - 1; i >= 0; --i) {
          double t = sh.e[i];
          for (int q = i + 1; q < n; ++q) t -= sh.H[i * kMaxBasis + q] * sh.y[q];
          sh.y[i] = t / sh.H[i * kMaxBasis + i];
        }
        for (int i = 0; i < n; ++i) sh.coef[i] = sh.y[i] * sh.sigma[i];
      }
      __syncthreads();
      for (int64_t s = s_lo + threadIdx.x; s < s_hi; s += kBsThreads) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t = fma(sh.coef[i], Ul[(int64_t)i * ust + (s - uoff)], t);
        V[s] += t;
      }
      __threadfence();
      cl.sync();  // theta complete before the next residual gathers it
    }
    inner += it;
    if (numeric) {
      status = MDP_ERR_NUMERIC;
      break;
    }
    ++k;
  }
  cl.sync();  // no block leaves while another may still read its shared memory
  if (rank == 0 && threadIdx.x == 0) {
    BsResult& R = results[blockIdx.x / c];
    R.outer = k;
    R.sweeps = sweeps;
    R.inner = inner;
    R.res = res;
    R.status = status;
  }
}

}  // namespace
}  // namespace mdp

using namespace mdp;

namespace {

// Blocks per cluster for a problem of S states: about kBsStatesPerBlock states per
// block, a power of two up to the portable cluster size.  It depends on S alone, so
// a problem's arithmetic (and result) does not depend on the rest of the batch.
int bs_cluster_size(int64_t S) {
  int c = 1;
  while (c < kBsMaxCluster && (int64_t)c * kBsStatesPerBlock < S) c *= 2;
  return c;
}

}  // namespace

extern "C" mdp_status mdp_solve_small_batch(int32_t n, const mdp_handle* handles, const mdp_solve_opts* opts,
                                            double* const* V, int32_t* const* pi, mdp_solve_stats* stats,
                                            mdp_status* status, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  NvtxRange range("mdp_solve_small_batch");
  if (n < 1 || !handles || !opts || !V || !pi || !status)
    return fail(MDP_ERR_INVALID_ARG, "need n >= 1 and non-null handles, opts, V, pi and status");
  int dev = -1;
  std::unordered_set<const mdp_s*> seen;
  for (int i = 0; i < n; ++i) {
    const mdp_s* h = handles[i];
    const mdp_solve_opts* o = opts + i;
    if (!h || !V[i] || !pi[i]) return fail(MDP_ERR_INVALID_ARG, "null handle or vector in the batch");
    if (!seen.insert(h).second) return fail(MDP_ERR_INVALID_ARG, "a handle appears twice in the batch");
    if (dev < 0) dev = h->device;
    if (h->device != dev) return fail(MDP_ERR_INVALID_ARG, "all handles must live on one device");
    if (h->S > kBsMaxStates) return fail(MDP_ERR_INVALID_ARG, "mdp_solve_small_batch takes at most 65536 states");
    if (!(o->gamma > 0.0 && o->gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
    if (!(o->atol_pi > 0.0) || !(o->alpha > 0.0 && o->alpha < 1.0))
      return fail(MDP_ERR_INVALID_ARG, "need atol_pi > 0 and 0 < alpha < 1");
    if (o->max_iter_pi < 0 || o->max_iter_ksp < 0) return fail(MDP_ERR_INVALID_ARG, "negative iteration cap");
    if (o->inner != MDP_GMRES || o->gmres_refine != MDP_REFINE_NEVER || o->precision != MDP_PREC_F64)
      return fail(MDP_ERR_INVALID_ARG,
                  "mdp_solve_small_batch runs GMRES with classical Gram-Schmidt (MDP_REFINE_NEVER) in binary64");
    if (o->gmres_restart < 1 || o->gmres_restart > kMaxBasis)
      return fail(MDP_ERR_INVALID_ARG, "GMRES restart must be in 1..32");
  }
  int cur = 0;
  MDP_CUDA(cudaGetDevice(&cur));
  if (cur != dev) return fail(MDP_ERR_INVALID_ARG, "the handles' device must be the current device");
  cudaStream_t st = (cudaStream_t)stream;
  // problems grouped by cluster size: one launch per size in use
  std::vector<BsProblem> probs(n);
  std::vector<int> order;
  order.reserve(n);
  int counts[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    mdp_s* h = handles[i];
    MDP_TRY(bind_stream(h, st));
    MDP_TRY(ensure_basis(h, opts[i].gmres_restart + 1));
    const int c = bs_cluster_size(h->S);
    counts[c == 1 ? 0 : c == 2 ? 1 : c == 4 ? 2 : 3]++;
  }
  for (int g = 0, c = 1; g < 4; ++g, c *= 2)
    for (int i = 0; i < n; ++i)
      if (bs_cluster_size(handles[i]->S) == c) order.push_back(i);
  for (int t = 0; t < n; ++t) {
    const int i = order[t];
    const mdp_s* h = handles[i];
    const mdp_solve_opts* o = opts + i;
    BsProblem& p = probs[t];
    p.val = h->P.val;
    p.col = h->P.col;
    p.off = h->P.off;
    p.len = h->P.len;
    p.g = h->g;
    p.V = V[i];
    p.pi = pi[i];
    p.basis = h->basis;
    p.w = h->w;
    p.S = h->S;
    p.A = h->A;
    p.k = h->P.uniform ? h->P.kmax : 0;
    p.uniform = h->P.uniform ? 1 : 0;
    p.m = o->gmres_restart;
    p.max_pi = o->max_iter_pi;
    p.max_ksp = o->max_iter_ksp;
    p.gamma = o->gamma;
    p.tol = o->atol_pi;
    p.alpha = o->alpha;
  }
  BsProblem* dprobs = nullptr;
  BsResult* dres = nullptr;
  if (cudaMallocAsync((void**)&dprobs, sizeof(BsProblem) * n, st) != cudaSuccess ||
      cudaMallocAsync((void**)&dres, sizeof(BsResult) * n, st) != cudaSuccess) {
    cudaGetLastError();
    if (dprobs) cudaFreeAsync(dprobs, st);
    return fail(MDP_ERR_OOM, "device allocation failed: batch descriptors");
  }
  struct Free {
    cudaStream_t st; BsProblem* a; BsResult* b;
    ~Free() { cudaFreeAsync(a, st); cudaFreeAsync(b, st); }
  } release{st, dprobs, dres};
  MDP_CUDA(cudaMemcpyAsync(dprobs, probs.data(), sizeof(BsProblem) * n, cudaMemcpyHostToDevice, st));
  int launches = 0;
  int sms = 0;
  MDP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  for (int g = 0, c = 1, at = 0; g < 4; ++g, c *= 2) {
    if (!counts[g]) continue;
    // A batch that leaves SMs free is latency-bound: each block then keeps its share of
    // the basis and w in shared memory (one block per SM).  A larger batch keeps them
    // in global memory, L2-resident, with several blocks per SM.  The results are the
    // same either way.
    int smem = 0;
    if ((int64_t)counts[g] * c <= 2 * (int64_t)sms) {
      for (int t = at; t < at + counts[g]; ++t) {
        const int64_t per = (probs[t].S + c - 1) / c;
        const int64_t need = (int64_t)(probs[t].m + 2) * per * (int64_t)sizeof(double);
        if (need <= kBsSmemCap) smem = std::max(smem, (int)need);
      }
      if (smem > 0) MDP_TRY(raise_dyn_smem((const void*)block_solve_kernel<1>, (size_t)smem));
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(counts[g] * c));
    cfg.blockDim = dim3(kBsThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const BsProblem* pp = dprobs + at;
    BsResult* rr = dres + at;
    if (smem > 0)
      MDP_CUDA(cudaLaunchKernelEx(&cfg, block_solve_kernel<1>, pp, rr, smem));
    else
      MDP_CUDA(cudaLaunchKernelEx(&cfg, block_solve_kernel<2>, pp, rr, smem));
    ++launches;
    at += counts[g];
  }
  std::vector<BsResult> res(n);
  MDP_CUDA(cudaMemcpyAsync(res.data(), dres, sizeof(BsResult) * n, cudaMemcpyDeviceToHost, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int t = 0; t < n; ++t) {
    const int i = order[t];
    mdp_s* h = handles[i];
    h->launches += launches;
    cudaEventRecord(h->done, st);
    status[i] = (mdp_status)res[t].status;
    if (stats) {
      mdp_solve_stats& s = stats[i];
      std::memset(&s, 0, sizeof(s));
      s.outer_iters = res[t].outer;
      s.inner_iters_total = res[t].inner;
      s.final_residual = res[t].res;
      s.converged = res[t].status == MDP_OK ? 1 : 0;
      s.bellman_sweeps = res[t].sweeps;
      s.seconds = secs;
      s.kernel_launches = launches;
      s.policy_value_bytes = 8;
      s.bellman_value_bytes = 8;
    }
  }
  return MDP_OK;
}
