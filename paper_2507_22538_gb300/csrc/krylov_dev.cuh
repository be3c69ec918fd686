// Device side of the inner solvers, shared by the single-problem kernels and the
// batched kernels (many problems per launch): the solver state in device memory,
// the row dot over the per-state sliced layout, the deterministic block/grid
// reductions and the bodies of the GMRES passes.  A body works on one problem
// with `nb` blocks of which the calling block is number `bid`.
#pragma once

#include "mdp_internal.cuh"

namespace mdp {

constexpr int kVecThreads = 256;

// ---- device state of an inner solve -------------------------------------------------

struct KrylovState {
  double H[(kMaxBasis + 1) * kMaxBasis];  // H[i * kMaxBasis + j]: rotated Hessenberg (upper triangle = R)
  double cs[kMaxBasis], sn[kMaxBasis];    // Givens rotations
  double e[kMaxBasis + 1];                // rotated right-hand side beta e_1
  double hc[kMaxBasis + 1];               // current column h_i = v_i . w
  double coef[kMaxBasis + 1];             // projection coefficients on the stored u_i
  double sigma[kMaxBasis + 1];            // v_i = sigma_i u_i
  double wnorm, beta, estimate, res2, tol;
  // TFQMR recurrences
  double t_rho, t_alpha, t_beta, t_theta, t_tau, t_eta;
  int it, maxit, m, jdone, flags, counter, result;  // result: Richardson buffer holding the answer
  int pstride;                                       // row stride of the transposed block partials
  // arrival counters of the two-level grid reductions: [0] for the groups, [1 + g] for
  // the blocks of group g (zero between kernels)
  int gcount[kMaxGroups + 2];
};

struct KrylovHeader {  // host copy of the int tail of KrylovState
  int it, maxit, m, jdone, flags, counter, result, pstride;
};

enum : int {
  kCycleStop = 1,  // this restart cycle is over
  kSolveDone = 2,  // the whole inner solve is over
  kReorth = 4,     // the current step needs its second Gram-Schmidt pass
  kNumeric = 8,    // a non-finite norm appeared
};

// sum_j P_pi[s, j] x[col_j] for state s (lane l of slice s/32), in the type of x.
// With 16-bit columns (TC = int16_t) each entry holds col_j - cbase[s].
template <bool UNIFORM, typename TP, typename TX, typename TC = int32_t>
__device__ __forceinline__ TX policy_row_dot(const TP* __restrict__ pval, const TC* __restrict__ pcol,
                                             const int64_t* __restrict__ poff, const int32_t* __restrict__ plen,
                                             int k, int64_t s, const TX* __restrict__ x,
                                             const int32_t* __restrict__ cbase = nullptr) {
  const int64_t q = s / kSlice;
  const int n = UNIFORM ? k : plen[s];
  const int w = UNIFORM ? k : (int)((poff[q + 1] - poff[q]) / kSlice);
  const int64_t base = UNIFORM ? q * kSlice * (int64_t)k : poff[q];
  const TX* xs = x;
  if constexpr (sizeof(TC) == sizeof(int16_t)) xs = x + cbase[s];
  return sell_row_dot<TP, TX, false, TC>(pval, pcol, base, w, (int)(s % kSlice), n, xs);
}

// Warp reduce-scatter of N values per lane (N a power of two, N <= 32): each
// butterfly level halves the values a lane carries (it keeps one half, adds the
// partner's copy of that half), so the warp spends about N additions per lane
// instead of 5 N for N separate shuffle trees; the last levels, once a lane
// carries one value, are plain butterflies.  Returns the warp sum of value
// index (lane >> (5 - log2 N)) in every lane.
template <int N, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&d)[N]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int half = N / 2, o = 16; half >= 1; half /= 2, o /= 2) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const T keep = upper ? d[i + half] : d[i];
      const T send = upper ? d[i] : d[i + half];
      d[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  T v = d[0];
  constexpr int kSplitLevels = (N >= 32) ? 5 : (N >= 16) ? 4 : (N >= 8) ? 3 : (N >= 4) ? 2 : (N >= 2) ? 1 : 0;
#pragma unroll
  for (int o = 16 >> kSplitLevels; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NT>
__device__ bool grid_finish(double* __restrict__ partials, int pstride, int* gcount, double* out, int bid, int nb);
template <int NT>
__device__ bool grid_finish1(double* __restrict__ partials, int pstride, int* counter, double* out, int nb);

// Block sums of NV per-thread values (NV a power of two) plus one extra value into
// partials[i * pstride + bid] (block bid of the nb blocks that work on one problem) (the extra one as column NV when HAS_EXTRA);
// the last block to finish then adds each column over all blocks in block order
// into out[] (shared memory) and returns true in all of its threads.
// Deterministic for a fixed grid.  The counter is left at zero for the next kernel.
template <int NV, bool HAS_EXTRA, typename TW>
__device__ bool grid_sum_at(TW (&d)[NV], double extra, double* __restrict__ partials, int pstride, int* counter,
                            double* out, int bid, int nb) {
  constexpr int NT = NV + (HAS_EXTRA ? 1 : 0);
  constexpr int kLog = (NV >= 32) ? 5 : (NV >= 16) ? 4 : (NV >= 8) ? 3 : (NV >= 4) ? 2 : (NV >= 2) ? 1 : 0;
  constexpr int kWarps = kVecThreads / 32;
  __shared__ double red[kWarps][NT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double v = (double)warp_reduce_scatter<NV>(d);  // the warp stage runs in the threads' type
  if ((lane & ((1 << (5 - kLog)) - 1)) == 0) red[warp][lane >> (5 - kLog)] = v;
  if (HAS_EXTRA) {
    for (int o = 16; o; o >>= 1) extra += __shfl_xor_sync(0xffffffffu, extra, o);
    if (lane == 0) red[warp][NT - 1] = extra;
  }
  __syncthreads();
  if (threadIdx.x < NT) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w][threadIdx.x];
    partials[(int64_t)threadIdx.x * pstride + bid] = t;
  }
  if constexpr (sizeof(TW) == sizeof(double))
    return grid_finish<NT>(partials, pstride, counter, out, bid, nb);
  else
    return grid_finish1<NT>(partials, pstride, counter, out, nb);
}

// Single-level tail: the last block to arrive adds each column over all blocks in
// block order (lanes stride the blocks) into out[] and returns true in all of its
// threads; the counter is left at zero.  Used by the binary32 passes of the mixed
// solver, where it measured faster than the two-level tail below.
template <int NT>
__device__ bool grid_finish1(double* __restrict__ partials, int pstride, int* counter, double* out, int nb) {
  constexpr int kWarps = kVecThreads / 32;
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1) == nb - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // warp w adds columns w, w + 8, ...: lanes stride the blocks (coalesced rows of
  // the transposed partials), two columns at a time with independent loads
  for (int i = warp; i < NT; i += 2 * kWarps) {
    const int i2 = i + kWarps;
    const double* p1 = partials + (int64_t)i * pstride;
    const double* p2 = partials + (int64_t)(i2 < NT ? i2 : i) * pstride;
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    int b = lane;
    for (; b + 32 < nb; b += 64) {
      a0 += __ldcg(p1 + b);
      a1 += __ldcg(p1 + b + 32);
      b0 += __ldcg(p2 + b);
      b1 += __ldcg(p2 + b + 32);
    }
    if (b < nb) {
      a0 += __ldcg(p1 + b);
      b0 += __ldcg(p2 + b);
    }
    double ta = a0 + a1, tb = b0 + b1;
    for (int o = 16; o; o >>= 1) {
      ta += __shfl_xor_sync(0xffffffffu, ta, o);
      tb += __shfl_xor_sync(0xffffffffu, tb, o);
    }
    if (lane == 0) {
      out[i] = ta;
      if (i2 < NT) out[i2] = tb;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
  return true;
}

// After every block wrote its NT block sums into column bid of the transposed
// partials: blocks form groups of 32 in index order; the last block of a group to
// arrive adds the group's sums per column (lane = block, fixed butterfly) into the
// second-level rows (after the kPartialRows rows of the partials, kMaxGroups
// apart), and the last group to arrive adds the group sums into out[] (shared
// memory) and returns true in all of its threads.  Two short steps instead of one
// block walking all nb columns: the latency of the tail stays near two L2 round
// trips.  Deterministic for a fixed grid; the counters are left at zero.
template <int NT>
__device__ bool grid_finish(double* __restrict__ partials, int pstride, int* gcount, double* out, int bid, int nb) {
  constexpr int kWarps = kVecThreads / 32;
  __shared__ int stage;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ngroups = (nb + kGroup - 1) / kGroup;
  const int g = bid / kGroup;
  const int gsize = min(kGroup, nb - g * kGroup);
  double* level2 = partials + (int64_t)kPartialRows * pstride;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) stage = (atomicAdd(gcount + 1 + g, 1) == gsize - 1) ? 1 : 0;
  __syncthreads();
  if (!stage) return false;
  __threadfence();
  for (int i = warp; i < NT; i += kWarps) {
    double a = lane < gsize ? __ldcg(partials + (int64_t)i * pstride + g * kGroup + lane) : 0.0;
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) level2[i * kMaxGroups + g] = a;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    gcount[1 + g] = 0;
    stage = (atomicAdd(gcount, 1) == ngroups - 1) ? 2 : 0;
  }
  __syncthreads();
  if (stage != 2) return false;
  __threadfence();
  for (int i = warp; i < NT; i += kWarps) {
    double a = 0.0;
    for (int q = lane; q < ngroups; q += 32) a += __ldcg(level2 + i * kMaxGroups + q);
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[i] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) gcount[0] = 0;
  return true;
}

template <int NV, bool HAS_EXTRA, typename TW>
__device__ __forceinline__ bool grid_sum(TW (&d)[NV], double extra, double* __restrict__ partials, int pstride,
                                         int* counter, double* out) {
  return grid_sum_at<NV, HAS_EXTRA>(d, extra, partials, pstride, counter, out, (int)blockIdx.x, (int)gridDim.x);
}

// Finish Arnoldi step j once beta = ||u_{j+1}|| is final (one thread).
__device__ inline void finish_step(KrylovState* K, int j) {
  double* H = K->H;
  for (int i = 0; i <= j; ++i) H[i * kMaxBasis + j] = K->hc[i];
  const double hn = K->beta;
  H[(j + 1) * kMaxBasis + j] = hn;
  for (int i = 0; i < j; ++i) {  // earlier rotations applied to column j
    const double a = H[i * kMaxBasis + j], b = H[(i + 1) * kMaxBasis + j];
    H[i * kMaxBasis + j] = K->cs[i] * a + K->sn[i] * b;
    H[(i + 1) * kMaxBasis + j] = -K->sn[i] * a + K->cs[i] * b;
  }
  const double a = H[j * kMaxBasis + j], b = H[(j + 1) * kMaxBasis + j];
  const double d = hypot(a, b);
  K->cs[j] = a / d;
  K->sn[j] = b / d;
  H[j * kMaxBasis + j] = d;
  H[(j + 1) * kMaxBasis + j] = 0.0;
  K->e[j + 1] = -K->sn[j] * K->e[j];
  K->e[j] = K->cs[j] * K->e[j];
  K->estimate = fabs(K->e[j + 1]);
  K->sigma[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
  K->it += 1;
  K->jdone = j + 1;
  if (!isfinite(hn) || !(d > 0.0) || !isfinite(d)) K->flags |= kNumeric | kCycleStop | kSolveDone;
  if (K->estimate < K->tol || K->it >= K->maxit || hn == 0.0 || j + 1 == K->m) K->flags |= kCycleStop;
}

// ---- GMRES pass bodies -------------------------------------------------------------

// GMRES (re)start: u_0 = r = b - J theta and beta_0 = ||r||_2; prepares the next
// cycle, or ends the solve when beta_0 < tol or the iteration cap is reached.  The
// policy's values come as binary64, or (TP 16-bit, with 16-bit column offsets from
// cbase) as the exact 16-bit copy of the mixed solver, widened exactly: the same
// binary64 sums either way.
template <bool U, typename T, typename TP = double, typename TC = int32_t>
__device__ __forceinline__ void gm_residual_body(int bid, int nb, const TP* __restrict__ pval,
                                                                   const TC* __restrict__ pcol,
                                                                   const int64_t* __restrict__ poff,
                                                                   const int32_t* __restrict__ plen, int k, int64_t S,
                                                                   double gamma, const double* __restrict__ theta,
                                                                   const double* __restrict__ b,
                                                                   T* __restrict__ u0, double* partials,
                                                                   KrylovState* K,
                                                                   const int32_t* __restrict__ cbase = nullptr) {
  if (K->flags & kSolveDone) return;
  double d[1] = {0.0};
  for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, theta, cbase);
    const double r = b[s] - (theta[s] - gamma * px);
    d[0] = fma(r, r, d[0]);
    u0[s] = (T)r;
  }
  __shared__ double out[1];
  if (grid_sum_at<1, false>(d, 0.0, partials, K->pstride, K->gcount, out, bid, nb) && threadIdx.x == 0) {
    const double beta = sqrt(out[0]);
    K->res2 = beta;
    K->sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    K->e[0] = beta;
    for (int i = 1; i <= kMaxBasis; ++i) K->e[i] = 0.0;
    K->jdone = 0;
    K->flags &= ~(kCycleStop | kReorth);
    if (!isfinite(beta)) K->flags |= kNumeric | kSolveDone;
    if (beta < K->tol || K->it >= K->maxit) K->flags |= kSolveDone;
  }
}

// Arnoldi step, part 1: w = J v_j = sigma_j (u_j - gamma P_pi u_j).  A lean
// kernel (no reductions, few registers) so that enough warps are resident to
// keep the row and gather loads of P_pi in flight.
template <bool U, typename TP, typename T, typename TC = int32_t>
__device__ __forceinline__ void gm_matvec_body(int bid, int nb, const TP* __restrict__ pval,
                                                                 const TC* __restrict__ pcol,
                                                                 const int64_t* __restrict__ poff,
                                                                 const int32_t* __restrict__ plen, int k, int64_t S,
                                                                 double gamma, const T* __restrict__ basis, int j,
                                                                 T* __restrict__ w, const KrylovState* K,
                                                                 const int32_t* __restrict__ cbase = nullptr) {
  if (K->flags & (kCycleStop | kSolveDone)) return;
  const T sj = (T)K->sigma[j];
  const T g = (T)gamma;
  const T* uj = basis + (int64_t)j * S;
  for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
    const T px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, uj, cbase);
    w[s] = sj * (uj[s] - g * px);
  }
}

// Smallest power of two >= n (n <= 32): the width of the warp reduce-scatter for
// NB accumulators.
__host__ __device__ constexpr int pow2_up(int n) { return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32; }

// Two consecutive elements of a vector (16 bytes of binary64, 8 of binary32).
template <typename T> struct Pair2;
template <> struct Pair2<double> { using type = double2; };
template <> struct Pair2<float> { using type = float2; };

// The dots of exactly NA basis vectors with w over this block's states.  In binary64
// with S even (every basis vector then starts on a 16-byte boundary) a thread takes
// two consecutive states per step with one 16-byte load per vector: half the load
// instructions and requests of one state per thread, which the strided streams of
// the basis need to overlap with the FP64 pipe (a microbenchmark at 25 vectors:
// 55 against 72 us, S = 1e6).  The binary32 cycle of the mixed solver keeps one
// state per thread: with pairs there, the mixed solve of the bfloat16-exact pendulum
// grid (10^6 states, gamma = 0.9999) stagnated at a residual of 2.7e-7 through 1000
// outer iterations, where one state per thread converges in about 105.
template <int NA, int NP, typename T>
__device__ __forceinline__ void dots_rows(int bid, int nb, int64_t S, const T* __restrict__ basis,
                                          const T* __restrict__ w, T (&d)[NP]) {
  if (sizeof(T) == sizeof(double) && (S & 1) == 0) {
    using T2 = typename Pair2<T>::type;
    const int64_t S2 = S >> 1;
    const T2* w2 = reinterpret_cast<const T2*>(w);
    for (int64_t p = bid * (int64_t)blockDim.x + threadIdx.x; p < S2; p += (int64_t)nb * blockDim.x) {
      const T2 ws = w2[p];
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const T2 b = reinterpret_cast<const T2*>(basis + (int64_t)i * S)[p];
        d[i] = fma(b.y, ws.y, fma(b.x, ws.x, d[i]));
      }
    }
    return;
  }
  for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
    const T ws = w[s];
#pragma unroll
    for (int i = 0; i < NA; ++i) d[i] = fma(basis[(int64_t)i * S + s], ws, d[i]);
  }
}

// Arnoldi step, part 2: raw dots u_i . w (i <= j) and ||w||^2; the last block
// turns them into the Hessenberg column h_i = v_i . w and the projection
// coefficients.  NB (>= j + 1) is the number of unrolled accumulators: the
// slots above j are predicated off but still issue.  FINE (the FP64 steps
// without re-orthogonalisation): NB is the smallest multiple of 4 that holds
// j + 1, and a uniform switch runs exactly j + 1 products per state, without
// ||w|| (read only by the re-orthogonalising modes).  Per thread each dot is the
// same chain of FMAs either way; the grid follows the kernel's occupancy, so the
// states a thread sums (and the last bits of the sums) depend on the variant, and
// the batched solver launches the same variant with the same grid.
template <int NB, typename T, bool FINE = false>
__device__ __forceinline__ void gm_dots_body(int bid, int nb, int64_t S, const T* __restrict__ basis, int j,
                                                               const T* __restrict__ w, double* partials,
                                                               KrylovState* K) {
  constexpr int NP = pow2_up(NB);
  if (K->flags & (kCycleStop | kSolveDone)) return;
  T d[NP];
  T ww = T(0);
#pragma unroll
  for (int i = 0; i < NP; ++i) d[i] = T(0);
  if constexpr (FINE) {
    static_assert(NB % 4 == 0, "fine widths are multiples of 4");
    switch (j + 1 - (NB - 4)) {  // 1..4: the caller picks NB from j
      case 1: dots_rows<NB - 3>(bid, nb, S, basis, w, d); break;
      case 2: dots_rows<NB - 2>(bid, nb, S, basis, w, d); break;
      case 3: dots_rows<NB - 1>(bid, nb, S, basis, w, d); break;
      default: dots_rows<NB>(bid, nb, S, basis, w, d); break;
    }
    __shared__ double fout[NP];
    if (grid_sum_at<NP, false>(d, 0.0, partials, K->pstride, K->gcount, fout, bid, nb) && threadIdx.x == 0) {
      for (int i = 0; i <= j; ++i) {
        const double h = K->sigma[i] * fout[i];
        K->hc[i] = h;
        K->coef[i] = h * K->sigma[i];
      }
      K->wnorm = 0.0;
    }
  } else {
    for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
      const T ws = w[s];
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i <= j) d[i] = fma(basis[(int64_t)i * S + s], ws, d[i]);
      ww = fma(ws, ws, ww);
    }
    __shared__ double out[NP + 1];  // warp sums in T, block and grid sums in double
    if (grid_sum_at<NP, true>(d, (double)ww, partials, K->pstride, K->gcount, out, bid, nb) && threadIdx.x == 0) {
      for (int i = 0; i <= j; ++i) {
        const double h = K->sigma[i] * out[i];
        K->hc[i] = h;
        K->coef[i] = h * K->sigma[i];
      }
      K->wnorm = sqrt(out[NP]);
    }
  }
}

// Arnoldi step of the binary64 solver with single-pass classical Gram-Schmidt, parts 1
// and 2 in one pass: w = J v_j = sigma_j (u_j - gamma P_pi u_j), written for the
// projection, and the raw dots u_i . w (i <= j) while w is still in a register, so w is
// not read back and one launch and its gap are saved per step.  w equals the
// separate mat-vec's bit for bit; the dots are sums of the same products grouped by
// this kernel's grid.  Exactly j + 1 products per state (NB as in gm_dots_body's FINE
// widths).  The last block turns the sums into the Hessenberg column and the
// projection coefficients.
template <int NA, bool U, int NP>
__device__ __forceinline__ void matvec_dots_rows(int bid, int nb, const double* __restrict__ pval,
                                                 const int32_t* __restrict__ pcol, const int64_t* __restrict__ poff,
                                                 const int32_t* __restrict__ plen, int k, int64_t S, double g,
                                                 double sj, const double* __restrict__ basis,
                                                 const double* __restrict__ uj, double* __restrict__ w,
                                                 double (&d)[NP]) {
  for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, uj);
    const double ws = sj * (uj[s] - g * px);
    w[s] = ws;
#pragma unroll
    for (int i = 0; i < NA; ++i) d[i] = fma(basis[(int64_t)i * S + s], ws, d[i]);
  }
}

// Blocks per SM the fused kernel's register budget is sized for: its row gathers want
// many resident warps, its NB accumulators want registers.  A microbenchmark at
// S = 1e6 put 13 products per state about level at 2 and 4 blocks per SM and 25
// products best at 2; the narrowest widths are mostly the mat-vec, which runs best
// with many warps.
__host__ __device__ constexpr int mvd_min_blocks(int NB) { return NB <= 8 ? 4 : NB <= 16 ? 3 : 2; }

template <bool U, int NB>
__device__ __forceinline__ void gm_matvec_dots_body(int bid, int nb, const double* __restrict__ pval,
                                                    const int32_t* __restrict__ pcol,
                                                    const int64_t* __restrict__ poff,
                                                    const int32_t* __restrict__ plen, int k, int64_t S,
                                                    double gamma, const double* __restrict__ basis, int j,
                                                    double* __restrict__ w, double* partials, KrylovState* K) {
  static_assert(NB % 4 == 0, "fine widths are multiples of 4");
  constexpr int NP = pow2_up(NB);
  if (K->flags & (kCycleStop | kSolveDone)) return;
  const double sj = K->sigma[j];
  const double* uj = basis + (int64_t)j * S;
  double d[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) d[i] = 0.0;
  switch (j + 1 - (NB - 4)) {  // 1..4: the caller picks NB from j
    case 1: matvec_dots_rows<NB - 3, U>(bid, nb, pval, pcol, poff, plen, k, S, gamma, sj, basis, uj, w, d); break;
    case 2: matvec_dots_rows<NB - 2, U>(bid, nb, pval, pcol, poff, plen, k, S, gamma, sj, basis, uj, w, d); break;
    case 3: matvec_dots_rows<NB - 1, U>(bid, nb, pval, pcol, poff, plen, k, S, gamma, sj, basis, uj, w, d); break;
    default: matvec_dots_rows<NB, U>(bid, nb, pval, pcol, poff, plen, k, S, gamma, sj, basis, uj, w, d); break;
  }
  __shared__ double fout[NP];
  if (grid_sum_at<NP, false>(d, 0.0, partials, K->pstride, K->gcount, fout, bid, nb) && threadIdx.x == 0) {
    for (int i = 0; i <= j; ++i) {
      const double h = K->sigma[i] * fout[i];
      K->hc[i] = h;
      K->coef[i] = h * K->sigma[i];
    }
    K->wnorm = 0.0;
  }
}

// Arnoldi projection passes.  First pass (MODE = kPlain, kDgks or kAlways):
// u_{j+1} = w - sum_i coef_i u_i and ||u_{j+1}||^2; kDgks and kAlways also form
// the raw dots u_i . u_{j+1} that a second classical Gram-Schmidt pass needs.
// The last block then finishes the step, or (kAlways; kDgks when the norm fell
// below 1/sqrt(2) of ||w||) turns the dots into corrections and requests the
// second pass (MODE = kSecond): u_{j+1} -= sum_i coef_i u_i, ||u_{j+1}||^2, finish.
enum { kPlain = 0, kDgks = 1, kAlways = 2, kSecond = 3 };

// The projection keeps every basis load of a state in flight (up to 2 (j + 1)
// registers) and the compiler takes up to 128 registers, two blocks per SM; a cap
// of 64 (four blocks) trades a few spills for twice the warps and measured 4%
// faster on the whole FP64 solve.
constexpr int kProjectMinBlocks = 3;

// u = src - sum of exactly NA coefficient-scaled basis vectors over this block's
// states; returns this thread's share of ||u||^2.  With S even, two consecutive
// states per step as in dots_rows: two independent chains of fused multiply-adds
// (each state's chain is the same as with one state per thread) and 16-byte loads
// (a microbenchmark at 25 vectors: 53 against 100 us, S = 1e6).
template <int NA, typename T>
__device__ __forceinline__ T project_rows(int bid, int nb, int64_t S, const T* __restrict__ basis,
                                          const T* __restrict__ src, T* __restrict__ u, const T* c) {
  T uu = T(0);
  if (sizeof(T) == sizeof(double) && (S & 1) == 0) {
    using T2 = typename Pair2<T>::type;
    const int64_t S2 = S >> 1;
    for (int64_t p = bid * (int64_t)blockDim.x + threadIdx.x; p < S2; p += (int64_t)nb * blockDim.x) {
      T2 x = reinterpret_cast<const T2*>(src)[p];
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const T2 b = reinterpret_cast<const T2*>(basis + (int64_t)i * S)[p];
        x.x = fma(-c[i], b.x, x.x);
        x.y = fma(-c[i], b.y, x.y);
      }
      reinterpret_cast<T2*>(u)[p] = x;
      uu = fma(x.x, x.x, uu);
      uu = fma(x.y, x.y, uu);
    }
    return uu;
  }
  for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
    T x = src[s];
#pragma unroll
    for (int i = 0; i < NA; ++i) x = fma(-c[i], basis[(int64_t)i * S + s], x);
    u[s] = x;
    uu = fma(x, x, uu);
  }
  return uu;
}

template <int NB, int MODE, typename T, bool FINE = false>
__device__ __forceinline__ void gm_project_body(int bid, int nb, int64_t S, T* __restrict__ basis, int j,
                                                                  const T* __restrict__ w, double* partials,
                                                                  KrylovState* K) {
  constexpr bool SECOND = (MODE == kSecond);
  constexpr bool DOTS = (MODE == kDgks || MODE == kAlways);
  static_assert(!FINE || MODE == kPlain, "fine widths are for the single-pass projection");
  if (K->flags & (kCycleStop | kSolveDone)) return;
  if (SECOND && !(K->flags & kReorth)) return;
  __shared__ T c[NB];
  if (threadIdx.x < NB) c[threadIdx.x] = ((int)threadIdx.x <= j) ? (T)K->coef[threadIdx.x] : T(0);
  __syncthreads();
  T* u = basis + (int64_t)(j + 1) * S;
  const T* src = SECOND ? u : w;
  if constexpr (FINE) {
    // as gm_dots_body: exactly j + 1 terms per state, in the order of the predicated loop
    T uu = T(0);
    switch (j + 1 - (NB - 4)) {
      case 1: uu = project_rows<NB - 3>(bid, nb, S, basis, src, u, c); break;
      case 2: uu = project_rows<NB - 2>(bid, nb, S, basis, src, u, c); break;
      case 3: uu = project_rows<NB - 1>(bid, nb, S, basis, src, u, c); break;
      default: uu = project_rows<NB>(bid, nb, S, basis, src, u, c); break;
    }
    T n1[1] = {uu};
    __shared__ double fout[1];
    if (grid_sum_at<1, false>(n1, 0.0, partials, K->pstride, K->gcount, fout, bid, nb) && threadIdx.x == 0) {
      K->beta = sqrt(fout[0]);
      K->flags &= ~kReorth;
      finish_step(K, j);
    }
  } else {
    constexpr int NV = DOTS ? pow2_up(NB) : 1;  // dots u_i . u_{j+1} (first pass with dots); ||u||^2 goes last
    T d[NV];
    T uu = T(0);
#pragma unroll
    for (int i = 0; i < NV; ++i) d[i] = T(0);
    for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
      T x = src[s];
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i <= j) x = fma(-c[i], basis[(int64_t)i * S + s], x);
      u[s] = x;
      uu = fma(x, x, uu);
      if (DOTS) {
#pragma unroll
        for (int i = 0; i < NB; ++i)
          if (i <= j) d[i] = fma(basis[(int64_t)i * S + s], x, d[i]);
      }
    }
    __shared__ double out[NV + 1];
    bool last;
    if (DOTS) {
      last = grid_sum_at<NV, true>(d, (double)uu, partials, K->pstride, K->gcount, out, bid, nb);
    } else {
      T n1[1] = {uu};
      last = grid_sum_at<1, false>(n1, 0.0, partials, K->pstride, K->gcount, out, bid, nb);
    }
    if (last && threadIdx.x == 0) {
      const double beta = sqrt(out[DOTS ? NV : 0]);
      K->beta = beta;
      const bool again = (MODE == kAlways && beta > 0.0) ||
                         (MODE == kDgks && beta > 0.0 && beta < 0.70710678118654752 * K->wnorm);
      if (again) {
        for (int i = 0; i <= j; ++i) {
          const double h2 = K->sigma[i] * out[i];
          K->hc[i] += h2;
          K->coef[i] = h2 * K->sigma[i];
        }
        K->flags |= kReorth;
      } else {
        K->flags &= ~kReorth;
        finish_step(K, j);
      }
    }
  }
}

// theta += sum_{i < jdone} y_i v_i, where every block solves R y = e by back
// substitution.  The correction is accumulated in the basis type (binary32 in
// the mixed solver, whose corrections only need that precision) and added to
// theta in binary64.
template <typename T>
__device__ __forceinline__ void gm_update_body(int bid, int nb, int64_t S, const T* __restrict__ basis,
                                                                 double* __restrict__ theta, KrylovState* K) {
  if (K->flags & kSolveDone) return;
  __shared__ T c[kMaxBasis];
  const int n = K->jdone;
  if (threadIdx.x == 0) {
    double y[kMaxBasis];
    for (int i = n - 1; i >= 0; --i) {
      double t = K->e[i];
      for (int q = i + 1; q < n; ++q) t -= K->H[i * kMaxBasis + q] * y[q];
      y[i] = t / K->H[i * kMaxBasis + i];
    }
    for (int i = 0; i < n; ++i) c[i] = (T)(y[i] * K->sigma[i]);
  }
  __syncthreads();
  for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
    T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);
    int i = 0;
    for (; i + 4 <= n; i += 4) {
      t0 = fma(c[i], basis[(int64_t)i * S + s], t0);
      t1 = fma(c[i + 1], basis[(int64_t)(i + 1) * S + s], t1);
      t2 = fma(c[i + 2], basis[(int64_t)(i + 2) * S + s], t2);
      t3 = fma(c[i + 3], basis[(int64_t)(i + 3) * S + s], t3);
    }
    for (; i < n; ++i) t0 = fma(c[i], basis[(int64_t)i * S + s], t0);
    theta[s] += (double)((t0 + t1) + (t2 + t3));
  }
}

}  // namespace mdp
