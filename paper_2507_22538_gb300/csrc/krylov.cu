// Inexact policy evaluation (Algorithm 1 steps 6-12): the matrix-free operator
// J_pi x = x - gamma P_pi x (Sec. III-B.3) over the policy's rows, and the inner
// solvers: Richardson (theta += omega (g_pi - J_pi theta)), Jacobi-Richardson,
// TFQMR (Freund 1993) and restarted GMRES(m) (Saad, Iterative Methods for Sparse
// Linear Systems, Sec. 6.5).
//
// GMRES runs a whole restart cycle without the host: classical Gram-Schmidt
// (one pass by default, PETSc's choice; optionally a second pass when the DGKS
// test asks for it -- Daniel, Gragg, Kaufman and Stewart, Math. Comp. 1976:
// re-orthogonalise when the norm after projection falls below 1/sqrt(2) of the
// norm before -- or always), the Givens rotations, the residual estimate and the
// stop test all on the device.  Each kernel
// reduces its dot products in its last finishing block (fixed order, so
// results are deterministic) and checks device flags on entry, so steps queued
// after the stop test fired return at once.  The host waits once per cycle.
//
// Basis vectors are stored unnormalised (u_i) with scales sigma_i (v_i =
// sigma_i u_i); the scales are folded into the projection coefficients, so no
// pass rescales a vector.
//
// Every pass is one thread per state over the per-state sliced layout of P_pi
// (lanes = consecutive states: values, columns and vector entries load
// coalesced; only x[col] is a gather).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "krylov_dev.cuh"

namespace mdp {

// ---- kernels ---------------------------------------------------------------------

// y = x - gamma P_pi x (states whose policy entry was invalid carry g_pi = NaN and get NaN)
template <bool U>
__global__ void __launch_bounds__(kVecThreads) policy_apply_kernel(const double* __restrict__ pval,
                                                                    const int32_t* __restrict__ pcol,
                                                                    const int64_t* __restrict__ poff,
                                                                    const int32_t* __restrict__ plen, int k, int64_t S,
                                                                    double gamma, const double* __restrict__ x,
                                                                    const double* __restrict__ gpi,
                                                                    double* __restrict__ y) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, x);
    const double gv = gpi[s];
    y[s] = (gv != gv) ? gv : x[s] - gamma * px;
  }
}

// GMRES passes (bodies in krylov_dev.cuh), one problem per launch.
template <bool U, typename T, typename TP = double, typename TC = int32_t>
__global__ void __launch_bounds__(kVecThreads) gm_residual_kernel(const TP* __restrict__ pval,
                                                                   const TC* __restrict__ pcol,
                                                                   const int64_t* __restrict__ poff,
                                                                   const int32_t* __restrict__ plen, int k, int64_t S,
                                                                   double gamma, const double* __restrict__ theta,
                                                                   const double* __restrict__ b,
                                                                   T* __restrict__ u0, double* partials,
                                                                   KrylovState* K, const int32_t* __restrict__ cbase) {
  pdl_begin();
  gm_residual_body<U, T, TP, TC>((int)blockIdx.x, (int)gridDim.x, pval, pcol, poff, plen, k, S, gamma, theta, b, u0,
                                 partials, K, cbase);
}

template <bool U, typename TP, typename T, typename TC = int32_t>
__global__ void __launch_bounds__(kVecThreads) gm_matvec_kernel(const TP* __restrict__ pval,
                                                                 const TC* __restrict__ pcol,
                                                                 const int64_t* __restrict__ poff,
                                                                 const int32_t* __restrict__ plen, int k, int64_t S,
                                                                 double gamma, const T* __restrict__ basis, int j,
                                                                 T* __restrict__ w, const KrylovState* K,
                                                                 const int32_t* __restrict__ cbase) {
  pdl_begin();
  gm_matvec_body<U, TP, T, TC>((int)blockIdx.x, (int)gridDim.x, pval, pcol, poff, plen, k, S, gamma, basis, j, w, K,
                               cbase);
}

template <int NB, typename T, bool FINE>
__global__ void __launch_bounds__(kVecThreads) gm_dots_kernel(int64_t S, const T* __restrict__ basis, int j,
                                                               const T* __restrict__ w, double* partials,
                                                               KrylovState* K) {
  pdl_begin();
  gm_dots_body<NB, T, FINE>((int)blockIdx.x, (int)gridDim.x, S, basis, j, w, partials, K);
}

// The binary64 mat-vec fused with the dots (single-pass classical Gram-Schmidt): one
// launch per step instead of two, and w not read back.  A microbenchmark of the two
// against the fused kernel at S = 1e6 (13 and 25 basis vectors): 120 -> 101 us and
// 144 -> 121 us.
template <bool U, int NB>
__global__ void __launch_bounds__(kVecThreads, mvd_min_blocks(NB)) gm_matvec_dots_kernel(const double* __restrict__ pval,
                                                                       const int32_t* __restrict__ pcol,
                                                                       const int64_t* __restrict__ poff,
                                                                       const int32_t* __restrict__ plen, int k,
                                                                       int64_t S, double gamma,
                                                                       const double* __restrict__ basis, int j,
                                                                       double* __restrict__ w, double* partials,
                                                                       KrylovState* K) {
  pdl_begin();
  gm_matvec_dots_body<U, NB>((int)blockIdx.x, (int)gridDim.x, pval, pcol, poff, plen, k, S, gamma, basis, j, w,
                             partials, K);
}

// The binary32 dots pass (mixed solver) at 4 blocks per SM (64 registers): measured
// 110.9 -> 107.1 ms per mixed solve.  The FP64 pass keeps the compiler's choice
// (80 registers, 3 blocks), faster there (147.8 against 150.3 ms at 4 blocks).
template <int NB, bool FINE>
__global__ void __launch_bounds__(kVecThreads, 4) gm_dots32_kernel(int64_t S, const float* __restrict__ basis, int j,
                                                                   const float* __restrict__ w, double* partials,
                                                                   KrylovState* K) {
  pdl_begin();
  gm_dots_body<NB, float, FINE>((int)blockIdx.x, (int)gridDim.x, S, basis, j, w, partials, K);
}

// The dots kernel of value type T.
template <int NB, typename T, bool FINE>
constexpr auto dots_kernel() {
  if constexpr (sizeof(T) == sizeof(float))
    return gm_dots32_kernel<NB, FINE>;
  else
    return gm_dots_kernel<NB, T, FINE>;
}

template <int NB, int MODE, typename T, bool FINE>
__global__ void __launch_bounds__(kVecThreads, kProjectMinBlocks) gm_project_kernel(int64_t S, T* __restrict__ basis, int j,
                                                                  const T* __restrict__ w, double* partials,
                                                                  KrylovState* K) {
  pdl_begin();
  gm_project_body<NB, MODE, T, FINE>((int)blockIdx.x, (int)gridDim.x, S, basis, j, w, partials, K);
}

template <typename T>
__global__ void __launch_bounds__(kVecThreads) gm_update_kernel(int64_t S, const T* __restrict__ basis,
                                                                 double* __restrict__ theta, KrylovState* K) {
  pdl_begin();
  gm_update_body<T>((int)blockIdx.x, (int)gridDim.x, S, basis, theta, K);
}

// One Richardson step from buffer `in`: r = b - J in, out = in + omega r, ||r||_2.
// The last block ends the solve when ||r|| < tol (the answer is then `in`) or
// when the step cap is reached (the answer is `out`).
template <bool U>
__global__ void __launch_bounds__(kVecThreads) rich_step_kernel(const double* __restrict__ pval,
                                                                 const int32_t* __restrict__ pcol,
                                                                 const int64_t* __restrict__ poff,
                                                                 const int32_t* __restrict__ plen, int k, int64_t S,
                                                                 double gamma, double omega,
                                                                 const double* __restrict__ in,
                                                                 const double* __restrict__ b,
                                                                 double* __restrict__ out, int in_index,
                                                                 double* partials, KrylovState* K) {
  if (K->flags & kSolveDone) return;
  double d[1] = {0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, in);
    const double th = in[s];
    const double r = b[s] - (th - gamma * px);
    d[0] = fma(r, r, d[0]);
    out[s] = fma(omega, r, th);
  }
  __shared__ double o[1];
  if (grid_sum<1, false>(d, 0.0, partials, K->pstride, K->gcount, o) && threadIdx.x == 0) {
    const double rn = sqrt(o[0]);
    K->res2 = rn;
    if (!isfinite(rn)) {
      K->flags |= kNumeric | kSolveDone;
      K->result = in_index;
    } else if (rn < K->tol) {
      K->flags |= kSolveDone;
      K->result = in_index;
    } else {
      K->it += 1;
      K->result = 1 - in_index;
      if (K->it >= K->maxit) K->flags |= kSolveDone;
    }
  }
}

// ---- TFQMR (Freund 1993) -------------------------------------------------------------
// Vectors (FP64, S each): rt (shadow residual r_0), w, y1, y2, u1 = J y1, u2 = J y2,
// v, d.  One half step (one product by J) is one iteration; it counts in K->it.

// r_0 = b - J x; rt = w = y1 = r_0; d = 0; tau = ||r_0||, rho = r_0 . r_0.
template <bool U>
__global__ void __launch_bounds__(kVecThreads) tf_init_kernel(const double* __restrict__ pval,
                                                               const int32_t* __restrict__ pcol,
                                                               const int64_t* __restrict__ poff,
                                                               const int32_t* __restrict__ plen, int k, int64_t S,
                                                               double gamma, const double* __restrict__ x,
                                                               const double* __restrict__ b, double* __restrict__ rt,
                                                               double* __restrict__ w, double* __restrict__ y1,
                                                               double* __restrict__ d, double* partials,
                                                               KrylovState* K) {
  double acc[1] = {0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, x);
    const double r = b[s] - (x[s] - gamma * px);
    rt[s] = r;
    w[s] = r;
    y1[s] = r;
    d[s] = 0.0;
    acc[0] = fma(r, r, acc[0]);
  }
  __shared__ double out[1];
  if (grid_sum<1, false>(acc, 0.0, partials, K->pstride, K->gcount, out) && threadIdx.x == 0) {
    const double tau = sqrt(out[0]);
    K->t_tau = tau;
    K->t_rho = out[0];
    K->t_theta = 0.0;
    K->t_eta = 0.0;
    K->res2 = tau;
    if (!isfinite(tau)) K->flags |= kNumeric | kSolveDone;
    if (tau < K->tol || K->maxit <= 0) K->flags |= kSolveDone;
  }
}

// y = J x with, optionally, v = y + beta (u2 + beta v) (TFQMR's v update) and u1 = y.
template <bool U, bool VUPD>
__global__ void __launch_bounds__(kVecThreads) tf_matvec_kernel(const double* __restrict__ pval,
                                                                 const int32_t* __restrict__ pcol,
                                                                 const int64_t* __restrict__ poff,
                                                                 const int32_t* __restrict__ plen, int k, int64_t S,
                                                                 double gamma, const double* __restrict__ x,
                                                                 double* __restrict__ y, const double* __restrict__ u2,
                                                                 double* __restrict__ v, const KrylovState* K) {
  if (K->flags & kSolveDone) return;
  const double beta = K->t_beta;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, x);
    const double ys = x[s] - gamma * px;
    y[s] = ys;
    if (VUPD) v[s] = fma(beta, fma(beta, v[s], u2[s]), ys);
  }
}

// sigma = rt . v; alpha = rho / sigma (a zero sigma or rho ends the solve).
__global__ void __launch_bounds__(kVecThreads) tf_sigma_kernel(int64_t S, const double* __restrict__ rt,
                                                                const double* __restrict__ v, double* partials,
                                                                KrylovState* K) {
  if (K->flags & kSolveDone) return;
  double acc[1] = {0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x)
    acc[0] = fma(rt[s], v[s], acc[0]);
  __shared__ double out[1];
  if (grid_sum<1, false>(acc, 0.0, partials, K->pstride, K->gcount, out) && threadIdx.x == 0) {
    const double sigma = out[0];
    if (sigma == 0.0 || K->t_rho == 0.0 || !isfinite(sigma)) {
      K->flags |= kSolveDone;
      if (!isfinite(sigma)) K->flags |= kNumeric;
    } else {
      K->t_alpha = K->t_rho / sigma;
    }
  }
}

// out = a + coef * b with coef = -alpha (y2 = y1 - alpha v) or beta (y1 = w + beta y2).
template <bool MINUS_ALPHA>
__global__ void __launch_bounds__(kVecThreads) tf_axpy_kernel(int64_t S, const double* __restrict__ a,
                                                               const double* __restrict__ b, double* __restrict__ out,
                                                               const KrylovState* K) {
  if (K->flags & kSolveDone) return;
  const double c = MINUS_ALPHA ? -K->t_alpha : K->t_beta;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x)
    out[s] = fma(c, b[s], a[s]);
}

// One quasi-minimal-residual half step: w -= alpha u; d = y + (theta^2 eta / alpha) d;
// then theta = ||w|| / tau, c = (1 + theta^2)^(-1/2), tau *= theta c, eta = c^2 alpha,
// one more iteration, and the stop test tau sqrt(it + 1) < tol (or the cap).
__global__ void __launch_bounds__(kVecThreads) tf_half_kernel(int64_t S, const double* __restrict__ y,
                                                               const double* __restrict__ u, double* __restrict__ w,
                                                               double* __restrict__ d, double* partials,
                                                               KrylovState* K) {
  if (K->flags & kSolveDone) return;
  const double alpha = K->t_alpha;
  const double cd = K->t_theta * K->t_theta * K->t_eta / alpha;
  double acc[1] = {0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double ws = fma(-alpha, u[s], w[s]);
    w[s] = ws;
    d[s] = fma(cd, d[s], y[s]);
    acc[0] = fma(ws, ws, acc[0]);
  }
  __shared__ double out[1];
  if (grid_sum<1, false>(acc, 0.0, partials, K->pstride, K->gcount, out) && threadIdx.x == 0) {
    const double theta = sqrt(out[0]) / K->t_tau;
    const double c = 1.0 / sqrt(1.0 + theta * theta);
    K->t_theta = theta;
    K->t_tau = K->t_tau * theta * c;
    K->t_eta = c * c * alpha;
    K->it += 1;
    K->jdone = K->it;  // the x update that follows checks this
    if (!isfinite(K->t_tau)) K->flags |= kNumeric | kSolveDone;
    if (K->t_tau * sqrt((double)K->it + 1.0) < K->tol || K->it >= K->maxit) K->flags |= kSolveDone;
  }
}

// x += eta d for half step number `half` (skipped when that half step did not run);
// with RHO also rho_new = rt . w, beta = rho_new / rho (a zero rho ends the solve).
template <bool RHO>
__global__ void __launch_bounds__(kVecThreads) tf_xupd_kernel(int64_t S, int half, const double* __restrict__ d,
                                                               double* __restrict__ x, const double* __restrict__ rt,
                                                               const double* __restrict__ w, double* partials,
                                                               KrylovState* K) {
  const bool apply = (K->jdone == half);
  if (!apply && (!RHO || (K->flags & kSolveDone))) return;
  const double eta = K->t_eta;
  const bool rho = RHO && !(K->flags & kSolveDone);
  double acc[1] = {0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    if (apply) x[s] = fma(eta, d[s], x[s]);
    if (rho) acc[0] = fma(rt[s], w[s], acc[0]);
  }
  if (!rho) return;
  __shared__ double out[1];
  if (grid_sum<1, false>(acc, 0.0, partials, K->pstride, K->gcount, out) && threadIdx.x == 0) {
    const double rn = out[0];
    if (rn == 0.0 || !isfinite(rn)) {
      K->flags |= kSolveDone;
      if (!isfinite(rn)) K->flags |= kNumeric;
    } else {
      K->t_beta = rn / K->t_rho;
      K->t_rho = rn;
    }
  }
}

// ||b - J x||_2 of the returned iterate into K->res2.
template <bool U>
__global__ void __launch_bounds__(kVecThreads) true_residual_kernel(const double* __restrict__ pval,
                                                                     const int32_t* __restrict__ pcol,
                                                                     const int64_t* __restrict__ poff,
                                                                     const int32_t* __restrict__ plen, int k,
                                                                     int64_t S, double gamma,
                                                                     const double* __restrict__ x,
                                                                     const double* __restrict__ b, double* partials,
                                                                     KrylovState* K) {
  double acc[1] = {0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, x);
    const double r = b[s] - (x[s] - gamma * px);
    acc[0] = fma(r, r, acc[0]);
  }
  __shared__ double out[1];
  if (grid_sum<1, false>(acc, 0.0, partials, K->pstride, K->gcount, out) && threadIdx.x == 0) {
    K->res2 = sqrt(out[0]);
    if (!isfinite(K->res2)) K->flags |= kNumeric;
  }
}

// One Jacobi-preconditioned Richardson step (J-VI, Table 2): r = b - J in,
// out = in + omega r / (1 - gamma P(s, s, pi(s))).  Stop logic as rich_step_kernel.
template <bool U>
__global__ void __launch_bounds__(kVecThreads) jacobi_step_kernel(const double* __restrict__ pval,
                                                                   const int32_t* __restrict__ pcol,
                                                                   const int64_t* __restrict__ poff,
                                                                   const int32_t* __restrict__ plen, int k, int64_t S,
                                                                   double gamma, double omega,
                                                                   const double* __restrict__ pdiag,
                                                                   const double* __restrict__ in,
                                                                   const double* __restrict__ b,
                                                                   double* __restrict__ out, int in_index,
                                                                   double* partials, KrylovState* K) {
  if (K->flags & kSolveDone) return;
  double acc[1] = {0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, in);
    const double th = in[s];
    const double r = b[s] - (th - gamma * px);
    acc[0] = fma(r, r, acc[0]);
    out[s] = th + omega * r / (1.0 - gamma * pdiag[s]);
  }
  __shared__ double o[1];
  if (grid_sum<1, false>(acc, 0.0, partials, K->pstride, K->gcount, o) && threadIdx.x == 0) {
    const double rn = sqrt(o[0]);
    K->res2 = rn;
    if (!isfinite(rn)) {
      K->flags |= kNumeric | kSolveDone;
      K->result = in_index;
    } else if (rn < K->tol) {
      K->flags |= kSolveDone;
      K->result = in_index;
    } else {
      K->it += 1;
      K->result = 1 - in_index;
      if (K->it >= K->maxit) K->flags |= kSolveDone;
    }
  }
}

// P(s, s, pi(s)): the self-transition entry of each policy row (0 when absent).
template <bool U>
__global__ void __launch_bounds__(kVecThreads) policy_diag_kernel(const double* __restrict__ pval,
                                                                   const int32_t* __restrict__ pcol,
                                                                   const int64_t* __restrict__ poff,
                                                                   const int32_t* __restrict__ plen, int k, int64_t S,
                                                                   double* __restrict__ pdiag) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = s / kSlice;
    const int n = U ? k : plen[s];
    const int w = U ? k : (int)((poff[q + 1] - poff[q]) / kSlice);
    const int64_t base = U ? q * kSlice * (int64_t)k : poff[q];
    double p = 0.0;
    for (int j = 0; j < n; ++j) {
      const int64_t i = sell_at(base, w, (int)(s % kSlice), j);
      if (pcol[i] == (int32_t)s) p += pval[i];
    }
    pdiag[s] = p;
  }
}

// ---- host side -------------------------------------------------------------------

#define MDP_LAUNCH_CHECK(h)       \
  do {                            \
    (h)->launches++;              \
    MDP_CUDA(cudaGetLastError()); \
  } while (0)

static KrylovState* kstate(mdp_s* h) { return (KrylovState*)h->kstate; }

// Grid of one full wave: as many 256-thread blocks as fit on every SM at once
// (from the occupancy calculator, cached per kernel), but no more blocks than
// 256-state chunks.  A partial second wave would leave most SMs idle for as long
// as the first.
template <typename Kern>
static int wave_grid(mdp_s* h, Kern kernel, int max_per_sm = kMaxBlocksPerSm) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find((const void*)kernel);
    if (it != cache.end()) {
      per_sm = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kVecThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
      }
      per_sm = std::max(1, std::min(per_sm, kMaxBlocksPerSm));
      cache[(const void*)kernel] = per_sm;
    }
  }
  const int64_t chunks = (h->S + kVecThreads - 1) / kVecThreads;
  const int64_t wave = std::min<int64_t>((int64_t)h->sm_count * std::min(per_sm, max_per_sm), h->partial_stride);
  return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, wave));
}

#define MDP_WAVE(kern) wave_grid(h, kern)  // kern in parentheses when it has template commas


// Zero the device state and set tol, maxit and m (through the pinned scratch).
static mdp_status init_state(mdp_s* h, double tol, int maxit, int m, cudaStream_t st) {
  KrylovState* K = kstate(h);
  double* pin = tls_pinned();
  MDP_CUDA(cudaMemsetAsync(K, 0, sizeof(KrylovState), st));
  pin[32] = tol;
  KrylovHeader hd{0, maxit, m, 0, 0, 0, 0, h->partial_stride};
  std::memcpy(pin + 34, &hd, sizeof(hd));
  MDP_CUDA(cudaMemcpyAsync(&K->tol, pin + 32, sizeof(double), cudaMemcpyHostToDevice, st));
  MDP_CUDA(cudaMemcpyAsync(&K->it, pin + 34, sizeof(hd), cudaMemcpyHostToDevice, st));
  MDP_CUDA(cudaStreamSynchronize(st));  // the pinned words are reused by the next call
  return MDP_OK;
}

static mdp_status read_header(mdp_s* h, KrylovHeader* out, double* res2, cudaStream_t st) {
  KrylovState* K = kstate(h);
  double* pin = tls_pinned();
  MDP_CUDA(cudaMemcpyAsync(pin + 40, &K->it, sizeof(KrylovHeader), cudaMemcpyDeviceToHost, st));
  MDP_CUDA(cudaMemcpyAsync(pin + 48, &K->res2, sizeof(double), cudaMemcpyDeviceToHost, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  std::memcpy(out, pin + 40, sizeof(KrylovHeader));
  *res2 = pin[48];
  return MDP_OK;
}

// Typed views of the Krylov workspace: FP64 (policy rows, basis and w in double)
// or mixed (FP32 copies of the policy rows, FP32 basis and w; the residual at
// each restart and the iterate theta stay FP64).
template <typename T>
struct KrylovBuffers {
  const void* pval;  // double (FP64 solver); float, binary16 or bfloat16 per h->pstore (mixed solver)
  T* basis;
  T* w;
};

static KrylovBuffers<double> buffers(mdp_s* h, double*) { return {h->Ppi.val, h->basis, h->w}; }
static KrylovBuffers<float> buffers(mdp_s* h, float*) {
  return {h->pstore == kStoreF32 ? (const void*)h->pval32 : (const void*)h->pval16, h->basis32, h->w32};
}

// The mat-vec of an Arnoldi step with policy values of type TP; the binary32 cycle of an
// MDP whose rows span at most 32767 columns reads 16-bit values with 16-bit column
// offsets (4 instead of 6 bytes per entry), with the same products and sums.
template <bool U, typename TP, typename T>
static mdp_status launch_matvec_as(mdp_s* h, const KrylovBuffers<T>& B, double gamma, int j, cudaStream_t st) {
  const Sell& Q = h->Ppi;
  const int k = U ? Q.kmax : 0;
  KrylovState* K = kstate(h);
  if constexpr (sizeof(T) == sizeof(float) && sizeof(TP) == 2) {
    if (h->pcol16) {
      MDP_CUDA(launch_pdl(gm_matvec_kernel<U, TP, T, int16_t>, MDP_WAVE((gm_matvec_kernel<U, TP, T, int16_t>)),
                          kVecThreads, 0, st, (const TP*)B.pval, (const int16_t*)h->pcol16, Q.off, Q.len, k, h->S,
                          gamma, B.basis, j, B.w, K, (const int32_t*)h->pcolbase));
      return MDP_OK;
    }
  }
  MDP_CUDA(launch_pdl(gm_matvec_kernel<U, TP, T>, MDP_WAVE((gm_matvec_kernel<U, TP, T>)), kVecThreads, 0, st,
                      (const TP*)B.pval, Q.col, Q.off, Q.len, k, h->S, gamma, B.basis, j, B.w, K,
                      (const int32_t*)nullptr));
  return MDP_OK;
}

template <bool U, typename T>
static mdp_status launch_matvec(mdp_s* h, const KrylovBuffers<T>& B, double gamma, int j, cudaStream_t st) {
  if (sizeof(T) == sizeof(double))
    MDP_TRY((launch_matvec_as<U, T, T>(h, B, gamma, j, st)));
  else if (h->pstore == kStoreF16)
    MDP_TRY((launch_matvec_as<U, __half, T>(h, B, gamma, j, st)));
  else if (h->pstore == kStoreBF16)
    MDP_TRY((launch_matvec_as<U, __nv_bfloat16, T>(h, B, gamma, j, st)));
  else
    MDP_TRY((launch_matvec_as<U, float, T>(h, B, gamma, j, st)));
  MDP_LAUNCH_CHECK(h);
  return MDP_OK;
}

template <bool U, int NB, bool FINE, typename T>
static mdp_status arnoldi_step(mdp_s* h, const KrylovBuffers<T>& B, double gamma, int j, int refine,
                               cudaStream_t st) {
  const int64_t S = h->S;
  KrylovState* K = kstate(h);
  const bool timed = h->timing && (j % kMatvecTimingStride) == 0;
  if (timed) MDP_CUDA(cudaEventRecord(h->mv_ev[2 * j], st));
  if constexpr (FINE && sizeof(T) == sizeof(double)) {
    // binary64, single pass: the mat-vec fused with the dots, then the projection
    const Sell& Q = h->Ppi;
    MDP_CUDA(launch_pdl(gm_matvec_dots_kernel<U, NB>, MDP_WAVE((gm_matvec_dots_kernel<U, NB>)), kVecThreads, 0, st,
        Q.val, Q.col, Q.off, Q.len, U ? Q.kmax : 0, S, gamma, B.basis, j, B.w, h->partials, K));
    MDP_LAUNCH_CHECK(h);
    if (timed) MDP_CUDA(cudaEventRecord(h->mv_ev[2 * j + 1], st));
    MDP_CUDA(launch_pdl(gm_project_kernel<NB, kPlain, T, FINE>, MDP_WAVE((gm_project_kernel<NB, kPlain, T, FINE>)), kVecThreads, 0, st,
        S, B.basis, j, B.w, h->partials, K));
    MDP_LAUNCH_CHECK(h);
    if (timed && h->gs_on) MDP_CUDA(cudaEventRecord(h->gs_ev[j], st));
    return MDP_OK;
  }
  mdp_status r = launch_matvec<U>(h, B, gamma, j, st);
  if (r != MDP_OK) return r;
  if (timed) MDP_CUDA(cudaEventRecord(h->mv_ev[2 * j + 1], st));
  MDP_CUDA(launch_pdl(dots_kernel<NB, T, FINE>(), MDP_WAVE((dots_kernel<NB, T, FINE>())), kVecThreads, 0, st, S, B.basis, j, B.w,
                                                                                            h->partials, K));
  MDP_LAUNCH_CHECK(h);
  if (refine == MDP_REFINE_NEVER) {
    MDP_CUDA(launch_pdl(gm_project_kernel<NB, kPlain, T, FINE>, MDP_WAVE((gm_project_kernel<NB, kPlain, T, FINE>)), kVecThreads, 0, st,
        S, B.basis, j, B.w, h->partials, K));
    MDP_LAUNCH_CHECK(h);
    if (timed && h->gs_on) MDP_CUDA(cudaEventRecord(h->gs_ev[j], st));
    return MDP_OK;
  }
  if constexpr (!FINE && (NB == 8 || NB == 16 || NB == 32)) {  // re-orthogonalised steps use the coarse widths only
    if (refine == MDP_REFINE_IFNEEDED)
      MDP_CUDA(launch_pdl(gm_project_kernel<NB, kDgks, T, false>, MDP_WAVE((gm_project_kernel<NB, kDgks, T, false>)), kVecThreads, 0, st, S, B.basis, j, B.w, h->partials, K));
    else
      MDP_CUDA(launch_pdl(gm_project_kernel<NB, kAlways, T, false>, MDP_WAVE((gm_project_kernel<NB, kAlways, T, false>)), kVecThreads, 0, st, S, B.basis, j, B.w, h->partials, K));
    MDP_LAUNCH_CHECK(h);
    MDP_CUDA(launch_pdl(gm_project_kernel<NB, kSecond, T, false>, MDP_WAVE((gm_project_kernel<NB, kSecond, T, false>)), kVecThreads, 0, st, S, B.basis, j, B.w, h->partials, K));
    MDP_LAUNCH_CHECK(h);
    return MDP_OK;
  } else {
    return fail(MDP_ERR_INVALID_ARG, "internal: re-orthogonalised Arnoldi step at a fine width");
  }
}

// Block count of the single-problem launch of a GMRES pass (FP64, or the binary32
// cycle of the mixed solver).  The batched path gives every problem these counts,
// so its grid reductions add the same partial sums in the same order and its
// iterates equal the stand-alone ones.
template <typename T>
static int matvec_grid(mdp_s* h, bool U) {
  if (sizeof(T) == sizeof(double))
    return U ? MDP_WAVE((gm_matvec_kernel<true, double, double>)) : MDP_WAVE((gm_matvec_kernel<false, double, double>));
  if (h->pstore == kStoreF16)
    return U ? MDP_WAVE((gm_matvec_kernel<true, __half, float>)) : MDP_WAVE((gm_matvec_kernel<false, __half, float>));
  if (h->pstore == kStoreBF16)
    return U ? MDP_WAVE((gm_matvec_kernel<true, __nv_bfloat16, float>))
             : MDP_WAVE((gm_matvec_kernel<false, __nv_bfloat16, float>));
  return U ? MDP_WAVE((gm_matvec_kernel<true, float, float>)) : MDP_WAVE((gm_matvec_kernel<false, float, float>));
}

template <typename T>
static int pass_grid(mdp_s* h, GmresPass pass, int NB) {
  // the passes the batched solver mirrors run at the fine widths (exact tails)
  constexpr bool FINE_T = true;
  const bool U = h->Ppi.uniform;
  switch (pass) {
    case kPassResidual:
      return U ? MDP_WAVE((gm_residual_kernel<true, T>)) : MDP_WAVE((gm_residual_kernel<false, T>));
    case kPassMatvec:
      return matvec_grid<T>(h, U);
    case kPassUpdate:
      return MDP_WAVE(gm_update_kernel<T>);
    case kPassDots:
      if (sizeof(T) == sizeof(double)) {  // binary64: the mat-vec fused with the dots
        switch (NB) {
#define MDP_MVD(nb) return U ? MDP_WAVE((gm_matvec_dots_kernel<true, nb>)) : MDP_WAVE((gm_matvec_dots_kernel<false, nb>))
          case 4: MDP_MVD(4);
          case 8: MDP_MVD(8);
          case 12: MDP_MVD(12);
          case 16: MDP_MVD(16);
          case 20: MDP_MVD(20);
          case 24: MDP_MVD(24);
          case 28: MDP_MVD(28);
          default: MDP_MVD(32);
#undef MDP_MVD
        }
      }
      switch (NB) {
        case 4: return MDP_WAVE((dots_kernel<4, T, FINE_T>()));
        case 8: return MDP_WAVE((dots_kernel<8, T, FINE_T>()));
        case 12: return MDP_WAVE((dots_kernel<12, T, FINE_T>()));
        case 16: return MDP_WAVE((dots_kernel<16, T, FINE_T>()));
        case 20: return MDP_WAVE((dots_kernel<20, T, FINE_T>()));
        case 24: return MDP_WAVE((dots_kernel<24, T, FINE_T>()));
        case 28: return MDP_WAVE((dots_kernel<28, T, FINE_T>()));
        default: return MDP_WAVE((dots_kernel<32, T, FINE_T>()));
      }
    case kPassProject:
      switch (NB) {
        case 4: return MDP_WAVE((gm_project_kernel<4, kPlain, T, FINE_T>));
        case 8: return MDP_WAVE((gm_project_kernel<8, kPlain, T, FINE_T>));
        case 12: return MDP_WAVE((gm_project_kernel<12, kPlain, T, FINE_T>));
        case 16: return MDP_WAVE((gm_project_kernel<16, kPlain, T, FINE_T>));
        case 20: return MDP_WAVE((gm_project_kernel<20, kPlain, T, FINE_T>));
        case 24: return MDP_WAVE((gm_project_kernel<24, kPlain, T, FINE_T>));
        case 28: return MDP_WAVE((gm_project_kernel<28, kPlain, T, FINE_T>));
        default: return MDP_WAVE((gm_project_kernel<32, kPlain, T, FINE_T>));
      }
  }
  return 1;
}

int gmres_grid(mdp_s* h, GmresPass pass, int NB, bool mixed) {
  return mixed ? pass_grid<float>(h, pass, NB) : pass_grid<double>(h, pass, NB);
}

// Classical Gram-Schmidt steps without re-orthogonalisation (the default), FP64
// and binary32 alike, run at the smallest multiple of 4 accumulators that holds
// j + 1 basis vectors, with exact tails (FINE): predicated-off slots cost issue
// cycles (FP64: FP64 pipe cycles; measured 160.6 -> 147.1 ms per FP64 solve and
// 121.2 -> 110.8 ms per mixed one).  The re-orthogonalising modes run at 8, 16, 32.
template <bool U, typename T>
static mdp_status arnoldi_dispatch(mdp_s* h, const KrylovBuffers<T>& B, double gamma, int j, int refine,
                                   cudaStream_t st) {
  if (refine != MDP_REFINE_NEVER) {
    if (j + 1 <= 8) return arnoldi_step<U, 8, false>(h, B, gamma, j, refine, st);
    if (j + 1 <= 16) return arnoldi_step<U, 16, false>(h, B, gamma, j, refine, st);
    return arnoldi_step<U, 32, false>(h, B, gamma, j, refine, st);
  }
  switch ((j + 4) / 4) {  // j + 1 in (NB - 4, NB]: the exact-tail (FINE) passes
    case 1: return arnoldi_step<U, 4, true>(h, B, gamma, j, refine, st);
    case 2: return arnoldi_step<U, 8, true>(h, B, gamma, j, refine, st);
    case 3: return arnoldi_step<U, 12, true>(h, B, gamma, j, refine, st);
    case 4: return arnoldi_step<U, 16, true>(h, B, gamma, j, refine, st);
    case 5: return arnoldi_step<U, 20, true>(h, B, gamma, j, refine, st);
    case 6: return arnoldi_step<U, 24, true>(h, B, gamma, j, refine, st);
    case 7: return arnoldi_step<U, 28, true>(h, B, gamma, j, refine, st);
    default: return arnoldi_step<U, 32, true>(h, B, gamma, j, refine, st);
  }
}

// FP64 residual of the policy system (the refinement residual in the mixed
// solver), stored into basis slot 0 in the basis type.
template <bool U, typename T>
static mdp_status gm_residual(mdp_s* h, const KrylovBuffers<T>& B, double gamma, const double* theta,
                              cudaStream_t st) {
  const Sell& Q = h->Ppi;
  // the grid of the binary64-row kernel in every variant: the batched solver sums the
  // same block partials in the same order
  const int grid = MDP_WAVE((gm_residual_kernel<U, T>));
  bool done = false;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (h->pcol16) {  // the mixed solver's exact 16-bit rows (the gather wrote no binary64 copy)
      done = true;
      if (h->pstore == kStoreF16)
        MDP_CUDA(launch_pdl(gm_residual_kernel<U, T, __half, int16_t>, grid, kVecThreads, 0, st,
                            (const __half*)h->pval16, (const int16_t*)h->pcol16, Q.off, Q.len, U ? Q.kmax : 0, h->S,
                            gamma, theta, h->gpi, B.basis, h->partials, kstate(h), (const int32_t*)h->pcolbase));
      else
        MDP_CUDA(launch_pdl(gm_residual_kernel<U, T, __nv_bfloat16, int16_t>, grid, kVecThreads, 0, st,
                            (const __nv_bfloat16*)h->pval16, (const int16_t*)h->pcol16, Q.off, Q.len,
                            U ? Q.kmax : 0, h->S, gamma, theta, h->gpi, B.basis, h->partials, kstate(h),
                            (const int32_t*)h->pcolbase));
    }
  }
  if (!done) {
    MDP_CUDA(launch_pdl(gm_residual_kernel<U, T>, grid, kVecThreads, 0, st, Q.val, Q.col, Q.off, Q.len,
                        U ? Q.kmax : 0, h->S, gamma, theta, h->gpi, B.basis, h->partials, kstate(h),
                        (const int32_t*)nullptr));
  }
  MDP_LAUNCH_CHECK(h);
  return MDP_OK;
}

// Algorithmic bytes of the inner solver: one application of P_pi reads the
// policy's rows (value + 4 B column per entry) and its x once; the other vector
// accesses move one element per state.
static void add_matvec_bytes(mdp_s* h, int n, size_t value_bytes, size_t vec_bytes, size_t col_bytes = 4) {
  const double entries = (double)h->S * (double)h->Ppi.kmax;
  h->inner_bytes += n * (entries * (double)(value_bytes + col_bytes) + (double)h->S * (double)vec_bytes);
}

static void add_vector_bytes(mdp_s* h, int64_t nvec, size_t vec_bytes) {
  h->inner_bytes += (double)nvec * (double)h->S * (double)vec_bytes;
}

// n restart residuals (binary64 sums over the policy's rows, x = theta): the binary64
// rows, or the mixed solver's exact 16-bit rows with 16-bit column offsets.
static void add_residual_bytes(mdp_s* h, int64_t n, bool mixed) {
  const bool r16 = mixed && h->pcol16;
  add_matvec_bytes(h, (int)n, r16 ? 2 : sizeof(double), sizeof(double), r16 ? 2 : 4);
}

// Work of `steps` Arnoldi steps without re-orthogonalisation (one pass would do):
// apply P_pi with x = u_j, read the other j basis vectors for the dots and write
// w; the projection reads w and the j+1 basis vectors and writes u_{j+1}.  Then
// the update (basis vectors and theta) and the FP64 residual of the restart.
template <typename T>
static void count_cycle(mdp_s* h, int steps) {
  const size_t vbytes = (sizeof(T) == sizeof(double) || h->pstore == kStoreF32) ? sizeof(T) : 2;
  for (int j = 0; j < steps; ++j) {
    h->matvecs += 1;
    h->vreads += j + (j + 2);
    h->vwrites += 2;
    add_matvec_bytes(h, 1, vbytes, sizeof(T), (sizeof(T) == sizeof(float) && h->pcol16) ? 2 : 4);
    add_vector_bytes(h, j + (j + 2) + 2, sizeof(T));
  }
  h->vreads += steps + 1;
  h->vwrites += 1;
  add_vector_bytes(h, steps, sizeof(T));
  add_vector_bytes(h, 2, sizeof(double));
  h->matvecs += 1;
  h->vreads += 1;
  h->vwrites += 1;
  add_residual_bytes(h, 1, sizeof(T) == sizeof(float));
  add_vector_bytes(h, 1, sizeof(double));
  add_vector_bytes(h, 1, sizeof(T));
}

// Bytes per probability the mat-vec of value type T reads.
template <typename T>
static size_t vbytes_of(const mdp_s* h) {
  return sizeof(T) == sizeof(double) ? 8 : (h->pstore == kStoreF32 ? 4 : 2);
}

// record_timing: add the device time of the timed mat-vecs among the first n
// steps of the cycle that just finished (their events completed before the host
// read the solver state).  Every kMatvecTimingStride-th step of a cycle is timed:
// all mat-vecs do the same work, and an event pair around every one of them cost
// about 2% of the solve.
//
// The FP64 single-pass Gram-Schmidt of the same steps (dots, then projection) is
// timed from the mat-vec's end event to one after the projection; it does
// 2 (j + 1) + 1 FP64 FMAs per state (j + 1 dots, j + 1 projection terms, ||u||^2).
static mdp_status add_matvec_times(mdp_s* h, int n, size_t value_bytes, size_t vec_bytes) {
  const double S = (double)h->S, entries = S * (double)h->Ppi.kmax;
  for (int j = 0; j < n; j += kMatvecTimingStride) {
    float ms = 0.f;
    MDP_CUDA(cudaEventElapsedTime(&ms, h->mv_ev[2 * j], h->mv_ev[2 * j + 1]));
    h->mv_ms += ms;
    h->mv_timed += 1;
    // algorithmic bytes of the timed launch: the policy's rows, u_j read and w written,
    // and with the fused binary64 dots the j other basis vectors
    const double col_bytes = (vec_bytes == sizeof(float) && h->pcol16) ? 2.0 : 4.0;  // 16-bit offsets
    h->mv_bytes += entries * ((double)value_bytes + col_bytes) + 2.0 * S * (double)vec_bytes;
    if (h->gs_on) {
      h->mv_bytes += (double)j * S * (double)vec_bytes;
      // the fused kernel's FP64 work: the row (k fused multiply-adds), the j + 1 dots and w
      h->mv_flops += 2.0 * ((double)h->Ppi.kmax + (double)j + 2.0) * S;
      MDP_CUDA(cudaEventElapsedTime(&ms, h->mv_ev[2 * j + 1], h->gs_ev[j]));
      h->gs_ms += ms;
      h->gs_flops += 2.0 * (double)(j + 2) * S;  // the projection: j + 1 products and ||u||^2
      h->gs_timed += 1;
    }
  }
  return MDP_OK;
}

template <bool U, typename T>
static mdp_status gmres(mdp_s* h, double gamma, double* theta, int m, int refine, double tol, int maxit,
                        int* iters, double* res2, cudaStream_t st) {
  if (h->timing && !h->mv_ev[0]) {
    for (cudaEvent_t& e : h->mv_ev) MDP_CUDA(cudaEventCreate(&e));
    for (cudaEvent_t& e : h->gs_ev) MDP_CUDA(cudaEventCreate(&e));
  }
  h->gs_on = refine == MDP_REFINE_NEVER && sizeof(T) == sizeof(double);
  mdp_status r = (sizeof(T) == sizeof(double)) ? ensure_basis(h, m + 1) : ensure_mixed(h, m + 1);
  if (r != MDP_OK) return r;
  const KrylovBuffers<T> B = buffers(h, (T*)nullptr);
  KrylovState* K = kstate(h);
  r = init_state(h, tol, maxit, m, st);
  if (r != MDP_OK) return r;
  r = gm_residual<U>(h, B, gamma, theta, st);
  if (r != MDP_OK) return r;
  h->matvecs += 1;
  h->vreads += 1;
  h->vwrites += 1;
  add_residual_bytes(h, 1, sizeof(T) == sizeof(float));
  add_vector_bytes(h, 1, sizeof(double));
  add_vector_bytes(h, 1, sizeof(T));
  KrylovHeader hd{};
  double rn = 0.0;
  int it_before = 0;
  for (;;) {
    r = read_header(h, &hd, &rn, st);
    if (r != MDP_OK) return r;
    if (hd.flags & kSolveDone) break;
    if (hd.it > it_before) count_cycle<T>(h, hd.it - it_before);
    if (h->timing) MDP_TRY(add_matvec_times(h, hd.it - it_before, vbytes_of<T>(h), sizeof(T)));
    it_before = hd.it;
    const int steps = std::min(m, maxit - hd.it);
    for (int j = 0; j < steps; ++j) {
      r = arnoldi_dispatch<U>(h, B, gamma, j, refine, st);
      if (r != MDP_OK) return r;
    }
    MDP_CUDA(launch_pdl(gm_update_kernel<T>, MDP_WAVE(gm_update_kernel<T>), kVecThreads, 0, st, h->S, B.basis, theta, K));
    MDP_LAUNCH_CHECK(h);
    r = gm_residual<U>(h, B, gamma, theta, st);
    if (r != MDP_OK) return r;
  }
  if (hd.it > it_before) count_cycle<T>(h, hd.it - it_before);
  if (h->timing) MDP_TRY(add_matvec_times(h, hd.it - it_before, vbytes_of<T>(h), sizeof(T)));
  if (hd.flags & kNumeric) return fail(MDP_ERR_NUMERIC, "non-finite residual in GMRES");
  *iters = hd.it;
  *res2 = rn;
  return MDP_OK;
}

// Richardson: before each step r = g_pi - J theta; stop when ||r||_2 < tol, else
// theta += omega r; at most maxit steps.  Steps are queued in batches and the
// host waits once per batch; steps queued after the stop return at once.
template <bool U>
static mdp_status richardson(mdp_s* h, double gamma, double* theta, double omega, double tol, int maxit, int* iters,
                             double* res2, cudaStream_t st) {
  KrylovState* K = kstate(h);
  mdp_status r = init_state(h, tol, maxit, 0, st);
  if (r != MDP_OK) return r;
  double* buf[2] = {theta, h->tmp};
  const Sell& Q = h->Ppi;
  KrylovHeader hd{};
  double rn = INFINITY;
  int issued = 0;
  if (maxit > 0) {
    for (;;) {
      const int batch = std::min(maxit - issued, issued < 8 ? 2 : 16);
      for (int b = 0; b < batch; ++b, ++issued) {
        const int in = issued & 1;
        rich_step_kernel<U><<<MDP_WAVE(rich_step_kernel<U>), kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, U ? Q.kmax : 0, h->S,
                                                                    gamma, omega, buf[in], h->gpi, buf[1 - in], in,
                                                                    h->partials, K);
        MDP_LAUNCH_CHECK(h);
      }
      r = read_header(h, &hd, &rn, st);
      if (r != MDP_OK) return r;
      if ((hd.flags & kSolveDone) || issued >= maxit) break;
    }
    const int worked = hd.it + ((hd.flags & kSolveDone) && hd.it < maxit ? 1 : 0);
    h->matvecs += worked;
    h->vreads += worked;
    h->vwrites += worked;
    add_matvec_bytes(h, worked, sizeof(double), sizeof(double));
    add_vector_bytes(h, 2 * (int64_t)worked, sizeof(double));
    if (hd.flags & kNumeric) return fail(MDP_ERR_NUMERIC, "non-finite residual in Richardson");
    if (hd.result == 1) MDP_CUDA(cudaMemcpyAsync(theta, h->tmp, h->S * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  *iters = maxit > 0 ? hd.it : 0;
  *res2 = rn;
  return MDP_OK;
}

// TFQMR on J_pi x = g_pi from x = theta: batches of outer steps (two half steps
// each) are queued and the host waits once per batch; kernels queued after the
// stop test return at once.
template <bool U>
static mdp_status tfqmr(mdp_s* h, double gamma, double* x, double tol, int maxit, int* iters, double* res2,
                        cudaStream_t st) {
  mdp_status r = ensure_tfqmr(h);
  if (r != MDP_OK) return r;
  KrylovState* K = kstate(h);
  r = init_state(h, tol, maxit, 0, st);
  if (r != MDP_OK) return r;
  const Sell& Q = h->Ppi;
  const int k = U ? Q.kmax : 0;
  const int64_t S = h->S;
  double* rt = h->tfq;
  double* w = rt + S;
  double* y1 = w + S;
  double* y2 = y1 + S;
  double* u1 = y2 + S;
  double* u2 = u1 + S;
  double* v = u2 + S;
  double* d = v + S;
  tf_init_kernel<U><<<MDP_WAVE(tf_init_kernel<U>), kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, k, S, gamma, x,
                                                                         h->gpi, rt, w, y1, d, h->partials, K);
  MDP_LAUNCH_CHECK(h);
  tf_matvec_kernel<U, false><<<MDP_WAVE((tf_matvec_kernel<U, false>)), kVecThreads, 0, st>>>(
      Q.val, Q.col, Q.off, Q.len, k, S, gamma, y1, v, nullptr, nullptr, K);
  MDP_LAUNCH_CHECK(h);
  MDP_CUDA(cudaMemcpyAsync(u1, v, S * sizeof(double), cudaMemcpyDeviceToDevice, st));
  add_matvec_bytes(h, 2, sizeof(double), sizeof(double));
  KrylovHeader hd{};
  double rn = 0.0;
  int half = 0;  // half steps queued so far
  for (;;) {
    r = read_header(h, &hd, &rn, st);
    if (r != MDP_OK) return r;
    if ((hd.flags & kSolveDone) || half >= maxit) break;
    const int outer = std::max(1, std::min(8, (maxit - half + 1) / 2));
    for (int q = 0; q < outer; ++q) {
      tf_sigma_kernel<<<MDP_WAVE(tf_sigma_kernel), kVecThreads, 0, st>>>(S, rt, v, h->partials, K);
      MDP_LAUNCH_CHECK(h);
      tf_axpy_kernel<true><<<MDP_WAVE(tf_axpy_kernel<true>), kVecThreads, 0, st>>>(S, y1, v, y2, K);
      MDP_LAUNCH_CHECK(h);
      tf_matvec_kernel<U, false><<<MDP_WAVE((tf_matvec_kernel<U, false>)), kVecThreads, 0, st>>>(
          Q.val, Q.col, Q.off, Q.len, k, S, gamma, y2, u2, nullptr, nullptr, K);
      MDP_LAUNCH_CHECK(h);
      tf_half_kernel<<<MDP_WAVE(tf_half_kernel), kVecThreads, 0, st>>>(S, y1, u1, w, d, h->partials, K);
      MDP_LAUNCH_CHECK(h);
      tf_xupd_kernel<false><<<MDP_WAVE(tf_xupd_kernel<false>), kVecThreads, 0, st>>>(S, ++half, d, x, rt, w,
                                                                                    h->partials, K);
      MDP_LAUNCH_CHECK(h);
      tf_half_kernel<<<MDP_WAVE(tf_half_kernel), kVecThreads, 0, st>>>(S, y2, u2, w, d, h->partials, K);
      MDP_LAUNCH_CHECK(h);
      tf_xupd_kernel<true><<<MDP_WAVE(tf_xupd_kernel<true>), kVecThreads, 0, st>>>(S, ++half, d, x, rt, w,
                                                                                  h->partials, K);
      MDP_LAUNCH_CHECK(h);
      tf_axpy_kernel<false><<<MDP_WAVE(tf_axpy_kernel<false>), kVecThreads, 0, st>>>(S, w, y2, y1, K);
      MDP_LAUNCH_CHECK(h);
      tf_matvec_kernel<U, true><<<MDP_WAVE((tf_matvec_kernel<U, true>)), kVecThreads, 0, st>>>(
          Q.val, Q.col, Q.off, Q.len, k, S, gamma, y1, u1, u2, v, K);
      MDP_LAUNCH_CHECK(h);
      if (half >= maxit) break;
    }
  }
  true_residual_kernel<U><<<MDP_WAVE(true_residual_kernel<U>), kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, k,
                                                                                     S, gamma, x, h->gpi,
                                                                                     h->partials, K);
  MDP_LAUNCH_CHECK(h);
  r = read_header(h, &hd, &rn, st);
  if (r != MDP_OK) return r;
  // per half step: one product by J (12 B/entry + x) and about six vector accesses
  add_matvec_bytes(h, hd.it + 1, sizeof(double), sizeof(double));
  add_vector_bytes(h, 6 * (int64_t)hd.it + 2, sizeof(double));
  h->matvecs += hd.it + 3;
  if (hd.flags & kNumeric) return fail(MDP_ERR_NUMERIC, "non-finite residual in TFQMR");
  *iters = hd.it;
  *res2 = rn;
  return MDP_OK;
}

// Richardson with the Jacobi preconditioner (J-VI): as richardson() with the
// step scaled by 1 / (1 - gamma P(s, s, pi(s))).
template <bool U>
static mdp_status jacobi_richardson(mdp_s* h, double gamma, double* theta, double omega, double tol, int maxit,
                                    int* iters, double* res2, cudaStream_t st) {
  mdp_status r = ensure_tfqmr(h);  // its first vector holds the diagonal
  if (r != MDP_OK) return r;
  KrylovState* K = kstate(h);
  r = init_state(h, tol, maxit, 0, st);
  if (r != MDP_OK) return r;
  const Sell& Q = h->Ppi;
  const int k = U ? Q.kmax : 0;
  double* pdiag = h->tfq;
  policy_diag_kernel<U><<<MDP_WAVE(policy_diag_kernel<U>), kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, k, h->S,
                                                                                 pdiag);
  MDP_LAUNCH_CHECK(h);
  double* buf[2] = {theta, h->tmp};
  KrylovHeader hd{};
  double rn = INFINITY;
  int issued = 0;
  if (maxit > 0) {
    for (;;) {
      const int batch = std::min(maxit - issued, issued < 8 ? 2 : 16);
      for (int b = 0; b < batch; ++b, ++issued) {
        const int in = issued & 1;
        jacobi_step_kernel<U><<<MDP_WAVE(jacobi_step_kernel<U>), kVecThreads, 0, st>>>(
            Q.val, Q.col, Q.off, Q.len, k, h->S, gamma, omega, pdiag, buf[in], h->gpi, buf[1 - in], in, h->partials,
            K);
        MDP_LAUNCH_CHECK(h);
      }
      r = read_header(h, &hd, &rn, st);
      if (r != MDP_OK) return r;
      if ((hd.flags & kSolveDone) || issued >= maxit) break;
    }
    const int worked = hd.it + ((hd.flags & kSolveDone) && hd.it < maxit ? 1 : 0);
    h->matvecs += worked;
    add_matvec_bytes(h, worked, sizeof(double), sizeof(double));
    add_vector_bytes(h, 3 * (int64_t)worked, sizeof(double));
    if (hd.flags & kNumeric) return fail(MDP_ERR_NUMERIC, "non-finite residual in Jacobi-Richardson");
    if (hd.result == 1) MDP_CUDA(cudaMemcpyAsync(theta, h->tmp, h->S * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  *iters = maxit > 0 ? hd.it : 0;
  *res2 = rn;
  return MDP_OK;
}

mdp_status launch_policy_apply(mdp_s* h, double gamma, const double* x, double* y, cudaStream_t st) {
  const Sell& Q = h->Ppi;
  if (Q.uniform)
    policy_apply_kernel<true><<<h->vec_blocks, kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, Q.kmax, h->S, gamma,
                                                                      x, h->gpi, y);
  else
    policy_apply_kernel<false><<<h->vec_blocks, kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, 0, h->S, gamma, x,
                                                                       h->gpi, y);
  MDP_LAUNCH_CHECK(h);
  return MDP_OK;
}

size_t krylov_state_bytes() { return sizeof(KrylovState); }

// ---- launch sequences of the GMRES solve for the graph-driven mdp_solve ------------------

// The restart residual r = g_pi - J_pi theta into basis slot 0 (and beta, the stop flags).
mdp_status gmres_residual_launch(mdp_s* h, bool mixed, double gamma, const double* theta, cudaStream_t st) {
  const bool U = h->Ppi.uniform;
  if (mixed) {
    const KrylovBuffers<float> B = buffers(h, (float*)nullptr);
    return U ? gm_residual<true>(h, B, gamma, theta, st) : gm_residual<false>(h, B, gamma, theta, st);
  }
  const KrylovBuffers<double> B = buffers(h, (double*)nullptr);
  return U ? gm_residual<true>(h, B, gamma, theta, st) : gm_residual<false>(h, B, gamma, theta, st);
}

template <bool U, typename T>
static mdp_status steps_launch(mdp_s* h, double gamma, int j0, int j1, int refine, cudaStream_t st) {
  const KrylovBuffers<T> B = buffers(h, (T*)nullptr);
  for (int j = j0; j < j1; ++j) MDP_TRY(arnoldi_dispatch<U>(h, B, gamma, j, refine, st));
  return MDP_OK;
}

template <bool U, typename T>
static mdp_status tail_launch(mdp_s* h, double gamma, double* theta, cudaStream_t st) {
  const KrylovBuffers<T> B = buffers(h, (T*)nullptr);
  MDP_CUDA(launch_pdl(gm_update_kernel<T>, MDP_WAVE(gm_update_kernel<T>), kVecThreads, 0, st, h->S, B.basis, theta, kstate(h)));
  MDP_LAUNCH_CHECK(h);
  return gm_residual<U>(h, B, gamma, theta, st);
}

// Arnoldi steps j0..j1-1 of a restart cycle as gmres() queues them (steps after
// the cycle's stop return at once; the iteration cap stops a cycle on the device).
mdp_status gmres_steps_launch(mdp_s* h, bool mixed, double gamma, int j0, int j1, int refine, cudaStream_t st) {
  const bool U = h->Ppi.uniform;
  if (mixed)
    return U ? steps_launch<true, float>(h, gamma, j0, j1, refine, st)
             : steps_launch<false, float>(h, gamma, j0, j1, refine, st);
  return U ? steps_launch<true, double>(h, gamma, j0, j1, refine, st)
           : steps_launch<false, double>(h, gamma, j0, j1, refine, st);
}

// The end of a restart cycle: the update of theta and the next restart residual.
mdp_status gmres_tail_launch(mdp_s* h, bool mixed, double gamma, double* theta, cudaStream_t st) {
  const bool U = h->Ppi.uniform;
  if (mixed) return U ? tail_launch<true, float>(h, gamma, theta, st) : tail_launch<false, float>(h, gamma, theta, st);
  return U ? tail_launch<true, double>(h, gamma, theta, st) : tail_launch<false, double>(h, gamma, theta, st);
}

// The work counters gmres() adds, summed over `solves` GMRES solves made of
// `cycles` restart cycles with `steps` Arnoldi steps in all, where `tri` is the
// sum over cycles of n (n - 1) / 2 for a cycle of n steps.
void gmres_count_work(mdp_s* h, bool mixed, int64_t solves, int64_t cycles, int64_t steps, int64_t tri) {
  const size_t sT = mixed ? sizeof(float) : sizeof(double);
  const size_t vbytes = (!mixed || h->pstore == kStoreF32) ? sT : 2;
  // the first restart residual of every solve
  h->matvecs += solves;
  h->vreads += solves;
  h->vwrites += solves;
  add_residual_bytes(h, solves, mixed);
  add_vector_bytes(h, solves, sizeof(double));
  add_vector_bytes(h, solves, sT);
  // count_cycle summed in closed form: sum_j (2 j + 2) = n^2 + n over a cycle of n steps
  const int64_t sq = 2 * tri + steps;
  h->matvecs += steps + cycles;
  h->vreads += sq + 2 * steps + 2 * cycles;
  h->vwrites += 2 * steps + 2 * cycles;
  add_matvec_bytes(h, (int)steps, vbytes, sT, (mixed && h->pcol16) ? 2 : 4);
  add_vector_bytes(h, 2 * tri + 5 * steps, sT);
  add_vector_bytes(h, 3 * cycles, sizeof(double));
  add_residual_bytes(h, cycles, mixed);
  add_vector_bytes(h, cycles, sT);
}

mdp_status inner_solve(mdp_s* h, double gamma, double* theta, int inner, int restart, int refine, int precision,
                       double omega, double tol, int max_it, int* iters, double* res2, cudaStream_t st) {
  *iters = 0;
  *res2 = 0.0;
  const bool U = h->Ppi.uniform;
  if (inner == MDP_GMRES && precision == MDP_PREC_MIXED)
    return U ? gmres<true, float>(h, gamma, theta, restart, refine, tol, max_it, iters, res2, st)
             : gmres<false, float>(h, gamma, theta, restart, refine, tol, max_it, iters, res2, st);
  if (inner == MDP_GMRES)
    return U ? gmres<true, double>(h, gamma, theta, restart, refine, tol, max_it, iters, res2, st)
             : gmres<false, double>(h, gamma, theta, restart, refine, tol, max_it, iters, res2, st);
  if (inner == MDP_TFQMR)
    return U ? tfqmr<true>(h, gamma, theta, tol, max_it, iters, res2, st)
             : tfqmr<false>(h, gamma, theta, tol, max_it, iters, res2, st);
  if (inner == MDP_RICHARDSON_JACOBI)
    return U ? jacobi_richardson<true>(h, gamma, theta, omega, tol, max_it, iters, res2, st)
             : jacobi_richardson<false>(h, gamma, theta, omega, tol, max_it, iters, res2, st);
  return U ? richardson<true>(h, gamma, theta, omega, tol, max_it, iters, res2, st)
           : richardson<false>(h, gamma, theta, omega, tol, max_it, iters, res2, st);
}

}  // namespace mdp
