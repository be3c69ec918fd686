// Inexact policy evaluation (Algorithm 1 steps 6-12): the matrix-free operator
// J_pi x = x - gamma P_pi x (Sec. III-B.3) over the policy's rows, and the two
// inner solvers, Richardson (theta += omega (g_pi - J_pi theta)) and restarted
// GMRES(m) with classical Gram-Schmidt plus one re-orthogonalisation (CGS2).
//
// Every pass is one thread per state over the per-state sliced layout of P_pi
// (lanes = consecutive states, so values, columns and vector entries load
// coalesced; only x[col] is a gather).  Reductions are deterministic: each
// block writes a partial per quantity, and a one-block kernel adds the
// partials in a fixed order.
#include <cmath>
#include <vector>

#include "mdp_internal.cuh"

namespace mdp {

constexpr int kVecThreads = 256;

// sum_j P_pi[s, j] x[col_j] for state s (lane l of slice s/32)
template <bool UNIFORM>
__device__ __forceinline__ double policy_row_dot(const double* __restrict__ pval, const int32_t* __restrict__ pcol,
                                                 const int64_t* __restrict__ poff, const int32_t* __restrict__ plen,
                                                 int k, int64_t s, const double* __restrict__ x) {
  const int64_t q = s / kSlice;
  const int n = UNIFORM ? k : plen[s];
  const int64_t base = (UNIFORM ? q * kSlice * (int64_t)k : poff[q]) + (s % kSlice);
  const double* vp = pval + base;
  const int32_t* cp = pcol + base;
  double acc = 0.0;
  int j = 0;
  for (; j + 4 <= n; j += 4) {
    double v[4];
    int c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = vp[(int64_t)(j + u) * kSlice];
      c[u] = cp[(int64_t)(j + u) * kSlice];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc = fma(v[u], __ldg(x + c[u]), acc);
  }
  for (; j < n; ++j) acc = fma(vp[(int64_t)j * kSlice], __ldg(x + cp[(int64_t)j * kSlice]), acc);
  return acc;
}

// Block sum of NV per-thread values; thread 0..NV-1 of the block then writes
// partials[blockIdx.x * kMaxBasis + i].  Fixed shuffle tree, fixed warp order.
template <int NV>
__device__ __forceinline__ void block_partials(double (&d)[NV], int nvalid, double* __restrict__ partials) {
  __shared__ double red[kVecThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < nvalid) {
      double v = d[i];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][i] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < nvalid) {
    double v = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) v += red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * kMaxBasis + threadIdx.x] = v;
  }
}

// y = x - gamma P_pi x
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
    // states whose policy entry was invalid carry g_pi = NaN: poison their output
    const double gv = gpi[s];
    y[s] = (gv != gv) ? gv : x[s] - gamma * px;
  }
}

// r = b - J theta written to r_out; partial ||r||^2.  Richardson variant also
// writes theta_out = theta + omega r.
template <bool U, bool RICH>
__global__ void __launch_bounds__(kVecThreads) residual_kernel(const double* __restrict__ pval,
                                                                const int32_t* __restrict__ pcol,
                                                                const int64_t* __restrict__ poff,
                                                                const int32_t* __restrict__ plen, int k, int64_t S,
                                                                double gamma, double omega,
                                                                const double* __restrict__ theta,
                                                                const double* __restrict__ b,
                                                                double* __restrict__ out, double* __restrict__ partials) {
  double d[1] = {0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, theta);
    const double th = theta[s];
    const double r = b[s] - (th - gamma * px);
    d[0] = fma(r, r, d[0]);
    out[s] = RICH ? fma(omega, r, th) : r;
  }
  block_partials<1>(d, 1, partials);
}

// Arnoldi pass 1: w = J v_j, and partial dots v_i . w for i <= j.
template <bool U, int NB>
__global__ void __launch_bounds__(kVecThreads) arnoldi_matvec_kernel(const double* __restrict__ pval,
                                                                      const int32_t* __restrict__ pcol,
                                                                      const int64_t* __restrict__ poff,
                                                                      const int32_t* __restrict__ plen, int k,
                                                                      int64_t S, double gamma,
                                                                      const double* __restrict__ basis, int j,
                                                                      double* __restrict__ w,
                                                                      double* __restrict__ partials) {
  double d[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) d[i] = 0.0;
  const double* vj = basis + (int64_t)j * S;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const double px = policy_row_dot<U>(pval, pcol, poff, plen, k, s, vj);
    const double ws = vj[s] - gamma * px;
    w[s] = ws;
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i <= j) d[i] = fma(basis[(int64_t)i * S + s], ws, d[i]);
  }
  block_partials<NB>(d, j + 1, partials);
}

// Arnoldi pass 2 (re-orthogonalisation): w' = w - sum_i h_i v_i, partial dots v_i . w'.
template <int NB>
__global__ void __launch_bounds__(kVecThreads) cgs_correct_kernel(int64_t S, const double* __restrict__ basis, int j,
                                                                   const double* __restrict__ h,
                                                                   const double* __restrict__ w,
                                                                   double* __restrict__ partials) {
  __shared__ double hc[NB];
  double d[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) d[i] = 0.0;
  if (threadIdx.x < NB) hc[threadIdx.x] = (threadIdx.x <= j) ? h[threadIdx.x] : 0.0;
  __syncthreads();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    double ws = w[s];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i <= j) ws = fma(-hc[i], basis[(int64_t)i * S + s], ws);
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i <= j) d[i] = fma(__ldca(basis + (int64_t)i * S + s), ws, d[i]);
  }
  block_partials<NB>(d, j + 1, partials);
}

// Arnoldi pass 3: u = w - sum_i h_i v_i (h = first + second coefficients) into
// basis slot j+1, partial ||u||^2.
template <int NB>
__global__ void __launch_bounds__(kVecThreads) cgs_final_kernel(int64_t S, double* __restrict__ basis, int j,
                                                                 const double* __restrict__ h,
                                                                 const double* __restrict__ w,
                                                                 double* __restrict__ partials) {
  __shared__ double hc[NB];
  double d[1] = {0.0};
  if (threadIdx.x < NB) hc[threadIdx.x] = (threadIdx.x <= j) ? h[threadIdx.x] : 0.0;
  __syncthreads();
  double* u = basis + (int64_t)(j + 1) * S;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    double ws = w[s];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i <= j) ws = fma(-hc[i], basis[(int64_t)i * S + s], ws);
    u[s] = ws;
    d[0] = fma(ws, ws, d[0]);
  }
  block_partials<1>(d, 1, partials);
}

// theta += sum_{i < n} y_i v_i
template <int NB>
__global__ void __launch_bounds__(kVecThreads) basis_update_kernel(int64_t S, const double* __restrict__ basis, int n,
                                                                    const double* __restrict__ y,
                                                                    double* __restrict__ theta) {
  __shared__ double yc[NB];
  if (threadIdx.x < NB) yc[threadIdx.x] = (threadIdx.x < n) ? y[threadIdx.x] : 0.0;
  __syncthreads();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    double t = theta[s];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i < n) t = fma(yc[i], basis[(int64_t)i * S + s], t);
    theta[s] = t;
  }
}

// v *= scale[0]
__global__ void scale_kernel(int64_t S, double* __restrict__ v, const double* __restrict__ scale) {
  const double c = scale[0];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x)
    v[s] *= c;
}

enum { kSum = 0, kAdd = 1, kNorm = 2 };

// One block: dst[i] = (mode == kAdd ? src[i] : 0) + sum_b partials[b][i] for i < n,
// or (kNorm) dst[0] = sqrt(sum), dst[1] = 1 / dst[0] (0 if dst[0] == 0).
__global__ void reduce_partials_kernel(const double* __restrict__ partials, int nblk, int n, int mode,
                                       const double* __restrict__ src, double* __restrict__ dst) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = 0; i < n; ++i) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += partials[(int64_t)b * kMaxBasis + i];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w];
      if (mode == kNorm) {
        const double nr = sqrt(t);
        dst[0] = nr;
        dst[1] = nr > 0.0 ? 1.0 / nr : 0.0;
      } else {
        dst[i] = (mode == kAdd ? src[i] : 0.0) + t;
      }
    }
    __syncthreads();
  }
}

// device scalar slots
enum {
  kSlotH1 = 0,      // first-pass coefficients [32]
  kSlotH = 64,      // Hessenberg column j: h_0..h_j, then norm at [j+1]
  kSlotNorm = 160,  // [0] = norm, [1] = 1/norm
  kSlotY = 192,     // update coefficients [32]
};

#define MDP_LAUNCH_CHECK(h) \
  do {                      \
    (h)->launches++;        \
    MDP_CUDA(cudaGetLastError()); \
  } while (0)

static mdp_status reduce(mdp_s* h, int n, int mode, const double* src, double* dst, cudaStream_t st) {
  reduce_partials_kernel<<<1, 256, 0, st>>>(h->partials, h->vec_blocks, n, mode, src, dst);
  MDP_LAUNCH_CHECK(h);
  return MDP_OK;
}

template <bool U>
static mdp_status residual(mdp_s* h, double gamma, double omega, const double* theta, double* out, bool rich,
                           cudaStream_t st) {
  const Sell& Q = h->Ppi;
  const int k = U ? Q.kmax : 0;
  if (rich)
    residual_kernel<U, true><<<h->vec_blocks, kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, k, h->S, gamma,
                                                                     omega, theta, h->gpi, out, h->partials);
  else
    residual_kernel<U, false><<<h->vec_blocks, kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, k, h->S, gamma,
                                                                      omega, theta, h->gpi, out, h->partials);
  MDP_LAUNCH_CHECK(h);
  h->matvecs += 1;
  h->vreads += 1;
  h->vwrites += 1;
  return reduce(h, 1, kNorm, nullptr, h->sc + kSlotNorm, st);
}

static mdp_status read_scalars(mdp_s* h, int slot, int n, cudaStream_t st) {
  MDP_CUDA(cudaMemcpyAsync(h->hpin + slot, h->sc + slot, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  return MDP_OK;
}

template <bool U, int NB>
static mdp_status arnoldi_step(mdp_s* h, double gamma, int j, cudaStream_t st) {
  const Sell& Q = h->Ppi;
  const int k = U ? Q.kmax : 0;
  const int64_t S = h->S;
  arnoldi_matvec_kernel<U, NB><<<h->vec_blocks, kVecThreads, 0, st>>>(Q.val, Q.col, Q.off, Q.len, k, S, gamma,
                                                                       h->basis, j, h->w, h->partials);
  MDP_LAUNCH_CHECK(h);
  mdp_status r = reduce(h, j + 1, kSum, nullptr, h->sc + kSlotH1, st);
  if (r != MDP_OK) return r;
  cgs_correct_kernel<NB><<<h->vec_blocks, kVecThreads, 0, st>>>(S, h->basis, j, h->sc + kSlotH1, h->w, h->partials);
  MDP_LAUNCH_CHECK(h);
  r = reduce(h, j + 1, kAdd, h->sc + kSlotH1, h->sc + kSlotH, st);
  if (r != MDP_OK) return r;
  cgs_final_kernel<NB><<<h->vec_blocks, kVecThreads, 0, st>>>(S, h->basis, j, h->sc + kSlotH, h->w, h->partials);
  MDP_LAUNCH_CHECK(h);
  r = reduce(h, 1, kNorm, nullptr, h->sc + kSlotNorm, st);
  if (r != MDP_OK) return r;
  scale_kernel<<<h->vec_blocks, kVecThreads, 0, st>>>(S, h->basis + (int64_t)(j + 1) * S, h->sc + kSlotNorm + 1);
  MDP_LAUNCH_CHECK(h);
  // pass 1: P_pi v_j plus the other j basis vectors, writes w; pass 2: w and j+1
  // basis vectors; pass 3: the same, writes v_{j+1}; scaling: one read, one write
  h->matvecs += 1;
  h->vreads += j + (j + 2) + (j + 2) + 1;
  h->vwrites += 1 + 1 + 1;
  return MDP_OK;
}

template <bool U>
static mdp_status arnoldi_dispatch(mdp_s* h, double gamma, int j, cudaStream_t st) {
  if (j + 1 <= 8) return arnoldi_step<U, 8>(h, gamma, j, st);
  if (j + 1 <= 16) return arnoldi_step<U, 16>(h, gamma, j, st);
  return arnoldi_step<U, 32>(h, gamma, j, st);
}

static mdp_status basis_update(mdp_s* h, int n, double* theta, cudaStream_t st) {
  const double* y = h->sc + kSlotY;
  if (n <= 8)
    basis_update_kernel<8><<<h->vec_blocks, kVecThreads, 0, st>>>(h->S, h->basis, n, y, theta);
  else if (n <= 16)
    basis_update_kernel<16><<<h->vec_blocks, kVecThreads, 0, st>>>(h->S, h->basis, n, y, theta);
  else
    basis_update_kernel<32><<<h->vec_blocks, kVecThreads, 0, st>>>(h->S, h->basis, n, y, theta);
  MDP_LAUNCH_CHECK(h);
  h->vreads += n + 1;
  h->vwrites += 1;
  return MDP_OK;
}

// Restarted GMRES(m) on J_pi theta = g_pi (Saad, Sec. 6.5), CGS2 Arnoldi on the
// device, Givens rotations and the triangular solve on the host (m <= 32).
template <bool U>
static mdp_status gmres(mdp_s* h, double gamma, double* theta, int m, double tol, int maxit, int* iters,
                        double* res2, cudaStream_t st) {
  mdp_status r = ensure_basis(h, m + 1);
  if (r != MDP_OK) return r;
  const int64_t S = h->S;
  int it = 0;
  r = residual<U>(h, gamma, 1.0, theta, h->basis, false, st);
  if (r != MDP_OK) return r;
  r = read_scalars(h, kSlotNorm, 2, st);
  if (r != MDP_OK) return r;
  double beta = h->hpin[kSlotNorm];
  std::vector<double> H((m + 1) * m), cs(m), sn(m), e(m + 1), y(m);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  while (beta >= tol && it < maxit) {
    if (!std::isfinite(beta)) return fail(MDP_ERR_NUMERIC, "non-finite residual in GMRES");
    scale_kernel<<<h->vec_blocks, kVecThreads, 0, st>>>(S, h->basis, h->sc + kSlotNorm + 1);
    MDP_LAUNCH_CHECK(h);
    h->vreads += 1;
    h->vwrites += 1;
    std::fill(e.begin(), e.end(), 0.0);
    e[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      r = arnoldi_dispatch<U>(h, gamma, j, st);
      if (r != MDP_OK) return r;
      // column j of H: h_0..h_j from slot H, h_{j+1} = norm
      MDP_CUDA(cudaMemcpyAsync(h->hpin + kSlotH, h->sc + kSlotH, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
      r = read_scalars(h, kSlotNorm, 1, st);
      if (r != MDP_OK) return r;
      for (int i = 0; i <= j; ++i) Hat(i, j) = h->hpin[kSlotH + i];
      const double hn = h->hpin[kSlotNorm];
      Hat(j + 1, j) = hn;
      if (!std::isfinite(hn)) return fail(MDP_ERR_NUMERIC, "non-finite Arnoldi norm in GMRES");
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hat(i, j) + sn[i] * Hat(i + 1, j);
        Hat(i + 1, j) = -sn[i] * Hat(i, j) + cs[i] * Hat(i + 1, j);
        Hat(i, j) = t;
      }
      const double d = std::hypot(Hat(j, j), Hat(j + 1, j));
      cs[j] = Hat(j, j) / d;
      sn[j] = Hat(j + 1, j) / d;
      Hat(j, j) = d;
      Hat(j + 1, j) = 0.0;
      e[j + 1] = -sn[j] * e[j];
      e[j] = cs[j] * e[j];
      ++it;
      jdone = j + 1;
      if (std::fabs(e[j + 1]) < tol || it >= maxit || hn == 0.0) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double t = e[i];
      for (int c = i + 1; c < jdone; ++c) t -= Hat(i, c) * y[c];
      y[i] = t / Hat(i, i);
    }
    for (int i = 0; i < jdone; ++i) h->hpin[kSlotY + i] = y[i];
    MDP_CUDA(cudaMemcpyAsync(h->sc + kSlotY, h->hpin + kSlotY, jdone * sizeof(double), cudaMemcpyHostToDevice, st));
    r = basis_update(h, jdone, theta, st);
    if (r != MDP_OK) return r;
    r = residual<U>(h, gamma, 1.0, theta, h->basis, false, st);
    if (r != MDP_OK) return r;
    r = read_scalars(h, kSlotNorm, 2, st);
    if (r != MDP_OK) return r;
    beta = h->hpin[kSlotNorm];
  }
  if (!std::isfinite(beta)) return fail(MDP_ERR_NUMERIC, "non-finite residual in GMRES");
  *iters = it;
  *res2 = beta;
  return MDP_OK;
}

// Richardson: before each step r = g_pi - J theta; stop when ||r||_2 < tol, else
// theta += omega r; at most maxit steps.
template <bool U>
static mdp_status richardson(mdp_s* h, double gamma, double* theta, double omega, double tol, int maxit, int* iters,
                             double* res2, cudaStream_t st) {
  double* a = theta;
  double* b = h->tmp;
  int it = 0;
  double rn = INFINITY;
  while (it < maxit) {
    mdp_status r = residual<U>(h, gamma, omega, a, b, true, st);
    if (r != MDP_OK) return r;
    r = read_scalars(h, kSlotNorm, 1, st);
    if (r != MDP_OK) return r;
    rn = h->hpin[kSlotNorm];
    if (!std::isfinite(rn)) return fail(MDP_ERR_NUMERIC, "non-finite residual in Richardson");
    if (rn < tol) break;
    std::swap(a, b);
    ++it;
  }
  if (a != theta) MDP_CUDA(cudaMemcpyAsync(theta, a, h->S * sizeof(double), cudaMemcpyDeviceToDevice, st));
  *iters = it;
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

mdp_status inner_solve(mdp_s* h, double gamma, double* theta, int inner, int restart, double omega, double tol,
                       int max_it, int* iters, double* res2, cudaStream_t st) {
  *iters = 0;
  *res2 = 0.0;
  const bool U = h->Ppi.uniform;
  if (inner == MDP_GMRES)
    return U ? gmres<true>(h, gamma, theta, restart, tol, max_it, iters, res2, st)
             : gmres<false>(h, gamma, theta, restart, tol, max_it, iters, res2, st);
  return U ? richardson<true>(h, gamma, theta, omega, tol, max_it, iters, res2, st)
           : richardson<false>(h, gamma, theta, omega, tol, max_it, iters, res2, st);
}

}  // namespace mdp
