// Fused Bellman sweep (Eq. 3-4, Algorithm 1 steps 2-3, Sec. III-B.3):
//   Q(s,a) = g(s,a) + gamma * sum_j P[s*A+a, j] V[col_j]   (the S*A-long PV, scaled, plus g)
//   TV(s) = min_a Q(s,a), pi(s) = lowest minimising a, residual = max_s |TV(s) - V(s)|
// in one pass over the stacked matrix; Q is never written to memory.
//
// Layout: rows of the stacked matrix in 32-row slices, column-major inside a
// slice, so lane l of a warp streams row 32q+l with fully coalesced loads of
// values and columns.  A CTA owns a tile of whole states; Q of the tile goes
// to shared memory and one thread per state takes the min/argmin.
#include "mdp_internal.cuh"

namespace mdp {

__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

constexpr int kBellThreads = 256;

template <bool UNIFORM>
__global__ void __launch_bounds__(kBellThreads) bellman_kernel(
    const double* __restrict__ sval, const int32_t* __restrict__ scol, const int64_t* __restrict__ off,
    const int32_t* __restrict__ len, int k, const double* __restrict__ g, const double* __restrict__ V, int64_t S,
    int A, int TS, double gamma, double* __restrict__ TV, int32_t* __restrict__ pi,
    unsigned long long* __restrict__ resmax) {
  extern __shared__ double q_s[];  // TS * A values of Q
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  double dmax = 0.0;
  const int64_t ntiles = (S + TS - 1) / TS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t s0 = t * TS;
    const int64_t s1 = min(S, s0 + TS);
    const int64_t r0 = s0 * A, r1 = s1 * A;
    const int64_t q0 = r0 / kSlice, q1 = (r1 - 1) / kSlice;
    // phase 1: one row per lane, one 32-row slice per warp
    for (int64_t q = q0 + warp; q <= q1; q += nwarps) {
      const int64_t r = q * kSlice + lane;
      if (r >= r0 && r < r1) {
        const int n = UNIFORM ? k : len[r];
        const int64_t base = (UNIFORM ? q * kSlice * (int64_t)k : off[q]) + lane;
        const double* vp = sval + base;
        const int32_t* cp = scol + base;
        double acc = 0.0;
        int j = 0;
        for (; j + 8 <= n; j += 8) {
          double v[8];
          int c[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            v[u] = vp[(int64_t)(j + u) * kSlice];
            c[u] = cp[(int64_t)(j + u) * kSlice];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) acc = fma(v[u], __ldg(V + c[u]), acc);
        }
        for (; j < n; ++j) acc = fma(vp[(int64_t)j * kSlice], __ldg(V + cp[(int64_t)j * kSlice]), acc);
        q_s[r - r0] = fma(gamma, acc, g[r]);
      }
    }
    __syncthreads();
    // phase 2: one thread per state, min / argmin over its A contiguous Q values
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
      const double* qs = q_s + (s - s0) * A;
      double best = qs[0];
      int ba = 0;
      bool bad = (best != best);
      for (int a = 1; a < A; ++a) {
        const double qv = qs[a];
        bad |= (qv != qv);
        if (qv < best) {
          best = qv;
          ba = a;
        }
      }
      if (bad) best = __longlong_as_double(0x7ff8000000000000ULL);
      TV[s] = best;
      pi[s] = ba;
      dmax = nan_max(dmax, fabs(best - V[s]));
    }
    __syncthreads();
  }
  // block max of |TV - V|, then one atomic per block on the bit pattern
  // (for nonnegative doubles, and NaN, the unsigned order is the numeric order)
  for (int o = 16; o; o >>= 1) dmax = nan_max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (lane == 0) red[warp] = dmax;
  __syncthreads();
  if (warp == 0) {
    double m = lane < nwarps ? red[lane] : 0.0;
    for (int o = 16; o; o >>= 1) m = nan_max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(resmax, (unsigned long long)__double_as_longlong(m));
  }
}

static size_t bellman_smem(const mdp_s* h) { return (size_t)h->bell_tile_states * h->A * sizeof(double); }

mdp_status configure_bellman(mdp_s* h) {
  const size_t smem = bellman_smem(h);
  if (smem > 48 * 1024) {
    MDP_CUDA(cudaFuncSetAttribute(bellman_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MDP_CUDA(cudaFuncSetAttribute(bellman_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int per_sm = 0;
  if (h->P.uniform)
    MDP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bellman_kernel<true>, kBellThreads, smem));
  else
    MDP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bellman_kernel<false>, kBellThreads, smem));
  if (per_sm < 1) return fail(MDP_ERR_INVALID_ARG, "Bellman tile does not fit on an SM (too many actions)");
  const int64_t ntiles = (h->S + h->bell_tile_states - 1) / h->bell_tile_states;
  h->bell_threads = kBellThreads;
  h->bell_blocks = (int)std::min<int64_t>(ntiles, (int64_t)h->sm_count * per_sm);
  return MDP_OK;
}

mdp_status launch_bellman(mdp_s* h, double gamma, const double* V, double* TV, int32_t* pi, cudaStream_t st) {
  MDP_CUDA(cudaMemsetAsync(h->resmax, 0, sizeof(unsigned long long), st));
  const size_t smem = bellman_smem(h);
  const Sell& P = h->P;
  if (P.uniform)
    bellman_kernel<true><<<h->bell_blocks, kBellThreads, smem, st>>>(P.val, P.col, P.off, P.len, P.kmax, h->g, V,
                                                                      h->S, h->A, h->bell_tile_states, gamma, TV, pi,
                                                                      h->resmax);
  else
    bellman_kernel<false><<<h->bell_blocks, kBellThreads, smem, st>>>(P.val, P.col, P.off, P.len, 0, h->g, V, h->S,
                                                                       h->A, h->bell_tile_states, gamma, TV, pi,
                                                                       h->resmax);
  h->launches++;
  MDP_CUDA(cudaGetLastError());
  return MDP_OK;
}

}  // namespace mdp
