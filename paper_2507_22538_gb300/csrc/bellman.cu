// Fused Bellman sweep (Eq. 3-4, Algorithm 1 steps 2-3) on one problem: the
// kernel (body in bellman_dev.cuh), its launch shape and its launcher.
#include <algorithm>

#include "bellman_dev.cuh"

namespace mdp {

// Resident blocks per SM the register budget is sized for: one row per lane fits
// in 40 registers (6 blocks); two rows per lane take about twice the row state.
__host__ __device__ constexpr int bell_min_blocks(int rpl) { return rpl == 1 ? kBellMinBlocks : 4; }

template <bool UNIFORM, int RPL, bool V256>
__global__ void __launch_bounds__(kBellThreads, bell_min_blocks(RPL)) bellman_kernel(
    const double* __restrict__ sval, const int32_t* __restrict__ scol, const int64_t* __restrict__ off,
    const int32_t* __restrict__ len, int k, const double* __restrict__ g, const double* __restrict__ V, int64_t S,
    int A, int TS, double gamma, double* __restrict__ TV, int32_t* __restrict__ pi,
    unsigned long long* __restrict__ resmax) {
  bellman_body<UNIFORM, RPL, V256>((int)blockIdx.x, (int)gridDim.x, sval, scol, off, len, k, g, V, S, A, TS, gamma,
                                   TV, pi, resmax);
}

namespace {

using BellKernel = void (*)(const double*, const int32_t*, const int64_t*, const int32_t*, int, const double*,
                            const double*, int64_t, int, int, double, double*, int32_t*, unsigned long long*);

// The kernel of a handle's launch-shape variant (rows per lane, value load width).
BellKernel bell_kernel(bool uniform, int rpl, bool v256) {
  if (uniform) {
    if (rpl == 2) return v256 ? bellman_kernel<true, 2, true> : bellman_kernel<true, 2, false>;
    return v256 ? bellman_kernel<true, 1, true> : bellman_kernel<true, 1, false>;
  }
  if (rpl == 2) return v256 ? bellman_kernel<false, 2, true> : bellman_kernel<false, 2, false>;
  return v256 ? bellman_kernel<false, 1, true> : bellman_kernel<false, 1, false>;
}

}  // namespace

static size_t bellman_smem(const mdp_s* h) { return (size_t)h->bell_tile_states * h->A * sizeof(double); }
size_t bellman_smem_bytes(const mdp_s* h) { return bellman_smem(h); }

mdp_status configure_bellman(mdp_s* h) {
  const size_t smem = bellman_smem(h);
  if (h->bell_rpl != 1 && h->bell_rpl != 2) h->bell_rpl = 1;
  const BellKernel kern = bell_kernel(h->P.uniform, h->bell_rpl, h->bell_v256 != 0);
  MDP_TRY(raise_dyn_smem((const void*)kern, smem));
  int per_sm = 0;
  MDP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBellThreads, smem));
  if (per_sm < 1) return fail(MDP_ERR_INVALID_ARG, "Bellman tile does not fit on an SM (too many actions)");
  h->bell_max_per_sm = per_sm;
  if (h->bell_per_sm_cap > 0) per_sm = std::min(per_sm, h->bell_per_sm_cap);  // chosen by mdp_tune
  const int64_t ntiles = (h->S + h->bell_tile_states - 1) / h->bell_tile_states;
  h->bell_threads = kBellThreads;
  h->bell_blocks = (int)std::min<int64_t>(ntiles, (int64_t)h->sm_count * per_sm);
  return MDP_OK;
}

mdp_status launch_bellman(mdp_s* h, double gamma, const double* V, double* TV, int32_t* pi, cudaStream_t st) {
  MDP_CUDA(cudaMemsetAsync(h->resmax, 0, sizeof(unsigned long long), st));
  const size_t smem = bellman_smem(h);
  const Sell& P = h->P;
  const BellKernel kern = bell_kernel(P.uniform, h->bell_rpl, h->bell_v256 != 0);
  kern<<<h->bell_blocks, kBellThreads, smem, st>>>(P.val, P.col, P.off, P.len, P.uniform ? P.kmax : 0, h->g, V, h->S,
                                                   h->A, h->bell_tile_states, gamma, TV, pi, h->resmax);
  h->launches++;
  MDP_CUDA(cudaGetLastError());
  return MDP_OK;
}

}  // namespace mdp
