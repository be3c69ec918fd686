// Fused Bellman sweep (Eq. 3-4, Algorithm 1 steps 2-3) on one problem: the
// kernel (body in bellman_dev.cuh), its launch shape and its launcher.
#include "bellman_dev.cuh"

namespace mdp {

template <bool UNIFORM>
__global__ void __launch_bounds__(kBellThreads, kBellMinBlocks) bellman_kernel(
    const double* __restrict__ sval, const int32_t* __restrict__ scol, const int64_t* __restrict__ off,
    const int32_t* __restrict__ len, int k, const double* __restrict__ g, const double* __restrict__ V, int64_t S,
    int A, int TS, double gamma, double* __restrict__ TV, int32_t* __restrict__ pi,
    unsigned long long* __restrict__ resmax) {
  bellman_body<UNIFORM>((int)blockIdx.x, (int)gridDim.x, sval, scol, off, len, k, g, V, S, A, TS, gamma, TV, pi, resmax);
}

static size_t bellman_smem(const mdp_s* h) { return (size_t)h->bell_tile_states * h->A * sizeof(double); }
size_t bellman_smem_bytes(const mdp_s* h) { return bellman_smem(h); }

mdp_status configure_bellman(mdp_s* h) {
  const size_t smem = bellman_smem(h);
  MDP_TRY(raise_dyn_smem((const void*)bellman_kernel<true>, smem));
  MDP_TRY(raise_dyn_smem((const void*)bellman_kernel<false>, smem));
  int per_sm = 0;
  if (h->P.uniform)
    MDP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bellman_kernel<true>, kBellThreads, smem));
  else
    MDP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bellman_kernel<false>, kBellThreads, smem));
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
