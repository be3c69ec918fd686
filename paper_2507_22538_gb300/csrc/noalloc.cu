// mdp_bellman_csr_noalloc: one Bellman application computed straight from the
// caller's CSR arrays, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// handed out by their own pool or a framework's caching allocator, which must
// not be fragmented or exhausted behind its back; plug-ins called back from a
// host program that owns the device and forbids allocation inside the call;
// and real-time control loops where an allocation (and the device-wide
// synchronisation it can cause) would break the loop's deadline.  They also
// cannot create an mdp_handle, because mdp_create allocates the device layout.
//
// This entry point needs no handle and allocates nothing.  The only scratch it
// uses (one residual maximum per 32-state tile, plus a completion counter) lives
// in a file-scope __device__ array of fixed size that every GPU loading the
// library keeps until the process exits.  Host code must not pass the array's
// name to a kernel (on the host that name is only a stand-in, not a device
// address), so its device address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include <mutex>

#include "mdp_internal.cuh"

namespace mdp {
namespace {

constexpr int kNaTileStates = 32;               // states per CTA tile
constexpr int64_t kNaMaxTiles = 65536;          // scratch slots: S <= 65536 * 32
constexpr int kNaMaxActions = 128;              // Q tile in shared memory: 32 * 128 doubles
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

// [0, kNaMaxTiles): per-tile residual maxima (bit patterns); [kNaMaxTiles]: tiles finished.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNaMaxTiles + 32];

std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_ptr[kNaMaxDevices] = {};

__device__ __forceinline__ double na_nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

// One CTA per tile of 32 states.  Phase 1: one warp per row of Eq. 5, lanes
// striding over the row's CSR entries, shuffle sum, Q = g + gamma * PV into
// shared memory.  Phase 2: one thread per state, min / lowest argmin, |TV - V|.
// The tile's maximum goes to scratch[tile]; the last CTA to finish reduces all
// tiles in index order into *residual_inf.
__global__ void __launch_bounds__(kNaThreads) bellman_csr_noalloc_kernel(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const double* __restrict__ val,
    const double* __restrict__ g, const double* __restrict__ V, int64_t S, int A, double gamma,
    double* __restrict__ TV, int32_t* __restrict__ pi, double* __restrict__ residual_inf,
    unsigned long long* __restrict__ scratch, int64_t ntiles) {
  __shared__ double q_s[kNaTileStates * kNaMaxActions];
  __shared__ double red[kNaThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = kNaThreads / 32;
  const int64_t tile = blockIdx.x;
  const int64_t s0 = tile * kNaTileStates;
  const int64_t s1 = min(S, s0 + kNaTileStates);
  const int64_t r0 = s0 * A, r1 = s1 * A;
  for (int64_t r = r0 + warp; r < r1; r += nwarps) {
    const int64_t lo = rp[r], hi = rp[r + 1];
    double acc = 0.0;
    for (int64_t j = lo + lane; j < hi; j += 32) acc = fma(val[j], __ldg(V + col[j]), acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) q_s[r - r0] = fma(gamma, acc, g[r]);
  }
  __syncthreads();
  double dmax = 0.0;
  for (int64_t s = s0 + threadIdx.x; s < s1; s += kNaThreads) {
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
    dmax = na_nan_max(dmax, fabs(best - V[s]));
  }
  for (int o = 16; o; o >>= 1) dmax = na_nan_max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (lane == 0) red[warp] = dmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < nwarps; ++w) m = na_nan_max(m, red[w]);
    scratch[tile] = (unsigned long long)__double_as_longlong(m);
    __threadfence();
    const unsigned long long done = atomicAdd(&scratch[kNaMaxTiles], 1ULL);
    last = (done == (unsigned long long)(ntiles - 1));
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double m = 0.0;
    for (int64_t t = threadIdx.x; t < ntiles; t += kNaThreads)
      m = na_nan_max(m, __longlong_as_double((long long)(((volatile unsigned long long*)scratch)[t])));
    for (int o = 16; o; o >>= 1) m = na_nan_max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) t = na_nan_max(t, red[w]);
      if (residual_inf) *residual_inf = t;
    }
  }
}

// Device address of the scratch array on the current device, looked up once per device.
mdp_status noalloc_scratch(unsigned long long** out) {
  int dev = 0;
  MDP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail(MDP_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = (unsigned long long*)p;
  }
  *out = g_noalloc_ptr[dev];
  return MDP_OK;
}

}  // namespace
}  // namespace mdp

using namespace mdp;

extern "C" mdp_status mdp_bellman_csr_noalloc(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col,
                                              const double* val, const double* g, double gamma, const double* V,
                                              double* TV, int32_t* pi, double* residual_inf, void* stream) {
  if (S < 1 || A < 1) return fail(MDP_ERR_INVALID_ARG, "need S >= 1 and A >= 1");
  if (A > kNaMaxActions)
    return fail(MDP_ERR_INVALID_ARG, "mdp_bellman_csr_noalloc supports at most 128 actions");
  const int64_t ntiles = (S + kNaTileStates - 1) / kNaTileStates;
  if (ntiles > kNaMaxTiles)
    return fail(MDP_ERR_INVALID_ARG,
                "mdp_bellman_csr_noalloc supports at most 2097152 states (65536 tiles of 32 in its fixed scratch)");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
  if (!row_ptr || !col || !val || !g || !V || !TV || !pi) return fail(MDP_ERR_INVALID_ARG, "null array");
  // the outputs are written while other tiles still read V, g and the row pointers:
  // no output may share a byte with another output or with those inputs
  {
    const uint64_t R = (uint64_t)S * (uint64_t)A;
    const struct { const void* p; uint64_t n; } in[] = {{V, (uint64_t)S * 8}, {g, R * 8}, {row_ptr, (R + 1) * 8}},
                                                 out[] = {{TV, (uint64_t)S * 8}, {pi, (uint64_t)S * 4},
                                                          {residual_inf, residual_inf ? 8u : 0u}};
    auto overlap = [](const void* a, uint64_t na, const void* b, uint64_t nb) {
      const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
      return na && nb && x < y + nb && y < x + na;
    };
    for (int i = 0; i < 3; ++i) {
      for (const auto& r : in)
        if (overlap(out[i].p, out[i].n, r.p, r.n))
          return fail(MDP_ERR_INVALID_ARG, "TV, pi and residual_inf may not overlap V, g or row_ptr");
      for (int j = i + 1; j < 3; ++j)
        if (overlap(out[i].p, out[i].n, out[j].p, out[j].n))
          return fail(MDP_ERR_INVALID_ARG, "TV, pi and residual_inf may not overlap one another");
    }
  }
  unsigned long long* scratch = nullptr;
  mdp_status s = noalloc_scratch(&scratch);
  if (s != MDP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // the completion counter must start at zero; the per-tile slots are overwritten
  MDP_CUDA(cudaMemsetAsync(scratch + kNaMaxTiles, 0, sizeof(unsigned long long), st));
  bellman_csr_noalloc_kernel<<<(unsigned)ntiles, kNaThreads, 0, st>>>(row_ptr, col, val, g, V, S, A, gamma, TV, pi,
                                                                     residual_inf, scratch, ntiles);
  MDP_CUDA(cudaGetLastError());
  return MDP_OK;
}
