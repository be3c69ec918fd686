// Device draw of one request of the counter-based serving stream
// (mdpgen.generators.serving_request_philox): input generation only, no MDP
// arithmetic.  One thread per row: Philox4x32-10 (Salmon et al., SC 2011) at
// row counter rid * 2^40 + r, k columns floor(U * S) sorted ascending, weights
// -log(1 - U) normalised by their sum, cost U[0, 1).  Columns and costs equal
// the numpy draw bit for bit; probabilities agree to rounding (log1p and the
// row sum may differ in the last bit between libraries).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u, kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
constexpr uint32_t kTagCols = 0x636F6C73u, kTagVals = 0x76616C73u, kTagCost = 0x636F7374u;
constexpr int kMaxK = 64;

__device__ __forceinline__ void philox(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kM0 * c[0], p1 = (uint64_t)kM1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += kW0;
    k1 += kW1;
  }
}

// uniform double in [0, 1) from words 0 and 1 of the block at (row, block)
__device__ __forceinline__ double uniform(uint32_t seed, uint32_t tag, uint64_t row, uint64_t block) {
  uint32_t c[4] = {(uint32_t)row, (uint32_t)(row >> 32), (uint32_t)block, (uint32_t)(block >> 32)};
  philox(c, seed, tag);
  const uint64_t m = ((uint64_t)(c[0] >> 5) << 26) + (c[1] >> 6);
  return (double)m * 0x1.0p-53;
}

__global__ void request_kernel(uint32_t seed, uint64_t base, int64_t S, int64_t R, int k, int32_t* __restrict__ col,
                               double* __restrict__ val, double* __restrict__ g) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t row = base + (uint64_t)r;
    int64_t c[kMaxK];
    for (int j = 0; j < k; ++j) {
      const double u = uniform(seed, kTagCols, row, (uint64_t)j);
      int64_t t = (int64_t)floor(u * (double)S);
      c[j] = t < S - 1 ? t : S - 1;
    }
    for (int j = 1; j < k; ++j) {  // insertion sort, ascending
      const int64_t x = c[j];
      int q = j - 1;
      while (q >= 0 && c[q] > x) {
        c[q + 1] = c[q];
        --q;
      }
      c[q + 1] = x;
    }
    double w[kMaxK];
    double sum = 0.0;
    for (int j = 0; j < k; ++j) {
      w[j] = -log1p(-uniform(seed, kTagVals, row, (uint64_t)(k + j)));
      sum += w[j];
    }
    for (int j = 0; j < k; ++j) {
      col[r * k + j] = (int32_t)c[j];
      val[r * k + j] = w[j] / sum;
    }
    g[r] = uniform(seed, kTagCost, row, 0);
  }
}

}  // namespace

extern "C" int mdpgen_request(uint32_t seed, uint64_t rid, int64_t S, int32_t A, int32_t k, int32_t* col, double* val,
                              double* g, void* stream) {
  if (S < 1 || A < 1 || k < 1 || k > kMaxK || !col || !val || !g) return 1;
  const int64_t R = S * (int64_t)A;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = (R + 127) / 128;
  const int grid = (int)(blocks < (int64_t)sms * 16 ? blocks : (int64_t)sms * 16);
  request_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(seed, rid << 40, S, R, k, col, val, g);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
