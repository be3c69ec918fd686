// Device helpers of the chunked sliced-ELL layout (the layout itself is described
// with `Sell` in mdp_internal.cuh): element addressing, 4-entry vector loads and
// the row dot product that every sweep and mat-vec uses.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace mdp {

constexpr int kSlice = 32;  // rows (or states) per sliced-ELL slice: one warp, one row per lane
constexpr int kChunk = 4;  // consecutive entries of one row stored together in a slice

// Index of entry j of lane l in a slice that starts at `base` and is w entries wide.
__host__ __device__ __forceinline__ int64_t sell_at(int64_t base, int w, int lane, int j) {
  const int wc = w & ~(kChunk - 1);
  return base + (j < wc ? (int64_t)(j / kChunk) * (kSlice * kChunk) + lane * kChunk + (j % kChunk)
                        : (int64_t)j * kSlice + lane);
}

// Four consecutive stored values or columns (one chunk) with vector loads; the
// chunk starts on a multiple of 4 elements from a 256-byte aligned slice.
__device__ __forceinline__ void load_chunk(const double* p, double (&v)[kChunk]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void load_chunk(const float* p, float (&v)[kChunk]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}
__device__ __forceinline__ void load_chunk(const __half* p, __half (&v)[kChunk]) {
  const uint2 a = *reinterpret_cast<const uint2*>(p);
  v[0] = __ushort_as_half((unsigned short)(a.x & 0xffffu)), v[1] = __ushort_as_half((unsigned short)(a.x >> 16));
  v[2] = __ushort_as_half((unsigned short)(a.y & 0xffffu)), v[3] = __ushort_as_half((unsigned short)(a.y >> 16));
}
__device__ __forceinline__ void load_chunk(const __nv_bfloat16* p, __nv_bfloat16 (&v)[kChunk]) {
  const uint2 a = *reinterpret_cast<const uint2*>(p);
  v[0] = __ushort_as_bfloat16((unsigned short)(a.x & 0xffffu)), v[1] = __ushort_as_bfloat16((unsigned short)(a.x >> 16));
  v[2] = __ushort_as_bfloat16((unsigned short)(a.y & 0xffffu)), v[3] = __ushort_as_bfloat16((unsigned short)(a.y >> 16));
}
__device__ __forceinline__ void load_chunk(const int32_t* p, int (&v)[kChunk]) {
  const int4 a = *reinterpret_cast<const int4*>(p);
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}

// sum_j val[j] * x[col[j]] over the n entries of lane `lane`'s row in a slice
// (start `base`, width w; n <= w), in ascending j, accumulated in TX.  Full
// chunks go two at a time (8 independent loads in flight), the rest one by one.
template <typename TP, typename TX>
__device__ __forceinline__ TX sell_row_dot(const TP* __restrict__ val, const int32_t* __restrict__ col, int64_t base,
                                           int w, int lane, int n, const TX* __restrict__ x) {
  const TP* vp = val + base + lane * kChunk;
  const int32_t* cp = col + base + lane * kChunk;
  constexpr int64_t kStride = kSlice * kChunk;
  const int nc = n / kChunk;  // n <= w, so full chunks all lie in the chunked part
  TX acc = TX(0);
  int c = 0;
  for (; c + 2 <= nc; c += 2) {
    TP v0[kChunk], v1[kChunk];
    int c0[kChunk], c1[kChunk];
    load_chunk(vp + c * kStride, v0);
    load_chunk(vp + (c + 1) * kStride, v1);
    load_chunk(cp + c * kStride, c0);
    load_chunk(cp + (c + 1) * kStride, c1);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) acc = fma(static_cast<TX>(v0[u]), __ldg(x + c0[u]), acc);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) acc = fma(static_cast<TX>(v1[u]), __ldg(x + c1[u]), acc);
  }
  if (c < nc) {
    TP v0[kChunk];
    int c0[kChunk];
    load_chunk(vp + c * kStride, v0);
    load_chunk(cp + c * kStride, c0);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) acc = fma(static_cast<TX>(v0[u]), __ldg(x + c0[u]), acc);
  }
  for (int j = nc * kChunk; j < n; ++j) {
    const int64_t i = sell_at(base, w, lane, j);
    acc = fma(static_cast<TX>(val[i]), __ldg(x + col[i]), acc);
  }
  return acc;
}

}  // namespace mdp
