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
// 16-bit column offsets (the mixed solver's policy rows of a near-diagonal matrix)
__device__ __forceinline__ void load_chunk(const int16_t* p, int (&v)[kChunk]) {
  const short4 a = *reinterpret_cast<const short4*>(p);
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}

// A stored value in the accumulation type TX.  A binary16 or bfloat16 value becomes
// binary64 by rebuilding its IEEE fields with integer operations and selects, no
// branch (normal numbers, zeros, subnormals -- normalised by their leading bit --,
// infinities and NaNs): the same value, without spending GB300's scarce FP64 pipe on
// a format conversion per entry.  `mb` mantissa bits, exponent field width `eb`.
template <int mb, int eb>
__device__ __forceinline__ double widen_bits(unsigned b) {
  constexpr unsigned kEmax = (1u << eb) - 1u;
  constexpr int kBias = (1 << (eb - 1)) - 1;
  const unsigned e = (b >> mb) & kEmax, m = b & ((1u << mb) - 1u);
  const int p = 31 - __clz(m);  // leading bit of a subnormal's mantissa (m > 0)
  // binary64 exponent field: normal e - bias + 1023; subnormal p - (bias - 1 + mb) + 1023
  const unsigned E = e == kEmax ? 2047u : (e != 0u ? e + (1023u - kBias) : (m != 0u ? (unsigned)(p + 1024 - kBias - mb) : 0u));
  const unsigned long long M = e != 0u ? (unsigned long long)m << (52 - mb)
                                       : ((unsigned long long)m << (52 - p)) & ((1ull << 52) - 1ull);  // m = 0: 0
  return __longlong_as_double((long long)(((unsigned long long)(b >> (mb + eb)) << 63) | ((unsigned long long)E << 52) | M));
}
template <typename TX, typename TP>
__device__ __forceinline__ TX widen(TP v) {
  return static_cast<TX>(v);
}
template <>
__device__ __forceinline__ double widen<double, __half>(__half v) {
  return widen_bits<10, 5>(__half_as_ushort(v));
}
template <>
__device__ __forceinline__ double widen<double, __nv_bfloat16>(__nv_bfloat16 v) {
  return widen_bits<7, 8>(__bfloat16_as_ushort(v));
}

// One chunk of binary64 values with a single 32-byte load (256-bit vector load of the
// read-only path); the chunk starts on a 32-byte boundary (a multiple of 4 elements
// from a 256-byte aligned slice).
__device__ __forceinline__ void load_chunk_v256(const double* p, double (&v)[kChunk]) {
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
}

// The value load of one chunk: two 16-byte loads (load_chunk), or with V256 (binary64
// only) one 32-byte load.  The launch-shape tuner picks the width per matrix.
template <bool V256, typename TP>
__device__ __forceinline__ void load_vals(const TP* p, TP (&v)[kChunk]) {
  if constexpr (V256 && sizeof(TP) == sizeof(double))
    load_chunk_v256(reinterpret_cast<const double*>(p), reinterpret_cast<double(&)[kChunk]>(v));
  else
    load_chunk(p, v);
}

// sum_j val[j] * x[col[j]] over the n entries of lane `lane`'s row in a slice
// (start `base`, width w; n <= w), in ascending j, accumulated in TX.  Full
// chunks go two at a time (8 independent loads in flight), the rest one by one.
// TC is int32_t (columns) or int16_t (offsets from a base the caller folds into x).
template <typename TP, typename TX, bool V256 = false, typename TC = int32_t>
__device__ __forceinline__ TX sell_row_dot(const TP* __restrict__ val, const TC* __restrict__ col, int64_t base,
                                           int w, int lane, int n, const TX* __restrict__ x) {
  const TP* vp = val + base + lane * kChunk;
  const TC* cp = col + base + lane * kChunk;
  constexpr int64_t kStride = kSlice * kChunk;
  const int nc = n / kChunk;  // n <= w, so full chunks all lie in the chunked part
  TX acc = TX(0);
  int c = 0;
  for (; c + 2 <= nc; c += 2) {
    TP v0[kChunk], v1[kChunk];
    int c0[kChunk], c1[kChunk];
    load_vals<V256>(vp + c * kStride, v0);
    load_vals<V256>(vp + (c + 1) * kStride, v1);
    load_chunk(cp + c * kStride, c0);
    load_chunk(cp + (c + 1) * kStride, c1);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) acc = fma(widen<TX>(v0[u]), __ldg(x + c0[u]), acc);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) acc = fma(widen<TX>(v1[u]), __ldg(x + c1[u]), acc);
  }
  if (c < nc) {
    TP v0[kChunk];
    int c0[kChunk];
    load_vals<V256>(vp + c * kStride, v0);
    load_chunk(cp + c * kStride, c0);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) acc = fma(widen<TX>(v0[u]), __ldg(x + c0[u]), acc);
  }
  for (int j = nc * kChunk; j < n; ++j) {
    const int64_t i = sell_at(base, w, lane, j);
    acc = fma(widen<TX>(val[i]), __ldg(x + col[i]), acc);
  }
  return acc;
}

// Two rows per lane (lane `lane` of two slices, starts base0/base1, widths w0/w1,
// n0/n1 entries; n = 0 for a row the lane does not own): the chunks of both rows are
// loaded side by side, so a warp keeps twice the loads in flight with the same
// registers per row, while each row's sum is the same chain of fused multiply-adds,
// in the same order, as sell_row_dot's: the results are equal bit for bit.
template <typename TP, typename TX, bool V256 = false>
__device__ __forceinline__ void sell_row_dot2(const TP* __restrict__ val, const int32_t* __restrict__ col,
                                              int64_t base0, int w0, int n0, int64_t base1, int w1, int n1,
                                              int lane, const TX* __restrict__ x, TX& acc0, TX& acc1) {
  constexpr int64_t kStride = kSlice * kChunk;
  const TP* vp0 = val + base0 + lane * kChunk;
  const int32_t* cp0 = col + base0 + lane * kChunk;
  const TP* vp1 = val + base1 + lane * kChunk;
  const int32_t* cp1 = col + base1 + lane * kChunk;
  const int nc0 = n0 / kChunk, nc1 = n1 / kChunk;
  const int nc = nc0 > nc1 ? nc0 : nc1;
  acc0 = TX(0);
  acc1 = TX(0);
  for (int c = 0; c < nc; ++c) {
    TP v0[kChunk], v1[kChunk];
    int c0[kChunk], c1[kChunk];
    const bool has0 = c < nc0, has1 = c < nc1;
    if (has0) {
      load_vals<V256>(vp0 + c * kStride, v0);
      load_chunk(cp0 + c * kStride, c0);
    }
    if (has1) {
      load_vals<V256>(vp1 + c * kStride, v1);
      load_chunk(cp1 + c * kStride, c1);
    }
    if (has0) {
#pragma unroll
      for (int u = 0; u < kChunk; ++u) acc0 = fma(widen<TX>(v0[u]), __ldg(x + c0[u]), acc0);
    }
    if (has1) {
#pragma unroll
      for (int u = 0; u < kChunk; ++u) acc1 = fma(widen<TX>(v1[u]), __ldg(x + c1[u]), acc1);
    }
  }
  for (int j = nc0 * kChunk; j < n0; ++j) {
    const int64_t i = sell_at(base0, w0, lane, j);
    acc0 = fma(widen<TX>(val[i]), __ldg(x + col[i]), acc0);
  }
  for (int j = nc1 * kChunk; j < n1; ++j) {
    const int64_t i = sell_at(base1, w1, lane, j);
    acc1 = fma(widen<TX>(val[i]), __ldg(x + col[i]), acc1);
  }
}

}  // namespace mdp
