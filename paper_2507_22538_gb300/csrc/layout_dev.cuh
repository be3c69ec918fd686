// Device side of the policy-row gather (Algorithm 1 step 4), shared by the
// single-problem kernel and the batched kernel.  The body works on one problem
// with `nb` blocks of which the calling block is number `bid`.
#pragma once

#include "mdp_internal.cuh"

namespace mdp {

// Algorithm 1 step 4: gather the policy's rows r(s) = s*A + pi(s) of the stacked
// matrix into the per-state sliced layout, and g_pi(s) = g(s, pi(s)).  One thread
// per (state, 4-entry chunk) with the state fastest: each warp writes whole
// contiguous chunks and each thread reads one 32-byte run of its row.  States
// whose pi(s) lies outside [0, A) get an empty row (zero values, column 0) and
// g_pi = NaN.  With pcol16 set (the mixed solver of an MDP with 16-bit values whose
// every row stays within 32767 columns of its first column), the rows go out as the
// 16-bit values and column - pcolbase[s] as int16 per entry (offsets 0 for an empty
// row; pcolbase written beforehand by policy_base_body), and no binary64 copy is
// written: every pass of that solver reads the 16-bit rows.
// The 16-bit pattern of a value that is exact in binary16 (store16 = kStoreF16) or
// bfloat16 (checked at creation), from its binary64 fields with integer operations for
// zeros and normal numbers (GB300's FP64 pipe is kept for arithmetic); other values
// take the library conversion.
__device__ __forceinline__ uint16_t narrow_exact(double v, int store16) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 63) << 15;
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  if ((b << 1) == 0ull) return (uint16_t)sign;  // +-0
  if (store16 == kStoreF16) {
    if (e - 1009u < 30u && (b & ((1ull << 42) - 1)) == 0ull)  // normal binary16, no bits lost
      return (uint16_t)(sign | ((e - 1008u) << 10) | (unsigned)((b >> 42) & 0x3ffu));
    return __half_as_ushort(__double2half(v));
  }
  if (e - 897u < 254u && (b & ((1ull << 45) - 1)) == 0ull)  // normal bfloat16, no bits lost
    return (uint16_t)(sign | ((e - 896u) << 7) | (unsigned)((b >> 45) & 0x7fu));
  return __bfloat16_as_ushort(__double2bfloat16(v));
}

__device__ __forceinline__ void put_narrow(float* p32, uint16_t* p16, int store16, int64_t i, double v) {
  if (p32) p32[i] = (float)v;
  if (p16) p16[i] = narrow_exact(v, store16);
}

// The base column of each policy row for the 16-bit offsets: the first column of
// row s*A + pi(s) (0 for an empty row), one thread per state, so that the gather's
// threads read it with one coalesced load per warp instead of each its own sector.
template <bool UNIFORM>
__device__ __forceinline__ void policy_base_body(int bid, int nb, const int32_t* __restrict__ scol,
                                                 const int64_t* __restrict__ off, const int32_t* __restrict__ len,
                                                 int kmax, const int32_t* __restrict__ pi, int64_t S, int A,
                                                 int32_t* __restrict__ pcolbase) {
  for (int64_t s = bid * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)nb * blockDim.x) {
    const int a = pi[s];
    const bool ok = (a >= 0 && a < A);
    const int64_t r = s * A + (ok ? a : 0);
    const int n = !ok ? 0 : (UNIFORM ? kmax : len[r]);
    const int64_t q = r / kSlice;
    const int sw = UNIFORM ? kmax : (int)((off[q + 1] - off[q]) / kSlice);
    const int64_t sbase = UNIFORM ? q * kSlice * (int64_t)kmax : off[q];
    pcolbase[s] = n > 0 ? scol[sell_at(sbase, sw, (int)(r % kSlice), 0)] : 0;
  }
}

template <bool UNIFORM>
__device__ __forceinline__ void extract_policy_body(int bid, int nb, const double* __restrict__ sval, const int32_t* __restrict__ scol,
                                      const int64_t* __restrict__ off, const int32_t* __restrict__ len, int kmax,
                                      const double* __restrict__ g, const int32_t* __restrict__ pi, int64_t S, int A,
                                      double* __restrict__ pval, int32_t* __restrict__ pcol,
                                      const int64_t* __restrict__ poff, int32_t* __restrict__ plen,
                                      double* __restrict__ gpi, float* __restrict__ pval32,
                                      uint16_t* __restrict__ pval16, int store16, int16_t* __restrict__ pcol16,
                                      const int32_t* __restrict__ pcolbase) {
  const int nunits = (kmax + kChunk - 1) / kChunk;
  // chunk u outermost, states grid-strided inside: the work of the flat (u, s) loop
  // without a 64-bit division per unit
  const int64_t start = bid * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)nb * blockDim.x;
  for (int u = 0; u < nunits; ++u) {
    for (int64_t s = start; s < S; s += stride) {
      const int a = pi[s];
      const bool ok = (a >= 0 && a < A);
      const int64_t r = s * A + (ok ? a : 0);
      const int n = !ok ? 0 : (UNIFORM ? kmax : len[r]);
      if (u == 0) {
        if (!UNIFORM) plen[s] = n;
        gpi[s] = ok ? g[r] : __longlong_as_double(0x7ff8000000000000ULL);
      }
      const int64_t ps = s / kSlice, q = r / kSlice;
      const int pw = UNIFORM ? kmax : (int)((poff[ps + 1] - poff[ps]) / kSlice);  // destination slice width
      const int sw = UNIFORM ? kmax : (int)((off[q + 1] - off[q]) / kSlice);      // source slice width
      const int64_t pbase = UNIFORM ? ps * kSlice * (int64_t)kmax : poff[ps];
      const int64_t sbase = UNIFORM ? q * kSlice * (int64_t)kmax : off[q];
      const int pl = (int)(s % kSlice), sl = (int)(r % kSlice);
      const int j0 = u * kChunk;
      const int cbase = pcol16 ? pcolbase[s] : 0;  // the row's first column (policy_base_body)
      if (UNIFORM && ok && j0 + kChunk <= (kmax & ~(kChunk - 1))) {  // whole chunk on both sides
        double v[kChunk];
        int c[kChunk];
        const int64_t si = sell_at(sbase, sw, sl, j0), di = sell_at(pbase, pw, pl, j0);
        load_chunk(sval + si, v);
        load_chunk(scol + si, c);
        if (!pcol16) {
          *reinterpret_cast<double2*>(pval + di) = make_double2(v[0], v[1]);
          *reinterpret_cast<double2*>(pval + di + 2) = make_double2(v[2], v[3]);
          *reinterpret_cast<int4*>(pcol + di) = make_int4(c[0], c[1], c[2], c[3]);
        }
        if (pval32) *reinterpret_cast<float4*>(pval32 + di) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
        if (pval16)
  #pragma unroll
          for (int e = 0; e < kChunk; ++e) put_narrow(nullptr, pval16, store16, di + e, v[e]);
        if (pcol16)
          *reinterpret_cast<short4*>(pcol16 + di) = make_short4((short)(c[0] - cbase), (short)(c[1] - cbase),
                                                                (short)(c[2] - cbase), (short)(c[3] - cbase));
        continue;
      }
      for (int j = j0; j < j0 + kChunk && j < pw; ++j) {
        const int64_t di = sell_at(pbase, pw, pl, j);
        if (j < n) {
          const int64_t si = sell_at(sbase, sw, sl, j);
          const double v = sval[si];
          const int c = scol[si];
          if (pcol16) {
            pcol16[di] = (int16_t)(c - cbase);
          } else {
            pval[di] = v;
            pcol[di] = c;
          }
          put_narrow(pval32, pval16, store16, di, v);
        } else if (UNIFORM) {
          if (pcol16) {
            pcol16[di] = 0;
          } else {
            pval[di] = 0.0;
            pcol[di] = 0;
          }
          put_narrow(pval32, pval16, store16, di, 0.0);
        }
      }
    }
  }
}

}  // namespace mdp
