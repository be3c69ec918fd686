// Device side of the fused Bellman sweep (Eq. 3-4, Algorithm 1 steps 2-3), shared by
// the single-problem kernel and the batched kernel:
//   Q(s,a) = g(s,a) + gamma * sum_j P[s*A+a, j] V[col_j]   (the S*A-long PV, scaled, plus g)
//   TV(s) = min_a Q(s,a), pi(s) = lowest minimising a, residual = max_s |TV(s) - V(s)|
// in one pass over the stacked matrix; Q is never written to memory.
//
// Layout: rows of the stacked matrix in 32-row slices, 4-entry chunks of a row
// side by side inside a slice, so lane l of a warp streams row 32q+l with vector
// loads while the warp reads whole contiguous lines of values and columns.  A
// CTA owns a tile of whole states; Q of the tile goes to shared memory and one
// thread per state takes the min/argmin.  The body works on one problem with
// `nb` blocks of which the calling block is number `bid`.
#pragma once

#include "mdp_internal.cuh"

namespace mdp {

constexpr int kBellThreads = 256;
// At least 6 resident blocks per SM: the register cap (40) keeps the chunk loads
// unspilled and gives 48 warps per SM for the V gathers; at 48 registers (5
// blocks) the full-size sweep measured 4% slower.
constexpr int kBellMinBlocks = 6;

__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }


// Launch-shape variants the tuner picks from (mdp_tune): RPL rows per lane (1: one
// 32-row slice per warp step; 2: two slices, their loads side by side) and V256
// (the binary64 values of a chunk in one 32-byte load instead of two 16-byte ones).
// Every variant computes each row's sum as the same chain of fused multiply-adds,
// so the outputs do not depend on the variant.
template <bool UNIFORM, int RPL = 1, bool V256 = false>
__device__ __forceinline__ void bellman_body(int bid, int nb, 
    const double* __restrict__ sval, const int32_t* __restrict__ scol, const int64_t* __restrict__ off,
    const int32_t* __restrict__ len, int k, const double* __restrict__ g, const double* __restrict__ V, int64_t S,
    int A, int TS, double gamma, double* __restrict__ TV, int32_t* __restrict__ pi,
    unsigned long long* __restrict__ resmax) {
  extern __shared__ double q_s[];  // TS * A values of Q
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  double dmax = 0.0;
  const int64_t ntiles = (S + TS - 1) / TS;
  for (int64_t t = bid; t < ntiles; t += nb) {
    const int64_t s0 = t * TS;
    const int64_t s1 = min(S, s0 + TS);
    const int64_t r0 = s0 * A, r1 = s1 * A;
    const int64_t q0 = r0 / kSlice, q1 = (r1 - 1) / kSlice;
    // phase 1: one row per lane, RPL 32-row slices per warp step
    if constexpr (RPL == 1) {
      for (int64_t q = q0 + warp; q <= q1; q += nwarps) {
        const int64_t r = q * kSlice + lane;
        if (r >= r0 && r < r1) {
          const int n = UNIFORM ? k : len[r];
          const int w = UNIFORM ? k : (int)((off[q + 1] - off[q]) / kSlice);
          const int64_t base = UNIFORM ? q * kSlice * (int64_t)k : off[q];
          const double acc = sell_row_dot<double, double, V256>(sval, scol, base, w, lane, n, V);
          q_s[r - r0] = fma(gamma, acc, g[r]);
        }
      }
    } else {
      static_assert(RPL == 2, "one or two rows per lane");
      for (int64_t q = q0 + 2 * warp; q <= q1; q += 2 * nwarps) {
        const int64_t ra = q * kSlice + lane, rb = ra + kSlice;
        const bool in_a = ra >= r0 && ra < r1, in_b = q + 1 <= q1 && rb >= r0 && rb < r1;
        int na = 0, nb_ = 0, wa = 0, wb = 0;
        int64_t ba = 0, bb = 0;
        if (in_a) {
          na = UNIFORM ? k : len[ra];
          wa = UNIFORM ? k : (int)((off[q + 1] - off[q]) / kSlice);
          ba = UNIFORM ? q * kSlice * (int64_t)k : off[q];
        }
        if (in_b) {
          nb_ = UNIFORM ? k : len[rb];
          wb = UNIFORM ? k : (int)((off[q + 2] - off[q + 1]) / kSlice);
          bb = UNIFORM ? (q + 1) * kSlice * (int64_t)k : off[q + 1];
        }
        double acc_a, acc_b;
        sell_row_dot2<double, double, V256>(sval, scol, ba, wa, na, bb, wb, nb_, lane, V, acc_a, acc_b);
        if (in_a) q_s[ra - r0] = fma(gamma, acc_a, g[ra]);
        if (in_b) q_s[rb - r0] = fma(gamma, acc_b, g[rb]);
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

}  // namespace mdp
