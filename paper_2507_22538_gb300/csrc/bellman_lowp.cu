// Certified low-precision Bellman sweep (Eq. 3-4, Algorithm 1 steps 2-3) for MDPs
// whose probabilities are exact in binary16 or bfloat16 (multiples of 2^-11 or
// 2^-8 summing to 1, the exact-dyadic inputs of the mixed-precision path).
//
// The sweep reads the stacked matrix as 16-bit values (2 B instead of 8 B per
// entry) and screens every row in binary32:
//   q~(s,a) = fl32(gamma_f * sum_j p_j Vf[col_j] + g_f),  Vf = fl32(V), g_f = fl32(g)
// with a rigorous bound e(s,a) >= |q~(s,a) - Q(s,a)|, where Q(s,a) is the value the
// binary64 sweep computes for that row (same summation order, fma(gamma, acc, g)).
// An action a can attain the binary64 minimum only if q~ - e <= min_b (q~ + e);
// every other action's Q exceeds the minimum.  Those candidate rows, and all rows
// of a state whose screen is not finite, are evaluated again in binary64 exactly as
// the binary64 sweep evaluates them, and the min/argmin/residual phase is the
// binary64 sweep's own.  TV, pi and ||TV - V||_inf are therefore bit for bit those
// of the binary64 sweep, while the bulk of the bytes moves in 16 bits and the bulk
// of the arithmetic runs on the binary32 pipe.
//
// The bound.  Let n be the row length, u = 2^-24 (binary32 unit roundoff) and
// M = fl32(sum_j p_j |Vf_j|) the screened magnitude sum.  With p_j >= 0 exact,
//   |sum p_j Vf_j - sum p_j V_j| <= u sum p_j |V_j|            (rounding V)
//   |acc - sum p_j Vf_j|          <= gamma_n sum p_j |Vf_j|     (recursive fma sum;
//                                     gamma_n = n u / (1 - n u), Higham Sec. 3.1)
//   sum p_j |Vf_j|                <= M / (1 - gamma_n)
// and the binary64 dot is off from the exact sum by at most gamma_n(binary64) times
// the same magnitude.  With n <= 16382 (n u <= 2^-10) these add up to less than
// (2n + 5.1) u M; the rounding of gamma to binary32 adds u gamma M, the final fma
// and the rounding of g add u (|q~| + |g_f|), the binary64 sweep's own last
// rounding is below 2^-53 |Q|, and gradual underflow adds at most n 2^-150.
//   e = gamma_f (n + 4) 2^-23 M + 2^-22 (|q~| + |g_f|) + 2^-120
// covers all of it with at least a factor 1.9 to spare, which also absorbs the
// rounding of e itself and of q~ -+ e.  Rows longer than 16382 entries, and any
// non-finite q~ or e (V beyond binary32 range, NaN, Inf), send every action of
// the state to binary64.
#include "bellman_dev.cuh"

namespace mdp {

constexpr int kLowpMaxRowLen = 16382;
// Shared memory per row of a tile: 8 bytes that hold the row's bounds (lo, hi in
// binary32) until its state's candidates are chosen and its binary64 Q after that,
// and the candidate list (row index within the tile, < 2^16).
constexpr int kLowpSmemPerRow = 8 + 2;

__device__ __forceinline__ float lp_to_float(__half v) { return __half2float(v); }
__device__ __forceinline__ float lp_to_float(__nv_bfloat16 v) { return __bfloat162float(v); }

// binary32 screen of one row: acc = sum_j p_j x[col_j] and mag = sum_j p_j |x[col_j]|
// in ascending j (the row walk of sell_row_dot).
template <typename TP, typename TC>
__device__ __forceinline__ void lowp_row_dot(const TP* __restrict__ val, const TC* __restrict__ col,
                                             int64_t base, int w, int lane, int n, const float* __restrict__ x,
                                             float& acc, float& mag) {
  const TP* vp = val + base + lane * kChunk;
  const TC* cp = col + base + lane * kChunk;
  constexpr int64_t kStride = kSlice * kChunk;
  const int nc = n / kChunk;
  float a = 0.f, m = 0.f;
  int c = 0;
  for (; c + 2 <= nc; c += 2) {
    TP v0[kChunk], v1[kChunk];
    int c0[kChunk], c1[kChunk];
    load_chunk(vp + c * kStride, v0);
    load_chunk(vp + (c + 1) * kStride, v1);
    load_chunk(cp + c * kStride, c0);
    load_chunk(cp + (c + 1) * kStride, c1);
    float x0[kChunk], x1[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) x0[u] = __ldg(x + c0[u]);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) x1[u] = __ldg(x + c1[u]);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const float p = lp_to_float(v0[u]);
      a = fmaf(p, x0[u], a);
      m = fmaf(p, fabsf(x0[u]), m);
    }
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const float p = lp_to_float(v1[u]);
      a = fmaf(p, x1[u], a);
      m = fmaf(p, fabsf(x1[u]), m);
    }
  }
  if (c < nc) {
    TP v0[kChunk];
    int c0[kChunk];
    load_chunk(vp + c * kStride, v0);
    load_chunk(cp + c * kStride, c0);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const float p = lp_to_float(v0[u]);
      const float xv = __ldg(x + c0[u]);
      a = fmaf(p, xv, a);
      m = fmaf(p, fabsf(xv), m);
    }
  }
  for (int j = nc * kChunk; j < n; ++j) {
    const int64_t i = sell_at(base, w, lane, j);
    const float p = lp_to_float(val[i]);
    const float xv = __ldg(x + col[i]);
    a = fmaf(p, xv, a);
    m = fmaf(p, fabsf(xv), m);
  }
  acc = a;
  mag = m;
}

// TC: int32_t columns, or int16_t offsets from each row's first column (cbase[r]; the
// MDP's every row within 32767 columns of its first): 4 instead of 6 bytes per entry.
template <bool UNIFORM, typename TP, typename TC>
__global__ void __launch_bounds__(kBellThreads, kBellMinBlocks) bellman_lowp_kernel(
    const TP* __restrict__ sval, const TC* __restrict__ scol, const int32_t* __restrict__ cbase,
    const int64_t* __restrict__ off,
    const int32_t* __restrict__ len, int k, const float* __restrict__ g32, const double* __restrict__ g,
    const float* __restrict__ Vf, const double* __restrict__ V, int64_t S, int A, int TS, double gamma, float gammaf,
    double* __restrict__ TV, int32_t* __restrict__ pi, unsigned long long* __restrict__ resmax,
    unsigned long long* __restrict__ rows64) {
  extern __shared__ double lp_smem[];
  __shared__ double red[32];
  __shared__ int ncand;
  const int nr = TS * A;
  double* qd = lp_smem;                                           // [nr] binary64 Q (phases 2-4)
  float2* lohi = reinterpret_cast<float2*>(lp_smem);              // [nr] the same bytes: bounds (phases 1-2)
  uint16_t* list = reinterpret_cast<uint16_t*>(qd + nr);          // [nr]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  double dmax = 0.0;
  unsigned long long cand_total = 0;
  const int64_t ntiles = (S + TS - 1) / TS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t s0 = t * TS;
    const int64_t s1 = min(S, s0 + TS);
    const int64_t r0 = s0 * A, r1 = s1 * A;
    const int64_t q0 = r0 / kSlice, q1 = (r1 - 1) / kSlice;
    if (threadIdx.x == 0) ncand = 0;
    // phase 1: binary32 screen, one row per lane, one 32-row slice per warp
    for (int64_t q = q0 + warp; q <= q1; q += nwarps) {
      const int64_t r = q * kSlice + lane;
      if (r >= r0 && r < r1) {
        const int n = UNIFORM ? k : len[r];
        const int w = UNIFORM ? k : (int)((off[q + 1] - off[q]) / kSlice);
        const int64_t base = UNIFORM ? q * kSlice * (int64_t)k : off[q];
        float acc, mag;
        const float* xr = Vf;
        if constexpr (sizeof(TC) == sizeof(int16_t)) xr = Vf + cbase[r];
        lowp_row_dot(sval, scol, base, w, lane, n, xr, acc, mag);
        const float gq = g32[r];
        const float qt = fmaf(gammaf, acc, gq);
        const float e = gammaf * ((float)(n + 4) * 0x1p-23f) * mag + 0x1p-22f * (fabsf(qt) + fabsf(gq)) + 0x1p-120f;
        const bool ok = n <= kLowpMaxRowLen && isfinite(qt) && isfinite(e);
        const float nan = __int_as_float(0x7fc00000);
        lohi[r - r0] = ok ? make_float2(qt - e, qt + e) : make_float2(nan, nan);
      }
    }
    __syncthreads();
    // phase 2: one thread per state picks the rows that can attain the binary64 minimum
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
      const int b = (int)(s - s0) * A;
      bool all = false;
      float U = __int_as_float(0x7f800000);
      for (int a = 0; a < A; ++a) {
        const float2 bnd = lohi[b + a];
        all |= (bnd.x != bnd.x);
        U = fminf(U, bnd.y);
      }
      for (int a = 0; a < A; ++a) {
        const bool cand = all || lohi[b + a].x <= U;  // read this row's bounds before its Q overwrites them
        qd[b + a] = __longlong_as_double(0x7ff0000000000000LL);  // +inf: never the minimum
        if (cand) list[atomicAdd(&ncand, 1)] = (uint16_t)(b + a);
      }
    }
    __syncthreads();
    // phase 3: the candidate rows in binary64, exactly as the binary64 sweep (the
    // 16-bit values widen exactly)
    const int nc = ncand;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
      const int lr = list[i];
      const int64_t r = r0 + lr;
      const int64_t q = r / kSlice;
      const int ln = (int)(r % kSlice);
      const int n = UNIFORM ? k : len[r];
      const int w = UNIFORM ? k : (int)((off[q + 1] - off[q]) / kSlice);
      const int64_t base = UNIFORM ? q * kSlice * (int64_t)k : off[q];
      const double* xr = V;
      if constexpr (sizeof(TC) == sizeof(int16_t)) xr = V + cbase[r];
      const double acc = sell_row_dot<TP, double, false, TC>(sval, scol, base, w, ln, n, xr);
      qd[lr] = fma(gamma, acc, g[r]);
    }
    if (threadIdx.x == 0) cand_total += (unsigned long long)nc;
    __syncthreads();
    // phase 4: the binary64 sweep's min / lowest argmin over the tile's Q
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
      const double* qs = qd + (s - s0) * A;
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
  for (int o = 16; o; o >>= 1) dmax = nan_max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (lane == 0) red[warp] = dmax;
  __syncthreads();
  if (warp == 0) {
    double m = lane < nwarps ? red[lane] : 0.0;
    for (int o = 16; o; o >>= 1) m = nan_max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(resmax, (unsigned long long)__double_as_longlong(m));
  }
  if (threadIdx.x == 0 && rows64) atomicAdd(rows64, cand_total);
}

// V -> binary32 (round to nearest) for the screen's gathers.
__global__ void __launch_bounds__(256) lowp_v32_kernel(const double* __restrict__ V, float* __restrict__ Vf, int64_t S) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x)
    Vf[s] = __double2float_rn(V[s]);
}

// The 16-bit copy of the stacked matrix's values (exact: checked at creation) and
// binary32 costs.
template <bool BF16>
__global__ void __launch_bounds__(256) lowp_pack_kernel(const double* __restrict__ sval, int64_t nstored,
                                                        uint16_t* __restrict__ out, const double* __restrict__ g,
                                                        int64_t R, float* __restrict__ g32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nstored; i += stride)
    out[i] = BF16 ? __bfloat16_as_ushort(__double2bfloat16(sval[i])) : __half_as_ushort(__double2half(sval[i]));
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += stride) g32[r] = __double2float_rn(g[r]);
}

// The 16-bit column offsets of the stacked matrix (with col16): each row's first
// column as its base, every entry's column minus that base (one thread per row).
template <bool UNIFORM>
__global__ void __launch_bounds__(256) lowp_col16_kernel(const int32_t* __restrict__ col, const int64_t* __restrict__ off,
                                                         const int32_t* __restrict__ len, int k, int64_t R,
                                                         int16_t* __restrict__ col16, int32_t* __restrict__ base) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = r / kSlice;
    const int lane = (int)(r % kSlice);
    const int n = UNIFORM ? k : len[r];
    const int w = UNIFORM ? k : (int)((off[q + 1] - off[q]) / kSlice);
    const int64_t sb = UNIFORM ? q * kSlice * (int64_t)k : off[q];
    const int c0 = n > 0 ? col[sell_at(sb, w, lane, 0)] : 0;
    base[r] = c0;
    for (int j = 0; j < n; ++j) {
      const int64_t i = sell_at(sb, w, lane, j);
      col16[i] = (int16_t)(col[i] - c0);
    }
  }
}

static size_t lowp_smem_for(int ts, int A) { return (size_t)ts * A * kLowpSmemPerRow + 16; }
static size_t lowp_smem(const mdp_s* h) { return lowp_smem_for(h->lp_ts, h->A); }

static int vec_grid(const mdp_s* h, int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)h->sm_count * 8));
}

// Whether the handle's probabilities are exact in 16 bits (the sweep's precondition).
bool lowp_available(const mdp_s* h) { return h->pstore == kStoreF16 || h->pstore == kStoreBF16; }

// The 16-bit values, binary32 costs and V, the counter, and the launch shape for the
// current tile size (set up on first use, reshaped when mdp_tune changes a tile).
static mdp_status ensure_lowp(mdp_s* h, cudaStream_t st) {
  if (!lowp_available(h))
    return fail(MDP_ERR_INVALID_ARG,
                "the low-precision sweep needs probabilities exact in binary16 or bfloat16 (multiples of 2^-11 or "
                "2^-8 per row, summing to 1)");
  if (!h->P16) {
    auto alloc = [&](void** p, size_t bytes, const char* what) -> mdp_status {
      cudaError_t e = cudaMallocAsync(p, bytes, st);
      if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(MDP_ERR_OOM, std::string("device allocation failed: ") + what);
      }
      return MDP_OK;
    };
    MDP_TRY(alloc((void**)&h->g32, (size_t)h->R * sizeof(float), "binary32 costs"));
    MDP_TRY(alloc((void**)&h->vf32, (size_t)h->S * sizeof(float), "binary32 V"));
    MDP_TRY(alloc((void**)&h->lp_rows, sizeof(unsigned long long), "sweep counter"));
    MDP_TRY(alloc((void**)&h->P16, (size_t)std::max<int64_t>(1, h->P.nstored) * sizeof(uint16_t), "16-bit values"));
    const int grid = vec_grid(h, std::max(h->P.nstored, h->R));
    if (h->pstore == kStoreBF16)
      lowp_pack_kernel<true><<<grid, 256, 0, st>>>(h->P.val, h->P.nstored, h->P16, h->g, h->R, h->g32);
    else
      lowp_pack_kernel<false><<<grid, 256, 0, st>>>(h->P.val, h->P.nstored, h->P16, h->g, h->R, h->g32);
    h->launches++;
    MDP_CUDA(cudaGetLastError());
    MDP_CUDA(cudaMemsetAsync(h->lp_rows, 0, sizeof(unsigned long long), st));
    if (h->col16) {
      MDP_TRY(alloc((void**)&h->P16col, (size_t)std::max<int64_t>(1, h->P.nstored) * sizeof(int16_t),
                    "16-bit column offsets"));
      MDP_TRY(alloc((void**)&h->P16base, (size_t)h->R * sizeof(int32_t), "row base columns"));
      const int rg = vec_grid(h, h->R);
      if (h->P.uniform)
        lowp_col16_kernel<true><<<rg, 256, 0, st>>>(h->P.col, h->P.off, h->P.len, h->P.kmax, h->R, h->P16col,
                                                    h->P16base);
      else
        lowp_col16_kernel<false><<<rg, 256, 0, st>>>(h->P.col, h->P.off, h->P.len, 0, h->R, h->P16col, h->P16base);
      h->launches++;
      MDP_CUDA(cudaGetLastError());
    }
  }
  // the tile mdp_tune chose for this sweep, else the binary64 sweep's, halved until
  // its 10 B per row fit in shared memory
  int ts = h->lp_ts_tuned > 0 ? h->lp_ts_tuned : h->bell_tile_states;
  while (ts > 1 && lowp_smem_for(ts, h->A) > 227 * 1024) ts /= 2;
  if (h->lp_ts != ts) {
    h->lp_ts = ts;
    const size_t smem = lowp_smem(h);
    if (smem > 227 * 1024) return fail(MDP_ERR_INVALID_ARG, "low-precision sweep tile does not fit on an SM");
    const void* kern[8] = {(const void*)bellman_lowp_kernel<true, __half, int32_t>,
                           (const void*)bellman_lowp_kernel<false, __half, int32_t>,
                           (const void*)bellman_lowp_kernel<true, __nv_bfloat16, int32_t>,
                           (const void*)bellman_lowp_kernel<false, __nv_bfloat16, int32_t>,
                           (const void*)bellman_lowp_kernel<true, __half, int16_t>,
                           (const void*)bellman_lowp_kernel<false, __half, int16_t>,
                           (const void*)bellman_lowp_kernel<true, __nv_bfloat16, int16_t>,
                           (const void*)bellman_lowp_kernel<false, __nv_bfloat16, int16_t>};
    for (const void* f : kern) MDP_TRY(raise_dyn_smem(f, smem));
    const int which = (h->P16col ? 4 : 0) + (h->pstore == kStoreBF16 ? 2 : 0) + (h->P.uniform ? 0 : 1);
    int per_sm = 0;
    MDP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[which], kBellThreads, smem));
    if (per_sm < 1) return fail(MDP_ERR_INVALID_ARG, "low-precision sweep tile does not fit on an SM");
    const int64_t ntiles = (h->S + ts - 1) / ts;
    h->lp_blocks = (int)std::min<int64_t>(ntiles, (int64_t)h->sm_count * per_sm);
  }
  return MDP_OK;
}

mdp_status prepare_lowp(mdp_s* h, cudaStream_t st) { return ensure_lowp(h, st); }

mdp_status launch_bellman_lowp(mdp_s* h, double gamma, const double* V, double* TV, int32_t* pi, cudaStream_t st) {
  MDP_TRY(ensure_lowp(h, st));
  MDP_CUDA(cudaMemsetAsync(h->resmax, 0, sizeof(unsigned long long), st));
  lowp_v32_kernel<<<vec_grid(h, h->S), 256, 0, st>>>(V, h->vf32, h->S);
  h->launches++;
  MDP_CUDA(cudaGetLastError());
  const size_t smem = lowp_smem(h);
  const Sell& P = h->P;
  const float gf = static_cast<float>(gamma);  // round to nearest, as on the device
  const int k = P.uniform ? P.kmax : 0;
#define MDP_LOWP_LAUNCH(U, TP, TC, COL, BASE)                                                               \
  bellman_lowp_kernel<U, TP, TC><<<h->lp_blocks, kBellThreads, smem, st>>>(                                  \
      reinterpret_cast<const TP*>(h->P16), COL, BASE, P.off, P.len, k, h->g32, h->g, h->vf32, V, h->S, h->A, \
      h->lp_ts, gamma, gf, TV, pi, h->resmax, h->lp_rows)
#define MDP_LOWP_COLS(U, TP)                                                                                \
  do {                                                                                                      \
    if (h->P16col)                                                                                          \
      MDP_LOWP_LAUNCH(U, TP, int16_t, (const int16_t*)h->P16col, (const int32_t*)h->P16base);               \
    else                                                                                                    \
      MDP_LOWP_LAUNCH(U, TP, int32_t, (const int32_t*)P.col, (const int32_t*)nullptr);                      \
  } while (0)
  if (h->pstore == kStoreBF16) {
    if (P.uniform) MDP_LOWP_COLS(true, __nv_bfloat16); else MDP_LOWP_COLS(false, __nv_bfloat16);
  } else {
    if (P.uniform) MDP_LOWP_COLS(true, __half); else MDP_LOWP_COLS(false, __half);
  }
#undef MDP_LOWP_COLS
#undef MDP_LOWP_LAUNCH
  h->launches++;
  MDP_CUDA(cudaGetLastError());
  return MDP_OK;
}

mdp_status launch_sweep(mdp_s* h, bool lowp, double gamma, const double* V, double* TV, int32_t* pi,
                        cudaStream_t st) {
  if (lowp && lowp_available(h)) return launch_bellman_lowp(h, gamma, V, TV, pi, st);
  return launch_bellman(h, gamma, V, TV, pi, st);
}

}  // namespace mdp

using namespace mdp;

extern "C" mdp_status mdp_bellman_lowp(mdp_handle h, double gamma, const double* V, double* TV, int32_t* pi,
                                       double* residual_inf, void* stream) {
  NvtxRange range("mdp_bellman_lowp");
  if (!h) return fail(MDP_ERR_INVALID_ARG, "null handle");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
  if (!V || !TV || !pi) return fail(MDP_ERR_INVALID_ARG, "null vector");
  if ((const void*)V == (const void*)TV) return fail(MDP_ERR_INVALID_ARG, "V and TV may not alias");
  cudaStream_t st = (cudaStream_t)stream;
  MDP_TRY(bind_stream(h, st));
  MDP_TRY(launch_bellman_lowp(h, gamma, V, TV, pi, st));
  if (residual_inf)
    MDP_CUDA(cudaMemcpyAsync(residual_inf, h->resmax, sizeof(double), cudaMemcpyDeviceToDevice, st));
  MDP_CUDA(cudaEventRecord(h->done, st));
  return MDP_OK;
}
