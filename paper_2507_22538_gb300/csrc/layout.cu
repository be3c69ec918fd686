// Handle lifetime: validation of the row-stacked CSR input (Eq. 5), conversion
// to the device layout, policy-row extraction (Algorithm 1 step 4) and errors.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "layout_dev.cuh"

namespace mdp {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

mdp_status fail(mdp_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

mdp_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  // a non-sticky error (a refused launch or argument) is reported here once; clear
  // the thread's error state so the next launch check does not report it again
  cudaGetLastError();
  return (e == cudaErrorMemoryAllocation) ? MDP_ERR_OOM : MDP_ERR_CUDA;
}

enum : int {
  kBadPtr = 1,
  kEmptyRow = 2,
  kBadCol = 4,
  kBadVal = 8,
  kRowSum = 16,
  kBadCost = 32,
  kLongRow = 64,
};

// Whether a finite double v >= 0 is exactly a binary16 / bfloat16 value, read off its
// IEEE-754 fields: with unbiased exponent e, a normal target (e >= emin) keeps `p`
// fraction bits, a subnormal one (emin - p <= e < emin) keeps e - (emin - p) of them,
// and every dropped fraction bit must be zero.  (binary16: p = 10, emin = -14;
// bfloat16: p = 7, emin = -126.)
__device__ __forceinline__ bool exact_in(uint64_t bits, int p, int emin, int emax) {
  if ((bits << 1) == 0) return true;  // +-0
  const int ebits = (int)((bits >> 52) & 0x7ff);
  if (ebits == 0) return false;  // a double subnormal is below both formats' range
  const int e = ebits - 1023;
  if (e > emax || e < emin - p) return false;
  const int kept = e >= emin ? p : e - (emin - p);
  const uint64_t dropped = (1ull << (52 - kept)) - 1;
  return (bits & dropped) == 0;
}

// Exact widening of the caller's value type to binary64.
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return (double)v; }
__device__ __forceinline__ double widen(__half v) { return (double)__half2float(v); }
__device__ __forceinline__ double widen(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// One thread per row of Eq. 5: check the row pointers and the stage cost, record
// the row length and the shortest and longest row.  Entries are read only after
// these checks have passed on every row (sell_rows_kernel).
__global__ void row_struct_kernel(const int64_t* __restrict__ rp, const double* __restrict__ g, int64_t R,
                                  int64_t nnz, int32_t* __restrict__ len, int* __restrict__ flags,
                                  int* __restrict__ kmin, int* __restrict__ kmax) {
  int bad = 0;
  int lmin = 0x7fffffff, lmax = 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = rp[r], hi = rp[r + 1];
    int l = 0;
    if (lo < 0 || hi < lo || hi > nnz || (r == 0 && lo != 0))
      bad |= kBadPtr;
    else if (hi == lo)
      bad |= kEmptyRow;
    else if (hi - lo > (1 << 30))
      bad |= kLongRow;
    else
      l = (int)(hi - lo);
    if (!isfinite(g[r])) bad |= kBadCost;
    len[r] = l;
    lmin = min(lmin, l);
    lmax = max(lmax, l);
  }
  if (bad) atomicOr(flags, bad);
  atomicMin(kmin, lmin);
  atomicMax(kmax, lmax);
}

// Width of each slice of `rows` rows: the longest row among its 32.
__global__ void slice_width_kernel(const int32_t* __restrict__ len, int64_t rows, int64_t nslices,
                                   int32_t* __restrict__ width) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nslices; q += (int64_t)gridDim.x * blockDim.x) {
    int w = 0;
    for (int l = 0; l < kSlice; ++l) {
      int64_t r = q * kSlice + l;
      if (r < rows) w = max(w, len[r]);
    }
    width[q] = w;
  }
}

// Per state: the longest of its A rows (sizes the policy-row slices).
__global__ void state_maxlen_kernel(const int32_t* __restrict__ len, int64_t S, int A, int32_t* __restrict__ out) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    int w = 0;
    for (int a = 0; a < A; ++a) w = max(w, len[s * A + a]);
    out[s] = w;
  }
}

// CSR -> sliced ELL for rows [r0, r1) of Eq. 5, one thread per row: copy the row's
// entries (values of type TV widened exactly to binary64) into their chunked slice
// positions and zero-fill the slice width beyond the row, and check the entries on
// the way: columns in [0, S), probabilities finite and >= 0 summing to 1 within
// 1e-12, whether every probability is exact in binary16 / bfloat16 (the narrowest
// exact storage for the mixed solver's copies of the policy rows) and whether every
// column lies within 32767 of its row's first one (16-bit column offsets).
// col and val hold the entries from index ebase on: the whole arrays (ebase 0) or
// one uploaded chunk that covers the rows' entries.  Row pointers were checked by
// row_struct_kernel.
template <typename TV>
__global__ void sell_rows_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const TV* __restrict__ val, int64_t r0, int64_t r1, int64_t ebase, int64_t S,
                                 const int64_t* __restrict__ off, int uniform_k, double* __restrict__ sval,
                                 int32_t* __restrict__ scol, int* __restrict__ flags, int* __restrict__ f16_ok,
                                 int* __restrict__ bf16_ok, int* __restrict__ near_ok) {
  int bad = 0;
  bool a16 = true, b16 = true, near = true;
  for (int64_t r = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < r1; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = r / kSlice;
    const int lane = (int)(r % kSlice);
    const int64_t base = uniform_k ? q * kSlice * (int64_t)uniform_k : off[q];
    const int width = uniform_k ? uniform_k : (int)((off[q + 1] - off[q]) / kSlice);
    const int64_t lo = rp[r] - ebase;
    const int n = (int)(rp[r + 1] - rp[r]);
    const int c0 = col[lo];  // the row's first column: the base of its 16-bit offsets
    double sum = 0.0;
    for (int j = 0; j < width; ++j) {
      const int64_t d = sell_at(base, width, lane, j);
      if (j < n) {
        const int c = col[lo + j];
        const double v = widen(val[lo + j]);
        if (c < 0 || (int64_t)c >= S) bad |= kBadCol;
        near &= ((int64_t)c - c0 >= -32768 && (int64_t)c - c0 <= 32767);
        if (!(v >= 0.0) || isinf(v)) bad |= kBadVal;
        const uint64_t bits = (uint64_t)__double_as_longlong(v);
        a16 &= exact_in(bits, 10, -14, 15);
        b16 &= exact_in(bits, 7, -126, 127);
        sum += v;
        sval[d] = v;
        scol[d] = c;
      } else {
        sval[d] = 0.0;
        scol[d] = 0;
      }
    }
    if (!(fabs(sum - 1.0) <= 1e-12)) bad |= kRowSum;
  }
  if (bad) atomicOr(flags, bad);
  if (!__all_sync(0xffffffffu, a16) && (threadIdx.x & 31) == 0) atomicAnd(f16_ok, 0);
  if (!__all_sync(0xffffffffu, b16) && (threadIdx.x & 31) == 0) atomicAnd(bf16_ok, 0);
  if (!__all_sync(0xffffffffu, near) && (threadIdx.x & 31) == 0) atomicAnd(near_ok, 0);
}

// Algorithm 1 step 4 on one problem (body in layout_dev.cuh).
template <bool UNIFORM>
__global__ void extract_policy_kernel(const double* __restrict__ sval, const int32_t* __restrict__ scol,
                                      const int64_t* __restrict__ off, const int32_t* __restrict__ len, int kmax,
                                      const double* __restrict__ g, const int32_t* __restrict__ pi, int64_t S, int A,
                                      double* __restrict__ pval, int32_t* __restrict__ pcol,
                                      const int64_t* __restrict__ poff, int32_t* __restrict__ plen,
                                      double* __restrict__ gpi, float* __restrict__ pval32,
                                      uint16_t* __restrict__ pval16, int store16, int16_t* __restrict__ pcol16,
                                      const int32_t* __restrict__ pcolbase) {
  extract_policy_body<UNIFORM>((int)blockIdx.x, (int)gridDim.x, sval, scol, off, len, kmax, g, pi, S, A, pval, pcol, poff, plen, gpi, pval32, pval16, store16, pcol16, pcolbase);
}

template <bool UNIFORM>
__global__ void policy_base_kernel(const int32_t* __restrict__ scol, const int64_t* __restrict__ off,
                                   const int32_t* __restrict__ len, int kmax, const int32_t* __restrict__ pi, int64_t S,
                                   int A, int32_t* __restrict__ pcolbase) {
  policy_base_body<UNIFORM>((int)blockIdx.x, (int)gridDim.x, scol, off, len, kmax, pi, S, A, pcolbase);
}

static int grid_for(int64_t n, int threads, int sm_count) {
  int64_t b = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sm_count * 8;
  return (int)std::max<int64_t>(1, std::min(b, cap));
}

double* tls_pinned() {
  static thread_local double* buf = nullptr;
  if (!buf && cudaMallocHost((void**)&buf, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    buf = nullptr;
  }
  return buf;
}

// Device memory comes from the stream-ordered pool on the handle's creation
// stream (no device-wide synchronisation, so handles of concurrent solves can be
// created and destroyed while others run).
template <typename T>
static mdp_status dalloc(mdp_s* h, T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), h->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(MDP_ERR_OOM, std::string("device allocation failed: ") + what);
  }
  return MDP_OK;
}

template <typename T>
static void dfree(cudaStream_t st, T*& p) {
  if (p) cudaFreeAsync((void*)p, st);
  p = nullptr;
}

mdp_status bind_stream(mdp_s* h, cudaStream_t st) {
  MDP_CUDA(cudaStreamWaitEvent(st, h->done, 0));
  h->stream = st;
  return MDP_OK;
}

// Build a sliced layout from per-row lengths (device) for `rows` rows.
static mdp_status build_sell(mdp_s* h, Sell* m, const int32_t* dlen, int64_t rows, int kmin, int kmax,
                             cudaStream_t st) {
  m->rows = rows;
  m->nslices = (rows + kSlice - 1) / kSlice;
  m->kmax = kmax;
  m->uniform = (kmin == kmax);
  if (m->uniform) {
    m->nstored = m->nslices * kSlice * (int64_t)kmax;
  } else {
    int32_t* dwidth = nullptr;
    MDP_TRY(dalloc(h, &dwidth, m->nslices, "slice widths"));
    slice_width_kernel<<<grid_for(m->nslices, 256, h->sm_count), 256, 0, st>>>(dlen, rows, m->nslices, dwidth);
    h->launches++;
    std::vector<int32_t> width(m->nslices);
    cudaError_t e = cudaMemcpyAsync(width.data(), dwidth, m->nslices * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(st, dwidth);
    if (e != cudaSuccess) return cuda_fail(e, "slice widths");
    std::vector<int64_t> off(m->nslices + 1);
    off[0] = 0;
    for (int64_t q = 0; q < m->nslices; ++q) off[q + 1] = off[q] + (int64_t)width[q] * kSlice;
    m->nstored = off[m->nslices];
    MDP_TRY(dalloc(h, &m->off, m->nslices + 1, "slice offsets"));
    MDP_CUDA(cudaMemcpyAsync(m->off, off.data(), (m->nslices + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    MDP_TRY(dalloc(h, &m->len, rows, "row lengths"));
  }
  MDP_TRY(dalloc(h, &m->val, m->nstored, "sliced values"));
  MDP_TRY(dalloc(h, &m->col, m->nstored, "sliced columns"));
  return MDP_OK;
}

static void free_sell(cudaStream_t st, Sell* m) {
  dfree(st, m->off);
  dfree(st, m->len);
  dfree(st, m->val);
  dfree(st, m->col);
  *m = Sell();
}

int extract_blocks(const mdp_s* h) {
  const int64_t work = h->S * (int64_t)((h->P.kmax + kChunk - 1) / kChunk);
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)h->sm_count * 16));
}

mdp_status extract_policy(mdp_s* h, const int32_t* pi, bool want32, cudaStream_t st) {
  const Sell& P = h->P;
  Sell& Q = h->Ppi;
  const int blocks = extract_blocks(h);
  if (want32 && h->pcol16) {  // the base columns of the 16-bit offsets first
    const int bb = grid_for(h->S, 256, h->sm_count);
    if (P.uniform)
      policy_base_kernel<true><<<bb, 256, 0, st>>>(P.col, P.off, P.len, P.kmax, pi, h->S, h->A, h->pcolbase);
    else
      policy_base_kernel<false><<<bb, 256, 0, st>>>(P.col, P.off, P.len, P.kmax, pi, h->S, h->A, h->pcolbase);
    h->launches++;
    MDP_CUDA(cudaGetLastError());
  }
  if (P.uniform)
    extract_policy_kernel<true><<<blocks, 256, 0, st>>>(
        P.val, P.col, P.off, P.len, P.kmax, h->g, pi, h->S, h->A, Q.val, Q.col, Q.off, Q.len, h->gpi,
        want32 && h->pstore == kStoreF32 ? h->pval32 : nullptr, want32 && h->pstore != kStoreF32 ? h->pval16 : nullptr,
        h->pstore, want32 ? h->pcol16 : nullptr, want32 ? h->pcolbase : nullptr);
  else
    extract_policy_kernel<false><<<blocks, 256, 0, st>>>(
        P.val, P.col, P.off, P.len, P.kmax, h->g, pi, h->S, h->A, Q.val, Q.col, Q.off, Q.len, h->gpi,
        want32 && h->pstore == kStoreF32 ? h->pval32 : nullptr, want32 && h->pstore != kStoreF32 ? h->pval16 : nullptr,
        h->pstore, want32 ? h->pcol16 : nullptr, want32 ? h->pcolbase : nullptr);
  h->launches++;
  MDP_CUDA(cudaGetLastError());
  return MDP_OK;
}

// Frees go to the legacy stream, ordered after everything the caller already
// completed; the caller makes sure no work on the handle is still in flight.
static void destroy_handle(mdp_s* h) {
  if (!h) return;
  if (h->done) cudaEventSynchronize(h->done);  // the last call's work has finished
  graph_cache_free(h);
  const cudaStream_t st = 0;
  free_sell(st, &h->P);
  free_sell(st, &h->Ppi);
  dfree(st, h->g);
  dfree(st, h->gpi);
  dfree(st, h->TV);
  dfree(st, h->piw);
  dfree(st, h->w);
  dfree(st, h->tmp);
  dfree(st, h->basis);
  dfree(st, h->pval32);
  dfree(st, h->pval16);
  dfree(st, h->pcol16);
  dfree(st, h->pcolbase);
  dfree(st, h->basis32);
  dfree(st, h->w32);
  dfree(st, h->tfq);
  dfree(st, h->partials);
  dfree(st, h->sc);
  dfree(st, h->resmax);
  dfree(st, h->P16);
  dfree(st, h->P16col);
  dfree(st, h->P16base);
  dfree(st, h->g32);
  dfree(st, h->vf32);
  dfree(st, h->lp_rows);
  char* ks = (char*)h->kstate;
  dfree(st, ks);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev2) cudaEventDestroy(h->ev2);
  if (h->ev3) cudaEventDestroy(h->ev3);
  if (h->done) cudaEventDestroy(h->done);
  for (cudaEvent_t e : h->mv_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->gs_ev)
    if (e) cudaEventDestroy(e);
  delete h;
}

mdp_status ensure_mixed(mdp_s* h, int nvec) {
  if (h->pstore == kStoreF32 && !h->pval32) MDP_TRY(dalloc(h, &h->pval32, h->Ppi.nstored, "FP32 policy values"));
  if (h->pstore != kStoreF32 && !h->pval16) MDP_TRY(dalloc(h, &h->pval16, h->Ppi.nstored, "16-bit policy values"));
  // 16-bit column offsets go with 16-bit values (4 instead of 6 bytes per entry); beside
  // binary32 values they measured 1% slower on the whole mixed solve than 32-bit columns
  if (h->col16 && h->pstore != kStoreF32) {
    if (!h->pcol16) MDP_TRY(dalloc(h, &h->pcol16, h->Ppi.nstored, "16-bit policy column offsets"));
    if (!h->pcolbase) MDP_TRY(dalloc(h, &h->pcolbase, h->S, "policy row base columns"));
  }
  if (!h->w32) MDP_TRY(dalloc(h, &h->w32, h->S, "FP32 w"));
  if (nvec > h->basis32_cap) {
    dfree(h->stream, h->basis32);
    h->basis32_cap = 0;
    MDP_TRY(dalloc(h, &h->basis32, (size_t)nvec * (size_t)h->S, "FP32 GMRES basis"));
    h->basis32_cap = nvec;
  }
  return MDP_OK;
}

mdp_status ensure_tfqmr(mdp_s* h) {
  if (!h->tfq) MDP_TRY(dalloc(h, &h->tfq, (size_t)8 * (size_t)h->S, "TFQMR vectors"));
  return MDP_OK;
}

mdp_status ensure_basis(mdp_s* h, int nvec) {
  if (nvec <= h->basis_cap) return MDP_OK;
  dfree(h->stream, h->basis);
  h->basis_cap = 0;
  MDP_TRY(dalloc(h, &h->basis, (size_t)nvec * (size_t)h->S, "GMRES basis"));
  h->basis_cap = nvec;
  return MDP_OK;
}

// The dynamic shared memory cap of a kernel is one attribute per kernel and
// device, shared by every handle and host thread of the process.  It is only ever
// raised (under a lock): a handle whose tile needs less must not lower the cap
// under a concurrent handle that needs more, whose next launch would then fail.
mdp_status raise_dyn_smem(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return MDP_OK;
  int dev = 0;
  MDP_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> caps;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cap = caps[{dev, func}];
  if (bytes <= cap) return MDP_OK;
  MDP_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cap = bytes;
  return MDP_OK;
}

// The stream-ordered pool that every device buffer of the library comes from
// keeps up to a sixteenth of the device's memory across synchronisations (the
// default returns all of it to the CUDA driver at each one), so handles created and
// destroyed in turn reuse their buffers instead of mapping memory again.  This is
// the process's default pool of the device: the setting ends with the process.
static mdp_status retain_pool(int device) {
  static std::mutex mu;
  static bool done[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (device < 0 || device >= 64 || done[device]) return MDP_OK;
  size_t free_b = 0, total_b = 0;
  MDP_CUDA(cudaMemGetInfo(&free_b, &total_b));
  cudaMemPool_t pool;
  MDP_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
  uint64_t keep = (uint64_t)(total_b / 16);
  MDP_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  done[device] = true;
  return MDP_OK;
}

// Entries of a host CSR: uploaded in row-aligned chunks of at most 2^25 entries (or
// one longest row) through a ring of four device buffers on a copy stream; each chunk
// is converted and checked on the creation stream as soon as it has arrived, so the
// copies of later chunks overlap the conversion of earlier ones, and device memory
// holds a few chunks instead of the whole CSR.  (Host-to-device copies from pinned
// memory run at the same rate from one stream as from two or four.)  The row pointers have been checked
// on the device beforehand, so the chunk boundaries found here by binary search on
// the host's row pointers are valid.
template <typename Convert>
static mdp_status upload_rows(mdp_s* h, const int64_t* row_ptr, const int32_t* col, const void* val, size_t vbytes,
                              int64_t R, int kmax, cudaStream_t st, Convert& convert) {
  constexpr int kRing = 4;
  const int64_t cap = std::min<int64_t>(row_ptr[R] - row_ptr[0], std::max<int64_t>(int64_t(1) << 25, kmax));
  std::vector<int64_t> cut{0};
  for (int64_t r0 = 0; r0 < R;) {
    int64_t r1 = std::upper_bound(row_ptr + r0 + 1, row_ptr + R + 1, row_ptr[r0] + cap) - row_ptr - 1;
    if (r1 <= r0 || row_ptr[r1] - row_ptr[r0] > cap)
      return fail(MDP_ERR_INVALID_ARG, "row_ptr changed during mdp_create");
    cut.push_back(r1);
    r0 = r1;
  }
  const int chunks = (int)cut.size() - 1;
  const int nb = std::min(kRing, chunks);
  struct Ring {
    cudaStream_t st;
    cudaStream_t cs = nullptr;
    cudaEvent_t ready = nullptr, copied[kRing] = {}, used[kRing] = {};
    int32_t* c[kRing] = {};
    uint16_t* v[kRing] = {};
    ~Ring() {  // copies still in flight (an error part-way) end before their buffers are freed
      if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
      }
      for (cudaEvent_t e : copied)
        if (e) cudaEventDestroy(e);
      for (cudaEvent_t e : used)
        if (e) cudaEventDestroy(e);
      if (ready) cudaEventDestroy(ready);
      for (int b = 0; b < kRing; ++b) {
        dfree(st, c[b]);
        dfree(st, v[b]);
      }
    }
  } ring{st};
  for (int b = 0; b < nb; ++b) {
    MDP_TRY(dalloc(h, &ring.c[b], (size_t)cap, "column chunk"));
    MDP_TRY(dalloc(h, &ring.v[b], (size_t)cap * (vbytes / 2), "value chunk"));
    MDP_CUDA(cudaEventCreateWithFlags(&ring.copied[b], cudaEventDisableTiming));
    MDP_CUDA(cudaEventCreateWithFlags(&ring.used[b], cudaEventDisableTiming));
  }
  MDP_CUDA(cudaEventCreateWithFlags(&ring.ready, cudaEventDisableTiming));
  MDP_CUDA(cudaStreamCreateWithFlags(&ring.cs, cudaStreamNonBlocking));
  MDP_CUDA(cudaEventRecord(ring.ready, st));  // the ring buffers are allocated on st
  for (int i = 0; i < chunks; ++i) {
    const int b = i % nb;
    cudaStream_t cs = ring.cs;
    const int64_t r0 = cut[i], r1 = cut[i + 1], e0 = row_ptr[r0], n = row_ptr[r1] - e0;
    MDP_CUDA(cudaStreamWaitEvent(cs, i < nb ? ring.ready : ring.used[b], 0));
    MDP_CUDA(cudaMemcpyAsync(ring.c[b], col + e0, n * sizeof(int32_t), cudaMemcpyHostToDevice, cs));
    MDP_CUDA(cudaMemcpyAsync(ring.v[b], (const char*)val + e0 * vbytes, n * vbytes, cudaMemcpyHostToDevice, cs));
    MDP_CUDA(cudaEventRecord(ring.copied[b], cs));
    MDP_CUDA(cudaStreamWaitEvent(st, ring.copied[b], 0));
    MDP_TRY(convert(ring.c[b], ring.v[b], r0, r1, e0));
    MDP_CUDA(cudaEventRecord(ring.used[b], st));
  }
  return MDP_OK;
}

static mdp_status create_impl(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const void* val,
                              mdp_dtype val_type, const double* g, int32_t on_device, cudaStream_t st,
                              mdp_s* h) {
  h->stream = st;
  MDP_CUDA(cudaGetDevice(&h->device));
  MDP_CUDA(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
  MDP_TRY(retain_pool(h->device));
  h->S = S;
  h->A = A;
  h->R = S * (int64_t)A;
  const int64_t R = h->R;

  int64_t nnz = 0;
  if (on_device) {
    MDP_CUDA(cudaMemcpyAsync(&nnz, row_ptr + R, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MDP_CUDA(cudaStreamSynchronize(st));
  } else {
    nnz = row_ptr[R];
  }
  if (nnz < R || nnz > (int64_t(1) << 40))
    return fail(MDP_ERR_NOT_STOCHASTIC, "row_ptr[S*A] must be between S*A (no empty rows) and 2^40");
  h->nnz = nnz;

  // Row pointers and stage costs first: the row structure is checked on every row
  // before any entry is read, and it fixes the sliced layout.
  const size_t vbytes = val_type == MDP_F64 ? 8 : val_type == MDP_F32 ? 4 : 2;
  const int64_t* drp = row_ptr;
  int64_t* trp = nullptr;  // device copy of host row pointers
  struct FreeRp { cudaStream_t st; int64_t** p; ~FreeRp() { dfree(st, *p); } } free_rp{st, &trp};
  if (!on_device) {
    MDP_TRY(dalloc(h, &trp, R + 1, "row pointers"));
    MDP_CUDA(cudaMemcpyAsync(trp, row_ptr, (R + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    drp = trp;
  }
  MDP_TRY(dalloc(h, &h->g, R, "stage costs"));
  MDP_CUDA(cudaMemcpyAsync(h->g, g, R * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));

  // validation flags, kmin, kmax and the exactness / offset flags live in the scalar area
  MDP_TRY(dalloc(h, &h->sc, kScalarSlots, "scalars"));
  MDP_TRY(dalloc(h, &h->resmax, 1, "residual"));
  int32_t* dlen = nullptr;
  MDP_TRY(dalloc(h, &dlen, R, "row lengths"));
  struct FreeLen { cudaStream_t st; int32_t** p; ~FreeLen() { dfree(st, *p); } } free_len{st, &dlen};
  int* dflags = (int*)h->sc;
  int init[6] = {0, 0x7fffffff, 0, 1, 1, 1};
  MDP_CUDA(cudaMemcpyAsync(dflags, init, sizeof(init), cudaMemcpyHostToDevice, st));
  row_struct_kernel<<<grid_for(R, 256, h->sm_count), 256, 0, st>>>(drp, h->g, R, nnz, dlen, dflags, dflags + 1,
                                                                     dflags + 2);
  h->launches++;
  MDP_CUDA(cudaGetLastError());
  int res[6];
  MDP_CUDA(cudaMemcpyAsync(res, dflags, sizeof(res), cudaMemcpyDeviceToHost, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  auto invalid = [](int f) {
    std::string m = "invalid MDP:";
    if (f & kBadPtr) m += " row_ptr[0] not 0, or row_ptr not monotone or out of [0, nnz];";
    if (f & kEmptyRow) m += " empty row;";
    if (f & kLongRow) m += " row longer than 2^30;";
    if (f & kBadCol) m += " column outside [0, S);";
    if (f & kBadVal) m += " negative or non-finite probability;";
    if (f & kRowSum) m += " row does not sum to 1 within 1e-12;";
    if (f & kBadCost) m += " non-finite stage cost;";
    return fail((f & (kBadCost | kBadPtr)) && !(f & (kEmptyRow | kBadCol | kBadVal | kRowSum))
                    ? MDP_ERR_INVALID_ARG : MDP_ERR_NOT_STOCHASTIC, m);
  };
  if (res[0] & (kBadPtr | kEmptyRow | kLongRow)) return invalid(res[0]);
  const int kmin = res[1], kmax = res[2];

  // stacked matrix in sliced layout: entries converted and checked row by row
  MDP_TRY(build_sell(h, &h->P, dlen, R, kmin, kmax, st));
  const int uk = h->P.uniform ? kmax : 0;
  auto convert_rows = [&](const int32_t* c, const void* v, int64_t r0, int64_t r1, int64_t ebase) -> mdp_status {
    const int cb = grid_for(r1 - r0, 256, h->sm_count);
    Sell& P = h->P;
    switch (val_type) {
      case MDP_F32:
        sell_rows_kernel<<<cb, 256, 0, st>>>(drp, c, (const float*)v, r0, r1, ebase, S, P.off, uk, P.val, P.col,
                                             dflags, dflags + 3, dflags + 4, dflags + 5);
        break;
      case MDP_F16:
        sell_rows_kernel<<<cb, 256, 0, st>>>(drp, c, (const __half*)v, r0, r1, ebase, S, P.off, uk, P.val, P.col,
                                             dflags, dflags + 3, dflags + 4, dflags + 5);
        break;
      case MDP_BF16:
        sell_rows_kernel<<<cb, 256, 0, st>>>(drp, c, (const __nv_bfloat16*)v, r0, r1, ebase, S, P.off, uk, P.val,
                                             P.col, dflags, dflags + 3, dflags + 4, dflags + 5);
        break;
      default:
        sell_rows_kernel<<<cb, 256, 0, st>>>(drp, c, (const double*)v, r0, r1, ebase, S, P.off, uk, P.val, P.col,
                                             dflags, dflags + 3, dflags + 4, dflags + 5);
    }
    h->launches++;
    MDP_CUDA(cudaGetLastError());
    return MDP_OK;
  };
  if (on_device)
    MDP_TRY(convert_rows(col, val, 0, R, 0));
  else
    MDP_TRY(upload_rows(h, row_ptr, col, val, vbytes, R, kmax, st, convert_rows));
  MDP_CUDA(cudaMemcpyAsync(res, dflags, sizeof(res), cudaMemcpyDeviceToHost, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  if (res[0]) return invalid(res[0]);

  // narrowest exact storage for the mixed solver's copies of the policy rows
  h->pstore = res[3] ? kStoreF16 : (res[4] ? kStoreBF16 : kStoreF32);
  // every column within 32767 states of its row's first column (banded and grid MDPs,
  // and every MDP of at most 32,768 states): the mixed solver's copy of the policy
  // rows then stores 16-bit column offsets (2 B per entry instead of 4)
  h->col16 = res[5] != 0;
  if (!h->P.uniform)
    MDP_CUDA(cudaMemcpyAsync(h->P.len, dlen, R * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));

  // policy rows: one per state, slice width = longest row of the slice's states
  if (h->P.uniform) {
    MDP_TRY(build_sell(h, &h->Ppi, dlen, S, kmax, kmax, st));
  } else {
    int32_t* smax = nullptr;
    MDP_TRY(dalloc(h, &smax, S, "state max length"));
    state_maxlen_kernel<<<grid_for(S, 256, h->sm_count), 256, 0, st>>>(dlen, S, A, smax);
    h->launches++;
    mdp_status s2 = build_sell(h, &h->Ppi, smax, S, 0, kmax, st);
    dfree(st, smax);
    MDP_TRY(s2);
  }

  // launch shapes
  h->vec_threads = 256;
  // vector passes: up to 4 blocks per SM (whole grid resident even at 128 registers
  // per thread), few enough that the last block's reduction of the partials is short
  h->vec_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((S + 255) / 256, (int64_t)h->sm_count * 4));
  h->mv_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((S + 255) / 256, (int64_t)h->sm_count * 8));
  {
    // Bellman tile: a multiple of 32 states whose rows fill whole warps where possible
    int64_t ts = 32;
    if (A <= 256) {
      int g256 = 1;
      for (int d = 1; d <= 256; d <<= 1)
        if (A % d == 0) g256 = d;
      int64_t need = 256 / g256;  // states per tile so that ts*A is a multiple of 256 rows
      ts = std::max<int64_t>(32, need);
      while (ts * A > 8192 && ts > 32) ts /= 2;
    }
    while (ts * A > 8192 && ts > 1) ts /= 2;
    if (ts > S) ts = std::max<int64_t>(1, S);
    h->bell_tile_states = (int)ts;
    MDP_TRY(configure_bellman(h));
  }
  MDP_TRY(dalloc(h, &h->gpi, S, "g_pi"));
  MDP_TRY(dalloc(h, &h->TV, S, "TV"));
  MDP_TRY(dalloc(h, &h->piw, S, "policy"));
  MDP_TRY(dalloc(h, &h->w, S, "w"));
  MDP_TRY(dalloc(h, &h->tmp, S, "tmp"));
  h->partial_stride = std::min(h->sm_count * kMaxBlocksPerSm, kMaxReduceBlocks);
  // block partials, then the second-level group sums of the grid reductions
  MDP_TRY(dalloc(h, &h->partials, (size_t)kPartialRows * (h->partial_stride + kMaxGroups), "partials"));
  {
    char* ks = nullptr;
    MDP_TRY(dalloc(h, &ks, krylov_state_bytes(), "solver state"));
    h->kstate = ks;
  }
  if (!tls_pinned()) return fail(MDP_ERR_OOM, "pinned host allocation failed");
  MDP_CUDA(cudaEventCreate(&h->ev0));
  MDP_CUDA(cudaEventCreate(&h->ev1));
  MDP_CUDA(cudaEventCreate(&h->ev2));
  MDP_CUDA(cudaEventCreate(&h->ev3));
  MDP_CUDA(cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming));
  MDP_CUDA(cudaStreamSynchronize(st));
  return MDP_OK;
}

}  // namespace mdp

using namespace mdp;

extern "C" {

void mdp_default_opts(mdp_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->gamma = 0.0;
  o->atol_pi = 1e-8;
  o->alpha = 1e-4;
  o->richardson_scale = 1.0;
  o->max_iter_pi = 1000;
  o->max_iter_ksp = 1000;
  o->gmres_restart = 30;
  o->inner = MDP_GMRES;
  o->record_timing = 0;
  o->gmres_refine = MDP_REFINE_NEVER;
  o->precision = MDP_PREC_F64;
}

const char* mdp_last_error(void) { return g_last_error.c_str(); }

mdp_status mdp_create(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const void* val,
                      mdp_dtype val_type, const double* g, int32_t inputs_on_device, void* stream,
                      mdp_handle* out) {
  NvtxRange range("mdp_create");
  if (!out) return fail(MDP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (S < 1 || A < 1 || A > 8192) return fail(MDP_ERR_INVALID_ARG, "need S >= 1 and 1 <= A <= 8192");
  if (S > (int64_t(1) << 31) - 1 || S * (int64_t)A > (int64_t(1) << 36))
    return fail(MDP_ERR_INVALID_ARG, "S must fit int32 and S*A must be below 2^36");
  if (!row_ptr || !col || !val || !g) return fail(MDP_ERR_INVALID_ARG, "null input array");
  if (val_type != MDP_F64 && val_type != MDP_F32 && val_type != MDP_F16 && val_type != MDP_BF16)
    return fail(MDP_ERR_INVALID_ARG, "val_type must be MDP_F64, MDP_F32, MDP_F16 or MDP_BF16");
  mdp_s* h = new mdp_s();
  mdp_status st = create_impl(S, A, row_ptr, col, val, val_type, g, inputs_on_device, (cudaStream_t)stream, h);
  if (st != MDP_OK) {
    std::string msg = g_last_error;
    cudaStreamSynchronize((cudaStream_t)stream);
    destroy_handle(h);
    cudaGetLastError();
    g_last_error = msg;
    return st;
  }
  *out = h;
  g_last_error.clear();
  return MDP_OK;
}

mdp_status mdp_destroy(mdp_handle h) {
  if (!h) return MDP_OK;
  destroy_handle(h);
  return MDP_OK;
}

mdp_status mdp_get_info(mdp_handle h, int64_t* S, int32_t* A, int64_t* nnz) {
  if (!h) return fail(MDP_ERR_INVALID_ARG, "null handle");
  if (S) *S = h->S;
  if (A) *A = h->A;
  if (nnz) *nnz = h->nnz;
  return MDP_OK;
}

}  // extern "C"
