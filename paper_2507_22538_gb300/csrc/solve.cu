// Entry points: the Bellman application, policy evaluation and Algorithm 1 (inexact policy iteration).
#include <chrono>
#include <cmath>
#include <cstring>

#include "mdp_internal.cuh"

using namespace mdp;

extern "C" {
mdp_status mdp_bellman(mdp_handle h, double gamma, const double* V, double* TV, int32_t* pi,
                                  double* residual_inf, void* stream) {
  NvtxRange range("mdp_bellman");
  if (!h) return fail(MDP_ERR_INVALID_ARG, "null handle");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
  if (!V || !TV || !pi) return fail(MDP_ERR_INVALID_ARG, "null vector");
  if ((const void*)V == (const void*)TV) return fail(MDP_ERR_INVALID_ARG, "V and TV may not alias");
  cudaStream_t st = (cudaStream_t)stream;
  MDP_TRY(bind_stream(h, st));
  mdp_status s = launch_bellman(h, gamma, V, TV, pi, st);
  if (s != MDP_OK) return s;
  if (residual_inf)
    MDP_CUDA(cudaMemcpyAsync(residual_inf, h->resmax, sizeof(double), cudaMemcpyDeviceToDevice, st));
  MDP_CUDA(cudaEventRecord(h->done, st));
  return MDP_OK;
}

mdp_status mdp_policy_apply(mdp_handle h, double gamma, const int32_t* pi, const double* x, double* y, void* stream) {
  if (!h) return fail(MDP_ERR_INVALID_ARG, "null handle");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
  if (!pi || !x || !y) return fail(MDP_ERR_INVALID_ARG, "null vector");
  if ((const void*)x == (const void*)y) return fail(MDP_ERR_INVALID_ARG, "x and y may not alias");
  cudaStream_t st = (cudaStream_t)stream;
  MDP_TRY(bind_stream(h, st));
  mdp_status s = extract_policy(h, pi, false, st);
  if (s != MDP_OK) return s;
  s = launch_policy_apply(h, gamma, x, y, st);
  if (s != MDP_OK) return s;
  MDP_CUDA(cudaEventRecord(h->done, st));
  return MDP_OK;
}

mdp_status mdp_policy_eval(mdp_handle h, double gamma, const int32_t* pi, const double* v0, double* v,
                           mdp_inner inner, int32_t restart, double omega, double abs_tol_2norm, int32_t max_it,
                           int32_t* iters, double* res_2norm, void* stream) {
  NvtxRange range("mdp_policy_eval");
  if (!h) return fail(MDP_ERR_INVALID_ARG, "null handle");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
  if (!pi || !v0 || !v) return fail(MDP_ERR_INVALID_ARG, "null vector");
  if (inner < MDP_GMRES || inner > MDP_RICHARDSON_JACOBI) return fail(MDP_ERR_INVALID_ARG, "unknown inner solver");
  if (inner == MDP_GMRES && (restart < 1 || restart > kMaxBasis))
    return fail(MDP_ERR_INVALID_ARG, "GMRES restart must be in 1..32");
  if (max_it < 0 || !(abs_tol_2norm >= 0.0)) return fail(MDP_ERR_INVALID_ARG, "bad tolerance or iteration cap");
  cudaStream_t st = (cudaStream_t)stream;
  MDP_TRY(bind_stream(h, st));
  mdp_status s = extract_policy(h, pi, false, st);
  if (s != MDP_OK) return s;
  if (v != v0) MDP_CUDA(cudaMemcpyAsync(v, v0, h->S * sizeof(double), cudaMemcpyDeviceToDevice, st));
  int it = 0;
  double r2 = 0.0;
  s = inner_solve(h, gamma, v, inner, restart, MDP_REFINE_NEVER, MDP_PREC_F64, omega, abs_tol_2norm, max_it, &it,
                  &r2, st);
  MDP_CUDA(cudaEventRecord(h->done, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  if (iters) *iters = it;
  if (res_2norm) *res_2norm = r2;
  if (s != MDP_OK) return s;
  if (!(r2 < abs_tol_2norm)) return fail(MDP_NOT_CONVERGED, "policy evaluation hit max_it");
  return MDP_OK;
}

mdp_status mdp_tune(mdp_handle h, double gamma, int32_t* tile_states, float* ms_per_sweep, void* stream) {
  NvtxRange range("mdp_tune");
  if (!h) return fail(MDP_ERR_INVALID_ARG, "null handle");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
  cudaStream_t st = (cudaStream_t)stream;
  MDP_TRY(bind_stream(h, st));
  // the sweep at V = 0 into the handle's own vectors (w, TV, the policy scratch)
  MDP_CUDA(cudaMemsetAsync(h->w, 0, h->S * sizeof(double), st));
  auto time_one = [&](float* ms) -> mdp_status {
    MDP_TRY(launch_bellman(h, gamma, h->w, h->TV, h->piw, st));  // warm-up
    MDP_CUDA(cudaEventRecord(h->ev0, st));
    for (int r = 0; r < 3; ++r) MDP_TRY(launch_bellman(h, gamma, h->w, h->TV, h->piw, st));
    MDP_CUDA(cudaEventRecord(h->ev1, st));
    MDP_CUDA(cudaEventSynchronize(h->ev1));
    MDP_CUDA(cudaEventElapsedTime(ms, h->ev0, h->ev1));
    *ms /= 3.f;
    return MDP_OK;
  };
  const int start = h->bell_tile_states;
  int best = start;
  float best_ms = 0.f;
  h->bell_per_sm_cap = 0;  // tiles are compared at full occupancy, one row per lane, 16-byte loads
  h->bell_rpl = 1;
  h->bell_v256 = 0;
  MDP_TRY(configure_bellman(h));
  MDP_TRY(time_one(&best_ms));
  static const int kCandidates[] = {8, 16, 32, 64, 128, 256, 512};
  for (int ts : kCandidates) {
    if (ts == start || ts > h->S || (size_t)ts * h->A * sizeof(double) > 227 * 1024) continue;
    h->bell_tile_states = ts;
    h->bell_per_sm_cap = 0;
    if (configure_bellman(h) != MDP_OK) continue;  // the tile does not fit: skip it
    float ms = 0.f;
    mdp_status s = time_one(&ms);
    if (s != MDP_OK) {
      h->bell_tile_states = best;
      configure_bellman(h);
      return s;
    }
    if (ms < 0.98f * best_ms) {  // a clear gain only
      best = ts;
      best_ms = ms;
    }
  }
  h->bell_tile_states = best;
  MDP_TRY(configure_bellman(h));
  // then, for that tile, rows per lane (32 or 64 rows per warp step) and the width of
  // the value loads (16 or 32 bytes), each at full occupancy
  {
    int best_rpl = 1, best_v = 0;
    static const int kVariants[3][2] = {{1, 1}, {2, 0}, {2, 1}};
    for (const auto& var : kVariants) {
      h->bell_rpl = var[0];
      h->bell_v256 = var[1];
      MDP_TRY(configure_bellman(h));
      float ms = 0.f;
      MDP_TRY(time_one(&ms));
      if (ms < 0.98f * best_ms) {
        best_rpl = var[0];
        best_v = var[1];
        best_ms = ms;
      }
    }
    h->bell_rpl = best_rpl;
    h->bell_v256 = best_v;
    MDP_TRY(configure_bellman(h));
  }
  // then the grid: resident blocks per SM from the occupancy limit down (fewer blocks
  // leave each SM's L1 and request queues to fewer tiles at a time)
  {
    const int top = h->bell_max_per_sm;
    int best_cap = 0;
    for (int cap = top - 1; cap >= 1; --cap) {
      h->bell_per_sm_cap = cap;
      MDP_TRY(configure_bellman(h));
      float ms = 0.f;
      MDP_TRY(time_one(&ms));
      if (ms < 0.98f * best_ms) {
        best_cap = cap;
        best_ms = ms;
      }
    }
    h->bell_per_sm_cap = best_cap;
    MDP_TRY(configure_bellman(h));
  }
  // the low-precision sweep has its own tile (10 B of shared memory per row, and a
  // binary64 re-evaluation phase whose latency larger tiles amortise)
  if (lowp_available(h)) {
    auto time_lp = [&](float* ms) -> mdp_status {
      MDP_TRY(launch_bellman_lowp(h, gamma, h->w, h->TV, h->piw, st));  // warm-up (and set-up)
      MDP_CUDA(cudaEventRecord(h->ev0, st));
      for (int r = 0; r < 3; ++r) MDP_TRY(launch_bellman_lowp(h, gamma, h->w, h->TV, h->piw, st));
      MDP_CUDA(cudaEventRecord(h->ev1, st));
      MDP_CUDA(cudaEventSynchronize(h->ev1));
      MDP_CUDA(cudaEventElapsedTime(ms, h->ev0, h->ev1));
      *ms /= 3.f;
      return MDP_OK;
    };
    int best_lp = 0;
    float best_lp_ms = 0.f;
    for (int ts : kCandidates) {
      if (ts > h->S || (size_t)ts * h->A * 10 + 16 > 227 * 1024) continue;
      h->lp_ts_tuned = ts;
      float ms = 0.f;
      const mdp_status s = time_lp(&ms);
      if (s != MDP_OK) {
        if (s == MDP_ERR_INVALID_ARG) continue;  // the tile does not fit: skip it
        h->lp_ts_tuned = best_lp;
        return s;
      }
      if (best_lp == 0 || ms < 0.98f * best_lp_ms) {
        best_lp = ts;
        best_lp_ms = ms;
      }
    }
    h->lp_ts_tuned = best_lp;
    MDP_TRY(prepare_lowp(h, st));
  }
  MDP_CUDA(cudaEventRecord(h->done, st));
  if (tile_states) *tile_states = best;
  if (ms_per_sweep) *ms_per_sweep = best_ms;
  return MDP_OK;
}

mdp_status mdp_set_sweep_shape(mdp_handle h, int32_t tile_states, int32_t rows_per_warp, int32_t value_load_bytes,
                               int32_t blocks_per_sm) {
  if (!h) return fail(MDP_ERR_INVALID_ARG, "null handle");
  if (tile_states < 1 || tile_states > 4096 || (rows_per_warp != 32 && rows_per_warp != 64) ||
      (value_load_bytes != 16 && value_load_bytes != 32) || blocks_per_sm < 0)
    return fail(MDP_ERR_INVALID_ARG,
                "need 1 <= tile_states <= 4096, rows_per_warp 32 or 64, value_load_bytes 16 or 32, blocks_per_sm >= 0");
  if ((size_t)tile_states * h->A * sizeof(double) > 227 * 1024)
    return fail(MDP_ERR_INVALID_ARG, "the tile's Q values do not fit in shared memory");
  const int old_ts = h->bell_tile_states, old_rpl = h->bell_rpl, old_v = h->bell_v256, old_cap = h->bell_per_sm_cap;
  h->bell_tile_states = tile_states;
  h->bell_rpl = rows_per_warp / kSlice;
  h->bell_v256 = value_load_bytes == 32 ? 1 : 0;
  h->bell_per_sm_cap = blocks_per_sm;
  const mdp_status s = configure_bellman(h);
  if (s != MDP_OK) {  // keep the previous shape
    h->bell_tile_states = old_ts;
    h->bell_rpl = old_rpl;
    h->bell_v256 = old_v;
    h->bell_per_sm_cap = old_cap;
    configure_bellman(h);
  }
  return s;
}

mdp_status mdp_get_sweep_shape(mdp_handle h, int32_t* tile_states, int32_t* blocks, int32_t* blocks_per_sm,
                               int32_t* rows_per_warp, int32_t* value_load_bytes) {
  if (!h) return fail(MDP_ERR_INVALID_ARG, "null handle");
  if (tile_states) *tile_states = h->bell_tile_states;
  if (blocks) *blocks = h->bell_blocks;
  if (blocks_per_sm) *blocks_per_sm = h->bell_per_sm_cap;
  if (rows_per_warp) *rows_per_warp = kSlice * h->bell_rpl;
  if (value_load_bytes) *value_load_bytes = h->bell_v256 ? 32 : 16;
  return MDP_OK;
}

mdp_status mdp_solve(mdp_handle h, const mdp_solve_opts* o, double* V, int32_t* pi, mdp_solve_stats* stats,
                     void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  NvtxRange range("mdp_solve");
  if (!h || !o) return fail(MDP_ERR_INVALID_ARG, "null handle or options");
  if (!V || !pi) return fail(MDP_ERR_INVALID_ARG, "null vector");
  if (!(o->gamma > 0.0 && o->gamma < 1.0)) return fail(MDP_ERR_INVALID_ARG, "gamma must lie in (0, 1)");
  if (!(o->atol_pi > 0.0) || !(o->alpha > 0.0 && o->alpha < 1.0))
    return fail(MDP_ERR_INVALID_ARG, "need atol_pi > 0 and 0 < alpha < 1");
  if (o->max_iter_pi < 0 || o->max_iter_ksp < 0) return fail(MDP_ERR_INVALID_ARG, "negative iteration cap");
  if (o->inner < MDP_GMRES || o->inner > MDP_RICHARDSON_JACOBI)
    return fail(MDP_ERR_INVALID_ARG, "unknown inner solver");
  if (o->inner == MDP_GMRES && (o->gmres_restart < 1 || o->gmres_restart > kMaxBasis))
    return fail(MDP_ERR_INVALID_ARG, "GMRES restart must be in 1..32");
  if (o->gmres_refine < MDP_REFINE_NEVER || o->gmres_refine > MDP_REFINE_ALWAYS)
    return fail(MDP_ERR_INVALID_ARG, "unknown gmres_refine");
  if (o->precision != MDP_PREC_F64 && o->precision != MDP_PREC_MIXED)
    return fail(MDP_ERR_INVALID_ARG, "unknown precision");
  const bool mixed = (o->precision == MDP_PREC_MIXED && o->inner == MDP_GMRES);
  cudaStream_t st = (cudaStream_t)stream;
  MDP_TRY(bind_stream(h, st));
  if (mixed) {
    mdp_status s0 = ensure_mixed(h, o->gmres_restart + 1);
    if (s0 != MDP_OK) return s0;
  }
  const bool lowp = o->lowp_sweep && lowp_available(h);
  if (lowp) {
    MDP_TRY(prepare_lowp(h, st));
    MDP_CUDA(cudaMemsetAsync(h->lp_rows, 0, sizeof(unsigned long long), st));
  }
  const int64_t launches0 = h->launches;
  const int64_t matvecs0 = h->matvecs, vreads0 = h->vreads, vwrites0 = h->vwrites;
  const double ibytes0 = h->inner_bytes;
  const double mv_ms0 = h->mv_ms, mv_bytes0 = h->mv_bytes, mv_flops0 = h->mv_flops;
  const int64_t mv_timed0 = h->mv_timed;
  const double gs_ms0 = h->gs_ms, gs_flops0 = h->gs_flops;
  const int64_t gs_timed0 = h->gs_timed;
  mdp_solve_stats local;
  std::memset(&local, 0, sizeof(local));
  mdp_status status = MDP_OK;
  int k = 0;
  if (o->graph && o->inner == MDP_GMRES && !o->record_timing) {
    // the whole loop below as one CUDA graph launch (graph.cu)
    NvtxRange graph_range("graph launch (Algorithm 1)");
    status = graph_solve(h, o, V, pi, &local, st);
    if (status != MDP_OK && status != MDP_NOT_CONVERGED && status != MDP_ERR_NUMERIC) return status;
    k = local.outer_iters;
  } else {
  h->timing = o->record_timing ? 1 : 0;
  struct TimingOff { mdp_s* h; ~TimingOff() { h->timing = 0; } } timing_off{h};
  for (;;) {
    // Algorithm 1 steps 2-3: TV, pi_{k+1} and ||r(V_k)||_inf in one sweep
    nvtxRangePushA("Bellman sweep and stop test");
    struct PopSweep { bool on = true; void pop() { if (on) nvtxRangePop(); on = false; } ~PopSweep() { pop(); } } sweep_range;
    if (o->record_timing) MDP_CUDA(cudaEventRecord(h->ev0, st));
    mdp_status s = launch_sweep(h, lowp, o->gamma, V, h->TV, pi, st);
    if (s != MDP_OK) return s;
    if (o->record_timing) MDP_CUDA(cudaEventRecord(h->ev1, st));
    local.bellman_sweeps++;
    double* pin = tls_pinned();
    MDP_CUDA(cudaMemcpyAsync(pin, h->resmax, sizeof(double), cudaMemcpyDeviceToHost, st));
    MDP_CUDA(cudaStreamSynchronize(st));
    const double res = pin[0];
    if (o->record_timing) {
      float ms = 0.f;
      MDP_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
      local.bellman_ms += ms;
    }
    local.final_residual = res;
    if (!std::isfinite(res)) {
      status = fail(MDP_ERR_NUMERIC, "non-finite Bellman residual");
      break;
    }
    if (res <= o->atol_pi) {
      local.converged = 1;
      break;
    }
    if (k >= o->max_iter_pi) {
      status = fail(MDP_NOT_CONVERGED, "max_iter_pi policy evaluations without reaching atol_pi");
      break;
    }
    sweep_range.pop();
    // step 4: the policy's rows P_pi and costs g_pi, gathered into the per-state layout
    NvtxRange eval_range("policy evaluation");
    s = extract_policy(h, pi, mixed, st);
    if (s != MDP_OK) {
      status = s;
      break;
    }
    // steps 5-12: theta_0 = V_k, solve J_pi theta = g_pi to ||.||_2 < alpha * ||r(V_k)||_inf
    int it = 0;
    double r2 = 0.0;
    if (o->record_timing) MDP_CUDA(cudaEventRecord(h->ev2, st));
    s = inner_solve(h, o->gamma, V, o->inner, o->gmres_restart, o->gmres_refine, o->precision,
                    o->richardson_scale, o->alpha * res, o->max_iter_ksp, &it, &r2, st);
    if (s != MDP_OK) {
      status = s;
      break;
    }
    if (o->record_timing) {
      MDP_CUDA(cudaEventRecord(h->ev3, st));
      MDP_CUDA(cudaEventSynchronize(h->ev3));
      float ms = 0.f;
      MDP_CUDA(cudaEventElapsedTime(&ms, h->ev2, h->ev3));
      local.inner_ms += ms;
    }
    local.inner_iters_total += it;
    ++k;
  }
  MDP_CUDA(cudaEventRecord(h->done, st));
  MDP_CUDA(cudaStreamSynchronize(st));
  }
  local.outer_iters = k;
  local.bellman_value_bytes = lowp ? 2 : 8;
  if (lowp) {
    double* pin = tls_pinned();
    MDP_CUDA(cudaMemcpyAsync(pin, h->lp_rows, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    MDP_CUDA(cudaStreamSynchronize(st));
    unsigned long long rows = 0;
    std::memcpy(&rows, pin, sizeof(rows));
    local.bellman_rows_fp64 = (int64_t)rows;
  }
  local.kernel_launches = h->launches - launches0;
  local.policy_matvecs = h->matvecs - matvecs0;
  local.vector_reads = h->vreads - vreads0;
  local.vector_writes = h->vwrites - vwrites0;
  local.inner_bytes = h->inner_bytes - ibytes0;
  local.matvec_ms = h->mv_ms - mv_ms0;
  local.matvec_bytes = h->mv_bytes - mv_bytes0;
  local.matvec_flops = h->mv_flops - mv_flops0;
  local.matvecs_timed = h->mv_timed - mv_timed0;
  local.gs_ms = h->gs_ms - gs_ms0;
  local.gs_flops = h->gs_flops - gs_flops0;
  local.gs_timed = h->gs_timed - gs_timed0;
  local.policy_value_bytes = !mixed ? 8 : (h->pstore == kStoreF32 ? 4 : 2);
  local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = local;
  return status;
}

}  // extern "C"
