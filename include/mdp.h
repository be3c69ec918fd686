/*
 * mdp.h -- C ABI of the GB300 inexact-policy-iteration library (libmdp).
 *
 * The library solves discounted infinite-horizon MDPs {S, A, P, g, gamma} with
 * finite state and action spaces (Sec. II of "Inside madupite", arXiv
 * 2507.22538) by inexact policy iteration (Algorithm 1).  All arithmetic runs
 * in the library's own CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *  - States are 0..S-1 and actions 0..A-1.  The transition tensor is passed
 *    row-stacked as in Eq. 5: an (S*A) x S CSR matrix whose row s*A + a holds
 *    P(s, ., a).  Stage costs are an S x A row-major array, g[s*A + a] = g(s, a).
 *  - Unless stated otherwise every array argument is a DEVICE pointer owned by
 *    the caller; the library reads/writes it in stream order on `stream` (a
 *    cudaStream_t passed as void*; NULL means the legacy default stream).
 *  - Every function returns an mdp_status and never aborts the process.  On
 *    failure mdp_last_error() returns a message for the calling thread.
 *  - A handle may be used by one host thread at a time.
 */
#ifndef MDP_H_
#define MDP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdp_s* mdp_handle; /* opaque; owns a device copy of P and g */

typedef enum {
  MDP_OK = 0,
  MDP_ERR_INVALID_ARG = 1,    /* bad size, null pointer, gamma outside (0,1), ... */
  MDP_ERR_NOT_STOCHASTIC = 2, /* a row is empty, has a column outside [0,S), a negative or
                                 non-finite probability, or does not sum to 1 */
  MDP_ERR_OOM = 3,            /* device or pinned-host allocation failed */
  MDP_ERR_CUDA = 4,           /* a CUDA runtime call failed */
  MDP_NOT_CONVERGED = 5,      /* an iteration cap was hit; outputs hold the last iterate */
  MDP_ERR_NUMERIC = 6         /* NaN or Inf appeared in a residual */
} mdp_status;

/* Storage type of the P values passed to mdp_create.  The library widens every value
   exactly to binary64 on the device, so an MDP whose probabilities are exact in a
   narrower type (multiples of 2^-11 summing to 1 are exact in binary16, of 2^-8 in
   bfloat16) gives the same handle, and the same results bit for bit, from either
   type; the narrower one only moves fewer bytes at upload. */
typedef enum { MDP_F64 = 0, MDP_F32 = 1, MDP_F16 = 2, MDP_BF16 = 3 } mdp_dtype;

/* Inner solvers of Algorithm 1 (Sec. III-B.3, Table 2): restarted GMRES (the
   default), Richardson (VI, OPI(W), beta-VI), TFQMR (used for the pendulum and
   maze studies, Sec. IV-C/D; one half step = one iteration), and Richardson with
   the Jacobi preconditioner D = diag(I - gamma P_pi) (J-VI). */
typedef enum { MDP_GMRES = 0, MDP_RICHARDSON = 1, MDP_TFQMR = 2, MDP_RICHARDSON_JACOBI = 3 } mdp_inner;

/* Gram-Schmidt refinement inside GMRES (the choices of PETSc's KSPGMRES, whose
   default madupite inherits, Sec. III-B.3): classical Gram-Schmidt with no second
   pass, a second pass when the projected norm drops below 1/sqrt(2) of the
   original (Daniel-Gragg-Kaufman-Stewart test), or always two passes. */
typedef enum { MDP_REFINE_NEVER = 0, MDP_REFINE_IFNEEDED = 1, MDP_REFINE_ALWAYS = 2 } mdp_refine;

/* Arithmetic of the GMRES inner solve.  MDP_PREC_F64: everything in binary64.
   MDP_PREC_MIXED: each restart forms the residual g_pi - J_pi theta and updates
   theta in binary64, while the Arnoldi cycle (mat-vec with binary32 copies of the
   policy's probabilities, basis vectors, Gram-Schmidt) runs in binary32 and the
   Hessenberg least-squares in binary64; restarted GMRES then acts as iterative
   refinement.  The Bellman sweep and the outer stop test are binary64 in both. */
typedef enum { MDP_PREC_F64 = 0, MDP_PREC_MIXED = 1 } mdp_precision;

/* Options of Algorithm 1 with the defaults of Table 1 (set by mdp_default_opts). */
typedef struct {
  double gamma;            /* discount factor, 0 < gamma < 1 (no default; must be set) */
  double atol_pi;          /* tol: outer stop when ||TV - V||_inf <= atol_pi          (1e-8) */
  double alpha;            /* inner stop when ||g_pi - J_pi theta||_2 < alpha*||r(V_k)||_inf (1e-4) */
  double richardson_scale; /* omega of the Richardson step theta += omega (b - J theta) (1.0) */
  int32_t max_iter_pi;     /* N_o: at most this many policy evaluations             (1000) */
  int32_t max_iter_ksp;    /* N_i: at most this many inner iterations per evaluation (1000) */
  int32_t gmres_restart;   /* GMRES restart length m, 1..32                            (30) */
  int32_t inner;           /* an mdp_inner value                                  (MDP_GMRES) */
  int32_t record_timing;   /* nonzero: time Bellman sweeps and inner solves (CUDA events) (0) */
  int32_t gmres_refine;    /* an mdp_refine value                          (MDP_REFINE_NEVER) */
  int32_t precision;       /* an mdp_precision value of the GMRES inner solve  (MDP_PREC_F64) */
  int32_t graph;           /* nonzero: with the GMRES inner solver and record_timing off, run the
                              whole of Algorithm 1 as one CUDA graph launch: conditional WHILE/IF
                              nodes over the sweep, the stop tests and the restart cycles, decided
                              on the device, with no host round trip until the solve ends.  Same
                              kernels and results, bit for bit, as the stream-driven solve.  The
                              instantiated graph stays in the handle and is rebuilt when V, pi,
                              gamma, the options or the Bellman launch shape change.  A batch
                              (mdp_solve_batch) runs as one graph launch when every member sets
                              it.                                                                 (0) */
  int32_t lowp_sweep;      /* nonzero: when every probability of the MDP is exact in binary16 or
                              bfloat16, run the Bellman sweeps as mdp_bellman_lowp does (16-bit
                              values, binary32 screen, binary64 re-evaluation of the rows that can
                              attain the minimum); V, pi, the iteration counts and the stop test are
                              bit for bit those of the binary64 sweep.  Otherwise ignored.  Ignored
                              by mdp_solve_batch.                                                 (0) */
} mdp_solve_opts;

/* Statistics of one mdp_solve call (host struct filled by the library). */
typedef struct {
  int32_t outer_iters;        /* policy evaluations performed (k at exit) */
  int32_t converged;          /* 1 when ||TV - V||_inf <= atol_pi at the returned V */
  int64_t inner_iters_total;  /* inner iterations summed over all evaluations */
  double final_residual;      /* ||TV - V||_inf at the returned V */
  double seconds;             /* host wall time of the call */
  int64_t kernel_launches;    /* CUDA kernels the call launched */
  int32_t bellman_sweeps;     /* Bellman sweeps launched */
  double bellman_ms;          /* summed device time of those sweeps (record_timing only) */
  double inner_ms;            /* summed device-timeline time of the inner solves, including
                                 host round trips between their kernels (record_timing only) */
  int64_t policy_matvecs;     /* applications of P_pi by the inner solver */
  int64_t vector_reads;       /* length-S double vectors the inner kernels must read, besides
                                 the P_pi applications (each counts its x once) */
  int64_t vector_writes;      /* length-S double vectors the inner kernels write */
  double inner_bytes;         /* algorithmic bytes the inner kernels must move, in their storage types */
  int32_t policy_value_bytes; /* bytes per probability the inner mat-vecs read: 8 (binary64), or with
                                 MDP_PREC_MIXED 4 (binary32) or 2 (binary16 / bfloat16, used when every
                                 probability of the MDP is exactly representable there) */
  double matvec_ms;           /* summed device time of the policy mat-vec kernels of GMRES steps
                                 j = 0, 8, 16, ... of every restart cycle, each between its own pair
                                 of CUDA events (record_timing only); in the FP64 single-pass solver the
                                 mat-vec kernel also forms the Gram-Schmidt dots */
  int64_t matvecs_timed;      /* mat-vec kernels timed in matvec_ms */
  double gs_ms;               /* summed device time of the FP64 single-pass Gram-Schmidt projection of
                                 the same steps (record_timing only) */
  double gs_flops;            /* its FP64 flops: 2 (j + 2) S for step j (j + 1 products and the norm) */
  int64_t gs_timed;           /* projections timed in gs_ms */
  int32_t bellman_value_bytes; /* bytes per probability the sweeps read: 8, or 2 with lowp_sweep */
  int64_t bellman_rows_fp64;  /* with lowp_sweep: rows the sweeps re-evaluated in binary64 (at least
                                 one per state and sweep: the rows that can attain the minimum) */
  double matvec_bytes;        /* algorithmic bytes of the kernels timed in matvec_ms: the policy's rows,
                                 u_j read, w written, and with the fused FP64 dots the j other basis
                                 vectors of step j (record_timing only) */
  double matvec_flops;        /* FP64 flops of the kernels timed in matvec_ms when the mat-vec also forms the
                                 Gram-Schmidt dots (FP64 single-pass steps): 2 (k + j + 2) per state for
                                 step j, k entries per row (record_timing only; 0 otherwise) */
} mdp_solve_stats;

/* Fill *opts with the Table 1 defaults (gamma is set to 0: the caller must set it). */
void mdp_default_opts(mdp_solve_opts* opts);

/*
 * mdp_create -- copy an MDP into device memory owned by the returned handle.
 * (Sec. III-B.2: row-stacked CSR of Eq. 5 and the dense S x A stage costs.)
 *
 *  S, A          number of states (1 .. 2^31-1) and actions (1 .. 8192), S*A < 2^36.
 *  row_ptr       int64[S*A + 1], row_ptr[0] = 0, nondecreasing.
 *  col           int32[nnz] column (successor state) of each entry, in [0, S).
 *  val           P values, nnz entries of val_type: double (MDP_F64), float (MDP_F32),
 *                IEEE binary16 (MDP_F16) or bfloat16 (MDP_BF16) bit patterns; widened
 *                exactly to binary64, so the row-sum test below applies to the widened
 *                values (MDP_ERR_INVALID_ARG for any other val_type).
 *  g             double[S*A] stage costs, finite.
 *  inputs_on_device  nonzero: the four arrays are device pointers; zero: host pointers
 *                (pinned host memory gives the fastest upload).  Host entries go up
 *                in row-aligned chunks of at most 2^25 entries on an internal copy
 *                stream, each converted to the device layout while later chunks are
 *                in flight; besides the handle, creation holds at most four chunks
 *                and the row pointers on the device.
 *  stream        stream for the upload and the layout kernels; the call returns
 *                after they complete.
 *  out           receives the handle (NULL on failure).
 * The caller keeps ownership of its arrays; the handle keeps its own copy in a
 * GPU-friendly layout.  Every row must be nonempty, have entries >= 0 that sum
 * to 1 within 1e-12, and columns in [0, S): otherwise MDP_ERR_NOT_STOCHASTIC.
 * A row_ptr that does not start at 0, decreases or leaves [0, nnz] (with no
 * empty row), or a non-finite cost with otherwise valid rows, gives
 * MDP_ERR_INVALID_ARG.
 */
mdp_status mdp_create(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const void* val,
                      mdp_dtype val_type, const double* g, int32_t inputs_on_device, void* stream,
                      mdp_handle* out);

/* Release every device and host resource of the handle (NULL is accepted).  Waits
   for the work of the handle's last call, then returns its memory to the
   stream-ordered pool without synchronising the device; calls on one handle must
   be ordered by the caller (one stream, or events between streams). */
mdp_status mdp_destroy(mdp_handle h);

/* Problem sizes of a handle (any out pointer may be NULL). */
mdp_status mdp_get_info(mdp_handle h, int64_t* S, int32_t* A, int64_t* nnz);

/*
 * mdp_bellman -- one application of the Bellman optimality operator (Eq. 3),
 * the greedy policy (Eq. 4) and the residual norm ||r(V)||_inf (Sec. II;
 * Algorithm 1 steps 2-3; computed as PV, reshaped S x A, scaled by gamma, plus
 * g, row-wise argmin: Sec. III-B.3), fused in one kernel.
 *
 *  V             double[S]  input value vector.
 *  TV            double[S]  TV(s) = min_a g(s,a) + gamma * sum_s' P(s,s',a) V(s').
 *  pi            int32[S]   the lowest action attaining the minimum.
 *  residual_inf  double[1]  max_s |TV(s) - V(s)| (device pointer; may be NULL).
 * Stream-ordered: returns without waiting for the kernel.
 */
mdp_status mdp_bellman(mdp_handle h, double gamma, const double* V, double* TV, int32_t* pi,
                       double* residual_inf, void* stream);

/*
 * mdp_bellman_lowp -- mdp_bellman for an MDP whose probabilities are all exact in
 * binary16 or bfloat16 (multiples of 2^-11 or 2^-8 summing to 1 per row, the
 * exact-dyadic inputs of the mixed-precision path; checked at mdp_create), with
 * the same outputs bit for bit and fewer bytes moved.  The sweep (Eq. 3-4,
 * Algorithm 1 steps 2-3) reads the stacked matrix as 16-bit values, screens every
 * row in binary32 against a rigorous rounding bound, and re-evaluates in binary64,
 * exactly as mdp_bellman does, every row that can attain the minimum (all rows of
 * a state whose screen is not finite); the min / lowest argmin / residual is then
 * mdp_bellman's own.  The first call on a handle builds the 16-bit copy of the
 * values (2 B per stored entry) and binary32 copies of g and V, which the handle
 * keeps.  The paper computes the greedy step in binary64 only (PETSc); this is the
 * same result computed with less memory traffic.
 *
 *  Arguments as for mdp_bellman.  MDP_ERR_INVALID_ARG when the probabilities are
 *  not exact in 16 bits.  Stream-ordered: returns without waiting for the kernel.
 */
mdp_status mdp_bellman_lowp(mdp_handle h, double gamma, const double* V, double* TV, int32_t* pi,
                            double* residual_inf, void* stream);

/*
 * mdp_policy_apply -- y = J_pi x = x - gamma * P_pi x, the matrix-free policy
 * operator of Sec. III-B.3 (Algorithm 1 step 4), for a policy pi.
 *  pi int32[S] with 0 <= pi[s] < A; x, y double[S] (may not alias).
 * Stream-ordered.
 */
mdp_status mdp_policy_apply(mdp_handle h, double gamma, const int32_t* pi, const double* x, double* y,
                            void* stream);

/*
 * mdp_policy_eval -- approximately solve (I - gamma P_pi) v = g_pi (Eq. 2), the
 * inexact policy evaluation of Algorithm 1 steps 4-12, from v0.
 *
 *  pi            int32[S] policy, 0 <= pi[s] < A.
 *  v0, v         double[S] start vector and result (may alias).
 *  inner         an mdp_inner value: MDP_GMRES (restart = `restart`), MDP_RICHARDSON or
 *                MDP_RICHARDSON_JACOBI (step scale `omega`), MDP_TFQMR.
 *  abs_tol_2norm stop when ||g_pi - J_pi v||_2 < abs_tol_2norm (Sec. III-B.3).
 *  max_it        at most this many iterations (a GMRES Arnoldi step or a Richardson step);
 *                GMRES uses classical Gram-Schmidt without refinement (MDP_REFINE_NEVER).
 *  iters, res_2norm  host outputs (may be NULL): iterations done and the last
 *                computed residual 2-norm.
 * Blocks until the solve completes.  Returns MDP_NOT_CONVERGED (with v filled)
 * when max_it is reached first.
 */
mdp_status mdp_policy_eval(mdp_handle h, double gamma, const int32_t* pi, const double* v0, double* v,
                           mdp_inner inner, int32_t restart, double omega, double abs_tol_2norm,
                           int32_t max_it, int32_t* iters, double* res_2norm, void* stream);

/*
 * mdp_solve -- inexact policy iteration, Algorithm 1.
 *
 *  opts   options (Table 1); opts->gamma must be in (0, 1).
 *  V      double[S]: in V_0, out the last iterate V_k (the first with
 *         ||TV_k - V_k||_inf <= atol_pi, or the last one when a cap is hit).
 *  pi     int32[S]: out the greedy policy of the returned V (ties: lowest action).
 *  stats  host struct (may be NULL).
 * Blocks until done.  MDP_NOT_CONVERGED when max_iter_pi evaluations did not
 * reach atol_pi (V, pi and stats are still filled).  With opts->graph set (GMRES,
 * record_timing off) the loop runs as one CUDA graph launch decided on the device,
 * with the same results bit for bit.
 */
mdp_status mdp_solve(mdp_handle h, const mdp_solve_opts* opts, double* V, int32_t* pi,
                     mdp_solve_stats* stats, void* stream);

/*
 * mdp_tune -- autotune the launch shape of the Bellman sweep (Eq. 3-4) on this
 * handle's matrix: times the fused sweep at V = 0 for each tile size (states per
 * block: 8 .. 512 that fit in shared memory) and keeps the fastest, then for that
 * tile the number of resident blocks per SM of its grid (from the occupancy limit
 * down to 1), which every later mdp_bellman, mdp_solve and mdp_solve_batch call on
 * the handle uses; when the probabilities are exact in 16 bits it also picks the
 * tile of the low-precision sweep (mdp_bellman_lowp).  The paper has no
 * counterpart (its sparse kernels are PETSc's).  Between the tile and the grid it
 * also picks, at full occupancy, the rows of the stacked matrix a warp takes per
 * step (32: one row per lane; 64: two rows per lane, their loads side by side) and
 * the width of the binary64 value loads (16 or 32 bytes per chunk of 4 entries).
 * Results do not depend on the launch shape: every state's Q values, minimum and
 * the residual are computed the same way in any tile, grid and variant.
 *
 *  gamma         discount factor of the timed sweeps, in (0, 1).
 *  tile_states   host out (may be NULL): the chosen tile size.
 *  ms_per_sweep  host out (may be NULL): the binary64 sweep's time per sweep with the
 *                chosen tile and grid.
 * Blocks until done.  Overwrites the handle's scratch vectors only.
 */
mdp_status mdp_tune(mdp_handle h, double gamma, int32_t* tile_states, float* ms_per_sweep, void* stream);

/*
 * mdp_get_sweep_shape -- the launch shape the Bellman sweep of this handle uses
 * (the creation defaults, or what mdp_tune or mdp_set_sweep_shape set).  Host
 * outputs, each may be NULL: states per block (tile), blocks of the grid, the cap on
 * resident blocks per SM (0: the occupancy limit), rows of the stacked matrix per
 * warp step (32 or 64) and bytes per binary64 value load (16 or 32); passing these
 * to mdp_set_sweep_shape restores the shape.  No device work.  The paper has no
 * counterpart.
 */
mdp_status mdp_get_sweep_shape(mdp_handle h, int32_t* tile_states, int32_t* blocks, int32_t* blocks_per_sm,
                               int32_t* rows_per_warp, int32_t* value_load_bytes);

/*
 * mdp_set_sweep_shape -- set the Bellman sweep's launch shape by hand, e.g. to reuse
 * what mdp_tune chose for the same matrix in an earlier run: states per block
 * (tile_states, whose Q values must fit in shared memory: tile_states * A * 8 bytes
 * <= 227 KB), rows per warp step (32 or 64), bytes per binary64 value load (16 or
 * 32) and resident blocks per SM of the grid (0: the occupancy limit).  Results do
 * not depend on the shape.  MDP_ERR_INVALID_ARG for an unsupported shape (the
 * handle keeps its previous one).  No device work.  The paper has no counterpart.
 */
mdp_status mdp_set_sweep_shape(mdp_handle h, int32_t tile_states, int32_t rows_per_warp, int32_t value_load_bytes,
                               int32_t blocks_per_sm);

/*
 * mdp_solve_batch -- Algorithm 1 on n independent MDPs at once (problems of
 * different S, A, row lengths and gamma), each with its own options, advanced
 * in lockstep: every kernel launch of the batch covers all problems that are
 * still running (per-problem descriptors and block ranges in device memory),
 * with one residual read per outer iteration and one solver-state read per
 * GMRES cycle for the whole batch.  The paper solves one MDP per call; this is
 * the same method applied to many, with the per-problem arithmetic unchanged:
 * each problem's V, pi, iteration counts and status equal those of mdp_solve on
 * that problem alone, bit for bit.  When every member's opts.graph is set, the
 * whole batch runs as one CUDA graph launch instead, whose independent branches
 * are the members' graph-driven solves (the nodes mdp_solve runs with opts.graph):
 * each problem's loops are decided on the device at its own pace, its kernels may
 * overlap with the other members', and nothing returns to the host until all have
 * stopped.  The graph is built and destroyed by the call (a handle's own cached
 * graph is dropped and rebuilt by its next graph-driven mdp_solve); the results
 * are the same bit for bit.
 *
 *  n        number of problems, >= 1.
 *  handles  [n] distinct handles on the current device (each used by this call only).
 *  opts     [n] options as for mdp_solve; inner must be MDP_GMRES and gmres_refine
 *           MDP_REFINE_NEVER; precision MDP_PREC_F64 or MDP_PREC_MIXED, per problem.
 *  V, pi    [n] device pointers: V[i] double[S_i] (in V_0, out V), pi[i] int32[S_i].
 *  stats    [n] host structs (may be NULL): per problem as mdp_solve, except that
 *           seconds and kernel_launches are those of the whole batch and the
 *           bellman_ms, inner_ms and byte counters are not filled (0).
 *  status   [n] host: each problem's mdp_solve status (MDP_OK, MDP_NOT_CONVERGED,
 *           MDP_ERR_NUMERIC).
 * Blocks until every problem has stopped.  Returns MDP_OK when the batch ran
 * (per-problem outcomes in status[]), MDP_ERR_INVALID_ARG for a bad argument
 * (nothing runs), MDP_ERR_OOM or MDP_ERR_CUDA when the batch could not run.
 */
mdp_status mdp_solve_batch(int32_t n, const mdp_handle* handles, const mdp_solve_opts* opts, double* const* V,
                           int32_t* const* pi, mdp_solve_stats* stats, mdp_status* status, void* stream);

/*
 * mdp_solve_small_batch -- Algorithm 1 on n small MDPs, each solved from start to
 * finish by one thread-block cluster (1 to 8 blocks, about 512 states per block),
 * the whole batch in one kernel launch per cluster size, with no host round trip
 * until every problem has stopped.  The sweep (Eq. 3-4), the stop tests, the
 * policy's rows and GMRES(m) with classical Gram-Schmidt and Givens rotations (the
 * method of mdp_solve) run inside the cluster; every reduction is a fixed-order
 * block sum followed by a fixed-order sum over the cluster's blocks.  The paper
 * solves one MDP per call with distributed PETSc kernels; this is the same method
 * for many small problems, where one grid-wide kernel per Arnoldi pass would be
 * bound by launch latency.
 *
 *  n        number of problems, >= 1.
 *  handles  [n] distinct handles on the current device, each with S <= 65536.
 *  opts     [n] options as for mdp_solve; inner MDP_GMRES, gmres_refine
 *           MDP_REFINE_NEVER and precision MDP_PREC_F64 (graph, record_timing and
 *           lowp_sweep are ignored).
 *  V, pi    [n] device pointers: V[i] double[S_i] (in V_0, out V), pi[i] int32[S_i].
 *  stats    [n] host structs (may be NULL): outer_iters, inner_iters_total,
 *           final_residual, converged, bellman_sweeps; seconds and kernel_launches
 *           are those of the whole batch.
 *  status   [n] host: each problem's outcome (MDP_OK, MDP_NOT_CONVERGED, MDP_ERR_NUMERIC).
 * Each problem's arithmetic depends on its own size only, so its V, pi and counts
 * are the same bit for bit alone and in any batch.  They are certified like
 * mdp_solve's results, but not bit-identical to them: the reductions add in a
 * different order.  Blocks until every problem has stopped.  Returns MDP_OK when
 * the batch ran, MDP_ERR_INVALID_ARG for a bad argument (nothing runs).
 */
mdp_status mdp_solve_small_batch(int32_t n, const mdp_handle* handles, const mdp_solve_opts* opts,
                                 double* const* V, int32_t* const* pi, mdp_solve_stats* stats,
                                 mdp_status* status, void* stream);

/*
 * mdp_bellman_csr_noalloc -- the Bellman application of mdp_bellman (TV, greedy pi,
 * ||TV - V||_inf) computed straight from the caller's row-stacked CSR arrays,
 * with no handle and no device allocation.  The paper has no counterpart: it is
 * for callers that cannot allocate device memory at the point of the call, such
 * as an application that hands out every device allocation through its own pool,
 * a plug-in whose host program forbids allocation inside the call, or a real-time
 * loop that cannot afford the synchronisation an allocation may cause.
 *
 *  S, A          at most 2,097,152 states and 128 actions (else MDP_ERR_INVALID_ARG).
 *  row_ptr, col, val, g   device arrays laid out as for mdp_create; the caller
 *                guarantees they are valid (this call does not check them).
 *  V, TV, pi, residual_inf   as for mdp_bellman (residual_inf may be NULL).  The outputs
 *                TV, pi and residual_inf must not share any byte with one another or
 *                with V, g or row_ptr (MDP_ERR_INVALID_ARG); col and val, whose length the
 *                call does not know, must not overlap them either.
 * Scratch: a fixed 512 KB array in the library's device memory, present on every
 * GPU that loads the library until the process exits.  Its device address is
 * looked up on the first call made on each device (that first call must not be
 * inside a stream capture); later calls only launch work.  All calls share the
 * array, so calls that may overlap on the GPU (different streams, no ordering
 * between them) race and must not be issued.  Stream-ordered: returns without
 * waiting for the kernel.
 */
mdp_status mdp_bellman_csr_noalloc(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col,
                                   const double* val, const double* g, double gamma, const double* V,
                                   double* TV, int32_t* pi, double* residual_inf, void* stream);

/* Message describing the last failure on the calling thread ("" if none). */
const char* mdp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MDP_H_ */
