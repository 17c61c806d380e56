/*
 * mdp.h -- C ABI of the GB300 (sm_103a) MDP path planner library
 *          (libmdp_gb300.so).
 *
 * The library builds and solves the finite-horizon, undiscounted, total-cost
 * MDP of Chowdhury & Subramani, "Optimal Path Planning of Autonomous Marine
 * Vehicles in Stochastic Dynamic Ocean Flows using a GPU-Accelerated
 * Algorithm" (arXiv 2109.00857):
 *   - model build (Sec. III-A/B/C, Alg. 1 and Alg. 2): for every (time step,
 *     grid cell, action) it draws N realizations of the dynamically orthogonal
 *     (DO) velocity v = vbar + mu_i v~_i (Sec. II-C), takes one Euler step
 *     x' = x + (v + a) dt (Sec. II-A), counts the landing cells on the
 *     neighbouring sub-grid and emits sparse P(s'|s,a) = count/N and the
 *     expected one-step reward R(s,a) for the time, energy and net-energy
 *     objectives (Eqs. Rsa_time, Rsa_energyConsumption, Rsa_NetEnergy, with
 *     the mean scalar field only, as proved in Sec. III-A);
 *   - sparse value iteration (Sec. II-B, Sec. III-D):
 *     v_{k+1}(s) = max_a sum_{s'} P(s'|s,a) [r + v_k(s')], greedy policy.
 *
 * Conventions used by every call
 *   - Pointers named *_h are HOST pointers; every other array pointer is a
 *     DEVICE pointer on the current CUDA device.  The caller owns every array
 *     it passes and keeps it alive until the work on `stream` completes.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work of a call is ordered on that stream.
 *   - Kinematics are in grid units: the agent starts at the centre of cell
 *     (i, j), i.e. x = (i + 1/2) dx, and cell(x) = floor(x / dx) with
 *     half-open cells.  Velocities are in length per time, dx and dt scale them.
 *   - State index s = t*Nc + j*Nx + i (Nc = Nx*Ny), |S| = Nt*Nc; the sink
 *     state (outside the domain, obstacle, beyond the horizon) is s = |S|
 *     with V(sink) = 0.
 *   - Exported rows follow the paper's appended layout: row = a*|S| + s
 *     (Sec. III-C, P appended over actions), successors ascending, sink last.
 *   - Errors: every call returns an mdp_status; mdp_last_error() gives a
 *     thread-local message.  The library never traps, asserts on the device,
 *     exits or aborts; device-side problems are reported through a status
 *     word read back once per call.  There is no CPU fallback: without a
 *     usable CUDA device every call returns MDP_ERR_CUDA.
 */
#ifndef MDP_GB300_H
#define MDP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MDP_OK = 0,
  MDP_ERR_ARG = -1,               /* invalid argument (message says which) */
  MDP_ERR_OOM = -2,               /* device allocation failed or pool capacity hit */
  MDP_ERR_SUBGRID_OVERFLOW = -3,  /* a landing fell outside the neighbouring sub-grid */
  MDP_ERR_ELL_OVERFLOW = -4,      /* a row had more successors than the row cap (batched
                                     builds and 3-D builds, which keep no spill area) */
  MDP_ERR_TIMEOUT = -5,           /* a bounded wait expired */
  MDP_ERR_CUDA = -6,              /* a CUDA runtime error (message has the CUDA string) */
  MDP_ERR_BUDGET = -7,            /* request does not fit the server's HBM budget */
  MDP_ERR_CANCELLED = -8,         /* request cancelled or server shutting down */
  MDP_ERR_NOT_FOUND = -9,         /* unknown ticket / env id */
  MDP_ERR_PENDING = -10           /* result not ready within the poll timeout */
} mdp_status;

/* prob_type (Alg. 1 input): the mission objective. */
typedef enum { MDP_OBJ_TIME = 0, MDP_OBJ_ENERGY = 1, MDP_OBJ_NET_ENERGY = 2 } mdp_objective;

/* Arithmetic of a build/solve.  FP32 is the production path.  FP64_CHECK runs
 * the literal FP64 formulas in the oracle's operation order (no contraction)
 * so that counts are bit-identical to an FP64 reference; it is slow and meant
 * for small problems. */
typedef enum { MDP_FP32 = 0, MDP_FP64_CHECK = 1 } mdp_precision;

/* grid_params (Alg. 1 input, Sec. IV): grid sizes, cell side dx, time step dt. */
typedef struct {
  int32_t nx, ny, nt;
  double dx, dt;
} mdp_grid;

/* prob_params (Alg. 1 input, Sec. II-A): the action space and reward constants.
 * Action a = f*n_headings + h has heading 2 pi h / n_headings and speed
 * f_max (f+1)/n_speeds.  If table_h is non-NULL it overrides that rule:
 * table_h[3a+0..2] = (F cos theta, F sin theta, F) in FP64.  A = n_headings *
 * n_speeds must be in [1, 32]. */
typedef struct {
  int32_t n_headings, n_speeds;
  double f_max;
  const double *table_h;  /* host [A][3] or NULL */
  double c_f;             /* energy function e(F) = c_f F^2 (Eq. Rsa_energyConsumption) */
  double c_r;             /* scalar-field coefficient (Eq. Rsa_NetEnergy) */
  double r_term;          /* reward added on reaching a target cell */
  double r_outbound;      /* reward for obstacle / outside / beyond the horizon */
} mdp_actions;

/* Environment data (Alg. 1 inputs: vbar, v~_i, mu_i, gbar, m).  Element type of
 * every floating array is float for MDP_FP32 and double for MDP_FP64_CHECK.
 * Alignment: vbar and modes to one (x, y) pair (8 B FP32, 16 B FP64), coeffs
 * to 16 B, gbar to 4 B; otherwise mdp_build returns MDP_ERR_ARG. */
typedef struct {
  int32_t K;               /* number of DO modes, 0..16 */
  int32_t precision;       /* mdp_precision */
  const void *vbar;        /* [nt][ny][nx][2] DO mean velocity */
  const void *modes;       /* [nt][K][ny][nx][2] DO modes */
  const void *coeffs;      /* [nt][N][K] DO coefficients mu_i(t; w), or NULL: drawn by the
                              library as sigma_h[k] * z, z ~ N(0,1) from Philox4x64-10 */
  const double *sigma_h;   /* host [K] coefficient standard deviations (used if coeffs NULL) */
  uint64_t seed;           /* Philox key word 0 (used if coeffs NULL) */
  uint64_t mdp_id;         /* Philox key word 1 (used if coeffs NULL) */
  const void *gbar;        /* [nt][ny][nx] mean scalar field, NULL unless net energy is asked */
  const uint8_t *obstacle; /* [nt][ny][nx] dynamic obstacle mask m (nonzero = obstacle) */
  const uint8_t *target;   /* [ny][nx] target (terminal) cells (nonzero = target) */
} mdp_env;

/* Build options (zero-initialise for defaults). */
typedef struct {
  int32_t row_cap;         /* in-domain successors a row keeps in the sliced-ELL columns, <= 255;
                              0 = 64.  The rest of a longer row goes to its slice's spill
                              block (HYB); the sink's count is stored apart in either case */
  int32_t no_compact;      /* 1: keep the worst-case entry pool instead of compacting it */
  int32_t threads;         /* CTA size of the FP32 full-window kernel (multiple of 64, <= 512);
                              0 = the autotuner's choice for the workload class (see
                              mdp_autotune) if one was recorded or loaded, else 256 */
  int32_t chunk;           /* realizations staged per pass by that kernel; 0 = the autotuner's
                              choice, else 1024 */
  int32_t hist_cap;        /* fine-count table cells (32-bit words) per warp of the
                              warp-per-slice kernel, <= 6144; 0 = the autotuner's choice,
                              else 2048; slices whose tables need more go to the
                              full-window kernel (1 sends every sampled slice there) */
} mdp_build_opts;

typedef struct mdp_model_t *mdp_model;

/* Builds P and R for n_obj objectives from one set of samples (Alg. 1; the
 * counts do not depend on the objective).  N in [1, 65535], subgrid_L odd in
 * [1, 255] (0 = smallest window that holds every landing, computed from the
 * field extremes as the paper sizes it from the component-wise maximum
 * velocity plus a buffer).  objs_h: host [n_obj], n_obj in [1, 3].
 * On success *out owns all model memory (free with mdp_model_free).
 * Rows of any length are stored: the first row_cap in-domain successors in
 * the sliced-ELL columns, the rest in a spill area (allocated only when some
 * row needs it; the build then runs a second time with the area sized
 * exactly).  Returns MDP_ERR_SUBGRID_OVERFLOW if any landing left the
 * sub-grid; *out is NULL then.  Synchronises `stream` once at the end to
 * read the status word (twice when the first attempt ran out of room). */
mdp_status mdp_build(const mdp_env *env, const mdp_grid *grid, const mdp_actions *actions,
                     int32_t N, int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj,
                     const mdp_build_opts *opts, void *stream, mdp_model *out);

typedef struct {
  int64_t n_states;        /* |S| = nt*nx*ny (sink excluded) */
  int32_t A;               /* actions */
  int32_t N;               /* realizations */
  int32_t L;               /* sub-grid side used */
  int32_t n_obj;           /* objectives with an R vector */
  int32_t objs[3];
  int32_t precision;
  int64_t rows;            /* A * |S| */
  int64_t nnz;             /* stored successors over all rows (sink entries included) */
  int32_t max_row_nnz;     /* widest row in the sliced-ELL columns (<= row_cap) */
  int64_t pool_columns;    /* 32-entry columns of the sliced-ELL entry pool in use */
  int64_t device_bytes;    /* device memory owned by the model */
  int64_t samples;         /* landing evaluations performed (N per sampled (s,a)) */
  double build_ms;         /* device time of sampler + build kernels (CUDA events) */
  double kernel_ms;        /* device time of the fused build kernel alone (CUDA events) */
  int32_t launches;        /* kernels the build launched */
  int64_t wide_slices;     /* slices built by the full-window kernel (tables > hist_cap) */
  int64_t nnz_domain;      /* stored successors inside the domain (sink entries excluded) */
  int64_t spill_rows;      /* rows longer than row_cap (their tails are in the spill area) */
  int64_t spill_words;     /* 32-bit words of the spill area (33 per spilling slice + entries) */
  int32_t max_row_len;     /* longest row: in-domain successors, spill included */
} mdp_model_info_t;

mdp_status mdp_model_info(mdp_model m, mdp_model_info_t *out);

/* Paper-layout CSR export of P and the R of objective slot obj (Sec. III-C COO
 * rows appended over actions).  rowptr: device int64 [A*|S|+1]; col: device
 * int64 [nnz] (sink = |S|); count: device int32 [nnz] with P = count/N;
 * R: device [A*|S|] float (FP32) or double (FP64_CHECK); any of col, count, R
 * may be NULL to skip it.  Synchronises `stream`. */
mdp_status mdp_export_csr(mdp_model m, int32_t obj, int64_t *rowptr, int64_t *col,
                          int32_t *count, void *R, void *stream);

/* Solve schedules. */
typedef enum {
  MDP_SOLVE_JACOBI = 0,       /* Jacobi sweeps V_{k+1} = T V_k with a device residual (Sec. II-B).
                                * A sweep recomputes only the time layers t whose own values or
                                * whose successor layer t+1 changed in the previous sweep; every
                                * other state has V_{k+1}(s) = V_k(s) exactly, so iterates, policy,
                                * residuals and sweep count equal MDP_SOLVE_JACOBI_FULL bit for bit */
  MDP_SOLVE_LAYERED = 1,      /* one backward pass over time layers t = nt-1..0 (same fixed point) */
  MDP_SOLVE_JACOBI_FULL = 2,  /* Jacobi sweeps over every state in every sweep */
  MDP_SOLVE_WARM = 16         /* flag, OR-ed into MDP_SOLVE_JACOBI or _JACOBI_FULL of mdp_solve
                                * (one objective): V on entry is V_0 (e.g. the previous plan's
                                * values when replanning, Sec. V) instead of 0; V[|S|] is reset to 0.
                                * This MDP reaches its exact fixed point from any V_0 within nt + 1
                                * sweeps, so with tol = 0 the result equals the cold start's bit for
                                * bit; a V_0 near the fixed point needs fewer sweeps */
} mdp_solve_method;

typedef struct {
  int32_t sweeps;          /* sweeps executed (layered: 1) */
  double residual;         /* max |V_k - V_{k-1}| of the last sweep (layered: 0) */
  double solve_ms;         /* device time of the solve kernels (CUDA events) */
  int64_t backups;         /* (s,a) Bellman backups computed (MDP_SOLVE_JACOBI: the
                            * recomputed layers only; fused solves: for all objectives) */
} mdp_solve_stats;

/* Value iteration on the model's P and the R of objective slot obj.
 * V: device [|S|+1] float (FP32) or double (FP64_CHECK), V[|S|] = 0 (sink);
 * policy: device int16 [|S|], argmax_a with the lowest index winning ties,
 * -1 for terminal and obstacle start states.  Jacobi starts from V = 0 (or,
 * with MDP_SOLVE_WARM, from V as given) and stops when max|V_{k+1} - V_k| <= tol
 * or after max_sweeps sweeps
 * (0 = nt + 1, which reaches the exact fixed point of this time-layered MDP).
 * Synchronises `stream` once to read the sweep count and residual. */
mdp_status mdp_solve(mdp_model m, int32_t obj, int32_t method, double tol, int32_t max_sweeps,
                     void *V, int16_t *policy, void *stream, mdp_solve_stats *stats);

/* Value iteration for n (1..3) objectives of one model at once (Sec. II-B
 * backup per objective; Sec. III-D solves each objective's MDP on the same
 * P).  Each sweep streams the transition slices once for all n objectives;
 * every objective keeps its own R, V, policy and residual, so objective o's
 * V, policy, sweeps and residual equal those of mdp_solve(m, objs[o], ...)
 * with the same method, tol and max_sweeps bit for bit (an objective that
 * met tol stops updating while the others continue).
 * objs: host [n] objective slots (repeats allowed); V, policy: host arrays of
 * n device pointers laid out as in mdp_solve; stats: host [n] or NULL.
 * solve_ms is the device time of the whole fused solve for every entry.
 * Errors: MDP_ERR_ARG for n outside 1..3, a NULL pointer or a slot out of
 * range; otherwise as mdp_solve.  Synchronises `stream` once. */
mdp_status mdp_solve_multi(mdp_model m, int32_t n, const int32_t *objs, int32_t method, double tol,
                           int32_t max_sweeps, void *const *V, int16_t *const *policy, void *stream,
                           mdp_solve_stats *stats);

/* The same Jacobi value iteration as mdp_solve (method MDP_SOLVE_JACOBI),
 * for callers that may not allocate device memory once they are running:
 * a real-time replanning loop that must not block or fragment its memory
 * budget, or a program whose device memory belongs to another allocator.
 * The paper has no counterpart of this call.  Its scratch (the second value
 * buffer, the residual slots, status words, per-sweep work counts and the
 * layer flags of the active-layer sweeps; models with more than 4095 time
 * layers run full sweeps, same results) is a fixed array inside the
 * library, 8 MiB + 76 KiB per GPU, held by every GPU that loads the library
 * until the process exits; it performs no cudaMalloc or cudaFree.
 * Limits: (|S| + 1) values must fit 8 MiB (at most 2,097,151 states in FP32,
 * 1,048,575 in FP64_CHECK) and max_sweeps (0 = nt + 1) must be <= 4092;
 * larger requests return MDP_ERR_ARG with a message (use mdp_solve).
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  Every call reuses the same array
 * and clears what must start at zero, so calls whose work overlaps on the
 * GPU (on different streams, or from different threads) race and must not
 * be issued.  Arguments, outputs and errors as in mdp_solve; solve_ms is 0. */
mdp_status mdp_solve_noalloc(mdp_model m, int32_t obj, double tol, int32_t max_sweeps, void *V,
                             int16_t *policy, void *stream, mdp_solve_stats *stats);

void mdp_model_free(mdp_model m);

/* DO coefficients alone (step a1): Y[t][w][k] = sigma_h[k] * z with z from the
 * Marsaglia polar method on Philox4x64-10 (Salmon et al., SC'11) counters
 * (t, w, pair k/2, attempt) under key (seed, mdp_id).  Y: device [nt][N][K],
 * float (FP32) or double (FP64_CHECK); the FP32 table is the FP64 draw rounded. */
mdp_status mdp_sample_coeffs(int32_t nt, int32_t N, int32_t K, const double *sigma_h,
                             uint64_t seed, uint64_t mdp_id, int32_t precision, void *Y,
                             void *stream);

/* ------------------------------------------------------------- 3-D grid --
 * The build on a 3-D grid (Sec. II-A: the formulation holds for n = 3).  Cube
 * cells, state s = t*Nc + (k*ny + j)*nx + i with Nc = nx*ny*nz, a cubic
 * neighbouring sub-grid of side subgrid_L (odd, 1..11; no automatic size).
 * The returned model has the 2-D layout (successor offsets dk*nx*ny + dj*nx
 * + di as signed 16 bits: subgrid half-width * (nx*ny + nx + 1) <= 32767),
 * so mdp_solve, mdp_solve_multi, mdp_export_csr, mdp_model_info and
 * mdp_model_free apply unchanged.  FP32 lands with the exact floor of
 * u + d per axis like the 2-D build; FP64_CHECK follows the oracle's
 * literal formulas.  Errors as mdp_build. */
typedef struct {
  int32_t nx, ny, nz, nt;
  double dx, dt;
} mdp_grid3d;

typedef struct {
  int32_t K;
  int32_t precision;        /* mdp_precision */
  const void *vbar;         /* [nt][nz][ny][nx][3] */
  const void *modes;        /* [nt][K][nz][ny][nx][3] */
  const void *coeffs;       /* [nt][N][K] or NULL (drawn as in mdp_env) */
  const double *sigma_h;    /* host [K] */
  uint64_t seed, mdp_id;
  const void *gbar;         /* [nt][nz][ny][nx] or NULL */
  const uint8_t *obstacle;  /* [nt][nz][ny][nx] */
  const uint8_t *target;    /* [nz][ny][nx] */
} mdp_env3d;

typedef struct {
  int32_t A;                /* 1..32 */
  const double *table_h;    /* host [A][4]: (d_x, d_y, d_z, F) per action */
  double c_f, c_r, r_term, r_outbound;
} mdp_actions3d;

mdp_status mdp_build3d(const mdp_env3d *env, const mdp_grid3d *grid, const mdp_actions3d *actions,
                       int32_t N, int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj,
                       void *stream, mdp_model *out);

/* FP32 counting, with at most 4 states per slice and at most 8 distinct step
 * thresholds per axis: each realization is counted once at its fine
 * coordinate (floor(u) - n0) S + rank(frac u) per axis, and every (action,
 * offset bin) count is a box sum of the fine table's prefix sums -- by one
 * warp per slice while the slice's tables fit the warp's 2048 words, else by
 * a CTA per slice (whose realizations must fit one staging chunk: N <= 5461
 * for one state per slice).  Other slices (and FP64_CHECK) count one
 * increment per (realization, action).  All ways give the same model.
 * per_action = 1 forces the last way for every slice (a reference for tests
 * and comparisons).  3-D models keep every row in the sliced-ELL columns (no
 * spill area): a row with more than 255 stored successors (possible for
 * sub-grids above 5 x 5 x 5 cells) makes the build return
 * MDP_ERR_ELL_OVERFLOW. */
typedef struct {
  int32_t per_action;
} mdp_build3d_opts;

/* mdp_build3d with options (opts may be NULL: the defaults). */
mdp_status mdp_build3d_ex(const mdp_env3d *env, const mdp_grid3d *grid, const mdp_actions3d *actions,
                          int32_t N, int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj,
                          const mdp_build3d_opts *opts, void *stream, mdp_model *out);

/* ------------------------------------------------------------- rollouts --
 * Policy rollouts (Sec. IV: the optimal policy applied to every flow
 * realization from the start; the mean returns are the expected mission
 * time, energy and net energy).  Path (q, w) starts at cell starts_h[2q],
 * starts_h[2q+1] at t = 0 and follows policy[s] (device int16 [nt*ny*nx], as
 * written by mdp_solve), moving with realization w's velocity of time t at
 * its state -- the build's kinematics with the same env, grid, actions and N
 * (coefficients from env->coeffs or drawn as mdp_build draws them), so each
 * move is one of the samples the build counted.  A path ends on a target cell
 * (status 0) or in the sink (status 1: outside the domain, an obstacle at
 * t+1, a move from the last layer, or policy -1), which pays r_outbound; each
 * step adds the one-step reward of objective objs_h[o].
 * Outputs (each may be NULL): ret device [n_starts][N][n_obj] float (FP32) or
 * double (FP64_CHECK), steps device int32 [n_starts][N], status device int8
 * [n_starts][N]; summary_h host [n_starts].  Synchronises `stream` once.
 * Errors: MDP_ERR_ARG for bad sizes, pointers, objectives or start cells. */
typedef struct {
  double mean_return[3];     /* per objective slot, over the N paths */
  double p_target;           /* fraction of paths that reached a target cell */
  double mean_steps_target;  /* mean steps of those paths (0 if none) */
  int64_t paths;             /* N */
} mdp_rollout_summary;

mdp_status mdp_rollout(const mdp_env *env, const mdp_grid *grid, const mdp_actions *actions,
                       int32_t N, const int16_t *policy, const int32_t *starts_h, int32_t n_starts,
                       const int32_t *objs_h, int32_t n_obj, void *ret, int32_t *steps,
                       int8_t *status, mdp_rollout_summary *summary_h, void *stream);

/* ------------------------------------------------------------ autotuner --
 * Launch shapes per workload class, chosen by timing candidates (the paper's
 * authors tuned threads per block by hand for each GPU, Sec. IV-D; here the
 * library does it).  A class is (actions padded to a power of two, modes, N
 * and cells rounded to powers of two, objectives, precision).  The shapes:
 * warps per CTA (4, 8) and fine-table words per warp (1536..4096) of the
 * warp-per-slice build kernel, the CTA size of the full-window kernel when the
 * calibration defers slices to it, and the shared memory of the
 * one-state-per-slice Bellman sweep (132, 160, 190 KiB: its slot size).
 * No choice changes a count, entry, R, value or policy -- only the speed.
 * mdp_build, mdp_solve, mdp_solve_multi and the batch use the process-wide
 * table's entry for a model's class wherever the caller leaves an option 0.
 *
 * mdp_autotune times every candidate on a calibration cut of the caller's
 * environment (its first layers, about 200,000 states; arguments as in
 * mdp_build), records the fastest in the table and, if json_path is not
 * NULL, merges it into that JSON file ({"<class>": {"build_warps": ..,
 * "hist_cap": .., "threads": .., "chunk": .., "sweep_smem_kb": ..}, ...}).
 * mdp_tuning_load installs a file's entries (MDP_ERR_ARG if it cannot be read
 * or parsed; entries outside the kernels' limits are skipped). */
typedef struct {
  int32_t build_warps, hist_cap, threads, chunk, sweep_smem_kb;
  double build_kernel_ms;    /* calibration build kernel time with the chosen shapes */
  double sweep_ms;           /* calibration solve time with the chosen sweep memory */
  int32_t candidates;        /* configurations timed */
  int32_t calibration_layers;
  char key[64];              /* workload class */
} mdp_tuning;

mdp_status mdp_autotune(const mdp_env *env, const mdp_grid *grid, const mdp_actions *actions, int32_t N,
                        int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj, const char *json_path,
                        void *stream, mdp_tuning *out);
mdp_status mdp_tuning_load(const char *json_path);

/* ------------------------------------------------------------- batching --
 * Builds and solves n (1..1023) independent MDPs of uneven sizes: one
 * persistent build launch per group of MDPs with the same mode count and
 * action count class over a shared work queue, and per batched step (a
 * Jacobi sweep, or a time layer of the layered pass) and solve class one
 * small plan launch plus one Bellman launch that spreads every MDP's
 * recomputed slices evenly over the GPU; all captured in a CUDA graph that is
 * replayed on each call with the same shapes.  Arrays are host arrays of
 * per-MDP descriptors; V[i] / policy[i] are device outputs as in mdp_solve
 * (FP32 only).  Objective slot 0 of each MDP is solved to tol: tol > 0 by
 * (active-layer) Jacobi sweeps, tol = 0 by the layered pass (one batched step
 * per time layer, every model's layer nt - k at step k; the exact fixed
 * point, equal to Jacobi's bit for bit; sweeps_h reports 1 as mdp_solve's
 * layered method does).  V and policy equal mdp_build + mdp_solve of each
 * MDP alone. */
typedef struct {
  mdp_env env;
  mdp_grid grid;
  mdp_actions actions;
  int32_t N, subgrid_L;
  int32_t objective;
  void *V;
  int16_t *policy;
} mdp_batch_item;

typedef struct mdp_batch_t *mdp_batch;

mdp_status mdp_batch_create(const mdp_batch_item *items_h, int32_t n, double tol, mdp_batch *out);
mdp_status mdp_batch_run(mdp_batch b, void *stream, int32_t *sweeps_h, double *ms);
void mdp_batch_free(mdp_batch b);

/* -------------------------------------------------------------- serving --
 * Replanning server (on-board re-planning, Sec. V): environment fields stay
 * resident on the device; requests carry a new start/target, a coefficient
 * variance scale, a seed and N.  Requests are admitted in arrival order while
 * the HBM budget and free slots allow, run concurrently on per-slot streams
 * (continuous batching), and retire independently.
 * Memory: each request is charged, at admission, an upper bound of all the
 * device memory its build and solve can hold with an entry pool of a given
 * size, and its build never allocates a larger pool.  The size is the largest
 * the slices can need when the budget has room for it, else the widest the
 * environment's earlier requests needed; after the build the charge drops to
 * that of the compacted model.  A request whose slices need more columns is
 * charged again for the exact need and goes back to the head of the queue (or
 * ends with MDP_ERR_BUDGET if that exceeds the whole budget), so the requests
 * in flight never hold more than the budget.
 * Scheduling: a request runs on a stream whose priority follows its age among
 * the requests in flight (the oldest highest).  The oldest request uses the
 * fastest (persistent) kernels; a younger one whose work (states x N) is at
 * most a quarter of the oldest one's runs beside it with kernels that leave
 * the SMs all along their run, filling the gaps; a larger one waits until it
 * is the oldest.  Idle workers are woken most recently idle first. */
typedef struct mdp_server_t *mdp_server;

typedef struct {
  int32_t env_id;
  int32_t start_i, start_j;      /* reported entry of V / pi */
  int32_t target_i, target_j;    /* lower-left corner of the target block */
  int32_t target_w, target_h;    /* target block size in cells */
  double sigma_scale;            /* multiplies the registered sigma_h */
  uint64_t seed;
  int32_t N;
  int32_t objective;             /* mdp_objective */
  double tol;                    /* 0: the exact fixed point by one layered pass (the
                                    Jacobi fixed point bit for bit); > 0: Jacobi sweeps
                                    until the residual is <= tol */
  int32_t start_t;               /* time step of the start, 0..nt-1: the request replans the
                                    remaining horizon t = start_t..nt-1 on the resident
                                    fields with freshly drawn coefficients (on-board
                                    re-planning, Sec. V); its V / policy cover those
                                    nt - start_t layers (index (t - start_t)*nx*ny + c) */
  const float *V0_h;             /* host [|S|+1] or NULL: starting values of a Jacobi request
                                    (tol > 0; MDP_SOLVE_WARM), e.g. the V polled from an
                                    earlier request on the same env and start_t; NULL: start
                                    from 0; exact requests ignore it.  Must stay valid until
                                    the request completes */
} mdp_request;

typedef struct {
  int32_t status;                /* mdp_status of the request */
  float V_start;                 /* V at (t = 0, start) */
  int16_t pi_start;              /* policy at (t = 0, start) */
  int32_t sweeps;                /* Jacobi sweeps (1 for the layered pass) */
  double latency_ms;             /* submit -> completion (host clock) */
  double queue_ms;               /* submit -> admission */
  int64_t device_bytes;          /* device memory the request was charged (an upper bound of
                                    what it held) */
} mdp_result;

/* hbm_budget_bytes: device memory the server may hold for requests;
 * max_slots: concurrently running requests. */
mdp_status mdp_serve_create(size_t hbm_budget_bytes, int32_t max_slots, mdp_server *out);
/* Copies the environment's device arrays into server-owned device memory
 * (FP32 only); sigma_h is copied too; coeffs must be NULL. */
mdp_status mdp_env_register(mdp_server s, const mdp_env *env, const mdp_grid *grid,
                            const mdp_actions *actions, int32_t subgrid_L, int32_t *env_id);
mdp_status mdp_serve_submit(mdp_server s, const mdp_request *req, uint64_t *ticket);
/* Waits up to timeout_ms (0 = do not wait) for the ticket; MDP_ERR_PENDING if
 * not done.  Copies V and pi of the whole problem to V_h / pi_h when non-NULL
 * (host [|S|+1] float / [|S|] int16), then releases the request. */
mdp_status mdp_serve_poll(mdp_server s, uint64_t ticket, int32_t timeout_ms, mdp_result *out,
                          float *V_h, int16_t *pi_h);
mdp_status mdp_serve_stats(mdp_server s, int64_t *in_flight, int64_t *queued,
                           int64_t *bytes_in_use);
mdp_status mdp_serve_destroy(mdp_server s);

const char *mdp_last_error(void);
const char *mdp_version(void);

/* Failure injection for tests (the library's own test suite; not for
 * production use).  Every device-side wait of the Bellman sweeps is bounded:
 * after a limit of clock cycles it gives up, the kernel drains its copies in
 * flight, records the failure in the call's status word and returns, and the
 * call reports MDP_ERR_TIMEOUT with the device context still usable.
 *   MDP_TEST_WAIT_NEVER_COMPLETES: the next mdp_solve / mdp_solve_multi's first
 *     round of the one-state-per-slice sweep expects `value` bytes (a multiple
 *     of 16, <= 1 MiB) that are never copied, so that wait runs out (one shot);
 *   MDP_TEST_WAIT_LIMIT_CYCLES: the limit of those waits (0 = the default,
 *     about 2 s).
 * Returns MDP_ERR_ARG for other keys or values.  The paper has no counterpart. */
enum { MDP_TEST_WAIT_NEVER_COMPLETES = 1, MDP_TEST_WAIT_LIMIT_CYCLES = 2 };
mdp_status mdp_test_inject(int32_t what, int64_t value);

#ifdef __cplusplus
}
#endif
#endif /* MDP_GB300_H */
