// mdp_internal.cuh -- internal types and device helpers of libmdp_gb300.
//
// Model layout in HBM (sliced ELLPACK, one slice per 32 internal rows):
//   internal row   ir = s * A_pad + a          (A_pad = A rounded up to a power of two <= 32)
//   slice          sl = ir / 32 = s / spw      (spw = 32 / A_pad states per slice)
//   lane           l  = ir % 32 = (s % spw) * A_pad + a
//   entries        pool[(slice_off[sl] + k) * 32 + l], k < nnz[ir]: the in-domain
//                  successors in ascending order, one 32-bit word each (columns
//                  nnz[ir] .. slice_w[sl]-1 of a row hold 0 = padding):
//                  bits 0..15 signed offset o = s' - (s + Nc) = dj*Nx + di,
//                  bits 16..31 count (realizations landing there, <= N <= 65535)
//   sink           sinkc[ir] realizations end in the sink s' = |S| (V = 0)
//   R              R[o * rows_pad + ir]        (float or double), rows_pad = n_slices * 32
// Warps read a slice column (32 lanes x 4 B = 128 B) per k: fully coalesced.
// A slice's columns are contiguous; the build allocates them in completion
// order and its compaction moves them into slice order (pool_ordered), so
// that the columns of consecutive slices are one contiguous range.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mdp.h"

namespace mdpgb {

constexpr int kMaxActions = 32;
constexpr int kMaxModes = 16;
constexpr uint32_t kSinkBin = 0xFFFFu;
constexpr uint32_t kNoSlice = 0xFFFFFFFFu;

// cell class bits, [nt][ny][nx]
enum : uint8_t { CLS_FREE = 0, CLS_OBSTACLE = 1, CLS_TARGET = 2 };

// device status counters (unsigned long long each)
enum {
  CNT_POOL_COLS = 0,     // 32-entry columns handed out
  CNT_OVERFLOW = 1,      // (s,a) rows / samples that left the sub-grid
  CNT_ROW_CAP = 2,       // rows longer than row_cap
  CNT_POOL_FULL = 3,     // slices that did not fit the pool
  CNT_CAPPED = 4,        // polar pairs that hit the attempt cap
  CNT_WORK = 5,          // dynamic work-queue head
  CNT_SAMPLES = 6,       // landing evaluations performed
  CNT_NNZ = 7,           // stored entries (sink included)
  CNT_MAXROW = 8,        // widest row
  CNT_DEFER_N = 9,       // slices the warp kernel handed to the CTA kernel
  CNT_DEFER_WORK = 10,   // work-queue head of the CTA kernel over the deferred list
  CNT_DOMAIN = 11,       // stored in-domain successors (sink entries excluded)
  CNT_SPILL_WORDS = 12,  // spill words requested (headers included), stored or not
  CNT_SPILL_FULL = 13,   // slices whose spill block did not fit the spill area
  CNT_SPILL_ROWS = 14,   // rows with entries beyond row_cap
  CNT_MAXLEN = 15,       // longest row (in-domain successors + sink), spill included
  CNT_N = 16
};

// HYB spill.  A row keeps its first row_cap in-domain successors in the
// slice's ELL columns; the rest of the row (still in ascending order) goes to
// its slice's spill block at spill[spill_off[slice]]: kSpillHdr words
// start[0..32] (start[l] = first entry of row l of the slice relative to the
// block's entries, start[32] = the block's entry count), then the entry words
// (the ELL's 16-bit offset | 16-bit count).  Summing a row's ELL columns and
// then its spill entries is the same ascending-order sum as over one plain
// row.  Slices without a spill block hold kNoSlice in spill_off.
constexpr int kSpillHdr = 33;

constexpr int kRankBuckets = 128;

struct ActionTable {
  float dxl[kMaxActions];   // F cos(theta) * dt/dx   (FP32 kinematics, grid units)
  float dyl[kMaxActions];
  float F[kMaxActions];
  double dx64[kMaxActions];  // F cos(theta), F sin(theta), F in FP64 (check mode)
  double dy64[kMaxActions];
  double F64[kMaxActions];
  // FP32 landing offsets: floor(u + d) of the exact sum of the floats u and
  // d = floor(u) + c + [u - floor(u) >= th] with c = floor(d) and th the
  // smallest float >= 1 - (d - c) (2 when d is an integer: never reached).
  int32_t cx[kMaxActions], cy[kMaxActions];
  float thx[kMaxActions], thy[kMaxActions];
  // The distinct thresholds below 2, ascending, padded with 2 (Dx, Dy of
  // them), and each action's rank le = #{T <= th}: a sample's fractional
  // rank rho = #{T <= u - floor(u)} decides [u - floor(u) >= th] = [rho >= le]
  // for every action at once.
  float Tx[kMaxActions + 2], Ty[kMaxActions + 2];
  int32_t lex[kMaxActions], ley[kMaxActions];
  int32_t Dx, Dy;
  // Rank lookup over kRankBuckets equal buckets of [0, 1]: entry b =
  // #{T in buckets < b}, bucket(v) = min(floor(128 v), 127) (exact: 128 is a
  // power of two); Mx, My = most thresholds in one bucket.
  uint8_t Lx[kRankBuckets], Ly[kRankBuckets];
  int32_t Mx, My;
};

struct RewardParams {
  double c_f, c_r, r_term, r_out, dt, dx;
  int32_t n_obj;
  int32_t objs[3];
};

// Everything the build kernels need, passed by value.
struct BuildArgs {
  int32_t nx, ny, nt, K, N, A, A_pad, spw, L, h, nbins, row_cap;
  int64_t Nc, nS, n_slices, rows_pad;
  float lam;                 // dt / dx
  const void *vbar, *modes, *Y, *gbar;
  const uint8_t *cls;
  ActionTable act;
  RewardParams rw;
  uint32_t *pool;
  uint64_t pool_cap_cols;
  uint32_t *slice_off;
  uint8_t *slice_w;
  uint8_t *nnz;
  uint16_t *sinkc;
  void *R;
  unsigned long long *cnt;
  int32_t chunk;             // realizations per staged pass (FP32 CTA kernel)
  int64_t slice_begin, slice_end;  // work range [begin, end)
  int32_t cap_bins;          // fine-table words per warp of the warp kernel
  uint32_t *defer;           // slices deferred by the warp kernel ([n_slices])
  const uint32_t *defer_in;  // non-NULL: the CTA kernel works on this list (count CNT_DEFER_N)
  // HYB spill area (nullptr: none; rows beyond row_cap then only count their
  // need in CNT_SPILL_WORDS / CNT_SPILL_FULL)
  uint32_t *spill;
  uint32_t *spill_off;       // [n_slices] word offset of the slice's block, or kNoSlice
  uint64_t spill_cap_words;
  // single-model warp kernel: 0 = persistent warps (one CTA wave pulls every
  // slice); q > 0 = each warp builds at most q slices and the grid covers the
  // model, so CTAs retire all along the build and the block scheduler can
  // place higher-priority work (another request's launches) between them
  int32_t slices_per_warp;
};

struct mdp_model_impl;

}  // namespace mdpgb

struct mdp_model_t {
  int32_t nx, ny, nt, K, N, A, A_pad, spw, L, h, nbins, row_cap, precision, n_obj;
  int32_t objs[3];
  int64_t Nc, nS, n_slices, rows_pad;
  double dx, dt;
  mdpgb::RewardParams rw;
  // device memory owned by the model
  uint32_t *pool;
  uint64_t pool_cols;         // columns in use (after compaction: capacity == in use)
  uint32_t *slice_off;
  uint8_t *slice_w;           // [n_slices] columns per slice
  uint8_t *nnz;               // [rows_pad] in-domain entries per row
  uint16_t *sinkc;            // [rows_pad] realizations ending in the sink
  void *R;                    // [n_obj][rows_pad]
  uint8_t *cls;               // [nt][ny][nx]
  int32_t *delta;             // [nbins] (unused by the solver)
  void *Vtmp;                 // [nS+1] Jacobi ping-pong partner
  unsigned long long *cnt;    // [CNT_N]
  double *solve_stats_d;      // [4] device scalars for the solver
  int64_t device_bytes;
  int64_t nnz_total;
  int64_t nnz_domain;
  int32_t max_row_nnz;
  int64_t samples;
  double build_ms;
  double kernel_ms;
  int32_t launches;
  int64_t deferred;           // slices the full-window kernel built
  int device;
  int32_t pool_ordered;       // 1: the pool holds the slices in slice order, back to back
                              // (slice_off[sl + 1] = slice_off[sl] + slice_w[sl])
  int32_t sweep_smem_kb;      // shared memory of the one-state-per-slice Bellman sweep (0: default)
  // HYB spill (nullptr when no row is longer than row_cap)
  uint32_t *spill;            // [spill_words] per-slice blocks (kSpillHdr words + entries)
  uint32_t *spill_off;        // [n_slices] block offset or kNoSlice
  uint64_t spill_words;
  int64_t spill_rows;         // rows with entries beyond row_cap
  int64_t spill_entries;      // entries held in the spill blocks
  int32_t max_row_len;        // longest row (in-domain successors + sink)
  int32_t sweep_small_ctas;   // 1: sweeps use CTAs that share an SM with other work (the server)
};

namespace mdpgb {

// ---------------------------------------------------------------- errors --
void set_error(const std::string &msg);
mdp_status cuda_fail(cudaError_t e, const char *what);
#define MDP_CUDA_TRY(expr)                                    \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::mdpgb::cuda_fail(_e, #expr); \
  } while (0)

// ---------------------------------------------------------------- memory --
// Stream-ordered allocations from the device's default memory pool, kept
// cached by the pool between builds (release threshold raised at init).
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);
int ensure_device_init();
// MDP_OK when a CUDA device is usable (sets the error message otherwise)
mdp_status check_device();
// validated action table of `ac` (FP32 displacements scaled by lam = dt/dx)
mdp_status make_actions(const mdp_actions *ac, double lam, ActionTable *t, int *A_out);

// ----------------------------------------------------------- launches ----
// sampler (FP64 draw; FP32 copy is the FP64 value rounded)
cudaError_t launch_sample_coeffs(int nt, int N, int K, const double *sigma_d, uint64_t seed,
                                 uint64_t mdp_id, double *Y64, float *Y32,
                                 unsigned long long *capped, cudaStream_t st);
// build
// warp-per-slice kernel (fast path) followed by the CTA kernel over the
// slices it deferred (fine tables larger than cap_bins)
cudaError_t launch_build_fp32(const BuildArgs &a, int threads, int sms, cudaStream_t st);
cudaError_t launch_build_warp(const BuildArgs &a, int warps_per_cta, int sms, cudaStream_t st);
cudaError_t launch_build_fp64(const BuildArgs &a, cudaStream_t st);
// cell classes + sub-grid delta table
cudaError_t launch_prepare(const uint8_t *obstacle, const uint8_t *target, uint8_t *cls,
                           int nx, int ny, int nt, int32_t *delta, int L, cudaStream_t st);
// out[g*C + c] = max |x| over group g, component c of data laid out
// [outer][G][inner][C] (n elements); out holds float bit patterns, zeroed by the caller
cudaError_t launch_absmax(const void *x, int precision, int64_t n, int G, int64_t inner, int C,
                          unsigned int *out, cudaStream_t st);
// solve
struct SolveArgs {
  const uint32_t *pool;
  const uint32_t *slice_off;
  const uint8_t *slice_w;
  int32_t wcap;               // widest slice (columns)
  int *err;                   // device error word (bounded waits that expired)
  const uint8_t *nnz;
  const void *R;              // objective slot base
  const uint8_t *cls;
  const int32_t *delta;
  int64_t nS, Nc, n_slices;
  int32_t A, A_pad, spw, N, nbins;
  double tol;
  // Active-layer Jacobi (nullptr: every state every sweep).  lflags holds
  // three rotating arrays of nt + 1 layer flags: sweep k reads
  // lflags[(k-1)%3] (layers whose V changed in sweep k-1; entry nt, the
  // sink, stays 0), sets lflags[k%3] and clears lflags[(k+1)%3].
  uint8_t *lflags = nullptr;
  unsigned long long *work = nullptr;   // [max_sweeps] slices computed per sweep (or nullptr)
  int32_t nt = 0;
  int32_t pool_ordered = 0;   // the model's pool_ordered: a run of slices is one contiguous copy
  int32_t sweep_smem_kb = 0;  // shared memory of the one-state-per-slice sweep (0: its default)
  long long wait_cycles = 0;  // bounded waits give up after this many clock cycles (0: ~2 s)
  uint32_t test_extra_tx = 0; // failure injection (tests): bytes one wait expects that never arrive
  const uint32_t *spill = nullptr;      // HYB spill blocks (nullptr: the model has none)
  const uint32_t *spill_off = nullptr;  // [n_slices]
  int32_t small_ctas = 0;     // 1: the warp-per-slice sweep also for one state per slice
};
// Launch shapes chosen by the autotuner (mdp_autotune) per workload class;
// every choice gives the same model and values bit for bit.
struct Tuning {
  int32_t build_warps = 8;       // warps per CTA of the warp-per-slice build kernel
  int32_t hist_cap = 2048;       // fine-table words per warp of that kernel
  int32_t threads = 256;         // CTA size of the full-window build kernel
  int32_t chunk = 1024;          // realizations staged per pass by that kernel
  int32_t sweep_smem_kb = 160;   // shared memory of the one-state-per-slice Bellman sweep
};
// Workload class of a model: actions (padded), modes, N and cells (rounded
// to powers of two), objectives and precision.
std::string tuning_key(int A_pad, int K, int N, int64_t Nc, int n_obj, int precision);
// The tuned shapes of a class, if the autotuner recorded (or loaded) them.
bool tuning_lookup(const std::string &key, Tuning *out);

// Failure injection for tests, set on the host by mdp_test_inject: the next
// solve's first round expects this many bytes too many (one shot), and the
// bounded waits' limit in clock cycles (0: the default).
void take_test_injection(SolveArgs &a);
// batched solve (FP32): one Jacobi sweep over many models per launch
struct BatchSolveItem {
  SolveArgs a;                // the model (R of the objective being solved)
  float *Va, *Vb;             // V ping-pong (Va = the caller's output)
  int16_t *policy;
  unsigned long long *res;    // [max_sweeps] residual bits, zeroed per run
  double *stats;              // [4] sweeps, residual
  int max_sweeps;
};
struct BatchCta {
  int item;
  int64_t sl_lo, sl_hi;   // slices of the entry
  int64_t s_lo, s_hi;     // states it may write (layered: one layer)
};
// grouped: models with one state per slice whose width fits the grouped
// sweep (bellman_grouped_fits); else the warp-per-slice sweep
bool bellman_grouped_fits(int spw, int wcap);
cudaError_t prepare_bellman_batch(int wcap, int grouped, int *stage_bytes, int *per_sm);
// sweep k: a plan launch spreads the models' recomputed slices over G + n
// CTA entries (ctas_d), then the sweep launch; n <= 1023 models
// layered: step k (1..max nt) is the in-place pass over layer nt - k of
// every model (the exact fixed point of tol = 0, Jacobi's bit for bit)
cudaError_t launch_bellman_batch(const BatchSolveItem *items_d, int n, BatchCta *ctas_d, int G, int k,
                                 int stage_bytes, int grouped, int layered, cudaStream_t st);
cudaError_t launch_finalize_batch(const BatchSolveItem *items_d, int n, int layered, cudaStream_t st);
// batched build (FP32): one persistent warp launch over the slices of n
// models that share the mode count K and the states per warp spw (prefix[m]
// = first slice of model m in the launch, prefix[n] = total); then the
// full-window CTA kernel over every model's deferred slices
cudaError_t launch_build_warp_batch(const BuildArgs *items_d, const int64_t *prefix_d, int n,
                                    unsigned long long *work_d, int cap_bins, int K, int spw,
                                    cudaStream_t st);
cudaError_t launch_build_fp32_batch(const BuildArgs *items_d, int n, size_t smem, int threads,
                                    cudaStream_t st);
size_t fp32_smem_bytes(const BuildArgs &a, int threads);
// per-objective arrays of one solve over n <= 3 objectives sharing P
struct SolveIO {
  int n;
  const void *R[3];           // objective slot bases of R
  void *V[3];                 // the caller's outputs
  void *Vtmp[3];              // n = 1: the Jacobi partner of V[0]
  void *table[2];             // n > 1: packed value tables [|S|+1][n == 3 ? 4 : n]
                              // (Jacobi: both, layered: table[0]), zeroed by the caller
  int16_t *policy[3];
};
// stats_d: objective o's block at stats_d + o*(4 + max_sweeps); the error
// word (a.err) is set by the caller
cudaError_t launch_jacobi_multi(const SolveArgs &a, int precision, int max_sweeps, const SolveIO &io,
                                double *stats_d, cudaStream_t st);
cudaError_t launch_layered_multi(const SolveArgs &a, int precision, int nt, const SolveIO &io,
                                 double *stats_d, cudaStream_t st);
cudaError_t launch_jacobi(const SolveArgs &a, int precision, int max_sweeps, void *Va, void *Vb,
                          int16_t *policy, double *stats_d, cudaStream_t st);
// Copies the slices' entry columns from `pool` (any order) into `out` in
// slice order, back to back, and rewrites slice_off accordingly (a slice
// without columns gets the offset where the next one starts).  `out` holds
// the sum of slice_w columns.
cudaError_t launch_pool_reorder(const uint32_t *pool, uint32_t *out, uint32_t *slice_off, const uint8_t *slice_w,
                                int64_t n_slices, cudaStream_t st);
// export
cudaError_t launch_export(const mdp_model_t *m, int obj, int64_t *rowptr, int64_t *col,
                          int32_t *count, void *R, cudaStream_t st);

int num_sms();

// Raises a kernel's dynamic shared-memory limit to the device maximum, once per
// (kernel, device).  Launches then pass their own size; the limit is never
// lowered, so concurrent launches with different sizes cannot race on it.
cudaError_t allow_max_smem(const void *func);

// Hand-over of a prepared (not yet built) model to the batched build.
struct BuildHook {
  uint64_t pool_cols = 0;     // in: entry-pool capacity in columns (0 = default guess); out: used
  BuildArgs args;             // out: kernel arguments
  void *Yown = nullptr;       // out: coefficient table owned by the caller now
  double *sigma_d = nullptr;  // out: device sigma (owned by the caller now)
  uint32_t *defer = nullptr;  // out: deferred-slice list (owned by the caller now)
  int threads = 256;          // out: CTA size of the full-window kernel
};
// A caller that accounts device memory (the server) fixes the entry pool's
// size: the build then never allocates a larger pool, and if the slices need
// more columns it returns MDP_ERR_BUDGET with the exact need.
struct BuildLimits {
  uint64_t pool_cols = 0;          // in: pool columns to allocate (0: the build's own guess)
  uint64_t pool_cols_needed = 0;   // out (MDP_ERR_BUDGET): the columns the slices need
  uint64_t spill_words = 0;        // in (with pool_cols): spill words to allocate (0: none)
  uint64_t spill_words_needed = 0; // out (MDP_ERR_BUDGET): the spill words the rows need
  int32_t slices_per_warp = 0;     // in: BuildArgs::slices_per_warp of the warp kernel
};
mdp_status build_impl(const mdp_env *env, const mdp_grid *grid, const mdp_actions *actions, int32_t N,
                      int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj, const mdp_build_opts *opts,
                      void *stream, mdp_model *out, BuildHook *hook, BuildLimits *lim = nullptr);

// Frees a model's device memory in the order of `st` (no device-wide sync):
// for callers that know the model's work was issued on that stream.
void free_model_on_stream(mdp_model_t *m, cudaStream_t st);

}  // namespace mdpgb
