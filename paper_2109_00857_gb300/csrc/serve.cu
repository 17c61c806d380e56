// serve.cu -- the replanning server (on-board re-planning, Sec. V) of
// include/mdp.h.
//
// Registered environments are copied into server-owned device memory and stay
// resident.  A request names an environment and carries a new start and target,
// a scale for the coefficient standard deviations, a seed, N, an objective and
// a tolerance.  Requests wait in a FIFO queue; max_slots worker threads, each
// with its own CUDA stream, take the head of the queue as soon as a slot is
// free and the request's device-memory charge fits the HBM budget, then build
// and solve it: mdp_build over the remaining horizon t = start_t..nt-1, then
// mdp_solve -- the layered pass for an exact request (tol = 0), Jacobi sweeps
// to tol otherwise (from the request's starting values V0_h when given).
// Requests admitted while others run overlap with them on the GPU (continuous
// batching); each retires on its own, copies V and the policy to host memory
// and releases its device memory.
//
// Memory accounting is a hard bound: a request is charged, at admission, the
// most device memory its build and solve can hold with an entry pool of a
// given size (every array the calls allocate, as if all were live at once),
// and the build is held to that pool size.  The size is the largest the
// slices can need (every slice as wide as the row limit) when the budget has
// room for it -- the build then never stops for want of columns -- else the
// widest the environment's earlier requests needed; once the model is built
// and compacted, the charge drops to that of the columns in use.  If a
// request's slices need more columns than its pool, the build stops before
// allocating them and reports the exact need, and the request goes back to
// the head of the queue charged for that need.
//
// Scheduling: requests run on CUDA streams of graded priority by admission
// order -- the oldest request in flight on the highest priority -- so the GPU
// serves them close to first come, first served while later requests fill
// the gaps the earlier ones leave (host round trips, short launches).  The
// oldest request in flight runs the persistent kernels (a build and sweeps
// that occupy every SM); a younger request runs beside it only when its work
// (states x N) is at most kServeShareFraction of the oldest one's, with
// kernels that leave the SMs along their run (build warps that take
// kServeSlicesPerWarp slices each, sweeps of small CTAs); a larger one waits
// until it is the oldest, since two full-GPU builds would only slow the older
// one down.  Idle workers wait on their own condition variables and a new
// request wakes the most recently idle one, whose stream and buffers are warm.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "mdp_internal.cuh"

using namespace mdpgb;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct EnvEntry {
  mdp_grid grid;
  mdp_actions actions;
  std::vector<double> table;     // host action table (owned copy)
  std::vector<double> sigma;
  int K = 0, L = 0;
  void *vbar = nullptr, *modes = nullptr, *gbar = nullptr;
  uint8_t *obstacle = nullptr;
  double cols_per_slice = 16.0;   // pool columns per slice to charge the next request for
  bool cols_seen = false;         // a request has measured it
};

struct Job {
  uint64_t ticket = 0;
  mdp_request req{};
  Clock::time_point submitted, admitted, finished;
  int64_t bytes = 0;             // device memory charged now
  int64_t peak_bytes = 0;        // the largest charge it held (reported)
  uint64_t pool_cols = 0;        // entry-pool size the charge covers
  uint64_t spill_words = 0;      // spill-area size the charge covers (rows beyond the row cap)
  int level = 0;                 // stream priority level (0 = highest)
  double work = 0;               // realizations to count: states x N
  mdp_status status = MDP_ERR_PENDING;
  std::string error;
  int32_t sweeps = 0;
  float V_start = 0.f;
  int16_t pi_start = -1;
  std::vector<float> V;
  std::vector<int16_t> pi;
  bool done = false;
};

}  // namespace

struct mdp_server_t {
  int device = 0;
  size_t budget = 0;
  int slots = 1;
  std::mutex mu;
  std::condition_variable cv_done;
  // idle workers wait on their own condition variable; a request wakes the
  // most recently idle one (its streams and buffers are warm), so a request
  // alone on the server runs like the one-slot server, and no other worker
  // is woken for nothing
  std::vector<std::unique_ptr<std::condition_variable>> wcv;
  std::vector<int> idle;
  std::condition_variable cv_front;   // a request left the running list
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::unique_ptr<EnvEntry>> envs;
  std::vector<std::thread> workers;
  int64_t bytes_in_use = 0;
  int64_t in_flight = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  int prio_levels = 1, prio_greatest = 0;   // stream priorities: greatest = numerically lowest
  std::deque<std::shared_ptr<Job>> running; // admitted requests, in admission order
};

namespace {

// Geometry of a request's model: the remaining horizon's states and slices.
// (S->mu held) wakes the most recently idle worker, or every idle worker
void wake_one(mdp_server_t *S) {
  if (S->idle.empty()) return;
  const int j = S->idle.back();
  S->idle.pop_back();
  S->wcv[j]->notify_one();
}
void wake_all(mdp_server_t *S) {
  for (int j : S->idle) S->wcv[j]->notify_one();
  S->idle.clear();
}
// (S->mu held) the queue's head may start now
bool head_fits(const mdp_server_t *S) {
  return !S->queue.empty() && S->bytes_in_use + S->queue.front()->bytes <= (int64_t)S->budget;
}

struct ReqShape {
  int64_t nt, nS, n_slices, rows_pad, nbins;
};
ReqShape req_shape(const EnvEntry &e, const mdp_request &r) {
  ReqShape g;
  g.nt = e.grid.nt - r.start_t;
  g.nS = (int64_t)e.grid.nx * e.grid.ny * g.nt;
  int A = e.actions.n_headings * e.actions.n_speeds, A_pad = 1;
  while (A_pad < A) A_pad <<= 1;
  const int64_t spw = 32 / A_pad;
  g.n_slices = (g.nS + spw - 1) / spw;
  g.rows_pad = g.n_slices * 32;
  const int64_t L = e.L > 0 ? e.L : 255;   // automatic sub-grid: at most 255 cells a side
  g.nbins = L * L;
  return g;
}

// The most device memory a request can hold with an entry pool of pool_cols
// columns: every allocation of its build (coefficients, pool, slice and row
// arrays, R, cell classes, offsets, deferred-slice list, the compacted pool and
// its scan while the first pool is still live), its solve (status words, the
// Jacobi partner vector and layer flags) and the request's own V and policy,
// each rounded up to 4 KiB, plus 1 MiB; with spill_words > 0 also a spill area
// of that many words and its per-slice offsets.
int64_t charge_bytes(const EnvEntry &e, const mdp_request &r, uint64_t pool_cols, uint64_t spill_words) {
  const ReqShape g = req_shape(e, r);
  auto al = [](int64_t x) { return (x + 4095) & ~(int64_t)4095; };
  const int64_t max_sweeps = g.nt + 1;
  int64_t b = 0;
  b += al(8 * 16) + al(4 * g.nt * r.N * e.K) + al(8 * (e.K + 1)) + al(4 * (2 + 3 * e.K));   // counters, Y, sigma, extremes
  b += 2 * al((int64_t)pool_cols * 128);                                                      // pool + compacted pool
  b += al(8 * (g.n_slices + 2) + 8 * (g.n_slices / 1000 + 64));                              // reorder scan
  b += al(4 * g.n_slices) + al(g.n_slices) + al(g.rows_pad) + al(2 * g.rows_pad) + al(4 * g.rows_pad);
  b += al(g.nS) + al(4 * g.nbins) + al(4 * g.n_slices);                                        // classes, offsets, defer
  b += al(8 * (4 + 2 * max_sweeps + (3 * (g.nt + 1) + 7) / 8 + 1));                           // solve status
  b += 3 * al(4 * (g.nS + 1)) + al(2 * g.nS);                                                  // V, partner, policy
  b += al((int64_t)e.grid.nx * e.grid.ny);                                                     // target mask
  if (spill_words) b += al(4 * g.n_slices) + al(4 * (int64_t)spill_words);                     // spill area
  return b + (1 << 20);
}

uint64_t pool_guess(const EnvEntry &e, const mdp_request &r) {
  return (uint64_t)(e.cols_per_slice * (double)req_shape(e, r).n_slices) + 64;
}

// The largest pool the request's slices can need (every slice as wide as the
// row limit): charged when the budget has room, so the build never stops for
// want of columns; the charge drops to the compacted model once it is built.
uint64_t pool_worst(const EnvEntry &e, const mdp_request &r) {
  const ReqShape g = req_shape(e, r);
  return (uint64_t)g.n_slices * (uint64_t)std::min<int64_t>(64, g.nbins + 1) + 64;
}

__global__ void target_block_kernel(uint8_t *tgt, int nx, int ny, int i0, int j0, int w, int h) {
  const int n = nx * ny;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const int i = c % nx, j = c / nx;
    tgt[c] = (i >= i0 && i < i0 + w && j >= j0 && j < j0 + h) ? 1 : 0;
  }
}

// slices per build warp when requests share the GPU (BuildArgs::slices_per_warp)
constexpr int kServeSlicesPerWarp = 8;
// a younger request runs beside the oldest one only when its work is at most
// this fraction of the oldest one's
constexpr double kServeShareFraction = 0.25;

// Returns true when the request must be charged again for a larger pool or
// for a spill area (job.pool_cols / job.spill_words then hold the exact need;
// a request is first charged without a spill area, which only rows longer
// than the row cap -- wide, high-sigma fields -- need).
bool run_job(mdp_server_t *S, Job &job, cudaStream_t st, uint8_t *tgt) {
  const EnvEntry &e = *S->envs[job.req.env_id];
  const mdp_request &r = job.req;
  const int nx = e.grid.nx, ny = e.grid.ny;
  target_block_kernel<<<(nx * ny + 255) / 256, 256, 0, st>>>(tgt, nx, ny, r.target_i, r.target_j,
                                                             r.target_w, r.target_h);
  std::vector<double> sig(e.sigma);
  for (double &x : sig) x *= r.sigma_scale;
  // the remaining horizon t = start_t..nt-1: the resident fields from layer
  // start_t on (float data, layer-major), coefficients drawn afresh
  const size_t Nc = (size_t)nx * ny, t0 = (size_t)r.start_t;
  mdp_grid grid = e.grid;
  grid.nt = e.grid.nt - r.start_t;
  mdp_env env{};
  env.K = e.K;
  env.precision = MDP_FP32;
  env.vbar = static_cast<const float *>(e.vbar) + t0 * Nc * 2;
  env.modes = e.modes ? static_cast<const float *>(e.modes) + t0 * (size_t)e.K * Nc * 2 : nullptr;
  env.coeffs = nullptr;
  env.sigma_h = sig.data();
  env.seed = r.seed;
  env.mdp_id = 0;
  env.gbar = e.gbar ? static_cast<const float *>(e.gbar) + t0 * Nc : nullptr;
  env.obstacle = e.obstacle + t0 * Nc;
  env.target = tgt;
  const int32_t obj = r.objective;
  mdp_model m = nullptr;
  BuildLimits lim;
  lim.pool_cols = job.pool_cols;
  lim.spill_words = job.spill_words;
  // The oldest running request takes the fastest (persistent) kernels.  A
  // younger one runs beside it with kernels that leave the SMs all along
  // their run -- the build's warps take a few slices each and the sweeps use
  // small CTAs -- so the stream priorities (older first) decide whose blocks
  // run next: the younger request fills the SMs the older one leaves idle.
  // A request far larger than the oldest one in flight would only slow that
  // one down (each build needs the whole GPU): it waits until it is the
  // oldest and then takes the persistent kernels.
  {
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_front.wait(lk, [&] {
      return S->running.empty() || S->running.front().get() == &job ||
             job.work <= kServeShareFraction * S->running.front()->work;
    });
  }
  auto younger = [&] {
    std::lock_guard<std::mutex> lk(S->mu);
    return !S->running.empty() && S->running.front().get() != &job;
  };
  lim.slices_per_warp = younger() ? kServeSlicesPerWarp : 0;
  mdp_status s = build_impl(&env, &grid, &e.actions, r.N, e.L, &obj, 1, nullptr, st, &m, nullptr, &lim);
  if (s == MDP_ERR_BUDGET &&
      (lim.pool_cols_needed > job.pool_cols || lim.spill_words_needed > job.spill_words)) {
    job.pool_cols = std::max(job.pool_cols, lim.pool_cols_needed);
    job.spill_words = std::max(job.spill_words, lim.spill_words_needed);
    cudaStreamSynchronize(st);
    return true;
  }
  if (s != MDP_OK) {
    job.status = s;
    job.error = mdp_last_error();
    return false;
  }
  {   // the model is compacted: the request now holds at most the charge of a
      // pool of the columns in use (the rest of its charge goes back)
    std::lock_guard<std::mutex> lk(S->mu);
    const int64_t now = charge_bytes(e, job.req, std::max<uint64_t>(m->pool_cols, 1), m->spill ? job.spill_words : 0);
    if (now < job.bytes) {
      S->bytes_in_use -= job.bytes - now;
      job.bytes = now;
    }
    if (head_fits(S)) wake_one(S);
  }
  {   // the widest pool per slice this environment's requests have needed (with
      // 10 % to spare) prices the next ones: widths vary with sigma and N, and
      // a charge that is too small costs the request a second build
    std::lock_guard<std::mutex> lk(S->mu);
    double &c = S->envs[job.req.env_id]->cols_per_slice;
    const double need = 1.1 * (double)m->pool_cols / (double)m->n_slices;
    if (!S->envs[job.req.env_id]->cols_seen || need > c) c = std::max(2.0, need);
    S->envs[job.req.env_id]->cols_seen = true;
  }
  m->sweep_small_ctas = younger() ? 1 : 0;
  const int64_t nS = m->nS;
  float *V = nullptr;
  int16_t *pi = nullptr;
  cudaError_t ce = dev_alloc((void **)&V, sizeof(float) * (size_t)(nS + 1), st);
  if (ce == cudaSuccess) ce = dev_alloc((void **)&pi, sizeof(int16_t) * (size_t)nS, st);
  if (ce != cudaSuccess) {
    job.status = cuda_fail(ce, "serve allocation");
    job.error = mdp_last_error();
    dev_free(V, st);
    free_model_on_stream(m, st);
    return false;
  }
  mdp_solve_stats ss{};
  // the exact fixed point is reached by one backward pass over the layers
  // (the same values as Jacobi to tol = 0) with far fewer Bellman backups;
  // a Jacobi request may start from the caller's values (replanning warm)
  int32_t method = r.tol == 0.0 ? MDP_SOLVE_LAYERED : MDP_SOLVE_JACOBI;
  if (method == MDP_SOLVE_JACOBI && r.V0_h) {
    ce = cudaMemcpyAsync(V, r.V0_h, sizeof(float) * (size_t)(nS + 1), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
      job.status = cuda_fail(ce, "serve warm start");
      job.error = mdp_last_error();
      dev_free(V, st);
      dev_free(pi, st);
      free_model_on_stream(m, st);
      cudaStreamSynchronize(st);
      return false;
    }
    method |= MDP_SOLVE_WARM;
  }
  s = mdp_solve(m, 0, method, r.tol, 0, V, pi, st, &ss);
  if (s == MDP_OK) {
    job.V.resize((size_t)nS + 1);
    job.pi.resize((size_t)nS);
    ce = cudaMemcpyAsync(job.V.data(), V, sizeof(float) * (size_t)(nS + 1), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(job.pi.data(), pi, sizeof(int16_t) * (size_t)nS, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
      s = cuda_fail(ce, "serve copy-out");
    } else {
      const int64_t s0 = (int64_t)r.start_j * nx + r.start_i;
      job.V_start = job.V[(size_t)s0];
      job.pi_start = job.pi[(size_t)s0];
      job.sweeps = ss.sweeps;
    }
  }
  job.status = s;
  if (s != MDP_OK) job.error = mdp_last_error();
  dev_free(V, st);
  dev_free(pi, st);
  // the model's memory goes back on this stream, without a device-wide sync
  // that would wait for the other slots' work
  free_model_on_stream(m, st);
  cudaStreamSynchronize(st);
  return false;
}

void worker_main(mdp_server_t *S, int id) {
  cudaSetDevice(S->device);
  // one stream per priority level; a request runs on the level it got at admission
  std::vector<cudaStream_t> streams(S->prio_levels);
  for (int l = 0; l < S->prio_levels; ++l)
    cudaStreamCreateWithPriority(&streams[l], cudaStreamNonBlocking, S->prio_greatest + l);
  size_t maxc = 0;
  uint8_t *tgt = nullptr;
  cudaStream_t tst = streams[0];   // the stream the target buffer was last used on
  for (;;) {
    std::shared_ptr<Job> job;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // FIFO admission: the head waits until its charge fits the budget
      while (!S->stopping && !head_fits(S)) {
        S->idle.push_back(id);
        S->wcv[id]->wait(lk);
        auto it = std::find(S->idle.begin(), S->idle.end(), id);   // a spurious wake-up
        if (it != S->idle.end()) S->idle.erase(it);
      }
      if (S->stopping) break;
      job = S->queue.front();
      S->queue.pop_front();
      S->bytes_in_use += job->bytes;
      S->in_flight += 1;
      job->admitted = Clock::now();
      // priority by age: behind the requests still running
      job->level = std::min<int>((int)S->running.size(), S->prio_levels - 1);
      S->running.push_back(job);
      if (head_fits(S)) wake_one(S);   // the next request may start beside this one
    }
    cudaStream_t st = streams[job->level];
    const EnvEntry &e = *S->envs[job->req.env_id];
    const size_t cells = (size_t)e.grid.nx * e.grid.ny;
    if (st != tst) {   // the target buffer's last use is ordered before this request's
      cudaStreamSynchronize(tst);
      tst = st;
    }
    if (cells > maxc) {
      dev_free(tgt, st);
      tgt = nullptr;
      if (dev_alloc((void **)&tgt, cells, st) == cudaSuccess) maxc = cells;
    }
    bool again = false;
    if (!tgt) {
      job->status = MDP_ERR_OOM;
      job->error = "target mask allocation failed";
    } else {
      again = run_job(S, *job, st, tgt);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->bytes_in_use -= job->bytes;
      S->in_flight -= 1;
      for (auto it = S->running.begin(); it != S->running.end(); ++it)
        if (*it == job) {
          S->running.erase(it);
          break;
        }
      S->cv_front.notify_all();
      if (again) {
        const double cps = (double)job->pool_cols / (double)req_shape(e, job->req).n_slices;
        S->envs[job->req.env_id]->cols_per_slice = std::max(S->envs[job->req.env_id]->cols_per_slice, 1.1 * cps);
        // the slices need a larger pool: charge the exact need and put the
        // request back at the head of the queue (or refuse it if the whole
        // budget is too small)
        job->bytes = charge_bytes(e, job->req, job->pool_cols, job->spill_words);
        job->peak_bytes = std::max(job->peak_bytes, job->bytes);
        if (job->bytes > (int64_t)S->budget) {
          job->status = MDP_ERR_BUDGET;
          job->error = "request needs more device memory than the whole HBM budget";
          again = false;
        } else if (S->stopping) {
          job->status = MDP_ERR_CANCELLED;
          job->error = "server destroyed before the request was admitted";
          again = false;
        } else {
          S->queue.push_front(job);
        }
      }
      if (!again) {
        job->finished = Clock::now();
        job->done = true;
      }
    }
    S->cv_done.notify_all();   // this worker itself takes the next request, if any
  }
  dev_free(tgt, tst);
  for (cudaStream_t x : streams) {
    cudaStreamSynchronize(x);
    cudaStreamDestroy(x);
  }
}

}  // namespace

extern "C" mdp_status mdp_serve_create(size_t hbm_budget_bytes, int32_t max_slots, mdp_server *out) {
  if (!out) {
    set_error("invalid argument: out is NULL");
    return MDP_ERR_ARG;
  }
  *out = nullptr;
  if (max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) {
    set_error("invalid argument: need 1 <= max_slots <= 64 and a nonzero budget");
    return MDP_ERR_ARG;
  }
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    set_error("no usable CUDA device (this library has no CPU fallback)");
    return MDP_ERR_CUDA;
  }
  ensure_device_init();
  auto *S = new mdp_server_t();
  cudaGetDevice(&S->device);
  S->budget = hbm_budget_bytes;
  S->slots = max_slots;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess && least > greatest) {
    S->prio_greatest = greatest;
    S->prio_levels = std::min(least - greatest + 1, max_slots);
  }
  for (int i = 0; i < max_slots; ++i) S->wcv.emplace_back(new std::condition_variable());
  for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(worker_main, S, i);
  *out = S;
  return MDP_OK;
}

extern "C" mdp_status mdp_env_register(mdp_server S, const mdp_env *env, const mdp_grid *grid,
                                       const mdp_actions *actions, int32_t subgrid_L, int32_t *env_id) {
  if (!S || !env || !grid || !actions || !env_id) {
    set_error("invalid argument: NULL server/env/grid/actions/env_id");
    return MDP_ERR_ARG;
  }
  if (env->precision != MDP_FP32 || env->coeffs) {
    set_error("invalid argument: the server takes FP32 fields and draws its own coefficients");
    return MDP_ERR_ARG;
  }
  if (env->K < 0 || env->K > kMaxModes || (env->K > 0 && (!env->sigma_h || !env->modes)) || !env->vbar ||
      !env->obstacle || grid->nx < 1 || grid->ny < 1 || grid->nt < 1) {
    set_error("invalid argument: incomplete environment");
    return MDP_ERR_ARG;
  }
  const int A = actions->n_headings * actions->n_speeds;
  if (A < 1 || A > kMaxActions) {
    set_error("invalid argument: n_headings * n_speeds must be in [1, 32]");
    return MDP_ERR_ARG;
  }
  auto e = std::make_unique<EnvEntry>();
  e->grid = *grid;
  e->actions = *actions;
  if (actions->table_h) {
    e->table.assign(actions->table_h, actions->table_h + 3 * A);
    e->actions.table_h = e->table.data();
  }
  e->K = env->K;
  e->L = subgrid_L;
  if (env->K > 0) e->sigma.assign(env->sigma_h, env->sigma_h + env->K);
  const size_t cells = (size_t)grid->nx * grid->ny, n = cells * grid->nt;
  cudaSetDevice(S->device);
  cudaError_t ce = cudaMalloc(&e->vbar, 8 * n);
  if (ce == cudaSuccess) ce = cudaMemcpy(e->vbar, env->vbar, 8 * n, cudaMemcpyDeviceToDevice);
  if (ce == cudaSuccess && env->K > 0) ce = cudaMalloc(&e->modes, 8 * n * env->K);
  if (ce == cudaSuccess && env->K > 0)
    ce = cudaMemcpy(e->modes, env->modes, 8 * n * env->K, cudaMemcpyDeviceToDevice);
  if (ce == cudaSuccess && env->gbar) ce = cudaMalloc(&e->gbar, 4 * n);
  if (ce == cudaSuccess && env->gbar) ce = cudaMemcpy(e->gbar, env->gbar, 4 * n, cudaMemcpyDeviceToDevice);
  if (ce == cudaSuccess) ce = cudaMalloc((void **)&e->obstacle, n);
  if (ce == cudaSuccess) ce = cudaMemcpy(e->obstacle, env->obstacle, n, cudaMemcpyDeviceToDevice);
  if (ce != cudaSuccess) {
    cudaFree(e->vbar);
    cudaFree(e->modes);
    cudaFree(e->gbar);
    cudaFree(e->obstacle);
    return cuda_fail(ce, "mdp_env_register");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  *env_id = (int32_t)S->envs.size();
  S->envs.push_back(std::move(e));
  return MDP_OK;
}

extern "C" mdp_status mdp_serve_submit(mdp_server S, const mdp_request *req, uint64_t *ticket) {
  if (!S || !req || !ticket) {
    set_error("invalid argument: NULL server/request/ticket");
    return MDP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stopping) {
    set_error("server is shutting down");
    return MDP_ERR_CANCELLED;
  }
  if (req->env_id < 0 || req->env_id >= (int32_t)S->envs.size()) {
    set_error("unknown env_id");
    return MDP_ERR_NOT_FOUND;
  }
  const EnvEntry &e = *S->envs[req->env_id];
  const mdp_grid &g = e.grid;
  if (req->N < 1 || req->N > 65535 || req->objective < 0 || req->objective > 2 ||
      (req->objective == MDP_OBJ_NET_ENERGY && !e.gbar) || !(req->sigma_scale >= 0) ||
      req->start_i < 0 || req->start_i >= g.nx || req->start_j < 0 || req->start_j >= g.ny ||
      req->target_w < 1 || req->target_h < 1 || req->start_t < 0 || req->start_t >= g.nt) {
    set_error("invalid argument: bad request fields");
    return MDP_ERR_ARG;
  }
  auto job = std::make_shared<Job>();
  job->req = *req;
  job->work = (double)req_shape(e, *req).nS * (double)req->N;
  job->pool_cols = pool_worst(e, *req);
  job->bytes = charge_bytes(e, *req, job->pool_cols, 0);
  if (job->bytes > (int64_t)S->budget) {   // too much for the budget: the widths seen so far
    job->pool_cols = pool_guess(e, *req);
    job->bytes = charge_bytes(e, *req, job->pool_cols, 0);
  }
  job->peak_bytes = job->bytes;
  if (job->bytes > (int64_t)S->budget) {
    set_error("request needs more device memory than the whole HBM budget");
    return MDP_ERR_BUDGET;
  }
  job->ticket = S->next_ticket++;
  job->submitted = Clock::now();
  S->jobs[job->ticket] = job;
  S->queue.push_back(job);
  *ticket = job->ticket;
  if (head_fits(S)) wake_one(S);
  return MDP_OK;
}

extern "C" mdp_status mdp_serve_poll(mdp_server S, uint64_t ticket, int32_t timeout_ms, mdp_result *out,
                                     float *V_h, int16_t *pi_h) {
  if (!S || !out) {
    set_error("invalid argument: NULL server/result");
    return MDP_ERR_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) {
    set_error("unknown ticket");
    return MDP_ERR_NOT_FOUND;
  }
  std::shared_ptr<Job> job = it->second;
  if (!job->done && timeout_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return job->done; });
  if (!job->done) return MDP_ERR_PENDING;
  memset(out, 0, sizeof(*out));
  out->status = job->status;
  out->V_start = job->V_start;
  out->pi_start = job->pi_start;
  out->sweeps = job->sweeps;
  out->latency_ms = ms_between(job->submitted, job->finished);
  out->queue_ms = ms_between(job->submitted, job->admitted);
  out->device_bytes = job->peak_bytes;
  if (job->status == MDP_OK) {
    if (V_h) memcpy(V_h, job->V.data(), sizeof(float) * job->V.size());
    if (pi_h) memcpy(pi_h, job->pi.data(), sizeof(int16_t) * job->pi.size());
  } else {
    set_error(job->error);
  }
  S->jobs.erase(it);   // released
  return MDP_OK;
}

extern "C" mdp_status mdp_serve_stats(mdp_server S, int64_t *in_flight, int64_t *queued,
                                      int64_t *bytes_in_use) {
  if (!S) {
    set_error("invalid argument: NULL server");
    return MDP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (in_flight) *in_flight = S->in_flight;
  if (queued) *queued = (int64_t)S->queue.size();
  if (bytes_in_use) *bytes_in_use = S->bytes_in_use;
  return MDP_OK;
}

extern "C" mdp_status mdp_serve_destroy(mdp_server S) {
  if (!S) return MDP_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    for (auto &j : S->queue) {   // queued requests are cancelled; running ones finish
      j->status = MDP_ERR_CANCELLED;
      j->error = "server destroyed before the request was admitted";
      j->done = true;
    }
    S->queue.clear();
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    wake_all(S);
  }
  S->cv_done.notify_all();
  for (auto &t : S->workers) t.join();
  cudaSetDevice(S->device);
  for (auto &e : S->envs) {
    cudaFree(e->vbar);
    cudaFree(e->modes);
    cudaFree(e->gbar);
    cudaFree(e->obstacle);
  }
  delete S;
  return MDP_OK;
}

