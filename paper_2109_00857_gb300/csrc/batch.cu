// batch.cu -- many independent MDPs of uneven sizes built and solved together
// (mdp_batch_* of include/mdp.h).
//
// Create: every item is first built once on its own to calibrate it (the
// autotuner): the sub-grid side (given or sized from the field extremes), the
// entry-pool columns it needs, its widest slice, and how many slices overflow
// the warp kernel's histogram; from these the batch picks the per-lane
// histogram capacity, sizes each item's pool exactly (plus a margin), and
// sizes the Bellman stages for the widest slice.  Then each item is set up
// through the same path as mdp_build (allocations, coefficient table, cell
// classes) without launching its build.
// Run: one persistent warp-per-slice launch per (states per warp, mode
// count) group builds its items' slices from one work queue; one CTA launch
// finishes the slices any item deferred;
// the solve runs batched steps -- with tol = 0 the layered pass (step k
// updates layer nt - k of every item that has it, in place: the exact fixed
// point), with tol > 0 Jacobi sweeps (the layers whose inputs changed in the
// previous sweep; an item stops on its own residual) -- each step, per solve
// class (grouped sweep or warp per slice), a one-block plan launch that cuts
// the items' slices into chunks of equal size and one launch whose CTAs take
// one chunk each; one launch finalizes all.  The whole sequence (with the per-item coefficient draws,
// cell classes, clears and the status copies) is captured once into a CUDA
// graph and replayed on every run.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "mdp_internal.cuh"

using namespace mdpgb;

namespace {

struct Item {
  mdp_batch_item desc;
  std::vector<double> sigma, table;
  mdp_model_t *m = nullptr;
  BuildHook hook;
  float *Vb = nullptr;
  uint8_t *lflags = nullptr;   // active-layer sweep flags, 3 x (nt + 1)
  unsigned long long *res = nullptr;
  double *stats = nullptr;
  int max_sweeps = 0;
  int L = 0;
  int64_t pool_cols = 0;
  int width = 1;       // widest slice (columns), from the calibration build
  int solve_cls = 0;   // 1: grouped sweep
};

}  // namespace

struct mdp_batch_t {
  int n = 0, device = 0;
  double tol = 0;
  std::vector<Item> items;
  BuildArgs *items_d = nullptr;
  int64_t *prefix_d = nullptr;
  unsigned long long *work_d = nullptr;
  BatchSolveItem *sitems_d = nullptr;   // [n]: the warp-per-slice class first, then the grouped class
  int cap_bins = 2048, kmax = 0, max_sweeps_all = 0, max_nt = 0, cta_threads = 256;
  // tol = 0: the exact fixed point by one layered pass per model (Jacobi's
  // result bit for bit, one step per time layer); tol > 0: Jacobi sweeps
  bool layered = false;
  // solve classes: 0 = warp-per-slice sweep, 1 = grouped sweep (one state
  // per slice, narrow enough); each with its own plan entries
  struct SolveClass {
    int first = 0, n = 0, wcap = 1, stage_bytes = 0, n_ctas = 0;
    BatchCta *ctas_d = nullptr;
  };
  SolveClass cls[2];
  // build launches: items grouped by (states per warp, mode count), each
  // group one persistent launch over its own zero-based prefix segment
  struct Group {
    int start, n, pstart, K, spw;
  };
  std::vector<Group> groups;
  size_t cta_smem = 0;
  cudaStream_t st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long *cnt_h = nullptr;
  double *stats_h = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

void batch_release(mdp_batch_t *b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (Item &it : b->items) {
    if (it.m) free_model_on_stream(it.m, b->st);
    dev_free(it.hook.Yown, b->st);
    dev_free(it.hook.sigma_d, b->st);
    dev_free(it.hook.defer, b->st);
    dev_free(it.Vb, b->st);
    dev_free(it.lflags, b->st);
    dev_free(it.res, b->st);
    dev_free(it.stats, b->st);
  }
  dev_free(b->items_d, b->st);
  dev_free(b->prefix_d, b->st);
  dev_free(b->work_d, b->st);
  dev_free(b->sitems_d, b->st);
  for (auto &c : b->cls) dev_free(c.ctas_d, b->st);
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->cnt_h) cudaFreeHost(b->cnt_h);
  if (b->stats_h) cudaFreeHost(b->stats_h);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

// Every stream operation of one run, in order (captured into the graph).
cudaError_t enqueue(mdp_batch_t *b) {
  cudaStream_t st = b->st;
  cudaError_t e = cudaMemsetAsync(b->work_d, 0, sizeof(unsigned long long) * b->groups.size(), st);
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    Item &it = b->items[i];
    const mdp_env &env = it.desc.env;
    const mdp_grid &g = it.desc.grid;
    e = cudaMemsetAsync(it.m->cnt, 0, sizeof(unsigned long long) * CNT_N, st);
    if (e == cudaSuccess && it.hook.Yown)
      e = launch_sample_coeffs(g.nt, it.desc.N, env.K, it.hook.sigma_d, env.seed, env.mdp_id, nullptr,
                               (float *)it.hook.Yown, it.m->cnt + CNT_CAPPED, st);
    if (e == cudaSuccess)
      e = launch_prepare(env.obstacle, env.target, it.m->cls, g.nx, g.ny, g.nt, it.m->delta, it.L, st);
  }
  for (size_t g = 0; g < b->groups.size() && e == cudaSuccess; ++g) {
    const auto &G = b->groups[g];
    e = launch_build_warp_batch(b->items_d + G.start, b->prefix_d + G.pstart, G.n, b->work_d + g, b->cap_bins,
                                G.K, G.spw, st);
  }
  if (e == cudaSuccess) e = launch_build_fp32_batch(b->items_d, b->n, b->cta_smem, b->cta_threads, st);
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    Item &it = b->items[i];
    const size_t vbytes = sizeof(float) * (size_t)(it.m->nS + 1);
    e = cudaMemsetAsync(it.res, 0, sizeof(unsigned long long) * (size_t)it.max_sweeps, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(it.stats, 0, sizeof(double) * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(it.desc.V, 0, vbytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(it.Vb, 0, vbytes, st);
    // sweep 1 recomputes every layer (flags [0][0..nt) = 1, the rest 0)
    const int nt = it.m->nt;
    if (e == cudaSuccess) e = cudaMemsetAsync(it.lflags, 1, (size_t)nt, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(it.lflags + nt, 0, 2 * (size_t)nt + 3, st);
  }
  const int steps = b->layered ? b->max_nt : b->max_sweeps_all;
  for (int k = 1; k <= steps && e == cudaSuccess; ++k) {
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
      const auto &C = b->cls[c];
      if (C.n > 0)
        e = launch_bellman_batch(b->sitems_d + C.first, C.n, C.ctas_d, C.n_ctas, k, C.stage_bytes, c,
                                 b->layered ? 1 : 0, st);
    }
  }
  if (e == cudaSuccess) e = launch_finalize_batch(b->sitems_d, b->n, b->layered ? 1 : 0, st);
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    Item &it = b->items[i];
    e = cudaMemcpyAsync(b->cnt_h + (size_t)i * CNT_N, it.m->cnt, sizeof(unsigned long long) * CNT_N,
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->stats_h + (size_t)i * 4, it.stats, sizeof(double) * 4, cudaMemcpyDeviceToHost, st);
  }
  return e;
}

}  // namespace

extern "C" mdp_status mdp_batch_create(const mdp_batch_item *items_h, int32_t n, double tol, mdp_batch *out) {
  if (!out) {
    set_error("invalid argument: out is NULL");
    return MDP_ERR_ARG;
  }
  *out = nullptr;
  if (!items_h || n < 1 || n > 1023) {
    set_error("invalid argument: need 1 <= n <= 1023 items");
    return MDP_ERR_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    set_error("no usable CUDA device (this library has no CPU fallback)");
    return MDP_ERR_CUDA;
  }
  ensure_device_init();
  mdp_batch_t *b = new mdp_batch_t();
  cudaGetDevice(&b->device);
  b->n = n;
  b->tol = tol;
  b->layered = (tol == 0.0);
  cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  auto fail = [&](mdp_status code) {
    batch_release(b);
    return code;
  };
  b->items.resize(n);
  // ---- calibration (autotuner): one plain build per item
  int64_t total_slices = 0, wide = 0;
  for (int i = 0; i < n; ++i) {
    Item &it = b->items[i];
    it.desc = items_h[i];
    if (it.desc.env.precision != MDP_FP32 || !it.desc.V || !it.desc.policy) {
      set_error("invalid argument: batch items are FP32 and need V and policy outputs (item " +
                std::to_string(i) + ")");
      return fail(MDP_ERR_ARG);
    }
    const int A = it.desc.actions.n_headings * it.desc.actions.n_speeds;
    if (it.desc.actions.table_h && A > 0) {
      it.table.assign(it.desc.actions.table_h, it.desc.actions.table_h + 3 * A);
      it.desc.actions.table_h = it.table.data();
    }
    if (it.desc.env.sigma_h && it.desc.env.K > 0) {
      it.sigma.assign(it.desc.env.sigma_h, it.desc.env.sigma_h + it.desc.env.K);
      it.desc.env.sigma_h = it.sigma.data();
    }
    mdp_model cm = nullptr;
    mdp_build_opts o{};
    o.hist_cap = 2048;
    const int32_t obj = it.desc.objective;
    mdp_status s = mdp_build(&it.desc.env, &it.desc.grid, &it.desc.actions, it.desc.N, it.desc.subgrid_L,
                             &obj, 1, &o, b->st, &cm);
    if (s != MDP_OK) {
      set_error("batch item " + std::to_string(i) + ": " + mdp_last_error());
      return fail(s);
    }
    if (cm->spill_words) {   // the batched build and sweeps keep rows in the ELL columns only
      free_model_on_stream(cm, b->st);
      set_error("batch item " + std::to_string(i) + ": a row has more than the row cap's successors "
                "(batched models keep no spill area; build it with mdp_build)");
      return fail(MDP_ERR_ELL_OVERFLOW);
    }
    it.L = cm->L;
    it.pool_cols = (int64_t)cm->pool_cols;
    it.width = std::max(1, cm->max_row_nnz);
    it.solve_cls = bellman_grouped_fits(cm->spw, it.width) ? 1 : 0;
    wide += cm->deferred;
    total_slices += cm->n_slices;
    b->kmax = std::max(b->kmax, it.desc.env.K);
    free_model_on_stream(cm, b->st);
  }
  cudaStreamSynchronize(b->st);
  // the fine-table capacity the autotuner chose for the members' classes (the
  // largest), else larger tables when more than 0.2% of the slices would be deferred
  int tuned_cap = 0;
  for (int i = 0; i < n; ++i) {
    const Item &it = b->items[i];
    const int A = it.desc.actions.n_headings * it.desc.actions.n_speeds;
    int A_pad = 1;
    while (A_pad < A) A_pad <<= 1;
    Tuning t;
    if (tuning_lookup(tuning_key(A_pad, it.desc.env.K, it.desc.N, (int64_t)it.desc.grid.nx * it.desc.grid.ny, 1,
                                 MDP_FP32), &t))
      tuned_cap = std::max(tuned_cap, t.hist_cap);
  }
  b->cap_bins = tuned_cap > 0 ? tuned_cap : ((wide * 500 > total_slices) ? 4096 : 2048);
  // ---- set-up of every item through the build path, without launching it
  std::vector<BuildArgs> args(n);
  std::vector<int64_t> prefix(n + 1, 0);
  std::vector<BatchSolveItem> sitems(n);

  // solve classes: the warp-per-slice items first, then the grouped ones
  // (the same item order within each), each with its own widest slice
  std::vector<int> slot(n);
  for (int c = 0, pos = 0; c < 2; ++c) {
    auto &C = b->cls[c];
    C.first = pos;
    for (int i = 0; i < n; ++i) {
      if (b->items[i].solve_cls != c) continue;
      slot[i] = pos++;
      C.wcap = std::max(C.wcap, b->items[i].width);
    }
    C.n = pos - C.first;
  }
  cudaError_t ce = cudaSuccess;
  for (int c = 0; c < 2; ++c) {
    auto &C = b->cls[c];
    if (C.n == 0) continue;
    int per_sm = 1;
    ce = prepare_bellman_batch(C.wcap, c, &C.stage_bytes, &per_sm);
    if (ce != cudaSuccess) return fail(cuda_fail(ce, "prepare_bellman_batch"));
    // two waves of CTAs share each sweep's recomputed slices (plus one entry
    // per model for the chunk remainders)
    C.n_ctas = num_sms() * std::max(per_sm, 1) * 2;
  }
  for (int i = 0; i < n; ++i) {
    Item &it = b->items[i];
    mdp_build_opts o{};
    o.hist_cap = b->cap_bins;
    it.hook.pool_cols = (uint64_t)(it.pool_cols + std::max<int64_t>(1024, it.pool_cols / 50));
    const int32_t obj = it.desc.objective;
    mdp_model m = nullptr;
    mdp_status s = build_impl(&it.desc.env, &it.desc.grid, &it.desc.actions, it.desc.N, it.L, &obj, 1, &o,
                              b->st, &m, &it.hook);
    if (s != MDP_OK) {
      set_error("batch item " + std::to_string(i) + ": " + mdp_last_error());
      return fail(s);
    }
    it.m = m;
    it.max_sweeps = m->nt + 1;
    b->max_sweeps_all = std::max(b->max_sweeps_all, it.max_sweeps);
    b->max_nt = std::max(b->max_nt, m->nt);
    b->cta_threads = it.hook.threads;
    const size_t vbytes = sizeof(float) * (size_t)(m->nS + 1);
    ce = dev_alloc((void **)&it.Vb, vbytes, b->st);
    if (ce == cudaSuccess) ce = dev_alloc((void **)&it.lflags, 3 * ((size_t)m->nt + 1), b->st);
    if (ce == cudaSuccess) ce = dev_alloc((void **)&it.res, sizeof(unsigned long long) * it.max_sweeps, b->st);
    if (ce == cudaSuccess) ce = dev_alloc((void **)&it.stats, sizeof(double) * 4, b->st);
    if (ce != cudaSuccess) return fail(cuda_fail(ce, "batch allocation"));
    args[i] = it.hook.args;
    args[i].defer_in = it.hook.defer;
    b->cta_smem = std::max(b->cta_smem, fp32_smem_bytes(args[i], b->cta_threads));
    prefix[i + 1] = prefix[i] + m->n_slices;
    BatchSolveItem &si = sitems[slot[i]];
    memset(&si, 0, sizeof(si));
    si.a.pool = m->pool; si.a.slice_off = m->slice_off; si.a.slice_w = m->slice_w; si.a.nnz = m->nnz;
    si.a.wcap = b->cls[it.solve_cls].wcap;
    si.a.err = reinterpret_cast<int *>(it.stats + 2);
    si.a.R = m->R; si.a.cls = m->cls; si.a.delta = m->delta;
    si.a.nS = m->nS; si.a.Nc = m->Nc; si.a.n_slices = m->n_slices;
    si.a.A = m->A; si.a.A_pad = m->A_pad; si.a.spw = m->spw; si.a.N = m->N; si.a.nbins = m->nbins;
    si.a.tol = tol;
    si.a.nt = m->nt;
    si.a.lflags = b->layered ? nullptr : it.lflags;
    si.a.work = nullptr;
    si.Va = static_cast<float *>(it.desc.V);
    si.Vb = it.Vb;
    si.policy = it.desc.policy;
    si.res = it.res;
    si.stats = it.stats;
    si.max_sweeps = it.max_sweeps;
  }
  // group the build items by (states per warp, mode count); prefix segments per group
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  auto cls = [&](int i) {
    const int sc = args[i].spw == 1 ? 0 : (args[i].spw == 2 ? 1 : 2);
    return sc * 64 + std::min<int>(args[i].K, 63);
  };
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cls(x) < cls(y); });
  std::vector<BuildArgs> sorted(n);
  std::vector<int64_t> gprefix;
  for (int j = 0; j < n;) {
    int e = j;
    while (e < n && cls(ord[e]) == cls(ord[j])) ++e;
    mdp_batch_t::Group G{j, e - j, (int)gprefix.size(), args[ord[j]].K, args[ord[j]].spw};
    if (G.spw != 1 && G.spw != 2) G.spw = 0;
    int64_t acc = 0;
    gprefix.push_back(0);
    for (int q = j; q < e; ++q) {
      sorted[q] = args[ord[q]];
      acc += args[ord[q]].n_slices;
      gprefix.push_back(acc);
    }
    b->groups.push_back(G);
    j = e;
  }
  (void)prefix;
  ce = dev_alloc((void **)&b->items_d, sizeof(BuildArgs) * n, b->st);
  if (ce == cudaSuccess) ce = dev_alloc((void **)&b->prefix_d, sizeof(int64_t) * gprefix.size(), b->st);
  if (ce == cudaSuccess) ce = dev_alloc((void **)&b->work_d, sizeof(unsigned long long) * b->groups.size(), b->st);
  if (ce == cudaSuccess) ce = dev_alloc((void **)&b->sitems_d, sizeof(BatchSolveItem) * n, b->st);
  for (auto &C : b->cls)
    if (ce == cudaSuccess && C.n > 0) ce = dev_alloc((void **)&C.ctas_d, sizeof(BatchCta) * (C.n_ctas + C.n), b->st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(b->items_d, sorted.data(), sizeof(BuildArgs) * n, cudaMemcpyHostToDevice, b->st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(b->prefix_d, gprefix.data(), sizeof(int64_t) * gprefix.size(), cudaMemcpyHostToDevice,
                         b->st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(b->sitems_d, sitems.data(), sizeof(BatchSolveItem) * n, cudaMemcpyHostToDevice, b->st);
  if (ce == cudaSuccess) ce = cudaMallocHost((void **)&b->cnt_h, sizeof(unsigned long long) * CNT_N * n);
  if (ce == cudaSuccess) ce = cudaMallocHost((void **)&b->stats_h, sizeof(double) * 4 * n);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->st);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "batch set-up"));
  cudaEventCreate(&b->e0);
  cudaEventCreate(&b->e1);
  *out = b;
  return MDP_OK;
}

extern "C" mdp_status mdp_batch_run(mdp_batch b, void *stream, int32_t *sweeps_h, double *ms) {
  if (!b) {
    set_error("invalid argument: NULL batch");
    return MDP_ERR_ARG;
  }
  cudaStream_t ust = (cudaStream_t)stream;
  if (!b->exec) {
    cudaError_t ce = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamBeginCapture");
    cudaError_t ee = enqueue(b);
    ce = cudaStreamEndCapture(b->st, &b->graph);
    if (ee != cudaSuccess) return cuda_fail(ee, "batch capture");
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
  }
  cudaEventRecord(b->e0, ust);
  cudaError_t ce = cudaGraphLaunch(b->exec, ust);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphLaunch");
  cudaEventRecord(b->e1, ust);
  ce = cudaStreamSynchronize(ust);
  if (ce != cudaSuccess) return cuda_fail(ce, "mdp_batch_run");
  float t = 0.f;
  cudaEventElapsedTime(&t, b->e0, b->e1);
  if (ms) *ms = t;
  for (int i = 0; i < b->n; ++i) {
    const unsigned long long *c = b->cnt_h + (size_t)i * CNT_N;
    std::string which = "batch item " + std::to_string(i) + ": ";
    if (c[CNT_OVERFLOW]) {
      set_error(which + "a landing left the neighbouring sub-grid");
      return MDP_ERR_SUBGRID_OVERFLOW;
    }
    if (c[CNT_ROW_CAP] || c[CNT_SPILL_FULL]) {
      set_error(which + "a row exceeded the row cap");
      return MDP_ERR_ELL_OVERFLOW;
    }
    if (c[CNT_POOL_FULL]) {
      set_error(which + "the calibrated entry pool is too small for these inputs (recreate the batch)");
      return MDP_ERR_OOM;
    }
    int errw = 0;
    memcpy(&errw, &b->stats_h[(size_t)i * 4 + 2], sizeof(int));
    if (errw) {
      set_error(which + "a bounded device wait expired in the Bellman pipeline");
      return MDP_ERR_TIMEOUT;
    }
    if (sweeps_h) sweeps_h[i] = (int32_t)b->stats_h[(size_t)i * 4];
  }
  return MDP_OK;
}

extern "C" void mdp_batch_free(mdp_batch b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  const int dev = b->device;
  if (cur != dev) cudaSetDevice(dev);
  batch_release(b);
  if (cur != dev) cudaSetDevice(cur);
}
