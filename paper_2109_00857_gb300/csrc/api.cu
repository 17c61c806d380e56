// api.cu -- the C ABI of include/mdp.h: argument checks, device memory,
// launch sequencing and status read-back for build, export, solve and the
// standalone coefficient sampler.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

#include "mdp_internal.cuh"

namespace mdpgb {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

mdp_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorName(e) + " (" +
            cudaGetErrorString(e) + ")");
  return MDP_ERR_CUDA;
}

static mdp_status arg_fail(const std::string &msg) {
  set_error("invalid argument: " + msg);
  return MDP_ERR_ARG;
}

static std::mutex g_init_mu;
static std::set<int> g_init_devices;

int ensure_device_init() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (g_init_devices.count(dev)) return dev;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed blocks cached for the next build
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  g_init_devices.insert(dev);
  return dev;
}

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  return cudaMallocAsync(p, bytes, st);
}

void dev_free(void *p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

cudaError_t allow_max_smem(const void *func) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({func, dev})) return cudaSuccess;
  int maxopt = 0;
  e = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  // static and dynamic shared memory together may not exceed the opt-in limit
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           maxopt - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({func, dev});
  return e;
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

static int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

mdp_status check_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    set_error("no usable CUDA device (this library has no CPU fallback)");
    return MDP_ERR_CUDA;
  }
  if (ensure_device_init() < 0) {
    set_error("cudaGetDevice failed");
    return MDP_ERR_CUDA;
  }
  return MDP_OK;
}

// Host action table (Sec. II-A): a = f*Nh + h, theta = 2 pi h/Nh, F = Fmax (f+1)/NF.
// Per-axis constants of the FP32 landing offset floor(u + d) (see
// ActionTable): c = floor(d); th = the smallest float >= 1 - frac(d), from
// the exact FP64 value of 1 - frac(d) (frac(d) of a float has at most 24
// significant bits; when 1 - frac(d) is not exact in FP64 it lies within
// 2^-29 of 1 and rounds up to 1 all the same); 2 when frac(d) = 0.
static void offset_thresholds(const float *d, int A, int32_t *c, float *th, float *T, int32_t *le, int32_t *D,
                              uint8_t *L, int32_t *M) {
  std::vector<float> u;
  for (int a = 0; a < A; ++a) {
    const double dd = (double)d[a];
    const double fl = std::floor(dd);
    c[a] = (int32_t)fl;
    if (dd == fl) {
      th[a] = 2.0f;
    } else {
      // 1 - frac(d) = (floor(d) + 1) - d, exact in FP64 unless 0 < d < 2^-29
      // (then it lies within 2^-29 of 1 and rounds up to 1 either way)
      const double t1 = (fl + 1.0) - dd;
      float f = (float)t1;
      if ((double)f < t1) f = std::nextafter(f, 2.0f);
      th[a] = f;
      u.push_back(f);
    }
  }
  std::sort(u.begin(), u.end());
  u.erase(std::unique(u.begin(), u.end()), u.end());
  *D = (int32_t)u.size();
  for (int i = 0; i < kMaxActions + 2; ++i) T[i] = i < (int)u.size() ? u[i] : 2.0f;
  for (int a = 0; a < kMaxActions; ++a) {
    int n = 0;
    if (a < A)
      for (float v : u) n += (v <= th[a]) ? 1 : 0;
    // an integer offset (th = 2) never steps: le = D + 1 exceeds every rank
    le[a] = (a < A && th[a] < 2.0f) ? n : (int32_t)u.size() + 1;
  }
  for (int a = A; a < kMaxActions; ++a) { c[a] = 0; th[a] = 2.0f; }
  // rank lookup: thresholds bucketed by floor(128 T) (clamped to the last bucket)
  std::vector<int> inb(kRankBuckets, 0);
  for (float v : u) inb[std::min((int)std::floor((double)v * kRankBuckets), kRankBuckets - 1)]++;
  int below = 0;
  *M = 0;
  for (int b = 0; b < kRankBuckets; ++b) {
    L[b] = (uint8_t)below;
    below += inb[b];
    *M = std::max(*M, inb[b]);
  }
}

mdp_status make_actions(const mdp_actions *ac, double lam, ActionTable *t, int *A_out) {
  if (!ac) return arg_fail("actions is NULL");
  const int A = ac->n_headings * ac->n_speeds;
  if (ac->n_headings < 1 || ac->n_speeds < 1 || A > kMaxActions)
    return arg_fail("n_headings * n_speeds must be in [1, 32]");
  memset(t, 0, sizeof(*t));
  for (int a = 0; a < A; ++a) {
    double dx, dy, F;
    if (ac->table_h) {
      dx = ac->table_h[3 * a];
      dy = ac->table_h[3 * a + 1];
      F = ac->table_h[3 * a + 2];
    } else {
      const int f = a / ac->n_headings, h = a % ac->n_headings;
      F = ac->f_max * (f + 1) / ac->n_speeds;
      const double th = 2.0 * M_PI * h / ac->n_headings;
      dx = F * std::cos(th);
      dy = F * std::sin(th);
    }
    if (!std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(F))
      return arg_fail("action table holds a non-finite value");
    t->dx64[a] = dx;
    t->dy64[a] = dy;
    t->F64[a] = F;
    t->dxl[a] = (float)(dx * lam);
    t->dyl[a] = (float)(dy * lam);
    t->F[a] = (float)F;
  }
  offset_thresholds(t->dxl, A, t->cx, t->thx, t->Tx, t->lex, &t->Dx, t->Lx, &t->Mx);
  offset_thresholds(t->dyl, A, t->cy, t->thy, t->Ty, t->ley, &t->Dy, t->Ly, &t->My);
  *A_out = A;
  return MDP_OK;
}

struct Pinned {
  unsigned long long *p = nullptr;
  Pinned() { cudaMallocHost((void **)&p, sizeof(unsigned long long) * CNT_N * 2); }
  ~Pinned() { if (p) cudaFreeHost(p); }
};

static void free_model_memory(mdp_model_t *m, cudaStream_t st) {
  dev_free(m->pool, st);
  dev_free(m->slice_off, st);
  dev_free(m->slice_w, st);
  dev_free(m->nnz, st);
  dev_free(m->sinkc, st);
  dev_free(m->R, st);
  dev_free(m->cls, st);
  dev_free(m->delta, st);
  dev_free(m->Vtmp, st);
  dev_free(m->cnt, st);
  dev_free(m->solve_stats_d, st);
  dev_free(m->spill, st);
  dev_free(m->spill_off, st);
  m->spill = nullptr;
  m->spill_off = nullptr;
  m->pool = nullptr;
  m->slice_off = nullptr;
  m->slice_w = nullptr;
  m->nnz = nullptr;
  m->sinkc = nullptr;
  m->R = nullptr;
  m->cls = nullptr;
  m->delta = nullptr;
  m->Vtmp = nullptr;
  m->cnt = nullptr;
  m->solve_stats_d = nullptr;
}

void free_model_on_stream(mdp_model_t *m, cudaStream_t st) {
  if (!m) return;
  free_model_memory(m, st);
  delete m;
}

}  // namespace mdpgb

using namespace mdpgb;

namespace mdpgb {
static std::atomic<long long> g_test_wait_cycles{0};
static std::atomic<uint32_t> g_test_extra_tx{0};
void take_test_injection(SolveArgs &a) {
  a.wait_cycles = g_test_wait_cycles.load();
  a.test_extra_tx = g_test_extra_tx.exchange(0u);
}
}  // namespace mdpgb

extern "C" mdp_status mdp_test_inject(int32_t what, int64_t value) {
  if (what == MDP_TEST_WAIT_NEVER_COMPLETES && value >= 0 && value <= (1 << 20) && (value % 16) == 0) {
    g_test_extra_tx.store((uint32_t)value);
    return MDP_OK;
  }
  if (what == MDP_TEST_WAIT_LIMIT_CYCLES && value >= 0) {
    g_test_wait_cycles.store((long long)value);
    return MDP_OK;
  }
  set_error("invalid argument: mdp_test_inject(what, value)");
  return MDP_ERR_ARG;
}

extern "C" const char *mdp_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *mdp_version(void) { return "mdp_gb300 1.0 (sm_103a)"; }

extern "C" mdp_status mdp_sample_coeffs(int32_t nt, int32_t N, int32_t K, const double *sigma_h,
                                        uint64_t seed, uint64_t mdp_id, int32_t precision, void *Y,
                                        void *stream) {
  mdp_status s = check_device();
  if (s != MDP_OK) return s;
  if (nt < 1 || N < 1 || K < 1 || K > kMaxModes) return arg_fail("need nt, N >= 1 and 1 <= K <= 16");
  if (!sigma_h || !Y) return arg_fail("sigma_h and Y must be non-NULL");
  if (precision != MDP_FP32 && precision != MDP_FP64_CHECK) return arg_fail("precision");
  cudaStream_t st = (cudaStream_t)stream;
  double *sig_d = nullptr;
  unsigned long long *cap_d = nullptr;
  MDP_CUDA_TRY(dev_alloc((void **)&sig_d, sizeof(double) * K, st));
  MDP_CUDA_TRY(dev_alloc((void **)&cap_d, sizeof(unsigned long long), st));
  MDP_CUDA_TRY(cudaMemcpyAsync(sig_d, sigma_h, sizeof(double) * K, cudaMemcpyHostToDevice, st));
  MDP_CUDA_TRY(cudaMemsetAsync(cap_d, 0, sizeof(unsigned long long), st));
  MDP_CUDA_TRY(launch_sample_coeffs(nt, N, K, sig_d, seed, mdp_id,
                                    precision == MDP_FP64_CHECK ? (double *)Y : nullptr,
                                    precision == MDP_FP32 ? (float *)Y : nullptr, cap_d, st));
  unsigned long long capped = 0;
  MDP_CUDA_TRY(cudaMemcpyAsync(&capped, cap_d, sizeof(capped), cudaMemcpyDeviceToHost, st));
  dev_free(sig_d, st);
  dev_free(cap_d, st);
  MDP_CUDA_TRY(cudaStreamSynchronize(st));
  (void)capped;  // a capped pair (probability ~1e-43 each) draws z = 0
  return MDP_OK;
}

namespace mdpgb {
// The whole build.  With a hook, it stops after the set-up (validation,
// coefficient draw, sub-grid size, allocations, cell classes) and hands the
// model and its kernel arguments to the caller instead of launching the build
// (the batched build launches them itself).
mdp_status build_impl(const mdp_env *env, const mdp_grid *grid, const mdp_actions *actions, int32_t N,
                      int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj, const mdp_build_opts *opts,
                      void *stream, mdp_model *out, BuildHook *hook, BuildLimits *lim) {
  if (out) *out = nullptr;
  mdp_status s = check_device();
  if (s != MDP_OK) return s;
  if (!env || !grid || !actions || !out || !objs_h) return arg_fail("NULL env/grid/actions/objs/out");
  if (grid->nx < 1 || grid->ny < 1 || grid->nt < 1) return arg_fail("grid sizes must be >= 1");
  if (!(grid->dx > 0) || !(grid->dt > 0) || !std::isfinite(grid->dx) || !std::isfinite(grid->dt))
    return arg_fail("dx and dt must be finite and > 0");
  if (env->K < 0 || env->K > kMaxModes) return arg_fail("K must be in [0, 16]");
  if (N < 1 || N > 65535) return arg_fail("N must be in [1, 65535]");
  if (env->precision != MDP_FP32 && env->precision != MDP_FP64_CHECK) return arg_fail("precision");
  if (n_obj < 1 || n_obj > 3) return arg_fail("n_obj must be in [1, 3]");
  for (int o = 0; o < n_obj; ++o) {
    if (objs_h[o] < 0 || objs_h[o] > 2) return arg_fail("unknown objective");
    if (objs_h[o] == MDP_OBJ_NET_ENERGY && !env->gbar) return arg_fail("net energy needs gbar");
  }
  if (!env->vbar || !env->obstacle || !env->target || (env->K > 0 && !env->modes))
    return arg_fail("vbar, modes, obstacle and target must be non-NULL");
  if (env->K > 0 && !env->coeffs && !env->sigma_h) return arg_fail("need coeffs or sigma_h");
  // the kernels load (x, y) pairs and coefficient rows as vectors
  if (((uintptr_t)env->vbar | (uintptr_t)env->modes) & (2 * (env->precision == MDP_FP64_CHECK ? 8 : 4) - 1))
    return arg_fail("vbar and modes must be aligned to one (x, y) pair");
  if ((uintptr_t)env->coeffs & 15) return arg_fail("coeffs must be 16-byte aligned");
  if ((uintptr_t)env->gbar & 3) return arg_fail("gbar must be 4-byte aligned");
  if (subgrid_L < 0 || subgrid_L > 255 || (subgrid_L > 0 && subgrid_L % 2 == 0))
    return arg_fail("subgrid_L must be 0 (auto) or odd in [1, 255]");
  const int row_cap = (opts && opts->row_cap > 0) ? opts->row_cap : 64;
  if (row_cap > 255) return arg_fail("row_cap must be <= 255");
  const int64_t Nc = (int64_t)grid->nx * grid->ny, nS = Nc * grid->nt;
  if (nS > ((int64_t)1 << 40)) return arg_fail("grid too large");
  const double lam = grid->dt / grid->dx;

  ActionTable at;
  int A = 0;
  s = make_actions(actions, lam, &at, &A);
  if (s != MDP_OK) return s;
  const int prec = env->precision;
  const size_t fsz = prec == MDP_FP64_CHECK ? 8 : 4;
  cudaStream_t st = (cudaStream_t)stream;

  mdp_model_t *m = new mdp_model_t();
  memset(m, 0, sizeof(*m));
  m->nx = grid->nx; m->ny = grid->ny; m->nt = grid->nt;
  m->K = env->K; m->N = N; m->A = A; m->precision = prec; m->n_obj = n_obj;
  for (int o = 0; o < n_obj; ++o) m->objs[o] = objs_h[o];
  m->Nc = Nc; m->nS = nS; m->dx = grid->dx; m->dt = grid->dt;
  m->A_pad = pow2_at_least(A);
  m->spw = 32 / m->A_pad;
  m->n_slices = (nS + m->spw - 1) / m->spw;
  m->rows_pad = m->n_slices * 32;
  m->row_cap = row_cap;
  cudaGetDevice(&m->device);
  RewardParams &rw = m->rw;
  rw.c_f = actions->c_f; rw.c_r = actions->c_r; rw.r_term = actions->r_term;
  rw.r_out = actions->r_outbound; rw.dt = grid->dt; rw.dx = grid->dx; rw.n_obj = n_obj;
  for (int o = 0; o < n_obj; ++o) rw.objs[o] = objs_h[o];

  auto fail = [&](mdp_status code) {
    free_model_memory(m, st);
    delete m;
    return code;
  };
#define TRY(expr)                                   \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return fail(cuda_fail(_e, #expr)); \
  } while (0)

  // -- coefficients: caller table or Philox draw (step a1)
  const void *Y = env->coeffs;
  void *Yown = nullptr;
  double *sig_d = nullptr;
  TRY(dev_alloc((void **)&m->cnt, sizeof(unsigned long long) * CNT_N, st));
  TRY(cudaMemsetAsync(m->cnt, 0, sizeof(unsigned long long) * CNT_N, st));
  // timing events, destroyed on every return path
  struct Events {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    Events() { for (auto &x : e) cudaEventCreate(&x); }
    ~Events() { for (auto &x : e) if (x) cudaEventDestroy(x); }
  } evs;
  cudaEvent_t ev0 = evs.e[0], ev1 = evs.e[1], evk = evs.e[2];
  cudaEventRecord(ev0, st);
  int launches = 0;
  if (!Y && env->K > 0) {
    TRY(dev_alloc(&Yown, fsz * (size_t)grid->nt * N * env->K, st));
    TRY(dev_alloc((void **)&sig_d, sizeof(double) * env->K, st));
    TRY(cudaMemcpyAsync(sig_d, env->sigma_h, sizeof(double) * env->K, cudaMemcpyHostToDevice, st));
    TRY(launch_sample_coeffs(grid->nt, N, env->K, sig_d, env->seed, env->mdp_id,
                             prec == MDP_FP64_CHECK ? (double *)Yown : nullptr,
                             prec == MDP_FP32 ? (float *)Yown : nullptr, m->cnt + CNT_CAPPED, st));
    Y = Yown;
    ++launches;
  }

  // -- sub-grid side: given, or from the component-wise field extremes (Sec. III-B)
  int L = subgrid_L;
  if (L == 0) {
    const int K = env->K;
    unsigned int *ex = nullptr;
    const int nex = 2 + 2 * K + K;
    TRY(dev_alloc((void **)&ex, sizeof(unsigned int) * nex, st));
    TRY(cudaMemsetAsync(ex, 0, sizeof(unsigned int) * nex, st));
    TRY(launch_absmax(env->vbar, prec, nS * 2, 1, 1, 2, ex, st));
    ++launches;
    if (K > 0) {
      TRY(launch_absmax(env->modes, prec, nS * K * 2, K, Nc, 2, ex + 2, st));
      TRY(launch_absmax(Y, prec, (int64_t)grid->nt * N * K, K, 1, 1, ex + 2 + 2 * K, st));
      launches += 2;
    }
    std::vector<unsigned int> hx(nex);
    TRY(cudaMemcpyAsync(hx.data(), ex, sizeof(unsigned int) * nex, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    dev_free(ex, st);
    auto f = [&](int i) { float v; memcpy(&v, &hx[i], 4); return (double)v; };
    double wmax[2] = {f(0), f(1)};
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < 2; ++c) wmax[c] += f(2 + 2 * K + k) * f(2 + 2 * k + c);
    double amax[2] = {0, 0};
    for (int a = 0; a < A; ++a) {
      amax[0] = std::max(amax[0], std::fabs(at.dx64[a]));
      amax[1] = std::max(amax[1], std::fabs(at.dy64[a]));
    }
    int h = 0;
    for (int c = 0; c < 2; ++c) {
      // |offset| <= ceil(1/2 + lam (max|v| + max|a|)), plus one cell of buffer
      const int hc = (int)std::ceil(0.5 + lam * (wmax[c] + amax[c]) * (1.0 + 1e-6)) + 1;
      h = std::max(h, hc);
    }
    if (2 * h + 1 > 255) return fail(arg_fail("automatic sub-grid would exceed 255 cells"));
    L = 2 * h + 1;
  }
  m->L = L;
  m->h = (L - 1) / 2;
  m->nbins = L * L;
  // successors are stored as signed 16-bit offsets dj*Nx + di
  if ((int64_t)m->h * (grid->nx + 1) > 32767)
    return fail(arg_fail("sub-grid half-width * (nx + 1) must be <= 32767 (16-bit successor offsets)"));

  // -- model memory.  The entry pool is sized for an average slice width of
  // kPoolGuess columns first; if the build runs out of columns it is rebuilt
  // once with a pool of exactly the columns needed.  A row holds at most
  // row_cap in-domain successors in the ELL columns (the sink has its own
  // count); the rest of a longer row goes to a spill area, which the first
  // attempt does not have: if some row needs it, the rebuild allocates it
  // with exactly the words counted.
  const int Wmax = std::min(row_cap, m->nbins);
  const int kPoolGuess = 16;
  // the pool may take at most 60 % of the free device memory; asking the
  // driver costs a round trip, so only pools above 256 MiB ask
  size_t free_b = (size_t)1 << 62, total_b = 0;
  if ((uint64_t)m->n_slices * (uint64_t)std::min(kPoolGuess, Wmax) * 128 > ((uint64_t)256 << 20))
    cudaMemGetInfo(&free_b, &total_b);
  const uint64_t budget_cols = (uint64_t)(0.6 * (double)free_b) / 128;
  auto pool_cols_for = [&](int width) {
    uint64_t c = (uint64_t)m->n_slices * (uint64_t)std::min(width, Wmax) + 64;
    if (c > budget_cols) c = budget_cols;
    return c < 1 ? (uint64_t)1 : c;
  };
  uint64_t cap_cols = (hook && hook->pool_cols) ? hook->pool_cols : pool_cols_for(kPoolGuess);
  if (lim && lim->pool_cols) cap_cols = lim->pool_cols;   // the caller's pool size (and limit)
  TRY(dev_alloc((void **)&m->pool, (size_t)cap_cols * 128, st));
  TRY(dev_alloc((void **)&m->slice_off, sizeof(uint32_t) * (size_t)m->n_slices, st));
  TRY(dev_alloc((void **)&m->slice_w, (size_t)m->n_slices, st));
  TRY(dev_alloc((void **)&m->nnz, (size_t)m->rows_pad, st));
  TRY(dev_alloc((void **)&m->sinkc, sizeof(uint16_t) * (size_t)m->rows_pad, st));
  TRY(dev_alloc(&m->R, fsz * (size_t)m->rows_pad * n_obj, st));
  TRY(dev_alloc((void **)&m->cls, (size_t)nS, st));
  TRY(dev_alloc((void **)&m->delta, sizeof(int32_t) * (size_t)m->nbins, st));
  TRY(launch_prepare(env->obstacle, env->target, m->cls, grid->nx, grid->ny, grid->nt, m->delta, L, st));
  ++launches;

  BuildArgs ba;
  memset(&ba, 0, sizeof(ba));
  ba.nx = grid->nx; ba.ny = grid->ny; ba.nt = grid->nt; ba.K = env->K; ba.N = N; ba.A = A;
  ba.A_pad = m->A_pad; ba.spw = m->spw; ba.L = L; ba.h = m->h; ba.nbins = m->nbins;
  ba.row_cap = Wmax; ba.Nc = Nc; ba.nS = nS; ba.n_slices = m->n_slices; ba.rows_pad = m->rows_pad;
  ba.lam = (float)lam;
  ba.vbar = env->vbar; ba.modes = env->modes; ba.Y = Y; ba.gbar = env->gbar; ba.cls = m->cls;
  ba.act = at; ba.rw = rw;
  ba.pool = m->pool; ba.pool_cap_cols = cap_cols; ba.slice_off = m->slice_off; ba.slice_w = m->slice_w; ba.nnz = m->nnz; ba.sinkc = m->sinkc;
  ba.R = m->R; ba.cnt = m->cnt;
  ba.slice_begin = 0; ba.slice_end = m->n_slices;
  ba.slices_per_warp = lim ? lim->slices_per_warp : 0;
  // spill area: the caller's size when it fixes the pool (the server), else none yet
  uint64_t spill_cap = (lim && lim->pool_cols) ? lim->spill_words : 0;
  auto alloc_spill = [&](uint64_t words) -> cudaError_t {
    dev_free(m->spill, st);
    m->spill = nullptr;
    cudaError_t e = cudaSuccess;
    if (!m->spill_off) e = dev_alloc((void **)&m->spill_off, sizeof(uint32_t) * (size_t)m->n_slices, st);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->spill, sizeof(uint32_t) * (size_t)std::max<uint64_t>(words, 1), st);
    ba.spill = m->spill;
    ba.spill_off = m->spill_off;
    ba.spill_cap_words = words;
    return e;
  };
  if (spill_cap) TRY(alloc_spill(spill_cap));
  // launch shapes: the caller's, else the autotuner's for this workload class, else defaults
  Tuning tun;
  tuning_lookup(tuning_key(m->A_pad, env->K, N, Nc, n_obj, prec), &tun);
  m->sweep_smem_kb = tun.sweep_smem_kb;
  int threads = (opts && opts->threads > 0) ? opts->threads : tun.threads;
  if (threads % 64 != 0 || threads > 512) return fail(arg_fail("threads must be a multiple of 64, <= 512"));
  int chunk = (opts && opts->chunk > 0) ? opts->chunk : tun.chunk;
  if (chunk > N) chunk = N;
  // the full-window kernels hold an [L*L][32] histogram in shared memory: the
  // FP32 one halves its realization chunk until it fits (the model does not
  // depend on the chunk); beyond that (sub-grids above 41 x 41 cells) only
  // the warp kernel's slices can be built
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device);
  const size_t window_limit = (size_t)smem_max - 1024;   // the kernels' static shared memory
  if (prec == MDP_FP64_CHECK && (size_t)m->nbins * 128 > window_limit)
    return fail(arg_fail("check mode needs a sub-grid of at most 41 x 41 cells (its histogram is in shared memory)"));
  ba.chunk = chunk;
  while (chunk > 32 && fp32_smem_bytes(ba, threads) > window_limit) ba.chunk = chunk = chunk / 2;
  const bool window_fits = fp32_smem_bytes(ba, threads) <= window_limit;
  int hist_cap = (opts && opts->hist_cap > 0) ? opts->hist_cap : tun.hist_cap;
  const int build_warps = tun.build_warps;
  if (hist_cap > 6144) return fail(arg_fail("hist_cap must be <= 6144"));
  uint32_t *defer = nullptr;
  if (prec == MDP_FP32) TRY(dev_alloc((void **)&defer, sizeof(uint32_t) * (size_t)m->n_slices, st));
  ba.cap_bins = hist_cap;
  ba.defer = defer;
  ba.defer_in = nullptr;
  if (hook) {
    hook->args = ba;
    hook->Yown = Yown;
    hook->sigma_d = sig_d;
    hook->defer = defer;
    hook->pool_cols = cap_cols;
    hook->threads = threads;
    *out = m;
    return MDP_OK;
  }
  static thread_local Pinned pin;
  if (!pin.p) return fail(cuda_fail(cudaErrorMemoryAllocation, "cudaMallocHost"));
  const unsigned long long *c = pin.p;
  for (int attempt = 0;; ++attempt) {
    cudaEventRecord(evk, st);
    if (prec == MDP_FP64_CHECK) {
      TRY(launch_build_fp64(ba, st));
      ++launches;
    } else {
      // warp-per-slice kernel, then the full-window CTA kernel over what it deferred
      TRY(launch_build_warp(ba, build_warps, num_sms(), st));
      BuildArgs bd = ba;
      bd.defer_in = defer;
      if (window_fits) TRY(launch_build_fp32(bd, threads, num_sms(), st));
      launches += window_fits ? 2 : 1;
    }
    cudaEventRecord(ev1, st);
    TRY(cudaMemcpyAsync(pin.p, m->cnt, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    const bool pool_full = c[CNT_POOL_FULL] != 0, spill_full = c[CNT_SPILL_FULL] != 0;
    if ((!pool_full && !spill_full) || attempt > 0) break;
    // The pool or the spill area ran out.  The column counter holds every
    // slice's width even for the slices that did not fit, and the spill
    // counter every spill block's words, i.e. exactly what the build needs:
    // rebuild once with those sizes (counters reset, sampled Y kept) --
    // unless the caller fixed the sizes, then report the need.
    const uint64_t need = pool_full ? c[CNT_POOL_COLS] : cap_cols;
    const uint64_t sneed = spill_full ? c[CNT_SPILL_WORDS] : spill_cap;
    if (lim && lim->pool_cols) {
      lim->pool_cols_needed = need;
      lim->spill_words_needed = sneed;
      char buf[200];
      snprintf(buf, sizeof buf, "the model needs %llu pool columns and %llu spill words, above the %llu and %llu allowed",
               (unsigned long long)need, (unsigned long long)sneed, (unsigned long long)lim->pool_cols,
               (unsigned long long)spill_cap);
      set_error(buf);
      if (Yown) dev_free(Yown, st);
      if (sig_d) dev_free(sig_d, st);
      if (defer) dev_free(defer, st);
      return fail(MDP_ERR_BUDGET);
    }
    // does not fit the device (or the 32-bit block offsets): reported as MDP_ERR_OOM below
    if (need > budget_cols || sneed > budget_cols * 32 || sneed >= (uint64_t)kNoSlice) break;
    if (pool_full) {
      dev_free(m->pool, st);
      cap_cols = std::max<uint64_t>(need, 1);
      TRY(dev_alloc((void **)&m->pool, (size_t)cap_cols * 128, st));
      ba.pool = m->pool;
      ba.pool_cap_cols = cap_cols;
    }
    if (spill_full) {
      spill_cap = sneed;
      TRY(alloc_spill(spill_cap));
    }
    TRY(cudaMemsetAsync(m->cnt, 0, sizeof(unsigned long long) * CNT_CAPPED, st));
    TRY(cudaMemsetAsync(m->cnt + CNT_WORK, 0, sizeof(unsigned long long) * (CNT_N - CNT_WORK), st));
  }
  if (Yown) dev_free(Yown, st);
  if (sig_d) dev_free(sig_d, st);
  if (defer) dev_free(defer, st);
  m->deferred = (int64_t)c[CNT_DEFER_N];

  float ms = 0.f, kms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventElapsedTime(&kms, evk, ev1);
  m->build_ms = ms;
  m->kernel_ms = kms;
  m->launches = launches;
  if (prec == MDP_FP32 && !window_fits && m->deferred > 0) {
    char buf[200];
    snprintf(buf, sizeof buf, "%lld slice(s) need the full-window kernel, whose histogram of a %dx%d sub-grid "
             "exceeds shared memory: raise hist_cap or use a sub-grid of at most 41 x 41 cells",
             (long long)m->deferred, L, L);
    set_error(buf);
    return fail(MDP_ERR_ARG);
  }
  if (c[CNT_OVERFLOW]) {
    char buf[256];
    snprintf(buf, sizeof buf, "%llu landing(s)/row(s) left the %dx%d neighbouring sub-grid; use a larger subgrid_L",
             c[CNT_OVERFLOW], L, L);
    set_error(buf);
    return fail(MDP_ERR_SUBGRID_OVERFLOW);
  }
  if (c[CNT_POOL_FULL] || c[CNT_SPILL_FULL]) {
    set_error(c[CNT_POOL_FULL] ? "entry pool capacity exhausted (device memory budget)"
                               : "spill area exhausted (device memory budget)");
    return fail(MDP_ERR_OOM);
  }
  m->pool_cols = c[CNT_POOL_COLS];
  m->nnz_total = (int64_t)c[CNT_NNZ];
  m->nnz_domain = (int64_t)c[CNT_DOMAIN];
  m->max_row_nnz = (int32_t)c[CNT_MAXROW];
  m->max_row_len = c[CNT_MAXLEN] ? (int32_t)c[CNT_MAXLEN] : m->max_row_nnz;
  m->samples = (int64_t)c[CNT_SAMPLES];
  m->spill_rows = (int64_t)c[CNT_SPILL_ROWS];
  m->spill_words = c[CNT_SPILL_WORDS];
  if (m->spill_words == 0) {   // no row beyond row_cap: no spill area
    dev_free(m->spill, st);
    dev_free(m->spill_off, st);
    m->spill = nullptr;
    m->spill_off = nullptr;
    spill_cap = 0;
  }
  // -- compaction: the columns in use move into a pool of exactly that size,
  // in slice order (a run of consecutive slices is then one contiguous copy
  // for the solver)
  if (!(opts && opts->no_compact)) {
    uint32_t *np = nullptr;
    TRY(dev_alloc((void **)&np, (size_t)std::max<uint64_t>(m->pool_cols, 1) * 128, st));
    TRY(launch_pool_reorder(m->pool, np, m->slice_off, m->slice_w, m->n_slices, st));
    dev_free(m->pool, st);
    m->pool = np;
    m->pool_ordered = 1;
    cap_cols = std::max<uint64_t>(m->pool_cols, 1);
  }
  m->device_bytes = (int64_t)cap_cols * 128 + 5 * m->n_slices + 3 * m->rows_pad + (int64_t)fsz * m->rows_pad * n_obj +
                    nS + 4 * m->nbins + 8 * CNT_N + (m->spill ? 4 * (int64_t)(m->n_slices + spill_cap) : 0);
  *out = m;
#undef TRY
  return MDP_OK;
}

}  // namespace mdpgb

extern "C" mdp_status mdp_build(const mdp_env *env, const mdp_grid *grid, const mdp_actions *actions,
                                int32_t N, int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj,
                                const mdp_build_opts *opts, void *stream, mdp_model *out) {
  return build_impl(env, grid, actions, N, subgrid_L, objs_h, n_obj, opts, stream, out, nullptr);
}

extern "C" mdp_status mdp_model_info(mdp_model m, mdp_model_info_t *o) {
  if (!m || !o) return arg_fail("NULL model or info");
  memset(o, 0, sizeof(*o));
  o->n_states = m->nS;
  o->A = m->A;
  o->N = m->N;
  o->L = m->L;
  o->n_obj = m->n_obj;
  for (int i = 0; i < m->n_obj; ++i) o->objs[i] = m->objs[i];
  o->precision = m->precision;
  o->rows = m->nS * m->A;
  o->nnz = m->nnz_total;
  o->max_row_nnz = m->max_row_nnz;
  o->pool_columns = (int64_t)m->pool_cols;
  o->device_bytes = m->device_bytes + (m->Vtmp ? (int64_t)(m->nS + 1) * (m->precision ? 8 : 4) : 0);
  o->samples = m->samples;
  o->build_ms = m->build_ms;
  o->kernel_ms = m->kernel_ms;
  o->launches = m->launches;
  o->wide_slices = m->deferred;
  o->nnz_domain = m->nnz_domain;
  o->spill_rows = m->spill_rows;
  o->spill_words = (int64_t)m->spill_words;
  o->max_row_len = m->max_row_len;
  return MDP_OK;
}

extern "C" mdp_status mdp_export_csr(mdp_model m, int32_t obj, int64_t *rowptr, int64_t *col,
                                     int32_t *count, void *R, void *stream) {
  if (!m || !rowptr) return arg_fail("NULL model or rowptr");
  if (obj < 0 || obj >= m->n_obj) return arg_fail("objective slot out of range");
  cudaStream_t st = (cudaStream_t)stream;
  MDP_CUDA_TRY(launch_export(m, obj, rowptr, col, count, R, st));
  MDP_CUDA_TRY(cudaStreamSynchronize(st));
  return MDP_OK;
}

// Value iteration for n objectives on one model: the Bellman kernels stream
// P once per sweep for all of them (mdp_solve is the n = 1 case).
static mdp_status solve_impl(mdp_model m, int32_t n, const int32_t *objs, int32_t method, double tol,
                             int32_t max_sweeps, void *const *V, int16_t *const *policy, void *stream,
                             mdp_solve_stats *stats) {
  if (!m) return arg_fail("NULL model");
  if (n < 1 || n > 3) return arg_fail("n must be 1, 2 or 3");
  if (!objs || !V || !policy) return arg_fail("NULL objs, V or policy");
  for (int o = 0; o < n; ++o) {
    if (!V[o] || !policy[o]) return arg_fail("NULL V or policy");
    if (objs[o] < 0 || objs[o] >= m->n_obj) return arg_fail("objective slot out of range");
  }
  const bool warm = (method & MDP_SOLVE_WARM) != 0;
  method &= ~MDP_SOLVE_WARM;
  if (method != MDP_SOLVE_JACOBI && method != MDP_SOLVE_LAYERED && method != MDP_SOLVE_JACOBI_FULL)
    return arg_fail("method");
  if (warm && (n != 1 || method == MDP_SOLVE_LAYERED))
    return arg_fail("MDP_SOLVE_WARM applies to single-objective Jacobi solves");
  if (!(tol >= 0) && !(tol < 0)) return arg_fail("tol is NaN");
  if (max_sweeps < 0) return arg_fail("max_sweeps must be >= 0");
  if (max_sweeps == 0) max_sweeps = m->nt + 1;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t fsz = m->precision == MDP_FP64_CHECK ? 8 : 4;
  const size_t vbytes = fsz * (size_t)(m->nS + 1);
  // the solver streams slices with 16-byte-aligned bulk copies and indexes
  // successors with 32-bit offsets
  if ((((uintptr_t)m->pool) | ((uintptr_t)m->R) | ((uintptr_t)m->nnz)) & 15) {
    set_error("model arrays are not 16-byte aligned");
    return MDP_ERR_CUDA;
  }
  if (m->nS + m->Nc >= ((int64_t)1 << 31)) return arg_fail("more than 2^31 states is not supported by the solver");
  const bool jac = method != MDP_SOLVE_LAYERED;
  const bool active = method == MDP_SOLVE_JACOBI;   // active-layer sweeps
  // n = 1 iterates in V and the model's cached partner buffer; n > 1 in
  // packed value tables (stream-ordered scratch) copied out to V[o] at the end
  if (n == 1 && jac && !m->Vtmp) MDP_CUDA_TRY(dev_alloc(&m->Vtmp, vbytes, st));
  const size_t tbytes = fsz * (size_t)(n == 3 ? 4 : n) * (size_t)(m->nS + 1);
  const int n_tables = n == 1 ? 0 : (jac ? 2 : 1);
  void *tables = nullptr;
  if (n_tables) MDP_CUDA_TRY(dev_alloc(&tables, tbytes * n_tables, st));
  // status blocks, then (active-layer Jacobi) the per-sweep work counts and
  // the three rotating layer-flag arrays
  const size_t blk = 4 + (size_t)max_sweeps;
  const size_t n_dbl = blk * (size_t)n + (active ? (size_t)max_sweeps + (3 * ((size_t)m->nt + 1) + 7) / 8 : 0);
  double *sd = nullptr;
  cudaError_t ce = dev_alloc((void **)&sd, sizeof(double) * n_dbl, st);
  if (ce != cudaSuccess) {
    if (tables) dev_free(tables, st);
    return cuda_fail(ce, "dev_alloc");
  }
  SolveIO io{};
  io.n = n;
  for (int o = 0; o < n; ++o) {
    io.R[o] = static_cast<const char *>(m->R) + fsz * (size_t)objs[o] * m->rows_pad;
    io.V[o] = V[o];
    io.policy[o] = policy[o];
  }
  io.Vtmp[0] = (n == 1 && jac) ? m->Vtmp : nullptr;
  for (int t = 0; t < n_tables; ++t) io.table[t] = static_cast<char *>(tables) + tbytes * t;
  for (int o = 0; o < n && ce == cudaSuccess; ++o) ce = cudaMemsetAsync(sd + o * blk, 0, sizeof(double) * 4, st);
  if (ce == cudaSuccess && n == 1) {
    if (warm)   // V_0 as given; the sink stays 0
      ce = cudaMemsetAsync(static_cast<char *>(V[0]) + fsz * (size_t)m->nS, 0, fsz, st);
    else
      ce = cudaMemsetAsync(V[0], 0, vbytes, st);
  }
  if (ce == cudaSuccess && io.Vtmp[0]) ce = cudaMemsetAsync(io.Vtmp[0], 0, vbytes, st);
  if (ce == cudaSuccess && tables) ce = cudaMemsetAsync(tables, 0, tbytes * n_tables, st);
  SolveArgs a;
  a.pool = m->pool; a.slice_off = m->slice_off; a.slice_w = m->slice_w; a.nnz = m->nnz;
  a.wcap = std::max(1, m->max_row_nnz);
  a.spill = m->spill;
  a.spill_off = m->spill_off;
  a.small_ctas = m->sweep_small_ctas;
  a.R = io.R[0];
  a.cls = m->cls; a.delta = m->delta;
  a.nS = m->nS; a.Nc = m->Nc; a.n_slices = m->n_slices;
  a.A = m->A; a.A_pad = m->A_pad; a.spw = m->spw; a.N = m->N; a.nbins = m->nbins; a.tol = tol;
  a.err = reinterpret_cast<int *>(sd + 2);
  a.nt = m->nt;
  a.pool_ordered = m->pool_ordered;
  a.sweep_smem_kb = m->sweep_smem_kb;
  take_test_injection(a);
  if (active) {
    a.work = reinterpret_cast<unsigned long long *>(sd + blk * n);
    a.lflags = reinterpret_cast<uint8_t *>(sd + blk * n + max_sweeps);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  if (ce == cudaSuccess) {
    if (jac) ce = launch_jacobi_multi(a, m->precision, max_sweeps, io, sd, st);
    else ce = launch_layered_multi(a, m->precision, m->nt, io, sd, st);
  }
  cudaEventRecord(e1, st);
  double hs[3][3] = {};
  for (int o = 0; o < n && ce == cudaSuccess; ++o)
    ce = cudaMemcpyAsync(hs[o], sd + o * blk, sizeof(hs[o]), cudaMemcpyDeviceToHost, st);
  std::vector<unsigned long long> work(active ? max_sweeps : 0);
  if (active && ce == cudaSuccess)
    ce = cudaMemcpyAsync(work.data(), a.work, sizeof(unsigned long long) * max_sweeps, cudaMemcpyDeviceToHost, st);
  dev_free(sd, st);
  if (tables) dev_free(tables, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (ce == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_fail(ce, "mdp_solve");
  int errw = 0;
  memcpy(&errw, &hs[0][2], sizeof(int));
  if (errw) {
    set_error("a bounded device wait expired in the Bellman pipeline");
    return MDP_ERR_TIMEOUT;
  }
  if (stats) {
    for (int o = 0; o < n; ++o) {
      stats[o].sweeps = jac ? (int32_t)hs[o][0] : 1;
      stats[o].residual = jac ? hs[o][1] : 0.0;
      stats[o].solve_ms = ms;
      if (active) {   // slices recomputed in the objective's sweeps
        int64_t sl = 0;
        for (int k = 0; k < stats[o].sweeps; ++k) sl += (int64_t)work[k];
        stats[o].backups = std::min<int64_t>(sl * m->spw, (int64_t)stats[o].sweeps * m->nS) * m->A;
      } else {
        stats[o].backups = (int64_t)stats[o].sweeps * m->nS * m->A;
      }
    }
  }
  return MDP_OK;
}

extern "C" mdp_status mdp_solve(mdp_model m, int32_t obj, int32_t method, double tol,
                                int32_t max_sweeps, void *V, int16_t *policy, void *stream,
                                mdp_solve_stats *stats) {
  if (!m || !V || !policy) return arg_fail("NULL model, V or policy");
  return solve_impl(m, 1, &obj, method, tol, max_sweeps, &V, &policy, stream, stats);
}

extern "C" mdp_status mdp_solve_multi(mdp_model m, int32_t n, const int32_t *objs, int32_t method,
                                      double tol, int32_t max_sweeps, void *const *V,
                                      int16_t *const *policy, void *stream, mdp_solve_stats *stats) {
  return solve_impl(m, n, objs, method, tol, max_sweeps, V, policy, stream, stats);
}

extern "C" void mdp_model_free(mdp_model m) {
  if (!m) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != m->device) cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  free_model_memory(m, 0);
  if (cur != m->device) cudaSetDevice(cur);
  delete m;
}
