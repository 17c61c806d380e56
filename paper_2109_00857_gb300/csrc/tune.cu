// tune.cu -- the autotuner: launch shapes per workload class, timed on a
// calibration cut of the caller's environment, kept in a process-wide table
// and in a JSON file that later processes load.
//
// A workload class is (actions padded to a power of two, modes, N and cells
// rounded to powers of two, objectives, precision).  The shapes tuned are the
// warps per CTA and the fine-table capacity of the warp-per-slice build
// kernel, the CTA size of the full-window build kernel (when the calibration
// defers slices to it), and the shared memory of the one-state-per-slice
// Bellman sweep (which sets its slot size).  None of them changes a count, an
// entry, an R value, a value or a policy: the table only picks the fastest
// launch.  mdp_build, mdp_solve and the batch use the table's entry for a
// model's class whenever the caller leaves the corresponding option at 0.
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "mdp_internal.cuh"

namespace mdpgb {

static std::mutex g_tune_mu;
static std::map<std::string, Tuning> g_tune;

static int64_t pow2_round(int64_t x) {   // nearest power of two (ties up)
  if (x <= 1) return 1;
  int64_t p = 1;
  while (p * 2 <= x) p *= 2;
  return (x - p < 2 * p - x) ? p : 2 * p;
}

std::string tuning_key(int A_pad, int K, int N, int64_t Nc, int n_obj, int precision) {
  char buf[96];
  snprintf(buf, sizeof buf, "A%d_K%d_N%lld_Nc%lld_o%d_%s", A_pad, K, (long long)pow2_round(N),
           (long long)pow2_round(Nc), n_obj, precision == MDP_FP64_CHECK ? "fp64" : "fp32");
  return buf;
}

bool tuning_lookup(const std::string &key, Tuning *out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

static void tuning_store(const std::string &key, const Tuning &t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = t;
}

static void tuning_erase(const std::string &key) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.erase(key);
}

// ------------------------------------------------------------------- JSON --
// The file is one object of objects of integers:
//   {"<class>": {"build_warps": 8, "hist_cap": 2048, ...}, ...}
static const char *kFields[] = {"build_warps", "hist_cap", "threads", "chunk", "sweep_smem_kb"};

static int32_t *field_of(Tuning &t, const std::string &name) {
  if (name == "build_warps") return &t.build_warps;
  if (name == "hist_cap") return &t.hist_cap;
  if (name == "threads") return &t.threads;
  if (name == "chunk") return &t.chunk;
  if (name == "sweep_smem_kb") return &t.sweep_smem_kb;
  return nullptr;
}

// Shapes the kernels accept (an edited file cannot ask for a launch that fails).
static bool tuning_valid(const Tuning &t) {
  return (t.build_warps == 4 || t.build_warps == 8) && t.hist_cap >= 256 && t.hist_cap <= 6144 &&
         t.threads >= 64 && t.threads <= 512 && t.threads % 64 == 0 && t.chunk >= 32 && t.chunk <= 8192 &&
         t.sweep_smem_kb >= 64 && t.sweep_smem_kb <= 220;
}

namespace {
struct Lexer {
  const std::string &s;
  size_t i = 0;
  explicit Lexer(const std::string &x) : s(x) {}
  void ws() {
    while (i < s.size() && isspace((unsigned char)s[i])) ++i;
  }
  bool eat(char c) {
    ws();
    if (i < s.size() && s[i] == c) {
      ++i;
      return true;
    }
    return false;
  }
  bool str(std::string *out) {
    ws();
    if (i >= s.size() || s[i] != '"') return false;
    size_t j = s.find('"', i + 1);
    if (j == std::string::npos) return false;
    *out = s.substr(i + 1, j - i - 1);
    i = j + 1;
    return true;
  }
  bool num(long long *out) {
    ws();
    size_t j = i;
    if (j < s.size() && s[j] == '-') ++j;
    while (j < s.size() && isdigit((unsigned char)s[j])) ++j;
    if (j == i) return false;
    *out = std::stoll(s.substr(i, j - i));
    i = j;
    return true;
  }
};
}  // namespace

static bool parse_table(const std::string &text, std::map<std::string, Tuning> *out) {
  Lexer L(text);
  if (!L.eat('{')) return false;
  if (L.eat('}')) return true;
  for (;;) {
    std::string key;
    if (!L.str(&key) || !L.eat(':') || !L.eat('{')) return false;
    Tuning t;
    if (!L.eat('}')) {
      for (;;) {
        std::string name;
        long long v = 0;
        if (!L.str(&name) || !L.eat(':') || !L.num(&v)) return false;
        if (int32_t *f = field_of(t, name)) *f = (int32_t)v;
        if (L.eat('}')) break;
        if (!L.eat(',')) return false;
      }
    }
    if (tuning_valid(t)) (*out)[key] = t;
    if (L.eat('}')) return true;
    if (!L.eat(',')) return false;
  }
}

static std::string format_table(const std::map<std::string, Tuning> &tab) {
  std::ostringstream o;
  o << "{\n";
  size_t n = 0;
  for (const auto &kv : tab) {
    Tuning t = kv.second;
    o << "  \"" << kv.first << "\": {";
    for (size_t f = 0; f < sizeof(kFields) / sizeof(kFields[0]); ++f)
      o << (f ? ", " : "") << "\"" << kFields[f] << "\": " << *field_of(t, kFields[f]);
    o << "}" << (++n < tab.size() ? "," : "") << "\n";
  }
  o << "}\n";
  return o.str();
}

static mdp_status load_file(const char *path, std::map<std::string, Tuning> *out, bool must_exist) {
  std::ifstream f(path);
  if (!f) {
    if (!must_exist) return MDP_OK;
    set_error(std::string("cannot read tuning file ") + path);
    return MDP_ERR_ARG;
  }
  std::stringstream ss;
  ss << f.rdbuf();
  if (!parse_table(ss.str(), out)) {
    set_error(std::string("tuning file is not a table of launch shapes: ") + path);
    return MDP_ERR_ARG;
  }
  return MDP_OK;
}

}  // namespace mdpgb

using namespace mdpgb;

extern "C" mdp_status mdp_tuning_load(const char *json_path) {
  if (!json_path) {
    set_error("invalid argument: NULL path");
    return MDP_ERR_ARG;
  }
  std::map<std::string, Tuning> tab;
  mdp_status s = load_file(json_path, &tab, true);
  if (s != MDP_OK) return s;
  for (const auto &kv : tab) tuning_store(kv.first, kv.second);
  return MDP_OK;
}

extern "C" mdp_status mdp_autotune(const mdp_env *env, const mdp_grid *grid, const mdp_actions *actions,
                                   int32_t N, int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj,
                                   const char *json_path, void *stream, mdp_tuning *out) {
  if (!env || !grid || !actions || !objs_h || n_obj < 1 || n_obj > 3) {
    set_error("invalid argument: NULL env/grid/actions/objs or n_obj outside 1..3");
    return MDP_ERR_ARG;
  }
  if (grid->nx < 1 || grid->ny < 1 || grid->nt < 1) {
    set_error("invalid argument: grid sizes must be >= 1");
    return MDP_ERR_ARG;
  }
  const int A = actions->n_headings * actions->n_speeds;
  int A_pad = 1;
  while (A_pad < A) A_pad <<= 1;
  const int64_t Nc = (int64_t)grid->nx * grid->ny;
  const std::string key = tuning_key(A_pad, env->K, N, Nc, n_obj, env->precision);
  // calibration cut: about 400,000 states of layers from the middle of the
  // horizon (the fields, masks and coefficients are layer-major, so the cut is
  // the caller's pointers advanced by t0 layers)
  mdp_grid g = *grid;
  g.nt = (int32_t)std::min<int64_t>(grid->nt, std::max<int64_t>(2, (400000 + Nc - 1) / Nc));
  const int64_t t0 = (grid->nt - g.nt) / 2;
  const size_t fsz0 = env->precision == MDP_FP64_CHECK ? 8 : 4;
  mdp_env ce_env = *env;
  ce_env.vbar = static_cast<const char *>(env->vbar) + fsz0 * 2 * (size_t)(t0 * Nc);
  if (env->modes) ce_env.modes = static_cast<const char *>(env->modes) + fsz0 * 2 * (size_t)(t0 * env->K * Nc);
  if (env->coeffs) ce_env.coeffs = static_cast<const char *>(env->coeffs) + fsz0 * (size_t)(t0 * N * env->K);
  if (env->gbar) ce_env.gbar = static_cast<const char *>(env->gbar) + fsz0 * (size_t)(t0 * Nc);
  ce_env.obstacle = env->obstacle + (size_t)(t0 * Nc);
  env = &ce_env;
  cudaStream_t st = (cudaStream_t)stream;
  Tuning prev;
  const bool had = tuning_lookup(key, &prev);
  std::vector<int32_t> objs(objs_h, objs_h + n_obj);
  auto restore = [&]() {
    if (had) tuning_store(key, prev);
    else tuning_erase(key);
  };
  // one calibration build with the candidate's shapes (read from the table)
  auto build_with = [&](const Tuning &t, mdp_model *m) -> mdp_status {
    tuning_store(key, t);
    return mdp_build(env, &g, actions, N, subgrid_L, objs.data(), n_obj, nullptr, stream, m);
  };
  Tuning best;
  double best_build = 1e300;
  int timed = 0;
  int64_t deferred = 0;
  for (int warps : {8, 4}) {
    for (int cap : {2048, 1536, 3072, 4096}) {
      Tuning t;
      t.build_warps = warps;
      t.hist_cap = cap;
      double ms = 1e300;
      for (int rep = 0; rep < 2; ++rep) {
        mdp_model m = nullptr;
        mdp_status s = build_with(t, &m);
        if (s != MDP_OK) {
          restore();
          return s;
        }
        ms = std::min(ms, m->kernel_ms);
        if (warps == 8 && cap == 2048) deferred = m->deferred;
        mdp_model_free(m);
      }
      ++timed;
      if (ms < best_build) {
        best_build = ms;
        best.build_warps = warps;
        best.hist_cap = cap;
      }
    }
  }
  if (deferred > 0) {   // the full-window kernel has work: tune its CTA size too
    double best_t = 1e300;
    for (int th : {256, 128, 512}) {
      Tuning t = best;
      t.threads = th;
      mdp_model m = nullptr;
      mdp_status s = build_with(t, &m);
      if (s != MDP_OK) {
        restore();
        return s;
      }
      ++timed;
      if (m->kernel_ms < best_t) {
        best_t = m->kernel_ms;
        best.threads = th;
      }
      mdp_model_free(m);
    }
  }
  // the Bellman sweep's shared memory, on one calibration model (fused
  // objectives, a few Jacobi sweeps)
  mdp_model m = nullptr;
  mdp_status s = build_with(best, &m);
  if (s != MDP_OK) {
    restore();
    return s;
  }
  double best_sweep = 1e300;
  const size_t fsz = env->precision == MDP_FP64_CHECK ? 8 : 4;
  std::vector<void *> V(n_obj, nullptr);
  std::vector<int16_t *> P(n_obj, nullptr);
  cudaError_t ce = cudaSuccess;
  for (int o = 0; o < n_obj && ce == cudaSuccess; ++o) {
    ce = dev_alloc(&V[o], fsz * (size_t)(m->nS + 1), st);
    if (ce == cudaSuccess) ce = dev_alloc((void **)&P[o], 2 * (size_t)m->nS, st);
  }
  if (ce == cudaSuccess && m->spw == 1) {
    std::vector<int32_t> slots(n_obj);
    for (int o = 0; o < n_obj; ++o) slots[o] = o;
    for (int kb : {160, 132, 190}) {
      m->sweep_smem_kb = kb;
      double ms = 1e300;
      for (int rep = 0; rep < 3 && s == MDP_OK; ++rep) {
        std::vector<mdp_solve_stats> sts(n_obj);
        s = mdp_solve_multi(m, n_obj, slots.data(), MDP_SOLVE_JACOBI_FULL, 0.0, std::min(4, g.nt + 1), V.data(),
                            P.data(), stream, sts.data());
        ms = std::min(ms, sts[0].solve_ms);
      }
      if (s != MDP_OK) break;
      ++timed;
      if (ms < best_sweep) {
        best_sweep = ms;
        best.sweep_smem_kb = kb;
      }
    }
  }
  for (int o = 0; o < n_obj; ++o) {
    dev_free(V[o], st);
    dev_free(P[o], st);
  }
  mdp_model_free(m);
  if (ce != cudaSuccess) {
    restore();
    return cuda_fail(ce, "mdp_autotune");
  }
  if (s != MDP_OK) {
    restore();
    return s;
  }
  tuning_store(key, best);
  if (json_path) {   // merge into the file: its other classes stay
    std::map<std::string, Tuning> tab;
    s = load_file(json_path, &tab, false);
    if (s != MDP_OK) return s;
    tab[key] = best;
    const std::string tmp = std::string(json_path) + ".tmp";
    {
      std::ofstream f(tmp);
      f << format_table(tab);
      if (!f) {
        set_error(std::string("cannot write tuning file ") + json_path);
        return MDP_ERR_ARG;
      }
    }
    if (std::rename(tmp.c_str(), json_path) != 0) {
      set_error(std::string("cannot write tuning file ") + json_path);
      return MDP_ERR_ARG;
    }
  }
  if (out) {
    memset(out, 0, sizeof(*out));
    out->build_warps = best.build_warps;
    out->hist_cap = best.hist_cap;
    out->threads = best.threads;
    out->chunk = best.chunk;
    out->sweep_smem_kb = best.sweep_smem_kb;
    out->build_kernel_ms = best_build;
    out->sweep_ms = best_sweep < 1e299 ? best_sweep : 0.0;
    out->candidates = timed;
    out->calibration_layers = g.nt;
    snprintf(out->key, sizeof out->key, "%s", key.c_str());
  }
  return MDP_OK;
}
