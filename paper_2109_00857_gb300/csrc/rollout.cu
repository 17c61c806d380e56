// rollout.cu -- policy rollouts over the flow realizations (Sec. IV: the
// optimal policy applied to every realization from the start; the mean
// returns are the expected mission time, energy and net energy).
//
// One thread per path (start q, realization w).  Path w follows the policy
// from its start at t = 0 and moves with realization w's velocity of time t
// at its current state -- the build's own kinematics, so every move is one of
// the samples the build counted: FP32 lands with the same landing offsets as
// the FP32 build, FP64 check mode with the oracle's literal FP64 formulas.
// A path ends on a target cell (status 0, absorbing) or in the sink (status
// 1: a landing outside the domain or on an obstacle at t + 1, a move from the
// last layer, or a state without an action), which pays r_outbound.
#include <vector>

#include "build_common.cuh"

namespace mdpgb {

struct RolloutArgs {
  int32_t nx, ny, nt, K, N, n_obj, n_starts;
  int64_t Nc, nS;
  double dx, dt;
  float lam;
  const void *vbar, *modes, *Y, *gbar;
  const uint8_t *obstacle, *target;
  const int16_t *policy;
  const int32_t *starts;   // [n_starts][2] (i, j)
  ActionTable act;
  RewardParams rw;
  void *ret;               // [n_starts][N][n_obj]
  int32_t *steps;          // [n_starts][N]
  int8_t *status;          // [n_starts][N]
};

template <typename RT>
__global__ void __launch_bounds__(256) rollout_kernel(RolloutArgs a) {
  const int64_t path = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (path >= (int64_t)a.n_starts * a.N) return;
  const int q = (int)(path / a.N), w = (int)(path % a.N);
  const int64_t Nc = a.Nc;
  const RT *vbar = static_cast<const RT *>(a.vbar);
  const RT *modes = static_cast<const RT *>(a.modes);
  const RT *Y = static_cast<const RT *>(a.Y);
  const RT *gbar = static_cast<const RT *>(a.gbar);
  RT ret[3] = {0, 0, 0};
  int i = a.starts[2 * q], j = a.starts[2 * q + 1];
  int n = 0, st = 1;
  for (int t = 0; t < a.nt; ++t) {
    const int64_t c = (int64_t)j * a.nx + i, s = (int64_t)t * Nc + c;
    if (a.target[c]) {   // arrived: terminal states are absorbing
      st = 0;
      break;
    }
    const int act = a.policy[s];
    ++n;
    if (a.obstacle[s] || t == a.nt - 1 || act < 0) {   // every move ends in the sink
      for (int o = 0; o < a.n_obj; ++o) ret[o] += (RT)a.rw.r_out;
      break;
    }
    const RT *yw = Y + ((int64_t)t * a.N + w) * a.K;
    int ip, jp;
    if constexpr (sizeof(RT) == 4) {
      // the FP32 build's velocity and landing offsets (FMA chain over
      // ascending k, u = w dt/dx + 1/2, exact floor of u + d_a)
      float wx = vbar[2 * s], wy = vbar[2 * s + 1];
      for (int k = 0; k < a.K; ++k) {
        const float y = yw[k];
        const float *ph = reinterpret_cast<const float *>(modes) + 2 * (((int64_t)t * a.K + k) * Nc + c);
        wx = fmaf(y, ph[0], wx);
        wy = fmaf(y, ph[1], wy);
      }
      float ux = fmaf(wx, a.lam, 0.5f), uy = fmaf(wy, a.lam, 0.5f);
      if (!(fabsf(ux) < 1e30f)) ux = 1e30f;
      if (!(fabsf(uy) < 1e30f)) uy = 1e30f;
      const int di = land_offset(ux, a.act.cx[act], a.act.thx[act]);
      const int dj = land_offset(uy, a.act.cy[act], a.act.thy[act]);
      ip = i + di;
      jp = j + dj;
    } else {
      // the oracle's literal FP64 kinematics, round-to-nearest, no contraction
      double vx = vbar[2 * s], vy = vbar[2 * s + 1];
      for (int k = 0; k < a.K; ++k) {
        const double *ph = reinterpret_cast<const double *>(modes) + 2 * (((int64_t)t * a.K + k) * Nc + c);
        vx = __dadd_rn(vx, __dmul_rn(yw[k], ph[0]));
        vy = __dadd_rn(vy, __dmul_rn(yw[k], ph[1]));
      }
      const double x = __dmul_rn((double)i + 0.5, a.dx), y = __dmul_rn((double)j + 0.5, a.dx);
      const double xp = __dadd_rn(x, __dmul_rn(__dadd_rn(vx, a.act.dx64[act]), a.dt));
      const double yp = __dadd_rn(y, __dmul_rn(__dadd_rn(vy, a.act.dy64[act]), a.dt));
      const double fx = floor(__ddiv_rn(xp, a.dx)), fy = floor(__ddiv_rn(yp, a.dx));
      // far outside the grid the cell index does not fit an int: the sink
      ip = (fx >= 0.0 && fx < (double)a.nx) ? (int)fx : -1;
      jp = (fy >= 0.0 && fy < (double)a.ny) ? (int)fy : -1;
    }
    if (ip < 0 || ip >= a.nx || jp < 0 || jp >= a.ny ||
        a.obstacle[(int64_t)(t + 1) * Nc + (int64_t)jp * a.nx + ip]) {
      for (int o = 0; o < a.n_obj; ++o) ret[o] += (RT)a.rw.r_out;
      break;
    }
    const int64_t cp = (int64_t)jp * a.nx + ip;
    const bool is_t = a.target[cp] != 0;
    const RT g_s = gbar ? gbar[s] : (RT)0, g_sp = gbar ? gbar[(int64_t)(t + 1) * Nc + cp] : (RT)0;
    for (int o = 0; o < a.n_obj; ++o) {
      if constexpr (sizeof(RT) == 4)
        ret[o] += step_reward32(a.rw, a.rw.objs[o], a.act.F[act], g_s, g_sp, is_t);
      else
        ret[o] = __dadd_rn(ret[o], step_reward64(a.rw, a.rw.objs[o], a.act.F64[act], g_s, g_sp, is_t));
    }
    i = ip;
    j = jp;
  }
  if (a.ret)
    for (int o = 0; o < a.n_obj; ++o) static_cast<RT *>(a.ret)[path * a.n_obj + o] = ret[o];
  if (a.steps) a.steps[path] = n;
  if (a.status) a.status[path] = (int8_t)st;
}

// Per start (one block each): sums of the returns per objective, paths at a
// target and their steps, in FP64 (a fixed tree order: deterministic).
template <typename RT>
__global__ void rollout_summary_kernel(const RT *ret, const int32_t *steps, const int8_t *status, int N,
                                       int n_obj, double *out) {
  __shared__ double sh[256][5];
  const int q = blockIdx.x, tid = threadIdx.x;
  double acc[5] = {0, 0, 0, 0, 0};   // returns x3, arrivals, steps of arrivals
  for (int w = tid; w < N; w += blockDim.x) {
    const int64_t p = (int64_t)q * N + w;
    for (int o = 0; o < n_obj; ++o) acc[o] += (double)ret[p * n_obj + o];
    if (status[p] == 0) {
      acc[3] += 1.0;
      acc[4] += (double)steps[p];
    }
  }
  for (int v = 0; v < 5; ++v) sh[tid][v] = acc[v];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (tid < h)
      for (int v = 0; v < 5; ++v) sh[tid][v] += sh[tid + h][v];
    __syncthreads();
  }
  if (tid < 5) out[q * 5 + tid] = sh[0][tid];
}

}  // namespace mdpgb

using namespace mdpgb;

static mdp_status rollout_arg_fail(const char *msg) {
  set_error(std::string("invalid argument: ") + msg);
  return MDP_ERR_ARG;
}

extern "C" mdp_status mdp_rollout(const mdp_env *env, const mdp_grid *grid, const mdp_actions *actions,
                                  int32_t N, const int16_t *policy, const int32_t *starts_h, int32_t n_starts,
                                  const int32_t *objs_h, int32_t n_obj, void *ret, int32_t *steps,
                                  int8_t *status, mdp_rollout_summary *summary_h, void *stream) {
  mdp_status s = check_device();
  if (s != MDP_OK) return s;
  if (!env || !grid || !actions || !policy || !starts_h || !objs_h) return rollout_arg_fail("NULL pointer");
  if (grid->nx < 1 || grid->ny < 1 || grid->nt < 1 || !(grid->dx > 0) || !(grid->dt > 0))
    return rollout_arg_fail("grid");
  if (N < 1 || N > 65535) return rollout_arg_fail("N must be in [1, 65535]");
  if (n_starts < 1 || n_obj < 1 || n_obj > 3) return rollout_arg_fail("n_starts >= 1, n_obj in [1, 3]");
  if (env->K < 0 || env->K > kMaxModes) return rollout_arg_fail("K");
  if (env->precision != MDP_FP32 && env->precision != MDP_FP64_CHECK) return rollout_arg_fail("precision");
  if (!env->vbar || !env->obstacle || !env->target || (env->K > 0 && !env->modes))
    return rollout_arg_fail("vbar, modes, obstacle and target must be non-NULL");
  if (env->K > 0 && !env->coeffs && !env->sigma_h) return rollout_arg_fail("need coeffs or sigma_h");
  for (int o = 0; o < n_obj; ++o) {
    if (objs_h[o] < 0 || objs_h[o] > 2) return rollout_arg_fail("unknown objective");
    if (objs_h[o] == MDP_OBJ_NET_ENERGY && !env->gbar) return rollout_arg_fail("net energy needs gbar");
  }
  for (int q = 0; q < n_starts; ++q)
    if (starts_h[2 * q] < 0 || starts_h[2 * q] >= grid->nx || starts_h[2 * q + 1] < 0 ||
        starts_h[2 * q + 1] >= grid->ny)
      return rollout_arg_fail("start cell outside the grid");
  const int64_t paths = (int64_t)n_starts * N;
  if (paths > ((int64_t)1 << 31)) return rollout_arg_fail("n_starts * N above 2^31");
  const int prec = env->precision;
  const size_t fsz = prec == MDP_FP64_CHECK ? 8 : 4;
  RolloutArgs a{};
  int A = 0;
  s = make_actions(actions, grid->dt / grid->dx, &a.act, &A);
  if (s != MDP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  a.nx = grid->nx; a.ny = grid->ny; a.nt = grid->nt; a.K = env->K; a.N = N; a.n_obj = n_obj;
  a.n_starts = n_starts;
  a.Nc = (int64_t)grid->nx * grid->ny;
  a.nS = a.Nc * grid->nt;
  a.dx = grid->dx; a.dt = grid->dt; a.lam = (float)(grid->dt / grid->dx);
  a.vbar = env->vbar; a.modes = env->modes; a.gbar = env->gbar;
  a.obstacle = env->obstacle; a.target = env->target; a.policy = policy;
  a.rw.c_f = actions->c_f; a.rw.c_r = actions->c_r; a.rw.r_term = actions->r_term;
  a.rw.r_out = actions->r_outbound; a.rw.dt = grid->dt; a.rw.dx = grid->dx; a.rw.n_obj = n_obj;
  for (int o = 0; o < n_obj; ++o) a.rw.objs[o] = objs_h[o];
  // scratch: starts, own coefficient table (when drawn here), outputs the
  // caller did not ask for but the summary needs
  const bool own_ret = !ret, own_steps = !steps, own_status = !status;
  const bool need_all = summary_h != nullptr;
  void *buf[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  auto release = [&]() {
    for (void *p : buf) dev_free(p, st);
  };
  cudaError_t ce = dev_alloc(&buf[0], sizeof(int32_t) * 2 * (size_t)n_starts, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(buf[0], starts_h, sizeof(int32_t) * 2 * (size_t)n_starts, cudaMemcpyHostToDevice, st);
  a.starts = static_cast<const int32_t *>(buf[0]);
  a.Y = env->coeffs;
  if (ce == cudaSuccess && !env->coeffs && env->K > 0) {
    ce = dev_alloc(&buf[1], fsz * (size_t)grid->nt * N * env->K, st);
    double *sig = nullptr;
    if (ce == cudaSuccess) ce = dev_alloc((void **)&sig, sizeof(double) * env->K, st);
    buf[5] = sig;
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(sig, env->sigma_h, sizeof(double) * env->K, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = dev_alloc(&buf[6], sizeof(unsigned long long), st);   // capped draws
    if (ce == cudaSuccess) ce = cudaMemsetAsync(buf[6], 0, sizeof(unsigned long long), st);
    if (ce == cudaSuccess)
      ce = launch_sample_coeffs(grid->nt, N, env->K, sig, env->seed, env->mdp_id,
                                prec == MDP_FP64_CHECK ? (double *)buf[1] : nullptr,
                                prec == MDP_FP32 ? (float *)buf[1] : nullptr,
                                static_cast<unsigned long long *>(buf[6]), st);
    a.Y = buf[1];
  }
  if (ce == cudaSuccess && need_all && own_ret) ce = dev_alloc(&buf[2], fsz * (size_t)paths * n_obj, st);
  if (ce == cudaSuccess && need_all && own_steps) ce = dev_alloc(&buf[3], sizeof(int32_t) * (size_t)paths, st);
  if (ce == cudaSuccess && need_all && own_status) ce = dev_alloc(&buf[4], (size_t)paths, st);
  if (ce != cudaSuccess) {
    release();
    return cuda_fail(ce, "mdp_rollout set-up");
  }
  a.ret = ret ? ret : buf[2];
  a.steps = steps ? steps : static_cast<int32_t *>(buf[3]);
  a.status = status ? status : static_cast<int8_t *>(buf[4]);
  const unsigned blocks = (unsigned)((paths + 255) / 256);
  if (prec == MDP_FP64_CHECK) rollout_kernel<double><<<blocks, 256, 0, st>>>(a);
  else rollout_kernel<float><<<blocks, 256, 0, st>>>(a);
  ce = cudaGetLastError();
  std::vector<double> sums;
  if (ce == cudaSuccess && need_all) {
    double *sd = nullptr;
    ce = dev_alloc((void **)&sd, sizeof(double) * 5 * (size_t)n_starts, st);
    if (ce == cudaSuccess) {
      if (prec == MDP_FP64_CHECK)
        rollout_summary_kernel<double><<<n_starts, 256, 0, st>>>(static_cast<const double *>(a.ret), a.steps,
                                                                 a.status, N, n_obj, sd);
      else
        rollout_summary_kernel<float><<<n_starts, 256, 0, st>>>(static_cast<const float *>(a.ret), a.steps,
                                                                a.status, N, n_obj, sd);
      ce = cudaGetLastError();
      sums.resize(5 * (size_t)n_starts);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sums.data(), sd, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, st);
      dev_free(sd, st);
    }
  }
  release();
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "mdp_rollout");
  if (need_all) {
    for (int q = 0; q < n_starts; ++q) {
      const double *v = &sums[5 * (size_t)q];
      mdp_rollout_summary &o = summary_h[q];
      for (int k = 0; k < 3; ++k) o.mean_return[k] = k < n_obj ? v[k] / N : 0.0;
      o.p_target = v[3] / N;
      o.mean_steps_target = v[3] > 0 ? v[4] / v[3] : 0.0;
      o.paths = N;
    }
  }
  return MDP_OK;
}
