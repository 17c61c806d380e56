/*
 * oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Follows the paper's steps in its order and notation:
 *   - DO velocity v = vbar + mu_i v~_i                      (Sec. II-C)
 *   - kinematics x' = x + (v + a) dt, t' = t + dt, s' = cell(x', t')
 *                                                           (Sec. II-A)
 *   - Monte-Carlo counting of successors, P = count / N     (Sec. II-A, Sec. III-B/C)
 *   - one-step rewards: time -dt, energy -c_f F^2 dt, net energy
 *     [-c_f F^2 + c_r (g(s) + g(s'))/2] dt with the mean scalar field,
 *     r_term on reaching the target, r_outbound for obstacle / outside /
 *     beyond the horizon                                    (Eqs. Rsa_time, Rsa_energyConsumption,
 *                                                            Rsa_NetEnergy; Sec. III-A theorem)
 *   - K_TRANSITION per-sample classification and counting (Alg. 2),
 *     K_COMPUTE_MEAN sum_R / N, K_COUNT / K_REDUCE_TO_COO    (Sec. III-C)
 *   - value iteration v_{k+1}(s) = max_a sum P [r + v_k(s')] and the greedy
 *     policy                                                (Sec. II-B)
 * Compile: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox -- */
/* Multipliers and Weyl key increments of Philox4x64 as published by
 * Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
 * (SC'11), Sec. 4 and Table 2. */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 prod = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(prod >> 64);
  *lo = (uint64_t)prod;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: bump the key between rounds */
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(PHILOX_M0, x0, &hi0, &lo0);
    mulhilo64(PHILOX_M1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 53-bit uniform in [0, 1) from the top 53 bits of a 64-bit word (exact). */
static double u01(uint64_t x) { return (double)(x >> 11) * 0x1p-53; }

/* ------------------------------------------------------------------- log -- */
/* ln s = e ln2 + 2 atanh((m-1)/(m+1)), s = m 2^e, m in [sqrt(1/2), sqrt(2)).
 * atanh(z) = sum_{n>=0} z^(2n+1)/(2n+1) (Abramowitz & Stegun 4.1.27); |z| <=
 * 0.1716 so twelve terms reach far below one ulp. */
#define ORC_LN2 0x1.62e42fefa39efp-1        /* ln 2 rounded to binary64 */
#define ORC_SQRT_HALF 0x1.6a09e667f3bcdp-1  /* sqrt(1/2) rounded to binary64 */
#define ORC_LN_TERMS 12

double orc_ln(double s) {
  int e;
  double m = frexp(s, &e); /* s = m * 2^e, m in [0.5, 1) -- exact */
  if (m < ORC_SQRT_HALF) {
    m = m * 2.0;
    e = e - 1;
  }
  double z = (m - 1.0) / (m + 1.0);
  double z2 = z * z;
  double poly = 1.0 / (double)(2 * (ORC_LN_TERMS - 1) + 1);
  for (int n = ORC_LN_TERMS - 2; n >= 0; --n) poly = poly * z2 + 1.0 / (double)(2 * n + 1);
  return (double)e * ORC_LN2 + 2.0 * (z * poly);
}

/* ----------------------------------------------------------- polar pairs -- */
#define ORC_MAX_ATTEMPTS 64

int orc_polar_pair(uint64_t seed, uint64_t mdp_id, uint64_t t, uint64_t w, uint64_t j,
                   double *z1, double *z2) {
  const uint64_t key[2] = {seed, mdp_id};
  for (uint64_t attempt = 0; attempt < ORC_MAX_ATTEMPTS; ++attempt) {
    const uint64_t ctr[4] = {t, w, j, attempt};
    uint64_t r[4];
    orc_philox4x64_10(ctr, key, r);
    double v1 = 2.0 * u01(r[0]) - 1.0;
    double v2 = 2.0 * u01(r[1]) - 1.0;
    double s = v1 * v1 + v2 * v2;
    if (s < 1.0 && s > 0.0) { /* Marsaglia & Bray (1964) polar method */
      double f = sqrt((-2.0 * orc_ln(s)) / s);
      *z1 = v1 * f;
      *z2 = v2 * f;
      return (int)attempt + 1;
    }
  }
  *z1 = 0.0;
  *z2 = 0.0;
  return 0;
}

int64_t orc_sample_coeffs(int32_t nt, int32_t N, int32_t K, const double *sigma,
                          uint64_t seed, uint64_t mdp_id, double *Y) {
  int64_t capped = 0;
  const int32_t pairs = (K + 1) / 2;
  for (int32_t t = 0; t < nt; ++t)
    for (int32_t w = 0; w < N; ++w)
      for (int32_t j = 0; j < pairs; ++j) {
        double z1, z2;
        if (orc_polar_pair(seed, mdp_id, (uint64_t)t, (uint64_t)w, (uint64_t)j, &z1, &z2) == 0)
          ++capped;
        double *y = Y + ((int64_t)t * N + w) * K;
        y[2 * j] = sigma[2 * j] * z1;
        if (2 * j + 1 < K) y[2 * j + 1] = sigma[2 * j + 1] * z2;
      }
  return capped;
}

/* ----------------------------------------------------------------- build -- */
/* One-step reward for a landing inside the domain and free of obstacles
 * (Eqs. Rsa_time, Rsa_energyConsumption, Rsa_NetEnergy; the net-energy
 * reward uses only the mean scalar field, Sec. III-A), plus r_term when the
 * landing cell is a target (Sec. II-A). */
static double step_reward(const orc_problem *p, int32_t obj, double F, double g_s, double g_sp,
                          int is_target) {
  double r;
  if (obj == ORC_OBJ_TIME) {
    r = -p->dt;
  } else if (obj == ORC_OBJ_ENERGY) {
    double eF = p->c_f * F * F;
    r = -eF * p->dt;
  } else {
    double eF = p->c_f * F * F;
    double half_cr = 0.5 * p->c_r;
    r = ((-eF + half_cr * g_s) + half_cr * g_sp) * p->dt;
  }
  if (is_target) r = r + p->r_term;
  return r;
}

int orc_build(const orc_problem *p, int64_t u_begin, int64_t u_end, int32_t max_nnz,
              const int32_t *objs, int32_t n_obj, int32_t *nnz, int64_t *col, int32_t *cnt,
              double *R, double *R_lit, int64_t *overflow) {
  if (p->L < 1 || (p->L % 2) == 0 || p->A < 1 || p->N < 1 || n_obj < 1 || n_obj > 3) return -2;
  for (int32_t o = 0; o < n_obj; ++o)
    if (objs[o] < 0 || objs[o] > 2 || (objs[o] == ORC_OBJ_NET_ENERGY && p->gbar == NULL)) return -2;
  const int64_t Nx = p->nx, Ny = p->ny, Nt = p->nt, Nc = Nx * Ny, nS = Nt * Nc;
  const int32_t L = p->L, h = (L - 1) / 2, A = p->A, K = p->K, N = p->N;
  const int64_t rows = (u_end - u_begin) * A;
  int32_t *hist = (int32_t *)malloc(sizeof(int32_t) * (size_t)L * (size_t)L);
  double *sumR = (double *)malloc(sizeof(double) * (size_t)n_obj);
  if (!hist || !sumR) { free(hist); free(sumR); return -2; }
  int status = 0;
  *overflow = 0;

  for (int64_t u = u_begin; u < u_end && status == 0; ++u) {
    const int64_t t = u / Nc, c = u % Nc, i = c % Nx, j = c / Nx;
    const int64_t s = t * Nc + c;
    const int start_terminal = p->target[c] != 0;
    const int start_obstacle = p->obstacle[s] != 0;
    const int horizon = (t == Nt - 1);
    for (int32_t a = 0; a < A; ++a) {
      const int64_t lr = (u - u_begin) * A + a;
      int64_t *rc = col + lr * max_nnz;
      int32_t *rn = cnt + lr * max_nnz;
      if (start_terminal) { /* terminal states are absorbing: no transitions */
        nnz[lr] = 0;
        for (int32_t o = 0; o < n_obj; ++o) {
          R[o * rows + lr] = 0.0;
          if (R_lit) R_lit[o * rows + lr] = 0.0;
        }
        continue;
      }
      if (start_obstacle || horizon) { /* every realization ends in the sink */
        if (max_nnz < 1) { status = -1; break; }
        nnz[lr] = 1;
        rc[0] = nS;
        rn[0] = N;
        for (int32_t o = 0; o < n_obj; ++o) {
          R[o * rows + lr] = ((double)N / (double)N) * p->r_outbound;
          if (R_lit) {
            double acc = 0.0;
            for (int32_t w = 0; w < N; ++w) acc = acc + p->r_outbound;
            R_lit[o * rows + lr] = acc / (double)N;
          }
        }
        continue;
      }
      const double dxa = p->act[3 * a + 0], dya = p->act[3 * a + 1], F = p->act[3 * a + 2];
      memset(hist, 0, sizeof(int32_t) * (size_t)L * (size_t)L);
      int32_t sink = 0;
      for (int32_t o = 0; o < n_obj; ++o) sumR[o] = 0.0;
      const double g_s = p->gbar ? p->gbar[s] : 0.0;
      for (int32_t w = 0; w < N; ++w) {
        /* v(s; w) = vbar + sum_k Y_k v~_k, modes in ascending order */
        double vx = p->vbar[2 * s + 0], vy = p->vbar[2 * s + 1];
        const double *yw = p->Y + (t * N + w) * K;
        for (int32_t k = 0; k < K; ++k) {
          const double *phi = p->modes + 2 * ((t * K + k) * Nc + c);
          vx = vx + yw[k] * phi[0];
          vy = vy + yw[k] * phi[1];
        }
        /* move: x' = x + (v + a) dt from the cell centre, cell() = floor(x'/dx) */
        const double x = ((double)i + 0.5) * p->dx, y = ((double)j + 0.5) * p->dx;
        const double xp = x + (vx + dxa) * p->dt, yp = y + (vy + dya) * p->dt;
        const int64_t ip = (int64_t)floor(xp / p->dx), jp = (int64_t)floor(yp / p->dx);
        const int64_t di = ip - i, dj = jp - j;
        if (di < -h || di > h || dj < -h || dj > h) { /* outside the neighbouring sub-grid */
          ++*overflow;
          continue;
        }
        if (ip < 0 || ip >= Nx || jp < 0 || jp >= Ny || p->obstacle[(t + 1) * Nc + jp * Nx + ip]) {
          ++sink;
          for (int32_t o = 0; o < n_obj; ++o) sumR[o] = sumR[o] + p->r_outbound;
          continue;
        }
        ++hist[(dj + h) * L + (di + h)];
        const int is_t = p->target[jp * Nx + ip] != 0;
        const double g_sp = p->gbar ? p->gbar[(t + 1) * Nc + jp * Nx + ip] : 0.0;
        for (int32_t o = 0; o < n_obj; ++o)
          sumR[o] = sumR[o] + step_reward(p, objs[o], F, g_s, g_sp, is_t);
      }
      /* K_COUNT / K_REDUCE_TO_COO: nonzero sub-grid cells in ascending order, sink last */
      int32_t e = 0;
      for (int32_t o = 0; o < n_obj; ++o) R[o * rows + lr] = 0.0;
      for (int32_t b = 0; b < L * L; ++b) {
        if (hist[b] == 0) continue;
        if (e >= max_nnz) { status = -1; break; }
        const int64_t dj = b / L - h, di = b % L - h;
        const int64_t ip = i + di, jp = j + dj;
        rc[e] = (t + 1) * Nc + jp * Nx + ip;
        rn[e] = hist[b];
        const int is_t = p->target[jp * Nx + ip] != 0;
        const double g_sp = p->gbar ? p->gbar[(t + 1) * Nc + jp * Nx + ip] : 0.0;
        const double prob = (double)hist[b] / (double)N;
        for (int32_t o = 0; o < n_obj; ++o)
          R[o * rows + lr] = R[o * rows + lr] + prob * step_reward(p, objs[o], F, g_s, g_sp, is_t);
        ++e;
      }
      if (status != 0) break;
      if (sink > 0) {
        if (e >= max_nnz) { status = -1; break; }
        rc[e] = nS;
        rn[e] = sink;
        const double prob = (double)sink / (double)N;
        for (int32_t o = 0; o < n_obj; ++o)
          R[o * rows + lr] = R[o * rows + lr] + prob * p->r_outbound;
        ++e;
      }
      nnz[lr] = e;
      /* K_COMPUTE_MEAN: the paper's literal sample mean of the per-sample rewards */
      if (R_lit)
        for (int32_t o = 0; o < n_obj; ++o) R_lit[o * rows + lr] = sumR[o] / (double)N;
    }
  }
  free(hist);
  free(sumR);
  return status;
}

/* ------------------------------------------------------- value iteration -- */
/* Q(s,a) = R(s,a) + sum_j P(s'_j|s,a) V(s'_j), successors in stored order. */
static double q_value(int64_t r, const int64_t *rowptr, const int64_t *col, const double *prob,
                      const double *R, const double *V) {
  double acc = 0.0;
  for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) acc = acc + prob[e] * V[col[e]];
  return R[r] + acc;
}

/* max_a Q(s,a); the lowest action index wins exact ties. */
static double backup(int64_t s, int64_t nS, int32_t A, const int64_t *rowptr, const int64_t *col,
                     const double *prob, const double *R, const double *V, int32_t *arg) {
  double best = 0.0;
  int32_t best_a = -1;
  for (int32_t a = 0; a < A; ++a) {
    double q = q_value((int64_t)a * nS + s, rowptr, col, prob, R, V);
    if (best_a < 0 || q > best) {
      best = q;
      best_a = a;
    }
  }
  *arg = best_a;
  return best;
}

void orc_q_values(int64_t nS, int32_t A, const int64_t *rowptr, const int64_t *col,
                  const double *prob, const double *R, const double *V, double *Q) {
  for (int64_t r = 0; r < (int64_t)A * nS; ++r) Q[r] = q_value(r, rowptr, col, prob, R, V);
}

int orc_vi_jacobi(int64_t nS, int32_t A, const int64_t *rowptr, const int64_t *col,
                  const double *prob, const double *R, const uint8_t *fixed, const double *V0,
                  double tol, int32_t max_sweeps, double *V, int32_t *pi, int32_t *sweeps,
                  double *residual) {
  double *Vold = (double *)malloc(sizeof(double) * (size_t)(nS + 1));
  if (!Vold) return -2;
  /* v_0: the caller's values (V0 != NULL) or 0 everywhere; V(sink) = 0 always */
  for (int64_t s = 0; s <= nS; ++s) {
    const double v0 = (V0 && s < nS) ? V0[s] : 0.0;
    V[s] = v0;
    Vold[s] = v0;
  }
  int32_t k = 0;
  double res = 0.0;
  while (k < max_sweeps) {
    res = 0.0;
    for (int64_t s = 0; s < nS; ++s) {
      int32_t arg;
      V[s] = backup(s, nS, A, rowptr, col, prob, R, Vold, &arg);
      pi[s] = fixed[s] ? -1 : arg;
      double d = fabs(V[s] - Vold[s]);
      if (d > res) res = d;
    }
    ++k;
    memcpy(Vold, V, sizeof(double) * (size_t)(nS + 1));
    if (res <= tol) break;
  }
  *sweeps = k;
  *residual = res;
  free(Vold);
  return 0;
}

int orc_vi_backward(int64_t nS, int32_t A, int32_t nt, int64_t Nc, const int64_t *rowptr,
                    const int64_t *col, const double *prob, const double *R,
                    const uint8_t *fixed, double *V, int32_t *pi) {
  for (int64_t s = 0; s <= nS; ++s) V[s] = 0.0;
  for (int32_t t = nt - 1; t >= 0; --t)
    for (int64_t c = 0; c < Nc; ++c) {
      const int64_t s = (int64_t)t * Nc + c;
      int32_t arg;
      V[s] = backup(s, nS, A, rowptr, col, prob, R, V, &arg);
      pi[s] = fixed[s] ? -1 : arg;
    }
  return 0;
}

/* -------------------------------------------------------------- rollouts -- */
int orc_rollout(const orc_problem *p, const int32_t *policy, int32_t i0, int32_t j0,
                const int32_t *objs, int32_t n_obj, double *ret, int32_t *steps, int32_t *status,
                int64_t *traj) {
  if (n_obj < 1 || n_obj > 3 || p->N < 1 || p->nt < 1) return -2;
  if (i0 < 0 || i0 >= p->nx || j0 < 0 || j0 >= p->ny) return -2;
  for (int32_t o = 0; o < n_obj; ++o)
    if (objs[o] < 0 || objs[o] > 2 || (objs[o] == ORC_OBJ_NET_ENERGY && p->gbar == NULL)) return -2;
  const int64_t Nx = p->nx, Ny = p->ny, Nt = p->nt, Nc = Nx * Ny, nS = Nt * Nc;
  const int32_t K = p->K, N = p->N;
  for (int32_t w = 0; w < N; ++w) {
    double *rw = ret + (int64_t)w * n_obj;
    int64_t *tr = traj ? traj + (int64_t)w * (Nt + 1) : NULL;
    for (int32_t o = 0; o < n_obj; ++o) rw[o] = 0.0;
    if (tr)
      for (int64_t k = 0; k <= Nt; ++k) tr[k] = -1;
    int64_t i = i0, j = j0;
    int32_t n = 0, st = 1;
    if (tr) tr[0] = j * Nx + i;
    for (int64_t t = 0; t < Nt; ++t) {
      const int64_t c = j * Nx + i, s = t * Nc + c;
      if (p->target[c]) { /* arrived: terminal states are absorbing */
        st = 0;
        break;
      }
      const int32_t a = policy[s];
      if (p->obstacle[s] || t == Nt - 1 || a < 0) { /* every move ends in the sink */
        for (int32_t o = 0; o < n_obj; ++o) rw[o] = rw[o] + p->r_outbound;
        ++n;
        if (tr) tr[n] = nS;
        st = 1;
        break;
      }
      const double dxa = p->act[3 * a + 0], dya = p->act[3 * a + 1], F = p->act[3 * a + 2];
      /* realization w's velocity at this state and time: vbar + sum_k Y_k v~_k */
      double vx = p->vbar[2 * s + 0], vy = p->vbar[2 * s + 1];
      const double *yw = p->Y + (t * N + w) * K;
      for (int32_t k = 0; k < K; ++k) {
        const double *phi = p->modes + 2 * ((t * K + k) * Nc + c);
        vx = vx + yw[k] * phi[0];
        vy = vy + yw[k] * phi[1];
      }
      const double x = ((double)i + 0.5) * p->dx, y = ((double)j + 0.5) * p->dx;
      const double xp = x + (vx + dxa) * p->dt, yp = y + (vy + dya) * p->dt;
      const int64_t ip = (int64_t)floor(xp / p->dx), jp = (int64_t)floor(yp / p->dx);
      ++n;
      if (ip < 0 || ip >= Nx || jp < 0 || jp >= Ny || p->obstacle[(t + 1) * Nc + jp * Nx + ip]) {
        for (int32_t o = 0; o < n_obj; ++o) rw[o] = rw[o] + p->r_outbound;
        if (tr) tr[n] = nS;
        st = 1;
        break;
      }
      const int is_t = p->target[jp * Nx + ip] != 0;
      const double g_s = p->gbar ? p->gbar[s] : 0.0;
      const double g_sp = p->gbar ? p->gbar[(t + 1) * Nc + jp * Nx + ip] : 0.0;
      for (int32_t o = 0; o < n_obj; ++o) rw[o] = rw[o] + step_reward(p, objs[o], F, g_s, g_sp, is_t);
      i = ip;
      j = jp;
      if (tr) tr[n] = (t + 1) * Nc + jp * Nx + ip;
    }
    steps[w] = n;
    status[w] = st;
  }
  return 0;
}

/* -------------------------------------------------------------- 3-D grid -- */
/* The 3-D build: the 2-D steps with a third spatial component everywhere. */
static double step_reward3d(const orc_problem3d *p, int32_t obj, double F, double g_s, double g_sp,
                            int is_target) {
  double r;
  if (obj == ORC_OBJ_TIME) {
    r = -p->dt;
  } else if (obj == ORC_OBJ_ENERGY) {
    double eF = p->c_f * F * F;
    r = -eF * p->dt;
  } else {
    double eF = p->c_f * F * F;
    double half_cr = 0.5 * p->c_r;
    r = ((-eF + half_cr * g_s) + half_cr * g_sp) * p->dt;
  }
  if (is_target) r = r + p->r_term;
  return r;
}

int orc_build3d(const orc_problem3d *p, int64_t u_begin, int64_t u_end, int32_t max_nnz,
                const int32_t *objs, int32_t n_obj, int32_t *nnz, int64_t *col, int32_t *cnt,
                double *R, int64_t *overflow) {
  if (p->L < 1 || (p->L % 2) == 0 || p->A < 1 || p->N < 1 || n_obj < 1 || n_obj > 3) return -2;
  for (int32_t o = 0; o < n_obj; ++o)
    if (objs[o] < 0 || objs[o] > 2 || (objs[o] == ORC_OBJ_NET_ENERGY && p->gbar == NULL)) return -2;
  const int64_t Nx = p->nx, Ny = p->ny, Nz = p->nz, Nt = p->nt, Nc = Nx * Ny * Nz, nS = Nt * Nc;
  const int32_t L = p->L, h = (L - 1) / 2, A = p->A, K = p->K, N = p->N;
  const int64_t nb = (int64_t)L * L * L;
  const int64_t rows = (u_end - u_begin) * A;
  int32_t *hist = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
  if (!hist) return -2;
  int status = 0;
  *overflow = 0;
  for (int64_t u = u_begin; u < u_end && status == 0; ++u) {
    const int64_t t = u / Nc, c = u % Nc, i = c % Nx, j = (c / Nx) % Ny, k = c / (Nx * Ny);
    const int64_t s = t * Nc + c;
    const int start_terminal = p->target[c] != 0;
    const int start_obstacle = p->obstacle[s] != 0;
    const int horizon = (t == Nt - 1);
    for (int32_t a = 0; a < A; ++a) {
      const int64_t lr = (u - u_begin) * A + a;
      int64_t *rc = col + lr * max_nnz;
      int32_t *rn = cnt + lr * max_nnz;
      if (start_terminal) {
        nnz[lr] = 0;
        for (int32_t o = 0; o < n_obj; ++o) R[o * rows + lr] = 0.0;
        continue;
      }
      if (start_obstacle || horizon) {
        if (max_nnz < 1) { status = -1; break; }
        nnz[lr] = 1;
        rc[0] = nS;
        rn[0] = N;
        for (int32_t o = 0; o < n_obj; ++o) R[o * rows + lr] = ((double)N / (double)N) * p->r_outbound;
        continue;
      }
      const double dxa = p->act[4 * a + 0], dya = p->act[4 * a + 1], dza = p->act[4 * a + 2];
      const double F = p->act[4 * a + 3];
      memset(hist, 0, sizeof(int32_t) * (size_t)nb);
      int32_t sink = 0;
      const double g_s = p->gbar ? p->gbar[s] : 0.0;
      for (int32_t w = 0; w < N; ++w) {
        double vx = p->vbar[3 * s + 0], vy = p->vbar[3 * s + 1], vz = p->vbar[3 * s + 2];
        const double *yw = p->Y + (t * N + w) * K;
        for (int32_t q = 0; q < K; ++q) {
          const double *phi = p->modes + 3 * ((t * K + q) * Nc + c);
          vx = vx + yw[q] * phi[0];
          vy = vy + yw[q] * phi[1];
          vz = vz + yw[q] * phi[2];
        }
        const double x = ((double)i + 0.5) * p->dx, y = ((double)j + 0.5) * p->dx;
        const double z = ((double)k + 0.5) * p->dx;
        const double xp = x + (vx + dxa) * p->dt, yp = y + (vy + dya) * p->dt, zp = z + (vz + dza) * p->dt;
        const int64_t ip = (int64_t)floor(xp / p->dx), jp = (int64_t)floor(yp / p->dx);
        const int64_t kp = (int64_t)floor(zp / p->dx);
        const int64_t di = ip - i, dj = jp - j, dk = kp - k;
        if (di < -h || di > h || dj < -h || dj > h || dk < -h || dk > h) {
          ++*overflow;
          continue;
        }
        if (ip < 0 || ip >= Nx || jp < 0 || jp >= Ny || kp < 0 || kp >= Nz ||
            p->obstacle[(t + 1) * Nc + (kp * Ny + jp) * Nx + ip]) {
          ++sink;
          continue;
        }
        ++hist[((dk + h) * L + (dj + h)) * L + (di + h)];
      }
      int32_t e = 0;
      for (int32_t o = 0; o < n_obj; ++o) R[o * rows + lr] = 0.0;
      for (int64_t b = 0; b < nb; ++b) {
        if (hist[b] == 0) continue;
        if (e >= max_nnz) { status = -1; break; }
        const int64_t dk = b / ((int64_t)L * L) - h, dj = (b / L) % L - h, di = b % L - h;
        const int64_t ip = i + di, jp = j + dj, kp = k + dk;
        const int64_t cp = (kp * Ny + jp) * Nx + ip;
        rc[e] = (t + 1) * Nc + cp;
        rn[e] = hist[b];
        const int is_t = p->target[cp] != 0;
        const double g_sp = p->gbar ? p->gbar[(t + 1) * Nc + cp] : 0.0;
        const double prob = (double)hist[b] / (double)N;
        for (int32_t o = 0; o < n_obj; ++o)
          R[o * rows + lr] = R[o * rows + lr] + prob * step_reward3d(p, objs[o], F, g_s, g_sp, is_t);
        ++e;
      }
      if (status != 0) break;
      if (sink > 0) {
        if (e >= max_nnz) { status = -1; break; }
        rc[e] = nS;
        rn[e] = sink;
        const double prob = (double)sink / (double)N;
        for (int32_t o = 0; o < n_obj; ++o) R[o * rows + lr] = R[o * rows + lr] + prob * p->r_outbound;
        ++e;
      }
      nnz[lr] = e;
    }
  }
  free(hist);
  return status;
}
