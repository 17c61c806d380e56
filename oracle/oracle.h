/*
 * oracle.h -- plain, slow FP64 CPU oracle for the MDP build and value iteration
 * of Chowdhury & Subramani, "Optimal Path Planning of Autonomous Marine
 * Vehicles in Stochastic Dynamic Ocean Flows using a GPU-Accelerated
 * Algorithm" (arXiv 2109.00857).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or constant table with the
 * CUDA library.
 *
 * Conventions (the readings of the paper this oracle takes):
 *   state index      s = t*Nc + j*Nx + i  (Nc = Nx*Ny), sink = |S| = Nt*Nc
 *   row index        paper layout, rows appended over actions: r = a*|S| + s
 *   sub-grid bin     b = (dj+h)*L + (di+h), h = (L-1)/2
 *   coefficients     Y[t][w][k]  (t < Nt, w < N realizations, k < K modes)
 *   fields           vbar[t][j][i][2], modes[t][k][j][i][2], gbar[t][j][i],
 *                    obstacle[t][j][i] (u8), target[j][i] (u8)
 *   actions          act[a][3] = (d_x, d_y, F): the action's velocity
 *                    components and speed (heading/speed table, Sec. II-A)
 *
 * Every function is single-threaded; floating point is IEEE binary64 with no
 * contraction (compile with -O2 -ffp-contract=off, no -ffast-math).
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OBJ_TIME = 0, ORC_OBJ_ENERGY = 1, ORC_OBJ_NET_ENERGY = 2 };

typedef struct {
  int32_t nx, ny, nt;          /* grid sizes */
  double dx, dt;               /* cell side and time step */
  int32_t K, N;                /* DO modes, velocity realizations */
  int32_t A;                   /* actions */
  int32_t L;                   /* neighbouring sub-grid side (odd) */
  const double *vbar;          /* [nt][ny][nx][2] DO mean */
  const double *modes;         /* [nt][K][ny][nx][2] DO modes */
  const double *Y;             /* [nt][N][K] DO coefficients */
  const double *gbar;          /* [nt][ny][nx] mean scalar field (may be NULL) */
  const uint8_t *obstacle;     /* [nt][ny][nx] dynamic obstacle mask */
  const uint8_t *target;       /* [ny][nx] terminal (target) cells */
  const double *act;           /* [A][3] (d_x, d_y, F) */
  double c_f, c_r, r_term, r_outbound;
} orc_problem;

/* Philox4x64-10 block function (Salmon et al., SC'11): out = bijection of ctr under key. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Natural log from + - * / only (frexp range reduction, atanh series,
 * Abramowitz & Stegun 4.1.27).  Defined for finite s > 0. */
double orc_ln(double s);

/* Marsaglia polar pair for (t, w, pair j) under (seed, mdp_id).  Returns the
 * number of attempts used (0 if the attempt cap was hit; z1 = z2 = 0 then). */
int orc_polar_pair(uint64_t seed, uint64_t mdp_id, uint64_t t, uint64_t w, uint64_t j,
                   double *z1, double *z2);

/* DO coefficients Y[t][w][k] = sigma[k] * z (Sec. II-C, coefficient matrix of
 * size Nm x Nr x Nt).  Returns the number of capped pairs (0 normally). */
int64_t orc_sample_coeffs(int32_t nt, int32_t N, int32_t K, const double *sigma,
                          uint64_t seed, uint64_t mdp_id, double *Y);

/* MDP build for the units u in [u_begin, u_end), unit u = t*Nc + c (Alg. 1 / Alg. 2).
 * Output rows are local: lr = (u - u_begin)*A + a.
 *   nnz[lr]                 number of stored successors (sink included)
 *   col[lr*max_nnz + e]     successor state index (sink = |S|), ascending
 *   cnt[lr*max_nnz + e]     realizations landing there
 *   R[o*rows + lr]          expected reward from counts, objective objs[o]
 *   R_lit[o*rows + lr]      the paper's literal form (sum of per-sample r)/N (may be NULL)
 *   *overflow               samples that left the sub-grid (a nonzero value is an error)
 * Returns 0, or -1 if a row had more than max_nnz successors, -2 on bad arguments. */
int orc_build(const orc_problem *p, int64_t u_begin, int64_t u_end, int32_t max_nnz,
              const int32_t *objs, int32_t n_obj, int32_t *nnz, int64_t *col, int32_t *cnt,
              double *R, double *R_lit, int64_t *overflow);

/* Gauss-Jacobi value iteration on the paper-layout CSR model (Sec. II-B).
 * rows = A*nS, row r = a*nS + s; col < nS or col == nS (sink, V = 0).
 * fixed[s] != 0 marks terminal/obstacle start states: pi[s] = -1 there.
 * v_0 = V0[0..nS) when V0 is non-NULL (e.g. a previous plan's values when
 * replanning), else 0.  Stops when max|V_{k+1}-V_k| <= tol or after
 * max_sweeps sweeps. */
int orc_vi_jacobi(int64_t nS, int32_t A, const int64_t *rowptr, const int64_t *col,
                  const double *prob, const double *R, const uint8_t *fixed, const double *V0,
                  double tol, int32_t max_sweeps, double *V, int32_t *pi, int32_t *sweeps,
                  double *residual);

/* Backward induction over time layers t = nt-1 .. 0 with the same per-(s,a)
 * operation order (transitions go from layer t to t+1 or the sink only). */
int orc_vi_backward(int64_t nS, int32_t A, int32_t nt, int64_t Nc, const int64_t *rowptr,
                    const int64_t *col, const double *prob, const double *R,
                    const uint8_t *fixed, double *V, int32_t *pi);

/* Q(s, a) = R + sum_j P_j V(s'_j) for all rows, given V ([nS+1]). */
void orc_q_values(int64_t nS, int32_t A, const int64_t *rowptr, const int64_t *col,
                  const double *prob, const double *R, const double *V, double *Q);

/* ------------------------------------------------------------- 3-D grid --
 * The same build in 3-D space (Sec. II-A: the formulation holds for n = 3):
 * cube cells, state s = t*Nc + (k*Ny + j)*Nx + i with Nc = Nx*Ny*Nz, velocity
 * and action displacements with three components, a cubic neighbouring
 * sub-grid of side L, bin b = ((dk+h)*L + (dj+h))*L + (di+h). */
typedef struct {
  int32_t nx, ny, nz, nt;
  double dx, dt;
  int32_t K, N, A, L;
  const double *vbar;          /* [nt][nz][ny][nx][3] */
  const double *modes;         /* [nt][K][nz][ny][nx][3] */
  const double *Y;             /* [nt][N][K] */
  const double *gbar;          /* [nt][nz][ny][nx] (may be NULL) */
  const uint8_t *obstacle;     /* [nt][nz][ny][nx] */
  const uint8_t *target;       /* [nz][ny][nx] */
  const double *act;           /* [A][4] (d_x, d_y, d_z, F) */
  double c_f, c_r, r_term, r_outbound;
} orc_problem3d;

/* orc_build for the 3-D grid: same outputs and return codes (no R_lit). */
int orc_build3d(const orc_problem3d *p, int64_t u_begin, int64_t u_end, int32_t max_nnz,
                const int32_t *objs, int32_t n_obj, int32_t *nnz, int64_t *col, int32_t *cnt,
                double *R, int64_t *overflow);

/* Policy rollouts (Sec. IV: the optimal policy applied to every flow
 * realization from the start).  Path w starts at cell (i0, j0) at t = 0 and
 * follows policy[s] (s = t*Nc + j*Nx + i), moving with realization w's
 * velocity of time t at its state (the build's kinematics), until:
 *   status 0  it stands on a target cell (absorbing, no further reward);
 *   status 1  it takes the sink: a landing outside the domain or on an
 *             obstacle at t+1, any move from the last layer t = Nt-1, or a
 *             state whose policy is -1 (an obstacle start); reward r_outbound.
 * Each step adds the one-step reward of objective objs[o] (target landings
 * add r_term), summed in path order.
 * Outputs: ret[w*n_obj + o], steps[w], status[w]; traj[w*(nt+1) + k] = state
 * after k steps (k = 0: the start; the sink = |S|; -1 after the end), or
 * NULL.  Returns 0, or -2 on bad arguments. */
int orc_rollout(const orc_problem *p, const int32_t *policy, int32_t i0, int32_t j0,
                const int32_t *objs, int32_t n_obj, double *ret, int32_t *steps, int32_t *status,
                int64_t *traj);

#ifdef __cplusplus
}
#endif
#endif
