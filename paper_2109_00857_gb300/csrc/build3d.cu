// build3d.cu -- the MDP build on a 3-D grid (Sec. II-A with n = 3: the
// formulation and the implementation hold in 3-D space).  The model it
// returns has the 2-D model's layout (sliced-ELL rows of signed 16-bit
// successor offsets dk*Nx*Ny + dj*Nx + di), so mdp_solve, mdp_solve_multi,
// mdp_export_csr and mdp_model_info apply unchanged.
//
// One CTA per slice (spw states x A_pad actions, 32 rows), persistent over a
// work queue.  Per chunk of realizations the threads form the velocity of
// their (state, realization) items once for all actions and stage it in
// shared memory (phase A).  Counting, two ways with the same result:
//  - per action (phase B): lane l of every warp bins row l's landings of the
//    staged realizations into a full L^3 window hist[bin][l] (a lane only
//    touches its own bank);
//  - FP32 rank counting, when every realization is staged at once: as in the
//    2-D build, the landing offset per axis is floor(u) + c + [rho >= le]
//    with rho = #{T <= frac u} over the axis' distinct step thresholds, so
//    one count per realization at the fine coordinate (floor(u) - n0) S + rho
//    in a per-state 3-D table (in the window memory), an in-place 3-D prefix
//    sum, and each (row, offset bin) count is an eight-corner box sum.
// Warp 0 then turns each row's counts into ascending entries with the sink
// folded and R(s,a) from the counts.  The landing offsets are monotone in the
// velocity, so the offsets of a state's smallest and largest u per axis bound
// every landing of a row: the emit scans that box instead of all L^3 bins.
// FP32 lands with the exact floor of u + d per axis (the 2-D path's landing
// offsets); FP64 check mode counts per action and evaluates the oracle's
// literal formulas in its order without contraction.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "build_common.cuh"

namespace mdpgb {

constexpr int kMaxL3 = 11;   // largest 3-D window side (11^3 bins x 128 B in shared memory)
constexpr int kRank3 = 8;    // most distinct step thresholds per axis for rank counting
constexpr int kRankSpw = 4;  // most states per slice for rank counting

struct Actions3 {
  float dl[3][kMaxActions];     // displacement * dt/dx per axis (FP32 kinematics)
  int32_t c[3][kMaxActions];    // floor(dl)
  float th[3][kMaxActions];     // smallest float >= 1 - frac(dl) (2: integer dl)
  float F[kMaxActions];
  double d64[3][kMaxActions];   // displacement in FP64 (check mode)
  double F64[kMaxActions];
  // rank counting (FP32): per axis the distinct thresholds T[0] < ... < T[D-1]
  // (integer displacements excluded), S = D + 1 fine positions per cell and
  // le[a] = #{T <= th[a]} (D + 1 for an integer displacement): the landing
  // steps past floor(u) + c exactly when rho(frac u) = #{T <= frac u} >= le
  float T[3][kRank3];
  int32_t D[3];
  int8_t le[3][kMaxActions];
};

struct Build3Args {
  int32_t nx, ny, nz, nt, K, N, A, A_pad, spw, L, h, row_cap, chunk;
  int32_t rank_ok;   // FP32 rank counting allowed (thresholds and states fit)
  int64_t Nc, nS, n_slices, rows_pad;
  float lam;
  double dx, dt;
  const void *vbar, *modes, *Y, *gbar;
  const uint8_t *cls, *target, *obstacle;
  Actions3 act;
  RewardParams rw;
  uint32_t *pool;
  uint64_t pool_cap_cols;
  uint32_t *slice_off;
  uint8_t *slice_w, *nnz;
  uint16_t *sinkc;
  void *R;
  unsigned long long *cnt;
  // warp-per-slice kernel (FP32 rank counting): table words per warp, the
  // list of slices it leaves to the CTA kernel, and (CTA kernel) that list
  int32_t cap3;
  uint32_t *defer;
  const uint32_t *defer_in;
};

template <typename RT>
struct U3 {
  RT x, y, z;
};

// Offset bound of one axis for the emit box: the landing offset of u clamped
// to [-h-1, h+1] (monotone in u like the landing itself).
__device__ __forceinline__ int box_offset(float u, int c, float th, int h) {
  const float n = floorf(u);
  const float f = n + (float)c + ((u - n) >= th ? 1.f : 0.f);
  return (int)fminf(fmaxf(f, (float)(-h - 1)), (float)(h + 1));
}

__device__ __forceinline__ int box_offset64(double v, double d, int64_t i, double dx, double dt, int h) {
  const double x = __dmul_rn((double)i + 0.5, dx);
  const double xp = __dadd_rn(x, __dmul_rn(__dadd_rn(v, d), dt));
  const double f = floor(__ddiv_rn(xp, dx)) - (double)i;
  if (f >= (double)(-h - 1) && f <= (double)(h + 1)) return (int)f;
  return f < 0.0 ? -h - 1 : h + 1;
}

// rho(f) = #{T <= f} for f in [0, 1) (D <= kRank3 thresholds, ascending).
__device__ __forceinline__ int rank3(float f, const float *T, int D) {
  int r = 0;
#pragma unroll
  for (int i = 0; i < kRank3; ++i) r += (i < D && T[i] <= f) ? 1 : 0;
  return r;
}

// Fine coordinate of u along one axis: (floor(u) - n0) S + rho(u - floor(u)).
__device__ __forceinline__ int fine3(float u, int n0, int S, const float *T, int D) {
  const float n = floorf(u);
  return ((int)n - n0) * S + rank3(u - n, T, D);
}

// Fine table of one state (rank counting): cells [1, G] per axis after a
// zero border, index ((x * (Gy + 1)) + y) * (Gz + 1) + z from word `base`.
struct Geo3 {
  int n0[3], fmin[3], G[3], base;
};

template <typename RT>
__global__ void __launch_bounds__(256, sizeof(RT) == 4 ? 4 : 1) build3d_kernel(Build3Args a) {
  extern __shared__ __align__(16) unsigned char smem3[];
  const int nb = a.L * a.L * a.L;
  uint32_t *hist = reinterpret_cast<uint32_t *>(smem3);   // [nb][32]
  U3<RT> *ubuf = reinterpret_cast<U3<RT> *>(smem3 + (size_t)nb * 128);   // [chunk][spw]
  RT *sbox = reinterpret_cast<RT *>(smem3 + (size_t)nb * 128 +
                                    (((size_t)a.chunk * a.spw * sizeof(U3<RT>) + 15) & ~(size_t)15));   // [warp][spw][6]
  __shared__ long long s_slice;
  __shared__ Geo3 s_geo[kRankSpw];       // rank counting: the states' fine tables
  __shared__ long long s_cells[kRankSpw];
  __shared__ int s_rank, s_total;        // rank counting used for this slice; table words
  unsigned long long loc_tot = 0, loc_dom = 0, loc_samp = 0, loc_max = 0;   // warp 0 lane 0
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int h = a.h, L = a.L;
  const int64_t Nc = a.Nc, nxy = (int64_t)a.nx * a.ny;
  const int q_l = lane / a.A_pad, a_l = lane % a.A_pad;
  const bool act_ok = a_l < a.A;
  const int q_t = tid % a.spw, w0 = tid / a.spw, wstride = blockDim.x / a.spw;
  const RT *vbar = static_cast<const RT *>(a.vbar);
  const RT *modes = static_cast<const RT *>(a.modes);
  const RT *Yall = static_cast<const RT *>(a.Y);
  for (int i = tid; i < nb * 32; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (;;) {
    if (tid == 0) {
      if (a.defer_in) {   // the slices the warp kernel left (count CNT_DEFER_N)
        const unsigned long long i = atomicAdd(&a.cnt[CNT_DEFER_WORK], 1ULL);
        s_slice = i < a.cnt[CNT_DEFER_N] ? (long long)a.defer_in[i] : (long long)a.n_slices;
      } else {
        s_slice = (long long)atomicAdd(&a.cnt[CNT_WORK], 1ULL);
      }
      s_rank = 0;
      s_total = 0;
    }
    __syncthreads();
    const int64_t sl = s_slice;
    if (sl >= a.n_slices) break;
    const int64_t s_l = sl * a.spw + q_l, s_t = sl * a.spw + q_t;
    // state kinds: terminal first, then obstacle start or last layer, else sampled
    auto kind = [&](int64_t s) {
      if (s >= a.nS) return (int)KIND_NONE;
      if (a.target[s % Nc]) return (int)KIND_TERMINAL;
      if (a.obstacle[s] || s / Nc == a.nt - 1) return (int)KIND_SINK;
      return (int)KIND_SAMPLE;
    };
    int kind_l = act_ok ? kind(s_l) : KIND_NONE;
    const int kind_t = kind(s_t);
    const int any = __syncthreads_or(kind_t == KIND_SAMPLE);
    // ---- phase B: lane l bins row l's landings of the first cn staged
    // realizations (one shared increment per realization and action)
    auto phase_b = [&](int cn) {
      if (kind_l == KIND_SAMPLE) {
        const int64_t sc = s_l % Nc;
        const int64_t li = sc % a.nx, lj = (sc / a.nx) % a.ny, lk = sc / nxy;
        const uint32_t hb = smem_u32(hist) + (uint32_t)lane * 4u;
        for (int w = warp; w < cn; w += nwarps) {
          const U3<RT> u = ubuf[(size_t)w * a.spw + q_l];
          int di, dj, dk;
          if constexpr (sizeof(RT) == 4) {
            di = land_offset(u.x, a.act.c[0][a_l], a.act.th[0][a_l]);
            dj = land_offset(u.y, a.act.c[1][a_l], a.act.th[1][a_l]);
            dk = land_offset(u.z, a.act.c[2][a_l], a.act.th[2][a_l]);
          } else {
            // x' = x + (v + a) dt from the cell centre, cell() = floor(x' / dx)
            const double x = __dmul_rn((double)li + 0.5, a.dx), y = __dmul_rn((double)lj + 0.5, a.dx);
            const double z = __dmul_rn((double)lk + 0.5, a.dx);
            const double xp = __dadd_rn(x, __dmul_rn(__dadd_rn(u.x, a.act.d64[0][a_l]), a.dt));
            const double yp = __dadd_rn(y, __dmul_rn(__dadd_rn(u.y, a.act.d64[1][a_l]), a.dt));
            const double zp = __dadd_rn(z, __dmul_rn(__dadd_rn(u.z, a.act.d64[2][a_l]), a.dt));
            const double fx = floor(__ddiv_rn(xp, a.dx)) - (double)li;
            const double fy = floor(__ddiv_rn(yp, a.dx)) - (double)lj;
            const double fz = floor(__ddiv_rn(zp, a.dx)) - (double)lk;
            di = (fabs(fx) <= (double)h) ? (int)fx : h + 1;
            dj = (fabs(fy) <= (double)h) ? (int)fy : h + 1;
            dk = (fabs(fz) <= (double)h) ? (int)fz : h + 1;
          }
          if (di < -h || di > h || dj < -h || dj > h || dk < -h || dk > h) {
            atomicAdd(&a.cnt[CNT_OVERFLOW], 1ULL);
            continue;
          }
          const uint32_t b = (uint32_t)(((dk + h) * L + (dj + h)) * L + (di + h));
          asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(hb + b * 128u), "r"(1u));
        }
      }
    };
    // FP32 rank counting needs every realization staged at once
    const bool try_rank = sizeof(RT) == 4 && a.rank_ok && a.N <= a.chunk;
    // rank counting: the count of row (q_l, a_l)'s offset bin (di, dj, dk) is
    // the fine table summed over X in [(di - c - n0 - 1) S + le, + S) per axis
    // (the realizations whose landing steps to exactly that offset): eight
    // corners of the prefix table
    auto rank_count = [&](const Geo3 &gl, int di, int dj, int dk) -> uint32_t {
      const int off[3] = {di, dj, dk};
      int c0[3], c1[3];
      for (int x = 0; x < 3; ++x) {
        const int S = a.act.D[x] + 1;
        const int f0 = (off[x] - a.act.c[x][a_l] - gl.n0[x] - 1) * S + a.act.le[x][a_l] - gl.fmin[x];
        c0[x] = max(f0, 0);
        c1[x] = min(f0 + S - 1, gl.G[x] - 1);
        if (c0[x] > c1[x]) return 0u;
      }
      const int Py = gl.G[1] + 1, Pz = gl.G[2] + 1;
      const uint32_t *P = hist + gl.base;
      auto at = [&](int x, int y, int z) { return P[(x * Py + y) * Pz + z]; };
      const int x0 = c0[0], y0 = c0[1], z0 = c0[2], x1 = c1[0] + 1, y1 = c1[1] + 1, z1 = c1[2] + 1;
      return at(x1, y1, z1) - at(x0, y1, z1) - at(x1, y0, z1) - at(x1, y1, z0) + at(x0, y0, z1) +
             at(x0, y1, z0) + at(x1, y0, z0) - at(x0, y0, z0);
    };
    RT mn[3] = {(RT)INFINITY, (RT)INFINITY, (RT)INFINITY}, mx[3] = {-(RT)INFINITY, -(RT)INFINITY, -(RT)INFINITY};
    if (any) {
      const int64_t t = s_t / Nc, c = s_t % Nc;
      const RT *Yt = Yall + (size_t)t * a.N * a.K;
      for (int c0 = 0; c0 < a.N; c0 += a.chunk) {
        const int cn = min(a.chunk, a.N - c0);
        // ---- phase A: velocity of (state q_t, realization w) once for all actions
        for (int w = w0; w < cn; w += wstride) {
          if (kind_t != KIND_SAMPLE) continue;
          const RT *yw = Yt + (size_t)(c0 + w) * a.K;
          U3<RT> u;
          if constexpr (sizeof(RT) == 4) {
            float vx = vbar[3 * s_t], vy = vbar[3 * s_t + 1], vz = vbar[3 * s_t + 2];
            for (int k = 0; k < a.K; ++k) {
              const float *ph = modes + 3 * ((t * a.K + k) * Nc + c);
              vx = fmaf(yw[k], ph[0], vx);
              vy = fmaf(yw[k], ph[1], vy);
              vz = fmaf(yw[k], ph[2], vz);
            }
            u.x = fmaf(vx, a.lam, 0.5f);
            u.y = fmaf(vy, a.lam, 0.5f);
            u.z = fmaf(vz, a.lam, 0.5f);
            if (!(fabsf(u.x) < 1e30f)) u.x = 1e30f;
            if (!(fabsf(u.y) < 1e30f)) u.y = 1e30f;
            if (!(fabsf(u.z) < 1e30f)) u.z = 1e30f;
          } else {
            double vx = vbar[3 * s_t], vy = vbar[3 * s_t + 1], vz = vbar[3 * s_t + 2];
            for (int k = 0; k < a.K; ++k) {
              const double *ph = modes + 3 * ((t * a.K + k) * Nc + c);
              vx = __dadd_rn(vx, __dmul_rn(yw[k], ph[0]));
              vy = __dadd_rn(vy, __dmul_rn(yw[k], ph[1]));
              vz = __dadd_rn(vz, __dmul_rn(yw[k], ph[2]));
            }
            u.x = vx;   // the velocity itself: the landing adds the position and action
            u.y = vy;
            u.z = vz;
          }
          ubuf[(size_t)w * a.spw + q_t] = u;
          mn[0] = fmin(mn[0], u.x); mn[1] = fmin(mn[1], u.y); mn[2] = fmin(mn[2], u.z);
          mx[0] = fmax(mx[0], u.x); mx[1] = fmax(mx[1], u.y); mx[2] = fmax(mx[2], u.z);
        }
        __syncthreads();
        if (!try_rank) {
          phase_b(cn);
          __syncthreads();
        }
      }
      // the extreme u of each state: lanes of equal q_t are lane + multiples of spw
      for (int off = 16; off >= a.spw; off >>= 1) {
        for (int x = 0; x < 3; ++x) {
          mn[x] = fmin(mn[x], __shfl_xor_sync(0xffffffffu, mn[x], off));
          mx[x] = fmax(mx[x], __shfl_xor_sync(0xffffffffu, mx[x], off));
        }
      }
      if (lane < a.spw) {
        RT *sb = sbox + ((size_t)warp * a.spw + lane) * 6;
        for (int x = 0; x < 3; ++x) {
          sb[x] = mn[x];
          sb[3 + x] = mx[x];
        }
      }
      __syncthreads();
      if (try_rank) {
        // ---- rank counting (FP32): per state a fine table over the fine
        // coordinates (floor(u) - n0) S + rho(frac u) of its extremes; the
        // slice falls back to phase B when a table cannot be formed or the
        // tables do not fit the window memory
        if (tid < a.spw) {
          const int q = tid;
          Geo3 g{};
          long long cells = 0;
          if (kind(sl * a.spw + q) == KIND_SAMPLE) {
            cells = 1;
            for (int x = 0; x < 3 && cells > 0; ++x) {
              float umn = INFINITY, umx = -INFINITY;
              for (int w = 0; w < nwarps; ++w) {
                umn = fminf(umn, (float)sbox[((size_t)w * a.spw + q) * 6 + x]);
                umx = fmaxf(umx, (float)sbox[((size_t)w * a.spw + q) * 6 + 3 + x]);
              }
              if (!(umn > -1e6f) || !(umx < 1e6f) || umx - umn > 1024.f) {
                cells = -1;   // non-finite, far or widely spread u (a sub-grid overflow): phase B
                break;
              }
              const int S = a.act.D[x] + 1;
              g.n0[x] = (int)floorf(umn);
              g.fmin[x] = fine3(umn, g.n0[x], S, a.act.T[x], a.act.D[x]);
              g.G[x] = fine3(umx, g.n0[x], S, a.act.T[x], a.act.D[x]) - g.fmin[x] + 1;
              cells *= (long long)(g.G[x] + 1);
            }
          }
          s_geo[q] = g;
          s_cells[q] = cells;
        }
        __syncthreads();
        if (tid == 0) {
          long long tot = 0;
          bool fit = true;
          for (int q = 0; q < a.spw; ++q) {
            if (s_cells[q] < 0) fit = false;
            s_geo[q].base = (int)min(tot, (long long)nb * 32);
            tot += max(s_cells[q], 0LL);
          }
          fit = fit && tot <= (long long)nb * 32;
          s_rank = fit ? 1 : 0;
          s_total = fit ? (int)tot : 0;
        }
        __syncthreads();
        if (s_rank) {
          // one count per realization at its fine coordinate (the window
          // memory is zero between slices)
          if (kind_t == KIND_SAMPLE) {
            const Geo3 g = s_geo[q_t];
            const int Py = g.G[1] + 1, Pz = g.G[2] + 1;
            const uint32_t hb = smem_u32(hist);
            for (int w = w0; w < a.N; w += wstride) {
              const U3<RT> u = ubuf[(size_t)w * a.spw + q_t];
              int X = fine3((float)u.x, g.n0[0], a.act.D[0] + 1, a.act.T[0], a.act.D[0]) - g.fmin[0];
              int Y = fine3((float)u.y, g.n0[1], a.act.D[1] + 1, a.act.T[1], a.act.D[1]) - g.fmin[1];
              int Z = fine3((float)u.z, g.n0[2], a.act.D[2] + 1, a.act.T[2], a.act.D[2]) - g.fmin[2];
              X = min(max(X, 0), g.G[0] - 1);
              Y = min(max(Y, 0), g.G[1] - 1);
              Z = min(max(Z, 0), g.G[2] - 1);
              const uint32_t idx = (uint32_t)(g.base + ((X + 1) * Py + (Y + 1)) * Pz + (Z + 1));
              asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(hb + 4u * idx), "r"(1u));
            }
          }
          __syncthreads();
          // in-place inclusive prefix sums along z, y and x (the zero border
          // planes stay zero): P[x][y][z] = sum of counts up to (x, y, z)
          for (int q = 0; q < a.spw; ++q) {
            if (s_cells[q] <= 0) continue;
            const Geo3 g = s_geo[q];
            const int Gx = g.G[0], Gy = g.G[1], Gz = g.G[2], Py = Gy + 1, Pz = Gz + 1;
            uint32_t *P = hist + g.base;
            for (int ln = tid; ln < Gx * Gy; ln += blockDim.x) {
              uint32_t *r = P + ((ln / Gy + 1) * Py + (ln % Gy + 1)) * Pz;
              for (int z = 1; z <= Gz; ++z) r[z] += r[z - 1];
            }
            __syncthreads();
            for (int ln = tid; ln < Gx * Gz; ln += blockDim.x) {
              uint32_t *r = P + (ln / Gz + 1) * Py * Pz + (ln % Gz + 1);
              for (int y = 1; y <= Gy; ++y) r[y * Pz] += r[(y - 1) * Pz];
            }
            __syncthreads();
            for (int ln = tid; ln < Gy * Gz; ln += blockDim.x) {
              uint32_t *r = P + (ln / Gz + 1) * Pz + (ln % Gz + 1);
              for (int x = 1; x <= Gx; ++x) r[x * Py * Pz] += r[(x - 1) * Py * Pz];
            }
            __syncthreads();
          }
        } else {
          phase_b(a.N);   // every realization is staged
          __syncthreads();
        }
      }
    }
    const int rank_mode = s_rank, rank_total = s_total;
    // ---- emit (warp 0): ascending bins (dk, dj, di) of the row's box, sink
    // folded, R from counts
    if (warp == 0) {
      const int64_t ir = sl * 32 + lane;
      const int64_t t = s_l / Nc, c = s_l % Nc;
      const int64_t li = c % a.nx, lj = (c / a.nx) % a.ny, lk = c / nxy;
      const int64_t nxt = (t + 1) * Nc;
      int e = 0;
      uint32_t sink = 0;
      int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
      Geo3 gl{};
      if (rank_mode && kind_l == KIND_SAMPLE) gl = s_geo[q_l];
      if (kind_l == KIND_SAMPLE) {
        RT umn[3] = {(RT)INFINITY, (RT)INFINITY, (RT)INFINITY}, umx[3] = {-(RT)INFINITY, -(RT)INFINITY, -(RT)INFINITY};
        for (int w = 0; w < nwarps; ++w) {
          const RT *sb = sbox + ((size_t)w * a.spw + q_l) * 6;
          for (int x = 0; x < 3; ++x) {
            umn[x] = fmin(umn[x], sb[x]);
            umx[x] = fmax(umx[x], sb[3 + x]);
          }
        }
        const int64_t pos[3] = {li, lj, lk};
        for (int x = 0; x < 3; ++x) {
          if constexpr (sizeof(RT) == 4) {
            lo[x] = box_offset(umn[x], a.act.c[x][a_l], a.act.th[x][a_l], h);
            hi[x] = box_offset(umx[x], a.act.c[x][a_l], a.act.th[x][a_l], h);
          } else {
            lo[x] = box_offset64(umn[x], a.act.d64[x][a_l], pos[x], a.dx, a.dt, h);
            hi[x] = box_offset64(umx[x], a.act.d64[x][a_l], pos[x], a.dx, a.dt, h);
          }
          // (phase B counted the landings outside the window; rank counting
          // counts the rows that have some)
          if (rank_mode && (lo[x] < -h || hi[x] > h)) atomicAdd(&a.cnt[CNT_OVERFLOW], 1ULL);
          lo[x] = max(lo[x], -h);
          hi[x] = min(hi[x], h);
        }
        for (int dk = lo[2]; dk <= hi[2]; ++dk)
          for (int dj = lo[1]; dj <= hi[1]; ++dj)
            for (int di = lo[0]; di <= hi[0]; ++di) {
              const int b = ((dk + h) * L + (dj + h)) * L + (di + h);
              const uint32_t n = rank_mode ? rank_count(gl, di, dj, dk) : hist[b * 32 + lane];
              if (!n) continue;
              const int64_t ip = li + di, jp = lj + dj, kp = lk + dk;
              const bool inside = ip >= 0 && ip < a.nx && jp >= 0 && jp < a.ny && kp >= 0 && kp < a.nz;
              if (!inside || a.obstacle[nxt + (kp * a.ny + jp) * a.nx + ip]) sink += n;
              else ++e;
            }
      } else if (kind_l == KIND_SINK) {
        sink = (uint32_t)a.N;
      }
      const bool cap_hit = e + (sink > 0 ? 1 : 0) > a.row_cap;
      if (cap_hit) {
        atomicAdd(&a.cnt[CNT_ROW_CAP], 1ULL);
        e = 0;
      }
      int W = e;
      for (int off = 16; off > 0; off >>= 1) W = max(W, __shfl_xor_sync(0xffffffffu, W, off));
      unsigned long long base = 0;
      if (lane == 0 && W > 0) base = atomicAdd(&a.cnt[CNT_POOL_COLS], (unsigned long long)W);
      base = __shfl_sync(0xffffffffu, base, 0);
      const bool fits = (W == 0) || (base + (unsigned long long)W <= a.pool_cap_cols);
      if (!fits && lane == 0) atomicAdd(&a.cnt[CNT_POOL_FULL], 1ULL);
      const bool write = fits && !cap_hit;
      RT Racc[3] = {0, 0, 0};
      uint32_t *dst = a.pool + base * 32 + lane;
      int k = 0;
      if (kind_l == KIND_SAMPLE) {
        const RT F = sizeof(RT) == 4 ? (RT)a.act.F[a_l] : (RT)a.act.F64[a_l];
        const RT g_s = a.gbar ? static_cast<const RT *>(a.gbar)[s_l] : (RT)0;
        for (int dk = lo[2]; dk <= hi[2]; ++dk)
          for (int dj = lo[1]; dj <= hi[1]; ++dj)
            for (int di = lo[0]; di <= hi[0]; ++di) {
              uint32_t n;
              if (rank_mode) {
                n = rank_count(gl, di, dj, dk);
              } else {
                uint32_t *hp = hist + (((dk + h) * L + (dj + h)) * L + (di + h)) * 32 + lane;
                n = *hp;
                *hp = 0;
              }
              if (!n) continue;
              const int64_t ip = li + di, jp = lj + dj, kp = lk + dk;
              const bool inside = ip >= 0 && ip < a.nx && jp >= 0 && jp < a.ny && kp >= 0 && kp < a.nz;
              const int64_t cp = (kp * a.ny + jp) * a.nx + ip;
              if (!inside || a.obstacle[nxt + cp]) continue;
              if (write) dst[(size_t)k * 32] = entry_word((int)(dk * nxy + dj * a.nx + di), n);
              ++k;
              const bool is_t = a.target[cp] != 0;
              const RT g_sp = a.gbar ? static_cast<const RT *>(a.gbar)[nxt + cp] : (RT)0;
              for (int o = 0; o < a.rw.n_obj; ++o) {
                if constexpr (sizeof(RT) == 4) {
                  Racc[o] = fmaf((float)n / (float)a.N, step_reward32(a.rw, a.rw.objs[o], F, g_s, g_sp, is_t), Racc[o]);
                } else {
                  const double p = __ddiv_rn((double)n, (double)a.N);
                  Racc[o] = __dadd_rn(Racc[o], __dmul_rn(p, step_reward64(a.rw, a.rw.objs[o], F, g_s, g_sp, is_t)));
                }
              }
            }
        if (sink) {
          for (int o = 0; o < a.rw.n_obj; ++o) {
            if constexpr (sizeof(RT) == 4)
              Racc[o] = fmaf((float)sink / (float)a.N, (float)a.rw.r_out, Racc[o]);
            else
              Racc[o] = __dadd_rn(Racc[o], __dmul_rn(__ddiv_rn((double)sink, (double)a.N), a.rw.r_out));
          }
        }
      } else if (kind_l == KIND_SINK) {
        for (int o = 0; o < a.rw.n_obj; ++o)
          Racc[o] = sizeof(RT) == 4 ? (RT)(float)a.rw.r_out : (RT)__dmul_rn(__ddiv_rn((double)a.N, (double)a.N), a.rw.r_out);
      }
      if (!write) {
        e = 0;
        k = 0;
      }
      if (write)
        for (int kk = k; kk < W; ++kk) dst[(size_t)kk * 32] = 0u;
      if (!fits) sink = 0;
      if (lane == 0) {
        a.slice_off[sl] = (fits && W > 0) ? (uint32_t)base : kNoSlice;
        a.slice_w[sl] = (fits && W > 0) ? (uint8_t)W : (uint8_t)0;
      }
      a.nnz[ir] = (uint8_t)e;
      a.sinkc[ir] = (uint16_t)sink;
      for (int o = 0; o < a.rw.n_obj; ++o) static_cast<RT *>(a.R)[(int64_t)o * a.rows_pad + ir] = Racc[o];
      int dom = e, tot = e + (sink > 0 ? 1 : 0);
      for (int off = 16; off > 0; off >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, off);
        dom += __shfl_xor_sync(0xffffffffu, dom, off);
      }
      const int sampled = __popc(__ballot_sync(0xffffffffu, kind_l == KIND_SAMPLE));
      loc_tot += (unsigned long long)tot;
      loc_dom += (unsigned long long)dom;
      loc_samp += (unsigned long long)sampled * (unsigned long long)a.N;
      loc_max = max(loc_max, (unsigned long long)W);
    }
    __syncthreads();
    if (rank_mode)   // the window memory goes back to zero for the next slice
      for (int i = tid; i < rank_total; i += blockDim.x) hist[i] = 0;
  }
  if (tid == 0) {
    atomicAdd(&a.cnt[CNT_NNZ], loc_tot);
    atomicAdd(&a.cnt[CNT_DOMAIN], loc_dom);
    atomicAdd(&a.cnt[CNT_SAMPLES], loc_samp);
    atomicMax(&a.cnt[CNT_MAXROW], loc_max);
  }
}

// ---- warp per slice (FP32 rank counting) ----
// A warp builds one slice alone, in private shared memory and without block
// barriers -- the 2-D warp kernel's scheme in three dimensions: pass 1 forms
// u for the warp's (state, realization) items and reduces each state's exact
// extremes per axis; the states' fine tables are laid out in the warp's table
// memory; pass 2 forms u again and counts each realization at its fine
// coordinate; an in-place 3-D prefix sum; then lane l emits row l exactly as
// the CTA kernel's rank path does (the same offsets, eight-corner box sums,
// entry order and R accumulation), so a slice's output does not depend on
// the kernel that built it.  Slices whose tables do not fit the warp's memory
// (or whose velocity extremes are not finite or widely spread) go to a list
// that the CTA kernel builds afterwards.
constexpr int kWarps3 = 8;   // warps per CTA of the warp kernel
constexpr int kCap3 = 2048;  // table words per warp (8 KB)

struct Warp3Acc {
  unsigned long long tot = 0, dom = 0, samp = 0, maxw = 0;
};

// u of realization w of state s (layer t, cell c): the CTA kernel's phase A
__device__ __forceinline__ void velocity3(const Build3Args &a, int64_t s, int64_t t, int64_t c, int w, float (&u)[3]) {
  const float *vbar = static_cast<const float *>(a.vbar);
  const float *modes = static_cast<const float *>(a.modes);
  const float *yw = static_cast<const float *>(a.Y) + ((size_t)t * a.N + w) * a.K;
  float vx = vbar[3 * s], vy = vbar[3 * s + 1], vz = vbar[3 * s + 2];
  for (int k = 0; k < a.K; ++k) {
    const float *ph = modes + 3 * ((t * a.K + k) * a.Nc + c);
    vx = fmaf(yw[k], ph[0], vx);
    vy = fmaf(yw[k], ph[1], vy);
    vz = fmaf(yw[k], ph[2], vz);
  }
  u[0] = fmaf(vx, a.lam, 0.5f);
  u[1] = fmaf(vy, a.lam, 0.5f);
  u[2] = fmaf(vz, a.lam, 0.5f);
#pragma unroll
  for (int x = 0; x < 3; ++x)
    if (!(fabsf(u[x]) < 1e30f)) u[x] = 1e30f;
}

// the same with the state's mode vectors in registers (K <= 4)
__device__ __forceinline__ void velocity3r(const Build3Args &a, int64_t s, int64_t t, int w, const float (&ph)[4][3],
                                           float (&u)[3]) {
  const float *vbar = static_cast<const float *>(a.vbar);
  const float *yw = static_cast<const float *>(a.Y) + ((size_t)t * a.N + w) * a.K;
  float vx = vbar[3 * s], vy = vbar[3 * s + 1], vz = vbar[3 * s + 2];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k < a.K) {
      const float y = yw[k];
      vx = fmaf(y, ph[k][0], vx);
      vy = fmaf(y, ph[k][1], vy);
      vz = fmaf(y, ph[k][2], vz);
    }
  }
  u[0] = fmaf(vx, a.lam, 0.5f);
  u[1] = fmaf(vy, a.lam, 0.5f);
  u[2] = fmaf(vz, a.lam, 0.5f);
#pragma unroll
  for (int x = 0; x < 3; ++x)
    if (!(fabsf(u[x]) < 1e30f)) u[x] = 1e30f;
}

__device__ __forceinline__ Geo3 shfl_geo3(const Geo3 &g, int src) {
  Geo3 o;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    o.n0[x] = __shfl_sync(0xffffffffu, g.n0[x], src);
    o.fmin[x] = __shfl_sync(0xffffffffu, g.fmin[x], src);
    o.G[x] = __shfl_sync(0xffffffffu, g.G[x], src);
  }
  o.base = __shfl_sync(0xffffffffu, g.base, src);
  return o;
}

// Slice sl by one warp; tab: the warp's cap words of table memory (zero).
// Returns false when the slice was put on the CTA kernel's list.
__device__ bool warp3_slice(const Build3Args &a, int64_t sl, uint32_t *tab, Warp3Acc &acc) {
  const int lane = threadIdx.x & 31;
  const int spw = a.spw, h = a.h, L = a.L;
  const int64_t Nc = a.Nc, nxy = (int64_t)a.nx * a.ny;
  const int q_l = lane / a.A_pad, a_l = lane % a.A_pad;
  const bool act_ok = a_l < a.A;
  const int q_t = lane % spw, wi = lane / spw, wstep = 32 / spw;
  auto kind = [&](int64_t s) {
    if (s >= a.nS) return (int)KIND_NONE;
    if (a.target[s % Nc]) return (int)KIND_TERMINAL;
    if (a.obstacle[s] || s / Nc == a.nt - 1) return (int)KIND_SINK;
    return (int)KIND_SAMPLE;
  };
  const int64_t s_l = sl * spw + q_l, s_t = sl * spw + q_t;
  const int kind_l = act_ok ? kind(s_l) : KIND_NONE;
  const int kind_t = kind(s_t);
  const int64_t t_t = s_t / Nc, c_t = s_t % Nc;
  // up to four modes: the state's mode vectors in registers for both passes
  // (else each realization reloads them, 3K floats, from L1)
  const bool preph = a.K <= 4;
  float ph[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int x = 0; x < 3; ++x)
      ph[k][x] = (preph && k < a.K && kind_t == KIND_SAMPLE)
                     ? static_cast<const float *>(a.modes)[3 * ((t_t * a.K + k) * Nc + c_t) + x] : 0.f;
  // ---- pass 1: exact extremes of u per state and axis
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  if (kind_t == KIND_SAMPLE) {
    for (int w = wi; w < a.N; w += wstep) {
      float u[3];
      if (preph) velocity3r(a, s_t, t_t, w, ph, u);
      else velocity3(a, s_t, t_t, c_t, w, u);
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        mn[x] = fminf(mn[x], u[x]);
        mx[x] = fmaxf(mx[x], u[x]);
      }
    }
  }
  for (int off = 16; off >= spw; off >>= 1) {
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      mn[x] = fminf(mn[x], __shfl_xor_sync(0xffffffffu, mn[x], off));
      mx[x] = fmaxf(mx[x], __shfl_xor_sync(0xffffffffu, mx[x], off));
    }
  }
  // lane q < spw: the fine table of state q (the CTA kernel's rules)
  Geo3 g{};
  long long cells = 0;
  if (lane < spw && kind(sl * spw + lane) == KIND_SAMPLE) {
    cells = 1;
    for (int x = 0; x < 3 && cells > 0; ++x) {
      if (!(mn[x] > -1e6f) || !(mx[x] < 1e6f) || mx[x] - mn[x] > 1024.f) {
        cells = -1;
        break;
      }
      const int S = a.act.D[x] + 1;
      g.n0[x] = (int)floorf(mn[x]);
      g.fmin[x] = fine3(mn[x], g.n0[x], S, a.act.T[x], a.act.D[x]);
      g.G[x] = fine3(mx[x], g.n0[x], S, a.act.T[x], a.act.D[x]) - g.fmin[x] + 1;
      cells *= (long long)(g.G[x] + 1);
    }
  }
  long long total = 0;
  bool fit = true;
  for (int q = 0; q < spw; ++q) {
    const long long cq = __shfl_sync(0xffffffffu, cells, q);
    if (lane == q) g.base = (int)min(total, (long long)a.cap3);
    if (cq < 0) fit = false;
    total += max(cq, 0LL);
  }
  if (!fit || total > (long long)a.cap3) {   // the CTA kernel builds it
    if (lane == 0) {
      const unsigned long long i = atomicAdd(&a.cnt[CNT_DEFER_N], 1ULL);
      a.defer[i] = (uint32_t)sl;
    }
    return false;
  }
  // ---- pass 2: one count per realization at its fine coordinate
  const Geo3 gt = shfl_geo3(g, q_t);
  if (kind_t == KIND_SAMPLE) {
    const int Py = gt.G[1] + 1, Pz = gt.G[2] + 1;
    const uint32_t hb = smem_u32(tab);
#pragma unroll 1
    for (int w = wi; w < a.N; w += wstep) {
      float u[3];
      if (preph) velocity3r(a, s_t, t_t, w, ph, u);
      else velocity3(a, s_t, t_t, c_t, w, u);
      int X = fine3(u[0], gt.n0[0], a.act.D[0] + 1, a.act.T[0], a.act.D[0]) - gt.fmin[0];
      int Y = fine3(u[1], gt.n0[1], a.act.D[1] + 1, a.act.T[1], a.act.D[1]) - gt.fmin[1];
      int Z = fine3(u[2], gt.n0[2], a.act.D[2] + 1, a.act.T[2], a.act.D[2]) - gt.fmin[2];
      X = min(max(X, 0), gt.G[0] - 1);
      Y = min(max(Y, 0), gt.G[1] - 1);
      Z = min(max(Z, 0), gt.G[2] - 1);
      const uint32_t idx = (uint32_t)(gt.base + ((X + 1) * Py + (Y + 1)) * Pz + (Z + 1));
      asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(hb + 4u * idx), "r"(1u));
    }
  }
  __syncwarp();
  // ---- in-place inclusive prefix sums along z, y and x (border planes stay zero)
  for (int q = 0; q < spw; ++q) {
    if (__shfl_sync(0xffffffffu, cells, q) <= 0) continue;
    const Geo3 gq = shfl_geo3(g, q);
    const int Gx = gq.G[0], Gy = gq.G[1], Gz = gq.G[2], Py = Gy + 1, Pz = Gz + 1;
    uint32_t *P = tab + gq.base;
    for (int ln = lane; ln < Gx * Gy; ln += 32) {
      uint32_t *r = P + ((ln / Gy + 1) * Py + (ln % Gy + 1)) * Pz;
      for (int z = 1; z <= Gz; ++z) r[z] += r[z - 1];
    }
    __syncwarp();
    for (int ln = lane; ln < Gx * Gz; ln += 32) {
      uint32_t *r = P + (ln / Gz + 1) * Py * Pz + (ln % Gz + 1);
      for (int y = 1; y <= Gy; ++y) r[y * Pz] += r[(y - 1) * Pz];
    }
    __syncwarp();
    for (int ln = lane; ln < Gy * Gz; ln += 32) {
      uint32_t *r = P + (ln / Gz + 1) * Pz + (ln % Gz + 1);
      for (int x = 1; x <= Gx; ++x) r[x * Py * Pz] += r[(x - 1) * Py * Pz];
    }
    __syncwarp();
  }
  // ---- emit: lane l = row (q_l, a_l), the CTA kernel's rank path
  const Geo3 gl = shfl_geo3(g, q_l);
  float umn[3], umx[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    umn[x] = __shfl_sync(0xffffffffu, mn[x], q_l);
    umx[x] = __shfl_sync(0xffffffffu, mx[x], q_l);
  }
  auto rank_count = [&](int di, int dj, int dk) -> uint32_t {
    const int off[3] = {di, dj, dk};
    int c0[3], c1[3];
    for (int x = 0; x < 3; ++x) {
      const int S = a.act.D[x] + 1;
      const int f0 = (off[x] - a.act.c[x][a_l] - gl.n0[x] - 1) * S + a.act.le[x][a_l] - gl.fmin[x];
      c0[x] = max(f0, 0);
      c1[x] = min(f0 + S - 1, gl.G[x] - 1);
      if (c0[x] > c1[x]) return 0u;
    }
    const int Py = gl.G[1] + 1, Pz = gl.G[2] + 1;
    const uint32_t *P = tab + gl.base;
    auto at = [&](int x, int y, int z) { return P[(x * Py + y) * Pz + z]; };
    const int x0 = c0[0], y0 = c0[1], z0 = c0[2], x1 = c1[0] + 1, y1 = c1[1] + 1, z1 = c1[2] + 1;
    return at(x1, y1, z1) - at(x0, y1, z1) - at(x1, y0, z1) - at(x1, y1, z0) + at(x0, y0, z1) +
           at(x0, y1, z0) + at(x1, y0, z0) - at(x0, y0, z0);
  };
  const int64_t ir = sl * 32 + lane;
  const int64_t t = s_l / Nc, c = s_l % Nc;
  const int64_t li = c % a.nx, lj = (c / a.nx) % a.ny, lk = c / nxy;
  const int64_t nxt = (t + 1) * Nc;
  int e = 0;
  uint32_t sink = 0;
  int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
  if (kind_l == KIND_SAMPLE) {
    for (int x = 0; x < 3; ++x) {
      lo[x] = box_offset(umn[x], a.act.c[x][a_l], a.act.th[x][a_l], h);
      hi[x] = box_offset(umx[x], a.act.c[x][a_l], a.act.th[x][a_l], h);
      if (lo[x] < -h || hi[x] > h) atomicAdd(&a.cnt[CNT_OVERFLOW], 1ULL);
      lo[x] = max(lo[x], -h);
      hi[x] = min(hi[x], h);
    }
    for (int dk = lo[2]; dk <= hi[2]; ++dk)
      for (int dj = lo[1]; dj <= hi[1]; ++dj)
        for (int di = lo[0]; di <= hi[0]; ++di) {
          const uint32_t n = rank_count(di, dj, dk);
          if (!n) continue;
          const int64_t ip = li + di, jp = lj + dj, kp = lk + dk;
          const bool inside = ip >= 0 && ip < a.nx && jp >= 0 && jp < a.ny && kp >= 0 && kp < a.nz;
          if (!inside || a.obstacle[nxt + (kp * a.ny + jp) * a.nx + ip]) sink += n;
          else ++e;
        }
  } else if (kind_l == KIND_SINK) {
    sink = (uint32_t)a.N;
  }
  (void)L;
  const bool cap_hit = e + (sink > 0 ? 1 : 0) > a.row_cap;
  if (cap_hit) {
    atomicAdd(&a.cnt[CNT_ROW_CAP], 1ULL);
    e = 0;
  }
  int W = e;
  for (int off = 16; off > 0; off >>= 1) W = max(W, __shfl_xor_sync(0xffffffffu, W, off));
  unsigned long long base = 0;
  if (lane == 0 && W > 0) base = atomicAdd(&a.cnt[CNT_POOL_COLS], (unsigned long long)W);
  base = __shfl_sync(0xffffffffu, base, 0);
  const bool fits = (W == 0) || (base + (unsigned long long)W <= a.pool_cap_cols);
  if (!fits && lane == 0) atomicAdd(&a.cnt[CNT_POOL_FULL], 1ULL);
  const bool write = fits && !cap_hit;
  float Racc[3] = {0.f, 0.f, 0.f};
  uint32_t *dst = a.pool + base * 32 + lane;
  int k = 0;
  if (kind_l == KIND_SAMPLE) {
    const float F = a.act.F[a_l];
    const float g_s = a.gbar ? static_cast<const float *>(a.gbar)[s_l] : 0.f;
    for (int dk = lo[2]; dk <= hi[2]; ++dk)
      for (int dj = lo[1]; dj <= hi[1]; ++dj)
        for (int di = lo[0]; di <= hi[0]; ++di) {
          const uint32_t n = rank_count(di, dj, dk);
          if (!n) continue;
          const int64_t ip = li + di, jp = lj + dj, kp = lk + dk;
          const bool inside = ip >= 0 && ip < a.nx && jp >= 0 && jp < a.ny && kp >= 0 && kp < a.nz;
          const int64_t cp = (kp * a.ny + jp) * a.nx + ip;
          if (!inside || a.obstacle[nxt + cp]) continue;
          if (write) dst[(size_t)k * 32] = entry_word((int)(dk * nxy + dj * a.nx + di), n);
          ++k;
          const bool is_t = a.target[cp] != 0;
          const float g_sp = a.gbar ? static_cast<const float *>(a.gbar)[nxt + cp] : 0.f;
          for (int o = 0; o < a.rw.n_obj; ++o)
            Racc[o] = fmaf((float)n / (float)a.N, step_reward32(a.rw, a.rw.objs[o], F, g_s, g_sp, is_t), Racc[o]);
        }
    if (sink)
      for (int o = 0; o < a.rw.n_obj; ++o) Racc[o] = fmaf((float)sink / (float)a.N, (float)a.rw.r_out, Racc[o]);
  } else if (kind_l == KIND_SINK) {
    for (int o = 0; o < a.rw.n_obj; ++o) Racc[o] = (float)a.rw.r_out;
  }
  if (!write) {
    e = 0;
    k = 0;
  }
  if (write)
    for (int kk = k; kk < W; ++kk) dst[(size_t)kk * 32] = 0u;
  if (!fits) sink = 0;
  if (lane == 0) {
    a.slice_off[sl] = (fits && W > 0) ? (uint32_t)base : kNoSlice;
    a.slice_w[sl] = (fits && W > 0) ? (uint8_t)W : (uint8_t)0;
  }
  a.nnz[ir] = (uint8_t)e;
  a.sinkc[ir] = (uint16_t)sink;
  for (int o = 0; o < a.rw.n_obj; ++o) static_cast<float *>(a.R)[(int64_t)o * a.rows_pad + ir] = Racc[o];
  int dom = e, tot = e + (sink > 0 ? 1 : 0);
  for (int off = 16; off > 0; off >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, off);
    dom += __shfl_xor_sync(0xffffffffu, dom, off);
  }
  const int sampled = __popc(__ballot_sync(0xffffffffu, kind_l == KIND_SAMPLE));
  acc.tot += (unsigned long long)tot;
  acc.dom += (unsigned long long)dom;
  acc.samp += (unsigned long long)sampled * (unsigned long long)a.N;
  acc.maxw = max(acc.maxw, (unsigned long long)W);
  __syncwarp();
  for (int i = lane; i < (int)total; i += 32) tab[i] = 0u;   // zero for the next slice
  __syncwarp();
  return true;
}

__global__ void __launch_bounds__(32 * kWarps3, 2) build3d_warp_kernel(Build3Args a) {
  extern __shared__ __align__(16) uint32_t smem3w[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *tab = smem3w + (size_t)warp * a.cap3;
  for (int i = lane; i < a.cap3; i += 32) tab[i] = 0u;
  __syncwarp();
  Warp3Acc acc;
  unsigned long long next = 0;
  if (lane == 0) next = atomicAdd(&a.cnt[CNT_WORK], 1ULL);
  for (;;) {
    const int64_t sl = (int64_t)__shfl_sync(0xffffffffu, next, 0);
    if (sl >= a.n_slices) break;
    if (lane == 0) next = atomicAdd(&a.cnt[CNT_WORK], 1ULL);
    warp3_slice(a, sl, tab, acc);
  }
  if (lane == 0) {
    if (acc.tot) atomicAdd(&a.cnt[CNT_NNZ], acc.tot);
    if (acc.dom) atomicAdd(&a.cnt[CNT_DOMAIN], acc.dom);
    if (acc.samp) atomicAdd(&a.cnt[CNT_SAMPLES], acc.samp);
    if (acc.maxw) atomicMax(&a.cnt[CNT_MAXROW], acc.maxw);
  }
}

// FP32 landing-offset constants of one axis (same rule as the 2-D tables).
static void axis_constants(const float *d, int A, int32_t *c, float *th) {
  for (int a = 0; a < A; ++a) {
    const double dd = (double)d[a], fl = std::floor(dd);
    c[a] = (int32_t)fl;
    if (dd == fl) {
      th[a] = 2.0f;
    } else {
      const double t1 = (fl + 1.0) - dd;
      float f = (float)t1;
      if ((double)f < t1) f = std::nextafter(f, 2.0f);
      th[a] = f;
    }
  }
}

}  // namespace mdpgb

using namespace mdpgb;

static mdp_status arg3(const char *msg) {
  set_error(std::string("invalid argument: ") + msg);
  return MDP_ERR_ARG;
}

extern "C" mdp_status mdp_build3d(const mdp_env3d *env, const mdp_grid3d *grid, const mdp_actions3d *actions,
                                  int32_t N, int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj,
                                  void *stream, mdp_model *out) {
  return mdp_build3d_ex(env, grid, actions, N, subgrid_L, objs_h, n_obj, nullptr, stream, out);
}

extern "C" mdp_status mdp_build3d_ex(const mdp_env3d *env, const mdp_grid3d *grid, const mdp_actions3d *actions,
                                     int32_t N, int32_t subgrid_L, const int32_t *objs_h, int32_t n_obj,
                                     const mdp_build3d_opts *opts, void *stream, mdp_model *out) {
  if (!out) return arg3("out is NULL");
  *out = nullptr;
  mdp_status s = check_device();
  if (s != MDP_OK) return s;
  if (!env || !grid || !actions || !objs_h) return arg3("NULL pointer");
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->nt < 1 || !(grid->dx > 0) || !(grid->dt > 0))
    return arg3("grid");
  if (N < 1 || N > 65535) return arg3("N must be in [1, 65535]");
  if (subgrid_L < 1 || subgrid_L > kMaxL3 || subgrid_L % 2 == 0) return arg3("subgrid_L must be odd in [1, 11]");
  if (n_obj < 1 || n_obj > 3) return arg3("n_obj must be 1, 2 or 3");
  if (env->K < 0 || env->K > kMaxModes) return arg3("K");
  if (env->precision != MDP_FP32 && env->precision != MDP_FP64_CHECK) return arg3("precision");
  if (!env->vbar || !env->obstacle || !env->target || (env->K > 0 && !env->modes))
    return arg3("vbar, modes, obstacle and target must be non-NULL");
  if (env->K > 0 && !env->coeffs && !env->sigma_h) return arg3("need coeffs or sigma_h");
  for (int o = 0; o < n_obj; ++o) {
    if (objs_h[o] < 0 || objs_h[o] > 2) return arg3("unknown objective");
    if (objs_h[o] == MDP_OBJ_NET_ENERGY && !env->gbar) return arg3("net energy needs gbar");
  }
  const int A = actions->A;
  if (A < 1 || A > kMaxActions || !actions->table_h) return arg3("A must be in [1, 32] with a table");
  const int h = (subgrid_L - 1) / 2;
  const int64_t nxy = (int64_t)grid->nx * grid->ny;
  if ((int64_t)h * (nxy + grid->nx + 1) > 32767)
    return arg3("sub-grid half-width * (nx*ny + nx + 1) must be <= 32767 (16-bit successor offsets)");
  const int prec = env->precision;
  const size_t fsz = prec == MDP_FP64_CHECK ? 8 : 4;
  const double lam = grid->dt / grid->dx;
  cudaStream_t st = (cudaStream_t)stream;

  Build3Args ba;
  memset(&ba, 0, sizeof(ba));
  for (int a = 0; a < A; ++a) {
    for (int x = 0; x < 3; ++x) {
      const double d = actions->table_h[4 * a + x];
      if (!std::isfinite(d)) return arg3("action table holds a non-finite value");
      ba.act.d64[x][a] = d;
      ba.act.dl[x][a] = (float)(d * lam);
    }
    ba.act.F64[a] = actions->table_h[4 * a + 3];
    ba.act.F[a] = (float)actions->table_h[4 * a + 3];
  }
  for (int x = 0; x < 3; ++x) axis_constants(ba.act.dl[x], A, ba.act.c[x], ba.act.th[x]);
  // rank counting tables: the distinct step thresholds of each axis
  bool rank_ok = prec == MDP_FP32 && !(opts && opts->per_action);
  for (int x = 0; x < 3; ++x) {
    std::vector<float> T;
    for (int a = 0; a < A; ++a)
      if (ba.act.th[x][a] < 2.0f) T.push_back(ba.act.th[x][a]);
    std::sort(T.begin(), T.end());
    T.erase(std::unique(T.begin(), T.end()), T.end());
    if ((int)T.size() > kRank3) {
      rank_ok = false;
      T.resize(kRank3);
    }
    ba.act.D[x] = (int32_t)T.size();
    for (int i = 0; i < kRank3; ++i) ba.act.T[x][i] = i < (int)T.size() ? T[i] : 2.0f;
    for (int a = 0; a < A; ++a) {
      int le = (int)T.size() + 1;   // an integer displacement never steps
      if (ba.act.th[x][a] < 2.0f) le = (int)(std::upper_bound(T.begin(), T.end(), ba.act.th[x][a]) - T.begin());
      ba.act.le[x][a] = (int8_t)le;
    }
  }

  mdp_model_t *m = new mdp_model_t();
  memset(m, 0, sizeof(*m));
  auto fail = [&](mdp_status code) {
    cudaStreamSynchronize(st);
    free_model_on_stream(m, st);
    return code;
  };
#define TRY3(expr)                                                \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return fail(cuda_fail(_e, #expr));     \
  } while (0)
  cudaGetDevice(&m->device);
  m->nx = grid->nx; m->ny = (int32_t)(grid->ny * grid->nz); m->nt = grid->nt;   // Nc = nx * (ny * nz)
  m->K = env->K; m->N = N; m->A = A; m->precision = prec; m->n_obj = n_obj;
  for (int o = 0; o < n_obj; ++o) m->objs[o] = objs_h[o];
  m->Nc = nxy * grid->nz; m->nS = m->Nc * grid->nt; m->dx = grid->dx; m->dt = grid->dt;
  int A_pad = 1;
  while (A_pad < A) A_pad <<= 1;
  m->A_pad = A_pad;
  m->spw = 32 / A_pad;
  m->n_slices = (m->nS + m->spw - 1) / m->spw;
  m->rows_pad = m->n_slices * 32;
  m->L = subgrid_L;
  m->h = h;
  m->nbins = subgrid_L * subgrid_L * subgrid_L;
  const int row_cap = std::min(255, m->nbins + 1);
  m->row_cap = row_cap;
  RewardParams rw;
  memset(&rw, 0, sizeof(rw));
  rw.c_f = actions->c_f; rw.c_r = actions->c_r; rw.r_term = actions->r_term;
  rw.r_out = actions->r_outbound; rw.dt = grid->dt; rw.dx = grid->dx; rw.n_obj = n_obj;
  for (int o = 0; o < n_obj; ++o) rw.objs[o] = objs_h[o];
  m->rw = rw;

  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaEventRecord(ev0, st);
  TRY3(dev_alloc((void **)&m->cnt, sizeof(unsigned long long) * CNT_N, st));
  TRY3(cudaMemsetAsync(m->cnt, 0, sizeof(unsigned long long) * CNT_N, st));
  const void *Y = env->coeffs;
  void *Yown = nullptr;
  double *sig_d = nullptr;
  int launches = 0;
  if (!Y && env->K > 0) {
    TRY3(dev_alloc(&Yown, fsz * (size_t)grid->nt * N * env->K, st));
    TRY3(dev_alloc((void **)&sig_d, sizeof(double) * env->K, st));
    TRY3(cudaMemcpyAsync(sig_d, env->sigma_h, sizeof(double) * env->K, cudaMemcpyHostToDevice, st));
    TRY3(launch_sample_coeffs(grid->nt, N, env->K, sig_d, env->seed, env->mdp_id,
                              prec == MDP_FP64_CHECK ? (double *)Yown : nullptr,
                              prec == MDP_FP32 ? (float *)Yown : nullptr, m->cnt + CNT_CAPPED, st));
    Y = Yown;
    ++launches;
  }
  auto release = [&]() {
    dev_free(Yown, st);
    dev_free(sig_d, st);
    Yown = nullptr;
    sig_d = nullptr;
  };
  // model memory: the entry pool sized for 8 columns per slice first, rebuilt
  // once with the worst case if that runs out
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const uint64_t budget_cols = (uint64_t)(0.6 * (double)free_b) / 128;
  auto cols_for = [&](int width) {
    uint64_t c = (uint64_t)m->n_slices * (uint64_t)std::min(width, row_cap) + 64;
    return std::max<uint64_t>(1, std::min(c, budget_cols));
  };
  uint64_t cap_cols = cols_for(8);
  TRY3(dev_alloc((void **)&m->pool, (size_t)cap_cols * 128, st));
  TRY3(dev_alloc((void **)&m->slice_off, sizeof(uint32_t) * (size_t)m->n_slices, st));
  TRY3(dev_alloc((void **)&m->slice_w, (size_t)m->n_slices, st));
  TRY3(dev_alloc((void **)&m->nnz, (size_t)m->rows_pad, st));
  TRY3(dev_alloc((void **)&m->sinkc, sizeof(uint16_t) * (size_t)m->rows_pad, st));
  TRY3(dev_alloc(&m->R, fsz * (size_t)m->rows_pad * n_obj, st));
  TRY3(dev_alloc((void **)&m->cls, (size_t)m->nS, st));
  TRY3(dev_alloc((void **)&m->delta, sizeof(int32_t) * (size_t)subgrid_L * subgrid_L, st));
  // cell classes over the flattened (k, j, i) cells (the solver's policy rule)
  TRY3(launch_prepare(env->obstacle, env->target, m->cls, grid->nx, m->ny, grid->nt, m->delta, subgrid_L, st));
  ++launches;

  ba.nx = grid->nx; ba.ny = grid->ny; ba.nz = grid->nz; ba.nt = grid->nt; ba.K = env->K; ba.N = N; ba.A = A;
  ba.A_pad = A_pad; ba.spw = m->spw; ba.L = subgrid_L; ba.h = h; ba.row_cap = row_cap;
  ba.rank_ok = (rank_ok && m->spw <= kRankSpw) ? 1 : 0;
  ba.Nc = m->Nc; ba.nS = m->nS; ba.n_slices = m->n_slices; ba.rows_pad = m->rows_pad;
  ba.lam = (float)lam; ba.dx = grid->dx; ba.dt = grid->dt;
  ba.vbar = env->vbar; ba.modes = env->modes; ba.Y = Y; ba.gbar = env->gbar;
  ba.cls = m->cls; ba.target = env->target; ba.obstacle = env->obstacle;
  ba.rw = rw;
  ba.slice_off = m->slice_off; ba.slice_w = m->slice_w; ba.nnz = m->nnz; ba.sinkc = m->sinkc;
  ba.R = m->R; ba.cnt = m->cnt;
  // shared memory: the L^3 window plus the staged velocities of one chunk
  const size_t win = (size_t)m->nbins * 128;
  const size_t per_item = 3 * fsz;
  int chunk = (int)std::min<size_t>((size_t)N, (64 * 1024) / (per_item * m->spw));
  chunk = std::max(chunk, 1);
  ba.chunk = chunk;
  const size_t smem = win + (((size_t)chunk * m->spw * per_item + 15) & ~(size_t)15) + (size_t)8 * m->spw * 6 * fsz;
  const void *kfn = prec == MDP_FP64_CHECK ? (const void *)build3d_kernel<double> : (const void *)build3d_kernel<float>;
  TRY3(allow_max_smem(kfn));
  int per_sm = 0;
  TRY3(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 256, smem));
  if (per_sm < 1) {
    release();
    set_error("the 3-D window does not fit shared memory (reduce subgrid_L)");
    return fail(MDP_ERR_ARG);
  }
  const int64_t blocks = std::min<int64_t>((int64_t)num_sms() * per_sm, m->n_slices);
  // FP32 rank counting: the warp-per-slice kernel first, the CTA kernel over
  // the slices it leaves
  const bool use_warp = prec == MDP_FP32 && ba.rank_ok;
  uint32_t *defer = nullptr;
  int64_t wblocks = 0;
  size_t wsmem = 0;
  if (use_warp) {
    ba.cap3 = kCap3;
    wsmem = (size_t)kWarps3 * kCap3 * 4;
    TRY3(dev_alloc((void **)&defer, sizeof(uint32_t) * (size_t)m->n_slices, st));
    ba.defer = defer;
    TRY3(allow_max_smem((const void *)build3d_warp_kernel));
    int wper = 0;
    TRY3(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper, build3d_warp_kernel, 32 * kWarps3, wsmem));
    if (wper < 1) {
      release();
      dev_free(defer, st);
      set_error("the 3-D warp kernel's tables do not fit shared memory");
      return fail(MDP_ERR_CUDA);
    }
    wblocks = std::min<int64_t>((int64_t)num_sms() * wper, (m->n_slices + kWarps3 - 1) / kWarps3);
  }
  unsigned long long c[CNT_N];
  for (int attempt = 0;; ++attempt) {
    ba.pool = m->pool;
    ba.pool_cap_cols = cap_cols;
    if (prec == MDP_FP64_CHECK) {
      build3d_kernel<double><<<(unsigned)blocks, 256, smem, st>>>(ba);
    } else if (use_warp) {
      build3d_warp_kernel<<<(unsigned)wblocks, 32 * kWarps3, wsmem, st>>>(ba);
      TRY3(cudaGetLastError());
      Build3Args bd = ba;
      bd.defer_in = defer;
      build3d_kernel<float><<<(unsigned)blocks, 256, smem, st>>>(bd);
      ++launches;
    } else {
      build3d_kernel<float><<<(unsigned)blocks, 256, smem, st>>>(ba);
    }
    TRY3(cudaGetLastError());
    ++launches;
    TRY3(cudaMemcpyAsync(c, m->cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    TRY3(cudaStreamSynchronize(st));
    const uint64_t worst = cols_for(row_cap);
    if (c[CNT_POOL_FULL] == 0 || attempt > 0 || worst <= cap_cols) break;
    dev_free(m->pool, st);
    cap_cols = worst;
    TRY3(dev_alloc((void **)&m->pool, (size_t)cap_cols * 128, st));
    TRY3(cudaMemsetAsync(m->cnt, 0, sizeof(unsigned long long) * CNT_CAPPED, st));
    TRY3(cudaMemsetAsync(m->cnt + CNT_WORK, 0, sizeof(unsigned long long) * (CNT_N - CNT_WORK), st));
  }
  release();
  dev_free(defer, st);
  cudaEventRecord(ev1, st);
  cudaEventSynchronize(ev1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (c[CNT_OVERFLOW]) {
    set_error(std::to_string(c[CNT_OVERFLOW]) + " landing(s) left the neighbouring 3-D sub-grid; use a larger subgrid_L");
    return fail(MDP_ERR_SUBGRID_OVERFLOW);
  }
  if (c[CNT_ROW_CAP]) {
    set_error("a row had more successors than the row cap");
    return fail(MDP_ERR_ELL_OVERFLOW);
  }
  if (c[CNT_POOL_FULL]) {
    set_error("entry pool capacity exhausted (device memory budget)");
    return fail(MDP_ERR_OOM);
  }
  m->pool_cols = c[CNT_POOL_COLS];
  m->nnz_total = (int64_t)c[CNT_NNZ];
  m->nnz_domain = (int64_t)c[CNT_DOMAIN];
  m->max_row_nnz = (int32_t)c[CNT_MAXROW];
  m->samples = (int64_t)c[CNT_SAMPLES];
  m->deferred = use_warp ? (int64_t)c[CNT_DEFER_N] : 0;   // slices the CTA kernel built
  {   // compaction into a pool of exactly the columns in use, in slice order
    uint32_t *np = nullptr;
    TRY3(dev_alloc((void **)&np, (size_t)std::max<uint64_t>(m->pool_cols, 1) * 128, st));
    TRY3(launch_pool_reorder(m->pool, np, m->slice_off, m->slice_w, m->n_slices, st));
    m->pool_ordered = 1;
    dev_free(m->pool, st);
    m->pool = np;
    cap_cols = std::max<uint64_t>(m->pool_cols, 1);
  }
  m->build_ms = ms;
  m->kernel_ms = ms;
  m->launches = launches;
  m->device_bytes = (int64_t)cap_cols * 128 + 5 * m->n_slices + 3 * m->rows_pad +
                    (int64_t)fsz * m->rows_pad * n_obj + m->nS + 8 * CNT_N;
  *out = m;
#undef TRY3
  return MDP_OK;
}
