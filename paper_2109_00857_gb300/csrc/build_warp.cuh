// build_warp.cuh -- the warp-per-slice FP32 build (steps a2-a6 fused) as a
// device function, shared by the single-model kernel (build_warp.cu) and the
// batched kernel (build_warp_batch.cu).
//
// A warp works alone on one slice (spw states x A_pad actions, 32 rows) with
// private shared memory and no block-level barrier.  The landing offset of
// realization w under action a along x is floor(u_w + d_a) (Sec. II-A move,
// cell(); u = 1/2 + w dt/dx from the DO velocity, Sec. II-C, d_a the action's
// displacement), taken for the exact sum of the two floats:
//   floor(u + d) = floor(u) + c_a + [u - floor(u) >= th_a]
// with per-action constants c_a, th_a (ActionTable).  Sorting the distinct
// th_a (T_0 < ... < T_{D-1}) gives each realization one fractional rank
// rho = #{T <= u - floor(u)} that decides the step for every action at once
// ([u - floor(u) >= th_a] = [rho >= le_a]).  So a realization needs one count,
// not one per action:
//   pass 1   lanes form u for (state, realization) items and reduce the exact
//            per-state extremes (the offset is monotone in u, so they bound
//            every action's offsets: sub-grid check, bounding boxes).
//   pass 2   the same items again: the fine coordinate X = (floor(u) - n0) S +
//            rho (S = D + 1) per axis, one shared-memory count into the
//            state's fine table H[X][Y] (sized from the extremes).
//   prefix   in-place 2-D inclusive prefix sums of H.
//   emit     lane l = row (state q, action a): an offset bin (dx, dy) collects
//            exactly the fine cells X in [(dx - c_a - 1 - n0) S + le_a, + S)
//            (and likewise in y) -- a box whose count is four prefix lookups;
//            two scans of the row's bounding box count the entries (sink
//            folded), allocate the slice's columns and write the entry words
//            in ascending order with R(s,a) from the counts.
// Slices whose fine tables do not fit cap_bins cells are appended to a list
// that the CTA kernel of build_fp32.cu finishes with a full-window histogram
// and the same landing offsets, so a slice's output does not depend on which
// kernel built it.
#pragma once
#include "build_common.cuh"

namespace mdpgb {

// per-warp rank tables (32-bit words): TPx[33], TPy[33] as float2 pairs
// (T[i], T[i+1]), then Lx, Ly as bytes
constexpr int kTabPairs = kMaxActions + 1;
constexpr int kTab = 4 * kTabPairs + 2 * kRankBuckets / 4 + 2;   // even: float2 alignment kept

// Shared-memory words per warp: rank tables + fine tables, a multiple of 4
// so every warp's tables start 16-byte aligned.
__host__ __device__ constexpr int warp_words(int cap) { return (kTab + cap + 3) & ~3; }

__device__ __forceinline__ void red_add_shared(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Same FP32 operations as the CTA kernel: u = fma(w, lam, 1/2), w by an FMA
// chain over ascending k; non-finite values are pushed outside every sub-grid.
// Mode-count variants: KT > 0 exactly KT modes; KT < 0 at most -KT modes
// (runtime K, coefficients in registers); KT == 0 up to kMaxModes (runtime).
template <int KT>
constexpr int kPhi = KT > 0 ? KT : (KT < 0 ? -KT : kMaxModes);

template <int KT, bool CLAMP = true>
__device__ __forceinline__ float2 velocity_u(const float *__restrict__ yw, const float (&phx)[kPhi<KT>],
                                             const float (&phy)[kPhi<KT>], float vbx,
                                             float vby, int K, float lam) {
  float wx = vbx, wy = vby;
  if constexpr (KT < 0) {
    if ((K & 1) == 0) {   // even K: rows are 8-byte aligned (coeffs 16-byte aligned)
#pragma unroll
      for (int k = 0; k < -KT; k += 2) {
        if (k < K) {
          const float2 v = __ldg(reinterpret_cast<const float2 *>(yw + k));
          wx = fmaf(v.x, phx[k], wx); wy = fmaf(v.x, phy[k], wy);
          wx = fmaf(v.y, phx[k + 1], wx); wy = fmaf(v.y, phy[k + 1], wy);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < -KT; ++k) {
        if (k < K) {
          const float yk = __ldg(yw + k);
          wx = fmaf(yk, phx[k], wx);
          wy = fmaf(yk, phy[k], wy);
        }
      }
    }
  } else if constexpr (KT > 0 && (KT % 4) == 0) {
#pragma unroll
    for (int k = 0; k < KT; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(yw + k));
      wx = fmaf(v.x, phx[k], wx); wy = fmaf(v.x, phy[k], wy);
      wx = fmaf(v.y, phx[k + 1], wx); wy = fmaf(v.y, phy[k + 1], wy);
      wx = fmaf(v.z, phx[k + 2], wx); wy = fmaf(v.z, phy[k + 2], wy);
      wx = fmaf(v.w, phx[k + 3], wx); wy = fmaf(v.w, phy[k + 3], wy);
    }
  } else if constexpr (KT > 0) {
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const float yk = __ldg(yw + k);
      wx = fmaf(yk, phx[k], wx);
      wy = fmaf(yk, phy[k], wy);
    }
  } else {
    for (int k = 0; k < K; ++k) {
      const float yk = __ldg(yw + k);
      wx = fmaf(yk, phx[k], wx);
      wy = fmaf(yk, phy[k], wy);
    }
  }
  float ux = fmaf(wx, lam, 0.5f), uy = fmaf(wy, lam, 0.5f);
  if constexpr (CLAMP) {
    if (!(fabsf(ux) < 1e30f)) ux = 1e30f;
    if (!(fabsf(uy) < 1e30f)) uy = 1e30f;
  }
  return make_float2(ux, uy);
}

// The same velocity from a coefficient row already loaded (KT a multiple of
// 4): the identical FMA chain, so both forms give the same u bit for bit.
template <int KT>
__device__ __forceinline__ void load_row4(const float *__restrict__ yw, float4 (&y)[KT / 4]) {
#pragma unroll
  for (int v = 0; v < KT / 4; ++v) y[v] = __ldg(reinterpret_cast<const float4 *>(yw) + v);
}
template <int KT, bool CLAMP = true>
__device__ __forceinline__ float2 velocity_row4(const float4 (&y)[KT / 4], const float (&phx)[kPhi<KT>],
                                                const float (&phy)[kPhi<KT>], float vbx, float vby, float lam) {
  float wx = vbx, wy = vby;
#pragma unroll
  for (int v = 0; v < KT / 4; ++v) {
    const int k = 4 * v;
    wx = fmaf(y[v].x, phx[k], wx); wy = fmaf(y[v].x, phy[k], wy);
    wx = fmaf(y[v].y, phx[k + 1], wx); wy = fmaf(y[v].y, phy[k + 1], wy);
    wx = fmaf(y[v].z, phx[k + 2], wx); wy = fmaf(y[v].z, phy[k + 2], wy);
    wx = fmaf(y[v].w, phx[k + 3], wx); wy = fmaf(y[v].w, phy[k + 3], wy);
  }
  float ux = fmaf(wx, lam, 0.5f), uy = fmaf(wy, lam, 0.5f);
  if constexpr (CLAMP) {
    if (!(fabsf(ux) < 1e30f)) ux = 1e30f;
    if (!(fabsf(uy) < 1e30f)) uy = 1e30f;
  }
  return make_float2(ux, uy);
}

// Rank tables of one axis in a warp's table memory.
struct RankTab {
  const float2 *TP;    // TP[i] = (T[i], T[i+1]); T[i] = 2 for i >= D
  const uint8_t *L;    // thresholds below each bucket
  int M;               // most thresholds in one bucket
};

// #{i : T[i] <= f} for f in [0, 1].  The thresholds below f's bucket come
// from the lookup; those in the bucket follow them in T, and every later
// one exceeds f, so with at most two per bucket two comparisons finish it.
__device__ __forceinline__ int frac_rank(const RankTab &rt, float f) {
  int r = rt.L[min((int)(f * (float)kRankBuckets), kRankBuckets - 1)];
  if (rt.M <= 2) {
    const float2 t = rt.TP[r];
    return r + (t.x <= f ? 1 : 0) + (t.y <= f ? 1 : 0);
  }
  while (rt.TP[r].x <= f) ++r;   // T[D] = 2 > f ends it
  return r;
}

// Fine coordinate of u along one axis: (floor(u) - n0) S + rho(u - floor(u)).
__device__ __forceinline__ int fine_coord(float u, int n0, int S, const RankTab &rt) {
  const float n = floorf(u);
  return ((int)n - n0) * S + frac_rank(rt, u - n);
}

// Copies a model's rank tables into a warp's table memory (whole warp).
__device__ __forceinline__ void load_rank_tables(const BuildArgs &a, float *tab) {
  const int lane = threadIdx.x & 31;
  float2 *TPx = reinterpret_cast<float2 *>(tab), *TPy = TPx + kTabPairs;
  uint8_t *L = reinterpret_cast<uint8_t *>(TPy + kTabPairs);
  for (int i = lane; i < kTabPairs; i += 32) {
    TPx[i] = make_float2(a.act.Tx[i], a.act.Tx[i + 1]);
    TPy[i] = make_float2(a.act.Ty[i], a.act.Ty[i + 1]);
  }
  for (int b = lane; b < kRankBuckets; b += 32) {
    L[b] = a.act.Lx[b];
    L[kRankBuckets + b] = a.act.Ly[b];
  }
  __syncwarp();
}

__device__ __forceinline__ RankTab rank_tab(const BuildArgs &a, const float *tab, int axis) {
  const float2 *TP = reinterpret_cast<const float2 *>(tab) + axis * kTabPairs;
  const uint8_t *L = reinterpret_cast<const uint8_t *>(reinterpret_cast<const float2 *>(tab) + 2 * kTabPairs) +
                     axis * kRankBuckets;
  return RankTab{TP, L, axis ? a.act.My : a.act.Mx};
}

// A state's fine table: X in [xmin, xmin + gx), Y in [ymin, ymin + gy);
// prefix layout P[i * pitch + j], i <= gx, j <= gy, at word `base` of the
// warp's table memory (row 0 and column 0 stay zero; pitch is odd, so a
// warp's lanes walking rows i, i+1, ... hit distinct banks).
struct FineGeo {
  int n0x, n0y, xmin, ymin, gx, gy, pitch, base;
};

__device__ __forceinline__ FineGeo shfl_geo(const FineGeo &g, int src) {
  FineGeo o;
  o.n0x = __shfl_sync(0xffffffffu, g.n0x, src);
  o.n0y = __shfl_sync(0xffffffffu, g.n0y, src);
  o.xmin = __shfl_sync(0xffffffffu, g.xmin, src);
  o.ymin = __shfl_sync(0xffffffffu, g.ymin, src);
  o.gx = __shfl_sync(0xffffffffu, g.gx, src);
  o.gy = __shfl_sync(0xffffffffu, g.gy, src);
  o.pitch = __shfl_sync(0xffffffffu, g.pitch, src);
  o.base = __shfl_sync(0xffffffffu, g.base, src);
  return o;
}

// Per-warp totals, added to the model's counters by warp_flush().
struct WarpAcc {
  unsigned long long samples = 0, nnz = 0, dom = 0, maxrow = 0;
};

__device__ __forceinline__ void warp_flush(const BuildArgs &a, WarpAcc &acc) {
  if ((threadIdx.x & 31) == 0) {
    if (acc.nnz) atomicAdd(&a.cnt[CNT_NNZ], acc.nnz);
    if (acc.dom) atomicAdd(&a.cnt[CNT_DOMAIN], acc.dom);
    if (acc.samples) atomicAdd(&a.cnt[CNT_SAMPLES], acc.samples);
    if (acc.maxrow) atomicMax(&a.cnt[CNT_MAXROW], acc.maxrow);
  }
  acc = WarpAcc();
}

// One warp builds slice sl of model a (see the file comment).  grid holds
// a.cap_bins words of fine-table memory, tab the model's rank tables
// (kTab words, filled by load_rank_tables).
// SPW > 0: states per warp fixed at compile time (1: A = 32, 2: A = 16);
// SPW == 0: runtime spw.  KT: see kPhi.  HYB: rows beyond row_cap keep
// their tail in the slice's spill block; without it (the batched build, whose
// models keep no spill area) such a row is counted in CNT_ROW_CAP and left
// empty -- the lighter emit keeps the batched kernel free of register spills.
template <int KT, int SPW, bool HYB>
__device__ __forceinline__ void warp_slice(const BuildArgs &a, int64_t sl, uint32_t *grid, float *tab,
                                           WarpAcc &acc) {
  const int lane = threadIdx.x & 31;
  const int spw = SPW > 0 ? SPW : a.spw;
  const int K = KT > 0 ? KT : a.K;
  // lane role: row (q_l, a_l)
  const int q_l = lane / a.A_pad, a_l = lane % a.A_pad;
  const bool act_ok = a_l < a.A;
  // item role: state q_t, realizations wi, wi + 32/spw, ...
  const int q_t = lane % spw, wi = lane / spw, wstep = 32 / spw;
  const float lam = a.lam;
  // model scalars in registers: the loops below also store to memory, so
  // loads through `a` (global memory in the batched kernel) would repeat
  const int N = a.N, nx = a.nx, ny = a.ny;
  const int64_t Nc = a.Nc;
  const uint8_t *__restrict__ cls = a.cls;
  const float *__restrict__ gbar = static_cast<const float *>(a.gbar);
  const float *Yall = static_cast<const float *>(a.Y);
  const float *vbar = static_cast<const float *>(a.vbar);
  const float *modes = static_cast<const float *>(a.modes);
  const float invN = 1.0f / (float)N;
  const RankTab rx = rank_tab(a, tab, 0), ry = rank_tab(a, tab, 1);   // (load_rank_tables)
  const int Sx = a.act.Dx + 1, Sy = a.act.Dy + 1;

  const int64_t s_l = sl * spw + q_l;
  int kind_l = state_kind(a, s_l);
  if (!act_ok) kind_l = KIND_NONE;
  const int64_t s_t = sl * spw + q_t;
  const int kind_t = state_kind(a, s_t);
  const bool any_sample = __any_sync(0xffffffffu, kind_t == KIND_SAMPLE);

  bool active = kind_l == KIND_SAMPLE;
  int lox = 0, hix = -1, loy = 0, hiy = -1;
  FineGeo gl{};   // fine table of state q_l (emit)
  if (any_sample) {
    float phx[kPhi<KT>], phy[kPhi<KT>];
    float vbx = 0.f, vby = 0.f;
    const float *Yt = Yall;
    if (kind_t == KIND_SAMPLE) {
      const int64_t t = s_t / Nc, c = s_t % Nc;
      vbx = vbar[2 * s_t];
      vby = vbar[2 * s_t + 1];
#pragma unroll
      for (int k = 0; k < kPhi<KT>; ++k) {
        if (KT == 0 && k >= K) break;
        if (KT < 0 && k >= K) {
          phx[k] = 0.f;
          phy[k] = 0.f;
          continue;
        }
        const float2 ph = *reinterpret_cast<const float2 *>(modes + 2 * ((t * K + k) * Nc + c));
        phx[k] = ph.x;
        phy[k] = ph.y;
      }
      Yt = Yall + (size_t)t * N * K;
    }
    // ---- pass 1: exact extremes of u per state
    float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    if (kind_t == KIND_SAMPLE) {
      for (int w = wi; w < N; w += wstep) {
        const float2 u = velocity_u<KT>(Yt + (size_t)w * K, phx, phy, vbx, vby, K, lam);
        mnx = fminf(mnx, u.x); mxx = fmaxf(mxx, u.x);
        mny = fminf(mny, u.y); mxy = fmaxf(mxy, u.y);
      }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      if (off < spw) break;
      mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, off));
      mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, off));
      mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, off));
      mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, off));
    }
    // every lane now holds the extremes of its item state q_t; lane q < spw
    // sizes state q's fine table
    FineGeo g{};
    int cells = 0;
    bool tame = true;
    if (kind_t == KIND_SAMPLE) {
      // non-finite (clamped to 1e30) or far velocities: the CTA kernel's path
      tame = mnx > -1e6f && mxx < 1e6f && mny > -1e6f && mxy < 1e6f;
    }
    if (kind_t == KIND_SAMPLE && !tame) {
      cells = a.cap_bins + 1;
    } else if (kind_t == KIND_SAMPLE) {
      g.n0x = (int)floorf(mnx);
      g.n0y = (int)floorf(mny);
      g.xmin = fine_coord(mnx, g.n0x, Sx, rx);
      g.ymin = fine_coord(mny, g.n0y, Sy, ry);
      const long long gx = (long long)fine_coord(mxx, g.n0x, Sx, rx) - g.xmin + 1;
      const long long gy = (long long)fine_coord(mxy, g.n0y, Sy, ry) - g.ymin + 1;
      const long long pitch = (gy + 1) | 1;
      const long long c = (gx + 1) * pitch;
      // a huge spread (only with a sub-grid overflow) cannot be tabled
      cells = (gx <= 65536 && gy <= 65536 && c <= (long long)a.cap_bins) ? (int)c : a.cap_bins + 1;
      g.gx = (int)min(gx, 65536LL);
      g.gy = (int)min(gy, 65536LL);
      g.pitch = (int)min(pitch, 65537LL);
    }
    int total = 0;
    for (int q = 0; q < spw; ++q) {   // table bases, states in order
      const int cq = __shfl_sync(0xffffffffu, cells, q);
      if (lane == q) g.base = total;
      total += cq;
    }
    const FineGeo gt = shfl_geo(g, q_t);
    gl = shfl_geo(g, q_l);
    const float lmnx = __shfl_sync(0xffffffffu, mnx, q_l), lmxx = __shfl_sync(0xffffffffu, mxx, q_l);
    const float lmny = __shfl_sync(0xffffffffu, mny, q_l), lmxy = __shfl_sync(0xffffffffu, mxy, q_l);
    const int cxa = act_ok ? a.act.cx[a_l] : 0, cya = act_ok ? a.act.cy[a_l] : 0;
    const float thxa = act_ok ? a.act.thx[a_l] : 2.f, thya = act_ok ? a.act.thy[a_l] : 2.f;
    if (active) {
      lox = land_offset(lmnx, cxa, thxa); hix = land_offset(lmxx, cxa, thxa);
      loy = land_offset(lmny, cya, thya); hiy = land_offset(lmxy, cya, thya);
      if (lox < -a.h || hix > a.h || loy < -a.h || hiy > a.h) {   // sub-grid overflow
        active = false;
        atomicAdd(&a.cnt[CNT_OVERFLOW], 1ULL);
      }
    }
    if (total > a.cap_bins) {   // too wide for this warp: the CTA kernel builds it
      if (lane == 0) {
        const unsigned long long i = atomicAdd(&a.cnt[CNT_DEFER_N], 1ULL);
        a.defer[i] = (uint32_t)sl;
      }
      return;
    }
    for (int i = lane; i < total; i += 32) grid[i] = 0;
    __syncwarp();
    // ---- pass 2: one count per realization in its state's fine table
    if (kind_t == KIND_SAMPLE) {
      const uint32_t gbase = smem_u32(grid + gt.base);
      // every u of the state is finite and within the extremes of pass 1 (the
      // same floats): X in [0, gx), Y in [0, gy) with no clamping
      auto count = [&](float2 u) {
        const int X = fine_coord(u.x, gt.n0x, Sx, rx) - gt.xmin;
        const int Y = fine_coord(u.y, gt.n0y, Sy, ry) - gt.ymin;
        red_add_shared(gbase + 4u * (uint32_t)((X + 1) * gt.pitch + Y + 1), 1u);
      };
      if constexpr (KT > 0 && KT % 4 == 0) {
        // the next realization's coefficient row is loaded while this one
        // is counted (its L2 latency overlaps the rank lookups); two trips
        // per loop iteration (measured: 127 ms against 131 ms unrolled once)
        float4 yn[KT / 4];
        if (wi < N) load_row4<KT>(Yt + (size_t)wi * K, yn);
#pragma unroll 2
        for (int w = wi; w < N; w += wstep) {
          float4 yc[KT / 4];
#pragma unroll
          for (int v = 0; v < KT / 4; ++v) yc[v] = yn[v];
          if (w + wstep < N) load_row4<KT>(Yt + (size_t)(w + wstep) * K, yn);
          count(velocity_row4<KT, false>(yc, phx, phy, vbx, vby, lam));
        }
      } else {
#pragma unroll 1
        for (int w = wi; w < N; w += wstep) count(velocity_u<KT, false>(Yt + (size_t)w * K, phx, phy, vbx, vby, K, lam));
      }
    }
    __syncwarp();
    // ---- prefix: P[i][j] = sum of H[X'][Y'] over X' < i, Y' < j
    for (int q = 0; q < spw; ++q) {
      const FineGeo gq = shfl_geo(g, q);
      if (gq.gx <= 0 || gq.gy <= 0 || __shfl_sync(0xffffffffu, cells, q) == 0) continue;
      uint32_t *P = grid + gq.base;
      for (int i = 1 + lane; i <= gq.gx; i += 32) {
        uint32_t *row = P + (size_t)i * gq.pitch;
        uint32_t v = 0;
        for (int j = 1; j <= gq.gy; ++j) {
          v += row[j];
          row[j] = v;
        }
      }
      __syncwarp();
      for (int j = 1 + lane; j <= gq.gy; j += 32) {
        uint32_t v = 0;
        for (int i = 1; i <= gq.gx; ++i) {
          v += P[(size_t)i * gq.pitch + j];
          P[(size_t)i * gq.pitch + j] = v;
        }
      }
      __syncwarp();
    }
  }

  // ---- emit: count entries, allocate the slice, write
  // count of offset bin (di, dj) of this lane's row: a box of the prefix table
  const uint32_t *P = grid + gl.base;
  const int cxa = act_ok ? a.act.cx[a_l] : 0, cya = act_ok ? a.act.cy[a_l] : 0;
  const int xoff = (-cxa - 1 - gl.n0x) * Sx + (act_ok ? a.act.lex[a_l] : 0) - gl.xmin;
  const int yoff = (-cya - 1 - gl.n0y) * Sy + (act_ok ? a.act.ley[a_l] : 0) - gl.ymin;
  auto bin_count = [&](int di, int dj) -> uint32_t {
    const int x0 = di * Sx + xoff, y0 = dj * Sy + yoff;
    const int i0 = min(max(x0, 0), gl.gx), i1 = min(max(x0 + Sx, 0), gl.gx);
    const int j0 = min(max(y0, 0), gl.gy), j1 = min(max(y0 + Sy, 0), gl.gy);
    const int r0 = i0 * gl.pitch, r1 = i1 * gl.pitch;
    return P[r1 + j1] - P[r0 + j1] - P[r1 + j0] + P[r0 + j0];
  };
  const int64_t ir = sl * 32 + lane;
  int e = 0;
  uint32_t sink = 0;
  const int64_t t = s_l / Nc, c = s_l % Nc;
  const int ci = (int)(c % nx), cj = (int)(c / nx);
  const int64_t nxt = (t + 1) * Nc;
  if (kind_l == KIND_SAMPLE && active) {
    for (int dj = loy; dj <= hiy; ++dj) {
      const int jp = cj + dj;
      for (int di = lox; di <= hix; ++di) {
        const uint32_t n = bin_count(di, dj);
        if (n == 0) continue;
        const int ip = ci + di;
        const bool inside = ip >= 0 && ip < nx && jp >= 0 && jp < ny;
        const uint8_t cc = inside ? cls[nxt + (int64_t)jp * nx + ip] : CLS_OBSTACLE;
        if (cc & CLS_OBSTACLE) sink += n;
        else ++e;
      }
    }
  } else if (kind_l == KIND_SINK) {
    sink = (uint32_t)N;
  }
  // the first row_cap in-domain successors go to the ELL columns, the rest to
  // the slice's spill block (HYB)
  bool cap_hit = false;
  if constexpr (!HYB) {
    cap_hit = e > a.row_cap;
    if (cap_hit) {
      atomicAdd(&a.cnt[CNT_ROW_CAP], 1ULL);
      e = 0;
    }
  }
  int ell = min(e, a.row_cap);
  int64_t sp_at = -1;
  if constexpr (HYB) sp_at = spill_alloc(a, sl, e - ell);
  int W = ell;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) W = max(W, __shfl_xor_sync(0xffffffffu, W, off));
  unsigned long long base = 0;
  if (lane == 0 && W > 0) base = atomicAdd(&a.cnt[CNT_POOL_COLS], (unsigned long long)W);
  base = __shfl_sync(0xffffffffu, base, 0);
  const bool fits = (W == 0) || (base + (unsigned long long)W <= a.pool_cap_cols);
  if (!fits && lane == 0) atomicAdd(&a.cnt[CNT_POOL_FULL], 1ULL);
  float Racc[3] = {0.f, 0.f, 0.f};
  uint32_t *dst = a.pool + base * 32 + lane;
  const bool write = fits && !cap_hit;
  int k = 0;
  if (kind_l == KIND_SAMPLE && active) {
    const float F = a.act.F[a_l];
    const float g_s = gbar ? gbar[s_l] : 0.f;
    for (int dj = loy; dj <= hiy; ++dj) {
      const int jp = cj + dj;
      for (int di = lox; di <= hix; ++di) {
        const uint32_t n = bin_count(di, dj);
        if (n == 0) continue;
        const int ip = ci + di;
        const bool inside = ip >= 0 && ip < nx && jp >= 0 && jp < ny;
        const uint8_t cc = inside ? cls[nxt + (int64_t)jp * nx + ip] : CLS_OBSTACLE;
        if (cc & CLS_OBSTACLE) continue;
        const uint32_t wd = entry_word(dj * nx + di, n);
        if (k < ell) {
          if (write) dst[(size_t)k * 32] = wd;
        } else if (sp_at >= 0) {
          a.spill[sp_at + (k - ell)] = wd;
        }
        ++k;
        const bool is_t = (cc & CLS_TARGET) != 0;
        const float g_sp = gbar ? gbar[nxt + (int64_t)jp * nx + ip] : 0.f;
        const float p = (float)n * invN;
        for (int o = 0; o < a.rw.n_obj; ++o)
          Racc[o] = fmaf(p, step_reward32(a.rw, a.rw.objs[o], F, g_s, g_sp, is_t), Racc[o]);
      }
    }
    if (sink)
      for (int o = 0; o < a.rw.n_obj; ++o) Racc[o] = fmaf((float)sink * invN, (float)a.rw.r_out, Racc[o]);
  } else if (kind_l == KIND_SINK) {
    for (int o = 0; o < a.rw.n_obj; ++o) Racc[o] = (float)a.rw.r_out;
  }
  if (!write) {
    e = 0;
    ell = 0;
  }
  if (write)   // zero padding up to the slice width
    for (int kk = ell; kk < W; ++kk) dst[(size_t)kk * 32] = 0u;
  if (e > ell) atomicMax(&a.cnt[CNT_MAXLEN], (unsigned long long)e);
  if (!fits) sink = 0;
  if (lane == 0) {
    a.slice_off[sl] = (fits && W > 0) ? (uint32_t)base : kNoSlice;
    a.slice_w[sl] = (fits && W > 0) ? (uint8_t)W : (uint8_t)0;
  }
  a.nnz[ir] = (uint8_t)ell;
  a.sinkc[ir] = (uint16_t)sink;
  for (int o = 0; o < a.rw.n_obj; ++o) static_cast<float *>(a.R)[(int64_t)o * a.rows_pad + ir] = Racc[o];
  int dom = e;
  e += (sink > 0 ? 1 : 0);   // stored successors incl. the sink, for the totals below
  int tot = e;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, off);
    dom += __shfl_xor_sync(0xffffffffu, dom, off);
  }
  const int sampled = __popc(__ballot_sync(0xffffffffu, kind_l == KIND_SAMPLE && active));
  if (lane == 0) {
    acc.nnz += (unsigned long long)tot;
    acc.dom += (unsigned long long)dom;
    acc.samples += (unsigned long long)sampled * (unsigned long long)N;
    if ((unsigned long long)W > acc.maxrow) acc.maxrow = W;
  }
}

}  // namespace mdpgb
