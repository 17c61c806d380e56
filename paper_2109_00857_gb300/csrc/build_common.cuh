// build_common.cuh -- state classification, one-step rewards and the emit
// (K_COUNT + K_REDUCE_TO_COO + K_COMPUTE_MEAN of Sec. III-C, fused) shared by
// the FP32 and FP64-check build kernels.
#pragma once
#include "mdp_internal.cuh"

namespace mdpgb {

// What a start state needs (Alg. 2 branches on terminal / obstacle).
enum : int {
  KIND_SAMPLE = 0,    // free state below the horizon: Monte-Carlo counting
  KIND_TERMINAL = 1,  // target cell: absorbing, no transitions (V = 0)
  KIND_SINK = 2,      // obstacle start state, or t = nt-1: every realization -> sink
  KIND_NONE = 3       // padding lane (s >= |S| or a >= A)
};

__device__ __forceinline__ int state_kind(const BuildArgs &a, int64_t s) {
  if (s >= a.nS) return KIND_NONE;
  const uint8_t c = a.cls[s];
  if (c & CLS_TARGET) return KIND_TERMINAL;     // terminal is tested first (Alg. 2)
  if (c & CLS_OBSTACLE) return KIND_SINK;
  if (s / a.Nc == a.nt - 1) return KIND_SINK;   // beyond the finite horizon
  return KIND_SAMPLE;
}

// FP32 landing offset along one axis (Sec. II-A move, cell()): floor(u + d)
// for the exact sum of the floats u and d, as floor(u) + c + [u - floor(u)
// >= th] with the per-action constants of ActionTable.  Monotone in u, so
// the offsets of a state's extreme u bound every sample's offset.
__device__ __forceinline__ int land_offset(float u, int c, float th) {
  const float n = floorf(u);
  return (int)n + c + ((u - n) >= th ? 1 : 0);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// --------------------------------------------------------------- rewards --
// One-step reward of a landing inside the domain and free of obstacles
// (Eqs. Rsa_time, Rsa_energyConsumption, Rsa_NetEnergy; mean scalar field
// only, Sec. III-A), plus r_term on a target cell.  FP64: explicit
// round-to-nearest operations in a fixed order (no contraction).
__device__ __forceinline__ double step_reward64(const RewardParams &rw, int obj, double F,
                                                double g_s, double g_sp, bool is_target) {
  double r;
  if (obj == MDP_OBJ_TIME) {
    r = -rw.dt;
  } else if (obj == MDP_OBJ_ENERGY) {
    double eF = __dmul_rn(__dmul_rn(rw.c_f, F), F);
    r = __dmul_rn(-eF, rw.dt);
  } else {
    double eF = __dmul_rn(__dmul_rn(rw.c_f, F), F);
    double hc = __dmul_rn(0.5, rw.c_r);
    r = __dmul_rn(__dadd_rn(__dadd_rn(-eF, __dmul_rn(hc, g_s)), __dmul_rn(hc, g_sp)), rw.dt);
  }
  if (is_target) r = __dadd_rn(r, rw.r_term);
  return r;
}

__device__ __forceinline__ float step_reward32(const RewardParams &rw, int obj, float F,
                                               float g_s, float g_sp, bool is_target) {
  float r;
  if (obj == MDP_OBJ_TIME) {
    r = -(float)rw.dt;
  } else if (obj == MDP_OBJ_ENERGY) {
    r = -((float)rw.c_f * F * F) * (float)rw.dt;
  } else {
    const float hc = 0.5f * (float)rw.c_r;
    r = ((-((float)rw.c_f * F * F) + hc * g_s) + hc * g_sp) * (float)rw.dt;
  }
  if (is_target) r += (float)rw.r_term;
  return r;
}

template <typename RT>
__device__ __forceinline__ RT load_field(const void *p, int64_t i) {
  return static_cast<const RT *>(p)[i];
}

// ------------------------------------------------------------------ emit --
// Entry word of an in-domain successor: low 16 bits the signed offset
// s' - (s + Nc) = dj*Nx + di, high 16 bits the count.  Padding words are 0
// (offset 0, count 0: a harmless zero term).  The sink's count lives in
// sinkc[ir], outside the entry pool.
__device__ __forceinline__ uint32_t entry_word(int off, uint32_t n) {
  return ((uint32_t)off & 0xFFFFu) | (n << 16);
}

// HYB spill of slice sl (the whole warp calls it): sp = this lane's in-domain
// successors beyond row_cap.  When any lane has some, allocates the slice's
// spill block (kSpillHdr header words + the entries) from the model's spill
// area, writes the header and spill_off[sl], and returns the word index of this
// lane's first spill entry; returns -1 when nothing is to be stored (no spill,
// or no room: the need is counted in CNT_SPILL_WORDS either way, and a slice
// without room in CNT_SPILL_FULL, so that the build can be rerun with an area
// of exactly the size needed).
__device__ __forceinline__ int64_t spill_alloc(const BuildArgs &a, int64_t sl, int sp) {
  const int lane = threadIdx.x & 31;
  int incl = sp;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int x = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += x;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) {
    if (lane == 0 && a.spill_off) a.spill_off[sl] = kNoSlice;
    return -1;
  }
  const unsigned rows = __popc(__ballot_sync(0xffffffffu, sp > 0));
  unsigned long long base = 0;
  if (lane == 0) {
    base = atomicAdd(&a.cnt[CNT_SPILL_WORDS], (unsigned long long)(total + kSpillHdr));
    atomicAdd(&a.cnt[CNT_SPILL_ROWS], (unsigned long long)rows);
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  const bool fits = a.spill && base + (unsigned long long)(total + kSpillHdr) <= a.spill_cap_words;
  if (lane == 0) {
    if (!fits) atomicAdd(&a.cnt[CNT_SPILL_FULL], 1ULL);
    if (a.spill_off) a.spill_off[sl] = fits ? (uint32_t)base : kNoSlice;
  }
  if (!fits) return -1;
  uint32_t *blk = a.spill + base;
  blk[lane] = (uint32_t)(incl - sp);
  if (lane == 31) blk[32] = (uint32_t)total;
  return (int64_t)base + kSpillHdr + (incl - sp);
}

// Executed by one full warp for one slice.  Lane l owns internal row
// ir = sl*32 + l.  Scans its histogram column hist[b*32 + l] over the bins of
// [lo_x, hi_x] x [lo_y, hi_y] (sub-grid offsets) in ascending bin order,
// zeroes what it reads, classifies each landing cell (outside the domain or an
// obstacle at t+1 -> sink), stages the k-th entry word in its own column at
// hist[k*32 + l] (bin k <= the bin just read, so already read and zeroed: the
// histogram is the stage, and the kernels need no shared memory for it),
// accumulates R = sum_b (count_b/N) r_b + (count_sink/N) r_outbound in that
// order, then allocates the slice's columns from the pool, writes them and
// zeroes the staged words again.
// Every entry is staged (entry k in histogram row k); those beyond row_cap
// then go to the slice's spill block (HYB).
template <typename RT>
__device__ void emit_slice(const BuildArgs &a, uint32_t *hist, int64_t sl,
                           int kind, bool row_ok, int lo_x, int hi_x, int lo_y, int hi_y) {
  const int lane = threadIdx.x & 31;
  const int q = lane / a.A_pad, act = lane % a.A_pad;
  const int64_t s = sl * a.spw + q;
  const int64_t ir = sl * 32 + lane;
  int e = 0;              // in-domain entries
  uint32_t sink = 0;      // realizations ending in the sink
  RT Racc[3] = {RT(0), RT(0), RT(0)};

  lo_x = max(lo_x, -a.h);
  lo_y = max(lo_y, -a.h);
  hi_x = min(hi_x, a.h);
  hi_y = min(hi_y, a.h);
  if (kind == KIND_SINK) {
    sink = (uint32_t)a.N;
    for (int o = 0; o < a.rw.n_obj; ++o) {
      if constexpr (sizeof(RT) == 8)
        Racc[o] = __dmul_rn(__ddiv_rn((double)a.N, (double)a.N), a.rw.r_out);
      else
        Racc[o] = (RT)a.rw.r_out;
    }
  } else if (kind == KIND_SAMPLE) {
    const int64_t t = s / a.Nc, c = s % a.Nc;
    const int i = (int)(c % a.nx), j = (int)(c / a.nx);
    const int64_t nxt = (t + 1) * a.Nc;
    RT F, g_s = RT(0);
    if constexpr (sizeof(RT) == 8) F = a.act.F64[act]; else F = a.act.F[act];
    if (a.gbar) g_s = load_field<RT>(a.gbar, s);
    const RT invN = RT(1) / RT(a.N);
    for (int dj = lo_y; dj <= hi_y; ++dj) {
      const int jp = j + dj;
      const int brow = (dj + a.h) * a.L + a.h;
      for (int di = lo_x; di <= hi_x; ++di) {
        const int b = brow + di;
        uint32_t *hp = hist + (size_t)b * 32 + lane;
        const uint32_t n = *hp;
        if (n == 0) continue;
        *hp = 0;
        const int ip = i + di;
        const bool inside = ip >= 0 && ip < a.nx && jp >= 0 && jp < a.ny;
        const uint8_t ccls = inside ? a.cls[nxt + (int64_t)jp * a.nx + ip] : CLS_OBSTACLE;
        if (!row_ok) continue;
        if (ccls & CLS_OBSTACLE) {   // obstacle at t+1 or outside: sink
          sink += n;
          continue;
        }
        hist[e * 32 + lane] = entry_word(dj * a.nx + di, n);
        ++e;
        const bool is_t = (ccls & CLS_TARGET) != 0;
        RT g_sp = RT(0);
        if (a.gbar) g_sp = load_field<RT>(a.gbar, nxt + (int64_t)jp * a.nx + ip);
        for (int o = 0; o < a.rw.n_obj; ++o) {
          if constexpr (sizeof(RT) == 8) {
            const double p = __ddiv_rn((double)n, (double)a.N);
            Racc[o] = __dadd_rn(Racc[o], __dmul_rn(p, step_reward64(a.rw, a.rw.objs[o], F, g_s, g_sp, is_t)));
          } else {
            const float p = (float)n * invN;
            Racc[o] = fmaf(p, step_reward32(a.rw, a.rw.objs[o], F, g_s, g_sp, is_t), Racc[o]);
          }
        }
      }
    }
    if (row_ok && sink > 0) {
      for (int o = 0; o < a.rw.n_obj; ++o) {
        if constexpr (sizeof(RT) == 8) {
          const double p = __ddiv_rn((double)sink, (double)a.N);
          Racc[o] = __dadd_rn(Racc[o], __dmul_rn(p, a.rw.r_out));
        } else {
          Racc[o] = fmaf((float)sink * invN, (float)a.rw.r_out, Racc[o]);
        }
      }
    }
    if (!row_ok) {
      e = 0;
      sink = 0;
    }
  }
  int ell = min(e, a.row_cap);   // entries in the ELL columns
  const int staged = e;          // histogram words holding the row's entries
  // the rest of the row goes to the slice's spill block (HYB)
  const int64_t sp_at = spill_alloc(a, sl, e - ell);
  if (sp_at >= 0)
    for (int k = ell; k < e; ++k) a.spill[sp_at + (k - ell)] = hist[k * 32 + lane];

  // slice width = widest row; allocate columns from the pool (bump allocator)
  int W = ell;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) W = max(W, __shfl_xor_sync(0xffffffffu, W, off));
  unsigned long long base = 0;
  if (lane == 0 && W > 0) base = atomicAdd(&a.cnt[CNT_POOL_COLS], (unsigned long long)W);
  base = __shfl_sync(0xffffffffu, base, 0);
  bool fits = (W == 0) || (base + (unsigned long long)W <= a.pool_cap_cols);
  if (!fits) {
    if (lane == 0) atomicAdd(&a.cnt[CNT_POOL_FULL], 1ULL);
    e = 0;
    ell = 0;
  }
  if (fits && W > 0) {
    uint32_t *dst = a.pool + base * 32 + lane;
    for (int k = 0; k < W; ++k) dst[(size_t)k * 32] = (k < ell) ? hist[k * 32 + lane] : 0u;
  }
  for (int k = 0; k < staged; ++k) hist[k * 32 + lane] = 0u;   // the histogram is zero again
  if (e > ell) atomicMax(&a.cnt[CNT_MAXLEN], (unsigned long long)e);
  if (lane == 0) {
    a.slice_off[sl] = (fits && W > 0) ? (uint32_t)base : kNoSlice;
    a.slice_w[sl] = (fits && W > 0) ? (uint8_t)W : (uint8_t)0;
  }
  a.nnz[ir] = (uint8_t)ell;
  a.sinkc[ir] = (uint16_t)sink;
  int tot = e + (sink > 0 ? 1 : 0), dom = e;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, off);
    dom += __shfl_xor_sync(0xffffffffu, dom, off);
  }
  if (lane == 0 && tot > 0) {
    atomicAdd(&a.cnt[CNT_NNZ], (unsigned long long)tot);
    atomicAdd(&a.cnt[CNT_DOMAIN], (unsigned long long)dom);
    atomicMax(&a.cnt[CNT_MAXROW], (unsigned long long)W);
  }
  for (int o = 0; o < a.rw.n_obj; ++o) static_cast<RT *>(a.R)[(int64_t)o * a.rows_pad + ir] = Racc[o];
}

}  // namespace mdpgb
