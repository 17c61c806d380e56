// build_warp.cuh -- the warp-per-slice FP32 build (steps a2-a6 fused) as a
// device function, shared by the single-model kernel (build_warp.cu) and the
// batched kernel (batch.cu).
//
// A warp works alone on one slice (spw states x A_pad actions, 32 rows) with
// a private shared-memory histogram and no block-level barrier:
//   pass 1   lanes form the DO velocity w = vbar + sum_k Y_k v~_k (Sec. II-C)
//            of (state, realization) items, u = 1/2 + w dt/dx, and reduce the
//            exact per-state extremes of u over all N realizations.  Floor and
//            rounded addition are monotone, so floor(ext(u) + d_a dt/dx) is the
//            exact range of every action's landing offsets: it checks the
//            neighbouring sub-grid (overflow is an error) and sizes each lane's
//            histogram to its own bounding box.
//   pass 2   per chunk of 64 items the lanes stage u in shared memory
//            (velocity once for all actions), then lane l = (state q, action a)
//            forms floor(u + d_a dt/dx) in x and y (Sec. II-A move, cell()) and
//            counts the bin with a shared-memory reduction into hist[bin][l]:
//            a lane only touches its own bank, so no conflicts.  The counting
//            loop over a full chunk is unrolled with constant shared offsets.
//   emit     two scans of each lane's bounding box: count the entries (sink
//            folded), allocate the slice's columns, then write the entry words
//            in ascending order with R(s,a) from the counts, zeroing the bins.
// Slices whose bounding box does not fit cap_bins are appended to a list that
// the CTA kernel of build_fp32.cu finishes with a full-window histogram; both
// kernels evaluate u, the floors and R with the same FP32 operations, so a
// slice's output does not depend on which kernel built it.
#pragma once
#include "build_common.cuh"

namespace mdpgb {

constexpr float kMagic = 12582912.0f;         // 1.5 * 2^23: floor via round-down add
constexpr uint32_t kMagicBits = 0x4B400000u;  // bit pattern of kMagic
constexpr int kItems = 64;                    // (state, realization) items per chunk per warp

__device__ __forceinline__ void red_add_shared(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Same FP32 operations as the CTA kernel: u = fma(w, lam, 1/2), w by an FMA
// chain over ascending k; non-finite values are pushed outside every sub-grid.
// Mode-count variants: KT > 0 exactly KT modes; KT < 0 at most -KT modes
// (runtime K, coefficients in registers); KT == 0 up to kMaxModes (runtime).
template <int KT>
constexpr int kPhi = KT > 0 ? KT : (KT < 0 ? -KT : kMaxModes);

template <int KT>
__device__ __forceinline__ float2 velocity_u(const float *__restrict__ yw, const float (&phx)[kPhi<KT>],
                                             const float (&phy)[kPhi<KT>], float vbx,
                                             float vby, int K, float lam) {
  float wx = vbx, wy = vby;
  if constexpr (KT < 0) {
#pragma unroll
    for (int k = 0; k < -KT; ++k) {
      if (k < K) {
        const float yk = __ldg(yw + k);
        wx = fmaf(yk, phx[k], wx);
        wy = fmaf(yk, phy[k], wy);
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
  if (!(fabsf(ux) < 1e30f)) ux = 1e30f;
  if (!(fabsf(uy) < 1e30f)) uy = 1e30f;
  return make_float2(ux, uy);
}

// Counts one landing: (x, y) = u + d_a rounded to nearest, then floor of both
// by a round-down add of the magic constant, in packed f32x2 adds (two
// lanes' worth of FP32 work per instruction, same IEEE results as scalar
// adds); the floors' bit patterns index the lane's histogram column.
// u, d: (x, y) pairs as 64-bit registers (x in the low word).
constexpr unsigned long long kMagic2 = ((unsigned long long)kMagicBits << 32) | kMagicBits;
__device__ __forceinline__ void count_sample(unsigned long long u, unsigned long long d, uint32_t rowstride,
                                             uint32_t hb) {
  unsigned long long p, f;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(u), "l"(d));
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(f) : "l"(p), "l"(kMagic2));
  red_add_shared((uint32_t)(f >> 32) * rowstride + (uint32_t)f * 128u + hb, 1u);
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

// One warp builds slice sl of model a: pass 1 (exact extremes), pass 2
// (counting into hist, sized by the bounding boxes), emit.  hist holds
// a.cap_bins * 32 zeroed words and is left zeroed; ubuf holds 64 float2.
// SPW > 0: states per warp fixed at compile time (1: A = 32, 2: A = 16);
// SPW == 0: runtime spw.  KT: see kPhi.
template <int KT, int SPW>
__device__ __forceinline__ void warp_slice(const BuildArgs &a, int64_t sl, uint32_t *hist, float2 *ubuf,
                                           WarpAcc &acc) {
  const int lane = threadIdx.x & 31;
  const int spw = SPW > 0 ? SPW : a.spw;
  const int CHq = kItems / spw;                    // realizations per state per chunk
  const int K = KT > 0 ? KT : a.K;
  const int cap = a.cap_bins;
  // lane role: row (q_l, a_l)
  const int q_l = lane / a.A_pad, a_l = lane % a.A_pad;
  const bool act_ok = a_l < a.A;
  const float dxl = act_ok ? a.act.dxl[a_l] : 0.f;
  const float dyl = act_ok ? a.act.dyl[a_l] : 0.f;
  // item role: state q_t, realizations wi and wi + 32/spw of each chunk
  const int q_t = lane % spw, wi = lane / spw, wstep = 32 / spw;
  const float lam = a.lam;
  const float *Yall = static_cast<const float *>(a.Y);
  const float *vbar = static_cast<const float *>(a.vbar);
  const float *modes = static_cast<const float *>(a.modes);
  const uint32_t hist_base = smem_u32(hist) + (uint32_t)lane * 4u;
  const float invN = 1.0f / (float)a.N;

  const int64_t s_l = sl * spw + q_l;
  int kind_l = state_kind(a, s_l);
  if (!act_ok) kind_l = KIND_NONE;
  const int64_t s_t = sl * spw + q_t;
  const int kind_t = state_kind(a, s_t);
  const bool any_sample = __any_sync(0xffffffffu, kind_t == KIND_SAMPLE);

  bool active = kind_l == KIND_SAMPLE;
  int lox = 0, hix = -1, loy = 0, hiy = -1, pitch = 0;
  if (any_sample) {
    float phx[kPhi<KT>], phy[kPhi<KT>];
    float vbx = 0.f, vby = 0.f;
    const float *Yt = Yall;
    if (kind_t == KIND_SAMPLE) {
      const int64_t t = s_t / a.Nc, c = s_t % a.Nc;
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
        const float2 ph = *reinterpret_cast<const float2 *>(modes + 2 * ((t * K + k) * a.Nc + c));
        phx[k] = ph.x;
        phy[k] = ph.y;
      }
      Yt = Yall + (size_t)t * a.N * K;
    }
    // ---- pass 1: exact extremes of u per state
    float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    if (kind_t == KIND_SAMPLE) {
      for (int w = wi; w < a.N; w += wstep) {
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
    // lane q (q < spw) holds state q's extremes
    mnx = __shfl_sync(0xffffffffu, mnx, q_l);
    mxx = __shfl_sync(0xffffffffu, mxx, q_l);
    mny = __shfl_sync(0xffffffffu, mny, q_l);
    mxy = __shfl_sync(0xffffffffu, mxy, q_l);
    if (active) {
      lox = (int)floorf(mnx + dxl); hix = (int)floorf(mxx + dxl);
      loy = (int)floorf(mny + dyl); hiy = (int)floorf(mxy + dyl);
      if (lox < -a.h || hix > a.h || loy < -a.h || hiy > a.h) {   // sub-grid overflow
        active = false;
        atomicAdd(&a.cnt[CNT_OVERFLOW], 1ULL);
      }
    }
    const int wx = active ? hix - lox + 1 : 0, wy = active ? hiy - loy + 1 : 0;
    int nrows = wy;
    pitch = wx;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      pitch = max(pitch, __shfl_xor_sync(0xffffffffu, pitch, off));
      nrows = max(nrows, __shfl_xor_sync(0xffffffffu, nrows, off));
    }
    if (pitch * nrows > cap) {   // too wide for this warp: the CTA kernel builds it
      if (lane == 0) {
        const unsigned long long i = atomicAdd(&a.cnt[CNT_DEFER_N], 1ULL);
        a.defer[i] = (uint32_t)sl;
      }
      return;
    }
    // ---- pass 2: count
    const uint32_t rowstride = (uint32_t)pitch * 128u;
    const uint32_t hb = hist_base - (kMagicBits + (uint32_t)loy) * rowstride -
                        (kMagicBits + (uint32_t)lox) * 128u;
    const ulonglong2 *ub4 = reinterpret_cast<const ulonglong2 *>(ubuf + q_l * CHq);
    const unsigned long long d2 = ((unsigned long long)__float_as_uint(dyl) << 32) | __float_as_uint(dxl);
    for (int c0 = 0; c0 < a.N; c0 += CHq) {
      if (kind_t == KIND_SAMPLE) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int wl = wi + j * wstep;
          const int w = c0 + wl;
          float2 u = make_float2(0.f, 0.f);
          if (w < a.N) u = velocity_u<KT>(Yt + (size_t)w * K, phx, phy, vbx, vby, K, lam);
          ubuf[q_t * CHq + wl] = u;
        }
      }
      __syncwarp();
      if (active) {
        if (c0 + CHq <= a.N) {
          if constexpr (SPW > 0) {
#pragma unroll
            for (int p = 0; p < kItems / SPW / 2; ++p) {
              const ulonglong2 u2 = ub4[p];
              count_sample(u2.x, d2, rowstride, hb);
              count_sample(u2.y, d2, rowstride, hb);
            }
          } else {
#pragma unroll 4
            for (int p = 0; p < CHq / 2; ++p) {
              const ulonglong2 u2 = ub4[p];
              count_sample(u2.x, d2, rowstride, hb);
              count_sample(u2.y, d2, rowstride, hb);
            }
          }
        } else {
          const unsigned long long *ub = reinterpret_cast<const unsigned long long *>(ubuf + q_l * CHq);
          for (int wl = 0; wl < a.N - c0; ++wl) count_sample(ub[wl], d2, rowstride, hb);
        }
      }
      __syncwarp();
    }
  }

  // ---- emit: count entries, allocate the slice, write
  const int64_t ir = sl * 32 + lane;
  int e = 0;
  uint32_t sink = 0;
  const int64_t t = s_l / a.Nc, c = s_l % a.Nc;
  const int ci = (int)(c % a.nx), cj = (int)(c / a.nx);
  const int64_t nxt = (t + 1) * a.Nc;
  if (kind_l == KIND_SAMPLE && active) {
    for (int dj = loy; dj <= hiy; ++dj) {
      const int jp = cj + dj;
      const uint32_t *row = hist + (size_t)(dj - loy) * pitch * 32 + lane;
      for (int di = lox; di <= hix; ++di) {
        const uint32_t n = row[(di - lox) * 32];
        if (n == 0) continue;
        const int ip = ci + di;
        const bool inside = ip >= 0 && ip < a.nx && jp >= 0 && jp < a.ny;
        const uint8_t cc = inside ? a.cls[nxt + (int64_t)jp * a.nx + ip] : CLS_OBSTACLE;
        if (cc & CLS_OBSTACLE) sink += n;
        else ++e;
      }
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
    const float g_s = a.gbar ? static_cast<const float *>(a.gbar)[s_l] : 0.f;
    for (int dj = loy; dj <= hiy; ++dj) {
      const int jp = cj + dj;
      uint32_t *row = hist + (size_t)(dj - loy) * pitch * 32 + lane;
      for (int di = lox; di <= hix; ++di) {
        uint32_t *hp = row + (di - lox) * 32;
        const uint32_t n = *hp;
        if (n == 0) continue;
        *hp = 0;
        const int ip = ci + di;
        const bool inside = ip >= 0 && ip < a.nx && jp >= 0 && jp < a.ny;
        const uint8_t cc = inside ? a.cls[nxt + (int64_t)jp * a.nx + ip] : CLS_OBSTACLE;
        if (cc & CLS_OBSTACLE) continue;
        if (write) dst[(size_t)k * 32] = entry_word(dj * a.nx + di, n);
        ++k;
        const bool is_t = (cc & CLS_TARGET) != 0;
        const float g_sp = a.gbar ? static_cast<const float *>(a.gbar)[nxt + (int64_t)jp * a.nx + ip] : 0.f;
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
    k = 0;
  }
  if (write)   // zero padding up to the slice width
    for (int kk = k; kk < W; ++kk) dst[(size_t)kk * 32] = 0u;
  if (!fits) sink = 0;
  if (lane == 0) {
    a.slice_off[sl] = (fits && W > 0) ? (uint32_t)base : kNoSlice;
    a.slice_w[sl] = (fits && W > 0) ? (uint8_t)W : (uint8_t)0;
  }
  a.nnz[ir] = (uint8_t)e;
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
    acc.samples += (unsigned long long)sampled * (unsigned long long)a.N;
    if ((unsigned long long)W > acc.maxrow) acc.maxrow = W;
  }
}

}  // namespace mdpgb
