// build_fp32.cu -- production FP32 MDP build (steps a2-a6), one fused kernel.
//
// Persistent CTAs pull slices (32 internal rows = spw states x A_pad actions)
// from a device work queue.  Per slice and per chunk of realizations:
//   phase A  threads form the DO velocity of their (state, realization),
//            w = vbar + sum_k Y_k v~_k (Sec. II-C), once for all actions, and
//            stage u = 1/2 + w dt/dx (position relative to the cell's lower
//            edge after the flow, in cells) in shared memory; the per-state
//            extremes of u bound every landing offset of every action.
//   phase B  lane l of every warp owns row (state q, action a) = (l / A_pad,
//            l % A_pad).  For each staged realization it forms the landing
//            offset floor(u + d_a dt/dx) in x and y (Sec. II-A move, cell();
//            land_offset, the floor of the exact sum of the two floats) and
//            counts the sub-grid bin with a shared-memory reduction into
//            hist[bin][l]: a lane only ever touches its own bank, so the
//            counting has no bank or address conflicts within a warp.
//   emit     warp 0 turns each lane's column into sparse (bin, count) entries,
//            folds out-of-domain / obstacle landings into the sink and forms
//            R(s,a) from the counts (build_common.cuh).
// Landing offsets are checked against the sub-grid from the per-state extremes
// before any count is made (the offset is monotone in u, so the extremes of u
// give the exact extremes of every action's offsets); a state
// whose offsets leave the sub-grid is reported as overflow and counts nothing.
#include "build_common.cuh"

namespace mdpgb {

__device__ __forceinline__ void red_add_shared(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

__device__ __forceinline__ float warp_min(float v, int from) {
  for (int off = 16; off >= from; off >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}
__device__ __forceinline__ float warp_max(float v, int from) {
  for (int off = 16; off >= from; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

template <int KT>
__device__ __forceinline__ void load_y(const float *__restrict__ yw, float (&y)[KT > 0 ? KT : 1]) {
  if constexpr (KT > 0 && (KT % 4) == 0) {
#pragma unroll
    for (int k = 0; k < KT; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(yw + k));
      y[k] = v.x; y[k + 1] = v.y; y[k + 2] = v.z; y[k + 3] = v.w;
    }
  } else if constexpr (KT > 0) {
#pragma unroll
    for (int k = 0; k < KT; ++k) y[k] = __ldg(yw + k);
  }
}

// KT > 0: the number of modes is a compile-time constant; KT == 0: runtime K.
// The whole CTA algorithm for one model: all threads of the CTA call it.
// s_slice is a __shared__ word of the calling kernel.
template <int KT>
__device__ __forceinline__ void cta_run(const BuildArgs &a, uint32_t *smem, long long &s_slice) {
  uint32_t *hist = smem;                                             // [nbins][32]
  float2 *ubuf = reinterpret_cast<float2 *>(hist + (size_t)a.nbins * 32);    // [chunk][spw]
  float *red = reinterpret_cast<float *>(ubuf + (size_t)a.chunk * a.spw);    // [nwarps][spw][4]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const int K = KT > 0 ? KT : a.K;
  for (int i = tid; i < a.nbins * 32; i += blockDim.x) hist[i] = 0;

  // lane role (phase B / emit): row (q_l, a_l) of the slice
  const int q_l = lane / a.A_pad, a_l = lane % a.A_pad;
  const bool act_ok = a_l < a.A;
  const int cxl = act_ok ? a.act.cx[a_l] : 0, cyl = act_ok ? a.act.cy[a_l] : 0;
  const float thxl = act_ok ? a.act.thx[a_l] : 2.f, thyl = act_ok ? a.act.thy[a_l] : 2.f;
  // hist byte address of (bin(dx, dy), lane): ((dy + h) * L + (dx + h)) * 128 + lane * 4
  const uint32_t rowstride = (uint32_t)a.L * 128u;
  const uint32_t hbase = smem_u32(hist) + (uint32_t)lane * 4u +
                         ((uint32_t)a.h * (uint32_t)a.L + (uint32_t)a.h) * 128u;
  // thread role (phase A): state q_t of the slice, realizations w0, w0 + wstride, ...
  const int q_t = tid % a.spw;
  const int w0 = tid / a.spw, wstride = blockDim.x / a.spw;
  const float lam = a.lam;
  const float *Yall = static_cast<const float *>(a.Y);
  const float *vbar = static_cast<const float *>(a.vbar);
  const float *modes = static_cast<const float *>(a.modes);
  __syncthreads();

  for (;;) {
    if (tid == 0) {
      if (a.defer_in) {
        const unsigned long long i = atomicAdd(&a.cnt[CNT_DEFER_WORK], 1ULL);
        s_slice = (i < *(volatile unsigned long long *)&a.cnt[CNT_DEFER_N]) ? (long long)a.defer_in[i]
                                                                              : (long long)a.slice_end;
      } else {
        s_slice = a.slice_begin + (long long)atomicAdd(&a.cnt[CNT_WORK], 1ULL);
      }
    }
    __syncthreads();
    const int64_t sl = s_slice;
    if (sl >= a.slice_end) break;

    const int64_t s_l = sl * a.spw + q_l;
    int kind_l = state_kind(a, s_l);
    if (!act_ok) kind_l = KIND_NONE;
    const int64_t s_t = sl * a.spw + q_t;
    const int kind_t = state_kind(a, s_t);
    const int any_sample = __syncthreads_or(kind_t == KIND_SAMPLE);

    float run_mnx = INFINITY, run_mxx = -INFINITY, run_mny = INFINITY, run_mxy = -INFINITY;
    bool active = (kind_l == KIND_SAMPLE);
    if (any_sample) {
      // per-thread DO mean and modes at (t, cell) of state q_t
      float phx[KT > 0 ? KT : kMaxModes], phy[KT > 0 ? KT : kMaxModes];
      float vbx = 0.f, vby = 0.f;
      const float *Yt = Yall;
      if (kind_t == KIND_SAMPLE) {
        const int64_t t = s_t / a.Nc, c = s_t % a.Nc;
        vbx = vbar[2 * s_t];
        vby = vbar[2 * s_t + 1];
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : kMaxModes); ++k) {
          if (KT == 0 && k >= K) break;
          const float2 ph = *reinterpret_cast<const float2 *>(modes + 2 * ((t * K + k) * a.Nc + c));
          phx[k] = ph.x;
          phy[k] = ph.y;
        }
        Yt = Yall + (size_t)t * a.N * K;
      }
      for (int c0 = 0; c0 < a.N; c0 += a.chunk) {
        const int cn = min(a.chunk, a.N - c0);
        // ---- phase A: velocities of this chunk
        float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
        if (kind_t == KIND_SAMPLE) {
          for (int w = w0; w < cn; w += wstride) {
            const float *yw = Yt + (size_t)(c0 + w) * K;
            float wx = vbx, wy = vby;
            if constexpr (KT > 0) {
              float y[KT];
              load_y<KT>(yw, y);
#pragma unroll
              for (int k = 0; k < KT; ++k) {
                wx = fmaf(y[k], phx[k], wx);
                wy = fmaf(y[k], phy[k], wy);
              }
            } else {
              for (int k = 0; k < K; ++k) {
                const float yk = __ldg(yw + k);
                wx = fmaf(yk, phx[k], wx);
                wy = fmaf(yk, phy[k], wy);
              }
            }
            float ux = fmaf(wx, lam, 0.5f), uy = fmaf(wy, lam, 0.5f);
            // a non-finite velocity must not reach the bin arithmetic: push it far
            // outside every sub-grid so the extreme check reports overflow
            if (!(fabsf(ux) < 1e30f)) ux = 1e30f;
            if (!(fabsf(uy) < 1e30f)) uy = 1e30f;
            ubuf[(size_t)w * a.spw + q_t] = make_float2(ux, uy);
            mnx = fminf(mnx, ux); mxx = fmaxf(mxx, ux);
            mny = fminf(mny, uy); mxy = fmaxf(mxy, uy);
          }
        }
        // extremes per state q over this chunk: lanes with equal q share lane % spw
        mnx = warp_min(mnx, a.spw); mxx = warp_max(mxx, a.spw);
        mny = warp_min(mny, a.spw); mxy = warp_max(mxy, a.spw);
        if (lane < a.spw) {
          float *r = red + ((size_t)warp * a.spw + lane) * 4;
          r[0] = mnx; r[1] = mxx; r[2] = mny; r[3] = mxy;
        }
        __syncthreads();
        float cmnx = INFINITY, cmxx = -INFINITY, cmny = INFINITY, cmxy = -INFINITY;
        for (int wv = 0; wv < nwarps; ++wv) {
          const float *r = red + ((size_t)wv * a.spw + q_l) * 4;
          cmnx = fminf(cmnx, r[0]); cmxx = fmaxf(cmxx, r[1]);
          cmny = fminf(cmny, r[2]); cmxy = fmaxf(cmxy, r[3]);
        }
        run_mnx = fminf(run_mnx, cmnx); run_mxx = fmaxf(run_mxx, cmxx);
        run_mny = fminf(run_mny, cmny); run_mxy = fmaxf(run_mxy, cmxy);
        if (active) {
          // far (or clamped non-finite) extremes leave the sub-grid; the
          // integer landing offsets below are only formed for moderate ones
          if (!(cmnx > -1e6f && cmxx < 1e6f && cmny > -1e6f && cmxy < 1e6f)) {
            active = false;
          } else {
            const int lox = land_offset(cmnx, cxl, thxl), hix = land_offset(cmxx, cxl, thxl);
            const int loy = land_offset(cmny, cyl, thyl), hiy = land_offset(cmxy, cyl, thyl);
            if (lox < -a.h || hix > a.h || loy < -a.h || hiy > a.h) active = false;
          }
        }
        // ---- phase B: count landings of this chunk
        if (active) {
          const float2 *ub = ubuf + q_l;
#pragma unroll 4
          for (int w = warp; w < cn; w += nwarps) {
            const float2 u = ub[(size_t)w * a.spw];
            const int bx = land_offset(u.x, cxl, thxl), by = land_offset(u.y, cyl, thyl);
            red_add_shared((uint32_t)by * rowstride + (uint32_t)bx * 128u + hbase, 1u);
          }
        }
        __syncthreads();
      }
    }
    // ---- emit (warp 0)
    if (warp == 0) {
      int lox = 0, hix = -1, loy = 0, hiy = -1;
      if (kind_l == KIND_SAMPLE && run_mnx <= run_mxx) {
        lox = land_offset(run_mnx, cxl, thxl); hix = land_offset(run_mxx, cxl, thxl);
        loy = land_offset(run_mny, cyl, thyl); hiy = land_offset(run_mxy, cyl, thyl);
      }
      const bool row_ok = active || kind_l != KIND_SAMPLE;
      if (kind_l == KIND_SAMPLE) {
        if (!row_ok) atomicAdd(&a.cnt[CNT_OVERFLOW], 1ULL);
        else atomicAdd(&a.cnt[CNT_SAMPLES], (unsigned long long)a.N);
      }
      emit_slice<float>(a, hist, sl, kind_l, row_ok, lox, hix, loy, hiy);
    }
    __syncthreads();
  }
}

template <int KT>
__global__ void __launch_bounds__(512) build_fp32_kernel(BuildArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ long long s_slice;
  cta_run<KT>(a, smem, s_slice);
}


// Many models: every CTA walks the models in order and helps finish each
// model's deferred list (items carry defer_in = their own list).
__global__ void __launch_bounds__(512) build_fp32_batch_kernel(const BuildArgs *__restrict__ items, int n) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ long long s_slice;
  for (int m = 0; m < n; ++m) {
    const BuildArgs &a = items[m];
    if (*(volatile unsigned long long *)&a.cnt[CNT_DEFER_N] == 0) continue;   // same value in every thread
    cta_run<0>(a, smem, s_slice);
    __syncthreads();
  }
}

cudaError_t launch_build_fp32_batch(const BuildArgs *items_d, int n, size_t smem, int threads,
                                    cudaStream_t st) {
  cudaError_t e = allow_max_smem((const void *)build_fp32_batch_kernel);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_fp32_batch_kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  build_fp32_batch_kernel<<<num_sms() * per_sm, threads, smem, st>>>(items_d, n);
  return cudaGetLastError();
}

size_t fp32_smem_bytes(const BuildArgs &a, int threads) {
  return (size_t)a.nbins * 32 * 4 + (size_t)a.chunk * a.spw * 8 +
         (size_t)(threads / 32) * a.spw * 16;
}

template <int KT>
static cudaError_t launch_kt(const BuildArgs &a, int threads, int sms, cudaStream_t st) {
  const size_t smem = fp32_smem_bytes(a, threads);
  cudaError_t e = allow_max_smem((const void *)build_fp32_kernel<KT>);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_fp32_kernel<KT>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t blocks = (int64_t)sms * per_sm;
  const int64_t work = a.slice_end - a.slice_begin;
  if (!a.defer_in && blocks > work) blocks = work > 0 ? work : 1;
  build_fp32_kernel<KT><<<(unsigned)blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_build_fp32(const BuildArgs &a, int threads, int sms, cudaStream_t st) {
  switch (a.K) {
    case 1: return launch_kt<1>(a, threads, sms, st);
    case 2: return launch_kt<2>(a, threads, sms, st);
    case 3: return launch_kt<3>(a, threads, sms, st);
    case 4: return launch_kt<4>(a, threads, sms, st);
    case 5: return launch_kt<5>(a, threads, sms, st);
    case 6: return launch_kt<6>(a, threads, sms, st);
    case 8: return launch_kt<8>(a, threads, sms, st);
    default: return launch_kt<0>(a, threads, sms, st);
  }
}

}  // namespace mdpgb
