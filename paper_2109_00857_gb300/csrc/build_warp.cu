// build_warp.cu -- production FP32 MDP build, warp-per-slice fast path
// (single-model kernel and launchers; the slice algorithm is in build_warp.cuh,
// the batched kernel in build_warp_batch.cu).
#include <algorithm>

#include "build_warp.cuh"

namespace mdpgb {

// Single model: warps pull slices from the model's work queue -- persistent
// warps, or at most a.slices_per_warp slices each (the grid then covers the
// model: capacity blocks x warps x q >= slices, so every slice is taken).
template <int KT, int SPW>
__global__ void __launch_bounds__(256, 3) build_warp_kernel(BuildArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *tab = reinterpret_cast<float *>(smem + (size_t)warp * warp_words(a.cap_bins));
  uint32_t *grid = smem + (size_t)warp * warp_words(a.cap_bins) + kTab;
  load_rank_tables(a, tab);
  WarpAcc acc;
  unsigned long long next = 0;
  if (lane == 0) next = atomicAdd(&a.cnt[CNT_WORK], 1ULL);
  for (int n = 1;; ++n) {
    const int64_t sl = a.slice_begin + (int64_t)__shfl_sync(0xffffffffu, next, 0);
    if (sl >= a.slice_end) break;
    // prefetch the next slice, unless this warp's share ends with this one
    const bool more = a.slices_per_warp == 0 || n < a.slices_per_warp;
    if (lane == 0) next = more ? atomicAdd(&a.cnt[CNT_WORK], 1ULL) : (unsigned long long)(a.slice_end - a.slice_begin);
    warp_slice<KT, SPW, true>(a, sl, grid, tab, acc);
    __syncwarp();
  }
  warp_flush(a, acc);
}

template <int KT, int SPW>
static cudaError_t launch_w(const BuildArgs &a, int warps, int sms, cudaStream_t st) {
  const size_t per_warp = (size_t)warp_words(a.cap_bins) * 4;
  const size_t smem = per_warp * warps;
  cudaError_t e = allow_max_smem((const void *)build_warp_kernel<KT, SPW>);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_warp_kernel<KT, SPW>, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t blocks = (int64_t)sms * per_sm;
  const int64_t need = (a.slice_end - a.slice_begin + warps - 1) / warps;
  if (blocks > need) blocks = need > 0 ? need : 1;
  if (a.slices_per_warp > 0) {   // bounded warps: a grid that covers every slice
    const int64_t per_cta = (int64_t)warps * a.slices_per_warp;
    blocks = std::max<int64_t>(1, (a.slice_end - a.slice_begin + per_cta - 1) / per_cta);
  }
  build_warp_kernel<KT, SPW><<<(unsigned)blocks, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int SPW>
static cudaError_t launch_spw(const BuildArgs &a, int warps, int sms, cudaStream_t st) {
  switch (a.K) {
    case 1: return launch_w<1, SPW>(a, warps, sms, st);
    case 2: return launch_w<2, SPW>(a, warps, sms, st);
    case 3: return launch_w<3, SPW>(a, warps, sms, st);
    case 4: return launch_w<4, SPW>(a, warps, sms, st);
    case 5: return launch_w<5, SPW>(a, warps, sms, st);
    case 6: return launch_w<6, SPW>(a, warps, sms, st);
    case 8: return launch_w<8, SPW>(a, warps, sms, st);
    default: return launch_w<0, SPW>(a, warps, sms, st);
  }
}

cudaError_t launch_build_warp(const BuildArgs &a, int warps, int sms, cudaStream_t st) {
  if (a.spw == 1) return launch_spw<1>(a, warps, sms, st);
  if (a.spw == 2) return launch_spw<2>(a, warps, sms, st);
  return launch_spw<0>(a, warps, sms, st);
}

}  // namespace mdpgb
