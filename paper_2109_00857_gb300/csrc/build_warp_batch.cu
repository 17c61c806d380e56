// build_warp_batch.cu -- the warp-per-slice FP32 build over many models in
// one persistent launch (mdp_batch_*); the slice algorithm is in
// build_warp.cuh.
#include "build_warp.cuh"

namespace mdpgb {

// Many models: persistent warps pull global slice indices; g -> (model m,
// slice g - prefix[m]) by binary search over the prefix sums.  The models of
// one launch share the mode count (KT > 0; KT == 0: runtime, up to
// kMaxModes) and the states per warp (SPW; 0: runtime).
template <int KT, int SPW>
__global__ void __launch_bounds__(256, 3) build_warp_batch_kernel(const BuildArgs *__restrict__ items,
                                                                 const int64_t *__restrict__ prefix, int n,
                                                                 unsigned long long *work, int cap) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *tab = reinterpret_cast<float *>(smem + (size_t)warp * warp_words(cap));
  uint32_t *grid = smem + (size_t)warp * warp_words(cap) + kTab;
  const int64_t total = prefix[n];
  WarpAcc acc;
  int cur = -1;
  unsigned long long next = 0;
  if (lane == 0) next = atomicAdd(work, 1ULL);
  for (;;) {
    const int64_t g = (int64_t)__shfl_sync(0xffffffffu, next, 0);
    if (g >= total) break;
    if (lane == 0) next = atomicAdd(work, 1ULL);
    int lo = 0, hi = n - 1;   // last m with prefix[m] <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
    }
    if (lo != cur) {
      if (cur >= 0) warp_flush(items[cur], acc);
      cur = lo;
      __syncwarp();
      load_rank_tables(items[lo], tab);
    }
    warp_slice<KT, SPW, false>(items[lo], g - prefix[lo], grid, tab, acc);
    __syncwarp();
  }
  if (cur >= 0) warp_flush(items[cur], acc);
}

template <int KT, int SPW>
static cudaError_t launch_wb(const BuildArgs *items_d, const int64_t *prefix_d, int n, unsigned long long *work_d,
                             int cap, cudaStream_t st) {
  const int warps = 8;
  const size_t smem = (size_t)warp_words(cap) * 4 * warps;
  cudaError_t e = allow_max_smem((const void *)build_warp_batch_kernel<KT, SPW>);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_warp_batch_kernel<KT, SPW>, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  build_warp_batch_kernel<KT, SPW><<<num_sms() * per_sm, warps * 32, smem, st>>>(items_d, prefix_d, n, work_d, cap);
  return cudaGetLastError();
}

template <int SPW>
static cudaError_t launch_wb_k(const BuildArgs *items_d, const int64_t *prefix_d, int n,
                               unsigned long long *work_d, int cap_bins, int K, cudaStream_t st) {
  switch (K) {
    case 1: return launch_wb<1, SPW>(items_d, prefix_d, n, work_d, cap_bins, st);
    case 2: return launch_wb<2, SPW>(items_d, prefix_d, n, work_d, cap_bins, st);
    case 3: return launch_wb<3, SPW>(items_d, prefix_d, n, work_d, cap_bins, st);
    case 4: return launch_wb<4, SPW>(items_d, prefix_d, n, work_d, cap_bins, st);
    case 5: return launch_wb<5, SPW>(items_d, prefix_d, n, work_d, cap_bins, st);
    case 6: return launch_wb<6, SPW>(items_d, prefix_d, n, work_d, cap_bins, st);
    case 8: return launch_wb<8, SPW>(items_d, prefix_d, n, work_d, cap_bins, st);
    default: return launch_wb<0, SPW>(items_d, prefix_d, n, work_d, cap_bins, st);
  }
}

cudaError_t launch_build_warp_batch(const BuildArgs *items_d, const int64_t *prefix_d, int n,
                                    unsigned long long *work_d, int cap_bins, int K, int spw,
                                    cudaStream_t st) {
  if (spw == 1) return launch_wb_k<1>(items_d, prefix_d, n, work_d, cap_bins, K, st);
  if (spw == 2) return launch_wb_k<2>(items_d, prefix_d, n, work_d, cap_bins, K, st);
  return launch_wb_k<0>(items_d, prefix_d, n, work_d, cap_bins, K, st);
}

}  // namespace mdpgb
