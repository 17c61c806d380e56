// check_fp64.cu -- the DO-coefficient sampler (step a1) and the FP64 check-mode
// build kernel.  Compiled with -fmad=false; every floating operation on the
// path is additionally written as an explicit round-to-nearest intrinsic so no
// contraction can change a rounding.  The check build evaluates the paper's
// kinematics literally, x' = x + (v + a) dt, cell = floor(x'/dx) (Sec. II-A),
// with v = vbar + sum_k Y_k v~_k summed in ascending k (Sec. II-C).
#include "build_common.cuh"

namespace mdpgb {

// ------------------------------------------------------- Philox4x64-10 ----
// Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds
// of two 64x64->128 multiplies with the published multipliers, key bumped by
// the published Weyl constants between rounds.
struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  U64x4 o;
  o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// ln s for a normal double s > 0: s = m 2^e with m in [sqrt(1/2), sqrt(2)),
// ln s = e ln2 + 2 atanh(z), z = (m-1)/(m+1), atanh(z) = sum z^(2n+1)/(2n+1)
// (Abramowitz & Stegun 4.1.27), twelve terms, Horner in z^2.  Only + - * /
// in round-to-nearest, so host and device agree bit for bit.
__device__ __forceinline__ double ln_series(double s) {
  const uint64_t bits = (uint64_t)__double_as_longlong(s);
  int e = (int)((bits >> 52) & 0x7FF) - 1022;
  double m = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFULL) | 0x3FE0000000000000ULL));
  const double kSqrtHalf = 0x1.6a09e667f3bcdp-1;   // sqrt(1/2) rounded to binary64
  const double kLn2 = 0x1.62e42fefa39efp-1;        // ln 2 rounded to binary64
  if (m < kSqrtHalf) {
    m = __dmul_rn(m, 2.0);
    e = e - 1;
  }
  const double z = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z2 = __dmul_rn(z, z);
  double poly = 1.0 / 23.0;
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 21.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 19.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 17.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 15.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 13.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 11.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 9.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 7.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 5.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0 / 3.0);
  poly = __dadd_rn(__dmul_rn(poly, z2), 1.0);
  return __dadd_rn(__dmul_rn((double)e, kLn2), __dmul_rn(2.0, __dmul_rn(z, poly)));
}

__device__ __forceinline__ double u01(uint64_t x) { return __dmul_rn((double)(x >> 11), 0x1p-53); }

// One thread per (t, w, pair j): Marsaglia-Bray polar method on Philox counters
// (t, w, j, attempt) under key (seed, mdp_id); Y[t][w][2j] = sigma_2j z1,
// Y[t][w][2j+1] = sigma_2j+1 z2.
__global__ void sample_coeffs_kernel(int nt, int N, int K, const double *__restrict__ sigma,
                                     uint64_t seed, uint64_t mdp_id, double *__restrict__ Y64,
                                     float *__restrict__ Y32, unsigned long long *capped) {
  const int pairs = (K + 1) / 2;
  const int64_t total = (int64_t)nt * N * pairs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % pairs);
    const int64_t tw = idx / pairs;
    const int w = (int)(tw % N), t = (int)(tw / N);
    double z1 = 0.0, z2 = 0.0;
    bool ok = false;
    for (uint64_t att = 0; att < 64 && !ok; ++att) {
      const U64x4 r = philox4x64_10((uint64_t)t, (uint64_t)w, (uint64_t)j, att, seed, mdp_id);
      const double v1 = __dsub_rn(__dmul_rn(2.0, u01(r.v[0])), 1.0);
      const double v2 = __dsub_rn(__dmul_rn(2.0, u01(r.v[1])), 1.0);
      const double s = __dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2));
      if (s < 1.0 && s > 0.0) {
        const double f = __dsqrt_rn(__ddiv_rn(__dmul_rn(-2.0, ln_series(s)), s));
        z1 = __dmul_rn(v1, f);
        z2 = __dmul_rn(v2, f);
        ok = true;
      }
    }
    if (!ok) atomicAdd(capped, 1ULL);
    const int64_t base = ((int64_t)t * N + w) * K;
    const double y1 = __dmul_rn(sigma[2 * j], z1);
    if (Y64) Y64[base + 2 * j] = y1;
    if (Y32) Y32[base + 2 * j] = (float)y1;
    if (2 * j + 1 < K) {
      const double y2 = __dmul_rn(sigma[2 * j + 1], z2);
      if (Y64) Y64[base + 2 * j + 1] = y2;
      if (Y32) Y32[base + 2 * j + 1] = (float)y2;
    }
  }
}

cudaError_t launch_sample_coeffs(int nt, int N, int K, const double *sigma_d, uint64_t seed,
                                 uint64_t mdp_id, double *Y64, float *Y32,
                                 unsigned long long *capped, cudaStream_t st) {
  const int64_t total = (int64_t)nt * N * ((K + 1) / 2);
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  const int64_t maxb = (int64_t)num_sms() * 16;
  if (blocks > maxb) blocks = maxb;
  sample_coeffs_kernel<<<(unsigned)blocks, threads, 0, st>>>(nt, N, K, sigma_d, seed, mdp_id, Y64,
                                                            Y32, capped);
  return cudaGetLastError();
}

// --------------------------------------------------- FP64 check build ----
// One CTA per slice at a time (dynamic work queue).  Every thread takes
// (realization, state-in-slice) items, forms the FP64 velocity, and for each
// action evaluates the literal move; landings inside the sub-grid are counted
// with shared atomics into hist[bin][lane], landings outside it are counted as
// overflow.  Warp 0 then emits the slice over the full sub-grid.
__global__ void build_fp64_kernel(BuildArgs a) {
  extern __shared__ uint32_t smem[];
  uint32_t *hist = smem;                                   // [nbins][32]
  __shared__ long long s_slice;
  const int tid = threadIdx.x;
  for (int i = tid; i < a.nbins * 32; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const double *vbar = static_cast<const double *>(a.vbar);
  const double *modes = static_cast<const double *>(a.modes);
  const double *Y = static_cast<const double *>(a.Y);
  for (;;) {
    if (tid == 0) s_slice = a.slice_begin + (long long)atomicAdd(&a.cnt[CNT_WORK], 1ULL);
    __syncthreads();
    const int64_t sl = s_slice;
    if (sl >= a.slice_end) break;
    unsigned long long ovf = 0, smp = 0;
    for (int64_t it = tid; it < (int64_t)a.N * a.spw; it += blockDim.x) {
      const int q = (int)(it % a.spw);
      const int w = (int)(it / a.spw);
      const int64_t s = sl * a.spw + q;
      if (state_kind(a, s) != KIND_SAMPLE) continue;
      const int64_t t = s / a.Nc, c = s % a.Nc;
      const int64_t i = c % a.nx, j = c / a.nx;
      double vx = vbar[2 * s], vy = vbar[2 * s + 1];
      const double *yw = Y + ((int64_t)t * a.N + w) * a.K;
      for (int k = 0; k < a.K; ++k) {
        const double *phi = modes + 2 * ((t * a.K + k) * a.Nc + c);
        vx = __dadd_rn(vx, __dmul_rn(yw[k], phi[0]));
        vy = __dadd_rn(vy, __dmul_rn(yw[k], phi[1]));
      }
      const double x = __dmul_rn(__dadd_rn((double)i, 0.5), a.rw.dx);
      const double y = __dmul_rn(__dadd_rn((double)j, 0.5), a.rw.dx);
      for (int act = 0; act < a.A; ++act) {
        const double xp = __dadd_rn(x, __dmul_rn(__dadd_rn(vx, a.act.dx64[act]), a.rw.dt));
        const double yp = __dadd_rn(y, __dmul_rn(__dadd_rn(vy, a.act.dy64[act]), a.rw.dt));
        const double fx = floor(__ddiv_rn(xp, a.rw.dx)), fy = floor(__ddiv_rn(yp, a.rw.dx));
        ++smp;
        // non-finite or far landings count as overflow before any integer conversion
        if (!(fabs(fx) < 1e15) || !(fabs(fy) < 1e15)) {
          ++ovf;
          continue;
        }
        const int64_t ip = (int64_t)fx, jp = (int64_t)fy;
        const int64_t di = ip - i, dj = jp - j;
        if (di < -a.h || di > a.h || dj < -a.h || dj > a.h) {
          ++ovf;
          continue;
        }
        const int b = (int)((dj + a.h) * a.L + (di + a.h));
        atomicAdd(&hist[(size_t)b * 32 + q * a.A_pad + act], 1u);
      }
    }
    if (ovf) atomicAdd(&a.cnt[CNT_OVERFLOW], ovf);
    if (smp) atomicAdd(&a.cnt[CNT_SAMPLES], smp);
    __syncthreads();
    if (tid < 32) {
      const int q = tid / a.A_pad, act = tid % a.A_pad;
      int kind = state_kind(a, sl * a.spw + q);
      if (act >= a.A) kind = KIND_NONE;
      emit_slice<double>(a, hist, sl, kind, true, -a.h, a.h, -a.h, a.h);
    }
    __syncthreads();
  }
}

cudaError_t launch_build_fp64(const BuildArgs &a, cudaStream_t st) {
  const size_t smem = (size_t)a.nbins * 32 * 4;
  cudaError_t e = allow_max_smem((const void *)build_fp64_kernel);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_fp64_kernel, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t blocks = (int64_t)num_sms() * per_sm;
  const int64_t work = a.slice_end - a.slice_begin;
  if (blocks > work) blocks = work > 0 ? work : 1;
  build_fp64_kernel<<<(unsigned)blocks, 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mdpgb
