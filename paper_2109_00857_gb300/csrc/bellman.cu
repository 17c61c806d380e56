// bellman.cu -- sparse value iteration (steps a7-a8) and the small helper
// kernels of the build (cell classes, sub-grid offset table, field extremes)
// and of the paper-layout export.
//
// Bellman backup (Sec. II-B): Q(s,a) = R(s,a) + sum_j P_j V(s'_j),
// V_{k+1}(s) = max_a Q(s,a), pi(s) = argmax_a Q(s,a) (lowest index wins ties).
// The slices' entry columns reach shared memory by TMA bulk copies and the
// successors' values V(s') are gathered from the next time layer.  Three
// sweeps with the same results bit for bit: the warp-specialized sweep for
// one state per slice (a producer warp copies rounds of slices into three
// slots, 31 consumer warps each sum one slice, lane l row l, and take the max
// and argmax with one redux.sync key per objective); warp per slice for
// several states per slice (a segmented butterfly over the A_pad lanes of a
// state); and the grouped sweep, kept for the batch's one-state-per-slice
// class (four states per warp step, each lane summing four rows and keeping
// a running max, a 3-step shuffle per state).  Residual max|V_{k+1} - V_k|
// is reduced on the device; a sweep whose predecessor met the tolerance
// exits at once, so a fixed launch sequence needs no host round trip between
// sweeps.
#include <algorithm>
#include <cfloat>

#include "build_common.cuh"

namespace mdpgb {

// ------------------------------------------------------------ prepare ----
__global__ void prepare_kernel(const uint8_t *__restrict__ obstacle, const uint8_t *__restrict__ target,
                               uint8_t *__restrict__ cls, int64_t Nc, int64_t n, int32_t *delta,
                               int L, int nx) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    uint8_t c = 0;
    if (obstacle[i]) c |= CLS_OBSTACLE;
    if (target[i % Nc]) c |= CLS_TARGET;
    cls[i] = c;
  }
  if (blockIdx.x == 0) {
    const int h = (L - 1) / 2;
    for (int b = threadIdx.x; b < L * L; b += blockDim.x) delta[b] = (b / L - h) * nx + (b % L - h);
  }
}

cudaError_t launch_prepare(const uint8_t *obstacle, const uint8_t *target, uint8_t *cls, int nx,
                           int ny, int nt, int32_t *delta, int L, cudaStream_t st) {
  const int64_t Nc = (int64_t)nx * ny, n = Nc * nt;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  prepare_kernel<<<(unsigned)blocks, 256, 0, st>>>(obstacle, target, cls, Nc, n, delta, L, nx);
  return cudaGetLastError();
}

// ------------------------------------------------------ field extremes ----
// out[g*C + c] = max |x| over the elements of group g, component c, for data
// laid out [outer][G][inner][C].  Non-negative floats order like their bits.
template <typename T>
__global__ void absmax_kernel(const T *__restrict__ x, int64_t n, int G, int64_t inner, int C,
                              unsigned int *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const int c = (int)(i % C);
    const int g = (int)((i / ((int64_t)C * inner)) % G);
    const float v = fabsf((float)x[i]);
    atomicMax(&out[g * C + c], __float_as_uint(v));
  }
}

cudaError_t launch_absmax(const void *x, int precision, int64_t n, int G, int64_t inner, int C,
                          unsigned int *out, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  if (blocks < 1) return cudaSuccess;
  if (precision == MDP_FP64_CHECK)
    absmax_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const double *>(x), n, G, inner, C, out);
  else
    absmax_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const float *>(x), n, G, inner, C, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------- backups ----
template <typename RT>
struct Acc;
template <>
struct Acc<float> {
  float v = 0.f;
  __device__ __forceinline__ void add(uint32_t cnt, float V, int) { v = fmaf((float)cnt, V, v); }
  __device__ __forceinline__ float q(float R, float invN) const { return fmaf(v, invN, R); }
};
template <>
struct Acc<double> {
  double v = 0.0;
  // the oracle's order: acc = acc + (count/N) * V(s'), then Q = R + acc
  __device__ __forceinline__ void add(uint32_t cnt, double V, int N) {
    v = __dadd_rn(v, __dmul_rn(__ddiv_rn((double)cnt, (double)N), V));
  }
  __device__ __forceinline__ double q(double R, double) const { return __dadd_rn(R, v); }
};

// ---- mbarrier / bulk-copy helpers (PTX) ----
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2 s of clock cycles so a lost arrival can
// never hang the GPU; the caller reports the timeout through the error word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;   // usual case: the data is there
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > 4000000000LL) return false;
  }
  return true;
}
// The same bounded wait, but each test may suspend the warp (up to ~20 us,
// resumed as soon as the phase completes) instead of spinning, so waiting
// warps leave the issue slots to the others.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_suspend(uint32_t bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait_suspend(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// The same copy marked for early L2 eviction (policy from l2_evict_first):
// the entry stream is read once per sweep and should not push the value
// tables, which every sweep gathers from, out of L2.
__device__ __forceinline__ void bulk_g2s_stream(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar,
                                                uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

constexpr int kWarps = 8;     // warps per CTA
constexpr int kDepth = 2;     // slices each warp keeps in flight

struct PipeRange {
  int64_t sl_lo, sl_hi;   // slices of this launch
  int64_t s_lo, s_hi;     // states whose V this launch writes
  int stage_bytes;        // bytes per stage
  int dtab_smem;          // 1: delta table staged in shared memory
  int grouped;            // 1: bellman_body_g (kGS states per warp step, batched sweeps); 2: bellman_kernel_ws
                          // (stage_bytes = entry bytes per slot)
};

// one stage holds a slice's entry columns (at most wcap of them)
static int stage_bytes_for(int wcap) { return wcap * 128; }

// A CTA streams a contiguous block of slices (so its V(s') gathers stay in a
// small window of layer t+1 that L1 keeps); warp w takes slices w, w+8, ...
// and keeps kDepth of them in flight in private stages: lane 0 copies a
// slice's entry columns with cp.async.bulk (TMA) into a stage whose mbarrier
// counts the bytes, while the warp works on an earlier stage: gathers V(s'),
// forms Q, reduces max/argmax over each state's A_pad lanes and writes V and
// the policy.  The slice's R values (one per row and objective) come with
// plain coalesced loads issued one slice ahead; slice offsets and widths of
// the next 32 slices are read in one coalesced load.
// res != nullptr: Jacobi sweep k (exits at once if sweep k-1 met the
// tolerance) with the residual reduced into res[k-1].
// One CTA, slices [b_lo, b_hi) of one model (all threads call it).
// Values of NO objectives of one state, stored side by side (objective o
// in v[o]; NO = 3 is padded to four) so that one vector load gathers V(s')
// of every objective of a fused solve.
template <typename RT, int NO>
struct alignas(sizeof(RT) * (NO == 3 ? 4 : NO)) VPack {
  static constexpr int W = (NO == 3) ? 4 : NO;
  RT v[W];
};

// Per-objective operands of one Bellman launch.  NO objectives share the
// streamed transition slices (each slice is copied once per sweep), each
// with its own R, policy and residual slots; their values live in one
// packed table (in = V_k, out = V_{k+1}; equal for the in-place layered
// pass).  res[o] == nullptr marks a layered pass (no residual, no early
// exit).
template <typename RT, int NO>
struct VSet {
  const RT *R[NO];
  const VPack<RT, NO> *in;
  VPack<RT, NO> *out;
  int16_t *pol[NO];
  unsigned long long *res[NO];
};

// The tail of row `lane` of slice sl that the build put in the slice's spill
// block (HYB), added to the row's sums in its stored (ascending) order after
// the ELL columns: the same sum as over one plain row.  Called only for
// models with a spill area (a.spill_off != nullptr).
template <typename RT, int NO>
__device__ __forceinline__ void add_spill(const SolveArgs &a, int64_t sl, int lane, const VPack<RT, NO> *Vn,
                                          Acc<RT> (&acc)[NO]) {
  const uint32_t off = __ldg(a.spill_off + sl);
  if (off == kNoSlice) return;
  const uint32_t *blk = a.spill + off;
  const uint32_t b = __ldg(blk + lane), e = __ldg(blk + lane + 1);
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t w = __ldg(blk + kSpillHdr + i);
    const VPack<RT, NO> g = Vn[(int)(int16_t)(w & 0xFFFFu)];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o].add(w >> 16, g.v[o], a.N);
  }
}

template <typename RT, int NO>
__device__ __forceinline__ void bellman_body(const SolveArgs &a, const VSet<RT, NO> &v, int k, int64_t b_lo,
                                             int64_t b_hi, const PipeRange &pr, unsigned char *sm,
                                             double *wmax, int *wst_s) {
  // objectives whose previous sweep met the tolerance are finished
  unsigned live = (1u << NO) - 1u;
  if (k > 1) {
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (v.res[o] && __longlong_as_double((long long)v.res[o][k - 2]) <= a.tol) live &= ~(1u << o);
  }
  if (!live) return;
  if (*(volatile int *)a.err) return;   // an earlier launch of this solve timed out
  if (a.work && k >= 1 && blockIdx.x == 0 && threadIdx.x == 0) a.work[k - 1] = (unsigned long long)(pr.sl_hi - pr.sl_lo);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm);   // [kWarps][kDepth]
  unsigned char *ring = sm + 256;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n_local = b_hi - b_lo;
  if (n_local <= 0) return;

  if (tid < kWarps * kDepth) mbar_init(smem_u32(full + tid), 1);
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  unsigned char *myring = ring + (size_t)warp * kDepth * pr.stage_bytes;

  // 32-bit slice/state indices (the host guarantees |S| + Nc < 2^31)
  const int n_mine = (n_local > warp) ? (int)((n_local - warp + kWarps - 1) / kWarps) : 0;
  const int sl0 = (int)b_lo + warp;                       // my j-th slice: sl0 + j*kWarps
  const uint32_t ring0 = smem_u32(myring), bar0 = smem_u32(full + warp * kDepth);
  uint32_t m_off = 0, m_w = 0;   // lane l: metadata of my slice 32*(j/32) + l
  const uint64_t stream_policy = l2_evict_first();

  // issue(j, st): copy my j-th slice into stage st = j % kDepth (whole warp calls it)
  auto issue = [&](int j, int st) {
    if ((j & 31) == 0) {
      const int jj = j + lane;
      if (jj < n_mine) {
        const int sl = sl0 + jj * kWarps;
        m_off = __ldg(a.slice_off + sl);
        m_w = __ldg(a.slice_w + sl);
      }
    }
    const uint32_t off = __shfl_sync(0xffffffffu, m_off, j & 31);
    const uint32_t W = __shfl_sync(0xffffffffu, m_w, j & 31);
    if (lane == 0) {
      wst_s[warp * kDepth + st] = (int)W;
      const uint32_t sbase = ring0 + (uint32_t)(st * pr.stage_bytes);
      const uint32_t fb = bar0 + 8u * (uint32_t)st;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the stage
      mbar_expect_tx(fb, W * 128u);
      if (W) bulk_g2s_stream(sbase, a.pool + (size_t)off * 32, W * 128u, fb, stream_policy);
    }
    __syncwarp();
  };
  // R of my j-th slice, lane = row: one coalesced 128-byte load per objective,
  // issued one slice ahead of its use
  auto load_r = [&](int j, RT (&Rr)[NO]) {
    const size_t sl = (size_t)(sl0 + j * kWarps);
#pragma unroll
    for (int o = 0; o < NO; ++o) Rr[o] = __ldcs(v.R[o] + sl * 32 + lane);   // streamed: read once
  };

  const int q = lane / a.A_pad, act = lane % a.A_pad;
  const int nS = (int)a.nS, Nc = (int)a.Nc;
  const int s_lo = (int)pr.s_lo, s_hi = (int)pr.s_hi;
  const RT invN = (RT)1 / (RT)a.N;
  float rf[NO];      // FP32 residuals
  double r[NO];      // FP64 residuals
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    rf[o] = 0.f;
    r[o] = 0.0;
  }
  for (int j = 0; j < kDepth && j < n_mine; ++j) issue(j, j);
  RT Rn[NO];   // R of the next slice
#pragma unroll
  for (int o = 0; o < NO; ++o) Rn[o] = (RT)0;
  if (n_mine > 0) load_r(0, Rn);
  int st = 0;
  uint32_t phase = 0;
  int s = sl0 * a.spw + q;                      // state of this lane's row in my j-th slice
  const int s_step = kWarps * a.spw;
  // active-layer Jacobi: layer t_cur of my state s (s < t_end = (t_cur+1) Nc)
  // and whether any of its values changed in this sweep
  uint8_t *chg_out = a.lflags ? a.lflags + (size_t)(k % 3) * (a.nt + 1) : nullptr;
  int t_cur = s / Nc, t_end = (t_cur + 1) * Nc;
  bool chg = false;
  for (int j = 0; j < n_mine; ++j, s += s_step) {
    if (!mbar_wait(bar0 + 8u * (uint32_t)st, phase)) {
      if (lane == 0) atomicOr(a.err, 1);
      // drain: wait (bounded) for the copies still in flight into my stages
      for (int jj = j + 1; jj < j + kDepth && jj < n_mine; ++jj)
        mbar_wait(bar0 + 8u * (uint32_t)(jj % kDepth), (uint32_t)(jj / kDepth) & 1);
      break;
    }
    const unsigned char *sb = myring + st * pr.stage_bytes;
    const uint32_t *ent = reinterpret_cast<const uint32_t *>(sb) + lane;
    const bool valid = s >= s_lo && s < s_hi && act < a.A;
    RT Rv[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) Rv[o] = Rn[o];
    if (j + 1 < n_mine) load_r(j + 1, Rn);
    const int W = wst_s[warp * kDepth + st];
    Acc<RT> acc[NO];
    // successor layer base of this state; rows without successors (last
    // layer, padding lanes) hold only padding words and read V[|S|] = 0
    const int sn = (s + Nc <= nS) ? s + Nc : nS;
    const VPack<RT, NO> *Vn = v.in + sn;
#pragma unroll 4
    for (int kk = 0; kk < W; ++kk) {   // every column of the slice, ascending
      const uint32_t w = ent[kk * 32];
      const VPack<RT, NO> g = Vn[(int)(int16_t)(w & 0xFFFFu)];
#pragma unroll
      for (int o = 0; o < NO; ++o) acc[o].add(w >> 16, g.v[o], a.N);
    }
    if (a.spill_off) add_spill<RT, NO>(a, sl0 + (int64_t)j * kWarps, lane, Vn, acc);
    __syncwarp();
    if (j + kDepth < n_mine) issue(j + kDepth, st);   // refill the stage just read
    if (++st == kDepth) {
      st = 0;
      phase ^= 1u;
    }
    const bool head = act == 0 && s >= s_lo && s < s_hi;   // the lane that writes state s
    const bool term = head && __ldg(a.cls + s) != CLS_FREE;
    VPack<RT, NO> old{}, nv;
    if (head) old = v.in[s];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      RT qv = valid ? acc[o].q(Rv[o], invN) : -(RT)INFINITY;
      int qa = act;
      if (sizeof(RT) == 4 && a.A_pad == 32) {
        // one state per warp: order-preserving integer key, warp max in one
        // redux, lowest lane (= lowest action) among the maxima by ballot
        const uint32_t bits = __float_as_uint((float)qv + 0.0f);   // -0 keys like +0
        const uint32_t key = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
        const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
        qa = __ffs(__ballot_sync(0xffffffffu, key == kmax)) - 1;
        qv = __shfl_sync(0xffffffffu, qv, qa);
      } else {
        for (int m = 1; m < a.A_pad; m <<= 1) {
          const RT oq = __shfl_xor_sync(0xffffffffu, qv, m);
          const int oa = __shfl_xor_sync(0xffffffffu, qa, m);
          if (oq > qv || (oq == qv && oa < qa)) {
            qv = oq;
            qa = oa;
          }
        }
      }
      // a finished objective carries its value forward unchanged
      const bool upd = (live >> o) & 1u;
      nv.v[o] = upd ? qv : old.v[o];
      if (head && upd) {
        v.pol[o][s] = term ? (int16_t)-1 : (int16_t)qa;
        if constexpr (sizeof(RT) == 4) rf[o] = fmaxf(rf[o], fabsf(qv - old.v[o]));
        else r[o] = fmax(r[o], fabs(qv - old.v[o]));
      }
    }
#pragma unroll
    for (int o = NO; o < VPack<RT, NO>::W; ++o) nv.v[o] = (RT)0;
    if (head) {
      v.out[s] = nv;
      if (chg_out) {
        if (s >= t_end) {   // entered a later layer: publish the finished one
          if (chg) chg_out[t_cur] = 1;
          chg = false;
          do { ++t_cur; t_end += Nc; } while (s >= t_end);
        }
#pragma unroll
        for (int o = 0; o < NO; ++o) {   // bitwise: -0 vs +0 counts as a change
          if constexpr (sizeof(RT) == 4) chg |= __float_as_uint(nv.v[o]) != __float_as_uint(old.v[o]);
          else chg |= __double_as_longlong(nv.v[o]) != __double_as_longlong(old.v[o]);
        }
      }
    }
  }
  if (chg_out && chg) chg_out[t_cur] = 1;
  if (v.res[0]) {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      double ro = (sizeof(RT) == 4) ? (double)rf[o] : r[o];
      for (int m = 16; m > 0; m >>= 1) ro = fmax(ro, __shfl_xor_sync(0xffffffffu, ro, m));
      if (lane == 0) wmax[warp * NO + o] = ro;
    }
    __syncthreads();
#pragma unroll
    for (int o = 0; o < NO; ++o) {   // thread o publishes objective o (no dynamic index into v)
      if (tid == o) {
        double m = 0.0;
        for (int i = 0; i < kWarps; ++i) m = fmax(m, wmax[i * NO + o]);
        if (m > 0.0) atomicMax(&v.res[o][k - 1], (unsigned long long)__double_as_longlong(m));
      }
    }
  }
}

// Active-layer Jacobi sweep k: layer t needs recomputing if its own values
// or those of layer t+1 changed in sweep k-1 (otherwise V_{k+1} = V_k on it
// and the output table already holds that value from sweep k-1).  Sets
// [sl_lo, sl_hi) to the slices of the first through the last such layer
// (layers in between are recomputed, which yields their unchanged values).
// The leader CTA (one per model) clears the flags that sweep k+1 will set.
// Returns false when no layer changed: V_{k+1} = V_k, the residual stays 0.
// All threads of the CTA call it.
__device__ __forceinline__ bool active_range(const SolveArgs &a, int k, PipeRange &pr, bool leader) {
  const int nt = a.nt;
  const uint8_t *prev = a.lflags + (size_t)((k - 1) % 3) * (nt + 1);
  if (leader) {
    uint8_t *clr = a.lflags + (size_t)((k + 1) % 3) * (nt + 1);
    for (int t = threadIdx.x; t <= nt; t += blockDim.x) clr[t] = 0;
  }
  __shared__ int s_tlo, s_thi;
  if (threadIdx.x == 0) {
    s_tlo = nt;
    s_thi = -1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    if (prev[t] | prev[t + 1]) {
      atomicMin(&s_tlo, t);
      atomicMax(&s_thi, t);
    }
  }
  __syncthreads();
  const int tlo = s_tlo, thi = s_thi;
  if (thi < 0) return false;
  pr.sl_lo = (int64_t)tlo * a.Nc / a.spw;
  pr.sl_hi = min(a.n_slices, ((int64_t)(thi + 1) * a.Nc + a.spw - 1) / a.spw);
  return true;
}

template <typename RT, int NO>
__global__ void __launch_bounds__(32 * kWarps, 4) bellman_kernel(SolveArgs a, VSet<RT, NO> v, int k,
                                                              PipeRange pr) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ double wmax[kWarps * NO];
  __shared__ int wst_s[kWarps * kDepth];   // columns of the slice in each stage
  if (a.lflags && k >= 1 && !active_range(a, k, pr, blockIdx.x == 0)) return;
  const int64_t total = pr.sl_hi - pr.sl_lo;
  const int64_t per_cta = (total + gridDim.x - 1) / gridDim.x;
  const int64_t b_lo = pr.sl_lo + (int64_t)blockIdx.x * per_cta;
  const int64_t b_hi = min(pr.sl_hi, b_lo + per_cta);
  bellman_body<RT, NO>(a, v, k, b_lo, b_hi, pr, sm, wmax, wst_s);
}

// ---- grouped sweep: kGS states per warp step (models with A_pad = 32) ----
// One slice per state (A_pad = 32) makes the per-slice epilogue of
// bellman_body (a max/argmax over 32 lanes per objective, the stage refill,
// the writes) cost as much as the slice's backups.  Here a warp takes kGS
// consecutive slices at a time: lane (q, g) owns state q of the group and the
// actions g, g + kGL, g + 2 kGL, ... (ascending), forms their Q values one
// after another in registers and keeps the running maximum (strict >, so the
// lowest action wins ties); a log2(kGL)-step shuffle reduction over the kGL
// lanes of each state finishes the max/argmax.  Each row is still summed by
// one lane in ascending column order, so values and policy equal
// bellman_body's bit for bit.  The kGS slices of a group are copied into
// fixed slots of one stage (slot = wcap columns + 32 bytes: the 8-bank skew
// between slots keeps the lanes' shared-memory reads conflict-free).
constexpr int kGS = 4;           // states (slices) per group
constexpr int kGL = 32 / kGS;    // lanes per state
constexpr int kWarpsG = 16;      // warps per CTA: one CTA per SM (one V(s') window per L1)

static int slot_bytes_g(int wcap) { return wcap * 128 + 32; }
static size_t grouped_smem(int wcap) { return 256 + (size_t)kWarpsG * kDepth * kGS * slot_bytes_g(wcap); }
// dynamic shared memory the grouped kernel may take: the opt-in maximum per
// CTA (227 KB) less its static arrays and a margin
constexpr size_t kGroupedSmemMax = 227 * 1024 - 2048;

template <typename RT, int NO>
__device__ __forceinline__ void bellman_body_g(const SolveArgs &a, const VSet<RT, NO> &v, int k, int64_t b_lo,
                                               int64_t b_hi, const PipeRange &pr, unsigned char *sm,
                                               double *wmax, int *wst_s) {
  unsigned live = (1u << NO) - 1u;
  if (k > 1) {
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (v.res[o] && __longlong_as_double((long long)v.res[o][k - 2]) <= a.tol) live &= ~(1u << o);
  }
  if (!live) return;
  if (*(volatile int *)a.err) return;   // an earlier launch of this solve timed out
  if (a.work && k >= 1 && blockIdx.x == 0 && threadIdx.x == 0) a.work[k - 1] = (unsigned long long)(pr.sl_hi - pr.sl_lo);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm);   // [kWarpsG][kDepth]
  unsigned char *ring = sm + 256;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n_local = b_hi - b_lo;
  if (n_local <= 0) return;

  if (tid < kWarpsG * kDepth) mbar_init(smem_u32(full + tid), 1);
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  const int slot = pr.stage_bytes / kGS;
  unsigned char *myring = ring + (size_t)warp * kDepth * pr.stage_bytes;
  const int n_groups = (int)((n_local + kGS - 1) / kGS);
  const int n_mine = (n_groups > warp) ? (n_groups - warp + kWarpsG - 1) / kWarpsG : 0;
  const int first0 = (int)b_lo + warp * kGS;      // first slice of my j-th group: first0 + j*gstep
  const int gstep = kWarpsG * kGS;
  const int hi = (int)b_hi;
  const uint32_t ring0 = smem_u32(myring), bar0 = smem_u32(full + warp * kDepth);
  const uint64_t stream_policy = l2_evict_first();
  const int q = lane / kGL, g = lane % kGL;

  // lane l: metadata of slice l % kGS of my group 32/kGS * (j / (32/kGS)) + l / kGS
  constexpr int kMetaG = 32 / kGS;
  uint32_t m_off = 0, m_w = 0;
  // issue(j, st): lanes 0..kGS-1 copy the slices of my j-th group into their
  // slots of stage st (whole warp calls it)
  auto issue = [&](int j, int st) {
    if (j % kMetaG == 0) {   // one coalesced load for the next kMetaG groups
      const int sl = first0 + (j + lane / kGS) * gstep + lane % kGS;
      m_off = 0;
      m_w = 0;
      if (sl < hi) {
        m_off = __ldg(a.slice_off + sl);
        m_w = __ldg(a.slice_w + sl);
      }
    }
    const int src = (j % kMetaG) * kGS + (lane % kGS);
    const uint32_t off = __shfl_sync(0xffffffffu, m_off, src);
    uint32_t W = __shfl_sync(0xffffffffu, m_w, src);
    if (lane >= kGS) W = 0;
    uint32_t tot = W;
#pragma unroll
    for (int m = 1; m < kGS; m <<= 1) tot += __shfl_xor_sync(0xffffffffu, tot, m);
    const uint32_t fb = bar0 + 8u * (uint32_t)st;
    if (lane < kGS) wst_s[(warp * kDepth + st) * kGS + lane] = (int)W;
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the stage
      mbar_expect_tx(fb, tot * 128u);
    }
    __syncwarp();
    if (lane < kGS && W) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_g2s_stream(ring0 + (uint32_t)(st * pr.stage_bytes + lane * slot), a.pool + (size_t)off * 32, W * 128u,
                      fb, stream_policy);
    }
    __syncwarp();
  };
  // R of my j-th group (lane (q, g): rows g + i*kGL of slice q) and, on the
  // head lanes, the state's current values and class: loaded one group ahead
  auto load_r = [&](int j, RT (&Rr)[kGS][NO], VPack<RT, NO> &old, uint8_t &cls) {
    const int sl = first0 + j * gstep + q;
    if (sl < hi) {
#pragma unroll
      for (int i = 0; i < kGS; ++i)
#pragma unroll
        for (int o = 0; o < NO; ++o) Rr[i][o] = __ldcs(v.R[o] + (size_t)sl * 32 + i * kGL + g);
      if (g == 0) {
        old = v.in[sl];
        cls = __ldg(a.cls + sl);
      }
    }
  };

  const int nS = (int)a.nS, Nc = (int)a.Nc;
  const int s_lo = (int)pr.s_lo, s_hi = (int)pr.s_hi;
  const RT invN = (RT)1 / (RT)a.N;
  float rf[NO];
  double r[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    rf[o] = 0.f;
    r[o] = 0.0;
  }
  for (int j = 0; j < kDepth && j < n_mine; ++j) issue(j, j);
  RT Rn[kGS][NO];
#pragma unroll
  for (int i = 0; i < kGS; ++i)
#pragma unroll
    for (int o = 0; o < NO; ++o) Rn[i][o] = (RT)0;
  VPack<RT, NO> old_n{};
  uint8_t cls_n = 0;
  if (n_mine > 0) load_r(0, Rn, old_n, cls_n);
  int st = 0;
  uint32_t phase = 0;
  int s = first0 + q;   // spw = 1: state = slice
  uint8_t *chg_out = a.lflags ? a.lflags + (size_t)(k % 3) * (a.nt + 1) : nullptr;
  int t_cur = s / Nc, t_end = (t_cur + 1) * Nc;
  bool chg = false;
  for (int j = 0; j < n_mine; ++j, s += gstep) {
    if (!mbar_wait(bar0 + 8u * (uint32_t)st, phase)) {
      if (lane == 0) atomicOr(a.err, 1);
      for (int jj = j + 1; jj < j + kDepth && jj < n_mine; ++jj)
        mbar_wait(bar0 + 8u * (uint32_t)(jj % kDepth), (uint32_t)(jj / kDepth) & 1);
      break;
    }
    const uint32_t *ent = reinterpret_cast<const uint32_t *>(myring + st * pr.stage_bytes + q * slot) + g;
    const int Wq = wst_s[(warp * kDepth + st) * kGS + q];
    RT Rv[kGS][NO];
#pragma unroll
    for (int i = 0; i < kGS; ++i)
#pragma unroll
      for (int o = 0; o < NO; ++o) Rv[i][o] = Rn[i][o];
    const VPack<RT, NO> old = old_n;
    const uint8_t cls_s = cls_n;
    if (j + 1 < n_mine) load_r(j + 1, Rn, old_n, cls_n);
    const bool in_rng = s < hi && s >= s_lo && s < s_hi;
    const int sn = (s + Nc <= nS) ? s + Nc : nS;
    const VPack<RT, NO> *Vn = v.in + sn;
    Acc<RT> acc[kGS][NO];
#pragma unroll(NO == 1 ? 4 : 1)
    for (int kk = 0; kk < Wq; ++kk) {   // every column of the slice, ascending
#pragma unroll
      for (int i = 0; i < kGS; ++i) {
        const uint32_t w = ent[kk * 32 + i * kGL];
        const VPack<RT, NO> gv = Vn[(int)(int16_t)(w & 0xFFFFu)];
#pragma unroll
        for (int o = 0; o < NO; ++o) acc[i][o].add(w >> 16, gv.v[o], a.N);
      }
    }
    __syncwarp();
    if (j + kDepth < n_mine) issue(j + kDepth, st);   // refill the stage just read
    if (++st == kDepth) {
      st = 0;
      phase ^= 1u;
    }
    // running max over my actions (ascending, strict >: the lowest wins ties)
    RT qv[NO];
    int qa[NO];
    // (states outside the range are not written, so only padding actions
    // need masking)
    const bool full_a = a.A == 32;
#pragma unroll
    for (int i = 0; i < kGS; ++i) {
      const int act = i * kGL + g;
      const bool valid = full_a || act < a.A;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const RT x = valid ? acc[i][o].q(Rv[i][o], invN) : -(RT)INFINITY;
        if (i == 0 || x > qv[o]) {
          qv[o] = x;
          qa[o] = act;
        }
      }
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) {
#pragma unroll
      for (int m = 1; m < kGL; m <<= 1) {
        const RT oq = __shfl_xor_sync(0xffffffffu, qv[o], m);
        const int oa = __shfl_xor_sync(0xffffffffu, qa[o], m);
        if (oq > qv[o] || (oq == qv[o] && oa < qa[o])) {
          qv[o] = oq;
          qa[o] = oa;
        }
      }
    }
    const bool head = g == 0 && in_rng;   // the lane that writes state s
    const bool term = head && cls_s != CLS_FREE;
    VPack<RT, NO> nv;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const bool upd = (live >> o) & 1u;
      nv.v[o] = upd ? qv[o] : old.v[o];
      if (head && upd) {
        v.pol[o][s] = term ? (int16_t)-1 : (int16_t)qa[o];
        if constexpr (sizeof(RT) == 4) rf[o] = fmaxf(rf[o], fabsf(qv[o] - old.v[o]));
        else r[o] = fmax(r[o], fabs(qv[o] - old.v[o]));
      }
    }
#pragma unroll
    for (int o = NO; o < VPack<RT, NO>::W; ++o) nv.v[o] = (RT)0;
    if (head) {
      v.out[s] = nv;
      if (chg_out) {
        if (s >= t_end) {
          if (chg) chg_out[t_cur] = 1;
          chg = false;
          do { ++t_cur; t_end += Nc; } while (s >= t_end);
        }
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          if constexpr (sizeof(RT) == 4) chg |= __float_as_uint(nv.v[o]) != __float_as_uint(old.v[o]);
          else chg |= __double_as_longlong(nv.v[o]) != __double_as_longlong(old.v[o]);
        }
      }
    }
  }
  if (chg_out && chg) chg_out[t_cur] = 1;
  if (v.res[0]) {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      double ro = (sizeof(RT) == 4) ? (double)rf[o] : r[o];
      for (int m = 16; m > 0; m >>= 1) ro = fmax(ro, __shfl_xor_sync(0xffffffffu, ro, m));
      if (lane == 0) wmax[warp * NO + o] = ro;
    }
    __syncthreads();
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      if (tid == o) {
        double m = 0.0;
        for (int i = 0; i < kWarpsG; ++i) m = fmax(m, wmax[i * NO + o]);
        if (m > 0.0) atomicMax(&v.res[o][k - 1], (unsigned long long)__double_as_longlong(m));
      }
    }
  }
}

// ---- warp-specialized sweep: a producer warp stages rounds of slices ----
// Models with one state per slice (A_pad = 32).  Each CTA has kWsCons
// consumer warps and one producer warp, and walks its block of consecutive
// slices in rounds: a round holds up to kWsCons consecutive slices (as many as
// fit a slot's entry capacity) and consumer warp w takes slice w of every
// round, so the CTA's warps gather V(s') from one small window of layer t+1
// that L1 keeps.  The producer copies a round into one of kWsSlots
// shared-memory slots with TMA bulk copies -- the slices' entry columns (one
// copy when the pool is in slice order, else one per slice), then for every
// objective the round's R values in one copy (consecutive slices have
// consecutive R rows) -- completing on the slot's full barrier, and writes
// each slice's columns, cell class and current values (loaded one round
// ahead) into the slot's table; the consumers arrive on the slot's empty
// barrier once they have read it, and the producer refills it.  Slots are
// sized by the bytes the slices really have, not by the widest slice.  Lane l
// of a consumer sums row l (action l) in ascending column order, so every Q is
// the same float as in the other kernels, and the max over the 32 actions is
// one redux.sync on an order-preserving key with the lowest winning action by
// ballot (FP64: a butterfly): values and policy equal theirs bit for bit.
constexpr int kWsCons = 31;     // consumer warps per CTA (+ 1 producer = 1024 threads)
constexpr int kWsSlots = 3;     // round slots
// slices per consumer warp and round (warp w takes slices w, w + 31, ...;
// its slices' column loops run interleaved).  Measured on the large
// workload: 1 (rounds of 31 slices in three slots) 99.5 ms per solve, 2
// (rounds of 62 in two slots) 108-117 ms.
constexpr int kWsPer = 1;
constexpr int kWsRound = kWsCons * kWsPer;   // most slices in a round
constexpr int kWsTab = 32 * kWsPer;          // table entries per slot

struct WsHdr {
  uint64_t full[kWsSlots];      // producer arrival + the round's copied bytes
  uint64_t empty[kWsSlots];     // one arrival per consumer warp
  int2 round[kWsSlots];         // (first slice, slices in the round); 0 slices ends the block
  int2 slice[kWsSlots][kWsTab]; // (entry byte offset in the slot, W | cell class << 8) per slice
};
__host__ __device__ constexpr size_t ws_hdr_bytes() { return (sizeof(WsHdr) + 127) & ~(size_t)127; }
// the slices' current values, [kWsSlots][kWsTab]
template <typename RT, int NO>
__host__ __device__ constexpr size_t ws_old_bytes() { return (kWsSlots * kWsTab * sizeof(VPack<RT, NO>) + 127) & ~(size_t)127; }
template <typename RT>
__host__ __device__ constexpr int ws_r_bytes(int n_obj) { return n_obj * kWsTab * 32 * (int)sizeof(RT); }

// Work of the slices [lo, x) of a slice-ordered pool, in entry columns: their
// columns plus kWsSliceWork per slice (a slice's own cost -- its R rows, its
// state's values, the max over the actions -- weighed in columns).
constexpr int64_t kWsSliceWork = 24;

// CTA b of G takes the slices [ws_cut(b), ws_cut(b + 1)) of [lo, hi): the cut
// is the first x whose work from lo reaches b/G of the whole, so every CTA
// gets the same work however the widths vary (a pool in slice order has
// slice_off = the prefix sums of the widths: the work is monotone in x).  A
// 32-ary search over slice_off, about five dependent loads.  One warp calls it
// with its lanes converged; every lane returns the cut.
__device__ int64_t ws_cut(const SolveArgs &a, int64_t lo, int64_t hi, int64_t b, int64_t G) {
  if (b <= 0) return lo;
  if (b >= G) return hi;
  const int lane = threadIdx.x & 31;
  const uint32_t c0 = __ldg(a.slice_off + lo);
  const int64_t c_end = (int64_t)__ldg(a.slice_off + hi - 1) + (int64_t)__ldg(a.slice_w + hi - 1);
  const int64_t total = (c_end - (int64_t)c0) + kWsSliceWork * (hi - lo);
  const int64_t tgt = total * b / G;   // < total: the cut lies in (lo, hi) or is hi
  if (tgt <= 0) return lo;
  // invariant: work(l) < tgt <= work(h)
  int64_t l = lo, h = hi;
  while (h - l > 1) {
    const int64_t step = (h - l + 31) / 32;   // probes l + step, l + 2 step, ... below h
    const int64_t x = l + (int64_t)(lane + 1) * step;
    bool below = false;
    if (x < h) below = (int64_t)(__ldg(a.slice_off + x) - c0) + kWsSliceWork * (x - lo) < tgt;
    const int c = __popc(__ballot_sync(0xffffffffu, below));   // a prefix of the lanes
    const int64_t nh = min(h, l + (int64_t)(c + 1) * step);
    l += (int64_t)c * step;
    h = nh;
  }
  return h;
}

template <typename RT, int NO>
__device__ __forceinline__ void bellman_body_ws(const SolveArgs &a, const VSet<RT, NO> &v, int k,
                                                const PipeRange &pr, unsigned char *sm, double *wmax, int *s_flag,
                                                int64_t *s_cut) {
  using Pk = VPack<RT, NO>;
  unsigned live = (1u << NO) - 1u;
  if (k > 1) {
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (v.res[o] && __longlong_as_double((long long)v.res[o][k - 2]) <= a.tol) live &= ~(1u << o);
  }
  if (!live) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // one read of the error word for the whole CTA (an earlier launch timed out)
  if (tid == 0) *s_flag = *(volatile int *)a.err;
  // this CTA's slices: equal work (slice-ordered pool) or equal counts
  if (warp < 2) {
    int64_t x;
    if (a.pool_ordered && pr.sl_hi > pr.sl_lo) {
      x = ws_cut(a, pr.sl_lo, pr.sl_hi, (int64_t)blockIdx.x + warp, gridDim.x);
    } else {
      const int64_t per_cta = (pr.sl_hi - pr.sl_lo + gridDim.x - 1) / gridDim.x;
      x = min(pr.sl_hi, pr.sl_lo + ((int64_t)blockIdx.x + warp) * per_cta);
    }
    if (lane == 0) s_cut[warp] = x;
  }
  __syncthreads();
  if (*s_flag) return;
  if (a.work && k >= 1 && blockIdx.x == 0 && tid == 0) a.work[k - 1] = (unsigned long long)(pr.sl_hi - pr.sl_lo);
  const int64_t b_lo = s_cut[0], b_hi = s_cut[1];
  if (b_hi <= b_lo) return;

  WsHdr *hdr = reinterpret_cast<WsHdr *>(sm);
  Pk *olds = reinterpret_cast<Pk *>(sm + ws_hdr_bytes());   // [kWsSlots][32]
  constexpr int kRB = 32 * (int)sizeof(RT);                // one objective's R values of a slice
  constexpr int kRBytes = ws_r_bytes<RT>(NO);
  const int ecap = pr.stage_bytes;                         // entry bytes per slot
  const int slot_bytes = kRBytes + ecap;
  unsigned char *slots = sm + ws_hdr_bytes() + ws_old_bytes<RT, NO>();
  if (tid < kWsSlots) {
    mbar_init(smem_u32(&hdr->full[tid]), 1);
    mbar_init(smem_u32(&hdr->empty[tid]), kWsCons);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint32_t full0 = smem_u32(&hdr->full[0]), empty0 = smem_u32(&hdr->empty[0]);
  const long long wait_limit = a.wait_cycles > 0 ? a.wait_cycles : 4000000000LL;   // ~2 s
  const uint32_t slots0 = smem_u32(slots);

  if (warp == kWsCons) {
    // ---------------------------------------------------------- producer
    const uint64_t stream_policy = l2_evict_first();
    const RT *myR = nullptr;   // lane o copies objective o's R rows
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (lane == o) myR = v.R[o];
    int64_t sl = b_lo;
    bool failed = false;
    // lane l: slices sl + l + 32 i of the next round -- pool column, columns, cell
    // class and current values -- loaded before the wait for its slot
    uint32_t off[kWsPer];
    int W[kWsPer], cls[kWsPer];
    Pk old[kWsPer];
    auto fetch = [&]() {
#pragma unroll
      for (int i = 0; i < kWsPer; ++i) {
        off[i] = 0;
        W[i] = 0;
        cls[i] = 0;
        if (lane + 32 * i < kWsRound && sl + lane + 32 * i < b_hi) {
          const int64_t x = sl + lane + 32 * i;
          off[i] = __ldg(a.slice_off + x);
          W[i] = __ldg(a.slice_w + x);
          cls[i] = __ldg(a.cls + x);   // spw = 1: state = slice
          old[i] = v.in[x];
        }
      }
    };
    fetch();
    int slot = 0;
    uint32_t ph = 0;   // phase parity of the slot's current round
    for (int r = 0;; ++r) {
      if (r >= kWsSlots && !mbar_wait_suspend(empty0 + 8u * (uint32_t)slot, ph ^ 1u, wait_limit)) {
        if (lane == 0) atomicOr(a.err, 1);
        failed = true;
        break;
      }
      int n = 0, tot = 0, e[kWsPer];
      const uint32_t off0 = __shfl_sync(0xffffffffu, off[0], 0);
#pragma unroll
      for (int i = 0; i < kWsPer; ++i) e[i] = 0;
      if (sl < b_hi) {
        int carry = 0;
        bool open = true;
#pragma unroll
        for (int i = 0; i < kWsPer; ++i) {
          int cum = W[i] * 128;   // inclusive scan of the entry bytes
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, cum, d);
            if (lane >= d) cum += x;
          }
          cum += carry;
          const bool valid = open && lane + 32 * i < kWsRound && sl + lane + 32 * i < b_hi;
          const int ni = __popc(__ballot_sync(0xffffffffu, valid && cum <= ecap));   // a prefix of the lanes
          if (ni > 0) tot = __shfl_sync(0xffffffffu, cum, ni - 1);
          e[i] = cum - W[i] * 128;
          if (lane < ni) {
            hdr->slice[slot][32 * i + lane] = make_int2(e[i], W[i] | (cls[i] << 8));
            olds[slot * kWsTab + 32 * i + lane] = old[i];
          }
          n += ni;
          if (ni < 32) open = false;
          carry = __shfl_sync(0xffffffffu, cum, 31);
        }
      }
      __syncwarp();   // the slot's table is written before lane 0 arrives (release)
      const uint32_t fb = full0 + 8u * (uint32_t)slot;
      if (lane == 0) {
        hdr->round[slot] = make_int2((int)sl, n);
        if (n > 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the slot's earlier reads
          // (a.test_extra_tx: bytes that never arrive, on the first round of CTA 0,
          // so that a bounded wait runs out -- failure injection for tests)
          const uint32_t extra = (r == 0 && blockIdx.x == 0) ? a.test_extra_tx : 0u;
          mbar_expect_tx(fb, (uint32_t)(tot + NO * n * kRB) + extra);
        } else {
          mbar_arrive(fb);   // no more rounds: the consumers stop here
        }
      }
      __syncwarp();
      if (n == 0) break;
      const uint32_t sbase = slots0 + (uint32_t)(slot * slot_bytes);
      if (a.pool_ordered) {
        // the round's slices are back to back in the pool: one copy
        if (lane == 0 && tot > 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bulk_g2s_stream(sbase + (uint32_t)kRBytes, a.pool + (size_t)off0 * 32, (uint32_t)tot, fb, stream_policy);
        }
      } else {
#pragma unroll
        for (int i = 0; i < kWsPer; ++i) {
          if (lane + 32 * i < n && W[i] > 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_g2s_stream(sbase + (uint32_t)(kRBytes + e[i]), a.pool + (size_t)off[i] * 32, (uint32_t)W[i] * 128u,
                            fb, stream_policy);
          }
        }
      }
      if (lane < NO) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bulk_g2s_stream(sbase + (uint32_t)(lane * kWsTab * kRB), myR + (size_t)sl * 32, (uint32_t)(n * kRB), fb,
                        stream_policy);
      }
      __syncwarp();
      sl += n;
      fetch();   // the next round's slices
      if (++slot == kWsSlots) {
        slot = 0;
        ph ^= 1u;
      }
    }
    // After a timeout the consumers may have stopped reading: wait (bounded)
    // for the copies of the last rounds issued, whose slots were not reused,
    // so that none is still in flight when the CTA exits.  (Normally every
    // round was waited for by the consumers, and the end-of-block round has
    // reused one of these slots, so this must not run then.)
    if (failed) {
      for (int i = 0; i < kWsSlots; ++i) {
        slot = (slot + kWsSlots - 1) % kWsSlots;   // the last rounds, newest first
        if (slot == kWsSlots - 1) ph ^= 1u;
        mbar_wait_suspend(full0 + 8u * (uint32_t)slot, ph, wait_limit);
      }
    }
  } else {
    // ---------------------------------------------------------- consumers
    const int nS = (int)a.nS, Nc = (int)a.Nc;
    const int s_lo = (int)pr.s_lo, s_hi = (int)pr.s_hi;
    const RT invN = (RT)1 / (RT)a.N;
    const bool act_ok = lane < a.A;
    int16_t *mypol = v.pol[0];   // lane o < NO writes objective o's policy
#pragma unroll
    for (int o = 1; o < NO; ++o)
      if (lane == o) mypol = v.pol[o];
    const bool mylive = lane < NO && ((live >> lane) & 1u);
    float rf[NO];
    double rd[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      rf[o] = 0.f;
      rd[o] = 0.0;
    }
    uint8_t *chg_out = a.lflags ? a.lflags + (size_t)(k % 3) * (a.nt + 1) : nullptr;
    int t_cur = -1, t_end = 0;
    bool chg = false;
    int slot = 0;
    uint32_t ph = 0;
    for (;;) {
      if (!mbar_wait_suspend(full0 + 8u * (uint32_t)slot, ph, wait_limit)) {
        if (lane == 0) atomicOr(a.err, 1);
        break;
      }
      const int2 rdesc = hdr->round[slot];
      if (rdesc.y == 0) break;
      Acc<RT> accs[kWsPer][NO];
      RT Rvs[kWsPer][NO];
      Pk olds_i[kWsPer];
      int wcs[kWsPer], Ws[kWsPer];
      const uint32_t *ents[kWsPer];
      const Pk *Vns[kWsPer];
      const unsigned char *sb = slots + (size_t)slot * slot_bytes;
      int Wm = 0;
#pragma unroll
      for (int i = 0; i < kWsPer; ++i) {
        const int j = warp + kWsCons * i;
        Ws[i] = 0;
        wcs[i] = 0;
        ents[i] = nullptr;
        Vns[i] = v.in;
        if (j < rdesc.y) {
          const int si = rdesc.x + j;
          const int2 sd = hdr->slice[slot][j];
          wcs[i] = sd.y;
          Ws[i] = sd.y & 0xFF;
          ents[i] = reinterpret_cast<const uint32_t *>(sb + kRBytes + sd.x) + lane;
          Vns[i] = v.in + ((si + Nc <= nS) ? si + Nc : nS);
          const RT *Rs = reinterpret_cast<const RT *>(sb) + j * 32 + lane;
#pragma unroll
          for (int o = 0; o < NO; ++o) Rvs[i][o] = Rs[o * kWsTab * 32];
          olds_i[i] = olds[slot * kWsTab + j];
        }
        Wm = max(Wm, Ws[i]);
      }
#pragma unroll 2
      for (int kk = 0; kk < Wm; ++kk) {   // every column of each slice, ascending
#pragma unroll
        for (int i = 0; i < kWsPer; ++i) {
          if (kk < Ws[i]) {
            const uint32_t w = ents[i][kk * 32];
            const Pk g = Vns[i][(int)(int16_t)(w & 0xFFFFu)];
#pragma unroll
            for (int o = 0; o < NO; ++o) accs[i][o].add(w >> 16, g.v[o], a.N);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8u * (uint32_t)slot);   // the slot is read
      if (++slot == kWsSlots) {
        slot = 0;
        ph ^= 1u;
      }
#pragma unroll
      for (int i = 0; i < kWsPer; ++i) {
        if (warp + kWsCons * i >= rdesc.y) continue;
        const int s = rdesc.x + warp + kWsCons * i;
        Acc<RT> (&acc)[NO] = accs[i];
        RT (&Rv)[NO] = Rvs[i];
        const Pk old = olds_i[i];
        const int wc = wcs[i];
        if (a.spill_off) add_spill<RT, NO>(a, s, lane, v.in + ((s + Nc <= nS) ? s + Nc : nS), acc);
        RT qv[NO];
        int qa[NO];
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          RT q = act_ok ? acc[o].q(Rv[o], invN) : -(RT)INFINITY;
          int ia = lane;
          if constexpr (sizeof(RT) == 4) {
            // order-preserving key (-0 keys like +0): the max in one redux,
            // the lowest lane (= lowest action) among the maxima by ballot
            const uint32_t bits = __float_as_uint((float)q + 0.0f);
            const uint32_t key = bits ^ ((uint32_t)((int32_t)bits >> 31) | 0x80000000u);
            const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
            ia = __ffs(__ballot_sync(0xffffffffu, key == kmax)) - 1;
            q = __shfl_sync(0xffffffffu, q, ia);
          } else {
#pragma unroll
            for (int m = 1; m < 32; m <<= 1) {
              const RT oq = __shfl_xor_sync(0xffffffffu, q, m);
              const int oa = __shfl_xor_sync(0xffffffffu, ia, m);
              if (oq > q || (oq == q && oa < ia)) {
                q = oq;
                ia = oa;
              }
            }
          }
          qv[o] = q;
          qa[o] = ia;
        }
        if (s < s_lo || s >= s_hi) continue;
        const bool term = (wc >> 8) != CLS_FREE;
        Pk nv;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          const bool upd = (live >> o) & 1u;
          nv.v[o] = upd ? qv[o] : old.v[o];
          if (upd) {
            if constexpr (sizeof(RT) == 4) rf[o] = fmaxf(rf[o], fabsf(qv[o] - old.v[o]));
            else rd[o] = fmax(rd[o], fabs(qv[o] - old.v[o]));
          }
        }
#pragma unroll
        for (int o = NO; o < Pk::W; ++o) nv.v[o] = (RT)0;
        int myqa = qa[0];
#pragma unroll
        for (int o = 1; o < NO; ++o)
          if (lane == o) myqa = qa[o];
        if (mylive) mypol[s] = term ? (int16_t)-1 : (int16_t)myqa;
        if (lane == 0) v.out[s] = nv;
        if (chg_out) {
          if (s >= t_end) {   // entered a later layer: publish the finished one
            if (chg && lane == 0) chg_out[t_cur] = 1;
            chg = false;
            t_cur = s / Nc;
            t_end = (t_cur + 1) * Nc;
          }
#pragma unroll
          for (int o = 0; o < NO; ++o) {   // bitwise: -0 vs +0 counts as a change
            if constexpr (sizeof(RT) == 4) chg |= __float_as_uint(nv.v[o]) != __float_as_uint(old.v[o]);
            else chg |= __double_as_longlong(nv.v[o]) != __double_as_longlong(old.v[o]);
          }
        }
      }
    }
    if (chg_out && chg && lane == 0) chg_out[t_cur] = 1;
    if (v.res[0] && lane == 0) {
#pragma unroll
      for (int o = 0; o < NO; ++o) wmax[warp * NO + o] = (sizeof(RT) == 4) ? (double)rf[o] : rd[o];
    }
  }
  if (v.res[0]) {
    __syncthreads();
#pragma unroll
    for (int o = 0; o < NO; ++o) {   // thread o publishes objective o
      if (tid == o) {
        double m = 0.0;
        for (int i = 0; i < kWsCons; ++i) m = fmax(m, wmax[i * NO + o]);
        if (m > 0.0) atomicMax(&v.res[o][k - 1], (unsigned long long)__double_as_longlong(m));
      }
    }
  }
}

template <typename RT, int NO>
__global__ void __launch_bounds__(32 * (kWsCons + 1), 1) bellman_kernel_ws(SolveArgs a, VSet<RT, NO> v, int k,
                                                                         PipeRange pr) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ double wmax[kWsCons * NO];
  __shared__ int s_flag;
  __shared__ int64_t s_cut[2];
  if (a.lflags && k >= 1 && !active_range(a, k, pr, blockIdx.x == 0)) return;
  bellman_body_ws<RT, NO>(a, v, k, pr, sm, wmax, &s_flag, s_cut);
}

// Plan of batched Jacobi sweep k (one block): per model, the slices of the
// layers whose inputs changed in sweep k-1 (nothing once the model met the
// tolerance or ran max_sweeps), with the model's flags for sweep k+1
// cleared; layered (tol = 0): the slices of layer nt - k of every model that
// has it.  Then the total is cut into chunks of about total / G slices,
// each model's range into whole chunks, so every CTA entry of the sweep
// holds one model's contiguous range (entries past the last: item -1).
// n <= blockDim.x.
__global__ void plan_batch_kernel(const BatchSolveItem *items, int n, int k, BatchCta *ctas, int G,
                                  int n_entries, int layered) {
  __shared__ long long s_cnt[1024];
  __shared__ int s_ctas[1024];
  __shared__ long long s_chunk;
  const int i = threadIdx.x;
  long long lo = 0, hi = 0, s_lo = 0, s_hi = 0;
  if (i < n && layered) {   // step k: layer nt - k of every model that has it
    const SolveArgs &a = items[i].a;
    const int t = a.nt - k;
    if (t >= 0 && !*(volatile int *)a.err) {
      s_lo = (long long)t * a.Nc;
      s_hi = s_lo + a.Nc;
      lo = s_lo / a.spw;
      hi = min((long long)a.n_slices, (s_hi + a.spw - 1) / a.spw);
    }
  } else if (i < n) {
    const BatchSolveItem &it = items[i];
    const SolveArgs &a = it.a;
    s_hi = a.nS;
    const bool done = k > it.max_sweeps ||
                      (k > 1 && __longlong_as_double((long long)it.res[k - 2]) <= a.tol) ||
                      *(volatile int *)a.err;
    if (a.lflags) {
      const int nt = a.nt;
      const uint8_t *prev = a.lflags + (size_t)((k - 1) % 3) * (nt + 1);
      uint8_t *clr = a.lflags + (size_t)((k + 1) % 3) * (nt + 1);
      int tlo = nt, thi = -1;
      for (int t = 0; t < nt; ++t) {
        if (prev[t] | prev[t + 1]) {
          tlo = min(tlo, t);
          thi = t;
        }
      }
      for (int t = 0; t <= nt; ++t) clr[t] = 0;
      if (thi >= 0 && !done) {
        lo = (long long)tlo * a.Nc / a.spw;
        hi = min((long long)a.n_slices, ((long long)(thi + 1) * a.Nc + a.spw - 1) / a.spw);
      }
    } else if (!done) {
      hi = a.n_slices;
    }
  }
  s_cnt[i] = hi - lo;
  __syncthreads();
  if (i == 0) {
    long long tot = 0;
    for (int j = 0; j < n; ++j) tot += s_cnt[j];
    s_chunk = max(32LL, (tot + G - 1) / G);
  }
  __syncthreads();
  const long long chunk = s_chunk;
  s_ctas[i] = (i < n) ? (int)((s_cnt[i] + chunk - 1) / chunk) : 0;
  __syncthreads();
  if (i < n) {
    int first = 0;
    for (int j = 0; j < i; ++j) first += s_ctas[j];
    for (int c = 0; c < s_ctas[i] && first + c < n_entries; ++c) {
      const long long a0 = lo + (long long)c * chunk;
      ctas[first + c] = BatchCta{i, a0, min(hi, a0 + chunk), s_lo, s_hi};
    }
  }
  if (i == n) {   // unused entries
    int used = 0;
    for (int j = 0; j < n; ++j) used += s_ctas[j];
    for (int e = used; e < n_entries; ++e) ctas[e] = BatchCta{-1, 0, 0, 0, 0};
  }
}

// Batched Jacobi sweep k over many models: CTA b works on ctas[b] (one
// model's contiguous slice range, from the plan); each model stops on its
// own residual.
__global__ void __launch_bounds__(32 * kWarps, 4) bellman_batch_kernel(const BatchSolveItem *items,
                                                                    const BatchCta *ctas, int k,
                                                                    int stage_bytes, int layered) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ double wmax[kWarps];
  __shared__ int wst_s[kWarps * kDepth];
  const BatchCta c = ctas[blockIdx.x];
  if (c.item < 0) return;
  const BatchSolveItem &it = items[c.item];
  PipeRange pr;
  pr.sl_lo = c.sl_lo;
  pr.sl_hi = c.sl_hi;
  pr.s_lo = c.s_lo;
  pr.s_hi = c.s_hi;
  pr.stage_bytes = stage_bytes;
  pr.dtab_smem = 0;
  pr.grouped = 0;
  VSet<float, 1> v;
  v.R[0] = static_cast<const float *>(it.a.R);
  // Jacobi: ping-pong (sweep k reads Va when k is odd); layered: in place in Va
  v.in = reinterpret_cast<const VPack<float, 1> *>((layered || (k & 1)) ? it.Va : it.Vb);
  v.out = reinterpret_cast<VPack<float, 1> *>((layered || !(k & 1)) ? it.Va : it.Vb);
  v.pol[0] = it.policy;
  v.res[0] = layered ? nullptr : it.res;
  bellman_body<float, 1>(it.a, v, layered ? 0 : k, pr.sl_lo, pr.sl_hi, pr, sm, wmax, wst_s);
}

// The same over models with one state per slice, by the grouped sweep.
__global__ void __launch_bounds__(32 * kWarpsG, 1) bellman_batch_kernel_g(const BatchSolveItem *items,
                                                                       const BatchCta *ctas, int k,
                                                                       int stage_bytes, int layered) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ double wmax[kWarpsG];
  __shared__ int wst_s[kWarpsG * kDepth * kGS];
  const BatchCta c = ctas[blockIdx.x];
  if (c.item < 0) return;
  const BatchSolveItem &it = items[c.item];
  PipeRange pr;
  pr.sl_lo = c.sl_lo;
  pr.sl_hi = c.sl_hi;
  pr.s_lo = c.s_lo;
  pr.s_hi = c.s_hi;
  pr.stage_bytes = stage_bytes;
  pr.dtab_smem = 0;
  pr.grouped = 1;
  VSet<float, 1> v;
  v.R[0] = static_cast<const float *>(it.a.R);
  // Jacobi: ping-pong (sweep k reads Va when k is odd); layered: in place in Va
  v.in = reinterpret_cast<const VPack<float, 1> *>((layered || (k & 1)) ? it.Va : it.Vb);
  v.out = reinterpret_cast<VPack<float, 1> *>((layered || !(k & 1)) ? it.Va : it.Vb);
  v.pol[0] = it.policy;
  v.res[0] = layered ? nullptr : it.res;
  bellman_body_g<float, 1>(it.a, v, layered ? 0 : k, pr.sl_lo, pr.sl_hi, pr, sm, wmax, wst_s);
}

// Per model (one block each): sweeps and residual, final iterate into Va.
__global__ void finalize_batch_kernel(const BatchSolveItem *items, int layered) {
  const BatchSolveItem &it = items[blockIdx.x];
  __shared__ int s_sweeps;
  if (layered) {   // one pass, in place in Va
    if (threadIdx.x == 0) {
      it.stats[0] = 1.0;
      it.stats[1] = 0.0;
    }
    return;
  }
  if (threadIdx.x == 0) {
    int sw = it.max_sweeps;
    for (int k = 1; k <= it.max_sweeps; ++k)
      if (__longlong_as_double((long long)it.res[k - 1]) <= it.a.tol) { sw = k; break; }
    s_sweeps = sw;
    it.stats[0] = (double)sw;
    it.stats[1] = sw > 0 ? __longlong_as_double((long long)it.res[sw - 1]) : 0.0;
  }
  __syncthreads();
  if ((s_sweeps & 1) == 0) return;
  for (int64_t i = threadIdx.x; i <= it.a.nS; i += blockDim.x) it.Va[i] = it.Vb[i];
}

cudaError_t launch_bellman_batch(const BatchSolveItem *items_d, int n, BatchCta *ctas_d, int G, int k,
                                 int stage_bytes, int grouped, int layered, cudaStream_t st) {
  if (n > 1023) return cudaErrorInvalidValue;
  plan_batch_kernel<<<1, 1024, 0, st>>>(items_d, n, k, ctas_d, G, G + n, layered);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (grouped) {
    const size_t smem = 256 + (size_t)kWarpsG * kDepth * stage_bytes;
    bellman_batch_kernel_g<<<G + n, 32 * kWarpsG, smem, st>>>(items_d, ctas_d, k, stage_bytes, layered);
  } else {
    const size_t smem = 256 + (size_t)kWarps * kDepth * stage_bytes;
    bellman_batch_kernel<<<G + n, 32 * kWarps, smem, st>>>(items_d, ctas_d, k, stage_bytes, layered);
  }
  return cudaGetLastError();
}

cudaError_t launch_finalize_batch(const BatchSolveItem *items_d, int n, int layered, cudaStream_t st) {
  finalize_batch_kernel<<<n, 256, 0, st>>>(items_d, layered);
  return cudaGetLastError();
}

bool bellman_grouped_fits(int spw, int wcap) { return spw == 1 && grouped_smem(wcap) <= kGroupedSmemMax; }

cudaError_t prepare_bellman_batch(int wcap, int grouped, int *stage_bytes, int *per_sm) {
  if (grouped) {
    *stage_bytes = kGS * slot_bytes_g(wcap);
    const size_t smem = grouped_smem(wcap);
    if (smem > kGroupedSmemMax) return cudaErrorInvalidConfiguration;
    cudaError_t e = allow_max_smem((const void *)bellman_batch_kernel_g);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, bellman_batch_kernel_g, 32 * kWarpsG, smem);
  }
  *stage_bytes = stage_bytes_for(wcap);
  const size_t smem = 256 + (size_t)kWarps * kDepth * (*stage_bytes);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = allow_max_smem((const void *)bellman_batch_kernel);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, bellman_batch_kernel, 32 * kWarps, smem);
}

// stats_d[0] = sweeps, [1] = residual of the last sweep.  Copies the final
// iterate into Va when it ended in Vb.
template <typename RT>
__global__ void finalize_kernel(const unsigned long long *res, int max_sweeps, double tol, RT *Va,
                                const RT *Vb, int64_t n, double *stats_d) {
  __shared__ int s_sweeps;
  if (threadIdx.x == 0) {
    int sw = max_sweeps;
    for (int k = 1; k <= max_sweeps; ++k)
      if (__longlong_as_double((long long)res[k - 1]) <= tol) { sw = k; break; }
    s_sweeps = sw;
    if (blockIdx.x == 0) {
      stats_d[0] = (double)sw;
      stats_d[1] = sw > 0 ? __longlong_as_double((long long)res[sw - 1]) : 0.0;
    }
  }
  __syncthreads();
  if ((s_sweeps & 1) == 0) return;   // V_sweeps lives in Va already
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Va[i] = Vb[i];
}

// Warp-specialized sweep: per slot the R rows of up to 32 slices and the
// entry bytes of a round; three slots of ~53 KB (FP32, three objectives) keep
// two full rounds of copies in flight while one is read and leave ~60 KB of
// the SM's 256 KB to L1 for the V(s') window.  A slot always holds the widest
// slice.  (Measured on the large instance: 132 KB 114 ms, 160 KB 104 ms,
// 190 KB 104 ms, 215 KB 107 ms per fused solve; four or five slots in the
// same memory make shorter rounds and are slower.)
constexpr size_t kWsSmem = 160 * 1024;

template <typename RT, int NO>
static int ws_entry_bytes(int wcap, int smem_kb) {
  const size_t budget = smem_kb > 0 ? (size_t)smem_kb * 1024 : kWsSmem;
  const long per_slot = (long)((budget - ws_hdr_bytes() - ws_old_bytes<RT, NO>()) / kWsSlots) - ws_r_bytes<RT>(NO);
  long e = std::max<long>(per_slot, (long)wcap * 128);
  return (int)(e & ~127L);
}

template <typename RT, int NO>
static cudaError_t pipe_config(const SolveArgs &a, int64_t slices, PipeRange *pr, size_t *smem, int *blocks) {
  pr->dtab_smem = 0;
  if (a.spw == 1 && !a.small_ctas) {   // one state per slice: the warp-specialized sweep, any width
    pr->grouped = 2;
    pr->stage_bytes = ws_entry_bytes<RT, NO>(a.wcap, a.sweep_smem_kb);
    *smem = ws_hdr_bytes() + ws_old_bytes<RT, NO>() + (size_t)kWsSlots * (ws_r_bytes<RT>(NO) + pr->stage_bytes);
    cudaError_t e = allow_max_smem((const void *)bellman_kernel_ws<RT, NO>);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bellman_kernel_ws<RT, NO>, 32 * (kWsCons + 1), *smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t b = (int64_t)num_sms() * per_sm;
    const int64_t want = (slices + 2 * kWsRound - 1) / (2 * kWsRound);   // >= 2 rounds per CTA
    if (b > want) b = want;
    if (b < 1) b = 1;
    *blocks = (int)b;
    return cudaSuccess;
  }
  pr->grouped = 0;   // several states per slice: the warp-per-slice kernel
  pr->stage_bytes = stage_bytes_for(a.wcap);
  *smem = 256 + (size_t)kWarps * kDepth * pr->stage_bytes;
  if (*smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = allow_max_smem((const void *)bellman_kernel<RT, NO>);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bellman_kernel<RT, NO>, 32 * kWarps, *smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t b = (int64_t)num_sms() * per_sm;
  const int64_t want = (slices + 4 * kWarps - 1) / (4 * kWarps);   // >= 4 slices per warp
  if (b > want) b = want;
  if (b < 1) b = 1;
  *blocks = (int)b;
  return cudaSuccess;
}

// Fused solve epilogue: objective o's sweep count is the first k whose
// residual met tol (else max_sweeps); the table of the last executed sweep
// (the largest count; 0 = the initial table) holds every objective's final
// values, since a finished objective is carried forward unchanged.  Writes
// the stats and copies objective o's column into V[o][0..n).
template <typename RT, int NO>
struct VOut {
  RT *V[NO];
};
template <typename RT, int NO>
__global__ void finalize_multi_kernel(const double *stats_base, size_t blk, int max_sweeps, double tol,
                                      const VPack<RT, NO> *ta, const VPack<RT, NO> *tb, VOut<RT, NO> out,
                                      int64_t n, double *stats_out, int layered) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    int last = 0;
    for (int o = 0; o < NO; ++o) {
      const unsigned long long *res = reinterpret_cast<const unsigned long long *>(stats_base + o * blk + 4);
      int sw = max_sweeps;
      if (!layered) {
        for (int k = 1; k <= max_sweeps; ++k)
          if (__longlong_as_double((long long)res[k - 1]) <= tol) { sw = k; break; }
      }
      last = max(last, sw);
      if (blockIdx.x == 0 && !layered) {
        stats_out[o * blk + 0] = (double)sw;
        stats_out[o * blk + 1] = sw > 0 ? __longlong_as_double((long long)res[sw - 1]) : 0.0;
      }
    }
    s_last = layered ? 0 : last;
  }
  __syncthreads();
  const VPack<RT, NO> *t = (s_last & 1) ? tb : ta;   // sweep k writes tb when k is odd
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const VPack<RT, NO> p = t[i];
#pragma unroll
    for (int o = 0; o < NO; ++o) out.V[o][i] = p.v[o];
  }
}

template <typename RT, int NO>
static void launch_sweep(const SolveArgs &a, const VSet<RT, NO> &v, int k, const PipeRange &pr, int blocks,
                         size_t smem, cudaStream_t st) {
  if (pr.grouped == 2)
    bellman_kernel_ws<RT, NO><<<blocks, 32 * (kWsCons + 1), smem, st>>>(a, v, k, pr);
  else
    bellman_kernel<RT, NO><<<blocks, 32 * kWarps, smem, st>>>(a, v, k, pr);
}

// Objective o's status block: stats_d + o*(4 + max_sweeps) holds sweeps,
// residual, (objective 0: the error word), spare, then one residual slot
// per sweep.  NO = 1 iterates in the caller's V and io.Vtmp[0]; NO > 1 in
// the packed tables io.table[0..1], copied out to V[o] at the end.
template <typename RT, int NO>
static cudaError_t jacobi_t(const SolveArgs &a, int max_sweeps, const SolveIO &io, double *stats_d,
                            cudaStream_t st) {
  using Pk = VPack<RT, NO>;
  const size_t blk = 4 + (size_t)max_sweeps;
  Pk *ta = static_cast<Pk *>(NO == 1 ? io.V[0] : io.table[0]);
  Pk *tb = static_cast<Pk *>(NO == 1 ? io.Vtmp[0] : io.table[1]);
  VSet<RT, NO> odd, even;   // sweep k reads ta when k is odd, tb when even
  odd.in = ta;
  odd.out = tb;
  even.in = tb;
  even.out = ta;
  for (int o = 0; o < NO; ++o) {
    unsigned long long *res = reinterpret_cast<unsigned long long *>(stats_d + o * blk + 4);
    cudaError_t e = cudaMemsetAsync(res, 0, sizeof(unsigned long long) * (size_t)max_sweeps, st);
    if (e != cudaSuccess) return e;
    odd.R[o] = even.R[o] = static_cast<const RT *>(io.R[o]);
    odd.pol[o] = even.pol[o] = io.policy[o];
    odd.res[o] = even.res[o] = res;
  }
  if (a.lflags) {   // sweep 1 recomputes every layer
    cudaError_t e = cudaMemsetAsync(a.lflags, 1, (size_t)a.nt, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.lflags + a.nt, 0, (size_t)a.nt + 2, st);
    if (e == cudaSuccess && a.work) e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long) * max_sweeps, st);
    if (e != cudaSuccess) return e;
  }
  PipeRange pr;
  size_t smem = 0;
  int blocks = 1;
  cudaError_t e = pipe_config<RT, NO>(a, a.n_slices, &pr, &smem, &blocks);
  if (e != cudaSuccess) return e;
  pr.sl_lo = 0;
  pr.sl_hi = a.n_slices;
  pr.s_lo = 0;
  pr.s_hi = a.nS;
  for (int k = 1; k <= max_sweeps; ++k)
    launch_sweep<RT, NO>(a, (k & 1) ? odd : even, k, pr, blocks, smem, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t fb = (a.nS + 1 + 255) / 256;
  if (fb > 1024) fb = 1024;
  if constexpr (NO == 1) {
    finalize_kernel<RT><<<(unsigned)fb, 256, 0, st>>>(odd.res[0], max_sweeps, a.tol, static_cast<RT *>(io.V[0]),
                                                       static_cast<const RT *>(io.Vtmp[0]), a.nS + 1, stats_d);
  } else {
    VOut<RT, NO> out;
    for (int o = 0; o < NO; ++o) out.V[o] = static_cast<RT *>(io.V[o]);
    finalize_multi_kernel<RT, NO><<<(unsigned)fb, 256, 0, st>>>(stats_d, blk, max_sweeps, a.tol, ta, tb, out,
                                                                 a.nS + 1, stats_d, 0);
  }
  return cudaGetLastError();
}

template <typename RT>
static cudaError_t jacobi_n(const SolveArgs &a, int max_sweeps, const SolveIO &io, double *stats_d,
                            cudaStream_t st) {
  switch (io.n) {
    case 1: return jacobi_t<RT, 1>(a, max_sweeps, io, stats_d, st);
    case 2: return jacobi_t<RT, 2>(a, max_sweeps, io, stats_d, st);
    case 3: return jacobi_t<RT, 3>(a, max_sweeps, io, stats_d, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_jacobi_multi(const SolveArgs &a, int precision, int max_sweeps, const SolveIO &io,
                                double *stats_d, cudaStream_t st) {
  if (precision == MDP_FP64_CHECK) return jacobi_n<double>(a, max_sweeps, io, stats_d, st);
  return jacobi_n<float>(a, max_sweeps, io, stats_d, st);
}

cudaError_t launch_jacobi(const SolveArgs &a, int precision, int max_sweeps, void *Va, void *Vb,
                          int16_t *policy, double *stats_d, cudaStream_t st) {
  SolveIO io{};
  io.n = 1;
  io.R[0] = a.R;
  io.V[0] = Va;
  io.Vtmp[0] = Vb;
  io.policy[0] = policy;
  return launch_jacobi_multi(a, precision, max_sweeps, io, stats_d, st);
}

// In place: layer t reads layer t+1, finished by the previous launch.
template <typename RT, int NO>
static cudaError_t layered_t(const SolveArgs &a, int nt, const SolveIO &io, double *stats_d,
                             cudaStream_t st) {
  using Pk = VPack<RT, NO>;
  PipeRange pr0;
  size_t smem = 0;
  int blocks = 1;
  // every layer has the same number of slices (up to one straddling slice)
  cudaError_t e = pipe_config<RT, NO>(a, (a.Nc + a.spw - 1) / a.spw + 1, &pr0, &smem, &blocks);
  if (e != cudaSuccess) return e;
  VSet<RT, NO> v;
  Pk *t = static_cast<Pk *>(NO == 1 ? io.V[0] : io.table[0]);
  v.in = t;
  v.out = t;
  for (int o = 0; o < NO; ++o) {
    v.R[o] = static_cast<const RT *>(io.R[o]);
    v.pol[o] = io.policy[o];
    v.res[o] = nullptr;
  }
  for (int t_ = nt - 1; t_ >= 0; --t_) {
    PipeRange pr = pr0;
    pr.s_lo = (int64_t)t_ * a.Nc;
    pr.s_hi = pr.s_lo + a.Nc;
    pr.sl_lo = pr.s_lo / a.spw;
    pr.sl_hi = (pr.s_hi + a.spw - 1) / a.spw;
    launch_sweep<RT, NO>(a, v, 0, pr, blocks, smem, st);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || NO == 1) return e;
  VOut<RT, NO> out;
  for (int o = 0; o < NO; ++o) out.V[o] = static_cast<RT *>(io.V[o]);
  int64_t fb = (a.nS + 1 + 255) / 256;
  if (fb > 1024) fb = 1024;
  finalize_multi_kernel<RT, NO><<<(unsigned)fb, 256, 0, st>>>(stats_d, 0, 0, a.tol, t, t, out, a.nS + 1,
                                                               stats_d, 1);
  return cudaGetLastError();
}

template <typename RT>
static cudaError_t layered_n(const SolveArgs &a, int nt, const SolveIO &io, double *stats_d,
                             cudaStream_t st) {
  switch (io.n) {
    case 1: return layered_t<RT, 1>(a, nt, io, stats_d, st);
    case 2: return layered_t<RT, 2>(a, nt, io, stats_d, st);
    case 3: return layered_t<RT, 3>(a, nt, io, stats_d, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_layered_multi(const SolveArgs &a, int precision, int nt, const SolveIO &io,
                                 double *stats_d, cudaStream_t st) {
  if (precision == MDP_FP64_CHECK) return layered_n<double>(a, nt, io, stats_d, st);
  return layered_n<float>(a, nt, io, stats_d, st);
}

// -------------------------------------------------------------- export ----
// Paper layout row r = a*|S| + s.
// entries of internal row ir = 32 sl + lane held in its slice's spill block
__device__ __forceinline__ int spill_len(const uint32_t *spill, const uint32_t *spill_off, int64_t sl, int lane) {
  if (!spill_off) return 0;
  const uint32_t off = spill_off[sl];
  return off == kNoSlice ? 0 : (int)(spill[off + lane + 1] - spill[off + lane]);
}

__global__ void export_count_kernel(const uint8_t *__restrict__ nnz, const uint16_t *__restrict__ sinkc,
                                    const uint32_t *__restrict__ spill, const uint32_t *__restrict__ spill_off,
                                    int64_t nS, int A, int A_pad, int64_t *__restrict__ rowlen) {
  const int64_t rows = nS * A;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t act = r / nS, s = r % nS;
    const int64_t ir = s * A_pad + act;
    rowlen[r] = nnz[ir] + spill_len(spill, spill_off, ir / 32, (int)(ir % 32)) + (sinkc[ir] ? 1 : 0);
  }
}

// in-place exclusive scan of x[0..n) (int64), tile = 1024 per block
__global__ void scan_tiles_kernel(int64_t *x, int64_t n, int64_t *tile_sums) {
  __shared__ int64_t sh[1024];
  const int64_t base = (int64_t)blockIdx.x * 1024;
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) sh[i] = (base + i < n) ? x[base + i] : 0;
  __syncthreads();
  // Hillis-Steele inclusive scan over 1024 entries with 256 threads x 4
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t v[4];
    for (int u = 0; u < 4; ++u) {
      const int i = threadIdx.x * 4 + u;
      v[u] = (i >= off) ? sh[i - off] : 0;
    }
    __syncthreads();
    for (int u = 0; u < 4; ++u) sh[threadIdx.x * 4 + u] += v[u];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
    if (base + i < n) x[base + i] = (i == 0) ? 0 : sh[i - 1];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = sh[1023];
}

__global__ void scan_add_kernel(int64_t *x, int64_t n, const int64_t *tile_offs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += tile_offs[i / 1024];
}

// exclusive scan in place; scratch must hold ceil(n/1024) + ceil(n/1024^2) + ... entries
static cudaError_t exclusive_scan(int64_t *x, int64_t n, int64_t *scratch, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = (n + 1023) / 1024;
  scan_tiles_kernel<<<(unsigned)tiles, 256, 0, st>>>(x, n, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || tiles == 1) return e;
  e = exclusive_scan(scratch, tiles, scratch + tiles, st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  scan_add_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, scratch);
  return cudaGetLastError();
}

// One warp per slice: the slice's W columns are W*128 contiguous bytes in
// both pools, copied as 16-byte vectors; then the new offset is recorded.
__global__ void pool_reorder_kernel(const uint32_t *__restrict__ pool, uint32_t *__restrict__ out,
                                    uint32_t *slice_off, const uint8_t *__restrict__ slice_w,
                                    const int64_t *__restrict__ new_off, int64_t n_slices) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = wid; sl < n_slices; sl += nwarps) {
    const int W = slice_w[sl];
    const int64_t no = new_off[sl];
    if (W) {
      const uint4 *src = reinterpret_cast<const uint4 *>(pool + (size_t)slice_off[sl] * 32);
      uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)no * 32);
      for (int i = lane; i < W * 8; i += 32) dst[i] = src[i];
    }
    __syncwarp();
    if (lane == 0) slice_off[sl] = (uint32_t)no;
  }
}

__global__ void slice_width_kernel(const uint8_t *__restrict__ slice_w, int64_t *x, int64_t n_slices) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n_slices; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = i < n_slices ? (int64_t)slice_w[i] : 0;
}

cudaError_t launch_pool_reorder(const uint32_t *pool, uint32_t *out, uint32_t *slice_off, const uint8_t *slice_w,
                                int64_t n_slices, cudaStream_t st) {
  const int64_t n = n_slices + 1;
  int64_t need = n, nn = n;   // offsets, then the scan's tile sums
  while (nn > 1) { nn = (nn + 1023) / 1024; need += nn; }
  int64_t *x = nullptr;
  cudaError_t e = dev_alloc((void **)&x, sizeof(int64_t) * (size_t)(need + 1), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = std::min<int64_t>(8192, (n + 255) / 256);
  slice_width_kernel<<<(unsigned)blocks, 256, 0, st>>>(slice_w, x, n_slices);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = exclusive_scan(x, n, x + n, st);
  if (e == cudaSuccess) {
    blocks = std::min<int64_t>(num_sms() * 16, (n_slices + 7) / 8);
    if (blocks < 1) blocks = 1;
    pool_reorder_kernel<<<(unsigned)blocks, 256, 0, st>>>(pool, out, slice_off, slice_w, x, n_slices);
    e = cudaGetLastError();
  }
  dev_free(x, st);
  return e;
}

template <typename RT>
__global__ void export_fill_kernel(const uint32_t *__restrict__ pool, const uint32_t *__restrict__ slice_off,
                                   const uint8_t *__restrict__ nnz, const uint16_t *__restrict__ sinkc,
                                   const uint32_t *__restrict__ spill, const uint32_t *__restrict__ spill_off,
                                   const RT *__restrict__ Rsrc, int64_t nS, int64_t Nc, int A, int A_pad,
                                   int spw, int64_t n_slices, const int64_t *__restrict__ rowptr,
                                   int64_t *col, int32_t *count, RT *Rdst) {
  const int64_t nrow = n_slices * 32;
  for (int64_t ir = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ir < nrow; ir += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = ir / 32;
    const int lane = (int)(ir % 32);
    const int q = lane / A_pad, act = lane % A_pad;
    const int64_t s = sl * spw + q;
    if (s >= nS || act >= A) continue;
    const int64_t r = (int64_t)act * nS + s;
    if (Rdst) Rdst[r] = Rsrc[ir];
    if (!col && !count) continue;
    int e = nnz[ir];
    const int64_t o = rowptr[r];
    if (e > 0) {
      const uint32_t off = slice_off[sl];
      for (int k = 0; k < e; ++k) {
        const uint32_t w = pool[((size_t)off + k) * 32 + lane];
        if (col) col[o + k] = s + Nc + (int64_t)(int16_t)(w & 0xFFFFu);
        if (count) count[o + k] = (int32_t)(w >> 16);
      }
    }
    const int ns = spill_len(spill, spill_off, sl, lane);
    if (ns > 0) {   // the row's tail, after its ELL entries (ascending order continues)
      const uint32_t *ent = spill + spill_off[sl] + kSpillHdr + spill[spill_off[sl] + lane];
      for (int k = 0; k < ns; ++k) {
        const uint32_t w = ent[k];
        if (col) col[o + e + k] = s + Nc + (int64_t)(int16_t)(w & 0xFFFFu);
        if (count) count[o + e + k] = (int32_t)(w >> 16);
      }
      e += ns;
    }
    if (sinkc[ir]) {
      if (col) col[o + e] = nS;
      if (count) count[o + e] = (int32_t)sinkc[ir];
    }
  }
}

cudaError_t launch_export(const mdp_model_t *m, int obj, int64_t *rowptr, int64_t *col,
                          int32_t *count, void *R, cudaStream_t st) {
  const int64_t rows = m->nS * m->A;
  int64_t blocks = (rows + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  export_count_kernel<<<(unsigned)blocks, 256, 0, st>>>(m->nnz, m->sinkc, m->spill, m->spill_off, m->nS, m->A,
                                                         m->A_pad, rowptr);
  cudaError_t e = cudaMemsetAsync(rowptr + rows, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  // scan scratch: geometric series of tile counts
  int64_t need = 0, nn = rows + 1;
  while (nn > 1) { nn = (nn + 1023) / 1024; need += nn; }
  int64_t *scratch = nullptr;
  e = dev_alloc((void **)&scratch, sizeof(int64_t) * (size_t)(need + 1), st);
  if (e != cudaSuccess) return e;
  e = exclusive_scan(rowptr, rows + 1, scratch, st);
  if (e != cudaSuccess) { dev_free(scratch, st); return e; }
  int64_t nrow = m->n_slices * 32;
  int64_t fb = (nrow + 255) / 256;
  if (fb > 8192) fb = 8192;
  const size_t esz = (m->precision == MDP_FP64_CHECK) ? 8 : 4;
  if (m->precision == MDP_FP64_CHECK)
    export_fill_kernel<double><<<(unsigned)fb, 256, 0, st>>>(
        m->pool, m->slice_off, m->nnz, m->sinkc, m->spill, m->spill_off,
        static_cast<const double *>(m->R) + (size_t)obj * m->rows_pad,
        m->nS, m->Nc, m->A, m->A_pad, m->spw, m->n_slices, rowptr, col, count, (double *)R);
  else
    export_fill_kernel<float><<<(unsigned)fb, 256, 0, st>>>(
        m->pool, m->slice_off, m->nnz, m->sinkc, m->spill, m->spill_off,
        static_cast<const float *>(m->R) + (size_t)obj * m->rows_pad,
        m->nS, m->Nc, m->A, m->A_pad, m->spw, m->n_slices, rowptr, col, count, (float *)R);
  (void)esz;
  e = cudaGetLastError();
  dev_free(scratch, st);
  return e;
}

}  // namespace mdpgb
