// bellman.cu -- sparse value iteration (steps a7-a8) and the small helper
// kernels of the build (cell classes, sub-grid offset table, field extremes)
// and of the paper-layout export.
//
// Bellman backup (Sec. II-B): Q(s,a) = R(s,a) + sum_j P_j V(s'_j),
// V_{k+1}(s) = max_a Q(s,a), pi(s) = argmax_a Q(s,a) (lowest index wins ties).
// One warp per slice: lane l streams its row's (bin, count) words from the
// slice's columns (128 B per k, coalesced), gathers V(s') from the next time
// layer (L2 resident), and a segmented butterfly over the A_pad lanes of a
// state gives the max and argmax.  Residual max|V_{k+1} - V_k| is reduced on
// the device; a sweep whose predecessor met the tolerance exits at once, so a
// fixed launch sequence needs no host round trip between sweeps.
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

// One warp per slice in [sl_lo, sl_hi).  Writes Vout[s] and policy[s] for
// states in [s_lo, s_hi); returns the warp's residual contribution.
template <typename RT>
__device__ __forceinline__ double backup_slice(const SolveArgs &a, int64_t sl, int64_t s_lo,
                                              int64_t s_hi, const RT *Vin, RT *Vout,
                                              int16_t *__restrict__ policy) {
  const int lane = threadIdx.x & 31;
  const int q = lane / a.A_pad, act = lane % a.A_pad;
  const int64_t s = sl * a.spw + q;
  const bool valid = s >= s_lo && s < s_hi && act < a.A;
  const int64_t ir = sl * 32 + lane;
  const uint32_t off = __ldg(a.slice_off + sl);
  const int e = valid ? (int)__ldg(a.nnz + ir) : 0;
  Acc<RT> acc;
  const int64_t nxt = s + a.Nc;
  const uint32_t *col = a.pool + (size_t)off * 32 + lane;
  for (int k = 0; k < e; ++k) {
    const uint32_t w = __ldcs(col + (size_t)k * 32);
    const uint32_t b = w & 0xFFFFu;
    const int64_t sp = (b == kSinkBin) ? a.nS : nxt + __ldg(a.delta + b);
    acc.add(w >> 16, Vin[sp], a.N);
  }
  RT qv;
  if (valid) qv = acc.q(__ldcs(static_cast<const RT *>(a.R) + ir), (RT)1 / (RT)a.N);
  else qv = -(RT)INFINITY;
  int qa = act;
  for (int o = 1; o < a.A_pad; o <<= 1) {
    const RT oq = __shfl_xor_sync(0xffffffffu, qv, o);
    const int oa = __shfl_xor_sync(0xffffffffu, qa, o);
    if (oq > qv || (oq == qv && oa < qa)) {
      qv = oq;
      qa = oa;
    }
  }
  double res = 0.0;
  if (act == 0 && s >= s_lo && s < s_hi) {
    const RT old = Vin[s];
    Vout[s] = qv;
    policy[s] = (a.cls[s] != CLS_FREE) ? (int16_t)-1 : (int16_t)qa;
    res = fabs((double)qv - (double)old);
  }
  return res;
}

// Jacobi sweep k (1-based) reads V_{k-1} and writes V_k.  res[k-1] holds the
// residual of sweep k (bits of a non-negative double), zero-initialised.
template <typename RT>
__global__ void __launch_bounds__(256) jacobi_kernel(SolveArgs a, const RT *Vin, RT *Vout,
                                                     int16_t *policy,
                                                     unsigned long long *res, int k) {
  if (k > 1 && __longlong_as_double((long long)res[k - 2]) <= a.tol) return;  // converged earlier
  __shared__ double wmax[8];
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double r = 0.0;
  for (int64_t sl = gw; sl < a.n_slices; sl += nw) r = fmax(r, backup_slice<RT>(a, sl, 0, a.nS, Vin, Vout, policy));
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, wmax[i]);
    if (m > 0.0) atomicMax(&res[k - 1], (unsigned long long)__double_as_longlong(m));
  }
}

// Backward layer t: V of layer t+1 is final, so one pass per layer suffices.
template <typename RT>
__global__ void __launch_bounds__(256) layer_kernel(SolveArgs a, RT *V, int16_t *policy, int64_t s_lo,
                                                    int64_t s_hi, int64_t sl_lo, int64_t sl_hi) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = sl_lo + gw; sl < sl_hi; sl += nw) backup_slice<RT>(a, sl, s_lo, s_hi, V, V, policy);
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

static int solve_blocks(int64_t slices) {
  int64_t warps = slices;
  int64_t blocks = (warps + 7) / 8;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <typename RT>
static cudaError_t jacobi_t(const SolveArgs &a, int max_sweeps, RT *Va, RT *Vb, int16_t *policy,
                            double *stats_d, cudaStream_t st) {
  // residual slots live after the 4 stats doubles
  unsigned long long *res = reinterpret_cast<unsigned long long *>(stats_d + 4);
  cudaError_t e = cudaMemsetAsync(res, 0, sizeof(unsigned long long) * (size_t)max_sweeps, st);
  if (e != cudaSuccess) return e;
  const int blocks = solve_blocks(a.n_slices);
  for (int k = 1; k <= max_sweeps; ++k) {
    const RT *vin = (k & 1) ? Va : Vb;
    RT *vout = (k & 1) ? Vb : Va;
    jacobi_kernel<RT><<<blocks, 256, 0, st>>>(a, vin, vout, policy, res, k);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t fb = (a.nS + 1 + 255) / 256;
  if (fb > 1024) fb = 1024;
  finalize_kernel<RT><<<(unsigned)fb, 256, 0, st>>>(res, max_sweeps, a.tol, Va, Vb, a.nS + 1, stats_d);
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const SolveArgs &a, int precision, int max_sweeps, void *Va, void *Vb,
                          int16_t *policy, double *stats_d, cudaStream_t st) {
  if (precision == MDP_FP64_CHECK)
    return jacobi_t<double>(a, max_sweeps, (double *)Va, (double *)Vb, policy, stats_d, st);
  return jacobi_t<float>(a, max_sweeps, (float *)Va, (float *)Vb, policy, stats_d, st);
}

template <typename RT>
static cudaError_t layered_t(const SolveArgs &a, int nt, RT *V, int16_t *policy, cudaStream_t st) {
  for (int t = nt - 1; t >= 0; --t) {
    const int64_t s_lo = (int64_t)t * a.Nc, s_hi = s_lo + a.Nc;
    const int64_t sl_lo = s_lo / a.spw, sl_hi = (s_hi + a.spw - 1) / a.spw;
    layer_kernel<RT><<<solve_blocks(sl_hi - sl_lo), 256, 0, st>>>(a, V, policy, s_lo, s_hi, sl_lo, sl_hi);
  }
  return cudaGetLastError();
}

cudaError_t launch_layered(const SolveArgs &a, int precision, int nt, void *V, int16_t *policy,
                           double *stats_d, cudaStream_t st) {
  (void)stats_d;
  if (precision == MDP_FP64_CHECK) return layered_t<double>(a, nt, (double *)V, policy, st);
  return layered_t<float>(a, nt, (float *)V, policy, st);
}

// -------------------------------------------------------------- export ----
// Paper layout row r = a*|S| + s.
__global__ void export_count_kernel(const uint8_t *__restrict__ nnz, int64_t nS, int A, int A_pad,
                                    int64_t *__restrict__ rowlen) {
  const int64_t rows = nS * A;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t act = r / nS, s = r % nS;
    rowlen[r] = nnz[s * A_pad + act];
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

template <typename RT>
__global__ void export_fill_kernel(const uint32_t *__restrict__ pool, const uint32_t *__restrict__ slice_off,
                                   const uint8_t *__restrict__ nnz, const RT *__restrict__ Rsrc,
                                   const int32_t *__restrict__ delta, int64_t nS, int64_t Nc, int A,
                                   int A_pad, int spw, int64_t n_slices, const int64_t *__restrict__ rowptr,
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
    const int e = nnz[ir];
    if (e == 0 || (!col && !count)) continue;
    const uint32_t off = slice_off[sl];
    const int64_t o = rowptr[r];
    for (int k = 0; k < e; ++k) {
      const uint32_t w = pool[((size_t)off + k) * 32 + lane];
      const uint32_t b = w & 0xFFFFu;
      if (col) col[o + k] = (b == kSinkBin) ? nS : s + Nc + delta[b];
      if (count) count[o + k] = (int32_t)(w >> 16);
    }
  }
}

cudaError_t launch_export(const mdp_model_t *m, int obj, int64_t *rowptr, int64_t *col,
                          int32_t *count, void *R, cudaStream_t st) {
  const int64_t rows = m->nS * m->A;
  int64_t blocks = (rows + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  export_count_kernel<<<(unsigned)blocks, 256, 0, st>>>(m->nnz, m->nS, m->A, m->A_pad, rowptr);
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
        m->pool, m->slice_off, m->nnz, static_cast<const double *>(m->R) + (size_t)obj * m->rows_pad,
        m->delta, m->nS, m->Nc, m->A, m->A_pad, m->spw, m->n_slices, rowptr, col, count, (double *)R);
  else
    export_fill_kernel<float><<<(unsigned)fb, 256, 0, st>>>(
        m->pool, m->slice_off, m->nnz, static_cast<const float *>(m->R) + (size_t)obj * m->rows_pad,
        m->delta, m->nS, m->Nc, m->A, m->A_pad, m->spw, m->n_slices, rowptr, col, count, (float *)R);
  (void)esz;
  e = cudaGetLastError();
  dev_free(scratch, st);
  return e;
}

}  // namespace mdpgb
