// noalloc.cu -- Jacobi value iteration that allocates no device memory.
//
// mdp_solve() obtains its scratch (the second value buffer of the Jacobi
// ping-pong, the per-sweep residual slots and a few status words) from the
// device memory pool on every call.  Some callers cannot allow that: a
// real-time replanning loop that must not allocate once it is running
// (an allocation can block and can fragment a tight memory budget), or an
// application whose device memory is owned by another allocator that hands
// out no extra space.  mdp_solve_noalloc() runs the same kernels with its
// scratch in the fixed array below instead.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "mdp_internal.cuh"

namespace mdpgb {

// Scratch layout: [0, kVBytes) the partner value buffer; then 4 status
// doubles (sweeps, residual, error word) and one residual slot per sweep;
// one work count per sweep; three arrays of kLayers layer flags for the
// active-layer sweeps (models with more than kLayers - 1 time layers run
// full sweeps, which give the same results).
constexpr size_t kNoAllocVBytes = 8u << 20;                        // 8 MiB
constexpr size_t kNoAllocSweeps = 4092;
constexpr size_t kNoAllocLayers = 4096;
constexpr size_t kNoAllocStatus = 8 * (4 + kNoAllocSweeps);
constexpr size_t kNoAllocWork = 8 * kNoAllocSweeps;
constexpr size_t kNoAllocBytes = kNoAllocVBytes + kNoAllocStatus + kNoAllocWork + 3 * kNoAllocLayers;   // 8 MiB + 76 KiB

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64];   // device address of the array, per device ordinal

// Device address of the array on the current device (the host-side name of a
// __device__ variable is only a stand-in, never a device address).
static mdp_status noalloc_scratch(unsigned char **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal out of range for the scratch table");
    return MDP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
  return MDP_OK;
}

}  // namespace mdpgb

using namespace mdpgb;

extern "C" mdp_status mdp_solve_noalloc(mdp_model m, int32_t obj, double tol, int32_t max_sweeps,
                                        void *V, int16_t *policy, void *stream,
                                        mdp_solve_stats *stats) {
  if (!m || !V || !policy) {
    set_error("invalid argument: NULL model, V or policy");
    return MDP_ERR_ARG;
  }
  if (obj < 0 || obj >= m->n_obj) {
    set_error("invalid argument: objective slot out of range");
    return MDP_ERR_ARG;
  }
  if (!(tol >= 0) && !(tol < 0)) {
    set_error("invalid argument: tol is NaN");
    return MDP_ERR_ARG;
  }
  if (max_sweeps < 0) {
    set_error("invalid argument: max_sweeps must be >= 0");
    return MDP_ERR_ARG;
  }
  if (max_sweeps == 0) max_sweeps = m->nt + 1;
  const size_t fsz = m->precision == MDP_FP64_CHECK ? 8 : 4;
  const size_t vbytes = fsz * (size_t)(m->nS + 1);
  if (vbytes > kNoAllocVBytes) {
    set_error("mdp_solve_noalloc: the model has " + std::to_string(m->nS) +
              " states; the fixed scratch holds a value vector of at most " +
              std::to_string(kNoAllocVBytes / fsz - 1) + " states (use mdp_solve)");
    return MDP_ERR_ARG;
  }
  if ((size_t)max_sweeps > kNoAllocSweeps) {
    set_error("mdp_solve_noalloc: max_sweeps above " + std::to_string(kNoAllocSweeps) +
              " does not fit the fixed scratch");
    return MDP_ERR_ARG;
  }
  if ((((uintptr_t)m->pool) | ((uintptr_t)m->R) | ((uintptr_t)m->nnz)) & 15) {
    set_error("model arrays are not 16-byte aligned");
    return MDP_ERR_CUDA;
  }
  if (m->nS + m->Nc >= ((int64_t)1 << 31)) {
    set_error("invalid argument: more than 2^31 states is not supported by the solver");
    return MDP_ERR_ARG;
  }
  unsigned char *scratch = nullptr;
  mdp_status s = noalloc_scratch(&scratch);
  if (s != MDP_OK) return s;
  void *Vb = scratch;
  double *sd = reinterpret_cast<double *>(scratch + kNoAllocVBytes);
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear what starts at zero
  MDP_CUDA_TRY(cudaMemsetAsync(sd, 0, sizeof(double) * 4, st));
  MDP_CUDA_TRY(cudaMemsetAsync(V, 0, vbytes, st));
  MDP_CUDA_TRY(cudaMemsetAsync(Vb, 0, vbytes, st));
  SolveArgs a;
  a.pool = m->pool; a.slice_off = m->slice_off; a.slice_w = m->slice_w; a.nnz = m->nnz;
  a.wcap = m->max_row_nnz > 1 ? m->max_row_nnz : 1;
  a.R = static_cast<const char *>(m->R) + fsz * (size_t)obj * m->rows_pad;
  a.cls = m->cls; a.delta = m->delta;
  a.nS = m->nS; a.Nc = m->Nc; a.n_slices = m->n_slices;
  a.A = m->A; a.A_pad = m->A_pad; a.spw = m->spw; a.N = m->N; a.nbins = m->nbins; a.tol = tol;
  a.err = reinterpret_cast<int *>(sd + 2);
  a.nt = m->nt;
  a.pool_ordered = m->pool_ordered;
  a.spill = m->spill;
  a.spill_off = m->spill_off;
  if ((size_t)m->nt + 1 <= kNoAllocLayers) {
    a.work = reinterpret_cast<unsigned long long *>(scratch + kNoAllocVBytes + kNoAllocStatus);
    a.lflags = scratch + kNoAllocVBytes + kNoAllocStatus + kNoAllocWork;
  }
  MDP_CUDA_TRY(launch_jacobi(a, m->precision, max_sweeps, V, Vb, policy, sd, st));
  double hs[3] = {0, 0, 0};
  unsigned long long wk[kNoAllocSweeps];   // per-sweep work counts (host stack, no allocation)
  MDP_CUDA_TRY(cudaMemcpyAsync(hs, sd, sizeof(hs), cudaMemcpyDeviceToHost, st));
  if (a.work)
    MDP_CUDA_TRY(cudaMemcpyAsync(wk, a.work, sizeof(unsigned long long) * max_sweeps, cudaMemcpyDeviceToHost, st));
  MDP_CUDA_TRY(cudaStreamSynchronize(st));
  int errw = 0;
  memcpy(&errw, &hs[2], sizeof(int));
  if (errw) {
    set_error("a bounded device wait expired in the Bellman pipeline");
    return MDP_ERR_TIMEOUT;
  }
  if (stats) {
    stats->sweeps = (int32_t)hs[0];
    stats->residual = hs[1];
    stats->solve_ms = 0.0;
    stats->backups = (int64_t)stats->sweeps * m->nS * m->A;
    if (a.work) {   // slices recomputed by the active-layer sweeps
      int64_t sl = 0;
      for (int k = 0; k < stats->sweeps; ++k) sl += (int64_t)wk[k];
      stats->backups = std::min<int64_t>(sl * m->spw, (int64_t)stats->sweeps * m->nS) * m->A;
    }
  }
  return MDP_OK;
}
