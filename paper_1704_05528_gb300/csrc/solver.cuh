// Shared pieces of the SVT driver: parameters, device work buffers, the R4SVD routine
// (Algorithm 3; Algorithm 2 when nothing is recycled) and the per-kernel-class profiler.
// Included by the fast-SVT driver and by the unrolled / adjoint driver.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {


using clk = std::chrono::steady_clock;
inline double seconds_since(clk::time_point t0) {
  return std::chrono::duration<double>(clk::now() - t0).count();
}

// ------------------------------------------------------------------ profiler
// When enabled, each kernel class launched by the solver's host loop is bracketed by CUDA
// events on the launching stream; elapsed times are folded in at the loop's sync points,
// together with the algorithmic bytes that the class must move.
struct ProfEntry {
  char name[32];
  int64_t launches = 0;
  double ms = 0.0, bytes = 0.0;
};
struct Pending {
  int id;
  cudaEvent_t a, b;
  double bytes;
  bool owned = false;  // events belong to a captured graph: not returned to the pool
};
// While a stream capture is being recorded on this thread, profiler scopes record their
// events as nodes of the graph (external event records) into this list instead of the
// pending list; every launch of the graph then re-queues them.
extern thread_local std::vector<Pending>* g_prof_capture;
extern std::mutex g_prof_mu;
extern bool g_prof_on;
extern std::vector<ProfEntry> g_prof;
extern std::vector<Pending> g_pending;
extern std::vector<cudaEvent_t> g_pool;

inline int prof_id(const char* name) {
  for (size_t i = 0; i < g_prof.size(); ++i)
    if (strncmp(g_prof[i].name, name, sizeof(g_prof[i].name)) == 0) return (int)i;
  ProfEntry e;
  strncpy(e.name, name, sizeof(e.name) - 1);
  e.name[sizeof(e.name) - 1] = 0;
  g_prof.push_back(e);
  return (int)g_prof.size() - 1;
}

inline cudaEvent_t pool_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Fold completed event pairs into the table (call after a stream synchronisation).
inline void prof_flush() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  size_t keep = 0;
  for (size_t i = 0; i < g_pending.size(); ++i) {
    Pending& p = g_pending[i];
    float ms = 0.f;
    if (cudaEventQuery(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_prof[p.id].launches += 1;
      g_prof[p.id].ms += ms;
      g_prof[p.id].bytes += p.bytes;
      if (!p.owned) {
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
      }
    } else {
      g_pending[keep++] = p;
    }
  }
  g_pending.resize(keep);
  cudaGetLastError();
}

// Count an event (no timing) in the table, when profiling is on.
inline void prof_count(const char* name) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof[prof_id(name)].launches += 1;
}

struct ProfScope {
  bool on;
  int id = -1;
  cudaEvent_t a = nullptr;
  double bytes;
  cudaStream_t s;
  ProfScope(const char* name, double b, cudaStream_t st) : on(g_prof_on), bytes(b), s(st) {
    if (!on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    id = prof_id(name);
    if (g_prof_capture) {
      cudaEventCreate(&a);
      cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
    } else {
      a = pool_event();
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (!on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t b = nullptr;
    if (g_prof_capture) {
      cudaEventCreate(&b);
      cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
      g_prof_capture->push_back(Pending{id, a, b, bytes, true});
    } else {
      b = pool_event();
      cudaEventRecord(b, s);
      g_pending.push_back(Pending{id, a, b, bytes});
    }
  }
};

#define SVT_CAT2(a, b) a##b
#define SVT_CAT(a, b) SVT_CAT2(a, b)
#define SVT_PROF(name, bytes, stream) ProfScope SVT_CAT(svt_prof_, __LINE__)(name, (double)(bytes), stream)

// Algorithmic bytes (what the method must move once) of the main kernel classes.
inline double spmm_bytes(int64_t nnz, int64_t rows, int64_t cols, int w, int sv) {
  return (double)nnz * (sv + 4) + 4.0 * (rows + 1) + (double)sv * ((double)cols * w + (double)rows * w);
}
inline double update_bytes(int64_t nnz, int64_t m, int64_t n, int k, int sv) {
  return (double)nnz * (4 + 3 * sv) + 4.0 * (m + 1) + (double)sv * k * (double)(m + n);
}
// the fused update: indices, A, Y read and written, U[:, :r] and W[:, :k] once, B^T written
inline double recycle_bytes(int64_t nnz, int64_t m, int64_t n, int k, int r, int sv) {
  return (double)nnz * (4 + 3 * sv) + 4.0 * (n + 1) +
         (double)sv * ((double)m * r + (double)n * k + (double)n * r);
}
inline double gemm_bytes(int64_t M, int p, int q, int sv, bool reads_c) {
  return (double)sv * (double)M * (p + q + (reads_c ? q : 0));
}

constexpr double kExhaustedRel = 1e-7;
constexpr uint32_t kPowerSeedIter = 0xFFFFFFFFu;
// Ogita-Aishima steps after the binary32 Jacobi: each squares the first-order coupling
// of a pair.  The Jacobi's rounding is relative to the largest eigenvalue, so the coupling
// it leaves is about 1e-7 for the large eigenvalues but up to 1e-2 for small ones a short
// distance apart: one step suffices for binary32 results, three reach binary64 (the
// acceptance test then adds steps where they are still needed).
template <typename T>
constexpr int refine_steps() { return sizeof(T) == 8 ? 3 : 1; }
// From the near-diagonal start of a recycled basis (couplings below 0.02 of their gaps)
// the error falls as 1e-4, 1e-8, 1e-16: three steps for binary32 results, four for binary64.
template <typename T>
constexpr int near_diagonal_steps() { return sizeof(T) == 8 ? 4 : 3; }
// Acceptance of that start: every off-diagonal entry of X^T G X below this fraction of
// the largest eigenvalue.  Clusters whose eigenvalues move next to another cluster's
// after diagonalisation stall well above it (1.6e-5 in a 40 x 40 example), converged
// runs end near 1e-10 (three steps) and 1e-15 (four).
template <typename T>
constexpr double near_diagonal_tol() { return sizeof(T) == 8 ? 1e-12 : 1e-8; }

struct Params {
  int64_t m, n;
  int r_cap, t_eff, dt, np, power_steps, recycle, stop;
  double beta, eps_thr0;
  uint64_t seed;
};

inline svt_status make_params(int64_t m, int64_t n, const svt_options* o, Params* P) {
  if (!o) return fail(SVT_ERR_ARG, "null options");
  if (o->dt <= 0 || o->n_power < 0 || !(o->beta > 0.0 && o->beta < 1.0) || o->power_steps < 1)
    return fail(SVT_ERR_ARG, "options: need dt > 0, n_power >= 0, 0 < beta < 1, power_steps >= 1");
  if (o->precision != SVT_FP64 && o->precision != SVT_MIXED_FP32)
    return fail(SVT_ERR_ARG, "options: unknown precision %d", o->precision);
  if (o->recycle < SVT_RECYCLE_ALL || o->recycle > SVT_RECYCLE_NONE)
    return fail(SVT_ERR_ARG, "options: unknown recycle mode %d", o->recycle);
  if (o->stop != SVT_STOP_RESIDUAL && o->stop != SVT_STOP_MAE)
    return fail(SVT_ERR_ARG, "options: unknown stop rule %d", o->stop);
  const int64_t mn = std::min(m, n);
  int64_t cap = o->r_max > 0 ? std::min<int64_t>(mn, o->r_max) : mn;
  if (cap > 1024)
    return fail(SVT_ERR_UNSUPPORTED, "rank cap min(m, n, r_max) = %lld exceeds 1024; set r_max",
                (long long)cap);
  int64_t t = o->t > 0 ? o->t : (int64_t)std::floor(0.05 * (double)mn);
  if (t < 1) t = 1;
  P->m = m; P->n = n; P->r_cap = (int)cap; P->t_eff = (int)std::min<int64_t>(t, 1 << 20);
  P->dt = o->dt; P->np = o->n_power; P->power_steps = o->power_steps; P->recycle = o->recycle;
  P->stop = o->stop;
  P->beta = o->beta; P->eps_thr0 = o->eps_thr0; P->seed = o->seed;
  return SVT_OK;
}

inline int64_t ld_of(int64_t cols) { return round_up(cols > 0 ? cols : 1, 4); }

namespace {
// out (r x kp, ld kp) = Ub[:, :k] diag(coef), with zero columns k .. kp-1
template <typename T>
__global__ void k_scale_cols(int r, int k, int kp, const double* __restrict__ Ub, int64_t ldu,
                             const double* __restrict__ coef, double* __restrict__ out) {
  const int64_t total = (int64_t)r * kp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / kp), j = (int)(t % kp);
    out[t] = j < k ? Ub[(int64_t)i * ldu + j] * coef[j] : 0.0;
  }
}

// dst (rows x ld, binary64) = src[:, :k] diag(scale) and zero columns k .. ld-1
template <typename T>
__global__ void k_export_scaled(int64_t rows, int k, int ld, const T* __restrict__ src, int64_t lds,
                                const double* __restrict__ scale, double* __restrict__ dst) {
  const int64_t total = rows * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ld;
    const int j = (int)(t - i * ld);
    dst[t] = j < k ? (double)src[i * lds + j] * scale[j] : 0.0;
  }
}

// C = (3 I - G) / 2 (r x r): one Newton-Schulz step towards the orthonormal polar factor,
// Q C, for a basis whose Gram matrix Q^T Q = G is close to the identity.
__global__ void k_ns_coeff(int r, const double* __restrict__ G, double* __restrict__ C) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)r * r;
       t += (int64_t)gridDim.x * blockDim.x)
    C[t] = (t / r == t % r ? 1.5 : 0.0) - 0.5 * G[t];
}

__global__ void k_normalize(int64_t n, const double* __restrict__ w, const double* __restrict__ ss,
                            double* __restrict__ v) {
  const double inv = 1.0 / sqrt(ss[0]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * inv;
}

}  // namespace

// Device buffers of one solve (or one R4SVD call).
// An executable graph of the recycled-basis eigen phase of R4SVD (see r4svd_run), with
// what its recorded launches depend on.
struct EigGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<Pending> scopes;  // profiler events recorded inside the graph
  int64_t launches = 0;         // kernels per launch of the graph
  int r = -1;
  const void *Q = nullptr, *Bt = nullptr, *Unew = nullptr;
  bool prof = false;
  uint64_t used = 0;
  EigGraph() = default;
  EigGraph(const EigGraph&) = delete;
  EigGraph& operator=(const EigGraph&) = delete;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);  // an in-flight graph is freed on completion
    exec = nullptr;
    for (auto& e : scopes) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    scopes.clear();
    r = -1;
  }
  ~EigGraph() { reset(); }
};

template <typename T>
struct Work {
  Params P;
  const svt_pattern* pat = nullptr;
  cudaStream_t s = nullptr;
  int wmax = 1;
  int64_t ldq = 0, ldb = 0, ldw = 0, ldk = 0;
  T *Qa = nullptr, *Qb = nullptr;   // m x ldq (basis / recycled U, ping-pong)
  T *Bt = nullptr;                  // n x ldb
  T *Om = nullptr, *Z = nullptr;    // n x ldw
  T *X = nullptr, *X2 = nullptr;    // m x ldw
  T *Wk = nullptr;                  // n x ldk (V_K scaled by sigma - tau, or V)
  T *y_csc = nullptr;               // nnz
  double *G = nullptr, *Ub = nullptr, *lam = nullptr, *Gs = nullptr;
  double *Gx = nullptr, *Rm = nullptr, *Rinv = nullptr, *cwork = nullptr, *Tsm = nullptr;
  double *coef = nullptr, *part = nullptr, *eigw = nullptr, *dsc = nullptr, *colss = nullptr;
  double *pv = nullptr, *pu = nullptr, *pw = nullptr;  // power-iteration vectors
  // status words: [0] FLAG bits, [1] cluster-start status, [2] Jacobi sweeps, [3] check
  // status, [4] sticky FLAG_TC_TIMEOUT / FLAG_GRID_TIMEOUT (tensor-core lift, grid Jacobi)
  unsigned* flags = nullptr;
  float* tcb = nullptr;             // split U_B^T for the tensor-core lift (binary32 path)
  void* spmm_scr = nullptr;         // partial rows of the entry-chunked SpMM
  // Set by a caller whose sampled update already formed Bt = Y^T Q for the s recycled
  // columns (the fused update); r4svd_run then skips that product and clears it.
  bool bt_ready = false;
  // Non-null: this CSR copy of Y is stale (the fused update wrote only the CSC copy);
  // r4svd_run refreshes it from y_csc before its first CSR product and clears it.
  T* y_csr_stale = nullptr;
  // Set when both full copies of Y are stale (the update wrote the sparse rest and the
  // dense core instead): r4svd_run calls it before its first product with Y and clears it.
  std::function<svt_status()> refresh_y;
  // Recycled iterations replay the eigen phase as a captured graph (two graphs: the basis
  // and B^T buffers alternate); host_pin is page-locked host memory of pin_doubles()
  // doubles for the graph's copies.  Off unless the caller provides host_pin.
  double* host_pin = nullptr;
  bool graph_broken = false;
  // the eigen-phase graph of the next R4SVD call was launched ahead by the caller
  bool graph_inflight = false;
  // set by the caller: re-orthonormalise the recycled basis at the start of the next
  // R4SVD call (binary32; see reorth_basis)
  bool reorth_due = false;
  uint64_t graph_clock = 0;
  EigGraph eg[2];
  // graphs are recorded on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured) and launched on the caller's
  struct OwnedStream {
    cudaStream_t s = nullptr;
    ~OwnedStream() { if (s) cudaStreamDestroy(s); }
  } cap;
  // [0, 2 r_cap + kFlagWords) for the graph's copies, 8 doubles for the caller, then r_cap
  // doubles staging the shrinkage coefficients of scaled_right
  static size_t pin_doubles(int r_cap) { return 3 * (size_t)r_cap + kFlagWords + 8; }
  double* pin_tail() const { return host_pin + 2 * (size_t)P.r_cap + kFlagWords; }
  double* pin_coef() const { return host_pin + 2 * (size_t)P.r_cap + kFlagWords + 8; }

  void layout(Arena& a) {
    const int64_t m = P.m, n = P.n, z = pat->nnz;
    const int rc = P.r_cap;
    wmax = std::max(std::min(P.t_eff, rc), std::min(P.dt, rc));
    ldq = ld_of(rc); ldb = ld_of(rc); ldw = ld_of(wmax); ldk = ld_of(rc);
    Qa = a.take<T>(m * ldq); Qb = a.take<T>(m * ldq);
    Bt = a.take<T>(n * ldb);
    Om = a.take<T>(n * ldw); Z = a.take<T>(n * ldw);
    X = a.take<T>(m * ldw); X2 = a.take<T>(m * ldw);
    Wk = a.take<T>(n * ldk);
    y_csc = a.take<T>(z);
    G = a.take<double>((int64_t)rc * rc);
    Ub = a.take<double>((int64_t)rc * rc);
    lam = a.take<double>(rc);
    Gs = a.take<double>((int64_t)rc * wmax);
    Gx = a.take<double>((int64_t)wmax * wmax);
    Rm = a.take<double>((int64_t)wmax * wmax);
    Rinv = a.take<double>((int64_t)wmax * wmax);
    cwork = a.take<double>((int64_t)wmax * wmax);
    Tsm = a.take<double>((int64_t)rc * ld_of(rc));
    coef = a.take<double>(rc);
    size_t pe = reduce_scratch();
    pe = std::max(pe, gemm_tn_scratch(m, rc, wmax));
    pe = std::max(pe, gemm_tn_scratch(m, wmax, wmax));
    pe = std::max(pe, gemm_tn_scratch(n, rc, rc));
    pe = std::max(pe, colsumsq_scratch(std::max(m, n), std::max(wmax, rc)));
    part = a.take<double>(pe);
    eigw = a.take<double>(eig_scratch(rc));
    dsc = a.take<double>(16);
    colss = a.take<double>(std::max(wmax, rc));
    pv = a.take<double>(n); pw = a.take<double>(n); pu = a.take<double>(m);
    flags = a.take<unsigned>(kFlagWords);
    if (sizeof(T) == 4) tcb = a.take<float>(lift_tc_scratch_floats());
    const size_t sb = std::max(spmm_scratch_bytes(z, std::max(wmax, rc), (int)sizeof(T)),
                               spmm_scratch_bytes(z, 1, 8));
    spmm_scr = a.take<char>(sb);
  }
};

template <typename T>
svt_status read_flags(Work<T>& W, unsigned* out) {
  SVT_CUDA(cudaMemcpyAsync(out, W.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, W.s));
  SVT_CUDA(cudaStreamSynchronize(W.s));
  return SVT_OK;
}

// Sum of squares of columns [c0, c0+w) of an M x w block, summed on the host in column order.
template <typename T>
svt_status block_sumsq(Work<T>& W, int64_t M, int w, const T* X, int64_t ldx, double* out,
                       double* maxcol = nullptr) {
  std::vector<double> h(w > 0 ? w : 1);
  if (w <= 0) { *out = 0.0; if (maxcol) *maxcol = 0.0; return SVT_OK; }
  SVT_TRY(colsumsq<T>(M, w, X, ldx, W.colss, W.part, W.s));
  SVT_CUDA(cudaMemcpyAsync(h.data(), W.colss, w * sizeof(double), cudaMemcpyDeviceToHost, W.s));
  SVT_CUDA(cudaStreamSynchronize(W.s));
  double s = 0.0, mx = 0.0;
  for (int c = 0; c < w; ++c) { s += h[c]; mx = std::max(mx, h[c]); }
  *out = s;
  if (maxcol) *maxcol = std::sqrt(mx);
  return SVT_OK;
}

struct R4Out {
  int r = 0, blocks = 0;
  bool exhausted = false;
  double eps = 0.0, normB = 0.0;
  std::vector<double> sigma;  // descending, r entries
};

// Algorithm 3 (Algorithm 2 when s == 0).  Q holds the recycled basis in columns [0, s);
// new blocks are appended in place.  On return U = Q U_B is written to Unew (m x ldq),
// Bt (n x r) = Y^T Q, W.Ub = U_B, sigma on the host.
// U = Q U_B (m x r times r x r, Algorithm 3): on the tensor cores in the binary32 path
template <typename T>
svt_status lift_basis(Work<T>& W, const T* Q, int r, T* Unew) {
  if constexpr (sizeof(T) == 4) {
    if (W.tcb && lift_tc_fits(W.P.m, r, r, Q, W.ldq, Unew, W.ldq))
      return lift_tc(W.P.m, r, r, Q, W.ldq, W.Ub, r, Unew, W.ldq, W.tcb, W.flags + 4, W.s);
  }
  return gemm_nn<T, T>(W.P.m, r, r, 1.0, Q, W.ldq, W.Ub, r, 0.0, nullptr, 0, Unew, W.ldq, W.s);
}

// C (M x r, ldc) = A (M x r, lda) B (r x r binary64, ld r): on the tensor cores in the
// binary32 path when the shape allows, else the SIMT kernel.
template <typename T>
svt_status times_small(Work<T>& W, int64_t M, int r, const T* A, int64_t lda, const double* B, T* C,
                       int64_t ldc) {
  if constexpr (sizeof(T) == 4) {
    if (W.tcb && lift_tc_fits(M, r, r, A, lda, C, ldc))
      return lift_tc(M, r, r, A, lda, B, r, C, ldc, W.tcb, W.flags + 4, W.s);
  }
  return gemm_nn<T, T>(M, r, r, 1.0, A, lda, B, r, 0.0, nullptr, 0, C, ldc, W.s);
}

// Re-orthonormalisation of a binary32 basis by one Newton-Schulz step: Q <- Q C with
// C = (3 I - Q^T Q) / 2 (the Gram matrix in binary64 accuracy) and, when Bt is given,
// B^T <- B^T C, which keeps B^T = Y^T Q.  In exact arithmetic Q is orthonormal and C = I; in
// binary32 each lift U = Q U_B moves Q^T Q away from the identity a little, while the
// energy test of R4SVD and the SVD of B = Q^T Y assume it is the identity.  The step takes
// max |Q^T Q - I| from e to about 1.5 e^2.  Qscr (m x ldq) and W.Wk serve as scratch.
template <typename T>
svt_status reorth_basis(Work<T>& W, T* Q, int r, T* Qscr, T* Bt, int64_t ldb) {
  if (r <= 0) return SVT_OK;
  const int64_t m = W.P.m, n = W.P.n;
  const int sv = (int)sizeof(T);
  cudaStream_t st = W.s;
  SVT_PROF("reorth", gemm_bytes(m, r, 0, sv, false) + 2 * gemm_bytes(m, r, r, sv, false) +
                         (Bt ? 2 * gemm_bytes(n, r, r, sv, false) : 0.0), st);
  SVT_TRY((gemm_tn<T, T>(m, r, r, Q, W.ldq, Q, W.ldq, W.G, r, W.part, st)));
  k_ns_coeff<<<(int)std::min<int64_t>(ceil_div((int64_t)r * r, 256), 256), 256, 0, st>>>(r, W.G, W.Tsm);
  SVT_LAUNCH_CHECK();
  SVT_TRY(times_small<T>(W, m, r, Q, W.ldq, W.Tsm, Qscr, W.ldq));
  SVT_CUDA(cudaMemcpy2DAsync(Q, W.ldq * sizeof(T), Qscr, W.ldq * sizeof(T), r * sizeof(T), m,
                             cudaMemcpyDeviceToDevice, st));
  if (Bt) {
    SVT_TRY(times_small<T>(W, n, r, Bt, ldb, W.Tsm, W.Wk, W.ldk));
    SVT_CUDA(cudaMemcpy2DAsync(Bt, ldb * sizeof(T), W.Wk, W.ldk * sizeof(T), r * sizeof(T), n,
                               cudaMemcpyDeviceToDevice, st));
  }
  return SVT_OK;
}

enum class EigFrom {
  kClusters,  // near-diagonal cluster start, checked refinement, second pass, else Jacobi
  kRejected,  // the checked refinement from the cluster start was refused: second pass
  kJacobi,    // full binary32 Jacobi, then refinement
};

// svt(B): eigen-decomposition of G = B B^T = (B^T)^T B^T (formed here when gram is set),
// Reads the acceptance status of the last checked refinement (flags[3]).
template <typename T>
svt_status eig_status(Work<T>& W, int* status) {
  SVT_CUDA(cudaMemcpyAsync(status, W.flags + 3, sizeof(int), cudaMemcpyDeviceToHost, W.s));
  SVT_CUDA(cudaStreamSynchronize(W.s));
  return SVT_OK;
}

// Eigenpairs of G (r x r, in W.G) from the full binary32 Jacobi, refined in binary64 until
// the acceptance test passes.  The Jacobi's rounding is relative to the largest
// eigenvalue, so the first-order coupling it leaves between two small eigenvalues a short
// distance apart can be close to the refinement's limit of 0.1: such pairs need more
// than the steps that suffice for the large ones, and are given up to four more.  Pairs
// coupled beyond that limit (eigenvalues that agree to about 4e-7 of the largest) are
// clusters for the refinement; they are diagonalised in the refined basis by the cluster
// pass, and refined again.
template <typename T>
svt_status eig_from_jacobi(Work<T>& W, int r) {
  cudaStream_t st = W.s;
  int* fl3 = reinterpret_cast<int*>(W.flags + 3);
  {
    SVT_PROF("eig_jacobi32", 8.0 * r * r, st);
    SVT_TRY(eig_start(r, W.G, r, W.eigw, st, reinterpret_cast<int*>(W.flags + 2), W.flags + 4));
  }
  int alt = 0;
  auto refine = [&](int steps) -> svt_status {
    SVT_PROF("eig_refine64", 8.0 * 3 * r * r, st);
    SVT_TRY(eig_refine(r, W.G, r, W.lam, W.Ub, r, W.eigw, steps, st, fl3, near_diagonal_tol<T>(), alt));
    alt = eig_x_alt(alt, steps);
    return SVT_OK;
  };
  int status = 0;
  SVT_TRY(refine(refine_steps<T>()));
  SVT_TRY(eig_status(W, &status));
  for (int round = 0; round < 2 && status != 0; ++round) {
    prof_count("eig_jacobi_more_steps");
    SVT_TRY(refine(2));
    SVT_TRY(eig_status(W, &status));
  }
  if (status != 0) {
    prof_count("eig_jacobi_clusters");
    {
      SVT_PROF("eig_refine64", 8.0 * 3 * r * r, st);
      SVT_TRY(eig_refine_clusters_again(r, W.G, r, W.lam, W.Ub, r, W.eigw, alt, 2, st, fl3,
                                        near_diagonal_tol<T>()));
    }
    alt = eig_x_alt(0, 2);
    SVT_TRY(eig_status(W, &status));
    for (int round = 0; round < 2 && status != 0; ++round) {
      SVT_TRY(refine(2));
      SVT_TRY(eig_status(W, &status));
    }
    if (status != 0) prof_count("eig_jacobi_unresolved");
  }
  return SVT_OK;
}

// U = Q U_B and sigma on the host.  A purely recycled basis (no new block) leaves G
// nearly diagonal: the binary64 refinement starts from the identity with the coupled
// clusters diagonalised, and the result is accepted only if no coupled pair was left;
// otherwise (or if a cluster is too large) it starts from the full binary32 Jacobi.
template <typename T>
svt_status eig_finish(Work<T>& W, T* Q, int r, T* Unew, EigFrom from, bool gram, R4Out* o) {
  const int64_t m = W.P.m, n = W.P.n;
  const int sv = (int)sizeof(T);
  cudaStream_t st = W.s;
  if (gram) {
    SVT_PROF("gram_B", gemm_bytes(n, r, 0, sv, false), st);
    SVT_TRY((gemm_tn<T, T>(n, r, r, W.Bt, W.ldb, W.Bt, W.ldb, W.G, r, W.part, st)));
  }
  bool near_diagonal = false;
  int status = 1;
  if (from == EigFrom::kClusters) {
    {
      SVT_PROF("eig_cluster", 8.0 * r * r, st);
      SVT_TRY(eig_start_clusters(r, W.G, r, W.eigw, st, reinterpret_cast<int*>(W.flags + 3)));
    }
    SVT_CUDA(cudaMemcpyAsync(&status, W.flags + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaStreamSynchronize(st));
    if (status != 0) prof_count("eig_start_oversize");
    if (status == 0) {
      {
        SVT_PROF("eig_refine64", 8.0 * 3 * r * r, st);
        SVT_TRY(eig_refine(r, W.G, r, W.lam, W.Ub, r, W.eigw, near_diagonal_steps<T>(), st,
                           reinterpret_cast<int*>(W.flags + 3), near_diagonal_tol<T>()));
      }
      SVT_CUDA(cudaMemcpyAsync(&status, W.flags + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
      SVT_CUDA(cudaStreamSynchronize(st));
      if (status != 0) from = EigFrom::kRejected;
      else near_diagonal = true;
    }
  }
  if (from == EigFrom::kRejected) {
    // an unresolved pair: resolve its cluster in the rotated basis, once
    prof_count("eig_start_rejected");
    {
      SVT_PROF("eig_refine64", 8.0 * 3 * r * r, st);
      SVT_TRY(eig_refine_clusters_again(r, W.G, r, W.lam, W.Ub, r, W.eigw,
                                        eig_x_alt(0, near_diagonal_steps<T>()), 2, st,
                                        reinterpret_cast<int*>(W.flags + 3), near_diagonal_tol<T>()));
    }
    SVT_CUDA(cudaMemcpyAsync(&status, W.flags + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaStreamSynchronize(st));
    if (status != 0) prof_count("eig_start_rejected_twice");
    near_diagonal = status == 0;  // else redo from the full Jacobi
  }
  if (!near_diagonal) SVT_TRY(eig_from_jacobi<T>(W, r));
  std::vector<double> lam(r);
  SVT_CUDA(cudaMemcpyAsync(lam.data(), W.lam, r * sizeof(double), cudaMemcpyDeviceToHost, st));
  // U = Q U_B (all r columns are recycled)
  {
    SVT_PROF("lift_U", gemm_bytes(m, r, r, sv, false), st);
    SVT_TRY(lift_basis<T>(W, Q, r, Unew));
  }
  unsigned tc_status = 0;
  SVT_CUDA(cudaMemcpyAsync(&tc_status, W.flags + 4, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  SVT_CUDA(cudaStreamSynchronize(st));
  if (tc_status & (FLAG_TC_TIMEOUT | FLAG_GRID_TIMEOUT))
    return fail(SVT_ERR_CUDA, "a bounded wait ran out (%s)",
                (tc_status & FLAG_TC_TIMEOUT) ? "tensor-core kernel" : "grid Jacobi");
  prof_flush();
  if (g_prof_on && !near_diagonal) {  // sweep count of the binary32 Jacobi stage (pseudo-entry)
    int sweeps = 0;
    if (cudaMemcpy(&sweeps, W.flags + 2, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(g_prof_mu);
      const int id = prof_id("jacobi_sweeps");
      g_prof[id].launches += 1;
      g_prof[id].bytes += sweeps;
    }
  }
  o->sigma.assign(r, 0.0);
  for (int j = 0; j < r; ++j) {
    if (!std::isfinite(lam[j])) return fail(SVT_ERR_NUMERIC, "R4SVD: non-finite eigenvalue");
    o->sigma[j] = std::sqrt(std::max(lam[j], 0.0));
  }
  return SVT_OK;
}

// The eigen phase of a purely recycled basis, enqueued without host synchronisation so
// that it can be captured: G = B B^T (its diagonal, ||B||_F^2 by columns, copied to
// host_pin[0, r)), the near-diagonal cluster start (identity if a cluster is too large, status in flags[1]),
// the checked binary64 refinement (status in flags[3]), the status words and the
// eigenvalues copied to host_pin, and U = Q U_B.
template <typename T>
svt_status eig_phase_enqueue(Work<T>& W, T* Q, int r, T* Unew) {
  const int64_t m = W.P.m, n = W.P.n;
  const int sv = (int)sizeof(T);
  cudaStream_t st = W.s;
  {
    SVT_PROF("gram_B", gemm_bytes(n, r, 0, sv, false), st);
    SVT_TRY((gemm_tn<T, T>(n, r, r, W.Bt, W.ldb, W.Bt, W.ldb, W.G, r, W.part, st)));
  }
  // ||B||_F^2 by columns is the diagonal of G: one strided copy of G_cc to host_pin[0, r)
  SVT_CUDA(cudaMemcpy2DAsync(W.host_pin, sizeof(double), W.G, (size_t)(r + 1) * sizeof(double),
                             sizeof(double), (size_t)r, cudaMemcpyDeviceToHost, st));
  {
    SVT_PROF("eig_cluster", 8.0 * r * r, st);
    SVT_TRY(eig_start_clusters(r, W.G, r, W.eigw, st, reinterpret_cast<int*>(W.flags + 1), true));
  }
  {
    SVT_PROF("eig_refine64", 8.0 * 3 * r * r, st);
    SVT_TRY(eig_refine(r, W.G, r, W.lam, W.Ub, r, W.eigw, near_diagonal_steps<T>(), st,
                       reinterpret_cast<int*>(W.flags + 3), near_diagonal_tol<T>()));
  }
  SVT_CUDA(cudaMemcpyAsync(W.host_pin + r, W.lam, r * sizeof(double), cudaMemcpyDeviceToHost, st));
  SVT_CUDA(cudaMemcpyAsync(W.host_pin + 2 * r, W.flags, kFlagWords * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  {
    SVT_PROF("lift_U", gemm_bytes(m, r, r, sv, false), st);
    SVT_TRY(lift_basis<T>(W, Q, r, Unew));
  }
  return SVT_OK;
}

// Launches eig_phase_enqueue as a graph, capturing it first when no cached graph matches
// (r, the buffers, the profiler state).  *ran = false when capture is unavailable; the
// caller then runs the phase eagerly.
template <typename T>
svt_status eig_phase_graph(Work<T>& W, T* Q, int r, T* Unew, bool* ran) {
  *ran = false;
  if (W.graph_broken || !W.host_pin) return SVT_OK;
  cudaStream_t st = W.s;
  EigGraph* g = nullptr;
  for (auto& c : W.eg)
    if (c.exec && c.r == r && c.Q == Q && c.Bt == W.Bt && c.Unew == Unew && c.prof == g_prof_on) g = &c;
  if (!g) {
    g = W.eg[0].used <= W.eg[1].used ? &W.eg[0] : &W.eg[1];
    g->reset();
    SVT_TRY(eig_prepare());
    if (sizeof(T) == 4) SVT_TRY(lift_tc_prepare());
    if (!W.cap.s) SVT_CUDA(cudaStreamCreateWithFlags(&W.cap.s, cudaStreamNonBlocking));
    std::vector<Pending> scopes;
    const int64_t l0 = launches_so_far();
    SVT_CUDA(cudaStreamBeginCapture(W.cap.s, cudaStreamCaptureModeThreadLocal));
    g_prof_capture = &scopes;
    W.s = W.cap.s;
    const svt_status es = eig_phase_enqueue<T>(W, Q, r, Unew);
    W.s = st;
    g_prof_capture = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(W.cap.s, &graph);
    const int64_t recorded = launches_so_far() - l0;
    count_launches(-recorded);  // counted when the graph runs
    cudaError_t ie = cudaErrorUnknown;
    if (es == SVT_OK && ce == cudaSuccess && graph) ie = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {  // leave graphs off for this solve and run eagerly
      for (auto& e : scopes) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
      g->exec = nullptr;
      cudaGetLastError();
      W.graph_broken = true;
      prof_count("eig_graph_unavailable");
      return SVT_OK;
    }
    g->scopes = std::move(scopes);
    g->launches = recorded;
    g->r = r; g->Q = Q; g->Bt = W.Bt; g->Unew = Unew; g->prof = g_prof_on;
  }
  g->used = ++W.graph_clock;
  SVT_CUDA(cudaGraphLaunch(g->exec, st));
  count_launches(g->launches);
  if (g->prof) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const auto& e : g->scopes) g_pending.push_back(e);
  }
  *ran = true;
  return SVT_OK;
}

// Algorithm 3 (Algorithm 2 when s == 0).  Q holds the recycled basis in columns [0, s);
// new blocks are appended in place.  On return U = Q U_B is written to Unew (m x ldq),
// Bt (n x r) = Y^T Q, W.Ub = U_B, sigma on the host.
template <typename T>
svt_status r4svd_run(Work<T>& W, const T* y_csr, const T* y_csc, T* Q, int s, double normY2,
                     double eps_thr, uint32_t iter, T* Unew, R4Out* o) {
  const Params& P = W.P;
  const svt_pattern* p = W.pat;
  const int64_t m = P.m, n = P.n;
  cudaStream_t st = W.s;
  int r = s;
  double normB = 0.0;
  const int sv = (int)sizeof(T);
  const int64_t z = p->nnz;
  auto eps_of = [&](double nb) { return normY2 > 0.0 ? (normY2 - nb) / normY2 : 0.0; };
  // binary32: a recycled basis is re-orthonormalised when the caller asks (periodically)
  if (sizeof(T) == 4 && W.reorth_due && s > 0 && !W.graph_inflight)
    SVT_TRY(reorth_basis<T>(W, Q, s, Unew, W.bt_ready ? W.Bt : nullptr, W.ldb));
  W.reorth_due = false;
  // A recycled basis whose B^T the fused update already formed usually needs no new block:
  // run the whole eigen phase as one graph and check that assumption afterwards.
  bool have_normB = false;
  if (s > 0 && W.bt_ready) {
    bool ran = W.graph_inflight;  // launched ahead with these buffers by the caller
    W.graph_inflight = false;
    if (!ran) SVT_TRY(eig_phase_graph<T>(W, Q, s, Unew, &ran));
    if (ran) {
      have_normB = true;
      SVT_CUDA(cudaStreamSynchronize(st));  // (profiler events are folded in later, off this path)
      const double* hp = W.host_pin;
      for (int c = 0; c < s; ++c) normB += hp[c];
      const double eps0 = eps_of(normB);
      if (!(eps0 > eps_thr && s < P.r_cap)) {  // no new block: the graph's results stand
        unsigned fl[kFlagWords];
        memcpy(fl, hp + 2 * s, sizeof(fl));
        if (fl[4] & (FLAG_TC_TIMEOUT | FLAG_GRID_TIMEOUT))
          return fail(SVT_ERR_CUDA, "a bounded wait ran out (%s)",
                      (fl[4] & FLAG_TC_TIMEOUT) ? "tensor-core kernel" : "grid Jacobi");
        o->r = s; o->blocks = 0; o->exhausted = false; o->eps = eps0; o->normB = normB;
        o->sigma.assign(s, 0.0);
        if (fl[1] == 0 && fl[3] == 0) {
          for (int j = 0; j < s; ++j) {
            const double lj = hp[s + j];
            if (!std::isfinite(lj)) return fail(SVT_ERR_NUMERIC, "R4SVD: non-finite eigenvalue");
            o->sigma[j] = std::sqrt(std::max(lj, 0.0));
          }
          return SVT_OK;
        }
        if (fl[1] != 0) prof_count("eig_start_oversize");
        // the near-diagonal start was refused: finish eagerly from G (already formed)
        return eig_finish<T>(W, Q, s, Unew, fl[1] != 0 ? EigFrom::kJacobi : EigFrom::kRejected,
                             false, o);
      }
      // the basis must grow: fall through with ||B||^2 known (G and U are redone below)
    }
  }
  if (s > 0 && !have_normB) {
    if (!W.bt_ready) {
      SVT_PROF("spmm_csc_recycled", spmm_bytes(z, n, m, s, sv), st);
      SVT_TRY((launch_spmm_rows<T, T>(n, p->col_ptr, p->row_idx, y_csc, Q, W.ldq, s, W.Bt, W.ldb, W.spmm_scr, z, st, p->chunk_row_csc)));
    }
    SVT_TRY(block_sumsq<T>(W, n, s, W.Bt, W.ldb, &normB));
  }
  W.bt_ready = false;
  double eps = eps_of(normB);
  bool first = (s == 0);
  int blocks = 0;
  bool exhausted = false;
  while ((first || eps > eps_thr) && r < P.r_cap) {
    const int w = first ? std::min(P.t_eff, P.r_cap) : std::min(P.dt, P.r_cap - r);
    {
      SVT_PROF("gaussian", (double)sv * n * w, st);
      SVT_TRY(launch_gaussian<T>(P.seed, iter, (uint32_t)blocks, n, w, W.Om, W.ldw, st));
    }
    ++blocks;
    if (W.refresh_y) {
      SVT_PROF("assemble_y", (double)z * (4 + 2 * sv) + (double)z * (4 + 2 * sv), st);
      SVT_TRY(W.refresh_y());
      W.refresh_y = nullptr;
    } else if (W.y_csr_stale) {
      SVT_PROF("scatter_csr", (double)z * (4 + 2 * sv), st);
      SVT_TRY(launch_scatter<T>(z, p->perm, y_csc, W.y_csr_stale, st));
      W.y_csr_stale = nullptr;
    }
    {
      SVT_PROF("spmm_csr", spmm_bytes(z, m, n, w, sv), st);
      SVT_TRY((launch_spmm_rows<T, T>(m, p->row_ptr, p->col_idx, y_csr, W.Om, W.ldw, w, W.X, W.ldw, W.spmm_scr, z, st, p->chunk_row_csr)));
    }
    for (int it = 0; it < P.np; ++it) {
      SVT_PROF("spmm_power", spmm_bytes(z, n, m, w, sv) + spmm_bytes(z, m, n, w, sv), st);
      SVT_TRY((launch_spmm_rows<T, T>(n, p->col_ptr, p->row_idx, y_csc, W.X, W.ldw, w, W.Z, W.ldw, W.spmm_scr, z, st, p->chunk_row_csc)));
      SVT_TRY((launch_spmm_rows<T, T>(m, p->row_ptr, p->col_idx, y_csr, W.Z, W.ldw, w, W.X, W.ldw, W.spmm_scr, z, st, p->chunk_row_csr)));
    }
    double ssum = 0.0, scale = 0.0;
    SVT_TRY(block_sumsq<T>(W, m, w, W.X, W.ldw, &ssum, &scale));
    if (r > 0) {
      for (int pass = 0; pass < 2; ++pass) {  // X <- X - Q (Q^T X), twice
        SVT_PROF("orthogonalise", gemm_bytes(m, r, w, sv, false) + gemm_bytes(m, r, w, sv, true), st);
        SVT_TRY((gemm_tn<T, T>(m, r, w, Q, W.ldq, W.X, W.ldw, W.Gs, w, W.part, st)));
        SVT_TRY((gemm_nn<T, T>(m, r, w, -1.0, Q, W.ldq, W.Gs, w, 1.0, W.X, W.ldw, W.X2, W.ldw, st)));
        std::swap(W.X, W.X2);
      }
    }
    // Cholesky-QR, twice: X = Q' R
    SVT_CUDA(cudaMemsetAsync(W.flags, 0, sizeof(unsigned), st));
    {
      SVT_PROF("cholqr", gemm_bytes(m, w, 0, sv, false), st);
      SVT_TRY((gemm_tn<T, T>(m, w, w, W.X, W.ldw, W.X, W.ldw, W.Gx, w, W.part, st)));
      SVT_TRY(chol_inv(w, W.Gx, w, W.Rm, W.Rinv, W.cwork, W.dsc + 0, W.flags, st));
    }
    double dmin = 0.0;
    unsigned fl = 0;
    SVT_CUDA(cudaMemcpyAsync(&dmin, W.dsc + 0, sizeof(double), cudaMemcpyDeviceToHost, st));
    SVT_TRY(read_flags(W, &fl));
    if (scale == 0.0 || (fl & FLAG_CHOLESKY) || !(dmin > kExhaustedRel * scale)) {
      exhausted = true;
      break;
    }
    {
      SVT_PROF("cholqr", gemm_bytes(m, w, w, sv, false) + gemm_bytes(m, w, 0, sv, false), st);
      SVT_TRY((gemm_nn<T, T>(m, w, w, 1.0, W.X, W.ldw, W.Rinv, w, 0.0, nullptr, 0, W.X2, W.ldw, st)));
      SVT_TRY((gemm_tn<T, T>(m, w, w, W.X2, W.ldw, W.X2, W.ldw, W.Gx, w, W.part, st)));
      SVT_TRY(chol_inv(w, W.Gx, w, W.Rm, W.Rinv, W.cwork, W.dsc + 1, W.flags, st));
    }
    SVT_TRY(read_flags(W, &fl));
    if (fl & FLAG_CHOLESKY) return fail(SVT_ERR_NUMERIC, "R4SVD: Cholesky-QR breakdown in block %d", blocks);
    {
      SVT_PROF("cholqr", gemm_bytes(m, w, w, sv, false), st);
      SVT_TRY((gemm_nn<T, T>(m, w, w, 1.0, W.X2, W.ldw, W.Rinv, w, 0.0, nullptr, 0, Q + r, W.ldq, st)));
    }
    // B'^T = Y^T Q'
    {
      SVT_PROF("spmm_csc", spmm_bytes(z, n, m, w, sv), st);
      SVT_TRY((launch_spmm_rows<T, T>(n, p->col_ptr, p->row_idx, y_csc, Q + r, W.ldq, w, W.Bt + r, W.ldb, W.spmm_scr, z, st, p->chunk_row_csc)));
    }
    double nb = 0.0;
    SVT_TRY(block_sumsq<T>(W, n, w, W.Bt + r, W.ldb, &nb));
    normB += nb;
    r += w;
    eps = eps_of(normB);
    first = false;
  }
  o->r = r; o->blocks = blocks; o->exhausted = exhausted; o->eps = eps; o->normB = normB;
  o->sigma.assign(r, 0.0);
  if (r == 0) return SVT_OK;
  return eig_finish<T>(W, Q, r, Unew, s > 0 && blocks == 0 ? EigFrom::kClusters : EigFrom::kJacobi,
                       true, o);
}

// Wk (n x k) = Bt (n x r) * Ub[:, :k] diag(coef).  Columns k .. round_up(k, 4) - 1 of Wk
// are written as exact zeros (zero coefficients times the finite Bt), so the sampled update
// may read them in whole vectors without masking.
template <typename T>
svt_status scaled_right(Work<T>& W, int r, int k, const std::vector<double>& coef) {
  if (k <= 0) return SVT_OK;
  const int kp = (int)round_up(k, 4);
  // page-locked staging when available: the previous iteration's copy has completed (the
  // caller waited for the update that follows it), so the buffer may be refilled
  const double* src = coef.data();
  if (W.host_pin && k <= W.P.r_cap) {
    memcpy(W.pin_coef(), coef.data(), k * sizeof(double));
    src = W.pin_coef();
  }
  SVT_CUDA(cudaMemcpyAsync(W.coef, src, k * sizeof(double), cudaMemcpyHostToDevice, W.s));
  const int64_t total = (int64_t)r * kp;
  k_scale_cols<T><<<(int)std::min<int64_t>(ceil_div(total, 256), 1024), 256, 0, W.s>>>(
      r, k, kp, W.Ub, r, W.coef, W.Tsm);
  SVT_LAUNCH_CHECK();
  SVT_PROF("lift_V", gemm_bytes(W.P.n, r, k, (int)sizeof(T), false), W.s);
  if constexpr (sizeof(T) == 4) {  // the same contraction shape as the lift of U
    if (W.tcb && lift_tc_fits(W.P.n, r, kp, W.Bt, W.ldb, W.Wk, W.ldk))
      return lift_tc(W.P.n, r, kp, W.Bt, W.ldb, W.Tsm, kp, W.Wk, W.ldk, W.tcb, W.flags + 4, W.s);
  }
  SVT_TRY((gemm_nn<T, T>(W.P.n, r, kp, 1.0, W.Bt, W.ldb, W.Tsm, kp, 0.0, nullptr, 0, W.Wk, W.ldk, W.s)));
  return SVT_OK;
}

// Copy the first k columns of a device T matrix into caller memory (double, ld = cap).
// With col_scale (device, k values) column j is multiplied by col_scale[j] in binary64.
template <typename T>
svt_status export_cols(Work<T>& W, int64_t rows, int k, const T* src, int64_t lds, double* dst,
                       int cap, const double* col_scale = nullptr) {
  if (rows <= 0 || cap <= 0) return SVT_OK;
  auto fill = [&](double* d) -> svt_status {
    if (col_scale && k > 0) {
      const int64_t total = rows * cap;
      k_export_scaled<T><<<(int)std::min<int64_t>(ceil_div(total, 256), 4096), 256, 0, W.s>>>(
          rows, k, cap, src, lds, col_scale, d);
      SVT_LAUNCH_CHECK();
      return SVT_OK;
    }
    SVT_CUDA(cudaMemsetAsync(d, 0, rows * cap * sizeof(double), W.s));
    return copy_convert<T, double>(rows, k, src, lds, d, cap, W.s);
  };
  const bool dev = is_device_pointer(dst);
  if (dev) return fill(dst);
  DeviceBlock tmp;
  SVT_TRY(tmp.alloc(rows * cap * sizeof(double), W.s));
  double* d = (double*)tmp.ptr;
  SVT_TRY(fill(d));
  SVT_CUDA(cudaMemcpyAsync(dst, d, rows * cap * sizeof(double), cudaMemcpyDeviceToHost, W.s));
  SVT_CUDA(cudaStreamSynchronize(W.s));
  return SVT_OK;
}


}  // namespace svt
