// Fast SVT driver (Algorithm 4) and R4SVD (Algorithm 3; Algorithm 2 on iteration 1).
//
// Host code here only sequences kernels and takes the scalar decisions of the
// algorithms (rank growth, cooling, stopping) from binary64 values read back after
// each step; every vector and matrix operation runs in the library's kernels.
//
// Readings of points the paper leaves open (shared with the CPU reference):
//  - residual eps^(i) = ||P_Lambda(A - X^(i))||_F / ||P_Lambda(A)||_F, after D_tau;
//    per iteration: R4SVD -> residual -> cooling -> stop (strict <) -> update;
//  - Y^(0) = k0 delta P_Lambda(A), k0 = ceil(tau / (delta ||P_Lambda(A)||_2)), the norm
//    from a fixed number of power steps from a seeded Gaussian start vector;
//  - power iterations X <- Y (Y^T X); QB error (||Y||^2 - ||B||^2) / ||Y||^2;
//  - new blocks are appended, orthogonalised against Q twice, and the range counts
//    as exhausted (block discarded, loop ended) when the smallest diagonal entry of
//    the block's triangular factor is at most 1e-7 of its largest column norm;
//  - the first iteration draws a block of width min(t, r_cap) unconditionally; all r
//    columns of U are recycled; r_cap = min(m, n, r_max);
//  - D_tau keeps sigma_j > tau.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dense_core.cuh"
#include "kernels.cuh"
#include "solver.cuh"

namespace svt {

// ------------------------------------------------------------------ error plumbing
static thread_local char g_err[512] = "no error";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

svt_status fail(svt_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

svt_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error '%s' in %s (%s:%d)", cudaGetErrorString(e), what, file, line);
  return SVT_ERR_CUDA;
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t delta) { g_launches.fetch_add(delta, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

int num_sms() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      cached = v;
    else
      return 132;
  }
  return cached;
}

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static thread_local Workspace* g_ws = nullptr;
Workspace* current_workspace() { return g_ws; }
WorkspaceScope::WorkspaceScope(void* base, size_t bytes) : prev(g_ws) {
  ws.base = static_cast<char*>(base);
  ws.cap = bytes;
  g_ws = base ? &ws : prev;
}
WorkspaceScope::~WorkspaceScope() { g_ws = prev; }

svt_status DeviceBlock::alloc(size_t bytes, cudaStream_t s) {
  release();
  stream = s;
  if (Workspace* w = g_ws) {
    const size_t off = (size_t)round_up((int64_t)w->top, 256);
    const size_t len = (size_t)round_up((int64_t)(bytes > 0 ? bytes : 256), 256);
    if (off + len > w->cap)
      return fail(SVT_ERR_ARG, "workspace of %zu bytes is too small (needs at least %zu)", w->cap, off + len);
    ptr = w->base + off;
    ws = w;
    ws_prev_top = w->top;
    ws_end = off + len;
    w->top = ws_end;
    return SVT_OK;
  }
  static std::once_flag once;
  std::call_once(once, []() {
    // keep freed stream-ordered memory in the pool between calls
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  });
  SVT_CUDA(cudaMallocAsync(&ptr, bytes > 0 ? bytes : 256, s));
  return SVT_OK;
}

// Page-locked host buffers for the solver's small device-to-host copies, kept for reuse
// by later solves (a solve takes one while it runs).
namespace {
std::mutex g_pin_mu;
std::vector<std::pair<void*, size_t>> g_pin_free;
}  // namespace

// *len receives the buffer's size (at least `bytes`), to be handed back to pinned_release.
svt_status pinned_acquire(size_t bytes, void** out, size_t* len) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (size_t i = 0; i < g_pin_free.size(); ++i)
      if (g_pin_free[i].second >= bytes) {
        *out = g_pin_free[i].first;
        *len = g_pin_free[i].second;
        g_pin_free.erase(g_pin_free.begin() + (int64_t)i);
        return SVT_OK;
      }
  }
  *len = std::max<size_t>(bytes, 64 * 1024);
  SVT_CUDA(cudaMallocHost(out, *len));
  return SVT_OK;
}

void pinned_release(void* p, size_t len) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.emplace_back(p, len);
}

// profiler state shared with solver.cuh
std::mutex g_prof_mu;
bool g_prof_on = false;
thread_local std::vector<Pending>* g_prof_capture = nullptr;
std::vector<ProfEntry> g_prof;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;

namespace {

// Rows with at least this fraction of n observed entries form the dense core (automatic
// choice).  On the tensor cores a core row costs its whole panel row (A read, Y read and
// written: 12 bytes per column); on the gather path each of its entries costs one
// gathered row of U (4r bytes from L2), so rows this full are far cheaper in the core.
constexpr double kCoreMinFrac = 0.1;

// Binary32 solves re-orthonormalise the recycled basis every this many iterations.  Lifted
// and recycled in binary32, the basis drifts from orthonormality by about 2e-6 per
// iteration (max |Q^T Q - I| of 1.1e-5, 1.5e-4 and 5.8e-4 after 5, 60 and 300 iterations
// of the 71,567 x 10,681 workload without it), so the drift stays near 1e-4.
constexpr int kReorthEvery = 50;

// The evaluation set of svt_complete_eval on the device: its own sorted pattern, the
// values in that pattern's CSR order, and a zero Y for the sampled pass (delta = 0).
template <typename T>
struct EvalSet {
  int64_t n = 0;
  svt_pattern* pat = nullptr;
  DeviceBlock blk;
  T* a = nullptr;
  T* y = nullptr;
  ~EvalSet() { if (pat) svt_pattern_destroy(pat); }
  svt_status init(int64_t m, int64_t nc, int64_t ne, const int32_t* r, const int32_t* c,
                  const T* v, cudaStream_t st) {
    n = ne;
    if (ne <= 0) return SVT_OK;
    Arena a0;
    a0.take<int32_t>(ne); a0.take<int32_t>(ne); a0.take<T>(ne); a0.take<T>(ne); a0.take<T>(ne);
    SVT_TRY(blk.alloc(a0.off, st));
    Arena b; b.base = (char*)blk.ptr;
    int32_t* r2 = b.take<int32_t>(ne);
    int32_t* c2 = b.take<int32_t>(ne);
    T* v2 = b.take<T>(ne);
    a = b.take<T>(ne);
    y = b.take<T>(ne);
    SVT_CUDA(cudaMemcpyAsync(r2, r, ne * sizeof(int32_t), cudaMemcpyDefault, st));
    SVT_CUDA(cudaMemcpyAsync(c2, c, ne * sizeof(int32_t), cudaMemcpyDefault, st));
    SVT_CUDA(cudaMemcpyAsync(v2, v, ne * sizeof(T), cudaMemcpyDefault, st));
    SVT_TRY(build_pattern(m, nc, ne, r2, c2, st, &pat));
    SVT_TRY((gather_convert<T, T>(ne, pat->csr_src, v2, a, st)));
    SVT_CUDA(cudaMemsetAsync(y, 0, ne * sizeof(T), st));
    return SVT_OK;
  }
};

// The solve's own device arrays next to the R4SVD work buffers: A and Y in both orders, a
// second B^T that the fused update fills while the solver still reads the current one, the
// fused update's block sums, and the dense core (binary32) when the plan has one.
template <typename T>
struct SolveBufs {
  T *a_csr = nullptr, *y_csr = nullptr, *a_csc = nullptr, *bt_alt = nullptr;
  double* fpart = nullptr;
  int64_t ldb_alt = 0;
  DenseCore core;
  int32_t* core_src = nullptr;
  void layout(Arena& ar, int64_t m, int64_t n, int64_t nnz, int r_cap, const CorePlan& plan) {
    ldb_alt = ld_of(r_cap);
    a_csr = ar.take<T>(nnz);
    y_csr = ar.take<T>(nnz);
    a_csc = ar.take<T>(nnz);
    bt_alt = ar.take<T>(n * ldb_alt);
    fpart = ar.take<double>(update_recycle_scratch(nnz));
    if (plan.rd > 0) {
      core_layout(ar, plan, m, n, r_cap, &core);
      core_src = ar.take<int32_t>(nnz);
    }
  }
};

// Peak bytes a solve takes from a caller workspace, replaying its allocations in order:
// the inputs' device copies (counted whether or not the inputs are host memory), the
// pattern with its sort scratch, the evaluation set with its pattern and scratch, the solve
// arena (with the largest core the plan could choose), and the staging of host outputs.
template <typename T>
size_t complete_ws_bytes(int64_t m, int64_t n, int64_t nnz, int64_t n_eval, int32_t cap,
                         const svt_options* opt, const Params& P) {
  auto blk = [](size_t bytes) { return (size_t)round_up((int64_t)(bytes > 0 ? bytes : 256), 256); };
  size_t in = 0;
  if (nnz > 0) {
    Arena a;
    a.take<int32_t>(nnz); a.take<int32_t>(nnz); a.take<T>(nnz);
    in = blk(a.off);
  }
  const size_t pat = blk(pattern_block_bytes(m, n, nnz));
  const size_t pat_scr = nnz > 0 ? blk(pattern_scratch_bytes(nnz)) : 0;
  size_t ev = 0, ev_pat = 0, ev_scr = 0;
  if (n_eval > 0) {
    Arena e;
    e.take<int32_t>(n_eval); e.take<int32_t>(n_eval);
    e.take<T>(n_eval); e.take<T>(n_eval); e.take<T>(n_eval);
    ev = blk(e.off);
    ev_pat = blk(pattern_block_bytes(m, n, n_eval));
    ev_scr = blk(pattern_scratch_bytes(n_eval));
  }
  size_t main = 0;
  if (nnz > 0) {
    CorePlan bound;
    if (sizeof(T) == 4 && opt->core_rows != 0)
      bound = core_plan_bound(m, n, nnz, opt->core_rows, kCoreMinFrac);
    svt_pattern fake;
    fake.m = m; fake.n = n; fake.nnz = nnz;
    Work<T> W;
    W.P = P; W.pat = &fake;
    SolveBufs<T> B;
    Arena a;
    B.layout(a, m, n, nnz, P.r_cap, bound);
    W.layout(a);
    main = blk(a.off);
  }
  const size_t out = blk((size_t)std::max(m, n) * (size_t)std::max(cap, 1) * sizeof(double));
  return in + pat + std::max(pat_scr, ev + ev_pat + std::max(ev_scr, main + out));
}

// Bytes svt_r4svd takes from a caller workspace: its work buffers.
template <typename T>
size_t r4svd_ws_bytes(int64_t m, int64_t n, int64_t nnz, const Params& P) {
  svt_pattern fake;
  fake.m = m; fake.n = n; fake.nnz = nnz;
  Work<T> W;
  W.P = P; W.pat = &fake;
  Arena a;
  W.layout(a);
  return (size_t)round_up((int64_t)(a.off > 0 ? a.off : 256), 256);
}

template <typename T>
svt_status complete_impl(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                         const int32_t* cols, const T* vals, double tau, double delta,
                         double tol, int32_t maxit, const svt_options* opt, double* Uo,
                         double* So, double* Vo, int32_t cap, svt_result* res,
                         svt_iter_log* log, int32_t log_cap, int64_t n_eval = 0,
                         const int32_t* eval_rows = nullptr, const int32_t* eval_cols = nullptr,
                         const T* eval_vals = nullptr) {
  const auto t_start = clk::now();
  Params P;
  SVT_TRY(make_params(m, n, opt, &P));
  if (cap < P.r_cap) return fail(SVT_ERR_ARG, "output capacity %d below the rank cap %d", cap, P.r_cap);
  cudaStream_t st = (cudaStream_t)opt->stream;

  // Inputs to device (copied when the caller passes host memory).
  DeviceBlock in_blk;
  const int32_t* d_rows = rows;
  const int32_t* d_cols = cols;
  const T* d_vals = vals;
  if (nnz > 0) {
    const bool dr = is_device_pointer(rows), dc = is_device_pointer(cols), dv = is_device_pointer(vals);
    if (!dr || !dc || !dv) {
      Arena a;
      a.take<int32_t>(nnz); a.take<int32_t>(nnz); a.take<T>(nnz);
      SVT_TRY(in_blk.alloc(a.off, st));
      Arena b; b.base = (char*)in_blk.ptr;
      int32_t* r2 = b.take<int32_t>(nnz);
      int32_t* c2 = b.take<int32_t>(nnz);
      T* v2 = b.take<T>(nnz);
      if (!dr) { SVT_CUDA(cudaMemcpyAsync(r2, rows, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st)); d_rows = r2; }
      if (!dc) { SVT_CUDA(cudaMemcpyAsync(c2, cols, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st)); d_cols = c2; }
      if (!dv) { SVT_CUDA(cudaMemcpyAsync(v2, vals, nnz * sizeof(T), cudaMemcpyHostToDevice, st)); d_vals = v2; }
    }
  }
  svt_pattern* pat = nullptr;
  const auto t_pat = clk::now();
  {
    SVT_PROF("pattern_build", 2.0 * nnz * 36.0, st);
    SVT_TRY(build_pattern(m, n, nnz, d_rows, d_cols, st, &pat));
  }
  struct PatGuard { svt_pattern* p; ~PatGuard() { svt_pattern_destroy(p); } } pg{pat};
  res->seconds_pattern = seconds_since(t_pat);
  EvalSet<T> ev;
  SVT_TRY(ev.init(m, n, n_eval, eval_rows, eval_cols, eval_vals, st));

  auto zero_outputs = [&]() -> svt_status {
    // X = 0: k = 0, outputs cleared
    std::vector<double> zeros;
    auto clear = [&](double* p, int64_t count) -> svt_status {
      if (!p || count <= 0) return SVT_OK;
      if (is_device_pointer(p)) { SVT_CUDA(cudaMemsetAsync(p, 0, count * sizeof(double), st)); }
      else memset(p, 0, count * sizeof(double));
      return SVT_OK;
    };
    SVT_TRY(clear(Uo, m * cap));
    SVT_TRY(clear(So, cap));
    SVT_TRY(clear(Vo, n * cap));
    SVT_CUDA(cudaStreamSynchronize(st));
    return SVT_OK;
  };

  res->k = 0; res->r = 0; res->iters = 0; res->k0 = 0; res->log_len = 0;
  res->rel_residual = 0.0; res->mae = 0.0; res->spec_norm = 0.0; res->eps_thr = P.eps_thr0;
  if (nnz == 0) {
    SVT_TRY(zero_outputs());
    res->status = SVT_OK;
    res->seconds_total = seconds_since(t_start);
    return SVT_OK;
  }

  // page-locked host words for the copies inside the captured eigen phase
  struct HostPin {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    ~HostPin() {
      if (!p) return;
      cudaStreamSynchronize(s);  // a graph launched ahead may still copy into it
      pinned_release(p, bytes);
    }
  } pin;
  pin.s = st;
  SVT_TRY(pinned_acquire(Work<T>::pin_doubles(P.r_cap) * sizeof(double), &pin.p, &pin.bytes));
  Work<T> W;
  W.P = P; W.pat = pat; W.s = st;
  W.host_pin = static_cast<double*>(pin.p);
  // binary32: the fullest rows may form a dense core updated on the tensor cores
  CorePlan cplan;
  if constexpr (sizeof(T) == 4) {
    if (opt->core_rows != 0 && P.r_cap >= 1) SVT_TRY(core_plan(pat, opt->core_rows, kCoreMinFrac, st, &cplan));
  }
  SolveBufs<T> B;
  Arena a;
  B.layout(a, m, n, nnz, P.r_cap, cplan);
  W.layout(a);
  DeviceBlock wblk;
  SVT_TRY(wblk.alloc(a.off, st));
  Arena b; b.base = (char*)wblk.ptr;
  B.layout(b, m, n, nnz, P.r_cap, cplan);
  W.layout(b);
  const int64_t ldb_alt = B.ldb_alt;
  T *a_csr = B.a_csr, *y_csr = B.y_csr, *a_csc = B.a_csc, *bt_alt = B.bt_alt;
  double* fpart = B.fpart;
  DenseCore& core = B.core;
  int32_t* core_src = B.core_src;
  SVT_CUDA(cudaMemsetAsync(W.flags, 0, kFlagWords * sizeof(unsigned), st));

  // P_Lambda(A) in CSR order; reject non-finite values.
  SVT_TRY((gather_convert<T, T>(nnz, pat->csr_src, d_vals, a_csr, st)));
  double nA2 = 0.0;
  SVT_TRY(sumsq<T>(nnz, a_csr, W.dsc + 2, W.part, st));
  SVT_CUDA(cudaMemcpyAsync(&nA2, W.dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
  SVT_CUDA(cudaStreamSynchronize(st));
  if (!std::isfinite(nA2)) return fail(SVT_ERR_NUMERIC, "non-finite observed value");
  if (nA2 == 0.0) {
    SVT_TRY(zero_outputs());
    res->status = SVT_OK;
    res->seconds_total = seconds_since(t_start);
    return SVT_OK;
  }
  const double nA = std::sqrt(nA2);

  // ||P_Lambda(A)||_2 by power steps v <- A^T A v / ||A^T A v||
  SVT_TRY(launch_gather<T>(nnz, pat->perm, a_csr, a_csc, st));
  SVT_TRY(launch_gaussian<double>(P.seed, kPowerSeedIter, 0, n, 1, W.pw, 1, st));
  SVT_TRY(sumsq<double>(n, W.pw, W.dsc + 3, W.part, st));
  k_normalize<<<(int)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(n, W.pw, W.dsc + 3, W.pv);
  SVT_LAUNCH_CHECK();
  for (int it = 0; it < P.power_steps; ++it) {
    SVT_PROF("init_power", spmm_bytes(nnz, m, n, 1, (int)sizeof(T)) + spmm_bytes(nnz, n, m, 1, (int)sizeof(T)), st);
    SVT_TRY((launch_spmm_rows<T, double>(m, pat->row_ptr, pat->col_idx, a_csr, W.pv, 1, 1, W.pu, 1,
                                         W.spmm_scr, nnz, st, pat->chunk_row_csr)));
    SVT_TRY((launch_spmm_rows<T, double>(n, pat->col_ptr, pat->row_idx, a_csc, W.pu, 1, 1, W.pw, 1,
                                         W.spmm_scr, nnz, st, pat->chunk_row_csc)));
    SVT_TRY(sumsq<double>(n, W.pw, W.dsc + 3, W.part, st));
    k_normalize<<<(int)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(n, W.pw, W.dsc + 3, W.pv);
    SVT_LAUNCH_CHECK();
  }
  double lam2 = 0.0;
  SVT_CUDA(cudaMemcpyAsync(&lam2, W.dsc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
  SVT_CUDA(cudaStreamSynchronize(st));
  const double s2 = std::sqrt(std::sqrt(lam2));
  const double kk = s2 > 0.0 ? std::ceil(tau / (delta * s2)) : 1.0;
  const int k0 = (int)std::min(kk, 2.0e9);
  res->k0 = k0;
  res->spec_norm = s2;
  SVT_TRY(scale_copy<T>(nnz, a_csr, (double)k0 * delta, y_csr, st));
  SVT_TRY(launch_gather<T>(nnz, pat->perm, y_csr, W.y_csc, st));
  bool core_active = false;  // Y lives in the sparse rest and the core panel
  if constexpr (sizeof(T) == 4) {
    if (cplan.rd > 0) SVT_TRY(core_build(pat, cplan, a_csc, core_src, st, &core));
  }
  double normY2 = 0.0;
  SVT_TRY(sumsq<T>(nnz, y_csr, W.dsc + 4, W.part, st));
  SVT_CUDA(cudaMemcpyAsync(&normY2, W.dsc + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
  SVT_CUDA(cudaStreamSynchronize(st));

  double eps_thr = P.eps_thr0, eps_min = INFINITY;
  int s = 0;
  T* Qcur = W.Qa;
  T* Qnext = W.Qb;
  int k = 0;
  R4Out ro;
  double rel = 0.0, mae = 0.0;
  int last_iter = 0;
  svt_status status = SVT_NOT_CONVERGED;
  std::vector<double> coef;
  bool fused = false;
  struct Event {
    cudaEvent_t e = nullptr;
    ~Event() { if (e) cudaEventDestroy(e); }
  } upd;
  SVT_CUDA(cudaEventCreateWithFlags(&upd.e, cudaEventDisableTiming));
  double* hsum = W.pin_tail();  // sums of the update, then its status word
  for (int i = 1; i <= maxit; ++i) {
    const auto t_it = clk::now();
    SVT_TRY(r4svd_run<T>(W, y_csr, W.y_csc, Qcur, s, normY2, eps_thr, (uint32_t)i, Qnext, &ro));
    const int r = ro.r;
    k = 0;
    while (k < r && ro.sigma[k] > tau) ++k;
    coef.assign(k, 0.0);
    for (int j = 0; j < k; ++j) coef[j] = (ro.sigma[j] - tau) / ro.sigma[j];
    SVT_TRY(scaled_right<T>(W, r, k, coef));
    SVT_CUDA(cudaMemsetAsync(W.flags, 0, sizeof(unsigned), st));
    // The first s_next columns of U (= Qnext) seed the next R4SVD call: all r of them
    // (Algorithm 3), the k kept ones, or none.  In CSC order the update also forms
    // B^T = Y^T U[:, :s_next] for that call.
    const int s_next = P.recycle == SVT_RECYCLE_ALL ? r : P.recycle == SVT_RECYCLE_KEPT ? k : 0;
    fused = s_next > 0 && update_recycle_fits<T>(s_next, nnz);
    bool use_core = false;
    if constexpr (sizeof(T) == 4) use_core = fused && cplan.rd > 0 && core_fits(s_next, k);
    if (core_active && !use_core) {  // back to the full copies of Y
      SVT_PROF("assemble_y", 2.0 * (double)nnz * (4 + 2 * sizeof(T)), st);
      if constexpr (sizeof(T) == 4) SVT_TRY(core_assemble(pat, core, y_csr, W.y_csc, st));
      core_active = false;
      W.refresh_y = nullptr;
      W.y_csr_stale = nullptr;
    }
    if (use_core) {
      if constexpr (sizeof(T) == 4) {
        if (!core_active) {
          SVT_TRY(core_enter(pat, W.y_csc, st, &core));
          core_active = true;
        }
        {
          SVT_PROF("update_recycled", recycle_bytes(core.rest.nnz, m, n, k, s_next, (int)sizeof(T)), st);
          SVT_TRY(update_recycle<T>(&core.rest, Qnext, W.ldq, s_next, W.Wk, W.ldk, k, core.a_rest,
                                    core.y_rest, delta, bt_alt, ldb_alt, W.dsc + 5, core.upd_part,
                                    W.flags, core.upd_scratch, st));
        }
        {
          SVT_PROF("update_core", (double)cplan.core_nnz * (4 + 3 * sizeof(T)), st);
          SVT_TRY(core_update(core, Qnext, W.ldq, s_next, W.Wk, W.ldk, k, delta, bt_alt, ldb_alt,
                              W.dsc + 5, W.flags, W.flags + 4, st));
        }
        W.y_csr_stale = nullptr;
        W.refresh_y = [&]() { return core_assemble(pat, core, y_csr, W.y_csc, W.s); };
      }
    } else if (fused) {
      SVT_PROF("update_recycled", recycle_bytes(nnz, m, n, k, s_next, (int)sizeof(T)), st);
      SVT_TRY(update_recycle<T>(pat, Qnext, W.ldq, s_next, W.Wk, W.ldk, k, a_csc, W.y_csc, delta,
                                bt_alt, ldb_alt, W.dsc + 5, fpart, W.flags, W.spmm_scr, st));
      W.y_csr_stale = y_csr;
    } else {
      if (W.y_csr_stale) {
        SVT_TRY(launch_scatter<T>(nnz, pat->perm, W.y_csc, y_csr, st));
        W.y_csr_stale = nullptr;
      }
      SVT_PROF("sampled_update", update_bytes(nnz, m, n, k, (int)sizeof(T)), st);
      SVT_TRY(sampled_update<T>(pat, Qnext, W.ldq, W.Wk, W.ldk, k, a_csr, y_csr, delta, W.dsc + 5,
                                W.part, W.flags, st, true));
    }
    if (ev.n > 0) {  // MAE of X^(i) = U[:, :k] W^T on the evaluation set (delta = 0: Y stays 0)
      SVT_TRY(sampled_update<T>(ev.pat, Qnext, W.ldq, W.Wk, W.ldk, k, ev.a, ev.y, 0.0, W.dsc + 8,
                                W.part, W.flags + 5, st, true));
      SVT_CUDA(cudaMemcpyAsync(hsum + 4, W.dsc + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    SVT_CUDA(cudaMemcpyAsync(hsum, W.dsc + 5, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaMemcpyAsync(hsum + 3, W.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaMemcpyAsync(reinterpret_cast<unsigned*>(hsum + 3) + 1, W.flags + 4, sizeof(unsigned),
                             cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaEventRecord(upd.e, st));
    if (fused) {  // the update formed Y^T U for the next iteration's recycled basis
      std::swap(W.Bt, bt_alt);
      W.bt_ready = true;
      // the next R4SVD call most likely needs no new block: launch its eigen phase now,
      // before this iteration's residual is known (r4svd_run checks the assumption); an
      // iteration that re-orthonormalises the basis first runs it there instead
      W.reorth_due = sizeof(T) == 4 && (i % kReorthEvery) == 0;
      if (i < maxit && !W.reorth_due) {
        bool ran = false;
        SVT_TRY(eig_phase_graph<T>(W, Qnext, s_next, Qcur, &ran));
        W.graph_inflight = ran;
      }
    }
    SVT_CUDA(cudaEventSynchronize(upd.e));
    double sums[3];
    unsigned fl = 0, fl_tc = 0;
    memcpy(sums, hsum, sizeof(sums));
    memcpy(&fl, hsum + 3, sizeof(unsigned));
    memcpy(&fl_tc, reinterpret_cast<const unsigned*>(hsum + 3) + 1, sizeof(unsigned));
    if (fl_tc & (FLAG_TC_TIMEOUT | FLAG_GRID_TIMEOUT))
      return fail(SVT_ERR_CUDA, "a bounded wait ran out (%s)",
                  (fl_tc & FLAG_TC_TIMEOUT) ? "tensor-core kernel" : "grid Jacobi");
    rel = std::sqrt(sums[0]) / nA;
    mae = sums[1] / (double)nnz;
    if (!std::isfinite(rel) || (fl & FLAG_NONFINITE))
      return fail(SVT_ERR_NUMERIC, "non-finite iterate at SVT iteration %d", i);
    const double thr_used = eps_thr;
    bool cooled = false;
    if (rel < eps_min) eps_min = rel;
    else { eps_thr *= P.beta; cooled = true; }
    last_iter = i;
    if (log && i - 1 < log_cap) {
      svt_iter_log& L = log[i - 1];
      L.iter = i; L.r = r; L.k = k; L.blocks = ro.blocks; L.cooled = cooled ? 1 : 0;
      L.exhausted = ro.exhausted ? 1 : 0; L.eps = ro.eps; L.eps_thr = thr_used;
      L.rel_residual = rel; L.mae = mae; L.sigma_max = r > 0 ? ro.sigma[0] : 0.0;
      L.mae_eval = ev.n > 0 ? hsum[5] / (double)ev.n : std::nan("");
      L.seconds = seconds_since(t_it);
      res->log_len = i;
    }
    res->r = r;
    if ((P.stop == SVT_STOP_MAE ? mae : rel) < tol) { status = SVT_OK; break; }
    if (!fused) {  // Y^(i+1) is in y_csr; refresh its CSC copy
      SVT_PROF("gather_csc", (double)nnz * (4 + 2 * sizeof(T)), st);
      SVT_TRY(launch_gather<T>(nnz, pat->perm, y_csr, W.y_csc, st));
    }
    prof_flush();
    normY2 = sums[2];
    std::swap(Qcur, Qnext);
    s = s_next;
  }
  res->iters = last_iter;
  res->k = k;
  res->rel_residual = rel;
  res->mae = mae;
  res->eps_thr = eps_thr;
  res->status = status;
  if (last_iter == 0) {
    SVT_TRY(zero_outputs());
    res->seconds_total = seconds_since(t_start);
    return status;
  }
  // X = U_K diag(sigma_K - tau) V_K^T with V_K = B^T U_B,K Sigma_K^-1.  The last update used
  // W = B^T U_B,K diag((sigma_K - tau) / sigma_K), so V_K = W diag(1 / (sigma_K - tau)); the
  // buffers of the eigen phase may already hold the next (speculated) iteration.
  std::vector<double> inv(k), shrunk(cap, 0.0);
  for (int j = 0; j < k; ++j) { inv[j] = 1.0 / (ro.sigma[j] - tau); shrunk[j] = ro.sigma[j] - tau; }
  if (k > 0) SVT_CUDA(cudaMemcpyAsync(W.coef, inv.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
  T* Ufinal = (last_iter > 0 && status == SVT_OK) ? Qnext : Qcur;
  // after a converged break Qnext holds U; after the loop ran out, the swap moved it to Qcur
  SVT_TRY(export_cols<T>(W, m, k, Ufinal, W.ldq, Uo, cap));
  SVT_TRY(export_cols<T>(W, n, k, W.Wk, W.ldk, Vo, cap, W.coef));
  if (So) SVT_CUDA(cudaMemcpyAsync(So, shrunk.data(), cap * sizeof(double), cudaMemcpyDefault, st));
  SVT_CUDA(cudaStreamSynchronize(st));
  prof_flush();
  res->seconds_total = seconds_since(t_start);
  return status;
}

template <typename T>
svt_status r4svd_impl(const svt_pattern* p, const T* y_csr, const T* U_prev, int64_t ld_prev,
                      int32_t s, double eps_thr, uint32_t iter, const svt_options* opt, T* U,
                      int64_t ldu, double* S, T* V, int64_t ldv, int32_t* r_out,
                      double* eps_out, int32_t* blocks_out) {
  Params P;
  SVT_TRY(make_params(p->m, p->n, opt, &P));
  if (s < 0 || s > P.r_cap) return fail(SVT_ERR_ARG, "r4svd: recycled rank %d outside [0, %d]", s, P.r_cap);
  if (s > 0 && (!U_prev || ld_prev < s)) return fail(SVT_ERR_ARG, "r4svd: bad recycled basis");
  if (!U || !V || ldu < P.r_cap || ldv < P.r_cap)
    return fail(SVT_ERR_ARG, "r4svd: outputs need capacity for %d columns", P.r_cap);
  cudaStream_t st = (cudaStream_t)opt->stream;
  Work<T> W;
  W.P = P; W.pat = p; W.s = st;
  Arena a;
  W.layout(a);
  DeviceBlock blk;
  SVT_TRY(blk.alloc(a.off, st));
  Arena b; b.base = (char*)blk.ptr;
  W.layout(b);
  SVT_CUDA(cudaMemsetAsync(W.flags, 0, kFlagWords * sizeof(unsigned), st));
  const int64_t nnz = p->nnz;
  SVT_TRY(launch_gather<T>(nnz, p->perm, y_csr, W.y_csc, st));
  double normY2 = 0.0;
  SVT_TRY(sumsq<T>(nnz, y_csr, W.dsc + 4, W.part, st));
  SVT_CUDA(cudaMemcpyAsync(&normY2, W.dsc + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (s > 0) SVT_TRY((copy_convert<T, T>(p->m, s, U_prev, ld_prev, W.Qa, W.ldq, st)));
  SVT_CUDA(cudaStreamSynchronize(st));
  R4Out ro;
  SVT_TRY(r4svd_run<T>(W, y_csr, W.y_csc, W.Qa, s, normY2, eps_thr, iter, W.Qb, &ro));
  const int r = ro.r;
  std::vector<double> inv(r);
  for (int j = 0; j < r; ++j) inv[j] = ro.sigma[j] > 0.0 ? 1.0 / ro.sigma[j] : 0.0;
  SVT_TRY(scaled_right<T>(W, r, r, inv));
  SVT_TRY((copy_convert<T, T>(p->m, r, W.Qb, W.ldq, U, ldu, st)));
  SVT_TRY((copy_convert<T, T>(p->n, r, W.Wk, W.ldk, V, ldv, st)));
  if (S && r > 0) SVT_CUDA(cudaMemcpyAsync(S, ro.sigma.data(), r * sizeof(double), cudaMemcpyDefault, st));
  SVT_CUDA(cudaStreamSynchronize(st));
  if (r_out) *r_out = r;
  if (eps_out) *eps_out = ro.eps;
  if (blocks_out) *blocks_out = ro.blocks;
  return SVT_OK;
}

}  // namespace
}  // namespace svt

// ====================================================================== C ABI
extern "C" int svt_abi_version(void) { return 3; }

extern "C" void svt_default_options(svt_options* o) {
  if (!o) return;
  o->t = -1;
  o->dt = 10;
  o->n_power = 0;
  o->r_max = 0;
  o->power_steps = 100;
  o->precision = SVT_FP64;
  o->recycle = SVT_RECYCLE_ALL;
  o->stop = SVT_STOP_RESIDUAL;
  o->core_rows = -1;
  o->reserved = 0;
  o->beta = 0.95;
  o->eps_thr0 = 0.9;
  o->seed = 0x5EEDull;
  o->stream = nullptr;
}

extern "C" const char* svt_status_string(int s) {
  switch (s) {
    case SVT_OK: return "ok";
    case SVT_NOT_CONVERGED: return "not converged within maxit";
    case SVT_ERR_ARG: return "invalid argument";
    case SVT_ERR_INDEX: return "observed index out of range";
    case SVT_ERR_DUPLICATE: return "duplicate observed entry";
    case SVT_ERR_CUDA: return "CUDA runtime error";
    case SVT_ERR_NUMERIC: return "non-finite value";
    case SVT_ERR_UNSUPPORTED: return "unsupported size";
    default: return "unknown status";
  }
}

extern "C" const char* svt_last_error(void) { return svt::g_err; }

extern "C" svt_status svt_spmm(const svt_pattern* p, int precision, int transpose, const void* y_csr,
                               const void* W, int64_t ldw, int32_t w, void* out, int64_t ldo,
                               void* stream) {
  using namespace svt;
  if (!p || w < 0 || (p->nnz > 0 && !y_csr)) return fail(SVT_ERR_ARG, "spmm: bad arguments");
  if (precision != SVT_FP64 && precision != SVT_MIXED_FP32) return fail(SVT_ERR_ARG, "spmm: unknown precision");
  if (w > 0 && (!W || !out || ldw < w || ldo < w)) return fail(SVT_ERR_ARG, "spmm: bad dense operands");
  if (w == 0) return SVT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t z = p->nnz;
  const int64_t rows_out = transpose ? p->n : p->m;
  const int elem = precision == SVT_FP64 ? 8 : 4;
  DeviceBlock tmp;
  Arena a;
  a.take<char>(z * elem);
  a.take<char>(spmm_scratch_bytes(z, w, elem));
  SVT_TRY(tmp.alloc(a.off, s));
  Arena b; b.base = (char*)tmp.ptr;
  char* ycsc = b.take<char>(z * elem);
  char* scr = b.take<char>(spmm_scratch_bytes(z, w, elem));
  auto run = [&](auto tag) -> svt_status {
    using T = decltype(tag);
    const T* y = (const T*)y_csr;
    if (transpose) {
      SVT_TRY(launch_gather<T>(z, p->perm, y, (T*)ycsc, s));
      SVT_TRY((launch_spmm_rows<T, T>(rows_out, p->col_ptr, p->row_idx, (const T*)ycsc, (const T*)W, ldw,
                                       w, (T*)out, ldo, scr, z, s, p->chunk_row_csc)));
    } else {
      SVT_TRY((launch_spmm_rows<T, T>(rows_out, p->row_ptr, p->col_idx, y, (const T*)W, ldw, w, (T*)out,
                                       ldo, scr, z, s, p->chunk_row_csr)));
    }
    return SVT_OK;
  };
  SVT_TRY(precision == SVT_FP64 ? run(double(0)) : run(float(0)));
  SVT_CUDA(cudaStreamSynchronize(s));
  return SVT_OK;
}

extern "C" svt_status svt_sampled_update(const svt_pattern* p, int precision, const void* U,
                                         int64_t ldu, const void* W, int64_t ldw, int32_t k,
                                         const void* a_csr, void* y_csr, double delta, double* sums,
                                         void* stream) {
  using namespace svt;
  if (!p || k < 0 || !sums || (k > 0 && (!U || !W || ldu < k || ldw < k)))
    return fail(SVT_ERR_ARG, "sampled_update: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceBlock blk;
  const size_t pe = reduce_scratch();
  SVT_TRY(blk.alloc(pe * sizeof(double) + 64 + 256, s));
  double* part = (double*)blk.ptr;
  double* out3 = part + pe;
  unsigned* flags = (unsigned*)(out3 + 4);
  SVT_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), s));
  if (precision == SVT_FP64)
    SVT_TRY(sampled_update<double>(p, (const double*)U, ldu, (const double*)W, ldw, k,
                                   (const double*)a_csr, (double*)y_csr, delta, out3, part, flags, s));
  else if (precision == SVT_MIXED_FP32)
    SVT_TRY(sampled_update<float>(p, (const float*)U, ldu, (const float*)W, ldw, k,
                                  (const float*)a_csr, (float*)y_csr, delta, out3, part, flags, s));
  else
    return fail(SVT_ERR_ARG, "sampled_update: unknown precision");
  SVT_CUDA(cudaMemcpyAsync(sums, out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  SVT_CUDA(cudaStreamSynchronize(s));
  return SVT_OK;
}

extern "C" svt_status svt_sampled_update_recycle(const svt_pattern* p, int precision,
                                                 const void* U, int64_t ldu, int32_t r,
                                                 const void* W, int64_t ldw, int32_t k,
                                                 const void* a_csc, void* y_csc, double delta,
                                                 void* Bt, int64_t ldb, double* sums,
                                                 void* stream) {
  using namespace svt;
  if (!p || !sums || !U || !Bt || r < 1 || k < 0 || k > r || ldb < r || ldu < r ||
      (k > 0 && (!W || ldw < k)) || (p->nnz > 0 && (!a_csc || !y_csc)))
    return fail(SVT_ERR_ARG, "sampled_update_recycle: bad arguments");
  if (precision != SVT_FP64 && precision != SVT_MIXED_FP32)
    return fail(SVT_ERR_ARG, "sampled_update_recycle: unknown precision");
  const bool f64 = precision == SVT_FP64;
  if (!(f64 ? update_recycle_fits<double>(r, p->nnz) : update_recycle_fits<float>(r, p->nnz)))
    return fail(SVT_ERR_ARG, "sampled_update_recycle: r = %d or nnz above the limit", r);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t z = p->nnz;
  const size_t pe = update_recycle_scratch(z);
  const size_t sb = spmm_scratch_bytes(z > 0 ? z : 1, r, f64 ? 8 : 4);
  DeviceBlock blk;
  SVT_TRY(blk.alloc(round_up((int64_t)(pe * sizeof(double)), 256) + 256 + sb, s));
  double* part = (double*)blk.ptr;
  double* out3 = (double*)((char*)blk.ptr + round_up((int64_t)(pe * sizeof(double)), 256));
  unsigned* flags = (unsigned*)(out3 + 4);
  void* scratch = (char*)out3 + 256;
  SVT_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), s));
  // W is only read when k > 0; a k = 0 call may pass any aligned pointer for it
  const void* Wp = k > 0 ? W : U;
  const int64_t ldw_ = k > 0 ? ldw : ldu;
  if (f64)
    SVT_TRY(update_recycle<double>(p, (const double*)U, ldu, r, (const double*)Wp, ldw_, k,
                                   (const double*)a_csc, (double*)y_csc, delta, (double*)Bt, ldb,
                                   out3, part, flags, scratch, s));
  else
    SVT_TRY(update_recycle<float>(p, (const float*)U, ldu, r, (const float*)Wp, ldw_, k,
                                  (const float*)a_csc, (float*)y_csc, delta, (float*)Bt, ldb, out3,
                                  part, flags, scratch, s));
  SVT_CUDA(cudaMemcpyAsync(sums, out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  SVT_CUDA(cudaStreamSynchronize(s));
  return SVT_OK;
}

extern "C" size_t svt_r4svd_workspace_size(int64_t m, int64_t n, int64_t nnz, const svt_options* opt) {
  using namespace svt;
  Params P;
  if (!opt || m <= 0 || n <= 0 || nnz < 0 || make_params(m, n, opt, &P) != SVT_OK) return 0;
  return opt->precision == SVT_FP64 ? r4svd_ws_bytes<double>(m, n, nnz, P) : r4svd_ws_bytes<float>(m, n, nnz, P);
}

extern "C" size_t svt_workspace_size(int64_t m, int64_t n, int64_t nnz, int64_t n_eval, int32_t cap,
                                     const svt_options* opt) {
  using namespace svt;
  Params P;
  if (!opt || m <= 0 || n <= 0 || nnz < 0 || n_eval < 0 || make_params(m, n, opt, &P) != SVT_OK)
    return 0;
  return opt->precision == SVT_FP64 ? complete_ws_bytes<double>(m, n, nnz, n_eval, cap, opt, P)
                                    : complete_ws_bytes<float>(m, n, nnz, n_eval, cap, opt, P);
}

extern "C" svt_status svt_r4svd(const svt_pattern* p, const void* y_csr, const void* U_prev,
                                int64_t ld_prev, int32_t s, double eps_thr, uint32_t iter,
                                const svt_options* opt, void* U, int64_t ldu, double* S, void* V,
                                int64_t ldv, int32_t* r_out, double* eps_out, int32_t* blocks_out,
                                void* workspace, size_t ws_bytes) {
  using namespace svt;
  if (!p || !opt || (p->nnz > 0 && !y_csr)) return fail(SVT_ERR_ARG, "r4svd: bad arguments");
  if (workspace) {
    const size_t need = svt_r4svd_workspace_size(p->m, p->n, p->nnz, opt);
    if (need == 0 || ws_bytes < need)
      return fail(SVT_ERR_ARG, "r4svd: workspace of %zu bytes is below the %zu bytes of "
                               "svt_r4svd_workspace_size", ws_bytes, need);
  }
  WorkspaceScope scope(workspace, ws_bytes);
  if (opt->precision == SVT_FP64)
    return r4svd_impl<double>(p, (const double*)y_csr, (const double*)U_prev, ld_prev, s, eps_thr,
                              iter, opt, (double*)U, ldu, S, (double*)V, ldv, r_out, eps_out,
                              blocks_out);
  if (opt->precision == SVT_MIXED_FP32)
    return r4svd_impl<float>(p, (const float*)y_csr, (const float*)U_prev, ld_prev, s, eps_thr, iter,
                             opt, (float*)U, ldu, S, (float*)V, ldv, r_out, eps_out, blocks_out);
  return fail(SVT_ERR_ARG, "r4svd: unknown precision");
}

extern "C" svt_status svt_complete(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                                   const int32_t* cols, const void* vals, double tau, double delta,
                                   double tol, int32_t maxit, const svt_options* opt, double* U,
                                   double* S, double* V, int32_t cap, svt_result* res,
                                   svt_iter_log* log, int32_t log_cap, void* workspace,
                                   size_t ws_bytes) {
  return svt_complete_eval(m, n, nnz, rows, cols, vals, 0, nullptr, nullptr, nullptr, tau, delta,
                           tol, maxit, opt, U, S, V, cap, res, log, log_cap, workspace, ws_bytes);
}

extern "C" svt_status svt_complete_eval(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                                        const int32_t* cols, const void* vals, int64_t n_eval,
                                        const int32_t* eval_rows, const int32_t* eval_cols,
                                        const void* eval_vals, double tau, double delta,
                                        double tol, int32_t maxit, const svt_options* opt,
                                        double* U, double* S, double* V, int32_t cap,
                                        svt_result* res, svt_iter_log* log, int32_t log_cap,
                                        void* workspace, size_t ws_bytes) {
  using namespace svt;
  if (!res) return fail(SVT_ERR_ARG, "complete: null result");
  memset(res, 0, sizeof(*res));
  res->status = SVT_ERR_ARG;
  if (!opt) return fail(SVT_ERR_ARG, "complete: null options");
  if (m <= 0 || n <= 0 || nnz < 0 || maxit < 0 || cap < 1)
    return fail(SVT_ERR_ARG, "complete: need m, n > 0, nnz >= 0, maxit >= 0, cap >= 1");
  if (!(tau > 0.0) || !(delta > 0.0) || !std::isfinite(tau) || !std::isfinite(delta) || std::isnan(tol))
    return fail(SVT_ERR_ARG, "complete: need finite tau > 0, delta > 0");
  if (nnz > 0 && (!rows || !cols || !vals)) return fail(SVT_ERR_ARG, "complete: null input array");
  if (n_eval < 0 || (n_eval > 0 && (!eval_rows || !eval_cols || !eval_vals)))
    return fail(SVT_ERR_ARG, "complete: bad evaluation set");
  if (workspace) {  // checked before any work is queued
    const size_t need = svt_workspace_size(m, n, nnz, n_eval, cap, opt);
    if (need == 0) {
      Params P;
      return make_params(m, n, opt, &P);  // sets the message of the invalid option
    }
    if (ws_bytes < need)
      return fail(SVT_ERR_ARG, "complete: workspace of %zu bytes is below the %zu bytes of "
                               "svt_workspace_size", ws_bytes, need);
  }
  WorkspaceScope scope(workspace, ws_bytes);
  svt_status st;
  if (opt->precision == SVT_FP64)
    st = complete_impl<double>(m, n, nnz, rows, cols, (const double*)vals, tau, delta, tol, maxit,
                               opt, U, S, V, cap, res, log, log_cap, n_eval, eval_rows, eval_cols,
                               (const double*)eval_vals);
  else if (opt->precision == SVT_MIXED_FP32)
    st = complete_impl<float>(m, n, nnz, rows, cols, (const float*)vals, tau, delta, tol, maxit,
                              opt, U, S, V, cap, res, log, log_cap, n_eval, eval_rows, eval_cols,
                              (const float*)eval_vals);
  else
    st = fail(SVT_ERR_ARG, "complete: unknown precision");
  if (st < 0) {
    cudaStreamSynchronize((cudaStream_t)opt->stream);
    res->status = st;
  }
  return st;
}

extern "C" void svt_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(svt::g_prof_mu);
  svt::g_prof_on = on != 0;
}

extern "C" void svt_profile_reset(void) {
  std::lock_guard<std::mutex> lk(svt::g_prof_mu);
  svt::g_prof.clear();
}

extern "C" int svt_profile_read(int cap, char* names, int64_t* launches, double* ms, double* bytes) {
  svt::prof_flush();
  std::lock_guard<std::mutex> lk(svt::g_prof_mu);
  const int count = (int)svt::g_prof.size();
  for (int i = 0; i < count && i < cap; ++i) {
    if (names) memcpy(names + 32 * i, svt::g_prof[i].name, 32);
    if (launches) launches[i] = svt::g_prof[i].launches;
    if (ms) ms[i] = svt::g_prof[i].ms;
    if (bytes) bytes[i] = svt::g_prof[i].bytes;
  }
  return count;
}

extern "C" int64_t svt_launch_count(void) { return svt::g_launches.load(); }
