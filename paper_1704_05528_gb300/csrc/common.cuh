// Shared device helpers, error plumbing and the scratch arena of the SVT library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <cstdio>

#include "svt_gb300.h"

namespace svt {

// ---------------------------------------------------------------- error plumbing
void set_error(const char* fmt, ...);
svt_status fail(svt_status code, const char* fmt, ...);
svt_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define SVT_CUDA(expr)                                                        \
  do {                                                                        \
    cudaError_t svt_e_ = (expr);                                              \
    if (svt_e_ != cudaSuccess) return ::svt::cuda_fail(svt_e_, #expr, __FILE__, __LINE__); \
  } while (0)

// Every kernel launch site is followed by this check; it also counts the launch.
void count_launch();
// Adjusts the launch counter (a captured graph's kernels are counted at each launch of
// the graph, not when they are recorded).
void count_launches(int64_t delta);
int64_t launches_so_far();
#define SVT_LAUNCH_CHECK()        \
  do {                            \
    ::svt::count_launch();        \
    SVT_CUDA(cudaGetLastError()); \
  } while (0)

#define SVT_TRY(expr)                                                         \
  do {                                                                        \
    svt_status svt_s_ = (expr);                                               \
    if (svt_s_ < 0) return svt_s_;                                            \
  } while (0)

int num_sms();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of one double per thread (blockDim.x a multiple of 32, <= 1024).
// Deterministic: fixed shuffle tree, then warp partials summed in warp order.
__device__ __forceinline__ double block_sum(double v, double* smem32) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) smem32[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? smem32[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0 (and the whole of warp 0)
}

// Running sums of the sampled updates.  Binary64 data sum in binary64; binary32 data sum in
// an unevaluated pair hi + lo of binary32 values.
template <typename T>
struct SumAcc;

template <>
struct SumAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_sq(double x) { s = fma(x, x, s); }
  __device__ __forceinline__ double value() const { return s; }
};

// hi + lo holds the sum.  Knuth's TwoSum gives the exact error of hi + p, and fma gives
// the exact error of a rounded product; the intrinsics keep the compiler from fusing
// the steps that must round separately.
template <>
struct SumAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add2(float p, float e) {
    const float t = __fadd_rn(hi, p);
    const float z = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    lo = __fadd_rn(lo, __fadd_rn(err, e));
    hi = t;
  }
  __device__ __forceinline__ void add(float x) { add2(x, 0.f); }
  __device__ __forceinline__ void add_sq(float x) {
    const float p = __fmul_rn(x, x);
    add2(p, fmaf(x, x, -p));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------- device flags
// Bits raised by kernels into a device status word and read back by the host.
// Words of the device status array of a solve.
constexpr int kFlagWords = 8;
enum : unsigned {
  FLAG_INDEX = 1u,       // index out of range in the pattern input
  FLAG_DUPLICATE = 2u,   // duplicate (row, col)
  FLAG_NONFINITE = 4u,   // non-finite value met in a reduction
  FLAG_CHOLESKY = 8u,    // non-positive pivot in a small Cholesky factorisation
  FLAG_TC_TIMEOUT = 16u, // a bounded wait of the tensor-core lift ran out (result not written)
  FLAG_GRID_TIMEOUT = 32u, // a grid barrier of the cooperative Jacobi ran out
};

// ---------------------------------------------------------------- scratch arena
// Sub-allocates 256-byte aligned slices from one stream-ordered device block.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = round_up((int64_t)(count * sizeof(T)), 256);
    if (bytes == 0) bytes = 256;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

// A caller-owned device workspace, used as a stack by the call that received it: while a
// WorkspaceScope is alive on a thread, every DeviceBlock allocated on that thread is carved
// from the top of the workspace and released in reverse order.
struct Workspace {
  char* base = nullptr;
  size_t cap = 0;
  size_t top = 0;
};
Workspace* current_workspace();
struct WorkspaceScope {
  Workspace ws;
  Workspace* prev;
  WorkspaceScope(void* base, size_t bytes);
  ~WorkspaceScope();
  WorkspaceScope(const WorkspaceScope&) = delete;
  WorkspaceScope& operator=(const WorkspaceScope&) = delete;
};

// RAII owner of device scratch: a stream-ordered allocation, or a slice of the thread's
// current workspace.
struct DeviceBlock {
  void* ptr = nullptr;
  cudaStream_t stream = nullptr;
  Workspace* ws = nullptr;    // non-null: a slice of this workspace
  size_t ws_prev_top = 0, ws_end = 0;
  DeviceBlock() = default;
  DeviceBlock(const DeviceBlock&) = delete;
  DeviceBlock& operator=(const DeviceBlock&) = delete;
  ~DeviceBlock() { release(); }
  void release() {
    if (ws) {
      if (ws->top == ws_end) ws->top = ws_prev_top;  // blocks are released in reverse order
      ws = nullptr;
    } else if (ptr) {
      cudaFreeAsync(ptr, stream);
    }
    ptr = nullptr;
  }
  svt_status alloc(size_t bytes, cudaStream_t s);
};

// Memory location of a user pointer (host or device).
bool is_device_pointer(const void* p);

}  // namespace svt

// The pattern object behind the opaque ABI handle.
struct svt_pattern {
  int64_t m = 0, n = 0, nnz = 0;
  int32_t* row_ptr = nullptr;   // m+1
  int32_t* col_idx = nullptr;   // nnz, CSR
  int32_t* csr_src = nullptr;   // nnz, input position of each CSR slot
  int32_t* col_ptr = nullptr;   // n+1
  int32_t* row_idx = nullptr;   // nnz, CSC
  int32_t* perm = nullptr;      // nnz, CSR slot of each CSC slot
  int32_t* csr_row = nullptr;   // nnz, row of each CSR slot
  int64_t chunk = 0;            // entries per work chunk of the entry-balanced kernels
  int64_t nchunks = 0;
  int32_t* chunk_row_csr = nullptr;  // first CSR row touched by each chunk
  int32_t* chunk_row_csc = nullptr;  // first CSC column touched by each chunk
  void* block = nullptr;        // single device allocation holding the arrays
  svt::DeviceBlock ws_block;    // or: the arrays' slice of a caller workspace
};
