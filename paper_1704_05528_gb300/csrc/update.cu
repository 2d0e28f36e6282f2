// Sampled shrinkage and dual update on the observed set (eq. (4)-(5)) plus reductions.
//
// X^(i) = D_tau(Y^(i)) is kept in factored form U W^T with U the m x k left singular
// vectors and W = V_K diag(sigma_K - tau) (n x k); it is only ever evaluated on Lambda.
// One warp owns a CSR row p; its lanes take the row's entries in turn, evaluate
// x_pq = U[p, :] . W[q, :], d = A_pq - x_pq, update Y_pq += delta d and accumulate
// sum d^2 (the residual of Algorithm 4), sum |d| (MAE) and sum Y_new^2 (the next
// ||Y||_F^2 of R4SVD).  Binary64 data sums in binary64; binary32 data sums in pairs of
// binary32 values with error-free updates, which keeps about 2^-44 of relative accuracy
// on the binary32 pipes (binary64 arithmetic runs at a small fraction of the binary32
// rate on this GPU, and one binary64 operation per entry already bounds the kernel).
// Block partials are summed in block order by a second pass, so the sums are
// reproducible.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

constexpr int kRedBlocksPerSm = 8;

int red_blocks() { return num_sms() * kRedBlocksPerSm; }

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

template <typename T, int VEC>
__device__ __forceinline__ void load_v(const T* p, T (&v)[VEC]) {
  if constexpr (VEC == 1) {
    v[0] = p[0];
  } else if constexpr (VEC == 2) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
}

// Entries are split into chunks of C (warp w takes chunks w, w + #warps, ...).  Groups of
// G lanes evaluate one entry each, UNR entries per group per step, so 32/G * UNR entries
// (and their row gathers) are in flight per warp; all loads of a step are issued before
// the dependent arithmetic.  Lane l of a group holds vectors l, l+G, ... (VEC elements
// each) of U[p, :] for the current row p (read from the stored row of each entry,
// reloaded when it changes) and multiplies them with the same slices of W[q, :]; a
// shuffle tree over the group gives x_pq.  Loop trip counts are uniform across the warp
// so every lane reaches the shuffles.
template <typename T, int VEC, int G, int MAXV, int UNR, bool WPAD>
__global__ void __launch_bounds__(256)
k_sampled_update(int64_t nnz, int64_t C, int64_t nchunks, const int32_t* __restrict__ csr_row,
                 const int32_t* __restrict__ col_idx, const T* __restrict__ U, int64_t ldu,
                 const T* __restrict__ W, int64_t ldw, int k, const T* __restrict__ a,
                 T* __restrict__ y, T delta, double* __restrict__ part, unsigned* __restrict__ flags) {
  __shared__ double red[32];
  constexpr int NG = 32 / G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane % G;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  SumAcc<T> acc_d2, acc_abs, acc_y2;
  bool bad = false;
  for (int64_t chunk = wid; chunk < nchunks; chunk += nw) {
    const int64_t beg = chunk * C;
    const int64_t end = (beg + C < nnz) ? beg + C : nnz;
    int64_t r = -1;
    T u[MAXV][VEC];
    for (int64_t base = beg; base < end; base += NG * UNR) {
      // 1. independent loads of UNR entries per group
      int64_t e[UNR];
      bool v[UNR];
      int32_t row[UNR], col[UNR];
      T av[UNR], yv[UNR];
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        e[j] = base + j * NG + grp;
        v[j] = e[j] < end;
        row[j] = v[j] ? csr_row[e[j]] : 0;
        col[j] = v[j] ? col_idx[e[j]] : 0;
        av[j] = v[j] ? a[e[j]] : T(0);
        yv[j] = v[j] ? y[e[j]] : T(0);
      }
      // 2. gathers of the W rows (independent of each other)
      T wx[UNR][MAXV][VEC];
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        const T* wq = W + (int64_t)col[j] * ldw;
#pragma unroll
        for (int t = 0; t < MAXV; ++t) {
          const int c0 = (gl + t * G) * VEC;
          if (v[j] && c0 < k) load_v<T, VEC>(wq + c0, wx[j][t]);  // may read padding: masked below
          else {
#pragma unroll
            for (int bb = 0; bb < VEC; ++bb) wx[j][t][bb] = T(0);
          }
        }
      }
      // 3. dot products with this lane's slices of U[row, :k] (reloaded on a new row)
      T px[UNR];
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        px[j] = T(0);
        if (v[j]) {
          if (row[j] != r) {
            r = row[j];
            const T* up = U + r * ldu;
#pragma unroll
            for (int t = 0; t < MAXV; ++t) {
              const int c0 = (gl + t * G) * VEC;
              if (c0 < k) {
                load_v<T, VEC>(up + c0, u[t]);
#pragma unroll
                for (int bb = 0; bb < VEC; ++bb)
                  if (c0 + bb >= k) u[t][bb] = T(0);
              } else {
#pragma unroll
                for (int bb = 0; bb < VEC; ++bb) u[t][bb] = T(0);
              }
            }
          }
#pragma unroll
          for (int t = 0; t < MAXV; ++t) {
            const int c0 = (gl + t * G) * VEC;
#pragma unroll
            for (int bb = 0; bb < VEC; ++bb) {
              // WPAD: W's columns up to the next vector boundary are finite (zeros) and u
              // is zero there, so whole vectors multiply without a per-element test
              if (WPAD || c0 + bb < k) px[j] = fma(u[t][bb], wx[j][t][bb], px[j]);
            }
          }
        }
      }
      // 4. group reductions (every lane takes part)
#pragma unroll
      for (int j = 0; j < UNR; ++j)
#pragma unroll
        for (int o = 1; o < G; o <<= 1) px[j] += __shfl_xor_sync(0xffffffffu, px[j], o);
      // 5. residual and dual update: lane j0 + l of a group takes entry j0 + l, so the
      //    group's UNR entries finish in one instruction stream
#pragma unroll
      for (int j0 = 0; j0 < UNR; j0 += G) {
        T xs = T(0), as = T(0), ys = T(0);
        int64_t es = 0;
        bool vs = false;
#pragma unroll
        for (int j = j0; j < UNR && j < j0 + G; ++j)
          if (gl == j - j0) { xs = px[j]; as = av[j]; ys = yv[j]; es = e[j]; vs = v[j]; }
        if (vs) {
          const T d = as - xs;
          const T yn = fma(delta, d, ys);
          y[es] = yn;
          acc_d2.add_sq(d);
          acc_abs.add(fabs(d));
          acc_y2.add_sq(yn);
          bad |= !isfinite(yn);
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_NONFINITE);
  double s_d2 = acc_d2.value(), s_abs = acc_abs.value(), s_y2 = acc_y2.value();
  s_d2 = block_sum(s_d2, red);
  __syncthreads();
  s_abs = block_sum(s_abs, red);
  __syncthreads();
  s_y2 = block_sum(s_y2, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 3 + 0] = s_d2;
    part[blockIdx.x * 3 + 1] = s_abs;
    part[blockIdx.x * 3 + 2] = s_y2;
  }
}

template <typename T>
__global__ void k_sumsq_part(int64_t count, const T* __restrict__ x, double* __restrict__ part,
                             unsigned* __restrict__ flags) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[i];
    s = fma(v, v, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[c] = sum_b part[b * stride + c] for c < ncomp (one block per component): thread t
// adds blocks t, t + 256, ... in order, then a fixed shuffle tree combines the threads,
// so the sum does not depend on scheduling.
__global__ void __launch_bounds__(256)
k_finish(int nblocks, int stride, int ncomp, const double* __restrict__ part,
         double* __restrict__ out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[(int64_t)b * stride + c];
  s = block_sum(s, red);
  if (threadIdx.x == 0 && c < ncomp) out[c] = s;
}

template <typename T>
__global__ void k_scale_copy(int64_t count, const T* __restrict__ a, double scale, T* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (T)(scale * (double)a[i]);
}

template <typename TS, typename T>
__global__ void k_gather_convert(int64_t count, const int32_t* __restrict__ src,
                                 const TS* __restrict__ vals, T* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)vals[src[i]];
}

int grid_for(int64_t work, int per_sm) {
  int64_t g = ceil_div(work > 0 ? work : 1, 256);
  const int64_t cap = (int64_t)num_sms() * per_sm;
  return (int)(g < cap ? g : cap);
}

}  // namespace

size_t reduce_scratch() { return (size_t)red_blocks() * 3 + 8; }

template <typename T>
svt_status sumsq(int64_t count, const T* x, double* out, double* part, cudaStream_t s) {
  const int blocks = red_blocks();
  k_sumsq_part<T><<<blocks, 256, 0, s>>>(count, x, part, nullptr);
  SVT_LAUNCH_CHECK();
  k_finish<<<1, 256, 0, s>>>(blocks, 1, 1, part, out);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template <typename T>
svt_status scale_copy(int64_t count, const T* a, double scale, T* y, cudaStream_t s) {
  if (count <= 0) return SVT_OK;
  k_scale_copy<T><<<grid_for(count, 16), 256, 0, s>>>(count, a, scale, y);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template <typename TS, typename T>
svt_status gather_convert(int64_t count, const int32_t* src, const TS* vals, T* a_csr,
                          cudaStream_t s) {
  if (count <= 0) return SVT_OK;
  k_gather_convert<TS, T><<<grid_for(count, 16), 256, 0, s>>>(count, src, vals, a_csr);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template <typename T, int VEC, int G, int MAXV, bool WPAD>
svt_status run_update(const svt_pattern* p, const T* U, int64_t ldu, const T* W, int64_t ldw,
                      int k, const T* a, T* y, double delta, double* part, unsigned* flags,
                      cudaStream_t s) {
  const int blocks = red_blocks();
  const int64_t C = chunk_size(p->nnz > 0 ? p->nnz : 1);
  const int64_t nchunks = ceil_div(p->nnz, C);
  constexpr int UNR = (MAXV * VEC <= 16) ? 2 : 1;
  k_sampled_update<T, VEC, G, MAXV, UNR, WPAD><<<blocks, 256, 0, s>>>(p->nnz, C, nchunks, p->csr_row,
                                                                p->col_idx, U, ldu, W, ldw, k, a, y,
                                                                (T)delta, part, flags);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template <typename T, int VEC, bool WPAD>
svt_status dispatch_update(const svt_pattern* p, const T* U, int64_t ldu, const T* W, int64_t ldw,
                           int k, const T* a, T* y, double delta, double* part, unsigned* flags,
                           cudaStream_t s) {
  const int nv = (int)ceil_div(k > 0 ? k : 1, VEC);
  // at most 4 vectors per lane, as few lanes per entry as that allows
#define SVT_RUN(G, MV) return run_update<T, VEC, G, MV, WPAD>(p, U, ldu, W, ldw, k, a, y, delta, part, flags, s)
  if (nv <= 4) SVT_RUN(1, 4);
  if (nv <= 8) SVT_RUN(2, 4);
  if (nv <= 16) SVT_RUN(4, 4);
  if (nv <= 32) SVT_RUN(8, 4);
  if (nv <= 64) SVT_RUN(16, 4);
  if (nv <= 128) SVT_RUN(32, 4);
  if (nv <= 256) SVT_RUN(32, 8);
  if (nv <= 512) SVT_RUN(32, 16);
  SVT_RUN(32, 32);
#undef SVT_RUN
}

template <typename T>
svt_status sampled_update(const svt_pattern* p, const T* U, int64_t ldu, const T* W,
                          int64_t ldw, int k, const T* a, T* y, double delta, double* out3,
                          double* part, unsigned* flags, cudaStream_t s, bool w_pad_zero) {
  if (k > 1024) return fail(SVT_ERR_UNSUPPORTED, "sampled update: k = %d exceeds 1024", k);
  constexpr int V = sizeof(T) == 4 ? 4 : 2;
  const bool aligned = (reinterpret_cast<uintptr_t>(U) % 16 == 0) && (ldu % V == 0) &&
                       (reinterpret_cast<uintptr_t>(W) % 16 == 0) && (ldw % V == 0) &&
                       (!w_pad_zero || ldw >= round_up(k, 4));
  if (p->nnz > 0) {
    if (aligned && w_pad_zero)
      SVT_TRY((dispatch_update<T, V, true>(p, U, ldu, W, ldw, k, a, y, delta, part, flags, s)));
    else if (aligned)
      SVT_TRY((dispatch_update<T, V, false>(p, U, ldu, W, ldw, k, a, y, delta, part, flags, s)));
    else SVT_TRY((dispatch_update<T, 1, false>(p, U, ldu, W, ldw, k, a, y, delta, part, flags, s)));
  } else {
    SVT_CUDA(cudaMemsetAsync(part, 0, 3 * red_blocks() * sizeof(double), s));
  }
  k_finish<<<3, 256, 0, s>>>(red_blocks(), 3, 3, part, out3);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template svt_status sumsq<double>(int64_t, const double*, double*, double*, cudaStream_t);
template svt_status sumsq<float>(int64_t, const float*, double*, double*, cudaStream_t);
template svt_status scale_copy<double>(int64_t, const double*, double, double*, cudaStream_t);
template svt_status scale_copy<float>(int64_t, const float*, double, float*, cudaStream_t);
template svt_status gather_convert<double, double>(int64_t, const int32_t*, const double*, double*,
                                                   cudaStream_t);
template svt_status gather_convert<float, float>(int64_t, const int32_t*, const float*, float*,
                                                 cudaStream_t);
template svt_status sampled_update<double>(const svt_pattern*, const double*, int64_t,
                                           const double*, int64_t, int, const double*, double*,
                                           double, double*, double*, unsigned*, cudaStream_t, bool);
template svt_status sampled_update<float>(const svt_pattern*, const float*, int64_t, const float*,
                                          int64_t, int, const float*, float*, double, double*,
                                          double*, unsigned*, cudaStream_t, bool);

}  // namespace svt
