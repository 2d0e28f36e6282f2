// Sampled shrinkage and dual update on the observed set (eq. (4)-(5)) plus reductions.
//
// X^(i) = D_tau(Y^(i)) is kept in factored form U W^T with U the m x k left singular
// vectors and W = V_K diag(sigma_K - tau) (n x k); it is only ever evaluated on Lambda.
// One warp owns a CSR row p; its lanes take the row's entries in turn, evaluate
// x_pq = U[p, :] . W[q, :], d = A_pq - x_pq, update Y_pq += delta d and accumulate
// sum d^2 (the residual of Algorithm 4), sum |d| (MAE) and sum Y_new^2 (the next
// ||Y||_F^2 of R4SVD) in binary64.  Block partials are summed in block order by a
// second pass, so the sums are reproducible.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

constexpr int kRedBlocksPerSm = 8;

int red_blocks() { return num_sms() * kRedBlocksPerSm; }

template <typename T>
__global__ void __launch_bounds__(256)
k_sampled_update(int64_t m, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                 const T* __restrict__ U, int64_t ldu, const T* __restrict__ W, int64_t ldw, int k,
                 const T* __restrict__ a, T* __restrict__ y, T delta, double* __restrict__ part,
                 unsigned* __restrict__ flags) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double s_d2 = 0.0, s_abs = 0.0, s_y2 = 0.0;
  bool bad = false;
  for (int64_t p = wid; p < m; p += nw) {
    const int beg = row_ptr[p], end = row_ptr[p + 1];
    const T* up = U + p * ldu;
    for (int e = beg + lane; e < end; e += 32) {
      const T* wq = W + (int64_t)col_idx[e] * ldw;
      T x = T(0);
      for (int j = 0; j < k; ++j) x = fma(up[j], wq[j], x);
      const T d = a[e] - x;
      const T yn = fma(delta, d, y[e]);
      y[e] = yn;
      const double dd = (double)d, yy = (double)yn;
      s_d2 = fma(dd, dd, s_d2);
      s_abs += fabs(dd);
      s_y2 = fma(yy, yy, s_y2);
      bad |= !isfinite(yy);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_NONFINITE);
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

// out[c] = sum_b part[b * stride + c] for c < ncomp, in block order.
__global__ void k_finish(int nblocks, int stride, int ncomp, const double* __restrict__ part,
                         double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c < ncomp) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * stride + c];
    out[c] = s;
  }
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
  k_finish<<<1, 32, 0, s>>>(blocks, 1, 1, part, out);
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

template <typename T>
svt_status sampled_update(const svt_pattern* p, const T* U, int64_t ldu, const T* W,
                          int64_t ldw, int k, const T* a, T* y, double delta, double* out3,
                          double* part, unsigned* flags, cudaStream_t s) {
  const int blocks = red_blocks();
  k_sampled_update<T><<<blocks, 256, 0, s>>>(p->m, p->row_ptr, p->col_idx, U, ldu, W, ldw, k, a,
                                             y, (T)delta, part, flags);
  SVT_LAUNCH_CHECK();
  k_finish<<<1, 32, 0, s>>>(blocks, 3, 3, part, out3);
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
                                           double, double*, double*, unsigned*, cudaStream_t);
template svt_status sampled_update<float>(const svt_pattern*, const float*, int64_t, const float*,
                                          int64_t, int, const float*, float*, double, double*,
                                          double*, unsigned*, cudaStream_t);

}  // namespace svt
