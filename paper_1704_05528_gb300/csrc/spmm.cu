// Sparse (Y on Lambda) times tall-skinny dense block: the matrix-block products that
// dominate Algorithms 1-3 (O((np+2) r T_mult), Section 2.2).
//
// One warp per compressed row (a row of Y in CSR order for Y W, a column of Y in CSC
// order for Y^T W).  The warp is split into 32/G groups of G lanes; each group walks
// every (32/G)-th entry of the row and its lanes cover the block's columns
// (lane, lane + G, ...), so one gathered row of W is read with consecutive lanes.
// The groups' partial sums are combined by a fixed xor-shuffle tree, so results are
// reproducible run to run.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

template <typename TV, typename TD, int G, int MAXC>
__global__ void __launch_bounds__(256)
k_spmm_rows(int64_t nrows, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
            const TV* __restrict__ val, const TD* __restrict__ W, int64_t ldw, int w,
            TD* __restrict__ out, int64_t ldo) {
  constexpr int NG = 32 / G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane % G;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = wid; row < nrows; row += nw) {
    TD acc[MAXC];
#pragma unroll
    for (int t = 0; t < MAXC; ++t) acc[t] = TD(0);
    const int beg = ptr[row], end = ptr[row + 1];
    for (int e = beg + grp; e < end; e += NG) {
      const TD v = (TD)val[e];
      const TD* wr = W + (int64_t)idx[e] * ldw;
#pragma unroll
      for (int t = 0; t < MAXC; ++t) {
        const int col = gl + t * G;
        if (col < w) acc[t] = fma(v, wr[col], acc[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < MAXC; ++t) {
#pragma unroll
      for (int o = G; o < 32; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    }
    if (grp == 0) {
#pragma unroll
      for (int t = 0; t < MAXC; ++t) {
        const int col = gl + t * G;
        if (col < w) out[row * ldo + col] = acc[t];
      }
    }
  }
}

template <typename T>
__global__ void k_gather(int64_t count, const int32_t* __restrict__ perm, const T* __restrict__ src,
                         T* __restrict__ dst) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = src[perm[q]];
}

template <typename TV, typename TD, int G, int MAXC>
svt_status run_spmm(int64_t nrows, const int32_t* ptr, const int32_t* idx, const TV* val,
                    const TD* W, int64_t ldw, int w, TD* out, int64_t ldo, cudaStream_t s) {
  const int64_t warps_wanted = nrows;
  const int64_t warps_cap = (int64_t)num_sms() * 64;
  const int64_t warps = warps_wanted < warps_cap ? warps_wanted : warps_cap;
  const int blocks = (int)ceil_div(warps, 8);
  k_spmm_rows<TV, TD, G, MAXC><<<blocks, 256, 0, s>>>(nrows, ptr, idx, val, W, ldw, w, out, ldo);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

}  // namespace

template <typename TV, typename TD>
svt_status launch_spmm_rows(int64_t nrows, const int32_t* ptr, const int32_t* idx,
                            const TV* val, const TD* W, int64_t ldw, int w, TD* out,
                            int64_t ldo, cudaStream_t s) {
  if (nrows <= 0 || w <= 0) return SVT_OK;
  for (int c0 = 0; c0 < w; c0 += 512) {
    const int wc = (w - c0) < 512 ? (w - c0) : 512;
    const TD* Wc = W + c0;
    TD* oc = out + c0;
    svt_status st;
    if (wc == 1) st = run_spmm<TV, TD, 1, 1>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else if (wc == 2) st = run_spmm<TV, TD, 2, 1>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else if (wc <= 4) st = run_spmm<TV, TD, 4, 1>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else if (wc <= 8) st = run_spmm<TV, TD, 8, 1>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else if (wc <= 16) st = run_spmm<TV, TD, 16, 1>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else if (wc <= 32) st = run_spmm<TV, TD, 32, 1>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else if (wc <= 64) st = run_spmm<TV, TD, 32, 2>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else if (wc <= 128) st = run_spmm<TV, TD, 32, 4>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else if (wc <= 256) st = run_spmm<TV, TD, 32, 8>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    else st = run_spmm<TV, TD, 32, 16>(nrows, ptr, idx, val, Wc, ldw, wc, oc, ldo, s);
    if (st < 0) return st;
  }
  return SVT_OK;
}

template <typename T>
svt_status launch_gather(int64_t count, const int32_t* perm, const T* src, T* dst,
                         cudaStream_t s) {
  if (count <= 0) return SVT_OK;
  int64_t g = ceil_div(count, 256);
  const int64_t cap = (int64_t)num_sms() * 32;
  if (g > cap) g = cap;
  k_gather<T><<<(int)g, 256, 0, s>>>(count, perm, src, dst);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template svt_status launch_spmm_rows<double, double>(int64_t, const int32_t*, const int32_t*,
                                                     const double*, const double*, int64_t, int,
                                                     double*, int64_t, cudaStream_t);
template svt_status launch_spmm_rows<float, float>(int64_t, const int32_t*, const int32_t*,
                                                   const float*, const float*, int64_t, int,
                                                   float*, int64_t, cudaStream_t);
template svt_status launch_spmm_rows<float, double>(int64_t, const int32_t*, const int32_t*,
                                                    const float*, const double*, int64_t, int,
                                                    double*, int64_t, cudaStream_t);
template svt_status launch_gather<double>(int64_t, const int32_t*, const double*, double*,
                                          cudaStream_t);
template svt_status launch_gather<float>(int64_t, const int32_t*, const float*, float*,
                                         cudaStream_t);

}  // namespace svt
