// Dense tall-skinny kernels of R4SVD (Algorithms 2-3): block orthogonalisation
// X <- X - Q (Q^T X), Cholesky-QR of the new block, the Gram matrix of B and the
// products U = Q U_B, V = B^T U_B Sigma^-1.
//
// gemm_tn: C = A^T B with the long dimension M split across blocks; each block writes a
//          binary64 partial tile and a second pass sums the partials in split order, so
//          the result does not depend on scheduling.  Binary32 inputs are accumulated
//          with error-free products and TwoSum in binary32 pairs (binary64-accurate at
//          binary32 speed); a Gram matrix (A == B) computes its upper tiles only.
// gemm_nn: C = alpha A B + beta Cin, A tall (M x p), B small binary64 (p x q), tiled
//          64 x 32 per block through shared memory.
// chol_inv: one-block Cholesky G = R^T R of a small SPD matrix and R^-1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

constexpr int TN_TILE = 32;

// Error-free accumulation in binary32 pairs: the product p = a*b is rounded and its error
// e = fma(a, b, -p) is exact; p enters hi by Knuth's TwoSum (exact), the two errors
// gather in lo.  hi + lo tracks the sum to about 2^-44 relative, at binary32 speed.
__device__ __forceinline__ void dd_fma(float a, float b, float& hi, float& lo) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float t = hi + p;
  const float z = t - hi;
  const float err = (hi - (t - z)) + (p - z);
  hi = t;
  lo += err + e;
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256)
k_gemm_tn_part(int64_t M, int p, int q, const TA* __restrict__ A, int64_t lda,
               const TB* __restrict__ B, int64_t ldb, int64_t rows_per_split,
               double* __restrict__ part, int symmetric) {
  // A symmetric product (A == B) computes its upper tiles only (lower tiles mirror them):
  // blockIdx.x then enumerates the tiles ta <= tb row by row, so that every CTA of the
  // grid has work and the CTAs spread evenly over the SMs.
  int ta = blockIdx.x, tb = blockIdx.y;
  if (symmetric) {
    const int T = (p + TN_TILE - 1) / TN_TILE;
    int t = blockIdx.x;
    ta = 0;
    while (t >= T - ta) { t -= T - ta; ++ta; }
    tb = ta + t;
  }
  constexpr bool kF32 = sizeof(TA) == 4 && sizeof(TB) == 4;
  using TS = typename std::conditional<kF32, float, double>::type;
  __shared__ TS As[TN_TILE][TN_TILE + 1];
  __shared__ TS Bs[TN_TILE][TN_TILE + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int a0 = ta * TN_TILE, b0 = tb * TN_TILE;
  const int64_t i_beg = (int64_t)blockIdx.z * rows_per_split;
  int64_t i_end = i_beg + rows_per_split;
  if (i_end > M) i_end = M;
  TS acc[4] = {TS(0), TS(0), TS(0), TS(0)};
  TS lo[4] = {TS(0), TS(0), TS(0), TS(0)};
  for (int64_t i0 = i_beg; i0 < i_end; i0 += TN_TILE) {
    for (int t = threadIdx.x; t < TN_TILE * TN_TILE; t += blockDim.x) {
      const int rr = t / TN_TILE, cc = t % TN_TILE;
      const int64_t i = i0 + rr;
      const bool in = i < i_end;
      As[rr][cc] = (in && a0 + cc < p) ? (TS)A[i * lda + a0 + cc] : TS(0);
      Bs[rr][cc] = (in && b0 + cc < q) ? (TS)B[i * ldb + b0 + cc] : TS(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TN_TILE; ++kk) {
      const TS x0 = As[kk][ty], x1 = As[kk][ty + 16];
      const TS y0 = Bs[kk][tx], y1 = Bs[kk][tx + 16];
      if constexpr (kF32) {
        dd_fma(x0, y0, acc[0], lo[0]);
        dd_fma(x0, y1, acc[1], lo[1]);
        dd_fma(x1, y0, acc[2], lo[2]);
        dd_fma(x1, y1, acc[3], lo[3]);
      } else {
        acc[0] = fma(x0, y0, acc[0]);
        acc[1] = fma(x0, y1, acc[1]);
        acc[2] = fma(x1, y0, acc[2]);
        acc[3] = fma(x1, y1, acc[3]);
      }
    }
    __syncthreads();
  }
  double* P = part + (int64_t)blockIdx.z * p * q;
  const int a_0 = a0 + ty, a_1 = a0 + ty + 16, b_0 = b0 + tx, b_1 = b0 + tx + 16;
  if (a_0 < p && b_0 < q) P[(int64_t)a_0 * q + b_0] = (double)acc[0] + (double)lo[0];
  if (a_0 < p && b_1 < q) P[(int64_t)a_0 * q + b_1] = (double)acc[1] + (double)lo[1];
  if (a_1 < p && b_0 < q) P[(int64_t)a_1 * q + b_0] = (double)acc[2] + (double)lo[2];
  if (a_1 < p && b_1 < q) P[(int64_t)a_1 * q + b_1] = (double)acc[3] + (double)lo[3];
}

// The binary32 case of k_gemm_tn_part with four times the work per thread: a 32 x 32
// output tile per block of 64 threads, 4 x 4 outputs per thread (rows ty + 8a, columns
// tx + 8b), so that each step reads 8 values from shared memory for 16 error-free products
// (the same accumulation per output as k_gemm_tn_part).
__global__ void __launch_bounds__(64)
k_gemm_tn_part4(int64_t M, int p, int q, const float* __restrict__ A, int64_t lda,
                const float* __restrict__ B, int64_t ldb, int64_t rows_per_split,
                double* __restrict__ part, int symmetric) {
  int ta = blockIdx.x, tb = blockIdx.y;
  if (symmetric) {
    const int T = (p + TN_TILE - 1) / TN_TILE;
    int t = blockIdx.x;
    ta = 0;
    while (t >= T - ta) { t -= T - ta; ++ta; }
    tb = ta + t;
  }
  __shared__ float As[TN_TILE][TN_TILE + 1];
  __shared__ float Bs[TN_TILE][TN_TILE + 1];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int a0 = ta * TN_TILE, b0 = tb * TN_TILE;
  const int64_t i_beg = (int64_t)blockIdx.z * rows_per_split;
  int64_t i_end = i_beg + rows_per_split;
  if (i_end > M) i_end = M;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { hi[a][b] = 0.f; lo[a][b] = 0.f; }
  for (int64_t i0 = i_beg; i0 < i_end; i0 += TN_TILE) {
    for (int t = threadIdx.x; t < TN_TILE * TN_TILE; t += blockDim.x) {
      const int rr = t / TN_TILE, cc = t % TN_TILE;
      const int64_t i = i0 + rr;
      const bool in = i < i_end;
      As[rr][cc] = (in && a0 + cc < p) ? A[i * lda + a0 + cc] : 0.f;
      Bs[rr][cc] = (in && b0 + cc < q) ? B[i * ldb + b0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TN_TILE; ++kk) {
      float x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) x[a] = As[kk][ty + 8 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) y[b] = Bs[kk][tx + 8 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dd_fma(x[a], y[b], hi[a][b], lo[a][b]);
    }
    __syncthreads();
  }
  double* P = part + (int64_t)blockIdx.z * p * q;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int ia = a0 + ty + 8 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int jb = b0 + tx + 8 * b;
      if (ia < p && jb < q) P[(int64_t)ia * q + jb] = (double)hi[a][b] + (double)lo[a][b];
    }
  }
}

// C[a][b] = sum_z part[z][a][b]; for a symmetric product the lower tiles read the
// mirrored upper entry.
__global__ void k_reduce_parts(int p, int q, int splits, const double* __restrict__ part,
                               double* __restrict__ C, int64_t ldc, int symmetric) {
  const int64_t pq = (int64_t)p * q;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pq;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t / q, b = t % q;
    const int64_t src = (symmetric && (a / TN_TILE) > (b / TN_TILE)) ? b * q + a : t;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * pq + src];
    C[a * ldc + b] = s;
  }
}

// The same sums when there are many splits and few outputs: one warp per output, lane l
// adding splits l, l + 32, ... in order, then a fixed shuffle tree.
__global__ void k_reduce_parts_warp(int p, int q, int splits, const double* __restrict__ part,
                                    double* __restrict__ C, int64_t ldc, int symmetric) {
  const int64_t pq = (int64_t)p * q;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < pq; t += nw) {
    const int64_t a = t / q, b = t % q;
    const int64_t src = (symmetric && (a / TN_TILE) > (b / TN_TILE)) ? b * q + a : t;
    double s = 0.0;
    for (int z = lane; z < splits; z += 32) s += part[(int64_t)z * pq + src];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) C[a * ldc + b] = s;
  }
}

int grid_cap(int64_t work, int threads, int per_sm);

void launch_reduce_parts(int p, int q, int splits, const double* part, double* C, int64_t ldc,
                         int symmetric, cudaStream_t s) {
  const int64_t pq = (int64_t)p * q;
  if (splits > 32 && pq <= 65536)
    k_reduce_parts_warp<<<grid_cap(pq * 32, 256, 8), 256, 0, s>>>(p, q, splits, part, C, ldc, symmetric);
  else
    k_reduce_parts<<<grid_cap(pq, 256, 8), 256, 0, s>>>(p, q, splits, part, C, ldc, symmetric);
}

int tn_splits(int64_t M, int p, int q) {
  const int64_t tiles = ceil_div(p, TN_TILE) * ceil_div(q, TN_TILE);
  int64_t want = ceil_div((int64_t)num_sms() * 4, tiles);
  const int64_t most = ceil_div(M, 64);  // at least 64 rows per split
  if (want > most) want = most;
  if (want < 1) want = 1;
  if (want > 4096) want = 4096;
  return (int)want;
}

template <typename TA, typename TC, typename TACC>
__global__ void __launch_bounds__(256)
k_gemm_nn(int64_t M, int p, int q, double alpha, const TA* __restrict__ A, int64_t lda,
          const double* __restrict__ B, int64_t ldb, double beta, const TC* Cin, int64_t ldcin,
          TC* C, int64_t ldc) {
  __shared__ TACC As[64][33];
  __shared__ TACC Bs[32][33];
  const int tx = threadIdx.x & 7;    // columns tx*4 .. tx*4+3
  const int ty = threadIdx.x >> 3;   // rows ty*2, ty*2+1
  const int64_t i0 = (int64_t)blockIdx.y * 64;
  const int j0 = blockIdx.x * 32;
  TACC acc[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = TACC(0);
  for (int k0 = 0; k0 < p; k0 += 32) {
    for (int t = threadIdx.x; t < 64 * 32; t += blockDim.x) {
      const int rr = t >> 5, cc = t & 31;
      const int64_t i = i0 + rr;
      As[rr][cc] = (i < M && k0 + cc < p) ? (TACC)A[i * lda + k0 + cc] : TACC(0);
    }
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
      const int rr = t >> 5, cc = t & 31;
      Bs[rr][cc] = (k0 + rr < p && j0 + cc < q) ? (TACC)B[(int64_t)(k0 + rr) * ldb + j0 + cc] : TACC(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const TACC x0 = As[ty * 2][kk], x1 = As[ty * 2 + 1][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const TACC y = Bs[kk][tx * 4 + b];
        acc[0][b] = fma(x0, y, acc[0][b]);
        acc[1][b] = fma(x1, y, acc[1][b]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int64_t i = i0 + ty * 2 + a;
    if (i >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx * 4 + b;
      if (j >= q) continue;
      double v = alpha * (double)acc[a][b];
      if (beta != 0.0) v += beta * (double)Cin[i * ldcin + j];
      C[i * ldc + j] = (TC)v;
    }
  }
}

// The binary32 case of k_gemm_nn: C = alpha A B + beta Cin with a 128 x 64 output tile per
// block and 8 x 4 outputs per thread (A staged k-major so each thread reads its 8 rows and
// 4 columns as float4), epilogue in binary32 (binary64 runs at a small fraction of the
// binary32 rate on this GPU).
__global__ void __launch_bounds__(256)
k_gemm_nn_f32(int64_t M, int p, int q, float alpha, const float* __restrict__ A, int64_t lda,
              const double* __restrict__ B, int64_t ldb, float beta, const float* Cin,
              int64_t ldcin, float* C, int64_t ldc) {
  __shared__ __align__(16) float As[32][132];  // As[k][row]
  __shared__ __align__(16) float Bs[32][64];   // Bs[k][col]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * 128;
  const int j0 = blockIdx.x * 64;
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < p; k0 += 32) {
    for (int t = threadIdx.x; t < 128 * 32; t += 256) {
      const int rr = t >> 5, cc = t & 31;
      const int64_t i = i0 + rr;
      As[cc][rr] = (i < M && k0 + cc < p) ? A[i * lda + k0 + cc] : 0.f;
    }
    for (int t = threadIdx.x; t < 32 * 64; t += 256) {
      const int rr = t >> 6, cc = t & 63;
      Bs[rr][cc] = (k0 + rr < p && j0 + cc < q) ? (float)B[(int64_t)(k0 + rr) * ldb + j0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
      const float4 bq = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t i = i0 + ty * 8 + a;
    if (i >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx * 4 + b;
      if (j >= q) continue;
      float v = alpha * acc[a][b];
      if (beta != 0.f) v = fmaf(beta, Cin[i * ldcin + j], v);
      C[i * ldc + j] = v;
    }
  }
}

template <typename T>
__global__ void k_colsumsq_part(int64_t M, int w, const T* __restrict__ X, int64_t ldx,
                                int64_t rows_per_block, double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  int64_t r1 = r0 + rows_per_block;
  if (r1 > M) r1 = M;
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    double s = 0.0;
    for (int64_t i = r0; i < r1; ++i) {
      const double v = (double)X[i * ldx + c];
      s = fma(v, v, s);
    }
    part[(int64_t)blockIdx.x * w + c] = s;
  }
}

template <typename TS, typename TD>
__global__ void k_copy_convert(int64_t M, int w, const TS* __restrict__ src, int64_t lds,
                               TD* __restrict__ dst, int64_t ldd) {
  const int64_t total = M * w;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / w;
    const int j = (int)(t - i * w);
    dst[i * ldd + j] = (TD)src[i * lds + j];
  }
}

// Right-looking Cholesky of G (w x w) into upper R, then R^-1 by rows from the bottom.
__global__ void k_chol_inv(int w, const double* __restrict__ G, int64_t ldg, double* __restrict__ R,
                           double* __restrict__ Rinv, double* __restrict__ work,
                           double* __restrict__ diag_min, unsigned* __restrict__ flags) {
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  // work holds the trailing matrix (w x w, full), R and Rinv are w x w row-major.
  for (int64_t t = threadIdx.x; t < (int64_t)w * w; t += blockDim.x) {
    const int a = (int)(t / w), b = (int)(t % w);
    work[t] = G[(int64_t)a * ldg + b];
    R[t] = 0.0;
    Rinv[t] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    if (threadIdx.x == 0) {
      const double d = work[(int64_t)j * w + j];
      if (!(d > 0.0) || !isfinite(d)) { bad = 1; piv = 0.0; }
      else piv = sqrt(d);
      R[(int64_t)j * w + j] = piv;
    }
    __syncthreads();
    if (bad) break;
    for (int c = j + 1 + threadIdx.x; c < w; c += blockDim.x)
      R[(int64_t)j * w + c] = work[(int64_t)j * w + c] / piv;
    __syncthreads();
    const int rem = w - j - 1;
    for (int64_t t = threadIdx.x; t < (int64_t)rem * rem; t += blockDim.x) {
      const int a = j + 1 + (int)(t / rem), b = j + 1 + (int)(t % rem);
      if (b >= a) work[(int64_t)a * w + b] -= R[(int64_t)j * w + a] * R[(int64_t)j * w + b];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) { atomicOr(flags, FLAG_CHOLESKY); *diag_min = 0.0; }
    return;
  }
  // R^-1: row i from the bottom; Rinv[i][c] = (delta_ic - sum_{k=i+1..c} R[i][k] Rinv[k][c]) / R[i][i]
  for (int i = w - 1; i >= 0; --i) {
    const double rii = R[(int64_t)i * w + i];
    for (int c = i + threadIdx.x; c < w; c += blockDim.x) {
      double s = (c == i) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) s -= R[(int64_t)i * w + k] * Rinv[(int64_t)k * w + c];
      Rinv[(int64_t)i * w + c] = s / rii;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double mn = R[0];
    for (int j = 1; j < w; ++j) mn = fmin(mn, R[(int64_t)j * w + j]);
    *diag_min = mn;
  }
}

int grid_cap(int64_t work, int threads, int per_sm) {
  int64_t g = ceil_div(work > 0 ? work : 1, threads);
  const int64_t cap = (int64_t)num_sms() * per_sm;
  return (int)(g < cap ? g : cap);
}

}  // namespace

// Bound valid for every p' <= p, q' <= q: splits * p' * q' <= (4 SMs + tiles) * 32 * 32.
// Splits of the binary32 kernel: about eight blocks of 64 threads per SM over the output
// tiles, at least 32 rows per split, and a partial-sum buffer of at most kTn4PartDoubles.
constexpr int64_t kTn4PartDoubles = int64_t(1) << 21;
int tn4_splits(int64_t M, int p, int q, int64_t tiles) {
  int64_t want = ceil_div((int64_t)num_sms() * 8, tiles);
  want = std::min<int64_t>(want, ceil_div(M, 32));
  want = std::min<int64_t>(want, kTn4PartDoubles / std::max<int64_t>((int64_t)p * q, 1));
  return (int)std::max<int64_t>(want, 1);
}

size_t gemm_tn_scratch(int64_t M, int p, int q) {
  (void)M;
  const int64_t tiles = ceil_div(p > 0 ? p : 1, TN_TILE) * ceil_div(q > 0 ? q : 1, TN_TILE);
  const size_t old = (size_t)((int64_t)num_sms() * 4 + tiles + 1) * TN_TILE * TN_TILE;
  return std::max<size_t>(old, (size_t)kTn4PartDoubles + (size_t)p * q);
}

template <typename TA, typename TB>
svt_status gemm_tn(int64_t M, int p, int q, const TA* A, int64_t lda, const TB* B, int64_t ldb,
                   double* C, int64_t ldc, double* part, cudaStream_t s) {
  if (p <= 0 || q <= 0) return SVT_OK;
  if (M <= 0) {
    for (int a = 0; a < p; ++a) SVT_CUDA(cudaMemsetAsync(C + (int64_t)a * ldc, 0, q * sizeof(double), s));
    return SVT_OK;
  }
  const int sym = (A == (const TA*)(const void*)B && p == q && lda == ldb) ? 1 : 0;
  const int64_t tp = ceil_div(p, TN_TILE);
  const int64_t tiles = sym ? tp * (tp + 1) / 2 : tp * ceil_div(q, TN_TILE);
  constexpr bool kF32 = sizeof(TA) == 4 && sizeof(TB) == 4;
  const int splits = kF32 ? tn4_splits(M, p, q, tiles) : tn_splits(M, p, q);
  const int64_t rows = round_up(ceil_div(M, splits), TN_TILE);
  const int used = (int)ceil_div(M, rows);
  dim3 grid(sym ? (unsigned)(tp * (tp + 1) / 2) : (unsigned)tp,
            sym ? 1u : (unsigned)ceil_div(q, TN_TILE), (unsigned)used);
  if constexpr (kF32) {
    k_gemm_tn_part4<<<grid, 64, 0, s>>>(M, p, q, (const float*)A, lda, (const float*)B, ldb, rows, part, sym);
  } else {
    k_gemm_tn_part<TA, TB><<<grid, 256, 0, s>>>(M, p, q, A, lda, B, ldb, rows, part, sym);
  }
  SVT_LAUNCH_CHECK();
  launch_reduce_parts(p, q, used, part, C, ldc, sym, s);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template <typename TA, typename TC>
svt_status gemm_nn(int64_t M, int p, int q, double alpha, const TA* A, int64_t lda,
                   const double* B, int64_t ldb, double beta, const TC* Cin, int64_t ldcin,
                   TC* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || q <= 0) return SVT_OK;
  dim3 grid((unsigned)ceil_div(q, 32), (unsigned)ceil_div(M, 64));
  if (grid.y > 65535u) {
    // process in row slabs of 65535*64 rows
    const int64_t slab = (int64_t)65535 * 64;
    for (int64_t r0 = 0; r0 < M; r0 += slab) {
      const int64_t mm = (M - r0) < slab ? (M - r0) : slab;
      SVT_TRY((gemm_nn<TA, TC>(mm, p, q, alpha, A + r0 * lda, lda, B, ldb, beta,
                               Cin ? Cin + r0 * ldcin : Cin, ldcin, C + r0 * ldc, ldc, s)));
    }
    return SVT_OK;
  }
  if constexpr (sizeof(TA) == 4 && sizeof(TC) == 4) {
    const dim3 g32((unsigned)ceil_div(q, 64), (unsigned)ceil_div(M, 128));
    k_gemm_nn_f32<<<g32, 256, 0, s>>>(M, p, q, (float)alpha, A, lda, B, ldb, (float)beta, Cin, ldcin,
                                      C, ldc);
  } else {
    using TACC = typename std::conditional<sizeof(TA) == 8 || sizeof(TC) == 8, double, float>::type;
    k_gemm_nn<TA, TC, TACC><<<grid, 256, 0, s>>>(M, p, q, alpha, A, lda, B, ldb, beta, Cin, ldcin,
                                                 C, ldc);
  }
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

size_t colsumsq_scratch(int64_t M, int w) {
  return (size_t)(num_sms() * 4) * (size_t)(w > 0 ? w : 1);
}

template <typename T>
svt_status colsumsq(int64_t M, int w, const T* X, int64_t ldx, double* sums, double* part,
                    cudaStream_t s) {
  if (w <= 0) return SVT_OK;
  const int64_t blocks_max = (int64_t)num_sms() * 4;
  int64_t rows = ceil_div(M > 0 ? M : 1, blocks_max);
  const int blocks = (int)ceil_div(M > 0 ? M : 1, rows);
  k_colsumsq_part<T><<<blocks, 256, 0, s>>>(M, w, X, ldx, rows, part);
  SVT_LAUNCH_CHECK();
  launch_reduce_parts(1, w, blocks, part, sums, w, 0, s);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template <typename TS, typename TD>
svt_status copy_convert(int64_t M, int w, const TS* src, int64_t lds, TD* dst, int64_t ldd,
                        cudaStream_t s) {
  if (M <= 0 || w <= 0) return SVT_OK;
  k_copy_convert<TS, TD><<<grid_cap(M * w, 256, 16), 256, 0, s>>>(M, w, src, lds, dst, ldd);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

svt_status chol_inv(int w, const double* G, int64_t ldg, double* R, double* Rinv,
                    double* work, double* diag_min, unsigned* flags, cudaStream_t s) {
  k_chol_inv<<<1, 1024, 0, s>>>(w, G, ldg, R, Rinv, work, diag_min, flags);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

#define SVT_INST_TN(TA, TB)                                                                     \
  template svt_status gemm_tn<TA, TB>(int64_t, int, int, const TA*, int64_t, const TB*, int64_t, \
                                      double*, int64_t, double*, cudaStream_t);
SVT_INST_TN(double, double)
SVT_INST_TN(float, float)
#define SVT_INST_NN(TA, TC)                                                                     \
  template svt_status gemm_nn<TA, TC>(int64_t, int, int, double, const TA*, int64_t,             \
                                      const double*, int64_t, double, const TC*, int64_t, TC*,   \
                                      int64_t, cudaStream_t);
SVT_INST_NN(double, double)
SVT_INST_NN(float, float)
template svt_status colsumsq<double>(int64_t, int, const double*, int64_t, double*, double*,
                                     cudaStream_t);
template svt_status colsumsq<float>(int64_t, int, const float*, int64_t, double*, double*,
                                    cudaStream_t);
template svt_status copy_convert<double, double>(int64_t, int, const double*, int64_t, double*,
                                                 int64_t, cudaStream_t);
template svt_status copy_convert<float, double>(int64_t, int, const float*, int64_t, double*,
                                                int64_t, cudaStream_t);
template svt_status copy_convert<double, float>(int64_t, int, const double*, int64_t, float*,
                                                int64_t, cudaStream_t);
template svt_status copy_convert<float, float>(int64_t, int, const float*, int64_t, float*,
                                               int64_t, cudaStream_t);

}  // namespace svt
