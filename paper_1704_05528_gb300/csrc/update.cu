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

// The same update in CSC order, fused with the next iteration's recycled product.
// R4SVD recycles the basis U that defines X (Algorithm 3), so B^T = Y_new^T U (eq. (5)
// gives Y_new) can be formed while the update holds the rows of U it gathers: each entry
// (p, q) gathers U[p, :r] once, dots its first k columns with W[q, :k] (held in registers
// while the warp stays in column q), writes Y_pq += delta (A_pq - x_pq) and adds
// Y_pq(new) U[p, :r] into row q of B^T.  Chunks, groups and the partial rows of columns
// that cross chunks follow launch_spmm_rows (head and tail slots, then the fix-up in chunk
// order), so B^T does not depend on scheduling.  The loop over a column's entries has the
// same trip count in every group of the warp (the group reductions need all lanes).
template <typename T, int VEC, int G, int MAXV, int UNR, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_update_recycle(int32_t n, int32_t nnz, int32_t C, int32_t nchunks,
                 const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                 const int32_t* __restrict__ chunk_col, const T* __restrict__ U, int64_t ldu,
                 int r, const T* __restrict__ W, int64_t ldw, int k, const T* __restrict__ a,
                 T* __restrict__ y, T delta, T* __restrict__ bt, int64_t ldb,
                 T* __restrict__ slots, int64_t ldp, int32_t* __restrict__ tail_col,
                 double* __restrict__ part, unsigned* __restrict__ flags) {
  constexpr int NG = 32 / G;
  __shared__ double s_wpart[8][3];
  __shared__ unsigned s_done;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G;
  // entry offsets fit in int32: the pattern's column pointers are int32
  const int32_t chunk = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (threadIdx.x == 0) s_done = 0;
  __syncthreads();
  SumAcc<T> acc_d2, acc_abs, acc_y2;
  bool bad = false;
  if (chunk < nchunks) {  // warp-uniform
    const int32_t beg = chunk * C;
    const int32_t end = (nnz - beg > C) ? beg + C : nnz;
    const bool last_chunk = (chunk == nchunks - 1);
    int32_t my_tail = -1;
    for (int32_t q = chunk_col[chunk]; q < n; ++q) {
      const int32_t cb = col_ptr[q], ce = col_ptr[q + 1];
      if (cb >= end && !(last_chunk && cb == nnz)) break;
      const int32_t sb = cb > beg ? cb : beg;
      const int32_t se = ce < end ? ce : end;
      // this lane's slices of W[q, :k], zero from column k on
      T wq[MAXV][VEC];
#pragma unroll
      for (int t = 0; t < MAXV; ++t) {
        const int c0 = (gl + t * G) * VEC;
        if (c0 < k) load_v<T, VEC>(W + (int64_t)q * ldw + c0, wq[t]);
#pragma unroll
        for (int b = 0; b < VEC; ++b)
          if (c0 + b >= k) wq[t][b] = T(0);
      }
      T acc[MAXV][VEC];
#pragma unroll
      for (int t = 0; t < MAXV; ++t)
#pragma unroll
        for (int b = 0; b < VEC; ++b) acc[t][b] = T(0);
      for (int32_t e0 = sb + grp; e0 - grp < se; e0 += NG * UNR) {
        T av[UNR], yv[UNR];
        T ux[UNR][MAXV][VEC];
#pragma unroll
        for (int j = 0; j < UNR; ++j) {
          const int32_t e = e0 + j * NG;
          const bool v = e < se;
          const T* up = U + (int64_t)(v ? row_idx[e] : 0) * ldu;
          av[j] = v ? a[e] : T(0);
          yv[j] = v ? y[e] : T(0);
#pragma unroll
          for (int t = 0; t < MAXV; ++t) {
            const int c0 = (gl + t * G) * VEC;
            if (v && c0 < r) load_v<T, VEC>(up + c0, ux[j][t]);
#pragma unroll
            for (int b = 0; b < VEC; ++b)
              if (!v || c0 + b >= r) ux[j][t][b] = T(0);
          }
        }
        T px[UNR];
#pragma unroll
        for (int j = 0; j < UNR; ++j) {
          px[j] = T(0);
#pragma unroll
          for (int t = 0; t < MAXV; ++t)
#pragma unroll
            for (int b = 0; b < VEC; ++b) px[j] = fma(ux[j][t][b], wq[t][b], px[j]);
        }
        // butterfly over the group: every lane ends with the same sum (a + b == b + a)
#pragma unroll
        for (int j = 0; j < UNR; ++j)
#pragma unroll
          for (int o = 1; o < G; o <<= 1) px[j] += __shfl_xor_sync(0xffffffffu, px[j], o);
        // every lane forms all UNR updated values (zero for a masked entry) ...
        T yn[UNR], d[UNR];
#pragma unroll
        for (int j = 0; j < UNR; ++j) {
          d[j] = av[j] - px[j];
          yn[j] = fma(delta, d[j], yv[j]);
        }
        // ... and lane j0 + l of the group stores entry j0 + l and adds it to the sums,
        // so the group's entries finish in one instruction stream
#pragma unroll
        for (int j0 = 0; j0 < UNR; j0 += G) {
          T ds = T(0), ys = T(0);
          bool vs = false;
#pragma unroll
          for (int j = j0; j < UNR && j < j0 + G; ++j)
            if (gl == j - j0) { ds = d[j]; ys = yn[j]; vs = e0 + j * NG < se; }
          if (vs) {
            y[e0 + (j0 + gl) * NG] = ys;
            acc_d2.add_sq(ds);
            acc_abs.add(fabs(ds));
            acc_y2.add_sq(ys);
            bad |= !isfinite(ys);
          }
        }
#pragma unroll
        for (int j = 0; j < UNR; ++j)
#pragma unroll
          for (int t = 0; t < MAXV; ++t)
#pragma unroll
            for (int b = 0; b < VEC; ++b) acc[t][b] = fma(yn[j], ux[j][t][b], acc[t][b]);
      }
#pragma unroll
      for (int t = 0; t < MAXV; ++t)
#pragma unroll
        for (int b = 0; b < VEC; ++b)
#pragma unroll
          for (int o = G; o < 32; o <<= 1) acc[t][b] += __shfl_xor_sync(0xffffffffu, acc[t][b], o);
      T* dst;
      if (cb >= beg && ce <= end) {
        dst = bt + (int64_t)q * ldb;
      } else if (cb < beg) {
        dst = slots + (int64_t)(2 * chunk) * ldp;      // head slot
      } else {
        dst = slots + (int64_t)(2 * chunk + 1) * ldp;  // tail slot
        my_tail = q;
      }
      if (grp == 0) {
#pragma unroll
        for (int t = 0; t < MAXV; ++t) {
          const int c0 = (gl + t * G) * VEC;
#pragma unroll
          for (int b = 0; b < VEC; ++b)
            if (c0 + b < r) dst[c0 + b] = acc[t][b];
        }
      }
    }
    if (lane == 0) tail_col[chunk] = my_tail;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_NONFINITE);
  // One partial per block, summed in block order by k_finish.  Each warp's sums (fixed
  // shuffle tree) go to shared memory, and the last warp of the block to finish adds them
  // in warp order: there is no block-wide barrier, so a warp leaves as soon as its chunk
  // is done.
  const double s_d2 = warp_sum(acc_d2.value());
  const double s_abs = warp_sum(acc_abs.value());
  const double s_y2 = warp_sum(acc_y2.value());
  unsigned last = 0;
  if (lane == 0) {
    s_wpart[warp][0] = s_d2;
    s_wpart[warp][1] = s_abs;
    s_wpart[warp][2] = s_y2;
    __threadfence_block();
    last = atomicAdd(&s_done, 1u) == (blockDim.x >> 5) - 1 ? 1u : 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last && lane < 3) {
    __threadfence_block();
    const volatile double* wp = &s_wpart[0][0];
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wp[w * 3 + lane];
    part[(int64_t)blockIdx.x * 3 + lane] = t;
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

namespace {

int64_t recycle_blocks(int64_t nnz) { return ceil_div(ceil_div(nnz, chunk_size(nnz)), 8); }

template <typename T, int VEC, int G, int MAXV, int UNR, int MINB>
svt_status run_recycle(const svt_pattern* p, const T* U, int64_t ldu, int r, const T* W,
                       int64_t ldw, int k, const T* a, T* y, double delta, T* bt, int64_t ldb,
                       double* part, unsigned* flags, void* scratch, cudaStream_t s) {
  const int64_t z = p->nnz;
  const int64_t C = chunk_size(z);
  const int64_t nchunks = ceil_div(z, C);
  T* slots;
  int64_t ldp;
  int32_t* tails;
  spmm_slots<T>(scratch, z, r, &slots, &ldp, &tails);
  k_update_recycle<T, VEC, G, MAXV, UNR, MINB><<<(int)recycle_blocks(z), 256, 0, s>>>(
      (int32_t)p->n, (int32_t)z, (int32_t)C, (int32_t)nchunks, p->col_ptr, p->row_idx, p->chunk_row_csc, U, ldu, r, W, ldw, k, a, y,
      (T)delta, bt, ldb, slots, ldp, tails, part, flags);
  SVT_LAUNCH_CHECK();
  return spmm_fixup<T>(z, p->n, p->col_ptr, p->chunk_row_csc, slots, ldp, tails, r, bt, ldb, s);
}

// Up to four vectors of U's row per lane, two entries in flight per group, as few lanes
// per entry as that allows.  On the 71,567 x 10,681 pattern at r = 100 (binary32) this
// shape (8 lanes per entry, 8 entries per warp, two blocks per SM) took 0.47 ms against
// 0.60-0.98 ms for 16 or 32 lanes per entry, more entries in flight, or more blocks per SM
// with fewer registers; prefetching the next step's indices gained nothing.
template <typename T, int VEC>
svt_status dispatch_recycle(const svt_pattern* p, const T* U, int64_t ldu, int r, const T* W,
                            int64_t ldw, int k, const T* a, T* y, double delta, T* bt,
                            int64_t ldb, double* part, unsigned* flags, void* scratch,
                            cudaStream_t s) {
  const int nv = (int)ceil_div(r, VEC);
#define SVT_RUN(G) return run_recycle<T, VEC, G, 4, 2, 2>(p, U, ldu, r, W, ldw, k, a, y, delta, bt, ldb, part, flags, scratch, s)
  if (nv <= 4) SVT_RUN(1);
  if (nv <= 8) SVT_RUN(2);
  if (nv <= 16) SVT_RUN(4);
  if (nv <= 32) SVT_RUN(8);
  if (nv <= 64) SVT_RUN(16);
  SVT_RUN(32);
#undef SVT_RUN
}

}  // namespace

template <typename T>
bool update_recycle_fits(int r, int64_t nnz) {
  // entry offsets run in int32 with up to a chunk and a step of headroom
  return r >= 1 && r <= (sizeof(T) == 4 ? 512 : 256) && nnz <= INT32_MAX - (int64_t)(1 << 16);
}

size_t update_recycle_scratch(int64_t nnz) {
  return (size_t)(3 * recycle_blocks(nnz > 0 ? nnz : 1) + 8);
}

template <typename T>
svt_status update_recycle(const svt_pattern* p, const T* U, int64_t ldu, int r, const T* W,
                          int64_t ldw, int k, const T* a, T* y, double delta, T* bt, int64_t ldb,
                          double* out3, double* part, unsigned* flags, void* scratch,
                          cudaStream_t s) {
  constexpr int V = sizeof(T) == 4 ? 4 : 2;
  if (!update_recycle_fits<T>(r, p->nnz) || k < 0 || k > r)
    return fail(SVT_ERR_UNSUPPORTED, "fused update: r = %d, k = %d", r, k);
  if ((reinterpret_cast<uintptr_t>(U) % 16) || (ldu % V) || (reinterpret_cast<uintptr_t>(W) % 16) ||
      (ldw % V) || ldw < round_up(k, V) || ldu < round_up(r, V))
    return fail(SVT_ERR_UNSUPPORTED, "fused update: unaligned operands");
  if (p->nnz == 0) {
    SVT_CUDA(cudaMemsetAsync(out3, 0, 3 * sizeof(double), s));
    if (p->n > 0) SVT_CUDA(cudaMemset2DAsync(bt, ldb * sizeof(T), 0, r * sizeof(T), p->n, s));
    return SVT_OK;
  }
  SVT_TRY((dispatch_recycle<T, V>(p, U, ldu, r, W, ldw, k, a, y, delta, bt, ldb, part, flags,
                                   scratch, s)));
  k_finish<<<3, 256, 0, s>>>((int)recycle_blocks(p->nnz), 3, 3, part, out3);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template bool update_recycle_fits<double>(int, int64_t);
template bool update_recycle_fits<float>(int, int64_t);
template svt_status update_recycle<double>(const svt_pattern*, const double*, int64_t, int,
                                           const double*, int64_t, int, const double*, double*,
                                           double, double*, int64_t, double*, double*, unsigned*,
                                           void*, cudaStream_t);
template svt_status update_recycle<float>(const svt_pattern*, const float*, int64_t, int,
                                          const float*, int64_t, int, const float*, float*,
                                          double, float*, int64_t, double*, double*, unsigned*,
                                          void*, cudaStream_t);
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
