// Sparse (Y on Lambda) times tall-skinny dense block: the matrix-block products that
// dominate Algorithms 1-3 (O((np+2) r T_mult), Section 2.2).
//
// Work is split by entries, not by rows: warp c owns entries [c*C, (c+1)*C) of the
// compressed order, so a column with 60k entries costs the same as 60k scattered
// entries; each chunk's first row is precomputed with the pattern.  Inside a warp,
// groups of G lanes each take one entry at a time and gather its row of W with 16-byte
// vector loads (lane l of a group holds vectors l, l+G, ...).
// A row lying entirely inside a chunk is written directly; a row crossing chunk
// boundaries leaves one partial per chunk (the chunk's first row in slot "head", its
// last row in slot "tail"), and a fix-up pass adds them in chunk order.  The result is
// therefore independent of scheduling.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

template <typename T, int VEC> struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<double, 2> { using type = double2; };
template <typename T> struct VecT<T, 1> { using type = T; };

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T* p, const T (&v)[VEC]) {
  if constexpr (VEC == 1) {
    p[0] = v[0];
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
}

template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T* p, T (&v)[VEC]) {
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

// First row of the chunk starting at entry `beg`: rows with ptr[r] == beg (possibly empty)
// belong to this chunk; a row that started earlier and covers `beg` comes first.
__device__ __forceinline__ int64_t chunk_first_row(const int32_t* __restrict__ ptr, int64_t nrows,
                                                   int64_t beg) {
  int64_t lo = 0, hi = nrows + 1;  // smallest r in [0, nrows] with ptr[r] >= beg
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ptr[mid] < beg) lo = mid + 1; else hi = mid;
  }
  if (lo > nrows || ptr[lo] > beg) return lo - 1;
  return lo;
}

template <typename TV, typename TD, int VEC, int G, int MAXV, int UNR>
__global__ void __launch_bounds__(256)
k_spmm_chunked(int64_t nrows, int64_t nnz, int64_t C, const int32_t* __restrict__ ptr,
               const int32_t* __restrict__ idx, const TV* __restrict__ val, const TD* __restrict__ W,
               int64_t ldw, int w, TD* __restrict__ out, int64_t ldo, TD* __restrict__ part,
               int64_t ldp, int32_t* __restrict__ tail_row, int64_t nchunks,
               const int32_t* __restrict__ chunk_row) {
  constexpr int NG = 32 / G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane % G;
  const int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (chunk >= nchunks) return;
  const int64_t beg = chunk * C;
  const int64_t end = (beg + C < nnz) ? beg + C : nnz;
  const bool last_chunk = (chunk == nchunks - 1);
  int64_t r = chunk_row ? chunk_row[chunk] : chunk_first_row(ptr, nrows, beg);
  int32_t my_tail = -1;
  for (; r < nrows; ++r) {
    const int64_t rb = ptr[r], re = ptr[r + 1];
    if (rb >= end && !(last_chunk && rb == nnz)) break;
    const int64_t sb = rb > beg ? rb : beg;
    const int64_t se = re < end ? re : end;
    TD acc[MAXV][VEC];
#pragma unroll
    for (int a = 0; a < MAXV; ++a)
#pragma unroll
      for (int b = 0; b < VEC; ++b) acc[a][b] = TD(0);
    // UNR entries per group per step: their index, value and row loads are all issued
    // before the dependent multiply-adds
    for (int64_t e0 = sb + grp; e0 < se; e0 += NG * UNR) {
      TD v[UNR];
      const TD* wr[UNR];
      bool ok[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int64_t e = e0 + (int64_t)u * NG;
        ok[u] = e < se;
        v[u] = ok[u] ? (TD)val[e] : TD(0);
        wr[u] = W + (int64_t)(ok[u] ? idx[e] : 0) * ldw;
      }
      TD x[UNR][MAXV][VEC];
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int a = 0; a < MAXV; ++a) {
          const int c0 = (gl + a * G) * VEC;
          if (ok[u] && c0 < w) {
            load_vec<TD, VEC>(wr[u] + c0, x[u][a]);
          } else {
#pragma unroll
            for (int b = 0; b < VEC; ++b) x[u][a][b] = TD(0);
          }
        }
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int a = 0; a < MAXV; ++a)
#pragma unroll
          for (int b = 0; b < VEC; ++b) acc[a][b] = fma(v[u], x[u][a][b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < MAXV; ++a)
#pragma unroll
      for (int b = 0; b < VEC; ++b)
#pragma unroll
        for (int o = G; o < 32; o <<= 1) acc[a][b] += __shfl_xor_sync(0xffffffffu, acc[a][b], o);
    const bool starts_before = rb < beg;
    const bool ends_after = re > end;
    TD* dst;
    if (!starts_before && !ends_after) {
      dst = out + r * ldo;
    } else if (starts_before) {
      dst = part + (2 * chunk) * ldp;         // head slot
    } else {
      dst = part + (2 * chunk + 1) * ldp;     // tail slot
      my_tail = (int32_t)r;
    }
    if (grp == 0) {
#pragma unroll
      for (int a = 0; a < MAXV; ++a) {
        const int c0 = (gl + a * G) * VEC;
#pragma unroll
        for (int b = 0; b < VEC; ++b)
          if (c0 + b < w) dst[c0 + b] = acc[a][b];
      }
    }
  }
  if (lane == 0) tail_row[chunk] = my_tail;
}

// out[r] = tail(c) + head(c+1) + ... + head(c_last) for the row r left in chunk c's tail,
// in two passes so that no warp walks a long row alone: a row spanning more than kFixSeg
// chunks (a popular column spans hundreds) is cut into segments of kFixSeg chunks, each
// summed in chunk order by the warp of its first chunk, whose own tail slot is free (the
// chunk lies inside that row), and the second pass adds tail(c) and the segment sums in
// segment order.  Rows spanning at most kFixSeg chunks are summed in chunk order by the
// first pass.  One warp per chunk, lanes over vectors of VEC columns (partial rows are
// 16-byte aligned with a padded leading dimension); eight independent loads per step.
constexpr int kFixSeg = 16;

template <typename TD, int VEC>
__device__ __forceinline__ void add_heads(const TD* __restrict__ part, int64_t ldp, int c,
                                          int64_t k0, int64_t k1, TD (&s)[VEC]) {
  int64_t k = k0;
  for (; k + 8 <= k1 + 1; k += 8) {
    TD v[8][VEC];
#pragma unroll
    for (int j = 0; j < 8; ++j) load_vec<TD, VEC>(part + (2 * (k + j)) * ldp + c, v[j]);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int b = 0; b < VEC; ++b) s[b] += v[j][b];
  }
  for (; k <= k1; ++k) {
    TD v[VEC];
    load_vec<TD, VEC>(part + (2 * k) * ldp + c, v);
#pragma unroll
    for (int b = 0; b < VEC; ++b) s[b] += v[b];
  }
}

template <typename TD>
__global__ void __launch_bounds__(256)
k_spmm_fixup(int64_t nchunks, int64_t C, int64_t nrows, const int32_t* __restrict__ ptr,
             const int32_t* __restrict__ chunk_row, TD* __restrict__ part, int64_t ldp,
             const int32_t* __restrict__ tail_row, int w, TD* __restrict__ out, int64_t ldo) {
  constexpr int VEC = sizeof(TD) == 4 ? 4 : 2;
  const int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (chunk >= nchunks) return;
  const int nvec = (w + VEC - 1) / VEC;
  const int32_t r = tail_row[chunk];
  if (r >= 0) {  // a row starts here and continues: sum it now if it is short
    const int64_t c_last = ((int64_t)ptr[r + 1] - 1) / C;
    if (c_last - chunk > kFixSeg) return;  // long: second pass
    for (int cv = lane; cv < nvec; cv += 32) {
      const int c = cv * VEC;
      TD s[VEC];
      load_vec<TD, VEC>(part + (2 * chunk + 1) * ldp + c, s);
      add_heads<TD, VEC>(part, ldp, c, chunk + 1, c_last, s);
#pragma unroll
      for (int b = 0; b < VEC; ++b)
        if (c + b < w) out[(int64_t)r * ldo + c + b] = s[b];
    }
    return;
  }
  // the first chunk of a segment of a long row that started before this chunk?
  const int64_t beg = chunk * C;
  const int64_t hr = chunk_row ? chunk_row[chunk] : chunk_first_row(ptr, nrows, beg);
  if (hr >= nrows || (int64_t)ptr[hr] >= beg) return;
  const int64_t c0 = (int64_t)ptr[hr] / C;
  const int64_t c_last = ((int64_t)ptr[hr + 1] - 1) / C;
  if (c_last - c0 <= kFixSeg || (chunk - (c0 + 1)) % kFixSeg != 0 || chunk >= c_last) return;
  const int64_t k1 = chunk + kFixSeg - 1 < c_last ? chunk + kFixSeg - 1 : c_last;
  for (int cv = lane; cv < nvec; cv += 32) {
    const int c = cv * VEC;
    TD s[VEC];
#pragma unroll
    for (int b = 0; b < VEC; ++b) s[b] = TD(0);
    add_heads<TD, VEC>(part, ldp, c, chunk, k1, s);
    store_vec<TD, VEC>(part + (2 * chunk + 1) * ldp + c, s);  // this chunk's free tail slot
  }
}

// Second pass: out[r] = tail(c) + the segment sums in order, for the long rows.
template <typename TD>
__global__ void __launch_bounds__(256)
k_spmm_fixup_long(int64_t nchunks, int64_t C, const int32_t* __restrict__ ptr,
                  const TD* __restrict__ part, int64_t ldp, const int32_t* __restrict__ tail_row,
                  int w, TD* __restrict__ out, int64_t ldo) {
  constexpr int VEC = sizeof(TD) == 4 ? 4 : 2;
  const int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (chunk >= nchunks) return;
  const int32_t r = tail_row[chunk];
  if (r < 0) return;
  const int64_t c_last = ((int64_t)ptr[r + 1] - 1) / C;
  if (c_last - chunk <= kFixSeg) return;
  const int nvec = (w + VEC - 1) / VEC;
  for (int cv = lane; cv < nvec; cv += 32) {
    const int c = cv * VEC;
    TD s[VEC];
    load_vec<TD, VEC>(part + (2 * chunk + 1) * ldp + c, s);
    int64_t ks = chunk + 1;
    for (; ks + 8 * kFixSeg <= c_last; ks += 8 * kFixSeg) {  // eight segments in flight
      TD v[8][VEC];
#pragma unroll
      for (int j = 0; j < 8; ++j) load_vec<TD, VEC>(part + (2 * (ks + j * kFixSeg) + 1) * ldp + c, v[j]);
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int b = 0; b < VEC; ++b) s[b] += v[j][b];
    }
    for (; ks <= c_last; ks += kFixSeg) {
      TD v[VEC];
      // a segment starting at the row's last chunk is that chunk's head alone
      load_vec<TD, VEC>(part + (ks < c_last ? 2 * ks + 1 : 2 * ks) * ldp + c, v);
#pragma unroll
      for (int b = 0; b < VEC; ++b) s[b] += v[b];
    }
#pragma unroll
    for (int b = 0; b < VEC; ++b)
      if (c + b < w) out[(int64_t)r * ldo + c + b] = s[b];
  }
}

template <typename T>
__global__ void k_gather(int64_t count, const int32_t* __restrict__ perm, const T* __restrict__ src,
                         T* __restrict__ dst) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = src[perm[q]];
}

template <typename T>
__global__ void k_scatter(int64_t count, const int32_t* __restrict__ perm, const T* __restrict__ src,
                          T* __restrict__ dst) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    dst[perm[q]] = src[q];
}

__global__ void k_zero_rows(int64_t nrows, int w, void* out_, int64_t ldo, int elem) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrows * w;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / w;
    const int j = (int)(t - i * w);
    if (elem == 8) reinterpret_cast<double*>(out_)[i * ldo + j] = 0.0;
    else reinterpret_cast<float*>(out_)[i * ldo + j] = 0.0f;
  }
}

}  // namespace

// Entries per work chunk (one warp each): about 32 chunks per SM, a multiple of 32 entries.
// Measured on the 71,567 x 10,681 pattern (9.0 M entries, and its 4.5 M-entry sparse rest):
// 256, 128, 64, 32 and 16 chunks per SM gave 1088, 1133, 1158, 1170 and 1148 SVT
// iterations/s; longer chunks cut the partial rows and per-column set-up of the fused
// update, until the width-1 products of the power steps lose more than it gains.
int64_t chunk_size(int64_t nnz) {
  int64_t c = ceil_div(nnz, (int64_t)num_sms() * 32);
  c = round_up(c < 32 ? 32 : c, 32);
  return c > 4096 ? 4096 : c;
}

namespace {

template <typename TV, typename TD, int VEC, int G, int MAXV, int UNR>
svt_status run_chunked(int64_t nrows, int64_t nnz, const int32_t* ptr, const int32_t* idx,
                       const TV* val, const TD* W, int64_t ldw, int w, TD* out, int64_t ldo,
                       TD* part, int32_t* tails, const int32_t* chunk_row, cudaStream_t s) {
  const int64_t C = chunk_size(nnz);
  const int64_t nchunks = ceil_div(nnz, C);
  const int64_t ldp = round_up(w, 4);
  const int blocks = (int)ceil_div(nchunks, 8);
  k_spmm_chunked<TV, TD, VEC, G, MAXV, UNR><<<blocks, 256, 0, s>>>(nrows, nnz, C, ptr, idx, val, W, ldw, w,
                                                              out, ldo, part, ldp, tails, nchunks,
                                                              chunk_row);
  SVT_LAUNCH_CHECK();
  k_spmm_fixup<TD><<<blocks, 256, 0, s>>>(nchunks, C, nrows, ptr, chunk_row, part, ldp, tails, w, out, ldo);
  SVT_LAUNCH_CHECK();
  k_spmm_fixup_long<TD><<<blocks, 256, 0, s>>>(nchunks, C, ptr, part, ldp, tails, w, out, ldo);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

// Dispatch on width (in vectors of VEC elements): G lanes per entry, MAXV vectors per lane.
template <typename TV, typename TD, int VEC>
svt_status dispatch(int64_t nrows, int64_t nnz, const int32_t* ptr, const int32_t* idx,
                    const TV* val, const TD* W, int64_t ldw, int w, TD* out, int64_t ldo,
                    TD* part, int32_t* tails, const int32_t* chunk_row, cudaStream_t s) {
  const int nv = (int)ceil_div(w, VEC);
  // narrow blocks: one vector per lane, several entries per warp; wide blocks: one entry
  // per warp, up to 16 vectors per lane
#define SVT_RUN(G, MV, U) return run_chunked<TV, TD, VEC, G, MV, U>(nrows, nnz, ptr, idx, val, W, ldw, w, out, ldo, part, tails, chunk_row, s)
  if (nv <= 1) SVT_RUN(1, 1, 1);
  if (nv <= 2) SVT_RUN(2, 1, 1);
  if (nv <= 4) SVT_RUN(4, 1, 1);
  if (nv <= 8) SVT_RUN(8, 1, 1);
  if (nv <= 16) SVT_RUN(16, 1, 1);
  // 17-32 vectors (65-128 binary32 columns, the recycled product's width): half a warp per
  // entry with two entries in flight measured 13% faster than a whole warp per entry
  if (nv <= 32) SVT_RUN(16, 2, 2);
  if (nv <= 64) SVT_RUN(32, 2, 1);
  if (nv <= 128) SVT_RUN(32, 4, 1);
  if (nv <= 256) SVT_RUN(32, 8, 1);
  SVT_RUN(32, 16, 1);
#undef SVT_RUN
}

}  // namespace

// Scratch of one SpMM call: per chunk two partial rows (head, tail) of up to 512
// columns, then one int32 per chunk naming the row left in its tail slot.
static int64_t part_bytes(int64_t nchunks, int w, int elem) {
  const int64_t wc = w < 512 ? w : 512;
  return round_up(2 * nchunks * round_up(wc, 4) * elem, 256);
}

size_t spmm_scratch_bytes(int64_t nnz, int w, int elem) {
  const int64_t nchunks = ceil_div(nnz > 0 ? nnz : 1, chunk_size(nnz > 0 ? nnz : 1));
  return (size_t)(part_bytes(nchunks, w, elem) + nchunks * 4 + 256);
}

template <typename TV, typename TD>
svt_status launch_spmm_rows(int64_t nrows, const int32_t* ptr, const int32_t* idx,
                            const TV* val, const TD* W, int64_t ldw, int w, TD* out,
                            int64_t ldo, void* scratch, int64_t nnz, cudaStream_t s,
                            const int32_t* chunk_row) {
  if (nrows <= 0 || w <= 0) return SVT_OK;
  if (nnz == 0) {
    const int64_t zb = ceil_div(nrows * w, 256);
    k_zero_rows<<<(int)(zb < 4096 ? zb : 4096), 256, 0, s>>>(
        nrows, w, out, ldo, (int)sizeof(TD));
    SVT_LAUNCH_CHECK();
    return SVT_OK;
  }
  const int64_t nchunks = ceil_div(nnz, chunk_size(nnz));
  TD* part = reinterpret_cast<TD*>(scratch);
  int32_t* tails = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(scratch) +
                                              part_bytes(nchunks, w, (int)sizeof(TD)));
  for (int c0 = 0; c0 < w; c0 += 512) {
    const int wc = (w - c0) < 512 ? (w - c0) : 512;
    const TD* Wc = W + c0;
    TD* oc = out + c0;
    constexpr int V = (sizeof(TD) == 4) ? 4 : 2;
    const bool aligned = ((reinterpret_cast<uintptr_t>(Wc) % 16) == 0) && (ldw % V == 0);
    svt_status st = aligned ? dispatch<TV, TD, V>(nrows, nnz, ptr, idx, val, Wc, ldw, wc, oc, ldo, part, tails, chunk_row, s)
                            : dispatch<TV, TD, 1>(nrows, nnz, ptr, idx, val, Wc, ldw, wc, oc, ldo, part, tails, chunk_row, s);
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

template <typename T>
svt_status launch_scatter(int64_t count, const int32_t* perm, const T* src, T* dst,
                          cudaStream_t s) {
  if (count <= 0) return SVT_OK;
  int64_t g = ceil_div(count, 256);
  const int64_t cap = (int64_t)num_sms() * 32;
  if (g > cap) g = cap;
  k_scatter<T><<<(int)g, 256, 0, s>>>(count, perm, src, dst);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template <typename TD>
void spmm_slots(void* scratch, int64_t nnz, int w, TD** part, int64_t* ldp, int32_t** tails) {
  const int64_t nchunks = ceil_div(nnz, chunk_size(nnz));
  *part = reinterpret_cast<TD*>(scratch);
  *ldp = round_up(w, 4);
  *tails = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(scratch) +
                                      part_bytes(nchunks, w, (int)sizeof(TD)));
}

template <typename TD>
svt_status spmm_fixup(int64_t nnz, int64_t nrows, const int32_t* ptr, const int32_t* chunk_row,
                      TD* part, int64_t ldp, const int32_t* tails, int w, TD* out, int64_t ldo,
                      cudaStream_t s) {
  if (nnz <= 0 || w <= 0) return SVT_OK;
  const int64_t C = chunk_size(nnz);
  const int64_t nchunks = ceil_div(nnz, C);
  const int blocks = (int)ceil_div(nchunks, 8);
  k_spmm_fixup<TD><<<blocks, 256, 0, s>>>(nchunks, C, nrows, ptr, chunk_row, part, ldp, tails, w, out, ldo);
  SVT_LAUNCH_CHECK();
  k_spmm_fixup_long<TD><<<blocks, 256, 0, s>>>(nchunks, C, ptr, part, ldp, tails, w, out, ldo);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

#define SVT_INST_SPMM(TV, TD)                                                                   \
  template svt_status launch_spmm_rows<TV, TD>(int64_t, const int32_t*, const int32_t*,          \
                                               const TV*, const TD*, int64_t, int, TD*, int64_t, \
                                               void*, int64_t, cudaStream_t, const int32_t*);
SVT_INST_SPMM(double, double)
SVT_INST_SPMM(float, float)
SVT_INST_SPMM(float, double)
template svt_status launch_gather<double>(int64_t, const int32_t*, const double*, double*,
                                          cudaStream_t);
template svt_status launch_gather<float>(int64_t, const int32_t*, const float*, float*,
                                         cudaStream_t);
template svt_status launch_scatter<double>(int64_t, const int32_t*, const double*, double*,
                                           cudaStream_t);
template svt_status launch_scatter<float>(int64_t, const int32_t*, const float*, float*,
                                          cudaStream_t);
template void spmm_slots<double>(void*, int64_t, int, double**, int64_t*, int32_t**);
template void spmm_slots<float>(void*, int64_t, int, float**, int64_t*, int32_t**);
template svt_status spmm_fixup<double>(int64_t, int64_t, const int32_t*, const int32_t*, double*,
                                       int64_t, const int32_t*, int, double*, int64_t, cudaStream_t);
template svt_status spmm_fixup<float>(int64_t, int64_t, const int32_t*, const int32_t*, float*,
                                      int64_t, const int32_t*, int, float*, int64_t, cudaStream_t);

}  // namespace svt
