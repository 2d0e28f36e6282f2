// Observed-set construction: COO -> CSR (row, col) + CSC (col, row) + CSC->CSR permutation.
//
// P_Lambda of eq. (4) is realised by the sparsity pattern: Y and A only ever exist on
// Lambda.  Both orders come from a stable least-significant-digit radix sort over the
// packed keys row*n + col (CSR) and col*m + row (CSC), 8-bit digits per pass.  Each
// pass is histogram -> exclusive scan (digit-major, tile-minor) -> stable scatter, with
// the in-tile rank of an item found by warp match masks, so the result is
// deterministic.  Out-of-range indices and duplicate pairs raise device flags.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;                 // items per thread per tile
constexpr int kTile = kThreads * kItems;  // 2048 keys per tile
constexpr int kRadix = 256;

__global__ void k_make_keys(int64_t nnz, const int32_t* __restrict__ rows,
                            const int32_t* __restrict__ cols, int64_t m, int64_t n,
                            uint64_t* __restrict__ keys, int32_t* __restrict__ vals,
                            unsigned* __restrict__ flags) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[e], c = cols[e];
    const bool ok = r >= 0 && r < m && c >= 0 && c < n;
    if (!ok) atomicOr(flags, FLAG_INDEX);
    keys[e] = ok ? (uint64_t)r * (uint64_t)n + (uint64_t)c : 0ull;
    vals[e] = (int32_t)e;
  }
}

// hist[d * ntiles + tile] = number of keys in `tile` whose digit is d.
__global__ void k_hist(int64_t nkeys, const uint64_t* __restrict__ keys, int shift,
                       int ntiles, int32_t* __restrict__ hist) {
  __shared__ int32_t h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += blockDim.x) {
    const int64_t e = base + i;
    if (e < nkeys) atomicAdd(&h[(keys[e] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Exclusive scan of `count` int32 values in place, one block of 1024 threads.
__global__ void k_scan(int32_t* __restrict__ data, int64_t count) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < count; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int32_t v = i < count ? data[i] : 0;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;  // inclusive prefix of warp totals
    }
    __syncthreads();
    const int32_t before = carry + (warp > 0 ? warp_tot[warp - 1] : 0);
    if (i < count) data[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + x;
    __syncthreads();
  }
}

// Stable scatter of one tile: items are visited in index order, 256 at a time; an item's
// destination is offset[d][tile] + (earlier items of the tile with the same digit).
__global__ void k_scatter(int64_t nkeys, const uint64_t* __restrict__ keys_in,
                          const int32_t* __restrict__ vals_in, uint64_t* __restrict__ keys_out,
                          int32_t* __restrict__ vals_out, int shift, int ntiles,
                          const int32_t* __restrict__ offsets) {
  __shared__ int32_t run[kRadix];                 // items of each digit seen so far
  __shared__ int32_t wcnt[kThreads / 32][kRadix + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) run[d] = 0;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int chunk = 0; chunk < kItems; ++chunk) {
    for (int i = threadIdx.x; i < (kThreads / 32) * (kRadix + 1); i += blockDim.x)
      (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t e = base + (int64_t)chunk * kThreads + threadIdx.x;
    const bool valid = e < nkeys;
    uint64_t key = valid ? keys_in[e] : 0ull;
    const int d = valid ? (int)((key >> shift) & 0xFF) : kRadix;  // sentinel bucket
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank_in_warp = __popc(peers & lt_mask);
    if (rank_in_warp == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int32_t pos = offsets[(int64_t)d * ntiles + blockIdx.x] + run[d] + rank_in_warp;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
      keys_out[pos] = key;
      vals_out[pos] = vals_in[e];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) {
      int32_t add = 0;
      for (int w = 0; w < kThreads / 32; ++w) add += wcnt[w][dd];
      run[dd] += add;
    }
    __syncthreads();
  }
}

__global__ void k_split_csr(int64_t nnz, const uint64_t* __restrict__ keys, int64_t n,
                            int32_t* __restrict__ row, int32_t* __restrict__ col,
                            unsigned* __restrict__ flags) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[e];
    row[e] = (int32_t)(k / (uint64_t)n);
    col[e] = (int32_t)(k % (uint64_t)n);
    if (e > 0 && keys[e - 1] == k) atomicOr(flags, FLAG_DUPLICATE);
  }
}

__global__ void k_make_csc_keys(int64_t nnz, const int32_t* __restrict__ row,
                                const int32_t* __restrict__ col, int64_t m,
                                uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    keys[e] = (uint64_t)col[e] * (uint64_t)m + (uint64_t)row[e];
    vals[e] = (int32_t)e;
  }
}

__global__ void k_split_csc(int64_t nnz, const uint64_t* __restrict__ keys, int64_t m,
                            int32_t* __restrict__ row_idx, int32_t* __restrict__ col_of) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[e];
    row_idx[e] = (int32_t)(k % (uint64_t)m);
    col_of[e] = (int32_t)(k / (uint64_t)m);
  }
}

// ptr[i] = first position e with sorted_key_major[e] >= i, for i in [0, len].
__global__ void k_offsets(int64_t nnz, const int32_t* __restrict__ major, int64_t len,
                          int32_t* __restrict__ ptr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= len;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (major[mid] < i) lo = mid + 1; else hi = mid;
    }
    ptr[i] = (int32_t)lo;
  }
}

// First compressed row touched by each chunk of C entries: the smallest r with
// ptr[r] >= beg if ptr[r] == beg (rows that start exactly at the chunk, possibly empty,
// belong to it), else the row that covers beg.
__global__ void k_chunk_rows(int64_t nrows, int64_t C, int64_t nchunks, const int32_t* __restrict__ ptr,
                             int32_t* __restrict__ out) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t beg = c * C;
    int64_t lo = 0, hi = nrows + 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ptr[mid] < beg) lo = mid + 1; else hi = mid;
    }
    out[c] = (int32_t)((lo > nrows || ptr[lo] > beg) ? lo - 1 : lo);
  }
}

int grid_for(int64_t n, int threads) {
  const int64_t g = ceil_div(n > 0 ? n : 1, threads);
  const int64_t cap = (int64_t)num_sms() * 16;
  return (int)(g < cap ? g : cap);
}

// Stable LSD radix sort of (keys, vals) by the low `bits` bits, ping-ponging between the
// two buffer pairs.  Returns the index (0 or 1) of the pair holding the result.
svt_status radix_sort(int64_t nkeys, int bits, uint64_t* keys[2], int32_t* vals[2],
                      int32_t* hist, cudaStream_t s, int* result) {
  const int ntiles = (int)ceil_div(nkeys, kTile);
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    k_hist<<<ntiles, kThreads, 0, s>>>(nkeys, keys[cur], shift, ntiles, hist);
    SVT_LAUNCH_CHECK();
    k_scan<<<1, 1024, 0, s>>>(hist, (int64_t)kRadix * ntiles);
    SVT_LAUNCH_CHECK();
    k_scatter<<<ntiles, kThreads, 0, s>>>(nkeys, keys[cur], vals[cur], keys[cur ^ 1],
                                          vals[cur ^ 1], shift, ntiles, hist);
    SVT_LAUNCH_CHECK();
    cur ^= 1;
  }
  *result = cur;
  return SVT_OK;
}

int bits_for(uint64_t range) {  // bits needed to represent values in [0, range)
  int b = 0;
  while (b < 64 && (range - 1) >> b) ++b;
  return b == 0 ? 1 : b;
}

}  // namespace

// The persistent arrays of a pattern, in one block.
void pattern_layout(Arena& ar, int64_t m, int64_t n, int64_t nnz, svt_pattern* p) {
  p->row_ptr = ar.take<int32_t>(m + 1);
  p->col_idx = ar.take<int32_t>(nnz);
  p->csr_src = ar.take<int32_t>(nnz);
  p->col_ptr = ar.take<int32_t>(n + 1);
  p->row_idx = ar.take<int32_t>(nnz);
  p->perm = ar.take<int32_t>(nnz);
  p->csr_row = ar.take<int32_t>(nnz);
  p->chunk = chunk_size(nnz > 0 ? nnz : 1);
  p->nchunks = ceil_div(nnz, p->chunk);
  p->chunk_row_csr = ar.take<int32_t>(p->nchunks);
  p->chunk_row_csc = ar.take<int32_t>(p->nchunks);
}

// Sort scratch of the build: two key/value buffer pairs, a histogram, a flags word.
void scratch_layout(Arena& sa, int64_t nnz, uint64_t** k0, uint64_t** k1, int32_t** v0, int32_t** v1,
                    int32_t** hist, unsigned** flags) {
  *k0 = sa.take<uint64_t>(nnz);
  *k1 = sa.take<uint64_t>(nnz);
  *v0 = sa.take<int32_t>(nnz);
  *v1 = sa.take<int32_t>(nnz);
  *hist = sa.take<int32_t>(kRadix * ceil_div(nnz, kTile));
  *flags = sa.take<unsigned>(1);
}

svt_status build_pattern(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                         const int32_t* cols, cudaStream_t s, svt_pattern** out) {
  if (!out) return fail(SVT_ERR_ARG, "pattern: null output handle");
  *out = nullptr;
  if (m <= 0 || n <= 0 || nnz < 0) return fail(SVT_ERR_ARG, "pattern: m, n must be positive and nnz >= 0");
  if (nnz >= (int64_t)INT32_MAX || m >= (int64_t)INT32_MAX || n >= (int64_t)INT32_MAX)
    return fail(SVT_ERR_UNSUPPORTED, "pattern: nnz, m and n must be below 2^31");
  if (nnz > 0 && (!rows || !cols)) return fail(SVT_ERR_ARG, "pattern: null index array");
  if (nnz > 0 && (!is_device_pointer(rows) || !is_device_pointer(cols)))
    return fail(SVT_ERR_ARG, "pattern: rows/cols must be device pointers");

  // One allocation for the persistent arrays.
  Arena a;
  auto layout = [&](Arena& ar, svt_pattern& p) { pattern_layout(ar, m, n, nnz, &p); };
  svt_pattern probe;
  layout(a, probe);
  svt_pattern* p = new svt_pattern;
  void* blk = nullptr;
  if (current_workspace()) {  // a slice of the caller's workspace, released with the pattern
    const svt_status st = p->ws_block.alloc(a.off, s);
    if (st < 0) { delete p; return st; }
    blk = p->ws_block.ptr;
  } else {
    const cudaError_t e = cudaMalloc(&blk, a.off);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaMalloc(pattern)", __FILE__, __LINE__); }
    p->block = blk;
  }
  p->m = m; p->n = n; p->nnz = nnz;
  Arena real; real.base = (char*)blk; real.cap = a.off;
  layout(real, *p);

  auto cleanup = [&](svt_status st) { svt_pattern_destroy(p); return st; };

  if (nnz == 0) {
    if (cudaMemsetAsync(p->row_ptr, 0, (m + 1) * sizeof(int32_t), s) != cudaSuccess ||
        cudaMemsetAsync(p->col_ptr, 0, (n + 1) * sizeof(int32_t), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return cleanup(cuda_fail(cudaGetLastError(), "pattern: zero fill", __FILE__, __LINE__));
    *out = p;
    return SVT_OK;
  }

  // Scratch: two key/value buffer pairs, a histogram, a flags word.
  uint64_t *k0, *k1;
  int32_t *v0, *v1, *hist;
  unsigned* flags;
  DeviceBlock scratch;
  {
    svt_status st = scratch.alloc(pattern_scratch_bytes(nnz), s);
    if (st < 0) return cleanup(st);
  }
  Arena sa;
  sa.base = (char*)scratch.ptr;
  scratch_layout(sa, nnz, &k0, &k1, &v0, &v1, &hist, &flags);

  auto run = [&]() -> svt_status {
    SVT_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), s));
    const int g = grid_for(nnz, 256);
    k_make_keys<<<g, 256, 0, s>>>(nnz, rows, cols, m, n, k0, v0, flags);
    SVT_LAUNCH_CHECK();
    unsigned hflags = 0;
    SVT_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SVT_CUDA(cudaStreamSynchronize(s));
    if (hflags & FLAG_INDEX) return fail(SVT_ERR_INDEX, "pattern: index out of range");

    uint64_t* keys[2] = {k0, k1};
    int32_t* vals[2] = {v0, v1};
    int res = 0;
    SVT_TRY(radix_sort(nnz, bits_for((uint64_t)m * (uint64_t)n), keys, vals, hist, s, &res));
    // CSR: rows and columns of the sorted keys; csr_src = payload.
    k_split_csr<<<g, 256, 0, s>>>(nnz, keys[res], n, p->csr_row, p->col_idx, flags);
    SVT_LAUNCH_CHECK();
    SVT_CUDA(cudaMemcpyAsync(p->csr_src, vals[res], nnz * sizeof(int32_t),
                             cudaMemcpyDeviceToDevice, s));
    k_offsets<<<grid_for(m + 1, 256), 256, 0, s>>>(nnz, p->csr_row, m, p->row_ptr);
    SVT_LAUNCH_CHECK();
    // CSC: sort CSR slots by (col, row); payload = CSR slot.
    k_make_csc_keys<<<g, 256, 0, s>>>(nnz, p->csr_row, p->col_idx, m, keys[0], vals[0]);
    SVT_LAUNCH_CHECK();
    SVT_TRY(radix_sort(nnz, bits_for((uint64_t)m * (uint64_t)n), keys, vals, hist, s, &res));
    int32_t* col_of = (int32_t*)keys[res ^ 1];  // free buffer reused as scratch
    k_split_csc<<<g, 256, 0, s>>>(nnz, keys[res], m, p->row_idx, col_of);
    SVT_LAUNCH_CHECK();
    SVT_CUDA(cudaMemcpyAsync(p->perm, vals[res], nnz * sizeof(int32_t),
                             cudaMemcpyDeviceToDevice, s));
    k_offsets<<<grid_for(n + 1, 256), 256, 0, s>>>(nnz, col_of, n, p->col_ptr);
    SVT_LAUNCH_CHECK();
    k_chunk_rows<<<grid_for(p->nchunks, 256), 256, 0, s>>>(m, p->chunk, p->nchunks, p->row_ptr,
                                                          p->chunk_row_csr);
    SVT_LAUNCH_CHECK();
    k_chunk_rows<<<grid_for(p->nchunks, 256), 256, 0, s>>>(n, p->chunk, p->nchunks, p->col_ptr,
                                                          p->chunk_row_csc);
    SVT_LAUNCH_CHECK();
    SVT_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SVT_CUDA(cudaStreamSynchronize(s));
    if (hflags & FLAG_DUPLICATE) return fail(SVT_ERR_DUPLICATE, "pattern: duplicate (row, col) entry");
    return SVT_OK;
  };
  svt_status st = run();
  if (st < 0) {
    cudaStreamSynchronize(s);
    return cleanup(st);
  }
  *out = p;
  return SVT_OK;
}

size_t pattern_block_bytes(int64_t m, int64_t n, int64_t nnz) {
  Arena a;
  svt_pattern probe;
  pattern_layout(a, m, n, nnz, &probe);
  return a.off;
}

size_t pattern_scratch_bytes(int64_t nnz) {
  if (nnz <= 0) return 0;
  Arena a;
  uint64_t *k0, *k1;
  int32_t *v0, *v1, *hist;
  unsigned* flags;
  scratch_layout(a, nnz, &k0, &k1, &v0, &v1, &hist, &flags);
  return a.off;
}

svt_status launch_chunk_rows(int64_t nrows, int64_t C, int64_t nchunks, const int32_t* ptr,
                             int32_t* out, cudaStream_t s) {
  if (nchunks <= 0) return SVT_OK;
  k_chunk_rows<<<grid_for(nchunks, 256), 256, 0, s>>>(nrows, C, nchunks, ptr, out);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

}  // namespace svt

extern "C" void svt_pattern_destroy(svt_pattern* p) {
  if (!p) return;
  if (p->block) cudaFree(p->block);
  delete p;
}

extern "C" int64_t svt_pattern_nnz(const svt_pattern* p) { return p ? p->nnz : -1; }

extern "C" svt_status svt_pattern_create(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                                         const int32_t* cols, void* stream, svt_pattern** out) {
  return svt::build_pattern(m, n, nnz, rows, cols, (cudaStream_t)stream, out);
}

extern "C" svt_status svt_pattern_export(const svt_pattern* p, int32_t* row_ptr, int32_t* col_idx,
                                         int32_t* csr_src, int32_t* col_ptr, int32_t* row_idx,
                                         int32_t* perm, void* stream) {
  using namespace svt;
  if (!p) return fail(SVT_ERR_ARG, "pattern_export: null pattern");
  cudaStream_t s = (cudaStream_t)stream;
  auto cp = [&](int32_t* dst, const int32_t* src, int64_t count) -> svt_status {
    if (dst && count > 0)
      SVT_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(int32_t), cudaMemcpyDefault, s));
    return SVT_OK;
  };
  SVT_TRY(cp(row_ptr, p->row_ptr, p->m + 1));
  SVT_TRY(cp(col_idx, p->col_idx, p->nnz));
  SVT_TRY(cp(csr_src, p->csr_src, p->nnz));
  SVT_TRY(cp(col_ptr, p->col_ptr, p->n + 1));
  SVT_TRY(cp(row_idx, p->row_idx, p->nnz));
  SVT_TRY(cp(perm, p->perm, p->nnz));
  SVT_CUDA(cudaStreamSynchronize(s));
  return SVT_OK;
}
