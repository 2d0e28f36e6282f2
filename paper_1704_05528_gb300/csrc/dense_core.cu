// The dense-row core of the fused sampled update and recycled product on the tensor cores
// (binary32 solver path).
//
// Every SVT iteration evaluates X = U W^T on Lambda, updates Y += delta P_Lambda(A - X)
// (eq. (4)-(5)) and, for the next R4SVD call, forms B^T = Y_new^T U (Algorithm 3 with the
// recycled basis U).  On the gather path each observed entry fetches a whole row of U
// from L2, which bounds that kernel.  Observation patterns with popular rows (ratings:
// a few thousand users rate a large share of all items) put a large part of Lambda into
// a few rows: on the 71,567 x 10,681 workload the 1,152 rows with at least n/10 entries
// hold half of the entries at 37% density.  Those rows form the "dense core", stored as
// a dense n x ldd panel in column-of-A order (element (q, slot) = entry (row[slot], q)),
// kept tile-major in 128 x 128 blocks, unobserved positions holding a NaN in A and a zero
// in Y.  On the core the two products
// are dense GEMMs on tcgen05 (three TF32 products per term, binary32 accuracy):
//   X^T[q, slot] = sum_j W[q, j] U[row[slot], j]          (k_core_update, M = q, N = slot)
//       epilogue: where A is observed, d = A - x, Y += delta d, sums of d^2, |d|, Y_new^2
//   B^T[q, j]   += sum_slot Y[q, slot] U[row[slot], j]     (k_core_bt, M = q, N = j)
// The remaining entries ("sparse rest") form their own CSC pattern and go through the
// gather kernel as before; the core adds its part of B^T after it, and its sums after the
// rest's, in a fixed order, so results do not depend on scheduling.
//
// Every wait is bounded: a wait that runs out raises FLAG_TC_TIMEOUT in the status word,
// the CTA stops issuing work, waits (bounded) for what it issued and releases its tensor
// memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "dense_core.cuh"
#include "kernels.cuh"
#include "solver.cuh"
#include "tc_common.cuh"

namespace svt {
namespace {
using namespace tc;

constexpr int kTile = 128;          // rows of an M tile, columns of an N tile
constexpr int kKC = 32;             // K columns per chunk: 128 bytes of binary32
constexpr int kChunkBytes = kTile * 128;  // one 128 x 32 binary32 chunk: 16 KB
constexpr int kThreads = 256;
constexpr int kKMax = 128;          // k <= 128 (four chunks)

// The core panels are stored tile-major: tile (q / 128, slot / 128) is one contiguous block
// of 128 x 128 values, element (q % 128, slot % 128) at (q % 128) * 128 + slot % 128, so a
// CTA working on one tile streams one 64 KB block.
__host__ __device__ __forceinline__ int64_t panel_off(int64_t q, int64_t slot, int64_t ldd) {
  const int64_t nptiles = ldd / kTile;
  return ((q / kTile) * nptiles + slot / kTile) * (int64_t)(kTile * kTile) + (q % kTile) * kTile +
         slot % kTile;
}
constexpr int kCoreMaxRows = 4096;  // largest automatic core

// ------------------------------------------------------------------ set-up kernels
// Per column q: number of entries of the sparse rest (rows without a core slot).
__global__ void k_count_rest(int32_t n, const int32_t* __restrict__ col_ptr,
                             const int32_t* __restrict__ row_idx, const int32_t* __restrict__ row_slot,
                             int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < n;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int c = 0;
    for (int32_t e = col_ptr[q] + lane; e < col_ptr[q + 1]; e += 32) c += row_slot[row_idx[e]] < 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) cnt[q] = c;
  }
}

// Exclusive prefix sum of cnt[0..len) into out[0..len] (out[len] = total), one block.
__global__ void __launch_bounds__(1024) k_scan_counts(int64_t len, const int32_t* __restrict__ cnt,
                                                      int32_t* __restrict__ out) {
  __shared__ int32_t s_part[1024];
  const int t = threadIdx.x;
  const int64_t per = (len + 1023) / 1024;
  const int64_t b = t * per, e = b + per < len ? b + per : len;
  int32_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += cnt[i];
  s_part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int32_t run = 0;
    for (int i = 0; i < 1024; ++i) { const int32_t v = s_part[i]; s_part[i] = run; run += v; }
  }
  __syncthreads();
  int32_t run = s_part[t];
  for (int64_t i = b; i < e; ++i) { out[i] = run; run += cnt[i]; }
  if (t == 1023) out[len] = run;
}

// Sparse-rest CSC arrays: for column q, its rest entries in CSC order (warp ballot
// compaction keeps the order), their rows and their slots in the full CSC order.
__global__ void k_compact_rest(int32_t n, const int32_t* __restrict__ col_ptr,
                               const int32_t* __restrict__ row_idx, const int32_t* __restrict__ row_slot,
                               const int32_t* __restrict__ rest_ptr, int32_t* __restrict__ rest_row,
                               int32_t* __restrict__ rest_full) {
  const int lane = threadIdx.x & 31;
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < n;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int32_t out = rest_ptr[q];
    for (int32_t e0 = col_ptr[q]; e0 < col_ptr[q + 1]; e0 += 32) {
      const int32_t e = e0 + lane;
      const bool in = e < col_ptr[q + 1];
      const int32_t row = in ? row_idx[e] : 0;
      const bool rest = in && row_slot[row] < 0;
      const unsigned bal = __ballot_sync(0xffffffffu, rest);
      if (rest) {
        const int32_t o = out + __popc(bal & ((1u << lane) - 1u));
        rest_row[o] = row;
        rest_full[o] = e;
      }
      out += __popc(bal);
    }
  }
}

// full_src[e] for each CSR slot e of the full pattern: the rest's CSC slot of the entry, or
// -(1 + panel offset of (q, slot)) for a core entry.
__global__ void k_full_src_core(int64_t z, const int32_t* __restrict__ csr_row,
                                const int32_t* __restrict__ col_idx, const int32_t* __restrict__ row_slot,
                                int64_t ldd, int32_t* __restrict__ full_src) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < z;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sl = row_slot[csr_row[e]];
    if (sl >= 0) full_src[e] = -(int32_t)(1 + panel_off(col_idx[e], sl, ldd));
  }
}
__global__ void k_full_src_rest(int64_t zr, const int32_t* __restrict__ rest_full,
                                const int32_t* __restrict__ perm, int32_t* __restrict__ full_src) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < zr;
       c += (int64_t)gridDim.x * blockDim.x)
    full_src[perm[rest_full[c]]] = (int32_t)c;
}

// Core panel from a full CSC-order vector: panel(q, slot) = src_csc[c] for core entries.
__global__ void k_scatter_core(int64_t z, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ csr_row, const int32_t* __restrict__ col_idx,
                               const int32_t* __restrict__ row_slot, int64_t ldd,
                               const float* __restrict__ src_csc, float* __restrict__ panel) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < z;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = perm[c];
    const int32_t sl = row_slot[csr_row[e]];
    if (sl >= 0) panel[panel_off(col_idx[e], sl, ldd)] = src_csc[c];
  }
}

// Full CSR-order Y from the rest (CSC order of the rest) and the core panel.
__global__ void k_assemble(int64_t z, const int32_t* __restrict__ full_src, const float* __restrict__ y_rest,
                           const float* __restrict__ y_core, float* __restrict__ y_csr) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < z;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = full_src[e];
    y_csr[e] = s >= 0 ? y_rest[s] : y_core[-(int64_t)s - 1];
  }
}

// W (n x k, ldw) copied to n x 128 (K-major, zero beyond k), for a W whose rows a tensor
// map cannot address directly (leading dimension not a multiple of four values).
__global__ void k_pad_w(int64_t n, int k, const float* __restrict__ W, int64_t ldw,
                        float* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * kKMax;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t >> 7;
    const int j = (int)(t & (kKMax - 1));
    out[t] = j < k ? W[q * ldw + j] : 0.f;
  }
}

// TF32 parts of the core rows of U (m x r, ldu): UD (ldd x 128, K-major, columns j < k)
// for the X product and UDt (npad x ldd, K-major, rows j < r) for the B^T product; zero in
// padding slots and beyond k / r.  A block (32 x 8 threads) takes 32 slots x 32 columns
// through shared memory, so both the row-major and the transposed writes are coalesced.
__global__ void __launch_bounds__(256) k_gather_ud(int64_t ldd, int k, int r, int npad,
                                                   const int32_t* __restrict__ slot_row,
                                                   const float* __restrict__ U, int64_t ldu,
                                                   float* __restrict__ ud_hi, float* __restrict__ ud_lo,
                                                   float* __restrict__ udt_hi, float* __restrict__ udt_lo) {
  __shared__ float th[32][33], tl[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t s0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int i = ty; i < 32; i += 8) {  // slot s0 + i, column j0 + tx
    const int64_t sl = s0 + i;
    const int j = j0 + tx;
    const int32_t row = sl < ldd ? slot_row[sl] : -1;
    const float u = (row >= 0 && j < r) ? U[(int64_t)row * ldu + j] : 0.f;
    const float h = tf32_round(u), l = u - h;
    th[i][tx] = h;
    tl[i][tx] = l;
    if (sl < ldd) {
      ud_hi[sl * kKMax + j] = j < k ? h : 0.f;
      ud_lo[sl * kKMax + j] = j < k ? l : 0.f;
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {  // column j0 + i, slot s0 + tx
    const int j = j0 + i;
    const int64_t sl = s0 + tx;
    if (j < npad && sl < ldd) {
      udt_hi[(int64_t)j * ldd + sl] = th[tx][i];
      udt_lo[(int64_t)j * ldd + sl] = tl[tx][i];
    }
  }
}

// ------------------------------------------------------------------ X^T and the update
constexpr int kUpdStages = 3;
constexpr int kUpdB = 2 * 4 * kChunkBytes;              // U_D tile, 4 chunks, hi and lo
constexpr int kUpdA = kUpdStages * 2 * kChunkBytes;     // ring of W chunks, hi and lo
constexpr int kUpdBytes = kUpdB + kUpdA + 256 + 1024;   // + barriers, 1024-byte alignment slack
constexpr uint32_t kUpdTmemCols = 256;                  // two 128-column accumulators

// CTA (pt, g): the slot tile pt (128 slots of the core) with its U_D tile resident in shared
// memory, and the q tiles g, g + G, ... of W streamed by TMA.  The MMA computes X[slot, q]
// (M = 128 slots, N = 128 q, K = k), so a tensor-memory lane is a slot and the 32 lanes of
// a warp read and write 32 consecutive slots of one panel row q: 128 contiguous bytes.
// Warp 0 loads (chunks of W as they are, zero beyond k), warps 2-3 split each chunk in
// place into its TF32 high part and a low-part copy, warp 1 issues the MMAs into one of two
// accumulators, warps 4-11 apply the update from the other (warp 4 + 4h + i: lanes
// 32i .. 32i + 31, q columns 64h .. 64h + 63).
constexpr int kUpdThreads = 384;
template <int NK>
__global__ void __launch_bounds__(kUpdThreads, 1)
k_core_update(int n, int nptiles, int nqgroups, const __grid_constant__ CUtensorMap mW,
              const __grid_constant__ CUtensorMap mUhi,
              const __grid_constant__ CUtensorMap mUlo, const float* __restrict__ A,
              float* __restrict__ Y, int64_t ldd, float delta, double* __restrict__ part,
              unsigned* __restrict__ flags, unsigned* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sB = smem;            // U_D tile: hi chunks 0..3, lo chunks 4..7
  unsigned char* sA = smem + kUpdB;    // ring of W chunks (hi, lo)
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kUpdB + kUpdA);
  uint64_t* barB = bar;
  uint64_t* barFull = bar + 1;                       // [S]
  uint64_t* barEmpty = barFull + kUpdStages;         // [S]
  uint64_t* barAccFull = barEmpty + kUpdStages;      // [2]
  uint64_t* barAccEmpty = barAccFull + 2;            // [2]
  uint64_t* barDrain = barAccEmpty + 2;
  uint64_t* barSplit = barDrain + 1;                 // [S] (64 arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barSplit + kUpdStages);
  __shared__ int s_abort;
  __shared__ double s_sum[8][3];
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pt = blockIdx.x % nptiles, g = blockIdx.x / nptiles;
  const int nq = (n + kTile - 1) / kTile;
  const int my_tiles = g < nq ? (nq - 1 - g) / nqgroups + 1 : 0;
  const int total = my_tiles * NK;
  if (tid == 0) {
    s_abort = 0;
    mbar_init(barB, 1);
    for (int s = 0; s < kUpdStages; ++s) {
      mbar_init(barFull + s, 1);
      mbar_init(barEmpty + s, 1);
      mbar_init(barSplit + s, 64);
    }
    for (int b = 0; b < 2; ++b) { mbar_init(barAccFull + b, 1); mbar_init(barAccEmpty + b, 256); }
    mbar_init(barDrain, 1);
    mbar_init_fence();
  }
  if (warp == 1) tmem_alloc(tmem_slot, kUpdTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  SumAcc<float> acc_d2, acc_abs, acc_y2;
  bool bad = false;

  if (warp == 0) {
    if (lane == 0) {  // producer
      mbar_expect_tx(barB, (uint32_t)(2 * NK * kChunkBytes));
      for (int c = 0; c < NK; ++c) {
        tma_load_2d(sB + c * kChunkBytes, &mUhi, c * kKC, pt * kTile, barB);
        tma_load_2d(sB + (4 + c) * kChunkBytes, &mUlo, c * kKC, pt * kTile, barB);
      }
      int issued = 0;
      for (int j = 0; j < total && !*abort_flag; ++j) {
        const int s = j % kUpdStages;
        if (j >= kUpdStages && !mbar_wait(barEmpty + s, (uint32_t)((j / kUpdStages - 1) & 1))) {
          *abort_flag = 1;
          break;
        }
        const int tile = g + (j / NK) * nqgroups, c = j % NK;
        mbar_expect_tx(barFull + s, (uint32_t)kChunkBytes);
        tma_load_2d(sA + s * 2 * kChunkBytes, &mW, c * kKC, tile * kTile, barFull + s);
        issued = j + 1;
      }
      // nothing may still land in shared memory when the CTA leaves
      mbar_wait(barB, 0);
      if (*abort_flag)
        for (int j = issued - kUpdStages > 0 ? issued - kUpdStages : 0; j < issued; ++j)
          mbar_wait(barFull + j % kUpdStages, (uint32_t)((j / kUpdStages) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer: A = U_D (slots), B = W (q)
      const uint32_t idesc = instr_desc_tf32(kTile, kTile);
      if (!mbar_wait(barB, 0)) *abort_flag = 1;
      int j = 0;
      for (int t = 0; t < my_tiles && !*abort_flag; ++t) {
        const int b = t & 1;
        const uint32_t acc = tmem + (uint32_t)(b * kTile);
        if (t >= 2 && !mbar_wait(barAccEmpty + b, (uint32_t)((t / 2 - 1) & 1))) { *abort_flag = 1; break; }
        fence_after_sync();
        for (int c = 0; c < NK; ++c, ++j) {
          const int s = j % kUpdStages;
          if (!mbar_wait(barSplit + s, (uint32_t)((j / kUpdStages) & 1))) { *abort_flag = 1; break; }
          fence_after_sync();
          const unsigned char* w_hi = sA + s * 2 * kChunkBytes;
          const unsigned char* w_lo = w_hi + kChunkBytes;
          const unsigned char* u_hi = sB + c * kChunkBytes;
          const unsigned char* u_lo = sB + (4 + c) * kChunkBytes;
#pragma unroll
          for (int kk = 0; kk < kKC / 8; ++kk) {
            const uint64_t uh = smem_desc(u_hi + kk * 32), ul = smem_desc(u_lo + kk * 32);
            const uint64_t wh = smem_desc(w_hi + kk * 32), wl = smem_desc(w_lo + kk * 32);
            mma_tf32(acc, uh, wh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(acc, uh, wl, idesc, 1u);
            mma_tf32(acc, ul, wh, idesc, 1u);
          }
          mma_commit(barEmpty + s);
          if (c == NK - 1) mma_commit(barAccFull + b);
        }
      }
    }
  } else if (warp == 2 || warp == 3) {  // split each landed chunk of W into TF32 parts
    const int t64 = tid - 64;
    for (int j = 0; j < total && !*abort_flag; ++j) {
      const int s = j % kUpdStages;
      if (!mbar_wait(barFull + s, (uint32_t)((j / kUpdStages) & 1))) { *abort_flag = 1; break; }
      float4* hi4 = reinterpret_cast<float4*>(sA + s * 2 * kChunkBytes);
      float4* lo4 = reinterpret_cast<float4*>(sA + s * 2 * kChunkBytes + kChunkBytes);
#pragma unroll 4
      for (int i = t64; i < kChunkBytes / 16; i += 64) {  // elementwise: the swizzle is the same
        const float4 x = hi4[i];
        float4 h;
        h.x = tf32_round(x.x); h.y = tf32_round(x.y); h.z = tf32_round(x.z); h.w = tf32_round(x.w);
        hi4[i] = h;
        lo4[i] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
      fence_proxy_async();
      mbar_arrive(barSplit + s);
    }
  } else if (warp >= 4) {  // epilogue: thread = one slot, 64 q columns per warp
    const int lq = warp & 3, half = (warp - 4) >> 2;
    // the panel blocks of A and Y a tile reads (64 KB each), fetched into L2 one tile ahead
    auto prefetch_tile = [&](int t) {
      const int64_t base = ((int64_t)(g + t * nqgroups) * nptiles + pt) * (int64_t)(kTile * kTile);
      prefetch_l2(A + base, kTile * kTile * 4);
      prefetch_l2(Y + base, kTile * kTile * 4);
    };
    if (tid == 128 && my_tiles > 0) prefetch_tile(0);
    // Batches of 16 q rows, four per tile; the loads of the next batch are issued before
    // the current one is processed, so one batch of A and Y is always in flight.
    constexpr int kRows = 16;
    const int nb = my_tiles * (64 / kRows);
    auto load_batch = [&](int j, float (&av)[kRows], float (&yv)[kRows]) {
      const int t = j / (64 / kRows), bi = j % (64 / kRows);
      if (bi == 0 && tid == 128 && t + 1 < my_tiles) prefetch_tile(t + 1);
      const int tq = g + t * nqgroups;
      const int64_t q0 = (int64_t)tq * kTile + half * 64 + bi * kRows;
      const int64_t off = ((int64_t)tq * nptiles + pt) * (int64_t)(kTile * kTile) +
                          (int64_t)(half * 64 + bi * kRows) * kTile + lq * 32 + lane;
      const int live_n = (int)max((int64_t)0, min((int64_t)kRows, (int64_t)n - q0));
#pragma unroll
      for (int i = 0; i < kRows; ++i) {
        const bool live = i < live_n;
        av[i] = live ? __ldcs(A + off + i * kTile) : __int_as_float(0x7fffffff);
        yv[i] = live ? __ldcs(Y + off + i * kTile) : 0.f;
      }
    };
    // false when the accumulator wait ran out
    auto process = [&](int j, const float (&av)[kRows], const float (&yv)[kRows]) -> bool {
      const int t = j / (64 / kRows), bi = j % (64 / kRows);
      const int b = t & 1;
      if (bi == 0) {
        if (!mbar_wait(barAccFull + b, (uint32_t)((t / 2) & 1))) return false;
        fence_after_sync();
      }
      const int tq = g + t * nqgroups;
      float* yp = Y + ((int64_t)tq * nptiles + pt) * (int64_t)(kTile * kTile) +
                  (int64_t)(half * 64 + bi * kRows) * kTile + lq * 32 + lane;
      float x[kRows];
      tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(b * kTile + half * 64 + bi * kRows), x);
#pragma unroll
      for (int i = 0; i < kRows; ++i) {
        if (!isnan(av[i])) {  // observed (and q < n): the update of eq. (4)
          const float d = av[i] - x[i];
          const float yn = fmaf(delta, d, yv[i]);
          acc_d2.add_sq(d);
          acc_abs.add(fabsf(d));
          acc_y2.add_sq(yn);
          bad |= !isfinite(yn);
          __stcs(yp + i * kTile, yn);
        }
      }
      if (bi == 64 / kRows - 1) {
        fence_before_sync();
        mbar_arrive(barAccEmpty + b);
      }
      return true;
    };
    float a0[kRows], y0[kRows], a1[kRows], y1[kRows];
    if (nb > 0) load_batch(0, a0, y0);
    for (int j = 0; j < nb && !*abort_flag; j += 2) {
      if (j + 1 < nb) load_batch(j + 1, a1, y1);
      if (!process(j, a0, y0)) { *abort_flag = 1; break; }
      if (j + 1 < nb) {
        if (j + 2 < nb) load_batch(j + 2, a0, y0);
        if (!process(j + 1, a1, y1)) { *abort_flag = 1; break; }
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_NONFINITE);
  if (warp >= 4) {
    const double s0 = warp_sum(acc_d2.value()), s1 = warp_sum(acc_abs.value()),
                 s2 = warp_sum(acc_y2.value());
    if (lane == 0) { s_sum[warp - 4][0] = s0; s_sum[warp - 4][1] = s1; s_sum[warp - 4][2] = s2; }
  }
  __syncthreads();
  if (tid < 3) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_sum[w][tid];
    part[(int64_t)blockIdx.x * 3 + tid] = t;
  }
  if (tid == 0 && *abort_flag) atomicOr(status, FLAG_TC_TIMEOUT);
  if (warp == 1) {
    if (lane == 0 && *abort_flag) {
      mma_commit(barDrain);
      mbar_wait(barDrain, 0);
    }
    __syncwarp();
    fence_after_sync();
    tmem_dealloc(tmem, kUpdTmemCols);
  }
}

// ------------------------------------------------------------------ B^T += Y_core U_D
constexpr int kBtStages = 3;
constexpr int kBtSplitters = 192;  // warps 2-7 split the chunks of Y

template <int NPAD>
struct BtLayout {
  static constexpr int kBChunk = NPAD * 128;                     // bytes of one chunk of U_D^T
  static constexpr int kStage = 2 * kChunkBytes + 2 * kBChunk;   // Y hi, Y lo, U hi, U lo
  static constexpr int bytes = kBtStages * kStage + 256 + 1024;
  static constexpr uint32_t tmem_cols = NPAD <= 32 ? 32 : NPAD <= 64 ? 64 : 128;
};

// One CTA per q tile: B^T[q tile, :r] += Y[q tile, :] U_D, with K = ldd slots in chunks of
// 32.  Warp 0 loads a chunk of Y and of U_D^T (high and low parts), warps 2-7 split the
// chunk of Y in place into its TF32 parts, warp 1 issues the MMAs, and at the end warps
// 4-7 add the accumulator to the rows of B^T.
template <int NPAD>
__global__ void __launch_bounds__(kThreads, 1)
k_core_bt(int n, int nchunks, int r, const __grid_constant__ CUtensorMap mY,
          const __grid_constant__ CUtensorMap mUthi, const __grid_constant__ CUtensorMap mUtlo,
          const float* __restrict__ Ypanel, float* __restrict__ bt, int64_t ldb,
          unsigned* __restrict__ status) {
  using L = BtLayout<NPAD>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBtStages * L::kStage);
  uint64_t* barFull = bar;                      // [S]
  uint64_t* barSplit = barFull + kBtStages;     // [S] (64 arrivals)
  uint64_t* barEmpty = barSplit + kBtStages;    // [S]
  uint64_t* barAcc = barEmpty + kBtStages;
  uint64_t* barDrain = barAcc + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barDrain + 1);
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < kBtStages; ++s) {
      mbar_init(barFull + s, 1);
      mbar_init(barSplit + s, kBtSplitters);
      mbar_init(barEmpty + s, 1);
    }
    mbar_init(barAcc, 1);
    mbar_init(barDrain, 1);
    mbar_init_fence();
  }
  if (warp == 1) tmem_alloc(tmem_slot, L::tmem_cols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  auto stage = [&](int s) { return smem + s * L::kStage; };

  if (warp == 0) {
    if (lane == 0) {
      // this q tile's panel blocks (64 KB each, one per 128 slots), fetched into L2 one
      // block ahead of the chunk loads
      const int nptiles = nchunks / (kTile / kKC);
      const float* yblk = Ypanel + (int64_t)tile * nptiles * (kTile * kTile);
      prefetch_l2(yblk, kTile * kTile * 4);
      int issued = 0;
      for (int c = 0; c < nchunks && !*abort_flag; ++c) {
        const int s = c % kBtStages;
        const int pb = c / (kTile / kKC) + 1;
        if (c % (kTile / kKC) == 0 && pb < nptiles)
          prefetch_l2(yblk + (int64_t)pb * (kTile * kTile), kTile * kTile * 4);
        if (c >= kBtStages && !mbar_wait(barEmpty + s, (uint32_t)((c / kBtStages - 1) & 1))) {
          *abort_flag = 1;
          break;
        }
        unsigned char* st = stage(s);
        mbar_expect_tx(barFull + s, (uint32_t)(kChunkBytes + 2 * L::kBChunk));
        tma_load_4d(st, &mY, (c % (kTile / kKC)) * kKC, 0, c / (kTile / kKC), tile, barFull + s);
        tma_load_2d(st + 2 * kChunkBytes, &mUthi, c * kKC, 0, barFull + s);
        tma_load_2d(st + 2 * kChunkBytes + L::kBChunk, &mUtlo, c * kKC, 0, barFull + s);
        issued = c + 1;
      }
      if (*abort_flag)
        for (int c = issued - kBtStages > 0 ? issued - kBtStages : 0; c < issued; ++c)
          mbar_wait(barFull + c % kBtStages, (uint32_t)((c / kBtStages) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc_tf32(kTile, NPAD);
      for (int c = 0; c < nchunks && !*abort_flag; ++c) {
        const int s = c % kBtStages;
        if (!mbar_wait(barSplit + s, (uint32_t)((c / kBtStages) & 1))) { *abort_flag = 1; break; }
        fence_after_sync();
        const unsigned char* a_hi = stage(s);
        const unsigned char* a_lo = a_hi + kChunkBytes;
        const unsigned char* b_hi = a_hi + 2 * kChunkBytes;
        const unsigned char* b_lo = b_hi + L::kBChunk;
#pragma unroll
        for (int kk = 0; kk < kKC / 8; ++kk) {
          const uint64_t ah = smem_desc(a_hi + kk * 32), al = smem_desc(a_lo + kk * 32);
          const uint64_t bh = smem_desc(b_hi + kk * 32), bl = smem_desc(b_lo + kk * 32);
          mma_tf32(tmem, ah, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, ah, bl, idesc, 1u);
          mma_tf32(tmem, al, bh, idesc, 1u);
        }
        mma_commit(barEmpty + s);
        if (c == nchunks - 1) mma_commit(barAcc);
      }
    }
  } else {  // warps 2-7 split the chunks of Y; then warps 4-7 add the accumulator to B^T
    const int ts = tid - 64;
    for (int c = 0; c < nchunks && !*abort_flag; ++c) {
      const int s = c % kBtStages;
      if (!mbar_wait(barFull + s, (uint32_t)((c / kBtStages) & 1))) { *abort_flag = 1; break; }
      float4* hi4 = reinterpret_cast<float4*>(stage(s));
      float4* lo4 = reinterpret_cast<float4*>(stage(s) + kChunkBytes);
#pragma unroll 2
      for (int i = ts; i < kChunkBytes / 16; i += kBtSplitters) {
        const float4 x = hi4[i];
        float4 h;
        h.x = tf32_round(x.x); h.y = tf32_round(x.y); h.z = tf32_round(x.z); h.w = tf32_round(x.w);
        hi4[i] = h;
        lo4[i] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
      fence_proxy_async();
      mbar_arrive(barSplit + s);
    }
    if (warp < 4) {
      // warps 2-3 are done
    } else if (!*abort_flag && mbar_wait(barAcc, 0)) {
      // Accumulator rows -> a shared tile (the stages are idle once the last MMA has
      // completed) -> whole rows of B^T, read, added to and written back coalesced.  Warp
      // qw owns tile rows 32 qw .. 32 qw + 31 in both steps.
      const int qw = warp - 4;
      fence_after_sync();
      float* tileT = reinterpret_cast<float*>(smem);
      constexpr int kLd = NPAD + 1;  // odd: the 32 rows of a column fall in 32 banks
      static_assert(kTile * kLd * 4 <= kBtStages * L::kStage, "B^T staging tile");
      const int ql = qw * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < NPAD; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int u = 0; u < 16; ++u) tileT[ql * kLd + c0 + u] = v[u];
      }
      __syncwarp();
      constexpr int kCols = (NPAD + 31) / 32;
#pragma unroll 1
      for (int i0 = 0; i0 < 32; i0 += 8) {
        float cur[8][kCols];
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          const int64_t q = (int64_t)tile * kTile + qw * 32 + i0 + ii;
#pragma unroll
          for (int c = 0; c < kCols; ++c) {
            const int j = c * 32 + lane;
            cur[ii][c] = (q < n && j < r) ? bt[q * ldb + j] : 0.f;
          }
        }
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          const int64_t q = (int64_t)tile * kTile + qw * 32 + i0 + ii;
#pragma unroll
          for (int c = 0; c < kCols; ++c) {
            const int j = c * 32 + lane;
            if (q < n && j < r) bt[q * ldb + j] = cur[ii][c] + tileT[(qw * 32 + i0 + ii) * kLd + j];
          }
        }
      }
    } else {
      *abort_flag = 1;
    }
  }
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(status, FLAG_TC_TIMEOUT);
  if (warp == 1) {
    if (lane == 0 && *abort_flag) {
      mma_commit(barDrain);
      mbar_wait(barDrain, 0);
    }
    __syncwarp();
    fence_after_sync();
    tmem_dealloc(tmem, L::tmem_cols);
  }
}

// out3[c] += sum over the core's CTA partials, in CTA order (one block per component).
__global__ void __launch_bounds__(256)
k_core_finish(int nparts, const double* __restrict__ part, double* __restrict__ out3) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(int64_t)b * 3 + c];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out3[c] += s;
}

// The tile-major Y panel as a 4-D tensor (slot in tile, q in tile, slot tile, q tile) whose
// box (32 slots, 128 q, 1, 1) is one K chunk of a q tile: the layout of a 2-D box of 32 x 128.
bool encode_panel_4d(CUtensorMap* map, const float* base, int64_t nptiles, int64_t nqt) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t gdim[4] = {(cuuint64_t)kTile, (cuuint64_t)kTile, (cuuint64_t)nptiles, (cuuint64_t)nqt};
  cuuint64_t gstr[3] = {(cuuint64_t)kTile * 4, (cuuint64_t)kTile * kTile * 4,
                        (cuuint64_t)nptiles * kTile * kTile * 4};
  cuuint32_t box[4] = {(cuuint32_t)kKC, (cuuint32_t)kTile, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int egrid(int64_t work) {
  const int64_t g = ceil_div(work > 0 ? work : 1, 256);
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)(g < cap ? g : cap);
}

std::mutex g_core_mu;
uint64_t g_core_devices = 0;

template <int NPAD>
cudaError_t bt_smem() {
  return cudaFuncSetAttribute(k_core_bt<NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              BtLayout<NPAD>::bytes);
}
template <int NK>
cudaError_t upd_smem() {
  return cudaFuncSetAttribute(k_core_update<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kUpdBytes);
}

svt_status core_prepare() {
  int dev = 0;
  SVT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_core_mu);
  const uint64_t bit = 1ull << (dev & 63);
  if (g_core_devices & bit) return SVT_OK;
  if (!encode_fn()) return fail(SVT_ERR_UNSUPPORTED, "dense core: no tensor map encoder");
  SVT_CUDA(upd_smem<1>()); SVT_CUDA(upd_smem<2>()); SVT_CUDA(upd_smem<3>()); SVT_CUDA(upd_smem<4>());
  SVT_CUDA(bt_smem<16>()); SVT_CUDA(bt_smem<32>()); SVT_CUDA(bt_smem<48>()); SVT_CUDA(bt_smem<64>());
  SVT_CUDA(bt_smem<80>()); SVT_CUDA(bt_smem<96>()); SVT_CUDA(bt_smem<112>()); SVT_CUDA(bt_smem<128>());
  g_core_devices |= bit;
  return SVT_OK;
}

}  // namespace

// ------------------------------------------------------------------ host interface
svt_status core_plan(const svt_pattern* p, int want_rows, double min_frac, cudaStream_t s,
                     CorePlan* plan) {
  *plan = CorePlan();
  const int64_t m = p->m, n = p->n, z = p->nnz;
  if (z == 0 || want_rows == 0 || n < 1) return SVT_OK;
  std::vector<int32_t> ptr(m + 1);
  SVT_CUDA(cudaMemcpyAsync(ptr.data(), p->row_ptr, (m + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SVT_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> order(m);
  std::iota(order.begin(), order.end(), 0);
  auto cnt = [&](int32_t r) { return ptr[r + 1] - ptr[r]; };
  // rows by entry count, most first (ties: lower row first)
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cnt(a) > cnt(b); });
  int64_t rd = 0;
  if (want_rows > 0) {
    rd = std::min<int64_t>(want_rows, m);
  } else {  // automatic: rows with at least min_frac * n entries, whole tiles of 128
    while (rd < m && rd < kCoreMaxRows && cnt(order[rd]) >= min_frac * (double)n) ++rd;
    rd = rd / kTile * kTile;
  }
  if (rd <= 0) return SVT_OK;
  const int64_t ldd = round_up(rd, kTile);
  if (round_up(n, kTile) * ldd >= (int64_t)INT32_MAX - 1) return SVT_OK;  // panel offsets fit int32
  std::vector<int32_t> rows(order.begin(), order.begin() + rd);
  std::sort(rows.begin(), rows.end());
  plan->rd = (int)rd;
  plan->ldd = ldd;
  plan->slot_row.assign(ldd, -1);
  plan->row_slot.assign(m, -1);
  int64_t core_nnz = 0;
  for (int64_t sl = 0; sl < rd; ++sl) {
    plan->slot_row[sl] = rows[sl];
    plan->row_slot[rows[sl]] = (int32_t)sl;
    core_nnz += cnt(rows[sl]);
  }
  plan->core_nnz = core_nnz;
  plan->rest_nnz = z - core_nnz;
  return SVT_OK;
}

CorePlan core_plan_bound(int64_t m, int64_t n, int64_t nnz, int want_rows, double min_frac) {
  CorePlan b;
  if (nnz == 0 || want_rows == 0 || n < 1) return b;
  int64_t rd;
  if (want_rows > 0) {
    rd = std::min<int64_t>(want_rows, m);
  } else {  // a row in the core holds at least ceil(min_frac * n) entries
    const int64_t per_row = std::max<int64_t>(1, (int64_t)std::ceil(min_frac * (double)n));
    rd = std::min<int64_t>({m, (int64_t)kCoreMaxRows, nnz / per_row});
    rd = rd / kTile * kTile;
  }
  if (rd <= 0) return b;
  const int64_t ldd = round_up(rd, kTile);
  if (round_up(n, kTile) * ldd >= (int64_t)INT32_MAX - 1) return b;
  b.rd = (int)rd;
  b.ldd = ldd;
  b.core_nnz = 0;
  b.rest_nnz = nnz;
  return b;
}

void core_layout(Arena& a, const CorePlan& plan, int64_t m, int64_t n, int r_cap, DenseCore* C) {
  const int64_t ldd = plan.ldd, zr = plan.rest_nnz;
  C->m = m; C->n = n; C->rd = plan.rd; C->ldd = ldd;
  C->slot_row = a.take<int32_t>(ldd);
  C->row_slot = a.take<int32_t>(m);
  C->rest_ptr = a.take<int32_t>(n + 1);
  C->rest_cnt = a.take<int32_t>(n);
  C->rest_row = a.take<int32_t>(zr);
  C->rest_full = a.take<int32_t>(zr);
  C->rest.chunk = chunk_size(zr > 0 ? zr : 1);
  C->rest.nchunks = ceil_div(zr, C->rest.chunk);
  C->rest_chunk_col = a.take<int32_t>(C->rest.nchunks);
  C->a_rest = a.take<float>(zr);
  C->y_rest = a.take<float>(zr);
  C->A = a.take<float>(round_up(n, kTile) * ldd);
  C->Y = a.take<float>(round_up(n, kTile) * ldd);
  C->w_pad = a.take<float>(n * kKMax);
  C->ud_hi = a.take<float>(ldd * kKMax);
  C->ud_lo = a.take<float>(ldd * kKMax);
  C->udt_hi = a.take<float>(kKMax * ldd);
  C->udt_lo = a.take<float>(kKMax * ldd);
  C->part = a.take<double>(3 * (size_t)std::max(num_sms(), 1) * 2 + 8);
  C->upd_part = a.take<double>(update_recycle_scratch(zr > 0 ? zr : 1));
  C->upd_scratch = a.take<char>(spmm_scratch_bytes(zr > 0 ? zr : 1, std::max(r_cap, 1), 4));
  C->full_src = nullptr;  // set by the caller: it aliases no other buffer
}

svt_status core_build(const svt_pattern* p, const CorePlan& plan, const float* a_csc, int32_t* full_src,
                      cudaStream_t s, DenseCore* C) {
  const int64_t n = p->n, z = p->nnz, ldd = C->ldd, zr = plan.rest_nnz;
  C->full_src = full_src;
  SVT_CUDA(cudaMemcpyAsync(C->slot_row, plan.slot_row.data(), ldd * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  SVT_CUDA(cudaMemcpyAsync(C->row_slot, plan.row_slot.data(), p->m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  // the sparse rest as a CSC pattern of its own
  k_count_rest<<<egrid(n * 32), 256, 0, s>>>((int32_t)n, p->col_ptr, p->row_idx, C->row_slot, C->rest_cnt);
  SVT_LAUNCH_CHECK();
  k_scan_counts<<<1, 1024, 0, s>>>(n, C->rest_cnt, C->rest_ptr);
  SVT_LAUNCH_CHECK();
  k_compact_rest<<<egrid(n * 32), 256, 0, s>>>((int32_t)n, p->col_ptr, p->row_idx, C->row_slot,
                                                C->rest_ptr, C->rest_row, C->rest_full);
  SVT_LAUNCH_CHECK();
  SVT_TRY(launch_chunk_rows(n, C->rest.chunk, C->rest.nchunks, C->rest_ptr, C->rest_chunk_col, s));
  C->rest.m = p->m; C->rest.n = n; C->rest.nnz = zr;
  C->rest.col_ptr = C->rest_ptr;
  C->rest.row_idx = C->rest_row;
  C->rest.chunk_row_csc = C->rest_chunk_col;
  // where each full CSR entry lives: the rest's CSC slot or the core panel
  k_full_src_core<<<egrid(z), 256, 0, s>>>(z, p->csr_row, p->col_idx, C->row_slot, ldd, full_src);
  SVT_LAUNCH_CHECK();
  if (zr > 0) {
    k_full_src_rest<<<egrid(zr), 256, 0, s>>>(zr, C->rest_full, p->perm, full_src);
    SVT_LAUNCH_CHECK();
    SVT_TRY(launch_gather<float>(zr, C->rest_full, a_csc, C->a_rest, s));
  }
  // observed values on the core panel, NaN (all bits set) where nothing is observed
  SVT_CUDA(cudaMemsetAsync(C->A, 0xFF, round_up(n, kTile) * ldd * sizeof(float), s));
  k_scatter_core<<<egrid(z), 256, 0, s>>>(z, p->perm, p->csr_row, p->col_idx, C->row_slot, ldd, a_csc, C->A);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

svt_status core_enter(const svt_pattern* p, const float* y_csc, cudaStream_t s, DenseCore* C) {
  const int64_t z = p->nnz, zr = C->rest.nnz;
  if (zr > 0) SVT_TRY(launch_gather<float>(zr, C->rest_full, y_csc, C->y_rest, s));
  SVT_CUDA(cudaMemsetAsync(C->Y, 0, round_up(C->n, kTile) * C->ldd * sizeof(float), s));
  k_scatter_core<<<egrid(z), 256, 0, s>>>(z, p->perm, p->csr_row, p->col_idx, C->row_slot, C->ldd, y_csc, C->Y);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

svt_status core_assemble(const svt_pattern* p, const DenseCore& C, float* y_csr, float* y_csc,
                         cudaStream_t s) {
  const int64_t z = p->nnz;
  k_assemble<<<egrid(z), 256, 0, s>>>(z, C.full_src, C.y_rest, C.Y, y_csr);
  SVT_LAUNCH_CHECK();
  return launch_gather<float>(z, p->perm, y_csr, y_csc, s);
}

bool core_fits(int r, int k) { return r >= 1 && r <= kKMax && k >= 0 && k <= r; }

svt_status core_update(const DenseCore& C, const float* U, int64_t ldu, int r, const float* W,
                       int64_t ldw, int k, double delta, float* bt, int64_t ldb, double* out3,
                       unsigned* flags, unsigned* tc_status, cudaStream_t s) {
  if (!core_fits(r, k)) return fail(SVT_ERR_UNSUPPORTED, "dense core: r = %d, k = %d", r, k);
  SVT_TRY(core_prepare());
  const int64_t n = C.n, ldd = C.ldd;
  const int npad = (int)round_up(r, 16);
  const int nk = (int)ceil_div(k, kKC);
  const int nptiles = (int)(ldd / kTile);
  const int nq = (int)ceil_div(n, kTile);
  // W is read by the update kernel through a tensor map (columns beyond k read as zero) and
  // split into its TF32 parts in shared memory; a W that a map cannot address is copied
  // into a padded buffer first, and k = 0 maps a zeroed one (X = 0 on the core)
  const bool w_direct = nk > 0 && ldw % 4 == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0;
  {
    SVT_PROF("core_split", 4.0 * (double)(ldd * r + 4 * ldd * kKMax) + (w_direct ? 0.0 : 4.0 * (double)(n * k + n * kKMax)), s);
    if (!w_direct) {
      if (nk > 0) {
        k_pad_w<<<egrid(n * kKMax), 256, 0, s>>>(n, k, W, ldw, C.w_pad);
        SVT_LAUNCH_CHECK();
      } else {
        SVT_CUDA(cudaMemsetAsync(C.w_pad, 0, n * kKMax * sizeof(float), s));
      }
    }
    k_gather_ud<<<dim3((unsigned)ceil_div(ldd, 32), kKMax / 32), 256, 0, s>>>(ldd, k, r, npad, C.slot_row, U, ldu,
                                                                           C.ud_hi, C.ud_lo, C.udt_hi, C.udt_lo);
    SVT_LAUNCH_CHECK();
  }
  CUtensorMap mW, mUh, mUl, mY, mTh, mTl;
  const uint64_t rowb = (uint64_t)kKMax * 4;
  const bool w_ok = w_direct ? encode_2d(&mW, W, (uint64_t)k, (uint64_t)n, (uint64_t)ldw * 4, kKC, kTile)
                             : encode_2d(&mW, C.w_pad, kKMax, (uint64_t)n, rowb, kKC, kTile);
  if (!w_ok ||
      !encode_2d(&mUh, C.ud_hi, kKMax, (uint64_t)ldd, rowb, kKC, kTile) ||
      !encode_2d(&mUl, C.ud_lo, kKMax, (uint64_t)ldd, rowb, kKC, kTile) ||
      !encode_panel_4d(&mY, C.Y, ldd / kTile, ceil_div(n, kTile)) ||
      !encode_2d(&mTh, C.udt_hi, (uint64_t)ldd, (uint64_t)npad, (uint64_t)ldd * 4, kKC, (uint32_t)npad) ||
      !encode_2d(&mTl, C.udt_lo, (uint64_t)ldd, (uint64_t)npad, (uint64_t)ldd * 4, kKC, (uint32_t)npad))
    return fail(SVT_ERR_CUDA, "dense core: tensor map encoding failed");
  // X on the core and the update (k = 0: X = 0, the update still applies)
  const int nqg = std::max(1, std::min(nq, num_sms() / std::max(nptiles, 1)));
  const int grid1 = nptiles * nqg;
#define SVT_UPD(NK)                                                                                  \
  case NK:                                                                                           \
    k_core_update<NK><<<grid1, kUpdThreads, kUpdBytes, s>>>((int)n, nptiles, nqg, mW, mUh, mUl,  \
                                                         C.A, C.Y, ldd, (float)delta, C.part, flags, \
                                                         tc_status);                                 \
    break
  {
    SVT_PROF("core_x_update", 12.0 * (double)(n * ldd) + 8.0 * (double)n * kKMax, s);
    switch (nk > 0 ? nk : 1) {
      SVT_UPD(1); SVT_UPD(2); SVT_UPD(3); SVT_UPD(4);
      default: return fail(SVT_ERR_UNSUPPORTED, "dense core: k = %d", k);
    }
    SVT_LAUNCH_CHECK();
  }
#undef SVT_UPD
  // B^T += Y_core U_D
  const int nchunks = (int)(ldd / kKC);
#define SVT_BT(NP)                                                                                   \
  case NP:                                                                                           \
    k_core_bt<NP><<<nq, kThreads, BtLayout<NP>::bytes, s>>>((int)n, nchunks, r, mY, mTh, mTl, C.Y, bt, ldb, \
                                                            tc_status);                              \
    break
  {
    SVT_PROF("core_bt", 4.0 * (double)(n * ldd) + 8.0 * (double)npad * ldd + 8.0 * (double)n * r, s);
    switch (npad) {
      SVT_BT(16); SVT_BT(32); SVT_BT(48); SVT_BT(64); SVT_BT(80); SVT_BT(96); SVT_BT(112); SVT_BT(128);
      default: return fail(SVT_ERR_UNSUPPORTED, "dense core: r = %d", r);
    }
    SVT_LAUNCH_CHECK();
  }
#undef SVT_BT
  k_core_finish<<<3, 256, 0, s>>>(grid1, C.part, out3);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

}  // namespace svt
