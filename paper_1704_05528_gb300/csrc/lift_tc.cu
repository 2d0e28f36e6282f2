// U = Q U_B on the fifth-generation tensor cores (binary32 solver path).
//
// The lift of the basis (Algorithm 3: U = Q U_B, Q m x r, U_B r x r) is the one dense
// contraction of the hot path with a long dimension: m x r x r multiply-adds, about
// 0.7 GFMA for the 71,567 x 100 workload.  Binary32 accuracy comes from three TF32 products
// per term, A_hi B_hi + A_hi B_lo + A_lo B_hi, where x_hi is x rounded to TF32 and x_lo the
// rounded remainder; the dropped A_lo B_lo term is below 2^-22 of |a b|.
//
// One CTA per SM walks 128-row tiles of Q with warp-specialised stages.  The tensor memory
// accelerator brings each tile in 32-column chunks (128-byte rows, 128-byte swizzle) into
// a ring of two or three stages.  Two warps split a landed chunk in place into its TF32
// high part and a low-part copy (an elementwise operation, so the swizzled layout is
// kept); one thread issues the tcgen05.mma instructions (M = 128, N = r rounded up to 16,
// K = 8 each) that accumulate the tile in one of two tensor-memory accumulators; four
// warps read the other accumulator back with tcgen05.ld and store the previous tile.
// U_B^T, split the same way by a small kernel, stays in shared memory for the whole call.
//
// Every wait is bounded: a wait that runs out raises FLAG_TC_TIMEOUT in the status word,
// the CTA stops issuing work, waits (bounded) for what it issued and releases its tensor
// memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace svt {
namespace {
using namespace tc;

constexpr int kBM = 128;        // rows per tile: one tensor-memory lane per row
constexpr int kKC = 32;         // K columns per chunk: 128 bytes of binary32
constexpr int kMaxChunks = 4;   // K <= 128
constexpr int kThreads = 256;
// Stages of the A ring: as many 32 KB stages (high and low part of a 128 x 32 chunk) as
// fit next to U_B^T.
template <int NPAD>
struct Layout {
  static constexpr int kBChunk = NPAD * 128;           // bytes of one K chunk of U_B^T
  static constexpr int kB = 2 * kMaxChunks * kBChunk;  // high and low parts
  static constexpr int kAChunk = kBM * 128;            // 16 KB
  static constexpr int kStages = (kB + 3 * 2 * kAChunk + 2048 <= 232448) ? 3 : 2;
  static constexpr int kA = kStages * 2 * kAChunk;
  static constexpr int kBar = 256;
  static constexpr int bytes = kB + kA + kBar + 1024;  // + 1024-byte alignment slack
  // two accumulators (tile t in buffer t & 1) 32-column aligned, in a power of two of
  // tensor-memory columns
  static constexpr int kAccStride = (NPAD + 31) / 32 * 32;
  static constexpr int kCols = kAccStride + NPAD;
  static constexpr int tmem_cols = kCols <= 32 ? 32 : kCols <= 64 ? 64 : kCols <= 128 ? 128 : kCols <= 256 ? 256 : 512;
};

// Warp roles: warp 0 requests chunks of A (TMA), warps 2-3 split them into TF32 parts,
// warp 1 issues the MMAs, warps 4-7 read the accumulators back (warp 4 + i owns tensor
// memory lanes 32i .. 32i + 31) and store the tiles.  Tiles alternate between two
// accumulators, so the store of tile t overlaps the MMAs of tile t + 1.
template <int NPAD>
__global__ void __launch_bounds__(kThreads, 1)
k_lift_tf32x3(int M, int N, int K, const __grid_constant__ CUtensorMap mapA,
              const __grid_constant__ CUtensorMap mapBhi, const __grid_constant__ CUtensorMap mapBlo,
              float* __restrict__ C, int64_t ldc, unsigned* __restrict__ status) {
  using L = Layout<NPAD>;
  constexpr int S = L::kStages;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sB = smem;
  unsigned char* sA = smem + L::kB;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::kB + L::kA);
  uint64_t* barB = bar;                  // U_B^T has landed
  uint64_t* barFull = bar + 1;           // [S] a chunk of A has landed
  uint64_t* barSplit = barFull + S;      // [S] the chunk is split (two arrivals)
  uint64_t* barEmpty = barSplit + S;     // [S] the MMAs that read the stage have completed
  uint64_t* barAccFull = barEmpty + S;   // [2] an accumulator holds a finished tile
  uint64_t* barAccEmpty = barAccFull + 2;  // [2] its tile has been stored (128 arrivals)
  uint64_t* barDrain = barAccEmpty + 2;    // every MMA issued so far has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barDrain + 1);
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nchunks = (K + kKC - 1) / kKC;
  const int ntiles = (M + kBM - 1) / kBM;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int total = my_tiles * nchunks;
  if (tid == 0) {
    s_abort = 0;
    mbar_init(barB, 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(barFull + s, 1);
      mbar_init(barSplit + s, 64);
      mbar_init(barEmpty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(barAccFull + b, 1);
      mbar_init(barAccEmpty + b, 128);
    }
    mbar_init(barDrain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tmem_slot)),
                 "r"((uint32_t)L::tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // producer
      mbar_expect_tx(barB, (uint32_t)(2 * nchunks * L::kBChunk));
      for (int c = 0; c < nchunks; ++c) {
        tma_load_2d(sB + c * L::kBChunk, &mapBhi, c * kKC, 0, barB);
        tma_load_2d(sB + (kMaxChunks + c) * L::kBChunk, &mapBlo, c * kKC, 0, barB);
      }
      int issued = 0;
      for (int j = 0; j < total && !*abort_flag; ++j) {
        const int s = j % S;
        if (j >= S && !mbar_wait(barEmpty + s, (uint32_t)((j / S - 1) & 1))) { *abort_flag = 1; break; }
        const int tile = blockIdx.x + (j / nchunks) * gridDim.x, c = j % nchunks;
        mbar_expect_tx(barFull + s, (uint32_t)L::kAChunk);
        tma_load_2d(sA + s * 2 * L::kAChunk, &mapA, c * kKC, tile * kBM, barFull + s);
        issued = j + 1;
      }
      // after a failure nothing may still land in shared memory when the CTA leaves:
      // bounded waits for the last load of each stage
      if (*abort_flag)
        for (int j = issued - S > 0 ? issued - S : 0; j < issued; ++j)
          mbar_wait(barFull + j % S, (uint32_t)((j / S) & 1));
    }
  } else if (warp == 2 || warp == 3) {  // split: 64 threads per chunk
    const int t64 = tid - 64;
    for (int j = 0; j < total && !*abort_flag; ++j) {
      const int s = j % S;
      if (!mbar_wait(barFull + s, (uint32_t)((j / S) & 1))) { *abort_flag = 1; break; }
      float4* hi4 = reinterpret_cast<float4*>(sA + s * 2 * L::kAChunk);
      float4* lo4 = reinterpret_cast<float4*>(sA + s * 2 * L::kAChunk + L::kAChunk);
#pragma unroll 4
      for (int i = t64; i < L::kAChunk / 16; i += 64) {
        const float4 x = hi4[i];
        float4 h;
        h.x = tf32_round(x.x); h.y = tf32_round(x.y); h.z = tf32_round(x.z); h.w = tf32_round(x.w);
        hi4[i] = h;
        lo4[i] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(barSplit + s)) : "memory");
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = instr_desc_tf32(kBM, NPAD);
      if (!mbar_wait(barB, 0)) *abort_flag = 1;
      int j = 0;
      for (int t = 0; t < my_tiles && !*abort_flag; ++t) {
        const int b = t & 1;
        const uint32_t acc = tmem + (uint32_t)(b * L::kAccStride);
        if (t >= 2 && !mbar_wait(barAccEmpty + b, (uint32_t)((t / 2 - 1) & 1))) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = 0; c < nchunks; ++c, ++j) {
          const int s = j % S;
          if (!mbar_wait(barSplit + s, (uint32_t)((j / S) & 1))) { *abort_flag = 1; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned char* a_hi = sA + s * 2 * L::kAChunk;
          const unsigned char* a_lo = a_hi + L::kAChunk;
          const unsigned char* b_hi = sB + c * L::kBChunk;
          const unsigned char* b_lo = sB + (kMaxChunks + c) * L::kBChunk;
#pragma unroll
          for (int kk = 0; kk < kKC / 8; ++kk) {  // K = 8 per instruction: 32 bytes along the row
            const uint64_t ah = smem_desc(a_hi + kk * 32), al = smem_desc(a_lo + kk * 32);
            const uint64_t bh = smem_desc(b_hi + kk * 32), bl = smem_desc(b_lo + kk * 32);
            mma_tf32(acc, ah, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(acc, ah, bl, idesc, 1u);
            mma_tf32(acc, al, bh, idesc, 1u);
          }
          mma_commit(barEmpty + s);
          if (c == nchunks - 1) mma_commit(barAccFull + b);
        }
      }
    }
  } else {  // warps 4-7: store the tiles
    const int q = warp - 4;
    for (int t = 0; t < my_tiles && !*abort_flag; ++t) {
      const int b = t & 1;
      if (!mbar_wait(barAccFull + b, (uint32_t)((t / 2) & 1))) { *abort_flag = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int tile = blockIdx.x + t * gridDim.x;
      const int64_t row = (int64_t)tile * kBM + q * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < NPAD; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * L::kAccStride + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
          float* dst = C + row * ldc + c0;
          if (c0 + 16 <= N) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              reinterpret_cast<float4*>(dst)[u] =
                  make_float4(__uint_as_float(v[4 * u]), __uint_as_float(v[4 * u + 1]),
                              __uint_as_float(v[4 * u + 2]), __uint_as_float(v[4 * u + 3]));
          } else {
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (c0 + u < N) dst[u] = __uint_as_float(v[u]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(barAccEmpty + b)) : "memory");
    }
  }
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(status, FLAG_TC_TIMEOUT);
  if (warp == 1) {
    // no MMA may still write the accumulators when they are released (bounded wait for a
    // commit that tracks everything issued)
    if (lane == 0 && *abort_flag) {
      mma_commit(barDrain);
      mbar_wait(barDrain, 0);
    }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)L::tmem_cols)
                 : "memory");
  }
}

// Bt_hi, Bt_lo (npad x 128, K-major) = TF32 parts of (binary32) B^T for B (K x N, binary64,
// row-major, ldb); zero outside K x N.
__global__ void k_split_bt(int K, int N, int npad, const double* __restrict__ B, int64_t ldb,
                           float* __restrict__ bhi, float* __restrict__ blo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npad * 128) return;
  const int n = t / 128, k = t % 128;
  float h = 0.f, l = 0.f;
  if (n < N && k < K) {
    const float b = (float)B[(int64_t)k * ldb + n];
    h = tf32_round(b);
    l = b - h;
  }
  bhi[t] = h;
  blo[t] = l;
}

template <int NPAD>
cudaError_t set_smem_limit() {
  return cudaFuncSetAttribute(k_lift_tf32x3<NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Layout<NPAD>::bytes);
}

// shared-memory limits of every instantiation, once per device
std::mutex g_prep_mu;
uint64_t g_prep_devices = 0;

template <int NPAD>
svt_status launch_lift(int64_t M, int K, int N, const CUtensorMap& mA, const CUtensorMap& mBh,
                       const CUtensorMap& mBl, float* C, int64_t ldc, unsigned* status,
                       cudaStream_t s) {
  using L = Layout<NPAD>;
  const int64_t ntiles = ceil_div(M, (int64_t)kBM);
  const int grid = (int)(ntiles < num_sms() ? ntiles : num_sms());
  k_lift_tf32x3<NPAD><<<grid, kThreads, L::bytes, s>>>((int)M, N, K, mA, mBh, mBl, C, ldc, status);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

}  // namespace

namespace tc {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

bool encode_2d(CUtensorMap* map, const float* base, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t gstr[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

// N rounded up to a tile width with an instantiated kernel (shared memory holds U_B^T
// for up to 160 columns next to the two-stage ring)
int lift_npad(int N) { return N <= 128 ? (int)round_up(N, 16) : N <= 144 ? 144 : 160; }

size_t lift_tc_scratch_floats() { return (size_t)2 * 160 * 128; }

svt_status lift_tc_prepare() {
  int dev = 0;
  SVT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_prep_mu);
  const uint64_t bit = 1ull << (dev & 63);
  if (g_prep_devices & bit) return SVT_OK;
  if (!tc::encode_fn()) return fail(SVT_ERR_UNSUPPORTED, "tensor-core lift: no tensor map encoder");
  SVT_CUDA(set_smem_limit<16>()); SVT_CUDA(set_smem_limit<32>()); SVT_CUDA(set_smem_limit<48>());
  SVT_CUDA(set_smem_limit<64>()); SVT_CUDA(set_smem_limit<80>()); SVT_CUDA(set_smem_limit<96>());
  SVT_CUDA(set_smem_limit<112>()); SVT_CUDA(set_smem_limit<128>()); SVT_CUDA(set_smem_limit<144>());
  SVT_CUDA(set_smem_limit<160>());
  g_prep_devices |= bit;
  return SVT_OK;
}

bool lift_tc_fits(int64_t M, int K, int N, const float* A, int64_t lda, const float* C, int64_t ldc) {
  return M > 0 && M < (int64_t)INT32_MAX - kBM && K >= 1 && K <= kMaxChunks * kKC && N >= 1 &&
         N <= 160 && lda % 4 == 0 && ldc % 4 == 0 && lda >= K && ldc >= N &&
         reinterpret_cast<uintptr_t>(A) % 16 == 0 && reinterpret_cast<uintptr_t>(C) % 16 == 0 &&
         tc::encode_fn() != nullptr;
}

svt_status lift_tc(int64_t M, int K, int N, const float* A, int64_t lda, const double* B,
                   int64_t ldb, float* C, int64_t ldc, float* scratch, unsigned* status,
                   cudaStream_t s) {
  if (!lift_tc_fits(M, K, N, A, lda, C, ldc))
    return fail(SVT_ERR_UNSUPPORTED, "tensor-core lift: unsupported shape or alignment");
  SVT_TRY(lift_tc_prepare());
  const int npad = lift_npad(N);
  float* bhi = scratch;
  float* blo = scratch + (size_t)npad * 128;
  k_split_bt<<<(int)ceil_div((int64_t)npad * 128, 256), 256, 0, s>>>(K, N, npad, B, ldb, bhi, blo);
  SVT_LAUNCH_CHECK();
  CUtensorMap mA, mBh, mBl;
  if (!tc::encode_2d(&mA, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda * 4, kKC, kBM) ||
      !tc::encode_2d(&mBh, bhi, 128, (uint64_t)npad, 128 * 4, kKC, (uint32_t)npad) ||
      !tc::encode_2d(&mBl, blo, 128, (uint64_t)npad, 128 * 4, kKC, (uint32_t)npad))
    return fail(SVT_ERR_CUDA, "tensor-core lift: tensor map encoding failed");
#define SVT_LIFT(NP) \
  case NP: return launch_lift<NP>(M, K, N, mA, mBh, mBl, C, ldc, status, s)
  switch (npad) {
    SVT_LIFT(16); SVT_LIFT(32); SVT_LIFT(48); SVT_LIFT(64); SVT_LIFT(80); SVT_LIFT(96);
    SVT_LIFT(112); SVT_LIFT(128); SVT_LIFT(144); SVT_LIFT(160);
    default: break;
  }
#undef SVT_LIFT
  return fail(SVT_ERR_UNSUPPORTED, "tensor-core lift: N = %d", N);
}

}  // namespace svt
