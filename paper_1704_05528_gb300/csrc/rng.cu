// Gaussian test blocks Omega (Algorithms 2-3) from a counter-based generator.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64-bit
// multiplications by the round constants 0xD2511F53 and 0xCD9E8D57, a word swap/xor
// with the key, and a Weyl bump of the key by (0x9E3779B9, 0xBB67AE85) between rounds.
// Entry (j, c) of the block drawn in SVT iteration `iter`, block `blk`, uses counter
// (j, c/2, iter, blk) and key (seed lo, seed hi).  Words 0-1 and 2-3 each give 52
// random bits u = (bits + 0.5) 2^-52 in (0, 1); Box-Muller turns (u1, u2) into the pair
// sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2) for columns 2c and 2c+1.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

struct Words { uint32_t x0, x1, x2, x3; };

__device__ __forceinline__ Words philox10(Words c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x0);
    const uint32_t lo1 = 0xCD9E8D57u * c.x2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.x2);
    c = Words{hi1 ^ c.x1 ^ k0, lo1, hi0 ^ c.x3 ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ double open_unit(uint32_t hi, uint32_t lo) {
  const uint64_t bits = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);   // 52 bits
  return ((double)bits + 0.5) * 0x1.0p-52;
}

template <typename T>
__global__ void k_gaussian(uint32_t k0, uint32_t k1, uint32_t iter, uint32_t blk, int64_t n,
                           int w, T* __restrict__ out, int64_t ld) {
  const int pairs = (w + 1) >> 1;
  const int64_t total = n * pairs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / pairs;
    const int c = (int)(t - j * pairs);
    const Words x = philox10(Words{(uint32_t)j, (uint32_t)c, iter, blk}, k0, k1);
    const double u1 = open_unit(x.x0, x.x1);
    const double u2 = open_unit(x.x2, x.x3);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[j * ld + 2 * c] = (T)(rad * cs);
    if (2 * c + 1 < w) out[j * ld + 2 * c + 1] = (T)(rad * sn);
  }
}

}  // namespace

template <typename T>
svt_status launch_gaussian(uint64_t seed, uint32_t iter, uint32_t blk, int64_t n, int w, T* out,
                           int64_t ld, cudaStream_t s) {
  if (n <= 0 || w <= 0) return SVT_OK;
  const int64_t total = n * ((w + 1) / 2);
  int64_t g = ceil_div(total, 256);
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  k_gaussian<T><<<(int)g, 256, 0, s>>>((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32),
                                       iter, blk, n, w, out, ld);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

template svt_status launch_gaussian<double>(uint64_t, uint32_t, uint32_t, int64_t, int, double*,
                                            int64_t, cudaStream_t);
template svt_status launch_gaussian<float>(uint64_t, uint32_t, uint32_t, int64_t, int, float*,
                                           int64_t, cudaStream_t);

}  // namespace svt

extern "C" svt_status svt_gaussian_block(uint64_t seed, uint32_t iter, uint32_t block, int64_t n,
                                         int32_t w, double* out, int64_t ld, void* stream) {
  using namespace svt;
  if (n < 0 || w < 0 || (n > 0 && w > 0 && (!out || ld < w)))
    return fail(SVT_ERR_ARG, "gaussian_block: bad sizes or null output");
  if (n > 0 && w > 0 && !is_device_pointer(out))
    return fail(SVT_ERR_ARG, "gaussian_block: output must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  SVT_TRY(launch_gaussian<double>(seed, iter, block, n, w, out, ld, s));
  SVT_CUDA(cudaStreamSynchronize(s));
  return SVT_OK;
}
