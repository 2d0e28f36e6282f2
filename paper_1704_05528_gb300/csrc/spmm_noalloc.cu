// svt_spmm_noalloc: the sparse-times-block product of svt_spmm, with its scratch memory
// taken from one fixed device array of this library instead of a fresh allocation.
//
// Some callers cannot allocate device memory at the moment they need this product: a
// host process whose other runtime has already reserved nearly all of the GPU's memory
// for its own pool, a latency-critical loop where a device allocation or free would
// stall the whole device, or an embedding application that only permits allocations
// during its start-up.  For them this entry point uses a statically sized array that the
// CUDA runtime places in device memory when this code is loaded, and allocates nothing.
//
// Limits and sharing:
//  - the array holds kNoAllocScratchBytes (32 MiB); a call whose scratch need is larger
//    is rejected with SVT_ERR_UNSUPPORTED before any work is queued;
//  - every GPU that loads this code keeps the array until the process exits;
//  - all calls share the one array and its contents persist between calls; nothing in it
//    has to start at zero (each call writes every scratch word before reading it), but
//    calls that overlap on the GPU (other threads or other streams) race on it;
//  - the first call on a device looks up the array's device address there
//    (cudaGetSymbolAddress, with that device current) and caches it for the process; a
//    cudaDeviceReset would leave that cached address stale, so resetting a device while
//    this library is in use is not supported; that first call belongs before any stream
//    capture.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "solver.cuh"

namespace svt {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per device).
svt_status noalloc_scratch(void** out) {
  int dev = -1;
  SVT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(SVT_ERR_UNSUPPORTED, "spmm_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return SVT_OK;
}

}  // namespace
}  // namespace svt

extern "C" svt_status svt_spmm_noalloc(const svt_pattern* p, int precision, int transpose,
                                       const void* y_csr, const void* W, int64_t ldw, int32_t w,
                                       void* out, int64_t ldo, void* stream) {
  using namespace svt;
  if (!p || w < 0 || (p->nnz > 0 && !y_csr)) return fail(SVT_ERR_ARG, "spmm_noalloc: bad arguments");
  if (precision != SVT_FP64 && precision != SVT_MIXED_FP32)
    return fail(SVT_ERR_ARG, "spmm_noalloc: unknown precision");
  if (w > 0 && (!W || !out || ldw < w || ldo < w)) return fail(SVT_ERR_ARG, "spmm_noalloc: bad dense operands");
  if (w == 0) return SVT_OK;
  const int64_t z = p->nnz;
  const int elem = precision == SVT_FP64 ? 8 : 4;
  // scratch: [Y in column order (transpose only) | partial rows and chunk tails of the SpMM]
  const size_t ycsc_bytes = transpose ? (size_t)round_up(z * elem, 256) : 0;
  const size_t need = ycsc_bytes + spmm_scratch_bytes(z, w, elem);
  if (need > kNoAllocScratchBytes)
    return fail(SVT_ERR_UNSUPPORTED,
                "spmm_noalloc: this product needs %zu bytes of scratch; the fixed array holds %zu",
                need, kNoAllocScratchBytes);
  void* base = nullptr;
  SVT_TRY(noalloc_scratch(&base));
  char* ycsc = static_cast<char*>(base);
  char* scr = ycsc + ycsc_bytes;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t rows_out = transpose ? p->n : p->m;
  auto run = [&](auto tag) -> svt_status {
    using T = decltype(tag);
    const T* y = (const T*)y_csr;
    if (transpose) {
      SVT_TRY(launch_gather<T>(z, p->perm, y, (T*)ycsc, s));
      SVT_TRY((launch_spmm_rows<T, T>(rows_out, p->col_ptr, p->row_idx, (const T*)ycsc, (const T*)W, ldw,
                                       w, (T*)out, ldo, scr, z, s, p->chunk_row_csc)));
    } else {
      SVT_TRY((launch_spmm_rows<T, T>(rows_out, p->row_ptr, p->col_idx, y, (const T*)W, ldw, w, (T*)out,
                                       ldo, scr, z, s, p->chunk_row_csr)));
    }
    return SVT_OK;
  };
  {
    // the product's kernels, timed as one class when the library's profiler is on
    SVT_PROF(transpose ? "api_spmm_csc" : "api_spmm_csr",
             spmm_bytes(z, rows_out, transpose ? p->m : p->n, w, elem), s);
    SVT_TRY(precision == SVT_FP64 ? run(double(0)) : run(float(0)));
  }
  SVT_CUDA(cudaStreamSynchronize(s));
  return SVT_OK;
}
