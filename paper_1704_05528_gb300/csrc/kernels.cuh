// Host-side launchers of the SVT kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace svt {

// pattern.cu ------------------------------------------------------------------
svt_status build_pattern(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                         const int32_t* cols, cudaStream_t s, svt_pattern** out);
// Device bytes of a pattern's arrays, and of the scratch its build sorts in.
size_t pattern_block_bytes(int64_t m, int64_t n, int64_t nnz);
size_t pattern_scratch_bytes(int64_t nnz);
// out[c] = first compressed row touched by chunk c of C entries (ptr: nrows + 1 offsets)
svt_status launch_chunk_rows(int64_t nrows, int64_t C, int64_t nchunks, const int32_t* ptr,
                             int32_t* out, cudaStream_t s);

// rng.cu ----------------------------------------------------------------------
template <typename T>
svt_status launch_gaussian(uint64_t seed, uint32_t iter, uint32_t blk, int64_t n, int w, T* out,
                           int64_t ld, cudaStream_t s);

// spmm.cu ---------------------------------------------------------------------
// out[r, 0:w] = sum_{e in ptr[r]..ptr[r+1]} val[e] * W[idx[e], 0:w] for r < nrows, with
// the nnz entries split into equal chunks; `scratch` holds spmm_scratch_bytes(nnz, w,
// sizeof(TD)) bytes.
int64_t chunk_size(int64_t nnz);
size_t spmm_scratch_bytes(int64_t nnz, int w, int elem);
template <typename TV, typename TD>
svt_status launch_spmm_rows(int64_t nrows, const int32_t* ptr, const int32_t* idx,
                            const TV* val, const TD* W, int64_t ldw, int w, TD* out,
                            int64_t ldo, void* scratch, int64_t nnz, cudaStream_t s,
                            const int32_t* chunk_row = nullptr);
// dst[q] = src[perm[q]]
template <typename T>
svt_status launch_gather(int64_t count, const int32_t* perm, const T* src, T* dst,
                         cudaStream_t s);
// dst[perm[q]] = src[q] (the inverse of launch_gather for a permutation)
template <typename T>
svt_status launch_scatter(int64_t count, const int32_t* perm, const T* src, T* dst,
                          cudaStream_t s);
// Where a kernel that follows the chunking of launch_spmm_rows (chunk_size(nnz) entries
// per warp) leaves the partial rows of rows that cross chunks: per chunk c, the head slot
// part[2c * ldp] (its first row) and the tail slot part[(2c + 1) * ldp] (its last row),
// and tails[c] = the row left in the tail slot, or -1.
template <typename TD>
void spmm_slots(void* scratch, int64_t nnz, int w, TD** part, int64_t* ldp, int32_t** tails);
// out[tails[c]] = tail(c) + head(c + 1) + ... for every chunk c with a tail: rows spanning
// more chunks than a segment are summed by segments (each in chunk order, their sums in
// segment order), which uses the free tail slots of the segments' first chunks.
// chunk_row (may be null) holds each chunk's first row.
template <typename TD>
svt_status spmm_fixup(int64_t nnz, int64_t nrows, const int32_t* ptr, const int32_t* chunk_row,
                      TD* part, int64_t ldp, const int32_t* tails, int w, TD* out, int64_t ldo,
                      cudaStream_t s);

// lift_tc.cu ------------------------------------------------------------------
// C (M x N, binary32, ldc) = A (M x K, binary32, lda) B (K x N, binary64, ldb) on the
// tensor cores (three TF32 products per term).  lift_tc_fits tells whether the shape and
// alignment are supported (K <= 128, N <= 160, 16-byte aligned A and C, leading dimensions
// in whole 16-byte vectors); `scratch` holds lift_tc_scratch_floats() floats; a wait that
// ran out raises FLAG_TC_TIMEOUT in *status and leaves C unwritten.
size_t lift_tc_scratch_floats();
// Per-device set-up (driver entry point, shared-memory limits); call it before a stream
// capture that records lift_tc.
svt_status lift_tc_prepare();
bool lift_tc_fits(int64_t M, int K, int N, const float* A, int64_t lda, const float* C, int64_t ldc);
svt_status lift_tc(int64_t M, int K, int N, const float* A, int64_t lda, const double* B,
                   int64_t ldb, float* C, int64_t ldc, float* scratch, unsigned* status,
                   cudaStream_t s);

// dense.cu --------------------------------------------------------------------
// C (p x q, binary64, ldc) = A^T B with A (M x p), B (M x q), reduction over M split
// across blocks; `part` must hold gemm_tn_scratch(M, p, q) doubles.
size_t gemm_tn_scratch(int64_t M, int p, int q);
template <typename TA, typename TB>
svt_status gemm_tn(int64_t M, int p, int q, const TA* A, int64_t lda, const TB* B, int64_t ldb,
                   double* C, int64_t ldc, double* part, cudaStream_t s);
// C (M x q) = alpha A (M x p) B (p x q) + beta Cin; B binary64; C must not alias A.
template <typename TA, typename TC>
svt_status gemm_nn(int64_t M, int p, int q, double alpha, const TA* A, int64_t lda,
                   const double* B, int64_t ldb, double beta, const TC* Cin, int64_t ldcin,
                   TC* C, int64_t ldc, cudaStream_t s);
// sums[c] = sum_i X[i, c]^2 for c < w (binary64), `part` holds colsumsq_scratch doubles.
size_t colsumsq_scratch(int64_t M, int w);
template <typename T>
svt_status colsumsq(int64_t M, int w, const T* X, int64_t ldx, double* sums, double* part,
                    cudaStream_t s);
// dst (M x w, ldd) = (TD) src (M x w, lds)
template <typename TS, typename TD>
svt_status copy_convert(int64_t M, int w, const TS* src, int64_t lds, TD* dst, int64_t ldd,
                        cudaStream_t s);
// Upper Cholesky factor R of the w x w SPD matrix G (R^T R = G) and its inverse, one
// block; raises FLAG_CHOLESKY and writes min_j R_jj (0 on failure) to *diag_min.
svt_status chol_inv(int w, const double* G, int64_t ldg, double* R, double* Rinv,
                    double* work, double* diag_min, unsigned* flags, cudaStream_t s);

// eig.cu ----------------------------------------------------------------------
size_t eig_scratch(int r);
// Symmetric eigendecomposition of the r x r binary64 matrix G (ldg), in two stages: a
// binary32 Jacobi start (eigenvectors in work), then the binary64 refinement, which leaves
// the eigenvalues in descending order (lam) and the eigenvectors as columns of Ub.
svt_status eig_start(int r, const double* G, int64_t ldg, double* work, cudaStream_t s,
                     int* sweeps_out, unsigned* status = nullptr);
// Near-diagonal start for eig_refine (recycled bases): *status (device int) = 0 when the
// start was written, 1 when a coupled cluster is too large (run eig_start instead; with
// identity_on_fail the start is then the identity, so a refinement can follow unchecked).
svt_status eig_start_clusters(int r, const double* G, int64_t ldg, double* work, cudaStream_t s,
                              int* status, bool identity_on_fail = false);
// Per-device set-up of the eigensolver kernels (shared-memory limits); call it before a
// stream capture that records eig_start_clusters.
svt_status eig_prepare();
// After a rejected eig_refine (from any start): diagonalise the clusters of pairs that
// X^T G X still couples, rotate X, refine again with the same acceptance test.  x_alt
// tells where the preceding refinement left X (see eig_refine); this one leaves it at
// eig_x_alt(0, refine_steps).
svt_status eig_refine_clusters_again(int r, const double* G, int64_t ldg, double* lam, double* Ub,
                                     int64_t ldu, double* work, int x_alt, int refine_steps,
                                     cudaStream_t s, int* status, double tol);
// Ogita-Aishima steps from the start X in the scratch; the refined X alternates between
// two scratch buffers step by step: it starts in the second one when start_alt, and ends
// in the one eig_x_alt(start_alt, refine_steps) names, where a further call can resume.
svt_status eig_refine(int r, const double* G, int64_t ldg, double* lam, double* Ub, int64_t ldu,
                      double* work, int refine_steps, cudaStream_t s, int* check_status = nullptr,
                      double check_tol = 0.0, int start_alt = 0);
inline int eig_x_alt(int start_alt, int steps) { return (start_alt ^ steps) & 1; }

// update.cu -------------------------------------------------------------------

size_t reduce_scratch();
// sum of squares of x[0..count) (binary64 result into *out, device)
template <typename T>
svt_status sumsq(int64_t count, const T* x, double* out, double* part, cudaStream_t s);
// y = (T)(scale * a)
template <typename T>
svt_status scale_copy(int64_t count, const T* a, double scale, T* y, cudaStream_t s);
// a_csr[k] = (T) vals[src[k]]
template <typename TS, typename T>
svt_status gather_convert(int64_t count, const int32_t* src, const TS* vals, T* a_csr,
                          cudaStream_t s);
// Sampled shrinkage + update over CSR rows; out3 (device) = {sum d^2, sum |d|, sum y^2}.
// w_pad_zero: columns k .. round_up(k, 4) - 1 of W hold zeros (the solver's own W), so
// whole vectors of a row multiply without per-element tests.
template <typename T>
svt_status sampled_update(const svt_pattern* p, const T* U, int64_t ldu, const T* W,
                          int64_t ldw, int k, const T* a, T* y, double delta, double* out3,
                          double* part, unsigned* flags, cudaStream_t s, bool w_pad_zero = false);
// The sampled update in CSC order fused with the next recycled product: Y (CSC order,
// a the observed values in CSC order) += delta (A - U[:, :k] W^T) on Lambda, out3 as
// above, and bt (n x r, ldb) = Y_new^T U[:, :r].  Needs U, W 16-byte aligned with leading
// dimensions of whole vectors covering r columns, r and nnz within update_recycle_fits,
// k <= r,
// `part` of update_recycle_scratch(nnz) doubles and `scratch` of
// spmm_scratch_bytes(nnz, r, sizeof(T)) bytes.
template <typename T>
bool update_recycle_fits(int r, int64_t nnz);
size_t update_recycle_scratch(int64_t nnz);
template <typename T>
svt_status update_recycle(const svt_pattern* p, const T* U, int64_t ldu, int r, const T* W,
                          int64_t ldw, int k, const T* a, T* y, double delta, T* bt, int64_t ldb,
                          double* out3, double* part, unsigned* flags, void* scratch,
                          cudaStream_t s);

}  // namespace svt
