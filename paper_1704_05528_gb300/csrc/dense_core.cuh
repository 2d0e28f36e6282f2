// The dense-row core of the binary32 fused update (dense_core.cu): which rows form it, the
// device buffers of the core panel and of the sparse rest, and the host calls.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "common.cuh"

namespace svt {

// Host-side choice of the core rows (core_plan).
struct CorePlan {
  int rd = 0;                    // rows in the core (0: no core)
  int64_t ldd = 0;               // slots of the panel: rd rounded up to a tile of 128
  int64_t core_nnz = 0, rest_nnz = 0;
  std::vector<int32_t> slot_row;  // [ldd] row of each slot, -1 for padding
  std::vector<int32_t> row_slot;  // [m] slot of each row, -1 outside the core
};

// Device state of the core (laid out by core_layout from one arena).
struct DenseCore {
  int64_t m = 0, n = 0, ldd = 0;
  int rd = 0;
  int32_t *slot_row = nullptr, *row_slot = nullptr;
  // the sparse rest as a CSC pattern: column pointers, rows, chunk start columns, and the
  // full-pattern CSC slot of each rest entry
  int32_t *rest_ptr = nullptr, *rest_cnt = nullptr, *rest_row = nullptr, *rest_full = nullptr;
  int32_t* rest_chunk_col = nullptr;
  svt_pattern rest;               // views of the arrays above (not owned)
  float *a_rest = nullptr, *y_rest = nullptr;  // observed values and Y of the rest (its CSC order)
  float *A = nullptr, *Y = nullptr;            // n x ldd core panels: A (NaN = unobserved), Y
  float* w_pad = nullptr;                      // n x 128: W zero-padded, where W itself cannot be mapped
  float *ud_hi = nullptr, *ud_lo = nullptr;    // ldd x 128: TF32 parts of the core rows of U
  float *udt_hi = nullptr, *udt_lo = nullptr;  // 128 x ldd: the same, transposed
  double* part = nullptr;                      // per-CTA sums of the core update
  double* upd_part = nullptr;                  // block sums of the rest's update
  void* upd_scratch = nullptr;                 // partial rows of the rest's update
  int32_t* full_src = nullptr;                 // [nnz] rest CSC slot, or -(1 + panel offset)
};

// Rows with at least min_frac * n observed entries, in whole tiles of 128 and at most 4096
// (want_rows > 0: exactly that many of the fullest rows).  plan->rd = 0 when there is no core.
svt_status core_plan(const svt_pattern* p, int want_rows, double min_frac, cudaStream_t s,
                     CorePlan* plan);
// The largest plan core_plan can return for a pattern of this size (the automatic core
// is at most 4096 rows); rest_nnz is taken as nnz.  Sizes caller workspaces.
CorePlan core_plan_bound(int64_t m, int64_t n, int64_t nnz, int want_rows, double min_frac);
void core_layout(Arena& a, const CorePlan& plan, int64_t m, int64_t n, int r_cap, DenseCore* C);
// Device arrays of the core from the full pattern and the observed values in CSC order.
svt_status core_build(const svt_pattern* p, const CorePlan& plan, const float* a_csc,
                      int32_t* full_src, cudaStream_t s, DenseCore* C);
// Split Y (full CSC order) into the rest and the core panel.
svt_status core_enter(const svt_pattern* p, const float* y_csc, cudaStream_t s, DenseCore* C);
// Full Y in CSR and CSC order from the rest and the core panel.
svt_status core_assemble(const svt_pattern* p, const DenseCore& C, float* y_csr, float* y_csc,
                         cudaStream_t s);
// r <= 128 and 0 <= k <= r.
bool core_fits(int r, int k);
// The core's part of the fused update, after the sparse rest's (update_recycle on
// C.rest, which wrote every row of bt and the sums): Y_core += delta (A - U[:, :k] W^T)
// where observed, out3 (device) += {sum d^2, sum |d|, sum Y_new^2} over the core, and
// bt (n x r, ldb) += Y_core^T U_core[:, :r].  A bounded wait that ran out raises
// FLAG_TC_TIMEOUT in *tc_status.
svt_status core_update(const DenseCore& C, const float* U, int64_t ldu, int r, const float* W,
                       int64_t ldw, int k, double delta, float* bt, int64_t ldb, double* out3,
                       unsigned* flags, unsigned* tc_status, cudaStream_t s);

}  // namespace svt
