// Differentiating unrolled fast SVT: the adjoint of D_tau and the reverse recursion of
// eq. (4).
//
// Forward: Y^(1) = k0 delta P_Lambda(A) (k0 held fixed), X^(i) = D_tau(Y^(i)) by R4SVD,
// Y^(i+1) = Y^(i) + delta P_Lambda(A - X^(i)) for i < T, loss L = mean over the held-out
// set H of (X^(T) - A)^2.  R4SVD stops at an energy threshold, which leaves the leading
// triplets only approximate when Y has a dense spectrum below them; each R4SVD result is
// therefore refined by power steps with Rayleigh-Ritz until the kept triplets meet a
// residual bound, so the forward map is D_tau itself and the gradient is that of exact
// unrolled SVT.  The solver state (Y, the recycled basis, the threshold) is checkpointed
// every `ckpt` iterations; the reverse pass replays one segment at a time.
//
// Jacobian of D_tau.  D_tau is the proximal map of tau ||.||_* (eq. (3)), so its
// Jacobian J is symmetric.  With the kept singular triplets (u_i, s_i, v_i), s_i > tau,
// f_i = s_i - tau, and Y_perp = (I - U U^T) Y (I - V V^T) the rest of Y, a direction Z
// maps to
//   J(Z) = U (C1 o G + C2 o G^T) V^T                                   (kept / kept)
//        + sum_i f_i [ u_i w_i^T + (P_Uperp Z v_i + Y_perp w_i) v_i^T / s_i ]  (kept / rest)
// with G = U^T Z V, C1_ij = 1 - tau/(s_i+s_j), C2_ij = tau/(s_i+s_j) (C1_ii = 1, C2_ii = 0),
// and w_i the solution of (s_i^2 I - Y_perp^T Y_perp) w_i = s_i P_Vperp Z^T u_i +
// Y_perp^T P_Uperp Z v_i in the complement of V.  Those k shifted systems are positive
// definite (every remaining singular value is below tau < s_i) and are solved together
// by conjugate gradients, one sparse product with Y and one with Y^T per step, so no
// full SVD is ever formed.  J(Z) is only needed on Lambda: it is a rank-2k product
// [U M + Zc | U diag(f)] [V | W]^T evaluated on the observed entries.
// dD_tau/dtau = -U V^T, so <Z, dD_tau/dtau> = -trace(G).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "solver.cuh"

namespace svt {
namespace {

template <typename T>
__global__ void k_cols_affine(int64_t M, int k, const T* __restrict__ A, int64_t lda,
                              const T* __restrict__ B, int64_t ldb, const double* __restrict__ cb,
                              T* __restrict__ out, int64_t ldo) {
  // out[:, j] = A[:, j] + cb[j] * B[:, j]   (A may be null: out = cb o B)
  const int64_t total = M * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    const double base = A ? (double)A[i * lda + j] : 0.0;
    out[i * ldo + j] = (T)(base + cb[j] * (double)B[i * ldb + j]);
  }
}

template <typename T>
__global__ void k_cg_step(int64_t M, int k, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                          const T* __restrict__ Ap, int64_t ld, const double* __restrict__ alpha) {
  const int64_t total = M * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    const double a = alpha[j];
    x[i * ld + j] = (T)((double)x[i * ld + j] + a * (double)p[i * ld + j]);
    r[i * ld + j] = (T)((double)r[i * ld + j] - a * (double)Ap[i * ld + j]);
  }
}

// AP[:, j] = sig2[j] * P[:, j] - AP[:, j]
template <typename T>
__global__ void k_shift_op(int64_t M, int k, const T* __restrict__ P, T* __restrict__ AP, int64_t ld,
                           const double* __restrict__ sig2) {
  const int64_t total = M * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    AP[i * ld + j] = (T)(sig2[j] * (double)P[i * ld + j] - (double)AP[i * ld + j]);
  }
}

template <typename T>
__global__ void k_vec_axpy(int64_t count, double a, const T* __restrict__ x, T* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (T)((double)y[i] + a * (double)x[i]);
}

template <typename T>
__global__ void k_dot_part(int64_t count, const T* __restrict__ x, const T* __restrict__ y,
                           double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)x[i], (double)y[i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[b];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_diag(int k, const double* __restrict__ C, double* __restrict__ d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) d[j] = C[(int64_t)j * k + j];
}

// alpha_j = rs_j / pAp_j for columns still running (rs_j > thr_j), else 0
__global__ void k_cg_alpha(int k, const double* __restrict__ rs, const double* __restrict__ pAp,
                           const double* __restrict__ thr, double* __restrict__ alpha) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) alpha[j] = (rs[j] > thr[j] && pAp[j] > 0.0) ? rs[j] / pAp[j] : 0.0;
}

__global__ void k_cg_beta(int k, const double* __restrict__ rs_new, double* __restrict__ rs,
                          const double* __restrict__ thr, double* __restrict__ beta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) {
    beta[j] = (rs_new[j] > thr[j] && rs[j] > 0.0) ? rs_new[j] / rs[j] : 0.0;
    rs[j] = rs_new[j];
  }
}

template <typename T>
__global__ void k_cg_dir(int64_t M, int k, const T* __restrict__ r, T* __restrict__ p, int64_t ld,
                         const double* __restrict__ beta) {
  const int64_t total = M * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    p[i * ld + j] = (T)((double)r[i * ld + j] + beta[j] * (double)p[i * ld + j]);
  }
}

int egrid(int64_t work) {
  int64_t g = ceil_div(work > 0 ? work : 1, 256);
  const int64_t cap = (int64_t)num_sms() * 16;
  return (int)(g < cap ? g : cap);
}

// Device buffers of the adjoint (blocks sized for kcap kept values).
template <typename T>
struct AdjWork {
  int64_t m = 0, n = 0, zl = 0, zmax = 0;
  int kcap = 1;
  int64_t ldk = 4, ld2 = 4;
  T *ZV, *ZtU, *YtZ, *Bv, *Xc, *Rc, *Pc, *APc, *Tm, *YW, *L, *R;
  T *zc, *zero_l, *Xr;
  double *Gh, *GhT, *M, *proj, *Cdot, *vec, *part, *Gx2, *Rm2, *Rinv2, *cw2;
  double *rs, *rs_new, *pAp, *alpha, *beta, *thr, *sig2, *cb;
  void* spmm_scr;

  void layout(Arena& a) {
    ldk = ld_of(kcap);
    ld2 = ld_of(2 * kcap);
    ZV = a.take<T>(m * ldk); Tm = a.take<T>(m * ldk); YW = a.take<T>(m * ldk);
    ZtU = a.take<T>(n * ldk); YtZ = a.take<T>(n * ldk); Bv = a.take<T>(n * ldk);
    Xc = a.take<T>(n * ldk); Rc = a.take<T>(n * ldk); Pc = a.take<T>(n * ldk); APc = a.take<T>(n * ldk);
    L = a.take<T>(m * ld2); R = a.take<T>(n * ld2);
    zc = a.take<T>(zmax); zero_l = a.take<T>(zmax);
    Xr = a.take<T>(m * ldk);
    const int64_t kk = (int64_t)kcap * kcap;
    Gh = a.take<double>(kk); GhT = a.take<double>(kk); M = a.take<double>(kk);
    proj = a.take<double>(kk); Cdot = a.take<double>(kk);
    Gx2 = a.take<double>(kk); Rm2 = a.take<double>(kk); Rinv2 = a.take<double>(kk); cw2 = a.take<double>(kk);
    vec = a.take<double>(8);
    size_t pe = gemm_tn_scratch(std::max(m, n), kcap, kcap);
    pe = std::max(pe, reduce_scratch());
    pe = std::max(pe, (size_t)num_sms() * 8 + 8);
    part = a.take<double>(pe);
    rs = a.take<double>(kcap); rs_new = a.take<double>(kcap); pAp = a.take<double>(kcap);
    alpha = a.take<double>(kcap); beta = a.take<double>(kcap); thr = a.take<double>(kcap);
    sig2 = a.take<double>(kcap); cb = a.take<double>(2 * kcap);
    spmm_scr = a.take<char>(std::max(spmm_scratch_bytes(zmax, 2 * kcap, (int)sizeof(T)),
                                     spmm_scratch_bytes(zl, 2 * kcap, (int)sizeof(T))));
  }
};

template <typename T>
svt_status dot(AdjWork<T>& A, int64_t count, const T* x, const T* y, double* out_host,
               cudaStream_t s) {
  const int blocks = num_sms() * 8;
  k_dot_part<T><<<blocks, 256, 0, s>>>(count, x, y, A.part);
  SVT_LAUNCH_CHECK();
  k_sum_parts<<<1, 256, 0, s>>>(blocks, A.part, A.vec);
  SVT_LAUNCH_CHECK();
  SVT_CUDA(cudaMemcpyAsync(out_host, A.vec, sizeof(double), cudaMemcpyDeviceToHost, s));
  SVT_CUDA(cudaStreamSynchronize(s));
  return SVT_OK;
}

// X <- X - B (B^T X) for an M x k block X and an M x k orthonormal B (both ld given).
template <typename T>
svt_status project_out(AdjWork<T>& A, int64_t M, int k, const T* B, int64_t ldb, T* X,
                       int64_t ldx, cudaStream_t s) {
  SVT_TRY((gemm_tn<T, T>(M, k, k, B, ldb, X, ldx, A.proj, k, A.part, s)));
  SVT_TRY((gemm_nn<T, T>(M, k, k, -1.0, B, ldb, A.proj, k, 1.0, X, ldx, X, ldx, s)));
  return SVT_OK;
}

// Kept singular triplets of one iterate and the iterate itself.
template <typename T>
struct Triplets {
  const T* U = nullptr;   // m x k (ldu)
  int64_t ldu = 0;
  const T* V = nullptr;   // n x k (ldv)
  int64_t ldv = 0;
  std::vector<double> sigma;
  int k = 0;
  const T* y_csr = nullptr;  // Y on Lambda
  const T* y_csc = nullptr;
};

struct CgStats {
  int iters = 0, capped = 0;
};

// out_y (on Lambda, CSR order) += coef * J(Z) restricted to Lambda, for Z given on the
// pattern pz (CSR order).  *trace = trace(U^T Z V).
template <typename T>
svt_status jvp_sampled(AdjWork<T>& A, const svt_pattern* pl, const svt_pattern* pz, const T* z_csr,
                       const Triplets<T>& X, double tau, T* out_y, double coef, double* trace,
                       double cg_tol, int cg_maxit, CgStats* cg, double* part3, unsigned* flags,
                       cudaStream_t s) {
  const int k = X.k;
  const int64_t m = A.m, n = A.n;
  *trace = 0.0;
  if (k == 0) return SVT_OK;
  const int64_t ldk = A.ldk;
  // Z in both orders; Z V and Z^T U
  SVT_TRY(launch_gather<T>(pz->nnz, pz->perm, z_csr, A.zc, s));
  SVT_TRY((launch_spmm_rows<T, T>(m, pz->row_ptr, pz->col_idx, z_csr, X.V, X.ldv, k, A.ZV, ldk,
                                   A.spmm_scr, pz->nnz, s, pz->chunk_row_csr)));
  SVT_TRY((launch_spmm_rows<T, T>(n, pz->col_ptr, pz->row_idx, A.zc, X.U, X.ldu, k, A.ZtU, ldk,
                                   A.spmm_scr, pz->nnz, s, pz->chunk_row_csc)));
  // G = U^T Z V (k x k) and the kept/kept coefficients (host, k^2 values)
  SVT_TRY((gemm_tn<T, T>(m, k, k, X.U, X.ldu, A.ZV, ldk, A.Gh, k, A.part, s)));
  std::vector<double> G((size_t)k * k), GT((size_t)k * k), Mh((size_t)k * k);
  SVT_CUDA(cudaMemcpyAsync(G.data(), A.Gh, G.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  SVT_CUDA(cudaStreamSynchronize(s));
  double tr = 0.0;
  for (int i = 0; i < k; ++i) {
    tr += G[(size_t)i * k + i];
    for (int j = 0; j < k; ++j) {
      GT[(size_t)i * k + j] = G[(size_t)j * k + i];
      if (i == j) {
        Mh[(size_t)i * k + j] = G[(size_t)i * k + i];
      } else {
        const double c2 = tau / (X.sigma[i] + X.sigma[j]);
        Mh[(size_t)i * k + j] = (1.0 - c2) * G[(size_t)i * k + j] + c2 * G[(size_t)j * k + i];
      }
    }
  }
  *trace = tr;
  SVT_CUDA(cudaMemcpyAsync(A.GhT, GT.data(), GT.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  SVT_CUDA(cudaMemcpyAsync(A.M, Mh.data(), Mh.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  // P_Uperp Z V = ZV - U G,  P_Vperp Z^T U = ZtU - V G^T
  SVT_TRY((gemm_nn<T, T>(m, k, k, -1.0, X.U, X.ldu, A.Gh, k, 1.0, A.ZV, ldk, A.ZV, ldk, s)));
  SVT_TRY((gemm_nn<T, T>(n, k, k, -1.0, X.V, X.ldv, A.GhT, k, 1.0, A.ZtU, ldk, A.ZtU, ldk, s)));
  // b_i = s_i P_Vperp Z^T u_i + P_Vperp Y^T (P_Uperp Z v_i)
  SVT_TRY((launch_spmm_rows<T, T>(n, pl->col_ptr, pl->row_idx, X.y_csc, A.ZV, ldk, k, A.YtZ, ldk,
                                   A.spmm_scr, pl->nnz, s, pl->chunk_row_csc)));
  SVT_TRY(project_out<T>(A, n, k, X.V, X.ldv, A.YtZ, ldk, s));
  std::vector<double> hs(2 * (size_t)k);
  for (int i = 0; i < k; ++i) { hs[i] = X.sigma[i]; hs[k + i] = X.sigma[i] * X.sigma[i]; }
  SVT_CUDA(cudaMemcpyAsync(A.cb, hs.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
  SVT_CUDA(cudaMemcpyAsync(A.sig2, hs.data() + k, k * sizeof(double), cudaMemcpyHostToDevice, s));
  k_cols_affine<T><<<egrid(n * k), 256, 0, s>>>(n, k, A.YtZ, ldk, A.ZtU, ldk, A.cb, A.Bv, ldk);
  SVT_LAUNCH_CHECK();
  // batched CG on (s_i^2 I - Y_perp^T Y_perp) w_i = b_i, iterates kept in the complement of V
  SVT_CUDA(cudaMemsetAsync(A.Xc, 0, n * ldk * sizeof(T), s));
  SVT_CUDA(cudaMemcpyAsync(A.Rc, A.Bv, n * ldk * sizeof(T), cudaMemcpyDeviceToDevice, s));
  SVT_CUDA(cudaMemcpyAsync(A.Pc, A.Bv, n * ldk * sizeof(T), cudaMemcpyDeviceToDevice, s));
  SVT_TRY((gemm_tn<T, T>(n, k, k, A.Rc, ldk, A.Rc, ldk, A.Cdot, k, A.part, s)));
  k_diag<<<1, 256, 0, s>>>(k, A.Cdot, A.rs);
  SVT_LAUNCH_CHECK();
  std::vector<double> b2(k), rsh(k), thr(k);
  SVT_CUDA(cudaMemcpyAsync(b2.data(), A.rs, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  SVT_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < k; ++j) thr[j] = cg_tol * cg_tol * b2[j];
  SVT_CUDA(cudaMemcpyAsync(A.thr, thr.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
  int it = 0;
  bool done = false;
  {
    bool all = true;
    for (int j = 0; j < k; ++j) all = all && !(b2[j] > thr[j]);
    done = all;
  }
  for (; it < cg_maxit && !done; ++it) {
    // A p = s^2 p - P_Vperp Y^T P_Uperp Y p
    SVT_TRY((launch_spmm_rows<T, T>(m, pl->row_ptr, pl->col_idx, X.y_csr, A.Pc, ldk, k, A.Tm, ldk,
                                     A.spmm_scr, pl->nnz, s, pl->chunk_row_csr)));
    SVT_TRY(project_out<T>(A, m, k, X.U, X.ldu, A.Tm, ldk, s));
    SVT_TRY((launch_spmm_rows<T, T>(n, pl->col_ptr, pl->row_idx, X.y_csc, A.Tm, ldk, k, A.APc, ldk,
                                     A.spmm_scr, pl->nnz, s, pl->chunk_row_csc)));
    SVT_TRY(project_out<T>(A, n, k, X.V, X.ldv, A.APc, ldk, s));
    k_shift_op<T><<<egrid(n * k), 256, 0, s>>>(n, k, A.Pc, A.APc, ldk, A.sig2);  // s^2 p - (.)
    SVT_LAUNCH_CHECK();
    SVT_TRY((gemm_tn<T, T>(n, k, k, A.Pc, ldk, A.APc, ldk, A.Cdot, k, A.part, s)));
    k_diag<<<1, 256, 0, s>>>(k, A.Cdot, A.pAp);
    SVT_LAUNCH_CHECK();
    k_cg_alpha<<<1, 256, 0, s>>>(k, A.rs, A.pAp, A.thr, A.alpha);
    SVT_LAUNCH_CHECK();
    k_cg_step<T><<<egrid(n * k), 256, 0, s>>>(n, k, A.Xc, A.Rc, A.Pc, A.APc, ldk, A.alpha);
    SVT_LAUNCH_CHECK();
    SVT_TRY((gemm_tn<T, T>(n, k, k, A.Rc, ldk, A.Rc, ldk, A.Cdot, k, A.part, s)));
    k_diag<<<1, 256, 0, s>>>(k, A.Cdot, A.rs_new);
    SVT_LAUNCH_CHECK();
    SVT_CUDA(cudaMemcpyAsync(rsh.data(), A.rs_new, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    k_cg_beta<<<1, 256, 0, s>>>(k, A.rs_new, A.rs, A.thr, A.beta);
    SVT_LAUNCH_CHECK();
    k_cg_dir<T><<<egrid(n * k), 256, 0, s>>>(n, k, A.Rc, A.Pc, ldk, A.beta);
    SVT_LAUNCH_CHECK();
    SVT_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int j = 0; j < k; ++j) {
      if (!std::isfinite(rsh[j])) return fail(SVT_ERR_NUMERIC, "adjoint: non-finite CG residual");
      all = all && !(rsh[j] > thr[j]);
    }
    done = all;
  }
  cg->iters += it;
  if (!done) cg->capped += 1;
  // Y_perp w = P_Uperp (Y w)
  SVT_TRY((launch_spmm_rows<T, T>(m, pl->row_ptr, pl->col_idx, X.y_csr, A.Xc, ldk, k, A.YW, ldk,
                                   A.spmm_scr, pl->nnz, s, pl->chunk_row_csr)));
  SVT_TRY(project_out<T>(A, m, k, X.U, X.ldu, A.YW, ldk, s));
  // L = [U M + (P_Uperp Z V + Y_perp W) diag(f/s) | U diag(f)],  R = [V | W]
  std::vector<double> fs(2 * (size_t)k);
  for (int i = 0; i < k; ++i) {
    fs[i] = (X.sigma[i] - tau) / X.sigma[i];
    fs[k + i] = X.sigma[i] - tau;
  }
  SVT_CUDA(cudaMemcpyAsync(A.cb, fs.data(), 2 * k * sizeof(double), cudaMemcpyHostToDevice, s));
  const int64_t ld2 = A.ld2;
  k_cols_affine<T><<<egrid(m * k), 256, 0, s>>>(m, k, nullptr, 0, A.ZV, ldk, A.cb, A.L, ld2);
  SVT_LAUNCH_CHECK();
  k_cols_affine<T><<<egrid(m * k), 256, 0, s>>>(m, k, A.L, ld2, A.YW, ldk, A.cb, A.L, ld2);
  SVT_LAUNCH_CHECK();
  SVT_TRY((gemm_nn<T, T>(m, k, k, 1.0, X.U, X.ldu, A.M, k, 1.0, A.L, ld2, A.L, ld2, s)));
  k_cols_affine<T><<<egrid(m * k), 256, 0, s>>>(m, k, nullptr, 0, X.U, X.ldu, A.cb + k, A.L + k, ld2);
  SVT_LAUNCH_CHECK();
  SVT_TRY((copy_convert<T, T>(n, k, X.V, X.ldv, A.R, ld2, s)));
  SVT_TRY((copy_convert<T, T>(n, k, A.Xc, ldk, A.R + k, ld2, s)));
  // out_y += coef * (L R^T) on Lambda: the sampled update with a = 0 and step -coef
  SVT_TRY(sampled_update<T>(pl, A.L, ld2, A.R, ld2, 2 * k, A.zero_l, out_y, -coef, part3, A.part,
                            flags, s));
  return SVT_OK;
}

struct RitzStats {
  int steps = 0, capped = 0, grown = 0;
};

// Refinement of one R4SVD result until D_tau is that of Y to a residual bound.
//
// Entry and exit state, as r4svd_run leaves it: Q (m x r, orthonormal, ld W.ldq) the
// basis, W.Bt = Y^T Q, W.Ub / ro->sigma the Rayleigh-Ritz rotation and values of
// B = Q^T Y, and U = Q U_B.  Each step is one power step Q <- orth(Y Y^T Q) = orth(Y W.Bt)
// (Cholesky-QR twice) followed by a new Rayleigh-Ritz step.  With v_i = B^T u_B,i / s_i,
// Y^T u_i = s_i v_i holds exactly, so e_i = ||Y v_i - s_i u_i|| is the whole residual of
// the pair and some singular value of Y lies within e_i of s_i.  The loop ends once every
// kept pair has e_i <= tol * s_1 and the first dropped pair has
// e_i <= max(tol * s_1, (tau - s_i) / 2), which places its singular value below tau
// (subspace iteration meets the leading triplets in order); or after maxit steps; or when
// five steps with the same kept set have not lowered the worst ratio of e_i to its bound
// by a fifth (the rounding floor).
// Rayleigh-Ritz on the basis Q (m x r): W.Bt = Y^T Q, B B^T = U_B Lambda U_B^T, U = Q U_B.
template <typename T>
svt_status rayleigh_ritz(Work<T>& W, const svt_pattern* pl, const T* y_csc, const T* Q, T* U,
                         int r, R4Out* ro) {
  cudaStream_t st = W.s;
  const int64_t m = W.P.m, n = W.P.n;
  SVT_TRY((launch_spmm_rows<T, T>(n, pl->col_ptr, pl->row_idx, y_csc, Q, W.ldq, r, W.Bt, W.ldb,
                                   W.spmm_scr, pl->nnz, st, pl->chunk_row_csc)));
  SVT_TRY((gemm_tn<T, T>(n, r, r, W.Bt, W.ldb, W.Bt, W.ldb, W.G, r, W.part, st)));
  SVT_TRY(eig_from_jacobi<T>(W, r));
  SVT_TRY(lift_basis<T>(W, Q, r, U));
  std::vector<double> lam(r);
  SVT_CUDA(cudaMemcpyAsync(lam.data(), W.lam, r * sizeof(double), cudaMemcpyDeviceToHost, st));
  SVT_CUDA(cudaStreamSynchronize(st));
  ro->r = r;
  ro->sigma.assign(r, 0.0);
  for (int j = 0; j < r; ++j) {
    if (!std::isfinite(lam[j])) return fail(SVT_ERR_NUMERIC, "unrolled: non-finite Ritz value");
    ro->sigma[j] = std::sqrt(std::max(lam[j], 0.0));
  }
  return SVT_OK;
}

// Appends one Gaussian block of min(dt, r_cap - r) columns to Q (m x r) as R4SVD does
// (two projections against Q, Cholesky-QR twice); *exhausted when the block has no
// direction left outside Q (the range of Y is spanned).  Philox blocks kGrowBlock0 + g of
// iteration `iter` keep the draws apart from R4SVD's.
constexpr uint32_t kGrowBlock0 = 0x10000u;

template <typename T>
svt_status grow_basis(Work<T>& W, const svt_pattern* pl, const T* y_csr, T* Q, int r, uint32_t iter,
                      int g, int* w_out, bool* exhausted) {
  const Params& P = W.P;
  const int64_t m = P.m, n = P.n, z = pl->nnz;
  cudaStream_t st = W.s;
  const int w = std::min(P.dt, P.r_cap - r);
  *w_out = 0;
  *exhausted = false;
  SVT_TRY(launch_gaussian<T>(P.seed, iter, kGrowBlock0 + (uint32_t)g, n, w, W.Om, W.ldw, st));
  SVT_TRY((launch_spmm_rows<T, T>(m, pl->row_ptr, pl->col_idx, y_csr, W.Om, W.ldw, w, W.X, W.ldw,
                                   W.spmm_scr, z, st, pl->chunk_row_csr)));
  double ssum = 0.0, scale = 0.0;
  SVT_TRY(block_sumsq<T>(W, m, w, W.X, W.ldw, &ssum, &scale));
  for (int pass = 0; pass < 2; ++pass) {
    SVT_TRY((gemm_tn<T, T>(m, r, w, Q, W.ldq, W.X, W.ldw, W.Gs, w, W.part, st)));
    SVT_TRY((gemm_nn<T, T>(m, r, w, -1.0, Q, W.ldq, W.Gs, w, 1.0, W.X, W.ldw, W.X2, W.ldw, st)));
    std::swap(W.X, W.X2);
  }
  SVT_CUDA(cudaMemsetAsync(W.flags, 0, sizeof(unsigned), st));
  SVT_TRY((gemm_tn<T, T>(m, w, w, W.X, W.ldw, W.X, W.ldw, W.Gx, w, W.part, st)));
  SVT_TRY(chol_inv(w, W.Gx, w, W.Rm, W.Rinv, W.cwork, W.dsc + 0, W.flags, st));
  double dmin = 0.0;
  unsigned fl = 0;
  SVT_CUDA(cudaMemcpyAsync(&dmin, W.dsc + 0, sizeof(double), cudaMemcpyDeviceToHost, st));
  SVT_TRY(read_flags(W, &fl));
  if (scale == 0.0 || (fl & FLAG_CHOLESKY) || !(dmin > kExhaustedRel * scale)) {
    *exhausted = true;
    return SVT_OK;
  }
  SVT_TRY((gemm_nn<T, T>(m, w, w, 1.0, W.X, W.ldw, W.Rinv, w, 0.0, nullptr, 0, W.X2, W.ldw, st)));
  SVT_TRY((gemm_tn<T, T>(m, w, w, W.X2, W.ldw, W.X2, W.ldw, W.Gx, w, W.part, st)));
  SVT_TRY(chol_inv(w, W.Gx, w, W.Rm, W.Rinv, W.cwork, W.dsc + 1, W.flags, st));
  SVT_TRY(read_flags(W, &fl));
  if (fl & FLAG_CHOLESKY) return fail(SVT_ERR_NUMERIC, "unrolled: Cholesky-QR breakdown growing the basis");
  SVT_TRY((gemm_nn<T, T>(m, w, w, 1.0, W.X2, W.ldw, W.Rinv, w, 0.0, nullptr, 0, Q + r, W.ldq, st)));
  *w_out = w;
  return SVT_OK;
}

template <typename T>
svt_status ritz_refine(Work<T>& W, AdjWork<T>& A, const svt_pattern* pl, const T* y_csr,
                       const T* y_csc, T* Q, T* U, double tau, double tol, int maxit, uint32_t iter,
                       R4Out* ro, RitzStats* rs) {
  const int64_t m = W.P.m, z = pl->nnz;
  const int64_t ldq = W.ldq, ldk = A.ldk;
  cudaStream_t st = W.s;
  if (ro->r <= 0) return SVT_OK;
  std::vector<double> ss(W.P.r_cap), hist;
  int k_prev = -1, grown = 0;
  bool exhausted = false;
  for (int step = 0;; ++step) {
    const int r = ro->r;
    int k = 0;
    while (k < r && ro->sigma[k] > tau) ++k;
    if (k == r && !exhausted) {
      // no dropped pair to certify the kept set: grow the basis by a block, as R4SVD does
      if (r >= W.P.r_cap)
        return fail(SVT_ERR_UNSUPPORTED,
                    "unrolled: all %d Ritz values exceed tau at the rank cap, so the kept set is "
                    "not certified; raise r_max", r);
      int w = 0;
      SVT_TRY(grow_basis<T>(W, pl, y_csr, Q, r, iter, grown++, &w, &exhausted));
      if (w > 0) SVT_TRY(rayleigh_ritz<T>(W, pl, y_csc, Q, U, r + w, ro));
      rs->grown += 1;
      continue;
    }
    if (k != k_prev) hist.clear();  // the bounds changed with the kept set
    k_prev = k;
    int c = k < r ? k + 1 : k;  // k == r only once the range of Y is exhausted
    while (c > 0 && !(ro->sigma[c - 1] > 0.0)) --c;
    bool ok = true;
    if (c > 0) {
      std::vector<double> inv(c), neg(c);
      for (int j = 0; j < c; ++j) { inv[j] = 1.0 / ro->sigma[j]; neg[j] = -ro->sigma[j]; }
      SVT_TRY(scaled_right<T>(W, r, c, inv));  // W.Wk = V_c
      SVT_TRY((launch_spmm_rows<T, T>(m, pl->row_ptr, pl->col_idx, y_csr, W.Wk, W.ldk, c, A.Tm, ldk,
                                       W.spmm_scr, z, st, pl->chunk_row_csr)));
      SVT_CUDA(cudaMemcpyAsync(A.cb, neg.data(), c * sizeof(double), cudaMemcpyHostToDevice, st));
      k_cols_affine<T><<<egrid(m * c), 256, 0, st>>>(m, c, A.Tm, ldk, U, ldq, A.cb, A.Tm, ldk);
      SVT_LAUNCH_CHECK();
      SVT_TRY(colsumsq<T>(m, c, A.Tm, ldk, W.colss, W.part, st));
      SVT_CUDA(cudaMemcpyAsync(ss.data(), W.colss, c * sizeof(double), cudaMemcpyDeviceToHost, st));
      SVT_CUDA(cudaStreamSynchronize(st));
      const double bound = tol * ro->sigma[0];
      double worst = 0.0;
      for (int j = 0; j < c; ++j) {
        if (!std::isfinite(ss[j])) return fail(SVT_ERR_NUMERIC, "unrolled: non-finite Ritz residual");
        const double bj = j < k ? bound : std::max(bound, 0.5 * (tau - ro->sigma[j]));
        worst = std::max(worst, std::sqrt(ss[j]) / bj);
      }
      ok = worst <= 1.0;
      hist.push_back(worst);
    }
    if (ok) return SVT_OK;
    const int h = (int)hist.size();
    if (step >= maxit || (h > 5 && hist[h - 1] > 0.8 * hist[h - 6])) {
      rs->capped += 1;
      return SVT_OK;
    }
    rs->steps += 1;
    // power step: Xr = Y (Y^T Q), then Q = orth(Xr) by Cholesky-QR twice (U as the middle)
    SVT_TRY((launch_spmm_rows<T, T>(m, pl->row_ptr, pl->col_idx, y_csr, W.Bt, W.ldb, r, A.Xr, ldk,
                                     W.spmm_scr, z, st, pl->chunk_row_csr)));
    const T* src = A.Xr;
    int64_t lds = ldk;
    for (int pass = 0; pass < 2; ++pass) {
      T* dst = pass == 0 ? U : Q;
      SVT_CUDA(cudaMemsetAsync(W.flags, 0, sizeof(unsigned), st));
      SVT_TRY((gemm_tn<T, T>(m, r, r, src, lds, src, lds, A.Gx2, r, A.part, st)));
      SVT_TRY(chol_inv(r, A.Gx2, r, A.Rm2, A.Rinv2, A.cw2, W.dsc + 0, W.flags, st));
      unsigned fl = 0;
      SVT_TRY(read_flags(W, &fl));
      if (fl & FLAG_CHOLESKY) return fail(SVT_ERR_NUMERIC, "unrolled: refinement basis lost rank");
      SVT_TRY((gemm_nn<T, T>(m, r, r, 1.0, src, lds, A.Rinv2, r, 0.0, nullptr, 0, dst, ldq, st)));
      src = dst;
      lds = ldq;
    }
    SVT_TRY(rayleigh_ritz<T>(W, pl, y_csc, Q, U, r, ro));
  }
}

template <typename T>
svt_status upload(const void* src, int64_t count, T* dst, bool from_double, cudaStream_t s,
                  DeviceBlock& tmp) {
  // copy caller values (host or device; binary64 or T) into a device T array
  if (count <= 0) return SVT_OK;
  const size_t bytes = count * (from_double ? sizeof(double) : sizeof(T));
  const void* dsrc = src;
  if (!is_device_pointer(src)) {
    SVT_TRY(tmp.alloc(bytes, s));
    SVT_CUDA(cudaMemcpyAsync(tmp.ptr, src, bytes, cudaMemcpyHostToDevice, s));
    dsrc = tmp.ptr;
  }
  if (from_double && sizeof(T) != sizeof(double)) {
    SVT_TRY((copy_convert<double, T>(count, 1, (const double*)dsrc, 1, dst, 1, s)));
  } else {
    SVT_CUDA(cudaMemcpyAsync(dst, dsrc, count * sizeof(T), cudaMemcpyDeviceToDevice, s));
  }
  return SVT_OK;
}

template <typename T>
svt_status upload_idx(const int32_t* src, int64_t count, int32_t* dst, cudaStream_t s) {
  if (count <= 0) return SVT_OK;
  SVT_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(int32_t), cudaMemcpyDefault, s));
  return SVT_OK;
}

// Unrolled SVT as a tape: forward() runs the T iterations and keeps the checkpoints,
// backward() replays them in reverse for a given gradient on the held-out predictions.
template <typename T>
struct UnrolledTape {
  int64_t m = 0, n = 0, nnz = 0, nh = 0;
  double tau = 0, delta = 0;
  svt_unrolled_params UP{};
  Params P{};
  cudaStream_t st = nullptr;
  bool dbl_in = false;
  std::chrono::steady_clock::time_point t0;
  RitzStats ritz;
  CgStats cg;
  DeviceBlock idx_blk, wb, t1, t2;
  svt_pattern* pl = nullptr;
  svt_pattern* ph = nullptr;
  Work<T> W;
  AdjWork<T> A;
  int nck = 0;
  int64_t ldq0 = 0;
  T *a_csr, *y_csr, *hv, *xh, *gH, *ybar, *abar, *tmpz, *ck_y, *ck_Q, *sg_y, *sg_yc, *sg_d, *sg_U,
      *sg_V, *fin_V, *vals_in, *hvals_in;
  double* part3;
  int k0 = 1;
  // one SVT iteration from state (y, Q[:, :s], eps_thr, eps_min, normY2)
  struct State {
    int s = 0;
    double eps_thr = 0, eps_min = INFINITY, normY2 = 0;
    T* Qcur = nullptr;
    T* Qnext = nullptr;
  };
  struct IterOut {
    int r = 0, k = 0;
    std::vector<double> sigma;
  };
  // What the reverse pass needs from one iterate: U_K, V_K (ld ldq0) and A - X on Lambda.
  struct Capture {
    T* U = nullptr;
    T* V = nullptr;
    T* d = nullptr;
  };
  std::vector<State> cks;
  State S;
  IterOut last;
  std::vector<T> hx;          // X^(T) on the held-out entries, held CSR order
  std::vector<int32_t> hsrc;  // caller position of each held CSR slot
  double t_fwd = 0;
  bool backward_done = false;

  ~UnrolledTape() {
    if (st) cudaStreamSynchronize(st);
    svt_pattern_destroy(pl);
    svt_pattern_destroy(ph);
  }

  svt_status iterate(State& Sx, int i, bool update_y, IterOut* io, const Capture* cap) {
    R4Out ro;
    SVT_TRY(launch_gather<T>(nnz, pl->perm, y_csr, W.y_csc, st));
    SVT_TRY(r4svd_run<T>(W, y_csr, W.y_csc, Sx.Qcur, Sx.s, Sx.normY2, Sx.eps_thr, (uint32_t)i, Sx.Qnext, &ro));
    if (UP.ritz_maxit > 0)
      SVT_TRY(ritz_refine<T>(W, A, pl, y_csr, W.y_csc, Sx.Qcur, Sx.Qnext, tau, UP.ritz_tol, UP.ritz_maxit,
                             (uint32_t)i, &ro, &ritz));
    int k = 0;
    while (k < ro.r && ro.sigma[k] > tau) ++k;
    std::vector<double> coef(k), inv(k);
    for (int j = 0; j < k; ++j) {
      coef[j] = (ro.sigma[j] - tau) / ro.sigma[j];
      inv[j] = 1.0 / ro.sigma[j];
    }
    if (cap) {  // V_K = B^T U_B,K Sigma_K^-1 and U_K
      SVT_TRY(scaled_right<T>(W, ro.r, k, inv));
      SVT_TRY((copy_convert<T, T>(n, k, W.Wk, W.ldk, cap->V, ldq0, st)));
      SVT_TRY((copy_convert<T, T>(m, k, Sx.Qnext, W.ldq, cap->U, ldq0, st)));
    }
    SVT_TRY(scaled_right<T>(W, ro.r, k, coef));
    if (cap) {  // A - X on Lambda: the sampled update of a zero vector with step 1
      SVT_CUDA(cudaMemsetAsync(cap->d, 0, nnz * sizeof(T), st));
      SVT_TRY(sampled_update<T>(pl, Sx.Qnext, W.ldq, W.Wk, W.ldk, k, a_csr, cap->d, 1.0, part3, W.part,
                                W.flags, st, true));
    }
    io->r = ro.r; io->k = k;
    io->sigma.assign(ro.sigma.begin(), ro.sigma.begin() + k);
    if (!update_y) return SVT_OK;
    SVT_TRY(sampled_update<T>(pl, Sx.Qnext, W.ldq, W.Wk, W.ldk, k, a_csr, y_csr, delta, W.dsc + 5,
                              W.part, W.flags, st, true));
    double sums[3];
    SVT_CUDA(cudaMemcpyAsync(sums, W.dsc + 5, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaStreamSynchronize(st));
    const double res = std::sqrt(sums[0]);  // cooling compares successive residuals only
    if (!std::isfinite(res)) return fail(SVT_ERR_NUMERIC, "unrolled: non-finite iterate at %d", i);
    if (res < Sx.eps_min) Sx.eps_min = res; else Sx.eps_thr *= P.beta;
    Sx.normY2 = sums[2];
    std::swap(Sx.Qcur, Sx.Qnext);
    Sx.s = ro.r;
    return SVT_OK;
  }

  svt_status norm_y(double* out) {
    SVT_TRY(sumsq<T>(nnz, y_csr, W.dsc + 4, W.part, st));
    SVT_CUDA(cudaMemcpyAsync(out, W.dsc + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaStreamSynchronize(st));
    return SVT_OK;
  }

  // Forward pass: T iterations from Y^(1) = k0 delta P_Lambda(A), checkpoints every ckpt
  // iterations, and X^(T) on the held-out entries (hx).
  svt_status forward(int64_t m_, int64_t n_, int64_t nnz_, const int32_t* rows, const int32_t* cols,
                     const void* vals, int64_t nh_, const int32_t* hrows, const int32_t* hcols,
                     double tau_, double delta_, const svt_unrolled_params& up, const svt_options* opt) {
    t0 = std::chrono::steady_clock::now();
    m = m_; n = n_; nnz = nnz_; nh = nh_; tau = tau_; delta = delta_; UP = up;
    SVT_TRY(make_params(m, n, opt, &P));
    st = (cudaStream_t)opt->stream;
    dbl_in = opt->precision == SVT_FP64;
    const int steps = UP.steps, ckpt = UP.checkpoint_every;
    // index arrays on the device
    Arena ia;
    ia.take<int32_t>(nnz); ia.take<int32_t>(nnz); ia.take<int32_t>(nh); ia.take<int32_t>(nh);
    SVT_TRY(idx_blk.alloc(ia.off, st));
    Arena ib; ib.base = (char*)idx_blk.ptr;
    int32_t* d_rows = ib.take<int32_t>(nnz);
    int32_t* d_cols = ib.take<int32_t>(nnz);
    int32_t* d_hrows = ib.take<int32_t>(nh);
    int32_t* d_hcols = ib.take<int32_t>(nh);
    SVT_TRY(upload_idx<T>(rows, nnz, d_rows, st));
    SVT_TRY(upload_idx<T>(cols, nnz, d_cols, st));
    SVT_TRY(upload_idx<T>(hrows, nh, d_hrows, st));
    SVT_TRY(upload_idx<T>(hcols, nh, d_hcols, st));
    SVT_TRY(build_pattern(m, n, nnz, d_rows, d_cols, st, &pl));
    SVT_TRY(build_pattern(m, n, nh, d_hrows, d_hcols, st, &ph));
    if (nnz == 0 || nh == 0) return fail(SVT_ERR_ARG, "unrolled: need observed and held-out entries");

    W.P = P; W.pat = pl; W.s = st;
    A.m = m; A.n = n; A.zl = nnz; A.zmax = std::max(nnz, nh); A.kcap = P.r_cap;
    nck = (steps + ckpt - 1) / ckpt;
    ldq0 = ld_of(P.r_cap);
    auto layout_all = [&](Arena& a) {
      a_csr = a.take<T>(nnz); y_csr = a.take<T>(nnz);
      hv = a.take<T>(nh); xh = a.take<T>(nh); gH = a.take<T>(nh);
      ybar = a.take<T>(nnz); abar = a.take<T>(nnz); tmpz = a.take<T>(nnz);
      ck_y = a.take<T>((int64_t)nck * nnz);
      ck_Q = a.take<T>((int64_t)nck * m * ldq0);
      sg_y = a.take<T>((int64_t)ckpt * nnz);
      sg_yc = a.take<T>((int64_t)ckpt * nnz);
      sg_d = a.take<T>((int64_t)ckpt * nnz);
      sg_U = a.take<T>((int64_t)ckpt * m * ldq0);
      sg_V = a.take<T>((int64_t)ckpt * n * ldq0);
      fin_V = a.take<T>(n * ldq0);
      vals_in = a.take<T>(nnz); hvals_in = a.take<T>(nh);
      part3 = a.take<double>(8);
      W.layout(a);
      A.layout(a);
    };
    Arena a0;
    layout_all(a0);
    SVT_TRY(wb.alloc(a0.off, st));
    Arena a1; a1.base = (char*)wb.ptr;
    layout_all(a1);
    SVT_CUDA(cudaMemsetAsync(W.flags, 0, kFlagWords * sizeof(unsigned), st));
    SVT_CUDA(cudaMemsetAsync(A.zero_l, 0, A.zmax * sizeof(T), st));
    SVT_TRY(upload<T>(vals, nnz, vals_in, dbl_in, st, t1));
    SVT_TRY((gather_convert<T, T>(nnz, pl->csr_src, vals_in, a_csr, st)));
    // initialisation (Algorithm 4): power steps for ||P_Lambda A||_2, k0, Y = k0 delta A
    SVT_TRY(launch_gather<T>(nnz, pl->perm, a_csr, W.y_csc, st));
    SVT_TRY(launch_gaussian<double>(P.seed, kPowerSeedIter, 0, n, 1, W.pw, 1, st));
    SVT_TRY(sumsq<double>(n, W.pw, W.dsc + 3, W.part, st));
    k_normalize<<<(int)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(n, W.pw, W.dsc + 3, W.pv);
    SVT_LAUNCH_CHECK();
    for (int it = 0; it < P.power_steps; ++it) {
      SVT_TRY((launch_spmm_rows<T, double>(m, pl->row_ptr, pl->col_idx, a_csr, W.pv, 1, 1, W.pu, 1,
                                           W.spmm_scr, nnz, st, pl->chunk_row_csr)));
      SVT_TRY((launch_spmm_rows<T, double>(n, pl->col_ptr, pl->row_idx, W.y_csc, W.pu, 1, 1, W.pw, 1,
                                           W.spmm_scr, nnz, st, pl->chunk_row_csc)));
      SVT_TRY(sumsq<double>(n, W.pw, W.dsc + 3, W.part, st));
      k_normalize<<<(int)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(n, W.pw, W.dsc + 3, W.pv);
      SVT_LAUNCH_CHECK();
    }
    double lam2 = 0.0;
    SVT_CUDA(cudaMemcpyAsync(&lam2, W.dsc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaStreamSynchronize(st));
    const double s2 = std::sqrt(std::sqrt(lam2));
    k0 = s2 > 0.0 ? (int)std::min(std::ceil(tau / (delta * s2)), 2.0e9) : 1;

    // forward with checkpoints
    cks.assign(nck, State());
    S = State();
    S.eps_thr = P.eps_thr0; S.Qcur = W.Qa; S.Qnext = W.Qb;
    SVT_TRY(scale_copy<T>(nnz, a_csr, (double)k0 * delta, y_csr, st));
    SVT_TRY(norm_y(&S.normY2));
    for (int i = 1; i <= steps; ++i) {
      if ((i - 1) % ckpt == 0) {
        const int c = (i - 1) / ckpt;
        cks[c] = S;
        SVT_CUDA(cudaMemcpyAsync(ck_y + (int64_t)c * nnz, y_csr, nnz * sizeof(T), cudaMemcpyDeviceToDevice, st));
        SVT_CUDA(cudaMemcpyAsync(ck_Q + (int64_t)c * m * ldq0, S.Qcur, m * ldq0 * sizeof(T),
                                 cudaMemcpyDeviceToDevice, st));
      }
      SVT_TRY(iterate(S, i, i < steps, &last, nullptr));
    }
    // X^(T) on the held-out set: sampled product with a = 0 and step -1 gives x
    SVT_CUDA(cudaMemsetAsync(xh, 0, nh * sizeof(T), st));
    SVT_TRY(sampled_update<T>(ph, S.Qnext, W.ldq, W.Wk, W.ldk, last.k, A.zero_l, xh, -1.0, part3,
                              W.part, W.flags, st));
    hx.resize(nh);
    hsrc.resize(nh);
    SVT_CUDA(cudaMemcpyAsync(hx.data(), xh, nh * sizeof(T), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaMemcpyAsync(hsrc.data(), ph->csr_src, nh * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaStreamSynchronize(st));
    t_fwd = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return SVT_OK;
  }

  // X^(T) on the held-out entries in the caller's order.
  void held_predictions(std::vector<double>* out) const {
    out->assign(nh, 0.0);
    for (int64_t e = 0; e < nh; ++e) (*out)[hsrc[e]] = (double)hx[e];
  }

  // Reverse pass for g = dL/dX^(T) on the held-out entries (caller order): grad (caller
  // order, nnz) = dL/dvals, *gtau, *gdelta.
  svt_status backward(const std::vector<double>& g_caller, std::vector<double>* grad, double* gtau_out,
                      double* gdelta_out) {
    const int steps = UP.steps, ckpt = UP.checkpoint_every;
    const double cg_tol = UP.cg_tol;
    const int cg_maxit = UP.cg_maxit;
    std::vector<T> g(nh);
    for (int64_t e = 0; e < nh; ++e) g[e] = (T)g_caller[hsrc[e]];
    double gtau = 0.0, gdelta = 0.0, trace = 0.0;
    SVT_CUDA(cudaMemcpyAsync(gH, g.data(), nh * sizeof(T), cudaMemcpyHostToDevice, st));
    // triplets of the last iterate: U = Qnext[:, :k], V = B^T U_B,K Sigma_K^-1
    {
      std::vector<double> inv(last.k);
      for (int j = 0; j < last.k; ++j) inv[j] = 1.0 / last.sigma[j];
      SVT_TRY(scaled_right<T>(W, last.r, last.k, inv));
    }
    // (W.Bt / W.Ub still hold the last iteration; scaled_right wrote V_K into W.Wk)
    SVT_TRY((copy_convert<T, T>(n, last.k, W.Wk, W.ldk, fin_V, ldq0, st)));
    Triplets<T> XT;
    XT.U = S.Qnext; XT.ldu = W.ldq; XT.V = fin_V; XT.ldv = ldq0; XT.sigma = last.sigma; XT.k = last.k;
    XT.y_csr = y_csr;
    SVT_TRY(launch_gather<T>(nnz, pl->perm, y_csr, tmpz, st));
    XT.y_csc = tmpz;
    SVT_CUDA(cudaMemsetAsync(ybar, 0, nnz * sizeof(T), st));
    SVT_CUDA(cudaMemsetAsync(abar, 0, nnz * sizeof(T), st));
    SVT_TRY(jvp_sampled<T>(A, pl, ph, gH, XT, tau, ybar, 1.0, &trace, cg_tol, cg_maxit, &cg, part3,
                           W.flags, st));
    gtau -= trace;  // <G, dX/dtau> = -trace(U^T G V)
    // segments in reverse: iterations 1..steps-1 need the backward step
    for (int c = nck - 1; c >= 0; --c) {
      const int i0 = c * ckpt + 1;
      const int i1 = std::min(i0 + ckpt - 1, steps - 1);
      if (i0 > i1) continue;
      // replay the segment from its checkpoint, keeping each iterate's Y, triplets and A - X
      State R = cks[c];
      SVT_CUDA(cudaMemcpyAsync(y_csr, ck_y + (int64_t)c * nnz, nnz * sizeof(T), cudaMemcpyDeviceToDevice, st));
      SVT_CUDA(cudaMemcpyAsync(R.Qcur, ck_Q + (int64_t)c * m * ldq0, m * ldq0 * sizeof(T),
                               cudaMemcpyDeviceToDevice, st));
      std::vector<IterOut> outs(i1 - i0 + 1);
      for (int i = i0; i <= i1; ++i) {
        const int j = i - i0;
        SVT_CUDA(cudaMemcpyAsync(sg_y + (int64_t)j * nnz, y_csr, nnz * sizeof(T), cudaMemcpyDeviceToDevice, st));
        SVT_TRY(launch_gather<T>(nnz, pl->perm, y_csr, sg_yc + (int64_t)j * nnz, st));
        Capture cap;
        cap.U = sg_U + (int64_t)j * m * ldq0;
        cap.V = sg_V + (int64_t)j * n * ldq0;
        cap.d = sg_d + (int64_t)j * nnz;
        SVT_TRY(iterate(R, i, true, &outs[j], &cap));
      }
      for (int i = i1; i >= i0; --i) {
        const int j = i - i0;
        const T* d_i = sg_d + (int64_t)j * nnz;
        // Y^(i+1) = Y^(i) + delta P(A - X^(i)):  abar += delta ybar, dbar += <ybar, A - X^(i)>
        k_vec_axpy<T><<<egrid(nnz), 256, 0, st>>>(nnz, delta, ybar, abar);
        SVT_LAUNCH_CHECK();
        double dd = 0.0;
        SVT_TRY(dot<T>(A, nnz, ybar, d_i, &dd, st));
        gdelta += dd;
        Triplets<T> Xi;
        Xi.U = sg_U + (int64_t)j * m * ldq0; Xi.ldu = ldq0;
        Xi.V = sg_V + (int64_t)j * n * ldq0; Xi.ldv = ldq0;
        Xi.sigma = outs[j].sigma; Xi.k = outs[j].k;
        Xi.y_csr = sg_y + (int64_t)j * nnz; Xi.y_csc = sg_yc + (int64_t)j * nnz;
        // ybar <- ybar - delta J_i(ybar);  tau: -delta <ybar, dX/dtau> = +delta trace
        SVT_TRY(jvp_sampled<T>(A, pl, pl, ybar, Xi, tau, ybar, -delta, &trace, cg_tol, cg_maxit, &cg,
                               part3, W.flags, st));
        gtau += delta * trace;
      }
    }
    // Y^(1) = k0 delta A
    k_vec_axpy<T><<<egrid(nnz), 256, 0, st>>>(nnz, (double)k0 * delta, ybar, abar);
    SVT_LAUNCH_CHECK();
    double ya = 0.0;
    SVT_TRY(dot<T>(A, nnz, ybar, a_csr, &ya, st));
    gdelta += (double)k0 * ya;
    // gradient in the caller's entry order
    std::vector<T> ab(nnz);
    std::vector<int32_t> src(nnz);
    SVT_CUDA(cudaMemcpyAsync(ab.data(), abar, nnz * sizeof(T), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaMemcpyAsync(src.data(), pl->csr_src, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SVT_CUDA(cudaStreamSynchronize(st));
    grad->assign(nnz, 0.0);
    for (int64_t e = 0; e < nnz; ++e) (*grad)[src[e]] = (double)ab[e];
    *gtau_out = gtau;
    *gdelta_out = gdelta;
    backward_done = true;
    return SVT_OK;
  }

  void fill_info(svt_unrolled_info* info, double loss) const {
    if (!info) return;
    info->k0 = k0;
    info->k_final = last.k;
    info->r_final = last.r;
    info->cg_iters = cg.iters;
    info->cg_capped = cg.capped;
    info->ritz_steps = ritz.steps;
    info->ritz_capped = ritz.capped;
    info->ritz_grown = ritz.grown;
    info->loss = loss;
    info->seconds_forward = t_fwd;
    info->seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

svt_status check_unrolled_args(int64_t m, int64_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                               const void* vals, int64_t nheld, const int32_t* held_rows,
                               const int32_t* held_cols, double tau, double delta,
                               const svt_unrolled_params& up) {
  if (m <= 0 || n <= 0 || nnz <= 0 || nheld <= 0 || !rows || !cols || !vals || !held_rows ||
      !held_cols || !(tau > 0.0) || !(delta > 0.0))
    return fail(SVT_ERR_ARG, "unrolled: bad arguments");
  if (up.steps < 1 || up.checkpoint_every < 1 || up.cg_maxit < 1 || up.ritz_maxit < 0 ||
      !(up.cg_tol > 0.0) || !(up.ritz_tol > 0.0))
    return fail(SVT_ERR_ARG, "unrolled: bad parameters (steps, checkpoint_every, cg_maxit >= 1; "
                             "ritz_maxit >= 0; cg_tol, ritz_tol > 0)");
  return SVT_OK;
}

// Copy n doubles (host or device) into a host vector.
svt_status fetch_doubles(const double* src, int64_t count, std::vector<double>* out) {
  out->resize(count);
  if (count <= 0) return SVT_OK;
  SVT_CUDA(cudaMemcpy(out->data(), src, count * sizeof(double), cudaMemcpyDefault));
  return SVT_OK;
}

svt_status store_doubles(const std::vector<double>& v, double* dst) {
  if (!dst || v.empty()) return SVT_OK;
  SVT_CUDA(cudaMemcpy(dst, v.data(), v.size() * sizeof(double), cudaMemcpyDefault));
  return SVT_OK;
}

}  // namespace
}  // namespace svt

// The opaque tape of the ABI: one precision's tape.
struct svt_unrolled_tape {
  int precision = SVT_FP64;
  svt::UnrolledTape<double>* d = nullptr;
  svt::UnrolledTape<float>* f = nullptr;
  ~svt_unrolled_tape() {
    delete d;
    delete f;
  }
};

extern "C" void svt_unrolled_default_params(svt_unrolled_params* p, int precision) {
  if (!p) return;
  p->steps = 20;
  p->checkpoint_every = 5;
  p->cg_maxit = 1000;
  p->ritz_maxit = 100;
  p->cg_tol = precision == SVT_MIXED_FP32 ? 1e-6 : 1e-10;
  p->ritz_tol = precision == SVT_MIXED_FP32 ? 2e-6 : 1e-11;
}

extern "C" svt_status svt_unrolled_forward(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                                           const int32_t* cols, const void* vals, int64_t nheld,
                                           const int32_t* held_rows, const int32_t* held_cols,
                                           double tau, double delta, const svt_unrolled_params* p,
                                           const svt_options* opt, double* x_held,
                                           svt_unrolled_info* info, svt_unrolled_tape** tape) {
  using namespace svt;
  if (info) memset(info, 0, sizeof(*info));
  if (tape) *tape = nullptr;
  if (!opt) return fail(SVT_ERR_ARG, "unrolled: null options");
  if (opt->precision != SVT_FP64 && opt->precision != SVT_MIXED_FP32)
    return fail(SVT_ERR_ARG, "unrolled: unknown precision");
  svt_unrolled_params up;
  if (p) up = *p;
  else svt_unrolled_default_params(&up, opt->precision);
  SVT_TRY(check_unrolled_args(m, n, nnz, rows, cols, vals, nheld, held_rows, held_cols, tau, delta, up));
  svt_unrolled_tape* t = new svt_unrolled_tape;
  t->precision = opt->precision;
  svt_status st;
  std::vector<double> xh;
  if (opt->precision == SVT_FP64) {
    t->d = new UnrolledTape<double>;
    st = t->d->forward(m, n, nnz, rows, cols, vals, nheld, held_rows, held_cols, tau, delta, up, opt);
    if (st >= 0) { t->d->held_predictions(&xh); t->d->fill_info(info, NAN); }
  } else {
    t->f = new UnrolledTape<float>;
    st = t->f->forward(m, n, nnz, rows, cols, vals, nheld, held_rows, held_cols, tau, delta, up, opt);
    if (st >= 0) { t->f->held_predictions(&xh); t->f->fill_info(info, NAN); }
  }
  if (st >= 0) st = store_doubles(xh, x_held);
  if (st < 0 || !tape) {
    delete t;  // synchronises the stream and releases the device memory
    return st;
  }
  *tape = t;
  return SVT_OK;
}

extern "C" svt_status svt_unrolled_backward(svt_unrolled_tape* tape, const double* g_held,
                                            double* grad_vals, double* grad_tau_delta,
                                            svt_unrolled_info* info) {
  using namespace svt;
  if (!tape || !g_held) return fail(SVT_ERR_ARG, "unrolled_backward: null tape or gradient");
  auto run = [&](auto* T_) -> svt_status {
    if (T_->backward_done) return fail(SVT_ERR_ARG, "unrolled_backward: the tape was already used");
    std::vector<double> g, grad;
    SVT_TRY(fetch_doubles(g_held, T_->nh, &g));
    double gt = 0.0, gd = 0.0;
    SVT_TRY(T_->backward(g, &grad, &gt, &gd));
    SVT_TRY(store_doubles(grad, grad_vals));
    if (grad_tau_delta) {
      const double two[2] = {gt, gd};
      SVT_CUDA(cudaMemcpy(grad_tau_delta, two, sizeof(two), cudaMemcpyDefault));
    }
    if (info) { memset(info, 0, sizeof(*info)); T_->fill_info(info, NAN); }
    return SVT_OK;
  };
  const svt_status st = tape->d ? run(tape->d) : run(tape->f);
  if (st < 0) cudaStreamSynchronize(tape->d ? tape->d->st : tape->f->st);
  return st;
}

extern "C" void svt_unrolled_tape_destroy(svt_unrolled_tape* tape) { delete tape; }

extern "C" svt_status svt_unrolled_grad(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                                        const int32_t* cols, const void* vals, int64_t nheld,
                                        const int32_t* held_rows, const int32_t* held_cols,
                                        const void* held_vals, double tau, double delta,
                                        const svt_unrolled_params* p, const svt_options* opt,
                                        double* grad_vals, double* x_held, double* out3,
                                        svt_unrolled_info* info) {
  using namespace svt;
  if (info) memset(info, 0, sizeof(*info));
  if (!opt) return fail(SVT_ERR_ARG, "unrolled_grad: null options");
  if (!held_vals) return fail(SVT_ERR_ARG, "unrolled_grad: bad arguments");
  // held-out values in binary64, caller order (host or device input)
  std::vector<double> hv(nheld > 0 ? nheld : 0);
  svt_unrolled_tape* tape = nullptr;
  std::vector<double> xh(nheld > 0 ? nheld : 0);
  svt_status st = svt_unrolled_forward(m, n, nnz, rows, cols, vals, nheld, held_rows, held_cols, tau,
                                       delta, p, opt, xh.data(), info, grad_vals ? &tape : nullptr);
  if (st < 0) return st;
  struct Guard { svt_unrolled_tape* t; ~Guard() { delete t; } } guard{tape};
  if (opt->precision == SVT_FP64) {
    SVT_CUDA(cudaMemcpy(hv.data(), held_vals, nheld * sizeof(double), cudaMemcpyDefault));
  } else {
    std::vector<float> h32(nheld);
    SVT_CUDA(cudaMemcpy(h32.data(), held_vals, nheld * sizeof(float), cudaMemcpyDefault));
    for (int64_t e = 0; e < nheld; ++e) hv[e] = (double)h32[e];
  }
  // L = mean over the held-out entries of (X^(T) - A)^2, dL/dX = 2 (X - A) / nheld
  double loss = 0.0;
  std::vector<double> g(nheld);
  for (int64_t e = 0; e < nheld; ++e) {
    const double r = xh[e] - hv[e];
    loss += r * r;
    g[e] = 2.0 * r / (double)nheld;
  }
  loss /= (double)nheld;
  if (x_held) SVT_TRY(store_doubles(xh, x_held));
  double gtd[2] = {NAN, NAN};
  if (tape) {
    st = svt_unrolled_backward(tape, g.data(), grad_vals, gtd, info);
    if (st < 0) return st;
  }
  if (info) info->loss = loss;
  if (out3) { out3[0] = loss; out3[1] = gtd[0]; out3[2] = gtd[1]; }
  return SVT_OK;
}
