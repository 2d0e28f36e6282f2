// Small symmetric eigenproblem G = U_B diag(lam) U_B^T for the SVD of B (Algorithm 3:
// [U_L, Sigma_L, V_L] = svd(B) with B B^T = G, sigma = sqrt(lam)).
//
// Binary64 arithmetic runs at about 1/58 of the binary32 rate on this part, so the
// decomposition is computed in two stages:
//  1. cyclic Jacobi in binary32 inside one thread block (round-robin pairing, so each
//     step rotates r/2 disjoint planes at once), stopped when no off-diagonal entry is
//     significant at binary32 resolution;
//  2. Ogita-Aishima refinement in binary64 (Ogita & Aishima, "Iterative refinement for
//     symmetric eigenvalue decomposition", 2018): with X the current eigenvector
//     estimate, R = I - X^T X, S = X^T G X, lam_i = S_ii / (1 - R_ii), and
//     E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) for well separated pairs,
//     E_ij = R_ij / 2 otherwise; X <- X + X E.  Each step is four r x r x r products
//     (spread over the whole GPU) and converges quadratically.
// The eigenpairs are finally sorted by descending eigenvalue.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

constexpr int kJacThreads = 1024;

__device__ __forceinline__ void rr_pair(int step, int i, int N, int* p, int* q) {
  // circle method over N (even) players; player 0 fixed
  if (i == 0) {
    *p = 0;
    *q = step % (N - 1) + 1;
  } else {
    *p = (step + i) % (N - 1) + 1;
    *q = (step - i + (N - 1)) % (N - 1) + 1;
  }
}

// A: r x r working copy (row-major), V: r x r eigenvector estimate (columns).
__global__ void __launch_bounds__(kJacThreads)
k_jacobi32(int r, const double* __restrict__ G, int64_t ldg, float* gA, float* gV,
           int max_sweeps, int use_smem) {
  extern __shared__ float dyn[];
  __shared__ float cs_c[kJacThreads / 2 + 1], cs_s[kJacThreads / 2 + 1];
  __shared__ int pp[kJacThreads / 2 + 1], qq[kJacThreads / 2 + 1];
  __shared__ int active_any;
  __shared__ float scale;
  float* A = use_smem ? dyn : gA;
  float* V = use_smem ? dyn + (int64_t)r * r : gV;
  const int64_t rr2 = (int64_t)r * r;
  for (int64_t t = threadIdx.x; t < rr2; t += blockDim.x) {
    const int a = (int)(t / r), b = (int)(t % r);
    A[t] = (float)G[(int64_t)a * ldg + b];
    V[t] = (a == b) ? 1.0f : 0.0f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float mx = 0.f;
    for (int i = 0; i < r; ++i) mx = fmaxf(mx, fabsf(A[(int64_t)i * r + i]));
    scale = mx;
  }
  __syncthreads();
  const int N = (r + 1) & ~1;
  const int npairs = N / 2;
  const float rel_thr = 1e-6f, abs_thr = 1e-7f * scale;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) active_any = 0;
    __syncthreads();
    for (int step = 0; step < N - 1; ++step) {
      for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
        int p, q;
        rr_pair(step, i, N, &p, &q);
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < r) {
          const float apq = A[(int64_t)p * r + q];
          const float app = A[(int64_t)p * r + p], aqq = A[(int64_t)q * r + q];
          if (fabsf(apq) > abs_thr && fabsf(apq) > rel_thr * sqrtf(fabsf(app) * fabsf(aqq))) {
            const float theta = (aqq - app) / (2.f * apq);
            float t;
            if (fabsf(theta) > 1e15f) t = 0.5f / theta;
            else t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(1.f + theta * theta));
            c = rsqrtf(1.f + t * t);
            s = t * c;
            active_any = 1;
          }
        }
        cs_c[i] = c; cs_s[i] = s; pp[i] = p; qq[i] = (q < r) ? q : -1;
      }
      __syncthreads();
      // rows p, q of A <- J^T A
      for (int64_t t = threadIdx.x; t < (int64_t)npairs * r; t += blockDim.x) {
        const int i = (int)(t / r), j = (int)(t % r);
        const int q = qq[i];
        if (q < 0 || cs_s[i] == 0.f) continue;
        const int p = pp[i];
        const float c = cs_c[i], s = cs_s[i];
        const float ap = A[(int64_t)p * r + j], aq = A[(int64_t)q * r + j];
        A[(int64_t)p * r + j] = c * ap - s * aq;
        A[(int64_t)q * r + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q of A and V <- (.) J
      for (int64_t t = threadIdx.x; t < (int64_t)npairs * r; t += blockDim.x) {
        const int i = (int)(t / r), j = (int)(t % r);
        const int q = qq[i];
        if (q < 0 || cs_s[i] == 0.f) continue;
        const int p = pp[i];
        const float c = cs_c[i], s = cs_s[i];
        const float ap = A[(int64_t)j * r + p], aq = A[(int64_t)j * r + q];
        A[(int64_t)j * r + p] = c * ap - s * aq;
        A[(int64_t)j * r + q] = s * ap + c * aq;
        const float vp = V[(int64_t)j * r + p], vq = V[(int64_t)j * r + q];
        V[(int64_t)j * r + p] = c * vp - s * vq;
        V[(int64_t)j * r + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    if (!active_any) break;
    __syncthreads();
  }
  if (use_smem) {
    for (int64_t t = threadIdx.x; t < rr2; t += blockDim.x) gV[t] = V[t];
  }
}

__global__ void k_to_double(int64_t count, const float* __restrict__ src, double* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = (double)src[t];
}

// One Ogita-Aishima update: given C = X^T X and S = X^T G X (r x r), write E and lam.
__global__ void __launch_bounds__(1024)
k_oa_coeffs(int r, const double* __restrict__ G, int64_t ldg, const double* __restrict__ C,
            const double* __restrict__ S, double* __restrict__ E, double* __restrict__ lam) {
  __shared__ double red[32];
  __shared__ double s_delta;
  const int64_t rr2 = (int64_t)r * r;
  for (int i = threadIdx.x; i < r; i += blockDim.x)
    lam[i] = S[(int64_t)i * r + i] / C[(int64_t)i * r + i];  // S_ii / (1 - R_ii)
  __syncthreads();
  double off = 0.0, rn = 0.0, gn = 0.0;
  for (int64_t t = threadIdx.x; t < rr2; t += blockDim.x) {
    const int a = (int)(t / r), b = (int)(t % r);
    const double sv = S[t] - (a == b ? lam[a] : 0.0);
    const double rv = (a == b ? 1.0 : 0.0) - C[t];
    const double gv = G[(int64_t)a * ldg + b];
    off = fma(sv, sv, off);
    rn = fma(rv, rv, rn);
    gn = fma(gv, gv, gn);
  }
  off = block_sum(off, red);
  __syncthreads();
  rn = block_sum(rn, red);
  __syncthreads();
  gn = block_sum(gn, red);
  if (threadIdx.x == 0) s_delta = 2.0 * (sqrt(off) + sqrt(gn) * sqrt(rn));
  __syncthreads();
  const double delta = s_delta;
  for (int64_t t = threadIdx.x; t < rr2; t += blockDim.x) {
    const int a = (int)(t / r), b = (int)(t % r);
    const double rab = (a == b ? 1.0 : 0.0) - C[t];
    double e;
    if (a == b) {
      e = 0.5 * rab;
    } else {
      const double gap = lam[b] - lam[a];
      if (fabs(gap) > delta) e = (S[t] + lam[b] * rab) / gap;
      else e = 0.5 * rab;
    }
    E[t] = e;
  }
}

// Sort eigenpairs by descending eigenvalue (bitonic over 1024 slots, r <= 1024).
__global__ void __launch_bounds__(1024)
k_sort_eig(int r, const double* __restrict__ lam_in, const double* __restrict__ X,
           double* __restrict__ lam_out, double* __restrict__ Ub, int64_t ldu) {
  __shared__ double key[1024];
  __shared__ int idx[1024];
  const int t = threadIdx.x;
  key[t] = t < r ? lam_in[t] : -INFINITY;
  idx[t] = t;
  __syncthreads();
  for (int k = 2; k <= 1024; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int ixj = t ^ j;
      if (ixj > t) {
        const bool desc = (t & k) == 0;
        const double a = key[t], b = key[ixj];
        const int ia = idx[t], ib = idx[ixj];
        // order: larger first (ties broken by index) when desc
        const bool a_first = (a > b) || (a == b && ia < ib);
        if (desc != a_first) {
          key[t] = b; key[ixj] = a; idx[t] = ib; idx[ixj] = ia;
        }
      }
      __syncthreads();
    }
  }
  if (t < r) lam_out[t] = key[t];
  for (int64_t e = t; e < (int64_t)r * r; e += blockDim.x) {
    const int a = (int)(e / r), j = (int)(e % r);
    Ub[(int64_t)a * ldu + j] = X[(int64_t)a * r + idx[j]];
  }
}

}  // namespace

size_t eig_scratch(int r) {
  // floats: A, V (2 r^2) as doubles-equivalent; doubles: X, Xn, C, P, S, E (6 r^2), lam (r)
  const size_t rr = (size_t)r * r;
  return rr + 6 * rr + (size_t)r + gemm_tn_scratch(r, r, r) + 64;
}

svt_status sym_eig(int r, const double* G, int64_t ldg, double* lam, double* Ub, int64_t ldu,
                   double* work, int refine_steps, cudaStream_t s) {
  if (r <= 0) return SVT_OK;
  if (r > 1024) return fail(SVT_ERR_UNSUPPORTED, "eigensolver: r = %d exceeds 1024", r);
  const size_t rr = (size_t)r * r;
  float* A32 = reinterpret_cast<float*>(work);          // r^2 floats
  float* V32 = A32 + rr;                                // r^2 floats (fits in rr doubles)
  double* X = work + rr;
  double* Xn = X + rr;
  double* C = Xn + rr;
  double* P = C + rr;
  double* S = P + rr;
  double* E = S + rr;
  double* lamw = E + rr;
  double* part = lamw + r + 8;

  const size_t smem = 2 * rr * sizeof(float);
  const int use_smem = smem <= 200 * 1024 ? 1 : 0;
  if (use_smem) {
    SVT_CUDA(cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  }
  k_jacobi32<<<1, kJacThreads, use_smem ? smem : 0, s>>>(r, G, ldg, A32, V32, 30, use_smem);
  SVT_LAUNCH_CHECK();
  k_to_double<<<(int)ceil_div((int64_t)rr, 256), 256, 0, s>>>((int64_t)rr, V32, X);
  SVT_LAUNCH_CHECK();
  for (int step = 0; step < refine_steps; ++step) {
    SVT_TRY((gemm_tn<double, double>(r, r, r, X, r, X, r, C, r, part, s)));          // X^T X
    SVT_TRY((gemm_nn<double, double>(r, r, r, 1.0, G, ldg, X, r, 0.0, nullptr, 0, P, r, s)));  // G X
    SVT_TRY((gemm_tn<double, double>(r, r, r, X, r, P, r, S, r, part, s)));          // X^T G X
    k_oa_coeffs<<<1, 1024, 0, s>>>(r, G, ldg, C, S, E, lamw);
    SVT_LAUNCH_CHECK();
    SVT_TRY((gemm_nn<double, double>(r, r, r, 1.0, X, r, E, r, 1.0, X, r, Xn, r, s)));  // X + X E
    double* t = X; X = Xn; Xn = t;
  }
  if (refine_steps == 0) {
    // eigenvalues as Rayleigh quotients of the binary32 vectors
    SVT_TRY((gemm_tn<double, double>(r, r, r, X, r, X, r, C, r, part, s)));
    SVT_TRY((gemm_nn<double, double>(r, r, r, 1.0, G, ldg, X, r, 0.0, nullptr, 0, P, r, s)));
    SVT_TRY((gemm_tn<double, double>(r, r, r, X, r, P, r, S, r, part, s)));
    k_oa_coeffs<<<1, 1024, 0, s>>>(r, G, ldg, C, S, E, lamw);
    SVT_LAUNCH_CHECK();
  }
  k_sort_eig<<<1, 1024, 0, s>>>(r, lamw, X, lam, Ub, ldu);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

}  // namespace svt
