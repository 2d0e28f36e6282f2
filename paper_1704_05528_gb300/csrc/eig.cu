// Small symmetric eigenproblem G = U_B diag(lam) U_B^T for the SVD of B (Algorithm 3:
// [U_L, Sigma_L, V_L] = svd(B) with B B^T = G, sigma = sqrt(lam)).
//
// Binary64 arithmetic runs at about 1/58 of the binary32 rate on this part, so the
// decomposition is computed in two stages:
//  1. cyclic Jacobi in binary32 inside one thread block (round-robin pairing, so each
//     step rotates r/2 disjoint planes at once); a pair is rotated while its coupling
//     exceeds 1e-6 of the gap between its diagonal entries and a few binary32 ulps of
//     the entries themselves, for at most 12 sweeps;
//  2. Ogita-Aishima refinement in binary64 (Ogita & Aishima, "Iterative refinement for
//     symmetric eigenvalue decomposition", 2018): with X the current eigenvector
//     estimate, R = I - X^T X, S = X^T G X, lam_i = S_ii / (1 - R_ii), and
//     E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) for well separated pairs,
//     E_ij = R_ij / 2 otherwise; X <- X + X E.  Each step is four r x r x r products
//     (spread over the whole GPU) and converges quadratically.  A pair counts as well
//     separated when its first-order correction is below 0.1 (a per-pair test: the
//     paper's global bound built from Frobenius norms lumps a dense spectrum together).
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

// Rotate the pair (p, q) while its coupling is significant against the gap of its
// diagonal entries (what limits the eigenvector accuracy) and above binary32 rounding
// noise of the entries themselves; the binary64 refinement resolves the rest.
__device__ __forceinline__ bool jac_active(float app, float aqq, float apq, float scale) {
  const float mag = fabsf(apq);
  return mag > 1e-6f * fabsf(app - aqq) && mag > 4e-7f * (fabsf(app) + fabsf(aqq)) &&
         mag > 1e-30f * scale;
}

// A: r x r working copy (row-major), V: r x r eigenvector estimate (columns).
// Each step of a sweep rotates the N/2 disjoint planes of the round-robin pairing at once.
// Because the planes are disjoint, the two-sided update A <- J^T A J and V <- V J splits
// into independent 2x2 blocks (rows of pair i, columns of pair j): thread (i, j) reads
// its block, applies J_i^T . J_j (V only . J_j) and writes it back, so a step needs two
// barriers; a step in which no pair rotates skips the update and its barrier.  After a
// sweep that rotated, one pass over all pairs decides whether another sweep would rotate
// anything (the matrix is unchanged by a sweep without rotations, so this is the same
// test as running that sweep).  With N = r rounded up to even, a pair whose partner is
// the padding index r rotates nothing and has a single row / column.
__global__ void __launch_bounds__(kJacThreads)
k_jacobi32(int r, const double* __restrict__ G, int64_t ldg, float* gA, float* gV,
           int max_sweeps, int use_smem, int* sweeps_out) {
  extern __shared__ float dyn[];
  __shared__ float cs_c[kJacThreads / 2 + 1], cs_s[kJacThreads / 2 + 1];
  __shared__ int pp[kJacThreads / 2 + 1], qq[kJacThreads / 2 + 1];
  __shared__ int active_any, check_any;
  __shared__ int step_flag[3];
  __shared__ float scale;
  float* A = use_smem ? dyn : gA;
  float* V = use_smem ? dyn + r * r : gV;
  const int tid = threadIdx.x;
  for (int a = tid / 32; a < r; a += kJacThreads / 32)
    for (int b = tid % 32; b < r; b += 32) {
      A[a * r + b] = (float)G[(int64_t)a * ldg + b];
      V[a * r + b] = (a == b) ? 1.0f : 0.0f;
    }
  __syncthreads();
  if (tid < 32) {
    float mx = 0.f;
    for (int i = tid; i < r; i += 32) mx = fmaxf(mx, fabsf(A[i * r + i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid == 0) scale = mx;
  }
  if (tid < 3) step_flag[tid] = 0;
  __syncthreads();
  const int N = (r + 1) & ~1;
  const int npairs = N / 2;
  // 2D layout of the block updates: ty = tid / 32 walks pairs i, tx = tid % 32 pairs j
  const int ty = tid >> 5, tx = tid & 31;
  int sweep = 0;
  int gstep = 0;  // steps over all sweeps: step_flag[gstep % 3] marks a rotating step
  if (tid == 0) active_any = 0;
  __syncthreads();
  for (; sweep < max_sweeps; ++sweep) {
    for (int step = 0; step < N - 1; ++step, ++gstep) {
      int* flag = &step_flag[gstep % 3];
      for (int i = tid; i < npairs; i += blockDim.x) {
        int p, q;
        rr_pair(step, i, N, &p, &q);
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, sn = 0.f;
        if (q < r) {
          const float apq = A[p * r + q];
          const float app = A[p * r + p], aqq = A[q * r + q];
          if (jac_active(app, aqq, apq, scale)) {
            const float theta = (aqq - app) / (2.f * apq);
            float t;
            if (fabsf(theta) > 1e15f) t = 0.5f / theta;
            else t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(1.f + theta * theta));
            c = rsqrtf(1.f + t * t);
            sn = t * c;
            *flag = 1;
          }
        }
        cs_c[i] = c; cs_s[i] = sn; pp[i] = p; qq[i] = q;
      }
      __syncthreads();
      // The slot two steps ahead is free: its writers have not passed this barrier's
      // successor yet.  Every thread reads the same *flag (no writer until step gstep + 3).
      if (tid == 0) step_flag[(gstep + 2) % 3] = 0;
      if (!*flag) continue;
      if (tid == 0) active_any = 1;
      for (int i = ty; i < npairs; i += kJacThreads / 32) {
        const int pi = pp[i], qi = qq[i];
        const float ci = cs_c[i], si = cs_s[i];
        const bool hq_i = qi < r;
        for (int j = tx; j < npairs; j += 32) {
          const float cj = cs_c[j], sj = cs_s[j];
          if (si == 0.f && sj == 0.f) continue;         // both planes fixed: block unchanged
          const int pj = pp[j], qj = qq[j];
          const bool hq_j = qj < r;
          // A block rows (pi, qi), columns (pj, qj)
          float a00 = A[pi * r + pj];
          float a01 = hq_j ? A[pi * r + qj] : 0.f;
          float a10 = hq_i ? A[qi * r + pj] : 0.f;
          float a11 = (hq_i && hq_j) ? A[qi * r + qj] : 0.f;
          // rows: J_i^T
          float b00 = ci * a00 - si * a10, b01 = ci * a01 - si * a11;
          float b10 = si * a00 + ci * a10, b11 = si * a01 + ci * a11;
          // columns: . J_j
          A[pi * r + pj] = cj * b00 - sj * b01;
          if (hq_j) A[pi * r + qj] = sj * b00 + cj * b01;
          if (hq_i) A[qi * r + pj] = cj * b10 - sj * b11;
          if (hq_i && hq_j) A[qi * r + qj] = sj * b10 + cj * b11;
          if (sj != 0.f) {  // V <- V J_j on rows (pi, qi)
            const float v00 = V[pi * r + pj], v01 = V[pi * r + qj];
            V[pi * r + pj] = cj * v00 - sj * v01;
            V[pi * r + qj] = sj * v00 + cj * v01;
            if (hq_i) {
              const float v10 = V[qi * r + pj], v11 = V[qi * r + qj];
              V[qi * r + pj] = cj * v10 - sj * v11;
              V[qi * r + qj] = sj * v10 + cj * v11;
            }
          }
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (!active_any) break;  // nothing rotated in this sweep
    // would another sweep rotate anything?
    if (tid == 0) check_any = 0;
    __syncthreads();
    for (int t = tid; t < r * r; t += blockDim.x) {
      const int a = t / r, b = t - (t / r) * r;
      if (a < b && jac_active(A[a * r + a], A[b * r + b], A[a * r + b], scale)) check_any = 1;
    }
    __syncthreads();
    if (!check_any) {
      ++sweep;
      break;
    }
    if (tid == 0) active_any = 0;
    __syncthreads();
  }
  if (use_smem) {
    for (int t = tid; t < r * r; t += blockDim.x) gV[t] = V[t];
  }
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// C = op(A) B + beta Cin for r x r row-major binary64 matrices (op(A) = A or A^T), one
// 8 x 8 output tile per block: binary64 runs at a small fraction of the binary32 rate, so
// small tiles spread an r = 100 product over all SMs instead of a third of them.
constexpr int kSgTile = 8;

template <bool TRANS_A>
__global__ void __launch_bounds__(kSgTile * kSgTile)
k_small_gemm(int r, const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
             double beta, const double* __restrict__ Cin, double* __restrict__ C) {
  constexpr int T = kSgTile;
  __shared__ double As[T][T + 1];
  __shared__ double Bs[T][T + 1];
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  const int i = blockIdx.y * T + ty, j = blockIdx.x * T + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < r; k0 += T) {
    const int ka = k0 + tx, kb = k0 + ty;
    if (TRANS_A) {
      // op(A)[i][k] = A[k][i]: load rows k0.. of A, columns blockIdx.y*T ..
      const int ia = blockIdx.y * T + tx, kk = k0 + ty;
      As[tx][ty] = (ia < r && kk < r) ? A[(int64_t)kk * lda + ia] : 0.0;
    } else {
      As[ty][tx] = (i < r && ka < r) ? A[(int64_t)i * lda + ka] : 0.0;
    }
    Bs[ty][tx] = (kb < r && j < r) ? B[(int64_t)kb * r + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < T; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (i < r && j < r) {
    const int64_t o = (int64_t)i * r + j;
    C[o] = beta != 0.0 ? acc + beta * Cin[o] : acc;
  }
}

__global__ void k_to_double(int64_t count, const float* __restrict__ src, double* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = (double)src[t];
}

// One Ogita-Aishima update from C = X^T X and S = X^T G X (r x r): lam_i = S_ii / C_ii
// (= S_ii / (1 - R_ii)), and E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) wherever that
// first-order correction is small (|E_ij| < 0.1); pairs too close for it to be
// trustworthy are left as a cluster with E_ij = R_ij / 2, as are the diagonal entries.
__global__ void k_oa_lambda(int r, const double* __restrict__ C, const double* __restrict__ S,
                            double* __restrict__ lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < r) lam[i] = S[i * r + i] / C[i * r + i];
}

__global__ void k_oa_coeffs(int r, const double* __restrict__ C, const double* __restrict__ S,
                            const double* __restrict__ lam, double* __restrict__ E) {
  const int rr2 = r * r;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rr2; t += gridDim.x * blockDim.x) {
    const int a = t / r, b = t - (t / r) * r;
    const double rab = (a == b ? 1.0 : 0.0) - C[t];
    double e = 0.5 * rab;
    if (a != b) {
      const double gap = lam[b] - lam[a];
      if (gap != 0.0) {
        const double f = (S[t] + lam[b] * rab) / gap;
        if (fabs(f) < 0.1) e = f;
      }
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
  int P = 2;  // bitonic network over the next power of two >= r
  while (P < r) P <<= 1;
  key[t] = t < r ? lam_in[t] : -INFINITY;
  idx[t] = t;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int ixj = t ^ j;
      if (ixj > t && ixj < P) {
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
  // row a of Ub, column j: warp w takes rows w, w + 32, ...; lanes take columns
  for (int a = t >> 5; a < r; a += blockDim.x >> 5)
    for (int j = t & 31; j < r; j += 32) Ub[(int64_t)a * ldu + j] = X[(int64_t)a * r + idx[j]];
}

}  // namespace

size_t eig_scratch(int r) {
  // floats: A, V (2 r^2) as doubles-equivalent; doubles: X, Xn, C, P, S, E (6 r^2), lam (r)
  const size_t rr = (size_t)r * r;
  return rr + 6 * rr + (size_t)r + gemm_tn_scratch(r, r, r) + 64;
}

svt_status eig_start(int r, const double* G, int64_t ldg, double* work, cudaStream_t s,
                     int* sweeps_out) {
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
  k_jacobi32<<<1, kJacThreads, use_smem ? smem : 0, s>>>(r, G, ldg, A32, V32, 12, use_smem,
                                                         sweeps_out);
  SVT_LAUNCH_CHECK();
  k_to_double<<<(int)ceil_div((int64_t)rr, 256), 256, 0, s>>>((int64_t)rr, V32, X);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

svt_status eig_refine(int r, const double* G, int64_t ldg, double* lam, double* Ub, int64_t ldu,
                      double* work, int refine_steps, cudaStream_t s) {
  if (r <= 0) return SVT_OK;
  const size_t rr = (size_t)r * r;
  double* X = work + rr;
  double* Xn = X + rr;
  double* C = Xn + rr;
  double* P = C + rr;
  double* S = P + rr;
  double* E = S + rr;
  double* lamw = E + rr;
  double* part = lamw + r + 8;
  (void)part;
  const dim3 grid((unsigned)ceil_div(r, kSgTile), (unsigned)ceil_div(r, kSgTile));
  auto gemm = [&](bool ta, const double* A_, int64_t lda_, const double* B_, double beta,
                  const double* Cin_, double* C_) -> svt_status {
    if (ta) k_small_gemm<true><<<grid, kSgTile * kSgTile, 0, s>>>(r, A_, lda_, B_, beta, Cin_, C_);
    else k_small_gemm<false><<<grid, kSgTile * kSgTile, 0, s>>>(r, A_, lda_, B_, beta, Cin_, C_);
    SVT_LAUNCH_CHECK();
    return SVT_OK;
  };
  const int steps = refine_steps > 0 ? refine_steps : 0;
  const int eb = (int)ceil_div((int64_t)r * r, 256);
  for (int step = 0; step <= steps; ++step) {
    SVT_TRY(gemm(true, X, r, X, 0.0, nullptr, C));     // X^T X
    SVT_TRY(gemm(false, G, ldg, X, 0.0, nullptr, P));  // G X
    SVT_TRY(gemm(true, X, r, P, 0.0, nullptr, S));     // X^T G X
    k_oa_lambda<<<(int)ceil_div(r, 256), 256, 0, s>>>(r, C, S, lamw);
    SVT_LAUNCH_CHECK();
    if (step == steps) break;                           // last pass: eigenvalues only
    k_oa_coeffs<<<eb < 1024 ? eb : 1024, 256, 0, s>>>(r, C, S, lamw, E);
    SVT_LAUNCH_CHECK();
    SVT_TRY(gemm(false, X, r, E, 1.0, X, Xn));          // X + X E
    double* t = X; X = Xn; Xn = t;
  }
  k_sort_eig<<<1, 1024, 0, s>>>(r, lamw, X, lam, Ub, ldu);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

svt_status sym_eig(int r, const double* G, int64_t ldg, double* lam, double* Ub, int64_t ldu,
                   double* work, int refine_steps, cudaStream_t s) {
  SVT_TRY(eig_start(r, G, ldg, work, s, nullptr));
  return eig_refine(r, G, ldg, lam, Ub, ldu, work, refine_steps, s);
}

}  // namespace svt
