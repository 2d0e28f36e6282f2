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
//     E_ij = R_ij / 2 otherwise; X <- X + X E.  P = G X is formed once and then carried
//     through the updates (G (X + X E) = P + P E), so a step is three launches: E, the
//     update of [X | P] and X^T [X | P] (r x r x r products spread over the whole GPU);
//     it converges quadratically.  A pair counts as well
//     separated when its first-order correction is below 0.1 (a per-pair test: the
//     paper's global bound built from Frobenius norms lumps a dense spectrum together).
// The eigenpairs are finally sorted by descending eigenvalue.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace svt {
namespace {

constexpr int kJacThreads = 1024;
constexpr int kJacGridThreads = 512;

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
// Cyclic Jacobi sweeps on an r x r binary32 matrix A (row-major, shared or global memory)
// accumulating the rotations into V; every thread of the (kJacThreads) block takes part.
// Returns the number of sweeps that rotated.
__device__ int jacobi_sweeps(int r, float* A, float* V, int max_sweeps) {
  __shared__ float cs_c[kJacThreads / 2 + 1], cs_s[kJacThreads / 2 + 1];
  __shared__ int pp[kJacThreads / 2 + 1], qq[kJacThreads / 2 + 1];
  __shared__ int active_any, check_any;
  __shared__ int step_flag[3];
  __shared__ float scale;
  const int tid = threadIdx.x;
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
  __syncthreads();
  return sweep;
}

__global__ void __launch_bounds__(kJacThreads)
k_jacobi32(int r, const double* __restrict__ G, int64_t ldg, float* gA, float* gV,
           int max_sweeps, int use_smem, int* sweeps_out) {
  extern __shared__ float dyn[];
  float* A = use_smem ? dyn : gA;
  float* V = use_smem ? dyn + r * r : gV;
  const int tid = threadIdx.x;
  for (int a = tid / 32; a < r; a += kJacThreads / 32)
    for (int b = tid % 32; b < r; b += 32) {
      A[a * r + b] = (float)G[(int64_t)a * ldg + b];
      V[a * r + b] = (a == b) ? 1.0f : 0.0f;
    }
  __syncthreads();
  const int sweep = jacobi_sweeps(r, A, V, max_sweeps);
  if (use_smem) {
    for (int t = tid; t < r * r; t += blockDim.x) gV[t] = V[t];
  }
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// C (M x N) = op(A) (M x K) B (K x N) + beta Cin for small row-major binary64 matrices
// (op(A) = A or A^T), one 8 x 8 output tile per block: binary64 runs at a small fraction
// of the binary32 rate, so small tiles spread an r = 100 product over all SMs.
constexpr int kSgTile = 8;

template <bool TRANS_A>
__global__ void __launch_bounds__(kSgTile * kSgTile)
k_small_gemm(int M, int N, int K, const double* __restrict__ A, int64_t lda,
             const double* __restrict__ B, int64_t ldb, double beta, const double* Cin,
             int64_t ldcin, double* C, int64_t ldc) {
  constexpr int T = kSgTile;
  __shared__ double As[T][T + 1];
  __shared__ double Bs[T][T + 1];
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  const int i = blockIdx.y * T + ty, j = blockIdx.x * T + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += T) {
    const int ka = k0 + tx, kb = k0 + ty;
    if (TRANS_A) {
      // op(A)[i][k] = A[k][i]: load rows k0.. of A, columns blockIdx.y*T ..
      const int ia = blockIdx.y * T + tx, kk = k0 + ty;
      As[tx][ty] = (ia < M && kk < K) ? A[(int64_t)kk * lda + ia] : 0.0;
    } else {
      As[ty][tx] = (i < M && ka < K) ? A[(int64_t)i * lda + ka] : 0.0;
    }
    Bs[ty][tx] = (kb < K && j < N) ? B[(int64_t)kb * ldb + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < T; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (i < M && j < N) C[(int64_t)i * ldc + j] = beta != 0.0 ? acc + beta * Cin[(int64_t)i * ldcin + j] : acc;
}

// dst (r x r, leading dimension ldd) from a dense binary32 r x r matrix
__global__ void k_to_double_ld(int r, const float* __restrict__ src, double* __restrict__ dst,
                               int64_t ldd) {
  const int64_t total = (int64_t)r * r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t / r, b = t - a * r;
    dst[a * ldd + b] = (double)src[t];
  }
}


// One Ogita-Aishima update from C = X^T X and S = X^T G X (r x r): lam_i = S_ii / C_ii
// (= S_ii / (1 - R_ii)), and E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) wherever that
// first-order correction is small (|E_ij| < 0.1); pairs too close for it to be
// trustworthy are left as a cluster with E_ij = R_ij / 2, as are the diagonal entries.
// CS = [C | S] is r x 2r (leading dimension 2r).
__device__ __forceinline__ double oa_coeff(int r, const double* __restrict__ CS, int a, int b) {
  const int64_t ld = 2 * (int64_t)r;
  const double cab = CS[a * ld + b], sab = CS[a * ld + r + b];
  const double rab = (a == b ? 1.0 : 0.0) - cab;
  double e = 0.5 * rab;
  if (a != b) {
    const double la = CS[a * ld + r + a] / CS[a * ld + a];
    const double lb = CS[b * ld + r + b] / CS[b * ld + b];
    const double gap = lb - la;
    if (gap != 0.0) {
      const double f = (sab + lb * rab) / gap;
      if (fabs(f) < 0.1) e = f;
    }
  }
  return e;
}

__global__ void k_oa_coeffs(int r, const double* __restrict__ CS, double* __restrict__ E) {
  const int rr2 = r * r;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rr2; t += gridDim.x * blockDim.x)
    E[t] = oa_coeff(r, CS, t / r, t - (t / r) * r);
}

// [X | P] <- [X | P] + [X | P] E, blockwise (X E and P E).  P = G X is carried through the
// update instead of being formed again from G: G (X + X E) = P + P E.  XP and XPn are
// r x 2r (leading dimension l2); blockIdx.z selects the X or the P block.  Each output is
// sum_l A[i][l] E[l][j] in the order of l, then + A[i][j].
__global__ void __launch_bounds__(kSgTile * kSgTile)
k_oa_update(int r, const double* __restrict__ XP, int64_t l2, const double* __restrict__ E,
            double* __restrict__ XPn) {
  constexpr int T = kSgTile;
  __shared__ double As[T][T + 1];
  __shared__ double Es[T][T + 1];
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  const int i = blockIdx.y * T + ty, j = blockIdx.x * T + tx;
  const double* Ab = XP + (int64_t)blockIdx.z * r;
  double acc = 0.0;
  for (int k0 = 0; k0 < r; k0 += T) {
    const int ka = k0 + tx, kb = k0 + ty;
    As[ty][tx] = (i < r && ka < r) ? Ab[(int64_t)i * l2 + ka] : 0.0;
    Es[ty][tx] = (kb < r && j < r) ? E[(int64_t)kb * r + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < T; ++kk) acc = fma(As[ty][kk], Es[kk][tx], acc);
    __syncthreads();
  }
  if (i < r && j < r) XPn[(int64_t)i * l2 + (int64_t)blockIdx.z * r + j] = acc + Ab[(int64_t)i * l2 + j];
}

// The end of a refinement, in one block of 1024 threads (r <= 1024): the eigenvalues
// lam_i = S_ii / C_ii; when `status` is given, the convergence test (*status = 1 when an
// off-diagonal entry of S = X^T G X exceeds tol times its largest diagonal entry, i.e. a
// coupled pair was left unresolved, else 0); then the eigenpairs sorted by descending
// eigenvalue (each thread counts the eigenvalues ranked before its own; ties by index)
// into lam_out and the columns of Ub.
__global__ void __launch_bounds__(1024)
k_oa_finish(int r, const double* __restrict__ CS, double tol, int* __restrict__ status,
            const double* __restrict__ X, int64_t ldx, double* __restrict__ lam_out,
            double* __restrict__ Ub, int64_t ldu) {
  __shared__ double key[1024];
  __shared__ unsigned long long okey[1024];
  __shared__ int idx[1024];
  __shared__ unsigned long long red_off[32], red_diag[32];
  const int t = threadIdx.x;
  const int64_t ld = 2 * (int64_t)r;
  // Comparisons run on the bit patterns in the integer pipes: binary64 runs at a small
  // fraction of the rate, and this kernel is one block.  |v| orders as its bits without
  // the sign (a NaN above infinity).
  constexpr unsigned long long kAbs = 0x7fffffffffffffffull;
  if (status) {
    unsigned long long off = 0ull, dg = 0ull;
    for (int e = t; e < r * r; e += blockDim.x) {
      const int a = e / r, b = e - (e / r) * r;
      const unsigned long long v = (unsigned long long)__double_as_longlong(CS[a * ld + r + b]) & kAbs;
      if (a == b) dg = v > dg ? v : dg; else off = v > off ? v : off;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long xo = __shfl_xor_sync(0xffffffffu, off, o);
      const unsigned long long xd = __shfl_xor_sync(0xffffffffu, dg, o);
      off = xo > off ? xo : off;
      dg = xd > dg ? xd : dg;
    }
    if ((t & 31) == 0) { red_off[t >> 5] = off; red_diag[t >> 5] = dg; }
  }
  if (t < r) {
    const double lam = CS[t * ld + r + t] / CS[t * ld + t];
    const unsigned long long bits = (unsigned long long)__double_as_longlong(lam);
    key[t] = lam;
    // order-preserving key: larger value, larger key; a NaN above every number
    okey[t] = (bits & kAbs) > 0x7ff0000000000000ull ? ~0ull
              : (bits >> 63) ? ~bits : (bits | 0x8000000000000000ull);
  }
  idx[t] = t < r ? t : 0;
  __syncthreads();
  if (status && t == 0) {
    unsigned long long off = red_off[0], dg = red_diag[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      off = red_off[w] > off ? red_off[w] : off;
      dg = red_diag[w] > dg ? red_diag[w] : dg;
    }
    const double offd = __longlong_as_double((long long)off), dgd = __longlong_as_double((long long)dg);
    *status = (offd <= tol * dgd) ? 0 : 1;  // NaN counts as not converged
  }
  // rank of each eigenvalue: the number of eigenvalues placed before it (larger key, or
  // the same key with a smaller index); the order is total, so the ranks are distinct,
  // and a NaN lands first, where the caller rejects it
  double kt = 0.0;
  int rank = 0;
  if (t < r) {
    kt = key[t];
    const unsigned long long ot = okey[t];
    for (int j = 0; j < r; ++j) {
      const unsigned long long oj = okey[j];
      rank += (oj > ot) || (oj == ot && j < t);
    }
  }
  __syncthreads();
  if (t < r) { idx[rank] = t; key[rank] = kt; }
  __syncthreads();
  if (t < r) lam_out[t] = key[t];
  // row a of Ub, column j: warp w takes rows w, w + 32, ...; lanes take columns
  for (int a = t >> 5; a < r; a += blockDim.x >> 5)
    for (int j = t & 31; j < r; j += 32) Ub[(int64_t)a * ldu + j] = X[(int64_t)a * ldx + idx[j]];
}

// Near-diagonal start.  In a recycled basis G = B B^T is close to diagonal: most pairs have
// a first-order coupling |G_ab| / |G_bb - G_aa| well below one, which the Ogita-Aishima
// steps resolve directly.  Pairs at or above kClusterTol are joined into clusters
// (connected components, by label propagation over the list of such pairs); each
// cluster's block of G is diagonalised by cyclic binary32 Jacobi inside one warp, and
// X0 is the identity outside the clusters.  *status = 1 (X0 not written) when a cluster
// has more than kBigClusterMax members or the pair list overflows: the caller then runs
// the full Jacobi.  Clusters of up to kClusterMax members are solved one per warp; larger
// ones (up to kBigClusterMax) one at a time by the whole block with the cyclic Jacobi of
// k_jacobi32 on the cluster's block.
constexpr double kClusterTol = 0.02;
constexpr int kClusterMax = 32;
constexpr int kBigClusterMax = 96;
constexpr int kClusterWarps = 8;  // warps solving small clusters at once
constexpr int kMaxEdges = 4096;

size_t cluster_smem_bytes() {
  return sizeof(int) * (3 * 1024 + 2 * kMaxEdges) +
         sizeof(float) * 2 * kClusterWarps * kClusterMax * (kClusterMax + 1) +
         sizeof(int) * kClusterWarps * kClusterMax +
         sizeof(float) * 2 * kBigClusterMax * kBigClusterMax + sizeof(int) * kBigClusterMax;
}

__global__ void __launch_bounds__(1024)
k_cluster_start(int r, const double* __restrict__ G, int64_t ldg, double* __restrict__ X,
                int64_t ldx, int* __restrict__ status, int identity_on_fail, int shift) {
  extern __shared__ int csm[];
  int* label = csm;                    // 1024
  int* cnt = label + 1024;             // 1024
  int* roots = cnt + 1024;             // 1024
  int* ea = roots + 1024;              // kMaxEdges
  int* eb = ea + kMaxEdges;            // kMaxEdges
  float* blkA = reinterpret_cast<float*>(eb + kMaxEdges);           // warps x 32 x 33
  float* blkV = blkA + kClusterWarps * kClusterMax * (kClusterMax + 1);
  int* mem = reinterpret_cast<int*>(blkV + kClusterWarps * kClusterMax * (kClusterMax + 1));
  float* bigA = reinterpret_cast<float*>(mem + kClusterWarps * kClusterMax);  // big cluster
  float* bigV = bigA + kBigClusterMax * kBigClusterMax;
  int* bigm = reinterpret_cast<int*>(bigV + kBigClusterMax * kBigClusterMax);
  __shared__ int nedges, nroots, bad, bigsz;
  __shared__ float diag[1024];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < r; i += blockDim.x) {
    label[i] = i;
    cnt[i] = 0;
    diag[i] = (float)G[(int64_t)i * ldg + i];
  }
  if (tid == 0) { nedges = 0; nroots = 0; bad = 0; }
  __syncthreads();
  // the pair test runs in binary32 (binary64 is a small fraction of the rate): rounding
  // can only add pairs whose diagonal entries agree to binary32 precision
  for (int64_t t = tid; t < (int64_t)r * r; t += blockDim.x) {
    const int a = (int)(t / r), b = (int)(t - (int64_t)a * r);
    if (a >= b) continue;
    const float gab = (float)G[(int64_t)a * ldg + b];
    const float gap = diag[b] - diag[a];
    if (gab != 0.f && !(fabsf(gab) < (float)kClusterTol * fabsf(gap))) {
      const int e = atomicAdd(&nedges, 1);
      if (e < kMaxEdges) { ea[e] = a; eb[e] = b; } else bad = 1;
    }
  }
  __syncthreads();
  const int ne = nedges < kMaxEdges ? nedges : kMaxEdges;
  for (int it = 0; it < r && !bad; ++it) {
    int moved = 0;
    for (int e = tid; e < ne; e += blockDim.x) {
      const int la = label[ea[e]], lb = label[eb[e]];
      if (la != lb) {
        const int m = la < lb ? la : lb;
        atomicMin(&label[ea[e]], m);
        atomicMin(&label[eb[e]], m);
        moved = 1;
      }
    }
    if (!__syncthreads_or(moved)) break;  // a barrier, and every thread gets the same answer
  }
  for (int i = tid; i < r; i += blockDim.x) atomicAdd(&cnt[label[i]], 1);
  __syncthreads();
  for (int i = tid; i < r; i += blockDim.x) {
    if (label[i] == i && cnt[i] >= 2) {
      if (cnt[i] > kBigClusterMax) bad = 1;
      else if (cnt[i] <= kClusterMax) roots[atomicAdd(&nroots, 1)] = i;
    }
  }
  __syncthreads();
  for (int64_t t = tid; t < (int64_t)r * r && (!bad || identity_on_fail); t += blockDim.x) {
    const int a = (int)(t / r), b = (int)(t - (int64_t)a * r);
    X[(int64_t)a * ldx + b] = a == b ? 1.0 : 0.0;
  }
  if (bad) {
    if (tid == 0) *status = 1;
    return;
  }
  __syncthreads();
  if (warp < kClusterWarps) {
    float* A = blkA + warp * kClusterMax * (kClusterMax + 1);
    float* V = blkV + warp * kClusterMax * (kClusterMax + 1);
    int* mb = mem + warp * kClusterMax;
    constexpr int LD = kClusterMax + 1;
    for (int c = warp; c < nroots; c += kClusterWarps) {
      const int root = roots[c];
      int sz = 0;
      for (int j0 = 0; j0 < r; j0 += 32) {
        const bool in = j0 + lane < r && label[j0 + lane] == root;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) mb[sz + __popc(m & ((1u << lane) - 1u))] = j0 + lane;
        sz += __popc(m);
      }
      __syncwarp();
      // With `shift` (the cluster pass after a refinement, whose clusters are pairs that
      // agree to binary32 rounding) the block is shifted by the mean of its diagonal (in
      // binary64) before it is rounded to binary32: a cluster's eigenvalues agree in their
      // leading digits, and the shift keeps the digits that tell them apart.  Rotations do
      // not depend on it.
      double mu = lane < sz && shift ? G[(int64_t)mb[lane] * ldg + mb[lane]] : 0.0;
      for (int o = 16; o > 0; o >>= 1) mu += __shfl_xor_sync(0xffffffffu, mu, o);
      mu /= (double)sz;
      for (int a = 0; a < sz; ++a)
        if (lane < sz) {
          A[a * LD + lane] = (float)(G[(int64_t)mb[a] * ldg + mb[lane]] - (a == lane ? mu : 0.0));
          V[a * LD + lane] = a == lane ? 1.f : 0.f;
        }
      __syncwarp();
      for (int sweep = 0; sweep < 20; ++sweep) {
        bool any = false;
        for (int p = 0; p < sz - 1; ++p)
          for (int q = p + 1; q < sz; ++q) {
            const float apq = A[p * LD + q], app = A[p * LD + p], aqq = A[q * LD + q];
            const float mag = fabsf(apq);
            if (!(mag > 1e-6f * fabsf(app - aqq) && mag > 4e-7f * (fabsf(app) + fabsf(aqq))))
              continue;
            const float theta = (aqq - app) / (2.f * apq);
            float t;
            if (fabsf(theta) > 1e15f) t = 0.5f / theta;
            else t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(1.f + theta * theta));
            const float cs = rsqrtf(1.f + t * t), sn = t * cs;
            __syncwarp();
            if (lane < sz) {  // rows p, q
              const float x = A[p * LD + lane], y = A[q * LD + lane];
              A[p * LD + lane] = cs * x - sn * y;
              A[q * LD + lane] = sn * x + cs * y;
            }
            __syncwarp();
            if (lane < sz) {  // columns p, q of A and V
              const float x = A[lane * LD + p], y = A[lane * LD + q];
              A[lane * LD + p] = cs * x - sn * y;
              A[lane * LD + q] = sn * x + cs * y;
              const float u = V[lane * LD + p], v = V[lane * LD + q];
              V[lane * LD + p] = cs * u - sn * v;
              V[lane * LD + q] = sn * u + cs * v;
            }
            __syncwarp();
            any = true;
          }
        if (!any) break;
      }
      for (int a = 0; a < sz; ++a)
        if (lane < sz) X[(int64_t)mb[a] * ldx + mb[lane]] = (double)V[a * LD + lane];
      __syncwarp();
    }
  }
  __syncthreads();
  // clusters above kClusterMax, one at a time, by the whole block (roots in index order)
  for (int root = 0; root < r; ++root) {
    if (!(label[root] == root && cnt[root] > kClusterMax)) continue;  // uniform: shared data
    if (warp == 0) {  // members in index order
      int sz = 0;
      for (int j0 = 0; j0 < r; j0 += 32) {
        const bool in = j0 + lane < r && label[j0 + lane] == root;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) bigm[sz + __popc(m & ((1u << lane) - 1u))] = j0 + lane;
        sz += __popc(m);
      }
      if (lane == 0) bigsz = sz;
    }
    __syncthreads();
    const int sz = bigsz;
    // the shift of the warp clusters above: every warp forms the same sum (lanes over
    // members, a fixed shuffle tree, then the lanes' partial sums in order)
    double mu = 0.0;
    for (int a0 = 0; a0 < sz && shift; a0 += 32) {
      double v = a0 + lane < sz ? G[(int64_t)bigm[a0 + lane] * ldg + bigm[a0 + lane]] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      mu += v;
    }
    mu /= (double)sz;
    for (int t = tid; t < sz * sz; t += blockDim.x) {
      const int a = t / sz, b = t - (t / sz) * sz;
      bigA[t] = (float)(G[(int64_t)bigm[a] * ldg + bigm[b]] - (a == b ? mu : 0.0));
      bigV[t] = a == b ? 1.f : 0.f;
    }
    __syncthreads();
    jacobi_sweeps(sz, bigA, bigV, 12);
    for (int t = tid; t < sz * sz; t += blockDim.x) {
      const int a = t / sz, b = t - (t / sz) * sz;
      X[(int64_t)bigm[a] * ldx + bigm[b]] = (double)bigV[t];
    }
    __syncthreads();
  }
  if (tid == 0) *status = 0;
}

}  // namespace

// Scratch (doubles): binary32 A and V of the Jacobi stage (r^2 doubles of room), then
// XP = [X | G X] and XPn (r x 2r each), CS = [X^T X | X^T G X] (r x 2r), E (r x r), lam (r).
size_t eig_scratch(int r) {
  const size_t rr = (size_t)r * r;
  return rr + 7 * rr + (size_t)r + 64;
}

namespace {
// Polls of a grid-barrier wait before it gives up (each poll sleeps about 32 ns): 2^24 in
// normal use; svt_test_set_grid_wait_limit lowers it so that a test can make a wait run out.
std::atomic<unsigned> g_grid_wait_polls{1u << 24};

// Grid-wide barrier of a cooperative launch: an arrival count and a generation word in
// global memory (zero before the launch).  Bounded: a wait that runs out after `limit`
// polls returns false.
__device__ bool grid_barrier(unsigned* bar, unsigned* gen_local, unsigned limit) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok_s = 1;
    const unsigned gen = *gen_local;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {  // last to arrive: reset and release
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const volatile unsigned* g = &bar[1];
      unsigned spins = 0;
      while (*g == gen) {
        if (++spins > limit) { ok_s = 0; break; }
        __nanosleep(32);
      }
    }
    __threadfence();
    *gen_local = gen + 1;
  }
  __syncthreads();
  return ok_s != 0;
}

// The binary32 cyclic Jacobi of jacobi_sweeps for r above what one CTA's shared memory
// holds, spread over a cooperative grid.  A is double-buffered: a rotating step reads
// A_src and writes every element of A_dst, so no CTA ever writes what another may still
// be reading, and one grid barrier per rotating step suffices.  Every CTA computes the
// step's rotations itself from A_src (the same values everywhere, hence the same rotations
// and the same decision to skip a step that rotates nothing), and the 2 x 2 block updates
// J_i^T A J_j of the step are divided over all threads of the grid, one block per thread:
// each element gets the same operations in the same order as in the single-CTA kernel.
// V is updated in place (each element belongs to one block of the step).  A and V live in
// global memory and are read around L1 (other CTAs write them).  A barrier that runs out
// raises FLAG_GRID_TIMEOUT in *status and every CTA stops.
__global__ void __launch_bounds__(kJacGridThreads)
k_jacobi32_grid(int r, const double* __restrict__ G, int64_t ldg, float* A, float* A2, float* V,
                int max_sweeps, int* sweeps_out, unsigned* bar, unsigned* status,
                unsigned wait_limit) {
  __shared__ float cs_c[512], cs_s[512];
  __shared__ int pp[512], qq[512];
  __shared__ float scale;
  const int tid = threadIdx.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  unsigned gen = 0;
  for (int64_t t = gtid; t < (int64_t)r * r; t += gthreads) {
    const int a = (int)(t / r), b = (int)(t - (t / r) * r);
    __stcg(&A[t], (float)G[(int64_t)a * ldg + b]);
    __stcg(&V[t], a == b ? 1.0f : 0.0f);
  }
  bool alive = grid_barrier(bar, &gen, wait_limit);
  if (tid < 32) {
    float mx = 0.f;
    for (int i = tid; i < r; i += 32) mx = fmaxf(mx, fabsf(__ldcg(&A[(int64_t)i * r + i])));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid == 0) scale = mx;
  }
  __syncthreads();
  const int N = (r + 1) & ~1;
  const int npairs = N / 2;
  float* src = A;
  float* dst = A2;
  int sweep = 0;
  for (; sweep < max_sweeps && alive; ++sweep) {
    int rotated = 0;
    for (int step = 0; step < N - 1 && alive; ++step) {
      int any = 0;
      for (int i = tid; i < npairs; i += blockDim.x) {
        int p, q;
        rr_pair(step, i, N, &p, &q);
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, sn = 0.f;
        if (q < r) {
          const float apq = __ldcg(&src[(int64_t)p * r + q]);
          const float app = __ldcg(&src[(int64_t)p * r + p]), aqq = __ldcg(&src[(int64_t)q * r + q]);
          if (jac_active(app, aqq, apq, scale)) {
            const float theta = (aqq - app) / (2.f * apq);
            float t;
            if (fabsf(theta) > 1e15f) t = 0.5f / theta;
            else t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(1.f + theta * theta));
            c = rsqrtf(1.f + t * t);
            sn = t * c;
            any = 1;
          }
        }
        cs_c[i] = c; cs_s[i] = sn; pp[i] = p; qq[i] = q;
      }
      // every CTA read the same A_src, so every CTA takes the same branch here
      if (!__syncthreads_or(any)) continue;
      rotated = 1;
      for (int64_t t = gtid; t < (int64_t)npairs * npairs; t += gthreads) {
        const int i = (int)(t / npairs), j = (int)(t - (t / npairs) * npairs);
        const float ci = cs_c[i], si = cs_s[i], cj = cs_c[j], sj = cs_s[j];
        const int pi = pp[i], qi = qq[i], pj = pp[j], qj = qq[j];
        const bool hq_i = qi < r, hq_j = qj < r;
        const float* a0 = src + (int64_t)pi * r;
        const float* a1 = src + (int64_t)qi * r;
        float* d0 = dst + (int64_t)pi * r;
        float* d1 = dst + (int64_t)qi * r;
        const float a00 = __ldcg(&a0[pj]);
        const float a01 = hq_j ? __ldcg(&a0[qj]) : 0.f;
        const float a10 = hq_i ? __ldcg(&a1[pj]) : 0.f;
        const float a11 = (hq_i && hq_j) ? __ldcg(&a1[qj]) : 0.f;
        if (si == 0.f && sj == 0.f) {  // no rotation touches this block: carry it over
          __stcg(&d0[pj], a00);
          if (hq_j) __stcg(&d0[qj], a01);
          if (hq_i) __stcg(&d1[pj], a10);
          if (hq_i && hq_j) __stcg(&d1[qj], a11);
          continue;
        }
        const float b00 = ci * a00 - si * a10, b01 = ci * a01 - si * a11;
        const float b10 = si * a00 + ci * a10, b11 = si * a01 + ci * a11;
        __stcg(&d0[pj], cj * b00 - sj * b01);
        if (hq_j) __stcg(&d0[qj], sj * b00 + cj * b01);
        if (hq_i) __stcg(&d1[pj], cj * b10 - sj * b11);
        if (hq_i && hq_j) __stcg(&d1[qj], sj * b10 + cj * b11);
        if (sj != 0.f) {
          float* v0 = V + (int64_t)pi * r;
          float* v1 = V + (int64_t)qi * r;
          const float v00 = __ldcg(&v0[pj]), v01 = __ldcg(&v0[qj]);
          __stcg(&v0[pj], cj * v00 - sj * v01);
          __stcg(&v0[qj], sj * v00 + cj * v01);
          if (hq_i) {
            const float v10 = __ldcg(&v1[pj]), v11 = __ldcg(&v1[qj]);
            __stcg(&v1[pj], cj * v10 - sj * v11);
            __stcg(&v1[qj], sj * v10 + cj * v11);
          }
        }
      }
      alive = grid_barrier(bar, &gen, wait_limit);
      float* const t = src; src = dst; dst = t;
    }
    if (!rotated || !alive) break;
    // would another sweep rotate anything?  (each CTA checks the whole of A_src, which no
    // CTA writes before the next barrier: the same answer everywhere)
    int more = 0;
    for (int64_t t = tid; t < (int64_t)r * r && !more; t += blockDim.x) {
      const int a = (int)(t / r), b = (int)(t - (t / r) * r);
      if (a < b && jac_active(__ldcg(&src[(int64_t)a * r + a]), __ldcg(&src[(int64_t)b * r + b]),
                              __ldcg(&src[t]), scale))
        more = 1;
    }
    if (!__syncthreads_or(more)) {
      ++sweep;
      break;
    }
  }
  if (!alive && tid == 0) atomicOr(status, FLAG_GRID_TIMEOUT);
  if (blockIdx.x == 0 && tid == 0 && sweeps_out) *sweeps_out = sweep;
}

struct EigWork {
  float *A32, *V32;
  double *XP, *XPn, *CS, *E, *lam;
  EigWork(int r, double* work) {
    const size_t rr = (size_t)r * r;
    A32 = reinterpret_cast<float*>(work);
    V32 = A32 + rr;
    XP = work + rr;
    XPn = XP + 2 * rr;
    CS = XPn + 2 * rr;
    E = CS + 2 * rr;
    lam = E + rr;
  }
};
}  // namespace

svt_status eig_start(int r, const double* G, int64_t ldg, double* work, cudaStream_t s,
                     int* sweeps_out, unsigned* status) {
  if (r <= 0) return SVT_OK;
  if (r > 1024) return fail(SVT_ERR_UNSUPPORTED, "eigensolver: r = %d exceeds 1024", r);
  const size_t rr = (size_t)r * r;
  EigWork w(r, work);
  const size_t smem = 2 * rr * sizeof(float);
  const int use_smem = smem <= 200 * 1024 ? 1 : 0;
  if (use_smem) {
    SVT_CUDA(cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    k_jacobi32<<<1, kJacThreads, smem, s>>>(r, G, ldg, w.A32, w.V32, 12, 1, sweeps_out);
    SVT_LAUNCH_CHECK();
  } else {
    // above one CTA's shared memory: the cooperative grid version (one CTA per SM at most,
    // and no more CTAs than 2 x 2 blocks of a step, r/2 squared, keep busy)
    unsigned* bar = reinterpret_cast<unsigned*>(w.lam + r);
    SVT_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    int per_sm = 0;
    SVT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi32_grid, kJacGridThreads, 0));
    if (per_sm < 1) return fail(SVT_ERR_UNSUPPORTED, "eigensolver: grid Jacobi does not fit an SM");
    const int64_t work_items = ((int64_t)(r + 1) / 2) * ((r + 1) / 2);
    const int64_t want = ceil_div(work_items, (int64_t)kJacGridThreads * 4);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, num_sms()));
    int rr_ = r, sweeps = 12;
    const double* G_ = G;
    int64_t ldg_ = ldg;
    float* A_ = w.A32;
    float* A2_ = reinterpret_cast<float*>(w.XPn);  // free until the refinement
    float* V_ = w.V32;
    int* so = sweeps_out;
    unsigned* st_ = status ? status : bar + 2;
    unsigned limit = g_grid_wait_polls.load(std::memory_order_relaxed);
    void* args[] = {&rr_, &G_, &ldg_, &A_, &A2_, &V_, &sweeps, &so, &bar, &st_, &limit};
    SVT_CUDA(cudaLaunchCooperativeKernel((const void*)k_jacobi32_grid, dim3(blocks),
                                         dim3(kJacGridThreads), args, 0, s));
    count_launch();
  }
  k_to_double_ld<<<(int)ceil_div((int64_t)rr, 256), 256, 0, s>>>(r, w.V32, w.XP, 2 * (int64_t)r);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

// The cluster kernel's shared-memory limit is raised once per device: the call is not a
// stream operation, so it must stay out of graph captures.
static std::atomic<uint64_t> g_cluster_attr_devices{0};

svt_status eig_prepare() {
  int dev = 0;
  SVT_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (g_cluster_attr_devices.load() & bit) return SVT_OK;
  SVT_CUDA(cudaFuncSetAttribute(k_cluster_start, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cluster_smem_bytes()));
  g_cluster_attr_devices.fetch_or(bit);
  return SVT_OK;
}

svt_status eig_start_clusters(int r, const double* G, int64_t ldg, double* work, cudaStream_t s,
                              int* status, bool identity_on_fail) {
  if (r <= 0 || r > 1024) return fail(SVT_ERR_UNSUPPORTED, "eigensolver: r = %d out of range", r);
  EigWork w(r, work);
  const size_t smem = cluster_smem_bytes();
  SVT_TRY(eig_prepare());
  k_cluster_start<<<1, 1024, smem, s>>>(r, G, ldg, w.XP, 2 * (int64_t)r, status,
                                        identity_on_fail ? 1 : 0, 0);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

svt_status eig_refine_clusters_again(int r, const double* G, int64_t ldg, double* lam, double* Ub,
                                     int64_t ldu, double* work, int x_alt, int refine_steps,
                                     cudaStream_t s, int* status, double tol) {
  EigWork w(r, work);
  const int64_t l2 = 2 * (int64_t)r;
  // the refined X of the preceding eig_refine (in XPn when x_alt)
  const double* Xr = x_alt ? w.XPn : w.XP;
  // clusters of the pairs that S = X^T G X still couples, diagonalised into X1 (identity
  // if a cluster is too large: the check below then fails again)
  const size_t smem = cluster_smem_bytes();
  SVT_TRY(eig_prepare());
  k_cluster_start<<<1, 1024, smem, s>>>(r, w.CS + r, l2, w.E, r, status, 1, 1);
  SVT_LAUNCH_CHECK();
  // X <- X X1, into XP (where the refinement starts)
  const dim3 grid((unsigned)ceil_div(r, kSgTile), (unsigned)ceil_div(r, kSgTile));
  double* Xo = Xr == w.XP ? w.XPn : w.XP;
  k_small_gemm<false><<<grid, kSgTile * kSgTile, 0, s>>>(r, r, r, Xr, l2, w.E, r, 0.0, nullptr, 0,
                                                          Xo, l2);
  SVT_LAUNCH_CHECK();
  if (Xo != w.XP)
    SVT_CUDA(cudaMemcpy2DAsync(w.XP, l2 * sizeof(double), Xo, l2 * sizeof(double),
                               (size_t)r * sizeof(double), r, cudaMemcpyDeviceToDevice, s));
  return eig_refine(r, G, ldg, lam, Ub, ldu, work, refine_steps, s, status, tol);
}

svt_status eig_refine(int r, const double* G, int64_t ldg, double* lam, double* Ub, int64_t ldu,
                      double* work, int refine_steps, cudaStream_t s, int* check_status,
                      double check_tol, int start_alt) {
  if (r <= 0) return SVT_OK;
  EigWork w(r, work);
  const int64_t l2 = 2 * (int64_t)r;
  auto gemm = [&](bool ta, int M, int N, int K, const double* A_, int64_t lda_, const double* B_,
                  int64_t ldb_, double beta, const double* Cin_, int64_t ldcin_, double* C_,
                  int64_t ldc_) -> svt_status {
    const dim3 grid((unsigned)ceil_div(N, kSgTile), (unsigned)ceil_div(M, kSgTile));
    if (ta) k_small_gemm<true><<<grid, kSgTile * kSgTile, 0, s>>>(M, N, K, A_, lda_, B_, ldb_, beta, Cin_, ldcin_, C_, ldc_);
    else k_small_gemm<false><<<grid, kSgTile * kSgTile, 0, s>>>(M, N, K, A_, lda_, B_, ldb_, beta, Cin_, ldcin_, C_, ldc_);
    SVT_LAUNCH_CHECK();
    return SVT_OK;
  };
  const int steps = refine_steps > 0 ? refine_steps : 0;
  double* XP = start_alt ? w.XPn : w.XP;
  double* XPn = start_alt ? w.XP : w.XPn;
  SVT_TRY(gemm(false, r, r, r, G, ldg, XP, l2, 0.0, nullptr, 0, XP + r, l2));  // P = G X
  SVT_TRY(gemm(true, r, 2 * r, r, XP, l2, XP, l2, 0.0, nullptr, 0, w.CS, l2));  // X^T [X | P]
  const dim3 ugrid((unsigned)ceil_div(r, kSgTile), (unsigned)ceil_div(r, kSgTile), 2);
  const int eb = (int)ceil_div((int64_t)r * r, 256);
  for (int step = 0; step < steps; ++step) {
    k_oa_coeffs<<<eb < 1024 ? eb : 1024, 256, 0, s>>>(r, w.CS, w.E);
    SVT_LAUNCH_CHECK();
    k_oa_update<<<ugrid, kSgTile * kSgTile, 0, s>>>(r, XP, l2, w.E, XPn);       // [X | P] (I + E)
    SVT_LAUNCH_CHECK();
    double* t = XP; XP = XPn; XPn = t;
    SVT_TRY(gemm(true, r, 2 * r, r, XP, l2, XP, l2, 0.0, nullptr, 0, w.CS, l2));  // X^T [X | P]
  }
  // The test cannot ask for less than the rounding of S = X^T G X itself, which grows with
  // r: about r units of roundoff of the largest eigenvalue (up to 23 r in a CPU emulation
  // of these steps on spectra like the workloads', r = 150-512).
  const double tol = fmax(check_tol, 64.0 * r * 0x1p-53);
  k_oa_finish<<<1, 1024, 0, s>>>(r, w.CS, tol, check_status, XP, l2, lam, Ub, ldu);
  SVT_LAUNCH_CHECK();
  return SVT_OK;
}

}  // namespace svt

extern "C" unsigned svt_test_set_grid_wait_limit(unsigned polls) {
  return svt::g_grid_wait_polls.exchange(polls == 0 ? 1u : polls);
}
