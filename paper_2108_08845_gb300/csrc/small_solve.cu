// Small (K+B) x (K+B) solve of the per-batch update (Algorithm 1 steps 2, 3, 5).
//
// The paper takes the SVD of the panel's R factor.  Here the panel is represented
// by H = R^T R = S G S (its scaled Gram), and its singular triplets follow from
// the eigen-decomposition H = V diag(lambda) V^T: sigma = sqrt(lambda),
// right singular vectors V, and Q U~ = P V diag(1/sigma) (step 4).
//
// The eigen-solve is built for a GPU whose FP64 rate is ~2 FMA/clk/SM (FP32
// ~114): O(n^3) FP64 work only appears as small GEMMs spread over all SMs.
//   1. eig_levels_launch (small_eig.cu): FP32 tridiagonal solves on successive
//      scale levels, FP64 projections between them; the leading eigenpairs come
//      out accurate to ~u32 / 1e-3 relative to their own size.
//   2. Ogita & Aishima (2018) iterative refinement (RefSyEv) of the leading
//      eigenpairs in FP64 (GEMMs), quadratically convergent from there.
// finalize_kernel sorts, truncates to k1 and forms T = S V_k1 diag(1/sigma).
#include <math.h>

#include "psvd_internal.cuh"

namespace psvd {
namespace {

// Resolution of a Gram-based factorisation: eigenvalues of the scaled Gram below
// lam_floor * lambda_max (singular values below sqrt of that times sigma_max)
// are at the rounding level of the Gram and are not resolved; such kept modes
// are set to zero and reported as PSVD_WARN_RANK_DEFICIENT.  The floor is the
// Gram's (lambda_floor(w)): 1e-9 for the FP32 and tensor-core Grams.

// Sort key with a total order: NaN ranks below every number (ties broken by index
// by the callers), so descending ranks are always a permutation.
__device__ __forceinline__ double sort_key(double x) { return isnan(x) ? -INFINITY : x; }

// C (m x nn) = alpha * op(A) * B + beta * Cin, FP64, column-major.
// op(A) = A (lda >= m) or A^T (A is k x m).  8 x 8 outputs per CTA; blockIdx.z is
// the problem of a batch (each operand offset by its stride).  With ls != nullptr
// the kernel does nothing for a problem whose level solve is no longer active.
template <bool TRANS_A>
__global__ void __launch_bounds__(64, 1) dgemm_kernel(int m, int nn, int k, double alpha,
                                                   const double* __restrict__ A, int lda, int64_t sA,
                                                   const double* __restrict__ B, int ldb, int64_t sB,
                                                   double beta, const double* __restrict__ Cin,
                                                   int ldci, int64_t sCin, double* __restrict__ C,
                                                   int ldc, int64_t sC,
                                                   const LevelState* __restrict__ ls, int64_t sls) {
  const int64_t z = blockIdx.z;
  if (ls && ls[z * sls].active == 0) return;
  A += z * sA;
  B += z * sB;
  C += z * sC;
  if (Cin) Cin += z * sCin;
  __shared__ double As[8][33];
  __shared__ double Bs[32][9];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int row = blockIdx.x * 8 + tx, col = blockIdx.y * 8 + ty;
  double acc = 0.0;
  for (int k0 = 0; k0 < k; k0 += 32) {
    for (int e = threadIdx.x; e < 8 * 32; e += 64) {
      const int r = e % 8, kk = e / 8;  // A tile: rows blockIdx.x*8 + r, k index k0 + kk
      const int gr = blockIdx.x * 8 + r, gk = k0 + kk;
      double v = 0.0;
      if (gr < m && gk < k) v = TRANS_A ? A[gk + (int64_t)gr * lda] : A[gr + (int64_t)gk * lda];
      As[r][kk] = v;
      const int c = e / 32, kb = e % 32;  // B tile: k index k0 + kb, column blockIdx.y*8 + c
      const int gc = blockIdx.y * 8 + c, gkb = k0 + kb;
      Bs[kb][c] = (gc < nn && gkb < k) ? B[gkb + (int64_t)gc * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) acc = fma(As[tx][kk], Bs[kk][ty], acc);
    __syncthreads();
  }
  if (row < m && col < nn) {
    double v = alpha * acc;
    if (beta != 0.0) v = fma(beta, Cin[row + (int64_t)col * ldci], v);
    C[row + (int64_t)col * ldc] = v;
  }
}

// One Ogita-Aishima correction for column j of the refined set J = [0, nJ):
//   RR = I - X^T X (column j),  lt_j = S_jj / (X^T X)_jj,
//   E_ij = (S_ij + lt_j RR_ij) / (lt_j - lt_i)   for well-separated i,
//   E_ij = RR_ij / 2                             within a cluster (and i = j),
// with eigenvalue estimates lt_i = S_ii/(X^T X)_ii for i < nJ and the FP32
// Jacobi values beyond.  The cluster test is relative, |lt_j - lt_i| <=
// tau * max(|lt_i|, |lt_j|), since the Jacobi stage is relatively accurate on
// graded matrices (OA's absolute threshold would merge every small eigenvalue).
// Eigenpairs below the Gram's resolution (lambda <= lam_floor * lambda_max)
// carry no information and are left unrefined (E column zero).
__global__ void oa_correct_kernel(int n, int nJ, const double* __restrict__ S,
                                  const double* __restrict__ XtX, const double* __restrict__ lam,
                                  double tau, double lam_floor, double* __restrict__ E,
                                  double* __restrict__ lamJ, int* __restrict__ info,
                                  SmallBatch bs) {
  const int j = blockIdx.x;
  const int64_t z = blockIdx.y;
  S += z * bs.nn;
  XtX += z * bs.nn;
  E += z * bs.nn;
  lam += z * bs.n;
  lamJ += z * bs.n;
  info += z * bs.info;
  const double* Sj = S + (int64_t)j * n;
  const double* Rj = XtX + (int64_t)j * n;
  const double ltj = Sj[j] / Rj[j];
  if (!(lam[j] > lam_floor * lam[0])) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) E[i + (int64_t)j * n] = 0.0;
    if (threadIdx.x == 0) lamJ[j] = lam[j];
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double rr = ((i == j) ? 1.0 : 0.0) - Rj[i];
    double e;
    if (i == j) {
      e = 0.5 * rr;
    } else {
      const double lti = (i < nJ) ? S[i + (int64_t)i * n] / XtX[i + (int64_t)i * n] : lam[i];
      const double gap = ltj - lti;
      e = 0.5 * rr;
      if (fabs(gap) > tau * fmax(fabs(ltj), fabs(lti))) {
        // first-order correction; one that is not small means the pair is not
        // separated at the current accuracy: treat it as a cluster
        const double f = (Sj[i] + ltj * rr) / gap;
        if (fabs(f) <= 0.25) e = f;
      }
    }
    E[i + (int64_t)j * n] = e;
  }
  if (threadIdx.x == 0) {
    lamJ[j] = ltj;
    if (!isfinite(ltj)) atomicOr(&info[2], 4);
  }
}

// lamJ[j] = x_j^T (H x_j) / x_j^T x_j for the refined columns (W = H X_J given).
__global__ void rayleigh_kernel(int n, int nJ, const double* __restrict__ X,
                                const double* __restrict__ W, double* __restrict__ lamJ,
                                SmallBatch bs) {
  __shared__ double s_num[256], s_den[256];
  const int j = blockIdx.x;
  const int64_t z = blockIdx.y;
  X += z * bs.nn;
  W += z * bs.nn;
  lamJ += z * bs.n;
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = X[i + (int64_t)j * n];
    num = fma(x, W[i + (int64_t)j * n], num);
    den = fma(x, x, den);
  }
  s_num[threadIdx.x] = num;
  s_den[threadIdx.x] = den;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_num[threadIdx.x] += s_num[threadIdx.x + o];
      s_den[threadIdx.x] += s_den[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) lamJ[j] = s_num[0] / s_den[0];
}

__global__ void copy_cols_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                 int64_t count, int64_t stride) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t z = blockIdx.y;
  if (e < count) dst[z * stride + e] = src[z * stride + e];
}

// Sort the refined eigenpairs, truncate to k1 and form the update coefficients.
constexpr int kFinCols = 8;  // output columns per finalize block

__global__ void finalize_kernel(int n, int nJ, int kc, int k1, const double* __restrict__ X,
                                const double* __restrict__ lamJ, const double* __restrict__ D,
                                double ff, double sig_floor, float* __restrict__ T,
                                __nv_bfloat16* __restrict__ T3, double* __restrict__ T64,
                                double* __restrict__ Dnew, int* __restrict__ info, SmallBatch bs) {
  {
    // problem blockIdx.y of a batch (T3 and D are only used unbatched)
    const int64_t z = blockIdx.y;
    X += z * bs.nn;
    lamJ += z * bs.n;
    T += z * bs.T;
    if (T64) T64 += z * bs.T64;
    Dnew += z * bs.Dnew;
    info += z * bs.info;
  }
  // block b takes output columns [kFinCols b, kFinCols (b + 1)); the ordering and
  // the singular values are formed by every block (a few hundred operations)
  __shared__ int order[kMaxN];
  __shared__ double sig[kMaxN], inv[kMaxN];
  const int tid = threadIdx.x;
  const int kb0 = blockIdx.x * kFinCols, kb1 = min(k1, kb0 + kFinCols);
  if (tid < kMaxN) order[tid] = 0;
  __syncthreads();
  if (tid < nJ) {
    const double ki = sort_key(lamJ[tid]);
    int rank = 0;
    for (int j = 0; j < nJ; ++j) {
      const double kj = sort_key(lamJ[j]);
      rank += (kj > ki) || (kj == ki && j < tid);
    }
    order[rank] = tid;
  }
  __syncthreads();
  if (tid < k1) {
    const double l = lamJ[order[tid]];
    sig[tid] = (l > 0.0) ? sqrt(l) : 0.0;
    if (!isfinite(l)) atomicOr(&info[2], 4);
  }
  __syncthreads();
  const double s0 = sig[0];
  if (tid < k1) {
    double s = sig[tid];
    if (!(s > sig_floor * s0) || !isfinite(s)) {
      if (!isfinite(s) || !isfinite(s0)) atomicOr(&info[2], 4);
      else atomicOr(&info[2], 1);
      s = 0.0;
    }
    if (blockIdx.x == 0) Dnew[tid] = s;
    // this block's columns: 1 / (sigma_k ||x_k||)
    if (tid >= kb0 && tid < kb1) {
      double x2 = 0.0;
      for (int i = 0; i < n; ++i) {
        const double x = X[i + (int64_t)order[tid] * n];
        x2 = fma(x, x, x2);
      }
      inv[tid] = (s > 0.0) ? 1.0 / (s * sqrt(x2)) : 0.0;
    }
  }
  __syncthreads();
  for (int e = tid; e < n * (kb1 - kb0); e += blockDim.x) {
    const int i = e % n, k = kb0 + e / n;
    const double scale = (i < kc) ? ff * D[i] : 1.0;
    const double t = scale * X[i + (int64_t)order[k] * n] * inv[k];
    T[i + (int64_t)k * n] = (float)t;
    if (T64) T64[i + (int64_t)k * n] = t;
    if (T3) {
      // exact triple split t = h + m + l (24 significant bits) for BF16 operands
      const __nv_bfloat16 h = __float2bfloat16_rn((float)t);
      const double r1 = t - (double)__bfloat162float(h);
      const __nv_bfloat16 md = __float2bfloat16_rn((float)r1);
      const double r2 = r1 - (double)__bfloat162float(md);
      const __nv_bfloat16 lo = __float2bfloat16_rn((float)r2);
      T3[i + (int64_t)k * 3 * n] = h;
      T3[n + i + (int64_t)k * 3 * n] = md;
      T3[2 * n + i + (int64_t)k * 3 * n] = lo;
    }
  }
  if (tid == 0 && blockIdx.x == 0) info[3] = k1;
}

// Upper Cholesky R^T R = G (FP64, one CTA): row i of R from rows < i.
__global__ void cholesky_kernel(const double* __restrict__ G, int n, double* __restrict__ R,
                                int* __restrict__ info) {
  __shared__ double piv;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) R[e] = 0.0;
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    if (threadIdx.x == 0) {
      double s = G[i + (int64_t)i * n];
      for (int k = 0; k < i; ++k) s -= R[k + (int64_t)i * n] * R[k + (int64_t)i * n];
      if (!(s > 0.0) || !isfinite(s)) {
        atomicOr(&info[2], 4);
        s = 0.0;
      }
      piv = sqrt(s);
      R[i + (int64_t)i * n] = piv;
    }
    __syncthreads();
    const double d = piv;
    for (int j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
      double s = G[i + (int64_t)j * n];
      for (int k = 0; k < i; ++k) s -= R[k + (int64_t)i * n] * R[k + (int64_t)j * n];
      R[i + (int64_t)j * n] = (d > 0.0) ? s / d : 0.0;
    }
    __syncthreads();
  }
}

template <bool TA>
cudaError_t dgemm_b(int m, int nn, int k, double alpha, const double* A, int lda, int64_t sA,
                    const double* B, int ldb, int64_t sB, double beta, const double* Cin, int ldci,
                    int64_t sCin, double* C, int ldc, int64_t sC, const LevelState* ls, int64_t sls,
                    int count, cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(m, 8), (unsigned)ceil_div(nn, 8), (unsigned)count);
  dgemm_kernel<TA><<<grid, 64, 0, st>>>(m, nn, k, alpha, A, lda, sA, B, ldb, sB, beta, Cin, ldci,
                                        sCin, C, ldc, sC, ls, sls);
  return cudaGetLastError();
}

// One GEMM per problem of the batch w.bat on the n x n workspaces (stride bs.nn).
template <bool TA>
cudaError_t dgemm_w(const SmallBatch& bs, int m, int nn, int k, double alpha, const double* A,
                    int lda, const double* B, int ldb, double beta, const double* Cin, int ldci,
                    double* C, int ldc, cudaStream_t st) {
  return dgemm_b<TA>(m, nn, k, alpha, A, lda, bs.nn, B, ldb, bs.nn, beta, Cin, ldci, bs.nn, C, ldc,
                     bs.nn, nullptr, 0, bs.count, st);
}

// info[0] = levels, info[1] = leading eigenpairs resolved; bit 2 when the levels
// ended before resolving nJ eigenpairs above the resolution floor.
__global__ void level_info_kernel(const LevelState* __restrict__ ls, int nJ, int* __restrict__ info,
                                  SmallBatch bs) {
  ls += blockIdx.x * bs.ls;
  info += blockIdx.x * bs.info;
  info[0] = ls->levels;
  info[1] = ls->b;
  if (ls->b < nJ && !ls->floored) atomicOr(&info[2], 2);
}

}  // namespace

cudaError_t small_solve_launch(const SmallWork& w, int n, int kc, int k1, const double* D,
                               double ff, int refine_steps, int max_levels, cudaStream_t st,
                               int* launches) {
  cudaError_t e;
  const SmallBatch& bs = w.bat;
  const unsigned nb = (unsigned)bs.count;
  const int nJ = (k1 + kRefineMargin < n) ? k1 + kRefineMargin : n;
  int nl = 0;
  // 1. basis X and eigenvalue estimates lam from the scale levels
  if ((e = eig_levels_launch(w, n, nJ, max_levels, st, &nl)) != cudaSuccess) return e;
  level_info_kernel<<<nb, 1, 0, st>>>(w.ls, nJ, w.info, bs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 2. Ogita-Aishima refinement of the leading nJ eigenpairs
  for (int it = 0; it < refine_steps; ++it) {
    // W = H X_J ; S = X^T W ; XtX = X^T X_J
    if ((e = dgemm_w<false>(bs, n, nJ, n, 1.0, w.H, n, w.X, n, 0.0, nullptr, n, w.W, n, st))) return e;
    if ((e = dgemm_w<true>(bs, n, nJ, n, 1.0, w.X, n, w.W, n, 0.0, nullptr, n, w.S, n, st))) return e;
    if ((e = dgemm_w<true>(bs, n, nJ, n, 1.0, w.X, n, w.X, n, 0.0, nullptr, n, w.R, n, st))) return e;
    oa_correct_kernel<<<dim3(nJ, nb), 256, 0, st>>>(n, nJ, w.S, w.R, w.lam, 1e-5, lambda_floor(w),
                                                    w.E, w.lamJ, w.info, bs);
    if ((e = cudaGetLastError())) return e;
    // X_J <- X_J + X E
    if ((e = dgemm_w<false>(bs, n, nJ, n, 1.0, w.X, n, w.E, n, 1.0, w.X, n, w.Xn, n, st))) return e;
    const int64_t cnt = (int64_t)n * nJ;
    copy_cols_kernel<<<dim3((unsigned)ceil_div(cnt, 256), nb), 256, 0, st>>>(w.Xn, w.X, cnt, bs.nn);
    if ((e = cudaGetLastError())) return e;
  }
  // eigenvalues consistent with the final vectors: sigma_j^2 = x_j^T H x_j / x_j^T x_j,
  // so that every new mode P x_j / sigma_j has unit norm
  if ((e = dgemm_w<false>(bs, n, nJ, n, 1.0, w.H, n, w.X, n, 0.0, nullptr, n, w.W, n, st))) return e;
  rayleigh_kernel<<<dim3(nJ, nb), 256, 0, st>>>(n, nJ, w.X, w.W, w.lamJ, bs);
  if ((e = cudaGetLastError())) return e;
  finalize_kernel<<<dim3((unsigned)ceil_div(k1 > 0 ? k1 : 1, kFinCols), nb), 256, 0, st>>>(
      n, nJ, kc, k1, w.X, w.lamJ, D, ff, sqrt(lambda_floor(w)), w.T, nullptr, w.T64, w.Dnew, w.info,
      bs);
  *launches = nl + 1 + 6 * refine_steps + 3;
  return cudaGetLastError();
}

cudaError_t dgemm_batched_launch(bool trans_a, int m, int nn, int k, double alpha, const double* A,
                                 int lda, int64_t sA, const double* B, int ldb, int64_t sB,
                                 double beta, const double* Cin, int ldci, int64_t sCin, double* C,
                                 int ldc, int64_t sC, const LevelState* ls, int64_t sls, int count,
                                 cudaStream_t st) {
  return trans_a ? dgemm_b<true>(m, nn, k, alpha, A, lda, sA, B, ldb, sB, beta, Cin, ldci, sCin, C,
                                 ldc, sC, ls, sls, count, st)
                 : dgemm_b<false>(m, nn, k, alpha, A, lda, sA, B, ldb, sB, beta, Cin, ldci, sCin, C,
                                  ldc, sC, ls, sls, count, st);
}

cudaError_t dgemm_launch(bool trans_a, int m, int nn, int k, double alpha, const double* A, int lda,
                         const double* B, int ldb, double beta, const double* Cin, int ldci,
                         double* C, int ldc, cudaStream_t st) {
  return dgemm_batched_launch(trans_a, m, nn, k, alpha, A, lda, 0, B, ldb, 0, beta, Cin, ldci, 0, C,
                              ldc, 0, nullptr, 0, 1, st);
}

cudaError_t cholesky_launch(const double* G, int n, double* R, int* info, cudaStream_t st) {
  cholesky_kernel<<<1, 256, 0, st>>>(G, n, R, info);
  return cudaGetLastError();
}

}  // namespace psvd
