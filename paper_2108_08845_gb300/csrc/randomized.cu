// Randomized low-rank SVD of the Algorithm 1 panel (Sec. 3.3), carried out in the
// panel's coefficient space.
//
// The paper replaces the SVD of each panel P = [U | A] S (S = diag(ff D, 1),
// n = kc + B columns) by the randomized range finder with q power iterations
// (Halko, Martinsson & Tropp 2011, Algorithms 4.3/4.4 and 5.1):
//   Y = P Omega, Q = orth(Y);  q times: Z = orth(P^T Q), Y = P Z, Q = orth(Y);
//   B = Q^T P = U~ Sigma V~^T;  U_new = Q U~_K, D_new = Sigma_K,
// each new mode signed so that (P 1)^T u_j >= 0 (the paper leaves signs free, but
// with a fixed Omega the next update depends on them).
// Every tall matrix here is P times a small one, and P^T P = H = S G S is the
// FP64 matrix the exact path already forms.  Writing Q = P W (W n x l):
//   Q^T Q = W^T H W,  P^T Q = H W,  B B^T = W^T H^2 W = C^T C with C = H W,
// so the whole range finder runs on n x l and l x l FP64 matrices, and the tall
// panel is read only by the Gram before and by the update U_new = [U | A] (S W U~_K)
// after.  orth() in the metric of H (Q^T Q = I) and in the Euclidean metric
// (for Z) is CholeskyQR2 with diagonal pivoting: directions whose pivot falls
// below a relative tolerance are numerically outside the range of P and are
// dropped (zero columns), which keeps rank-deficient panels well defined.
#include <math.h>

#include "psvd_internal.cuh"

namespace psvd {
namespace {

constexpr int PCT = 512;                 // threads of the pivoted Cholesky kernel
constexpr int kSmemMaxL = 160;           // l x l FP64 working matrix kept in shared memory up to here
constexpr double kPivotTolRel = 1e-12;   // drop tolerance relative to the largest diagonal entry

#define RCK(x)                                     \
  do {                                             \
    cudaError_t err_ = (x);                        \
    if (err_ != cudaSuccess) return err_;          \
  } while (0)

unsigned blocks_for(int64_t count, int threads) { return (unsigned)ceil_div(count, threads); }

__global__ void widen_kernel(const float* __restrict__ x, int64_t count, double* __restrict__ y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) y[e] = (double)x[e];
}

__device__ __forceinline__ double warp_max_arg(double v, int* idx) {
  // maximum with the smallest index among ties; idx < 0 marks an empty slot
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oi = __shfl_xor_sync(0xffffffffu, *idx, off);
    if (oi >= 0 && (*idx < 0 || ov > v || (ov == v && oi < *idx))) {
      v = ov;
      *idx = oi;
    }
  }
  return v;
}

// Pivoted Cholesky (diagonal pivoting, outer-product form) of the symmetric
// positive semi-definite M (l x l, ld l):  Pi^T M Pi = R^T R.  Stops at the first
// pivot <= kPivotTolRel * max diag(M); the number of pivots taken is the rank r.
// Outputs: Rr[k + j*l] = R's row k at original column j (zero where unset),
// piv[k] = original index of pivot k, rank[0] = r.  Aw: l x l FP64 scratch used
// when l > kSmemMaxL.
__global__ void __launch_bounds__(PCT) pchol_kernel(const double* __restrict__ M, int l,
                                                    double* __restrict__ Rr, int* __restrict__ piv,
                                                    int* __restrict__ rank,
                                                    double* __restrict__ Aw_global) {
  extern __shared__ __align__(16) double sm_aw[];
  __shared__ double rk[kMaxN];
  __shared__ int active[kMaxN];
  __shared__ int s_p;
  __shared__ double s_piv_val, s_tol;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* Aw = (l <= kSmemMaxL) ? sm_aw : Aw_global;
  const int ll = l * l;
  for (int e = tid; e < ll; e += PCT) {
    Aw[e] = M[e];
    Rr[e] = 0.0;
  }
  for (int j = tid; j < l; j += PCT) active[j] = 1;
  __syncthreads();
  if (warp == 0) {
    double dmax = 0.0;
    for (int j = lane; j < l; j += 32) {
      const double d = Aw[j + j * l];
      if (d > dmax) dmax = d;
    }
    for (int off = 16; off > 0; off >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
    if (lane == 0) s_tol = isfinite(dmax) ? kPivotTolRel * dmax : INFINITY;
  }
  __syncthreads();
  const double tol = s_tol;
  int r = 0;
  for (int k = 0; k < l; ++k) {
    if (warp == 0) {
      double best = 0.0;
      int bi = -1;
      for (int j = lane; j < l; j += 32) {
        const double d = Aw[j + j * l];
        if (active[j] && !isnan(d) && (bi < 0 || d > best)) {
          best = d;
          bi = j;
        }
      }
      best = warp_max_arg(best, &bi);
      if (lane == 0) {
        const bool ok = bi >= 0 && best > tol;  // false for NaN as well
        s_p = ok ? bi : -1;
        s_piv_val = ok ? sqrt(best) : 0.0;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) break;  // uniform: every thread read the same shared value
    const double rkk = s_piv_val;
    // row k of R: rk[j] = Aw[p, j] / rkk for active j != p, zero elsewhere
    for (int j = tid; j < l; j += PCT) {
      const double v = (j != p && active[j]) ? Aw[p + j * l] / rkk : 0.0;
      rk[j] = v;
      Rr[k + (int64_t)j * l] = (j == p) ? rkk : v;
    }
    __syncthreads();
    // trailing update Aw -= rk rk^T (rows / columns outside the active set see zeros)
    for (int e = tid; e < ll; e += PCT) {
      const int i = e % l, j = e / l;
      Aw[e] -= rk[i] * rk[j];
    }
    if (tid == 0) {
      piv[k] = p;
      active[p] = 0;
    }
    r = k + 1;
    __syncthreads();
  }
  if (tid == 0) rank[0] = r;
}

// W = V Pi R11^{-1} row by row (W R11 = (V Pi)[:, 0:r], forward substitution),
// columns r..l-1 of W set to zero.  V, W: n x l (ld n); one thread per row.
__global__ void trsm_rows_kernel(const double* __restrict__ V, int n, int l,
                                 const double* __restrict__ Rr, const int* __restrict__ piv,
                                 const int* __restrict__ rank, double* __restrict__ W) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = rank[0];
  for (int c = 0; c < r; ++c) {
    const int pc = piv[c];
    double s = V[i + (int64_t)pc * n];
    for (int b = 0; b < c; ++b) s -= W[i + (int64_t)b * n] * Rr[b + (int64_t)pc * l];
    W[i + (int64_t)c * n] = s / Rr[c + (int64_t)pc * l];
  }
  for (int c = r; c < l; ++c) W[i + (int64_t)c * n] = 0.0;
}

// Sign convention of the new modes u_j = Q U~_j: (P 1)^T u_j >= 0.  With
// C = P^T Q (n x l) that is 1^T C U~_j >= 0; sgn[j] = -1 where it is negative.
// One CTA: column sums of C, then one dot product per kept mode.
__global__ void sign_kernel(const double* __restrict__ C, int n, int l, int k1,
                            const float* __restrict__ Tsmall, double* __restrict__ sgn) {
  __shared__ double csum[kMaxN];
  for (int c = threadIdx.x; c < l; c += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += C[i + (int64_t)c * n];
    csum[c] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k1; j += blockDim.x) {
    double g = 0.0;
    for (int c = 0; c < l; ++c) g = fma(csum[c], (double)Tsmall[c + (int64_t)j * l], g);
    sgn[j] = (g < 0.0) ? -1.0 : 1.0;
  }
}

// T_upd (n x k1, ld n, FP32) = S W U~ diag(sgn) with U~[c, j] = T_small[c, j] * sigma_j
// (T_small = U~ diag(1/sigma) from the eigen-solve of C^T C, ld l).
__global__ void coef_kernel(const double* __restrict__ W, int n, int l, int k1,
                            const float* __restrict__ Tsmall, const double* __restrict__ sigma,
                            const double* __restrict__ sgn, int kc, const double* __restrict__ D,
                            double ff, float* __restrict__ Tupd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * k1) return;
  const int i = (int)(e % n), j = (int)(e / n);
  double acc = 0.0;
  for (int c = 0; c < l; ++c)
    acc = fma(W[i + (int64_t)c * n], (double)Tsmall[c + (int64_t)j * l], acc);
  const double s = (i < kc) ? ff * D[i] : 1.0;
  Tupd[e] = (float)(s * acc * sigma[j] * sgn[j]);
}

size_t pchol_smem(int l) { return (l <= kSmemMaxL) ? sizeof(double) * (size_t)l * l : 0; }

cudaError_t pchol(const RandWork& r, const double* M, int l, cudaStream_t st) {
  const size_t smem = pchol_smem(l);
  RCK(cudaFuncSetAttribute(pchol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pchol_smem(kSmemMaxL)));
  pchol_kernel<<<1, PCT, smem, st>>>(M, l, r.Rr, r.piv, r.rank, r.Aw);
  return cudaGetLastError();
}

cudaError_t trsm_rows(const RandWork& r, const double* V, int n, int l, double* W, cudaStream_t st) {
  trsm_rows_kernel<<<blocks_for(n, 64), 64, 0, st>>>(V, n, l, r.Rr, r.piv, r.rank, W);
  return cudaGetLastError();
}

// out = basis of span(in) orthonormal in the metric of H (out^T H out = I_r + 0),
// two pivoted-CholeskyQR passes; tmp and hv are n x l scratch, out may alias in.
cudaError_t h_orth(const RandWork& r, const double* H, int n, int l, const double* in, double* tmp,
                   double* hv, double* out, cudaStream_t st, int* nl) {
  const double* src = in;
  for (int pass = 0; pass < 2; ++pass) {
    double* dst = pass == 0 ? tmp : out;
    RCK(dgemm_launch(false, n, l, n, 1.0, H, n, src, n, 0.0, nullptr, n, hv, n, st));
    RCK(dgemm_launch(true, l, l, n, 1.0, src, n, hv, n, 0.0, nullptr, l, r.Mm, l, st));
    RCK(pchol(r, r.Mm, l, st));
    RCK(trsm_rows(r, src, n, l, dst, st));
    src = dst;
  }
  *nl += 8;
  return cudaSuccess;
}

// out = Euclidean orthonormal basis of span(in); tmp is n x l scratch.
cudaError_t e_orth(const RandWork& r, int n, int l, const double* in, double* tmp, double* out,
                   cudaStream_t st, int* nl) {
  const double* src = in;
  for (int pass = 0; pass < 2; ++pass) {
    double* dst = pass == 0 ? tmp : out;
    RCK(dgemm_launch(true, l, l, n, 1.0, src, n, src, n, 0.0, nullptr, l, r.Mm, l, st));
    RCK(pchol(r, r.Mm, l, st));
    RCK(trsm_rows(r, src, n, l, dst, st));
    src = dst;
  }
  *nl += 6;
  return cudaSuccess;
}

}  // namespace

cudaError_t randomized_solve_launch(const RandWork& r, const SmallWork& w, int n, int kc, int k1,
                                    int l, int q, const double* D, double ff, uint64_t seed,
                                    uint64_t sketch_id, cudaStream_t st, int* launches) {
  int nl = 0;
  const int64_t nlc = (int64_t)n * l;
  double* B0 = r.B[0];
  double* B1 = r.B[1];
  double* B2 = r.B[2];
  // Omega (n x l, Philox stream sketch_id), W = h_orth(Omega): Q = P W spans P Omega
  RCK(gaussian_sketch_launch(seed, sketch_id, n, l, r.Om, st));
  widen_kernel<<<blocks_for(nlc, 256), 256, 0, st>>>(r.Om, nlc, B0);
  RCK(cudaGetLastError());
  nl += 2;
  RCK(h_orth(r, w.H, n, l, B0, B1, B2, B0, st, &nl));
  for (int it = 0; it < q; ++it) {
    // Z = P^T Q = H W, Z^ = orth(Z), then Q = orth(P Z^): W = h_orth(Z^)
    RCK(dgemm_launch(false, n, l, n, 1.0, w.H, n, B0, n, 0.0, nullptr, n, B2, n, st));
    nl += 1;
    RCK(e_orth(r, n, l, B2, B1, B0, st, &nl));
    RCK(h_orth(r, w.H, n, l, B0, B1, B2, B0, st, &nl));
  }
  // C = P^T Q = H W;  B B^T = C^T C (l x l)
  RCK(dgemm_launch(false, n, l, n, 1.0, w.H, n, B0, n, 0.0, nullptr, n, B2, n, st));
  RCK(dgemm_launch(true, l, l, n, 1.0, B2, n, B2, n, 0.0, nullptr, l, r.Bb, l, st));
  nl += 2;
  // B B^T = U~ Sigma^2 U~^T: the eigen-solve returns T_small = U~_K diag(1/sigma), Dnew
  SmallWork wb = w;
  wb.H = r.Bb;
  int ns = 0;
  RCK(small_solve_launch(wb, l, 0, k1, nullptr, 1.0, /*refine_steps=*/3, kMaxLevels, st,
                         &ns));
  nl += ns;
  sign_kernel<<<1, 256, 0, st>>>(B2, n, l, k1, w.T, r.sgn);
  RCK(cudaGetLastError());
  coef_kernel<<<blocks_for((int64_t)n * k1, 128), 128, 0, st>>>(B0, n, l, k1, w.T, w.Dnew, r.sgn,
                                                               kc, D, ff, r.Tupd);
  RCK(cudaGetLastError());
  nl += 2;
  *launches = nl;
  return cudaSuccess;
}

cudaError_t randomized_wide_launch(const RandWork& r, const SmallWork& w, const double* W,
                                   const double* WW, int N, int m, int k, int l, int q,
                                   uint64_t seed, uint64_t sketch_id, double* Tout,
                                   cudaStream_t st, int* launches) {
  int nl = 0;
  const int64_t mlc = (int64_t)m * l;
  double* B0 = r.B[0];  // m x l: the widened sketch, then n x l scratch
  double* B1 = r.B[1];  // N x l: Q
  double* B2 = r.B[2];  // N x l: products with W W^T
  RCK(gaussian_sketch_launch(seed, sketch_id, m, l, r.Om, st));
  widen_kernel<<<blocks_for(mlc, 256), 256, 0, st>>>(r.Om, mlc, B0);
  RCK(cudaGetLastError());
  // Y = W Omega, Q = orth(Y)
  RCK(dgemm_launch(false, N, l, m, 1.0, W, N, B0, m, 0.0, nullptr, N, B1, N, st));
  nl += 3;
  RCK(e_orth(r, N, l, B1, B2, B1, st, &nl));
  // power steps: span(W W^T Q) is span(W Q^) with Q^ = orth(W^T Q)
  for (int it = 0; it < q; ++it) {
    RCK(dgemm_launch(false, N, l, N, 1.0, WW, N, B1, N, 0.0, nullptr, N, B2, N, st));
    nl += 1;
    RCK(e_orth(r, N, l, B2, B0, B1, st, &nl));
  }
  // B B^T = Q^T W W^T Q (l x l)
  RCK(dgemm_launch(false, N, l, N, 1.0, WW, N, B1, N, 0.0, nullptr, N, B2, N, st));
  RCK(dgemm_launch(true, l, l, N, 1.0, B1, N, B2, N, 0.0, nullptr, l, r.Bb, l, st));
  nl += 2;
  // B B^T = U_B diag(s^2) U_B^T: w.T64 = U_B[:, :k] diag(1/s), w.Dnew = s
  SmallWork wb = w;
  wb.H = r.Bb;
  int ns = 0;
  RCK(small_solve_launch(wb, l, 0, k, nullptr, 1.0, /*refine_steps=*/3, kMaxLevels, st, &ns));
  nl += ns;
  // X diag(1/s) = Q U_B[:, :k] diag(1/s)
  RCK(dgemm_launch(false, N, k, l, 1.0, B1, N, w.T64, l, 0.0, nullptr, N, Tout, N, st));
  nl += 1;
  *launches = nl;
  return cudaSuccess;
}

}  // namespace psvd
