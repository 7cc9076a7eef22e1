// Adjoint (reverse-mode derivative) of one step of Algorithm 1 (Sec. 3.1, steps
// 1-5, or the initialisation I1-I2 when kc = 0).
//
// The step maps the panel P = [ff U diag(D) | A] (M x n, n = kc + B) to its
// leading k1 left singular vectors U' = Y_k and singular values D' = s_k.  Given
// the cotangents (Ybar, sbar) of (U', D'), the panel's cotangent is
//
//   Pbar = Y [diag(sbar) + (F o (X - X^T)) S] V^T + (I - Y Y^T) Ybar S^-1 V^T,
//   X = Y^T Ybar,  F_ij = 1 / (s_j^2 - s_i^2)
//
// (the SVD backward with the 1/(s_i^2 - s_j^2) terms).  Neither Q nor the M x n
// singular basis Y is kept or formed: with Y = P V S^-1 the cotangent is
//
//   Pbar = P N + Ybar E,  E = S_k^-1 V_k^T,
//   N = V_k W V_k^T + Xc S_k^-1 V_k^T + V_k S_k^-1 Xc^T,
//
// where V_k = P^T U' S_k^-1 is recovered from the stored output modes (the role
// the stored R plays for Q = P R^-1), W (k1 x k1) holds the kept-kept terms, and
// the dropped directions enter only through the shifted solves
//   Xc_j = (s_j^2 I - Pi H Pi)^-1 Pi P^T ybar_j,  H = P^T P,  Pi = I - V_k V_k^T,
// which are symmetric positive definite when s_j exceeds every dropped singular
// value.  Everything the small side needs comes from one pass over the rows:
//   G = [U | A]^T [U | A | U' | Ybar]   (FP32 products, float-float slab sums,
//                                        FP64 fixed-order reduction over chunks)
// and the result from a second:  [Ubar | Abar] = [U | A | Ybar] Cf  (FP32),
// with Cf = [S N ; E] and the chain rule of P = [ff U diag(D) | A] folded in:
//   Ubar = ff Pbar_U diag(D),  Dbar_k = ff <U_k, Pbar_U,k>,  Abar = Pbar_A.
#include <math.h>

#include <algorithm>
#include <new>

#include "psvd_internal.cuh"

namespace psvd {
namespace {

constexpr int AT = 64;   // output tile of the tall kernels (rows and columns)
constexpr int AK = 32;   // rows (Gram) or inner columns (apply) per shared-memory slab
constexpr int ATH = 256; // threads of the tall kernels
constexpr double kGapTol = 1e-13;  // relative squared-gap / pivot floor

// Column view of up to four column-major pieces (FP32 or BF16).
struct Pieces {
  const void* p[4];
  int64_t ld[4];
  int bf16[4];
  int start[5];  // piece q holds columns [start[q], start[q + 1])
  int np;
};

// (unrolled so that the kernel parameter is indexed with constants only)
__device__ __forceinline__ float piece_load(const Pieces& P, int c, int64_t r) {
  float v = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < P.np && c >= P.start[q] && c < P.start[q + 1]) {
      const int64_t off = r + (int64_t)(c - P.start[q]) * P.ld[q];
      v = P.bf16[q] ? __bfloat162float(static_cast<const __nv_bfloat16*>(P.p[q])[off])
                    : static_cast<const float*>(P.p[q])[off];
    }
  }
  return v;
}

// partial[z] (nl x nr, row-major) = L^T R over the rows of chunk z.
__global__ void __launch_bounds__(ATH) adj_gram_kernel(Pieces L, int nl, Pieces R, int nr,
                                                       int64_t M, int64_t rows_per_chunk,
                                                       double* partial) {
  __shared__ float Ls[AK][AT + 1];
  __shared__ float Rs[AK][AT + 1];
  const int i0 = blockIdx.x * AT, j0 = blockIdx.y * AT;
  const int64_t r0 = (int64_t)blockIdx.z * rows_per_chunk;
  const int64_t r1 = min(M, r0 + rows_per_chunk);
  const int t = threadIdx.x, tx = t % 16, ty = t / 16, lane = t % 32, warp = t / 32;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) hi[u][v] = lo[u][v] = 0.f;
  for (int64_t rb = r0; rb < r1; rb += AK) {
    const int64_t r = rb + lane;
    for (int c = warp; c < AT; c += ATH / 32) {
      const int cl = i0 + c, cr = j0 + c;
      Ls[lane][c] = (r < r1 && cl < nl) ? piece_load(L, cl, r) : 0.f;
      Rs[lane][c] = (r < r1 && cr < nr) ? piece_load(R, cr, r) : 0.f;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 8
    for (int k = 0; k < AK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Ls[k][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Rs[k][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    // fold the slab sum into the running float-float total (TwoSum)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float s = hi[u][v] + acc[u][v];
        const float bb = s - hi[u][v];
        lo[u][v] += (hi[u][v] - (s - bb)) + (acc[u][v] - bb);
        hi[u][v] = s;
      }
    __syncthreads();
  }
  double* out = partial + (size_t)blockIdx.z * nl * nr;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < nl && j < nr) out[(size_t)i * nr + j] = (double)hi[u][v] + (double)lo[u][v];
    }
}

// G (nl x nr, column-major) = sum over chunks in chunk order.
__global__ void adj_reduce_kernel(const double* partial, int nchunk, int nl, int nr, double* G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nl * nr) return;
  const int i = idx % nl, j = idx / nl;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += partial[(size_t)c * nl * nr + (size_t)i * nr + j];
  G[idx] = s;
}

__device__ __forceinline__ double panel_scale(int i, int kc, const double* D, double ff) {
  return i < kc ? ff * D[i] : 1.0;
}

// H = S G_PP S, V = S G_PY S_k^-1 (the kept right singular vectors), Cb = S G_PB.
__global__ void adj_scale_kernel(const double* G, int n, int k1, int kc, const double* D,
                                 double ff, const double* s, double* H, double* V, double* Cb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * (n + 2 * k1)) return;
  const int i = idx % n, j = idx / n;
  const double si = panel_scale(i, kc, D, ff);
  const double g = G[idx];
  if (j < n)
    H[i + (size_t)j * n] = si * g * panel_scale(j, kc, D, ff);
  else if (j < n + k1)
    V[i + (size_t)(j - n) * n] = si * g / s[j - n];
  else
    Cb[i + (size_t)(j - n - k1) * n] = si * g;
}

// C (m x nn, ldc) = alpha op(A) op(B) + beta C0 (C0 may be C; A and B must not alias C).
__global__ void adj_gemm_kernel(int ta, int tb, int m, int nn, int k, double alpha, const double* A,
                                int lda, const double* B, int ldb, double beta, const double* C0,
                                double* C, int ldc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nn) return;
  const int i = idx % m, j = idx / m;
  double acc = 0.0;
  for (int p = 0; p < k; ++p) {
    const double a = ta ? A[p + (size_t)i * lda] : A[i + (size_t)p * lda];
    const double b = tb ? B[j + (size_t)p * ldb] : B[p + (size_t)j * ldb];
    acc = fma(a, b, acc);
  }
  double v = alpha * acc;
  if (beta != 0.0) v += beta * C0[i + (size_t)j * ldc];
  C[i + (size_t)j * ldc] = v;
}

__device__ __forceinline__ int pk(int r, int c) { return r * (r + 1) / 2 + c; }  // r >= c

// X[:, j] = (s_j^2 I - Hp)^-1 Bp[:, j] for j = blockIdx.x: Cholesky of the packed
// lower triangle in shared memory, then the two triangular solves.  A pivot below
// kGapTol s_j^2 (the kept s_j meets a dropped singular value) sets info bit 2.
__global__ void adj_shift_solve_kernel(const double* Hp, const double* Bp, const double* s, int n,
                                       double* X, int* info) {
  extern __shared__ double sm[];
  double* Lp = sm;
  double* y = sm + n * (n + 1) / 2;
  const int j = blockIdx.x, t = threadIdx.x, bd = blockDim.x;
  const double sh = s[j] * s[j];
  for (int idx = t; idx < n * n; idx += bd) {
    const int r = idx % n, c = idx / n;
    if (c <= r) Lp[pk(r, c)] = (r == c ? sh : 0.0) - Hp[idx];
  }
  for (int r = t; r < n; r += bd) y[r] = Bp[r + (size_t)j * n];
  bool bad = false;
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    const double d = Lp[pk(k, k)];
    const bool small = !(d > kGapTol * sh);
    bad |= small;
    const double dd = sqrt(small ? kGapTol * sh : d);
    __syncthreads();
    if (t == 0) Lp[pk(k, k)] = dd;
    for (int i = k + 1 + t; i < n; i += bd) Lp[pk(i, k)] /= dd;
    __syncthreads();
    const int m = n - k - 1;
    const int cnt = m * (m + 1) / 2;
    for (int e = t; e < cnt; e += bd) {
      int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while (a * (a + 1) / 2 > e) --a;
      while ((a + 1) * (a + 2) / 2 <= e) ++a;
      const int b = e - a * (a + 1) / 2;
      const int r = k + 1 + a, c = k + 1 + b;
      Lp[pk(r, c)] -= Lp[pk(r, k)] * Lp[pk(c, k)];
    }
  }
  // L z = y
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    const double zk = y[k] / Lp[pk(k, k)];
    __syncthreads();
    if (t == 0) y[k] = zk;
    for (int i = k + 1 + t; i < n; i += bd) y[i] -= Lp[pk(i, k)] * zk;
  }
  // L^T x = z
  for (int k = n - 1; k >= 0; --k) {
    __syncthreads();
    const double xk = y[k] / Lp[pk(k, k)];
    __syncthreads();
    if (t == 0) y[k] = xk;
    for (int i = t; i < k; i += bd) y[i] -= Lp[pk(k, i)] * xk;
  }
  __syncthreads();
  for (int r = t; r < n; r += bd) X[r + (size_t)j * n] = y[r];
  if (bad && t == 0) atomicOr(info, 2);
}

// W (k1 x k1): the kept-kept block of S^-1 [diag(sbar) + (F o (X - X^T)) S - X S^-1] in the
// coordinates Z = V_k^T P^T Ybar (Y^T Ybar = S^-1 Z); Vs = V_k S_k^-1, Xs = Xc S_k^-1.
// Two kept singular values closer than kGapTol s_0^2 (squared) set info bit 1.
__global__ void adj_w_kernel(const double* Z, const double* s, const double* sbar, const double* V,
                             const double* Xc, int n, int k1, double* W, double* Vs, double* Xs,
                             int* info) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < k1 * k1) {
    const int i = idx % k1, j = idx / k1;
    const double si = s[i], sj = s[j];
    double w;
    if (i == j) {
      w = (sbar[i] - Z[idx] / (si * si)) / si;
    } else {
      const double d = sj * sj - si * si;
      if (!(fabs(d) > kGapTol * s[0] * s[0])) atomicOr(info, 1);
      const double F = 1.0 / d;
      w = (F * (Z[idx] * sj / si - Z[j + i * k1]) - Z[idx] / (si * sj)) / si;
    }
    if (!isfinite(w)) atomicOr(info, 4);
    W[idx] = w;
  }
  if (idx < n * k1) {
    const int j = idx / n;
    Vs[idx] = V[idx] / s[j];
    Xs[idx] = Xc[idx] / s[j];
  }
}

// Cf ((n + k1) x n, ld n + k1): rows r < n hold S N, rows n + j hold E = S_k^-1 V_k^T;
// output columns c < kc are scaled by ff D_c (Ubar = ff Pbar_U diag(D)).
__global__ void adj_coef_kernel(const double* N, const double* Vs, int n, int k1, int kc,
                                const double* D, double ff, float* Cf, int* info) {
  const int kin = n + k1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kin * n) return;
  const int r = idx % kin, c = idx / kin;
  double v = r < n ? panel_scale(r, kc, D, ff) * N[r + (size_t)c * n] : Vs[c + (size_t)(r - n) * n];
  if (c < kc) v *= ff * D[c];
  if (!isfinite(v)) atomicOr(info, 4);
  Cf[idx] = (float)v;
}

// Dbar_c = ff (sum_r G[c, r] (S N)[r, c] + sum_j G[c, n + k1 + j] E[j, c]), one warp per c < kc.
__global__ void adj_dbar_kernel(const double* G, const double* N, const double* Vs, int n, int k1,
                                int kc, const double* D, double ff, double* Dbar) {
  const int c = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (c >= kc) return;
  double acc = 0.0;
  for (int r = lane; r < n; r += 32)
    acc += G[c + (size_t)r * n] * panel_scale(r, kc, D, ff) * N[r + (size_t)c * n];
  for (int j = lane; j < k1; j += 32)
    acc += G[c + (size_t)(n + k1 + j) * n] * Vs[c + (size_t)j * n];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) Dbar[c] = ff * acc;
}

// [Ubar | Abar] (M x n) = [U | A | Ybar] (M x (n + k1)) Cf, FP32.
__global__ void __launch_bounds__(ATH) adj_apply_kernel(Pieces In, int kin, const float* Cf,
                                                        int nout, int64_t M, int kc, float* Ubar,
                                                        int64_t ldub, float* Abar, int64_t ldab) {
  __shared__ float Is[AK][AT + 1];
  __shared__ float Cs[AK][AT + 1];
  const int64_t m0 = (int64_t)blockIdx.x * AT;
  const int c0 = blockIdx.y * AT;
  const int t = threadIdx.x, tr = t % 16, tc = t / 16, lane = t % 32, warp = t / 32;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  for (int kb = 0; kb < kin; kb += AK) {
    for (int kk = warp; kk < AK; kk += ATH / 32) {
      const int k = kb + kk;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t r = m0 + lane + 32 * h;
        Is[kk][lane + 32 * h] = (k < kin && r < M) ? piece_load(In, k, r) : 0.f;
      }
    }
    for (int e = t; e < AK * AT; e += ATH) {
      const int kk = e % AK, c = e / AK;
      Cs[kk][c] = (kb + kk < kin && c0 + c < nout) ? Cf[(kb + kk) + (size_t)(c0 + c) * kin] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < AK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Is[k][tr + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Cs[k][tc + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t m = m0 + tr + 16 * u;
    if (m >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = c0 + tc + 16 * v;
      if (c >= nout) continue;
      if (c < kc)
        Ubar[m + (int64_t)c * ldub] = acc[u][v];
      else
        Abar[m + (int64_t)(c - kc) * ldab] = acc[u][v];
    }
  }
}

cudaError_t gemm(cudaStream_t st, int ta, int tb, int m, int nn, int k, double alpha,
                 const double* A, int lda, const double* B, int ldb, double beta, const double* C0,
                 double* C, int ldc) {
  const int tot = m * nn;
  if (tot == 0) return cudaSuccess;
  adj_gemm_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(ta, tb, m, nn, k, alpha, A, lda, B,
                                                                ldb, beta, C0, C, ldc);
  return cudaGetLastError();
}

}  // namespace

struct AdjWork {
  double* arena = nullptr;
  size_t arena_cap = 0;
  double* partial = nullptr;
  size_t partial_cap = 0;
  float* Cf = nullptr;
  size_t cf_cap = 0;
  int* info = nullptr;
  ~AdjWork() {
    cudaFree(arena);
    cudaFree(partial);
    cudaFree(Cf);
    cudaFree(info);
  }
};

AdjWork* adj_work_create() { return new (std::nothrow) AdjWork(); }
void adj_work_destroy(AdjWork* w) { delete w; }

size_t adjoint_shift_solve_smem(int n) { return sizeof(double) * ((size_t)n * (n + 1) / 2 + n); }

namespace {
template <typename T>
bool grow(T** p, size_t* cap, size_t need) {
  if (need <= *cap) return true;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc((void**)p, sizeof(T) * need) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  *cap = need;
  return true;
}
}  // namespace

int adjoint_run(AdjWork* aw, cudaStream_t st, int num_sms, int64_t M, double ff, int kc,
                const float* U, int64_t ldu, const double* D, const void* A, int64_t lda,
                int a_bf16, int B, int k1, const float* Unew, int64_t ldun, const double* Dnew,
                const float* Ybar, int64_t ldyb, const double* sbar, float* Ubar, int64_t ldub,
                double* Dbar, float* Abar, int64_t ldab, int* status) {
#define ACK(x)                  \
  do {                          \
    if ((x) != cudaSuccess) {   \
      cudaGetLastError();       \
      return PSVD_ERR_CUDA;     \
    }                           \
  } while (0)
  const int n = kc + B;
  const int w = n + 2 * k1;
  const int kin = n + k1;
  // row chunks of the Gram pass: a few CTAs per SM over the output tiles
  const int tiles = (int)(ceil_div(n, AT) * ceil_div(w, AT));
  int64_t nchunk = ceil_div(4LL * num_sms, tiles);
  nchunk = std::max<int64_t>(1, std::min<int64_t>(nchunk, ceil_div(M, 256)));
  const int64_t rpc = ceil_div(ceil_div(M, nchunk), AK) * AK;
  nchunk = ceil_div(M, rpc);
  // the buffers may still be in use by an earlier call on this stream
  ACK(cudaStreamSynchronize(st));
  const size_t nn = (size_t)n * n, nk = (size_t)n * k1, kk = (size_t)k1 * k1;
  const size_t need = (size_t)n * w + 3 * nn + 9 * nk + 3 * kk + 2 * (size_t)kc + 2 * (size_t)k1;
  if (!grow(&aw->arena, &aw->arena_cap, need) ||
      !grow(&aw->partial, &aw->partial_cap, (size_t)nchunk * n * w) ||
      !grow(&aw->Cf, &aw->cf_cap, (size_t)kin * n))
    return PSVD_ERR_ALLOC;
  if (!aw->info && cudaMalloc((void**)&aw->info, sizeof(int) * 4) != cudaSuccess) {
    cudaGetLastError();
    aw->info = nullptr;
    return PSVD_ERR_ALLOC;
  }
  double* p = aw->arena;
  auto take = [&p](size_t count) {
    double* q = p;
    p += count;
    return q;
  };
  double* G = take((size_t)n * w);
  double* H = take(nn);
  double* Hp = take(nn);
  double* N = take(nn);
  double* V = take(nk);
  double* Cb = take(nk);
  double* Bp = take(nk);
  double* HV = take(nk);
  double* Qm = take(nk);
  double* Xc = take(nk);
  double* Vs = take(nk);
  double* Xs = take(nk);
  double* T1 = take(nk);
  double* Z = take(kk);
  double* Mk = take(kk);
  double* W = take(kk);
  double* Dd = take(kc);
  double* Dbd = take(kc);
  double* sd = take(k1);
  double* sbd = take(k1);
  int* info = aw->info;
  ACK(cudaMemsetAsync(info, 0, sizeof(int) * 4, st));
  if (kc > 0) ACK(cudaMemcpyAsync(Dd, D, sizeof(double) * kc, cudaMemcpyDefault, st));
  ACK(cudaMemcpyAsync(sd, Dnew, sizeof(double) * k1, cudaMemcpyDefault, st));
  ACK(cudaMemcpyAsync(sbd, sbar, sizeof(double) * k1, cudaMemcpyDefault, st));

  // pass 1: G = [U | A]^T [U | A | U' | Ybar]
  Pieces R{};
  auto add = [](Pieces& P, const void* ptr, int64_t ld, int bf, int cols) {
    if (cols <= 0) return;
    P.p[P.np] = ptr;
    P.ld[P.np] = ld;
    P.bf16[P.np] = bf;
    P.start[P.np + 1] = P.start[P.np] + cols;
    ++P.np;
  };
  add(R, U, ldu, 0, kc);
  add(R, A, lda, a_bf16, B);
  Pieces L = R;  // the panel's own columns
  add(R, Unew, ldun, 0, k1);
  add(R, Ybar, ldyb, 0, k1);
  dim3 gg((unsigned)ceil_div(n, AT), (unsigned)ceil_div(w, AT), (unsigned)nchunk);
  adj_gram_kernel<<<gg, ATH, 0, st>>>(L, n, R, w, M, rpc, aw->partial);
  ACK(cudaGetLastError());
  adj_reduce_kernel<<<(unsigned)ceil_div((int64_t)n * w, 256), 256, 0, st>>>(aw->partial,
                                                                             (int)nchunk, n, w, G);
  ACK(cudaGetLastError());
  // small side (FP64)
  adj_scale_kernel<<<(unsigned)ceil_div((int64_t)n * w, 256), 256, 0, st>>>(G, n, k1, kc, Dd, ff,
                                                                            sd, H, V, Cb);
  ACK(cudaGetLastError());
  ACK(gemm(st, 1, 0, k1, k1, n, 1.0, V, n, Cb, n, 0.0, nullptr, Z, k1));      // Z = V^T Cb
  ACK(gemm(st, 0, 0, n, k1, k1, -1.0, V, n, Z, k1, 1.0, Cb, Bp, n));          // Bp = Pi Cb
  ACK(gemm(st, 0, 0, n, k1, n, 1.0, H, n, V, n, 0.0, nullptr, HV, n));        // HV = H V
  ACK(gemm(st, 1, 0, k1, k1, n, 1.0, V, n, HV, n, 0.0, nullptr, Mk, k1));     // Mk = V^T H V
  ACK(gemm(st, 0, 0, n, k1, k1, 1.0, V, n, Mk, k1, 0.0, nullptr, Qm, n));     // Qm = V Mk
  ACK(gemm(st, 0, 1, n, n, k1, -1.0, HV, n, V, n, 1.0, H, Hp, n));           // Hp = Pi H Pi
  ACK(gemm(st, 0, 1, n, n, k1, -1.0, V, n, HV, n, 1.0, Hp, Hp, n));
  ACK(gemm(st, 0, 1, n, n, k1, 1.0, Qm, n, V, n, 1.0, Hp, Hp, n));
  const size_t smem = adjoint_shift_solve_smem(n);
  ACK(cudaFuncSetAttribute(adj_shift_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem));
  adj_shift_solve_kernel<<<k1, 256, smem, st>>>(Hp, Bp, sd, n, Xc, info);
  ACK(cudaGetLastError());
  adj_w_kernel<<<(unsigned)ceil_div((int64_t)std::max(kk, nk), 256), 256, 0, st>>>(Z, sd, sbd, V, Xc, n, k1,
                                                                          W, Vs, Xs, info);
  ACK(cudaGetLastError());
  ACK(gemm(st, 0, 0, n, k1, k1, 1.0, V, n, W, k1, 1.0, Xs, T1, n));   // T1 = V W + Xs
  ACK(gemm(st, 0, 1, n, n, k1, 1.0, T1, n, V, n, 0.0, nullptr, N, n));  // N = T1 V^T
  ACK(gemm(st, 0, 1, n, n, k1, 1.0, V, n, Xs, n, 1.0, N, N, n));       //   + V Xs^T
  adj_coef_kernel<<<(unsigned)ceil_div((int64_t)kin * n, 256), 256, 0, st>>>(N, Vs, n, k1, kc, Dd,
                                                                             ff, aw->Cf, info);
  ACK(cudaGetLastError());
  if (kc > 0) {
    adj_dbar_kernel<<<(unsigned)ceil_div(kc, 8), 256, 0, st>>>(G, N, Vs, n, k1, kc, Dd, ff, Dbd);
    ACK(cudaGetLastError());
  }
  // pass 2: [Ubar | Abar] = [U | A | Ybar] Cf
  Pieces In{};
  add(In, U, ldu, 0, kc);
  add(In, A, lda, a_bf16, B);
  add(In, Ybar, ldyb, 0, k1);
  dim3 ga((unsigned)ceil_div(M, AT), (unsigned)ceil_div(n, AT));
  adj_apply_kernel<<<ga, ATH, 0, st>>>(In, kin, aw->Cf, n, M, kc, Ubar, ldub, Abar, ldab);
  ACK(cudaGetLastError());
  if (kc > 0) ACK(cudaMemcpyAsync(Dbar, Dbd, sizeof(double) * kc, cudaMemcpyDefault, st));
  int hinfo[4] = {0, 0, 0, 0};
  ACK(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, st));
  ACK(cudaStreamSynchronize(st));
#undef ACK
  *status = hinfo[0];
  return PSVD_OK;
}

}  // namespace psvd
