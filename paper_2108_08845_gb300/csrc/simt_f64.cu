// FP64 panel kernels of the per-batch update of Algorithm 1 (Sec. 3.1), for
// handles created with PSVD_PREC_FP64: modes stored in FP64, snapshots of any
// input type widened exactly.
//   * gram_f64_partial_kernel: the Gram [U|A]^T [U|A] of the (never materialised)
//     panel over row chunks (step 1's R^T R), FP64 FMAs.  Same tiling and partial
//     layout as the FP32 kernel, so gram_reduce_launch sums the chunks in the same
//     fixed order.
//   * update_f64_kernel: step 4, U <- [U | A] T with the FP64 T of the small solve.
// FP64 runs at a small fraction of the FP32 rate on this GPU: this path is the
// full-precision reference on the device, not the fast one.
#include "psvd_internal.cuh"

namespace psvd {
namespace {

constexpr int GB = 64;        // column block of the Gram tile
constexpr int GRS = 32;       // rows per shared-memory stage (the FP32 kernel's chunking)
constexpr int GLD = GRS + 1;  // padded stage leading dimension
constexpr int GTHREADS = 256;

__device__ __forceinline__ double panel_at(const PanelF64& p, int col, int64_t row) {
  if (col < p.kc) return p.U[row + (int64_t)col * p.ldu];
  const int64_t off = row + (int64_t)(col - p.kc) * p.lda;
  switch (p.a_dtype) {
    case PSVD_BF16: return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p.A)[off]);
    case PSVD_F64: return reinterpret_cast<const double*>(p.A)[off];
    default: return (double)reinterpret_cast<const float*>(p.A)[off];
  }
}

__device__ __forceinline__ void decode_pair(int pair, int nb, int* bi, int* bj) {
  int i = 0;
  while (pair >= nb - i) {
    pair -= nb - i;
    ++i;
  }
  *bi = i;
  *bj = i + pair;
}

// Block pair (bi, bj) of 64-column blocks over rows [chunk * rows_per_chunk, ...):
// thread (tx, ty) accumulates rows 16 k + ty x columns 16 l + tx of the tile.
__global__ void __launch_bounds__(GTHREADS) gram_f64_partial_kernel(PanelF64 p, int nb,
                                                                    int64_t rows_per_chunk,
                                                                    double* __restrict__ partial) {
  __shared__ double Xi[GB * GLD];
  __shared__ double Xj[GB * GLD];
  int bi, bj;
  decode_pair(blockIdx.x, nb, &bi, &bj);
  const bool diag = (bi == bj);
  const int npairs = gridDim.x;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r_end = min(p.M, r_begin + rows_per_chunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
  double acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[k][l] = 0.0;
  const double* Yj = diag ? Xi : Xj;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += GRS) {
    __syncthreads();
    const int64_t row = r0 + lane;
    const bool row_ok = row < r_end;
    for (int c = warp; c < GB; c += GTHREADS / 32) {
      const int ci = bi * GB + c;
      Xi[c * GLD + lane] = (row_ok && ci < p.n) ? panel_at(p, ci, row) : 0.0;
      if (!diag) {
        const int cj = bj * GB + c;
        Xj[c * GLD + lane] = (row_ok && cj < p.n) ? panel_at(p, cj, row) : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < GRS; ++r) {
      double a[4], b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = Xi[(ty + 16 * k) * GLD + r];
#pragma unroll
      for (int l = 0; l < 4; ++l) b[l] = Yj[(tx + 16 * l) * GLD + r];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l) acc[k][l] = fma(a[k], b[l], acc[k][l]);
    }
  }
  double* out = partial + ((size_t)blockIdx.y * npairs + blockIdx.x) * (GB * GB);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) out[(ty + 16 * k) + GB * (tx + 16 * l)] = acc[k][l];
}

constexpr int UR = 64;  // rows per update tile
constexpr int UC = 64;  // output columns per update tile
constexpr int UK = 32;  // panel columns per stage

// Unew[r0 .. r0+63, j0 .. j0+63] = P T: thread (warp w, lane l) owns rows l, l + 32
// and columns 8 w .. 8 w + 7 of the tile.
__global__ void __launch_bounds__(256) update_f64_kernel(PanelF64 p, const double* __restrict__ T,
                                                         int k1, double* __restrict__ Unew,
                                                         int64_t ldo) {
  __shared__ double Ps[UK * UR];
  __shared__ double Ts[UK * UC];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * UR;
  const int j0 = blockIdx.y * UC;
  double acc[2][8];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
  for (int c0 = 0; c0 < p.n; c0 += UK) {
    __syncthreads();
    for (int e = tid; e < UK * UR; e += 256) {
      const int c = e / UR, r = e % UR;
      const int64_t row = r0 + r;
      Ps[e] = (row < p.M && c0 + c < p.n) ? panel_at(p, c0 + c, row) : 0.0;
    }
    for (int e = tid; e < UK * UC; e += 256) {
      const int c = e / UC, j = e % UC;
      Ts[e] = (c0 + c < p.n && j0 + j < k1) ? T[(c0 + c) + (int64_t)(j0 + j) * p.n] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < UK; ++c) {
      double pv[2], tv[8];
#pragma unroll
      for (int i = 0; i < 2; ++i) pv[i] = Ps[c * UR + lane + 32 * i];
#pragma unroll
      for (int j = 0; j < 8; ++j) tv[j] = Ts[c * UC + 8 * warp + j];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(pv[i], tv[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int64_t row = r0 + lane + 32 * i;
    if (row >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = j0 + 8 * warp + j;
      if (col < k1) Unew[row + (int64_t)col * ldo] = acc[i][j];
    }
  }
}

__global__ void modes_f64_to_f32_kernel(const double* __restrict__ U, int64_t ldu, int64_t M, int k,
                                        float* __restrict__ out, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * k) return;
  const int64_t r = e % M, c = e / M;
  out[r + c * ldo] = (float)U[r + c * ldu];
}

}  // namespace

cudaError_t gram_f64_launch(const PanelF64& p, int nchunk, int64_t rows_per_chunk, double* partial,
                            cudaStream_t st) {
  const int nb = (int)ceil_div(p.n, GB);
  dim3 grid(nb * (nb + 1) / 2, nchunk);
  gram_f64_partial_kernel<<<grid, GTHREADS, 0, st>>>(p, nb, rows_per_chunk, partial);
  return cudaGetLastError();
}

cudaError_t update_f64_launch(const PanelF64& p, const double* T, int k1, double* Unew, int64_t ldo,
                              cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(p.M, UR), (unsigned)ceil_div(k1, UC));
  update_f64_kernel<<<grid, 256, 0, st>>>(p, T, k1, Unew, ldo);
  return cudaGetLastError();
}

cudaError_t modes_f64_to_f32_launch(const double* U, int64_t ldu, int64_t M, int k, float* out,
                                    int64_t ldo, cudaStream_t st) {
  const int64_t tot = M * k;
  if (tot == 0) return cudaSuccess;
  modes_f64_to_f32_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(U, ldu, M, k, out, ldo);
  return cudaGetLastError();
}

}  // namespace psvd
