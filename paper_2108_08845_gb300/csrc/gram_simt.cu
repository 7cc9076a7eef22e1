// FP32 CUDA-core ("plain FP32") panel kernels of the per-batch update of
// Algorithm 1 (Sec. 3.1):
//   * gram_partial_kernel: the Gram [U|A]^T [U|A] of the (never materialised)
//     panel over row chunks.  This is step 1's QR expressed through its R^T R:
//     R^T R = P^T P with P = [ff U D | A] = [U | A] diag(ff D, 1).
//   * gram_reduce_kernel: fixed-order FP64 reduction of the chunk partials and
//     the diag(ff D, 1) scaling on the small side.
//   * update_kernel: step 4, U <- Q U~ = [U | A] T with T = S V~ D~^-1.
// Column-major row tiles are staged through shared memory; FP32 FMAs run in
// short chains (fold_rows rows, 4 to 32) that are folded into float-float
// accumulators with Knuth's TwoSum, so the only rounding left in a chunk partial
// is that of the short chains.  A Gram-based factorisation amplifies the Gram's
// relative error by (sigma_1/sigma_i)^2, so the chains shrink as M shrinks
// (relative error ~ u * fold_rows / sqrt(M), kept near 1e-9).
#include <math.h>

#include <vector>

#include "psvd_internal.cuh"

namespace psvd {
namespace {

constexpr int GB = 64;         // column block of the Gram tile
constexpr int GRS = 32;        // rows per shared-memory stage
constexpr int GLD = GRS + 4;   // padded stage leading dimension (16-byte rows, no conflicts)
constexpr int GTHREADS = 256;

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ float panel_at(const PanelF32& p, int col, int64_t row) {
  if (col < p.kc) return p.U[row + (int64_t)col * p.ldu];
  const int64_t off = row + (int64_t)(col - p.kc) * p.lda;
  return p.a_bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p.A)[off])
                  : reinterpret_cast<const float*>(p.A)[off];
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

// Row chunk blockIdx.y: rows [blockIdx.y * rows_per_chunk, ...) of the panel, or,
// with a work list, rows [items[y].r0, items[y].r1) with that item's chain length
// (the row blocks of Algorithm 2 in one launch).
__global__ void __launch_bounds__(GTHREADS) gram_partial_kernel(PanelF32 p, int nb,
                                                                int64_t rows_per_chunk,
                                                                int fold_steps,
                                                                const GramItem* __restrict__ items,
                                                                double* __restrict__ partial) {
  __shared__ __align__(16) float Xi[GB * GLD];
  __shared__ __align__(16) float Xj[GB * GLD];
  int bi, bj;
  decode_pair(blockIdx.x, nb, &bi, &bj);
  const bool diag = (bi == bj);
  const int npairs = gridDim.x;
  int64_t r_begin = (int64_t)blockIdx.y * rows_per_chunk;
  int64_t r_end = min(p.M, r_begin + rows_per_chunk);
  if (items) {
    const GramItem it = items[blockIdx.y];
    r_begin = it.r0;
    r_end = it.r1;
    fold_steps = it.fold_steps;
  }
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;

  float acc[4][4], hi[4][4], lo[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[k][l] = hi[k][l] = lo[k][l] = 0.f;

  int since = 0;  // 4-row steps since the last fold
  const float* Yj = diag ? Xi : Xj;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += GRS) {
    __syncthreads();
    const int64_t row = r0 + lane;
    const bool row_ok = row < r_end;
    for (int c = warp; c < GB; c += GTHREADS / 32) {
      const int ci = bi * GB + c;
      Xi[c * GLD + lane] = (row_ok && ci < p.n) ? panel_at(p, ci, row) : 0.f;
      if (!diag) {
        const int cj = bj * GB + c;
        Xj[c * GLD + lane] = (row_ok && cj < p.n) ? panel_at(p, cj, row) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < GRS; r += 4) {
      float4 a[4], b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = *reinterpret_cast<const float4*>(&Xi[(ty + 16 * k) * GLD + r]);
#pragma unroll
      for (int l = 0; l < 4; ++l) b[l] = *reinterpret_cast<const float4*>(&Yj[(tx + 16 * l) * GLD + r]);
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          float s = acc[k][l];
          s = fmaf(a[k].x, b[l].x, s);
          s = fmaf(a[k].y, b[l].y, s);
          s = fmaf(a[k].z, b[l].z, s);
          s = fmaf(a[k].w, b[l].w, s);
          acc[k][l] = s;
        }
      if (++since == fold_steps) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            two_sum_acc(hi[k][l], lo[k][l], acc[k][l]);
            acc[k][l] = 0.f;
          }
        since = 0;
      }
    }
  }
  double* out = partial + ((size_t)blockIdx.y * npairs + blockIdx.x) * (GB * GB);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      two_sum_acc(hi[k][l], lo[k][l], acc[k][l]);
      out[(ty + 16 * k) + GB * (tx + 16 * l)] = (double)hi[k][l] + (double)lo[k][l];
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nchunk, int nb, int n,
                                   int kc, const double* __restrict__ D, double ff,
                                   double* __restrict__ G, double* __restrict__ H,
                                   int* __restrict__ info) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  int i = (int)(e % n), j = (int)(e / n);
  int bi = i / GB, bj = j / GB, il = i % GB, jl = j % GB;
  // read the stored orientation: block row <= block column, and in diagonal
  // blocks the entry with il <= jl, so H is exactly symmetric
  if (bi > bj || (bi == bj && il > jl)) {
    int t = bi; bi = bj; bj = t;
    t = il; il = jl; jl = t;
  }
  const int npairs = nb * (nb + 1) / 2;
  const int pair = bi * nb - bi * (bi - 1) / 2 + (bj - bi);
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += partial[((size_t)c * npairs + pair) * (GB * GB) + il + GB * jl];
  if (G) G[e] = s;
  const double si = (i < kc) ? ff * D[i] : 1.0;
  const double sj = (j < kc) ? ff * D[j] : 1.0;
  H[e] = si * sj * s;
  if (!isfinite(s)) atomicOr(&info[2], 4);
}

constexpr int UK = 32;   // panel columns per stage

// Tile of UR = 32 RI rows x UC = 8 NW columns, NW warps; each thread holds RI rows x 8
// columns.  Every output element sums the panel columns in the same order whatever
// the tile, so all tile shapes give the same bits.
template <int RI, int NW>
__global__ void __launch_bounds__(32 * NW) update_kernel(PanelF32 p, const float* __restrict__ T,
                                                         int k1, float* __restrict__ Unew,
                                                         int64_t ldo) {
  constexpr int UR = 32 * RI;
  constexpr int UC = 8 * NW;
  constexpr int NT = 32 * NW;
  __shared__ __align__(16) float Ps[UK * UR];
  __shared__ __align__(16) float Ts[UK * UC];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * UR;
  const int j0 = blockIdx.y * UC;
  float acc[RI][8];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  for (int c0 = 0; c0 < p.n; c0 += UK) {
    __syncthreads();
    for (int e = tid; e < UK * UR; e += NT) {
      const int c = e / UR, r = e % UR;
      const int64_t row = r0 + r;
      Ps[e] = (row < p.M && c0 + c < p.n) ? panel_at(p, c0 + c, row) : 0.f;
    }
    for (int e = tid; e < UK * UC; e += NT) {
      const int c = e / UC, j = e % UC;
      Ts[e] = (c0 + c < p.n && j0 + j < k1) ? T[(c0 + c) + (int64_t)(j0 + j) * p.n] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < UK; ++c) {
      float pv[RI];
#pragma unroll
      for (int i = 0; i < RI; ++i) pv[i] = Ps[c * UR + lane + 32 * i];
      const float4 t0 = *reinterpret_cast<const float4*>(&Ts[c * UC + 8 * warp]);
      const float4 t1 = *reinterpret_cast<const float4*>(&Ts[c * UC + 8 * warp + 4]);
      const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(pv[i], tv[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const int64_t row = r0 + lane + 32 * i;
    if (row >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = j0 + 8 * warp + j;
      if (col < k1) Unew[row + (int64_t)col * ldo] = acc[i][j];
    }
  }
}

__global__ void copy_modes_kernel(const float* __restrict__ U, int64_t ldu, int64_t M, int k,
                                  float* __restrict__ out, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * k) return;
  const int64_t r = e % M, c = e / M;
  out[r + c * ldo] = U[r + c * ldu];
}

}  // namespace

void gram_simt_plan(int64_t M, int n, int num_sms, int* nchunk, int64_t* rows_per_chunk,
                    int64_t* partial_doubles, int ctas_per_sm) {
  const int nb = (int)ceil_div(n, GB);
  const int npairs = nb * (nb + 1) / 2;
  // about ctas_per_sm CTAs per SM in total, chunks a multiple of the stage height
  int64_t want = (int64_t)num_sms * (ctas_per_sm > 0 ? ctas_per_sm : 4) / npairs;
  if (want < 1) want = 1;
  int64_t rpc = ceil_div(ceil_div(M, want), GRS) * GRS;
  if (rpc < GRS) rpc = GRS;
  *rows_per_chunk = rpc;
  *nchunk = (int)ceil_div(M, rpc);
  *partial_doubles = (int64_t)(*nchunk) * npairs * GB * GB;
}

// Rows per FP32 chain: about 0.029 sqrt(M) (relative Gram error ~1e-9), in {4, 8, 16, 32}.
int gram_simt_fold_steps(int64_t M) {
  const double rows = 0.029 * sqrt((double)M);
  int steps = 1;
  while (steps < 8 && 4.0 * (2 * steps) <= rows) steps *= 2;
  return steps;
}

cudaError_t gram_simt_launch(const PanelF32& p, int nchunk, int64_t rows_per_chunk,
                             double* partial, cudaStream_t st) {
  const int nb = (int)ceil_div(p.n, GB);
  dim3 grid(nb * (nb + 1) / 2, nchunk);
  gram_partial_kernel<<<grid, GTHREADS, 0, st>>>(p, nb, rows_per_chunk,
                                                 gram_simt_fold_steps(p.M), nullptr, partial);
  return cudaGetLastError();
}

void gram_items_plan(const int64_t* off, int nparts, int n, int num_sms, std::vector<GramItem>* items,
                     std::vector<int>* first, int64_t* partial_doubles) {
  const int nb = (int)ceil_div(n, GB);
  const int npairs = nb * (nb + 1) / 2;
  const int64_t total = off[nparts] - off[0];
  // about 4 CTAs per SM over all blocks, chunks a multiple of the stage height
  int64_t want = (int64_t)num_sms * 4 / npairs;
  if (want < 1) want = 1;
  int64_t rpc = ceil_div(ceil_div(total, want), GRS) * GRS;
  if (rpc < GRS) rpc = GRS;
  items->clear();
  first->assign(nparts + 1, 0);
  for (int b = 0; b < nparts; ++b) {
    (*first)[b] = (int)items->size();
    const int64_t mb = off[b + 1] - off[b];
    const int fs = gram_simt_fold_steps(mb);  // the chain length of a lone Gram of this block
    for (int64_t r = off[b]; r < off[b + 1]; r += rpc)
      items->push_back(GramItem{r, r + rpc < off[b + 1] ? r + rpc : off[b + 1], fs});
  }
  (*first)[nparts] = (int)items->size();
  *partial_doubles = (int64_t)items->size() * npairs * GB * GB;
}

cudaError_t gram_items_launch(const PanelF32& p, const GramItem* items, int nitems, double* partial,
                              cudaStream_t st) {
  const int nb = (int)ceil_div(p.n, GB);
  dim3 grid(nb * (nb + 1) / 2, nitems);
  gram_partial_kernel<<<grid, GTHREADS, 0, st>>>(p, nb, 0, 1, items, partial);
  return cudaGetLastError();
}

// H_z = sum of the partials of items [first[z], first[z+1]) (fixed order), z < count;
// H_z at H + z * sH (n x n), info_z at info + 4 z.
__global__ void gram_reduce_items_kernel(const double* __restrict__ partial,
                                         const int* __restrict__ first, int nb, int n,
                                         double* __restrict__ H, int64_t sH, int* __restrict__ info) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int z = blockIdx.y;
  if (e >= (int64_t)n * n) return;
  int i = (int)(e % n), j = (int)(e / n);
  int bi = i / GB, bj = j / GB, il = i % GB, jl = j % GB;
  if (bi > bj || (bi == bj && il > jl)) {
    int t = bi; bi = bj; bj = t;
    t = il; il = jl; jl = t;
  }
  const int npairs = nb * (nb + 1) / 2;
  const int pair = bi * nb - bi * (bi - 1) / 2 + (bj - bi);
  double s = 0.0;
  for (int c = first[z]; c < first[z + 1]; ++c)
    s += partial[((size_t)c * npairs + pair) * (GB * GB) + il + GB * jl];
  H[z * sH + e] = s;
  if (!isfinite(s)) atomicOr(&info[4 * z + 2], 4);
}

cudaError_t gram_reduce_items_launch(const double* partial, const int* first, int count, int n,
                                     double* H, int64_t sH, int* info, cudaStream_t st) {
  const int nb = (int)ceil_div(n, GB);
  const int64_t tot = (int64_t)n * n;
  gram_reduce_items_kernel<<<dim3((unsigned)ceil_div(tot, 256), (unsigned)count), 256, 0, st>>>(
      partial, first, nb, n, H, sH, info);
  return cudaGetLastError();
}

cudaError_t gram_reduce_launch(const double* partial, int nchunk, int n, int kc, const double* D,
                               double ff, double* G, double* H, int* info, cudaStream_t st) {
  const int nb = (int)ceil_div(n, GB);
  const int64_t tot = (int64_t)n * n;
  gram_reduce_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(partial, nchunk, nb, n, kc, D,
                                                                    ff, G, H, info);
  return cudaGetLastError();
}

namespace {
template <int RI, int NW>
void launch_update(const PanelF32& p, const float* T, int k1, float* Unew, int64_t ldo,
                   cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(p.M, 32 * RI), (unsigned)ceil_div(k1, 8 * NW));
  update_kernel<RI, NW><<<grid, 32 * NW, 0, st>>>(p, T, k1, Unew, ldo);
}
template <int RI>
void launch_update_cols(const PanelF32& p, const float* T, int k1, float* Unew, int64_t ldo,
                        cudaStream_t st) {
  // the narrowest tile of 16, 32 or 64 columns that covers k1 (or 64-column tiles)
  if (k1 <= 16)
    launch_update<RI, 2>(p, T, k1, Unew, ldo, st);
  else if (k1 <= 32)
    launch_update<RI, 4>(p, T, k1, Unew, ldo, st);
  else
    launch_update<RI, 8>(p, T, k1, Unew, ldo, st);
}
}  // namespace

cudaError_t update_simt_launch(const PanelF32& p, const float* T, int k1, float* Unew, int64_t ldo,
                               cudaStream_t st, int tile_rows) {
  if (tile_rows == 64)
    launch_update_cols<2>(p, T, k1, Unew, ldo, st);
  else
    launch_update_cols<4>(p, T, k1, Unew, ldo, st);
  return cudaGetLastError();
}

cudaError_t copy_modes_f32_launch(const float* U, int64_t ldu, int64_t M, int k, float* out,
                                  int64_t ldo, cudaStream_t st) {
  const int64_t tot = M * k;
  if (tot == 0) return cudaSuccess;
  copy_modes_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(U, ldu, M, k, out, ldo);
  return cudaGetLastError();
}

}  // namespace psvd
