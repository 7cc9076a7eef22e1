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

// Row stages are copied into shared memory with cp.async (no registers tied up while
// the copies fly).  Thread (warp w, lane l) copies rows r0 + 2 (l % 16) and the next
// of the columns c = 2 (w + 8 q) + l / 16, q < 4: FP32 columns element by element
// into the FP32 stage, BF16 columns as one 4-byte pair into a BF16 staging area that
// the same thread widens into the FP32 stage once its copies have landed.  Rows
// beyond the chunk and columns beyond n are zero-filled.
constexpr int SLD = GRS / 2 + 1;  // staging words per column (pairs of BF16 rows)

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gsrc), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Issues the copies of the stage rows [r0, r0 + GRS) of slab `blk` (64 columns) into
// X (FP32, column stride GLD) and stg (BF16 pairs, column stride SLD).
__device__ __forceinline__ void issue_slab(const PanelF32& p, int blk, int64_t r0, int64_t r_end,
                                           float* X, uint32_t* stg, int lane, int warp,
                                           bool pairs) {
  const int k = lane & 15, half = lane >> 4;
  const int64_t row = r0 + 2 * k;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = 2 * (warp + 8 * q) + half;
    const int col = blk * GB + c;
    float* xd = X + c * GLD + 2 * k;
    if (col >= p.n) {
      xd[0] = 0.f;
      xd[1] = 0.f;
    } else if (col < p.kc) {
      const float* src = p.U + (int64_t)col * p.ldu;
      cp_async4(xd, src + (row < r_end ? row : 0), row < r_end ? 4 : 0);
      cp_async4(xd + 1, src + (row + 1 < r_end ? row + 1 : 0), row + 1 < r_end ? 4 : 0);
    } else if (!p.a_bf16) {
      const float* src = reinterpret_cast<const float*>(p.A) + (int64_t)(col - p.kc) * p.lda;
      cp_async4(xd, src + (row < r_end ? row : 0), row < r_end ? 4 : 0);
      cp_async4(xd + 1, src + (row + 1 < r_end ? row + 1 : 0), row + 1 < r_end ? 4 : 0);
    } else if (pairs) {
      const __nv_bfloat16* src =
          reinterpret_cast<const __nv_bfloat16*>(p.A) + (int64_t)(col - p.kc) * p.lda;
      const int bytes = row + 1 < r_end ? 4 : row < r_end ? 2 : 0;
      cp_async4(stg + c * SLD + k, src + (bytes ? row : 0), bytes);
    } else {
      // a pair not 4-byte aligned: two plain loads
      const __nv_bfloat16* src =
          reinterpret_cast<const __nv_bfloat16*>(p.A) + (int64_t)(col - p.kc) * p.lda;
      xd[0] = row < r_end ? __bfloat162float(src[row]) : 0.f;
      xd[1] = row + 1 < r_end ? __bfloat162float(src[row + 1]) : 0.f;
    }
  }
}

// Widens this thread's BF16 pairs of slab `blk` (copied by issue_slab) into X.
__device__ __forceinline__ void widen_slab(const PanelF32& p, int blk, float* X, const uint32_t* stg,
                                           int lane, int warp, bool pairs) {
  if (!p.a_bf16 || !pairs) return;
  const int k = lane & 15, half = lane >> 4;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = 2 * (warp + 8 * q) + half;
    const int col = blk * GB + c;
    if (col < p.n && col >= p.kc) {
      const uint32_t w = stg[c * SLD + k];
      X[c * GLD + 2 * k] = __uint_as_float(w << 16);
      X[c * GLD + 2 * k + 1] = __uint_as_float(w & 0xffff0000u);
    }
  }
}

// Partial Gram of block pair (bi, bj) over rows [r_begin, r_end).  Thread (tx, ty)
// owns outputs (ty + 16 k, tx + 16 l), k, l < 4; in a diagonal block only k <= l,
// which covers every entry on or above the diagonal (the reduction reads that
// orientation).  The row stages are double-buffered in shared memory: the next
// stage's copies are issued before the current stage's FMAs and waited for behind
// them, one barrier per stage.
template <bool DIAG>
__device__ __forceinline__ void gram_block(const PanelF32& p, int bi, int bj, int64_t r_begin,
                                           int64_t r_end, int fold_steps, double* __restrict__ out,
                                           float* sm, float* hl, uint32_t* stg) {
  // stage b: Xi at sm + 2 b GB GLD, Xj right after it; staging: Xi's pairs, then Xj's.
  // The float-float running sums (touched once per fold) live in shared memory:
  // output (k, l) of thread t at hl[(4 k + l) GTHREADS + t] (hi) and 16 GTHREADS
  // further on (lo).
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
  float* shi = hl + tid;
  float* slo = hl + 16 * GTHREADS + tid;
  uint32_t* stg_i = stg;
  uint32_t* stg_j = stg + GB * SLD;
  // BF16 rows are copied as 4-byte pairs when every pair starts on a 4-byte
  // boundary: an even leading dimension and base, and an even first row (the row
  // blocks of Algorithm 2 may start anywhere)
  const bool pairs = !p.a_pairs_unaligned && (r_begin & 1) == 0;
  float acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      acc[k][l] = 0.f;
      shi[(4 * k + l) * GTHREADS] = 0.f;
      slo[(4 * k + l) * GTHREADS] = 0.f;
    }
  if (r_begin < r_end) {
    issue_slab(p, bi, r_begin, r_end, sm, stg_i, lane, warp, pairs);
    if (!DIAG) issue_slab(p, bj, r_begin, r_end, sm + GB * GLD, stg_j, lane, warp, pairs);
    cp_async_commit();
    cp_async_wait_all();
    widen_slab(p, bi, sm, stg_i, lane, warp, pairs);
    if (!DIAG) widen_slab(p, bj, sm + GB * GLD, stg_j, lane, warp, pairs);
  }
  __syncthreads();
  int since = 0;  // 4-row steps since the last fold
  int buf = 0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += GRS) {
    const bool more = r0 + GRS < r_end;
    float* nxt = sm + (buf ^ 1) * (2 * GB * GLD);
    if (more) {
      issue_slab(p, bi, r0 + GRS, r_end, nxt, stg_i, lane, warp, pairs);
      if (!DIAG) issue_slab(p, bj, r0 + GRS, r_end, nxt + GB * GLD, stg_j, lane, warp, pairs);
      cp_async_commit();
    }
    const float* A = sm + buf * (2 * GB * GLD);
    const float* Bm = DIAG ? A : A + GB * GLD;
#pragma unroll
    for (int r = 0; r < GRS; r += 4) {
      float4 a[4], b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = *reinterpret_cast<const float4*>(&A[(ty + 16 * k) * GLD + r]);
#pragma unroll
      for (int l = 0; l < 4; ++l) b[l] = *reinterpret_cast<const float4*>(&Bm[(tx + 16 * l) * GLD + r]);
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          if (DIAG && k > l) continue;
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
            if (DIAG && k > l) continue;
            float h = shi[(4 * k + l) * GTHREADS], o = slo[(4 * k + l) * GTHREADS];
            two_sum_acc(h, o, acc[k][l]);
            shi[(4 * k + l) * GTHREADS] = h;
            slo[(4 * k + l) * GTHREADS] = o;
            acc[k][l] = 0.f;
          }
        since = 0;
      }
    }
    if (more) {
      cp_async_wait_all();
      widen_slab(p, bi, nxt, stg_i, lane, warp, pairs);
      if (!DIAG) widen_slab(p, bj, nxt + GB * GLD, stg_j, lane, warp, pairs);
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      if (DIAG && k > l) continue;
      float h = shi[(4 * k + l) * GTHREADS], o = slo[(4 * k + l) * GTHREADS];
      two_sum_acc(h, o, acc[k][l]);
      out[(ty + 16 * k) + GB * (tx + 16 * l)] = (double)h + (double)o;
    }
}

// Row chunk blockIdx.y: rows [blockIdx.y * rows_per_chunk, ...) of the panel, or,
// with a work list, rows [items[y].r0, items[y].r1) with that item's chain length
// (the row blocks of Algorithm 2 in one launch).
__global__ void __launch_bounds__(GTHREADS, 2) gram_partial_kernel(PanelF32 p, int nb,
                                                                int64_t rows_per_chunk,
                                                                int fold_steps,
                                                                const GramItem* __restrict__ items,
                                                                double* __restrict__ partial) {
  __shared__ __align__(16) float sm[4 * GB * GLD];  // two stages of [Xi | Xj]
  __shared__ float hl[32 * GTHREADS];              // float-float running sums
  __shared__ uint32_t stg[2 * GB * SLD];           // BF16 pairs of one stage
  int bi, bj;
  decode_pair(blockIdx.x, nb, &bi, &bj);
  const int npairs = gridDim.x;
  int64_t r_begin = (int64_t)blockIdx.y * rows_per_chunk;
  int64_t r_end = min(p.M, r_begin + rows_per_chunk);
  if (items) {
    const GramItem it = items[blockIdx.y];
    r_begin = it.r0;
    r_end = it.r1;
    fold_steps = it.fold_steps;
  }
  double* out = partial + ((size_t)blockIdx.y * npairs + blockIdx.x) * (GB * GB);
  if (bi == bj)
    gram_block<true>(p, bi, bj, r_begin, r_end, fold_steps, out, sm, hl, stg);
  else
    gram_block<false>(p, bi, bj, r_begin, r_end, fold_steps, out, sm, hl, stg);
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

constexpr int UK = 16;   // panel columns per stage

// Tile of UR = 32 RI rows x UC = 8 NW columns, NW warps; each thread holds RI rows x 8
// columns.  Every output element sums the panel columns in the same order whatever
// the tile, so all tile shapes give the same bits.  The stages (UK panel columns of
// the tile's rows, and the matching rows of T) are double-buffered in shared memory
// and filled with cp.async while the previous stage's FMAs run: FP32 columns
// element by element, BF16 columns as 4-byte row pairs widened after they land
// (plain loads when a pair is not 4-byte aligned).
template <int RI, int NW>
__global__ void __launch_bounds__(32 * NW) update_kernel(PanelF32 p, const float* __restrict__ T,
                                                         int k1, float* __restrict__ Unew,
                                                         int64_t ldo) {
  constexpr int UR = 32 * RI;
  constexpr int UC = 8 * NW;
  constexpr int NT = 32 * NW;
  constexpr int UP = UR / 2;  // row pairs per column
  __shared__ __align__(16) float Ps[2][UK * UR];
  __shared__ __align__(16) float Ts[2][UK * UC];
  __shared__ uint32_t Stg[UK * UP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * UR;
  const int j0 = blockIdx.y * UC;
  const bool pairs = !p.a_pairs_unaligned;  // r0 is even
  float acc[RI][8];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  auto issue = [&](int c0, int b) {
    for (int e = tid; e < UK * UP; e += NT) {
      const int c = e / UP, pi = e % UP;
      const int64_t row = r0 + 2 * pi;
      const int col = c0 + c;
      float* dst = &Ps[b][c * UR + 2 * pi];
      if (col >= p.n) {
        dst[0] = 0.f;
        dst[1] = 0.f;
      } else if (col < p.kc || !p.a_bf16) {
        const float* src = col < p.kc ? p.U + (int64_t)col * p.ldu
                                      : reinterpret_cast<const float*>(p.A) + (int64_t)(col - p.kc) * p.lda;
        cp_async4(dst, src + (row < p.M ? row : 0), row < p.M ? 4 : 0);
        cp_async4(dst + 1, src + (row + 1 < p.M ? row + 1 : 0), row + 1 < p.M ? 4 : 0);
      } else {
        const __nv_bfloat16* src =
            reinterpret_cast<const __nv_bfloat16*>(p.A) + (int64_t)(col - p.kc) * p.lda;
        if (pairs) {
          const int bytes = row + 1 < p.M ? 4 : row < p.M ? 2 : 0;
          cp_async4(&Stg[c * UP + pi], src + (bytes ? row : 0), bytes);
        } else {
          dst[0] = row < p.M ? __bfloat162float(src[row]) : 0.f;
          dst[1] = row + 1 < p.M ? __bfloat162float(src[row + 1]) : 0.f;
        }
      }
    }
    for (int e = tid; e < UK * UC; e += NT) {
      const int c = e / UC, j = e % UC;
      const bool ok = c0 + c < p.n && j0 + j < k1;
      cp_async4(&Ts[b][e], T + (ok ? (c0 + c) + (int64_t)(j0 + j) * p.n : 0), ok ? 4 : 0);
    }
    cp_async_commit();
  };
  auto widen = [&](int c0, int b) {
    if (!p.a_bf16 || !pairs) return;
    for (int e = tid; e < UK * UP; e += NT) {
      const int c = e / UP, pi = e % UP;
      const int col = c0 + c;
      if (col < p.n && col >= p.kc) {
        const uint32_t w = Stg[c * UP + pi];
        Ps[b][c * UR + 2 * pi] = __uint_as_float(w << 16);
        Ps[b][c * UR + 2 * pi + 1] = __uint_as_float(w & 0xffff0000u);
      }
    }
  };

  issue(0, 0);
  cp_async_wait_all();
  widen(0, 0);
  __syncthreads();
  int b = 0;
  for (int c0 = 0; c0 < p.n; c0 += UK) {
    const bool more = c0 + UK < p.n;
    if (more) issue(c0 + UK, b ^ 1);
#pragma unroll 4
    for (int c = 0; c < UK; ++c) {
      float pv[RI];
#pragma unroll
      for (int i = 0; i < RI; ++i) pv[i] = Ps[b][c * UR + lane + 32 * i];
      const float4 t0 = *reinterpret_cast<const float4*>(&Ts[b][c * UC + 8 * warp]);
      const float4 t1 = *reinterpret_cast<const float4*>(&Ts[b][c * UC + 8 * warp + 4]);
      const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(pv[i], tv[j], acc[i][j]);
    }
    if (more) {
      cp_async_wait_all();
      widen(c0 + UK, b ^ 1);
    }
    __syncthreads();
    b ^= 1;
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

// The panel as the Gram kernel reads it (BF16 row pairs copied as 4-byte words when
// the snapshots' base and leading dimension allow it).
static PanelF32 gram_panel(const PanelF32& p0) {
  PanelF32 p = p0;
  p.a_pairs_unaligned = (p.a_bf16 && ((p.lda & 1) || ((uintptr_t)p.A & 3))) ? 1 : 0;
  return p;
}

cudaError_t gram_simt_launch(const PanelF32& p, int nchunk, int64_t rows_per_chunk,
                             double* partial, cudaStream_t st) {
  const int nb = (int)ceil_div(p.n, GB);
  dim3 grid(nb * (nb + 1) / 2, nchunk);
  gram_partial_kernel<<<grid, GTHREADS, 0, st>>>(gram_panel(p), nb, rows_per_chunk,
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
  gram_partial_kernel<<<grid, GTHREADS, 0, st>>>(gram_panel(p), nb, 0, 1, items, partial);
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
  update_kernel<RI, NW><<<grid, 32 * NW, 0, st>>>(gram_panel(p), T, k1, Unew, ldo);
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
  else if (tile_rows == 256)
    launch_update_cols<8>(p, T, k1, Unew, ldo, st);
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
