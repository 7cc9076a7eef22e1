// Eigen-decomposition of the small symmetric matrix H (n x n, n = K + B <= 192)
// by scale levels: FP32 tridiagonal solves on one CTA, FP64 projections between
// levels.  Sets up the basis that the FP64 refinement in small_solve.cu polishes.
//
// An FP32 eigensolver is backward stable: its eigenpairs are exact for H + E with
// ||E|| ~ u32 ||H||.  Eigenvalues far below ||H|| (the graded tail of a streaming
// panel spans 9+ decades) are therefore not resolved by one FP32 solve.  Level l
// works on the block H_l = X_l^T H X_l (formed in FP64) of the directions not yet
// resolved, whose norm is the largest remaining eigenvalue.  Its FP32 solve
// resolves the eigenpairs with lambda >= tau * lambda_max(H_l) to
// ~u32 / tau relative accuracy, which is what the FP64 refinement needs to
// converge.  The rest of the block becomes the next level:
//   level_eig_kernel (one CTA, FP32, every hot loop on shared memory or registers):
//     1. power-of-two scaling of the block, Householder tridiagonalisation
//        (Golub & Van Loan, Algorithm 8.3.1); the reflectors are then copied out;
//     2. all eigenvalues of the tridiagonal by Sturm-count multisection,
//        32 shifts per warp and round;
//     3. eigenvectors of the resolved eigenvalues: twisted factorisations for
//        isolated eigenvalues (one thread each), inverse iteration with partial
//        pivoting and modified Gram-Schmidt (Peters & Wilkinson; as in LAPACK's
//        stein) inside clusters of close eigenvalues;
//     4. an orthonormal complement of the resolved vectors from their
//        Householder QR (the next level's basis).
//   level_backtransform_kernel (one warp per column, all SMs): applies the
//   tridiagonalisation reflectors and writes Y_l = blockdiag(I_b, Z).
//   Between levels (FP64 GEMMs on all SMs): W = H X, H_l = X^T W, X <- X Y_l.
// The number of levels is decided on the device (LevelState), so the host
// enqueues a fixed number of launches and no synchronisation.
#include <math.h>

#include "psvd_internal.cuh"

namespace psvd {
namespace {

constexpr int LT = 512;           // threads of the level kernel (128 registers each)
constexpr int LW = LT / 32;       // warps
constexpr int TRR = kMaxN / LW;   // rows of the register tile of a thread (12)
constexpr int TRC = kMaxN / 32;   // columns of the register tile of a thread (6)
constexpr int NB3 = kMaxN / (LT / 8);  // eigenvalues per thread in the multisection (3)
constexpr int LWI = 8;            // warps running inverse iteration on clusters
constexpr int NE = kMaxN / 32;    // eigenvalues per warp in the multisection
constexpr float kEps32 = 5.9604645e-8f;
constexpr int kRegion = kMaxN * (kMaxN | 1);  // floats of the reusable shared region

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Uniform value in (-1, 1) from a counter (integer hash, no state).
__device__ __forceinline__ float hash_uniform(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f + (1.0f / 16777216.0f);
}

struct LevelArgs {
  const double* Hf;   // n x n FP64 (ld n): the level block is Hf[b:, b:]
  int n;
  int nJ;             // eigenpairs needed (levels stop once b >= nJ)
  int last;           // 1 on the last level launched
  LevelState* ls;
  double* lam;        // n eigenvalue estimates (level l writes lam[b:])
  float* Zs;          // m x m FP32 (ld n): eigenvectors of T, then the complement
  float* V;           // m x m FP32 (ld n): tridiagonalisation reflectors (column k)
  float* vb;          // m reflector coefficients
  double tau;         // resolved: lambda >= tau * lambda_max(level)
  double floor_rel;   // stop once lambda_max(level) <= floor_rel * lambda_max(H)
  double ctol;        // cluster: consecutive eigenvalues closer than ctol * ||T||
  // batch: CTA z solves problem z, its arrays offset by z times these strides
  int64_t sHf, sLam, sFs, sLs;
};

__global__ void __launch_bounds__(LT) level_eig_kernel(LevelArgs a0) {
  // problem blockIdx.x of a batch
  LevelArgs a = a0;
  {
    const int64_t z = blockIdx.x;
    a.Hf += z * a0.sHf;
    a.lam += z * a0.sLam;
    a.Zs += z * a0.sFs;
    a.V += z * a0.sFs;
    a.vb += z * a0.sFs;
    a.ls += z * a0.sLs;
  }
  extern __shared__ __align__(16) float smem[];
  __shared__ float d[kMaxN], e[kMaxN], e2[kMaxN], lamf[kMaxN], qbeta[kMaxN];
  __shared__ float red[LW];
  __shared__ int cl_start[kMaxN + 1], cl_of[kMaxN], fb[kMaxN];
  __shared__ int s_ncl, s_r, s_b, s_go;
  __shared__ float s_gl, s_gu, s_pivmin, s_tn, s_lmax_est;
  __shared__ int s_rcount, s_reflect;
  __shared__ double s_scale;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  LevelState* ls = a.ls;

  if (tid == 0) {
    s_b = ls->b;
    s_go = ls->active;
    if (!s_go) ls->skip = 1;
  }
  __syncthreads();
  if (!s_go) return;
  const int b = s_b, m = n - b;
  const int LDA = m | 1;  // odd leading dimension: conflict-free row and column access
  // dynamic shared memory: region R (kRegion floats), reused phase by phase
  // (tridiagonalisation matrix, twisted factorisations, cluster solver, QR),
  // then 4 x kMaxN matvec partials
  float* R = smem;
  float* A = R;                       // m x LDA
  float* pv = R + kRegion;            // 4 x kMaxN
  const double* Hf = a.Hf;
  const int ldz = n;

  // ---- 0. load the block, scaled by a power of two so that FP32 neither
  //         overflows nor underflows
  // warp w takes columns w, w + 16, ...; lane l rows l, l + 32, ... (all loads of a
  // column issued before they are used)
  constexpr int NQ = kMaxN / 32;
  float amax_l = 0.f;
  for (int j = warp; j < m; j += LW) {
    const double* col = Hf + b + (int64_t)(b + j) * n;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int i = lane + 32 * q;
      v[q] = i < m ? col[i] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) amax_l = fmaxf(amax_l, (float)fabs(v[q]));
  }
  amax_l = warp_max(amax_l);
  if (lane == 0) red[warp] = amax_l;
  __syncthreads();
  if (tid == 0) {
    float am = 0.f;
    for (int w = 0; w < LW; ++w) am = fmaxf(am, red[w]);
    int ex = 0;
    frexpf(am > 0.f && isfinite(am) ? am : 1.f, &ex);
    s_scale = ldexp(1.0, -ex);  // block entries scaled into [0.5, 1)
  }
  __syncthreads();
  const double sc = s_scale;
  for (int j = warp; j < m; j += LW) {
    const double* col = Hf + b + (int64_t)(b + j) * n;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int i = lane + 32 * q;
      v[q] = i < m ? col[i] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int i = lane + 32 * q;
      if (i < m) A[i + j * LDA] = (float)(v[q] * sc);
    }
  }
  __syncthreads();

  // ---- 1. Householder tridiagonalisation with the matrix in registers: thread
  //         (warp w, lane l) holds rows 12w .. 12w+11 x columns 6l .. 6l+5 (the
  //         192 x 192 FP32 block fills about half the register file).  Per column k:
  //           (a) the owners of column k publish rows > k and d[k];
  //           (b) warp 0 forms the unit reflector u (H = I - 2 u u^T; no
  //               1 / ||v||^2 intermediate, which overflows FP32 on near-null
  //               columns) and stores it for the back-transformation;
  //           (c) p = A u: register FMAs, rows reduced across lanes by
  //               interleaved shuffles;
  //           (d) A -= u w^T + w u^T, w = 2 (p - (u^T p) u), in registers.
  //         Rows and columns <= k are never read again, so (c) and (d) leave them
  //         unmasked; warps whose rows are all <= k skip both.
  {
    float* xcol = pv;               // kMaxN: column k
    float* uvec = pv + kMaxN;       // kMaxN: reflector
    float* pvec = pv + 2 * kMaxN;   // kMaxN: p = A u
    const int r0 = warp * TRR, c0 = lane * TRC;
    float at[TRR][TRC];
#pragma unroll
    for (int r = 0; r < TRR; ++r)
#pragma unroll
      for (int c = 0; c < TRC; ++c) {
        const int i = r0 + r, j = c0 + c;
        at[r][c] = (i < m && j < m) ? A[i + j * LDA] : 0.f;
      }
    // the reflector buffer starts at zero; (b) then rewrites entries k .. m-1
    for (int i = tid; i < kMaxN; i += LT) uvec[i] = 0.f;
    for (int k = 0; k < m - 2; ++k) {
      // (a) column k below the diagonal, and d[k]
      if (lane == k / TRC) {
#pragma unroll
        for (int c = 0; c < TRC; ++c)
          if (c0 + c == k) {
#pragma unroll
            for (int r = 0; r < TRR; ++r) {
              const int i = r0 + r;
              if (i >= k && i < m) {
                if (i == k) d[k] = at[r][c];
                else xcol[i] = at[r][c];
              }
            }
          }
      }
      __syncthreads();
      // (b) reflector from xcol[k+1 .. m-1]: one warp, element i = k+1+lane+32j
      //     in xv[j]; loads issued together and the sum taken as a tree (this
      //     step is a serial chain that the other warps wait for)
      if (warp == 0) {
        float xv[TRC];
#pragma unroll
        for (int j = 0; j < TRC; ++j) {
          const int i = k + 1 + lane + 32 * j;
          xv[j] = i < m ? xcol[i] : 0.f;
        }
        const float x0 = __shfl_sync(0xffffffffu, xv[0], 0);  // xcol[k+1]
        float s01 = lane == 0 ? 0.f : xv[0] * xv[0];
        s01 = fmaf(xv[1], xv[1], s01);
        const float s23 = fmaf(xv[3], xv[3], xv[2] * xv[2]);
        const float s45 = fmaf(xv[5], xv[5], xv[4] * xv[4]);
        const float sq = warp_sum((s01 + s23) + s45);
        const bool refl = sq > 0.f && isfinite(sq);
        float alpha = x0, inv = 0.f, v0 = 0.f;
        if (refl) {
          const float nrm = sqrtf(fmaf(x0, x0, sq));
          alpha = (x0 >= 0.f) ? -nrm : nrm;
          v0 = x0 - alpha;
          inv = rsqrtf(fmaf(v0, v0, sq));
        }
        // entries <= k were zeroed when their columns were reduced; uvec[k] is
        // the previous reflector's first entry
        if (lane == 0) uvec[k] = 0.f;
#pragma unroll
        for (int j = 0; j < TRC; ++j) {
          const int i = k + 1 + lane + 32 * j;
          if (i < m) {
            const float ui = !refl ? 0.f : (i == k + 1) ? v0 * inv : xv[j] * inv;
            uvec[i] = ui;
            a.V[i + (int64_t)k * ldz] = ui;
          }
        }
        if (lane == 0) {
          e[k] = alpha;
          a.vb[k] = refl ? 2.f : 0.f;
          s_reflect = refl ? 1 : 0;
        }
      }
      __syncthreads();
      if (!s_reflect) continue;  // uniform: column already reduced
      const bool live = r0 + TRR - 1 > k;  // warp has rows in the trailing block
      // (c) p = A u.  The 12 row sums of a warp are reduced across its lanes by
      //     halving exchanges (12 -> 6 -> 3 values per lane, xor 16 and 8), then
      //     butterflies over the remaining 8 lanes: 20 shuffles instead of 60.
      //     Lane l ends with rows rb .. rb+2, rb = 6 bit4(l) + 3 bit3(l).
      {
        float a3[3] = {0.f, 0.f, 0.f};
        if (live) {
          float uc[TRC];
#pragma unroll
          for (int c = 0; c < TRC; ++c) uc[c] = uvec[c0 + c];
          float acc[TRR];
#pragma unroll
          for (int r = 0; r < TRR; ++r) {
            float t = 0.f;
#pragma unroll
            for (int c = 0; c < TRC; ++c) t = fmaf(at[r][c], uc[c], t);
            acc[r] = t;
          }
          const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
          float a6[6];
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            const float send = h16 ? acc[j] : acc[j + 6];
            const float keep = h16 ? acc[j + 6] : acc[j];
            a6[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
          }
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float send = h8 ? a6[j] : a6[j + 3];
            const float keep = h8 ? a6[j + 3] : a6[j];
            a3[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
          }
#pragma unroll
          for (int o = 4; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < 3; ++j) a3[j] += __shfl_xor_sync(0xffffffffu, a3[j], o);
        }
        // one lane of each group of 8 publishes its three rows
        const int rb = r0 + ((lane >> 4) & 1) * 6 + ((lane >> 3) & 1) * 3;
        float up = 0.f;
        if ((lane & 7) == 0) {
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            pvec[rb + j] = a3[j];
            up = fmaf(a3[j], uvec[rb + j], up);
          }
        }
        up += __shfl_xor_sync(0xffffffffu, up, 8);
        up += __shfl_xor_sync(0xffffffffu, up, 16);
        if (lane == 0) red[warp] = up;
      }
      __syncthreads();
      // (d) rank-2 update in registers
      if (live) {
        // u^T A u from the warps' partials: every thread sums them in the same order
        float uau = 0.f;
#pragma unroll
        for (int i = 0; i < LW; ++i) uau += red[i];
        float ur[TRR], wr[TRR], ucv[TRC], wc[TRC];
#pragma unroll
        for (int r = 0; r < TRR; ++r) {
          ur[r] = uvec[r0 + r];
          wr[r] = 2.f * fmaf(-uau, ur[r], pvec[r0 + r]);
        }
#pragma unroll
        for (int c = 0; c < TRC; ++c) {
          ucv[c] = uvec[c0 + c];
          wc[c] = 2.f * fmaf(-uau, ucv[c], pvec[c0 + c]);
        }
#pragma unroll
        for (int r = 0; r < TRR; ++r)
#pragma unroll
          for (int c = 0; c < TRC; ++c) at[r][c] = fmaf(-ur[r], wc[c], fmaf(-wr[r], ucv[c], at[r][c]));
      }
    }
    // the trailing 2 x 2 block
#pragma unroll
    for (int r = 0; r < TRR; ++r)
#pragma unroll
      for (int c = 0; c < TRC; ++c) {
        const int i = r0 + r, j = c0 + c;
        if (m >= 2 && i == m - 2 && j == m - 2) d[m - 2] = at[r][c];
        if (m >= 2 && i == m - 1 && j == m - 2) e[m - 2] = at[r][c];
        if (i == m - 1 && j == m - 1) d[m - 1] = at[r][c];
      }
  }
  __syncthreads();
  if (tid == 0) {
    e[m - 1] = 0.f;
    for (int k = max(m - 2, 0); k < m; ++k) a.vb[k] = 0.f;
    float gl = INFINITY, gu = -INFINITY, emax2 = 0.f;
    for (int i = 0; i < m; ++i) {
      const float r = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i < m - 1 ? fabsf(e[i]) : 0.f);
      gl = fminf(gl, d[i] - r);
      gu = fmaxf(gu, d[i] + r);
      if (i < m - 1) emax2 = fmaxf(emax2, e[i] * e[i]);
    }
    for (int i = 0; i < m - 1; ++i) e2[i] = e[i] * e[i];
    const float tn = fmaxf(fabsf(gl), fabsf(gu));
    s_pivmin = 1.17549435e-38f * fmaxf(1.f, emax2);
    s_tn = (tn > 0.f && isfinite(tn)) ? tn : 1.f;
    s_gl = gl - 2.f * kEps32 * s_tn - s_pivmin;
    s_gu = gu + 2.f * kEps32 * s_tn + s_pivmin;
  }
  __syncthreads();

  // ---- 2. eigenvalues (descending) by multisection: a group of 8 lanes tests 8
  //         shifts per eigenvalue and round (9 subintervals); each thread carries
  //         NB3 eigenvalues (g, g + 64, g + 128).  Three rounds for all
  //         eigenvalues, then the number resolved (lambda >= tau * lambda_max) by
  //         one exact Sturm count, then five more rounds for the resolved ones and
  //         a margin of 8 (the rest only seed estimates for the next level).
  {
    const int grp = tid >> 3, gl8 = tid & 7;
    float lo[NB3], hi[NB3];
    int qidx[NB3];
#pragma unroll
    for (int t = 0; t < NB3; ++t) {
      lo[t] = s_gl;
      hi[t] = s_gu;
      const int jj = grp + (LT / 8) * t;
      qidx[t] = (jj < m) ? m - 1 - jj : 0;  // ascending index
    }
    const float pivmin = s_pivmin;
    const bool fin = isfinite(s_gl) && isfinite(s_gu);
    auto rounds = [&](int nr, int jlimit) {
      for (int round = 0; round < nr; ++round) {
        float x[NB3], q[NB3];
        int cnt[NB3];
        bool act[NB3];
#pragma unroll
        for (int t = 0; t < NB3; ++t) {
          act[t] = fin && (grp + (LT / 8) * t) < jlimit;
          x[t] = lo[t] + (hi[t] - lo[t]) * (float)(gl8 + 1) * (1.f / 9.f);
          q[t] = d[0] - x[t];
          if (fabsf(q[t]) < pivmin) q[t] = -pivmin;
          cnt[t] = q[t] < 0.f;
        }
        if (act[0] || act[1] || act[2]) {
          for (int i = 1; i < m; ++i) {
            const float di = d[i], ei = e2[i - 1];
#pragma unroll
            for (int t = 0; t < NB3; ++t) {
              q[t] = (di - x[t]) - __fdividef(ei, q[t]);
              if (fabsf(q[t]) < pivmin) q[t] = -pivmin;
              cnt[t] += q[t] < 0.f;
            }
          }
        }
#pragma unroll
        for (int t = 0; t < NB3; ++t) {
          const unsigned bal = __ballot_sync(0xffffffffu, cnt[t] <= qidx[t]);
          const int nle = __popc((bal >> (lane & 24)) & 0xffu);
          const float span = hi[t] - lo[t];
          const float nlo = (nle > 0) ? lo[t] + span * (float)nle * (1.f / 9.f) : lo[t];
          const float nhi = (nle < 8) ? lo[t] + span * (float)(nle + 1) * (1.f / 9.f) : hi[t];
          if (act[t]) {
            lo[t] = nlo;
            hi[t] = nhi;
          }
        }
      }
    };
    rounds(3, m);
    if (gl8 == 0 && grp == 0) s_lmax_est = 0.5f * (lo[0] + hi[0]);
    __syncthreads();
    if (tid == 0) {
      // eigenvalues >= tau * lambda_max: m minus the Sturm count below the threshold
      const float x = (float)a.tau * s_lmax_est;
      int cnt = 0;
      if (fin && s_lmax_est > 0.f) {
        float q = d[0] - x;
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt = q < 0.f;
        for (int i = 1; i < m; ++i) {
          q = (d[i] - x) - e2[i - 1] / q;
          if (fabsf(q) < pivmin) q = -pivmin;
          cnt += q < 0.f;
        }
      } else {
        cnt = m;
      }
      s_rcount = m - cnt;
    }
    __syncthreads();
    rounds(5, min(m, s_rcount + 8));
    if (gl8 == 0) {
#pragma unroll
      for (int t = 0; t < NB3; ++t) {
        const int jj = grp + (LT / 8) * t;
        if (jj < m) lamf[jj] = 0.5f * (lo[t] + hi[t]);
      }
    }
  }
  __syncthreads();

  // ---- resolved count, level bookkeeping
  if (tid == 0) {
    const double lmax_level = (double)lamf[0] / sc;
    if (b == 0) ls->lmax = lmax_level;
    const double lmax = ls->lmax;
    int r = 0;
    if (isfinite(lmax_level) && lmax_level > 0.0 && lmax_level > a.floor_rel * lmax) {
      r = min(max(s_rcount, 1), m);
    }
    s_r = r;
    // clusters among the resolved eigenvalues
    int ncl = 0;
    const float ct = (float)a.ctol * s_tn;
    for (int j = 0; j < r; ++j) {
      if (j == 0 || lamf[j - 1] - lamf[j] > ct) cl_start[ncl++] = j;
      cl_of[j] = ncl - 1;
    }
    cl_start[ncl] = r;
    s_ncl = ncl;
  }
  __syncthreads();
  const int r = s_r;
  for (int j = tid; j < m; j += LT) a.lam[b + j] = (double)lamf[j] / sc;
  if (r == 0) {
    if (tid == 0) {
      ls->active = 0;
      ls->skip = 1;
      ls->r = 0;
      ls->b0 = b;
      ls->floored = 1;
    }
    return;
  }

  // ---- 3. eigenvectors of the resolved eigenvalues
  //   (a) singletons: one thread each, twisted factorisation of T - lambda I
  //       (stationary and progressive qd transforms, twist at min |gamma_k|;
  //       Fernando 1997, Parlett & Dhillon 2000), vector by the two recurrences
  //       from the twist; D+ and D- go to global scratch, written once and
  //       read back once, never in a dependent chain.
  //   (b) clusters (and singletons whose twisted vector failed): warp w < LWI
  //       runs inverse iteration with partial pivoting and modified Gram-Schmidt
  //       against the cluster's earlier members, factors in shared memory.
  float* Zs = a.Zs;
  if (tid < r) fb[tid] = 0;
  {
    const float pivmin = s_pivmin;
    const int tpr = min(LT, kRegion / (2 * m));  // threads per round
    for (int base = 0; base < r; base += tpr) {
      const int j = base + tid;
      if (tid < tpr && j < r && cl_start[cl_of[j] + 1] - cl_start[cl_of[j]] == 1) {
        float* Dp = R + tid;            // D+_i at Dp[i * tpr]
        float* Dm = R + m * tpr + tid;  // D-_i at Dm[i * tpr]
        const float lam = lamf[j];
        float dp = d[0] - lam;
        if (fabsf(dp) < pivmin) dp = -pivmin;
        Dp[0] = dp;
        for (int i = 0; i < m - 1; ++i) {
          dp = (d[i + 1] - lam) - __fdividef(e2[i], dp);
          if (fabsf(dp) < pivmin) dp = -pivmin;
          Dp[(i + 1) * tpr] = dp;
        }
        float dm = d[m - 1] - lam;
        if (fabsf(dm) < pivmin) dm = -pivmin;
        Dm[(m - 1) * tpr] = dm;
        float best = fabsf(Dp[(m - 1) * tpr]);
        int tw = m - 1;
        for (int i = m - 2; i >= 0; --i) {
          dm = (d[i] - lam) - __fdividef(e2[i], dm);
          if (fabsf(dm) < pivmin) dm = -pivmin;
          Dm[i * tpr] = dm;
          const float g = fabsf(Dp[i * tpr] + dm - (d[i] - lam));
          if (g < best) {
            best = g;
            tw = i;
          }
        }
        // z from the twist: z_i = -(e_i / D+_i) z_{i+1} above, z_{i+1} = -(e_i / D-_{i+1}) z_i below;
        // kept in the D+ / D- slots it replaces
        float zi = 1.f, nn = 1.f;
        for (int i = tw - 1; i >= 0; --i) {
          zi = -__fdividef(e[i], Dp[i * tpr]) * zi;
          Dp[i * tpr] = zi;
          nn = fmaf(zi, zi, nn);
        }
        zi = 1.f;
        for (int i = tw; i < m - 1; ++i) {
          zi = -__fdividef(e[i], Dm[(i + 1) * tpr]) * zi;
          Dm[(i + 1) * tpr] = zi;
          nn = fmaf(zi, zi, nn);
        }
        float* z = Zs + (int64_t)j * ldz;
        if (nn > 0.f && isfinite(nn)) {
          const float rn = rsqrtf(nn);
          for (int i = 0; i < m; ++i)
            z[i] = rn * ((i < tw) ? Dp[i * tpr] : (i == tw) ? 1.f : Dm[i * tpr]);
        } else {
          fb[j] = 1;
        }
      }
      __syncthreads();
    }
  }
  if (warp < LWI) {
    const float tiny = kEps32 * s_tn, sep = 10.f * kEps32 * s_tn;
    float* xv = R + warp * kMaxN;                        // LWI x kMaxN vectors
    float* la = R + LWI * kMaxN + warp * 5 * kMaxN;      // diag of U, 1st super, 2nd super, multipliers, pivots
    float* bu = la + kMaxN;
    float* du2 = bu + kMaxN;
    float* ll = du2 + kMaxN;
    float* pv2 = ll + kMaxN;
    for (int cl = warp; cl < s_ncl; cl += LWI) {
      const int j0 = cl_start[cl], j1 = cl_start[cl + 1];
      if (j1 - j0 == 1 && !fb[j0]) continue;  // done by path (a)
      float prev = 0.f;
      for (int j = j0; j < j1; ++j) {
        float shift = lamf[j];
        if (j > j0 && prev - shift < sep) shift = prev - sep;
        prev = shift;
        if (lane == 0) {
          // LU of T - shift I with partial pivoting (rows k, k+1 exchanged when |c_k| > |a_k|)
          for (int i = 0; i < m; ++i) {
            la[i] = d[i] - shift;
            bu[i] = (i < m - 1) ? e[i] : 0.f;
            du2[i] = 0.f;
          }
          for (int k = 0; k < m - 1; ++k) {
            const float ak = la[k], ck = e[k];
            if (fabsf(ak) >= fabsf(ck)) {
              const float mult = (ak != 0.f) ? ck / ak : 0.f;
              ll[k] = mult;
              pv2[k] = 0.f;
              la[k + 1] = fmaf(-mult, bu[k], la[k + 1]);
            } else {
              const float mult = ak / ck;
              ll[k] = mult;
              pv2[k] = 1.f;
              la[k] = ck;
              const float tmp = la[k + 1];
              la[k + 1] = fmaf(-mult, tmp, bu[k]);
              bu[k] = tmp;
              if (k < m - 2) {
                du2[k] = bu[k + 1];
                bu[k + 1] = -mult * du2[k];
              }
            }
          }
        }
        for (int i = lane; i < m; i += 32) xv[i] = hash_uniform((uint32_t)(b * 256 + j), (uint32_t)i);
        __syncwarp();
        for (int it = 0; it < 3; ++it) {
          float mx = 0.f;
          for (int i = lane; i < m; i += 32) mx = fmaxf(mx, fabsf(xv[i]));
          mx = warp_max(mx);
          const float inv = (mx > 0.f && isfinite(mx)) ? 1.f / mx : 1.f;
          for (int i = lane; i < m; i += 32) xv[i] *= inv;
          __syncwarp();
          if (lane == 0) {
            for (int k = 0; k < m - 1; ++k) {
              if (pv2[k] != 0.f) {
                const float t0 = xv[k];
                xv[k] = xv[k + 1];
                xv[k + 1] = fmaf(-ll[k], xv[k], t0);
              } else {
                xv[k + 1] = fmaf(-ll[k], xv[k], xv[k + 1]);
              }
            }
            for (int k = m - 1; k >= 0; --k) {
              float s = xv[k];
              if (k + 1 < m) s = fmaf(-bu[k], xv[k + 1], s);
              if (k + 2 < m) s = fmaf(-du2[k], xv[k + 2], s);
              float ak = la[k];
              if (fabsf(ak) < tiny) ak = (ak >= 0.f) ? tiny : -tiny;
              float xk = s / ak;
              if (!(fabsf(xk) <= 1e30f)) {
                // growth through several tiny pivots: rescale the system (the
                // solution is only needed up to a factor) and redo this row
                const float f = (fabsf(s) > 0.f && isfinite(s)) ? fabsf(ak) / fabsf(s) : 0.f;
                for (int i = 0; i < m; ++i) xv[i] *= f;
                s *= f;
                xk = (f > 0.f) ? s / ak : 0.f;
              }
              xv[k] = xk;
            }
          }
          __syncwarp();
          // orthogonalise against the cluster's earlier members
          for (int t = j0; t < j; ++t) {
            const float* zt = Zs + (int64_t)t * ldz;
            float dt = 0.f;
            for (int i = lane; i < m; i += 32) dt = fmaf(zt[i], xv[i], dt);
            dt = warp_sum(dt);
            for (int i = lane; i < m; i += 32) xv[i] = fmaf(-dt, zt[i], xv[i]);
            __syncwarp();
          }
          float nn = 0.f;
          for (int i = lane; i < m; i += 32) nn = fmaf(xv[i], xv[i], nn);
          nn = warp_sum(nn);
          const float rn = (nn > 0.f && isfinite(nn)) ? rsqrtf(nn) : 0.f;
          for (int i = lane; i < m; i += 32) xv[i] = (rn > 0.f) ? xv[i] * rn : (i == j ? 1.f : 0.f);
          __syncwarp();
        }
        float* zj = Zs + (int64_t)j * ldz;
        for (int i = lane; i < m; i += 32) zj[i] = xv[i];
        __syncwarp();
      }
    }
  }
  __syncthreads();

  // ---- 4. orthonormal complement of span(Z[:, 0:r]): Householder QR of a copy
  //         in shared memory, complement = H_0 ... H_{r-1} [0; I_{m-r}] (warp per
  //         column, held in registers)
  if (r < m) {
    float* Zq = R;  // m x r, ld m
    for (int e0 = tid; e0 < m * r; e0 += LT) {
      const int i = e0 % m, j = e0 / m;
      Zq[e0] = Zs[i + (int64_t)j * ldz];
    }
    __syncthreads();
    // column c belongs to warp c % LW; step t: every warp applies reflector t
    // to its columns c > t, and the owner of column t + 1 then forms reflector
    // t + 1 from its now updated column, so one block barrier per step suffices
    auto form_reflector = [&](int t) {
      float* zc = Zq + t * m;
      float zv[NE];
#pragma unroll
      for (int q = 0; q < NE; ++q) {
        const int i = lane + 32 * q;
        zv[q] = (i >= t && i < m) ? zc[i] : 0.f;
      }
      const float x0 = zc[t];
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < NE; ++q) {
        const int i = lane + 32 * q;
        s = fmaf(i > t ? zv[q] : 0.f, zv[q], s);
      }
      const float s1 = warp_sum(s);
      float bt = 0.f, v0 = x0, inv = 1.f;
      if (s1 > 0.f && isfinite(s1)) {  // unit reflector u = v / ||v||, H = I - 2 u u^T
        const float nrm = sqrtf(fmaf(x0, x0, s1));
        v0 = x0 - ((x0 >= 0.f) ? -nrm : nrm);
        inv = rsqrtf(fmaf(v0, v0, s1));
        bt = 2.f;
      }
      __syncwarp();
      if (bt != 0.f) {
#pragma unroll
        for (int q = 0; q < NE; ++q) {
          const int i = lane + 32 * q;
          if (i >= t && i < m) zc[i] = (i == t) ? v0 * inv : zv[q] * inv;
        }
      }
      if (lane == 0) qbeta[t] = bt;
      __syncwarp();
    };
    if (warp == 0) form_reflector(0);
    __syncthreads();
    for (int t = 0; t < r; ++t) {
      const float bt = qbeta[t];
      const float* zc = Zq + t * m;
      int c0 = t + 1 + ((warp - (t + 1)) % LW + LW) % LW;  // first c > t owned by this warp
      if (bt != 0.f && c0 < r) {
        float zv[NE];
#pragma unroll
        for (int q = 0; q < NE; ++q) {
          const int i = lane + 32 * q;
          zv[q] = (i >= t && i < m) ? zc[i] : 0.f;
        }
        // this warp's columns c0, c0 + 16, ..., four at a time: dot products and
        // warp sums interleaved
        for (int cb = c0; cb < r; cb += 4 * LW) {
          float dt[4];
#pragma unroll
          for (int w4 = 0; w4 < 4; ++w4) {
            const int c = cb + w4 * LW;
            float acc = 0.f;
            if (c < r) {
              const float* zk = Zq + c * m;
#pragma unroll
              for (int q = 0; q < NE; ++q) {
                const int i = lane + 32 * q;
                acc = fmaf(zv[q], (i < m) ? zk[i] : 0.f, acc);
              }
            }
            dt[w4] = acc;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int w4 = 0; w4 < 4; ++w4) dt[w4] += __shfl_xor_sync(0xffffffffu, dt[w4], o);
#pragma unroll
          for (int w4 = 0; w4 < 4; ++w4) {
            const int c = cb + w4 * LW;
            if (c < r) {
              float* zk = Zq + c * m;
              const float f = dt[w4] * bt;
#pragma unroll
              for (int q = 0; q < NE; ++q) {
                const int i = lane + 32 * q;
                if (i >= t && i < m) zk[i] = fmaf(-f, zv[q], zk[i]);
              }
            }
          }
        }
        __syncwarp();
      }
      if (t + 1 < r && warp == (t + 1) % LW) form_reflector(t + 1);
      __syncthreads();
    }
    // complement columns c = r .. m-1, four per warp at a time: their dot products
    // and warp sums interleave, so one reflector costs one reduction latency
    constexpr int NCW = 4;
    for (int cb = r + warp; cb < m; cb += NCW * LW) {
      float x[NCW][NE];
#pragma unroll
      for (int w4 = 0; w4 < NCW; ++w4)
#pragma unroll
        for (int q = 0; q < NE; ++q) x[w4][q] = (lane + 32 * q == cb + w4 * LW) ? 1.f : 0.f;
      for (int t = r - 1; t >= 0; --t) {
        const float bt = qbeta[t];
        if (bt == 0.f) continue;
        const float* zc = Zq + t * m;
        float zv[NE];
#pragma unroll
        for (int q = 0; q < NE; ++q) {
          const int i = lane + 32 * q;
          zv[q] = (i >= t && i < m) ? zc[i] : 0.f;
        }
        float dt[NCW];
#pragma unroll
        for (int w4 = 0; w4 < NCW; ++w4) {
          float acc = 0.f;
#pragma unroll
          for (int q = 0; q < NE; ++q) acc = fmaf(zv[q], x[w4][q], acc);
          dt[w4] = acc;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int w4 = 0; w4 < NCW; ++w4) dt[w4] += __shfl_xor_sync(0xffffffffu, dt[w4], o);
#pragma unroll
        for (int w4 = 0; w4 < NCW; ++w4)
#pragma unroll
          for (int q = 0; q < NE; ++q) x[w4][q] = fmaf(-dt[w4] * bt, zv[q], x[w4][q]);
      }
#pragma unroll
      for (int w4 = 0; w4 < NCW; ++w4) {
        const int c = cb + w4 * LW;
        if (c < m) {
          float* zk = Zs + (int64_t)c * ldz;
#pragma unroll
          for (int q = 0; q < NE; ++q) {
            const int i = lane + 32 * q;
            if (i < m) zk[i] = x[w4][q];
          }
        }
      }
    }
  }
  if (tid == 0) {
    ls->r = r;
    ls->b0 = b;
    ls->b = b + r;
    ls->skip = 0;
    ls->levels += 1;
    ls->active = (b + r < a.nJ && r < m && !a.last) ? 1 : 0;
  }
}

// Y = blockdiag(I_b, Q_T Z) for the level just solved (b = ls->b0, m = n - b):
// each CTA stages the reflectors in shared memory, then warp c handles column c
// with the column of Z in registers (lane l holds rows l, l + 32, ...).  When the
// level was skipped, level 0 (first != 0) writes the identity and later levels
// nothing.
constexpr int BTW = 8;  // warps (columns) per CTA of the back-transformation
__global__ void __launch_bounds__(BTW * 32) level_backtransform_kernel(
    int n, const float* __restrict__ Zs, const float* __restrict__ V, const float* __restrict__ vb,
    double* __restrict__ Y, const LevelState* __restrict__ ls, int first, int64_t sFs, int64_t sY,
    int64_t sLs) {
  extern __shared__ __align__(16) float vs[];  // m x m reflectors (ld m), then m coefficients
  {
    // problem blockIdx.y of a batch
    const int64_t z = blockIdx.y;
    Zs += z * sFs;
    V += z * sFs;
    vb += z * sFs;
    Y += z * sY;
    ls += z * sLs;
  }
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * BTW + (threadIdx.x >> 5);
  const bool skip = ls->skip != 0;
  const int b = ls->b0, m = n - b;
  if (skip) {
    if (first && c < n)
      for (int i = lane; i < n; i += 32) Y[i + (int64_t)c * n] = (i == c) ? 1.0 : 0.0;
    return;
  }
  float* vbs = vs + m * m;
  for (int k = threadIdx.x >> 5; k < m; k += BTW)
    for (int i = lane; i < m; i += 32) vs[i + k * m] = V[i + (int64_t)k * n];
  for (int k = threadIdx.x; k < m; k += BTW * 32) vbs[k] = vb[k];
  __syncthreads();
  if (c >= n) return;
  double* yc = Y + (int64_t)c * n;
  if (c < b) {
    for (int i = lane; i < n; i += 32) yc[i] = (i == c) ? 1.0 : 0.0;
    return;
  }
  const float* z = Zs + (int64_t)(c - b) * n;
  float x[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int i = lane + 32 * q;
    x[q] = (i < m) ? z[i] : 0.f;
  }
  for (int k = m - 3; k >= 0; --k) {
    const float bt = vbs[k];
    if (bt == 0.f) continue;
    const float* v = vs + k * m;
    float dt = 0.f;
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      const int i = lane + 32 * q;
      if (i > k && i < m) dt = fmaf(v[i], x[q], dt);
    }
    dt = warp_sum(dt) * bt;
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      const int i = lane + 32 * q;
      if (i > k && i < m) x[q] = fmaf(-dt, v[i], x[q]);
    }
  }
  for (int i = lane; i < b; i += 32) yc[i] = 0.0;
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int i = lane + 32 * q;
    if (i < m) yc[b + i] = (double)x[q];
  }
}

__global__ void level_init_kernel(LevelState* ls, int64_t sLs) {
  ls += blockIdx.x * sLs;
  ls->b = 0;
  ls->active = 1;
  ls->skip = 0;
  ls->r = 0;
  ls->levels = 0;
  ls->floored = 0;
  ls->lmax = 0.0;
}

// C = A B (n x n FP64) unless the last level was skipped, in which case C = A.
__global__ void __launch_bounds__(64) level_update_kernel(int n, const double* __restrict__ A,
                                                          const double* __restrict__ B,
                                                          double* __restrict__ C,
                                                          const LevelState* __restrict__ ls,
                                                          int64_t sNN, int64_t sLs) {
  __shared__ double As[8][33];
  __shared__ double Bs[32][9];
  {
    // problem blockIdx.z of a batch
    const int64_t z = blockIdx.z;
    A += z * sNN;
    B += z * sNN;
    C += z * sNN;
    ls += z * sLs;
  }
  const bool skip = ls->skip != 0;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int row = blockIdx.x * 8 + tx, col = blockIdx.y * 8 + ty;
  if (skip) {
    if (row < n && col < n) C[row + (int64_t)col * n] = A[row + (int64_t)col * n];
    return;
  }
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int e0 = threadIdx.x; e0 < 8 * 32; e0 += 64) {
      const int r = e0 % 8, kk = e0 / 8;
      const int gr = blockIdx.x * 8 + r, gk = k0 + kk;
      As[r][kk] = (gr < n && gk < n) ? A[gr + (int64_t)gk * n] : 0.0;
      const int c = e0 / 32, kb = e0 % 32;
      const int gc = blockIdx.y * 8 + c, gkb = k0 + kb;
      Bs[kb][c] = (gc < n && gkb < n) ? B[gkb + (int64_t)gc * n] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) acc = fma(As[tx][kk], Bs[kk][ty], acc);
    __syncthreads();
  }
  if (row < n && col < n) C[row + (int64_t)col * n] = acc;
}

size_t level_smem_bytes() { return sizeof(float) * ((size_t)kRegion + 4 * (size_t)kMaxN); }

}  // namespace

size_t eig_levels_scratch_floats(int nmax) { return 2 * (size_t)nmax * nmax + (size_t)nmax; }

cudaError_t eig_levels_launch(const SmallWork& w, int n, int nJ, int max_levels, cudaStream_t st,
                              int* launches) {
  cudaError_t e;
  const SmallBatch& bs = w.bat;
  const unsigned nb = (unsigned)bs.count;
  const size_t smem = level_smem_bytes();
  if ((e = cudaFuncSetAttribute(level_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess)
    return e;
  LevelArgs a;
  a.n = n;
  a.nJ = nJ;
  a.ls = w.ls;
  a.lam = w.lam;
  a.Zs = w.fs;
  a.V = w.fs + (size_t)n * n;
  a.vb = w.fs + 2 * (size_t)n * n;
  a.tau = 1e-3;
  a.floor_rel = lambda_floor(w);
  a.ctol = 1e-5;
  a.sHf = bs.nn;
  a.sLam = bs.n;
  a.sFs = bs.fs;
  a.sLs = bs.ls;
  int nl = 0;
  level_init_kernel<<<nb, 1, 0, st>>>(w.ls, bs.ls);
  ++nl;
  // buffers: X ping-pong between w.Xn and w.X so that the result ends in w.X
  double* cur = ((max_levels - 1) % 2 == 0) ? w.X : w.Xn;
  double* nxt = (cur == w.X) ? w.Xn : w.X;
  const dim3 gbt((unsigned)ceil_div(n, BTW), nb);
  const size_t bt_smem = sizeof(float) * ((size_t)n * n + n);
  if ((e = cudaFuncSetAttribute(level_backtransform_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem)) !=
      cudaSuccess)
    return e;
  // level 0 on H itself: Y_0 is X
  a.Hf = w.H;
  a.last = (max_levels == 1);
  level_eig_kernel<<<nb, LT, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  level_backtransform_kernel<<<gbt, BTW * 32, bt_smem, st>>>(n, a.Zs, a.V, a.vb, cur, w.ls, 1,
                                                             bs.fs, bs.nn, bs.ls);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  nl += 2;
  const dim3 g8((unsigned)ceil_div(n, 8), (unsigned)ceil_div(n, 8), nb);
  for (int lev = 1; lev < max_levels; ++lev) {
    // H_l = X^T H X (FP64); both products are no-ops once a problem's levels are done
    if ((e = dgemm_batched_launch(false, n, n, n, 1.0, w.H, n, bs.nn, cur, n, bs.nn, 0.0, nullptr, n,
                                  0, w.W, n, bs.nn, w.ls, bs.ls, bs.count, st)))
      return e;
    if ((e = dgemm_batched_launch(true, n, n, n, 1.0, cur, n, bs.nn, w.W, n, bs.nn, 0.0, nullptr, n,
                                  0, w.S, n, bs.nn, w.ls, bs.ls, bs.count, st)))
      return e;
    a.Hf = w.S;
    a.last = (lev == max_levels - 1);
    level_eig_kernel<<<nb, LT, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    level_backtransform_kernel<<<gbt, BTW * 32, bt_smem, st>>>(n, a.Zs, a.V, a.vb, w.R, w.ls, 0,
                                                               bs.fs, bs.nn, bs.ls);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    level_update_kernel<<<g8, 64, 0, st>>>(n, cur, w.R, nxt, w.ls, bs.nn, bs.ls);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    nl += 5;
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  *launches = nl;
  return cudaSuccess;
}

}  // namespace psvd
