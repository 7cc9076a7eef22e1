// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "psvd.h"

namespace psvd {

// Largest panel width n = K + B handled by the single-CTA eigen-solver (its packed
// symmetric matrix plus eigenvector matrix, FP32, must fit in 227 KB of shared memory).
constexpr int kMaxN = 192;
// Extra eigenpairs refined beyond the kept K (covers the truncation boundary).
constexpr int kRefineMargin = 8;
// Scale levels of the small eigen-solve launched per update (device-side early exit).
constexpr int kMaxLevels = 4;

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }

// ---------------------------------------------------------------- FP32 SIMT path
// Panel [U | A]: U is M x kc FP32 (ldu), A is M x B (lda) of type TA.
struct PanelF32 {
  const float* U;
  int64_t ldu;
  int kc;
  const void* A;
  int64_t lda;
  int a_bf16;  // 1: A is bfloat16, 0: float
  int64_t M;
  int n;  // kc + B
  // set by the Gram launchers: 1 when a BF16 A cannot be read as 4-byte row pairs
  // (odd leading dimension or base), so its rows are loaded one at a time
  int a_pairs_unaligned = 0;
};

// Number of row chunks and partial-buffer doubles used by gram_simt for a panel,
// sized for about ctas_per_sm resident CTAs per SM over the Gram's 64 x 64 blocks.
void gram_simt_plan(int64_t M, int n, int num_sms, int* nchunk, int64_t* rows_per_chunk,
                    int64_t* partial_doubles, int ctas_per_sm = 4);
// Partial Grams of the panel over row chunks (FP64 per chunk, float-float inside).
cudaError_t gram_simt_launch(const PanelF32& p, int nchunk, int64_t rows_per_chunk,
                             double* partial, cudaStream_t st);
// Gram of row blocks of one panel in one launch (Algorithm 2's local Grams): a work
// list of row chunks [r0, r1) with the chain length of their block.
struct GramItem {
  int64_t r0, r1;
  int fold_steps;
};
// Chunks for the row blocks [off[b], off[b+1]) of an n-column panel, about 4 CTAs per
// SM in all; first[b] is block b's first item (first[nparts] = the item count).
void gram_items_plan(const int64_t* off, int nparts, int n, int num_sms, std::vector<GramItem>* items,
                     std::vector<int>* first, int64_t* partial_doubles);
// Partials of the items (device work list) of the panel p (p.M = all rows).
cudaError_t gram_items_launch(const PanelF32& p, const GramItem* items, int nitems, double* partial,
                              cudaStream_t st);
// H_z (n x n, stride sH) = fixed-order sum of the partials of items [first[z], first[z+1])
// (first: device array), z < count; non-finite entries set bit 4 of info[4 z + 2].
cudaError_t gram_reduce_items_launch(const double* partial, const int* first, int count, int n,
                                     double* H, int64_t sH, int* info, cudaStream_t st);
// G = sum of partials (fixed order), H = S G S with S = diag(ff*D[0:kc], 1).
// G may be null.  ldg = ldh = n.  A non-finite Gram entry sets info[2] bit 4.
cudaError_t gram_reduce_launch(const double* partial, int nchunk, int n, int kc,
                               const double* D, double ff, double* G, double* H, int* info,
                               cudaStream_t st);
// Unew (M x k1, ldo) = [U | A] * T (n x k1, FP32, ldt = n), in tiles of tile_rows
// (64, 128 or 256) rows by the narrowest of 16, 32 or 64 columns covering k1.
cudaError_t update_simt_launch(const PanelF32& p, const float* T, int k1, float* Unew,
                               int64_t ldo, cudaStream_t st, int tile_rows = 128);

// Tile choices of the FP32 path (psvd_autotune picks them per panel shape).
struct SimtTune {
  int gram_ctas_per_sm = 4;
  int update_rows = 128;
};

// ---------------------------------------------------------------- FP64 SIMT path
// Panel [U | A]: U is M x kc FP64 (ldu), A is M x B (lda) of psvd_dtype a_dtype.
struct PanelF64 {
  const double* U;
  int64_t ldu;
  int kc;
  const void* A;
  int64_t lda;
  int a_dtype;  // PSVD_F32, PSVD_BF16 or PSVD_F64
  int64_t M;
  int n;  // kc + B
};
// Partial Grams over row chunks (chunks as gram_simt_plan), FP64 throughout; the
// partial layout is gram_simt's, so gram_reduce_launch sums them.
cudaError_t gram_f64_launch(const PanelF64& p, int nchunk, int64_t rows_per_chunk, double* partial,
                            cudaStream_t st);
// Unew (M x k1 FP64, ldo) = [U | A] * T (n x k1, FP64, ldt = n).
cudaError_t update_f64_launch(const PanelF64& p, const double* T, int k1, double* Unew, int64_t ldo,
                              cudaStream_t st);
// out (M x k FP32, ldo) = U rounded to FP32.
cudaError_t modes_f64_to_f32_launch(const double* U, int64_t ldu, int64_t M, int k, float* out,
                                    int64_t ldo, cudaStream_t st);

// ------------------------------------------------------------- small solve
// Device-side progress of the level-by-level eigen-solve (small_eig.cu).
struct LevelState {
  int b;        // leading eigenpairs resolved so far
  int b0;       // first column of the block the last level solved
  int active;   // 1 while another level is needed
  int skip;     // 1 when the last level kernel produced no transform
  int r;        // eigenpairs resolved by the last level
  int levels;   // levels run
  int floored;  // 1 when the levels stopped at the resolution floor
  double lmax;  // largest eigenvalue of H
};

// Batched small solves: `count` independent problems of the same size, problem z's
// arrays at the SmallWork pointers plus z times these element strides (count = 1:
// one problem, strides unused).
struct SmallBatch {
  int count = 1;
  int64_t nn = 0;    // H, X, W, S, R, E, Xn (each n x n)
  int64_t n = 0;     // lam, lamJ
  int64_t T = 0;     // T (FP32)
  int64_t T64 = 0;   // T64
  int64_t Dnew = 0;  // Dnew
  int64_t info = 0;  // info (ints)
  int64_t ls = 0;    // ls (LevelState elements)
  int64_t fs = 0;    // fs (floats)
};

struct SmallWork {
  double* H;      // n x n FP64 (scaled Gram), ld n
  double* X;      // n x n FP64 eigenvector estimates (sorted), ld n
  double* lam;    // n eigenvalue estimates (sorted, descending)
  double* W;      // n x nJ scratch
  double* S;      // n x nJ
  double* R;      // n x nJ
  double* E;      // n x nJ
  double* Xn;     // n x nJ
  double* lamJ;   // nJ refined eigenvalues
  float* T;       // n x K FP32 update coefficients
  __nv_bfloat16* T3;  // (3 n) x K BF16 triple split of T (tensor-core path)
  double* Dnew;   // K new singular values
  int* info;      // device int[4]: levels, resolved count, status, k1
  LevelState* ls; // level-solve progress
  float* fs;      // FP32 scratch of the level solve (eig_levels_scratch_floats)
  double* T64;    // optional (may be null): n x K FP64 copy of T
  // Resolution of the Gram relative to lambda_max: eigenvalues below it are not
  // resolved (modes zeroed, PSVD_WARN_RANK_DEFICIENT).  0 means 1e-9 (the FP32 and
  // tensor-core Grams); FP64 Grams resolve far deeper.
  double lam_floor;
  SmallBatch bat;  // several problems in each launch (small_solve_launch)
};
__host__ __device__ inline double lambda_floor(const SmallWork& w) {
  return w.lam_floor > 0.0 ? w.lam_floor : 1e-9;
}

// Eigen-decomposition of H (n x n) and the update coefficients:
//   H = X diag(lam) X^T (descending), sigma = sqrt(lam[0:k1]),
//   T = S X[:, 0:k1] diag(1/sigma), Dnew = sigma.
// *launches receives the number of kernels enqueued.
cudaError_t small_solve_launch(const SmallWork& w, int n, int kc, int k1, const double* D,
                               double ff, int refine_steps, int max_levels, cudaStream_t st,
                               int* launches);
// Eigenvectors and eigenvalues of H (n x n, w.H) by FP32 tridiagonal solves on
// successive scale levels with FP64 projections between them: w.X (n x n) holds
// the basis, w.lam the eigenvalue estimates (descending); the leading nJ are
// resolved to ~u32 / 1e-3 relative accuracy.  Uses w.W, w.S, w.R, w.Xn, w.fs, w.ls.
cudaError_t eig_levels_launch(const SmallWork& w, int n, int nJ, int max_levels, cudaStream_t st,
                              int* launches);
size_t eig_levels_scratch_floats(int nmax);
// Batched FP64 GEMM: for z < count, C_z (m x nn) = alpha op(A_z) B_z + beta Cin_z with
// X_z = X + z * sX (element strides), skipped for problem z when ls != null and
// ls[z * sls].active == 0.
cudaError_t dgemm_batched_launch(bool trans_a, int m, int nn, int k, double alpha, const double* A,
                                 int lda, int64_t sA, const double* B, int ldb, int64_t sB,
                                 double beta, const double* Cin, int ldci, int64_t sCin, double* C,
                                 int ldc, int64_t sC, const LevelState* ls, int64_t sls, int count,
                                 cudaStream_t st);
// C (m x nn) = alpha * op(A) * B + beta * Cin (FP64, column-major), op(A) = A or A^T.
cudaError_t dgemm_launch(bool trans_a, int m, int nn, int k, double alpha, const double* A, int lda,
                         const double* B, int ldb, double beta, const double* Cin, int ldci,
                         double* C, int ldc, cudaStream_t st);
// FP64 Cholesky R^T R = G (n x n) into R (ld n, upper); info[2] = status.
cudaError_t cholesky_launch(const double* G, int n, double* R, int* info, cudaStream_t st);

// ------------------------------------------------- randomized range finder
struct RandWork {
  float* Om;      // n x l Gaussian sketch (FP32)
  double* B[3];   // n x l FP64 coefficient bases / products
  double* Mm;     // l x l metric Gram of a basis
  double* Rr;     // l x l pivoted Cholesky factor (row k, original column j)
  double* Aw;     // l x l working matrix (used when l exceeds the shared-memory limit)
  int* piv;       // l pivot order
  int* rank;      // 1 numerical rank of the last pivoted Cholesky
  double* Bb;     // l x l  B B^T of the projected panel
  float* Tupd;    // n x K FP32 update coefficients (ld n)
  double* sgn;    // K signs of the new modes
};
// Randomized rank-k1 SVD of the panel whose scaled Gram H = S G S sits in w.H
// (n x n): Gaussian sketch of l columns (Philox stream sketch_id), q power
// iterations; writes the update coefficients r.Tupd (U_new = [U | A] T_upd) and
// the singular values w.Dnew.  Uses w's eigen-solver scratch.
cudaError_t randomized_solve_launch(const RandWork& r, const SmallWork& w, int n, int kc, int k1,
                                    int l, int q, const double* D, double ff, uint64_t seed,
                                    uint64_t sketch_id, cudaStream_t st, int* launches);

// Randomized rank-k SVD of an explicit N x m FP64 matrix W (N <= 192, any m):
// Halko, Martinsson & Tropp Alg. 4.4 with the Gaussian sketch Omega (m x l, Philox
// stream sketch_id of seed), Y = W Omega, Q = orth(Y) and q power steps written
// through WW = W W^T (N x N FP64; span(W W^T Q) = span(W orth(W^T Q))), then the
// eigen-solve of Q^T W W^T Q (l x l).  Outputs Tout (N x k FP64, ld N) =
// X diag(1/s) with X = Q U_B the left singular vectors, w.Dnew = s (k); w.T64 (l x k)
// is scratch.  r.Om holds m x l floats and r.B[0] m x l doubles; r.B[1], r.B[2]
// N x l; r.Mm, r.Rr, r.Aw, r.Bb l x l.
cudaError_t randomized_wide_launch(const RandWork& r, const SmallWork& w, const double* W,
                                   const double* WW, int N, int m, int k, int l, int q,
                                   uint64_t seed, uint64_t sketch_id, double* Tout,
                                   cudaStream_t st, int* launches);

// ------------------------------------------------------------------- APMOS
// Algorithm 2 on device data: A (Mtot x N, lda, FP32 or BF16) in row blocks
// [off[b], off[b+1]) (host array), r1 local and r2 global modes; U (Mtot x r2,
// FP32, ldu) and L (r2, FP64) on the device.  *status receives the accumulated
// status bits (1 rank deficient, 4 non-finite).  Workspaces, lane streams and the
// captured launch graph live in the cache; synchronises the stream.
struct ApmosCache;
ApmosCache* apmos_cache_create();
void apmos_cache_destroy(ApmosCache* c);
// With low_rank set, the global SVD of the gathered W = [V_b S_b] is the paper's
// low_rank_svd: randomized, l = min(r2 + p, N, r1 nparts) sketch columns from the
// Philox stream kApmosSketchStream of seed, q power steps; each local factor
// column is signed so that its entries sum to >= 0 (the sketch depends on signs).
constexpr uint64_t kApmosSketchStream = 0x41504D4F53ull;
int apmos_run(const void* A, int64_t lda, int a_bf16, int64_t Mtot, const int64_t* off, int nparts,
              int N, int r1, int r2, float* U, int64_t ldu, double* L, int num_sms,
              cudaStream_t st, ApmosCache* cache, int low_rank, int p, int q, uint64_t seed,
              int* status);

// ------------------------------------------------------------------ adjoint
// Reverse-mode derivative of one update of Algorithm 1 (adjoint.cu).  Inputs: the
// step's panel pieces U (M x kc FP32; kc = 0 at the initialisation), D (kc), A
// (M x B, FP32 or BF16), its outputs U' (M x k1 FP32) and D' (k1), and their
// cotangents Ybar (M x k1 FP32) and sbar (k1).  Outputs Ubar (M x kc), Dbar (kc),
// Abar (M x B, FP32).  M-sized arrays are device pointers; D, D', sbar and Dbar may
// be host or device.  Workspaces live in the AdjWork; synchronises the stream.
// *status receives bits: 1 two kept singular values coincide, 2 a kept singular
// value meets a dropped one, 4 a non-finite coefficient.
struct AdjWork;
AdjWork* adj_work_create();
void adj_work_destroy(AdjWork* w);
int adjoint_run(AdjWork* aw, cudaStream_t st, int num_sms, int64_t M, double ff, int kc,
                const float* U, int64_t ldu, const double* D, const void* A, int64_t lda,
                int a_bf16, int B, int k1, const float* Unew, int64_t ldun, const double* Dnew,
                const float* Ybar, int64_t ldyb, const double* sbar, float* Ubar, int64_t ldub,
                double* Dbar, float* Abar, int64_t ldab, int* status);

// -------------------------------------------------------------------- Philox
cudaError_t gaussian_sketch_launch(uint64_t seed, uint64_t stream_id, int64_t rows, int64_t cols,
                                   float* out, cudaStream_t st);

// ---------------------------------------------------------------- misc kernels
cudaError_t copy_modes_f32_launch(const float* U, int64_t ldu, int64_t M, int k, float* out,
                                  int64_t ldo, cudaStream_t st);

}  // namespace psvd
