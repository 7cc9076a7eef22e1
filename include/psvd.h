/*
 * psvd.h - C-ABI of the GB300-native streaming, partitioned, randomized SVD
 * (Maulik & Mengaldo, "PyParSVD", arXiv 2108.08845).
 *
 * One handle holds one stream of snapshots: the current left singular vectors
 * (modes) U (M x k, k <= K) and singular values D (k) of Algorithm 1 (Sec. 3.1).
 * Every compute step runs in the library's own CUDA kernels for sm_103a; there is
 * no host or library fallback.
 *
 * Conventions shared by all entry points
 *   - Matrices are column-major: element (i, j) of a matrix with leading
 *     dimension ld is at ptr[i + j*ld].  Rows are grid points (degrees of
 *     freedom), columns are snapshots (Sec. 3.1/3.2), so each snapshot is
 *     contiguous.
 *   - Data pointers may be device pointers or host pointers (pageable or
 *     pinned); the library detects which with cudaPointerGetAttributes.  Host
 *     inputs are staged through a device buffer owned by the handle.  On the
 *     tensor-core path, device inputs whose base address or leading dimension
 *     (in bytes) is not a multiple of 16 are also re-staged (one extra copy);
 *     aligned inputs are read in place.
 *   - Work is enqueued on the handle's CUDA stream.  Calls that return data to
 *     the caller (psvd_get_*, psvd_parallel_qr, psvd_parallel_svd) synchronise
 *     that stream before returning.  Calls that only consume inputs
 *     (psvd_initialize, psvd_incorporate_data) return as soon as the work is
 *     enqueued when the input is a device pointer; the caller must keep device
 *     inputs alive and unmodified until the stream reaches that point.
 *   - Ownership: the caller owns every pointer it passes; the handle owns its
 *     modes, singular values, workspaces and random-number state.
 *   - Errors: every int-returning call returns PSVD_OK (0), a positive warning,
 *     or a negative error code; no exception or abort crosses the ABI.  After a
 *     PSVD_ERR_CUDA the handle must be destroyed.
 *   - Threading: a handle is not thread-safe; distinct handles are independent.
 */
#ifndef PSVD_H
#define PSVD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define PSVD_OK 0
#define PSVD_WARN_RANK_DEFICIENT 1   /* a kept singular value is (numerically) zero;
                                        its mode is set to zero (Alg. 2, Lambda_j = 0) */
#define PSVD_WARN_NOT_CONVERGED 2    /* the small eigen-solve used all of its scale levels
                                        (4; 6 on a PSVD_PREC_FP64 handle) before it had
                                        resolved the K + 8 leading eigenpairs of the
                                        scaled Gram down to the Gram's resolution floor
                                        (1e-9 of the largest eigenvalue; 1e-13 for FP64);
                                        the unresolved kept pairs carry only the FP32
                                        accuracy of the last level */
#define PSVD_WARN_DEGENERATE 3       /* psvd_update_adjoint: two kept singular values, or
                                        the last kept and the first dropped one, coincide
                                        (to 1e-13 relative in s^2); the derivative is
                                        undefined and the returned one is not meaningful */
#define PSVD_ERR_INVALID_ARG -1      /* null handle/pointer, ld < M, bad enum, ff not in (0,1] */
#define PSVD_ERR_NOT_INITIALIZED -2  /* psvd_incorporate_data / get before psvd_initialize */
#define PSVD_ERR_SHAPE -3            /* B > max_batch, M < K + B, K + max_batch > 192, ... */
#define PSVD_ERR_NONFINITE -4        /* a NaN or Inf reached the small factor */
#define PSVD_ERR_CUDA -5             /* a CUDA runtime call failed */
#define PSVD_ERR_ALLOC -6            /* device or host allocation failed */
#define PSVD_ERR_IO -7               /* psvd_save / psvd_load file error or bad format */
#define PSVD_ERR_UNSUPPORTED -8      /* feature not available for this precision/shape */
#define PSVD_ERR_TIMEOUT -9          /* a device-side wait exceeded its time budget; the
                                        kernel abandoned its work (results are invalid) */

/* ----------------------------------------------------------------- enums */
typedef enum {
  PSVD_F32 = 0,  /* IEEE binary32 */
  PSVD_BF16 = 1, /* bfloat16 (8-bit exponent, 7-bit fraction) */
  PSVD_F64 = 2   /* IEEE binary64: the small outputs, and snapshots of a
                    PSVD_PREC_FP64 handle */
} psvd_dtype;

typedef enum {
  /* "plain FP32": panel Gram and mode update on the FP32 CUDA cores with
     compensated (float-float) accumulation and an FP64 cross-block reduction;
     modes stored in FP32. */
  PSVD_PREC_FP32 = 0,
  /* tcgen05 tensor cores: snapshots in BF16, modes stored as a BF16 hi/lo pair
     (16 significant bits), panel Gram and mode update on the tensor cores with
     FP32 accumulation in tensor memory and an FP64 cross-block reduction. */
  PSVD_PREC_BF16_TC = 1,
  /* FP64 CUDA cores: modes stored in FP64, panel Gram and mode update in FP64
     (snapshots PSVD_F32, PSVD_BF16 or PSVD_F64, widened exactly).  The
     full-precision reference on the device: FP64 runs at a small fraction of
     the FP32 rate on this GPU.  No randomized front end (low_rank must be 0). */
  PSVD_PREC_FP64 = 2
} psvd_precision;

/* --------------------------------------------------------------- config */
typedef struct {
  int64_t M;          /* rows (grid points) of every snapshot, >= 1 */
  int32_t K;          /* modes kept after every batch (Alg. 1 steps 3 and 5), >= 1 */
  int32_t max_batch;  /* largest snapshot count B per call; K + max_batch <= 192;
                         PSVD_PREC_BF16_TC also needs K <= 80 and
                         2*roundup(K,8) + roundup(max_batch,8) <= 256 */
  double ff;          /* forget factor in (0, 1] (Sec. 3.1): scales U*D, i.e. sigma */
  int32_t precision;  /* psvd_precision */
  int32_t low_rank;   /* 1: the SVD of each panel is the randomized low-rank SVD
                         of Sec. 3.3 (range finder Y = P*Omega, Omega Gaussian
                         n x l, n = k + B); 0: exact.  PSVD_PREC_FP32 or
                         PSVD_PREC_BF16_TC (PSVD_ERR_UNSUPPORTED with FP64). */
  int32_t oversample; /* p >= 0: the sketch has l = min(K + p, k + B) columns */
  int32_t power_iters;/* q in [0, 16]: power iterations of the range finder */
  uint64_t seed;      /* Philox4x32-10 key of the Gaussian sketches: the sketch of
                         batch t (t = 0 for psvd_initialize) is
                         psvd_gaussian_sketch(seed, t, n, l) */
  void* stream;       /* cudaStream_t the handle enqueues on; NULL = default stream */
} psvd_config;

typedef struct psvd_ctx* psvd_handle;

/* psvd_create: allocates a handle for config *cfg (copied).  Device memory:
 * two M x K mode buffers (FP32, a BF16 hi/lo pair, or FP64) plus O(M) staging
 * and O((K+max_batch)^2) workspaces.  *out is set to NULL on failure. */
int psvd_create(psvd_handle* out, const psvd_config* cfg);

/* psvd_destroy: synchronises the handle's stream and frees everything it owns.
 * Null is a no-op. */
void psvd_destroy(psvd_handle h);

/* psvd_initialize: Algorithm 1 steps I1-I2 (Sec. 3.1) on the first batch
 * A0 (M x B, leading dimension lda >= M, dtype PSVD_F32 or PSVD_BF16, or
 * PSVD_F64 on a PSVD_PREC_FP64 handle; the tensor-core path takes PSVD_BF16):
 * QR of A0, SVD of R, U0 = Q U' truncated to k = min(K, B) modes.
 * Implemented as the Gram of A0, its eigen-decomposition, and U0 = A0 V D^-1. */
int psvd_initialize(psvd_handle h, const void* A0, int64_t lda, int32_t B, int32_t dtype);

/* psvd_incorporate_data: Algorithm 1 steps 1-5 (Sec. 3.1) for one new batch
 * A (M x B, lda >= M, B <= max_batch, M >= k + B): QR of [ff*U*D | A], SVD of
 * its R, keep min(K, k+B) modes, U <- Q U~.  The panel is never materialised:
 * its Gram [U|A]^T[U|A] is scaled by diag(ff*D, 1) on the small side. */
int psvd_incorporate_data(psvd_handle h, const void* A, int64_t lda, int32_t B, int32_t dtype);

/* psvd_incorporate_batches: psvd_incorporate_data on `count` batches in order,
 * A[0], ..., A[count-1] (host array of pointers; each batch M x B with leading
 * dimension lda and the given dtype, device or host memory).  Host batches are
 * copied to the device on a copy stream of the handle into two alternating staging
 * buffers, so the copy of batch i+1 runs while batch i is processed (pinned host
 * memory makes the copies asynchronous; pageable memory still works, with less
 * overlap); the result is then bit for bit that of the count single calls, as on
 * the FP32 and FP64 paths.  On the tensor-core path, when batch i+1 is in device
 * memory (16-byte aligned base and lda * 2) and the panel splits as one mode slab
 * and one snapshot slab (2 * roundup(K, 8) == 128, B <= 128), its A^T A block is
 * summed on a side stream of the handle while batch i's small solve runs and its
 * Gram computes only the blocks with the modes: the same Gram in another
 * summation order, so the result agrees with the single calls to rounding, not
 * bit for bit.  Every side-stream launch is joined back into the handle's stream
 * before the call's last batch is done.  s_out (may be
 * null; host or device, FP64, count x K with leading dimension K) receives each
 * batch's singular values (the current mode count of them, descending) as soon as
 * that batch is done.  Returns after enqueuing; the caller keeps every batch and
 * s_out valid until the handle's stream has finished (psvd_get_* or a stream
 * synchronisation).  Every batch is checked before the first is enqueued, so an
 * argument or shape error (as for psvd_incorporate_data) leaves the handle
 * unchanged; a CUDA error part-way leaves the batches before it applied.  A
 * pageable host s_out makes each read synchronous, which stalls the pipeline. */
int psvd_incorporate_batches(psvd_handle h, const void* const* A, int32_t count, int64_t lda,
                             int32_t B, int32_t dtype, double* s_out);

/* psvd_parallel_qr: the R factor of the row-partitioned QR of Sec. 4.2 for a
 * tall panel P (M x n, ldp >= M, n <= K + max_batch, dtype F32 or BF16), with
 * the handle's M.  R (n x n, upper triangular, diag >= 0) is written to R_out
 * (column-major, leading dimension n, FP64; host or device).  R is the
 * Cholesky factor of the panel's Gram, computed in FP64 from the Gram that the
 * update kernels use.  Returns PSVD_ERR_NONFINITE if the Gram is not positive
 * definite. */
int psvd_parallel_qr(psvd_handle h, const void* P, int64_t ldp, int32_t n, int32_t dtype,
                     double* R_out);

/* psvd_parallel_svd: Algorithm 2 (APMOS, Sec. 3.2) on the row blocks
 * [part_offsets[b], part_offsets[b+1]) of A (Mtot x N, lda >= Mtot; dtype F32
 * or BF16), part_offsets a host array of nparts+1 increasing values with
 * part_offsets[0] = 0 and part_offsets[nparts] = Mtot; every block needs
 * >= N rows.  Local right singular vectors (r1 kept per block), gather of
 * W = [V~^1 S~^1, ...], SVD of W (r2 kept), then U~^b_j = A^b X~_j / L~_j.
 * Outputs: U_out (Mtot x r2, FP32, ldu >= Mtot), L_out (r2, FP64, descending),
 * host or device.  N <= 192, r1 <= N, r2 <= min(N, r1*nparts).  Runs on the
 * FP32 path for either handle precision and uses the handle for its stream,
 * staging buffer and randomization settings: with low_rank set, the SVD of W is
 * the paper's low_rank_svd (Listing 3), a randomized SVD with l = min(r2 +
 * oversample, N, r1*nparts) Gaussian sketch columns from Philox stream
 * 0x41504D4F53 of the handle's seed and power_iters power steps, each local factor
 * column signed so that its entries sum to >= 0.  Its workspaces (one per concurrent lane: the
 * blocks' local solves run on up to 16 streams of the handle's own) are kept
 * by the handle after the first call and grown when a call needs more.  The
 * launch sequence is captured into a CUDA graph on the first call with a given
 * argument set and replayed by later calls with the same pointers and sizes.
 * The call synchronises the stream.  Returns PSVD_WARN_RANK_DEFICIENT when a kept
 * L~_j is numerically zero (that mode is returned as zero). */
int psvd_parallel_svd(psvd_handle h, const void* A, int64_t lda, const int64_t* part_offsets,
                      int32_t nparts, int32_t N, int32_t dtype, int32_t r1, int32_t r2,
                      float* U_out, int64_t ldu, double* L_out);

/* psvd_parallel_qr_static: the same R factor as psvd_parallel_qr, computed
 * without allocating anything (the paper has no counterpart: this serves
 * callers that cannot allocate device memory when they need the factor, e.g.
 * a process whose device memory is reserved by another allocator, or a
 * latency-critical loop where cudaMalloc's implicit device synchronisation
 * would stall other streams).  No handle is needed.
 *   P      pointer to the panel in the current device's memory (or managed
 *          memory), M x n column-major, ldp >= M, dtype PSVD_F32 or PSVD_BF16;
 *          host pointers (no staging buffer to copy them into) and pointers to
 *          another GPU's memory are rejected with PSVD_ERR_INVALID_ARG
 *   R_out  n x n FP64, leading dimension n, upper triangular with diag >= 0
 *          (host or device); stream: cudaStream_t, NULL = default stream
 * Limits: n <= 128 and M >= n, else PSVD_ERR_SHAPE.  Scratch: a 3.4 MB
 * file-scope device array (the Gram's row-chunk partials, the Gram and a
 * status word) that every GPU loading the library holds until the process
 * exits.  The first call on a device looks up the array's device address
 * (once per device); make that first call before any stream capture.  All
 * calls share the one array and every call overwrites it, so calls whose work
 * overlaps on the GPU (different streams or host threads) race: serialise
 * them.  The call synchronises `stream` before returning.  Returns
 * PSVD_ERR_NONFINITE if the Gram is not positive definite. */
int psvd_parallel_qr_static(const void* P, int64_t ldp, int64_t M, int32_t n, int32_t dtype,
                            double* R_out, void* stream);

/* psvd_get_modes: copies the current modes (M x k, FP32; a BF16 hi/lo pair is
 * summed exactly, FP64 modes are rounded) into U_out (ldu >= M, host or device). */
int psvd_get_modes(psvd_handle h, float* U_out, int64_t ldu);

/* psvd_get_modes_f64: the current modes of a PSVD_PREC_FP64 handle (M x k, FP64)
 * into U_out (ldu >= M, host or device); PSVD_ERR_UNSUPPORTED for the other
 * precisions.  Synchronises the handle's stream. */
int psvd_get_modes_f64(psvd_handle h, double* U_out, int64_t ldu);

/* psvd_get_singular_values: copies the current k singular values (descending,
 * FP64) into s_out (host or device). */
int psvd_get_singular_values(psvd_handle h, double* s_out);

/* psvd_num_modes: current mode count k (0 before psvd_initialize), or < 0. */
int psvd_num_modes(psvd_handle h);

/* psvd_save: writes (config, iteration, k, D, U as FP32, Philox counter; the
 * BF16 hi/lo planes or the FP64 modes of those precisions) to a binary file;
 * psvd_load recreates a handle from it on the given stream.  A loaded handle
 * continues bit-identically to the one that was saved. */
int psvd_save(psvd_handle h, const char* path);
int psvd_load(psvd_handle* out, const char* path, void* stream);

/* psvd_gaussian_sketch: the Philox4x32-10 Gaussian test matrix of Sec. 3.3
 * used by the randomized path: out (rows x cols, column-major, ld = rows,
 * FP32, device) gets variates i + j*rows of stream (seed, stream_id), each a
 * Box-Muller transform computed in FP64 from IEEE-exact operations and rounded
 * to FP32.  Enqueued on `stream` (cudaStream_t, NULL = default). */
int psvd_gaussian_sketch(uint64_t seed, uint64_t stream_id, int64_t rows, int64_t cols,
                         float* out, void* stream);

/* Adjoint (reverse-mode derivative) of one step of Algorithm 1 (Sec. 3.1, steps 1-5),
 * or of the initialisation I1-I2 when kc = 0: the hand-written backward of the
 * panel factorisation and truncated SVD of R, with the 1/(s_i^2 - s_j^2) terms.
 *
 * The forward step maps P = [ff U diag(D) | A] (M x n, n = kc + B; P = A when
 * kc = 0) to its leading k1 left singular vectors U_new and singular values D_new
 * (what psvd_initialize / psvd_incorporate_data computed, read back with
 * psvd_get_modes / psvd_get_singular_values).  Given the cotangents U_new_bar
 * (M x k1) and D_new_bar (k1) of a scalar loss, this returns the cotangents of the
 * step's inputs:  U_bar (M x kc), D_bar (kc) and A_bar (M x B).  Q is not kept:
 * the right singular vectors are recovered from U_new (V_k = P^T U_new / D_new) and
 * the dropped directions enter through shifted FP64 solves on the (n x n) Gram, so
 * a sweep over a run needs only the per-step modes and singular values.
 *
 * Arguments: M and ff are the handle's; U (FP32, ldu), A (dtype PSVD_F32 or
 * PSVD_BF16, lda), U_new, U_new_bar (FP32) and the outputs U_bar, A_bar (FP32) are
 * DEVICE pointers with leading dimensions >= M; D, D_new, D_new_bar, D_bar (FP64)
 * may be host or device.  U, D, U_bar, D_bar may be null when kc = 0.
 * kc + B <= 192, 1 <= k1 <= min(kc + B, 64), M >= kc + B.  The handle's stream is
 * used and synchronised; workspaces are kept by the handle.  Arithmetic: FP32
 * panel passes (float-float row sums, FP64 reduction), FP64 small side.
 * Returns PSVD_OK, PSVD_WARN_DEGENERATE, PSVD_ERR_NONFINITE, or an argument /
 * CUDA / allocation error (outputs then undefined). */
int psvd_update_adjoint(psvd_handle h, int32_t kc, const float* U, int64_t ldu, const double* D,
                        const void* A, int64_t lda, int32_t B, int32_t dtype, int32_t k1,
                        const float* U_new, int64_t ld_new, const double* D_new,
                        const float* U_new_bar, int64_t ld_new_bar, const double* D_new_bar,
                        float* U_bar, int64_t ld_bar, double* D_bar, float* A_bar,
                        int64_t lda_bar);

/* psvd_autotune: picks this handle's launch shapes for its steady-state panel (M
 * rows, n = K + B columns) by timing the candidates on the handle's stream with a
 * representative batch A (DEVICE pointer, M x B, lda >= M).  The fastest of each
 * is kept by the handle and cached for the process under the shape and SM count, so
 * later calls with the same shape take it without timing.
 *   FP32 handles (A PSVD_F32 or PSVD_BF16): Gram row chunks sized for 1, 2, 4 or
 *   8 resident CTAs per SM, and mode-update tiles of 64, 128 or 256 rows; choice
 *   receives {CTAs per SM, update tile rows, 0}.
 *   Tensor-core handles (A PSVD_BF16): the Gram's cluster count (the resident
 *   maximum, 2/3, 1/2 or 1/3 of it), the update's CTA count (one per SM or half
 *   of that) and its pipeline stages (2 to 4, those that fit in shared memory at
 *   this panel width); choice receives {Gram clusters, update CTAs, update
 *   stages}.
 * The Gram choices change only the summation order of its row partial sums
 * (results stay within the same rounding bounds); the update choices leave the
 * results unchanged.  choice may be null, else int32_t[3].  FP64 handles:
 * PSVD_ERR_UNSUPPORTED.  Synchronises; the handle's modes, singular values and
 * status are unchanged.  Call it between updates; a group whose member was retuned
 * captures its graphs again. */
int psvd_autotune(psvd_handle h, const void* A, int64_t lda, int32_t B, int32_t dtype,
                  int32_t* choice);

/* ------------------------------------------------------------------ groups
 * Many independent snapshot streams updated together (the batching form of the
 * method: one Algorithm 1 state per stream).  psvd_group_create makes `count`
 * handles with the same configuration, each on a CUDA stream of its own; cfg->stream
 * is the stream the group's calls are ordered on (their work starts after the
 * caller's earlier work on it, and later work on it waits for theirs).
 *
 * psvd_group_initialize / psvd_group_incorporate_data apply psvd_initialize /
 * psvd_incorporate_data to every member i with its own batch A[i] (A: host array
 * of `count` pointers; each batch M x B, leading dimension lda, dtype as for the
 * single-handle calls).  The members' update sequences run concurrently.  Once
 * every member holds K modes (and the handles use neither the randomized front
 * end nor the tensor-core path), the fork / updates / join sequence is captured
 * into a CUDA graph, one per double-buffer parity, and replayed by later calls
 * whose batch pointers, lda, B and dtype repeat (a ring of input buffers reuses
 * the graphs; new pointers are captured anew).  The calls do not synchronise;
 * psvd_group_status reads every member's status (synchronising) and returns the
 * most severe.  Members are ordinary handles for psvd_get_modes,
 * psvd_get_singular_values, psvd_save, ... (psvd_group_member); do not update a
 * member outside the group or destroy it.  psvd_group_stats reports how many
 * calls captured a graph and how many replayed one. */
typedef struct psvd_group* psvd_group_handle;
int psvd_group_create(psvd_group_handle* out, int32_t count, const psvd_config* cfg);
void psvd_group_destroy(psvd_group_handle g);
int psvd_group_initialize(psvd_group_handle g, const void* const* A, int64_t lda, int32_t B,
                          int32_t dtype);
int psvd_group_incorporate_data(psvd_group_handle g, const void* const* A, int64_t lda,
                                int32_t B, int32_t dtype);
psvd_handle psvd_group_member(psvd_group_handle g, int32_t i);
int psvd_group_status(psvd_group_handle g);
int psvd_group_stats(psvd_group_handle g, int64_t* captures, int64_t* replays);

/* psvd_set_profiling: enable (1) or disable (0) per-phase CUDA-event timing on
 * the handle's stream and reset its counters.  Phases: 0 panel Gram (partials
 * and reduction), 1 small solve (eigen-decomposition, refinement, T), 2 mode
 * update.  Timing adds two event records per phase and nothing else. */
int psvd_set_profiling(psvd_handle h, int32_t enable);

/* psvd_get_profile: synchronises, then writes the accumulated device time of
 * each phase in milliseconds (ms_out[3]), the number of timed executions of each
 * phase (count_out[3]) and the number of kernels the handle launched since
 * profiling was enabled (*launches_out).  Any output pointer may be NULL. */
int psvd_get_profile(psvd_handle h, double* ms_out, int64_t* count_out, int64_t* launches_out);

/* psvd_debug_set_wait_budget: testing hook of the device-side failure detection
 * (no counterpart in the paper).  Every wait of the tensor-core kernels on a copy or
 * on the tensor cores is bounded (about 2 s); when a budget runs out the kernel
 * stops issuing work, waits with the full budget for the copies and matrix
 * products it has already issued, frees its tensor memory and returns, and the
 * handle reports PSVD_ERR_TIMEOUT.  This call sets the budget, in SM clock cycles,
 * of the pipeline waits of the tensor-core mode-update kernel (kernel = 1) for the
 * launches that follow, process-wide; cycles = 0 restores the default.  A budget
 * shorter than any copy's latency makes the next update time out without a fault,
 * which is how the tests exercise that path.  Returns PSVD_ERR_INVALID_ARG for
 * another kernel or a negative budget.  Not synchronised with concurrent updates. */
int psvd_debug_set_wait_budget(int32_t kernel, int64_t cycles);

/* psvd_status_string: static description of a status code. */
const char* psvd_status_string(int status);

/* psvd_last_info: diagnostics of the most recent update (synchronises): info4[0]
 * is the number of scale levels of the small eigen-solve, info4[1] the leading
 * eigenpairs they resolved before refinement, info4[2] the accumulated status
 * bits since psvd_initialize (1 rank deficient, 2 not converged, 4 non-finite,
 * 8 timeout), info4[3] the kept mode count.  info4 is a host int32[4]. */
int psvd_last_info(psvd_handle h, int32_t* info4);

#ifdef __cplusplus
}
#endif

#endif /* PSVD_H */
