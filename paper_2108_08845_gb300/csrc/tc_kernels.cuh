// tcgen05 tensor-core kernels of the BF16 path (internal).
#pragma once

#include "psvd_internal.cuh"

namespace psvd {

// Modes of the tensor-core path: U = Uh + Ul (two BF16 planes) stored slot-tiled.
// For every block of 128 rows, 64-row half h and plane p (0: Uh, 1: Ul), column c
// (c < Kp = roundup(K, 8)) holds its 64 rows as one contiguous 128-byte line, so
// a run of columns of one half and plane is contiguous memory and TMA streams it
// at the HBM rate (a column-major panel, with its columns M rows apart, is
// capped well below it by address translation).  Rows beyond M are zero.
__host__ __device__ inline int64_t tc_mode_index(int64_t row, int plane, int col, int Kp) {
  return ((((row >> 7) * 2 + ((row >> 6) & 1)) * 2 + plane) * (int64_t)Kp + col) * 64 + (row & 63);
}
// BF16 elements of one tiled mode buffer (both planes) for M rows and K modes.
size_t tc_modes_elems(int64_t M, int K);
// Launch shapes of the tensor-core path chosen by psvd_autotune (0 = default):
// clusters of the Gram (at most the resident maximum), CTAs of the update (at most
// one per SM: each holds all of its SM's TMEM) and the update's pipeline stages (2
// or more, as many as fit in shared memory at the panel width).  The cluster count
// sets how the Gram's rows are split into partial sums; the update's shape does not
// change its results.
struct TcTune {
  int gram_clusters = 0;
  int upd_ctas = 0;
  int upd_stages = 2;
};
// The resident maximum of Gram clusters for the panel of kc modes and B snapshots.
int tc_gram_clusters_max(int kc, int B, int num_sms);
// The most update pipeline stages that fit in shared memory for kc modes, B
// snapshots and k1 kept modes (0 if not even two fit).
int tc_update_max_stages(int kc, int B, int k1);
// Partial Grams of the panel [Uh | Ul | A] (BF16; U = Uh + Ul, tiled as above with
// column stride Kp) over row slots, written to *partial (grown if needed).  A
// timed-out wait ORs 8 into *status.  Returns a PSVD status.
// split: only the blocks [Uh | Ul]^T [Uh | Ul] and [Uh | Ul]^T A, in clusters of two
// CTAs (tc_gram_can_split), the block A^T A coming from tc_gram_aa.
int tc_gram(const __nv_bfloat16* Ut, int Kp, int kc, const void* A, int64_t lda, int B, int dtype,
            int64_t M, int num_sms, const TcTune& tune, bool split, double** partial,
            int64_t* partial_cap, int* status, cudaStream_t st);
// Whether the panel of kc modes and B snapshots splits as [Uh | Ul] (one 128-column
// slab) and A (a second one).
bool tc_gram_can_split(int kc, int B);
// A^T A (128 x 128 FP64, entries x <= y, ld 128) of a BF16 batch into AAsum, with at
// most `clusters` CTAs (0 = as many as are resident), partials in *partial (grown
// if needed).  Returns a PSVD status.
int tc_gram_aa(const void* A, int64_t lda, int B, int64_t M, int num_sms, int clusters,
               double** partial, int64_t* partial_cap, double* AAsum, int* status,
               cudaStream_t st);
// G = fixed-order FP64 sum of the partials (U^T U from the hi/lo blocks), H = S G S.
// AAsum != null: the partials are those of a split Gram and A^T A is AAsum.
cudaError_t tc_gram_reduce(const double* partial, int64_t M, int kc, int B, int num_sms,
                           const TcTune& tune, const double* AAsum, double ff, const double* D,
                           double* G, double* H, int* status, cudaStream_t st);
// BF16 elements of the packed update coefficients for K modes and batches <= maxB.
size_t tc_t3_elems(int K, int maxB);
// Ut_new = [Uh | Ul | A] * T on the tensor cores (modes tiled, column stride Kp):
// T (n x k1 FP32, ld n) is split exactly into three BF16 parts packed into T3
// (tc_t3_elems) first.
int tc_update(const __nv_bfloat16* Ut, int Kp, int kc, const void* A, int64_t lda, int B, int dtype,
              int64_t M, const float* T, int n, int k1, __nv_bfloat16* T3, __nv_bfloat16* Ut_new,
              int num_sms, const TcTune& tune, int* status, cudaStream_t st);
// Testing hook of the device-side failure detection: the clock-cycle budget of the
// pipeline waits of tc_update_kernel (kernel = 1) for later launches; 0 = default.
int tc_set_wait_budget(int kernel, long long cycles);
// out = float(Uh) + float(Ul) (exact), M x k column-major with leading dimension ldo.
cudaError_t tc_modes_to_f32(const __nv_bfloat16* Ut, int Kp, int64_t M, int k, float* out,
                            int64_t ldo, cudaStream_t st);

}  // namespace psvd
