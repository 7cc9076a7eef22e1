// tcgen05 tensor-core kernels of the BF16 path (internal).
#pragma once

#include "psvd_internal.cuh"

namespace psvd {

// Partial Grams of the panel [Uh | Ul | A] (BF16; U = Uh + Ul) over row chunks,
// written to *partial (grown if needed).  A timed-out wait ORs 8 into *status.
// Returns a PSVD status.
int tc_gram(const __nv_bfloat16* Uh, const __nv_bfloat16* Ul, int64_t ldu, int kc, const void* A,
            int64_t lda, int B, int dtype, int64_t M, int num_sms, double** partial,
            int64_t* partial_cap, int* status, cudaStream_t st);
// G = fixed-order FP64 sum of the partials (U^T U from the hi/lo blocks), H = S G S.
cudaError_t tc_gram_reduce(const double* partial, int64_t M, int kc, int B, int num_sms, double ff,
                           const double* D, double* G, double* H, int* status, cudaStream_t st);
// BF16 elements of the packed update coefficients for K modes and batches <= maxB.
size_t tc_t3_elems(int K, int maxB);
// [Uh_new + Ul_new] = [Uh | Ul | A] * T on the tensor cores: T (n x k1 FP32, ld n) is
// split exactly into three BF16 parts packed into T3 (tc_t3_elems) first.
int tc_update(const __nv_bfloat16* Uh, const __nv_bfloat16* Ul, int64_t ldu, int kc, const void* A,
              int64_t lda, int B, int dtype, int64_t M, const float* T, int n, int k1,
              __nv_bfloat16* T3, __nv_bfloat16* Uh_new, __nv_bfloat16* Ul_new, int num_sms,
              int* status, cudaStream_t st);
// out = float(Uh) + float(Ul) (exact), M x k, ld ldu.
cudaError_t tc_modes_to_f32(const __nv_bfloat16* Uh, const __nv_bfloat16* Ul, int64_t ldu,
                            int64_t M, int k, float* out, cudaStream_t st);

}  // namespace psvd
