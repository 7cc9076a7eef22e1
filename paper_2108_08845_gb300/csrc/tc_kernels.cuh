// tcgen05 tensor-core kernels of the BF16 path (internal).
#pragma once

#include "psvd_internal.cuh"

namespace psvd {

// Partial Grams of the panel [Uh | Ul | A] (BF16; U = Uh + Ul) over row blocks,
// written to *partial (grown if needed).  Returns a PSVD status.
int tc_gram(const __nv_bfloat16* Uh, const __nv_bfloat16* Ul, int64_t ldu, int kc, const void* A,
            int64_t lda, int B, int dtype, int64_t M, int num_sms, double** partial,
            int64_t* partial_cap, cudaStream_t st);
// G = fixed-order FP64 sum of the partials (U^T U from the hi/lo blocks), H = S G S.
cudaError_t tc_gram_reduce(const double* partial, int64_t M, int kc, int B, int num_sms, double ff,
                           const double* D, double* G, double* H, cudaStream_t st);
// [Uh_new + Ul_new] = [Uh | Ul | A] * T3 on the tensor cores (T3: BF16 triple split).
int tc_update(const __nv_bfloat16* Uh, const __nv_bfloat16* Ul, int64_t ldu, int kc, const void* A,
              int64_t lda, int B, int dtype, int64_t M, const __nv_bfloat16* T3, int n, int k1,
              __nv_bfloat16* Uh_new, __nv_bfloat16* Ul_new, int num_sms, cudaStream_t st);
// out = float(Uh) + float(Ul) (exact), M x k, ld ldu.
cudaError_t tc_modes_to_f32(const __nv_bfloat16* Uh, const __nv_bfloat16* Ul, int64_t ldu,
                            int64_t M, int k, float* out, cudaStream_t st);

}  // namespace psvd
