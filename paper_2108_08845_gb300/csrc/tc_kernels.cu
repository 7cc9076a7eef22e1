// Placeholder until the tcgen05 kernels land: the BF16 tensor-core path reports
// PSVD_ERR_UNSUPPORTED.
#include "tc_kernels.cuh"

namespace psvd {

int tc_gram(const __nv_bfloat16*, const __nv_bfloat16*, int64_t, int, const void*, int64_t, int,
            int, int64_t, int, double**, int64_t*, cudaStream_t) {
  return PSVD_ERR_UNSUPPORTED;
}
cudaError_t tc_gram_reduce(const double*, int64_t, int, int, int, double, const double*, double*,
                           double*, cudaStream_t) {
  return cudaErrorNotSupported;
}
int tc_update(const __nv_bfloat16*, const __nv_bfloat16*, int64_t, int, const void*, int64_t, int,
              int, int64_t, const __nv_bfloat16*, int, int, __nv_bfloat16*, __nv_bfloat16*, int,
              cudaStream_t) {
  return PSVD_ERR_UNSUPPORTED;
}
cudaError_t tc_modes_to_f32(const __nv_bfloat16*, const __nv_bfloat16*, int64_t, int64_t, int,
                            float*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace psvd
