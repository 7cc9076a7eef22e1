// psvd_parallel_qr_static: the R factor of psvd_parallel_qr, computed without
// allocating any memory.
//
// Some callers cannot allocate device memory at the moment they need this
// factorisation: a process whose device memory is already fully reserved by
// another allocator (for example a framework's caching allocator), a
// latency-critical loop in which cudaMalloc's implicit device synchronisation
// would stall every other stream, or a service that runs under a fixed,
// pre-committed memory budget.  This entry point serves them: its scratch (the
// Gram's chunk partials, the Gram itself and a status word) lives in a
// file-scope __device__ array that every GPU loading the library holds until the
// process exits.  The caller passes the panel and the output buffer.
#include <mutex>

#include "psvd_internal.cuh"

namespace {

// Limits of the static scratch.
constexpr int kStaticMaxN = 128;            // panel columns
constexpr int kStaticChunks = 32;           // row chunks of the Gram
constexpr int kStaticPairs = 3;             // 64-column tile pairs for n <= 128
constexpr int64_t kPartialDoubles = (int64_t)kStaticChunks * kStaticPairs * 64 * 64;
constexpr int64_t kGramDoubles = (int64_t)kStaticMaxN * kStaticMaxN;
constexpr int64_t kScratchDoubles = kPartialDoubles + 2 * kGramDoubles + 4;  // partials, G, H, status

// 3,407,904 bytes: the Gram partials (3 MiB), G and H (128 KiB each), status word.
__device__ __align__(256) double g_static_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per
// device (the host-side symbol is only a stand-in and must never reach a kernel).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return PSVD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PSVD_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PSVD_OK;
}

// True for managed memory and for device memory of the current device (the
// kernels run there; a panel on another GPU is rejected rather than read across
// the interconnect or faulted on).
bool is_current_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.device == dev;
}

}  // namespace

extern "C" int psvd_parallel_qr_static(const void* P, int64_t ldp, int64_t M, int32_t n,
                                       int32_t dtype, double* R_out, void* stream) {
  if (!P || !R_out || M < 1 || n < 1 || ldp < M) return PSVD_ERR_INVALID_ARG;
  if (dtype != PSVD_F32 && dtype != PSVD_BF16) return PSVD_ERR_INVALID_ARG;
  if (n > kStaticMaxN || M < n) return PSVD_ERR_SHAPE;
  // host panels: no staging buffer to copy them into; other GPUs: see above
  if (!is_current_device_pointer(P)) return PSVD_ERR_INVALID_ARG;
  double* scratch = nullptr;
  if (int rc = scratch_for_current_device(&scratch)) return rc;
  double* partial = scratch;
  double* G = scratch + kPartialDoubles;
  double* H = G + kGramDoubles;
  int* status = reinterpret_cast<int*>(H + kGramDoubles);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // every partial and every Gram entry is overwritten below; only the status
  // word carries state from one call to the next, so it is cleared first
  if (cudaMemsetAsync(status, 0, 4 * sizeof(int), st) != cudaSuccess) return PSVD_ERR_CUDA;
  int64_t rows = psvd::ceil_div(psvd::ceil_div(M, kStaticChunks), 32) * 32;
  const int nchunk = (int)psvd::ceil_div(M, rows);
  psvd::PanelF32 p{nullptr, 0, 0, P, ldp, dtype == PSVD_BF16 ? 1 : 0, M, n};
  if (psvd::gram_simt_launch(p, nchunk, rows, partial, st) != cudaSuccess) return PSVD_ERR_CUDA;
  if (psvd::gram_reduce_launch(partial, nchunk, n, 0, nullptr, 1.0, G, H, status, st) != cudaSuccess)
    return PSVD_ERR_CUDA;
  // R (n x n, leading dimension n) is factored in H's place, then copied out
  if (psvd::cholesky_launch(G, n, H, status, st) != cudaSuccess) return PSVD_ERR_CUDA;
  if (cudaMemcpyAsync(R_out, H, sizeof(double) * n * n, cudaMemcpyDefault, st) != cudaSuccess)
    return PSVD_ERR_CUDA;
  int host_status[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(host_status, status, sizeof(host_status), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PSVD_ERR_CUDA;
  return (host_status[2] & 4) ? PSVD_ERR_NONFINITE : PSVD_OK;
}
