// Algorithm 2 (APMOS, Sec. 3.2) on one GPU.  The paper's ranks hold row blocks
// A^b of the snapshot matrix; here the blocks are row ranges of one matrix:
//   per block b: right singular vectors and values of A^b, kept to r1:
//     the Gram A^b^T A^b (compensated FP32 partials, FP64 reduction) and its
//     eigen-decomposition give V~^b and S~^b (the small solve of the streaming
//     update, with T = V~ diag(1/S~), so V~^b S~^b = T diag(S~^2));
//   gather: W W^T = sum_b (V~^b S~^b)(V~^b S~^b)^T (N x N, FP64), whose
//     eigenvectors are the left singular vectors X~ of W and whose eigenvalues
//     are L~^2;
//   U~ = A X~ diag(1/L~) over all rows at once (the same T = X~ diag(1/L~)).
#include <stdint.h>

#include <vector>

#include "psvd_internal.cuh"

namespace psvd {
namespace {

// WW += Vs Vs^T with Vs = T64[:, 0:r1] diag(sigma^2) (N x N, FP64).
__global__ void wwt_accumulate_kernel(int N, int r1, const double* __restrict__ T64,
                                      const double* __restrict__ sigma, double* __restrict__ WW) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e % N, j = e / N;
  double acc = 0.0;
  for (int k = 0; k < r1; ++k) {
    const double s2 = sigma[k] * sigma[k];
    acc = fma(T64[i + (int64_t)k * N] * s2, T64[j + (int64_t)k * N] * s2, acc);
  }
  WW[e] += acc;
}

struct Buffers {
  std::vector<void*> ptrs;
  bool failed = false;
  ~Buffers() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

}  // namespace

int apmos_run(const void* A, int64_t lda, int a_bf16, int64_t Mtot, const int64_t* off, int nparts,
              int N, int r1, int r2, float* U, int64_t ldu, double* L, int num_sms,
              cudaStream_t st, int* status) {
  const size_t es = a_bf16 ? 2 : 4;
  const size_t nn = (size_t)N * N;
  Buffers buf;
  SmallWork w{};
  w.H = buf.get<double>(nn);
  w.X = buf.get<double>(nn);
  w.lam = buf.get<double>(N);
  w.W = buf.get<double>(nn);
  w.S = buf.get<double>(nn);
  w.R = buf.get<double>(nn);
  w.E = buf.get<double>(nn);
  w.Xn = buf.get<double>(nn);
  w.lamJ = buf.get<double>(N);
  w.T = buf.get<float>(nn);
  w.T64 = buf.get<double>(nn);
  w.Dnew = buf.get<double>(N);
  w.info = buf.get<int>(4);
  w.ls = buf.get<LevelState>(1);
  w.fs = buf.get<float>(eig_levels_scratch_floats(N));
  double* WW = buf.get<double>(nn);
  int64_t pmax = 0;
  for (int b = 0; b < nparts; ++b) {
    int nchunk;
    int64_t rpc, pd;
    gram_simt_plan(off[b + 1] - off[b], N, num_sms, &nchunk, &rpc, &pd);
    if (pd > pmax) pmax = pd;
  }
  double* partial = buf.get<double>((size_t)pmax);
  if (buf.failed) return PSVD_ERR_ALLOC;
#define ACK(x)                                     \
  do {                                             \
    if ((x) != cudaSuccess) return PSVD_ERR_CUDA;  \
  } while (0)
  ACK(cudaMemsetAsync(w.info, 0, sizeof(int) * 4, st));
  ACK(cudaMemsetAsync(WW, 0, sizeof(double) * nn, st));
  int nl = 0;
  for (int b = 0; b < nparts; ++b) {
    // local block: Gram, eigen-decomposition, W_b W_b^T
    const int64_t mb = off[b + 1] - off[b];
    const void* Ab = static_cast<const char*>(A) + (size_t)off[b] * es;
    PanelF32 p{nullptr, 0, 0, Ab, lda, a_bf16, mb, N};
    int nchunk;
    int64_t rpc, pd;
    gram_simt_plan(mb, N, num_sms, &nchunk, &rpc, &pd);
    ACK(gram_simt_launch(p, nchunk, rpc, partial, st));
    ACK(gram_reduce_launch(partial, nchunk, N, 0, nullptr, 1.0, nullptr, w.H, w.info, st));
    ACK(small_solve_launch(w, N, 0, r1, nullptr, 1.0, 3, kMaxLevels, st, &nl));
    wwt_accumulate_kernel<<<(unsigned)ceil_div((int64_t)nn, 256), 256, 0, st>>>(N, r1, w.T64,
                                                                              w.Dnew, WW);
    ACK(cudaGetLastError());
  }
  // global: eigen-decomposition of W W^T, T = X~ diag(1/L~), U = A T
  ACK(cudaMemcpyAsync(w.H, WW, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
  ACK(small_solve_launch(w, N, 0, r2, nullptr, 1.0, 3, kMaxLevels, st, &nl));
  PanelF32 pa{nullptr, 0, 0, A, lda, a_bf16, Mtot, N};
  ACK(update_simt_launch(pa, w.T, r2, U, ldu, st));
  ACK(cudaMemcpyAsync(L, w.Dnew, sizeof(double) * r2, cudaMemcpyDeviceToDevice, st));
  int info[4] = {0, 0, 0, 0};
  ACK(cudaMemcpyAsync(info, w.info, sizeof(info), cudaMemcpyDeviceToHost, st));
  ACK(cudaStreamSynchronize(st));
#undef ACK
  *status = info[2];
  return PSVD_OK;
}

}  // namespace psvd
