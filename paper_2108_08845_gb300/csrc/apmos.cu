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
// The local solves are latency-bound chains (the eigen-solve's level kernel runs
// on one SM), so the blocks run concurrently: up to kLanes streams, each with its
// own workspace, take the blocks round-robin; every block writes its factors to
// its own slot, and W W^T sums the slots in block order after the join, so the
// result does not depend on which lane finished first.
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

#include "psvd_internal.cuh"

namespace psvd {
namespace {

constexpr int kLanes = 16;

// WW = sum_b Vs_b Vs_b^T, blocks in order, with Vs_b = T64_b[:, 0:r1] diag(sigma_b^2)
// (T64_b: N x r1 FP64 at T64 + b * N * r1, sigma_b at sigma + b * r1).
__global__ void wwt_kernel(int N, int r1, int nparts, const double* __restrict__ T64,
                           const double* __restrict__ sigma, double* __restrict__ WW) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e % N, j = e / N;
  double acc = 0.0;
  for (int b = 0; b < nparts; ++b) {
    const double* Tb = T64 + (size_t)b * N * r1;
    const double* sb = sigma + (size_t)b * r1;
    for (int k = 0; k < r1; ++k) {
      const double s2 = sb[k] * sb[k];
      acc = fma(Tb[i + (int64_t)k * N] * s2, Tb[j + (int64_t)k * N] * s2, acc);
    }
  }
  WW[e] = acc;
}

// The gathered W (N x m, m = r1 nparts): column (b, k) = +-V_b[:, k] s_bk =
// +-T64_b[:, k] s_bk^2, signed so that its entries sum to >= 0.  One warp per column.
__global__ void wide_w_kernel(int N, int r1, int nparts, const double* __restrict__ T64,
                              const double* __restrict__ sigma, double* __restrict__ W) {
  const int c = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (c >= r1 * nparts) return;
  const int b = c / r1, k = c % r1;
  const double* col = T64 + (size_t)b * N * r1 + (size_t)k * N;
  double sum = 0.0;
  for (int i = lane; i < N; i += 32) sum += col[i];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const double sk = sigma[(size_t)b * r1 + k];
  const double scale = (sum >= 0.0 ? 1.0 : -1.0) * sk * sk;
  for (int i = lane; i < N; i += 32) W[i + (size_t)c * N] = col[i] * scale;
}

__global__ void to_f32_kernel(const double* __restrict__ x, int64_t count, float* __restrict__ y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) y[e] = (float)x[e];
}

// The local Grams run nlanes at a time: each is chunked for its share of the SMs
// (chunking one for the whole GPU multiplies the partials its reduction reads).
inline int local_sms(int num_sms, int nlanes) {
  const int s = num_sms / (nlanes > 0 ? nlanes : 1);
  return s > 0 ? s : 1;
}

// OR of the lanes' status words into info[2].
__global__ void merge_info_kernel(const int* __restrict__ lane_info, int nlanes, int* __restrict__ info) {
  int bits = 0;
  for (int l = 0; l < nlanes; ++l) bits |= lane_info[4 * l + 2];
  info[2] |= bits;
}

// Device buffer that grows on demand (contents are not kept across growth).
template <typename T>
struct Grow {
  T* p = nullptr;
  size_t cap = 0;
  bool ensure(size_t count) {
    if (count == 0) count = 1;
    if (count <= cap) return true;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc((void**)&p, sizeof(T) * count) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cap = count;
    return true;
  }
  ~Grow() { cudaFree(p); }
};

struct Lane {
  Grow<double> H, X, lam, W, S, R, E, Xn, lamJ, T64, Dnew, partial;
  Grow<float> T, fs;
  Grow<LevelState> ls;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};

}  // namespace

// Workspaces and streams of apmos_run, kept by the handle across calls so that a
// call only enqueues work (no allocation once the sizes have been seen).
// The launch sequence of a call (thousands of small kernels: the local solves are
// chains of ~45 launches each) is captured into a CUDA graph; a later call with
// the same arguments and buffers replays it with one launch.
struct ApmosCache {
  Lane lane[kLanes];
  Grow<int> lane_info;
  Grow<double> T64_all, S_all, WW;
  // the randomized global SVD (low_rank): explicit W, X diag(1/s), RandWork arrays
  Grow<double> Wexp, Tout, rB0, rB1, rB2, rMm, rRr, rAw, rBb;
  Grow<float> rOm;
  Grow<int> rpiv, rrank;
  int low_rank = 0, p = 0, q = 0;  // this call's settings (read by apmos_enqueue)
  uint64_t seed = 0;
  cudaEvent_t fork = nullptr;
  // the sequence is captured and replayed on this stream (capture cannot start
  // on the legacy default stream); it is ordered after and before the caller's
  cudaStream_t origin = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> key;  // arguments and buffer addresses the graph was captured with
  ~ApmosCache() {
    if (exec) cudaGraphExecDestroy(exec);
    for (Lane& l : lane) {
      if (l.st) cudaStreamDestroy(l.st);
      if (l.done) cudaEventDestroy(l.done);
    }
    if (fork) cudaEventDestroy(fork);
    if (origin) cudaStreamDestroy(origin);
    if (in) cudaEventDestroy(in);
    if (out) cudaEventDestroy(out);
  }
};

ApmosCache* apmos_cache_create() { return new (std::nothrow) ApmosCache(); }

int apmos_enqueue(ApmosCache* c, const std::vector<SmallWork>& lw, int nlanes, const void* A,
                  size_t es, int64_t lda, int a_bf16, int64_t Mtot, const int64_t* off, int nparts,
                  int N, int r1, int r2, float* U, int64_t ldu, double* L, int num_sms,
                  cudaStream_t st);
void apmos_cache_destroy(ApmosCache* c) { delete c; }

int apmos_run(const void* A, int64_t lda, int a_bf16, int64_t Mtot, const int64_t* off, int nparts,
              int N, int r1, int r2, float* U, int64_t ldu, double* L, int num_sms,
              cudaStream_t st, ApmosCache* c, int low_rank, int p, int q, uint64_t seed,
              int* status) {
  if (!c) return PSVD_ERR_INVALID_ARG;
  c->low_rank = low_rank ? 1 : 0;
  c->p = p;
  c->q = q;
  c->seed = seed;
  const size_t es = a_bf16 ? 2 : 4;
  const size_t nn = (size_t)N * N;
  const int nlanes = nparts < kLanes ? nparts : kLanes;
  int64_t pmax = 0;
  for (int b = 0; b < nparts; ++b) {
    int nchunk;
    int64_t rpc, pd;
    gram_simt_plan(off[b + 1] - off[b], N, local_sms(num_sms, nlanes), &nchunk, &rpc, &pd);
    if (pd > pmax) pmax = pd;
  }
  // growing a buffer frees the old one: nothing may still be using it
  if (cudaStreamSynchronize(st) != cudaSuccess) return PSVD_ERR_CUDA;
  bool ok = c->lane_info.ensure(4 * (size_t)nlanes) && c->T64_all.ensure((size_t)nparts * N * r1) &&
            c->S_all.ensure((size_t)nparts * r1) && c->WW.ensure(nn);
  std::vector<SmallWork> lw(nlanes);
  for (int l = 0; l < nlanes && ok; ++l) {
    Lane& ln = c->lane[l];
    ok = ln.H.ensure(nn) && ln.X.ensure(nn) && ln.lam.ensure(N) && ln.W.ensure(nn) &&
         ln.S.ensure(nn) && ln.R.ensure(nn) && ln.E.ensure(nn) && ln.Xn.ensure(nn) &&
         ln.lamJ.ensure(N) && ln.T.ensure(nn) && ln.T64.ensure(nn) && ln.Dnew.ensure(N) &&
         ln.ls.ensure(1) && ln.fs.ensure(eig_levels_scratch_floats(N)) &&
         ln.partial.ensure((size_t)pmax);
    if (ok && !ln.st) ok = cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking) == cudaSuccess;
    if (ok && !ln.done) ok = cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) == cudaSuccess;
    SmallWork& w = lw[l];
    w = SmallWork{};
    w.H = ln.H.p;
    w.X = ln.X.p;
    w.lam = ln.lam.p;
    w.W = ln.W.p;
    w.S = ln.S.p;
    w.R = ln.R.p;
    w.E = ln.E.p;
    w.Xn = ln.Xn.p;
    w.lamJ = ln.lamJ.p;
    w.T = ln.T.p;
    w.T64 = ln.T64.p;
    w.Dnew = ln.Dnew.p;
    w.info = c->lane_info.p + 4 * l;
    w.ls = ln.ls.p;
    w.fs = ln.fs.p;
  }
  if (ok && c->low_rank) {
    const size_t m = (size_t)r1 * nparts, lmax = (size_t)N;
    ok = c->Wexp.ensure((size_t)N * m) && c->Tout.ensure((size_t)N * r2) &&
         c->rB0.ensure(std::max(m, (size_t)N) * lmax) && c->rB1.ensure((size_t)N * lmax) &&
         c->rB2.ensure((size_t)N * lmax) && c->rMm.ensure(lmax * lmax) &&
         c->rRr.ensure(lmax * lmax) && c->rAw.ensure(lmax * lmax) && c->rBb.ensure(lmax * lmax) &&
         c->rOm.ensure(m * lmax) && c->rpiv.ensure(lmax) && c->rrank.ensure(1);
  }
  if (ok && !c->fork) ok = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) == cudaSuccess;
  if (ok && !c->origin) ok = cudaStreamCreateWithFlags(&c->origin, cudaStreamNonBlocking) == cudaSuccess;
  if (ok && !c->in) ok = cudaEventCreateWithFlags(&c->in, cudaEventDisableTiming) == cudaSuccess;
  if (ok && !c->out) ok = cudaEventCreateWithFlags(&c->out, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return PSVD_ERR_ALLOC;
  }
#define ACK(x)                                    \
  do {                                            \
    if ((x) != cudaSuccess) {                     \
      cudaGetLastError();                         \
      return PSVD_ERR_CUDA;                       \
    }                                             \
  } while (0)
  int* lane_info = c->lane_info.p;
  double* T64_all = c->T64_all.p;  // block b's N x r1 factor
  double* WW = c->WW.p;
  std::vector<int64_t> key = {(int64_t)(uintptr_t)A, lda, a_bf16, Mtot, nparts, N, r1, r2,
                              (int64_t)(uintptr_t)U, ldu, (int64_t)(uintptr_t)L, num_sms,
                              (int64_t)(uintptr_t)st, (int64_t)(uintptr_t)lane_info,
                              (int64_t)(uintptr_t)T64_all, (int64_t)(uintptr_t)WW};
  for (int b = 0; b <= nparts; ++b) key.push_back(off[b]);
  for (int l = 0; l < nlanes; ++l) key.push_back((int64_t)(uintptr_t)c->lane[l].partial.p);
  key.push_back(c->low_rank);
  if (c->low_rank) {
    for (int64_t v : {(int64_t)c->p, (int64_t)c->q, (int64_t)c->seed,
                      (int64_t)(uintptr_t)c->Wexp.p, (int64_t)(uintptr_t)c->rB0.p,
                      (int64_t)(uintptr_t)c->rOm.p})
      key.push_back(v);
  }
  // origin runs after the work already on st
  cudaStream_t o = c->origin;
  ACK(cudaEventRecord(c->in, st));
  ACK(cudaStreamWaitEvent(o, c->in, 0));
  if (!(c->exec && key == c->key)) {
    if (c->exec) {
      cudaGraphExecDestroy(c->exec);
      c->exec = nullptr;
    }
    c->key.clear();
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(o, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      const int rc = apmos_enqueue(c, lw, nlanes, A, es, lda, a_bf16, Mtot, off, nparts, N, r1, r2,
                                   U, ldu, L, num_sms, o);
      const cudaError_t ec = cudaStreamEndCapture(o, &graph);
      if (rc == PSVD_OK && ec == cudaSuccess && graph &&
          cudaGraphInstantiate(&c->exec, graph, 0) == cudaSuccess)
        c->key = key;
      else
        c->exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
  }
  if (c->exec) {
    ACK(cudaGraphLaunch(c->exec, o));
  } else {
    // no graph (capture unavailable): enqueue the sequence directly
    if (int rc = apmos_enqueue(c, lw, nlanes, A, es, lda, a_bf16, Mtot, off, nparts, N, r1, r2, U,
                               ldu, L, num_sms, o))
      return rc;
  }
  ACK(cudaEventRecord(c->out, o));
  ACK(cudaStreamWaitEvent(st, c->out, 0));
  int info[4] = {0, 0, 0, 0};
  ACK(cudaMemcpyAsync(info, lane_info, sizeof(info), cudaMemcpyDeviceToHost, st));
  ACK(cudaStreamSynchronize(st));
#undef ACK
  *status = info[2];
  return PSVD_OK;
}

// Enqueues one APMOS run on st and the lanes' streams (captured by the caller).
int apmos_enqueue(ApmosCache* c, const std::vector<SmallWork>& lw, int nlanes, const void* A,
                  size_t es, int64_t lda, int a_bf16, int64_t Mtot, const int64_t* off, int nparts,
                  int N, int r1, int r2, float* U, int64_t ldu, double* L, int num_sms,
                  cudaStream_t st) {
#define ACK(x)                  \
  do {                          \
    if ((x) != cudaSuccess) {   \
      cudaGetLastError();       \
      return PSVD_ERR_CUDA;     \
    }                           \
  } while (0)
  const size_t nn = (size_t)N * N;
  int* lane_info = c->lane_info.p;
  double* T64_all = c->T64_all.p;
  double* S_all = c->S_all.p;
  double* WW = c->WW.p;
  ACK(cudaMemsetAsync(lane_info, 0, sizeof(int) * 4 * nlanes, st));
  // fork: every lane starts after the work already on st
  ACK(cudaEventRecord(c->fork, st));
  for (int l = 0; l < nlanes; ++l) ACK(cudaStreamWaitEvent(c->lane[l].st, c->fork, 0));
  int nl = 0;
  for (int b = 0; b < nparts; ++b) {
    // local block: Gram, eigen-decomposition, factor V~ S~ into slot b
    const int l = b % nlanes;
    Lane& ln = c->lane[l];
    SmallWork w = lw[l];
    w.T64 = T64_all + (size_t)b * N * r1;
    w.Dnew = S_all + (size_t)b * r1;
    const int64_t mb = off[b + 1] - off[b];
    const void* Ab = static_cast<const char*>(A) + (size_t)off[b] * es;
    PanelF32 p{nullptr, 0, 0, Ab, lda, a_bf16, mb, N};
    int nchunk;
    int64_t rpc, pd;
    gram_simt_plan(mb, N, local_sms(num_sms, nlanes), &nchunk, &rpc, &pd);
    ACK(gram_simt_launch(p, nchunk, rpc, ln.partial.p, ln.st));
    ACK(gram_reduce_launch(ln.partial.p, nchunk, N, 0, nullptr, 1.0, nullptr, w.H, w.info, ln.st));
    ACK(small_solve_launch(w, N, 0, r1, nullptr, 1.0, 3, kMaxLevels, ln.st, &nl));
  }
  // join, then W W^T in block order
  for (int l = 0; l < nlanes; ++l) {
    ACK(cudaEventRecord(c->lane[l].done, c->lane[l].st));
    ACK(cudaStreamWaitEvent(st, c->lane[l].done, 0));
  }
  SmallWork w = lw[0];
  wwt_kernel<<<(unsigned)ceil_div((int64_t)nn, 256), 256, 0, st>>>(N, r1, nparts, T64_all, S_all, WW);
  ACK(cudaGetLastError());
  merge_info_kernel<<<1, 1, 0, st>>>(lane_info, nlanes, lane_info);
  ACK(cudaGetLastError());
  PanelF32 pa{nullptr, 0, 0, A, lda, a_bf16, Mtot, N};
  if (c->low_rank) {
    // global: the paper's low_rank_svd of the explicit W, T = X~ diag(1/L~), U = A T
    const int m = r1 * nparts;
    const int l = std::min(std::min(r2 + c->p, N), m);
    wide_w_kernel<<<(unsigned)ceil_div(m, 8), 256, 0, st>>>(N, r1, nparts, T64_all, S_all,
                                                            c->Wexp.p);
    ACK(cudaGetLastError());
    RandWork rw{};
    rw.Om = c->rOm.p;
    rw.B[0] = c->rB0.p;
    rw.B[1] = c->rB1.p;
    rw.B[2] = c->rB2.p;
    rw.Mm = c->rMm.p;
    rw.Rr = c->rRr.p;
    rw.Aw = c->rAw.p;
    rw.piv = c->rpiv.p;
    rw.rank = c->rrank.p;
    rw.Bb = c->rBb.p;
    ACK(randomized_wide_launch(rw, w, c->Wexp.p, WW, N, m, r2, l, c->q, c->seed,
                               kApmosSketchStream, c->Tout.p, st, &nl));
    const int64_t cnt = (int64_t)N * r2;
    to_f32_kernel<<<(unsigned)ceil_div(cnt, 256), 256, 0, st>>>(c->Tout.p, cnt, w.T);
    ACK(cudaGetLastError());
  } else {
    // global: eigen-decomposition of W W^T, T = X~ diag(1/L~), U = A T
    ACK(cudaMemcpyAsync(w.H, WW, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
    ACK(small_solve_launch(w, N, 0, r2, nullptr, 1.0, 3, kMaxLevels, st, &nl));
  }
  ACK(update_simt_launch(pa, w.T, r2, U, ldu, st));
  ACK(cudaMemcpyAsync(L, w.Dnew, sizeof(double) * r2, cudaMemcpyDeviceToDevice, st));
#undef ACK
  return PSVD_OK;
}

}  // namespace psvd
