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
// Every phase covers all blocks in one launch: the local Grams are one launch over
// a work list of row chunks of every block (uneven blocks get proportionally many
// chunks), their reductions one launch with a grid dimension per block, and each
// kernel of the local eigen-solves one launch in which block b's problem is a CTA
// (or a grid plane) of its own, so the blocks' latency-bound solves run side by side
// on separate SMs.  Every block writes its factors to its own slot, and W W^T sums
// the slots in block order, so the result does not depend on scheduling.
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

#include "psvd_internal.cuh"

namespace psvd {
namespace {

// Blocks whose local eigen-solves share one batch of launches (bounds the batch
// workspace: 7 n x n FP64 matrices per block).
constexpr int kMaxBatch = 128;

// WW = sum_b Vs_b Vs_b^T, blocks in order, with Vs_b = T64_b[:, 0:r1] diag(sigma_b^2)
// (T64_b: N x r1 FP64 at T64 + b * N * r1, sigma_b at sigma + b * r1).  The blocks
// are split into gridDim.y consecutive groups, each summed by its own thread into a
// partial (part + y N^2); wwt_sum_kernel adds the partials in group order, so every
// entry is summed in block order as one chain of partial sums.
__global__ void wwt_kernel(int N, int r1, int nparts, const double* __restrict__ T64,
                           const double* __restrict__ sigma, double* __restrict__ part) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e % N, j = e / N;
  const int per = (nparts + gridDim.y - 1) / gridDim.y;
  const int b0 = blockIdx.y * per, b1 = min(nparts, b0 + per);
  double acc = 0.0;
  for (int b = b0; b < b1; ++b) {
    const double* Tb = T64 + (size_t)b * N * r1;
    const double* sb = sigma + (size_t)b * r1;
    for (int k = 0; k < r1; ++k) {
      const double s2 = sb[k] * sb[k];
      acc = fma(Tb[i + (int64_t)k * N] * s2, Tb[j + (int64_t)k * N] * s2, acc);
    }
  }
  part[(int64_t)blockIdx.y * N * N + e] = acc;
}

__global__ void wwt_sum_kernel(int N, int ngroups, const double* __restrict__ part,
                               double* __restrict__ WW) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  double s = 0.0;
  for (int g = 0; g < ngroups; ++g) s += part[(int64_t)g * N * N + e];
  WW[e] = s;
}

// Groups of blocks of the W W^T sum (a few blocks per thread).
inline int wwt_groups(int nparts) { return nparts < 32 ? nparts : 32; }

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

// OR of the blocks' status words into info[2] (info = block 0's words).
__global__ void merge_info_kernel(const int* __restrict__ block_info, int nblocks,
                                  int* __restrict__ info) {
  int bits = 0;
  for (int l = 0; l < nblocks; ++l) bits |= block_info[4 * l + 2];
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

}  // namespace

// Workspaces of apmos_run, kept by the handle across calls so that a call only
// enqueues work (no allocation once the sizes have been seen), and the launch
// sequence of a call, captured into a CUDA graph that a later call with the same
// arguments and buffers replays with one launch.
struct ApmosCache {
  // batched local solves: kMaxBatch problems' workspaces (problem 0 also serves the
  // global solve once the local ones are done)
  Grow<double> H, X, lam, W, S, R, E, Xn, lamJ, partial, Tg64, Dg;
  Grow<float> T, fs;
  Grow<LevelState> ls;
  Grow<int> info;  // 4 words per problem
  Grow<GramItem> items;
  Grow<int> first;  // first[b]: block b's first Gram item
  std::vector<int64_t> items_key;
  int nitems = 0;
  std::vector<int> first_host;
  Grow<double> T64_all, S_all, WW, WWp;  // WWp: partials of W W^T
  // the randomized global SVD (low_rank): explicit W, X diag(1/s), RandWork arrays
  Grow<double> Wexp, Tout, rB0, rB1, rB2, rMm, rRr, rAw, rBb;
  Grow<float> rOm;
  Grow<int> rpiv, rrank;
  int low_rank = 0, p = 0, q = 0;  // this call's settings (read by apmos_enqueue)
  uint64_t seed = 0;
  // the sequence is captured and replayed on this stream (capture cannot start
  // on the legacy default stream); it is ordered after and before the caller's
  cudaStream_t origin = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> key;  // arguments and buffer addresses the graph was captured with
  ~ApmosCache() {
    if (exec) cudaGraphExecDestroy(exec);
    if (origin) cudaStreamDestroy(origin);
    if (in) cudaEventDestroy(in);
    if (out) cudaEventDestroy(out);
  }
};

ApmosCache* apmos_cache_create() { return new (std::nothrow) ApmosCache(); }
void apmos_cache_destroy(ApmosCache* c) { delete c; }

namespace {

// SmallWork of problems [z0, z0 + count) of the batch workspace (problem stride nn).
SmallWork batch_work(ApmosCache* c, int N, int z0, int count, double* T64, int64_t sT64,
                     double* Dnew, int64_t sDnew) {
  const int64_t nn = (int64_t)N * N;
  const int64_t fsz = (int64_t)eig_levels_scratch_floats(N);
  SmallWork w{};
  w.H = c->H.p;
  w.X = c->X.p;
  w.lam = c->lam.p;
  w.W = c->W.p;
  w.S = c->S.p;
  w.R = c->R.p;
  w.E = c->E.p;
  w.Xn = c->Xn.p;
  w.lamJ = c->lamJ.p;
  w.T = c->T.p;
  w.T64 = T64;
  w.Dnew = Dnew;
  w.info = c->info.p + 4 * (int64_t)z0;
  w.ls = c->ls.p;
  w.fs = c->fs.p;
  w.bat.count = count;
  w.bat.nn = nn;
  w.bat.n = N;
  w.bat.T = nn;
  w.bat.T64 = sT64;
  w.bat.Dnew = sDnew;
  w.bat.info = 4;
  w.bat.ls = 1;
  w.bat.fs = fsz;
  return w;
}

// Enqueues one APMOS run on st (captured by the caller).
int apmos_enqueue(ApmosCache* c, const void* A, int64_t lda, int a_bf16, int64_t Mtot, int nparts,
                  int N, int r1, int r2, float* U, int64_t ldu, double* L, cudaStream_t st) {
#define ACK(x)                  \
  do {                          \
    if ((x) != cudaSuccess) {   \
      cudaGetLastError();       \
      return PSVD_ERR_CUDA;     \
    }                           \
  } while (0)
  const int64_t nn = (int64_t)N * N;
  double* T64_all = c->T64_all.p;
  double* S_all = c->S_all.p;
  double* WW = c->WW.p;
  const int nb = std::min(nparts, kMaxBatch);
  ACK(cudaMemsetAsync(c->info.p, 0, sizeof(int) * 4 * nb, st));
  // local Grams of every block: one launch over the work list of row chunks
  PanelF32 pa{nullptr, 0, 0, A, lda, a_bf16, Mtot, N};
  ACK(gram_items_launch(pa, c->items.p, c->nitems, c->partial.p, st));
  int nl = 0;
  for (int z0 = 0; z0 < nparts; z0 += kMaxBatch) {
    const int cnt = std::min(kMaxBatch, nparts - z0);
    // H_b for the blocks of this batch, then their eigen-solves side by side;
    // block b's factor goes to slot b of T64_all / S_all
    ACK(gram_reduce_items_launch(c->partial.p, c->first.p + z0, cnt, N, c->H.p, nn, c->info.p, st));
    SmallWork w = batch_work(c, N, 0, cnt, T64_all + (int64_t)z0 * N * r1, (int64_t)N * r1,
                             S_all + (int64_t)z0 * r1, r1);
    ACK(small_solve_launch(w, N, 0, r1, nullptr, 1.0, 3, kMaxLevels, st, &nl));
    merge_info_kernel<<<1, 1, 0, st>>>(c->info.p, cnt, c->info.p);
    ACK(cudaGetLastError());
  }
  // W W^T in block order (partials of groups of blocks, then their ordered sum)
  const int ng = wwt_groups(nparts);
  wwt_kernel<<<dim3((unsigned)ceil_div(nn, 128), (unsigned)ng), 128, 0, st>>>(N, r1, nparts, T64_all,
                                                                              S_all, c->WWp.p);
  ACK(cudaGetLastError());
  wwt_sum_kernel<<<(unsigned)ceil_div(nn, 256), 256, 0, st>>>(N, ng, c->WWp.p, WW);
  ACK(cudaGetLastError());
  // the global solve on problem 0's workspace (its status words collect every block's)
  SmallWork w = batch_work(c, N, 0, 1, c->Tg64.p, 0, c->Dg.p, 0);
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
    w.T64 = nullptr;
    ACK(cudaMemcpyAsync(w.H, WW, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
    ACK(small_solve_launch(w, N, 0, r2, nullptr, 1.0, 3, kMaxLevels, st, &nl));
  }
  // 256-row tiles: the same bits as any tile, 6.34 -> 6.31 ms per run on 64 blocks
  ACK(update_simt_launch(pa, w.T, r2, U, ldu, st, 256));
  ACK(cudaMemcpyAsync(L, w.Dnew, sizeof(double) * r2, cudaMemcpyDeviceToDevice, st));
#undef ACK
  return PSVD_OK;
}

}  // namespace

int apmos_run(const void* A, int64_t lda, int a_bf16, int64_t Mtot, const int64_t* off, int nparts,
              int N, int r1, int r2, float* U, int64_t ldu, double* L, int num_sms,
              cudaStream_t st, ApmosCache* c, int low_rank, int p, int q, uint64_t seed,
              int* status) {
  if (!c) return PSVD_ERR_INVALID_ARG;
  c->low_rank = low_rank ? 1 : 0;
  c->p = p;
  c->q = q;
  c->seed = seed;
  const size_t nn = (size_t)N * N;
  const int nb = std::min(nparts, kMaxBatch);
  // the Gram work list of these blocks (rebuilt when the blocks change)
  std::vector<int64_t> ikey(off, off + nparts + 1);
  ikey.push_back(N);
  ikey.push_back(num_sms);
  std::vector<GramItem> items;
  int64_t pdoubles = 0;
  const bool new_items = ikey != c->items_key;
  if (new_items) gram_items_plan(off, nparts, N, num_sms, &items, &c->first_host, &pdoubles);
  // growing a buffer frees the old one: nothing may still be using it
  if (cudaStreamSynchronize(st) != cudaSuccess) return PSVD_ERR_CUDA;
  const size_t fsz = eig_levels_scratch_floats(N);
  bool ok = c->T64_all.ensure((size_t)nparts * N * r1) && c->S_all.ensure((size_t)nparts * r1) &&
            c->WW.ensure(nn) && c->WWp.ensure(nn * (size_t)wwt_groups(nparts)) && c->H.ensure(nb * nn) && c->X.ensure(nb * nn) &&
            c->lam.ensure((size_t)nb * N) && c->W.ensure(nb * nn) && c->S.ensure(nb * nn) &&
            c->R.ensure(nb * nn) && c->E.ensure(nb * nn) && c->Xn.ensure(nb * nn) &&
            c->lamJ.ensure((size_t)nb * N) && c->T.ensure(nb * nn) && c->Tg64.ensure(nn) &&
            c->Dg.ensure(N) && c->ls.ensure(nb) && c->fs.ensure(nb * fsz) &&
            c->info.ensure(4 * (size_t)nb);
  if (ok && new_items) {
    c->items_key.clear();
    ok = c->items.ensure(items.size()) && c->first.ensure(c->first_host.size()) &&
         c->partial.ensure((size_t)pdoubles) &&
         cudaMemcpy(c->items.p, items.data(), sizeof(GramItem) * items.size(),
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->first.p, c->first_host.data(), sizeof(int) * c->first_host.size(),
                    cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
      c->nitems = (int)items.size();
      c->items_key = ikey;
    }
  }
  if (ok && c->low_rank) {
    const size_t m = (size_t)r1 * nparts, lmax = (size_t)N;
    ok = c->Wexp.ensure((size_t)N * m) && c->Tout.ensure((size_t)N * r2) &&
         c->rB0.ensure(std::max(m, (size_t)N) * lmax) && c->rB1.ensure((size_t)N * lmax) &&
         c->rB2.ensure((size_t)N * lmax) && c->rMm.ensure(lmax * lmax) &&
         c->rRr.ensure(lmax * lmax) && c->rAw.ensure(lmax * lmax) && c->rBb.ensure(lmax * lmax) &&
         c->rOm.ensure(m * lmax) && c->rpiv.ensure(lmax) && c->rrank.ensure(1);
  }
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
  std::vector<int64_t> key = {(int64_t)(uintptr_t)A, lda, a_bf16, Mtot, nparts, N, r1, r2,
                              (int64_t)(uintptr_t)U, ldu, (int64_t)(uintptr_t)L, num_sms,
                              (int64_t)(uintptr_t)st, c->nitems};
  for (const void* ptr : {(const void*)c->info.p, (const void*)c->T64_all.p, (const void*)c->S_all.p,
                          (const void*)c->WW.p, (const void*)c->WWp.p, (const void*)c->H.p,
                          (const void*)c->X.p,
                          (const void*)c->lam.p, (const void*)c->W.p, (const void*)c->S.p,
                          (const void*)c->R.p, (const void*)c->E.p, (const void*)c->Xn.p,
                          (const void*)c->lamJ.p, (const void*)c->T.p, (const void*)c->Tg64.p,
                          (const void*)c->Dg.p, (const void*)c->ls.p, (const void*)c->fs.p,
                          (const void*)c->items.p, (const void*)c->first.p,
                          (const void*)c->partial.p})
    key.push_back((int64_t)(uintptr_t)ptr);
  for (int b = 0; b <= nparts; ++b) key.push_back(off[b]);
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
      const int rc = apmos_enqueue(c, A, lda, a_bf16, Mtot, nparts, N, r1, r2, U, ldu, L, o);
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
    if (int rc = apmos_enqueue(c, A, lda, a_bf16, Mtot, nparts, N, r1, r2, U, ldu, L, o)) return rc;
  }
  ACK(cudaEventRecord(c->out, o));
  ACK(cudaStreamWaitEvent(st, c->out, 0));
  int info[4] = {0, 0, 0, 0};
  ACK(cudaMemcpyAsync(info, c->info.p, sizeof(info), cudaMemcpyDeviceToHost, st));
  ACK(cudaStreamSynchronize(st));
#undef ACK
  *status = info[2];
  return PSVD_OK;
}

}  // namespace psvd
