// C-ABI entry points (include/psvd.h): handle lifetime, argument checks, and the
// launch sequence of the per-batch update of Algorithm 1 (Sec. 3.1):
//
//   Gram of [U | A] over row chunks  ->  FP64 reduction + diag(ff D, 1) scaling
//   ->  eigen-decomposition of the small (K+B)^2 matrix (FP32 tridiagonal
//   solves on scale levels + FP64 refinement)  ->  T = S V diag(1/sigma)
//   ->  U_new = [U | A] T.
//
// All device work is enqueued on the handle's stream; nothing runs on the host
// but argument checks, pointer classification and launch configuration.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "psvd_internal.cuh"
#include "tc_kernels.cuh"

using namespace psvd;

struct psvd_ctx {
  psvd_config cfg;
  cudaStream_t st = nullptr;
  int num_sms = 0;
  int64_t M = 0, ldu = 0;
  int K = 0, maxB = 0, nmax = 0;
  int kc = 0;  // current mode count
  int64_t iteration = 0;
  uint64_t sketch_counter = 0;
  int cur = 0;
  // FP32 modes (double-buffered) or BF16 hi/lo planes (tensor-core path)
  float* U[2] = {nullptr, nullptr};
  // tensor-core path: both BF16 planes of the modes, slot-tiled (tc_kernels.cuh)
  __nv_bfloat16* Ut[2] = {nullptr, nullptr};
  int Kp = 0;  // column stride of the tiled planes, roundup(K, 8)
  // FP64 path: modes in FP64 (double-buffered)
  double* U64[2] = {nullptr, nullptr};
  double* D[2] = {nullptr, nullptr};
  double* partial = nullptr;
  int64_t partial_cap = 0;  // doubles
  double* G = nullptr;
  SmallWork w{};
  RandWork rw{};  // randomized range finder (low_rank handles only)
  int lmax = 0;   // sketch columns K + p, capped at K + max_batch
  void* staging = nullptr;
  size_t staging_bytes = 0;
  float* Uf32_tmp = nullptr;  // FP32 view of hi/lo modes for get_modes / save
  // psvd_incorporate_batches: host batches are copied on their own stream into two
  // alternating staging buffers while the previous batch is processed
  cudaStream_t copy_st = nullptr;
  void* hstg[2] = {nullptr, nullptr};
  size_t hstg_bytes = 0;
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
  bool hstg_used[2] = {false, false};
  // psvd_incorporate_batches on the tensor-core path: A^T A of the next device batch
  // is summed on its own stream while this batch's small solve runs (it needs no
  // modes), and the next Gram computes only the blocks that involve the modes
  cudaStream_t aa_st = nullptr;
  cudaEvent_t aa_go = nullptr, aa_done = nullptr;
  double* aa_partial = nullptr;
  int64_t aa_cap = 0;
  double* aa_sum = nullptr;      // 128 x 128 FP64
  const void* aa_src = nullptr;  // the batch aa_sum belongs to ...
  int64_t aa_iter = -1;          // ... and the step that may use it
  ApmosCache* apmos = nullptr;  // psvd_parallel_svd workspaces and streams (lazily made)
  AdjWork* adj = nullptr;       // psvd_update_adjoint workspaces (lazily made)
  SimtTune tune;                // FP32-path tile choices (psvd_autotune)
  TcTune tctune;                // tensor-core launch shapes (psvd_autotune)
  int host_info[4] = {0, 0, 0, 0};
  int sticky_status = 0;
  // per-phase event timing (psvd_set_profiling)
  bool profiling = false;
  struct Rec {
    cudaEvent_t a, b;
    int phase;
  };
  std::vector<Rec> recs;      // recorded, not yet read
  std::vector<Rec> free_recs; // event pairs available for reuse
  double prof_ms[3] = {0, 0, 0};
  int64_t prof_count[3] = {0, 0, 0};
  int64_t launches = 0;
};

namespace {

#define CK(x)                                     \
  do {                                            \
    cudaError_t err_ = (x);                       \
    if (err_ != cudaSuccess) return PSVD_ERR_CUDA; \
  } while (0)

int elem_size(int dtype) {
  switch (dtype) {
    case PSVD_F32: return 4;
    case PSVD_BF16: return 2;
    case PSVD_F64: return 8;
    default: return 0;
  }
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
int dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return PSVD_ERR_ALLOC;
  }
  return PSVD_OK;
}

// Device copy of a column-major input: host inputs are staged; with align16 (the
// tensor-core path, whose TMA copies need 16-byte aligned columns) device inputs
// whose base or leading dimension is not 16-byte aligned are re-staged with a
// padded leading dimension.
int stage_input(psvd_ctx* h, const void* A, int64_t lda, int64_t rows, int cols, int dtype,
                bool align16, const void** dev, int64_t* ld_dev) {
  const size_t es = (size_t)elem_size(dtype);
  const bool on_dev = is_device_ptr(A);
  const bool aligned = (((uintptr_t)A & 15) == 0) && (((size_t)lda * es) % 16 == 0);
  if (on_dev && (!align16 || aligned)) {
    *dev = A;
    *ld_dev = lda;
    return PSVD_OK;
  }
  const int64_t ld = align16 ? ceil_div(rows, 8) * 8 : rows;
  const size_t need = es * (size_t)ld * (size_t)cols;
  if (need > h->staging_bytes) {
    if (h->staging) {
      CK(cudaStreamSynchronize(h->st));
      cudaFree(h->staging);
      h->staging = nullptr;
    }
    if (cudaMalloc(&h->staging, need) != cudaSuccess) {
      cudaGetLastError();
      h->staging_bytes = 0;
      return PSVD_ERR_ALLOC;
    }
    h->staging_bytes = need;
  }
  CK(cudaMemcpy2DAsync(h->staging, es * ld, A, es * lda, es * rows, cols,
                       on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  *dev = h->staging;
  *ld_dev = ld;
  return PSVD_OK;
}

int ensure_partial(psvd_ctx* h, int64_t doubles) {
  if (doubles <= h->partial_cap) return PSVD_OK;
  if (h->partial) {
    CK(cudaStreamSynchronize(h->st));
    cudaFree(h->partial);
    h->partial = nullptr;
  }
  if (dalloc(&h->partial, (size_t)doubles)) return PSVD_ERR_ALLOC;
  h->partial_cap = doubles;
  return PSVD_OK;
}

bool use_tc(const psvd_ctx* h) { return h->cfg.precision == PSVD_PREC_BF16_TC; }
bool use_f64(const psvd_ctx* h) { return h->cfg.precision == PSVD_PREC_FP64; }

// Starts timing a phase (returns the record index, or -1 when not profiling).
int prof_begin(psvd_ctx* h, int phase) {
  if (!h->profiling) return -1;
  psvd_ctx::Rec r;
  if (!h->free_recs.empty()) {
    r = h->free_recs.back();
    h->free_recs.pop_back();
  } else if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  r.phase = phase;
  cudaEventRecord(r.a, h->st);
  h->recs.push_back(r);
  return (int)h->recs.size() - 1;
}

void prof_end(psvd_ctx* h, int idx) {
  if (idx >= 0) cudaEventRecord(h->recs[idx].b, h->st);
}

// Folds completed records into the per-phase totals (synchronises).
void prof_collect(psvd_ctx* h) {
  cudaStreamSynchronize(h->st);
  for (auto& r : h->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      h->prof_ms[r.phase] += ms;
      h->prof_count[r.phase] += 1;
    }
    cudaGetLastError();
    h->free_recs.push_back(r);
  }
  h->recs.clear();
}

// Gram of the panel [U | A] (U = current modes, kc columns) -> H = S G S.
// With G != nullptr the unscaled Gram is stored too.
int panel_gram(psvd_ctx* h, const void* A, int64_t lda, int B, int dtype, int kc, double ff,
               const double* D, double* G) {
  const int n = kc + B;
  if (use_tc(h)) {
    // A^T A already summed for this batch (psvd_incorporate_batches): split Gram
    const bool split = kc > 0 && h->aa_iter == h->iteration && h->aa_src == A &&
                       tc_gram_can_split(kc, B);
    h->aa_iter = -1;
    int rc = tc_gram(h->Ut[h->cur], h->Kp, kc, A, lda, B, dtype, h->M, h->num_sms, h->tctune,
                     split, &h->partial, &h->partial_cap, &h->w.info[2], h->st);
    if (rc) return rc;
    if (split) CK(cudaStreamWaitEvent(h->st, h->aa_done, 0));
    return tc_gram_reduce(h->partial, h->M, kc, B, h->num_sms, h->tctune,
                          split ? h->aa_sum : nullptr, ff, D, G, h->w.H, &h->w.info[2], h->st)
               ? PSVD_ERR_CUDA
               : PSVD_OK;
  }
  int nchunk;
  int64_t rpc, pd;
  gram_simt_plan(h->M, n, h->num_sms, &nchunk, &rpc, &pd, h->tune.gram_ctas_per_sm);
  if (int rc = ensure_partial(h, pd)) return rc;
  if (use_f64(h)) {
    PanelF64 p{h->U64[h->cur], h->ldu, kc, A, lda, dtype, h->M, n};
    CK(gram_f64_launch(p, nchunk, rpc, h->partial, h->st));
  } else {
    PanelF32 p{h->U[h->cur], h->ldu, kc, A, lda, dtype == PSVD_BF16 ? 1 : 0, h->M, n};
    CK(gram_simt_launch(p, nchunk, rpc, h->partial, h->st));
  }
  CK(gram_reduce_launch(h->partial, nchunk, n, kc, D, ff, G, h->w.H, h->w.info, h->st));
  return PSVD_OK;
}

// One application of Algorithm 1's small solve + mode update; kc = 0 is the
// initialisation I1-I2 (the panel is A0 alone).
// A_next (may be null): the next batch (device memory, the same B and dtype, leading
// dimension ld_next, no staging needed), whose A^T A block the tensor-core path sums
// during this step's small solve.
int step(psvd_ctx* h, const void* A, int64_t lda, int B, int dtype, const void* A_next = nullptr,
         int64_t ld_next = 0) {
  const int kc = h->kc;
  const int n = kc + B;
  const int k1 = (h->K < n) ? h->K : n;
  const double* Dcur = h->D[h->cur];
  double* Dnext = h->D[h->cur ^ 1];
  int pr = prof_begin(h, 0);
  if (int rc = panel_gram(h, A, lda, B, dtype, kc, h->cfg.ff, Dcur, nullptr)) return rc;
  prof_end(h, pr);
  h->launches += use_tc(h) ? 3 : 2;
  if (A_next && use_tc(h) && tc_gram_can_split(k1, B)) {
    // on the side stream, after this Gram's blocks are assembled (aa_sum is free),
    // with SMs left over for the small solve's kernels
    CK(cudaEventRecord(h->aa_go, h->st));
    CK(cudaStreamWaitEvent(h->aa_st, h->aa_go, 0));
    const int ctas = h->num_sms > 32 ? h->num_sms - 16 : h->num_sms / 2;
    if (int rc = tc_gram_aa(A_next, ld_next, B, h->M, h->num_sms, ctas, &h->aa_partial,
                            &h->aa_cap, h->aa_sum, &h->w.info[2], h->aa_st))
      return rc;
    CK(cudaEventRecord(h->aa_done, h->aa_st));
    h->aa_src = A_next;
    h->aa_iter = h->iteration + 1;
    h->launches += 2;
  }
  SmallWork w = h->w;
  w.Dnew = Dnext;
  pr = prof_begin(h, 1);
  int nl = 0;
  const float* T = w.T;
  if (h->cfg.low_rank) {
    // Sec. 3.3: randomized rank-k1 SVD of the panel, sketch stream = batch index
    int l = (h->lmax < n) ? h->lmax : n;
    if (l < k1) l = k1;
    CK(randomized_solve_launch(h->rw, w, n, kc, k1, l, h->cfg.power_iters, Dcur, h->cfg.ff,
                               h->cfg.seed, (uint64_t)h->iteration, h->st, &nl));
    T = h->rw.Tupd;
  } else {
    // an FP64 Gram resolves eigenvalues down to ~1e-13 lambda_max: up to six
    // levels of three decades each reach them.  The refinement converges
    // quadratically from the levels' ~u32/tau accuracy: two steps reach FP64
    // rounding for the FP32 Gram (resolved to ~1e-10 lambda_max), the FP64 path
    // takes three, and one already lies below the tensor-core Gram's own error
    // (~1e-9 lambda_max, from its FP32 accumulation chains)
    const int refine = use_f64(h) ? 3 : use_tc(h) ? 1 : 2;
    CK(small_solve_launch(w, n, kc, k1, Dcur, h->cfg.ff, refine, use_f64(h) ? 6 : kMaxLevels,
                          h->st, &nl));
  }
  prof_end(h, pr);
  h->launches += nl;
  pr = prof_begin(h, 2);
  if (use_tc(h)) {
    int rc = tc_update(h->Ut[h->cur], h->Kp, kc, A, lda, B, dtype, h->M, T, n, k1, w.T3,
                       h->Ut[h->cur ^ 1], h->num_sms, h->tctune, &h->w.info[2], h->st);
    if (rc) return rc;
  } else if (use_f64(h)) {
    PanelF64 p{h->U64[h->cur], h->ldu, kc, A, lda, dtype, h->M, n};
    CK(update_f64_launch(p, w.T64, k1, h->U64[h->cur ^ 1], h->ldu, h->st));
  } else {
    PanelF32 p{h->U[h->cur], h->ldu, kc, A, lda, dtype == PSVD_BF16 ? 1 : 0, h->M, n};
    CK(update_simt_launch(p, T, k1, h->U[h->cur ^ 1], h->ldu, h->st, h->tune.update_rows));
  }
  prof_end(h, pr);
  h->launches += use_tc(h) ? 2 : 1;
  h->cur ^= 1;
  h->kc = k1;
  h->iteration += 1;
  return PSVD_OK;
}

int check_batch(psvd_ctx* h, const void* A, int64_t lda, int B, int dtype) {
  if (!A || B < 1 || lda < h->M) return PSVD_ERR_INVALID_ARG;
  if (dtype != PSVD_F32 && dtype != PSVD_BF16 && dtype != PSVD_F64) return PSVD_ERR_INVALID_ARG;
  if (use_tc(h) && dtype != PSVD_BF16) return PSVD_ERR_UNSUPPORTED;
  if (dtype == PSVD_F64 && !use_f64(h)) return PSVD_ERR_UNSUPPORTED;
  if (B > h->maxB) return PSVD_ERR_SHAPE;
  if (h->M < (int64_t)h->kc + B) return PSVD_ERR_SHAPE;
  return PSVD_OK;
}

// Reads the device status word (synchronising) and folds it into a status code.
int collect_status(psvd_ctx* h) {
  CK(cudaMemcpyAsync(h->host_info, h->w.info, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const int bits = h->host_info[2];
  if (bits & 8) h->sticky_status = PSVD_ERR_TIMEOUT;
  if (bits & 4) h->sticky_status = PSVD_ERR_NONFINITE;
  if (h->sticky_status < 0) return h->sticky_status;
  if (bits & 1) return PSVD_WARN_RANK_DEFICIENT;
  if (bits & 2) return PSVD_WARN_NOT_CONVERGED;
  return PSVD_OK;
}

}  // namespace

// Autotuner helpers (psvd_autotune).
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int, int, int>, SimtTune> g_tune_cache;  // (M, n, dtype, SMs)
std::map<std::tuple<int64_t, int, int>, TcTune> g_tc_tune_cache;      // (M, n, SMs)

// Mean time of `reps` launches of fn on st (after one warm-up launch), in ms.
template <typename F>
int time_ms(cudaStream_t st, int reps, F fn, float* ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return PSVD_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return PSVD_ERR_CUDA;
  }
  int rc = fn();
  if (rc == PSVD_OK && cudaEventRecord(a, st) != cudaSuccess) rc = PSVD_ERR_CUDA;
  for (int i = 0; rc == PSVD_OK && i < reps; ++i) rc = fn();
  if (rc == PSVD_OK && cudaEventRecord(b, st) != cudaSuccess) rc = PSVD_ERR_CUDA;
  if (rc == PSVD_OK && cudaEventSynchronize(b) != cudaSuccess) rc = PSVD_ERR_CUDA;
  float t = 0.f;
  if (rc == PSVD_OK && cudaEventElapsedTime(&t, a, b) != cudaSuccess) rc = PSVD_ERR_CUDA;
  *ms = t / reps;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}
}  // namespace

extern "C" {

int psvd_debug_set_wait_budget(int32_t kernel, int64_t cycles) {
  return tc_set_wait_budget(kernel, (long long)cycles);
}

const char* psvd_status_string(int s) {
  switch (s) {
    case PSVD_OK: return "ok";
    case PSVD_WARN_RANK_DEFICIENT: return "warning: a kept singular value is numerically zero";
    case PSVD_WARN_NOT_CONVERGED:
      return "warning: the eigen-solve used all its scale levels before resolving every kept pair";
    case PSVD_WARN_DEGENERATE:
      return "warning: coincident singular values at a kept index; the derivative is undefined";
    case PSVD_ERR_INVALID_ARG: return "invalid argument";
    case PSVD_ERR_NOT_INITIALIZED: return "handle not initialized (call psvd_initialize first)";
    case PSVD_ERR_SHAPE: return "unsupported shape";
    case PSVD_ERR_NONFINITE: return "non-finite value in the small factor";
    case PSVD_ERR_CUDA: return "CUDA runtime error";
    case PSVD_ERR_ALLOC: return "allocation failed";
    case PSVD_ERR_IO: return "file I/O error or bad file";
    case PSVD_ERR_UNSUPPORTED: return "unsupported for this precision or configuration";
    case PSVD_ERR_TIMEOUT: return "a device-side wait timed out (kernel aborted its work)";
    default: return "unknown status";
  }
}

int psvd_create(psvd_handle* out, const psvd_config* cfg) {
  if (!out) return PSVD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || cfg->M < 1 || cfg->K < 1 || cfg->max_batch < 1) return PSVD_ERR_INVALID_ARG;
  if (!(cfg->ff > 0.0 && cfg->ff <= 1.0)) return PSVD_ERR_INVALID_ARG;
  if (cfg->precision != PSVD_PREC_FP32 && cfg->precision != PSVD_PREC_BF16_TC &&
      cfg->precision != PSVD_PREC_FP64)
    return PSVD_ERR_INVALID_ARG;
  if ((int64_t)cfg->K + cfg->max_batch > kMaxN) return PSVD_ERR_SHAPE;
  if (cfg->precision == PSVD_PREC_BF16_TC &&
      (cfg->K > 80 || ((2 * ((cfg->K + 7) & ~7) + ((cfg->max_batch + 7) & ~7) + 15) & ~15) > 256))
    return PSVD_ERR_SHAPE;
  if (cfg->low_rank != 0 &&
      (cfg->low_rank != 1 || cfg->oversample < 0 || cfg->power_iters < 0 || cfg->power_iters > 16))
    return PSVD_ERR_INVALID_ARG;
  if (cfg->low_rank && cfg->precision == PSVD_PREC_FP64) return PSVD_ERR_UNSUPPORTED;
  psvd_ctx* h = new (std::nothrow) psvd_ctx();
  if (!h) return PSVD_ERR_ALLOC;
  h->cfg = *cfg;
  h->st = (cudaStream_t)cfg->stream;
  h->M = cfg->M;
  h->ldu = ceil_div(cfg->M, 64) * 64;
  h->Kp = (cfg->K + 7) & ~7;
  h->K = cfg->K;
  h->maxB = cfg->max_batch;
  h->nmax = cfg->K + cfg->max_batch;
  int dev = 0;
  int rc = PSVD_OK;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return PSVD_ERR_CUDA;
  }
  const size_t nm = (size_t)h->nmax;
  const size_t ucount = (size_t)h->ldu * (size_t)h->K;
  for (int b = 0; b < 2 && !rc; ++b) {
    if (use_tc(h)) {
      rc = dalloc(&h->Ut[b], tc_modes_elems(h->M, h->K));
    } else if (use_f64(h)) {
      rc = dalloc(&h->U64[b], ucount);
    } else {
      rc = dalloc(&h->U[b], ucount);
    }
    if (!rc) rc = dalloc(&h->D[b], (size_t)h->K);
  }
  if (!rc) rc = dalloc(&h->G, nm * nm);
  if (!rc) rc = dalloc(&h->w.H, nm * nm);
  if (!rc) rc = dalloc(&h->w.X, nm * nm);
  if (!rc) rc = dalloc(&h->w.lam, nm);
  if (!rc) rc = dalloc(&h->w.W, nm * nm);
  if (!rc) rc = dalloc(&h->w.S, nm * nm);
  if (!rc) rc = dalloc(&h->w.R, nm * nm);
  if (!rc) rc = dalloc(&h->w.E, nm * nm);
  if (!rc) rc = dalloc(&h->w.Xn, nm * nm);
  if (!rc) rc = dalloc(&h->w.lamJ, nm);
  if (!rc) rc = dalloc(&h->w.T, nm * (size_t)h->K);
  if (!rc && use_f64(h)) rc = dalloc(&h->w.T64, nm * (size_t)h->K);
  // Gram resolution: FP64 sums over M rows keep ~u64 sqrt(M) of lambda_max
  h->w.lam_floor = use_f64(h) ? 1e-13 : 0.0;
  if (!rc) rc = dalloc(&h->w.T3, tc_t3_elems(h->K, h->maxB));
  if (!rc) rc = dalloc(&h->w.info, 4);
  if (!rc) rc = dalloc(&h->w.fs, eig_levels_scratch_floats(h->nmax));
  if (!rc) rc = dalloc(reinterpret_cast<char**>(&h->w.ls), sizeof(LevelState));
  if (!rc && cfg->low_rank) {
    const int64_t l = (int64_t)cfg->K + cfg->oversample;
    h->lmax = (int)((l < h->nmax) ? l : h->nmax);
    const size_t nl = nm * (size_t)h->lmax, ll = (size_t)h->lmax * h->lmax;
    rc = dalloc(&h->rw.Om, nl);
    for (int b = 0; b < 3 && !rc; ++b) rc = dalloc(&h->rw.B[b], nl);
    if (!rc) rc = dalloc(&h->rw.Mm, ll);
    if (!rc) rc = dalloc(&h->rw.Rr, ll);
    if (!rc) rc = dalloc(&h->rw.Aw, ll);
    if (!rc) rc = dalloc(&h->rw.piv, (size_t)h->lmax);
    if (!rc) rc = dalloc(&h->rw.rank, 1);
    if (!rc) rc = dalloc(&h->rw.Bb, ll);
    if (!rc) rc = dalloc(&h->rw.Tupd, nm * (size_t)h->K);
    if (!rc) rc = dalloc(&h->rw.sgn, (size_t)h->K);
  }
  if (!rc && cudaMemsetAsync(h->w.info, 0, sizeof(int) * 4, h->st) != cudaSuccess) rc = PSVD_ERR_CUDA;
  if (!rc) {
    // zero the mode buffers once so that padded rows stay zero
    for (int b = 0; b < 2 && !rc; ++b) {
      if (use_tc(h)) {
        if (cudaMemsetAsync(h->Ut[b], 0, tc_modes_elems(h->M, h->K) * 2, h->st)) rc = PSVD_ERR_CUDA;
      } else if (use_f64(h)) {
        if (cudaMemsetAsync(h->U64[b], 0, ucount * 8, h->st)) rc = PSVD_ERR_CUDA;
      } else if (cudaMemsetAsync(h->U[b], 0, ucount * 4, h->st)) {
        rc = PSVD_ERR_CUDA;
      }
      if (!rc && cudaMemsetAsync(h->D[b], 0, sizeof(double) * h->K, h->st)) rc = PSVD_ERR_CUDA;
    }
  }
  if (rc) {
    psvd_destroy(h);
    return rc;
  }
  *out = h;
  return PSVD_OK;
}

void psvd_destroy(psvd_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  for (auto& r : h->recs) h->free_recs.push_back(r);
  for (auto& r : h->free_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (int b = 0; b < 2; ++b) {
    cudaFree(h->U[b]);
    cudaFree(h->Ut[b]);
    cudaFree(h->U64[b]);
    cudaFree(h->D[b]);
  }
  cudaFree(h->partial);
  cudaFree(h->G);
  cudaFree(h->w.H);
  cudaFree(h->w.X);
  cudaFree(h->w.lam);
  cudaFree(h->w.W);
  cudaFree(h->w.S);
  cudaFree(h->w.R);
  cudaFree(h->w.E);
  cudaFree(h->w.Xn);
  cudaFree(h->w.lamJ);
  cudaFree(h->w.T);
  cudaFree(h->w.T3);
  cudaFree(h->w.info);
  cudaFree(h->w.fs);
  cudaFree(h->w.ls);
  cudaFree(h->rw.Om);
  for (int b = 0; b < 3; ++b) cudaFree(h->rw.B[b]);
  cudaFree(h->rw.Mm);
  cudaFree(h->rw.Rr);
  cudaFree(h->rw.Aw);
  cudaFree(h->rw.piv);
  cudaFree(h->rw.rank);
  cudaFree(h->rw.Bb);
  cudaFree(h->rw.Tupd);
  cudaFree(h->rw.sgn);
  cudaFree(h->staging);
  cudaFree(h->Uf32_tmp);
  for (int j = 0; j < 2; ++j) {
    cudaFree(h->hstg[j]);
    if (h->copied[j]) cudaEventDestroy(h->copied[j]);
    if (h->consumed[j]) cudaEventDestroy(h->consumed[j]);
  }
  if (h->copy_st) {
    cudaStreamSynchronize(h->copy_st);
    cudaStreamDestroy(h->copy_st);
  }
  if (h->aa_st) {
    cudaStreamSynchronize(h->aa_st);
    cudaStreamDestroy(h->aa_st);
  }
  if (h->aa_go) cudaEventDestroy(h->aa_go);
  if (h->aa_done) cudaEventDestroy(h->aa_done);
  cudaFree(h->aa_partial);
  cudaFree(h->aa_sum);
  apmos_cache_destroy(h->apmos);
  adj_work_destroy(h->adj);
  cudaFree(h->w.T64);
  cudaGetLastError();
  delete h;
}

int psvd_initialize(psvd_handle h, const void* A0, int64_t lda, int32_t B, int32_t dtype) {
  if (!h) return PSVD_ERR_INVALID_ARG;
  h->kc = 0;
  if (int rc = check_batch(h, A0, lda, B, dtype)) return rc;
  const void* Ad;
  int64_t ldd;
  if (int rc = stage_input(h, A0, lda, h->M, B, dtype, use_tc(h), &Ad, &ldd)) return rc;
  CK(cudaMemsetAsync(h->w.info, 0, sizeof(int) * 4, h->st));
  h->sticky_status = 0;
  h->iteration = 0;
  h->aa_iter = -1;
  return step(h, Ad, ldd, B, dtype);
}

int psvd_incorporate_data(psvd_handle h, const void* A, int64_t lda, int32_t B, int32_t dtype) {
  if (!h) return PSVD_ERR_INVALID_ARG;
  if (h->kc == 0) return PSVD_ERR_NOT_INITIALIZED;
  if (int rc = check_batch(h, A, lda, B, dtype)) return rc;
  h->aa_iter = -1;  // a look-ahead left by a failed batches call is never used
  const void* Ad;
  int64_t ldd;
  if (int rc = stage_input(h, A, lda, h->M, B, dtype, use_tc(h), &Ad, &ldd)) return rc;
  return step(h, Ad, ldd, B, dtype);
}

int psvd_incorporate_batches(psvd_handle h, const void* const* A, int32_t count, int64_t lda,
                             int32_t B, int32_t dtype, double* s_out) {
  if (!h || !A || count < 1) return PSVD_ERR_INVALID_ARG;
  if (h->kc == 0) return PSVD_ERR_NOT_INITIALIZED;
  // a look-ahead is made and used within one call: none survives from an earlier one
  // (its batch buffer may hold other data by now)
  h->aa_iter = -1;
  // every batch is checked before the first one is enqueued
  for (int i = 0; i < count; ++i)
    if (int rc = check_batch(h, A[i], lda, B, dtype)) return rc;
  const size_t es = (size_t)elem_size(dtype);
  // staging of host batches: the tensor-core path wants 16-byte aligned columns
  const int64_t ldst = use_tc(h) ? ceil_div(h->M, 8) * 8 : h->M;
  const size_t need = es * (size_t)ldst * (size_t)B;
  bool any_host = false;
  for (int i = 0; i < count && !any_host; ++i) any_host = !is_device_ptr(A[i]);
  if (any_host) {
    if (!h->copy_st) {
      if (cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->copy_st = nullptr;
        return PSVD_ERR_CUDA;
      }
      for (int j = 0; j < 2; ++j)
        if (cudaEventCreateWithFlags(&h->copied[j], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->consumed[j], cudaEventDisableTiming) != cudaSuccess) {
          cudaGetLastError();
          return PSVD_ERR_CUDA;
        }
    }
    if (need > h->hstg_bytes) {
      // a buffer may still feed an earlier call's update, or receive its copy
      CK(cudaStreamSynchronize(h->copy_st));
      CK(cudaStreamSynchronize(h->st));
      for (int j = 0; j < 2; ++j) {
        cudaFree(h->hstg[j]);
        h->hstg[j] = nullptr;
        h->hstg_used[j] = false;
      }
      h->hstg_bytes = 0;
      for (int j = 0; j < 2; ++j)
        if (cudaMalloc(&h->hstg[j], need) != cudaSuccess) {
          cudaGetLastError();
          return PSVD_ERR_ALLOC;
        }
      h->hstg_bytes = need;
    }
  }
  // device batches that need no staging: each step sums the next one's A^T A
  // during its small solve (tensor-core path)
  auto direct = [&](const void* p) {
    return is_device_ptr(p) && ((uintptr_t)p & 15) == 0 && ((size_t)lda * es) % 16 == 0;
  };
  bool lookahead = false;
  if (use_tc(h) && count > 1 && tc_gram_can_split(h->K, B)) {
    for (int i = 1; i < count && !lookahead; ++i) lookahead = direct(A[i]);
    if (lookahead && !h->aa_st) {
      if (cudaStreamCreateWithFlags(&h->aa_st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->aa_go, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->aa_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return PSVD_ERR_CUDA;
      }
    }
    if (lookahead && !h->aa_sum) {
      if (cudaMalloc(&h->aa_sum, sizeof(double) * 128 * 128) != cudaSuccess) {
        cudaGetLastError();
        return PSVD_ERR_ALLOC;
      }
    }
  }
  for (int i = 0; i < count; ++i) {
    const void* Ad;
    int64_t ldd;
    const int j = i & 1;
    const bool host = any_host && !is_device_ptr(A[i]);
    if (host) {
      // staging j is free once the update that read it (two batches back) is done
      if (h->hstg_used[j]) CK(cudaStreamWaitEvent(h->copy_st, h->consumed[j], 0));
      CK(cudaMemcpy2DAsync(h->hstg[j], es * ldst, A[i], es * lda, es * h->M, B,
                           cudaMemcpyHostToDevice, h->copy_st));
      CK(cudaEventRecord(h->copied[j], h->copy_st));
      CK(cudaStreamWaitEvent(h->st, h->copied[j], 0));
      Ad = h->hstg[j];
      ldd = ldst;
    } else if (int rc = stage_input(h, A[i], lda, h->M, B, dtype, use_tc(h), &Ad, &ldd)) {
      return rc;
    }
    const void* nxt = (lookahead && i + 1 < count && direct(A[i + 1])) ? A[i + 1] : nullptr;
    if (int rc = step(h, Ad, ldd, B, dtype, nxt, lda)) return rc;
    if (host) {
      CK(cudaEventRecord(h->consumed[j], h->st));
      h->hstg_used[j] = true;
    }
    if (s_out)
      CK(cudaMemcpyAsync(s_out + (int64_t)i * h->K, h->D[h->cur], sizeof(double) * h->kc,
                         cudaMemcpyDefault, h->st));
  }
  return PSVD_OK;
}

int psvd_num_modes(psvd_handle h) { return h ? h->kc : PSVD_ERR_INVALID_ARG; }

int psvd_get_modes(psvd_handle h, float* U_out, int64_t ldo) {
  if (!h || !U_out || ldo < h->M) return PSVD_ERR_INVALID_ARG;
  if (h->kc == 0) return PSVD_ERR_NOT_INITIALIZED;
  const float* src = h->U[h->cur];
  if (use_tc(h) || use_f64(h)) {
    if (!h->Uf32_tmp && dalloc(&h->Uf32_tmp, (size_t)h->ldu * h->K)) return PSVD_ERR_ALLOC;
    if (use_tc(h))
      CK(tc_modes_to_f32(h->Ut[h->cur], h->Kp, h->M, h->kc, h->Uf32_tmp, h->ldu, h->st));
    else
      CK(modes_f64_to_f32_launch(h->U64[h->cur], h->ldu, h->M, h->kc, h->Uf32_tmp, h->ldu, h->st));
    src = h->Uf32_tmp;
  }
  CK(cudaMemcpy2DAsync(U_out, sizeof(float) * ldo, src, sizeof(float) * h->ldu,
                       sizeof(float) * h->M, h->kc, cudaMemcpyDefault, h->st));
  return collect_status(h);
}

int psvd_get_modes_f64(psvd_handle h, double* U_out, int64_t ldo) {
  if (!h || !U_out || ldo < h->M) return PSVD_ERR_INVALID_ARG;
  if (!use_f64(h)) return PSVD_ERR_UNSUPPORTED;
  if (h->kc == 0) return PSVD_ERR_NOT_INITIALIZED;
  CK(cudaMemcpy2DAsync(U_out, sizeof(double) * ldo, h->U64[h->cur], sizeof(double) * h->ldu,
                       sizeof(double) * h->M, h->kc, cudaMemcpyDefault, h->st));
  return collect_status(h);
}

int psvd_get_singular_values(psvd_handle h, double* s_out) {
  if (!h || !s_out) return PSVD_ERR_INVALID_ARG;
  if (h->kc == 0) return PSVD_ERR_NOT_INITIALIZED;
  CK(cudaMemcpyAsync(s_out, h->D[h->cur], sizeof(double) * h->kc, cudaMemcpyDefault, h->st));
  return collect_status(h);
}

int psvd_last_info(psvd_handle h, int32_t* info4) {
  if (!h || !info4) return PSVD_ERR_INVALID_ARG;
  int rc = collect_status(h);
  for (int i = 0; i < 4; ++i) info4[i] = h->host_info[i];
  return rc;
}

int psvd_parallel_qr(psvd_handle h, const void* P, int64_t ldp, int32_t n, int32_t dtype,
                     double* R_out) {
  if (!h || !P || !R_out || n < 1 || ldp < h->M) return PSVD_ERR_INVALID_ARG;
  if (dtype != PSVD_F32 && dtype != PSVD_BF16 && dtype != PSVD_F64) return PSVD_ERR_INVALID_ARG;
  if (dtype == PSVD_F64 && !use_f64(h)) return PSVD_ERR_UNSUPPORTED;
  if (n > h->nmax || h->M < n) return PSVD_ERR_SHAPE;
  if (use_tc(h) && dtype != PSVD_BF16) return PSVD_ERR_UNSUPPORTED;
  const void* Pd;
  int64_t ldd;
  if (int rc = stage_input(h, P, ldp, h->M, n, dtype, use_tc(h), &Pd, &ldd)) return rc;
  CK(cudaMemsetAsync(h->w.info, 0, sizeof(int) * 4, h->st));
  if (int rc = panel_gram(h, Pd, ldd, n, dtype, 0, 1.0, h->D[h->cur], h->G)) return rc;
  CK(cholesky_launch(h->G, n, h->w.X, h->w.info, h->st));
  CK(cudaMemcpyAsync(R_out, h->w.X, sizeof(double) * n * n, cudaMemcpyDefault, h->st));
  int rc = collect_status(h);
  CK(cudaMemsetAsync(h->w.info, 0, sizeof(int) * 4, h->st));
  h->sticky_status = 0;
  return rc == PSVD_ERR_NONFINITE ? PSVD_ERR_NONFINITE : PSVD_OK;
}

int psvd_parallel_svd(psvd_handle h, const void* A, int64_t lda, const int64_t* part_offsets,
                      int32_t nparts, int32_t N, int32_t dtype, int32_t r1, int32_t r2,
                      float* U_out, int64_t ldu, double* L_out) {
  if (!h || !A || !part_offsets || !U_out || !L_out || nparts < 1) return PSVD_ERR_INVALID_ARG;
  if (dtype != PSVD_F32 && dtype != PSVD_BF16) return PSVD_ERR_INVALID_ARG;
  if (N < 1 || N > kMaxN || r1 < 1 || r1 > N || r2 < 1 || r2 > N || (int64_t)r2 > (int64_t)r1 * nparts)
    return PSVD_ERR_SHAPE;
  if (part_offsets[0] != 0) return PSVD_ERR_INVALID_ARG;
  for (int b = 0; b < nparts; ++b)
    if (part_offsets[b + 1] - part_offsets[b] < N) return PSVD_ERR_SHAPE;
  const int64_t Mtot = part_offsets[nparts];
  if (lda < Mtot || ldu < Mtot) return PSVD_ERR_INVALID_ARG;
  const void* Ad;
  int64_t ldd;
  if (int rc = stage_input(h, A, lda, Mtot, N, dtype, false, &Ad, &ldd)) return rc;
  // outputs: device pointers are written in place, host ones through temporaries
  const bool u_dev = is_device_ptr(U_out), l_dev = is_device_ptr(L_out);
  float* Ud = U_out;
  double* Ld = L_out;
  int64_t ldud = ldu;
  if (!u_dev) {
    ldud = Mtot;
    if (dalloc(&Ud, (size_t)Mtot * r2)) return PSVD_ERR_ALLOC;
  }
  if (!l_dev && dalloc(&Ld, (size_t)r2)) {
    if (!u_dev) cudaFree(Ud);
    return PSVD_ERR_ALLOC;
  }
  int bits = 0;
  if (!h->apmos) h->apmos = apmos_cache_create();
  int rc = h->apmos ? apmos_run(Ad, ldd, dtype == PSVD_BF16 ? 1 : 0, Mtot, part_offsets, nparts, N,
                                r1, r2, Ud, ldud, Ld, h->num_sms, h->st, h->apmos,
                                h->cfg.low_rank, h->cfg.oversample, h->cfg.power_iters,
                                h->cfg.seed, &bits)
                    : PSVD_ERR_ALLOC;
  if (rc == PSVD_OK && !u_dev &&
      cudaMemcpy2DAsync(U_out, sizeof(float) * ldu, Ud, sizeof(float) * ldud, sizeof(float) * Mtot,
                        r2, cudaMemcpyDeviceToHost, h->st) != cudaSuccess)
    rc = PSVD_ERR_CUDA;
  if (rc == PSVD_OK && !l_dev &&
      cudaMemcpyAsync(L_out, Ld, sizeof(double) * r2, cudaMemcpyDeviceToHost, h->st) != cudaSuccess)
    rc = PSVD_ERR_CUDA;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) rc = PSVD_ERR_CUDA;
  if (!u_dev) cudaFree(Ud);
  if (!l_dev) cudaFree(Ld);
  if (rc != PSVD_OK) return rc;
  if (bits & 4) return PSVD_ERR_NONFINITE;
  return (bits & 1) ? PSVD_WARN_RANK_DEFICIENT : PSVD_OK;
}

int psvd_update_adjoint(psvd_handle h, int32_t kc, const float* U, int64_t ldu, const double* D,
                        const void* A, int64_t lda, int32_t B, int32_t dtype, int32_t k1,
                        const float* U_new, int64_t ld_new, const double* D_new,
                        const float* U_new_bar, int64_t ld_new_bar, const double* D_new_bar,
                        float* U_bar, int64_t ld_bar, double* D_bar, float* A_bar,
                        int64_t lda_bar) {
  if (!h || kc < 0 || B < 1 || k1 < 1) return PSVD_ERR_INVALID_ARG;
  if (dtype != PSVD_F32 && dtype != PSVD_BF16) return PSVD_ERR_INVALID_ARG;
  const int64_t M = h->M;
  const int n = kc + B;
  if (n > kMaxN || k1 > n || k1 > 64 || M < n) return PSVD_ERR_SHAPE;
  if (!A || !U_new || !D_new || !U_new_bar || !D_new_bar || !A_bar) return PSVD_ERR_INVALID_ARG;
  if (kc > 0 && (!U || !D || !U_bar || !D_bar)) return PSVD_ERR_INVALID_ARG;
  if (lda < M || ld_new < M || ld_new_bar < M || lda_bar < M || (kc > 0 && (ldu < M || ld_bar < M)))
    return PSVD_ERR_INVALID_ARG;
  // the M-row operands are read and written in place on the device
  if (!is_device_ptr(A) || !is_device_ptr(U_new) || !is_device_ptr(U_new_bar) ||
      !is_device_ptr(A_bar) || (kc > 0 && (!is_device_ptr(U) || !is_device_ptr(U_bar))))
    return PSVD_ERR_INVALID_ARG;
  if (!h->adj) h->adj = adj_work_create();
  if (!h->adj) return PSVD_ERR_ALLOC;
  int bits = 0;
  const int rc = adjoint_run(h->adj, h->st, h->num_sms, M, h->cfg.ff, kc, U, ldu, D, A, lda,
                             dtype == PSVD_BF16 ? 1 : 0, B, k1, U_new, ld_new, D_new, U_new_bar,
                             ld_new_bar, D_new_bar, U_bar, ld_bar, D_bar, A_bar, lda_bar, &bits);
  if (rc != PSVD_OK) return rc;
  if (bits & 4) return PSVD_ERR_NONFINITE;
  return (bits & 3) ? PSVD_WARN_DEGENERATE : PSVD_OK;
}

// ------------------------------------------------------------------ groups
// Many independent snapshot streams (one handle each, on its own stream) updated
// together: one call forks the members' update sequences onto their streams and
// joins them.  In steady state (every member at K modes, no randomized front end,
// not the tensor-core path) the whole fork/updates/join sequence is captured into
// a CUDA graph, one per double-buffer parity, and replayed while the arguments
// (batch pointers, lda, B, dtype, member states) repeat.
struct psvd_group {
  std::vector<psvd_handle> m;
  std::vector<cudaStream_t> ms;   // member streams (owned)
  std::vector<cudaEvent_t> done;  // per-member join events
  cudaStream_t user = nullptr;    // the configuration's stream
  cudaStream_t origin = nullptr;  // capture origin (owned, non-blocking)
  cudaEvent_t in = nullptr, out = nullptr, fork = nullptr;
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> key;
    std::vector<int64_t> launches;  // per member
  } graph[2];
  int64_t replays = 0, captures = 0;
};

namespace {

void group_free(psvd_group* g) {
  if (!g) return;
  if (g->origin) cudaStreamSynchronize(g->origin);
  for (auto& gr : g->graph)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  for (psvd_handle h : g->m) psvd_destroy(h);
  for (cudaStream_t st : g->ms) cudaStreamDestroy(st);
  for (cudaEvent_t e : g->done) cudaEventDestroy(e);
  if (g->origin) cudaStreamDestroy(g->origin);
  if (g->in) cudaEventDestroy(g->in);
  if (g->out) cudaEventDestroy(g->out);
  if (g->fork) cudaEventDestroy(g->fork);
  cudaGetLastError();
  delete g;
}

// Forks the members' steps off the origin stream and joins them back.
int group_enqueue(psvd_group* g, const void* const* A, int64_t lda, int B, int dtype, bool init) {
  CK(cudaEventRecord(g->fork, g->origin));
  for (size_t i = 0; i < g->m.size(); ++i) {
    psvd_handle h = g->m[i];
    CK(cudaStreamWaitEvent(h->st, g->fork, 0));
    const int rc = init ? psvd_initialize(h, A[i], lda, B, dtype)
                        : psvd_incorporate_data(h, A[i], lda, B, dtype);
    if (rc < 0) return rc;
    CK(cudaEventRecord(g->done[i], h->st));
    CK(cudaStreamWaitEvent(g->origin, g->done[i], 0));
  }
  return PSVD_OK;
}

int group_step(psvd_group* g, const void* const* A, int64_t lda, int32_t B, int32_t dtype,
               bool init) {
  if (!g || !A) return PSVD_ERR_INVALID_ARG;
  const size_t n = g->m.size();
  bool steady = !init;
  for (size_t i = 0; i < n; ++i) {
    psvd_handle h = g->m[i];
    if (!init && h->kc == 0) return PSVD_ERR_NOT_INITIALIZED;
    if (int rc = check_batch(h, A[i], lda, B, dtype)) return rc;
    steady = steady && h->kc == h->K && !h->cfg.low_rank && !use_tc(h) && !h->profiling &&
             is_device_ptr(A[i]);
  }
  CK(cudaEventRecord(g->in, g->user));
  CK(cudaStreamWaitEvent(g->origin, g->in, 0));
  std::vector<int64_t> key;
  if (steady) {
    key = {lda, B, dtype};
    for (size_t i = 0; i < n; ++i) {
      key.push_back((int64_t)(uintptr_t)A[i]);
      key.push_back(g->m[i]->cur);
      // a member retuned by psvd_autotune launches other shapes: capture again
      key.push_back(g->m[i]->tune.gram_ctas_per_sm);
      key.push_back(g->m[i]->tune.update_rows);
    }
  }
  const int parity = n ? g->m[0]->cur : 0;
  psvd_group::Graph& gr = g->graph[parity];
  bool graph_ran = false;
  if (steady && gr.exec && gr.key == key) {
    graph_ran = true;
    CK(cudaGraphLaunch(gr.exec, g->origin));
    // the host-side state the captured steps advanced (kc stays K)
    for (size_t i = 0; i < n; ++i) {
      psvd_handle h = g->m[i];
      h->cur ^= 1;
      h->iteration += 1;
      h->launches += gr.launches[i];
    }
    ++g->replays;
  } else {
    bool captured = false;
    if (steady) {
      // grow the members' Gram partials outside the capture (growing synchronises)
      for (size_t i = 0; i < n; ++i) {
        psvd_handle h = g->m[i];
        int nchunk;
        int64_t rpc, pd;
        gram_simt_plan(h->M, h->kc + B, h->num_sms, &nchunk, &rpc, &pd, h->tune.gram_ctas_per_sm);
        if (int rc = ensure_partial(h, pd)) return rc;
      }
      struct Saved {
        int cur, kc;
        int64_t iteration, launches;
      };
      std::vector<Saved> saved(n);
      for (size_t i = 0; i < n; ++i)
        saved[i] = {g->m[i]->cur, g->m[i]->kc, g->m[i]->iteration, g->m[i]->launches};
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(g->origin, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const int rc = group_enqueue(g, A, lda, B, dtype, false);
        const cudaError_t ec = cudaStreamEndCapture(g->origin, &graph);
        cudaGraphExec_t exec = nullptr;
        if (rc == PSVD_OK && ec == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
          if (gr.exec) cudaGraphExecDestroy(gr.exec);
          gr.exec = exec;
          gr.key = key;
          gr.launches.assign(n, 0);
          for (size_t i = 0; i < n; ++i) gr.launches[i] = g->m[i]->launches - saved[i].launches;
          captured = true;
        }
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();
      if (captured) {
        CK(cudaGraphLaunch(gr.exec, g->origin));
        graph_ran = true;
        ++g->captures;
      } else {
        // nothing was enqueued: undo the host-side steps and run them directly
        for (size_t i = 0; i < n; ++i) {
          psvd_handle h = g->m[i];
          h->cur = saved[i].cur;
          h->kc = saved[i].kc;
          h->iteration = saved[i].iteration;
          h->launches = saved[i].launches;
        }
      }
    }
    if (!captured)
      if (int rc = group_enqueue(g, A, lda, B, dtype, init)) return rc;
  }
  CK(cudaEventRecord(g->out, g->origin));
  CK(cudaStreamWaitEvent(g->user, g->out, 0));
  // a graph runs the members' work on the origin stream: later work on a member's
  // own stream (psvd_get_modes, a direct step) must wait for it
  if (graph_ran)
    for (size_t i = 0; i < n; ++i) CK(cudaStreamWaitEvent(g->m[i]->st, g->out, 0));
  return PSVD_OK;
}

}  // namespace

int psvd_group_create(psvd_group_handle* out, int32_t count, const psvd_config* cfg) {
  if (!out) return PSVD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || count < 1) return PSVD_ERR_INVALID_ARG;
  psvd_group* g = new (std::nothrow) psvd_group();
  if (!g) return PSVD_ERR_ALLOC;
  g->user = (cudaStream_t)cfg->stream;
  bool ok = cudaStreamCreateWithFlags(&g->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->out, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess;
  int rc = ok ? PSVD_OK : PSVD_ERR_CUDA;
  for (int i = 0; rc == PSVD_OK && i < count; ++i) {
    cudaStream_t st = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      rc = PSVD_ERR_CUDA;
      break;
    }
    g->ms.push_back(st);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      rc = PSVD_ERR_CUDA;
      break;
    }
    g->done.push_back(e);
    psvd_config c = *cfg;
    c.stream = st;
    psvd_handle h = nullptr;
    rc = psvd_create(&h, &c);
    if (rc == PSVD_OK) g->m.push_back(h);
  }
  if (rc != PSVD_OK) {
    cudaGetLastError();
    group_free(g);
    return rc;
  }
  *out = g;
  return PSVD_OK;
}

void psvd_group_destroy(psvd_group_handle g) { group_free(g); }

int psvd_group_initialize(psvd_group_handle g, const void* const* A, int64_t lda, int32_t B,
                          int32_t dtype) {
  return group_step(g, A, lda, B, dtype, true);
}

int psvd_group_incorporate_data(psvd_group_handle g, const void* const* A, int64_t lda,
                                int32_t B, int32_t dtype) {
  return group_step(g, A, lda, B, dtype, false);
}

psvd_handle psvd_group_member(psvd_group_handle g, int32_t i) {
  if (!g || i < 0 || (size_t)i >= g->m.size()) return nullptr;
  return g->m[i];
}

int psvd_group_stats(psvd_group_handle g, int64_t* captures, int64_t* replays) {
  if (!g) return PSVD_ERR_INVALID_ARG;
  if (captures) *captures = g->captures;
  if (replays) *replays = g->replays;
  return PSVD_OK;
}

int psvd_group_status(psvd_group_handle g) {
  if (!g) return PSVD_ERR_INVALID_ARG;
  int worst = PSVD_OK;
  for (psvd_handle h : g->m) {
    const int rc = collect_status(h);
    if (rc < 0 && (worst >= 0 || rc < worst)) worst = rc;
    if (worst >= 0 && rc > worst) worst = rc;
  }
  return worst;
}

// ---------------------------------------------------------------- autotuner

namespace {
// psvd_autotune on a tensor-core handle: the Gram's cluster count, then the
// update's CTA count and stage count, each timed on the steady-state panel.
int autotune_tc(psvd_handle h, const void* A, int64_t lda, int32_t B, int32_t* choice) {
  const int n = h->K + B;
  const auto key = std::make_tuple(h->M, n, h->num_sms);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tc_tune_cache.find(key);
    if (it != g_tc_tune_cache.end()) {
      h->tctune = it->second;
      if (choice) {
        choice[0] = h->tctune.gram_clusters;
        choice[1] = h->tctune.upd_ctas;
        choice[2] = h->tctune.upd_stages;
      }
      return PSVD_OK;
    }
  }
  const int max_st = tc_update_max_stages(h->K, B, h->K);
  if (max_st < 2) return PSVD_ERR_SHAPE;
  // the trials read the current modes and write only scratch (the other mode
  // buffer, the Gram partials, w.H, w.T3) and the status word, restored afterwards
  int saved_info[4];
  CK(cudaMemcpyAsync(saved_info, h->w.info, sizeof(saved_info), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const int mx = tc_gram_clusters_max(h->K, B, h->num_sms);
  TcTune best, trial;
  float best_ms = 1e30f;
  const int cands[] = {mx, (2 * mx) / 3, mx / 2, mx / 3};
  for (int i = 0; i < 4; ++i) {
    const int c = cands[i];
    if (c < 1 || (i > 0 && c == cands[i - 1])) continue;
    trial.gram_clusters = c;
    float ms = 0.f;
    int rc = time_ms(h->st, 3, [&]() -> int {
      int r = tc_gram(h->Ut[h->cur], h->Kp, h->K, A, lda, B, PSVD_BF16, h->M, h->num_sms, trial,
                      false, &h->partial, &h->partial_cap, &h->w.info[2], h->st);
      if (r) return r;
      return tc_gram_reduce(h->partial, h->M, h->K, B, h->num_sms, trial, nullptr, 1.0, h->D[h->cur],
                            nullptr, h->w.H, &h->w.info[2], h->st) == cudaSuccess
                 ? PSVD_OK
                 : PSVD_ERR_CUDA;
    }, &ms);
    if (rc) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      best.gram_clusters = c;
    }
  }
  best_ms = 1e30f;
  const int ctas[] = {h->num_sms, h->num_sms / 2};
  for (int c : ctas) {
    for (int stg = 2; stg <= (max_st < 4 ? max_st : 4); ++stg) {
      trial.upd_ctas = c;
      trial.upd_stages = stg;
      float ms = 0.f;
      int rc = time_ms(h->st, 3, [&]() -> int {
        return tc_update(h->Ut[h->cur], h->Kp, h->K, A, lda, B, PSVD_BF16, h->M, h->w.T, n, h->K,
                         h->w.T3, h->Ut[h->cur ^ 1], h->num_sms, trial, &h->w.info[2], h->st);
      }, &ms);
      if (rc) return rc;
      if (ms < best_ms) {
        best_ms = ms;
        best.upd_ctas = c;
        best.upd_stages = stg;
      }
    }
  }
  CK(cudaMemcpyAsync(h->w.info, saved_info, sizeof(saved_info), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  h->tctune = best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tc_tune_cache[key] = best;
  }
  if (choice) {
    choice[0] = best.gram_clusters;
    choice[1] = best.upd_ctas;
    choice[2] = best.upd_stages;
  }
  return PSVD_OK;
}
}  // namespace

int psvd_autotune(psvd_handle h, const void* A, int64_t lda, int32_t B, int32_t dtype,
                  int32_t* choice) {
  if (!h) return PSVD_ERR_INVALID_ARG;
  if (h->cfg.precision == PSVD_PREC_BF16_TC) {
    if (!A || B < 1 || B > h->maxB || lda < h->M || dtype != PSVD_BF16) return PSVD_ERR_INVALID_ARG;
    if (!is_device_ptr(A)) return PSVD_ERR_INVALID_ARG;
    if (h->M < (int64_t)h->K + B) return PSVD_ERR_SHAPE;
    return autotune_tc(h, A, lda, B, choice);
  }
  if (h->cfg.precision != PSVD_PREC_FP32) return PSVD_ERR_UNSUPPORTED;
  if (!A || B < 1 || B > h->maxB || lda < h->M || (dtype != PSVD_F32 && dtype != PSVD_BF16))
    return PSVD_ERR_INVALID_ARG;
  if (!is_device_ptr(A)) return PSVD_ERR_INVALID_ARG;
  const int n = h->K + B;  // the steady-state panel
  if (h->M < n) return PSVD_ERR_SHAPE;
  const auto key = std::make_tuple(h->M, n, (int)dtype, h->num_sms);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      h->tune = it->second;
      if (choice) {
        choice[0] = h->tune.gram_ctas_per_sm;
        choice[1] = h->tune.update_rows;
        choice[2] = 0;
      }
      return PSVD_OK;
    }
  }
  // the trials read the current modes and write only scratch: the other mode
  // buffer (free between steps), the Gram partials, w.H and the status word, which
  // is saved here and restored afterwards
  int saved_info[4];
  CK(cudaMemcpyAsync(saved_info, h->w.info, sizeof(saved_info), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  PanelF32 p{h->U[h->cur], h->ldu, h->K, A, lda, dtype == PSVD_BF16 ? 1 : 0, h->M, n};
  SimtTune best;
  float best_ms = 1e30f;
  static const int kCps[] = {1, 2, 4, 8};
  for (int cps : kCps) {
    int nchunk;
    int64_t rpc, pd;
    gram_simt_plan(h->M, n, h->num_sms, &nchunk, &rpc, &pd, cps);
    if (int rc = ensure_partial(h, pd)) return rc;
    float ms = 0.f;
    int rc = time_ms(h->st, 3, [&]() -> int {
      if (gram_simt_launch(p, nchunk, rpc, h->partial, h->st) != cudaSuccess) return PSVD_ERR_CUDA;
      if (gram_reduce_launch(h->partial, nchunk, n, h->K, h->D[h->cur], 1.0, nullptr, h->w.H,
                             h->w.info, h->st) != cudaSuccess)
        return PSVD_ERR_CUDA;
      return PSVD_OK;
    }, &ms);
    if (rc) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      best.gram_ctas_per_sm = cps;
    }
  }
  best_ms = 1e30f;
  static const int kRows[] = {64, 128, 256};
  for (int rows : kRows) {
    float ms = 0.f;
    int rc = time_ms(h->st, 3, [&]() -> int {
      return update_simt_launch(p, h->w.T, h->K, h->U[h->cur ^ 1], h->ldu, h->st, rows) ==
                     cudaSuccess
                 ? PSVD_OK
                 : PSVD_ERR_CUDA;
    }, &ms);
    if (rc) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      best.update_rows = rows;
    }
  }
  CK(cudaMemcpyAsync(h->w.info, saved_info, sizeof(saved_info), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  h->tune = best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  if (choice) {
    choice[0] = best.gram_ctas_per_sm;
    choice[1] = best.update_rows;
    choice[2] = 0;
  }
  return PSVD_OK;
}

int psvd_set_profiling(psvd_handle h, int32_t enable) {
  if (!h) return PSVD_ERR_INVALID_ARG;
  prof_collect(h);
  h->profiling = enable != 0;
  for (int i = 0; i < 3; ++i) {
    h->prof_ms[i] = 0.0;
    h->prof_count[i] = 0;
  }
  h->launches = 0;
  return PSVD_OK;
}

int psvd_get_profile(psvd_handle h, double* ms_out, int64_t* count_out, int64_t* launches_out) {
  if (!h) return PSVD_ERR_INVALID_ARG;
  prof_collect(h);
  for (int i = 0; i < 3; ++i) {
    if (ms_out) ms_out[i] = h->prof_ms[i];
    if (count_out) count_out[i] = h->prof_count[i];
  }
  if (launches_out) *launches_out = h->launches;
  return PSVD_OK;
}

int psvd_gaussian_sketch(uint64_t seed, uint64_t stream_id, int64_t rows, int64_t cols, float* out,
                         void* stream) {
  if (!out || rows < 0 || cols < 0) return PSVD_ERR_INVALID_ARG;
  CK(gaussian_sketch_launch(seed, stream_id, rows, cols, out, (cudaStream_t)stream));
  return PSVD_OK;
}

// File layout: magic "PSVD0001", psvd_config (stream zeroed), int64 iteration,
// uint64 sketch counter, int32 kc, pad, kc doubles D, M*kc floats U (ld M); then,
// for a tensor-core handle, the Uh and Ul planes (M*kc BF16 each, ld M), for an
// FP64 handle M*kc doubles U (ld M).
int psvd_save(psvd_handle h, const char* path) {
  if (!h || !path) return PSVD_ERR_INVALID_ARG;
  if (h->kc == 0) return PSVD_ERR_NOT_INITIALIZED;
  const size_t nu = (size_t)h->M * h->kc;
  float* U = (float*)malloc(sizeof(float) * (nu ? nu : 1));
  double* D = (double*)malloc(sizeof(double) * h->kc);
  if (!U || !D) { free(U); free(D); return PSVD_ERR_ALLOC; }
  int rc = psvd_get_modes(h, U, h->M);
  if (rc >= 0) rc = psvd_get_singular_values(h, D);
  // TC handles keep the exact hi/lo pair: save it too so a reload is bit-identical
  unsigned short* hl = nullptr;
  if (rc >= 0 && use_tc(h)) {
    // file layout: Uh then Ul, each M x kc column-major
    const size_t nt = tc_modes_elems(h->M, h->K);
    hl = (unsigned short*)malloc(sizeof(unsigned short) * 2 * (nu ? nu : 1));
    unsigned short* tiled = (unsigned short*)malloc(sizeof(unsigned short) * nt);
    if (!hl || !tiled) rc = PSVD_ERR_ALLOC;
    if (rc >= 0 && cudaMemcpy(tiled, h->Ut[h->cur], 2 * nt, cudaMemcpyDeviceToHost)) rc = PSVD_ERR_CUDA;
    if (rc >= 0)
      for (int p = 0; p < 2; ++p)
        for (int c = 0; c < h->kc; ++c)
          for (int64_t r = 0; r < h->M; ++r)
            hl[p * nu + (size_t)c * h->M + r] = tiled[tc_mode_index(r, p, c, h->Kp)];
    free(tiled);
  }
  // FP64 handles keep their FP64 modes: save them too
  double* u64 = nullptr;
  if (rc >= 0 && use_f64(h)) {
    u64 = (double*)malloc(sizeof(double) * (nu ? nu : 1));
    if (!u64) rc = PSVD_ERR_ALLOC;
    if (rc >= 0 && cudaMemcpy2D(u64, sizeof(double) * h->M, h->U64[h->cur], sizeof(double) * h->ldu,
                                sizeof(double) * h->M, h->kc, cudaMemcpyDeviceToHost))
      rc = PSVD_ERR_CUDA;
  }
  FILE* f = nullptr;
  if (rc >= 0) f = fopen(path, "wb");
  if (rc >= 0 && !f) rc = PSVD_ERR_IO;
  if (rc >= 0) {
    psvd_config c = h->cfg;
    c.stream = nullptr;
    const int32_t kc = h->kc, pad = 0;
    bool ok = fwrite("PSVD0001", 1, 8, f) == 8 && fwrite(&c, sizeof c, 1, f) == 1 &&
              fwrite(&h->iteration, 8, 1, f) == 1 && fwrite(&h->sketch_counter, 8, 1, f) == 1 &&
              fwrite(&kc, 4, 1, f) == 1 && fwrite(&pad, 4, 1, f) == 1 &&
              fwrite(D, sizeof(double), kc, f) == (size_t)kc && fwrite(U, sizeof(float), nu, f) == nu;
    if (ok && hl) ok = fwrite(hl, 2, 2 * nu, f) == 2 * nu;
    if (ok && u64) ok = fwrite(u64, sizeof(double), nu, f) == nu;
    if (!ok) rc = PSVD_ERR_IO;
  }
  if (f) fclose(f);
  free(U);
  free(D);
  free(hl);
  free(u64);
  return rc < 0 ? rc : PSVD_OK;
}

int psvd_load(psvd_handle* out, const char* path, void* stream) {
  if (!out || !path) return PSVD_ERR_INVALID_ARG;
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return PSVD_ERR_IO;
  char magic[8];
  psvd_config c;
  int64_t iteration;
  uint64_t counter;
  int32_t kc, pad;
  int rc = PSVD_OK;
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, "PSVD0001", 8) || fread(&c, sizeof c, 1, f) != 1 ||
      fread(&iteration, 8, 1, f) != 1 || fread(&counter, 8, 1, f) != 1 || fread(&kc, 4, 1, f) != 1 ||
      fread(&pad, 4, 1, f) != 1 || kc < 1 || kc > c.K || c.M < 1)
    rc = PSVD_ERR_IO;
  psvd_handle h = nullptr;
  if (!rc) {
    c.stream = stream;
    rc = psvd_create(&h, &c);
    // the buffers are zeroed on the handle's stream: finish that before the copies
    if (!rc && cudaStreamSynchronize(h->st) != cudaSuccess) rc = PSVD_ERR_CUDA;
  }
  const size_t nu = rc ? 0 : (size_t)c.M * kc;
  float* U = rc ? nullptr : (float*)malloc(sizeof(float) * nu);
  double* D = rc ? nullptr : (double*)malloc(sizeof(double) * kc);
  unsigned short* hl = nullptr;
  if (!rc && (!U || !D)) rc = PSVD_ERR_ALLOC;
  if (!rc && (fread(D, sizeof(double), kc, f) != (size_t)kc || fread(U, sizeof(float), nu, f) != nu))
    rc = PSVD_ERR_IO;
  if (!rc && use_tc(h)) {
    hl = (unsigned short*)malloc(2 * 2 * nu);
    if (!hl || fread(hl, 2, 2 * nu, f) != 2 * nu) rc = PSVD_ERR_IO;
  }
  double* u64 = nullptr;
  if (!rc && use_f64(h)) {
    u64 = (double*)malloc(sizeof(double) * nu);
    if (!u64 || fread(u64, sizeof(double), nu, f) != nu) rc = PSVD_ERR_IO;
  }
  fclose(f);
  if (!rc) {
    if (use_tc(h)) {
      // rows beyond M and columns beyond kc stay zero
      const size_t nt = tc_modes_elems(c.M, c.K);
      unsigned short* tiled = (unsigned short*)calloc(nt, sizeof(unsigned short));
      if (!tiled) {
        rc = PSVD_ERR_ALLOC;
      } else {
        for (int p = 0; p < 2; ++p)
          for (int cc = 0; cc < kc; ++cc)
            for (int64_t r = 0; r < c.M; ++r)
              tiled[tc_mode_index(r, p, cc, h->Kp)] = hl[p * nu + (size_t)cc * c.M + r];
        if (cudaMemcpy(h->Ut[0], tiled, 2 * nt, cudaMemcpyHostToDevice)) rc = PSVD_ERR_CUDA;
        free(tiled);
      }
    } else if (use_f64(h)) {
      if (cudaMemcpy2D(h->U64[0], 8 * h->ldu, u64, 8 * c.M, 8 * c.M, kc, cudaMemcpyHostToDevice))
        rc = PSVD_ERR_CUDA;
    } else if (cudaMemcpy2D(h->U[0], 4 * h->ldu, U, 4 * c.M, 4 * c.M, kc, cudaMemcpyHostToDevice)) {
      rc = PSVD_ERR_CUDA;
    }
    if (!rc && cudaMemcpy(h->D[0], D, sizeof(double) * kc, cudaMemcpyHostToDevice)) rc = PSVD_ERR_CUDA;
  }
  free(U);
  free(D);
  free(hl);
  free(u64);
  if (rc) {
    psvd_destroy(h);
    return rc;
  }
  h->cur = 0;
  h->kc = kc;
  h->iteration = iteration;
  h->sketch_counter = counter;
  *out = h;
  return PSVD_OK;
}

}  // extern "C"
