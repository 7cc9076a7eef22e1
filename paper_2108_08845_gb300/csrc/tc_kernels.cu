// tcgen05 tensor-core kernels of the BF16 path of the per-batch update of
// Algorithm 1 (Sec. 3.1).
//
// The modes are stored as a pair of BF16 planes, U = Uh + Ul (16 significant
// bits), slot-tiled (tc_kernels.cuh), the snapshots A in BF16 column-major, so the
// padded panel
//     P' = [Uh (kcp cols) | Ul (kcp cols) | A (Bp cols)],  kcp = roundup(kc, 8)
// is an exact BF16 representation of [U | A] and every product on the tensor
// cores is exact; accumulation is FP32 in tensor memory (TMEM).
//
// tc_gram_kernel: the panel Gram P'^T P' (step 1's R^T R).  P' is streamed in
//   128-row slots by TMA (SWIZZLE_128B, each column's 64-row block one 128-byte
//   row, i.e. the K-major canonical layout with K = rows).  A cluster of CTAs, one
//   per 128 x 128 block (pair of 128-column slabs i <= j), takes every nrange-th
//   slot; each slab is read once and multicast to the CTAs whose blocks use it.
//   Each CTA issues one tcgen05.mma per 16 rows into an FP32 TMEM accumulator;
//   after every slot the epilogue folds that accumulator into a float-float sum
//   held in registers (Fast2Sum), so FP32 rounding only acts on 8-MMA chains.  The
//   cluster blocks are summed in FP64 in a fixed order and Uh/Ul are folded back
//   into U on the small side.
// tc_update_kernel: step 4, U_new = [U | A] T.  T (n x k1, FP32) is split
//   exactly into three BF16 parts, so one MMA with N = 3 * k1p computes the
//   three partial products; P' row tiles of 128 rows are the MN-major A operand
//   (the same TMA layout, two 64-row halves), T3 the K-major B operand resident
//   in shared memory.  Two TMEM accumulators alternate so the epilogue (sum of
//   the three parts, hi/lo split, stores) overlaps the next tile's MMAs.
//
// Warp roles (both kernels): warp 0 issues TMA loads, warp 1 allocates TMEM
// and issues MMAs (one elected thread), the other warps drain TMEM (warp w reads
// the TMEM lanes 32*(w%4) .. 32*(w%4)+31; the Gram has 16 of them, the update 4).
// Every mbarrier wait is bounded by a
// clock budget; on expiry the kernel records an error, stops issuing work,
// waits (bounded) for its own copies and frees its TMEM before returning.
#include <cuda.h>
#include <stdio.h>
#include <stdlib.h>

#include "tc_kernels.cuh"

namespace psvd {
namespace {

constexpr int kRowsStage = 64;            // rows per Gram stage (one 128-byte swizzle row per column)
constexpr int kSlab = 128;                // panel columns per MMA slab (UMMA M)
constexpr int kGramStages = 3;
// Rows per Gram pipeline slot: two 64-row blocks of every column, issued back to
// back, so that DRAM sees 256 contiguous bytes per column instead of 128 (the
// panel is column-major and its columns are far apart).
constexpr int kGramSubs = 2;
// 64-row stages per FP32 accumulation chain before it is folded into the
// float-float totals.  The tensor-core FP32 accumulation has a relative bias that
// grows with the chain (measured about -1.5e-8 per MMA on the Gram diagonal); with
// 8 MMAs per chain the 64-mode subspace of the 256-mode travelling-wave recipe
// (K = 64, B = 128) stays within 5.3e-4 rad of the FP64 result (2.2e-3 with 16).
// One slot (128 rows) is 8 MMAs.
constexpr int kFoldStages = 1;
// Gram CTA: warp 0 issues TMA loads, warp 1 issues MMAs, warps 2-17 drain TMEM
// (warp w reads lane quadrant w % 4; four warps per quadrant, 32 columns each,
// their float-float sums in registers).  Eighteen warps cap the registers at 112
// per thread.
constexpr int kGramEpiWarp0 = 2;
// TMEM accumulators of a Gram CTA (128 columns each, 512 allocated): the MMA warp
// fills one while the draining warps fold the others, so a fold's latency is hidden
// as long as it is shorter than (kGramAcc - 1) slots of MMAs.
constexpr int kGramAcc = 3;
constexpr int kGramEpiWarps = 16;
constexpr int kGramThreads = (kGramEpiWarp0 + kGramEpiWarps) * 32;
constexpr int kUpdRows = 128;             // rows per update tile (UMMA M)
constexpr int kUpdMaxStages = 8;          // bound of the runtime stage count (barrier space)
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on phase `parity`; on expiry sets *abort and the error word.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          int* err, long long budget = kWaitCycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > budget) {
      *abort = 1;
      atomicOr(err, 8);  // err points at the handle's status word
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// As tma_load_2d, delivered to the same shared-memory offset (data and barrier
// bytes) in every CTA of the cluster named in mask.
__device__ __forceinline__ void tma_load_2d_mc(const CUtensorMap* map, uint64_t* bar, void* dst,
                                               int x, int y, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "h"(mask)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// All threads of every CTA of the cluster (a CTA launched without a cluster is one).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols));
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// Arrives (once the issued MMAs complete) on the mbarrier at this offset in every
// CTA of the cluster named in mask.
__device__ __forceinline__ void umma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}
// 16 consecutive TMEM columns of this thread's lane, without waiting.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}


// Fast2Sum fold (Dekker): hi + lo accumulates x, lo collecting the rounding error of
// hi + x.  The error term is exact when |hi| >= |x|, which holds for a running Gram
// total once its first chains are in (one 128-row chain is small next to the sum);
// otherwise at most one rounding of the sum is lost.  Done on packed FP32 pairs
// (add/sub.rn.f32x2: each half rounded exactly as the scalar operation, half the
// instructions).
__device__ __forceinline__ uint64_t add_f32x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub_f32x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ void fold2(uint64_t& hi, uint64_t& lo, uint64_t x) {
  const uint64_t s = add_f32x2(hi, x);
  const uint64_t z = sub_f32x2(s, hi);
  lo = add_f32x2(lo, sub_f32x2(x, z));
  hi = s;
}
__device__ __forceinline__ uint64_t pack_f32x2(uint32_t a, uint32_t b) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ void unpack_f32x2(uint64_t v, float& a, float& b) {
  uint32_t x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(x), "=r"(y) : "l"(v));
  a = __uint_as_float(x);
  b = __uint_as_float(y);
}

// Shared-memory matrix descriptor, SWIZZLE_128B (layout type 2), version 1.
//   K-major:  rows of 128 bytes (64 bf16 along K), 8-row groups SBO = 1024 bytes.
//   MN-major: rows of 128 bytes (64 bf16 along M/N) per K index, 8 K indices per
//             1024-byte atom (SBO), LBO = stride between 64-element M/N atoms.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;  // SWIZZLE_128B
  return d;
}
// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int N, int a_mn_major, int b_mn_major) {
  return (1u << 4)                        // D format: F32
         | (1u << 7)                      // A format: BF16
         | (1u << 10)                     // B format: BF16
         | ((uint32_t)a_mn_major << 15)   // A major-ness (0: K-major, 1: MN-major)
         | ((uint32_t)b_mn_major << 16)   // B major-ness
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(128 >> 4) << 24);  // M / 16
}

struct GramGeom {
  int64_t M;
  int kcp;     // padded mode columns per plane (multiple of 8), 0 at initialisation
  int Bp;      // padded snapshot columns (multiple of 8)
  int np;      // 2*kcp + Bp
  int nslab;   // ceil(np / 128)
  int npair;   // nslab*(nslab+1)/2
  int Kp;              // column stride of the tiled mode planes
  int64_t nslot;       // 128-row slots covering M
  int64_t nrange;      // clusters; cluster r takes slots r, r + nrange, ...
  int fold_stages;     // 64-row stages (4 MMAs each) per FP32 accumulation chain
  int split;           // 1: blocks (0,0) and (0,1) only, slab 0 = [Uh | Ul], slab 1 = A
};

// Tensor maps of the three panel planes (Uh, Ul, A) with boxes of 64 rows x
// {64, 32, 16, 8} columns, so that any 8-aligned column range is tiled exactly.
struct PanelMaps {
  CUtensorMap m[3][4];
};

__device__ __forceinline__ void pair_of(int p, int nslab, int* i, int* j) {
  int a = 0;
  while (p >= nslab - a) {
    p -= nslab - a;
    ++a;
  }
  *i = a;
  *j = a + p;
}

__device__ __forceinline__ int slab_width16(int s, int np) {
  const int w = min(kSlab, np - s * kSlab);
  return (w + 15) & ~15;
}

// Loads slab s (padded-panel columns [128 s, 128 s + 128)) for rows [row, row + 64)
// into dst: each plane's column range inside the slab is tiled by boxes of 64,
// 32, 16 and 8 columns.  The mode planes (src 0, 1) are slot-tiled: their box
// starts at line ((row / 128 * 2 + row / 64 % 2) * 2 + src) * Kp + column; the
// snapshots (src 2) are column-major.  mask != 0: multicast to those CTAs of the
// cluster.
__device__ __forceinline__ void load_slab(const PanelMaps& pm, const GramGeom& g, int s,
                                          uint64_t* bar, uint8_t* dst, int row, uint16_t mask) {
  const int lo = s * kSlab, hi = min(g.np, (s + 1) * kSlab);
  const int start[3] = {0, g.kcp, 2 * g.kcp};
  const int end[3] = {g.kcp, 2 * g.kcp, g.np};
  for (int src = 0; src < 3; ++src) {
    int c = max(lo, start[src]);
    const int c_end = min(hi, end[src]);
    while (c < c_end) {
      const int left = c_end - c;
      const int wi = left >= 64 ? 0 : left >= 32 ? 1 : left >= 16 ? 2 : 3;
      int x = row, y = c - start[src];
      if (src < 2) {
        x = 0;
        y += (((row >> 7) * 2 + ((row >> 6) & 1)) * 2 + src) * g.Kp;
      }
      if (mask)
        tma_load_2d_mc(&pm.m[src][wi], bar, dst + (c - lo) * 128, x, y, mask);
      else
        tma_load_2d(&pm.m[src][wi], bar, dst + (c - lo) * 128, x, y);
      c += 64 >> wi;
    }
  }
}

// One CTA = one 128 x 128 block (slab pair si <= sj) of the Gram over the slots of
// its cluster.  The cluster has one CTA per block (rank = pair index); all CTAs
// use the same stage layout, per 64-row block [slab 0 | slab 1], so a slab lands
// at the same offset in every CTA that uses it.  The 64-row blocks of a slab are
// split between its users: each issues its share as TMA loads multicast to all of
// them (slab 0 to the (0,0) and (0,1) CTAs, slab 1 to the (0,1) and (1,1) CTAs).
// A CTA's full barrier expects all bytes it receives; its empty barrier collects
// the MMA commits of every CTA of the cluster, so no CTA's copy lands in a stage
// that another CTA still reads.
// TMEM: kGramAcc FP32 accumulators (128 columns each) rotate between the MMA warp
// and the epilogue, which folds each finished 128-row partial into a float-float
// running sum held in the draining warps' registers.  The block is written as
// FP64 (hi + lo) to partial[range][pair][128][128].
__global__ void __launch_bounds__(kGramThreads, 1) tc_gram_kernel(const __grid_constant__ PanelMaps pm,
                                                         GramGeom g, double* __restrict__ partial,
                                                         int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int pair = g.npair > 1 ? (int)cluster_rank() : 0;
  const int64_t range = blockIdx.x / g.npair;
  int si, sj;
  pair_of(pair, g.nslab, &si, &sj);
  const bool diag = (si == sj);
  const int sub_bytes = g.nslab * kSlab * 128;    // one 64-row block of every slab
  const int stage_bytes = kGramSubs * sub_bytes;  // one pipeline slot
  uint8_t* stages = base;
  uint64_t* full = (uint64_t*)(stages + (size_t)kGramStages * stage_bytes);
  uint64_t* empty = full + kGramStages;
  uint64_t* acc_full = empty + kGramStages;  // [kGramAcc]
  uint64_t* acc_empty = acc_full + kGramAcc;  // [kGramAcc]
  uint64_t* mma_done = acc_empty + kGramAcc;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nst = range < g.nslot ? (int)((g.nslot - 1 - range) / g.nrange + 1) : 0;
  const int nfold = (int)ceil_div(nst, g.fold_stages);
  const int w = slab_width16(sj, g.np);

  // zero the stage buffers once: columns beyond np inside a slab stay zero
  for (int i = threadIdx.x; i < kGramStages * stage_bytes / 16; i += blockDim.x)
    reinterpret_cast<int4*>(stages)[i] = make_int4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGramStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], g.npair);
    }
    for (int b = 0; b < kGramAcc; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kGramEpiWarps);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  fence_proxy_async_smem();
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // every CTA's barriers exist before any multicast or commit reaches them
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- TMA producer
      // bytes of one 64-row block of slab s; this CTA receives both blocks of
      // slab si and of slab sj
      uint32_t bytes_s[2];
      for (int s = 0; s < 2; ++s)
        bytes_s[s] = s < g.nslab ? (uint32_t)(min(g.np, (s + 1) * kSlab) - s * kSlab) * 128u : 0u;
      const uint32_t expect = kGramSubs * (bytes_s[si] + (diag ? 0u : bytes_s[sj]));
      int stage = 0, issued = 0;
      uint32_t phase = 0;
      for (int st = 0; st < nst && !*abort_flag; ++st) {
        if (issued >= kGramStages && !mbar_wait(&empty[stage], phase ^ 1, abort_flag, err)) break;
        uint8_t* dst = stages + (size_t)stage * stage_bytes;
        const int row = (int)((range + (int64_t)st * g.nrange) * (kGramSubs * kRowsStage));
        mbar_expect_tx(&full[stage], expect);
        // rows of the last slot beyond M are zero-filled by the tensor map
        for (int h = 0; h < kGramSubs; ++h) {
          uint8_t* d = dst + h * sub_bytes;
          if (g.npair == 1) {
            load_slab(pm, g, 0, &full[stage], d, row + h * kRowsStage, 0);
          } else if (g.split) {
            // blocks (0,0) and (0,1): block h of slab 0 from CTA h to both; slab 1
            // only to CTA 1, which loads it itself
            if (pair == h)
              load_slab(pm, g, 0, &full[stage], d, row + h * kRowsStage, (uint16_t)0x3);
            if (pair == 1)
              load_slab(pm, g, 1, &full[stage], d + kSlab * 128, row + h * kRowsStage, 0);
          } else {
            // block h of slab 0: CTA h (h = 0: (0,0), h = 1: (0,1)); of slab 1:
            // CTA 2 - h (h = 0: (1,1), h = 1: (0,1))
            if (pair == h)
              load_slab(pm, g, 0, &full[stage], d, row + h * kRowsStage, (uint16_t)0x3);
            if (pair == 2 - h)
              load_slab(pm, g, 1, &full[stage], d + kSlab * 128, row + h * kRowsStage, (uint16_t)0x6);
          }
        }
        ++issued;
        if (++stage == kGramStages) {
          stage = 0;
          phase ^= 1;
        }
      }
      const int inflight = issued < kGramStages ? issued : kGramStages;
      for (int i = 0; i < inflight; ++i) {
        if (--stage < 0) {
          stage = kGramStages - 1;
          phase ^= 1;
        }
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[stage], phase) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // --------------------------------------------------------- MMA issuer
      const uint32_t idesc = idesc_bf16(w, 0, 0);
      const uint16_t all = (uint16_t)((1u << g.npair) - 1u);
      int stage = 0;
      uint32_t phase = 0;
      int st = 0;
      for (int f = 0; f < nfold; ++f) {
        const int b = f % kGramAcc;
        const uint32_t use = (uint32_t)((f / kGramAcc) & 1);
        if (f >= kGramAcc && !mbar_wait(&acc_empty[b], use ^ 1, abort_flag, err)) break;
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * kSlab);
        bool ok = true;
        for (int k4 = 0; k4 < g.fold_stages && st < nst; ++k4, ++st) {
          if (!mbar_wait(&full[stage], phase, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sbase = smem_u32(stages + (size_t)stage * stage_bytes);
#pragma unroll
          for (int h = 0; h < kGramSubs; ++h) {
            const uint32_t abase = sbase + h * sub_bytes + si * kSlab * 128;
            const uint32_t bbase = sbase + h * sub_bytes + sj * kSlab * 128;
#pragma unroll
            for (int k = 0; k < kRowsStage / 16; ++k) {
              const uint64_t ad = smem_desc(abase + k * 32, 16, 1024);
              const uint64_t bd = smem_desc(bbase + k * 32, 16, 1024);
              umma_bf16(d_tmem, ad, bd, idesc, (k4 > 0 || h > 0 || k > 0) ? 1u : 0u);
            }
          }
          if (g.npair > 1)
            umma_commit_mc(&empty[stage], all);
          else
            umma_commit(&empty[stage]);
          if (++stage == kGramStages) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(&acc_full[b]);
      }
      umma_commit(mma_done);
      const long long t0 = clock64();
      while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else if (warp >= kGramEpiWarp0) {
    // ------------------------------------------------------------- epilogue
    // Warps 2 .. 17: TMEM lane quadrant q = warp % 4 (block rows 32q .. 32q+31),
    // column chunk ch (columns 32 ch .. 32 ch + 31).  The running float-float sums
    // (hi, lo) live in registers.  In a diagonal block a chunk wholly below the
    // diagonal of the quadrant is skipped (the assembly reads the mirror entry).
    const int q = warp & 3, ch = (warp - kGramEpiWarp0) >> 2;
    const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16);
    const int c0 = 32 * ch;
    const bool need = c0 < w && (!diag || c0 + 32 > 32 * q);
    uint64_t hi[16], lo[16];  // columns c0 + 2i, c0 + 2i + 1 packed
    bool ok = true;
    for (int f = 0; f < nfold; ++f) {
      const int b = f % kGramAcc;
      const uint32_t use = (uint32_t)((f / kGramAcc) & 1);
      if (!mbar_wait(&acc_full[b], use, abort_flag, err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (need) {
        // two 16-column pieces, one in registers at a time (the sums take 64)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          uint32_t a[16];
          tmem_ld16_nowait(lane_base + (uint32_t)(b * kSlab + c0 + 16 * p), a);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint64_t x = pack_f32x2(a[2 * i], a[2 * i + 1]);
            if (f == 0) {
              hi[8 * p + i] = x;
              lo[8 * p + i] = 0ull;
            } else {
              fold2(hi[8 * p + i], lo[8 * p + i], x);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    if (ok && nfold > 0 && need) {
      const int row_in_slab = q * 32 + lane;
      double* orow = partial + (((size_t)range * g.npair + pair) * kSlab + row_in_slab) * kSlab;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float h0, h1, l0, l1;
        unpack_f32x2(hi[i], h0, h1);
        unpack_f32x2(lo[i], l0, l1);
        orow[c0 + 2 * i] = (double)h0 + (double)l0;
        orow[c0 + 2 * i + 1] = (double)h1 + (double)l1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no CTA leaves while the cluster may still copy into it or commit to it
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, 512);
}

// Ssum[pair][x][y] = sum over the clusters of the FP64 blocks, in a fixed order.
__global__ void tc_gram_sum_kernel(const double* __restrict__ partial, int64_t nrange, int npair,
                                   double* __restrict__ Ssum) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)npair * kSlab * kSlab;
  if (e >= per) return;
  double s = 0.0;
  for (int64_t r = 0; r < nrange; ++r) s += partial[r * per + e];
  Ssum[e] = s;
}

// G (n x n, logical columns [U (kc) | A (B)]) from Ssum; H = S G S.  A mode
// column of U appears twice in the padded panel (hi and lo plane); its Gram
// entries are the sums over both.
__global__ void tc_gram_assemble_kernel(const double* __restrict__ Ssum,
                                        const double* __restrict__ AAsum, GramGeom g, int kc,
                                        int B, const double* __restrict__ D, double ff,
                                        double* __restrict__ G, double* __restrict__ H,
                                        int* __restrict__ status) {
  const int n = kc + B;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  if (i > j) return;  // computed once, mirrored
  int ci[2], cj[2], ni, nj;
  if (i < kc) { ci[0] = i; ci[1] = g.kcp + i; ni = 2; } else { ci[0] = 2 * g.kcp + (i - kc); ni = 1; }
  if (j < kc) { cj[0] = j; cj[1] = g.kcp + j; nj = 2; } else { cj[0] = 2 * g.kcp + (j - kc); nj = 1; }
  double s = 0.0;
  for (int a = 0; a < ni; ++a)
    for (int b = 0; b < nj; ++b) {
      // each block holds its entries for x <= y (a diagonal block only those)
      const int x = min(ci[a], cj[b]), y = max(ci[a], cj[b]);
      const int sx = x / kSlab, sy = y / kSlab;
      if (g.split && sx == 1) {
        // block (1,1) = A^T A, summed by its own launch
        s += AAsum[(size_t)(x % kSlab) * kSlab + (y % kSlab)];
        continue;
      }
      const int p = sx * g.nslab - sx * (sx - 1) / 2 + (sy - sx);
      s += Ssum[((size_t)p * kSlab + (x % kSlab)) * kSlab + (y % kSlab)];
    }
  const double si = (i < kc) ? ff * D[i] : 1.0;
  const double sj = (j < kc) ? ff * D[j] : 1.0;
  if (G) {
    G[i + (int64_t)j * n] = s;
    G[j + (int64_t)i * n] = s;
  }
  H[i + (int64_t)j * n] = si * sj * s;
  H[j + (int64_t)i * n] = si * sj * s;
  if (!isfinite(s)) atomicOr(status, 4);
}

struct UpdGeom {
  int64_t M;
  int kcp, Bp, np;  // padded panel (as in the Gram)
  int k1, k1p;      // kept modes, padded to 16
  int N;            // 3 * k1p
  int nkb;          // K blocks of 64 panel columns: ceil(np / 64)
  int64_t ntiles;   // row tiles of 128
  int Kp;           // column stride of the tiled mode planes
  int stages;       // pipeline stages (2 .. kUpdMaxStages)
  long long wait;   // clock-cycle budget of the pipeline waits (drains keep kWaitCycles)
};

// T3 (N x npk row-major BF16, npk = 64 * nkb): row part*k1p + j, column = padded
// panel column; the value is the part-th BF16 term of T[logical col][j].
__global__ void tc_pack_T_kernel(const float* __restrict__ T, int n, int kc, UpdGeom u, int npk,
                                 __nv_bfloat16* __restrict__ T3) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)u.N * npk) return;
  const int col = (int)(e % npk), row = (int)(e / npk);
  const int part = row / u.k1p, j = row % u.k1p;
  int lc = -1;  // logical panel column
  if (col < u.kcp) lc = (col < kc) ? col : -1;
  else if (col < 2 * u.kcp) lc = (col - u.kcp < kc) ? col - u.kcp : -1;
  else if (col - 2 * u.kcp < n - kc) lc = kc + (col - 2 * u.kcp);
  float v = 0.f;
  if (lc >= 0 && j < u.k1) {
    const float t = T[lc + (int64_t)j * n];
    const __nv_bfloat16 h = __float2bfloat16_rn(t);
    const float r1 = t - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    v = part == 0 ? __bfloat162float(h) : part == 1 ? __bfloat162float(m) : r2;
  }
  T3[e] = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(192, 1) tc_update_kernel(const __grid_constant__ CUtensorMap mU,
                                                           const __grid_constant__ CUtensorMap mA,
                                                           const __grid_constant__ CUtensorMap mT,
                                                           UpdGeom u, __nv_bfloat16* __restrict__ Ut_new,
                                                           int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int half_bytes = u.np * 128;         // one 64-row half of a tile
  const int stage_bytes = 2 * half_bytes;    // 128 rows
  const int tb_bytes = u.N * 128;            // one 64-column K block of T3
  uint8_t* stages = base;
  uint8_t* tsm = stages + (size_t)u.stages * stage_bytes;
  uint64_t* full = (uint64_t*)(tsm + (size_t)u.nkb * tb_bytes);
  uint64_t* empty = full + u.stages;
  uint64_t* t_full = empty + u.stages;
  uint64_t* acc_full = t_full + 1;   // [2]
  uint64_t* acc_empty = acc_full + 2;  // [2]
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < u.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(t_full, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t tx_bytes = (uint32_t)stage_bytes;

  if (warp == 0) {
    if (lane == 0) {
      // T3 once (K blocks of 64 columns, N rows each)
      mbar_expect_tx(t_full, (uint32_t)(u.nkb * tb_bytes));
      for (int kb = 0; kb < u.nkb; ++kb) tma_load_2d(&mT, t_full, tsm + (size_t)kb * tb_bytes, kb * 64, 0);
      int stage = 0, issued = 0;
      uint32_t phase = 0;
      for (int64_t t = blockIdx.x; t < u.ntiles && !*abort_flag; t += gridDim.x) {
        if (issued >= u.stages && !mbar_wait(&empty[stage], phase ^ 1, abort_flag, err, u.wait))
          break;
        uint8_t* dst = stages + (size_t)stage * stage_bytes;
        mbar_expect_tx(&full[stage], tx_bytes);
        for (int h = 0; h < 2; ++h) {
          const int row = (int)(t * kUpdRows + h * 64);
          uint8_t* d = dst + h * half_bytes;
          if (u.kcp > 0) {
            const int y = (int)((t * 2 + h) * 2) * u.Kp;
            tma_load_2d(&mU, &full[stage], d, 0, y);
            tma_load_2d(&mU, &full[stage], d + u.kcp * 128, 0, y + u.Kp);
          }
          tma_load_2d(&mA, &full[stage], d + 2 * u.kcp * 128, row, 0);
        }
        ++issued;
        if (++stage == u.stages) {
          stage = 0;
          phase ^= 1;
        }
      }
      const int inflight = issued < u.stages ? issued : u.stages;
      for (int i = 0; i < inflight; ++i) {
        if (--stage < 0) {
          stage = u.stages - 1;
          phase ^= 1;
        }
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[stage], phase) && clock64() - t0 < kWaitCycles) {
        }
      }
      const long long t0 = clock64();
      while (!mbar_try_wait(t_full, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // --------------------------------------------------------- MMA issuer
      const uint32_t idesc = idesc_bf16(u.N, 1, 0);  // A MN-major (rows contiguous), B K-major
      bool ok = mbar_wait(t_full, 0, abort_flag, err, u.wait);
      tc_fence_after();
      const uint32_t tbase = smem_u32(tsm);
      int stage = 0;
      uint32_t phase = 0;
      int64_t it = 0;
      for (int64_t t = blockIdx.x; ok && t < u.ntiles; t += gridDim.x, ++it) {
        const int buf = (int)(it & 1);
        const uint32_t use = (uint32_t)((it >> 1) & 1);
        if (it >= 2 && !mbar_wait(&acc_empty[buf], use ^ 1, abort_flag, err, u.wait)) break;
        if (!mbar_wait(&full[stage], phase, abort_flag, err, u.wait)) break;
        tc_fence_after();
        const uint32_t abase = smem_u32(stages + (size_t)stage * stage_bytes);
        const uint32_t d_tmem = tmem_base + (uint32_t)(buf * 256);
        for (int k = 0; k < u.np / 16; ++k) {
          // A: 16 panel columns = two 1024-byte K atoms; LBO = the other 64-row half
          const uint64_t ad = smem_desc(abase + k * 2048, (uint32_t)half_bytes, 1024);
          // B: K block k/4, 32-byte step inside the 128-byte swizzle row
          const uint64_t bd = smem_desc(tbase + (k >> 2) * tb_bytes + (k & 3) * 32, 16, 1024);
          umma_bf16(d_tmem, ad, bd, idesc, k > 0 ? 1u : 0u);
        }
        umma_commit(&empty[stage]);
        umma_commit(&acc_full[buf]);
        if (++stage == u.stages) {
          stage = 0;
          phase ^= 1;
        }
      }
      umma_commit(mma_done);
      const long long t0 = clock64();
      while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int sub = warp & 3;
    int64_t it = 0;
    for (int64_t t = blockIdx.x; t < u.ntiles; t += gridDim.x, ++it) {
      const int buf = (int)(it & 1);
      const uint32_t use = (uint32_t)((it >> 1) & 1);
      if (!mbar_wait(&acc_full[buf], use, abort_flag, err, u.wait)) break;
      tc_fence_after();
      const int64_t row = t * kUpdRows + sub * 32 + lane;
      const uint32_t tl = tmem_base + ((uint32_t)(sub * 32) << 16) + (uint32_t)(buf * 256);
      for (int j0 = 0; j0 < u.k1p; j0 += 32) {
        float h[32], m[32], l[32];
        tmem_ld32(tl + j0, h);
        tmem_ld32(tl + u.k1p + j0, m);
        tmem_ld32(tl + 2 * u.k1p + j0, l);
        if (row < u.M) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int j = j0 + i;
            if (j < u.k1) {
              const float v = (h[i] + m[i]) + l[i];
              const __nv_bfloat16 vh = __float2bfloat16_rn(v);
              const __nv_bfloat16 vl = __float2bfloat16_rn(v - __bfloat162float(vh));
              Ut_new[tc_mode_index(row, 0, j, u.Kp)] = vh;
              Ut_new[tc_mode_index(row, 1, j, u.Kp)] = vl;
            }
          }
        }
      }
      tc_fence_before();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, 512);
}

__global__ void tc_modes_to_f32_kernel(const __nv_bfloat16* __restrict__ Ut, int Kp, int64_t M,
                                       int k, float* __restrict__ out, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * k) return;
  const int64_t r = e % M, c = e / M;
  out[r + c * ldo] = __bfloat162float(Ut[tc_mode_index(r, 0, (int)c, Kp)]) +
                     __bfloat162float(Ut[tc_mode_index(r, 1, (int)c, Kp)]);
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2-D BF16 tensor map of a column-major matrix (rows x cols, leading dim ld),
// box = 64 rows x box_cols columns, 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap* m, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || box_cols < 1 || box_cols > 256) return false;
  if (((uintptr_t)ptr & 15) || ((ld * 2) & 15)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {64u, (cuuint32_t)box_cols};
  const cuuint32_t estr[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D BF16 tensor map of a tiled mode buffer seen as nlines lines of 64 elements
// (128 bytes), box = box_lines lines, 128-byte swizzle.
bool make_map_lines(CUtensorMap* m, const void* ptr, int64_t nlines, int box_lines) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || box_lines < 1 || box_lines > 256 || ((uintptr_t)ptr & 15)) return false;
  const cuuint64_t dims[2] = {64, (cuuint64_t)nlines};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {64u, (cuuint32_t)box_lines};
  const cuuint32_t estr[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

GramGeom gram_geom(int64_t M, int kc, int B, int max_clusters, int Kp, bool split = false) {
  GramGeom g;
  g.M = M;
  g.Kp = Kp;
  g.kcp = (kc + 7) & ~7;
  g.Bp = (B + 7) & ~7;
  g.np = 2 * g.kcp + g.Bp;
  g.nslab = (int)ceil_div(g.np, kSlab);
  g.split = split ? 1 : 0;
  g.npair = split ? 2 : g.nslab * (g.nslab + 1) / 2;
  // every cluster resident at once; the clusters interleave slot by slot, so that
  // the CTAs in flight read neighbouring rows of every column
  g.nslot = ceil_div(M, (int64_t)kGramSubs * kRowsStage);
  int64_t want = max_clusters;
  if (want > g.nslot) want = g.nslot;
  g.nrange = want < 1 ? 1 : want;
  g.fold_stages = kFoldStages;
  return g;
}

size_t gram_smem() { return 1024 + (size_t)kGramStages * kGramSubs * 2 * kSlab * 128 + 256; }

// Clusters of npair Gram CTAs that are resident at once (cached per cluster size).
int gram_max_clusters(int npair, int num_sms) {
  static int cached[4] = {0, 0, 0, 0};
  if (npair < 1 || npair > 3) return 1;
  if (cached[npair] > 0) return cached[npair];
  int n = 0;
  const size_t smem = gram_smem();
  if (cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
      cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(npair * (num_sms / npair)));
    cfg.blockDim = dim3(kGramThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)npair;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, tc_gram_kernel, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  if (n < 1) n = num_sms / npair;
  if (n < 1) n = 1;
  cached[npair] = n;
  return n;
}

}  // namespace

// Pipeline-wait budget of tc_update_kernel (psvd_debug_set_wait_budget; 0 = default).
long long g_update_wait = 0;

int tc_set_wait_budget(int kernel, long long cycles) {
  if (kernel != 1 || cycles < 0) return PSVD_ERR_INVALID_ARG;
  g_update_wait = cycles;
  return PSVD_OK;
}

size_t tc_t3_elems(int K, int maxB) {
  const int k1p = (K + 15) & ~15;
  const int np = (2 * ((K + 7) & ~7) + ((maxB + 7) & ~7) + 15) & ~15;
  return (size_t)3 * k1p * (size_t)(ceil_div(np, 64) * 64);
}

namespace {

}  // namespace

size_t tc_modes_elems(int64_t M, int K) {
  return (size_t)ceil_div(M, (int64_t)128) * 4 * (size_t)((K + 7) & ~7) * 64;
}

int tc_gram_clusters_max(int kc, int B, int num_sms) {
  const int np = 2 * ((kc + 7) & ~7) + ((B + 7) & ~7);
  return gram_max_clusters(np > kSlab ? 3 : 1, num_sms);
}

namespace {
// Clusters of one Gram launch: the tuned count, capped at the resident maximum.
int gram_clusters(int kc, int B, int num_sms, const TcTune& tune) {
  const int mx = tc_gram_clusters_max(kc, B, num_sms);
  return (tune.gram_clusters > 0 && tune.gram_clusters < mx) ? tune.gram_clusters : mx;
}
}  // namespace

bool tc_gram_can_split(int kc, int B) {
  return 2 * ((kc + 7) & ~7) == kSlab && B >= 1 && ((B + 7) & ~7) <= kSlab;
}

namespace {
// Geometry of one Gram launch: split mode (blocks (0,0) and (0,1) in clusters of
// two) takes the resident maximum of such clusters; at most `clusters` > 0 of the
// others when given, else the tuned count.
GramGeom launch_geom(int64_t M, int kc, int B, int num_sms, const TcTune& tune, int Kp, bool split,
                     int clusters) {
  if (split) return gram_geom(M, kc, B, gram_max_clusters(2, num_sms), Kp, true);
  int c = gram_clusters(kc, B, num_sms, tune);
  if (clusters > 0 && clusters < c) c = clusters;
  return gram_geom(M, kc, B, c, Kp);
}

int gram_launch(const __nv_bfloat16* Ut, int Kp, int kc, const void* A, int64_t lda, int B,
                const GramGeom& g, double** partial, int64_t* partial_cap, int* status,
                cudaStream_t st);
}  // namespace

int tc_gram(const __nv_bfloat16* Ut, int Kp, int kc, const void* A, int64_t lda, int B, int dtype,
            int64_t M, int num_sms, const TcTune& tune, bool split, double** partial,
            int64_t* partial_cap, int* status, cudaStream_t st) {
  if (dtype != PSVD_BF16) return PSVD_ERR_UNSUPPORTED;
  const int np = 2 * ((kc + 7) & ~7) + ((B + 7) & ~7);
  if (np > 256 || M > 0x7fffffffll - 256) return PSVD_ERR_SHAPE;
  if (kc > Kp) return PSVD_ERR_SHAPE;
  if (split && !tc_gram_can_split(kc, B)) return PSVD_ERR_SHAPE;
  const GramGeom g = launch_geom(M, kc, B, num_sms, tune, Kp, split, 0);
  return gram_launch(Ut, Kp, kc, A, lda, B, g, partial, partial_cap, status, st);
}

int tc_gram_aa(const void* A, int64_t lda, int B, int64_t M, int num_sms, int clusters,
               double** partial, int64_t* partial_cap, double* AAsum, int* status,
               cudaStream_t st) {
  if (B < 1 || B > kSlab || M > 0x7fffffffll - 256) return PSVD_ERR_SHAPE;
  TcTune none;
  const GramGeom g = launch_geom(M, 0, B, num_sms, none, 0, false, clusters);
  if (int rc = gram_launch(nullptr, 0, 0, A, lda, B, g, partial, partial_cap, status, st)) return rc;
  tc_gram_sum_kernel<<<(unsigned)ceil_div((int64_t)kSlab * kSlab, 256), 256, 0, st>>>(*partial,
                                                                                  g.nrange, 1, AAsum);
  return cudaGetLastError() == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

namespace {
int gram_launch(const __nv_bfloat16* Ut, int Kp, int kc, const void* A, int64_t lda, int B,
                const GramGeom& g, double** partial, int64_t* partial_cap, int* status,
                cudaStream_t st) {
  const int64_t M = g.M;
  PanelMaps pm;
  const int64_t nlines = ceil_div(M, (int64_t)128) * 4 * Kp;
  for (int wi = 0; wi < 4; ++wi) {
    const int bw = 64 >> wi;
    if (!make_map(&pm.m[2][wi], A, M, B, lda, bw)) return PSVD_ERR_INVALID_ARG;
    if (kc > 0) {
      if (!make_map_lines(&pm.m[0][wi], Ut, nlines, bw)) return PSVD_ERR_INVALID_ARG;
      pm.m[1][wi] = pm.m[0][wi];
    } else {
      pm.m[0][wi] = pm.m[2][wi];
      pm.m[1][wi] = pm.m[2][wi];
    }
  }
  // FP64 range blocks followed by their sums (one buffer)
  const int64_t per = (int64_t)g.npair * kSlab * kSlab;
  const int64_t need = g.nrange * per + per;
  if (need > *partial_cap) {
    if (*partial) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return PSVD_ERR_CUDA;
      cudaFree(*partial);
      *partial = nullptr;
    }
    if (cudaMalloc((void**)partial, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      *partial_cap = 0;
      return PSVD_ERR_ALLOC;
    }
    *partial_cap = need;
  }
  // columns of a block beyond the slab width are never written: keep them zero
  if (cudaMemsetAsync(*partial, 0, sizeof(double) * g.nrange * per, st) != cudaSuccess)
    return PSVD_ERR_CUDA;
  const size_t smem = gram_smem();
  if (cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
    return PSVD_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(g.nrange * g.npair));
  cfg.blockDim = dim3(kGramThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)g.npair;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, tc_gram_kernel, pm, g, *partial, status) != cudaSuccess) {
    cudaGetLastError();
    return PSVD_ERR_CUDA;
  }
  return PSVD_OK;
}
}  // namespace

cudaError_t tc_gram_reduce(const double* partial, int64_t M, int kc, int B, int num_sms,
                           const TcTune& tune, const double* AAsum, double ff, const double* D,
                           double* G, double* H, int* status, cudaStream_t st) {
  const GramGeom g = launch_geom(M, kc, B, num_sms, tune, 0, AAsum != nullptr, 0);
  const int64_t per = (int64_t)g.npair * kSlab * kSlab;
  double* Ssum = const_cast<double*>(partial) + g.nrange * per;
  tc_gram_sum_kernel<<<(unsigned)ceil_div(per, 256), 256, 0, st>>>(partial, g.nrange, g.npair, Ssum);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = kc + B;
  const int64_t tot = (int64_t)n * n;
  tc_gram_assemble_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Ssum, AAsum, g, kc, B, D, ff,
                                                                        G, H, status);
  return cudaGetLastError();
}

namespace {
// Shared memory of the update kernel: stages of 128 panel rows, T3 resident,
// barriers.
size_t update_smem(int np, int nkb, int N, int stages) {
  return 1024 + (size_t)stages * 2 * np * 128 + (size_t)nkb * N * 128 + 256;
}
constexpr size_t kMaxDynSmem = 232448;
}  // namespace

int tc_update_max_stages(int kc, int B, int k1) {
  const int np = (2 * ((kc + 7) & ~7) + ((B + 7) & ~7) + 15) & ~15;
  const int N = 3 * ((k1 + 15) & ~15);
  const int nkb = (int)ceil_div(np, 64);
  int s = 0;
  while (s < kUpdMaxStages && update_smem(np, nkb, N, s + 1) <= kMaxDynSmem) ++s;
  return s >= 2 ? s : 0;
}

int tc_update(const __nv_bfloat16* Ut, int Kp, int kc, const void* A, int64_t lda, int B, int dtype,
              int64_t M, const float* T, int n, int k1, __nv_bfloat16* T3, __nv_bfloat16* Ut_new,
              int num_sms, const TcTune& tune, int* status, cudaStream_t st) {
  if (dtype != PSVD_BF16) return PSVD_ERR_UNSUPPORTED;
  UpdGeom u{};
  u.M = M;
  u.kcp = (kc + 7) & ~7;
  u.Bp = (B + 7) & ~7;
  u.np = 2 * u.kcp + u.Bp;
  u.np = (u.np + 15) & ~15;  // MMA K steps of 16 columns (extra columns read as zero)
  u.k1 = k1;
  u.k1p = (k1 + 15) & ~15;
  u.N = 3 * u.k1p;
  u.nkb = (int)ceil_div(u.np, 64);
  u.ntiles = ceil_div(M, kUpdRows);
  u.Kp = Kp;
  u.wait = g_update_wait > 0 ? g_update_wait : kWaitCycles;
  if (u.np > 256 || u.N > 256 || M > 0x7fffffffll) return PSVD_ERR_SHAPE;
  const int npk = u.nkb * 64;
  const int64_t tcount = (int64_t)u.N * npk;
  tc_pack_T_kernel<<<(unsigned)ceil_div(tcount, 256), 256, 0, st>>>(T, n, kc, u, npk, T3);
  if (cudaGetLastError() != cudaSuccess) return PSVD_ERR_CUDA;
  CUtensorMap mU, mA, mT;
  // the A operand spans np (16-padded) columns: the maps deliver zeros past the data
  if (!make_map(&mA, A, M, B, lda, u.np - 2 * u.kcp)) return PSVD_ERR_INVALID_ARG;
  if (kc > 0) {
    if (u.kcp > Kp || !make_map_lines(&mU, Ut, ceil_div(M, (int64_t)128) * 4 * Kp, u.kcp))
      return PSVD_ERR_INVALID_ARG;
  } else {
    mU = mA;
  }
  // T3 is N rows x npk columns, row-major: a "column-major" npk x N matrix
  if (!make_map(&mT, T3, npk, u.N, npk, u.N)) return PSVD_ERR_INVALID_ARG;
  // the tuned stage count, capped at what fits; two at least
  const int max_st = tc_update_max_stages(kc, B, k1);
  if (max_st < 2) return PSVD_ERR_SHAPE;
  u.stages = tune.upd_stages < 2 ? 2 : (tune.upd_stages > max_st ? max_st : tune.upd_stages);
  const size_t smem = update_smem(u.np, u.nkb, u.N, u.stages);
  if (cudaFuncSetAttribute(tc_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
    return PSVD_ERR_CUDA;
  const int ctas = (tune.upd_ctas > 0 && tune.upd_ctas < num_sms) ? tune.upd_ctas : num_sms;
  const int grid = (int)(u.ntiles < ctas ? u.ntiles : ctas);
  tc_update_kernel<<<grid, 192, smem, st>>>(mU, mA, mT, u, Ut_new, status);
  return cudaGetLastError() == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

cudaError_t tc_modes_to_f32(const __nv_bfloat16* Ut, int Kp, int64_t M, int k, float* out,
                            int64_t ldo, cudaStream_t st) {
  const int64_t tot = M * k;
  if (tot == 0) return cudaSuccess;
  tc_modes_to_f32_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Ut, Kp, M, k, out, ldo);
  return cudaGetLastError();
}

}  // namespace psvd
