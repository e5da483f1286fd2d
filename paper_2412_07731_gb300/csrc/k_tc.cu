// Tensor-core trailing update of the FP32 block factors (sm_103a: tcgen05,
// tensor memory, bulk TMA).
//
// Step k of the batched partial Cholesky (the block factorisation and Schur-
// contribution steps of Alg. 2, here on the augmented matrices
// [M_i G_i; G_i' C_i]) subtracts L_Ik L_Jk' from every trailing tile pair
// (I, J), J <= I.  After the panel kernel has solved panel column k, it also
// writes each panel tile in the operand layout of the tensor core, split
// into two TF32 words: hi = tf32(x), lo = tf32(x - hi) (the "3xTF32"
// product hi*hi + hi*lo + lo*hi keeps FP32-level accuracy; only lo*lo,
// about 2^-22 relative, is dropped).  One CTA here computes a 128 x 64 block
// of the update -- rows of the tile pair (I0, I0 + 1), columns of tile J:
//
//   * one thread issues bulk copies (cp.async.bulk, completion counted on an
//     mbarrier) of the pre-laid-out operand tiles into shared memory;
//   * one thread issues 3 x 8 tcgen05.mma (kind::tf32, M = 128, N = 64,
//     K = 8 each) accumulating the product in tensor memory, then commits
//     them to a second mbarrier;
//   * the four warps read the 128 x 64 FP32 accumulator back (tcgen05.ld,
//     warp w owns TMEM lanes 32w..32w+31 = rows), write -P into a shared-
//     memory tile (zero where the global row is above the column, so the
//     upper triangle of diagonal tiles is left as it is), and one thread
//     issues a bulk tensor reduce-add (cp.reduce.async.bulk.tensor) of that
//     tile into the block's matrix: the read-modify-write of C happens in L2,
//     and rows past the matrix order are clipped by the tensor map.
//
// Every wait is bounded (1 s of %globaltimer); on expiry the kernel records
// the failure in the factor's status word, waits (bounded again) for its own
// operations in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <new>

#include "ahlp_internal.h"

namespace ahlp {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128, kTcN = 64;
constexpr uint32_t kTileBytes = NB * NB * 4;            // one staged 64x64 FP32 tile
constexpr uint32_t kSmemA = 2 * kTileBytes;             // 128 rows x 64 k
constexpr uint32_t kSmemB = kTileBytes;                 // 64 rows x 64 k
constexpr uint32_t kSmemBytes = 2 * kSmemA + 2 * kSmemB + 1024;   // hi/lo of A and B + alignment
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for phase `parity` of the barrier; false when it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try(bar, parity))
    if (globaltimer() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand without swizzling:
// 8-row x 16-byte core matrices, LBO = byte distance between core matrices
// adjacent in K, SBO = byte distance between adjacent 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the tcgen05 family
  return d;                 // base offset 0, absolute LBO, no swizzle
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, M = 128, N = 64.
constexpr uint32_t kIdescTf32 = (1u << 4)                    // D format F32
                                | (2u << 7)                  // A format TF32
                                | (2u << 10)                 // B format TF32
                                | ((uint32_t)(kTcN >> 3) << 17)
                                | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescTf32), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                   "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 bits, 32 consecutive columns: register j <- column col + j of
// this warp's lane quarter
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
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
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// One update job of step k: block b, the row tile pair (I0, I0 + 1) (the
// second one only when has_i1) and the column tile J.  The jobs of a step are
// numbered block after block (joff: prefix over the blocks); inside a block
// with t trailing tiles, row pair R holds min(2R + 2, t) jobs, so the jobs
// before it number R(R + 1).
struct Job {
  int b, I0, J;
  bool has_i1;
};

__device__ __forceinline__ Job decode_job(const int *joff, int nblk, int k, const BlkInfo *blk,
                                          int q, const int4 *jt) {
  if (jt) {   // tile-sparse: the kept jobs of this step, in the dense order
    const int4 v = jt[q];
    Job j;
    j.b = v.x;
    j.I0 = v.y;
    j.J = v.z;
    j.has_i1 = v.w != 0;
    return j;
  }
  int lo = 0, hi = nblk;   // joff[lo] <= q < joff[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (joff[mid] <= q) lo = mid;
    else hi = mid;
  }
  const int t = blk[lo].T - k - 1;
  const long long local = q - joff[lo];
  long long R = (long long)((sqrt(4.0 * (double)local + 1.0) - 1.0) * 0.5);
  while (R * (R + 1) > local) --R;
  while ((R + 1) * (R + 2) <= local) ++R;
  Job j;
  j.b = lo;
  j.I0 = k + 1 + 2 * (int)R;
  j.J = k + 1 + (int)(local - R * (R + 1));
  j.has_i1 = 2 * R + 1 < t;
  return j;
}

struct TcArgs {
  const float *stage;      // staged panel tiles: per slot 4096 hi then 4096 lo words
  const int *joff;         // [nblk + 1] job prefix of this step over the blocks
  const BlkInfo *blk;
  const CUtensorMap *tmap; // [nblk] each block's FP32 augmented matrix
  int nblk, k;
  int *status;             // status[4] := 1 when a bounded wait ran out
  const int4 *jt;          // this step's tile-sparse job table, or nullptr
};

__global__ void __launch_bounds__(kTcThreads) pchol_update_tc_kernel(const TcArgs args) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  // operands, 1024-aligned: A hi, A lo (128 x 64 each), B hi, B lo (64 x 64)
  unsigned char *base =
      tc_raw + ((1024 - (smem_u32(tc_raw) & 1023)) & 1023);
  float *a_hi = reinterpret_cast<float *>(base);
  float *a_lo = reinterpret_cast<float *>(base + kSmemA);
  float *b_hi = reinterpret_cast<float *>(base + 2 * kSmemA);
  float *b_lo = reinterpret_cast<float *>(base + 2 * kSmemA + kSmemB);

  // ---- which block and tiles ------------------------------------------------
  const Job jb = decode_job(args.joff, args.nblk, args.k, args.blk, blockIdx.x, args.jt);
  const int b = jb.b, I0 = jb.I0, J = jb.J;
  const bool has_i1 = jb.has_i1;
  const BlkInfo bi = args.blk[b];
  const float *st0 = args.stage + (bi.soff + I0) * 8192LL;
  const float *st1 = args.stage + (bi.soff + I0 + 1) * 8192LL;
  const float *stJ = args.stage + (bi.soff + J) * 8192LL;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar_ld = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"((uint32_t)kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(bar_ld, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // ---- operands into shared memory (bulk copies) ---------------------------
  if (threadIdx.x == 0) {
    const uint32_t bytes = (has_i1 ? 6u : 4u) * kTileBytes;
    mbar_expect_tx(bar_ld, bytes);
    bulk_g2s(smem_u32(a_hi), st0, kTileBytes, bar_ld);
    bulk_g2s(smem_u32(a_lo), st0 + 4096, kTileBytes, bar_ld);
    if (has_i1) {
      bulk_g2s(smem_u32(a_hi) + kTileBytes, st1, kTileBytes, bar_ld);
      bulk_g2s(smem_u32(a_lo) + kTileBytes, st1 + 4096, kTileBytes, bar_ld);
    }
    bulk_g2s(smem_u32(b_hi), stJ, kTileBytes, bar_ld);
    bulk_g2s(smem_u32(b_lo), stJ + 4096, kTileBytes, bar_ld);
    // ---- the product: lo*hi, hi*lo, then hi*hi, each over K = 64 ----------
    bool ok = mbar_wait(bar_ld, 0);
    if (ok) {
      tc_fence_after();
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
      const uint32_t bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      const uint32_t pa[3] = {al, ah, ah}, pb[3] = {bh, bl, bh};
#pragma unroll
      for (int pass = 0; pass < 3; ++pass)
#pragma unroll
        for (int s = 0; s < NB / 8; ++s) {
          // K step s: two 16-byte core-matrix columns, 2 x 128 bytes further
          const uint64_t da = smem_desc(pa[pass] + s * 256, 128, 2048);
          const uint64_t db = smem_desc(pb[pass] + s * 256, 128, 2048);
          mma_tf32(tmem, da, db, (pass | s) != 0);
        }
      mma_commit(bar_mma);
      ok = mbar_wait(bar_mma, 0);
      if (!ok) s_fail = 2;
    } else {
      s_fail = 1;
    }
  }
  __syncthreads();
  tc_fence_after();
  const int fail = s_fail;
  if (fail) {
    if (threadIdx.x == 0) {
      atomicExch(&args.status[4], 1);
      // what is still in flight must land before the memory goes away
      if (fail == 1) mbar_wait(bar_ld, 0);
      else mbar_wait(bar_mma, 0);
    }
    __syncthreads();
  } else {
    // ---- epilogue: -P into a 64-column x 128-row tile, then reduce-add ----
    // (A's operands are dead once the MMAs completed: reuse their memory)
    float *out = a_hi;   // [64 columns][128 rows], the tensor map's box order
    const int r = warp * 32 + lane;            // row of the 128-row block
    const int grow = I0 * NB + r;              // row in the block's matrix
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(half * 32), v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int gcol = J * NB + half * 32 + j;
        out[(half * 32 + j) * kTcM + r] = grow >= gcol ? -v[j] : 0.0f;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      const CUtensorMap *tm = args.tmap + b;
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
      asm volatile(
          "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], "
          "[%3];" ::"l"(tm),
          "r"(I0 * NB), "r"(J * NB), "r"(smem_u32(out))
          : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)kTcN)
                 : "memory");
}



// --------------------------------------------------------------------------
// The same FP32 update as a persistent, warp-specialised pipeline: one CTA
// per SM walks the step's jobs (job blockIdx.x, + gridDim.x, ...), and its
// warps overlap consecutive jobs --
//   warp 0  producer: bulk copies of job j's operands into smem stage j % 2,
//           once the MMAs of job j - 2 have released that stage;
//   warp 1  MMA issuer: the 24 MMAs of job j into TMEM accumulator j % 2, once
//           its operands have landed and the epilogue has drained job j - 2
//           from that accumulator; its commits release the stage and hand the
//           accumulator to the epilogue;
//   warps 2-5  epilogue: accumulator -> -P in a staging tile -> one tensor
//           reduce-add into the block's matrix, while the next job's copies
//           and MMAs run.
// mbarrier phases alternate per use of a stage / accumulator; every wait is
// bounded as in the kernel above.
// --------------------------------------------------------------------------
constexpr int kTc2Threads = 192;
constexpr uint32_t kTc2Stage = 2 * kSmemA + 2 * kSmemB;             // 96 KB of operands
constexpr uint32_t kTc2Smem = 2 * kTc2Stage + kTcM * kTcN * 4 + 1024;  // 2 stages + staging

__global__ void __launch_bounds__(kTc2Threads, 1) pchol_update_tc2_kernel(const TcArgs args,
                                                                         int njobs) {
  extern __shared__ __align__(1024) unsigned char tc2_raw[];
  __shared__ __align__(8) uint64_t full[2], empty[2], tfull[2], tempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail, s_epi_fail;
  unsigned char *base = tc2_raw + ((1024 - (smem_u32(tc2_raw) & 1023)) & 1023);
  float *stage_out = reinterpret_cast<float *>(base + 2 * kTc2Stage);   // [64 cols][128 rows]
  volatile int *vfail = &s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int myjobs = (int)blockIdx.x < njobs ? (njobs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                                             : 0;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(2u * kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    s_fail = 0;
    s_epi_fail = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), 1);
      mbar_init(smem_u32(&tfull[i]), 1);
      mbar_init(smem_u32(&tempty[i]), kTcM);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- producer: operands of job j into stage j % 2 -----------------------
    if (lane == 0) {
      int issued = 0;
      for (int j = 0; j < myjobs && !*vfail; ++j) {
        const int st = j & 1;
        if (!mbar_wait(smem_u32(&empty[st]), ((j >> 1) & 1) ^ 1)) {
          atomicExch(&s_fail, 1);
          break;
        }
        const Job jb = decode_job(args.joff, args.nblk, args.k, args.blk,
                                (int)blockIdx.x + j * (int)gridDim.x, args.jt);
        const BlkInfo bi = args.blk[jb.b];
        const float *st0 = args.stage + (bi.soff + jb.I0) * 8192LL;
        const float *stJ = args.stage + (bi.soff + jb.J) * 8192LL;
        const uint32_t sa = smem_u32(base + st * kTc2Stage);
        const uint32_t bar = smem_u32(&full[st]);
        mbar_expect_tx(bar, (jb.has_i1 ? 6u : 4u) * kTileBytes);
        bulk_g2s(sa, st0, kTileBytes, bar);                                 // A hi, rows 0..63
        bulk_g2s(sa + kSmemA, st0 + 4096, kTileBytes, bar);                 // A lo
        if (jb.has_i1) {                                                    // rows 64..127
          bulk_g2s(sa + kTileBytes, st0 + 8192, kTileBytes, bar);
          bulk_g2s(sa + kSmemA + kTileBytes, st0 + 8192 + 4096, kTileBytes, bar);
        }
        bulk_g2s(sa + 2 * kSmemA, stJ, kTileBytes, bar);                    // B hi
        bulk_g2s(sa + 2 * kSmemA + kSmemB, stJ + 4096, kTileBytes, bar);    // B lo
        issued = j + 1;
      }
      if (*vfail)   // copies still in flight (the last two jobs) land before exit
        for (int j = issued >= 2 ? issued - 2 : 0; j < issued; ++j)
          mbar_wait(smem_u32(&full[j & 1]), (j >> 1) & 1);
    }
  } else if (warp == 1) {
    // ---- MMA issuer: job j into accumulator j % 2 ---------------------------
    if (lane == 0) {
      int committed = 0;
      for (int j = 0; j < myjobs && !*vfail; ++j) {
        const int st = j & 1;
        if (!mbar_wait(smem_u32(&full[st]), (j >> 1) & 1) ||
            !mbar_wait(smem_u32(&tempty[st]), ((j >> 1) & 1) ^ 1)) {
          atomicExch(&s_fail, 2);
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(base + st * kTc2Stage);
        const uint32_t ah = sa, al = sa + kSmemA, bh = sa + 2 * kSmemA, bl = bh + kSmemB;
        const uint32_t pa[3] = {al, ah, ah}, pb[3] = {bh, bl, bh};
        const uint32_t d = tmem + (uint32_t)(st * kTcN);
#pragma unroll
        for (int pass = 0; pass < 3; ++pass)
#pragma unroll
          for (int ks = 0; ks < NB / 8; ++ks)
            mma_tf32(d, smem_desc(pa[pass] + ks * 256, 128, 2048),
                     smem_desc(pb[pass] + ks * 256, 128, 2048), (pass | ks) != 0);
        mma_commit(smem_u32(&empty[st]));   // operands read: stage free
        mma_commit(smem_u32(&tfull[st]));   // product complete: epilogue may read it
        committed = j + 1;
      }
      if (*vfail && committed > 0) {   // MMAs in flight finish before TMEM is freed
        const int j = committed - 1;
        mbar_wait(smem_u32(&tfull[j & 1]), (j >> 1) & 1);
      }
    }
  } else {
    // ---- epilogue: warps 2..5 read TMEM lane quarters 2, 3, 0, 1 -------------
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;   // row of the 128-row block
    const bool leader = threadIdx.x == 64;
    for (int j = 0; j < myjobs; ++j) {
      const int acc = j & 1;
      // one lane waits, the warp follows its verdict (tcgen05.ld is warp-wide)
      int ok = 0;
      if (lane == 0) ok = mbar_wait(smem_u32(&tfull[acc]), (j >> 1) & 1) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      float v[2][32];
      if (ok) {
        tc_fence_after();
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * kTcN), v[0]);
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * kTcN + 32), v[1]);
        tc_fence_before();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[acc]))
                     : "memory");
      } else if (lane == 0) {
        s_epi_fail = 1;
      }
      // the previous job's reduce has finished reading the staging tile
      if (leader) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (s_epi_fail) {   // the same verdict in all four warps
        if (leader) atomicExch(&s_fail, 3);
        break;
      }
      const Job jb = decode_job(args.joff, args.nblk, args.k, args.blk,
                                (int)blockIdx.x + j * (int)gridDim.x, args.jt);
      const int grow = jb.I0 * NB + r;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int col = h * 32 + c;
          stage_out[col * kTcM + r] = grow >= jb.J * NB + col ? -v[h][c] : 0.0f;
        }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (leader) {
        const CUtensorMap *tm = args.tmap + jb.b;
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
        asm volatile(
            "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, "
            "%2}], [%3];" ::"l"(tm),
            "r"(jb.I0 * NB), "r"(jb.J * NB), "r"(smem_u32(stage_out))
            : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  __syncwarp();
  if (threadIdx.x == 0 && *vfail) atomicExch(&args.status[4], 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2u * kTcN)
                 : "memory");
}

// --------------------------------------------------------------------------
// Float-float trailing update on the tensor cores.  The panel kernel leaves
// every panel tile as six planes of FP16 integer digits with one exponent per
// row, x = 2^E_r sum_s d_s 2^(-9-8s) (|d_0| <= 512, |d_s| <= 128).  Then
//     sum_k x_rk y_ck = 2^(E_r + E_c - 18) sum_q 2^(-8q) D_q,
//     D_q = sum_{s+t=q} sum_k d_s(r,k) d_t(c,k),
// and every D_q (q <= 5) is an integer below 2^24 in magnitude over the 64
// pivot columns (|D_0| <= 64 * 512^2, the others below 1.5 * 2^23), so the
// tensor core's FP32 accumulation of FP16 products computes each one exactly.
// The 21 digit products with s + t <= 5 run as kind::f16 MMAs (M = 128,
// N = 64, K = 16) into six TMEM accumulators; the epilogue sums
// 2^(-8q) D_q as a float-float pair (oz_combine), scales it by the row and
// column exponents and subtracts it from C's hi/lo pair.  The
// truncated digits and the dropped products (s + t >= 6) sit near 2^-47 of
// sum_k |x_rk| |y_ck|, the accuracy of the double-float FP32-pipe kernel.
// --------------------------------------------------------------------------
constexpr int kOzQ = 6;                                   // digits per entry
constexpr uint32_t kOzPlaneA = 2 * NB * NB * 2;           // 128 rows x 64 k FP16
constexpr uint32_t kOzPlaneB = NB * NB * 2;               // 64 rows x 64 k FP16
constexpr uint32_t kOzCTile = kTcM * kTcN * 4;           // one word of the 128 x 64 C tile
constexpr uint32_t kOzSmem = kOzQ * kOzPlaneA + kOzQ * kOzPlaneB + 2 * kOzCTile + 1024;
constexpr uint32_t kOzCols = 512;                         // TMEM: 6 accumulators of 64 columns

// kind::f16 instruction descriptor: FP32 accumulator, FP16 A and B, both
// K-major, M = 128, N = 64
constexpr uint32_t kIdescF16 = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) |
                               ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescF16), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void two_sum(float &a, float &b) {   // (a, b) <- fl(a+b), error
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  a = s;
  b = err;
}

// sum_q 2^(-8q) D_q (q = 0..5) as a float-float pair (h, l): each term is
// exact (a power-of-two scaling of an integer below 2^24), added to the high
// word by an error-free two-sum whose error goes to the low word.
__device__ __forceinline__ void oz_combine(const float (&D)[kOzQ], float &h, float &l) {
  h = D[0];
  l = 0.0f;
  const float pw[kOzQ] = {1.0f, 0x1p-8f, 0x1p-16f, 0x1p-24f, 0x1p-32f, 0x1p-40f};
#pragma unroll
  for (int q = 1; q < kOzQ; ++q) {
    float t = __fmul_rn(D[q], pw[q]);   // exact: an integer times a power of two
    two_sum(h, t);
    l = __fadd_rn(l, t);
  }
  two_sum(h, l);
}

struct OzArgs {
  const __half *dstage;    // digit planes: per slot 6 x 4096 halves
  const int *dexp;         // per slot 64 row exponents
  const int *joff;
  const BlkInfo *blk;
  const CUtensorMap *tmap; // [2 nblk]: each block's hi matrix, then its lo matrix
  int nblk, k;
  int *status;
  float *hi, *lo;          // the augmented matrices' words (persistent kernel)
  const int4 *jt;          // this step's tile-sparse job table, or nullptr
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(dst),
      "l"(tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *tm, int x, int y, uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tm),
      "r"(x), "r"(y), "r"(src)
      : "memory");
}

__global__ void __launch_bounds__(kTcThreads) pchol_update_oz_kernel(const OzArgs args) {
  extern __shared__ __align__(1024) unsigned char oz_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ int eA[kTcM], eB[kTcN];
  unsigned char *base = oz_raw + ((1024 - (smem_u32(oz_raw) & 1023)) & 1023);
  const uint32_t sA = smem_u32(base), sB = sA + kOzQ * kOzPlaneA;
  // the C tile (hi, then lo), [64 columns][128 rows], the tensor maps' box order
  float *c_hi = reinterpret_cast<float *>(base + kOzQ * kOzPlaneA + kOzQ * kOzPlaneB);
  float *c_lo = c_hi + kTcM * kTcN;

  const Job jb = decode_job(args.joff, args.nblk, args.k, args.blk, blockIdx.x, args.jt);
  const int b = jb.b, I0 = jb.I0, J = jb.J;
  const bool has_i1 = jb.has_i1;
  const BlkInfo bi = args.blk[b];
  const long long slot0 = bi.soff + I0, slotJ = bi.soff + J;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar_ld = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);

  {
    const int r = threadIdx.x;   // 128 threads: the A rows, then the B columns
    eA[r] = (r < NB || has_i1) ? args.dexp[slot0 * NB + r] : 0;
    if (r < kTcN) eB[r] = args.dexp[slotJ * NB + r];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kOzCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(bar_ld, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (threadIdx.x == 0) {
    const __half *st0 = args.dstage + slot0 * (kOzQ * NB * NB);
    const __half *stJ = args.dstage + slotJ * (kOzQ * NB * NB);
    const uint32_t plane = NB * NB * 2;   // bytes of one 64-row plane
    const CUtensorMap *tmh = args.tmap + b, *tml = args.tmap + args.nblk + b;
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmh) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tml) : "memory");
    // the whole box counts, rows past the matrix included (zero-filled)
    mbar_expect_tx(bar_ld, (has_i1 ? 3u : 2u) * kOzQ * plane + 2 * kOzCTile);
    tma_load_2d(smem_u32(c_hi), tmh, I0 * NB, J * NB, bar_ld);
    tma_load_2d(smem_u32(c_lo), tml, I0 * NB, J * NB, bar_ld);
    // A plane q: K half h holds rows 0..63 (tile I0) then rows 64..127 (tile
    // I0 + 1), 4 KB each; a B plane is the staged plane as it is
#pragma unroll
    for (int q = 0; q < kOzQ; ++q) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        bulk_g2s(sA + q * kOzPlaneA + h * plane, st0 + q * NB * NB + h * (NB * NB / 2),
                 plane / 2, bar_ld);
        if (has_i1)
          bulk_g2s(sA + q * kOzPlaneA + h * plane + plane / 2,
                   st0 + (kOzQ + q) * NB * NB + h * (NB * NB / 2), plane / 2, bar_ld);
      }
      bulk_g2s(sB + q * kOzPlaneB, stJ + q * NB * NB, plane, bar_ld);
    }
    bool ok = mbar_wait(bar_ld, 0);
    if (ok) {
      tc_fence_after();
#pragma unroll
      for (int q = 0; q < kOzQ; ++q)
#pragma unroll
        for (int sd = 0; sd <= q; ++sd)
#pragma unroll
          for (int ks = 0; ks < NB / 16; ++ks) {
            // K step ks: K half ks / 2, two 16-byte core-matrix columns into it
            // (an A half is 128 rows = 8 KB, a B half 64 rows = 4 KB)
            const uint32_t kin = (ks & 1) * 256;
            const uint64_t da = smem_desc(sA + sd * kOzPlaneA + (ks >> 1) * plane + kin, 128, 512);
            const uint64_t db =
                smem_desc(sB + (q - sd) * kOzPlaneB + (ks >> 1) * (plane / 2) + kin, 128, 512);
            mma_f16(tmem + q * kTcN, da, db, (sd | ks) != 0);
          }
      mma_commit(bar_mma);
      ok = mbar_wait(bar_mma, 0);
      if (!ok) s_fail = 2;
    } else {
      s_fail = 1;
    }
  }
  __syncthreads();
  tc_fence_after();
  const int fail = s_fail;
  if (fail) {
    if (threadIdx.x == 0) {
      atomicExch(&args.status[4], 1);
      if (fail == 1) mbar_wait(bar_ld, 0);
      else mbar_wait(bar_mma, 0);
    }
    __syncthreads();
  } else {
    const int r = warp * 32 + lane;
    const int grow = I0 * NB + r;
    const int er = eA[r];
#pragma unroll 1
    for (int ch = 0; ch < kTcN / 16; ++ch) {
      float D[kOzQ][16];
#pragma unroll
      for (int q = 0; q < kOzQ; ++q)
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * kTcN + ch * 16), D[q]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = ch * 16 + j, gcol = J * NB + c;
        // entries above the diagonal keep their value (the tile goes back
        // whole); rows and columns past the matrix are clipped by the store
        if (gcol > grow) continue;
        float Dq[kOzQ], sh, sl;
#pragma unroll
        for (int q = 0; q < kOzQ; ++q) Dq[q] = D[q][j];
        oz_combine(Dq, sh, sl);
        const int sc = er + eB[c] - 18;
        sh = ldexpf(sh, sc);
        sl = ldexpf(sl, sc);
        // (ch + cl) - (sh + sl): two-sum of the high parts, low parts added
        const int e = c * kTcM + r;
        const float chv = c_hi[e], clv = c_lo[e];
        const float tt = __fsub_rn(chv, sh);
        const float bv = __fsub_rn(tt, chv);
        const float err = __fadd_rn(__fsub_rn(chv, __fsub_rn(tt, bv)), __fsub_rn(-sh, bv));
        const float el = __fadd_rn(err, __fsub_rn(clv, sl));
        const float h = __fadd_rn(tt, el);
        c_hi[e] = h;
        c_lo[e] = __fsub_rn(el, __fsub_rn(h, tt));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_store_2d(args.tmap + b, I0 * NB, J * NB, smem_u32(c_hi));
      tma_store_2d(args.tmap + args.nblk + b, I0 * NB, J * NB, smem_u32(c_lo));
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kOzCols)
                 : "memory");
}

// --------------------------------------------------------------------------
// The float-float digit update as a persistent, warp-specialised pipeline:
// one CTA per SM walks the step's jobs (job blockIdx.x, + gridDim.x, ...).
// A job's operands come in two units, one per K half (all six A and B digit
// planes over 32 pivot columns, 72 KB), through a ring of three shared-memory
// stages, so the producer runs one and a half jobs ahead --
//   warp 0  producer: bulk copies of unit u into stage u % 3 once the MMAs of
//           unit u - 3 have released it, and an L2 prefetch of each job's C
//           tile (hi and lo) when its first unit goes out;
//   warp 1  MMA issuer: the 2 x 42 MMAs of job j into the six TMEM
//           accumulators, once both units have landed and the epilogue has
//           read job j - 1 out of tensor memory;
//   warps 2-9  epilogue: two warps per TMEM lane quarter, each owning a
//           32-row x 32-column quarter of the output tile.  A warp requests
//           its quarter of C (hi, lo) by cp.async into its own shared memory
//           before the job's products are ready, then, four columns at a
//           time, reads the six accumulators, turns them into a float-float
//           value and writes C - P back with plain stores; tensor memory is
//           released to the next job's MMAs after the last four columns.
// Warps of the epilogue never wait for each other.  The D_q are exact
// integers whatever the order of their products, so the factor equals the
// one-CTA-per-job kernel's bit for bit.  Every wait is bounded as above.
// --------------------------------------------------------------------------
constexpr int kOz2Threads = 320;
constexpr int kOz2Stages = 2;
constexpr uint32_t kOz2HalfA = kTcM * (NB / 2) * 2;             // one K half of an A plane: 8 KB
constexpr uint32_t kOz2HalfB = kTcN * (NB / 2) * 2;             // 4 KB
constexpr uint32_t kOz2Stage = kOzQ * (kOz2HalfA + kOz2HalfB);  // 72 KB
constexpr uint32_t kOz2Smem = kOz2Stages * kOz2Stage + 8 * 8192 + 1024;   // + C quarters

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void cp_async16_oz(float *dst, const float *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}

__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *tm, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(tm),
               "r"(x), "r"(y)
               : "memory");
}

__global__ void __launch_bounds__(kOz2Threads, 1) pchol_update_oz2_kernel(const OzArgs args,
                                                                         int njobs) {
  extern __shared__ __align__(1024) unsigned char oz2_raw[];
  __shared__ __align__(8) uint64_t full[kOz2Stages], empty[kOz2Stages], tfull, tempty;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  unsigned char *base = oz2_raw + ((1024 - (smem_u32(oz2_raw) & 1023)) & 1023);
  volatile int *vfail = &s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int myjobs = (int)blockIdx.x < njobs ? (njobs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                                             : 0;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kOzCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < kOz2Stages; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), 1);
    }
    mbar_init(smem_u32(&tfull), 1);
    mbar_init(smem_u32(&tempty), 8 * 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- producer: unit u = (job u / 2, K half u % 2) into stage u % 3 ----------
    if (lane == 0) {
      int issued = 0;   // units
      Job jb{};
      for (int u = 0; u < 2 * myjobs && !*vfail; ++u) {
        const int j = u >> 1, h = u & 1, st = u % kOz2Stages, use = u / kOz2Stages;
        if (!mbar_wait(smem_u32(&empty[st]), (use & 1) ^ 1)) {
          atomicExch(&s_fail, 1);
          break;
        }
        if (h == 0) {   // next job: its C tile towards L2 ahead of the epilogue's loads
          jb = decode_job(args.joff, args.nblk, args.k, args.blk,
                                (int)blockIdx.x + j * (int)gridDim.x, args.jt);
          const CUtensorMap *th = args.tmap + jb.b, *tl = args.tmap + args.nblk + jb.b;
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(th) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tl) : "memory");
          tma_prefetch_2d(th, jb.I0 * NB, jb.J * NB);
          tma_prefetch_2d(tl, jb.I0 * NB, jb.J * NB);
        }
        const BlkInfo bi = args.blk[jb.b];
        const __half *st0 = args.dstage + (bi.soff + jb.I0) * (kOzQ * NB * NB) + h * (NB * NB / 2);
        const __half *stJ = args.dstage + (bi.soff + jb.J) * (kOzQ * NB * NB) + h * (NB * NB / 2);
        const uint32_t sa = smem_u32(base + st * kOz2Stage), sb = sa + kOzQ * kOz2HalfA;
        const uint32_t bar = smem_u32(&full[st]);
        const uint32_t q4 = NB * NB;   // bytes of one 64-row K half = 4 KB
        mbar_expect_tx(bar, (jb.has_i1 ? 3u : 2u) * kOzQ * q4);
#pragma unroll
        for (int q = 0; q < kOzQ; ++q) {
          bulk_g2s(sa + q * kOz2HalfA, st0 + q * NB * NB, q4, bar);                 // rows 0..63
          if (jb.has_i1)
            bulk_g2s(sa + q * kOz2HalfA + q4, st0 + (kOzQ + q) * NB * NB, q4, bar);  // 64..127
          bulk_g2s(sb + q * kOz2HalfB, stJ + q * NB * NB, q4, bar);
        }
        issued = u + 1;
      }
      if (*vfail)   // copies still in flight (the last three units) land before exit
        for (int u = issued >= kOz2Stages ? issued - kOz2Stages : 0; u < issued; ++u)
          mbar_wait(smem_u32(&full[u % kOz2Stages]), (u / kOz2Stages) & 1);
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----------------------------------------------------------------
    if (lane == 0) {
      int last = -1;   // last unit whose MMAs were committed
      for (int j = 0; j < myjobs && !*vfail; ++j) {
        if (!mbar_wait(smem_u32(&tempty), (j & 1) ^ 1)) {
          atomicExch(&s_fail, 2);
          break;
        }
        bool ok = true;
        for (int h = 0; h < 2; ++h) {
          const int u = 2 * j + h, st = u % kOz2Stages;
          if (!mbar_wait(smem_u32(&full[st]), (u / kOz2Stages) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(base + st * kOz2Stage), sb = sa + kOzQ * kOz2HalfA;
#pragma unroll
          for (int q = 0; q < kOzQ; ++q)
#pragma unroll
            for (int sd = 0; sd <= q; ++sd)
#pragma unroll
              for (int ks = 0; ks < 2; ++ks)
                mma_f16(tmem + q * kTcN, smem_desc(sa + sd * kOz2HalfA + ks * 256, 128, 512),
                        smem_desc(sb + (q - sd) * kOz2HalfB + ks * 256, 128, 512),
                        (h | sd | ks) != 0);
          mma_commit(smem_u32(&empty[st]));   // stage free once these MMAs complete
          last = u;
        }
        if (!ok) {
          atomicExch(&s_fail, 2);
          break;
        }
        mma_commit(smem_u32(&tfull));   // all 84 products of job j complete
      }
      if (*vfail && last >= 0)   // MMAs in flight finish before tensor memory is freed
        mbar_wait(smem_u32(&empty[last % kOz2Stages]), (last / kOz2Stages) & 1);
    }
  } else {
    // ---- epilogue ------------------------------------------------------------------
    const int quarter = warp & 3;                // TMEM lanes 32 quarter .. + 31
    const int cbase = ((warp - 2) >> 2) * 32;    // this warp's 32 columns of the tile
    const int r = quarter * 32 + lane;           // row of the 128-row tile
    // this warp's quarter of the C tile, [column][row] for hi then lo
    float *cs = reinterpret_cast<float *>(base + kOz2Stages * kOz2Stage + (warp - 2) * 8192);
    for (int j = 0; j < myjobs; ++j) {
      const Job jb = decode_job(args.joff, args.nblk, args.k, args.blk,
                                (int)blockIdx.x + j * (int)gridDim.x, args.jt);
      const BlkInfo bi = args.blk[jb.b];
      const long long slot0 = bi.soff + jb.I0, slotJ = bi.soff + jb.J;
      const int row0 = jb.I0 * NB + quarter * 32;   // first row of the warp's quarter
      const int grow = row0 + lane;
      const int col0 = jb.J * NB + cbase;
      // C quarter -> shared memory by cp.async before the products are ready:
      // 16-byte copies of 4 rows, 8 per column, rows past the matrix
      // zero-filled, columns past it skipped
      __syncwarp();   // every lane has finished reading the previous job's quarter
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int arr = t >> 3, c = ((t & 7) << 2) | (lane >> 3), part = lane & 7;
        const int rr = row0 + part * 4;
        const int valid = col0 + c < bi.a ? max(0, min(4, bi.a - rr)) : 0;
        const float *src = (arr ? args.lo : args.hi) + bi.base;
        const float *g = valid ? src + (long long)(col0 + c) * bi.lda + rr : src;
        cp_async16_oz(cs + arr * 1024 + c * 32 + part * 4, g, valid * 4);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      const int er = (r < NB || jb.has_i1) ? args.dexp[slot0 * NB + r] : 0;
      const int ec = args.dexp[slotJ * NB + cbase + lane];   // lane u: column cbase + u
      int ok = 0;
      if (lane == 0) ok = mbar_wait(smem_u32(&tfull), j & 1) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        atomicExch(&s_fail, 3);
        break;
      }
      tc_fence_after();
      // the six accumulators -> sum_q 2^(-8q) D_q as a float-float pair
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp();   // the other lanes' copies are visible
      // four columns at a time: accumulators -> float-float value -> C - P on
      // the lower triangle of the matrix (rows and columns past it, and
      // entries above the diagonal, keep their values); the loop stays rolled
      // so that the epilogue's code stays short
      const long long g0 = bi.base + (long long)col0 * bi.lda + grow;
#pragma unroll 1
      for (int c4 = 0; c4 < 8; ++c4) {
        float D[kOzQ][4];
#pragma unroll
        for (int q = 0; q < kOzQ; ++q)
          tmem_ld4(tmem + ((uint32_t)(quarter * 32) << 16) +
                       (uint32_t)(q * kTcN + cbase + c4 * 4),
                   D[q]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int u = c4 * 4 + v;
          float Dq[kOzQ], shv, slv;
#pragma unroll
          for (int q = 0; q < kOzQ; ++q) Dq[q] = D[q][v];
          oz_combine(Dq, shv, slv);
          const int sc = er + __shfl_sync(0xffffffffu, ec, u) - 18;
          if (!(grow < bi.a && col0 + u <= grow)) continue;
          const float chv = cs[u * 32 + lane], clv = cs[1024 + u * 32 + lane];
          const float ph = ldexpf(shv, sc), pl = ldexpf(slv, sc);
          const float tt = __fsub_rn(chv, ph);
          const float bv = __fsub_rn(tt, chv);
          const float err = __fadd_rn(__fsub_rn(chv, __fsub_rn(tt, bv)), __fsub_rn(-ph, bv));
          const float el = __fadd_rn(err, __fsub_rn(clv, pl));
          const float hh = __fadd_rn(tt, el);
          args.hi[g0 + (long long)u * bi.lda] = hh;
          args.lo[g0 + (long long)u * bi.lda] = __fsub_rn(el, __fsub_rn(hh, tt));
        }
      }
      // all six accumulators read: the next job's MMAs may overwrite them
      tc_fence_before();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty))
                   : "memory");
    }
  }
  __syncwarp();
  if (threadIdx.x == 0 && *vfail) atomicExch(&args.status[4], 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kOzCols)
                 : "memory");
}

// the number of update jobs of a block with t trailing tiles: row pairs R
// cover tiles (2R, 2R+1) and the columns up to their last tile
long long tc_jobs_of(int t) {
  if (t <= 0) return 0;
  const long long nR = (t + 1) / 2;
  long long n = 0;
  for (long long R = 0; R < nR; ++R) n += std::min<long long>(2 * R + 2, t);
  return n;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tile-sparse jobs of the tensor-core trailing updates (host only).  A
// tile-level symbolic factorisation of each block's augmented matrix: tile
// (I, J) of L is nonzero if the formed matrix has entries there or if some
// pivot step k < J has nonzero tiles (I, k) and (J, k) (right-looking fill).
// The update of step k adds L_Ik L_Jk' to the tile pair's rows and column J;
// a job whose two row tiles are both zero in column k, or whose column tile J
// is, adds exact zeros and is left out.  The kept jobs stay in the dense
// enumeration's order (step, block, row pair, column), so the CTAs that run
// them and the factor are the same.  nz[b]: block b's T[b] x T[b] row-major
// tile pattern (lower triangle read), or nullptr for a dense block.  Fills
// tab and off (maxTp + 1 step offsets into tab); returns the jobs kept.
long long tile_sparse_jobs(int nblk, const int *T, const int *Tp,
                           const unsigned char *const *nz, int maxTp, std::vector<int4> &tab,
                           std::vector<long long> &off) {
  std::vector<std::vector<unsigned char>> L(nblk);
  for (int b = 0; b < nblk; ++b) {
    const int Tb = T[b];
    if (!nz[b]) {
      L[b].assign((size_t)Tb * Tb, 1);
      continue;
    }
    L[b].assign(nz[b], nz[b] + (size_t)Tb * Tb);
    bool dense = true;
    for (int I = 0; I < Tb && dense; ++I)
      for (int J = 0; J <= I; ++J)
        if (!L[b][(size_t)I * Tb + J]) {
          dense = false;
          break;
        }
    if (dense) continue;
    std::vector<int> rows;
    for (int k = 0; k < Tp[b]; ++k) {
      rows.clear();
      for (int I = k + 1; I < Tb; ++I)
        if (L[b][(size_t)I * Tb + k]) rows.push_back(I);
      for (size_t x = 0; x < rows.size(); ++x)
        for (size_t y = 0; y <= x; ++y) L[b][(size_t)rows[x] * Tb + rows[y]] = 1;
    }
  }
  tab.clear();
  off.assign((size_t)maxTp + 1, 0);
  for (int k = 0; k < maxTp; ++k) {
    off[k] = (long long)tab.size();
    for (int b = 0; b < nblk; ++b) {
      if (k >= Tp[b]) continue;
      const int Tb = T[b], t = Tb - k - 1;
      const unsigned char *Lb = L[b].data();
      for (int R = 0; 2 * R < t; ++R) {
        const int I0 = k + 1 + 2 * R;
        const bool has_i1 = 2 * R + 1 < t;
        if (!Lb[(size_t)I0 * Tb + k] && !(has_i1 && Lb[(size_t)(I0 + 1) * Tb + k])) continue;
        const int jend = k + std::min(2 * R + 2, t);
        for (int J = k + 1; J <= jend; ++J)
          if (Lb[(size_t)J * Tb + k]) tab.push_back(make_int4(b, I0, J, has_i1 ? 1 : 0));
      }
    }
  }
  off[maxTp] = (long long)tab.size();
  return (long long)tab.size();
}

// job offsets per step, over the blocks (shared by both tensor-core updates)
void jobs_setup(ahlp_problem *p) {
  if (p->tc_joff) return;
  const int N = (int)p->h_blk.size();
  const int maxTp = p->maxTp;
  std::vector<int> joff((size_t)std::max(maxTp, 1) * (N + 1), 0);
  p->tc_jobs.assign(maxTp, 0);
  for (int k = 0; k < maxTp; ++k) {
    long long acc = 0;
    for (int b = 0; b < N; ++b) {
      joff[(size_t)k * (N + 1) + b] = (int)acc;
      const BlkInfo &bi = p->h_blk[b];
      if (k < bi.Tp) acc += tc_jobs_of(bi.T - k - 1);
    }
    joff[(size_t)k * (N + 1) + N] = (int)acc;
    p->tc_jobs[k] = acc;
    p->tc_jobs_dense += acc;
  }
  p->tc_joff = static_cast<int *>(dupload_bytes(p, joff.data(), joff.size() * sizeof(int)));
  p->tc_jobs_kept = p->tc_jobs_dense;
  if (!p->opt.tile_sparse || (int)p->tile_nz.size() != N) return;
  std::vector<int> T(N), Tp(N);
  std::vector<const unsigned char *> nz(N);
  for (int b = 0; b < N; ++b) {
    T[b] = p->h_blk[b].T;
    Tp[b] = p->h_blk[b].Tp;
    // no pattern: every tile counts as nonzero
    nz[b] = p->tile_nz[b].size() == (size_t)T[b] * T[b] ? p->tile_nz[b].data() : nullptr;
  }
  std::vector<int4> tab;
  const long long kept =
      tile_sparse_jobs(N, T.data(), Tp.data(), nz.data(), maxTp, tab, p->tc_jtab_off);
  for (int k = 0; k < maxTp; ++k) p->tc_jobs[k] = p->tc_jtab_off[k + 1] - p->tc_jtab_off[k];
  p->tc_jobs_kept = kept;
  if (p->opt.verbose)
    printf("       tile-sparse trailing updates: %lld of %lld tile jobs kept\n", kept,
           p->tc_jobs_dense);
  // Nothing left out (every block tile-dense): the kernels keep decoding the
  // dense enumeration and no table is uploaded.
  if (kept < p->tc_jobs_dense && !tab.empty())
    p->tc_jtab = static_cast<int4 *>(dupload_bytes(p, tab.data(), tab.size() * sizeof(int4)));
}

}  // namespace

// Staging slots, per-step job offsets and the per-block tensor maps of the
// tensor-core update (FP32 factors).  Returns false (nothing changed) when
// the driver offers no tensor-map encoder.
bool tc_setup(ahlp_problem *p) {
  if (p->tc_ready) return true;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  auto encode = reinterpret_cast<EncodeTiledFn>(fn);
  const int N = (int)p->h_blk.size();
  std::vector<CUtensorMap> maps(std::max(N, 1));
  for (int b = 0; b < N; ++b) {
    const BlkInfo &bi = p->h_blk[b];
    const cuuint64_t dims[2] = {(cuuint64_t)bi.a, (cuuint64_t)bi.a};
    const cuuint64_t strides[1] = {(cuuint64_t)bi.lda * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kTcM, (cuuint32_t)kTcN};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&maps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->aug32 + bi.base, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  jobs_setup(p);
  p->tc_tmap = dupload_bytes(p, maps.data(), sizeof(CUtensorMap) * maps.size());
  p->pstage = static_cast<float *>(
      dalloc_bytes(p, (size_t)std::max(p->stage_slots, 1LL) * 8192 * sizeof(float)));
  ck(cudaFuncSetAttribute(pchol_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)kSmemBytes),
     "tensor-core update shared memory");
  ck(cudaFuncSetAttribute(pchol_update_tc2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)kTc2Smem),
     "tensor-core update shared memory");
  {
    int dev = 0, sms = 0;
    ck(cudaGetDevice(&dev), "device");
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    p->num_sms = std::max(sms, 1);
  }
  p->tc_ready = true;
  return true;
}

cudaError_t launch_update_tc(ahlp_problem *p, int k, cudaStream_t s) {
  const long long jobs = p->tc_jobs[k];
  if (jobs <= 0) return cudaSuccess;
  TcArgs a{p->pstage, p->tc_joff + (size_t)k * (p->h_blk.size() + 1), p->blk,
           reinterpret_cast<const CUtensorMap *>(p->tc_tmap), (int)p->h_blk.size(), k,
           p->status, p->tc_jtab ? p->tc_jtab + p->tc_jtab_off[k] : nullptr};
  if (p->fp32_update == 3) {   // persistent pipeline: one CTA per SM
    const int grid = (int)std::min<long long>(jobs, p->num_sms);
    count_launch(), pchol_update_tc2_kernel<<<grid, kTc2Threads, kTc2Smem, s>>>(a, (int)jobs);
  } else {
    count_launch(), pchol_update_tc_kernel<<<(unsigned)jobs, kTcThreads, kSmemBytes, s>>>(a);
  }
  return cudaGetLastError();
}

// FP16 digit staging and job offsets of the float-float tensor-core update
bool oz_setup(ahlp_problem *p) {
  if (p->oz_ready) return true;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  auto encode = reinterpret_cast<EncodeTiledFn>(fn);
  const int N = (int)p->h_blk.size();
  std::vector<CUtensorMap> maps(std::max(2 * N, 1));
  for (int w = 0; w < 2; ++w)
    for (int b = 0; b < N; ++b) {
      const BlkInfo &bi = p->h_blk[b];
      const cuuint64_t dims[2] = {(cuuint64_t)bi.a, (cuuint64_t)bi.a};
      const cuuint64_t strides[1] = {(cuuint64_t)bi.lda * sizeof(float)};
      const cuuint32_t box[2] = {(cuuint32_t)kTcM, (cuuint32_t)kTcN};
      const cuuint32_t estr[2] = {1, 1};
      CUresult r = encode(&maps[(size_t)w * N + b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                          (w == 0 ? p->aug32 : p->aug_lo) + bi.base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
  jobs_setup(p);
  p->oz_tmap = dupload_bytes(p, maps.data(), sizeof(CUtensorMap) * maps.size());
  p->dstage = static_cast<__half *>(
      dalloc_bytes(p, (size_t)std::max(p->stage_slots, 1LL) * kOzQ * NB * NB * sizeof(__half)));
  p->dexp = static_cast<int *>(
      dalloc_bytes(p, (size_t)std::max(p->stage_slots, 1LL) * NB * sizeof(int)));
  ck(cudaFuncSetAttribute(pchol_update_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)kOzSmem),
     "float-float tensor-core update shared memory");
  ck(cudaFuncSetAttribute(pchol_update_oz2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)kOz2Smem),
     "float-float tensor-core update shared memory");
  {
    int dev = 0, sms = 0;
    ck(cudaGetDevice(&dev), "device");
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    p->num_sms = std::max(sms, 1);
  }
  p->oz_ready = true;
  return true;
}

cudaError_t launch_update_oz(ahlp_problem *p, int k, cudaStream_t s) {
  const long long jobs = p->tc_jobs[k];
  if (jobs <= 0) return cudaSuccess;
  OzArgs a{p->dstage, p->dexp, p->tc_joff + (size_t)k * (p->h_blk.size() + 1), p->blk,
           reinterpret_cast<const CUtensorMap *>(p->oz_tmap), (int)p->h_blk.size(), k,
           p->status, p->aug32, p->aug_lo,
           p->tc_jtab ? p->tc_jtab + p->tc_jtab_off[k] : nullptr};
  if (p->ff_update == 3) {   // persistent pipeline: one CTA per SM
    const int grid = (int)std::min<long long>(jobs, p->num_sms);
    count_launch(), pchol_update_oz2_kernel<<<grid, kOz2Threads, kOz2Smem, s>>>(a, (int)jobs);
  } else {
    count_launch(), pchol_update_oz_kernel<<<(unsigned)jobs, kTcThreads, kOzSmem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace ahlp

extern "C" int ahlp_tile_sparse_jobs(int32_t nblk, const int32_t *T, const int32_t *Tp,
                                     const uint8_t *nz, int32_t *jobs, int64_t *step_off,
                                     int64_t cap, int64_t *njobs, int64_t *ndense) {
  using namespace ahlp;
  if (nblk < 0 || (nblk > 0 && (!T || !Tp)) || !njobs) return AHLP_ERR_INVALID_ARG;
  int maxTp = 0;
  long long dense = 0;
  std::vector<const unsigned char *> pat(nblk, nullptr);
  size_t at = 0;
  for (int b = 0; b < nblk; ++b) {
    if (T[b] < 1 || T[b] > 32768 || Tp[b] < 0 || Tp[b] > T[b]) return AHLP_ERR_INVALID_ARG;
    maxTp = std::max(maxTp, (int)Tp[b]);
    for (int k = 0; k < Tp[b]; ++k) dense += tc_jobs_of(T[b] - k - 1);
    if (nz) pat[b] = nz + at;
    at += (size_t)T[b] * T[b];
  }
  std::vector<int> Ti(T, T + nblk), Tpi(Tp, Tp + nblk);
  std::vector<int4> tab;
  std::vector<long long> off;
  long long kept = 0;
  try {
    kept = tile_sparse_jobs(nblk, Ti.data(), Tpi.data(), pat.data(), maxTp, tab, off);
  } catch (const std::bad_alloc &) {
    return AHLP_ERR_OOM;
  }
  *njobs = kept;
  if (ndense) *ndense = dense;
  if (step_off)
    for (int k = 0; k <= maxTp; ++k) step_off[k] = off[k];
  if (jobs) {
    if (cap < kept) return AHLP_ERR_INVALID_ARG;
    for (long long j = 0; j < kept; ++j) {
      jobs[4 * j + 0] = tab[j].x;
      jobs[4 * j + 1] = tab[j].y;
      jobs[4 * j + 2] = tab[j].z;
      jobs[4 * j + 3] = tab[j].w;
    }
  }
  return AHLP_OK;
}
