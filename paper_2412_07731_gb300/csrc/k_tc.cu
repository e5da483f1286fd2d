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

// TF32 rounding (round to nearest, ties away) as a 32-bit pattern
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
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

__device__ __forceinline__ Job decode_job(const int *joff, int nblk, int k, const BlkInfo *blk) {
  const int q = blockIdx.x;
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
  const Job jb = decode_job(args.joff, args.nblk, args.k, args.blk);
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
// 2^(-8q) D_q as a float-float pair (each term exact, two-sum), scales it by
// the row and column exponents and subtracts it from C's hi/lo pair.  The
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

struct OzArgs {
  const __half *dstage;    // digit planes: per slot 6 x 4096 halves
  const int *dexp;         // per slot 64 row exponents
  const int *joff;
  const BlkInfo *blk;
  const CUtensorMap *tmap; // [2 nblk]: each block's hi matrix, then its lo matrix
  int nblk, k;
  int *status;
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

  const Job jb = decode_job(args.joff, args.nblk, args.k, args.blk);
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
#pragma unroll
    for (int q = 0; q < kOzQ; ++q) {
      bulk_g2s(sA + q * kOzPlaneA, st0 + q * NB * NB, plane, bar_ld);
      if (has_i1) bulk_g2s(sA + q * kOzPlaneA + plane, st0 + (kOzQ + q) * NB * NB, plane, bar_ld);
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
            // K step ks: two 16-byte core-matrix columns, 2 x 128 bytes further
            const uint64_t da = smem_desc(sA + sd * kOzPlaneA + ks * 256, 128, 1024);
            const uint64_t db = smem_desc(sB + (q - sd) * kOzPlaneB + ks * 256, 128, 1024);
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
        float sh = D[0][j], sl = 0.0f;
#pragma unroll
        for (int q = 1; q < kOzQ; ++q) {
          float t = ldexpf(D[q][j], -8 * q);   // exact
          two_sum(sh, t);
          sl = __fadd_rn(sl, t);
        }
        two_sum(sh, sl);
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
  }
  p->tc_joff = static_cast<int *>(dupload_bytes(p, joff.data(), joff.size() * sizeof(int)));
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
  p->tc_ready = true;
  return true;
}

cudaError_t launch_update_tc(ahlp_problem *p, int k, cudaStream_t s) {
  const long long jobs = p->tc_jobs[k];
  if (jobs <= 0) return cudaSuccess;
  TcArgs a{p->pstage, p->tc_joff + (size_t)k * (p->h_blk.size() + 1), p->blk,
           reinterpret_cast<const CUtensorMap *>(p->tc_tmap), (int)p->h_blk.size(), k,
           p->status};
  count_launch(), pchol_update_tc_kernel<<<(unsigned)jobs, kTcThreads, kSmemBytes, s>>>(a);
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
  p->oz_ready = true;
  return true;
}

cudaError_t launch_update_oz(ahlp_problem *p, int k, cudaStream_t s) {
  const long long jobs = p->tc_jobs[k];
  if (jobs <= 0) return cudaSuccess;
  OzArgs a{p->dstage, p->dexp, p->tc_joff + (size_t)k * (p->h_blk.size() + 1), p->blk,
           reinterpret_cast<const CUtensorMap *>(p->oz_tmap), (int)p->h_blk.size(), k,
           p->status};
  count_launch(), pchol_update_oz_kernel<<<(unsigned)jobs, kTcThreads, kOzSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ahlp
