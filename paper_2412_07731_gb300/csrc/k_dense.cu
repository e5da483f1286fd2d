// Dense per-block kernels: formation of the augmented matrices, the batched
// tiled partial Cholesky, and the forward / backward solves with its factor.
//
// Every block i owns an augmented lower-triangular matrix
//     [ M_i   .  ]        M_i = A_i D_i A_i' + delta I      (m_i x m_i)
//     [ G_i'  C_i]        G_i = [W_i | A_i D_i U_i' | A_i D_i Fg_i']
// stored column-major.  Eliminating its first m_i pivots (the block factor and
// Schur-contribution steps of Alg. 2 in normal-equation form) leaves L_i on
// top, Y_i' = (L_i^-1 G_i)' below it and C_i - G_i' M_i^-1 G_i in the corner
// -- the block's Schur contribution.
//
// The factor is stored in FP64, FP32 or float-float (two FP32 words); in the
// mixed modes it only preconditions an FP64 Krylov solve.  Kernels shared by
// FP64 and FP32 are templated on the storage type; the FP32 and float-float
// trailing updates and the FP32 diagonal tile have their own kernels.
// Entries are always formed in FP64 and rounded once.
#include <cuda_fp16.h>
#include <math.h>

#include "ahlp_internal.h"

namespace ahlp {

namespace {

// --------------------------------------------------------------------------
// formation: one CTA per 64x64 lower tile, written exactly once
// --------------------------------------------------------------------------
template <typename T>
struct FormArgs {
  float *lo;   // float-float: receives v - (double)(float)v (nullptr otherwise)
  const FormTile *tiles;
  const long long *tile_ent;
  const int *ent_pos;
  const long long *ent_cb;
  const int *con_idx;
  const double *con_coef;
  const double *d;
  const BlkInfo *blk;
  T *aug;
  double *diag0;
  double *cdiag0;
  double delta;
};

template <typename T, bool kLo>
__global__ void __launch_bounds__(kThreads) form_aug_kernel(FormArgs<T> A) {
  __shared__ T t[NB * NB];   // column-major tile
  __shared__ float tl[kLo ? NB * NB : 1];
  const FormTile ft = A.tiles[blockIdx.x];
  const BlkInfo bi = A.blk[ft.blk];
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    t[i] = T(0);
    if constexpr (kLo) tl[i] = 0.0f;
  }
  __syncthreads();
  const long long e0 = A.tile_ent[blockIdx.x], e1 = A.tile_ent[blockIdx.x + 1];
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int pos = A.ent_pos[e];
    const long long q0 = A.ent_cb[e], q1 = A.ent_cb[e + 1];
    double v = 0.0;
    for (long long q = q0; q < q1; ++q) {
      const int di = A.con_idx[q];
      const double cf = A.con_coef[q];
      v += (di >= 0) ? cf * A.d[di] : cf;
    }
    const int rt = (pos >> 8) & 0xff, ct = pos & 0xff;
    if (pos & (1 << 16)) {   // diagonal of M_i: regularise, remember for pivot test
      v += A.delta;
      A.diag0[bi.d0off + (long long)ft.I * NB + rt] = v;
    } else if (pos & (1 << 17)) {   // corner diagonal: reference for link / y_g pivots
      A.cdiag0[bi.cdoff + (long long)ft.I * NB + rt - bi.p] = v;
    }
    t[ct * NB + rt] = T(v);
    if constexpr (kLo) tl[ct * NB + rt] = (float)(v - (double)(float)v);
  }
  __syncthreads();
  const int r0 = ft.I * NB, c0 = ft.J * NB;
  const int nr = min(NB, bi.a - r0), nc = min(NB, bi.a - c0);
  const long long g0 = bi.base + (long long)c0 * bi.lda + r0;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    if (r < nr && c < nc) {
      A.aug[g0 + (long long)c * bi.lda + r] = t[i];
      if constexpr (kLo) A.lo[g0 + (long long)c * bi.lda + r] = tl[i];
    }
  }
}

// d = x / z; on the block variables x / (z + rho_x x) with the factor's primal
// regularisation, i.e. D^-1 + rho_x (caps d at 1 / rho_x).  The linking
// variables get theirs in the Schur border (-D_0^-1 - rho).  With them, the
// two per-variable quotients every solve at this point needs (FP64 division
// is a long instruction sequence on this part): xinv = 1 / x and
// w = 1 / (1 / d + rho on the linking variables).
__global__ void dscale_kernel(const double *x, const double *z, double *d, double *xinv,
                              double *w, long long n, double rho_x, double rho,
                              const unsigned char *is_x0) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = (rho_x > 0.0 && !is_x0[i]) ? x[i] / (z[i] + rho_x * x[i]) : x[i] / z[i];
  d[i] = di;
  xinv[i] = 1.0 / x[i];
  w[i] = 1.0 / (1.0 / di + (is_x0[i] ? rho : 0.0));
}

// --------------------------------------------------------------------------
// partial Cholesky, step k: diagonal tile
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) pchol_potrf_kernel(T *buf, const BlkInfo *blk, int k,
                                                               const double *diag0, double tol,
                                                               int *status, double drop) {
  const BlkInfo bi = blk[blockIdx.x];
  if (k >= bi.Tp) return;
  __shared__ T t[NB][NB + 1];
  __shared__ T s_inv;
  const int r0 = k * NB;
  const int nr = min(NB, bi.a - r0);
  const int npiv = min(NB, bi.p - r0);
  T *g = buf + bi.base + (long long)r0 * bi.lda + r0;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    t[r][c] = (r < nr && c < nr && r >= c) ? g[(long long)c * bi.lda + r] : T(0);
  }
  __syncthreads();
  for (int c = 0; c < npiv; ++c) {
    if (threadIdx.x == 0) {
      double piv = (double)t[c][c];
      pivot_fix(piv, diag0[bi.d0off + r0 + c], tol, status, bi.tag + (int)blockIdx.x, r0 + c,
                drop, sizeof(T) == 4 ? kDropCapFP32 : 1e300);
      const T l = (T)sqrt(piv);
      t[c][c] = l;
      s_inv = T(1) / l;
    }
    __syncthreads();
    const T inv = s_inv;
    for (int r = c + 1 + threadIdx.x; r < nr; r += blockDim.x) t[r][c] *= inv;
    __syncthreads();
    const int m = nr - c - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int rr = idx % m, ss = idx / m;
      if (rr >= ss) t[c + 1 + rr][c + 1 + ss] -= t[c + 1 + rr][c] * t[c + 1 + ss][c];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    if (r < nr && c < nr && r >= c) g[(long long)c * bi.lda + r] = t[r][c];
  }
}

// panel tiles below the diagonal tile: X = A_Ik L_kk^-T on the pivot columns,
// and the non-pivot (Schur) columns of the tile updated with the new X.
template <typename T>
__global__ void __launch_bounds__(kThreads) pchol_trsm_kernel(T *buf, const BlkInfo *blk, int k) {
  const BlkInfo bi = blk[blockIdx.y];
  if (k >= bi.Tp) return;
  const int I = k + 1 + blockIdx.x;
  if (I >= bi.T) return;
  extern __shared__ __align__(16) unsigned char trsm_raw[];   // two (NB x NB+1) tiles
  T(*L)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(trsm_raw);
  T(*X)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(trsm_raw + sizeof(T) * NB * (NB + 1));
  const int r0 = k * NB;
  const int nr = min(NB, bi.a - r0);
  const int npiv = min(NB, bi.p - r0);
  const int ri = I * NB;
  const int nri = min(NB, bi.a - ri);
  const T *gl = buf + bi.base + (long long)r0 * bi.lda + r0;
  T *gx = buf + bi.base + (long long)r0 * bi.lda + ri;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    L[r][c] = (r < nr && c < nr && r >= c) ? gl[(long long)c * bi.lda + r] : T(0);
    X[r][c] = (r < nri && c < nr) ? gx[(long long)c * bi.lda + r] : T(0);
  }
  __syncthreads();
  for (int c = 0; c < npiv; ++c) {
    const T inv = T(1) / L[c][c];
    for (int r = threadIdx.x; r < nri; r += blockDim.x) X[r][c] *= inv;
    __syncthreads();
    const int ns = nr - c - 1;
    for (int idx = threadIdx.x; idx < nri * ns; idx += blockDim.x) {
      const int r = idx % nri, s = c + 1 + idx / nri;
      X[r][s] -= X[r][c] * L[s][c];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    if (r < nri && c < nr) gx[(long long)c * bi.lda + r] = X[r][c];
  }
}

// --------------------------------------------------------------------------
// FP32 factors: diagonal tile, then the inverse of its pivot triangle,
// written in the layout the block solves use (inverse on the pivot rows, the
// factor on the non-pivot rows of a block's last pivot tile).  The panel
// below then is a product with that inverse instead of a column-by-column
// substitution.
//
// The 64x64 tile sits in shared memory and is factored in four 16-column
// panels.  Warp 0 factors a panel in registers: lane l holds rows l and
// l + 32 of the panel's 16 columns, the pivot and the scaled column entries
// are broadcast with shuffles, so the sequential path has no shared-memory
// round trip.  All 256 threads then apply the panel to the columns right of
// it (a rank-16 update).  The code of a panel step is small and runs four
// times; a fully unrolled 64-column version was bound by instruction fetch.
// The inverse goes by 16x16 blocks: the diagonal blocks by substitution in
// parallel, then each block row below as two small products with the rows
// above it, so its sequential depth is 16 rows rather than 64.
// --------------------------------------------------------------------------
constexpr int kPotrf32Threads = 256;
constexpr int kPW = 16;   // panel width

__global__ void __launch_bounds__(kPotrf32Threads) pchol_potrf_f32_kernel(
    float *buf, float *tinv, const BlkInfo *blk, int k, const double *diag0, float tol,
    int *status, float drop) {
  const BlkInfo bi = blk[blockIdx.x];
  if (k >= bi.Tp) return;
  __shared__ float t[NB][NB + 1];
  __shared__ float X[NB][NB + 1];
  __shared__ float Tm[kPW][NB];
  const int r0 = k * NB;
  const int nr = min(NB, bi.a - r0);
  const int npiv = min(NB, bi.p - r0);
  float *g = buf + bi.base + (long long)r0 * bi.lda + r0;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    t[r][c] = (r < nr && c < nr && r >= c) ? g[(long long)c * bi.lda + r] : 0.0f;
    X[r][c] = 0.0f;
  }
  __syncthreads();
  const double *d0 = diag0 + bi.d0off + r0;
  for (int c0 = 0; c0 < npiv; c0 += kPW) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      float ra[kPW], rb[kPW];   // rows lane and lane + 32, columns c0 .. c0 + 15
#pragma unroll
      for (int u = 0; u < kPW; ++u) {
        ra[u] = t[lane][c0 + u];
        rb[u] = t[lane + 32][c0 + u];
      }
      const float dref_a = lane < npiv ? (float)d0[lane] : 0.0f;
      const float dref_b = lane + 32 < npiv ? (float)d0[lane + 32] : 0.0f;
#pragma unroll
      for (int u = 0; u < kPW; ++u) {
        const int c = c0 + u;
        if (c < npiv) {   // uniform over the warp
          // values, not array elements, are selected (a select of two
          // array elements would force the arrays into local memory)
          const float va = ra[u], vb = rb[u];
          const bool hi = c >= 32;
          float piv = __shfl_sync(0xffffffffu, hi ? vb : va, c & 31);
          const float dref = __shfl_sync(0xffffffffu, hi ? dref_b : dref_a, c & 31);
          const float lim = tol * dref;
          // the same safeguard as pivot_fix, in FP32
          const float repl = drop > 0.0f ? fminf(drop * fmaxf(dref, 1.0f), (float)kDropCapFP32)
                             : lim > 0.0f ? lim
                                          : 1.0f;
          if (!(piv == piv)) {
            if (lane == 0 && atomicAdd(&status[0], 1) == 0) {
              status[2] = bi.tag + (int)blockIdx.x;
              status[3] = r0 + c;
            }
            piv = repl;
          } else if (!(piv > lim) || !(piv > 0.0f)) {
            if (lane == 0) atomicAdd(&status[1], 1);
            piv = repl;
          }
          const float lcc = sqrtf(piv), inv = 1.0f / lcc;
          const float la = lane == c ? lcc : va * inv;
          const float lb = lane + 32 == c ? lcc : vb * inv;
          ra[u] = la;
          rb[u] = lb;
#pragma unroll
          for (int w = u + 1; w < kPW; ++w) {
            const int q = c0 + w;
            const float lq = __shfl_sync(0xffffffffu, q >= 32 ? lb : la, q & 31);
            ra[w] = fmaf(-la, lq, ra[w]);
            rb[w] = fmaf(-lb, lq, rb[w]);
          }
        }
      }
      // write the panel back (entries above the diagonal stay zero)
#pragma unroll
      for (int u = 0; u < kPW; ++u) {
        const int c = c0 + u;
        if (lane >= c) t[lane][c] = ra[u];
        if (lane + 32 >= c) t[lane + 32][c] = rb[u];
      }
    }
    __syncthreads();
    // rank-16 update of the lower triangle right of the panel:
    // t[r][q] -= sum_c t[r][c] t[q][c], c0 + 16 <= q <= r < nr, c < npiv
    const int q0 = c0 + kPW;
    const int cend = min(c0 + kPW, npiv);
    if (q0 < nr) {
      const int w = nr - q0;
      for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        const int rr = idx % w, qq = idx / w;
        if (rr < qq) continue;
        const int r = q0 + rr, q = q0 + qq;
        float s0 = 0.0f, s1 = 0.0f;
        int c = c0;
        for (; c + 1 < cend; c += 2) {
          s0 = fmaf(t[r][c], t[q][c], s0);
          s1 = fmaf(t[r][c + 1], t[q][c + 1], s1);
        }
        if (c < cend) s0 = fmaf(t[r][c], t[q][c], s0);
        t[r][q] -= s0 + s1;
      }
    }
    __syncthreads();
  }
  // inverse of the pivot triangle by 16x16 blocks: warp w inverts diagonal
  // block w by substitution (lane = column); then block rows 1..3 in turn,
  // X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj, all threads on the entries.
  // Rows at or past npiv are zero.
  const int nbk = (npiv + kPW - 1) / kPW;
  {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < 4 && lane < kPW) {
      const int b0 = w * kPW, j = b0 + lane;
      for (int i = b0; i < b0 + kPW; ++i) {
        float v = 0.0f;
        if (i < npiv && i >= j) {
          float s0 = i == j ? 1.0f : 0.0f, s1 = 0.0f;
          int q = j;
          for (; q + 1 < i; q += 2) {
            s0 = fmaf(-t[i][q], X[q][j], s0);
            s1 = fmaf(-t[i][q + 1], X[q + 1][j], s1);
          }
          if (q < i) s0 = fmaf(-t[i][q], X[q][j], s0);
          v = (s0 + s1) / t[i][i];
        }
        X[i][j] = v;
      }
    }
  }
  __syncthreads();
  for (int bi2 = 1; bi2 < nbk; ++bi2) {
    const int i0 = bi2 * kPW, wc = i0;   // columns 0 .. i0-1 of block row bi2
    for (int e = threadIdx.x; e < kPW * wc; e += blockDim.x) {
      const int r = e % kPW, c = e / kPW;
      float s0 = 0.0f, s1 = 0.0f;
      int q = (c / kPW) * kPW;
      for (; q + 1 < i0; q += 2) {
        s0 = fmaf(t[i0 + r][q], X[q][c], s0);
        s1 = fmaf(t[i0 + r][q + 1], X[q + 1][c], s1);
      }
      if (q < i0) s0 = fmaf(t[i0 + r][q], X[q][c], s0);
      Tm[r][c] = s0 + s1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kPW * wc; e += blockDim.x) {
      const int r = e % kPW, c = e / kPW;
      float s = 0.0f;
      for (int q = 0; q <= r; ++q) s = fmaf(X[i0 + r][i0 + q], Tm[q][c], s);
      X[i0 + r][c] = i0 + r < npiv ? -s : 0.0f;
    }
    __syncthreads();
  }
  float *out = tinv + bi.ioff + (long long)k * NB * NB;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    if (r < nr && c < nr && r >= c) g[(long long)c * bi.lda + r] = t[r][c];
    out[i] = r < npiv ? X[r][c] : (c < npiv ? t[r][c] : 0.0f);
  }
}

// Panel tile (I, k) below the diagonal: X = A_Ik L_kk^-T on the pivot columns
// (a 64x64x64 product with the stored inverse), then the non-pivot columns of
// a block's last pivot tile: A_Is -= X L_sk'.
// TF32 rounding (round to nearest, ties away), the value with its low 13
// mantissa bits zero
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// With pstage (FP32 factors, tensor-core update) the finished panel tile is
// also written to its staging slot as two TF32 words, hi = tf32(x) and
// lo = tf32(x - hi), in the K-major operand layout of tcgen05.mma without
// swizzling: 8-row x 4-column core matrices of 16-byte rows, the 16 core
// matrices of an 8-row group along the pivot columns, then the next group
// (entry (r, c) at (r/8)*512 + (c/4)*32 + (r%8)*4 + c%4; hi in words
// 0..4095, lo in 4096..8191).  Rows past the matrix and columns past the
// pivots are zero.
template <typename T>
__global__ void __launch_bounds__(kThreads) pchol_trsm_inv_kernel(T *buf, const T *tinv,
                                                                  const BlkInfo *blk, int k,
                                                                  float *pstage) {
  const BlkInfo bi = blk[blockIdx.y];
  if (k >= bi.Tp) return;
  const int I = k + 1 + blockIdx.x;
  if (I >= bi.T) return;
  extern __shared__ __align__(16) unsigned char trsm_raw[];   // two (NB x NB+1) tiles
  T(*A)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(trsm_raw);
  T(*V)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(trsm_raw + sizeof(T) * NB * (NB + 1));
  const int r0 = k * NB;
  const int nr = min(NB, bi.a - r0);
  const int npiv = min(NB, bi.p - r0);
  const int ri = I * NB;
  const int nri = min(NB, bi.a - ri);
  T *gx = buf + bi.base + (long long)r0 * bi.lda + ri;
  const T *ti = tinv + bi.ioff + (long long)k * NB * NB;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    A[r][c] = (r < nri && c < nr) ? gx[(long long)c * bi.lda + r] : T(0);
    V[r][c] = ti[i];   // V[r][c]: inverse (r < npiv) or factor (r >= npiv) entry (r, c)
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int q = 0; q < npiv; ++q) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = A[tx + 16 * a][q];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = V[ty + 16 * b][q];   // (L^-1)(c, q), zero for q > c
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = ty + 16 * b;
      if (c < npiv) A[tx + 16 * a][c] = acc[a][b];
    }
  __syncthreads();
  if (npiv < nr) {
    const int ns = nr - npiv;
    for (int idx = threadIdx.x; idx < nri * ns; idx += blockDim.x) {
      const int r = idx % nri, sc = npiv + idx / nri;
      T u = A[r][sc];
      for (int c = 0; c < npiv; ++c) u = fma(-A[r][c], V[sc][c], u);
      A[r][sc] = u;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    if (r < nri && c < nr) gx[(long long)c * bi.lda + r] = A[r][c];
  }
  if constexpr (sizeof(T) == sizeof(float)) {
    if (pstage) {
      float *st = pstage + (bi.soff + I) * 8192LL;
      for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = (e >> 9) * 8 + ((e >> 2) & 7), c = ((e >> 5) & 15) * 4 + (e & 3);
        const float v = (r < nri && c < npiv) ? (float)A[r][c] : 0.0f;
        const float h = tf32_round(v);
        st[e] = h;
        st[NB * NB + e] = tf32_round(v - h);
      }
    }
  }
}

// --------------------------------------------------------------------------
// float-float factors (hi + lo, both FP32).  The diagonal tile and the panel
// run in FP64 arithmetic on the converted values (a small share of the work);
// the trailing update -- nearly all the flops -- runs in double-float
// arithmetic on the FP32 pipe: each product by an FMA-based exact product, the
// sum by error-free two-sum, the low parts in FP32, renormalised per chunk.
// The __f*_rn intrinsics keep the compiler from contracting the error-free
// transformations into FMAs.
// --------------------------------------------------------------------------
__device__ __forceinline__ double ff_get(const float *hi, const float *lo, long long i) {
  return (double)hi[i] + (double)lo[i];
}

__device__ __forceinline__ void ff_put(float *hi, float *lo, long long i, double v) {
  const float h = (float)v;
  hi[i] = h;
  lo[i] = (float)(v - (double)h);
}

// (sh, sl) += (ah + al)(bh + bl), al*bl dropped
__device__ __forceinline__ void ff_mac(float &sh, float &sl, float ah, float al, float bh,
                                       float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);   // exact rounding error of ah*bh
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = __fadd_rn(sh, p);
  const float bv = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

__device__ __forceinline__ void ff_renorm(float &sh, float &sl) {
  const float h = __fadd_rn(sh, sl);
  sl = __fsub_rn(sl, __fsub_rn(h, sh));
  sh = h;
}

// hi + lo -> FP64 copy of the float-float factor, used by the solves; four
// entries per thread and step (16-byte loads of each word, two 16-byte
// stores; the buffers are cudaMalloc-aligned), the last n % 4 one by one
__global__ void ff_expand_kernel(const float *__restrict__ hi, const float *__restrict__ lo,
                                 double *__restrict__ out, long long n) {
  const long long n4 = n / 4;
  const float4 *h4 = reinterpret_cast<const float4 *>(hi);
  const float4 *l4 = reinterpret_cast<const float4 *>(lo);
  double2 *o2 = reinterpret_cast<double2 *>(out);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 h = __ldcs(h4 + i), l = __ldcs(l4 + i);
    __stcs(o2 + 2 * i, make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y));
    __stcs(o2 + 2 * i + 1, make_double2((double)h.z + (double)l.z, (double)h.w + (double)l.w));
  }
  for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += stride)
    out[i] = (double)hi[i] + (double)lo[i];
}

__global__ void __launch_bounds__(kThreads) pchol_potrf_ff_kernel(float *hi, float *lo,
                                                                  const BlkInfo *blk, int k,
                                                                  const double *diag0, double tol,
                                                                  int *status, double drop) {
  const BlkInfo bi = blk[blockIdx.x];
  if (k >= bi.Tp) return;
  __shared__ double t[NB][NB + 1];
  __shared__ double s_inv;
  const int r0 = k * NB;
  const int nr = min(NB, bi.a - r0);
  const int npiv = min(NB, bi.p - r0);
  const long long g0 = bi.base + (long long)r0 * bi.lda + r0;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    t[r][c] = (r < nr && c < nr && r >= c) ? ff_get(hi, lo, g0 + (long long)c * bi.lda + r) : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < npiv; ++c) {
    if (threadIdx.x == 0) {
      double piv = t[c][c];
      pivot_fix(piv, diag0[bi.d0off + r0 + c], tol, status, bi.tag + (int)blockIdx.x, r0 + c,
                drop, kDropCapFF);
      const double l = sqrt(piv);
      t[c][c] = l;
      s_inv = 1.0 / l;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int r = c + 1 + threadIdx.x; r < nr; r += blockDim.x) t[r][c] *= inv;
    __syncthreads();
    const int m = nr - c - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int rr = idx % m, ss = idx / m;
      if (rr >= ss) t[c + 1 + rr][c + 1 + ss] -= t[c + 1 + rr][c] * t[c + 1 + ss][c];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    if (r < nr && c < nr && r >= c) ff_put(hi, lo, g0 + (long long)c * bi.lda + r, t[r][c]);
  }
}

// With dstage (the tensor-core float-float update, k_tc.cu) the finished
// panel tile is also written as exact integer digits: per row r, E_r is the
// exponent with max_c |x_rc| < 2^E_r, and x = 2^E_r sum_s d_s 2^(-9-8s),
// s = 0..5, with |d_0| <= 512 and |d_s| <= 128 (s > 0), each digit an FP16
// integer (49 bits in all).  The digits are taken from the stored pair
// (hi, lo), scaled by a power of two and peeled off in FP32 with every
// remainder kept exactly (a two-word remainder, renormalised by two-sum).
// Digit plane s of the tile is a 64 x 64 FP16 K-major operand without
// swizzling, split into two K halves so that either half is one contiguous
// 4 KB run: entry (r, c) at (c/32)*2048 + (r/8)*256 + ((c%32)/8)*64 +
// (r%8)*8 + c%8; the six planes follow each other (4096 entries each).  Rows
// past the matrix and columns past the pivots are zero.
constexpr int kOzDigits = 6;

__device__ __forceinline__ void two_sum_f(float &a, float &b) {   // (a, b) <- fl(a+b), error
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  a = s;
  b = err;
}

__device__ __forceinline__ void oz_digits(float h, float l, int e, float (&d)[kOzDigits]) {
  h = ldexpf(h, 9 - e);
  l = ldexpf(l, 9 - e);
#pragma unroll
  for (int s = 0; s < kOzDigits; ++s) {
    if (s > 0) {
      h = __fmul_rn(h, 256.0f);
      l = __fmul_rn(l, 256.0f);
    }
    const float q = rintf(h);
    d[s] = q;
    h = __fsub_rn(h, q);   // exact: q is the integer nearest to h
    two_sum_f(h, l);
  }
}

// The panel in double-float arithmetic on the FP32 pipe (FP64 runs at 1/74
// of the FP32 rate on this part): column c of X = A_Ik L_kk^-T is scaled by
// the pivot's reciprocal (taken in FP64 and split into two words), then
// removed from the columns right of it, every product an FMA-based exact
// product and every difference an error-free two-sum.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph,
                                       float &pl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  ph = __fadd_rn(p, e);
  pl = __fsub_rn(e, __fsub_rn(ph, p));
}

__device__ __forceinline__ void df_sub(float &xh, float &xl, float ph, float pl) {
  const float s = __fsub_rn(xh, ph);
  const float bv = __fsub_rn(s, xh);
  const float err = __fadd_rn(__fsub_rn(xh, __fsub_rn(s, bv)), __fsub_rn(-ph, bv));
  const float el = __fadd_rn(err, __fsub_rn(xl, pl));
  xh = __fadd_rn(s, el);
  xl = __fsub_rn(el, __fsub_rn(xh, s));
}

// Rows of X are independent (X_r = A_r L^-T), so one thread solves one row
// and no step waits for another thread.  A row is taken in chunks of 16
// columns held in registers: first every finished column left of the chunk
// (kept in shared memory) is removed from it, then the chunk's own triangle
// is solved.  Every entry so receives the same operations in the same order
// as in column-by-column substitution (the subtractions of columns
// 0, 1, ..., c - 1, then the scaling), and the same rounding.  Two tiles of
// the same block and step per CTA share the pivot tile.
constexpr int kFFRowTiles = 2;
constexpr int kFFRowThreads = kFFRowTiles * NB;
constexpr int kFFChunk = 16;
constexpr size_t kTrsmFFSmem =
    (2 * NB * NB + 2 * kFFRowTiles * NB * NB + 2 * NB) * sizeof(float);

__global__ void __launch_bounds__(kFFRowThreads) pchol_trsm_ff_kernel(float *hi, float *lo,
                                                                     const BlkInfo *blk, int k,
                                                                     __half *dstage, int *dexp) {
  const BlkInfo bi = blk[blockIdx.y];
  if (k >= bi.Tp) return;
  const int I0 = k + 1 + kFFRowTiles * blockIdx.x;
  if (I0 >= bi.T) return;
  extern __shared__ __align__(16) float trsm_f[];
  float *Lth = trsm_f;                     // [c][sc] = L_kk(sc, c): pivot column c contiguous
  float *Ltl = Lth + NB * NB;
  float *Xsh = Ltl + NB * NB;              // [tile][c][r]: finished columns of the rows
  float *Xsl = Xsh + kFFRowTiles * NB * NB;
  float *s_ih = Xsl + kFFRowTiles * NB * NB;   // pivot reciprocals, split in two words
  float *s_il = s_ih + NB;
  const int r0 = k * NB;
  const int nr = min(NB, bi.a - r0);
  const int npiv = min(NB, bi.p - r0);
  const long long gl = bi.base + (long long)r0 * bi.lda + r0;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int sc = i % NB, c = i / NB;
    const bool lin = sc < nr && c < nr && sc >= c;
    const long long el = gl + (long long)c * bi.lda + sc;
    Lth[c * NB + sc] = lin ? hi[el] : 0.0f;
    Ltl[c * NB + sc] = lin ? lo[el] : 0.0f;
  }
  __syncthreads();
  if (threadIdx.x < npiv) {
    const int c = threadIdx.x;
    const double inv = 1.0 / ((double)Lth[c * NB + c] + (double)Ltl[c * NB + c]);
    s_ih[c] = (float)inv;
    s_il[c] = (float)(inv - (double)s_ih[c]);
  }
  __syncthreads();

  const int t = threadIdx.x / NB, r = threadIdx.x % NB;
  const int I = I0 + t;
  const bool tile_ok = I < bi.T;
  const int ri = I * NB;
  const int nri = tile_ok ? min(NB, bi.a - ri) : 0;
  const bool row_ok = r < nri;
  const long long gx = bi.base + (long long)r0 * bi.lda + ri;
  float *xsh = Xsh + t * NB * NB + r, *xsl = Xsl + t * NB * NB + r;   // column c at [c * NB]
  for (int c0 = 0; c0 < nr; c0 += kFFChunk) {
    float xh[kFFChunk], xl[kFFChunk];
#pragma unroll
    for (int j = 0; j < kFFChunk; ++j) {
      const int c = c0 + j;
      const bool in = row_ok && c < nr;
      xh[j] = in ? hi[gx + (long long)c * bi.lda + r] : 0.0f;
      xl[j] = in ? lo[gx + (long long)c * bi.lda + r] : 0.0f;
    }
    // the finished pivot columns left of the chunk
    const int cend = min(c0, npiv);
    for (int c = 0; c < cend; ++c) {
      const float ah = xsh[c * NB], al = xsl[c * NB];
      const float4 *Lh4 = reinterpret_cast<const float4 *>(Lth + c * NB + c0);
      const float4 *Ll4 = reinterpret_cast<const float4 *>(Ltl + c * NB + c0);
#pragma unroll
      for (int q = 0; q < kFFChunk / 4; ++q) {
        const float4 bh = Lh4[q], bl = Ll4[q];
        const float bhv[4] = {bh.x, bh.y, bh.z, bh.w}, blv[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float ph, pl;
          df_mul(ah, al, bhv[u], blv[u], ph, pl);
          df_sub(xh[4 * q + u], xl[4 * q + u], ph, pl);
        }
      }
    }
    // the chunk's own triangle
#pragma unroll
    for (int j = 0; j < kFFChunk; ++j) {
      const int c = c0 + j;
      if (c < npiv) {
        df_mul(xh[j], xl[j], s_ih[c], s_il[c], xh[j], xl[j]);
#pragma unroll
        for (int jj = j + 1; jj < kFFChunk; ++jj) {
          float ph, pl;
          df_mul(xh[j], xl[j], Lth[c * NB + c0 + jj], Ltl[c * NB + c0 + jj], ph, pl);
          df_sub(xh[jj], xl[jj], ph, pl);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kFFChunk; ++j) {
      const int c = c0 + j;
      xsh[c * NB] = xh[j];
      xsl[c * NB] = xl[j];
      if (row_ok && c < nr) {
        hi[gx + (long long)c * bi.lda + r] = xh[j];
        lo[gx + (long long)c * bi.lda + r] = xl[j];
      }
    }
  }
  if (dstage && tile_ok) {
    const long long slot = bi.soff + I;
    float mx = 0.0f;
    if (row_ok)
      for (int c = 0; c < npiv; ++c) mx = fmaxf(mx, fabsf(xsh[c * NB]));
    int e = 0;
    if (mx > 0.0f) frexpf(mx, &e);   // mx = f 2^e, f in [0.5, 1)
    dexp[slot * NB + r] = e;
    __half *st = dstage + slot * (kOzDigits * NB * NB) + (r >> 3) * 256 + (r & 7) * 8;
#pragma unroll 1
    for (int cg = 0; cg < NB / 8; ++cg) {   // 8 consecutive columns: one 16-byte run per plane
      __align__(16) __half dv[kOzDigits][8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = cg * 8 + u;
        float d[kOzDigits];
        if (row_ok && c < npiv) {
          oz_digits(xsh[c * NB], xsl[c * NB], e, d);
        } else {
#pragma unroll
          for (int q = 0; q < kOzDigits; ++q) d[q] = 0.0f;
        }
#pragma unroll
        for (int q = 0; q < kOzDigits; ++q) dv[q][u] = __float2half_rn(d[q]);
      }
      const int off = (cg >> 2) * 2048 + (cg & 3) * 64;
#pragma unroll
      for (int q = 0; q < kOzDigits; ++q)
        *reinterpret_cast<uint4 *>(st + q * NB * NB + off) =
            *reinterpret_cast<const uint4 *>(dv[q]);
    }
  }
}

// trailing update: C_IJ -= L_Ik L_Jk' over the pivot columns of step k (the
// FP64 factor; FP32 and float-float have their own kernels below).
constexpr int KC = 16;
template <typename T>
__global__ void __launch_bounds__(kThreads) pchol_update_kernel(T *buf, const BlkInfo *blk, int k) {
  const BlkInfo bi = blk[blockIdx.y];
  if (k >= bi.Tp) return;
  const long long t = bi.T - k - 1;
  const long long q = blockIdx.x;
  if (q >= t * (t + 1) / 2) return;
  long long ii = (long long)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
  while (ii * (ii + 1) / 2 > q) --ii;
  while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
  const long long jj = q - ii * (ii + 1) / 2;
  const int I = k + 1 + (int)ii, J = k + 1 + (int)jj;
  const int npiv = min(NB, bi.p - k * NB);
  const int rI = I * NB, rJ = J * NB;
  const int nrI = min(NB, bi.a - rI), nrJ = min(NB, bi.a - rJ);
  __shared__ T As[KC][NB];
  __shared__ T Bs[KC][NB];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const T *colk = buf + bi.base + (long long)(k * NB) * bi.lda;
  for (int kc = 0; kc < npiv; kc += KC) {
    for (int idx = threadIdx.x; idx < KC * NB; idx += blockDim.x) {
      const int r = idx % NB, kk = idx / NB;
      const bool kin = (kc + kk) < npiv;
      const T *col = colk + (long long)(kc + kk) * bi.lda;
      As[kk][r] = (kin && r < nrI) ? col[rI + r] : T(0);
      Bs[kk][r] = (kin && r < nrJ) ? col[rJ + r] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  T *gc = buf + bi.base + (long long)rJ * bi.lda + rI;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = ty + 16 * j;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = tx + 16 * i;
      if (r < nrI && c < nrJ && (I != J || r >= c)) gc[(long long)c * bi.lda + r] -= acc[i][j];
    }
  }
}

// FP32 trailing update.  The FP64 kernel's 4x4-per-thread tile above, run in
// FP32, leaves the FP32 pipe waiting on shared-memory issue (8 scalar loads
// per 16 FMAs); here 64
// threads cover the 64x64 tile with an 8x8 register tile each, reading it
// with four 16-byte shared loads per 64 FMAs.  Rows 4tx..4tx+3 and
// 32+4tx..35+4tx, columns likewise with ty, so that the 16-byte loads of a
// quarter warp cover 128 contiguous bytes.  The whole 64-column panel is
// requested up front with cp.async, in four 16-column groups, and the
// arithmetic on a group starts as soon as it has landed, so the later groups
// arrive behind the arithmetic; ragged rows and columns past the pivots are
// zero-filled by the copy itself.
constexpr int kUpdF32Threads = 64;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(kUpdF32Threads) pchol_update_f32_kernel(float *buf,
                                                                         const BlkInfo *blk,
                                                                         int k) {
  const BlkInfo bi = blk[blockIdx.y];
  if (k >= bi.Tp) return;
  const long long t = bi.T - k - 1;
  const long long q = blockIdx.x;
  if (q >= t * (t + 1) / 2) return;
  long long ii = (long long)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
  while (ii * (ii + 1) / 2 > q) --ii;
  while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
  const long long jj = q - ii * (ii + 1) / 2;
  const int I = k + 1 + (int)ii, J = k + 1 + (int)jj;
  const int npiv = min(NB, bi.p - k * NB);
  const int rI = I * NB, rJ = J * NB;
  const int nrI = min(NB, bi.a - rI), nrJ = min(NB, bi.a - rJ);
  __shared__ __align__(16) float As[NB][NB];   // [pivot column][row]
  __shared__ __align__(16) float Bs[NB][NB];
  const int tid = threadIdx.x;
  const int tx = tid & 7, ty = tid >> 3;
  // copies: thread moves float4 number (tid & 15) of columns (tid >> 4) + 4u
  const int lv = (tid & 15) * 4, lk = tid >> 4;
  const float *colk = buf + bi.base + (long long)(k * NB) * bi.lda;
  const int nchunk = (npiv + 15) / 16;
  const int na = 4 * max(0, min(4, nrI - lv)), nb = 4 * max(0, min(4, nrJ - lv));
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    if (ch < nchunk) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kk = ch * 16 + lk + 4 * u;
        const bool kin = kk < npiv;
        // a zero-byte copy still names a valid address: row rI / rJ of a pivot column
        const float *col = colk + (long long)(kin ? kk : 0) * bi.lda;
        cp_async16(&As[kk][lv], col + rI + (kin && na ? lv : 0), kin ? na : 0);
        cp_async16(&Bs[kk][lv], col + rJ + (kin && nb ? lv : 0), kin ? nb : 0);
      }
    }
    cp_async_commit();
  }
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  for (int ch = 0; ch < nchunk; ++ch) {
    if (ch == 0) cp_async_wait<3>();
    else if (ch == 1) cp_async_wait<2>();
    else if (ch == 2) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
#pragma unroll
    for (int kq = 0; kq < 16; ++kq) {
      const int kk = ch * 16 + kq;
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][4 * tx]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][32 + 4 * tx]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][4 * ty]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][32 + 4 * ty]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
  }
  float *gc = buf + bi.base + (long long)rJ * bi.lda + rI;
  const bool diag = I == J;
  if (!diag && nrI == NB && nrJ == NB) {
    // interior tile: the eight loads of a row quad are issued before any store
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = h == 0 ? 4 * tx : 32 + 4 * tx;
      float4 cv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = (j < 4 ? 4 * ty : 32 + 4 * ty) + (j & 3);
        cv[j] = *reinterpret_cast<const float4 *>(gc + (long long)c * bi.lda + r);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = (j < 4 ? 4 * ty : 32 + 4 * ty) + (j & 3);
        cv[j].x -= acc[4 * h][j];
        cv[j].y -= acc[4 * h + 1][j];
        cv[j].z -= acc[4 * h + 2][j];
        cv[j].w -= acc[4 * h + 3][j];
        *reinterpret_cast<float4 *>(gc + (long long)c * bi.lda + r) = cv[j];
      }
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = (j < 4 ? 4 * ty : 32 + 4 * ty) + (j & 3);
    if (c >= nrJ) continue;
    float *col = gc + (long long)c * bi.lda;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = (h == 0 ? 4 * tx : 32 + 4 * tx);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (r + e < nrI && (!diag || r + e >= c)) col[r + e] -= acc[4 * h + e][j];
    }
  }
}

// Float-float trailing update with an 8x4 register tile per thread (128
// threads per 64x64 tile): rows 4tx..4tx+3 and 32+4tx..35+4tx, columns
// 4ty..4ty+3, read with six 16-byte shared loads per 32 multiply-adds of 12
// FP32 operations each.  The whole panel (high and low words of both tile
// rows, 64 KB) is requested up front with cp.async in four 16-column groups.
constexpr int kUpdFFThreads = 128;
constexpr size_t kUpdFFSmem = 4 * NB * NB * sizeof(float);

__global__ void __launch_bounds__(kUpdFFThreads) pchol_update_ff8_kernel(float *hi, float *lo,
                                                                        const BlkInfo *blk,
                                                                        int k) {
  const BlkInfo bi = blk[blockIdx.y];
  if (k >= bi.Tp) return;
  const long long t = bi.T - k - 1;
  const long long q = blockIdx.x;
  if (q >= t * (t + 1) / 2) return;
  long long ii = (long long)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
  while (ii * (ii + 1) / 2 > q) --ii;
  while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
  const long long jj = q - ii * (ii + 1) / 2;
  const int I = k + 1 + (int)ii, J = k + 1 + (int)jj;
  const int npiv = min(NB, bi.p - k * NB);
  const int rI = I * NB, rJ = J * NB;
  const int nrI = min(NB, bi.a - rI), nrJ = min(NB, bi.a - rJ);
  extern __shared__ __align__(16) float ffsm[];
  float(*Ah)[NB] = reinterpret_cast<float(*)[NB]>(ffsm);
  float(*Al)[NB] = reinterpret_cast<float(*)[NB]>(ffsm + NB * NB);
  float(*Bh)[NB] = reinterpret_cast<float(*)[NB]>(ffsm + 2 * NB * NB);
  float(*Bl)[NB] = reinterpret_cast<float(*)[NB]>(ffsm + 3 * NB * NB);
  const int tid = threadIdx.x;
  const int tx = tid & 7, ty = tid >> 3;
  // copies: thread moves float4 number (tid & 15) of column (tid >> 4) of a
  // chunk, for both words of both tile rows (8 x 16-byte copies per chunk)
  const int lv = (tid & 15) * 4, lk = tid >> 4;
  const long long colk = bi.base + (long long)(k * NB) * bi.lda;
  const int nchunk = (npiv + 15) / 16;
  const int na = 4 * max(0, min(4, nrI - lv)), nb = 4 * max(0, min(4, nrJ - lv));
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    if (ch < nchunk) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int kk = ch * 16 + lk + 8 * u;
        const bool kin = kk < npiv;
        const long long col = colk + (long long)(kin ? kk : 0) * bi.lda;
        const long long oa = col + rI + (kin && na ? lv : 0);
        const long long ob = col + rJ + (kin && nb ? lv : 0);
        cp_async16(&Ah[kk][lv], hi + oa, kin ? na : 0);
        cp_async16(&Al[kk][lv], lo + oa, kin ? na : 0);
        cp_async16(&Bh[kk][lv], hi + ob, kin ? nb : 0);
        cp_async16(&Bl[kk][lv], lo + ob, kin ? nb : 0);
      }
    }
    cp_async_commit();
  }
  float sh[8][4], sl[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.0f;
  for (int ch = 0; ch < nchunk; ++ch) {
    if (ch == 0) cp_async_wait<3>();
    else if (ch == 1) cp_async_wait<2>();
    else if (ch == 2) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
#pragma unroll 4
    for (int kq = 0; kq < 16; ++kq) {
      const int kk = ch * 16 + kq;
      const float4 h0 = *reinterpret_cast<const float4 *>(&Ah[kk][4 * tx]);
      const float4 h1 = *reinterpret_cast<const float4 *>(&Ah[kk][32 + 4 * tx]);
      const float4 l0 = *reinterpret_cast<const float4 *>(&Al[kk][4 * tx]);
      const float4 l1 = *reinterpret_cast<const float4 *>(&Al[kk][32 + 4 * tx]);
      const float4 bh4 = *reinterpret_cast<const float4 *>(&Bh[kk][4 * ty]);
      const float4 bl4 = *reinterpret_cast<const float4 *>(&Bl[kk][4 * ty]);
      const float ah[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
      const float al[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
      const float bh[4] = {bh4.x, bh4.y, bh4.z, bh4.w};
      const float bl[4] = {bl4.x, bl4.y, bl4.z, bl4.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ff_mac(sh[i][j], sl[i][j], ah[i], al[i], bh[j], bl[j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) ff_renorm(sh[i][j], sl[i][j]);
  }
  const long long g = bi.base + (long long)rJ * bi.lda + rI;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = 4 * ty + j;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = (i < 4 ? 4 * tx : 32 + 4 * tx) + (i & 3);
      if (r < nrI && c < nrJ && (I != J || r >= c)) {
        const long long e = g + (long long)c * bi.lda + r;
        // (ch + cl) - (sh + sl): two-sum of the high parts, low parts added
        const float chv = hi[e], clv = lo[e], s = sh[i][j];
        const float tt = __fsub_rn(chv, s);
        const float bv = __fsub_rn(tt, chv);
        const float err = __fadd_rn(__fsub_rn(chv, __fsub_rn(tt, bv)), __fsub_rn(-s, bv));
        const float el = __fadd_rn(err, __fsub_rn(clv, sl[i][j]));
        const float h = __fadd_rn(tt, el);
        hi[e] = h;
        lo[e] = __fsub_rn(el, __fsub_rn(h, tt));
      }
    }
  }
}

// --------------------------------------------------------------------------
// solves with the partial factor (one CTA per problem, vector in smem)
// forward : v <- [L11 0; L21 I]^-1 v
// backward: v_top <- L11^-T (v_top - L21' v_bottom), v_bottom unchanged
// The arithmetic runs in the factor's precision; the vector in global memory
// is FP64 either way.  Per 64-column step the diagonal tile and its
// reciprocal pivots are staged in shared memory (the sequential part runs
// there), and the panel below it is streamed with eight independent loads
// per thread in flight so the step is bandwidth-, not latency-bound.
// --------------------------------------------------------------------------
constexpr int kSolveThreads = 1024;

template <typename T>
__device__ __forceinline__ void stage_diag_tile(const T *L, long long lda, int c0, int nr,
                                                int npiv, T (*dt)[NB + 1], T *dinv) {
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    if (r < nr && c < npiv) dt[r][c] = L[(long long)(c0 + c) * lda + c0 + r];
  }
  for (int c = threadIdx.x; c < npiv; c += blockDim.x)
    dinv[c] = T(1) / L[(long long)(c0 + c) * lda + c0 + c];
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads) ptri_fwd_kernel(const T *__restrict__ buf,
                                                                 const BlkInfo *blk,
                                                                 double *vec) {
  extern __shared__ __align__(16) unsigned char vraw[];
  __shared__ T dt[NB][NB + 1];   // diagonal tile, dt[r][c]
  __shared__ T dinv[NB];
  T *v = reinterpret_cast<T *>(vraw);
  const BlkInfo bi = blk[blockIdx.x];
  double *gv = vec + bi.voff;
  const T *__restrict__ L = buf + bi.base;
  const int a = bi.a;
  const long long lda = bi.lda;
  for (int i = threadIdx.x; i < a; i += blockDim.x) v[i] = (T)gv[i];
  for (int kt = 0; kt < bi.Tp; ++kt) {
    const int c0 = kt * NB;
    const int npiv = min(NB, bi.p - c0);
    const int rend = min(c0 + NB, a);
    const int nr = rend - c0;
    stage_diag_tile(L, lda, c0, nr, npiv, dt, dinv);
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int c = 0; c < npiv; ++c) {
        const T vc = v[c0 + c] * dinv[c];
        __syncwarp();
        if (lane == 0) v[c0 + c] = vc;
        for (int r = c + 1 + lane; r < nr; r += 32) v[c0 + r] -= dt[r][c] * vc;
        __syncwarp();
      }
    }
    __syncthreads();
    const T *__restrict__ P = L + (long long)c0 * lda;   // panel columns c0..c0+npiv
    for (int r = rend + threadIdx.x; r < a; r += blockDim.x) {
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      int c = 0;
      for (; c + 8 <= npiv; c += 8) {
        const T l0 = P[(long long)(c + 0) * lda + r], l1 = P[(long long)(c + 1) * lda + r];
        const T l2 = P[(long long)(c + 2) * lda + r], l3 = P[(long long)(c + 3) * lda + r];
        const T l4 = P[(long long)(c + 4) * lda + r], l5 = P[(long long)(c + 5) * lda + r];
        const T l6 = P[(long long)(c + 6) * lda + r], l7 = P[(long long)(c + 7) * lda + r];
        s0 = fma(l0, v[c0 + c + 0], s0);
        s1 = fma(l1, v[c0 + c + 1], s1);
        s2 = fma(l2, v[c0 + c + 2], s2);
        s3 = fma(l3, v[c0 + c + 3], s3);
        s0 = fma(l4, v[c0 + c + 4], s0);
        s1 = fma(l5, v[c0 + c + 5], s1);
        s2 = fma(l6, v[c0 + c + 6], s2);
        s3 = fma(l7, v[c0 + c + 7], s3);
      }
      for (; c < npiv; ++c) s0 = fma(P[(long long)c * lda + r], v[c0 + c], s0);
      v[r] -= (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < a; i += blockDim.x) gv[i] = (double)v[i];
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads) ptri_bwd_kernel(const T *__restrict__ buf,
                                                                 const BlkInfo *blk,
                                                                 double *vec) {
  extern __shared__ __align__(16) unsigned char vraw[];
  __shared__ T dt[NB][NB + 1];   // diagonal tile, dt[r][c]
  __shared__ T dinv[NB];
  T *v = reinterpret_cast<T *>(vraw);
  const BlkInfo bi = blk[blockIdx.x];
  double *gv = vec + bi.voff;
  const T *__restrict__ L = buf + bi.base;
  const int a = bi.a;
  const long long lda = bi.lda;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int i = threadIdx.x; i < a; i += blockDim.x) v[i] = (T)gv[i];
  __syncthreads();
  for (int kt = bi.Tp - 1; kt >= 0; --kt) {
    const int c0 = kt * NB;
    const int npiv = min(NB, bi.p - c0);
    const int rend = min(c0 + NB, a);
    const int nr = rend - c0;
    stage_diag_tile(L, lda, c0, nr, npiv, dt, dinv);
    // v[c] -= L(rend:a, c)' v(rend:a): one warp per column, lanes over rows
    for (int cc = warp; cc < npiv; cc += nwarp) {
      const T *__restrict__ col = L + (long long)(c0 + cc) * lda;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      int r = rend + lane;
      for (; r + 96 < a; r += 128) {
        const T l0 = col[r], l1 = col[r + 32], l2 = col[r + 64], l3 = col[r + 96];
        s0 = fma(l0, v[r], s0);
        s1 = fma(l1, v[r + 32], s1);
        s2 = fma(l2, v[r + 64], s2);
        s3 = fma(l3, v[r + 96], s3);
      }
      for (; r < a; r += 32) s0 = fma(col[r], v[r], s0);
      T s = (s0 + s1) + (s2 + s3);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) v[c0 + cc] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      for (int c = npiv - 1; c >= 0; --c) {
        T s = T(0);
        for (int r = c + 1 + lane; r < nr; r += 32) s = fma(dt[r][c], v[c0 + r], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) v[c0 + c] = (v[c0 + c] - s) * dinv[c];
        __syncwarp();
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < a; i += blockDim.x) gv[i] = (double)v[i];
}

// --------------------------------------------------------------------------
// Wavefront solves with the block partial factors: one CTA per (block, 64-row
// tile), so every block's factor is streamed by many SMs at once.
//
// Each CTA draws a ticket from an atomic counter and takes the job the
// schedule lists under that ticket.  The schedule is in wavefront order (tile
// r of every block before tile r+1 of any block; reversed for the backward
// sweep), so a tile only ever waits for tiles holding smaller tickets, which
// are already running: the waits cannot deadlock.  A CTA prefetches its part
// of the factor before it waits for the tile it needs, solves its diagonal
// tile, writes its solution rows and publishes them with a release store on
// its ready flag.  Every wait is bounded: after kWaitLimitNs the error word
// is set, the CTA stops waiting and the host reports AHLP_ERR_TIMEOUT.
//
// forward : v <- [L11 0; L21 I]^-1 v     (all a rows; pivot tiles publish)
// backward: v_top <- L11^-T (v_top - L21' v_bottom), v_bottom unchanged
// --------------------------------------------------------------------------
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int load_acquire(const int *f) {
  int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
  return v;
}

__device__ __forceinline__ void store_release(int *f, int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}

// Thread-level bounded wait until *f != 0.  Gives up at once when another CTA
// has already timed out, so a failure does not cascade into more waits.
__device__ void wait_ready(const int *f, int *err) {
  if (load_acquire(f)) return;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(128);
    if (load_acquire(f)) return;
    if (load_acquire(err)) return;
    if (global_ns() - t0 > kWaitLimitNs) {
      atomicExch(err, 1);
      return;
    }
  }
}

// Inverted diagonal tiles, one CTA (one thread per column) per pivot tile.
// Column j of X = L_kk^-1 by forward substitution against e_j.  The
// non-pivot rows of a block's last pivot tile keep the factor entries, so
// the solves stage one 64x64 tile that covers their whole diagonal step.
template <typename T>
__global__ void __launch_bounds__(NB) tinv_kernel(const T *__restrict__ buf, T *__restrict__ tinv,
                                                  const BlkInfo *__restrict__ blk,
                                                  const int *__restrict__ sched) {
  extern __shared__ __align__(16) unsigned char tinv_raw[];   // tinv_smem<T>() bytes
  T(*Ls)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(tinv_raw);
  T(*Xs)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(tinv_raw + sizeof(T) * NB * (NB + 1));
  T *rinv = reinterpret_cast<T *>(tinv_raw + 2 * sizeof(T) * NB * (NB + 1));
  const int b = sched[2 * blockIdx.x], k = sched[2 * blockIdx.x + 1];
  const BlkInfo bi = blk[b];
  const T *__restrict__ L = buf + bi.base;
  const int r0 = k * NB, nr = min(NB, bi.a - r0), npiv = min(NB, bi.p - r0);
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    Ls[r][c] = (r < nr && c < npiv && r >= c) ? L[(long long)(r0 + c) * bi.lda + r0 + r] : T(0);
    Xs[r][c] = T(0);
  }
  __syncthreads();
  if (threadIdx.x < npiv) rinv[threadIdx.x] = T(1) / Ls[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int j = threadIdx.x;
  if (j < npiv) {
    for (int i = j; i < npiv; ++i) {
      T s0 = (i == j) ? T(1) : T(0), s1 = T(0);
      int q = j;
      for (; q + 1 < i; q += 2) {
        s0 = fma(-Ls[i][q], Xs[q][j], s0);
        s1 = fma(-Ls[i][q + 1], Xs[q + 1][j], s1);
      }
      if (q < i) s0 = fma(-Ls[i][q], Xs[q][j], s0);
      Xs[i][j] = (s0 + s1) * rinv[i];
    }
  }
  __syncthreads();
  T *__restrict__ out = tinv + bi.ioff + (long long)k * NB * NB;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    out[i] = r < npiv ? Xs[r][c] : Ls[r][c];
  }
}

// Called by all threads when the next needed tile k may not be published.
// Warp 0 scans up to 32 flags fl[k + dir*i] in one round (tiles publish in
// order, so the set flags form a run starting at k), waits (bounded) when
// none is set yet, and the barrier count broadcasts the length of the run.
__device__ __forceinline__ int published_run(const int *fl, int k, int dir, int limit, int *err) {
  const int lane = threadIdx.x & 31;
  int c = 0;
  if (threadIdx.x < 32) {
    for (;;) {
      const int idx = k + dir * lane;
      const bool in = dir > 0 ? idx < limit : idx > limit;
      const bool set = in && load_acquire(fl + idx) != 0;
      const unsigned bal = __ballot_sync(0xffffffffu, set);
      c = bal == 0xffffffffu ? 32 : __ffs(~bal) - 1;
      if (c > 0) break;
      if (lane == 0) wait_ready(fl + k, err);
      __syncwarp();
      if (__any_sync(0xffffffffu, load_acquire(err) != 0)) {   // timed out: the host reports it
        c = 1;
        break;
      }
    }
  }
  return __syncthreads_count(threadIdx.x < 32 && lane < c);
}

// thread = (row rho of a 64-row tile or chunk, column lane q); lane q owns the
// columns q, q + kQL, ... of a 64-column tile.  The factor tiles a CTA reads
// are streamed into a ring of shared-memory stages by cp.async (16 bytes per
// copy, rows past the matrix zero-filled), kTrsvStages - 1 tiles ahead of
// the one in use, so each SM keeps several tiles of the factor in flight
// without holding them in registers; the inverse of the diagonal tile comes
// in with the first stage.

// FP64 factors go through the ring (two 32 KB stages, 512 threads, two CTAs
// per SM); FP32 factors hold the next tile in registers instead, which
// measured faster for their 16 KB tiles than a ring with a barrier per tile:
// the forward sweep with 256 threads (sixteen entries each, three CTAs per
// SM), the backward one, which also keeps sixteen accumulators per thread at
// that width, with 512 threads (eight entries each, two CTAs per SM).
template <typename T, bool Bwd>
struct TrsvCfg {
  static constexpr bool narrow = sizeof(T) == 4 && !Bwd;
  static constexpr int threads = narrow ? 256 : 512;
  static constexpr int min_ctas = narrow ? 3 : 2;   // per SM
  static constexpr int stages = sizeof(T) == 4 ? 0 : 2;
  static constexpr int ql = threads / NB;   // column lanes
  static constexpr int jc = NB / ql;        // columns per thread
};
template <typename T>
constexpr size_t trsv_smem() {
  return (size_t)TrsvCfg<T, false>::stages * NB * NB * sizeof(T);
}

// One 64 x 64 tile of a column-major factor into dst ([c][row], 64 entries per
// column): columns [0, ncols) of the tile starting at src, rows below
// `rows` are zero, so are the other columns.  Every copy reads only entries
// of the matrix.
template <typename T>
__device__ __forceinline__ void stage_factor_tile(T *dst, const T *src, long long lda, int ncols,
                                                  int rows) {
  constexpr int EPC = 16 / sizeof(T);   // entries per 16-byte copy
  constexpr int CPC = NB / EPC;         // copies per column
  for (int ch = threadIdx.x; ch < NB * CPC; ch += blockDim.x) {
    const int c = ch / CPC, rr = (ch % CPC) * EPC;
    const int valid = c < ncols ? max(0, min(EPC, rows - rr)) : 0;
    const T *g = valid ? src + (long long)c * lda + rr : src;
    cp_async16(dst + c * NB + rr, g, valid * (int)sizeof(T));
  }
}

// n contiguous entries (a multiple of 16 bytes)
template <typename T>
__device__ __forceinline__ void stage_contiguous(T *dst, const T *src, int n) {
  constexpr int EPC = 16 / sizeof(T);
  for (int i = threadIdx.x * EPC; i < n; i += blockDim.x * EPC) cp_async16(dst + i, src + i, 16);
}

template <typename T>
__global__ void __launch_bounds__(TrsvCfg<T, false>::threads, TrsvCfg<T, false>::min_ctas)
    trsv_fwd_kernel(const T *__restrict__ buf, const T *__restrict__ tinv,
                    const BlkInfo *__restrict__ blk, const int *__restrict__ sched,
                    const int *__restrict__ flag_off, int *flags, int *ticket, int *err,
                    double *vec, T *vecT) {
  constexpr int S = TrsvCfg<T, false>::stages;
  constexpr int kQL = TrsvCfg<T, false>::ql, kJC = TrsvCfg<T, false>::jc;
  extern __shared__ __align__(16) unsigned char trsv_raw[];
  T *ring = reinterpret_cast<T *>(trsv_raw);   // S tiles, [c][row]
  __shared__ __align__(16) T Xs[NB * NB];      // column-major, Xs[c * NB + r]
  __shared__ T red[kQL][NB];
  __shared__ T u[NB];
  __shared__ T xs[NB];
  __shared__ int s_job;
  if (threadIdx.x == 0) s_job = atomicAdd(ticket, 1);
  __syncthreads();
  const int b = sched[2 * s_job], r = sched[2 * s_job + 1];
  const BlkInfo bi = blk[b];
  const T *__restrict__ L = buf + bi.base;
  const long long lda = bi.lda;
  double *gv = vec + bi.voff;
  T *gvT = vecT + bi.voff;   // solution in the factor's precision (gv itself for FP64)
  int *fl = flags + flag_off[b];
  const int r0 = r * NB, nr = min(NB, bi.a - r0);
  const bool pivtile = r < bi.Tp;
  const int npiv = pivtile ? min(NB, bi.p - r0) : 0;
  const int rho = threadIdx.x & (NB - 1), q = threadIdx.x / NB;
  const int nct = min(r, bi.Tp);   // pivot column tiles left of this tile
  if (pivtile) stage_contiguous(Xs, tinv + bi.ioff + (long long)r * NB * NB, NB * NB);
  cp_async_commit();
  T acc0 = T(0), acc1 = T(0);
  int ready = 0;   // column tiles [0, ready) are published
  if constexpr (S > 0) {
    auto issue = [&](int k) {
      const int c0 = k * NB;
      stage_factor_tile(ring + (k % S) * NB * NB, L + (long long)c0 * lda + r0, lda,
                        min(NB, bi.p - c0), nr);
    };
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
      if (s < nct) issue(s);
      cp_async_commit();
    }
    for (int k = 0; k < nct; ++k) {
      const int c0 = k * NB, nc = min(NB, bi.p - c0);
      cp_async_wait<S - 2>();   // tile k has landed (this thread's copies) ...
      __syncthreads();          // ... everyone's, and stage (k - 1) % S is free
      if (k + S - 1 < nct) issue(k + S - 1);
      cp_async_commit();
      if (k >= ready) ready = k + published_run(fl, k, 1, nct, err);
      const T *t = ring + (k % S) * NB * NB;
#pragma unroll
      for (int j = 0; j < kJC; ++j) {
        const int c = q + kQL * j;
        if (c < nc) {
          const T xv = __ldcg(gvT + c0 + c);
          if (j & 1)
            acc1 = fma(t[c * NB + rho], xv, acc1);
          else
            acc0 = fma(t[c * NB + rho], xv, acc0);
        }
      }
    }
  } else {
    // the next tile's entries are loaded into registers while this one is used
    const bool rok = rho < nr;
    const T *__restrict__ Lr = L + r0 + rho;
    T l[kJC], ln[kJC];
    auto load_tile = [&](int k, T(&dst)[kJC]) {
      const int c0 = k * NB, nc = min(NB, bi.p - c0);
#pragma unroll
      for (int j = 0; j < kJC; ++j) {
        const int c = q + kQL * j;
        dst[j] = (rok && c < nc) ? Lr[(long long)(c0 + c) * lda] : T(0);
      }
    };
    if (nct > 0) load_tile(0, l);
    for (int k = 0; k < nct; ++k) {
      const int c0 = k * NB, nc = min(NB, bi.p - c0);
      if (k + 1 < nct) load_tile(k + 1, ln);
      if (k >= ready) ready = k + published_run(fl, k, 1, nct, err);
#pragma unroll
      for (int j = 0; j < kJC; ++j) {
        const int c = q + kQL * j;
        if (c < nc) {
          const T xv = __ldcg(gvT + c0 + c);
          if (j & 1)
            acc1 = fma(l[j], xv, acc1);
          else
            acc0 = fma(l[j], xv, acc0);
        }
      }
#pragma unroll
      for (int j = 0; j < kJC; ++j) l[j] = ln[j];
    }
  }
  cp_async_wait<0>();
  auto sum_lanes = [&](int t) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kQL; ++i) s += red[i][t];
    return s;
  };
  red[q][rho] = acc0 + acc1;
  __syncthreads();
  if (threadIdx.x < nr) u[threadIdx.x] = (T)gv[r0 + threadIdx.x] - sum_lanes(threadIdx.x);
  __syncthreads();
  if (pivtile) {
    // pivot rows: x = L_rr^-1 u
    T s = T(0);
    if (rho < npiv) {
#pragma unroll
      for (int j = 0; j < kJC; ++j) {
        const int c = q + kQL * j;
        if (c < npiv) s = fma(Xs[c * NB + rho], u[c], s);
      }
    }
    red[q][rho] = s;
    __syncthreads();
    if (threadIdx.x < npiv) xs[threadIdx.x] = sum_lanes(threadIdx.x);
    __syncthreads();
    if (npiv < nr) {
      // non-pivot rows of the last pivot tile: u -= L(rows, pivots) x
      T s2 = T(0);
      if (rho >= npiv && rho < nr) {
#pragma unroll
        for (int j = 0; j < kJC; ++j) {
          const int c = q + kQL * j;
          if (c < npiv) s2 = fma(Xs[c * NB + rho], xs[c], s2);
        }
      }
      red[q][rho] = s2;
      __syncthreads();
      if (threadIdx.x >= npiv && threadIdx.x < nr) u[threadIdx.x] -= sum_lanes(threadIdx.x);
    }
    if (threadIdx.x < npiv) u[threadIdx.x] = xs[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x < nr) {
    gv[r0 + threadIdx.x] = (double)u[threadIdx.x];
    if constexpr (sizeof(T) != sizeof(double)) gvT[r0 + threadIdx.x] = u[threadIdx.x];
  }
  if (pivtile) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      store_release(fl + r, 1);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(TrsvCfg<T, true>::threads, TrsvCfg<T, true>::min_ctas)
    trsv_bwd_kernel(const T *__restrict__ buf, const T *__restrict__ tinv,
                    const BlkInfo *__restrict__ blk, const int *__restrict__ sched,
                    const int *__restrict__ flag_off, int *flags, int *ticket, int *err,
                    double *vec) {
  constexpr int S = TrsvCfg<T, true>::stages;
  constexpr int kQL = TrsvCfg<T, true>::ql, kJC = TrsvCfg<T, true>::jc;
  extern __shared__ __align__(16) unsigned char trsv_raw[];
  T *ring = reinterpret_cast<T *>(trsv_raw);   // S chunks of 64 rows, [c][row]
  __shared__ __align__(16) T Xs[NB * NB];      // column-major, Xs[c * NB + r]
  __shared__ T red[TrsvCfg<T, true>::threads / 32][kJC];
  __shared__ T u[NB];
  __shared__ int s_job;
  if (threadIdx.x == 0) s_job = atomicAdd(ticket, 1);
  __syncthreads();
  const int b = sched[2 * s_job], r = sched[2 * s_job + 1];   // r < Tp
  const BlkInfo bi = blk[b];
  const T *__restrict__ L = buf + bi.base;
  const long long lda = bi.lda;
  double *gv = vec + bi.voff;
  int *fl = flags + flag_off[b];
  const int r0 = r * NB, nr = min(NB, bi.a - r0), npiv = min(NB, bi.p - r0);
  // lane q dots the tile's columns q, q + kQL, ... with the rows of each chunk
  const int rho = threadIdx.x & (NB - 1), q = threadIdx.x / NB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T *__restrict__ Lc = L + (long long)r0 * lda;
  // chunks of rows below the pivots, bottom first: non-pivot rows are inputs,
  // pivot tiles publish upwards.  Chunk r itself holds the non-pivot rows of
  // the last pivot tile (if any).
  const int kend = npiv < nr ? r : r + 1;
  const int nch = bi.T - kend;   // chunks, taken k = T - 1, T - 2, ..., kend
  stage_contiguous(Xs, tinv + bi.ioff + (long long)r * NB * NB, NB * NB);
  cp_async_commit();
  T acc[kJC];
#pragma unroll
  for (int j = 0; j < kJC; ++j) acc[j] = T(0);
  int ready_from = bi.Tp;   // chunks k >= ready_from are final
  if constexpr (S > 0) {
    auto issue = [&](int i) {      // i-th chunk taken: k = T - 1 - i
      const int k = bi.T - 1 - i;
      stage_factor_tile(ring + (i % S) * NB * NB, Lc + (long long)k * NB, lda, npiv,
                        bi.a - k * NB);
    };
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
      if (s < nch) issue(s);
      cp_async_commit();
    }
    for (int i = 0; i < nch; ++i) {
      const int k = bi.T - 1 - i;
      cp_async_wait<S - 2>();
      __syncthreads();
      if (i + S - 1 < nch) issue(i + S - 1);
      cp_async_commit();
      // tiles publish in decreasing order
      if (k > r && k < ready_from) ready_from = k + 1 - published_run(fl, k, -1, r, err);
      const int row = k * NB + rho;
      // rows past the matrix are zero in the stage; the pivot rows of chunk r
      // (entries of L_rr) take no part
      if (row < bi.a && (k > r || rho >= npiv)) {
        const T xv = (T)__ldcg(gv + row);
        const T *t = ring + (i % S) * NB * NB;
#pragma unroll
        for (int j = 0; j < kJC; ++j) acc[j] = fma(t[(q + kQL * j) * NB + rho], xv, acc[j]);
      }
    }
  } else {
    // the next chunk's entries are loaded into registers while this one is used
    T l[kJC], ln[kJC];
    auto load_chunk = [&](int k, T(&dst)[kJC]) {
      const int row = k * NB + rho;
      const bool ok = row < bi.a && (k > r || rho >= npiv);
#pragma unroll
      for (int j = 0; j < kJC; ++j) {
        const int c = q + kQL * j;
        dst[j] = (ok && c < npiv) ? Lc[(long long)c * lda + row] : T(0);
      }
    };
    if (nch > 0) load_chunk(bi.T - 1, l);
    for (int k = bi.T - 1; k >= kend; --k) {
      if (k - 1 >= kend) load_chunk(k - 1, ln);
      // tiles publish in decreasing order
      if (k > r && k < ready_from) ready_from = k + 1 - published_run(fl, k, -1, r, err);
      const int row = k * NB + rho;
      const bool ok = row < bi.a && (k > r || rho >= npiv);
      const T xv = ok ? (T)__ldcg(gv + row) : T(0);
#pragma unroll
      for (int j = 0; j < kJC; ++j) acc[j] = fma(l[j], xv, acc[j]);
#pragma unroll
      for (int j = 0; j < kJC; ++j) l[j] = ln[j];
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // column c = q + kQL j is summed over the two warps of lane q
  auto col_sum = [&](int c) {
    const int cq = c % kQL, cj = c / kQL;
    return red[2 * cq][cj] + red[2 * cq + 1][cj];
  };
#pragma unroll
  for (int j = 0; j < kJC; ++j) {
    T s = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][j] = s;
  }
  __syncthreads();
  if (threadIdx.x < npiv) u[threadIdx.x] = (T)gv[r0 + threadIdx.x] - col_sum(threadIdx.x);
  __syncthreads();
  // x = L_rr^-T u: column c = q + kQL j collects X(rho, c) u(rho) over the rows
  const T uv = rho < npiv ? u[rho] : T(0);
#pragma unroll
  for (int j = 0; j < kJC; ++j) {
    T s = (rho < npiv) ? Xs[(q + kQL * j) * NB + rho] * uv : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][j] = s;
  }
  __syncthreads();
  if (threadIdx.x < npiv) gv[r0 + threadIdx.x] = (double)col_sum(threadIdx.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    store_release(fl + r, 1);
  }
}

template <typename T>
constexpr size_t trsm_smem() {
  return 2 * NB * (NB + 1) * sizeof(T);
}

template <typename T>
constexpr size_t tinv_smem() {
  return (2 * NB * (NB + 1) + NB) * sizeof(T);
}

template <typename T>
cudaError_t pchol_t(T *buf, T *tinv, const BlkInfo *info, const std::vector<BlkInfo> &h,
                    const double *diag0, double tol, int *status, cudaStream_t s,
                    ahlp_problem *tc = nullptr, ahlp_problem *prof = nullptr,
                    double drop = 0.0) {
  int nblk = (int)h.size();
  if (nblk == 0) return cudaSuccess;
  int maxTp = 0;
  for (auto &b : h) maxTp = b.Tp > maxTp ? b.Tp : maxTp;
  for (int k = 0; k < maxTp; ++k) {
    long long maxPanel = 0, maxTrail = 0;
    for (auto &b : h) {
      if (k >= b.Tp) continue;
      long long t = b.T - k - 1;
      if (t > maxPanel) maxPanel = t;
      if (t * (t + 1) / 2 > maxTrail) maxTrail = t * (t + 1) / 2;
    }
    if constexpr (sizeof(T) == sizeof(float)) {
      if (prof) kt_mark(prof, 0, s);
      count_launch(), pchol_potrf_f32_kernel<<<nblk, kPotrf32Threads, 0, s>>>(
                          buf, tinv, info, k, diag0, (float)tol, status, (float)drop);
      if (prof) kt_mark(prof, 1, s);
      if (maxPanel > 0)
        count_launch(), pchol_trsm_inv_kernel<T><<<dim3((unsigned)maxPanel, nblk), kThreads,
                                                   trsm_smem<T>(), s>>>(
                            buf, tinv, info, k, tc ? tc->pstage : nullptr);
    } else {
      if (prof) kt_mark(prof, 0, s);
      count_launch(), pchol_potrf_kernel<T><<<nblk, kThreads, 0, s>>>(buf, info, k, diag0, tol,
                                                                      status, drop);
      if (prof) kt_mark(prof, 1, s);
      if (maxPanel > 0)
        count_launch(), pchol_trsm_kernel<T><<<dim3((unsigned)maxPanel, nblk), kThreads,
                                               trsm_smem<T>(), s>>>(buf, info, k);
    }
    if (prof) kt_mark(prof, 2, s);
    if (maxTrail > 0) {
      if constexpr (sizeof(T) == sizeof(float)) {
        if (tc) {
          cudaError_t e = launch_update_tc(tc, k, s);
          if (e != cudaSuccess) return e;
        } else {
          count_launch(), pchol_update_f32_kernel<<<dim3((unsigned)maxTrail, nblk),
                                                    kUpdF32Threads, 0, s>>>(buf, info, k);
        }
      } else
        count_launch(), pchol_update_kernel<T><<<dim3((unsigned)maxTrail, nblk), kThreads, 0, s>>>(
                            buf, info, k);
    }
    if (prof) kt_mark(prof, 3, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t launch_dscale(ahlp_problem *p) {
  if (p->n <= 0) return cudaSuccess;
  count_launch(), dscale_kernel<<<(unsigned)((p->n + 255) / 256), 256, 0, p->stream>>>(
      p->x, p->z, p->dscale, p->xinv, p->wfin, p->n, p->fac_rho_x, p->fac_rho, p->is_x0);
  return cudaGetLastError();
}

cudaError_t launch_form(ahlp_problem *p, double delta) {
  if (p->ntiles <= 0) return cudaSuccess;
  if (p->fac_prec == kPrecFP32) {
    FormArgs<float> A{nullptr, p->ftiles, p->tile_ent, p->ent_pos, p->ent_cb, p->con_idx,
                      p->con_coef, p->dscale, p->blk, p->aug32, p->diag0, p->cdiag0, delta};
    count_launch(), form_aug_kernel<float, false><<<(unsigned)p->ntiles, kThreads, 0, p->stream>>>(A);
  } else if (p->fac_prec == kPrecFF) {
    FormArgs<float> A{p->aug_lo, p->ftiles, p->tile_ent, p->ent_pos, p->ent_cb, p->con_idx,
                      p->con_coef, p->dscale, p->blk, p->aug32, p->diag0, p->cdiag0, delta};
    count_launch(), form_aug_kernel<float, true><<<(unsigned)p->ntiles, kThreads, 0, p->stream>>>(A);
  } else {
    FormArgs<double> A{nullptr, p->ftiles, p->tile_ent, p->ent_pos, p->ent_cb, p->con_idx,
                       p->con_coef, p->dscale, p->blk, p->aug, p->diag0, p->cdiag0, delta};
    count_launch(), form_aug_kernel<double, false><<<(unsigned)p->ntiles, kThreads, 0, p->stream>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_pchol_ff(float *hi, float *lo, double *out, long long elems,
                            const BlkInfo *info, const std::vector<BlkInfo> &h,
                            const double *diag0, double tol, int *status, cudaStream_t s,
                            ahlp_problem *oz, ahlp_problem *prof, double drop) {
  int nblk = (int)h.size();
  if (nblk == 0) return cudaSuccess;
  int maxTp = 0;
  for (auto &b : h) maxTp = b.Tp > maxTp ? b.Tp : maxTp;
  for (int k = 0; k < maxTp; ++k) {
    long long maxPanel = 0, maxTrail = 0;
    for (auto &b : h) {
      if (k >= b.Tp) continue;
      long long t = b.T - k - 1;
      if (t > maxPanel) maxPanel = t;
      if (t * (t + 1) / 2 > maxTrail) maxTrail = t * (t + 1) / 2;
    }
    if (prof) kt_mark(prof, 0, s);
    count_launch(), pchol_potrf_ff_kernel<<<nblk, kThreads, 0, s>>>(hi, lo, info, k, diag0, tol,
                                                                    status, drop);
    if (prof) kt_mark(prof, 1, s);
    if (maxPanel > 0)
      count_launch(), pchol_trsm_ff_kernel<<<dim3((unsigned)((maxPanel + kFFRowTiles - 1) /
                                                             kFFRowTiles),
                                                  nblk),
                                             kFFRowThreads, kTrsmFFSmem, s>>>(
                          hi, lo, info, k, oz ? oz->dstage : nullptr, oz ? oz->dexp : nullptr);
    if (prof) kt_mark(prof, 2, s);
    if (maxTrail > 0) {
      if (oz) {
        cudaError_t e = launch_update_oz(oz, k, s);
        if (e != cudaSuccess) return e;
      } else {
        count_launch(), pchol_update_ff8_kernel<<<dim3((unsigned)maxTrail, nblk), kUpdFFThreads,
                                                  kUpdFFSmem, s>>>(hi, lo, info, k);
      }
    }
    if (prof) kt_mark(prof, 3, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (elems > 0)
    count_launch(), ff_expand_kernel<<<152 * 8, 256, 0, s>>>(hi, lo, out, elems);
  return cudaGetLastError();
}

cudaError_t launch_pchol(double *buf, const BlkInfo *info, const std::vector<BlkInfo> &h,
                         const double *diag0, double tol, int *status, cudaStream_t s,
                         ahlp_problem *prof, double drop) {
  return pchol_t<double>(buf, nullptr, info, h, diag0, tol, status, s, nullptr, prof, drop);
}

cudaError_t launch_pchol_f32(float *buf, float *tinv, const BlkInfo *info,
                             const std::vector<BlkInfo> &h, const double *diag0, double tol,
                             int *status, cudaStream_t s, ahlp_problem *tc,
                             ahlp_problem *prof, double drop) {
  return pchol_t<float>(buf, tinv, info, h, diag0, tol, status, s, tc, prof, drop);
}

cudaError_t launch_ptri(const double *buf, const BlkInfo *info, int nblk, int amax, double *vec,
                        bool forward, cudaStream_t s) {
  if (nblk == 0 || amax == 0) return cudaSuccess;
  size_t sm = (size_t)amax * sizeof(double);
  if (forward)
    count_launch(), ptri_fwd_kernel<double><<<nblk, kSolveThreads, sm, s>>>(buf, info, vec);
  else
    count_launch(), ptri_bwd_kernel<double><<<nblk, kSolveThreads, sm, s>>>(buf, info, vec);
  return cudaGetLastError();
}

cudaError_t launch_trsv(ahlp_problem *p, bool forward) {
  const int njobs = forward ? p->trsv_nf : p->trsv_nb;
  if (njobs == 0) return cudaSuccess;
  cudaStream_t s = p->stream;
  cudaError_t e =
      cudaMemsetAsync(p->trsv_flags, 0, (size_t)(p->trsv_nflags + 2) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  int *ticket = p->trsv_flags + p->trsv_nflags + (forward ? 0 : 1);
  const int *sched = forward ? p->trsv_fsched : p->trsv_bsched;
  if (p->fac_prec == kPrecFP32) {
    if (forward)
      count_launch(), trsv_fwd_kernel<float><<<njobs, TrsvCfg<float, false>::threads, trsv_smem<float>(), s>>>(
          p->aug32, p->tinv32, p->blk, sched, p->trsv_flag_off, p->trsv_flags, ticket,
          p->trsv_err, p->vec, p->vec32);
    else
      count_launch(), trsv_bwd_kernel<float><<<njobs, TrsvCfg<float, true>::threads, trsv_smem<float>(), s>>>(
          p->aug32, p->tinv32, p->blk, sched, p->trsv_flag_off, p->trsv_flags, ticket,
          p->trsv_err, p->vec);
  } else {
    if (forward)
      count_launch(), trsv_fwd_kernel<double><<<njobs, TrsvCfg<double, false>::threads, trsv_smem<double>(), s>>>(
          p->aug, p->tinv, p->blk, sched, p->trsv_flag_off, p->trsv_flags, ticket, p->trsv_err,
          p->vec, p->vec);
    else
      count_launch(), trsv_bwd_kernel<double><<<njobs, TrsvCfg<double, true>::threads, trsv_smem<double>(), s>>>(
          p->aug, p->tinv, p->blk, sched, p->trsv_flag_off, p->trsv_flags, ticket, p->trsv_err,
          p->vec);
  }
  return cudaGetLastError();
}

cudaError_t launch_tinv(ahlp_problem *p) {
  // FP32 factors write their inverse tiles in pchol_potrf_f32_kernel; FP64 and
  // float-float factors (through their FP64 copy) get them here
  if (p->trsv_nb == 0 || p->fac_prec == kPrecFP32) return cudaSuccess;
  count_launch(), tinv_kernel<double><<<p->trsv_nb, NB, tinv_smem<double>(), p->stream>>>(
      p->aug, p->tinv, p->blk, p->trsv_bsched);
  return cudaGetLastError();
}

cudaError_t set_dense_smem_limits(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(tinv_kernel<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tinv_smem<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(trsv_fwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsv_smem<float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(trsv_bwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsv_smem<float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(trsv_fwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsv_smem<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(trsv_bwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsv_smem<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pchol_update_ff8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kUpdFFSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pchol_trsm_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTrsmFFSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pchol_trsm_kernel<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)trsm_smem<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(ptri_fwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(ptri_bwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes);
  return e;
}

}  // namespace ahlp
