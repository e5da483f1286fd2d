// Dense per-block kernels: formation of the augmented matrices, the batched
// tiled partial Cholesky, and the forward / backward solves with its factor.
//
// Every block i owns an augmented lower-triangular matrix
//     [ M_i   .  ]        M_i = A_i D_i A_i' + delta I      (m_i x m_i)
//     [ G_i'  C_i]        G_i = [W_i | A_i D_i U_i' | A_i D_i Fg_i']
// stored column-major.  Eliminating its first m_i pivots (Alg. 2 lines 1-2
// in normal-equation form) leaves L_i on top, Y_i' = (L_i^-1 G_i)' below it
// and C_i - G_i' M_i^-1 G_i in the corner -- the block's Schur contribution.
#include <math.h>

#include "ahlp_internal.h"

namespace ahlp {

namespace {

// --------------------------------------------------------------------------
// formation: one CTA per 64x64 lower tile, written exactly once
// --------------------------------------------------------------------------
struct FormArgs {
  const FormTile *tiles;
  const long long *tile_ent;
  const int *ent_pos;
  const long long *ent_cb;
  const int *con_idx;
  const double *con_coef;
  const double *d;
  const BlkInfo *blk;
  double *aug;
  double *diag0;
  double *cdiag0;
  double delta;
};

__global__ void __launch_bounds__(kThreads) form_aug_kernel(FormArgs A) {
  __shared__ double t[NB * NB];   // column-major tile
  const FormTile ft = A.tiles[blockIdx.x];
  const BlkInfo bi = A.blk[ft.blk];
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) t[i] = 0.0;
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
    t[ct * NB + rt] = v;
  }
  __syncthreads();
  const int r0 = ft.I * NB, c0 = ft.J * NB;
  const int nr = min(NB, bi.a - r0), nc = min(NB, bi.a - c0);
  double *g = A.aug + bi.base + (long long)c0 * bi.lda + r0;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    if (r < nr && c < nc) g[(long long)c * bi.lda + r] = t[i];
  }
}

__global__ void dscale_kernel(const double *x, const double *z, double *d, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = x[i] / z[i];
}

// --------------------------------------------------------------------------
// partial Cholesky, step k: diagonal tile
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) pchol_potrf_kernel(double *buf, const BlkInfo *blk,
                                                               int k, const double *diag0,
                                                               double tol, int *status) {
  const BlkInfo bi = blk[blockIdx.x];
  if (k >= bi.Tp) return;
  __shared__ double t[NB][NB + 1];
  __shared__ double s_inv;
  const int r0 = k * NB;
  const int nr = min(NB, bi.a - r0);
  const int npiv = min(NB, bi.p - r0);
  double *g = buf + bi.base + (long long)r0 * bi.lda + r0;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    t[r][c] = (r < nr && c < nr && r >= c) ? g[(long long)c * bi.lda + r] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < npiv; ++c) {
    if (threadIdx.x == 0) {
      double piv = t[c][c];
      pivot_fix(piv, diag0[bi.d0off + r0 + c], tol, status, blockIdx.x, r0 + c);
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
    if (r < nr && c < nr && r >= c) g[(long long)c * bi.lda + r] = t[r][c];
  }
}

// panel tiles below the diagonal tile: X = A_Ik L_kk^-T on the pivot columns,
// and the non-pivot (Schur) columns of the tile updated with the new X.
__global__ void __launch_bounds__(kThreads) pchol_trsm_kernel(double *buf, const BlkInfo *blk,
                                                              int k) {
  const BlkInfo bi = blk[blockIdx.y];
  if (k >= bi.Tp) return;
  const int I = k + 1 + blockIdx.x;
  if (I >= bi.T) return;
  extern __shared__ double trsm_sm[];   // two (NB x NB+1) tiles, opt-in size
  double(*L)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(trsm_sm);
  double(*X)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(trsm_sm + NB * (NB + 1));
  const int r0 = k * NB;
  const int nr = min(NB, bi.a - r0);
  const int npiv = min(NB, bi.p - r0);
  const int ri = I * NB;
  const int nri = min(NB, bi.a - ri);
  const double *gl = buf + bi.base + (long long)r0 * bi.lda + r0;
  double *gx = buf + bi.base + (long long)r0 * bi.lda + ri;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
    const int r = i % NB, c = i / NB;
    L[r][c] = (r < nr && c < nr && r >= c) ? gl[(long long)c * bi.lda + r] : 0.0;
    X[r][c] = (r < nri && c < nr) ? gx[(long long)c * bi.lda + r] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < npiv; ++c) {
    const double inv = 1.0 / L[c][c];
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

// trailing update: C_IJ -= L_Ik L_Jk' over the pivot columns of step k.
constexpr int KC = 16;
__global__ void __launch_bounds__(kThreads) pchol_update_kernel(double *buf, const BlkInfo *blk,
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
  __shared__ double As[KC][NB];
  __shared__ double Bs[KC][NB];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const double *colk = buf + bi.base + (long long)(k * NB) * bi.lda;
  for (int kc = 0; kc < npiv; kc += KC) {
    for (int idx = threadIdx.x; idx < KC * NB; idx += blockDim.x) {
      const int r = idx % NB, kk = idx / NB;
      const bool kin = (kc + kk) < npiv;
      const double *col = colk + (long long)(kc + kk) * bi.lda;
      As[kk][r] = (kin && r < nrI) ? col[rI + r] : 0.0;
      Bs[kk][r] = (kin && r < nrJ) ? col[rJ + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double av[4], bv[4];
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
  double *gc = buf + bi.base + (long long)rJ * bi.lda + rI;
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

// --------------------------------------------------------------------------
// solves with the partial factor (one CTA per problem, vector in smem)
// forward : v <- [L11 0; L21 I]^-1 v
// backward: v_top <- L11^-T (v_top - L21' v_bottom), v_bottom unchanged
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) ptri_fwd_kernel(const double *__restrict__ buf,
                                                            const BlkInfo *blk, double *vec) {
  extern __shared__ double v[];
  const BlkInfo bi = blk[blockIdx.x];
  double *gv = vec + bi.voff;
  const double *L = buf + bi.base;
  const int a = bi.a;
  const long long lda = bi.lda;
  for (int i = threadIdx.x; i < a; i += blockDim.x) v[i] = gv[i];
  __syncthreads();
  for (int kt = 0; kt < bi.Tp; ++kt) {
    const int c0 = kt * NB;
    const int npiv = min(NB, bi.p - c0);
    const int rend = min(c0 + NB, a);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int c = c0; c < c0 + npiv; ++c) {
        const double *col = L + (long long)c * lda;
        const double vc = v[c] / col[c];
        __syncwarp();
        if (lane == 0) v[c] = vc;
        for (int r = c + 1 + lane; r < rend; r += 32) v[r] -= col[r] * vc;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int r = rend + threadIdx.x; r < a; r += blockDim.x) {
      double s = 0.0;
      const double *Lr = L + (long long)c0 * lda + r;
      for (int c = 0; c < npiv; ++c) s = fma(Lr[(long long)c * lda], v[c0 + c], s);
      v[r] -= s;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < a; i += blockDim.x) gv[i] = v[i];
}

__global__ void __launch_bounds__(kThreads) ptri_bwd_kernel(const double *__restrict__ buf,
                                                            const BlkInfo *blk, double *vec) {
  extern __shared__ double v[];
  const BlkInfo bi = blk[blockIdx.x];
  double *gv = vec + bi.voff;
  const double *L = buf + bi.base;
  const int a = bi.a;
  const long long lda = bi.lda;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int i = threadIdx.x; i < a; i += blockDim.x) v[i] = gv[i];
  __syncthreads();
  for (int kt = bi.Tp - 1; kt >= 0; --kt) {
    const int c0 = kt * NB;
    const int npiv = min(NB, bi.p - c0);
    const int rend = min(c0 + NB, a);
    for (int cc = warp; cc < npiv; cc += nwarp) {
      const int c = c0 + cc;
      const double *col = L + (long long)c * lda;
      double s = 0.0;
      for (int r = rend + lane; r < a; r += 32) s = fma(col[r], v[r], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) v[c] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      for (int c = c0 + npiv - 1; c >= c0; --c) {
        const double *col = L + (long long)c * lda;
        double s = 0.0;
        for (int r = c + 1 + lane; r < rend; r += 32) s = fma(col[r], v[r], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) v[c] = (v[c] - s) / col[c];
        __syncwarp();
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < a; i += blockDim.x) gv[i] = v[i];
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t launch_dscale(ahlp_problem *p) {
  if (p->n <= 0) return cudaSuccess;
  count_launch(), dscale_kernel<<<(unsigned)((p->n + 255) / 256), 256, 0, p->stream>>>(p->x, p->z, p->dscale,
                                                                       p->n);
  return cudaGetLastError();
}

cudaError_t launch_form(ahlp_problem *p, double delta) {
  if (p->ntiles <= 0) return cudaSuccess;
  FormArgs A{p->ftiles, p->tile_ent, p->ent_pos, p->ent_cb, p->con_idx, p->con_coef,
             p->dscale, p->blk, p->aug, p->diag0, p->cdiag0, delta};
  count_launch(), form_aug_kernel<<<(unsigned)p->ntiles, kThreads, 0, p->stream>>>(A);
  return cudaGetLastError();
}

constexpr size_t kTrsmSmem = 2 * NB * (NB + 1) * sizeof(double);

cudaError_t launch_pchol(double *buf, const BlkInfo *info, const std::vector<BlkInfo> &h,
                         const double *diag0, double tol, int *status, cudaStream_t s) {
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
    count_launch(), pchol_potrf_kernel<<<nblk, kThreads, 0, s>>>(buf, info, k, diag0, tol, status);
    if (maxPanel > 0)
      count_launch(), pchol_trsm_kernel<<<dim3((unsigned)maxPanel, nblk), kThreads, kTrsmSmem, s>>>(buf, info, k);
    if (maxTrail > 0)
      count_launch(), pchol_update_kernel<<<dim3((unsigned)maxTrail, nblk), kThreads, 0, s>>>(buf, info, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_ptri(const double *buf, const BlkInfo *info, int nblk, int amax, double *vec,
                        bool forward, cudaStream_t s) {
  if (nblk == 0 || amax == 0) return cudaSuccess;
  size_t sm = (size_t)amax * sizeof(double);
  if (forward)
    count_launch(), ptri_fwd_kernel<<<nblk, kThreads, sm, s>>>(buf, info, vec);
  else
    count_launch(), ptri_bwd_kernel<<<nblk, kThreads, sm, s>>>(buf, info, vec);
  return cudaGetLastError();
}

cudaError_t set_dense_smem_limits(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(pchol_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTrsmSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(ptri_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(ptri_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace ahlp
