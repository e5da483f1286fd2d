// Block cyclic reduction of the link chain (the block-tridiagonal part T of
// the Schur complement, App. A), its border coupling Z = L^-1 E' and its
// solves.
//
// In a chain segment of n link pairs, position i is eliminated at level
// ctz(i + 1): level 0 takes every other pair, level 1 every other remaining
// one, and so on, so a segment of n pairs needs ceil(log2(n + 1)) levels and
// the positions of one level are independent of each other.  At level v the
// remaining neighbours of position j are a = j - 2^v and b = j + 2^v (when
// inside the segment).  Eliminating j (all FP64):
//   T_j  -= sum over the earlier levels v' of  GR_m' GR_m  (m = j - 2^v')
//                                          and GL_m' GL_m  (m = j + 2^v');
//   L_j L_j' = T_j;  Linv_j = L_j^-1;
//   GL_j = Linv_j C(j, a),  GR_j = Linv_j C(b, j)'   (couplings to a and b);
//   E_j' -= the same earlier-level terms applied to their Z, Z_j = Linv_j E_j'.
// The coupling C(b, a) that appears between j's neighbours is -GR_j' GL_j,
// built on demand one level later by whoever needs it (at level 0 the
// couplings are the assembled H blocks).  In elimination order the factor's
// off-diagonal blocks are GL_j' (row a) and GR_j' (row b), so
//   forward:  u_j = Linv_j (r_j - sum_m GR_m' u_m (m left of j) - sum_m GL_m' u_m (m right)),
//   backward: x_j = Linv_j' (u_j - GL_j x_a - GR_j x_b),
// level by level upwards and downwards.  Z' Z over all rows equals
// E T^-1 E' for any elimination order, so the border factor and its solves
// are unchanged.  The sequential depth is the number of levels, not the
// number of pairs.
#include <algorithm>

#include "ahlp_internal.h"

namespace ahlp {

namespace {

constexpr int kBcrThreads = 128;
constexpr int kBcrSmallL = 32;   // link blocks up to this size: one-warp Cholesky

struct BArgs {
  const int *l;                        // [N-1] link rows per pair
  const long long *td_off, *h_off, *link_off;
  const int *order;                    // pairs of the current level
  const int *info;                     // [N-1][4]: level, segment first pair, segment end, -
  int lmax;
  double *Td;                          // in: assembled T_j; out: L_j (lower)
  const double *Hd;                    // assembled H_j (l_{j+1} x l_j, ld l_{j+1})
  double *Linv;                        // L_j^-1 (layout of T_j)
  double *GL, *GR;                     // [N-1][lmax^2], ld l_j
  double *Et;                          // [B][nl]: E' in, Z out
  const double *Td_diag0;
  double tol;
  int *status;
  int B, nl;
};

__device__ __forceinline__ void pair_info(const BArgs &A, int j, int &lv, int &jb, int &je) {
  lv = A.info[4 * j];
  jb = A.info[4 * j + 1];
  je = A.info[4 * j + 2];
}

// dst (rows x cols, ld rows) -= G' H for G (k x rows, ld k), H (k x cols, ld k)
__device__ void sub_gtg(double *dst, int rows, int cols, const double *G, const double *H, int k,
                        int tid, int bd) {
  for (int i = tid; i < rows * cols; i += bd) {
    const int r = i % rows, c = i / rows;
    double a0 = 0.0, a1 = 0.0;
    int q = 0;
    for (; q + 1 < k; q += 2) {
      a0 = fma(G[q + (long long)r * k], H[q + (long long)c * k], a0);
      a1 = fma(G[q + 1 + (long long)r * k], H[q + 1 + (long long)c * k], a1);
    }
    if (q < k) a0 = fma(G[q + (long long)r * k], H[q + (long long)c * k], a0);
    dst[i] -= a0 + a1;
  }
}

// Factor of the pairs of one level: earlier-level updates of T_j, its
// Cholesky and inverse, and GL_j, GR_j.  One CTA per pair.
__global__ void __launch_bounds__(kBcrThreads) bcr_factor_kernel(BArgs A) {
  extern __shared__ double sm[];
  const int lm = A.lmax;
  double *T = sm, *Li = sm + lm * lm, *C = sm + 2 * lm * lm;
  __shared__ double Tinv[96];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int j = A.order[blockIdx.x];
  int lv, jb, je;
  pair_info(A, j, lv, jb, je);
  const int lj = A.l[j];
  double *Tg = A.Td + A.td_off[j];
  for (int i = tid; i < lj * lj; i += bd) T[i] = Tg[i];
  __syncthreads();
  // T_j -= GR_m' GR_m (m = j - 2^v') and GL_m' GL_m (m = j + 2^v'), v' < lv
  for (int v = 0; v < lv; ++v) {
    const int ml = j - (1 << v), mr = j + (1 << v);
    if (ml >= jb) sub_gtg(T, lj, lj, A.GR + (long long)ml * lm * lm,
                          A.GR + (long long)ml * lm * lm, A.l[ml], tid, bd);
    __syncthreads();
    if (mr < je) sub_gtg(T, lj, lj, A.GL + (long long)mr * lm * lm,
                         A.GL + (long long)mr * lm * lm, A.l[mr], tid, bd);
    __syncthreads();
  }
  // Cholesky of T_j (pivot safeguard against the link rows' full diagonal)
  if (lj <= kBcrSmallL) {
    if (tid < 32) {
      const int lane = tid;
      for (int c = 0; c < lj; ++c) {
        double piv = T[c + c * lj];
        const double orig = A.Td_diag0[A.link_off[j] + c];
        const double lim = A.tol * orig, floor_v = lim > 0.0 ? lim : 1.0;
        if (!(piv == piv)) {
          if (lane == 0 && atomicAdd(&A.status[0], 1) == 0) {
            A.status[2] = -1 - j;
            A.status[3] = c;
          }
          piv = floor_v;
        } else if (!(piv > lim) || !(piv > 0.0)) {
          if (lane == 0) atomicAdd(&A.status[1], 1);
          piv = floor_v;
        }
        const double inv = rsqrt(piv);
        __syncwarp();
        if (lane == c) {
          T[c + c * lj] = piv * inv;
          Tinv[c] = inv;
        } else if (lane > c && lane < lj) {
          T[lane + c * lj] *= inv;
        }
        __syncwarp();
        if (lane > c && lane < lj) {
          const double lr = T[lane + c * lj];
          for (int q = c + 1; q <= lane; ++q) T[lane + q * lj] = fma(-lr, T[q + c * lj], T[lane + q * lj]);
        }
        __syncwarp();
      }
    }
  } else {
    for (int c = 0; c < lj; ++c) {
      if (tid == 0) {
        double piv = T[c + c * lj];
        pivot_fix(piv, A.Td_diag0[A.link_off[j] + c], A.tol, A.status, -1 - j, c);
        const double lcc = sqrt(piv);
        T[c + c * lj] = lcc;
        Tinv[c] = 1.0 / lcc;
      }
      __syncthreads();
      const double inv = Tinv[c];
      for (int r = c + 1 + tid; r < lj; r += bd) T[r + c * lj] *= inv;
      __syncthreads();
      const int m = lj - c - 1;
      for (int i = tid; i < m * m; i += bd) {
        const int rr = i % m, ss = i / m;
        if (rr >= ss)
          T[(c + 1 + rr) + (c + 1 + ss) * lj] -= T[(c + 1 + rr) + c * lj] * T[(c + 1 + ss) + c * lj];
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // Linv_j: column c by forward substitution (one thread per column)
  for (int c = tid; c < lj; c += bd) {
    for (int r = 0; r < c; ++r) Li[r + c * lj] = 0.0;
    Li[c + c * lj] = Tinv[c];
    for (int r = c + 1; r < lj; ++r) {
      double acc = 0.0;
      for (int q = c; q < r; ++q) acc = fma(T[r + q * lj], Li[q + c * lj], acc);
      Li[r + c * lj] = -acc * Tinv[r];
    }
  }
  __syncthreads();
  for (int i = tid; i < lj * lj; i += bd) {
    const int r = i % lj, s = i / lj;
    Tg[i] = r >= s ? T[i] : 0.0;
    A.Linv[A.td_off[j] + i] = Li[i];
  }
  // GL_j = Linv_j C(j, a), a = j - 2^lv
  const int a = j - (1 << lv), b = j + (1 << lv);
  for (int side = 0; side < 2; ++side) {
    const int nb = side == 0 ? a : b;
    if (side == 0 ? nb < jb : nb >= je) continue;
    const int ln = A.l[nb];
    // C = the coupling as (l_j x l_nb): C(j, a) for the left side, C(b, j)'
    // for the right side
    if (lv == 0) {
      if (side == 0) {   // H_{j-1}: l_j x l_{j-1}, ld l_j
        const double *H = A.Hd + A.h_off[j - 1];
        for (int i = tid; i < lj * ln; i += bd) C[i] = H[i];
      } else {           // H_j: l_{j+1} x l_j, ld l_{j+1}; transposed
        const double *H = A.Hd + A.h_off[j];
        for (int i = tid; i < lj * ln; i += bd) {
          const int r = i % lj, c = i / lj;
          C[i] = H[c + (long long)r * ln];
        }
      }
    } else {
      // the coupling created by the position m between j and its neighbour:
      // C(j, a) = -GR_m' GL_m (m = j - 2^(lv-1)); C(b, j) = -GR_m' GL_m
      // (m = j + 2^(lv-1)), so C(b, j)' = -GL_m' GR_m
      const int m = side == 0 ? j - (1 << (lv - 1)) : j + (1 << (lv - 1));
      const int lmm = A.l[m];
      const double *G1 = (side == 0 ? A.GR : A.GL) + (long long)m * lm * lm;   // l_m x l_j
      const double *G2 = (side == 0 ? A.GL : A.GR) + (long long)m * lm * lm;   // l_m x l_nb
      for (int i = tid; i < lj * ln; i += bd) C[i] = 0.0;
      __syncthreads();
      sub_gtg(C, lj, ln, G1, G2, lmm, tid, bd);
    }
    __syncthreads();
    double *G = (side == 0 ? A.GL : A.GR) + (long long)j * lm * lm;
    for (int i = tid; i < lj * ln; i += bd) {
      const int r = i % lj, c = i / lj;
      double acc = 0.0;
      for (int q = 0; q <= r; ++q) acc = fma(Li[r + q * lj], C[q + c * lj], acc);
      G[i] = acc;
    }
    __syncthreads();
  }
}

// Z_j = Linv_j (E_j' - earlier-level terms), thread (row, column) over 32 x 4,
// blockIdx.y over groups of four border columns
__global__ void __launch_bounds__(kBcrThreads) bcr_z_kernel(BArgs A) {
  const int j = A.order[blockIdx.x];
  int lv, jb, je;
  pair_info(A, j, lv, jb, je);
  const int lj = A.l[j], lm = A.lmax;
  const int cl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.y * 4 + cl;
  __shared__ double e[4][96];
  const bool col = rb < A.B;
  double *ez = A.Et + (long long)(col ? rb : 0) * A.nl;
  for (int r = lane; r < lj; r += 32) {
    double v = col ? ez[A.link_off[j] + r] : 0.0;
    for (int w = 0; w < lv && col; ++w) {
      const int ml = j - (1 << w), mr = j + (1 << w);
      if (ml >= jb) {   // GR_ml' Z_ml
        const double *G = A.GR + (long long)ml * lm * lm;
        const int k = A.l[ml];
        const double *z = ez + A.link_off[ml];
        for (int q = 0; q < k; ++q) v = fma(-G[q + (long long)r * k], z[q], v);
      }
      if (mr < je) {    // GL_mr' Z_mr
        const double *G = A.GL + (long long)mr * lm * lm;
        const int k = A.l[mr];
        const double *z = ez + A.link_off[mr];
        for (int q = 0; q < k; ++q) v = fma(-G[q + (long long)r * k], z[q], v);
      }
    }
    e[cl][r] = v;
  }
  __syncwarp();
  if (!col) return;
  const double *Li = A.Linv + A.td_off[j];
  for (int r = lane; r < lj; r += 32) {
    double a0 = 0.0, a1 = 0.0;
    int q = 0;
    for (; q + 1 <= r; q += 2) {
      a0 = fma(Li[r + q * lj], e[cl][q], a0);
      a1 = fma(Li[r + (q + 1) * lj], e[cl][q + 1], a1);
    }
    if (q <= r) a0 = fma(Li[r + q * lj], e[cl][q], a0);
    ez[A.link_off[j] + r] = a0 + a1;
  }
}

// forward solve of one level, in place on the link part of u (one warp per
// row group, one CTA per pair): u_j = Linv_j (r_j - earlier-level terms)
__global__ void __launch_bounds__(kBcrThreads) bcr_fwd_kernel(BArgs A, double *u) {
  const int j = A.order[blockIdx.x];
  int lv, jb, je;
  pair_info(A, j, lv, jb, je);
  const int lj = A.l[j], lm = A.lmax;
  __shared__ double r[96];
  const int tid = threadIdx.x;
  for (int i = tid; i < lj; i += blockDim.x) {
    double v = u[A.link_off[j] + i];
    for (int w = 0; w < lv; ++w) {
      const int ml = j - (1 << w), mr = j + (1 << w);
      if (ml >= jb) {
        const double *G = A.GR + (long long)ml * lm * lm;
        const int k = A.l[ml];
        const double *z = u + A.link_off[ml];
        for (int q = 0; q < k; ++q) v = fma(-G[q + (long long)i * k], z[q], v);
      }
      if (mr < je) {
        const double *G = A.GL + (long long)mr * lm * lm;
        const int k = A.l[mr];
        const double *z = u + A.link_off[mr];
        for (int q = 0; q < k; ++q) v = fma(-G[q + (long long)i * k], z[q], v);
      }
    }
    r[i] = v;
  }
  __syncthreads();
  const double *Li = A.Linv + A.td_off[j];
  for (int i = tid; i < lj; i += blockDim.x) {
    double a0 = 0.0, a1 = 0.0;
    int q = 0;
    for (; q + 1 <= i; q += 2) {
      a0 = fma(Li[i + q * lj], r[q], a0);
      a1 = fma(Li[i + (q + 1) * lj], r[q + 1], a1);
    }
    if (q <= i) a0 = fma(Li[i + q * lj], r[q], a0);
    u[A.link_off[j] + i] = a0 + a1;
  }
}

// backward solve of one level: x_j = Linv_j' (u_j - GL_j x_a - GR_j x_b)
__global__ void __launch_bounds__(kBcrThreads) bcr_bwd_kernel(BArgs A, double *u) {
  const int j = A.order[blockIdx.x];
  int lv, jb, je;
  pair_info(A, j, lv, jb, je);
  const int lj = A.l[j], lm = A.lmax;
  __shared__ double r[96];
  const int tid = threadIdx.x;
  const int a = j - (1 << lv), b = j + (1 << lv);
  for (int i = tid; i < lj; i += blockDim.x) {
    double v = u[A.link_off[j] + i];
    if (a >= jb) {
      const double *G = A.GL + (long long)j * lm * lm;   // l_j x l_a
      const double *x = u + A.link_off[a];
      for (int q = 0; q < A.l[a]; ++q) v = fma(-G[i + (long long)q * lj], x[q], v);
    }
    if (b < je) {
      const double *G = A.GR + (long long)j * lm * lm;   // l_j x l_b
      const double *x = u + A.link_off[b];
      for (int q = 0; q < A.l[b]; ++q) v = fma(-G[i + (long long)q * lj], x[q], v);
    }
    r[i] = v;
  }
  __syncthreads();
  const double *Li = A.Linv + A.td_off[j];
  for (int i = tid; i < lj; i += blockDim.x) {
    double a0 = 0.0, a1 = 0.0;
    int q = i;
    for (; q + 1 < lj; q += 2) {
      a0 = fma(Li[q + i * lj], r[q], a0);
      a1 = fma(Li[q + 1 + i * lj], r[q + 1], a1);
    }
    if (q < lj) a0 = fma(Li[q + i * lj], r[q], a0);
    u[A.link_off[j] + i] = a0 + a1;
  }
}

BArgs bargs(ahlp_problem *p) {
  BArgs A{};
  A.l = p->l_d;
  A.td_off = p->td_off_d;
  A.h_off = p->h_off_d;
  A.link_off = p->link_off_d;
  A.order = p->bcr_order;
  A.info = p->bcr_info;
  A.lmax = p->bcr_lmax;
  A.Td = p->Td;
  A.Hd = p->Hd;
  A.Linv = p->Linv;
  A.GL = p->bcr_GL;
  A.GR = p->bcr_GR;
  A.Et = p->Et;
  A.Td_diag0 = p->Td_diag0;
  A.tol = p->fac_pivot_tol;
  A.status = p->status;
  A.B = p->B;
  A.nl = p->nl;
  return A;
}

}  // namespace

cudaError_t launch_bcr_factor(ahlp_problem *p) {
  cudaStream_t s = p->stream;
  const int nlev = (int)p->bcr_loff.size() - 1;
  const size_t smem = (size_t)3 * p->bcr_lmax * p->bcr_lmax * sizeof(double);
  for (int v = 0; v < nlev; ++v) {
    const int n = p->bcr_loff[v + 1] - p->bcr_loff[v];
    if (n == 0) continue;
    BArgs A = bargs(p);
    A.order = p->bcr_order + p->bcr_loff[v];
    count_launch(), bcr_factor_kernel<<<n, kBcrThreads, smem, s>>>(A);
    if (p->B > 0)
      count_launch(), bcr_z_kernel<<<dim3(n, (p->B + 3) / 4), kBcrThreads, 0, s>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_bcr_solve(ahlp_problem *p, double *u, bool forward) {
  cudaStream_t s = p->stream;
  const int nlev = (int)p->bcr_loff.size() - 1;
  for (int w = 0; w < nlev; ++w) {
    const int v = forward ? w : nlev - 1 - w;
    const int n = p->bcr_loff[v + 1] - p->bcr_loff[v];
    if (n == 0) continue;
    BArgs A = bargs(p);
    A.order = p->bcr_order + p->bcr_loff[v];
    if (forward)
      count_launch(), bcr_fwd_kernel<<<n, kBcrThreads, 0, s>>>(A, u);
    else
      count_launch(), bcr_bwd_kernel<<<n, kBcrThreads, 0, s>>>(A, u);
  }
  return cudaGetLastError();
}

cudaError_t set_bcr_smem_limits(int lmax) {
  return cudaFuncSetAttribute(bcr_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              3 * lmax * lmax * (int)sizeof(double));
}

}  // namespace ahlp
