// Schur complement of the block system (App. A) and the solve pipeline.
//
// Ordering of the Schur unknowns: [local link rows (pair 1..N-1) | x_0 | y_g].
// With local links the matrix is
//     S = [ T   E' ]     T block tridiagonal: T_j (l_j x l_j) on the diagonal,
//         [ E   SB ]     H_j (l_{j+1} x l_j) below it; E, SB the dense border.
// T is positive definite and SB quasi-definite (x_0 part negative, y_g part
// positive), so S = [L_T 0; Z' I] diag(I, SB - Z'Z) [L_T' Z; 0 I] with
// Z = L_T^-1 E' is factored by a block Cholesky along the link chain
// followed by a partial Cholesky of -(SB - Z'Z) over the x_0 pivots and a
// Cholesky of the remaining y_g Schur complement.
#include <algorithm>

#include "ahlp_internal.h"

namespace ahlp {

namespace {

struct SArgs {
  const double *aug;      // FP64 factors (prec kPrecFP64 / kPrecFF)
  const float *aug32;     // FP32 factors (prec == kPrecFP32)
  int prec;
  const BlkInfo *blk;
  const SchurBlk *sb;
  int N, n0, mg, B, nl;
  const long long *td_off, *h_off, *link_off;
  const int *l;
  double *Td, *Hd, *Et, *SB, *Td_diag0;
  const double *dscale;
  long long x0off;
  double delta, rho;
  const double *cdiag0;   // per-block corner diagonal before elimination
  double *sb_ref;         // reference diagonal of the border pivots
};

// entry (r, c) of block i's Schur contribution, local indices, symmetric
__device__ __forceinline__ double cget(const SArgs &A, const BlkInfo &bi, int m, int r, int c) {
  const int R = m + max(r, c), C = m + min(r, c);
  const long long idx = bi.base + (long long)C * bi.lda + R;
  // FP64 factors, or the FP64 copy of float-float ones
  return A.prec == kPrecFP32 ? (double)A.aug32[idx] : A.aug[idx];
}

// local Schur column of border index rb (linking variable rb < n0, else global
// row rb - n0) in block s, or -1 when the block does not touch it
__device__ __forceinline__ int border_local(const SchurBlk &s, int n0, int rb) {
  if (rb < n0) {
    const int t = rb - s.x0lo;
    return (t >= 0 && t < s.x0n) ? t : -1;
  }
  const int g = rb - n0 - s.glo;
  return (g >= 0 && g < s.gn) ? s.x0n + s.lprev + s.lnext + g : -1;
}

__global__ void assemble_T_kernel(SArgs A) {
  const int j = blockIdx.y;
  const int lj = A.l[j];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= lj * lj) return;
  const int r = idx % lj, s = idx / lj;
  const BlkInfo b0 = A.blk[j], b1 = A.blk[j + 1];
  const SchurBlk s0 = A.sb[j], s1 = A.sb[j + 1];
  double v = cget(A,b0, s0.m, s0.x0n + s0.lprev + r, s0.x0n + s0.lprev + s)   // block j, next
           + cget(A,b1, s1.m, s1.x0n + r, s1.x0n + s);                          // block j+1, prev
  if (r == s) {
    v += A.delta;
    // pivot reference: the link row's diagonal of the full normal matrix,
    // sum_i (U_i D_i U_i')_qq + delta, i.e. before the block eliminations
    // cancel most of it
    A.Td_diag0[A.link_off[j] + r] = A.cdiag0[b0.cdoff + s0.x0n + s0.lprev + r] +
                                    A.cdiag0[b1.cdoff + s1.x0n + r] + A.delta;
  }
  A.Td[A.td_off[j] + (long long)s * lj + r] = v;
}

__global__ void assemble_H_kernel(SArgs A) {
  const int j = blockIdx.y;   // H_j couples pair j+1 (rows) and pair j (cols) through block j+1
  const int lr = A.l[j + 1], lc = A.l[j];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= lr * lc) return;
  const int r = idx % lr, s = idx / lr;
  const BlkInfo b1 = A.blk[j + 1];
  const SchurBlk s1 = A.sb[j + 1];
  A.Hd[A.h_off[j] + (long long)s * lr + r] =
      cget(A,b1, s1.m, s1.x0n + s1.lprev + r, s1.x0n + s);
}

__global__ void assemble_E_kernel(SArgs A) {
  const int j = blockIdx.y;
  const int lj = A.l[j];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= lj * A.B) return;
  const int r = idx % lj, rb = idx / lj;
  const BlkInfo b0 = A.blk[j], b1 = A.blk[j + 1];
  const SchurBlk s0 = A.sb[j], s1 = A.sb[j + 1];
  const int t0 = border_local(s0, A.n0, rb), t1 = border_local(s1, A.n0, rb);
  const double v = (t0 >= 0 ? cget(A,b0, s0.m, t0, s0.x0n + s0.lprev + r) : 0.0) +
                   (t1 >= 0 ? cget(A,b1, s1.m, t1, s1.x0n + r) : 0.0);
  A.Et[(long long)rb * A.nl + A.link_off[j] + r] = v;
}

__global__ void assemble_SB_kernel(SArgs A) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= A.B * A.B) return;
  const int rb = idx % A.B, sb = idx / A.B;
  double v = 0.0;
  for (int i = 0; i < A.N; ++i) {   // fixed order over blocks
    const SchurBlk s = A.sb[i];
    const int tr = border_local(s, A.n0, rb), ts = border_local(s, A.n0, sb);
    if (tr >= 0 && ts >= 0) v += cget(A,A.blk[i], s.m, tr, ts);
  }
  if (rb == sb) v += (rb < A.n0) ? (-1.0 / A.dscale[A.x0off + rb] - A.rho) : A.delta;
  A.SB[(long long)sb * A.B + rb] = v;
  if (rb == sb && rb >= A.n0) {   // y_g pivot reference, as for the link rows
    double ref = A.delta;
    for (int i = 0; i < A.N; ++i) {
      const SchurBlk s = A.sb[i];
      const int t = border_local(s, A.n0, rb);
      if (t >= 0) ref += A.cdiag0[A.blk[i].cdoff + t];
    }
    A.sb_ref[rb] = ref;
  }
}

__global__ void scatter_add_kernel(double *dst, const long long *idx, const double *val,
                                   long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] += val[i];
}

// --------------------------------------------------------------------------
// link chain: block Cholesky of T, X_j = H_j L_j^-T, Z = L_T^-1 E'
// one CTA, sequential over the chain
// --------------------------------------------------------------------------
struct CArgs {
  int N, B, nl;
  const int *l;
  const long long *td_off, *h_off, *link_off;
  double *Td, *Hd, *Et;
  const double *Td_diag0;
  double tol;
  int *status;
  // explicit chain operators: Linv_j = L_j^-1 (layout of T_j),
  // Yf_j = L_j^-1 X_{j-1} (layout of H_{j-1}, ld l_j),
  // Yb_j = L_j^-T X_j'     (stored at H_j's offset, ld l_j)
  double *Linv, *Yf, *Yb;
  double *tmp;             // [nl] scratch of the chain solve
  const int *link_pair;    // [nl] pair of each link row
  // the chain falls apart at pairs without link rows: segment s covers pairs
  // [seg[2s], seg[2s+1]) and runs in CTA s (one per LP of a batch)
  const int *seg;
  int nseg;
};

// Forward substitution z <- L^-1 z for one right-hand side of at most 32 rows
// held in registers.  Axpy order: once z_q is final, every later row takes its
// update from it at once, so the dependent chain is two operations per row
// rather than the length of a dot product (FP64 latency dominates these
// small solves on this part).  L: column-major, ld lj; Tinv: its reciprocal
// pivots.
constexpr int kChainRegL = 32;

__device__ __forceinline__ void fwd_subst_regs(double (&z)[kChainRegL], int lj, const double *L,
                                               const double *Tinv) {
#pragma unroll
  for (int q = 0; q < kChainRegL; ++q) {
    if (q < lj) {
      const double zq = z[q] * Tinv[q];
      z[q] = zq;
#pragma unroll
      for (int r = q + 1; r < kChainRegL; ++r)
        if (r < lj) z[r] = fma(-L[r + q * lj], zq, z[r]);
    }
  }
}

__global__ void __launch_bounds__(512) chain_factor_kernel(CArgs A) {
  extern __shared__ double T[];   // lmax * lmax
  __shared__ double s_inv;
  __shared__ double Tinv[128];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int jb = A.seg[2 * blockIdx.x], je = A.seg[2 * blockIdx.x + 1];
  for (int j = jb; j < je; ++j) {
    const int lj = A.l[j];
    if (lj == 0) continue;
    const int lp = (j > jb) ? A.l[j - 1] : 0;
    const int ln = (j + 1 < je) ? A.l[j + 1] : 0;
    const bool small = lj <= kChainRegL;
    double *Tg = A.Td + A.td_off[j];
    for (int i = tid; i < lj * lj; i += bd) T[i] = Tg[i];
    __syncthreads();
    // T_j -= X_{j-1} X_{j-1}' (lower part), four partial sums per entry
    if (lp > 0) {
      const double *X = A.Hd + A.h_off[j - 1];   // l_j x l_{j-1}, ld l_j
      for (int i = tid; i < lj * lj; i += bd) {
        const int r = i % lj, s = i / lj;
        if (r < s) continue;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 4 <= lp; c += 4) {
          a0 = fma(X[r + (long long)c * lj], X[s + (long long)c * lj], a0);
          a1 = fma(X[r + (long long)(c + 1) * lj], X[s + (long long)(c + 1) * lj], a1);
          a2 = fma(X[r + (long long)(c + 2) * lj], X[s + (long long)(c + 2) * lj], a2);
          a3 = fma(X[r + (long long)(c + 3) * lj], X[s + (long long)(c + 3) * lj], a3);
        }
        for (; c < lp; ++c) a0 = fma(X[r + (long long)c * lj], X[s + (long long)c * lj], a0);
        T[i] -= (a0 + a1) + (a2 + a3);
      }
    }
    __syncthreads();
    if (small) {
      // Cholesky of T_j by warp 0, lane r owning row r; every lane takes the
      // pivot from shared memory, so no barrier or shuffle sits between the
      // pivot and its reciprocal square root
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
            for (int q = c + 1; q <= lane; ++q)
              T[lane + q * lj] = fma(-lr, T[q + c * lj], T[lane + q * lj]);
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
          s_inv = 1.0 / lcc;
        }
        __syncthreads();
        for (int r = c + 1 + tid; r < lj; r += bd) T[r + c * lj] *= s_inv;
        __syncthreads();
        const int m = lj - c - 1;
        for (int i = tid; i < m * m; i += bd) {
          const int rr = i % m, ss = i / m;
          if (rr >= ss) T[(c + 1 + rr) + (c + 1 + ss) * lj] -= T[(c + 1 + rr) + c * lj] * T[(c + 1 + ss) + c * lj];
        }
        __syncthreads();
      }
      // reciprocal pivots (FP64 divides are expensive on this part)
      for (int c = tid; c < lj; c += bd) Tinv[c] = 1.0 / T[c + c * lj];
    }
    __syncthreads();
    for (int i = tid; i < lj * lj; i += bd) {
      const int r = i % lj, s = i / lj;
      Tg[i] = (r >= s) ? T[i] : 0.0;
    }
    // E_j' -= X_{j-1} Z_{j-1}, one thread per entry, four partial sums
    if (lp > 0) {
      const double *X = A.Hd + A.h_off[j - 1];
      for (int i = tid; i < lj * A.B; i += bd) {
        const int r = i % lj, rb = i / lj;
        const double *zp = A.Et + (long long)rb * A.nl + A.link_off[j - 1];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 4 <= lp; c += 4) {
          a0 = fma(X[r + (long long)c * lj], zp[c], a0);
          a1 = fma(X[r + (long long)(c + 1) * lj], zp[c + 1], a1);
          a2 = fma(X[r + (long long)(c + 2) * lj], zp[c + 2], a2);
          a3 = fma(X[r + (long long)(c + 3) * lj], zp[c + 3], a3);
        }
        for (; c < lp; ++c) a0 = fma(X[r + (long long)c * lj], zp[c], a0);
        A.Et[(long long)rb * A.nl + A.link_off[j] + r] -= (a0 + a1) + (a2 + a3);
      }
      __syncthreads();
    }
    double *Li = A.Linv + A.td_off[j];
    double *H = A.Hd + A.h_off[j];   // l_{j+1} x l_j, ld l_{j+1}; becomes X_j = H_j L_j^-T
    if (small) {
      // three families of forward substitutions with L_j, all at once:
      // columns of Linv_j (e_c), rows of X_j (rows of H_j) and the columns
      // of Z_j (E_j' after the update above)
      const int nrhs = lj + ln + A.B;
      for (int w = tid; w < nrhs; w += bd) {
        double z[kChainRegL];
        double *dst;
        long long stride;
        if (w < lj) {
          dst = Li + (long long)w * lj;
          stride = 1;
        } else if (w < lj + ln) {
          dst = H + (w - lj);
          stride = ln;
        } else {
          dst = A.Et + (long long)(w - lj - ln) * A.nl + A.link_off[j];
          stride = 1;
        }
#pragma unroll
        for (int q = 0; q < kChainRegL; ++q)
          z[q] = q < lj ? (w < lj ? (q == w ? 1.0 : 0.0) : dst[q * stride]) : 0.0;
        fwd_subst_regs(z, lj, T, Tinv);
#pragma unroll
        for (int q = 0; q < kChainRegL; ++q)
          if (q < lj) dst[q * stride] = z[q];
      }
    } else {
      // Linv_j = L_j^-1, one thread per column
      for (int c = tid; c < lj; c += bd) {
        for (int r = 0; r < c; ++r) Li[r + c * lj] = 0.0;
        Li[c + c * lj] = Tinv[c];
        for (int r = c + 1; r < lj; ++r) {
          double acc = 0.0;
          for (int q = c; q < r; ++q) acc = fma(T[r + q * lj], Li[q + c * lj], acc);
          Li[r + c * lj] = -acc * Tinv[r];
        }
      }
      for (int rb = tid; rb < A.B; rb += bd) {
        double *zc = A.Et + (long long)rb * A.nl + A.link_off[j];
        for (int r = 0; r < lj; ++r) {
          double acc = zc[r];
          for (int c = 0; c < r; ++c) acc = fma(-T[r + c * lj], zc[c], acc);
          zc[r] = acc * Tinv[r];
        }
      }
      for (int r = tid; r < ln; r += bd) {
        for (int c = 0; c < lj; ++c) {
          double acc = H[r + (long long)c * ln];
          for (int q = 0; q < c; ++q) acc = fma(-H[r + (long long)q * ln], T[c + q * lj], acc);
          H[r + (long long)c * ln] = acc * Tinv[c];
        }
      }
    }
    __syncthreads();
    // chain operators for the solves: Yf_j = Linv_j X_{j-1}, Yb_j = Linv_j' X_j'
    if (lp > 0) {
      const double *X = A.Hd + A.h_off[j - 1];   // l_j x l_{j-1}
      double *Y = A.Yf + A.h_off[j - 1];
      for (int i = tid; i < lj * lp; i += bd) {
        const int r = i % lj, c = i / lj;
        double a0 = 0.0, a1 = 0.0;
        int q = 0;
        for (; q + 1 <= r; q += 2) {
          a0 = fma(Li[r + q * lj], X[q + (long long)c * lj], a0);
          a1 = fma(Li[r + (q + 1) * lj], X[q + 1 + (long long)c * lj], a1);
        }
        if (q <= r) a0 = fma(Li[r + q * lj], X[q + (long long)c * lj], a0);
        Y[r + (long long)c * lj] = a0 + a1;
      }
    }
    if (ln > 0) {
      const double *X = A.Hd + A.h_off[j];       // l_{j+1} x l_j
      double *Y = A.Yb + A.h_off[j];             // l_j x l_{j+1}
      for (int i = tid; i < lj * ln; i += bd) {
        const int r = i % lj, c = i / lj;
        double a0 = 0.0, a1 = 0.0;
        int q = r;
        for (; q + 1 < lj; q += 2) {
          a0 = fma(Li[q + r * lj], X[c + (long long)q * ln], a0);
          a1 = fma(Li[q + 1 + r * lj], X[c + (long long)(q + 1) * ln], a1);
        }
        if (q < lj) a0 = fma(Li[q + r * lj], X[c + (long long)q * ln], a0);
        Y[r + (long long)c * lj] = a0 + a1;
      }
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Link chain for link blocks of at most 32 rows, in three launches.  Only the
// block Cholesky of T and X_j = H_j L_j^-T are sequential along the chain;
// the solve operators (Linv_j, Yf_j, Yb_j) and Z = L_T^-1 E' hang off it.
// On one SM the FP64 pipe (about two FMA lanes per clock here) would carry
// all of that work; split this way the chain's CTA does the sequential part
// only, the operators take one CTA per pair, and Z one warp per border column.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) chain_critical_kernel(CArgs A) {
  extern __shared__ double T[];   // lmax * lmax
  __shared__ double Tinv[kChainRegL], Dg[kChainRegL];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int jb = A.seg[2 * blockIdx.x], je = A.seg[2 * blockIdx.x + 1];
  for (int j = jb; j < je; ++j) {
    const int lj = A.l[j];
    if (lj == 0) continue;
    const int lp = (j > jb) ? A.l[j - 1] : 0;
    const int ln = (j + 1 < je) ? A.l[j + 1] : 0;
    double *Tg = A.Td + A.td_off[j];
    for (int i = tid; i < lj * lj; i += bd) T[i] = Tg[i];
    if (tid < lj) Dg[tid] = A.Td_diag0[A.link_off[j] + tid];
    __syncthreads();
    if (lp > 0) {   // T_j -= X_{j-1} X_{j-1}', four partial sums per entry
      const double *X = A.Hd + A.h_off[j - 1];   // l_j x l_{j-1}, ld l_j
      for (int i = tid; i < lj * lj; i += bd) {
        const int r = i % lj, s = i / lj;
        if (r < s) continue;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 4 <= lp; c += 4) {
          a0 = fma(X[r + (long long)c * lj], X[s + (long long)c * lj], a0);
          a1 = fma(X[r + (long long)(c + 1) * lj], X[s + (long long)(c + 1) * lj], a1);
          a2 = fma(X[r + (long long)(c + 2) * lj], X[s + (long long)(c + 2) * lj], a2);
          a3 = fma(X[r + (long long)(c + 3) * lj], X[s + (long long)(c + 3) * lj], a3);
        }
        for (; c < lp; ++c) a0 = fma(X[r + (long long)c * lj], X[s + (long long)c * lj], a0);
        T[i] -= (a0 + a1) + (a2 + a3);
      }
    }
    __syncthreads();
    // Cholesky of T_j by warp 0, lane r owning row r; every lane reads the
    // pivot from shared memory, so no barrier or shuffle sits between the
    // pivot and its reciprocal square root
    if (tid < 32) {
      const int lane = tid;
      for (int c = 0; c < lj; ++c) {
        double piv = T[c + c * lj];
        const double lim = A.tol * Dg[c], floor_v = lim > 0.0 ? lim : 1.0;
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
          for (int q = c + 1; q <= lane; ++q)
            T[lane + q * lj] = fma(-lr, T[q + c * lj], T[lane + q * lj]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = tid; i < lj * lj; i += bd) {
      const int r = i % lj, s = i / lj;
      Tg[i] = (r >= s) ? T[i] : 0.0;
    }
    // X_j = H_j L_j^-T in place: row w of H_j is a forward substitution with L_j
    if (tid < ln) {
      double *H = A.Hd + A.h_off[j] + tid;   // l_{j+1} x l_j, ld l_{j+1}
      double z[kChainRegL];
#pragma unroll
      for (int q = 0; q < kChainRegL; ++q) z[q] = q < lj ? H[(long long)q * ln] : 0.0;
      fwd_subst_regs(z, lj, T, Tinv);
#pragma unroll
      for (int q = 0; q < kChainRegL; ++q)
        if (q < lj) H[(long long)q * ln] = z[q];
    }
    __syncthreads();
  }
}

// Linv_j = L_j^-1, Yf_j = Linv_j X_{j-1}, Yb_j = Linv_j' X_j': one CTA per pair
__global__ void __launch_bounds__(128) chain_ops_kernel(CArgs A) {
  extern __shared__ double Ls[];   // L_j then Linv_j, lmax * lmax each
  __shared__ double Tinv[kChainRegL];
  const int j = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  int jb = -1, je = -1;
  for (int s = 0; s < A.nseg; ++s)
    if (A.seg[2 * s] <= j && j < A.seg[2 * s + 1]) {
      jb = A.seg[2 * s];
      je = A.seg[2 * s + 1];
    }
  const int lj = A.l[j];
  if (jb < 0 || lj == 0) return;
  const int lp = (j > jb) ? A.l[j - 1] : 0;
  const int ln = (j + 1 < je) ? A.l[j + 1] : 0;
  double *L = Ls, *Li = Ls + lj * lj;
  const double *Tg = A.Td + A.td_off[j];
  for (int i = tid; i < lj * lj; i += bd) L[i] = Tg[i];
  __syncthreads();
  if (tid < lj) Tinv[tid] = 1.0 / L[tid + tid * lj];
  __syncthreads();
  double *Lg = A.Linv + A.td_off[j];
  if (tid < lj) {   // column tid of Linv_j
    double z[kChainRegL];
#pragma unroll
    for (int q = 0; q < kChainRegL; ++q) z[q] = q == tid ? 1.0 : 0.0;
    fwd_subst_regs(z, lj, L, Tinv);
#pragma unroll
    for (int q = 0; q < kChainRegL; ++q)
      if (q < lj) {
        Li[q + tid * lj] = z[q];
        Lg[q + tid * lj] = z[q];
      }
  }
  __syncthreads();
  if (lp > 0) {
    const double *X = A.Hd + A.h_off[j - 1];   // l_j x l_{j-1}
    double *Y = A.Yf + A.h_off[j - 1];
    for (int i = tid; i < lj * lp; i += bd) {
      const int r = i % lj, c = i / lj;
      double a0 = 0.0, a1 = 0.0;
      int q = 0;
      for (; q + 1 <= r; q += 2) {
        a0 = fma(Li[r + q * lj], X[q + (long long)c * lj], a0);
        a1 = fma(Li[r + (q + 1) * lj], X[q + 1 + (long long)c * lj], a1);
      }
      if (q <= r) a0 = fma(Li[r + q * lj], X[q + (long long)c * lj], a0);
      Y[r + (long long)c * lj] = a0 + a1;
    }
  }
  if (ln > 0) {
    const double *X = A.Hd + A.h_off[j];   // l_{j+1} x l_j
    double *Y = A.Yb + A.h_off[j];         // l_j x l_{j+1}
    for (int i = tid; i < lj * ln; i += bd) {
      const int r = i % lj, c = i / lj;
      double a0 = 0.0, a1 = 0.0;
      int q = r;
      for (; q + 1 < lj; q += 2) {
        a0 = fma(Li[q + r * lj], X[c + (long long)q * ln], a0);
        a1 = fma(Li[q + 1 + r * lj], X[c + (long long)(q + 1) * ln], a1);
      }
      if (q < lj) a0 = fma(Li[q + r * lj], X[c + (long long)q * ln], a0);
      Y[r + (long long)c * lj] = a0 + a1;
    }
  }
}

// Z = L_T^-1 E' along the chain, one warp per border column rb (lane r holds
// row r of the current link block): Z_j = Linv_j (E_j' - X_{j-1} Z_{j-1}).
// Segments outside the column's link rows [zlo, zhi) hold zeros and are skipped.
__global__ void __launch_bounds__(256) chain_z_kernel(CArgs A, const int *zlo, const int *zhi) {
  const int rb = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (rb >= A.B) return;   // whole warps leave together
  const int lo = zlo[rb], hi = zhi[rb];
  for (int s = 0; s < A.nseg; ++s) {
    const int jb = A.seg[2 * s], je = A.seg[2 * s + 1];
    if (A.link_off[je] <= lo || A.link_off[jb] >= hi) continue;
    double zprev = 0.0;
    int lp = 0;
    for (int j = jb; j < je; ++j) {
      const int lj = A.l[j];
      if (lj == 0) {
        lp = 0;
        continue;
      }
      double *zc = A.Et + (long long)rb * A.nl + A.link_off[j];
      double e = lane < lj ? zc[lane] : 0.0;
      if (lp > 0) {
        const double *X = A.Hd + A.h_off[j - 1];   // l_j x l_{j-1}, ld l_j
        double a0 = 0.0, a1 = 0.0;
        for (int c = 0; c < lp; c += 2) {
          const double z0 = __shfl_sync(0xffffffffu, zprev, c);
          const double z1 = __shfl_sync(0xffffffffu, zprev, c + 1 < 32 ? c + 1 : 31);
          if (lane < lj) {
            a0 = fma(X[lane + (long long)c * lj], z0, a0);
            if (c + 1 < lp) a1 = fma(X[lane + (long long)(c + 1) * lj], z1, a1);
          }
        }
        e -= a0 + a1;
      }
      const double *Li = A.Linv + A.td_off[j];
      double a0 = 0.0, a1 = 0.0;
      for (int q = 0; q < lj; q += 2) {
        const double e0 = __shfl_sync(0xffffffffu, e, q);
        const double e1 = __shfl_sync(0xffffffffu, e, q + 1 < 32 ? q + 1 : 31);
        if (lane < lj) {
          if (q <= lane) a0 = fma(Li[lane + q * lj], e0, a0);
          if (q + 1 <= lane && q + 1 < lj) a1 = fma(Li[lane + (q + 1) * lj], e1, a1);
        }
      }
      const double z = a0 + a1;
      if (lane < lj) zc[lane] = z;
      zprev = z;
      lp = lj;
    }
  }
}

// SB' = SB - Z'Z, written negated into the lower part of the border buffer.
// Column rb of Z can be nonzero only on the link rows [zlo[rb], zhi[rb]) (its
// LP's links in a batch), so each dot product runs over the overlap, in four
// independent partial sums.
__global__ void border_prep_kernel(const double *SB, const double *Z, int B, int nl, double *bd,
                                   int ld, double *bdiag0, const int *zlo, const int *zhi) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * B) return;
  const int rb = idx % B, sb = idx / B;
  if (rb < sb) return;
  double a0 = SB[(long long)sb * B + rb], a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const double *zr = Z + (long long)rb * nl, *zs = Z + (long long)sb * nl;
  const int q0 = max(zlo[rb], zlo[sb]), q1 = min(zhi[rb], zhi[sb]);
  int q = q0;
  for (; q + 4 <= q1; q += 4) {
    a0 -= zr[q] * zs[q];
    a1 -= zr[q + 1] * zs[q + 1];
    a2 -= zr[q + 2] * zs[q + 2];
    a3 -= zr[q + 3] * zs[q + 3];
  }
  for (; q < q1; ++q) a0 -= zr[q] * zs[q];
  const double acc = (a0 + a1) + (a2 + a3);
  bd[(long long)sb * ld + rb] = -acc;
  if (rb == sb) bdiag0[rb] = -acc;
}

// after eliminating the x_0 pivots the y_g corner holds -P; flip its sign
__global__ void negate_corner_kernel(double *bd, int ld, int n0, int mg, double *bdiag0,
                                     const double *sb_ref) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mg * mg) return;
  const int r = idx % mg, s = idx / mg;
  if (r < s) return;
  double *e = bd + (long long)(n0 + s) * ld + n0 + r;
  *e = -*e;
  if (r == s) {
    const double ref = sb_ref[n0 + r];
    bdiag0[n0 + r] = ref > 0.0 ? ref : *e;
  }
}

// --------------------------------------------------------------------------
// solve pipeline kernels
// --------------------------------------------------------------------------
// f = r_d - X^-1 r_c (forward) or g_x - Z X^-1 g_z (adjoint); g = D f on block columns
__global__ void prep_f_kernel(double *f, double *g, const double *rd, const double *rc,
                              const double *xinv, const double *z, const double *d,
                              const unsigned char *is_x0, long long n, int adjoint) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double fi = adjoint ? rd[i] - z[i] * rc[i] * xinv[i] : rd[i] - rc[i] * xinv[i];
  f[i] = fi;
  g[i] = is_x0[i] ? 0.0 : d[i] * fi;
}

__global__ void pack_rhs_kernel(const BlkInfo *blk, const SchurBlk *sb, const long long *yoff,
                                const double *rhat, double *vec) {
  const int i = blockIdx.y;
  const BlkInfo bi = blk[i];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= bi.a) return;
  vec[bi.voff + r] = (r < sb[i].m) ? rhat[yoff[i] + r] : 0.0;
}

struct RArgs {
  int N, n0, mg, B, nl;
  const BlkInfo *blk;
  const SchurBlk *sb;
  const int *link_pair;
  const double *vec, *rhat, *f;
  long long msum, x0off;
  double *svec;
};

// Schur right-hand side: base rows plus every block's -L21 w_i, fixed order.
// A link row touches two blocks (one thread each); a border row touches every
// block, so one warp takes it: lane i sums blocks i, i + 32, ... in order, then
// a fixed shuffle tree adds the lanes.  Launch: link_ctas CTAs of 256 threads
// for the link rows, then ceil(B / 8) CTAs for the border rows.
__global__ void schur_rhs_kernel(RArgs A, int link_ctas) {
  if ((int)blockIdx.x < link_ctas) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.nl) return;
    const int j = A.link_pair[q];
    const SchurBlk s0 = A.sb[j], s1 = A.sb[j + 1];
    const int r = q - s0.link_next_off;
    double v = A.rhat[A.msum + q];
    v += A.vec[A.blk[j].voff + s0.m + s0.x0n + s0.lprev + r];
    v += A.vec[A.blk[j + 1].voff + s1.m + s1.x0n + r];
    A.svec[q] = v;
    return;
  }
  const int lane = threadIdx.x & 31;
  const int rb = ((int)blockIdx.x - link_ctas) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (rb >= A.B) return;
  double v = 0.0;
  for (int i = lane; i < A.N; i += 32) {
    const SchurBlk s = A.sb[i];
    const int t = border_local(s, A.n0, rb);
    if (t >= 0) v += A.vec[A.blk[i].voff + s.m + t];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0)
    A.svec[A.nl + rb] =
        ((rb < A.n0) ? A.f[A.x0off + rb] : A.rhat[A.msum + A.nl + (rb - A.n0)]) + v;
}

// forward (dir = 0) or backward (dir = 1) solve with the block-bidiagonal L_T,
// using the operators precomputed by the factor:
//   forward  u_j = Linv_j r_j  - Yf_j u_{j-1}
//   backward s_j = Linv_j' v_j - Yb_j s_{j+1}
// The pre-multiplications are independent across pairs.  The recurrence is
// sequential; its operators lie contiguously in pair order, so they are
// staged into shared memory in batches of `stages` steps (one burst of
// loads per batch), and each step then costs one barrier.
constexpr int kChainMaxL = 96;         // link rows per pair handled by the chain kernels
constexpr int kChainMaxStages = 512;   // steps staged per batch, at most
constexpr size_t kChainSmem = 200 * 1024;

constexpr int kChainSolveThreads = 1024;
__global__ void __launch_bounds__(kChainSolveThreads) chain_solve_kernel(CArgs A, double *u,
                                                                         int dir, int stages,
                                                                         int lmax) {
  extern __shared__ double opbuf[];               // operators of one batch, then its tmp rows
  double *tbuf = opbuf + (size_t)stages * lmax * lmax;
  __shared__ double ubuf[2][kChainMaxL];          // solution of the previous pair
  __shared__ int meta[kChainMaxStages][4];        // l_j, l_other, operator offset, pair
  const int tid = threadIdx.x, bd = blockDim.x;
  const int jb = A.seg[2 * blockIdx.x], je = A.seg[2 * blockIdx.x + 1];
  const int npairs = je - jb;   // steps of this segment
  const long long q0 = A.link_off[jb], q1 = A.link_off[je - 1] + A.l[je - 1];
  for (long long q = q0 + tid; q < q1; q += bd) {
    const int j = A.link_pair[q];
    const int lj = A.l[j], r = q - (int)A.link_off[j];
    const double *Li = A.Linv + A.td_off[j];
    const double *uj = u + A.link_off[j];
    double acc = 0.0;
    if (dir == 0)
      for (int c = 0; c <= r; ++c) acc = fma(Li[r + c * lj], uj[c], acc);
    else
      for (int c = r; c < lj; ++c) acc = fma(Li[c + r * lj], uj[c], acc);
    A.tmp[q] = acc;
  }
  for (int s0 = 0; s0 < npairs; s0 += stages) {
    const int ns = min(stages, npairs - s0);
    // global range [g0, g1) holding the operators of steps s0 .. s0+ns-1
    long long g0 = 0, g1 = 0;
    if (dir == 0) {   // operators of pairs jb+1 .. : at h_off[j-1]
      const int a = jb + max(s0, 1), e = jb + s0 + ns - 1;
      if (e >= a) {
        g0 = A.h_off[a - 1];
        g1 = A.h_off[e - 1] + (long long)A.l[e] * A.l[e - 1];
      }
    } else {          // operators of pairs .. je-2: at h_off[j]
      const int jlo = je - s0 - ns, jtop = min(je - 1 - s0, je - 2);
      if (jtop >= jlo) {
        g0 = A.h_off[jlo];
        g1 = A.h_off[jtop] + (long long)A.l[jtop] * A.l[jtop + 1];
      }
    }
    const double *src = (dir == 0 ? A.Yf : A.Yb) + g0;
    __syncthreads();   // the previous batch is no longer read; tmp is complete
    const long long cnt = g1 - g0;
    for (long long i = tid; i < cnt; i += 8LL * bd) {   // eight loads in flight per thread
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = i + k * bd < cnt ? src[i + k * bd] : 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (i + k * bd < cnt) opbuf[i + k * bd] = v[k];
    }
    for (int t = tid; t < ns; t += bd) {
      const int j = dir == 0 ? jb + s0 + t : je - 1 - (s0 + t);
      const int jo = dir == 0 ? j - 1 : j + 1;
      const bool has = jo >= jb && jo < je;
      meta[t][0] = A.l[j];
      meta[t][1] = has ? A.l[jo] : 0;
      meta[t][2] = has ? (int)((dir == 0 ? A.h_off[j - 1] : A.h_off[j]) - g0) : 0;
      meta[t][3] = (int)A.link_off[j];
    }
    // the pre-multiplied rows of the batch's pairs (a contiguous range of tmp)
    {
      const int jf = dir == 0 ? jb + s0 : je - s0 - ns;   // first pair in memory order
      const int jl = dir == 0 ? jb + s0 + ns - 1 : je - 1 - s0;
      const long long t0 = A.link_off[jf], t1 = A.link_off[jl] + A.l[jl];
      for (long long i = tid; i < t1 - t0; i += bd) tbuf[i] = A.tmp[t0 + i];
      if (tid == 0) meta[kChainMaxStages - 1][3] = (int)t0;
    }
    __syncthreads();
    // the recurrence itself: one warp, lanes over the rows of a pair, so a
    // step needs only a warp barrier
    if (tid < 32) {
      const int tb0 = meta[kChainMaxStages - 1][3];
      for (int t = 0; t < ns; ++t) {
        const int b = (s0 + t) & 1;   // ubuf[b]: the previous pair's solution
        const int lj = meta[t][0], lo = meta[t][1], off = meta[t][3];
        const double *Yop = opbuf + meta[t][2];
        for (int r = tid; r < lj; r += 32) {
          // four independent partial sums keep the FP64 dependency chain short
          double a0 = tbuf[off - tb0 + r], a1 = 0.0, a2 = 0.0, a3 = 0.0;
          int c = 0;
          for (; c + 4 <= lo; c += 4) {
            a0 = fma(-Yop[r + (c + 0) * lj], ubuf[b][c + 0], a0);
            a1 = fma(-Yop[r + (c + 1) * lj], ubuf[b][c + 1], a1);
            a2 = fma(-Yop[r + (c + 2) * lj], ubuf[b][c + 2], a2);
            a3 = fma(-Yop[r + (c + 3) * lj], ubuf[b][c + 3], a3);
          }
          for (; c < lo; ++c) a0 = fma(-Yop[r + c * lj], ubuf[b][c], a0);
          const double acc = (a0 + a1) + (a2 + a3);
          u[off + r] = acc;
          ubuf[b ^ 1][r] = acc;
        }
        __syncwarp();
      }
    }
  }
}

// border rhs: sB -= Z' uT      (one warp per border row, lanes over link rows)
__global__ void border_rhs_kernel(const double *Z, int B, int nl, double *svec) {
  const int rb = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (rb >= B) return;
  const double *zc = Z + (long long)rb * nl;
  double acc = 0.0;
  for (int q = lane; q < nl; q += 32) acc = fma(zc[q], svec[q], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) svec[nl + rb] -= acc;
}

// uT -= Z sB      (one thread per link row)
__global__ void link_back_kernel(const double *Z, int B, int nl, double *svec) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nl) return;
  double acc = 0.0;
  for (int rb = 0; rb < B; ++rb) acc = fma(Z[(long long)rb * nl + q], svec[nl + rb], acc);
  svec[q] -= acc;
}

__global__ void scale_kernel(double *v, double a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] *= a;
}

__global__ void gather_schur_kernel(const BlkInfo *blk, const SchurBlk *sb, const int *kmap,
                                    const long long *kmap_off, const double *svec, double *vec) {
  const int i = blockIdx.y;
  const SchurBlk s = sb[i];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.k) return;
  vec[blk[i].voff + s.m + t] = svec[kmap[kmap_off[i] + t]];
}

__global__ void scatter_dy_kernel(const BlkInfo *blk, const SchurBlk *sb, const long long *yoff,
                                  const double *vec, double *dy) {
  const int i = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= sb[i].m) return;
  dy[yoff[i] + r] = vec[blk[i].voff + r];
}

__global__ void schur_dy_kernel(const double *svec, int nl, int n0, int mg, long long msum,
                                double *dy) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nl) dy[msum + q] = svec[q];
  else if (q < nl + mg) dy[msum + q] = svec[n0 + q];
}

// dx = (A'dy - f) / (1/d + rho[x0]);  dz = X^-1 (r_c - Z dx)  or  X^-1 (g_z - dx)
// dx = (A'dy - f) / (D^-1 + rho on the linking variables), dz from dx; w and
// xinv are those quotients' reciprocals, taken once per factor point
__global__ void finish_kernel(double *dx, double *dz, const double *aty, const double *f,
                              const double *w, const double *xinv, const double *z,
                              const double *rc, long long n, int adjoint) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dxi = (aty[i] - f[i]) * w[i];
  dx[i] = dxi;
  dz[i] = adjoint ? (rc[i] - dxi) * xinv[i] : (rc[i] - z[i] * dxi) * xinv[i];
}

// residual blocks of J d = r (forward) or J' d = r (adjoint)
__global__ void residual_tail_kernel(double *e_d, double *e_c, const double *dx,
                                     const double *dz, const double *rc, const double *x,
                                     const double *z, long long n, int adjoint) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (adjoint) {
    e_d[i] -= z[i] * dz[i];
    e_c[i] = rc[i] - dx[i] - x[i] * dz[i];
  } else {
    e_d[i] -= dz[i];
    e_c[i] = rc[i] - z[i] * dx[i] - x[i] * dz[i];
  }
}

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

SArgs sargs(ahlp_problem *p, double delta, double rho) {
  return SArgs{p->aug, p->aug32, p->fac_prec, p->blk, p->sblk, p->N, p->n0, p->mg, p->B, p->nl,
               p->td_off_d, p->h_off_d, p->link_off_d, p->l_d,
               p->Td, p->Hd, p->Et, p->SB, p->Td_diag0, p->dscale,
               p->xoff[p->N], delta, rho, p->cdiag0, p->sb_ref};
}

CArgs cargs(ahlp_problem *p) {
  return CArgs{p->N, p->B, p->nl, p->l_d, p->td_off_d, p->h_off_d, p->link_off_d,
               p->Td, p->Hd, p->Et, p->Td_diag0, p->fac_pivot_tol, p->status,
               p->Linv, p->Yf, p->Yb, p->chain_tmp, p->link_pair_d, p->chain_seg, p->nchain_seg};
}

}  // namespace

cudaError_t launch_schur_assemble(ahlp_problem *p, double delta, double rho) {
  cudaStream_t s = p->stream;
  SArgs A = sargs(p, delta, rho);
  int lmax = 0;
  for (int j = 0; j + 1 < p->N; ++j) lmax = std::max(lmax, (int)(p->link_off[j + 1] - p->link_off[j]));
  if (p->N > 1 && lmax > 0) {
    count_launch(), assemble_T_kernel<<<dim3(nb((long long)lmax * lmax, 256), p->N - 1), 256, 0, s>>>(A);
    if (p->N > 2)
      count_launch(), assemble_H_kernel<<<dim3(nb((long long)lmax * lmax, 256), p->N - 2), 256, 0, s>>>(A);
    if (p->B > 0)
      count_launch(), assemble_E_kernel<<<dim3(nb((long long)lmax * p->B, 256), p->N - 1), 256, 0, s>>>(A);
  }
  if (p->B > 0) count_launch(), assemble_SB_kernel<<<nb((long long)p->B * p->B, 256), 256, 0, s>>>(A);
  if (p->nf0 > 0) count_launch(), scatter_add_kernel<<<nb(p->nf0, 256), 256, 0, s>>>(p->Et, p->f0_idx, p->f0_val, p->nf0);
  if (p->nfg0 > 0)
    count_launch(), scatter_add_kernel<<<nb(p->nfg0, 256), 256, 0, s>>>(p->SB, p->fg0_idx, p->fg0_val, p->nfg0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // keep the assembled matrix for diagnostics
  if (p->td_elems) cudaMemcpyAsync(p->Td_asm, p->Td, p->td_elems * 8, cudaMemcpyDeviceToDevice, s);
  if (p->h_elems) cudaMemcpyAsync(p->Hd_asm, p->Hd, p->h_elems * 8, cudaMemcpyDeviceToDevice, s);
  if ((long long)p->nl * p->B != 0)
    cudaMemcpyAsync(p->Et_asm, p->Et, (size_t)p->nl * p->B * 8, cudaMemcpyDeviceToDevice, s);
  if (p->B) cudaMemcpyAsync(p->SB_asm, p->SB, (size_t)p->B * p->B * 8, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

cudaError_t launch_schur_factor(ahlp_problem *p) {
  cudaStream_t s = p->stream;
  int lmax = 0;
  for (int j = 0; j + 1 < p->N; ++j) lmax = std::max(lmax, (int)(p->link_off[j + 1] - p->link_off[j]));
  // the solves must use the factor that was built: remember which one
  p->fac_bcr = p->opt.schur_chain == 0 && p->bcr_order != nullptr;
  if (p->N > 1 && lmax > 0) {
    if (p->fac_bcr) {
      cudaError_t e = launch_bcr_factor(p);
      if (e != cudaSuccess) return e;
    } else if (p->nchain_seg > 0 && lmax <= kChainRegL) {
      const CArgs A = cargs(p);
      count_launch(), chain_critical_kernel<<<p->nchain_seg, 256, (size_t)lmax * lmax * 8, s>>>(A);
      count_launch(), chain_ops_kernel<<<p->N - 1, 128, (size_t)2 * lmax * lmax * 8, s>>>(A);
      if (p->B > 0)
        count_launch(), chain_z_kernel<<<(unsigned)((p->B + 7) / 8), 256, 0, s>>>(A, p->zlo,
                                                                                   p->zhi);
    } else if (p->nchain_seg > 0) {
      count_launch(), chain_factor_kernel<<<p->nchain_seg, 512, (size_t)lmax * lmax * 8, s>>>(
          cargs(p));
    }
  }
  if (p->B > 0) {
    count_launch(), border_prep_kernel<<<nb((long long)p->B * p->B, 256), 256, 0, s>>>(
        p->SB, p->Et, p->B, p->nl, p->border, p->Bld, p->border_diag0, p->zlo, p->zhi);
    std::vector<BlkInfo> hx(1, p->h_bx);
    if (p->n0 > 0) {
      cudaError_t e = launch_pchol(p->border, p->bx_info, hx, p->border_diag0, p->fac_pivot_tol,
                                   p->status, s);
      if (e != cudaSuccess) return e;
    }
    if (p->mg > 0) {
      count_launch(), negate_corner_kernel<<<nb((long long)p->mg * p->mg, 256), 256, 0, s>>>(
          p->border, p->Bld, p->n0, p->mg, p->border_diag0, p->sb_ref);
      std::vector<BlkInfo> hp(1, p->h_bp);
      cudaError_t e = launch_pchol(p->border, p->bp_info, hp, p->border_diag0, p->fac_pivot_tol,
                                   p->status, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_solve(ahlp_problem *p, const double *r_d, const double *r_p,
                         const double *r_c, double *dx, double *dy, double *dz, bool adjoint) {
  cudaStream_t s = p->stream;
  const long long n = p->n;
  cudaError_t e;
  count_launch(), prep_f_kernel<<<nb(n, 256), 256, 0, s>>>(p->f, p->g, r_d, r_c, p->xinv, p->z, p->dscale, p->is_x0,
                                          n, adjoint ? 1 : 0);
  e = launch_spmv(p->Amat, p->g, p->rhat, 1.0, r_p, s);
  if (e != cudaSuccess) return e;
  count_launch(), pack_rhs_kernel<<<dim3(nb(p->amax, 256), p->N), 256, 0, s>>>(p->blk, p->sblk, p->yoff_d,
                                                                p->rhat, p->vec);
  e = launch_trsv(p, true);
  if (e != cudaSuccess) return e;
  if (p->nS > 0) {
    int lmax = 0;
    for (int j = 0; j + 1 < p->N; ++j)
      lmax = std::max(lmax, (int)(p->link_off[j + 1] - p->link_off[j]));
    RArgs R{p->N, p->n0, p->mg, p->B, p->nl, p->blk, p->sblk,
            p->link_pair_d, p->vec, p->rhat, p->f, p->msum,
            p->xoff[p->N], p->svec};
    {
      const int link_ctas = (int)nb(p->nl, 256);
      count_launch(), schur_rhs_kernel<<<link_ctas + (int)nb(p->B, 8), 256, 0, s>>>(R, link_ctas);
    }
    CArgs C = cargs(p);
    // one stage = one operator (<= lmax^2) plus one pair's rows (<= lmax); the
    // last meta slot is reserved
    const int stages = (int)std::max<long long>(
        1, std::min<long long>(kChainMaxStages - 1,
                               (long long)kChainSmem /
                                   std::max(1LL, 8LL * ((long long)lmax * lmax + lmax))));
    const size_t csm = (size_t)stages * ((size_t)lmax * lmax + lmax) * sizeof(double);
    if (p->nl > 0 && lmax > 0 && p->nchain_seg > 0) {
      if (p->fac_bcr) {
        e = launch_bcr_solve(p, p->svec, true);
        if (e != cudaSuccess) return e;
      } else {
        count_launch(), chain_solve_kernel<<<p->nchain_seg, kChainSolveThreads, csm, s>>>(
            C, p->svec, 0, stages, lmax);
      }
    }
    if (p->B > 0) {
      if (p->nl > 0) count_launch(), border_rhs_kernel<<<nb((long long)p->B * 32, 256), 256, 0, s>>>(p->Et, p->B, p->nl, p->svec);
      double *sb = p->svec + p->nl;
      if (p->n0 > 0) {
        e = launch_ptri(p->border, p->bx_info, 1, p->B, sb, true, s);
        if (e != cudaSuccess) return e;
        count_launch(), scale_kernel<<<nb(p->n0, 256), 256, 0, s>>>(sb, -1.0, p->n0);
      }
      if (p->mg > 0) {
        e = launch_ptri(p->border, p->bp_info, 1, p->B, sb, true, s);
        if (e != cudaSuccess) return e;
        e = launch_ptri(p->border, p->bp_info, 1, p->B, sb, false, s);
        if (e != cudaSuccess) return e;
      }
      if (p->n0 > 0) {
        e = launch_ptri(p->border, p->bx_info, 1, p->B, sb, false, s);
        if (e != cudaSuccess) return e;
      }
      if (p->nl > 0) count_launch(), link_back_kernel<<<nb(p->nl, 128), 128, 0, s>>>(p->Et, p->B, p->nl, p->svec);
    }
    if (p->nl > 0 && lmax > 0 && p->nchain_seg > 0) {
      if (p->fac_bcr) {
        e = launch_bcr_solve(p, p->svec, false);
        if (e != cudaSuccess) return e;
      } else {
        count_launch(), chain_solve_kernel<<<p->nchain_seg, kChainSolveThreads, csm, s>>>(
            C, p->svec, 1, stages, lmax);
      }
    }
    int kmax = 0;
    for (int k : p->ki) kmax = std::max(kmax, k);
    if (kmax > 0)
      count_launch(), gather_schur_kernel<<<dim3(nb(kmax, 256), p->N), 256, 0, s>>>(p->blk, p->sblk, p->kmap,
                                                                  p->kmap_off_d, p->svec, p->vec);
  }
  e = launch_trsv(p, false);
  if (e != cudaSuccess) return e;
  int mmax = 0;
  for (int v : p->mi) mmax = std::max(mmax, v);
  count_launch(), scatter_dy_kernel<<<dim3(nb(mmax, 256), p->N), 256, 0, s>>>(
      p->blk, p->sblk, p->yoff_d, p->vec, dy);
  if (p->nl + p->mg > 0)
    count_launch(), schur_dy_kernel<<<nb(p->nl + p->mg, 256), 256, 0, s>>>(p->svec, p->nl, p->n0, p->mg, p->msum,
                                                          dy);
  // dx, dz
  e = launch_spmv(p->ATmat, dy, p->g, 1.0, nullptr, s);
  if (e != cudaSuccess) return e;
  count_launch(), finish_kernel<<<nb(n, 256), 256, 0, s>>>(dx, dz, p->g, p->f, p->wfin, p->xinv,
                                                            p->z, r_c, n, adjoint ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_residual(ahlp_problem *p, const double *r_d, const double *r_p,
                            const double *r_c, const double *dx, const double *dy,
                            const double *dz, double *e_d, double *e_p, double *e_c,
                            bool adjoint) {
  cudaStream_t s = p->stream;
  cudaError_t e = launch_spmv(p->ATmat, dy, e_d, -1.0, r_d, s);
  if (e != cudaSuccess) return e;
  e = launch_spmv(p->Amat, dx, e_p, -1.0, r_p, s);
  if (e != cudaSuccess) return e;
  count_launch(), residual_tail_kernel<<<nb(p->n, 256), 256, 0, s>>>(e_d, e_c, dx, dz, r_c, p->x, p->z, p->n,
                                                    adjoint ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t set_schur_smem_limits(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(chain_factor_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(chain_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kChainSmem);
}

}  // namespace ahlp
