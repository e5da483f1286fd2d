// Vector kernels of the IPM: sparse mat-vecs, deterministic reductions and
// elementwise updates.  All bandwidth-bound FP64.
#include "ahlp_internal.h"

namespace ahlp {

namespace {

constexpr int kRedBlocks = 304;   // 2 x 152 SMs, fixed so sums are reproducible
constexpr int kRedThreads = 256;

struct RedArgs {
  int op;
  const double *a, *b, *c, *d;
  double s1, s2;
  long long len;
};

__device__ __forceinline__ double red_identity(int op) {
  return (op == RED_MAXABS) ? 0.0 : ((op == RED_MINSTEP || op == RED_MIN) ? 1e300 : 0.0);
}

__device__ __forceinline__ double red_combine(int op, double u, double v) {
  switch (op) {
    case RED_MAXABS: return fmax(u, v);
    case RED_MINSTEP:
    case RED_MIN: return fmin(u, v);
    default: return u + v;
  }
}

__device__ __forceinline__ double red_elem(const RedArgs &r, long long i) {
  switch (r.op) {
    case RED_DOT: return r.a[i] * r.b[i];
    case RED_MAXABS: return fabs(r.a[i]);
    case RED_MINSTEP: {
      // largest step keeping a + t b >= 0
      double bi = r.b[i];
      return bi < 0.0 ? -r.a[i] / bi : 1e300;
    }
    case RED_MIN: return r.a[i];
    case RED_SUM: return r.a[i];
    case 5:  // (a + s1 b)(c + s2 d)
      return (r.a[i] + r.s1 * r.b[i]) * (r.c[i] + r.s2 * r.d[i]);
    default: return 0.0;
  }
}

__device__ double block_reduce(int op, double v, double *sh) {
  int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] = red_combine(op, sh[t], sh[t + s]);
    __syncthreads();
  }
  return sh[0];
}

__global__ void __launch_bounds__(kRedThreads) reduce_stage1(RedArgs r, double *part) {
  __shared__ double sh[kRedThreads];
  double acc = red_identity(r.op);
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < r.len; i += stride)
    acc = red_combine(r.op, acc, red_elem(r, i));
  double v = block_reduce(r.op, acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kRedThreads) reduce_stage2(int op, const double *part, int np,
                                                             double *out) {
  __shared__ double sh[kRedThreads];
  double acc = red_identity(op);
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc = red_combine(op, acc, part[i]);
  double v = block_reduce(op, acc, sh);
  if (threadIdx.x == 0) *out = v;
}

cudaError_t run_reduce(const RedArgs &r, double *part, double *out, cudaStream_t s) {
  count_launch(), reduce_stage1<<<kRedBlocks, kRedThreads, 0, s>>>(r, part);
  count_launch(), reduce_stage2<<<1, kRedThreads, 0, s>>>(r.op, part, kRedBlocks, out);
  return cudaGetLastError();
}

// y[r] = yadd[r] + alpha * sum_k v[k] x[ci[k]].  Short rows: one 8-lane group
// per row (four rows per warp); rows longer than kShortRow are skipped here
// and done by spmv_long_rows.  Each row is summed in a fixed order.
constexpr int kRowLanes = 8;
__global__ void spmv_short_rows(const int *__restrict__ rp, const int *__restrict__ ci,
                                const double *__restrict__ v, long long rows,
                                const double *__restrict__ x, double *y, double alpha,
                                const double *yadd) {
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kRowLanes;
  const int lane = threadIdx.x & (kRowLanes - 1);
  int k0 = 0, k1 = 0;
  if (row < rows) {
    k0 = rp[row];
    k1 = rp[row + 1];
    if (k1 - k0 > kShortRow) k1 = k0;   // long row: its own kernel
  }
  double s0 = 0.0, s1 = 0.0;
  int k = k0 + lane;
  for (; k + kRowLanes < k1; k += 2 * kRowLanes) {
    s0 = fma(v[k], x[ci[k]], s0);
    s1 = fma(v[k + kRowLanes], x[ci[k + kRowLanes]], s1);
  }
  if (k < k1) s0 = fma(v[k], x[ci[k]], s0);
  double s = s0 + s1;
#pragma unroll
  for (int o = kRowLanes / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, kRowLanes);
  if (lane == 0 && row < rows && rp[row + 1] - rp[row] <= kShortRow)
    y[row] = (yadd ? yadd[row] : 0.0) + alpha * s;
}

// one CTA per long row, fixed-order tree reduction
__global__ void __launch_bounds__(256) spmv_long_rows(const int *__restrict__ rp,
                                                      const int *__restrict__ ci,
                                                      const double *__restrict__ v,
                                                      const int *__restrict__ long_rows,
                                                      const double *__restrict__ x, double *y,
                                                      double alpha, const double *yadd) {
  __shared__ double part[8];
  const int row = long_rows[blockIdx.x];
  const int k0 = rp[row], k1 = rp[row + 1];
  double s0 = 0.0, s1 = 0.0;
  int k = k0 + threadIdx.x;
  for (; k + 256 < k1; k += 512) {
    s0 = fma(v[k], x[ci[k]], s0);
    s1 = fma(v[k + 256], x[ci[k + 256]], s1);
  }
  if (k < k1) s0 = fma(v[k], x[ci[k]], s0);
  double s = s0 + s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += part[w];
    y[row] = (yadd ? yadd[row] : 0.0) + alpha * t;
  }
}

__global__ void axpby_k(double *y, const double *x, double a, double b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void fill_k(double *y, double v, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = v;
}

__global__ void mul_k(double *y, const double *a, const double *b, double sc, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = sc * a[i] * b[i];
}

// r_c = sigma_mu - x z - dxa dza
__global__ void ipm_rc_k(double *rc, const double *x, const double *z, const double *dxa,
                         const double *dza, double smu, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rc[i] = smu - x[i] * z[i] - (dxa ? dxa[i] * dza[i] : 0.0);
}

__global__ void centrality_rc_k(double *rc2, const double *rc, const double *x, const double *dx,
                                double ap, const double *z, const double *dz, double ad,
                                double lo, double hi, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = (x[i] + ap * dx[i]) * (z[i] + ad * dz[i]);
  double t = v < lo ? lo - v : (v > hi ? hi - v : 0.0);
  if (t < -hi) t = -hi;
  rc2[i] = rc[i] + t;
}

__global__ void add_scalar_k(double *y, const double *x, double s, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] + s;
}

// part[i * gridDim.x + block] = partial of <V_i, w> for i < k (vectors of
// length len, stride ld); fixed assignment of entries to threads
__global__ void __launch_bounds__(kRedThreads) mdot_stage1(const double *V, long long ld, int k,
                                                           const double *w, long long len,
                                                           double *part) {
  __shared__ double sh[kRedThreads];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int i = 0; i < k; ++i) {
    const double *v = V + (long long)i * ld;
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride)
      acc = fma(v[e], w[e], acc);
    const double s = block_reduce(RED_DOT, acc, sh);
    if (threadIdx.x == 0) part[(long long)i * gridDim.x + blockIdx.x] = s;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRedThreads) mdot_stage2(const double *part, int np,
                                                           double *out) {
  __shared__ double sh[kRedThreads];
  const double *pp = part + (long long)blockIdx.x * np;
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += pp[i];
  const double v = block_reduce(RED_DOT, acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// w[e] += sum_i coef[i] V_i[e], fixed order over i
__global__ void maxpy_k(const double *V, long long ld, int k, const double *coef, double sc,
                        double *w, long long len) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  double acc = w[e];
  for (int i = 0; i < k; ++i) acc = fma(sc * coef[i], V[(long long)i * ld + e], acc);
  w[e] = acc;
}

// w *= 1 / sqrt(*nrm2) when *nrm2 > 0 (the norm stays on the device)
__global__ void scale_inv_norm_k(double *w, long long len, const double *nrm2) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double q = *nrm2;
  if (e >= len || !(q > 0.0)) return;
  w[e] = (1.0 / sqrt(q)) * w[e];
}

// J v tail: oz = z vx + x vz (Newton), oz = vx + x vz (transposed); ox += z vz (transposed)
__global__ void jmul_tail_k(double *ox, double *oz, const double *vx, const double *vz,
                            const double *x, const double *z, long long n, int adjoint) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (adjoint) {
    ox[i] += z[i] * vz[i];
    oz[i] = vx[i] + x[i] * vz[i];
  } else {
    oz[i] = z[i] * vx[i] + x[i] * vz[i];
  }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_mdot(ahlp_problem *p, const double *V, long long ld, int k, const double *w,
                        long long len, double *out) {
  if (k <= 0) return cudaSuccess;
  count_launch(), mdot_stage1<<<kRedBlocks, kRedThreads, 0, p->stream>>>(V, ld, k, w, len, p->mdot_part);
  count_launch(), mdot_stage2<<<k, kRedThreads, 0, p->stream>>>(p->mdot_part, kRedBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_maxpy(const double *V, long long ld, int k, const double *coef, double *w,
                         long long len, cudaStream_t s, double sign) {
  if (k <= 0 || len <= 0) return cudaSuccess;
  count_launch(), maxpy_k<<<blocks_for(len, 256), 256, 0, s>>>(V, ld, k, coef, sign, w, len);
  return cudaGetLastError();
}

cudaError_t launch_scale_inv_norm(double *w, long long len, const double *nrm2, cudaStream_t s) {
  if (len <= 0) return cudaSuccess;
  count_launch(), scale_inv_norm_k<<<blocks_for(len, 256), 256, 0, s>>>(w, len, nrm2);
  return cudaGetLastError();
}

// o = J v (adjoint: J' v) for v = [vx; vy; vz], o = [ox; oy; oz]
cudaError_t launch_jmul(ahlp_problem *p, const double *vx, const double *vy, const double *vz,
                        double *ox, double *oy, double *oz, bool adjoint) {
  cudaStream_t s = p->stream;
  cudaError_t e = launch_spmv(p->ATmat, vy, ox, 1.0, adjoint ? nullptr : vz, s);
  if (e != cudaSuccess) return e;
  e = launch_spmv(p->Amat, vx, oy, 1.0, nullptr, s);
  if (e != cudaSuccess) return e;
  if (p->n > 0)
    count_launch(), jmul_tail_k<<<blocks_for(p->n, 256), 256, 0, s>>>(ox, oz, vx, vz, p->x, p->z, p->n,
                                                       adjoint ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_add_scalar(double *y, const double *x, double s, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch(), add_scalar_k<<<blocks_for(n, 256), 256, 0, st>>>(y, x, s, n);
  return cudaGetLastError();
}

cudaError_t launch_reduce(ahlp_problem *p, int op, const double *a, const double *b,
                          long long len, double *out) {
  RedArgs r{op, a, b, nullptr, nullptr, 0.0, 0.0, len};
  return run_reduce(r, p->red_part, out, p->stream);
}

cudaError_t launch_step_dot(const double *x, const double *dx, double ap, const double *z,
                            const double *dz, double ad, long long n, double *part, double *out,
                            cudaStream_t s) {
  RedArgs r{5, x, dx, z, dz, ap, ad, n};
  return run_reduce(r, part, out, s);
}

cudaError_t launch_spmv(const SpMat &A, const double *x, double *y, double alpha,
                        const double *yadd, cudaStream_t s) {
  if (A.rows <= 0) return cudaSuccess;
  count_launch(), spmv_short_rows<<<blocks_for(A.rows * kRowLanes, 256), 256, 0, s>>>(
      A.rp, A.ci, A.v, A.rows, x, y, alpha, yadd);
  if (A.n_long > 0)
    count_launch(), spmv_long_rows<<<A.n_long, 256, 0, s>>>(A.rp, A.ci, A.v, A.long_rows, x, y,
                                                             alpha, yadd);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double *y, const double *x, double a, double b, long long n,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  count_launch(), axpby_k<<<blocks_for(n, 256), 256, 0, s>>>(y, x, a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(double *y, double v, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  count_launch(), fill_k<<<blocks_for(n, 256), 256, 0, s>>>(y, v, n);
  return cudaGetLastError();
}

cudaError_t launch_mul(double *y, const double *a, const double *b, double scale, long long n,
                       cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  count_launch(), mul_k<<<blocks_for(n, 256), 256, 0, s>>>(y, a, b, scale, n);
  return cudaGetLastError();
}

cudaError_t launch_ipm_rc(double *rc, const double *x, const double *z, const double *dxa,
                          const double *dza, double sigma_mu, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  count_launch(), ipm_rc_k<<<blocks_for(n, 256), 256, 0, s>>>(rc, x, z, dxa, dza, sigma_mu, n);
  return cudaGetLastError();
}

cudaError_t launch_centrality_rc(double *rc2, const double *rc, const double *x,
                                 const double *dx, double ap, const double *z, const double *dz,
                                 double ad, double lo, double hi, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  count_launch(), centrality_rc_k<<<blocks_for(n, 256), 256, 0, s>>>(rc2, rc, x, dx, ap, z, dz, ad,
                                                                     lo, hi, n);
  return cudaGetLastError();
}

}  // namespace ahlp
