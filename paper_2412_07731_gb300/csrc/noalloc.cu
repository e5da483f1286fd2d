// kkt_residual_noalloc: the relative Newton residual of a direction, computed
// without allocating any memory.
//
// kkt_solve measures the same quantity with residual vectors and reduction
// partials that live in the handle's device buffers.  Some callers cannot
// allocate device memory at the moment they need this number -- code running
// under a memory budget that forbids new allocations, callers whose allocator
// is owned by someone else, or code that must not trigger the implicit
// synchronisation cudaMalloc/cudaFree can cause.  This variant fuses the
// residual into the reduction and keeps its partial sums in one fixed,
// file-scope device array, so it needs nothing beyond the caller's vectors and
// the handle that already exists.
#include <algorithm>
#include <mutex>

#include "ahlp_internal.h"

namespace {

constexpr int kChunk = 16384;       // vector entries (or matrix rows) handled by one CTA
constexpr int kMaxParts = 4096;     // CTAs per residual block
constexpr long long kMaxLen = (long long)kChunk * kMaxParts;   // 67,108,864 entries
constexpr int kThreadsNA = 256;
constexpr int kMaxDevices = 64;

// Partial sums: for residual block b (0: dual rows, 1: primal rows,
// 2: complementarity rows) and CTA c, ||e||^2 at [(2b) * kMaxParts + c] and
// ||r||^2 at [(2b+1) * kMaxParts + c].  Every call writes every slot it later
// reads, so nothing has to be cleared between calls.  192 KB per device,
// held from the library's load until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[6 * kMaxParts];

__device__ double block_sum(double v, double *sh) {
  // fixed-order tree sum over the CTA
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

struct NAArgs {
  const int *A_rp, *A_ci, *AT_rp, *AT_ci;
  const double *A_v, *AT_v;
  const double *x, *z;
  const double *rd, *rp, *rc, *dx, *dy, *dz;
  long long n, m;
  double *scratch;
};

// grid (parts, 3): blockIdx.y selects the residual block
//   0: e_d = r_d - A'dy - dz   (rows of A', warp per row)
//   1: e_p = r_p - A dx        (rows of A, warp per row)
//   2: e_c = r_c - Z dx - X dz (elementwise)
__global__ void __launch_bounds__(kThreadsNA) residual_partials_kernel(NAArgs a) {
  __shared__ double sh[kThreadsNA];
  const int blk = blockIdx.y;
  const long long len = (blk == 1) ? a.m : a.n;
  const long long lo = (long long)blockIdx.x * kChunk;
  double e2 = 0.0, r2 = 0.0;
  if (lo < len) {
    const long long hi = min(lo + kChunk, len);
    if (blk == 2) {
      for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double e = a.rc[i] - a.z[i] * a.dx[i] - a.x[i] * a.dz[i];
        e2 += e * e;
        r2 += a.rc[i] * a.rc[i];
      }
    } else {
      const int *rp = blk == 0 ? a.AT_rp : a.A_rp;
      const int *ci = blk == 0 ? a.AT_ci : a.A_ci;
      const double *v = blk == 0 ? a.AT_v : a.A_v;
      const double *xv = blk == 0 ? a.dy : a.dx;
      const double *rhs = blk == 0 ? a.rd : a.rp;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
      for (long long row = lo + warp; row < hi; row += nwarp) {
        double s = 0.0;
        for (int k = rp[row] + lane; k < rp[row + 1]; k += 32) s = fma(v[k], xv[ci[k]], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
          const double e = rhs[row] - s - (blk == 0 ? a.dz[row] : 0.0);
          e2 += e * e;
          r2 += rhs[row] * rhs[row];
        }
      }
    }
  }
  const double se = block_sum(e2, sh);
  const double sr = block_sum(r2, sh);
  if (threadIdx.x == 0) {
    a.scratch[(2 * blk) * kMaxParts + blockIdx.x] = se;
    a.scratch[(2 * blk + 1) * kMaxParts + blockIdx.x] = sr;
  }
}

// one CTA: sum the partials of the three blocks in a fixed order
__global__ void __launch_bounds__(kThreadsNA) residual_final_kernel(const double *scratch,
                                                                    int parts_d, int parts_p,
                                                                    int parts_c, double *out) {
  __shared__ double sh[kThreadsNA];
  const int parts[3] = {parts_d, parts_p, parts_c};
  double e2 = 0.0, r2 = 0.0;
  for (int b = 0; b < 3; ++b) {
    double pe = 0.0, pr = 0.0;
    for (int c = threadIdx.x; c < parts[b]; c += blockDim.x) {
      pe += scratch[(2 * b) * kMaxParts + c];
      pr += scratch[(2 * b + 1) * kMaxParts + c];
    }
    e2 += block_sum(pe, sh);
    r2 += block_sum(pr, sh);
  }
  if (threadIdx.x == 0) out[0] = r2 > 0.0 ? sqrt(e2 / r2) : sqrt(e2);
}

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once
// per device (host code cannot take the address of a __device__ variable).
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int kkt_residual_noalloc(ahlp_problem *p, const double *r_d, const double *r_p,
                                    const double *r_c, const double *dx, const double *dy,
                                    const double *dz, double *rel_out) {
  using namespace ahlp;
  if (!p) return AHLP_ERR_INVALID_ARG;
  if (!r_d || !r_p || !r_c || !dx || !dy || !dz || !rel_out)
    return set_err(p, AHLP_ERR_INVALID_ARG, "kkt_residual_noalloc: NULL argument");
  if (!p->factored)
    return set_err(p, AHLP_ERR_INVALID_ARG,
                   "kkt_residual_noalloc: no factored point; call kkt_factor first");
  if (p->n > kMaxLen || p->m > kMaxLen)
    return set_err(p, AHLP_ERR_UNSUPPORTED,
                   "kkt_residual_noalloc: n_total and m_total must not exceed 67108864 "
                   "(the fixed scratch holds 4096 partial sums of 16384 entries per block)");
  // the scratch address is looked up for the current device, and the
  // kernels run on the handle's stream: both must be the handle's device, and
  // so must every vector
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device) {
    cudaGetLastError();
    return set_err(p, AHLP_ERR_INVALID_ARG,
                   "kkt_residual_noalloc: the current device is not the handle's device");
  }
  const void *ptrs[7] = {r_d, r_p, r_c, dx, dy, dz, rel_out};
  for (const void *q : ptrs) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
      cudaGetLastError();
      return set_err(p, AHLP_ERR_INVALID_ARG,
                     "kkt_residual_noalloc: every vector must be device memory");
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
        (at.type == cudaMemoryTypeDevice && at.device != p->device))
      return set_err(p, AHLP_ERR_INVALID_ARG,
                     "kkt_residual_noalloc: every vector must be device memory of the "
                     "handle's device");
  }
  double *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(p, AHLP_ERR_CUDA,
                   std::string("kkt_residual_noalloc: cudaGetSymbolAddress: ") +
                       cudaGetErrorString(e));
  }
  const int parts_d = (int)((p->n + kChunk - 1) / kChunk);
  const int parts_p = (int)((p->m + kChunk - 1) / kChunk);
  const int parts = std::max(std::max(parts_d, parts_p), 1);
  NAArgs a{p->A_rp, p->A_ci, p->AT_rp, p->AT_ci, p->A_v, p->AT_v, p->x, p->z,
           r_d, r_p, r_c, dx, dy, dz, p->n, p->m, scratch};
  count_launch(), residual_partials_kernel<<<dim3(parts, 3), kThreadsNA, 0, p->stream>>>(a);
  count_launch(), residual_final_kernel<<<1, kThreadsNA, 0, p->stream>>>(scratch, parts_d,
                                                                          parts_p, parts_d,
                                                                          rel_out);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_err(p, AHLP_ERR_CUDA,
                   std::string("kkt_residual_noalloc: launch: ") + cudaGetErrorString(e));
  return AHLP_OK;
}
