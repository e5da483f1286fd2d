// Host runtime of the C ABI: validation, symbolic analysis, device memory,
// and the kkt_factor / kkt_solve / kkt_adjoint_solve entry points.
#include <algorithm>
#include <deque>
#include <exception>
#include <mutex>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <tuple>
#include <utility>
#include <vector>

#include "ahlp_internal.h"

using namespace ahlp;

namespace ahlp {
cudaError_t set_dense_smem_limits(int bytes);
cudaError_t set_schur_smem_limits(int bytes);
cudaError_t set_bcr_smem_limits(int lmax);
}

static std::string g_create_err;

namespace {

// ---------------------------------------------------------------------------
// canonical sparse matrices on the host
// ---------------------------------------------------------------------------
struct Csc {
  int m = 0, n = 0;
  std::vector<int> cp, ri;
  std::vector<double> v;
  long long nnz() const { return (long long)ri.size(); }
};

[[noreturn]] void fail(int code, const std::string &msg) { throw Fail{code, msg}; }

bool finite(double v) { return std::isfinite(v); }

// Validate and canonicalise (sort rows, sum duplicates).  in == NULL means the
// zero matrix of the expected shape.
Csc canon(const ahlp_csc *in, int m, int n, const std::string &what) {
  Csc out;
  out.m = m;
  out.n = n;
  out.cp.assign(n + 1, 0);
  if (in == nullptr) return out;
  if (in->m != m || in->n != n)
    fail(AHLP_ERR_DIM_MISMATCH, what + ": shape " + std::to_string(in->m) + "x" +
                                    std::to_string(in->n) + ", expected " + std::to_string(m) +
                                    "x" + std::to_string(n));
  if (n == 0) return out;
  if (!in->colptr) fail(AHLP_ERR_INVALID_ARG, what + ": colptr is NULL");
  if (in->colptr[0] != 0) fail(AHLP_ERR_INVALID_ARG, what + ": colptr[0] != 0");
  for (int j = 0; j < n; ++j)
    if (in->colptr[j + 1] < in->colptr[j])
      fail(AHLP_ERR_INVALID_ARG, what + ": colptr not monotone");
  const int nnz = in->colptr[n];
  if (nnz > 0 && (!in->rowidx || !in->val))
    fail(AHLP_ERR_INVALID_ARG, what + ": rowidx/val NULL");
  std::vector<std::pair<int, double>> col;
  for (int j = 0; j < n; ++j) {
    col.clear();
    for (int k = in->colptr[j]; k < in->colptr[j + 1]; ++k) {
      const int r = in->rowidx[k];
      const double v = in->val[k];
      if (r < 0 || r >= m) fail(AHLP_ERR_INVALID_ARG, what + ": row index out of range");
      if (!finite(v)) fail(AHLP_ERR_INVALID_ARG, what + ": non-finite value");
      col.push_back({r, v});
    }
    std::sort(col.begin(), col.end(),
              [](const std::pair<int, double> &a, const std::pair<int, double> &b) {
                return a.first < b.first;
              });
    for (size_t k = 0; k < col.size(); ++k) {
      if (!out.ri.empty() && (int)out.ri.size() > out.cp[j] && out.ri.back() == col[k].first)
        out.v.back() += col[k].second;
      else {
        out.ri.push_back(col[k].first);
        out.v.push_back(col[k].second);
      }
    }
    out.cp[j + 1] = (int)out.ri.size();
  }
  return out;
}

std::vector<double> vec_in(const double *p, long long n, const std::string &what) {
  std::vector<double> v((size_t)n);
  if (n == 0) return v;
  if (!p) fail(AHLP_ERR_INVALID_ARG, what + " is NULL");
  for (long long i = 0; i < n; ++i) {
    if (!finite(p[i])) fail(AHLP_ERR_INVALID_ARG, what + ": non-finite entry");
    v[(size_t)i] = p[i];
  }
  return v;
}

void check_bounds(const double *lb, const double *ub, int n, const std::string &what) {
  for (int j = 0; j < n; ++j) {
    if (lb && lb[j] != 0.0)
      fail(AHLP_ERR_UNSUPPORTED, what + ": only lower bounds of 0 are supported");
    if (ub && !(std::isinf(ub[j]) && ub[j] > 0))
      fail(AHLP_ERR_UNSUPPORTED, what + ": finite upper bounds are not supported");
  }
}

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

template <class T>
T *dalloc(ahlp_problem *p, long long count) {
  if (count <= 0) count = 1;
  void *ptr = nullptr;
  size_t bytes = (size_t)count * sizeof(T);
  cudaError_t e = cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? AHLP_ERR_OOM : AHLP_ERR_CUDA,
         std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  p->allocs.push_back({ptr, bytes});
  return reinterpret_cast<T *>(ptr);
}

// the concatenation of member `f` of every part, uploaded part by part
template <class P, class T>
T *dupload_parts(ahlp_problem *p, const std::vector<P> &parts, std::vector<T> P::*f) {
  long long total = 0;
  for (const P &q : parts) total += (long long)(q.*f).size();
  T *d = dalloc<T>(p, total);
  long long off = 0;
  for (const P &q : parts) {
    const std::vector<T> &h = q.*f;
    if (!h.empty()) {
      cudaError_t e = cudaMemcpy(d + off, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
      p->bytes_h2d += (long long)(h.size() * sizeof(T));
      if (e != cudaSuccess) fail(AHLP_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    off += (long long)h.size();
  }
  return d;
}

template <class T>
T *dupload(ahlp_problem *p, const std::vector<T> &h) {
  T *d = dalloc<T>(p, (long long)h.size());
  if (!h.empty()) {
    cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    p->bytes_h2d += (long long)(h.size() * sizeof(T));
    if (e != cudaSuccess) fail(AHLP_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  return d;
}

// ---------------------------------------------------------------------------
// formation pattern of one block (the block step of Alg. 2 in normal-equation form):
// entries of M_i, G_i' and C_i as sums coef * d[j] (j = -1: constant 1)
// ---------------------------------------------------------------------------
struct Con {
  long long key;   // tile id * NB*NB + ct*NB + rt
  int didx;
  double coef;
};

struct Pattern {
  std::vector<unsigned char> nz;     // T x T (row I, column J <= I): the tile has entries
  std::vector<FormTile> tiles;
  std::vector<long long> tile_ent;   // entry begin per tile (absolute)
  std::vector<int> ent_pos;
  std::vector<long long> ent_cb;     // contribution begin per entry (absolute)
  std::vector<int> con_idx;
  std::vector<double> con_coef;
};

// fn(i) for i in [0, n) on up to 16 host threads (work taken in index order).
// An exception thrown by fn stops no other index; the first one caught is
// rethrown on the calling thread once every thread has joined.
template <class F>
void parallel_for(int n, F fn) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nthr = (int)std::min<long long>(n, std::min(16u, hw));
  std::atomic<int> next{0};
  std::exception_ptr err;
  std::mutex mu;
  auto worker = [&]() {
    for (int i = next++; i < n; i = next++) {
      try {
        fn(i);
      } catch (...) {
        std::lock_guard<std::mutex> g(mu);
        if (!err) err = std::current_exception();
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nthr; ++t) pool.emplace_back(worker);
  worker();
  for (auto &th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

struct URow {   // one link / global row restricted to the block's columns
  std::vector<int> j;
  std::vector<double> u;
};

void build_block_pattern(int blk, const Csc &A, const Csc &W, const std::vector<URow> &urows,
                         int x0lo, int x0n, int m, int k, long long xoff, Pattern &P) {
  const int a = m + k;
  const int T = (a + NB - 1) / NB;
  auto tile_id = [T](long long It, long long Jt) { return Jt * T - Jt * (Jt - 1) / 2 + (It - Jt); };
  std::vector<Con> cons;
  {   // exact count of the contributions below, so the buffer is allocated once
    long long nc = m + (long long)(W.cp[x0lo + x0n] - W.cp[x0lo]);
    std::vector<int> uc(A.n, 0);
    for (const URow &u : urows)
      for (int j : u.j) {
        nc += A.cp[j + 1] - A.cp[j];
        ++uc[j];
      }
    for (int j = 0; j < A.n; ++j) {
      const long long d = A.cp[j + 1] - A.cp[j];
      nc += d * (d + 1) / 2 + (long long)uc[j] * (uc[j] + 1) / 2;
    }
    cons.reserve((size_t)nc);
  }
  auto add = [&](int R, int C, int didx, double coef) {
    if (R < C) std::swap(R, C);
    const long long key = tile_id(R / NB, C / NB) * (long long)(NB * NB) + (long long)(C % NB) * NB +
                          (R % NB);
    cons.push_back({key, didx, coef});
  };
  // M_i = A_i D_i A_i'
  for (int j = 0; j < A.n; ++j)
    for (int p = A.cp[j]; p < A.cp[j + 1]; ++p)
      for (int q = A.cp[j]; q <= p; ++q)
        add(A.ri[p], A.ri[q], (int)(xoff + j), A.v[p] * A.v[q]);
  for (int r = 0; r < m; ++r) add(r, r, -1, 0.0);   // every diagonal entry exists
  // G_i' rows: W_i part (constant, the block's slice of the linking variables) ...
  for (int t = 0; t < x0n; ++t)
    for (int q = W.cp[x0lo + t]; q < W.cp[x0lo + t + 1]; ++q) add(m + t, W.ri[q], -1, W.v[q]);
  // ... and A_i D_i u' for every link / global row u touching the block
  std::vector<std::vector<std::pair<int, double>>> ucol(A.n);
  for (size_t tt = 0; tt < urows.size(); ++tt) {
    const int t = x0n + (int)tt;
    const URow &u = urows[tt];
    for (size_t e = 0; e < u.j.size(); ++e) {
      const int j = u.j[e];
      ucol[j].push_back({t, u.u[e]});
      for (int q = A.cp[j]; q < A.cp[j + 1]; ++q)
        add(m + t, A.ri[q], (int)(xoff + j), A.v[q] * u.u[e]);
    }
  }
  // C_i = [U_i; Fg_i] D_i [U_i; Fg_i]'
  for (int j = 0; j < A.n; ++j)
    for (size_t x = 0; x < ucol[j].size(); ++x)
      for (size_t y = 0; y <= x; ++y)
        add(m + ucol[j][x].first, m + ucol[j][y].first, (int)(xoff + j),
            ucol[j][x].second * ucol[j][y].second);
  // stable sort by key = tile id * NB*NB + position in the tile: two stable
  // counting passes (position, then tile), the same order as a stable
  // comparison sort in linear time
  {
    const long long ntile = (long long)T * (T + 1) / 2;
    std::vector<Con> tmp(cons.size());
    std::vector<long long> cnt((size_t)std::max<long long>(ntile, NB * NB) + 1);
    auto pass = [&](std::vector<Con> &src, std::vector<Con> &dst, long long nb, auto digit) {
      std::fill(cnt.begin(), cnt.begin() + nb + 1, 0);
      for (const Con &x : src) ++cnt[digit(x) + 1];
      for (long long d = 0; d < nb; ++d) cnt[d + 1] += cnt[d];
      for (const Con &x : src) dst[cnt[digit(x)]++] = x;
    };
    pass(cons, tmp, NB * NB, [](const Con &x) { return x.key % (NB * NB); });
    pass(tmp, cons, ntile, [](const Con &x) { return x.key / (NB * NB); });
  }
  // tiles in id order (J-major lower), entries grouped by key
  size_t c = 0;
  P.nz.assign((size_t)T * T, 0);
  for (int Jt = 0; Jt < T; ++Jt)
    for (int It = Jt; It < T; ++It) {
      const long long id = tile_id(It, Jt);
      P.tiles.push_back({blk, It, Jt, 0});
      P.tile_ent.push_back((long long)P.ent_pos.size());
      if (c < cons.size() && cons[c].key / (NB * NB) == id) P.nz[(size_t)It * T + Jt] = 1;
      while (c < cons.size() && cons[c].key / (NB * NB) == id) {
        const long long key = cons[c].key;
        const int within = (int)(key % (NB * NB));
        const int ct = within / NB, rt = within % NB;
        const int R = It * NB + rt, C = Jt * NB + ct;
        int pos = (rt << 8) | ct;
        if (R == C && R < m) pos |= (1 << 16);
        else if (R == C) pos |= (1 << 17);
        P.ent_pos.push_back(pos);
        P.ent_cb.push_back((long long)P.con_idx.size());
        while (c < cons.size() && cons[c].key == key) {
          P.con_idx.push_back(cons[c].didx);
          P.con_coef.push_back(cons[c].coef);
          ++c;
        }
      }
    }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void ahlp_default_options(ahlp_options *o) {
  if (!o) return;
  o->precision = AHLP_PREC_FP64;
  o->max_iter = 200;
  o->tol = 1e-8;
  o->eta = 0.9995;
  o->delta = 1e-8;
  o->rho = 0.0;
  o->refine_max = 40;
  o->refine_tol = 1e-10;
  o->pivot_tol = 1e-12;
  o->verbose = 0;
  o->max_correctors = 4;
  o->fp32_cond_max = 1e14;
  o->ipm_refine_tol = 1e-6;
  o->correctors_by_cost = 1;
  o->fp32_update = 0;
  o->ff_update = 0;
  o->schur_chain = 0;
  o->profile_kernels = 0;
  o->iter_cb = nullptr;
  o->iter_cb_ctx = nullptr;
  o->pivot_mode = 0;
  o->tile_sparse = 1;
}

const char *ahlp_status_string(int s) {
  switch (s) {
    case AHLP_OK: return "OK";
    case AHLP_ERR_INVALID_ARG: return "INVALID_ARG";
    case AHLP_ERR_DIM_MISMATCH: return "DIM_MISMATCH";
    case AHLP_ERR_UNSUPPORTED: return "UNSUPPORTED";
    case AHLP_ERR_NOT_SPD: return "NOT_SPD";
    case AHLP_ERR_REFINE_FAIL: return "REFINE_FAIL";
    case AHLP_ERR_MAX_ITER: return "MAX_ITER";
    case AHLP_ERR_INFEASIBLE: return "INFEASIBLE_OR_UNBOUNDED";
    case AHLP_ERR_CUDA: return "CUDA";
    case AHLP_ERR_OOM: return "OOM";
    case AHLP_ERR_TIMEOUT: return "TIMEOUT";
    case AHLP_ERR_STOPPED: return "STOPPED";
    default: return "UNKNOWN";
  }
}

const char *ahlp_last_error(const ahlp_problem *p) {
  return p ? p->err.c_str() : g_create_err.c_str();
}

void arrowhead_lp_destroy(ahlp_problem *p) {
  if (!p) return;
  for (auto e : p->kt_pool) cudaEventDestroy(e);
  for (auto &b : p->allocs) cudaFree(b.ptr);
  if (p->gm_V) cudaFree(p->gm_V);
  if (p->gm_Z) cudaFree(p->gm_Z);
  if (p->h_scal) cudaFreeHost(p->h_scal);
  for (auto &e : p->ev)
    if (e) cudaEventDestroy(e);
  delete p;
}

int arrowhead_lp_sizes(const ahlp_problem *p, int64_t *n_total, int64_t *m_total) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  if (n_total) *n_total = p->n;
  if (m_total) *m_total = p->m;
  return AHLP_OK;
}

int arrowhead_lp_set_stream(ahlp_problem *p, void *stream) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  p->stream = reinterpret_cast<cudaStream_t>(stream);
  return AHLP_OK;
}

static int check_options(const ahlp_options &o, std::string &err) {
  if (o.precision != AHLP_PREC_FP64 && o.precision != AHLP_PREC_MIXED) {
    err = "precision must be AHLP_PREC_FP64 or AHLP_PREC_MIXED";
    return AHLP_ERR_INVALID_ARG;
  }
  if (o.max_iter < 0 || !(o.tol > 0) || !(o.eta > 0 && o.eta < 1) || o.delta < 0 || o.rho < 0 ||
      o.refine_max < 0 || !(o.refine_tol > 0) || !(o.pivot_tol >= 0) ||
      !(o.fp32_cond_max >= 1) || o.max_correctors < 0 || o.max_correctors > 8 ||
      !(o.ipm_refine_tol >= 0 && o.ipm_refine_tol < 1) ||
      (o.correctors_by_cost != 0 && o.correctors_by_cost != 1) || o.fp32_update < 0 ||
      o.fp32_update > 3 || o.ff_update < 0 || o.ff_update > 3 || o.schur_chain < 0 ||
      o.schur_chain > 1 || o.profile_kernels < 0 || o.profile_kernels > 1 ||
      o.pivot_mode < 0 || o.pivot_mode > 1 || o.tile_sparse < 0 || o.tile_sparse > 1) {
    err = "invalid option value";
    return AHLP_ERR_INVALID_ARG;
  }
  return AHLP_OK;
}

int arrowhead_lp_set_options(ahlp_problem *p, const ahlp_options *opt) {
  if (!p || !opt) return AHLP_ERR_INVALID_ARG;
  int s = check_options(*opt, p->err);
  if (s != AHLP_OK) return s;
  p->opt = *opt;
  return AHLP_OK;
}

int arrowhead_lp_set_cb(ahlp_problem *p, const double *c, const double *b) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  try {
    // stage, check for NaN/Inf, then replace; returns the max norm
    auto replace = [&](const double *src, double *dst, long long len, double *staging,
                       double &norm) -> bool {
      const double *d = stage_in(p, src, len, staging);
      ck(launch_reduce(p, RED_MAXABS, d, nullptr, len, p->scal + 0), "reduce");
      read_scalars(p, 1);
      if (!std::isfinite(p->h_scal[0])) return false;
      ck(cudaMemcpyAsync(dst, d, len * 8, cudaMemcpyDeviceToDevice, p->stream), "copy");
      norm = p->h_scal[0];
      return true;
    };
    if (c && p->n > 0 && !replace(c, p->c, p->n, p->stg[0], p->cnorm_inf))
      return set_err(p, AHLP_ERR_INVALID_ARG, "arrowhead_lp_set_cb: c has NaN or Inf entries");
    if (b && p->m > 0 && !replace(b, p->b, p->m, p->stg[1], p->bnorm_inf))
      return set_err(p, AHLP_ERR_INVALID_ARG, "arrowhead_lp_set_cb: b has NaN or Inf entries");
    ck(cudaStreamSynchronize(p->stream), "sync");
    return AHLP_OK;
  } catch (const Fail &f) {
    return set_err(p, f.code, f.msg);
  }
}

namespace {

// A batch of independent arrowhead LPs solved as one: their direct sum is an
// arrowhead LP whose blocks are all the LPs' blocks in order, whose linking
// variables and global rows are the LPs' ones stacked, and in which a pair of
// consecutive blocks of different LPs has no link rows.  W, F0 and Fg0 get
// their columns moved to the LP's slice of x_0, Fg and Fg0 their rows to the
// LP's slice of the global rows; everything else is reused as given.
struct BatchDesc {
  ahlp_desc d{};
  std::vector<ahlp_csc> A, W, Fg, FL, FR, F0;
  ahlp_csc Fg0{};
  std::vector<const double *> b, c, blink, lb, ub;
  std::vector<int32_t> l;
  std::vector<double> c0, bg, lb0, ub0;
  std::deque<std::vector<int32_t>> ints;   // owned index arrays (stable addresses)
  std::deque<std::vector<double>> dbls;
  std::vector<long long> blk0, x0off, goff;   // per LP: first block, x_0 and row offsets

  const int32_t *zeros(int n) {
    ints.emplace_back(n + 1, 0);
    return ints.back().data();
  }
  // columns [0, n) of M become columns [off, off + n) of an ncols-wide matrix
  ahlp_csc shift_cols(const ahlp_csc *M, int m, int n, int off, int ncols) {
    if (M && (M->m != m || M->n != n)) fail(AHLP_ERR_DIM_MISMATCH, "batch: W or F0 shape");
    ahlp_csc o{m, ncols, nullptr, nullptr, nullptr};
    ints.emplace_back(ncols + 1, 0);
    std::vector<int32_t> &cp = ints.back();
    const int nnz = (M && n > 0 && M->colptr) ? M->colptr[n] : 0;
    for (int j = 0; j <= ncols; ++j) {
      const int jj = j - off;
      cp[j] = jj <= 0 ? 0 : (jj >= n ? nnz : M->colptr[jj]);
    }
    o.colptr = cp.data();
    o.rowidx = nnz ? M->rowidx : nullptr;
    o.val = nnz ? M->val : nullptr;
    return o;
  }
  // rows [0, m) of M become rows [off, off + m) of an nrows-high matrix
  ahlp_csc shift_rows(const ahlp_csc *M, int m, int n, int off, int nrows) {
    if (M && (M->m != m || M->n != n)) fail(AHLP_ERR_DIM_MISMATCH, "batch: Fg shape");
    ahlp_csc o{nrows, n, nullptr, nullptr, nullptr};
    if (!M || n == 0 || !M->colptr) {
      o.colptr = zeros(n);
      return o;
    }
    const int nnz = M->colptr[n];
    ints.emplace_back(M->rowidx, M->rowidx + nnz);
    for (auto &r : ints.back()) r += off;
    o.colptr = M->colptr;
    o.rowidx = ints.back().data();
    o.val = M->val;
    return o;
  }
};

void compose_batch(const ahlp_desc *D, int B, BatchDesc &S) {
  int N = 0, n0 = 0, mg = 0;
  for (int b = 0; b < B; ++b) {
    if (D[b].N < 1 || D[b].n0 < 0 || D[b].mg < 0)
      fail(AHLP_ERR_INVALID_ARG, "batch item " + std::to_string(b) + ": N >= 1, n0 >= 0, mg >= 0 required");
    if (!D[b].A || !D[b].W || !D[b].b || !D[b].c)
      fail(AHLP_ERR_INVALID_ARG, "batch item " + std::to_string(b) + ": A, W, b, c must be given");
    S.blk0.push_back(N);
    S.x0off.push_back(n0);
    S.goff.push_back(mg);
    N += D[b].N;
    n0 += D[b].n0;
    mg += D[b].mg;
  }
  bool bounds = false, bounds0 = false;
  for (int b = 0; b < B; ++b) {
    const ahlp_desc &d = D[b];
    const std::string tag = "batch item " + std::to_string(b);
    if (d.N > 1 && !d.l) fail(AHLP_ERR_INVALID_ARG, tag + ": l must be given when N > 1");
    for (int i = 0; i < d.N; ++i) {
      const int mi = d.A[i].m, ni = d.A[i].n;
      S.A.push_back(d.A[i]);
      S.W.push_back(S.shift_cols(&d.W[i], mi, d.n0, (int)S.x0off[b], n0));
      S.Fg.push_back(S.shift_rows(d.Fg ? &d.Fg[i] : nullptr, d.mg, ni, (int)S.goff[b], mg));
      S.b.push_back(d.b[i]);
      S.c.push_back(d.c[i]);
      S.lb.push_back(d.lb ? d.lb[i] : nullptr);
      S.ub.push_back(d.ub ? d.ub[i] : nullptr);
      bounds = bounds || d.lb || d.ub;
      if (i + 1 < d.N) {
        const int l = d.l[i];
        S.l.push_back(l);
        const ahlp_csc empty_l{l, d.A[i].n, S.zeros(d.A[i].n), nullptr, nullptr};
        const ahlp_csc empty_r{l, d.A[i + 1].n, S.zeros(d.A[i + 1].n), nullptr, nullptr};
        S.FL.push_back(d.FL ? d.FL[i] : empty_l);
        S.FR.push_back(d.FR ? d.FR[i] : empty_r);
        S.F0.push_back(S.shift_cols(d.F0 ? &d.F0[i] : nullptr, l, d.n0, (int)S.x0off[b], n0));
        S.blink.push_back(d.blink ? d.blink[i] : nullptr);
      } else if (b + 1 < B) {   // between LPs: no link rows
        S.l.push_back(0);
        S.FL.push_back(ahlp_csc{0, d.A[i].n, S.zeros(d.A[i].n), nullptr, nullptr});
        S.FR.push_back(ahlp_csc{0, D[b + 1].A[0].n, S.zeros(D[b + 1].A[0].n), nullptr, nullptr});
        S.F0.push_back(ahlp_csc{0, n0, S.zeros(n0), nullptr, nullptr});
        S.blink.push_back(nullptr);
      }
    }
    for (int k = 0; k < d.n0; ++k) S.c0.push_back(d.c0 ? d.c0[k] : 0.0);
    for (int k = 0; k < d.mg; ++k) S.bg.push_back(d.bg ? d.bg[k] : 0.0);
    bounds0 = bounds0 || d.lb0 || d.ub0;
  }
  if (bounds0)
    for (int b = 0; b < B; ++b)
      for (int k = 0; k < D[b].n0; ++k) {
        S.lb0.push_back(D[b].lb0 ? D[b].lb0[k] : 0.0);
        S.ub0.push_back(D[b].ub0 ? D[b].ub0[k] : INFINITY);
      }
  // Fg0: block diagonal over the LPs
  {
    std::vector<int32_t> cp(n0 + 1, 0), ri;
    std::vector<double> v;
    for (int b = 0; b < B; ++b) {
      const ahlp_desc &d = D[b];
      for (int j = 0; j < d.n0; ++j) {
        const int col = (int)S.x0off[b] + j;
        if (d.Fg0 && d.Fg0->colptr && d.Fg0->n == d.n0 && d.Fg0->m == d.mg)
          for (int q = d.Fg0->colptr[j]; q < d.Fg0->colptr[j + 1]; ++q) {
            ri.push_back(d.Fg0->rowidx[q] + (int)S.goff[b]);
            v.push_back(d.Fg0->val[q]);
          }
        else if (d.Fg0 && (d.Fg0->n != d.n0 || d.Fg0->m != d.mg))
          fail(AHLP_ERR_DIM_MISMATCH, "batch item " + std::to_string(b) + " Fg0: wrong shape");
        cp[col + 1] = (int32_t)ri.size();
      }
    }
    for (int j = 0; j < n0; ++j) cp[j + 1] = std::max(cp[j + 1], cp[j]);
    S.ints.push_back(std::move(cp));
    const int32_t *cpp = S.ints.back().data();
    S.ints.push_back(std::move(ri));
    const int32_t *rip = S.ints.back().data();
    S.dbls.push_back(std::move(v));
    S.Fg0 = ahlp_csc{mg, n0, cpp, rip, S.dbls.back().data()};
  }
  ahlp_desc &o = S.d;
  o.N = N;
  o.n0 = n0;
  o.mg = mg;
  o.c0 = S.c0.data();
  o.A = S.A.data();
  o.W = S.W.data();
  o.b = S.b.data();
  o.c = S.c.data();
  o.l = S.l.data();
  o.FL = S.FL.data();
  o.FR = S.FR.data();
  o.F0 = S.F0.data();
  o.blink = S.blink.data();
  o.Fg = S.Fg.data();
  o.Fg0 = &S.Fg0;
  o.bg = S.bg.data();
  o.lb = bounds ? S.lb.data() : nullptr;
  o.ub = bounds ? S.ub.data() : nullptr;
  o.lb0 = bounds0 ? S.lb0.data() : nullptr;
  o.ub0 = bounds0 ? S.ub0.data() : nullptr;
}

}  // namespace

int arrowhead_lp_create(const ahlp_desc *descs, int32_t batch, const ahlp_options *opt,
                        ahlp_problem **out) {
  if (!out) return AHLP_ERR_INVALID_ARG;
  *out = nullptr;
  g_create_err.clear();
  if (!descs) {
    g_create_err = "descs is NULL";
    return AHLP_ERR_INVALID_ARG;
  }
  if (batch < 1) {
    g_create_err = "batch must be >= 1";
    return AHLP_ERR_INVALID_ARG;
  }
  // LPs in the full statement (bounds, inequality rows): their equality form
  std::deque<StdDesc> stds;
  std::vector<ahlp_desc> eqform;
  std::vector<ahlp_problem::LpRecov> recov(batch);
  try {
    bool any = false;
    for (int b = 0; b < batch; ++b) {
      any = any || desc_is_general(descs[b]);
      // original sizes (for the map back) of an LP already in equality form
      if (descs[b].A && descs[b].N > 0 && !desc_is_general(descs[b])) {
        for (int i = 0; i < descs[b].N; ++i) recov[b].n_orig.push_back(descs[b].A[i].n);
        recov[b].n0_orig = descs[b].n0;
      }
    }
    if (any) {
      for (int b = 0; b < batch; ++b) {
        if (desc_is_general(descs[b])) {
          stds.emplace_back();
          standardize(descs[b], stds.back());
          eqform.push_back(stds.back().d);
          recov[b].recov = stds.back().recov;
          recov[b].n_orig = stds.back().n_orig;
          recov[b].n0_orig = stds.back().n0_orig;
          recov[b].const_obj = stds.back().const_obj;
        } else {
          eqform.push_back(descs[b]);
        }
      }
      descs = eqform.data();
    }
  } catch (const Fail &f) {
    g_create_err = f.msg;
    return f.code;
  } catch (const std::bad_alloc &) {
    g_create_err = "host memory exhausted while reducing the LP to equality form";
    return AHLP_ERR_OOM;
  }
  BatchDesc composed;
  if (batch > 1) {
    try {
      compose_batch(descs, batch, composed);
    } catch (const Fail &f) {
      g_create_err = f.msg;
      return f.code;
    }
    descs = &composed.d;
  }
  ahlp_problem *p = new ahlp_problem();
  p->batch = batch;
  p->lp_recov = std::move(recov);
  if (batch > 1) {
    p->lp_blk0 = composed.blk0;
    p->lp_x0off = composed.x0off;
    p->lp_goff = composed.goff;
  }
  ahlp_default_options(&p->opt);
  if (opt) {
    int s = check_options(*opt, g_create_err);
    if (s != AHLP_OK) {
      delete p;
      return s;
    }
    p->opt = *opt;
  }
  try {
    const ahlp_desc &D = descs[0];
    if (D.N < 1 || D.n0 < 0 || D.mg < 0) fail(AHLP_ERR_INVALID_ARG, "N >= 1, n0 >= 0, mg >= 0 required");
    if (!D.A || !D.W || !D.b || !D.c) fail(AHLP_ERR_INVALID_ARG, "A, W, b, c must be given");
    if (D.N > 1 && !D.l) fail(AHLP_ERR_INVALID_ARG, "l must be given when N > 1");
    const int N = D.N, n0 = D.n0, mg = D.mg;
    p->N = N;
    p->n0 = n0;
    p->mg = mg;
    p->B = n0 + mg;
    // ---- blocks -----------------------------------------------------------
    std::vector<Csc> A(N), W(N), Fg(N), FL(N > 1 ? N - 1 : 0), FR(FL.size()), F0(FL.size());
    std::vector<std::vector<double>> b(N), c(N), blink(FL.size());
    {   // blocks are independent: validated on host threads, the first failing
        // block reported (as a sequential pass would)
      std::vector<int> vcode(N, 0);
      std::vector<std::string> vmsg(N);
      parallel_for(N, [&](int i) {
        try {
          const std::string tag = "block " + std::to_string(i);
          if (D.A[i].m < 0 || D.A[i].n < 0) fail(AHLP_ERR_INVALID_ARG, tag + ": negative size");
          A[i] = canon(&D.A[i], D.A[i].m, D.A[i].n, tag + " A");
          W[i] = canon(&D.W[i], A[i].m, n0, tag + " W");
          Fg[i] = canon(D.Fg ? &D.Fg[i] : nullptr, mg, A[i].n, tag + " Fg");
          b[i] = vec_in(D.b[i], A[i].m, tag + " b");
          c[i] = vec_in(D.c[i], A[i].n, tag + " c");
          check_bounds(D.lb ? D.lb[i] : nullptr, D.ub ? D.ub[i] : nullptr, A[i].n, tag);
        } catch (const Fail &f) {
          vcode[i] = f.code;
          vmsg[i] = f.msg;
        } catch (const std::bad_alloc &) {
          vcode[i] = AHLP_ERR_OOM;
          vmsg[i] = "host memory exhausted while reading block " + std::to_string(i);
        } catch (...) {   // nothing may leave a host thread
          vcode[i] = AHLP_ERR_INVALID_ARG;
          vmsg[i] = "block " + std::to_string(i) + ": could not be read";
        }
      });
      for (int i = 0; i < N; ++i)
        if (vcode[i]) fail(vcode[i], vmsg[i]);
      for (int i = 0; i < N; ++i) {
        p->mi.push_back(A[i].m);
        p->ni.push_back(A[i].n);
      }
    }
    check_bounds(D.lb0, D.ub0, n0, "x0");
    std::vector<int> l(FL.size());
    for (size_t j = 0; j < FL.size(); ++j) {
      const std::string tag = "pair " + std::to_string(j);
      if (D.l[j] < 0) fail(AHLP_ERR_INVALID_ARG, tag + ": negative link count");
      l[j] = D.l[j];
      if (l[j] > 0 && (!D.FL || !D.FR)) fail(AHLP_ERR_INVALID_ARG, tag + ": FL/FR missing");
      FL[j] = canon(D.FL ? &D.FL[j] : nullptr, l[j], A[j].n, tag + " FL");
      FR[j] = canon(D.FR ? &D.FR[j] : nullptr, l[j], A[j + 1].n, tag + " FR");
      F0[j] = canon(D.F0 ? &D.F0[j] : nullptr, l[j], n0, tag + " F0");
      blink[j] = vec_in(D.blink ? D.blink[j] : nullptr, l[j], tag + " blink");
    }
    Csc Fg0 = canon(D.Fg0, mg, n0, "Fg0");
    std::vector<double> c0 = vec_in(D.c0, n0, "c0");
    std::vector<double> bg = vec_in(D.bg, mg, "bg");
    // ---- global sizes and offsets --------------------------------------------
    p->xoff.resize(N + 1);
    p->yoff.resize(N);
    long long xo = 0, yo = 0;
    for (int i = 0; i < N; ++i) {
      p->xoff[i] = xo;
      p->yoff[i] = yo;
      xo += A[i].n;
      yo += A[i].m;
    }
    p->xoff[N] = xo;
    p->msum = yo;
    p->n = xo + n0;
    p->link_off.assign(N, 0);
    for (int j = 0; j + 1 < N; ++j) p->link_off[j + 1] = p->link_off[j] + l[j];
    p->nl = (int)p->link_off[N - 1];
    p->m = p->msum + p->nl + mg;
    p->nS = p->nl + p->B;
    // ---- monolithic A (CSR) and A' (CSR) for residuals ------------------------
    // Built by counting and filling, block by block (and pair by pair) on host
    // threads.  A block's rows hold its A_i columns then its linking-variable
    // columns; a pair's link rows its FL, FR, F0 columns; global rows take the
    // blocks in order, then Fg0 -- so every row of A is sorted.  In A', a
    // block's columns hold its own rows, then the previous pair's link rows,
    // the next pair's, then the global rows; a linking variable's column the
    // blocks' rows, the link rows, the global rows -- sorted as well.
    const long long grow0 = p->msum + p->nl;
    const int nP = (int)FL.size();
    auto each = [](const Csc &M, auto &&f) {   // f(row, col, value), column-major order
      for (int j = 0; j < M.n; ++j)
        for (int q = M.cp[j]; q < M.cp[j + 1]; ++q) f(M.ri[q], j, M.v[q]);
    };
    std::vector<int> Arp(p->m + 1, 0), Aci, ATrp(p->n + 1, 0), ATci;
    std::vector<double> Av, ATv;
    parallel_for(N, [&](int i) {
      int *cnt = Arp.data() + 1 + p->yoff[i];
      each(A[i], [&](int r, int, double) { ++cnt[r]; });
      each(W[i], [&](int r, int, double) { ++cnt[r]; });
    });
    parallel_for(nP, [&](int j) {
      int *cnt = Arp.data() + 1 + p->msum + p->link_off[j];
      each(FL[j], [&](int r, int, double) { ++cnt[r]; });
      each(FR[j], [&](int r, int, double) { ++cnt[r]; });
      each(F0[j], [&](int r, int, double) { ++cnt[r]; });
    });
    {
      int *cnt = Arp.data() + 1 + grow0;
      for (int i = 0; i < N; ++i) each(Fg[i], [&](int r, int, double) { ++cnt[r]; });
      each(Fg0, [&](int r, int, double) { ++cnt[r]; });
    }
    for (long long r = 0; r < p->m; ++r) {
      if ((long long)Arp[r] + Arp[r + 1] >= (1LL << 31))
        fail(AHLP_ERR_UNSUPPORTED, "more than 2^31 nonzeros");
      Arp[r + 1] += Arp[r];
    }
    const long long nnz = Arp[p->m];
    Aci.resize(nnz);
    Av.resize(nnz);
    // fill: the row starts of the rows M's local row indices refer to
    auto put_rows = [&](std::vector<int> &fill, const Csc &M, long long c0_) {
      each(M, [&](int r, int j, double v) {
        const int pos = fill[r]++;
        Aci[pos] = (int)(c0_ + j);
        Av[pos] = v;
      });
    };
    parallel_for(N, [&](int i) {
      std::vector<int> fill(Arp.begin() + p->yoff[i], Arp.begin() + p->yoff[i] + A[i].m);
      put_rows(fill, A[i], p->xoff[i]);
      put_rows(fill, W[i], p->xoff[N]);
    });
    parallel_for(nP, [&](int j) {
      const long long r0 = p->msum + p->link_off[j];
      std::vector<int> fill(Arp.begin() + r0, Arp.begin() + r0 + l[j]);
      put_rows(fill, FL[j], p->xoff[j]);
      put_rows(fill, FR[j], p->xoff[j + 1]);
      put_rows(fill, F0[j], p->xoff[N]);
    });
    {
      std::vector<int> fill(Arp.begin() + grow0, Arp.begin() + grow0 + mg);
      for (int i = 0; i < N; ++i) put_rows(fill, Fg[i], p->xoff[i]);
      put_rows(fill, Fg0, p->xoff[N]);
    }
    // A': column counts, then each column's rows in increasing order
    parallel_for(N, [&](int i) {
      int *cnt = ATrp.data() + 1 + p->xoff[i];
      for (int j = 0; j < A[i].n; ++j) {
        int c = (A[i].cp[j + 1] - A[i].cp[j]) + (Fg[i].cp[j + 1] - Fg[i].cp[j]);
        if (i > 0) c += FR[i - 1].cp[j + 1] - FR[i - 1].cp[j];
        if (i + 1 < N) c += FL[i].cp[j + 1] - FL[i].cp[j];
        cnt[j] = c;
      }
    });
    {
      int *cnt = ATrp.data() + 1 + p->xoff[N];
      for (int t = 0; t < n0; ++t) {
        int c = Fg0.cp[t + 1] - Fg0.cp[t];
        for (int i = 0; i < N; ++i) c += W[i].cp[t + 1] - W[i].cp[t];
        for (int j = 0; j < nP; ++j) c += F0[j].cp[t + 1] - F0[j].cp[t];
        cnt[t] = c;
      }
    }
    for (long long c2 = 0; c2 < p->n; ++c2) ATrp[c2 + 1] += ATrp[c2];
    ATci.resize(nnz);
    ATv.resize(nnz);
    auto put_col = [&](int &pos, const Csc &M, int j, long long r0) {
      for (int q = M.cp[j]; q < M.cp[j + 1]; ++q) {
        ATci[pos] = (int)(r0 + M.ri[q]);
        ATv[pos] = M.v[q];
        ++pos;
      }
    };
    parallel_for(N, [&](int i) {
      for (int j = 0; j < A[i].n; ++j) {
        int pos = ATrp[p->xoff[i] + j];
        put_col(pos, A[i], j, p->yoff[i]);
        if (i > 0) put_col(pos, FR[i - 1], j, p->msum + p->link_off[i - 1]);
        if (i + 1 < N) put_col(pos, FL[i], j, p->msum + p->link_off[i]);
        put_col(pos, Fg[i], j, grow0);
      }
    });
    for (int t = 0; t < n0; ++t) {
      int pos = ATrp[p->xoff[N] + t];
      for (int i = 0; i < N; ++i) put_col(pos, W[i], t, p->yoff[i]);
      for (int j = 0; j < nP; ++j) put_col(pos, F0[j], t, p->msum + p->link_off[j]);
      put_col(pos, Fg0, t, grow0);
    }
    std::vector<double> bgl, cgl;
    for (int i = 0; i < N; ++i) bgl.insert(bgl.end(), b[i].begin(), b[i].end());
    for (auto &v : blink) bgl.insert(bgl.end(), v.begin(), v.end());
    bgl.insert(bgl.end(), bg.begin(), bg.end());
    for (int i = 0; i < N; ++i) cgl.insert(cgl.end(), c[i].begin(), c[i].end());
    cgl.insert(cgl.end(), c0.begin(), c0.end());
    for (double v : bgl) p->bnorm_inf = std::max(p->bnorm_inf, std::fabs(v));
    for (double v : cgl) p->cnorm_inf = std::max(p->cnorm_inf, std::fabs(v));
    for (int b = 0; b < p->batch && p->batch > 1; ++b) {
      ahlp_problem::LpRange r{};
      const long long blo = p->lp_blk0[b], bhi = b + 1 < p->batch ? p->lp_blk0[b + 1] : N;
      const long long x0hi = b + 1 < p->batch ? p->lp_x0off[b + 1] : n0;
      const long long ghi = b + 1 < p->batch ? p->lp_goff[b + 1] : mg;
      r.xb0 = p->xoff[blo];
      r.xb1 = p->xoff[bhi];
      r.x00 = p->xoff[N] + p->lp_x0off[b];
      r.x01 = p->xoff[N] + x0hi;
      r.yb0 = p->yoff[blo];
      r.yb1 = bhi < N ? p->yoff[bhi] : p->msum;
      r.yl0 = p->msum + p->link_off[blo];
      r.yl1 = p->msum + p->link_off[bhi - 1];
      r.yg0 = p->msum + p->nl + p->lp_goff[b];
      r.yg1 = p->msum + p->nl + ghi;
      r.bnorm = r.cnorm = 0.0;
      for (long long k : {0, 1, 2})
        for (long long q = (k == 0 ? r.yb0 : k == 1 ? r.yl0 : r.yg0);
             q < (k == 0 ? r.yb1 : k == 1 ? r.yl1 : r.yg1); ++q)
          r.bnorm = std::max(r.bnorm, std::fabs(bgl[q]));
      for (long long q = r.xb0; q < r.xb1; ++q) r.cnorm = std::max(r.cnorm, std::fabs(cgl[q]));
      for (long long q = r.x00; q < r.x01; ++q) r.cnorm = std::max(r.cnorm, std::fabs(cgl[q]));
      p->lp_rng.push_back(r);
    }
    std::vector<unsigned char> isx0(p->n, 0);
    for (long long k = p->xoff[N]; k < p->n; ++k) isx0[k] = 1;
    // ---- per-block layout ------------------------------------------------------
    p->h_blk.resize(N);
    p->h_sblk.resize(N);
    long long base = 0, voff = 0, d0 = 0, cd = 0, ioff = 0;
    // each block's slice of the linking variables and global rows: all of
    // them for one LP, its own LP's ones in a batch (W_i, Fg_i are zero elsewhere)
    std::vector<int> bx0lo(N, 0), bx0n(N, n0), bglo(N, 0), bgn(N, mg);
    for (int b = 0; b < p->batch && p->batch > 1; ++b) {
      const long long blo = p->lp_blk0[b], bhi = b + 1 < p->batch ? p->lp_blk0[b + 1] : N;
      const long long x0hi = b + 1 < p->batch ? p->lp_x0off[b + 1] : n0;
      const long long ghi = b + 1 < p->batch ? p->lp_goff[b + 1] : mg;
      for (long long i = blo; i < bhi; ++i) {
        bx0lo[i] = (int)p->lp_x0off[b];
        bx0n[i] = (int)(x0hi - p->lp_x0off[b]);
        bglo[i] = (int)p->lp_goff[b];
        bgn[i] = (int)(ghi - p->lp_goff[b]);
      }
    }
    for (int i = 0; i < N; ++i) {
      const int lp = i > 0 ? l[i - 1] : 0, ln = i + 1 < N ? l[i] : 0;
      const int k = bx0n[i] + lp + ln + bgn[i];
      const int m = A[i].m, a = m + k;
      p->ki.push_back(k);
      p->lprev.push_back(lp);
      p->lnext.push_back(ln);
      BlkInfo bi{};
      bi.base = base;
      bi.voff = voff;
      bi.d0off = d0;
      bi.cdoff = cd;
      bi.lda = (int)round_up(std::max(a, 1), 8);
      bi.a = a;
      bi.p = m;
      bi.T = (a + NB - 1) / NB;
      bi.Tp = (m + NB - 1) / NB;
      bi.ioff = ioff;
      ioff += (long long)bi.Tp * NB * NB;
      bi.soff = p->stage_slots;
      p->stage_slots += bi.T;
      p->h_blk[i] = bi;
      // algorithmic work of this block's partial Cholesky (column c updates the
      // r = a - c - 1 entries below its pivot and the r(r+1)/2 trailing pairs)
      for (int cc = 0; cc < m; ++cc) {
        const double r = (double)(a - cc - 1);
        p->fac_flops += r + r * (r + 1.0);
      }
      p->tri_elems += (double)a * (a + 1) / 2.0;
      base += round_up((long long)bi.lda * a, 32);
      voff += a;
      d0 += m;
      cd += k;
      p->amax = std::max(p->amax, a);
      p->maxT = std::max(p->maxT, bi.T);
      p->maxTp = std::max(p->maxTp, bi.Tp);
      SchurBlk sb{};
      sb.m = m;
      sb.k = k;
      sb.lprev = lp;
      sb.lnext = ln;
      sb.link_prev_off = i > 0 ? (int)p->link_off[i - 1] : 0;
      sb.link_next_off = i + 1 < N ? (int)p->link_off[i] : 0;
      sb.x0lo = bx0lo[i];
      sb.x0n = bx0n[i];
      sb.glo = bglo[i];
      sb.gn = bgn[i];
      p->h_sblk[i] = sb;
    }
    p->aug_elems = base;
    p->tinv_elems = ioff;
    p->vec_elems = voff;
    // the border solves keep the border vector in shared memory next to a
    // staged 64x64 tile; the link-chain kernels keep one l x l block there
    if ((long long)p->B * 8 > kSmemVecBytes)
      fail(AHLP_ERR_UNSUPPORTED, "the border (linking variables + global rows) exceeds 20480");
    for (int v : l)
      if (v > 96) fail(AHLP_ERR_UNSUPPORTED, "more than 96 local link rows per block pair");
    // ---- formation patterns --------------------------------------------------
    // Independent per block: built on host threads into block-local patterns,
    // then concatenated in block order, so the result does not depend on the
    // thread count.  A failure reports the first failing block, as a
    // sequential pass would.
    std::vector<Pattern> part(N);
    p->tile_nz.assign(N, {});
    std::vector<int> pcode(N, 0);
    std::vector<std::string> pmsg(N);
    auto one_block = [&](int i) {
      try {
        std::vector<URow> urows(p->ki[i] - bx0n[i]);
        auto rows_of = [&](const Csc &F, int off, int shift, int nrows) {
          for (int j = 0; j < F.n; ++j)
            for (int q = F.cp[j]; q < F.cp[j + 1]; ++q) {
              const int r = F.ri[q] - shift;
              if (r < 0 || r >= nrows)
                fail(AHLP_ERR_INVALID_ARG, "block " + std::to_string(i) + ": a global row outside its LP");
              urows[off + r].j.push_back(j);
              urows[off + r].u.push_back(F.v[q]);
            }
        };
        if (i > 0) rows_of(FR[i - 1], 0, 0, p->lprev[i]);
        if (i + 1 < N) rows_of(FL[i], p->lprev[i], 0, p->lnext[i]);
        rows_of(Fg[i], p->lprev[i] + p->lnext[i], bglo[i], bgn[i]);
        for (int t = 0; t < n0; ++t)
          if ((t < bx0lo[i] || t >= bx0lo[i] + bx0n[i]) && W[i].cp[t + 1] > W[i].cp[t])
            fail(AHLP_ERR_INVALID_ARG, "block " + std::to_string(i) + ": a linking variable outside its LP");
        build_block_pattern(i, A[i], W[i], urows, bx0lo[i], bx0n[i], A[i].m, p->ki[i], p->xoff[i],
                            part[i]);
      } catch (const Fail &f) {
        pcode[i] = f.code;
        pmsg[i] = f.msg;
      } catch (const std::bad_alloc &) {
        pcode[i] = AHLP_ERR_OOM;
        pmsg[i] = "host memory exhausted while building the formation pattern";
      } catch (...) {   // nothing may leave a host thread
        pcode[i] = AHLP_ERR_INVALID_ARG;
        pmsg[i] = "block " + std::to_string(i) + ": formation pattern could not be built";
      }
    };
    parallel_for(N, one_block);
    for (int i = 0; i < N; ++i)
      if (pcode[i]) fail(pcode[i], pmsg[i]);
    // the block patterns stay separate: their entry and contribution offsets
    // are made absolute here and each part is uploaded at its offset
    std::vector<long long> tb(N + 1, 0), eb(N + 1, 0), cb(N + 1, 0);
    for (int i = 0; i < N; ++i) {
      tb[i + 1] = tb[i] + (long long)part[i].tiles.size();
      p->tile_nz[i] = std::move(part[i].nz);
      eb[i + 1] = eb[i] + (long long)part[i].ent_pos.size();
      cb[i + 1] = cb[i] + (long long)part[i].con_idx.size();
    }
    parallel_for(N, [&](int i) {
      for (long long &v : part[i].tile_ent) v += eb[i];
      for (long long &v : part[i].ent_cb) v += cb[i];
    });
    part[N - 1].tile_ent.push_back(eb[N]);   // end sentinels
    part[N - 1].ent_cb.push_back(cb[N]);
    p->ntiles = tb[N];
    p->nent = eb[N];
    p->ncon = cb[N];
    // ---- Schur maps ---------------------------------------------------------------
    std::vector<int> kmap;
    for (int i = 0; i < N; ++i) {
      p->kmap_off.push_back((long long)kmap.size());
      const int xn = bx0n[i], lpv = p->lprev[i], lnx = p->lnext[i];
      for (int t = 0; t < p->ki[i]; ++t) {
        int s;
        if (t < xn) s = p->nl + bx0lo[i] + t;
        else if (t < xn + lpv) s = (int)p->link_off[i - 1] + (t - xn);
        else if (t < xn + lpv + lnx) s = (int)p->link_off[i] + (t - xn - lpv);
        else s = p->nl + n0 + bglo[i] + (t - xn - lpv - lnx);
        kmap.push_back(s);
      }
    }
    std::vector<int> link_pair(p->nl);
    for (size_t j = 0; j < FL.size(); ++j)
      for (int r = 0; r < l[j]; ++r) link_pair[p->link_off[j] + r] = (int)j;
    long long te = 0, he = 0;
    for (size_t j = 0; j < FL.size(); ++j) {
      p->td_off.push_back(te);
      te += (long long)l[j] * l[j];
      if (j + 1 < FL.size()) {
        p->h_off.push_back(he);
        he += (long long)l[j + 1] * l[j];
      }
    }
    p->td_elems = te;
    p->h_elems = he;
    std::vector<long long> f0i, fg0i;
    std::vector<double> f0v, fg0v;
    for (size_t j = 0; j < FL.size(); ++j)
      for (int cc = 0; cc < n0; ++cc)
        for (int q = F0[j].cp[cc]; q < F0[j].cp[cc + 1]; ++q) {
          f0i.push_back((long long)cc * p->nl + p->link_off[j] + F0[j].ri[q]);
          f0v.push_back(F0[j].v[q]);
        }
    for (int cc = 0; cc < n0; ++cc)
      for (int q = Fg0.cp[cc]; q < Fg0.cp[cc + 1]; ++q) {
        const long long g = n0 + Fg0.ri[q];
        fg0i.push_back((long long)cc * p->B + g);
        fg0v.push_back(Fg0.v[q]);
        fg0i.push_back(g * p->B + cc);
        fg0v.push_back(Fg0.v[q]);
      }
    p->nf0 = (long long)f0i.size();
    p->nfg0 = (long long)fg0i.size();
    p->Bld = (int)round_up(std::max(p->B, 1), 8);
    p->h_bx = BlkInfo{0, 0, 0, p->Bld, p->B, n0, (p->B + NB - 1) / NB, (n0 + NB - 1) / NB,
                      kTagBorderX, 0, 0, 0};
    p->h_bp = BlkInfo{(long long)n0 * p->Bld + n0, n0, n0, p->Bld, mg, mg, (mg + NB - 1) / NB,
                      (mg + NB - 1) / NB, kTagBorderG, 0, 0, 0};
    // ---- device memory ----------------------------------------------------------
    ck(cudaGetDevice(&p->device), "cudaGetDevice");
    p->b = dupload(p, bgl);
    p->c = dupload(p, cgl);
    p->A_rp = dupload(p, Arp);
    p->A_ci = dupload(p, Aci);
    p->A_v = dupload(p, Av);
    p->AT_rp = dupload(p, ATrp);
    p->AT_ci = dupload(p, ATci);
    p->AT_v = dupload(p, ATv);
    p->is_x0 = dupload(p, isx0);
    auto make_spmat = [&](const std::vector<int> &rp, const int *drp, const int *dci,
                          const double *dv) {
      SpMat M;
      M.rp = drp;
      M.ci = dci;
      M.v = dv;
      M.rows = (long long)rp.size() - 1;
      std::vector<int> lr;
      for (long long r = 0; r < M.rows; ++r)
        if (rp[r + 1] - rp[r] > kShortRow) lr.push_back((int)r);
      M.n_long = (int)lr.size();
      if (!lr.empty()) M.long_rows = dupload(p, lr);
      return M;
    };
    p->Amat = make_spmat(Arp, p->A_rp, p->A_ci, p->A_v);
    p->ATmat = make_spmat(ATrp, p->AT_rp, p->AT_ci, p->AT_v);
    if (p->opt.precision == AHLP_PREC_MIXED) {
      p->aug32 = dalloc<float>(p, p->aug_elems);
      p->tinv32 = dalloc<float>(p, std::max(p->tinv_elems, 1LL));
      p->vec32 = dalloc<float>(p, std::max(p->vec_elems, 1LL));
    } else {
      p->aug = dalloc<double>(p, p->aug_elems);
      p->tinv = dalloc<double>(p, std::max(p->tinv_elems, 1LL));
    }
    p->fac_prec = p->opt.precision == AHLP_PREC_MIXED ? kPrecFP32 : kPrecFP64;
    p->blk = dupload(p, p->h_blk);
    p->sblk = dupload(p, p->h_sblk);
    {
      // wavefront schedules of the block solves: forward in increasing row
      // tile, backward in decreasing pivot tile, blocks interleaved per wave
      std::vector<int> fs, bs, foff(N);
      int nflags = 0, maxT = 0, maxTp = 0;
      for (int i = 0; i < N; ++i) {
        foff[i] = nflags;
        nflags += p->h_blk[i].T;
        maxT = std::max(maxT, p->h_blk[i].T);
        maxTp = std::max(maxTp, p->h_blk[i].Tp);
      }
      for (int r = 0; r < maxT; ++r)
        for (int i = 0; i < N; ++i)
          if (r < p->h_blk[i].T) fs.insert(fs.end(), {i, r});
      for (int w = 0; w < maxTp; ++w)
        for (int i = 0; i < N; ++i)
          if (w < p->h_blk[i].Tp) bs.insert(bs.end(), {i, p->h_blk[i].Tp - 1 - w});
      p->trsv_nf = (int)fs.size() / 2;
      p->trsv_nb = (int)bs.size() / 2;
      p->trsv_nflags = nflags;
      if (!fs.empty()) p->trsv_fsched = dupload(p, fs);
      if (!bs.empty()) p->trsv_bsched = dupload(p, bs);
      if (N > 0) p->trsv_flag_off = dupload(p, foff);
      p->trsv_flags = dalloc<int>(p, nflags + 2);
      p->trsv_err = dalloc<int>(p, 1);
      ck(cudaMemset(p->trsv_err, 0, sizeof(int)), "memset");
    }
    p->diag0 = dalloc<double>(p, std::max(d0, 1LL));
    p->cdiag0 = dalloc<double>(p, std::max(cd, 1LL));
    p->cdiag_elems = cd;
    p->sb_ref = dalloc<double>(p, p->B);
    p->ftiles = dupload_parts(p, part, &Pattern::tiles);
    p->tile_ent = dupload_parts(p, part, &Pattern::tile_ent);
    p->ent_pos = dupload_parts(p, part, &Pattern::ent_pos);
    p->ent_cb = dupload_parts(p, part, &Pattern::ent_cb);
    p->con_idx = dupload_parts(p, part, &Pattern::con_idx);
    p->con_coef = dupload_parts(p, part, &Pattern::con_coef);
    std::vector<Pattern>().swap(part);
    p->Td = dalloc<double>(p, te);
    p->Hd = dalloc<double>(p, he);
    p->Et = dalloc<double>(p, (long long)p->nl * p->B);
    p->SB = dalloc<double>(p, (long long)p->B * p->B);
    p->Td_asm = dalloc<double>(p, te);
    p->Hd_asm = dalloc<double>(p, he);
    p->Et_asm = dalloc<double>(p, (long long)p->nl * p->B);
    p->SB_asm = dalloc<double>(p, (long long)p->B * p->B);
    p->Td_diag0 = dalloc<double>(p, p->nl);
    p->Linv = dalloc<double>(p, te);
    p->Yf = dalloc<double>(p, he);
    p->Yb = dalloc<double>(p, he);
    p->chain_tmp = dalloc<double>(p, p->nl);
    p->td_off_d = dupload(p, p->td_off);
    p->h_off_d = dupload(p, p->h_off);
    {
      // chain segments: maximal runs of pairs that all have link rows
      std::vector<int> seg;
      for (int j = 0; j + 1 < N;) {
        if (l[j] == 0) {
          ++j;
          continue;
        }
        int e = j;
        while (e + 1 < N && l[e] > 0) ++e;
        seg.push_back(j);
        seg.push_back(e);
        j = e;
      }
      p->nchain_seg = (int)seg.size() / 2;
      if (!seg.empty()) p->chain_seg = dupload(p, seg);
      // cyclic-reduction schedule: in a segment of n pairs position i is
      // eliminated at level ctz(i + 1); per level the list of its pairs, per
      // pair its level and its segment
      {
        std::vector<int> info((size_t)4 * std::max(N - 1, 1), 0), lvl(std::max(N - 1, 1), -1);
        int nlev = 0;
        for (size_t sgi = 0; sgi < seg.size(); sgi += 2) {
          const int jb = seg[sgi], je = seg[sgi + 1];
          for (int j = jb; j < je; ++j) {
            int v = 0;
            while (((j - jb + 1) >> v & 1) == 0) ++v;
            lvl[j] = v;
            info[4 * j] = v;
            info[4 * j + 1] = jb;
            info[4 * j + 2] = je;
            nlev = std::max(nlev, v + 1);
          }
        }
        std::vector<int> order;
        p->bcr_loff.assign(1, 0);
        for (int v = 0; v < nlev; ++v) {
          for (int j = 0; j + 1 < N; ++j)
            if (lvl[j] == v) order.push_back(j);
          p->bcr_loff.push_back((int)order.size());
        }
        int lm = 0;
        for (int v : l) lm = std::max(lm, v);
        p->bcr_lmax = lm;
        if (!order.empty()) {
          p->bcr_order = dupload(p, order);
          p->bcr_info = dupload(p, info);
          p->bcr_GL = dalloc<double>(p, (long long)(N - 1) * lm * lm);
          p->bcr_GR = dalloc<double>(p, (long long)(N - 1) * lm * lm);
          ck(set_bcr_smem_limits(lm), "smem limit");
        }
      }
      // link-row range of each border column of Z = L_T^-1 E': all links for one
      // LP; in a batch, the links of the LP that owns the linking variable or
      // global row
      std::vector<int> zl(std::max(p->B, 1), 0), zh(std::max(p->B, 1), p->nl);
      if (p->batch > 1) {
        const int Bt = p->batch;
        for (int b = 0; b < Bt; ++b) {
          const long long blo = p->lp_blk0[b];
          const long long bhi = b + 1 < Bt ? p->lp_blk0[b + 1] : N;
          const int lo = (int)p->link_off[blo];
          const int hi = (int)(bhi - 1 < N - 1 ? p->link_off[bhi - 1] : p->nl);
          const long long x0hi = b + 1 < Bt ? p->lp_x0off[b + 1] : n0;
          const long long ghi = b + 1 < Bt ? p->lp_goff[b + 1] : mg;
          for (long long k = p->lp_x0off[b]; k < x0hi; ++k) zl[k] = lo, zh[k] = hi;
          for (long long k = p->lp_goff[b]; k < ghi; ++k) zl[n0 + k] = lo, zh[n0 + k] = hi;
        }
      }
      p->zlo = dupload(p, zl);
      p->zhi = dupload(p, zh);
    }
    p->l_d = dupload(p, l);
    p->link_off_d = dupload(p, p->link_off);
    p->kmap = dupload(p, kmap);
    p->kmap_off_d = dupload(p, p->kmap_off);
    p->link_pair_d = dupload(p, link_pair);
    p->yoff_d = dupload(p, p->yoff);
    p->f0_idx = dupload(p, f0i);
    p->f0_val = dupload(p, f0v);
    p->fg0_idx = dupload(p, fg0i);
    p->fg0_val = dupload(p, fg0v);
    p->border = dalloc<double>(p, (long long)p->Bld * std::max(p->B, 1));
    p->bx_info = dupload(p, std::vector<BlkInfo>(1, p->h_bx));
    p->bp_info = dupload(p, std::vector<BlkInfo>(1, p->h_bp));
    p->border_diag0 = dalloc<double>(p, p->B);
    p->x = dalloc<double>(p, p->n);
    p->z = dalloc<double>(p, p->n);
    p->dscale = dalloc<double>(p, p->n);
    p->xinv = dalloc<double>(p, p->n);
    p->wfin = dalloc<double>(p, p->n);
    p->vec = dalloc<double>(p, p->vec_elems);
    p->svec = dalloc<double>(p, p->nS);
    p->f = dalloc<double>(p, p->n);
    p->g = dalloc<double>(p, std::max(p->n, p->m));
    p->rhat = dalloc<double>(p, p->m);
    const long long mx = std::max(p->n, p->m);
    for (auto &s : p->stg) s = dalloc<double>(p, mx);
    for (auto &s : p->res) s = dalloc<double>(p, mx);
    for (auto &s : p->cor) s = dalloc<double>(p, mx);
    for (auto &s : p->ipmv) s = dalloc<double>(p, mx);
    p->red_part = dalloc<double>(p, 1024);
    p->mdot_part = dalloc<double>(p, (long long)(kMaxKrylov + 1) * 304);
    p->gm_coef = dalloc<double>(p, kMaxKrylov + 1);
    p->gm_h = dalloc<double>(p, 2 * (kMaxKrylov + 1) + 1);
    p->scal = dalloc<double>(p, 64);
    p->status = dalloc<int>(p, 8);
    ck(cudaMallocHost(&p->h_scal, 512 * sizeof(double)), "cudaMallocHost");
    for (auto &e : p->ev) ck(cudaEventCreate(&e), "cudaEventCreate");
    ck(set_dense_smem_limits((int)kSmemVecBytes), "smem limit");
    ck(set_schur_smem_limits(128 * 128 * 8), "smem limit");
    ck(cudaDeviceSynchronize(), "create sync");
  } catch (const Fail &f) {
    g_create_err = f.msg;
    arrowhead_lp_destroy(p);
    return f.code;
  } catch (const std::bad_alloc &) {
    g_create_err = "host allocation failed";
    arrowhead_lp_destroy(p);
    return AHLP_ERR_OOM;
  } catch (const std::exception &e) {
    g_create_err = std::string("create: ") + e.what();
    arrowhead_lp_destroy(p);
    return AHLP_ERR_INVALID_ARG;
  }
  *out = p;
  return AHLP_OK;
}

}  // extern "C"

// ===========================================================================
// helpers for the compute entry points
// ===========================================================================
namespace ahlp {

void *dalloc_bytes(ahlp_problem *p, size_t bytes) {
  return dalloc<unsigned char>(p, (long long)std::max<size_t>(bytes, 1));
}

void *dupload_bytes(ahlp_problem *p, const void *h, size_t bytes) {
  void *d = dalloc_bytes(p, bytes);
  if (bytes) {
    cudaError_t e = cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice);
    p->bytes_h2d += (long long)bytes;
    if (e != cudaSuccess) fail(AHLP_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  return d;
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void ck(cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Fail{AHLP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

bool is_device_ptr(const void *ptr) {
  if (!ptr) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// device view of an input vector (copied into staging when it is on the host)
const double *stage_in(ahlp_problem *p, const double *v, long long n, double *staging) {
  if (is_device_ptr(v)) return v;
  if (n > 0) ck(cudaMemcpyAsync(staging, v, n * 8, cudaMemcpyHostToDevice, p->stream), "H2D");
  p->bytes_h2d += n * 8;
  return staging;
}

int set_err(ahlp_problem *p, int code, const std::string &msg) {
  p->err = msg;
  return code;
}

// read k device scalars into p->h_scal (synchronises the stream)
void read_scalars(ahlp_problem *p, int k) {
  p->bytes_d2h += k * (long long)sizeof(double);
  ck(cudaMemcpyAsync(p->h_scal, p->scal, k * sizeof(double), cudaMemcpyDeviceToHost, p->stream),
     "D2H scalars");
  ck(cudaStreamSynchronize(p->stream), "stream sync");
}

void kt_mark(ahlp_problem *p, int cls, cudaStream_t s) {
  const size_t i = p->kt_cls.size();
  if (i == p->kt_pool.size()) {
    cudaEvent_t e;
    ck(cudaEventCreate(&e), "event");
    p->kt_pool.push_back(e);
  }
  ck(cudaEventRecord(p->kt_pool[i], s), "event");
  p->kt_cls.push_back(cls);
}

void kt_collect(ahlp_problem *p) {
  for (int c = 0; c < 3; ++c) {
    p->kt_ms[c] = 0.0;
    p->kt_n[c] = 0;
  }
  for (size_t i = 0; i + 1 < p->kt_cls.size(); ++i) {
    const int c = p->kt_cls[i];
    if (c < 0 || c > 2) continue;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p->kt_pool[i], p->kt_pool[i + 1]) == cudaSuccess) {
      p->kt_ms[c] += ms;
      ++p->kt_n[c];
    }
  }
  p->kt_cls.clear();
}

int factor_impl(ahlp_problem *p, double delta, double rho, double pivot_tol, bool ff_nan_up) {
  // an FP32 pivot that lost six digits, a float-float one that lost eleven,
  // is rounding noise
  p->fac_pivot_tol = p->fac_prec == kPrecFP32 ? std::max(pivot_tol, kFp32PivotTol)
                     : p->fac_prec == kPrecFF ? std::max(pivot_tol, kFFPivotTol)
                                              : pivot_tol;
  if (p->fac_prec != kPrecFP64 && !p->aug32) {
    p->aug32 = dalloc<float>(p, p->aug_elems);
    p->tinv32 = dalloc<float>(p, std::max(p->tinv_elems, 1LL));
    p->vec32 = dalloc<float>(p, std::max(p->vec_elems, 1LL));
  }
  if (p->fac_prec == kPrecFF && !p->aug_lo) p->aug_lo = dalloc<float>(p, p->aug_elems);
  if (p->fac_prec != kPrecFP32 && !p->aug) {
    p->aug = dalloc<double>(p, p->aug_elems);
    p->tinv = dalloc<double>(p, std::max(p->tinv_elems, 1LL));
  }
  cudaStream_t s = p->stream;
  // strictly positive point required (Sec. 2.3: x, z > 0)
  ck(launch_reduce(p, RED_MIN, p->x, nullptr, p->n, p->scal + 0), "reduce");
  ck(launch_reduce(p, RED_MIN, p->z, nullptr, p->n, p->scal + 1), "reduce");
  read_scalars(p, 2);
  if (p->n > 0 && (!(p->h_scal[0] > 0) || !(p->h_scal[1] > 0)))
    return set_err(p, AHLP_ERR_INVALID_ARG, "kkt_factor: x and z must be strictly positive");
  p->factored = false;
  p->fac_delta = delta;
  p->fac_rho = rho;
  ck(cudaMemsetAsync(p->status, 0, 8 * sizeof(int), s), "memset");
  ck(cudaEventRecord(p->ev[0], s), "event");
  ck(cudaMemsetAsync(p->cdiag0, 0, std::max(p->cdiag_elems, 1LL) * sizeof(double), s), "memset");
  ck(launch_dscale(p), "dscale");
  if (p->fac_prec == kPrecFP32 && p->n > 0) {
    // adaptive precision: once D = X Z^-1 spans more than fp32_cond_max the
    // block normal matrices are too ill-conditioned for FP32 factors, and the
    // factor moves to float-float
    ck(launch_reduce(p, RED_MAXABS, p->dscale, nullptr, p->n, p->scal + 2), "reduce");
    ck(launch_reduce(p, RED_MIN, p->dscale, nullptr, p->n, p->scal + 3), "reduce");
    p->bytes_d2h += 2 * sizeof(double);
    ck(cudaMemcpyAsync(p->h_scal + 2, p->scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s),
       "D2H");
    ck(cudaStreamSynchronize(s), "sync");
    if (!(p->h_scal[2] <= p->opt.fp32_cond_max * p->h_scal[3])) {
      if (p->opt.verbose)
        printf("D spans %.2e > fp32_cond_max: block factors move to float-float\n",
               p->h_scal[2] / p->h_scal[3]);
      p->fac_prec = kPrecFF;
      return factor_impl(p, delta, rho, pivot_tol, ff_nan_up);
    }
  }
  ck(launch_form(p, delta), "form");
  ck(cudaEventRecord(p->ev[1], s), "event");
  ahlp_problem *prof = p->opt.profile_kernels ? p : nullptr;
  const bool drop = p->opt.pivot_mode == 1;
  p->kt_cls.clear();
  if (p->fac_prec == kPrecFP32) {
    // trailing updates on the tensor cores unless the FP32 pipe is asked for
    ahlp_problem *tc = nullptr;
    if (p->opt.fp32_update != 1) {
      if (tc_setup(p))
        tc = p;
      else if (p->opt.fp32_update >= 2)
        return set_err(p, AHLP_ERR_UNSUPPORTED,
                       "kkt_factor: tensor-core update requested, but the driver cannot "
                       "encode tensor maps");
    }
    p->fp32_update = tc ? (p->opt.fp32_update == 3 ? 3 : 2) : 1;
    ck(launch_pchol_f32(p->aug32, p->tinv32, p->blk, p->h_blk, p->diag0, p->fac_pivot_tol,
                        p->status, s, tc, prof, drop ? kDropFP32 : 0.0),
       "pchol");
  }
  else if (p->fac_prec == kPrecFF) {
    ahlp_problem *oz = (p->opt.ff_update != 1 && oz_setup(p)) ? p : nullptr;
    p->ff_update = oz ? (p->opt.ff_update == 3 ? 3 : 2) : 1;
    ck(launch_pchol_ff(p->aug32, p->aug_lo, p->aug, p->aug_elems, p->blk, p->h_blk, p->diag0,
                       p->fac_pivot_tol, p->status, s, oz, prof, drop ? kDropFF : 0.0),
       "pchol");
  }
  else
    ck(launch_pchol(p->aug, p->blk, p->h_blk, p->diag0, p->fac_pivot_tol, p->status, s, prof,
                    drop ? kDropFP64 : 0.0),
       "pchol");
  ck(launch_tinv(p), "diagonal tile inverses");
  ck(cudaEventRecord(p->ev[2], s), "event");
  ck(launch_schur_assemble(p, delta, rho), "schur assemble");
  p->assembled = true;
  ck(launch_schur_factor(p), "schur factor");
  ck(cudaEventRecord(p->ev[3], s), "event");
  int st[8];
  p->bytes_d2h += sizeof(st);
  ck(cudaMemcpyAsync(st, p->status, sizeof(st), cudaMemcpyDeviceToHost, s), "D2H status");
  ck(cudaStreamSynchronize(s), "factor sync");
  cudaEventElapsedTime(&p->stage_ms[0], p->ev[0], p->ev[1]);
  cudaEventElapsedTime(&p->stage_ms[1], p->ev[1], p->ev[2]);
  cudaEventElapsedTime(&p->stage_ms[2], p->ev[2], p->ev[3]);
  if (prof) kt_collect(p);
  p->tiny_pivots = st[1];
  if (st[4] != 0)
    return set_err(p, AHLP_ERR_TIMEOUT,
                   "kkt_factor: a bounded wait of the tensor-core update ran out");
  if (st[0] > 0) {
    char buf[160];
    if (st[2] >= kTagBorderG)
      snprintf(buf, sizeof buf, "kkt_factor: NaN pivot in the border (global row %d)", st[3]);
    else if (st[2] >= kTagBorderX)
      snprintf(buf, sizeof buf, "kkt_factor: NaN pivot in the border (linking variable %d)",
               st[3]);
    else if (st[2] >= 0)
      snprintf(buf, sizeof buf, "kkt_factor: NaN pivot in block %d row %d", st[2], st[3]);
    else
      snprintf(buf, sizeof buf, "kkt_factor: NaN pivot in link pair %d row %d", -1 - st[2], st[3]);
    if (p->fac_prec == kPrecFP32 || (p->fac_prec == kPrecFF && ff_nan_up)) {
      // range or accuracy exceeded: one precision up
      const int up = p->fac_prec == kPrecFP32 ? kPrecFF : kPrecFP64;
      if (p->opt.verbose)
        printf("%s with %s block factors; refactoring in %s\n", buf,
               p->fac_prec == kPrecFP32 ? "FP32" : "float-float", up == kPrecFF ? "float-float" : "FP64");
      p->fac_prec = up;
      return factor_impl(p, delta, rho, pivot_tol, ff_nan_up);
    }
    return set_err(p, AHLP_ERR_NOT_SPD, buf);
  }
  p->factored = true;
  return AHLP_OK;
}

// one solve + refinement, all arguments device pointers
int solve_impl(ahlp_problem *p, const double *rd, const double *rp, const double *rc, double *dx,
               double *dy, double *dz, bool adjoint, ahlp_solve_info *info, double tol_override) {
  cudaStream_t s = p->stream;
  ck(cudaEventRecord(p->ev[4], s), "event");
  ck(cudaMemsetAsync(p->trsv_err, 0, sizeof(int), s), "memset");
  ck(launch_solve(p, rd, rp, rc, dx, dy, dz, adjoint), "solve");
  ck(launch_reduce(p, RED_DOT, rd, rd, p->n, p->scal + 10), "reduce");
  ck(launch_reduce(p, RED_DOT, rp, rp, p->m, p->scal + 11), "reduce");
  ck(launch_reduce(p, RED_DOT, rc, rc, p->n, p->scal + 12), "reduce");
  const long long n = p->n, m = p->m, L = 2 * n + m;
  // e = r - J d; returns (||e||, ||r||)
  auto residual_norms = [&]() {
    ck(launch_residual(p, rd, rp, rc, dx, dy, dz, p->res[0], p->res[1], p->res[2], adjoint),
       "residual");
    ck(launch_reduce(p, RED_DOT, p->res[0], p->res[0], n, p->scal + 13), "reduce");
    ck(launch_reduce(p, RED_DOT, p->res[1], p->res[1], m, p->scal + 14), "reduce");
    ck(launch_reduce(p, RED_DOT, p->res[2], p->res[2], n, p->scal + 15), "reduce");
    p->bytes_d2h += 6 * sizeof(double);
    ck(cudaMemcpyAsync(p->h_scal + 10, p->scal + 10, 6 * sizeof(double), cudaMemcpyDeviceToHost, s),
       "D2H");
    ck(cudaStreamSynchronize(s), "sync");
    return std::make_pair(std::sqrt(p->h_scal[13] + p->h_scal[14] + p->h_scal[15]),
                          std::sqrt(p->h_scal[10] + p->h_scal[11] + p->h_scal[12]));
  };
  auto [en, rn] = residual_norms();
  double rel = rn > 0 ? en / rn : en;
  int steps = 0;
  const double tol = tol_override > 0 ? tol_override : p->opt.refine_tol;
  const int kmax = std::min(p->opt.refine_max, kMaxKrylov);
  // Right-preconditioned FGMRES on the unregularised Newton system: the
  // (regularised) block factorisation is the preconditioner, so the result
  // solves J d = r itself, not the regularised system.  The cycle's own
  // residual estimate can run ahead of the true residual when the
  // preconditioned vectors are badly scaled; the true residual is then
  // recomputed and, while it is above the target, another cycle starts from
  // it (restarted FGMRES, refine_max steps in all), as long as each cycle at
  // least halves it.
  for (double prev = rel; rel > tol && steps < kmax && en > 0 && std::isfinite(en);) {
    const int kc = kmax - steps;
    if (p->gm_cap < kmax) {
      if (p->gm_V) cudaFree(p->gm_V);
      if (p->gm_Z) cudaFree(p->gm_Z);
      p->gm_V = p->gm_Z = nullptr;
      p->gm_cap = 0;
      ck(cudaMalloc(&p->gm_V, (size_t)(kmax + 1) * L * sizeof(double)), "Krylov alloc");
      ck(cudaMalloc(&p->gm_Z, (size_t)kmax * L * sizeof(double)), "Krylov alloc");
      p->gm_cap = kmax;
    }
    double *V = p->gm_V, *Z = p->gm_Z;
    double *cbuf = p->h_scal + 64, *hcol = p->h_scal + 256;
    ck(cudaMemcpyAsync(V, p->res[0], n * 8, cudaMemcpyDeviceToDevice, s), "copy");
    ck(cudaMemcpyAsync(V + n, p->res[1], m * 8, cudaMemcpyDeviceToDevice, s), "copy");
    ck(cudaMemcpyAsync(V + n + m, p->res[2], n * 8, cudaMemcpyDeviceToDevice, s), "copy");
    ck(launch_axpby(V, V, 1.0 / en, 0.0, L, s), "scale");
    std::vector<double> H((size_t)(kc + 1) * kc, 0.0), cs(kc), sn(kc), g(kc + 1, 0.0);
    g[0] = en;
    int j = 0;
    for (; j < kc;) {
      double *Vj = V + (long long)j * L, *Zj = Z + (long long)j * L, *W = V + (long long)(j + 1) * L;
      ck(launch_solve(p, Vj, Vj + n, Vj + n + m, Zj, Zj + n, Zj + n + m, adjoint), "precond");
      ck(launch_jmul(p, Zj, Zj + n, Zj + n + m, W, W + n, W + n + m, adjoint), "jmul");
      double *h = &H[(size_t)j * (kc + 1)];
      // classical Gram-Schmidt, twice, and the normalisation, all on the
      // device (the coefficients never leave it in between); the host reads
      // the column once per step, for the Givens update and the stopping test
      const int nh = j + 1;
      double *gh = p->gm_h;
      ck(launch_mdot(p, V, L, nh, W, L, gh), "mdot");
      ck(launch_maxpy(V, L, nh, gh, W, L, s, -1.0), "maxpy");
      ck(launch_mdot(p, V, L, nh, W, L, gh + nh), "mdot");
      ck(launch_maxpy(V, L, nh, gh + nh, W, L, s, -1.0), "maxpy");
      ck(launch_reduce(p, RED_DOT, W, W, L, gh + 2 * nh), "reduce");
      ck(launch_scale_inv_norm(W, L, gh + 2 * nh, s), "scale");
      p->bytes_d2h += (2 * nh + 1) * 8;
      ck(cudaMemcpyAsync(hcol, gh, (2 * nh + 1) * 8, cudaMemcpyDeviceToHost, s), "D2H");
      ck(cudaStreamSynchronize(s), "sync");
      for (int i = 0; i <= j; ++i) h[i] = (h[i] + hcol[i]) + hcol[nh + i];
      const double hn = std::sqrt(hcol[2 * nh]);
      h[j + 1] = hn;
      for (int i = 0; i < j; ++i) {   // previous Givens rotations
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
      }
      const double rr = std::hypot(h[j], h[j + 1]);
      cs[j] = rr > 0 ? h[j] / rr : 1.0;
      sn[j] = rr > 0 ? h[j + 1] / rr : 0.0;
      h[j] = rr;
      h[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++j;
      if (p->opt.verbose >= 2)
        printf("         krylov step %d  residual estimate %.3e\n", steps + j,
               std::fabs(g[j]) / (rn > 0 ? rn : 1.0));
      if (!(std::fabs(g[j]) > tol * rn) || !(hn > 1e-300 * en)) break;
    }
    // y = R^-1 g, d += Z y
    std::vector<double> y(j, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k < j; ++k) t -= H[(size_t)k * (kc + 1) + i] * y[k];
      const double d = H[(size_t)i * (kc + 1) + i];
      y[i] = d != 0.0 ? t / d : 0.0;
    }
    for (int i = 0; i < j; ++i) cbuf[i] = y[i];
    p->bytes_h2d += j * 8;
    ck(cudaMemcpyAsync(p->gm_coef, cbuf, j * 8, cudaMemcpyHostToDevice, s), "H2D");
    ck(launch_maxpy(Z, L, j, p->gm_coef, dx, n, s), "maxpy");
    ck(launch_maxpy(Z + n, L, j, p->gm_coef, dy, m, s), "maxpy");
    ck(launch_maxpy(Z + n + m, L, j, p->gm_coef, dz, n, s), "maxpy");
    steps += j;
    std::tie(en, rn) = residual_norms();
    rel = rn > 0 ? en / rn : en;
    if (!(rel <= 0.5 * prev)) break;
    prev = rel;
  }
  ck(cudaEventRecord(p->ev[5], s), "event");
  int timed_out = 0;
  p->bytes_d2h += sizeof(int);
  ck(cudaMemcpyAsync(&timed_out, p->trsv_err, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H");
  ck(cudaEventSynchronize(p->ev[5]), "sync");
  ck(cudaStreamSynchronize(s), "sync");
  cudaEventElapsedTime(&p->stage_ms[3], p->ev[4], p->ev[5]);
  if (timed_out)
    return set_err(p, AHLP_ERR_TIMEOUT, "kkt_solve: a block-solve wait exceeded its time limit");
  if (info) {
    info->refine_steps = steps;
    info->rel_residual = rel;
  }
  if (!(rel == rel)) return set_err(p, AHLP_ERR_NOT_SPD, "kkt_solve: NaN in the direction");
  return AHLP_OK;
}

}  // namespace ahlp

extern "C" {

int kkt_factor(ahlp_problem *p, const double *x, const double *z, double delta, double rho) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  if (!x || !z) return set_err(p, AHLP_ERR_INVALID_ARG, "kkt_factor: x and z are required");
  try {
    const double *dx = stage_in(p, x, p->n, p->stg[0]);
    const double *dz = stage_in(p, z, p->n, p->stg[1]);
    // rho regularises every primal variable: D^-1 + rho on the blocks (through
    // d = x / (z + rho x)) and on the linking variables (in the Schur border)
    const double r = rho < 0 ? p->opt.rho : rho;
    p->fac_rho_x = r > 0 ? r : 0.0;
    if (p->n > 0) {
      ck(cudaMemcpyAsync(p->x, dx, p->n * 8, cudaMemcpyDeviceToDevice, p->stream), "copy x");
      ck(cudaMemcpyAsync(p->z, dz, p->n * 8, cudaMemcpyDeviceToDevice, p->stream), "copy z");
    }
    p->fac_prec = p->opt.precision == AHLP_PREC_MIXED ? kPrecFP32 : kPrecFP64;
    return factor_impl(p, delta < 0 ? p->opt.delta : delta, rho < 0 ? p->opt.rho : rho,
                       p->opt.pivot_tol);
  } catch (const Fail &f) {
    return set_err(p, f.code, f.msg);
  }
}

static int solve_entry(ahlp_problem *p, const double *a, const double *b, const double *c,
                       double *o1, double *o2, double *o3, ahlp_solve_info *info, bool adjoint) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  if (!p->factored) return set_err(p, AHLP_ERR_INVALID_ARG, "no factor: call kkt_factor first");
  if (!a || !b || !c || !o1 || !o2 || !o3)
    return set_err(p, AHLP_ERR_INVALID_ARG, "NULL vector argument");
  try {
    const double *da = stage_in(p, a, p->n, p->stg[0]);
    const double *db = stage_in(p, b, p->m, p->stg[1]);
    const double *dc = stage_in(p, c, p->n, p->stg[2]);
    const bool d1 = is_device_ptr(o1), d2 = is_device_ptr(o2), d3 = is_device_ptr(o3);
    double *w1 = d1 ? o1 : p->stg[3], *w2 = d2 ? o2 : p->stg[4], *w3 = d3 ? o3 : p->stg[5];
    int st = solve_impl(p, da, db, dc, w1, w2, w3, adjoint, info);
    if (!d1) ck(cudaMemcpyAsync(o1, w1, p->n * 8, cudaMemcpyDeviceToHost, p->stream), "D2H");
    if (!d2) ck(cudaMemcpyAsync(o2, w2, p->m * 8, cudaMemcpyDeviceToHost, p->stream), "D2H");
    if (!d3) ck(cudaMemcpyAsync(o3, w3, p->n * 8, cudaMemcpyDeviceToHost, p->stream), "D2H");
    p->bytes_d2h += (d1 ? 0 : p->n * 8) + (d2 ? 0 : p->m * 8) + (d3 ? 0 : p->n * 8);
    if (!(d1 && d2 && d3)) ck(cudaStreamSynchronize(p->stream), "sync");
    return st;
  } catch (const Fail &f) {
    return set_err(p, f.code, f.msg);
  }
}

int kkt_solve(ahlp_problem *p, const double *r_d, const double *r_p, const double *r_c,
              double *dx, double *dy, double *dz, ahlp_solve_info *info) {
  return solve_entry(p, r_d, r_p, r_c, dx, dy, dz, info, false);
}

int kkt_adjoint_solve(ahlp_problem *p, const double *g_x, const double *g_y, const double *g_z,
                      double *lam_x, double *lam_y, double *lam_z, ahlp_solve_info *info) {
  return solve_entry(p, g_x, g_y, g_z, lam_x, lam_y, lam_z, info, true);
}

int kkt_schur_dense(ahlp_problem *p, double *S, int64_t ld) {
  if (!p || !S) return AHLP_ERR_INVALID_ARG;
  if (!p->assembled)
    return set_err(p, AHLP_ERR_INVALID_ARG, "no Schur complement: call kkt_factor first");
  const int dim = p->nS;
  if (ld < dim) return set_err(p, AHLP_ERR_INVALID_ARG, "ld < dimension");
  try {
    std::vector<double> Td(p->td_elems), Hd(p->h_elems), Et((size_t)p->nl * p->B),
        SB((size_t)p->B * p->B);
    ck(cudaStreamSynchronize(p->stream), "sync");
    if (!Td.empty()) ck(cudaMemcpy(Td.data(), p->Td_asm, Td.size() * 8, cudaMemcpyDeviceToHost), "D2H");
    if (!Hd.empty()) ck(cudaMemcpy(Hd.data(), p->Hd_asm, Hd.size() * 8, cudaMemcpyDeviceToHost), "D2H");
    if (!Et.empty()) ck(cudaMemcpy(Et.data(), p->Et_asm, Et.size() * 8, cudaMemcpyDeviceToHost), "D2H");
    if (!SB.empty()) ck(cudaMemcpy(SB.data(), p->SB_asm, SB.size() * 8, cudaMemcpyDeviceToHost), "D2H");
    for (long long cidx = 0; cidx < dim; ++cidx)
      for (long long r = 0; r < dim; ++r) S[cidx * ld + r] = 0.0;
    for (int j = 0; j + 1 < p->N; ++j) {
      const int lj = (int)(p->link_off[j + 1] - p->link_off[j]);
      const long long o = p->link_off[j];
      for (int s = 0; s < lj; ++s)
        for (int r = 0; r < lj; ++r) S[(o + s) * ld + o + r] = Td[p->td_off[j] + (long long)s * lj + r];
      if (j + 2 < p->N) {
        const int ln = (int)(p->link_off[j + 2] - p->link_off[j + 1]);
        const long long on = p->link_off[j + 1];
        for (int s = 0; s < lj; ++s)
          for (int r = 0; r < ln; ++r) {
            const double v = Hd[p->h_off[j] + (long long)s * ln + r];
            S[(o + s) * ld + on + r] = v;
            S[(on + r) * ld + o + s] = v;
          }
      }
    }
    for (int rb = 0; rb < p->B; ++rb) {
      for (int q = 0; q < p->nl; ++q) {
        const double v = Et[(size_t)rb * p->nl + q];
        S[(long long)q * ld + p->nl + rb] = v;
        S[(long long)(p->nl + rb) * ld + q] = v;
      }
      for (int sb = 0; sb < p->B; ++sb) S[(long long)(p->nl + sb) * ld + p->nl + rb] = SB[(size_t)sb * p->B + rb];
    }
    return AHLP_OK;
  } catch (const Fail &f) {
    return set_err(p, f.code, f.msg);
  }
}

int64_t ahlp_launch_count(void) { return ahlp::launch_count(); }

int arrowhead_lp_autotune(ahlp_problem *p, const double *x, const double *z, double *ms6) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  const ahlp_options saved = p->opt;
  const int saved_prec = p->fac_prec;
  double best[6] = {0, 0, 0, 0, 0, 0};
  try {
    const double *xx = x ? stage_in(p, x, p->n, p->stg[0]) : nullptr;
    const double *zz = z ? stage_in(p, z, p->n, p->stg[1]) : nullptr;
    if (!xx || !zz) {
      ck(launch_fill(p->stg[0], 1.0, p->n, p->stream), "fill");
      xx = zz = p->stg[0];
    }
    ck(cudaMemcpyAsync(p->x, xx, p->n * 8, cudaMemcpyDeviceToDevice, p->stream), "copy");
    ck(cudaMemcpyAsync(p->z, zz, p->n * 8, cudaMemcpyDeviceToDevice, p->stream), "copy");
    // (precision, update option value) of the six candidates
    const int prec[6] = {kPrecFP32, kPrecFP32, kPrecFF, kPrecFF, kPrecFP32, kPrecFF};
    const int val[6] = {2, 1, 2, 1, 3, 3};
    for (int c = 0; c < 6; ++c) {
      p->opt = saved;
      p->opt.precision = AHLP_PREC_MIXED;
      p->opt.fp32_cond_max = prec[c] == kPrecFP32 ? 1e300 : 1.0;
      if (prec[c] == kPrecFP32) p->opt.fp32_update = val[c];
      else p->opt.ff_update = val[c];
      double t = 1e300;
      for (int rep = 0; rep < 3; ++rep) {
        p->fac_prec = prec[c];
        const int st = factor_impl(p, p->opt.delta, p->opt.rho, p->opt.pivot_tol);
        if (st != AHLP_OK) throw Fail{st, p->err};
        if (rep > 0) t = std::min(t, (double)p->stage_ms[1]);
      }
      best[c] = t;
    }
    p->opt = saved;
    p->opt.fp32_update = best[4] <= std::min(best[0], best[1]) ? 3 : best[0] <= best[1] ? 2 : 1;
    p->opt.ff_update = best[5] <= std::min(best[2], best[3]) ? 3 : best[2] <= best[3] ? 2 : 1;
    p->fac_prec = saved_prec;
    p->factored = false;
    if (ms6)
      for (int c = 0; c < 6; ++c) ms6[c] = best[c];
    return AHLP_OK;
  } catch (const Fail &f) {
    p->opt = saved;
    p->fac_prec = saved_prec;
    p->factored = false;
    return set_err(p, f.code, f.msg);
  }
}

int arrowhead_lp_original_size(const ahlp_problem *p, int64_t *n_orig) {
  if (!p || !n_orig) return AHLP_ERR_INVALID_ARG;
  long long n = 0;
  for (auto &r : p->lp_recov) {
    for (int v : r.n_orig) n += v;
    n += r.n0_orig;
  }
  *n_orig = n;
  return AHLP_OK;
}

int arrowhead_lp_recover(ahlp_problem *p, const double *x, double *x_orig, double *obj_offset) {
  if (!p || !x || !x_orig) return AHLP_ERR_INVALID_ARG;
  try {
    std::vector<double> xs(p->n);
    if (p->n > 0) {
      const bool dev = is_device_ptr(x);
      ck(cudaMemcpyAsync(xs.data(), x, p->n * 8, dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                         p->stream),
         "copy");
      ck(cudaStreamSynchronize(p->stream), "sync");
    }
    // standard-form offsets of every LP's blocks and linking variables
    long long norig = 0, n0orig_total = 0;
    for (auto &r : p->lp_recov) {
      for (int v : r.n_orig) norig += v;
      n0orig_total += r.n0_orig;
    }
    std::vector<double> xo(norig + n0orig_total, 0.0);
    long long blk = 0, ob = 0, o0 = norig, x0s = 0;
    double off = 0.0;
    const long long x0base = p->xoff[p->N];
    for (size_t b = 0; b < p->lp_recov.size(); ++b) {
      const auto &r = p->lp_recov[b];
      const int Nb = (int)r.n_orig.size();
      std::vector<long long> obase(Nb);
      for (int i = 0; i < Nb; ++i) {
        obase[i] = ob;
        ob += r.n_orig[i];
      }
      const long long n0std = b + 1 < p->lp_recov.size()
                                  ? (p->batch > 1 ? p->lp_x0off[b + 1] : p->n0) - x0s
                                  : p->n0 - x0s;
      if (r.recov.empty()) {   // already in equality form: copied as it is
        for (int i = 0; i < Nb; ++i)
          for (int t = 0; t < r.n_orig[i]; ++t) xo[obase[i] + t] = xs[p->xoff[blk + i] + t];
        for (int t = 0; t < r.n0_orig; ++t) xo[o0 + t] = xs[x0base + x0s + t];
      } else {
        for (const auto &q : r.recov) {
          const long long base = q.blk >= 0 ? p->xoff[blk + q.blk] : x0base + x0s;
          double v = q.shift + q.sign * xs[base + q.k];
          if (q.k2 >= 0) v -= xs[base + q.k2];
          if (q.blk >= 0) xo[obase[q.blk] + q.orig] = v;
          else xo[o0 + q.orig] = v;
        }
        off += r.const_obj;
      }
      blk += Nb;
      o0 += r.n0_orig;
      x0s += n0std;
    }
    const bool dev = is_device_ptr(x_orig);
    ck(cudaMemcpyAsync(x_orig, xo.data(), xo.size() * 8,
                       dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, p->stream),
       "copy");
    ck(cudaStreamSynchronize(p->stream), "sync");
    if (obj_offset) *obj_offset = off;
    return AHLP_OK;
  } catch (const Fail &f) {
    return set_err(p, f.code, f.msg);
  }
}

int kkt_factor_kernel_times(const ahlp_problem *p, double *ms3, int64_t *launches3) {
  if (!p || !ms3) return AHLP_ERR_INVALID_ARG;
  for (int c = 0; c < 3; ++c) {
    ms3[c] = p->kt_ms[c];
    if (launches3) launches3[c] = p->kt_n[c];
  }
  return AHLP_OK;
}

int kkt_update_jobs(const ahlp_problem *p, int64_t *kept, int64_t *dense) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  if (kept) *kept = p->tc_jobs_kept;
  if (dense) *dense = p->tc_jobs_dense;
  return AHLP_OK;
}

int ahlp_transfer_bytes(const ahlp_problem *p, int64_t *h2d, int64_t *d2h) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  if (h2d) *h2d = p->bytes_h2d;
  if (d2h) *d2h = p->bytes_d2h;
  return AHLP_OK;
}

int kkt_block_factor_dense(ahlp_problem *p, int32_t block, double *A, int64_t ld,
                           int32_t *order) {
  if (!p || !A) return AHLP_ERR_INVALID_ARG;
  if (!p->assembled)
    return set_err(p, AHLP_ERR_INVALID_ARG, "no factor: call kkt_factor first");
  if (block < 0 || block >= p->N) return set_err(p, AHLP_ERR_INVALID_ARG, "block out of range");
  const BlkInfo &bi = p->h_blk[block];
  if (order) *order = bi.a;
  if (ld < bi.a) return set_err(p, AHLP_ERR_INVALID_ARG, "ld < order");
  try {
    ck(cudaStreamSynchronize(p->stream), "sync");
    const size_t cnt = (size_t)bi.lda * bi.a;
    std::vector<double> h(cnt);
    if (p->fac_prec == kPrecFP32) {
      std::vector<float> hf(cnt);
      if (cnt) ck(cudaMemcpy(hf.data(), p->aug32 + bi.base, cnt * 4, cudaMemcpyDeviceToHost), "D2H");
      for (size_t i = 0; i < cnt; ++i) h[i] = hf[i];
    } else if (cnt) {   // FP64, or the FP64 copy of a float-float factor
      ck(cudaMemcpy(h.data(), p->aug + bi.base, cnt * 8, cudaMemcpyDeviceToHost), "D2H");
    }
    for (long long c = 0; c < bi.a; ++c)
      for (long long r = 0; r < bi.a; ++r) A[c * ld + r] = r >= c ? h[c * bi.lda + r] : 0.0;
    if (order) *order = bi.a;
    return AHLP_OK;
  } catch (const Fail &f) {
    return set_err(p, f.code, f.msg);
  }
}

int kkt_stage_times(ahlp_problem *p, double *out4) {
  if (!p || !out4) return AHLP_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i) out4[i] = p->stage_ms[i];
  return AHLP_OK;
}

}  // extern "C"
