// Internal declarations shared by the host runtime and the kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/ahlp.h"

namespace ahlp {

constexpr int NB = 64;            // tile edge of the dense kernels
constexpr int kPrecFP64 = 0;      // factor storage of the block matrices
constexpr int kPrecFP32 = 1;
// float-float: value = hi + lo with two FP32 arrays (aug32 = hi, aug_lo = lo);
// the factorisation runs in double-float arithmetic on the FP32 pipe (about
// 46 significant bits); the finished factor is expanded into the FP64 buffer,
// which the Schur assembly and the solves read as for an FP64 factor
constexpr int kPrecFF = 2;
constexpr double kFp32PivotTol = 1e-6;    // smallest clamp threshold for FP32 pivots
constexpr double kFFPivotTol = 1e-12;     // smallest clamp threshold for float-float pivots
// pivot_mode 1: a failing pivot becomes scale * max(its starting diagonal, 1),
// capped so that its square root and reciprocal stay normal in the factor's
// storage words
constexpr double kDropFP64 = 1e32, kDropFF = 1e16, kDropFP32 = 1e16;
constexpr double kDropCapFF = 1e60, kDropCapFP32 = 1e30;
constexpr long long kSmemVecBytes = 160 * 1024;   // dynamic smem of the border solves
constexpr int kThreads = 256;     // threads per CTA of the dense kernels

// One dense lower-triangular "partial Cholesky" problem: an a x a matrix
// (column-major, leading dimension lda, element offset base) whose first p
// pivots are eliminated.  After the factorisation the (p..a) x (p..a) corner
// holds the Schur complement of the leading p x p block.
// CSR matrix on the device with its rows binned by length: rows up to
// kShortRow nonzeros go to 8-lane groups, the rest (the dense linking-variable
// rows of A') to one CTA each.
constexpr int kShortRow = 256;
struct SpMat {
  const int *rp = nullptr, *ci = nullptr;
  const double *v = nullptr;
  long long rows = 0;
  const int *long_rows = nullptr;   // [n_long] rows with more than kShortRow nonzeros
  int n_long = 0;
};

struct BlkInfo {
  long long base;    // offset of element (0,0) in its buffer
  long long voff;    // offset of this problem's vector segment in solve vectors
  long long d0off;   // offset of its original diagonal in the diag0 array
  int lda, a, p;
  int T, Tp;         // tiles of a, tiles holding pivots
  int tag;           // added to the problem index in pivot reports (kTag*)
  long long cdoff;   // offset of the corner (non-pivot) diagonal in cdiag0
  long long ioff;    // offset of its Tp inverted diagonal tiles (block solves)
  long long soff;    // first staging slot of its panel tiles (tensor-core update)
};
constexpr int kTagBorderX = 1 << 20;   // pivot reports of the border x_0 factor
constexpr int kTagBorderG = 2 << 20;   // pivot reports of the border y_g factor

#ifdef __CUDACC__
// Pivot safeguard shared by every Cholesky in the library.  A pivot that is
// not above tol * (the diagonal entry it started from) has lost all its
// significant digits to cancellation.  It is clamped to that threshold, which
// keeps the factor nonsingular (the Krylov refinement of kkt_solve then
// corrects the solve against the exact Newton matrix); or, with drop > 0, it
// becomes drop * max(orig, 1) (at most cap), which leaves the row out of the
// factor: its column below the pivot and its solution entry come out ~0, the
// treatment of nearly dependent rows of A D A' in interior-point codes.  NaN
// pivots are counted in status[0] with the first location, failing pivots in
// status[1].
__device__ __forceinline__ void pivot_fix(double &piv, double orig, double tol, int *status,
                                          int where, int row, double drop = 0.0,
                                          double cap = 1e300) {
  const double floor_v = tol * orig > 0.0 ? tol * orig : 1.0;
  const double repl = drop > 0.0 ? fmin(drop * fmax(orig, 1.0), cap) : floor_v;
  if (!(piv == piv)) {
    if (atomicAdd(&status[0], 1) == 0) {
      status[2] = where;
      status[3] = row;
    }
    piv = repl;
  } else if (!(piv > tol * orig) || !(piv > 0.0)) {
    atomicAdd(&status[1], 1);
    piv = repl;
  }
}
#endif

// One formation tile: block, tile row, tile column.
struct FormTile {
  int blk, I, J, pad;
};

// Per-block layout of the local Schur columns k_i = n0 + lprev + lnext + mg.
struct SchurBlk {
  int m;       // pivots (rows of A_i)
  int k;       // local Schur columns: [x_0 slice | links i-1 | links i | global-row slice]
  int lprev, lnext;
  int link_prev_off, link_next_off;   // offsets of pairs i-1 and i in the link block
  int x0lo, x0n;   // the block's slice of the linking variables (all of them for one LP;
  int glo, gn;     // its LP's ones in a batch) and of the global rows
};

// A sparse matrix assembled column by column (host), and the equality-form
// description of an LP given in the full statement (general.cpp), with the
// map back to its original variables.
struct StdCsc {
  using Entry = std::pair<int, double>;   // (row, value)
  using Col = std::vector<Entry>;
  int m = 0;
  std::vector<int32_t> cp{0}, ri;
  std::vector<double> v;
  void push(const Col &c) {
    for (auto &e : c) {
      ri.push_back(e.first);
      v.push_back(e.second);
    }
    cp.push_back((int32_t)ri.size());
  }
  int n() const { return (int)cp.size() - 1; }
  ahlp_csc csc() const {
    return ahlp_csc{m, n(), cp.data(), ri.empty() ? nullptr : ri.data(),
                    v.empty() ? nullptr : v.data()};
  }
};

struct StdDesc {
  // original variable `orig` of block blk (-1: of x_0) = shift + sign x'_k
  // (- x'_k2 when k2 >= 0), k and k2 indices among its block's (x_0's)
  // standard-form columns
  struct Recov {
    int blk, orig;
    double shift;
    int k;
    double sign;
    int k2;
  };
  int N = 0;
  std::vector<StdCsc> A, W, Fg, FL, FR, F0;
  StdCsc Fg0;
  std::vector<std::vector<double>> b, c, blink;
  std::vector<double> bg, c0;
  std::vector<int32_t> l;
  std::vector<ahlp_csc> Ac, Wc, Fgc, FLc, FRc, F0c;
  ahlp_csc Fg0c{};
  std::vector<const double *> bp, cp, blp;
  ahlp_desc d{};
  std::vector<Recov> recov;
  double const_obj = 0.0;
  std::vector<int> n_orig;
  int n0_orig = 0;
};

// true when the description uses bounds or inequality rows
bool desc_is_general(const ahlp_desc &d);
// the equality form with x >= 0 of a description in the full statement
// (throws Fail on invalid input)
void standardize(const ahlp_desc &d, StdDesc &S);

struct DeviceBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace ahlp

struct ahlp_problem {
  // ---- sizes -------------------------------------------------------------
  int N = 0, n0 = 0, mg = 0, B = 0, nl = 0, nS = 0;
  // batch > 1: the direct sum of independent LPs; per LP its first block and
  // the offsets of its slices of x_0 and of the global rows
  int batch = 1;
  std::vector<long long> lp_blk0, lp_x0off, lp_goff;
  struct LpRange {   // index ranges of one LP of a batch in the global vectors
    long long xb0, xb1, x00, x01;            // x: its blocks, its linking variables
    long long yb0, yb1, yl0, yl1, yg0, yg1;  // y: block rows, link rows, global rows
    double bnorm, cnorm;                      // its ||b||_inf and ||c||_inf
  };
  std::vector<LpRange> lp_rng;
  // LPs given in the full statement: per LP its map back to the original
  // variables (empty: the LP was already in equality form with x >= 0)
  struct LpRecov {
    std::vector<ahlp::StdDesc::Recov> recov;
    std::vector<int> n_orig;
    int n0_orig = 0;
    double const_obj = 0.0;
  };
  std::vector<LpRecov> lp_recov;
  long long n = 0, m = 0, msum = 0;   // n_total, m_total, sum of m_i
  std::vector<int> mi, ni, ki, lprev, lnext;
  std::vector<long long> xoff, yoff, link_off;   // link_off has N entries (pairs + 1)
  int amax = 0;          // largest augmented order
  ahlp_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  double bnorm_inf = 0, cnorm_inf = 0;
  int device = 0;

  // ---- LP data on the device ----------------------------------------------
  double *b = nullptr, *c = nullptr;               // global rhs, cost
  int *A_rp = nullptr, *A_ci = nullptr;            // CSR of A (m x n)
  double *A_v = nullptr;
  int *AT_rp = nullptr, *AT_ci = nullptr;          // CSR of A' (n x m)
  double *AT_v = nullptr;
  unsigned char *is_x0 = nullptr;                  // [n] 1 for x_0 columns
  ahlp::SpMat Amat, ATmat;                         // A and A' with their long-row lists

  // ---- factor storage -----------------------------------------------------
  double *aug = nullptr;            // all augmented matrices, FP64 (allocated when first used)
  float *aug32 = nullptr;           // the same layout in FP32 (mixed mode; hi part of FF)
  float *aug_lo = nullptr;          // lo part of float-float factors
  long long aug_elems = 0;
  // per pivot tile of every block, a 64x64 column-major tile: the inverse of
  // the pivot triangle on its pivot rows, the factor itself on the non-pivot
  // rows of a block's last pivot tile, zeros elsewhere
  double *tinv = nullptr;
  float *tinv32 = nullptr;
  long long tinv_elems = 0;
  int fac_prec = 0;                 // precision of the current factor (kPrec*)
  ahlp::BlkInfo *blk = nullptr;     // [N]
  std::vector<ahlp::BlkInfo> h_blk;
  ahlp::SchurBlk *sblk = nullptr;   // [N]
  std::vector<ahlp::SchurBlk> h_sblk;
  double *diag0 = nullptr;          // original diagonals (blocks)
  double *cdiag0 = nullptr;         // corner diagonals before elimination ([U;Fg] D [U;Fg]')
  double *sb_ref = nullptr;         // reference diagonal of the border pivots
  long long cdiag_elems = 0;
  long long vec_elems = 0;          // sum of a_i
  int maxT = 0, maxTp = 0;
  // tensor-core trailing update of FP32 factors (k_tc.cu): each panel tile
  // of the current step staged as TF32 hi / lo words in the MMA operand
  // layout (one 8192-word slot per tile of every block), the update jobs of
  // every step as prefix offsets over the blocks, and one tensor map per
  // block over its FP32 augmented matrix
  float *pstage = nullptr;
  long long stage_slots = 0;
  int *tc_joff = nullptr;            // [maxTp][N + 1]
  std::vector<long long> tc_jobs;    // [maxTp]
  void *tc_tmap = nullptr;           // [N] CUtensorMap
  bool tc_ready = false;
  // float-float factors on the tensor cores: each panel tile as six FP16
  // digit planes (6 x 4096 halves per slot) and one exponent per row
  __half *dstage = nullptr;
  int *dexp = nullptr;
  bool oz_ready = false;
  void *oz_tmap = nullptr;           // [2N] CUtensorMap: each block's hi, then lo matrix
  int ff_update = 0;                 // trailing update of float-float factors: 1 FP32 pipe, 2 tensor cores
  // per block, T x T: lower tile (I, J) of the formed augmented matrix has entries
  std::vector<std::vector<unsigned char>> tile_nz;
  // tile-sparse update jobs (option tile_sparse): per step, the kept jobs of the
  // dense enumeration as {block, I0, J, has_i1}; nullptr = the dense triangle
  int4 *tc_jtab = nullptr;
  std::vector<long long> tc_jtab_off;
  long long tc_jobs_dense = 0, tc_jobs_kept = 0;
  int fp32_update = 0;               // trailing update of FP32 factors: 1 SIMT, 2 tensor
                                     // cores (one CTA per job), 3 tensor cores (persistent
                                     // warp-specialised pipeline)
  int num_sms = 1;
  double fac_flops = 0;   // algorithmic flops of one batched partial Cholesky
  double tri_elems = 0;   // lower-triangle entries of all augmented matrices

  // ---- formation pattern --------------------------------------------------
  ahlp::FormTile *ftiles = nullptr;
  long long *tile_ent = nullptr;    // [ntiles+1]
  int *ent_pos = nullptr;           // [nent]
  long long *ent_cb = nullptr;      // [nent+1]
  int *con_idx = nullptr;           // [ncon]
  double *con_coef = nullptr;       // [ncon]
  long long ntiles = 0, nent = 0, ncon = 0;

  // ---- Schur complement ---------------------------------------------------
  std::vector<long long> td_off, h_off;   // offsets of T_j (l_j^2) and H_j (l_{j+1} l_j)
  long long td_elems = 0, h_elems = 0;
  double *Td = nullptr, *Hd = nullptr, *Et = nullptr, *SB = nullptr;
  double *Td_asm = nullptr, *Hd_asm = nullptr, *Et_asm = nullptr, *SB_asm = nullptr;
  double *Td_diag0 = nullptr;        // assembled diagonal of T (pivot test)
  double *Linv = nullptr;            // L_j^-1 per pair (layout of Td)
  double *Yf = nullptr, *Yb = nullptr;   // chain coupling operators (layout of Hd)
  double *chain_tmp = nullptr;       // [nl] chain-solve scratch
  long long *td_off_d = nullptr, *h_off_d = nullptr;
  int *l_d = nullptr;                // [N-1]
  long long *link_off_d = nullptr;   // [N]
  int *kmap = nullptr;               // local Schur index -> global S index
  int *link_pair_d = nullptr;        // [nl] pair of each link row
  int *chain_seg = nullptr;          // [2 nchain_seg] pair ranges with link rows throughout
  int nchain_seg = 0;
  int *zlo = nullptr, *zhi = nullptr;   // [B] link rows a border column of Z can touch
  // cyclic reduction of the link chain (k_bcr.cu): pairs in level order,
  // per pair (level, segment first pair, segment end, -), the level offsets
  // into the order, and per pair its couplings GL_j, GR_j (lmax^2 each)
  int *bcr_order = nullptr, *bcr_info = nullptr;
  std::vector<int> bcr_loff;
  int bcr_lmax = 0;
  double *bcr_GL = nullptr, *bcr_GR = nullptr;
  bool fac_bcr = false;   // the current Schur factor's chain is the cyclic-reduction one
  long long *yoff_d = nullptr;       // [N] start of y_i
  long long *kmap_off_d = nullptr;   // [N]
  std::vector<long long> kmap_off;
  long long *f0_idx = nullptr; double *f0_val = nullptr; long long nf0 = 0;   // Et constants
  long long *fg0_idx = nullptr; double *fg0_val = nullptr; long long nfg0 = 0; // SB constants
  // border (quasi-definite) factor
  double *border = nullptr; int Bld = 0;
  ahlp::BlkInfo *bx_info = nullptr, *bp_info = nullptr;
  ahlp::BlkInfo h_bx{}, h_bp{};
  double *border_diag0 = nullptr;

  // ---- vectors ------------------------------------------------------------
  double *x = nullptr, *z = nullptr, *dscale = nullptr;   // current point, d = x/z
  double *xinv = nullptr, *wfin = nullptr;   // 1 / x, 1 / (1 / d + rho on x_0)
  double *vec = nullptr;      // block solve segments [sum a_i]
  float *vec32 = nullptr;     // FP32 copy of the forward solution (FP32 factors)
  double *svec = nullptr;     // Schur vector [nS]
  double *f = nullptr, *g = nullptr, *rhat = nullptr;      // solve scratch
  double *stg[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // staging for host I/O
  double *res[3] = {nullptr, nullptr, nullptr};            // refinement residual
  double *cor[3] = {nullptr, nullptr, nullptr};            // refinement correction
  double *ipmv[19] = {};      // IPM work vectors (the last three: a batch's balanced rhs)
  double *red_part = nullptr; // reduction partials
  double *mdot_part = nullptr;  // multi-dot partials [kMaxKrylov+1][304]
  double *gm_V = nullptr, *gm_Z = nullptr;   // Krylov bases, allocated on first use
  double *gm_coef = nullptr;    // device coefficients for multi-axpy
  double *gm_h = nullptr;       // Arnoldi column on the device: both Gram-Schmidt passes and |w|^2
  int gm_cap = 0;               // vectors allocated in gm_Z (gm_V has one more)
  double *scal = nullptr;     // device scalars
  double *h_scal = nullptr;   // pinned host scalars
  int *status = nullptr;      // device status words [4]
  // wavefront block solves: (block, row tile) jobs in ticket order, one ready
  // flag per tile, then the forward and backward ticket counters
  int *trsv_fsched = nullptr, *trsv_bsched = nullptr;   // [2 * jobs]
  int *trsv_flag_off = nullptr;   // [N] first flag of each block
  int *trsv_flags = nullptr;      // [trsv_nflags + 2]
  int *trsv_err = nullptr;        // set when a wait timed out
  int trsv_nf = 0, trsv_nb = 0, trsv_nflags = 0;
  int tiny_pivots = 0;
  bool factored = false;
  bool assembled = false;     // the Schur complement of the last kkt_factor exists
  double fac_delta = 0, fac_rho = 0, fac_pivot_tol = 0;
  double fac_rho_x = 0;   // primal regularisation of the preconditioner's D (ipm_solve's last safeguard)

  // ---- host <-> device traffic since create (ahlp_transfer_bytes) ----------
  long long bytes_h2d = 0, bytes_d2h = 0;

  // ---- timing -------------------------------------------------------------
  cudaEvent_t ev[8] = {};
  std::vector<cudaEvent_t> kt_pool;     // kernel-class timer: events, and per
  std::vector<int> kt_cls;              // recorded event the class it opens
  double kt_ms[3] = {0, 0, 0};          // last factor: diagonal tiles, panels, updates
  long long kt_n[3] = {0, 0, 0};        // and their launch groups
  float stage_ms[4] = {0, 0, 0, 0};

  std::vector<ahlp::DeviceBuf> allocs;
};

namespace ahlp {

// Every kernel launch of the library is written `count_launch(), k<<<...>>>(...)`
// so the number of launches can be reported (arrowhead_lp_launch_count).
void count_launch();
long long launch_count();

// ---- kernels (launch wrappers) --------------------------------------------
// All wrappers enqueue on p->stream and return the cudaError_t of the launch.
cudaError_t launch_dscale(ahlp_problem *p);   // dscale = x / (z + fac_rho_x x)
cudaError_t launch_form(ahlp_problem *p, double delta);
// prof (nullable): a handle whose kernel-class timer records the launches
// (kt_mark); classes 0 diagonal tiles, 1 panels, 2 trailing updates
cudaError_t launch_pchol(double *buf, const BlkInfo *info, const std::vector<BlkInfo> &h,
                         const double *diag0, double tol, int *status, cudaStream_t s,
                         ahlp_problem *prof = nullptr, double drop = 0.0);
// float-float (hi = aug32, lo): diagonal tiles and panels in FP64 arithmetic,
// trailing updates in double-float; then hi + lo is expanded into out (the
// FP64 factor buffer, elems entries), which the Schur assembly and the solves use
// with oz (a handle set up by oz_setup) the trailing updates run on the
// tensor cores as exact FP16 digit products (k_tc.cu)
cudaError_t launch_pchol_ff(float *hi, float *lo, double *out, long long elems,
                            const BlkInfo *info, const std::vector<BlkInfo> &h,
                            const double *diag0, double tol, int *status, cudaStream_t s,
                            ahlp_problem *oz = nullptr, ahlp_problem *prof = nullptr,
                            double drop = 0.0);
// FP32: also writes the inverted diagonal tiles into tinv (see launch_tinv);
// with tc (a handle set up by tc_setup) the trailing updates run on the
// tensor cores (k_tc.cu), else on the FP32 pipe
cudaError_t launch_pchol_f32(float *buf, float *tinv, const BlkInfo *info,
                             const std::vector<BlkInfo> &h, const double *diag0, double tol,
                             int *status, cudaStream_t s, ahlp_problem *tc = nullptr,
                             ahlp_problem *prof = nullptr, double drop = 0.0);
// forward / backward solves with one partial factor per CTA (the border
// factors; vectors FP64, held in shared memory)
cudaError_t launch_ptri(const double *buf, const BlkInfo *info, int nblk, int amax, double *vec,
                        bool forward, cudaStream_t s);
// inverted diagonal tiles of the current block factors (p->tinv / tinv32)
cudaError_t launch_tinv(ahlp_problem *p);
// forward / backward wavefront solves with all block factors (p->vec, in the
// precision of the current factor); wait timeouts set p->trsv_err
cudaError_t launch_trsv(ahlp_problem *p, bool forward);
cudaError_t launch_schur_assemble(ahlp_problem *p, double delta, double rho);
cudaError_t launch_schur_factor(ahlp_problem *p);
// cyclic reduction of the link chain: factor (T_j, Linv_j, GL_j, GR_j, and Z
// into Et) and the forward / backward solves in place on the link part of u
cudaError_t launch_bcr_factor(ahlp_problem *p);
cudaError_t launch_bcr_solve(ahlp_problem *p, double *u, bool forward);
cudaError_t launch_solve(ahlp_problem *p, const double *r_d, const double *r_p,
                         const double *r_c, double *dx, double *dy, double *dz, bool adjoint);
cudaError_t launch_residual(ahlp_problem *p, const double *r_d, const double *r_p,
                            const double *r_c, const double *dx, const double *dy,
                            const double *dz, double *e_d, double *e_p, double *e_c,
                            bool adjoint);

// ---- vector utilities ------------------------------------------------------
enum RedOp { RED_DOT = 0, RED_MAXABS = 1, RED_MINSTEP = 2, RED_MIN = 3, RED_SUM = 4 };
// out <- reduce(op, a, b) over len entries, deterministic order; out is a
// device scalar.
cudaError_t launch_reduce(ahlp_problem *p, int op, const double *a, const double *b,
                          long long len, double *out);
cudaError_t launch_spmv(const SpMat &A, const double *x, double *y, double alpha,
                        const double *yadd, cudaStream_t s);   // y = yadd + alpha A x (yadd may be null)
cudaError_t launch_axpby(double *y, const double *x, double a, double b, long long n,
                         cudaStream_t s);  // y = a x + b y
// generic elementwise kernels for the IPM
cudaError_t launch_ipm_rc(double *rc, const double *x, const double *z, const double *dxa,
                          const double *dza, double sigma_mu, long long n, cudaStream_t s);
cudaError_t launch_fill(double *y, double v, long long n, cudaStream_t s);
cudaError_t launch_add_scalar(double *y, const double *x, double s, long long n,
                              cudaStream_t st);   // y = x + s
constexpr int kMaxKrylov = 64;   // cap on GMRES iterations per solve
// out[i] = <V_i, w>, i < k (V_i = V + i*ld), deterministic
cudaError_t launch_mdot(ahlp_problem *p, const double *V, long long ld, int k, const double *w,
                        long long len, double *out);
// w += sum_i coef[i] V_i   (coef in device memory)
// w += sign * sum_i coef[i] V_i (coef on the device, fixed order over i)
cudaError_t launch_maxpy(const double *V, long long ld, int k, const double *coef, double *w,
                         long long len, cudaStream_t s, double sign = 1.0);
// w *= 1 / sqrt(*nrm2) when *nrm2 > 0, nrm2 a device scalar
cudaError_t launch_scale_inv_norm(double *w, long long len, const double *nrm2, cudaStream_t s);
// o = J v (Newton matrix of Sec. 2.3) or J' v
cudaError_t launch_jmul(ahlp_problem *p, const double *vx, const double *vy, const double *vz,
                        double *ox, double *oy, double *oz, bool adjoint);
cudaError_t launch_mul(double *y, const double *a, const double *b, double scale, long long n,
                       cudaStream_t s);   // y = scale * a .* b
// centrality corrector right-hand side: rc2 = rc + t, where v = (x + ap dx) .* (z + ad dz)
// is projected onto [lo, hi] and t = proj(v) - v, bounded below by -hi
cudaError_t launch_centrality_rc(double *rc2, const double *rc, const double *x,
                                 const double *dx, double ap, const double *z, const double *dz,
                                 double ad, double lo, double hi, long long n, cudaStream_t s);
cudaError_t launch_step_dot(const double *x, const double *dx, double ap, const double *z,
                            const double *dz, double ad, long long n, double *part,
                            double *out, cudaStream_t s);  // (x+ap dx)'(z+ad dz)

// ---- tensor-core trailing update (k_tc.cu) -----------------------------------
// staging, job offsets and tensor maps for the FP32 factors (needs aug32);
// false when the driver has no tensor-map encoder
bool tc_setup(ahlp_problem *p);
cudaError_t launch_update_tc(ahlp_problem *p, int k, cudaStream_t s);
// the same for float-float factors: FP16 digit staging and job offsets
bool oz_setup(ahlp_problem *p);
cudaError_t launch_update_oz(ahlp_problem *p, int k, cudaStream_t s);

// ---- kernel-class timer (option profile_kernels) -----------------------------
// kt_mark records an event on s that ends the previous mark's interval and
// opens one of class cls (0 diagonal tiles, 1 panels, 2 trailing updates,
// 3 closes without opening); kt_collect, after the stream has synchronised,
// sums the intervals per class into kt_ms and their counts into kt_n
void kt_mark(ahlp_problem *p, int cls, cudaStream_t s);
void kt_collect(ahlp_problem *p);

// ---- host runtime helpers (api.cpp) -------------------------------------------
// device allocations owned by the handle (freed at destroy); throw Fail
void *dalloc_bytes(ahlp_problem *p, size_t bytes);
void *dupload_bytes(ahlp_problem *p, const void *h, size_t bytes);
bool is_device_ptr(const void *ptr);
const double *stage_in(ahlp_problem *p, const double *v, long long n, double *staging);
int set_err(ahlp_problem *p, int code, const std::string &msg);
void read_scalars(ahlp_problem *p, int k);
// ff_nan_up: a NaN pivot of a float-float factor refactors in FP64 (else the
// call returns AHLP_ERR_NOT_SPD and the caller picks the next safeguard)
int factor_impl(ahlp_problem *p, double delta, double rho, double pivot_tol,
                bool ff_nan_up = true);
// tol_override > 0 replaces refine_tol as the FGMRES target
int solve_impl(ahlp_problem *p, const double *rd, const double *rp, const double *rc, double *dx,
               double *dy, double *dz, bool adjoint, ahlp_solve_info *info,
               double tol_override = 0.0);
void ck(cudaError_t e, const char *what);   // throws on error

struct Fail {
  int code;
  std::string msg;
};

}  // namespace ahlp
