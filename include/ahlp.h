/*
 * ahlp.h -- C ABI of a GB300 (sm_103a) library that solves arrowhead linear
 * programs with local linking structure by a primal-dual interior-point
 * method whose per-iteration KKT systems are factored and solved through a
 * block Schur-complement decomposition on one GPU.
 *
 * Problem (Sec. 3.2, eq. fig:blockstructure, equality rows and x >= 0; local
 * and global linking rows as in Sec. 3.3):
 *
 *     min  c_0'x_0 + sum_i c_i'x_i
 *     s.t. W_i x_0 + A_i x_i                     = b_i       i = 1..N
 *          F0_j x_0 + FL_j x_j + FR_j x_{j+1}    = blink_j   j = 1..N-1
 *          Fg0 x_0 + sum_i Fg_i x_i              = bg
 *          x >= 0
 *
 * (The paper calls the block matrices B_i and the linking-variable blocks
 * A_i; here they are A_i and W_i.)
 *
 * Global vector orderings used by every entry point:
 *     x, z, dx, dz, r_d, r_c : [x_1 .. x_N, x_0]                    length n_total
 *     y, dy, r_p             : [y_1 .. y_N, y_link(pair 1..N-1), y_g] length m_total
 *
 * Pointers.  Every vector argument may be a host pointer or a device
 * pointer of the current CUDA device; the library tells them apart with
 * cudaPointerGetAttributes.  Host vectors are staged through the library's
 * own device buffers (the call then synchronises its stream before
 * returning); device vectors are used in place on the problem's stream.
 * Matrix data in ahlp_desc are host pointers and are copied at create: the
 * caller keeps ownership of everything it passes in.
 *
 * Errors.  Every call returns an int status (AHLP_OK = 0 or a negative
 * code below).  Nothing aborts, prints or traps; the text of the last error
 * is available from ahlp_last_error().  A handle is not thread-safe.
 */
#ifndef AHLP_H
#define AHLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define AHLP_OK                   0
#define AHLP_ERR_INVALID_ARG     -1  /* NaN/Inf, negative size, bad index, NULL where required */
#define AHLP_ERR_DIM_MISMATCH    -2  /* block sizes disagree with each other                 */
#define AHLP_ERR_UNSUPPORTED     -3  /* a size limit or a feature not available            */
#define AHLP_ERR_NOT_SPD         -4  /* a pivot became NaN / negative beyond repair            */
#define AHLP_ERR_REFINE_FAIL     -5  /* refinement did not reach refine_tol                    */
#define AHLP_ERR_MAX_ITER        -6  /* ipm_solve hit max_iter                                 */
#define AHLP_ERR_INFEASIBLE      -7  /* iterates diverge (primal or dual infeasible LP)        */
#define AHLP_ERR_CUDA            -8  /* a CUDA runtime call failed                             */
#define AHLP_ERR_OOM             -9  /* device allocation failed                               */
#define AHLP_ERR_TIMEOUT        -10  /* a bounded device wait ran out                          */
#define AHLP_ERR_STOPPED        -11  /* ipm_solve: the iteration callback asked to stop        */

#define AHLP_PREC_FP64   0   /* every stage in FP64                                    */
#define AHLP_PREC_MIXED  1   /* FP32 block factors (float-float near the optimum), FP64 Schur factor and refinement */

/* ---- problem description (host memory, copied at create) --------------- */

/* Compressed sparse column matrix, 0-based.  colptr has n+1 entries,
 * rowidx/val have colptr[n] entries; rows within a column may be in any
 * order, duplicates are summed.  m or n may be 0 (then all pointers may be
 * NULL). */
typedef struct {
  int32_t m, n;
  const int32_t *colptr;
  const int32_t *rowidx;
  const double *val;
} ahlp_csc;

/* The arrowhead LP (Sec. 3.2/3.3).  Arrays of per-block items have N
 * entries, per-pair items N-1.  lb/ub: NULL means x >= 0, no upper bound;
 * otherwise any bounds -inf <= lb <= ub <= +inf (free, fixed, one- and
 * two-sided variables).  With bounds or inequality rows the LP is in the
 * full statement of Sec. 3.2; arrowhead_lp_create reduces it to the
 * equality form with x >= 0 that the solver works on (an inequality row gets
 * a bounded slack variable in its block -- the left block for a local link
 * row, the last block for a global row; a variable bounded below is shifted,
 * one bounded above negated and shifted, a free one split into two, a boxed
 * one given a new row in its block (a global row for a linking variable)
 * and a new column).  Every entry point after create then works on that
 * form; arrowhead_lp_recover maps its x back to the original variables. */
typedef struct {
  int32_t N;                       /* number of blocks (>= 1)                  */
  int32_t n0;                      /* linking variables x_0 (>= 0)             */
  int32_t mg;                      /* global linking rows (>= 0)               */
  const double *c0;                /* [n0]                                     */
  const ahlp_csc *A;               /* [N]  m_i x n_i block matrices            */
  const ahlp_csc *W;               /* [N]  m_i x n0 linking-variable blocks    */
  const double *const *b;          /* [N]  -> [m_i]                            */
  const double *const *c;          /* [N]  -> [n_i]                            */
  const int32_t *l;                /* [N-1] local link rows of pair (j, j+1)   */
  const ahlp_csc *FL;              /* [N-1] l_j x n_j                          */
  const ahlp_csc *FR;              /* [N-1] l_j x n_{j+1}                      */
  const ahlp_csc *F0;              /* [N-1] l_j x n0                           */
  const double *const *blink;      /* [N-1] -> [l_j]                           */
  const ahlp_csc *Fg;              /* [N]  mg x n_i                            */
  const ahlp_csc *Fg0;             /* mg x n0 (may be NULL when mg*n0 == 0)    */
  const double *bg;                /* [mg]                                     */
  const double *const *lb;         /* [N] -> [n_i] or NULL                     */
  const double *const *ub;         /* [N] -> [n_i] or NULL                     */
  const double *lb0, *ub0;         /* [n0] or NULL                             */
  /* Inequality rows of the full statement (Sec. 3.2), d <= (row) x <= f with
   * entries of d possibly -inf and of f +inf.  Every pointer may be NULL (no
   * rows of that kind; then the counts must be 0 or NULL too). */
  const int32_t *mD;               /* [N]  inequality rows of block i          */
  const ahlp_csc *D;               /* [N]  mD_i x n_i  (the paper's D_i)      */
  const ahlp_csc *C;               /* [N]  mD_i x n0   (the paper's C_i)      */
  const double *const *dlo;        /* [N] -> [mD_i]                            */
  const double *const *dhi;        /* [N] -> [mD_i]                            */
  const int32_t *lG;               /* [N-1] local link inequality rows of pair j */
  const ahlp_csc *GL;              /* [N-1] lG_j x n_j                         */
  const ahlp_csc *GR;              /* [N-1] lG_j x n_{j+1}                     */
  const ahlp_csc *G0;              /* [N-1] lG_j x n0                          */
  const double *const *glo;        /* [N-1] -> [lG_j]                          */
  const double *const *ghi;        /* [N-1] -> [lG_j]                          */
  int32_t mgG;                     /* global linking inequality rows           */
  const ahlp_csc *Gg;              /* [N]  mgG x n_i                           */
  const ahlp_csc *Gg0;             /* mgG x n0                                 */
  const double *gglo, *gghi;       /* [mgG]                                    */
} ahlp_desc;

struct ahlp_result_s;

/* Progress callback of ipm_solve (option iter_cb): called on the host thread
 * once per iteration, after the iterate's residuals, objective values and mu
 * have been evaluated and before the convergence test, with the iteration
 * index and the result record as it stands (pobj, dobj, rel_gap, pinf, dinf,
 * mu, iterations and the counters so far).  The device work of every earlier
 * iteration has been issued on the handle's stream (not necessarily
 * finished).  A nonzero return value stops the solve: ipm_solve then writes
 * the current iterate out and returns AHLP_ERR_STOPPED.  The callback must
 * not call into this handle. */
typedef int (*ahlp_iter_cb)(void *ctx, int32_t iteration, const struct ahlp_result_s *progress);

typedef struct {
  int32_t precision;    /* AHLP_PREC_FP64 (default) or AHLP_PREC_MIXED            */
  int32_t max_iter;     /* IPM iteration cap (200)                                */
  double  tol;          /* relative infeasibility and gap tolerance (1e-8)        */
  double  eta;          /* step-to-boundary factor (0.9995)                       */
  double  delta;        /* dual regularisation of the factor: +delta on the diagonal
                           of M_i, of the link rows and of the global rows (1e-8).
                           Only the preconditioner is regularised: kkt_solve
                           solves the unregularised Newton system.  ipm_solve
                           raises it x100 (up to 1e-4) when a NaN persists after
                           the FP64 and pivot-threshold safeguards            */
  double  rho;          /* primal regularisation of the factor: D^-1 + rho on every
                           primal variable (block variables through
                           d = x / (z + rho x)) (0); ipm_solve raises it from
                           1e-10 up to 1e-6 when a NaN persists after the other
                           safeguards                                           */
  int32_t refine_max;   /* FGMRES iterations per KKT solve, at most 64, counted
                           over restarts (40)                                     */
  double  refine_tol;   /* target relative Newton residual (1e-10)                */
  double  pivot_tol;    /* a pivot not above pivot_tol * (its diagonal before
                           elimination) has lost its digits to cancellation and
                           is clamped to that value (1e-12); ipm_solve coarsens
                           it x100 (up to 1e-8) when a direction's residual
                           stays above 1e-6 or a NaN appears, once the block
                           factors are FP64                                      */
  int32_t verbose;      /* 0: silent; 1: one line per IPM iteration; 2: also the
                           Krylov residual estimate of every refinement step */
  int32_t max_correctors; /* multiple centrality correctors per iteration, each
                           one more solve with the same factor, tried while the
                           step length stays below 0.9 (4; 0..8); see
                           correctors_by_cost                                  */
  double  fp32_cond_max;/* mixed precision: the block factors run in FP32 while
                           max(d)/min(d), d = x/z, stays at or below this value,
                           and in float-float (two FP32 words, ~46 bits) beyond
                           it; a float-float factor that fails moves to FP64
                           (1e14)                                                */
  double  ipm_refine_tol; /* target relative Newton residual of the directions
                           inside ipm_solve (1e-6): an inexact-Newton forcing
                           term, the residual is ~1e-6 of |r| >= mu sqrt(n).
                           The larger of it and refine_tol applies; kkt_solve
                           and kkt_adjoint_solve always use refine_tol        */
  int32_t correctors_by_cost; /* 1: at most as many correctors as the factor costs
                           in solves (Gondzio's rule), both costs from a fixed
                           model of the work (flops of the block factor at its
                           precision's rate; factor bytes read per
                           preconditioner application times the last solve's
                           Krylov steps), so the iterates do not depend on
                           timings; 0: up to max_correctors regardless (1)     */
  int32_t fp32_update;  /* trailing updates of FP32 block factors: 0 = tensor
                           cores when available (tcgen05, TF32 hi/lo split
                           operands, FP32 accumulation), 1 = FP32 pipe,
                           2 = tensor cores, one CTA per 128 x 64 output tile,
                           3 = tensor cores, one persistent CTA per SM that
                           overlaps the copies, products and reduce of
                           consecutive tiles (2 and 3: AHLP_ERR_UNSUPPORTED
                           when the driver cannot encode tensor maps) (0)      */
  int32_t ff_update;    /* trailing updates of float-float block factors: 0 or 2 =
                           tensor cores (each panel entry as six FP16 integer
                           digits under a per-row exponent, the digit products
                           accumulated exactly in FP32, 49 bits in all), one
                           CTA per 128 x 64 output tile; 3 = the same products
                           in one persistent CTA per SM that overlaps the
                           copies, products and C-tile update of consecutive
                           tiles (bitwise the same factor); 1 = double-float
                           arithmetic on the FP32 pipe.  0, 2 and 3 fall back
                           to 1 when the driver cannot encode tensor maps (0) */
  int32_t schur_chain;  /* factor and solves of the block-tridiagonal link chain
                           of the Schur complement: 0 = block cyclic reduction
                           (log2 of the chain length sequential levels),
                           1 = sequential block Cholesky along the chain (0)   */
  int32_t profile_kernels; /* 1: kkt_factor records CUDA events around each group
                           of block-factor launches (diagonal tiles, panels,
                           trailing updates) for kkt_factor_kernel_times (0) */
  ahlp_iter_cb iter_cb; /* progress callback of ipm_solve, or NULL (NULL)        */
  void   *iter_cb_ctx;  /* passed to iter_cb (NULL)                              */
  int32_t pivot_mode;   /* pivots of the block factors M_i that fail the
                           pivot_tol test (cancellation or NaN): 0 = clamp to
                           pivot_tol times their starting diagonal; 1 = drop:
                           replace by a huge value, so the row is left out of
                           the factor (its solution entry ~0, its column ~0)
                           and the Krylov refinement, which solves the exact
                           Newton system, sees it unpreconditioned.  The Schur
                           complement's pivots are always clamped (0)        */
  int32_t tile_sparse;  /* 1: the tensor-core trailing updates skip the tile
                           jobs whose product is structurally zero (a tile-level
                           symbolic factorisation of each block's augmented
                           matrix, from its formation pattern); the factor is
                           bitwise the same, banded blocks cost less.  0: every
                           tile pair of the trailing triangle.  Read when a
                           handle first factors on the tensor cores (1)       */
} ahlp_options;

typedef struct ahlp_result_s {
  int32_t status;         /* same code the call returned                          */
  int32_t iterations;
  double  pobj, dobj;     /* c'x and b'y                                          */
  double  rel_gap;        /* |c'x - b'y| / (1 + |c'x|)                            */
  double  pinf, dinf;     /* ||b-Ax||_inf/(1+||b||_inf), ||c-A'y-z||_inf/(1+||c||_inf) */
  double  mu;             /* x'z / n                                              */
  double  ms_total;       /* wall time of the solve                               */
  double  ms_factor;      /* summed kkt_factor time                               */
  double  ms_solve;       /* summed kkt_solve time (incl. refinement)             */
  int32_t refine_steps;   /* summed refinement steps                              */
  int32_t tiny_pivots;    /* pivots clamped in the last factor                    */
  double  kkt_residual;   /* largest relative Newton residual seen                */
  int32_t escalations;    /* FP32->FP64 switches plus pivot-threshold coarsenings  */
  int32_t fp64_switch_iter; /* mixed mode: first iteration whose block factors are
                             no longer FP32 (-1: never); FP64 mode: 0             */
  int32_t factors_fp32, factors_fp64;   /* block factorisations per precision     */
  int32_t correctors;     /* accepted centrality correctors                      */
  double  ms_block_fp32, ms_block_fp64; /* their summed device time (the batched
                                           partial Cholesky stage alone)         */
  int32_t factors_ff;     /* float-float block factorisations (mixed mode)       */
  double  ms_block_ff;    /* their summed device time                            */
} ahlp_result;

typedef struct {
  int32_t refine_steps;   /* refinement steps taken                               */
  double  rel_residual;   /* ||J d - r||_2 / ||r||_2 of the returned direction    */
} ahlp_solve_info;

typedef struct ahlp_problem ahlp_problem;   /* opaque; owns its device memory */

/* Fill *opt with the defaults listed above. */
void ahlp_default_options(ahlp_options *opt);

/* Human-readable name of a status code (static storage). */
const char *ahlp_status_string(int status);

/*
 * arrowhead_lp_create -- validate the LP, copy it to the current CUDA device
 * and run the symbolic analysis (storage layout of the per-block augmented
 * matrices, formation patterns, Schur-complement index maps).
 *   descs : [batch] problem descriptions (host memory)
 *   batch : number of independent LPs in descs (>= 1).  A batch is solved as
 *           their direct sum, one arrowhead LP whose blocks are all the LPs'
 *           blocks in order (consecutive blocks of different LPs share no link
 *           rows), so every stage runs all LPs in the same launches.  The
 *           global vectors of the handle follow the direct sum's ordering:
 *           x = [blocks of LP 0, blocks of LP 1, ..., x_0 of LP 0, x_0 of LP 1,
 *           ...]; y = [block rows of all LPs, link rows of all LPs, global rows
 *           of all LPs], each part in LP order.  ipm_solve stops when every LP
 *           meets the tolerances on its own and reports the worst LP.
 *   opt   : options, or NULL for defaults
 *   out   : receives the handle; *out is NULL on error
 * The structure follows Sec. 3.2 (blocks, linking variables and rows) and
 * Sec. 3.3 (local two-links vs global rows); the Schur layout is App. A.
 */
int arrowhead_lp_create(const ahlp_desc *descs, int32_t batch, const ahlp_options *opt,
                        ahlp_problem **out);

/* Free every device and host resource of the handle (NULL is a no-op). */
void arrowhead_lp_destroy(ahlp_problem *p);

/* Text of the last error on this handle (or of the last failed create when
 * p is NULL).  Valid until the next call on the handle. */
const char *ahlp_last_error(const ahlp_problem *p);

/*
 * arrowhead_lp_recover -- the original variables of an LP given in the full
 * statement (bounds or inequality rows, Sec. 3.2) from a point x of the
 * equality form the handle works on.  x [n_total] (host or device); x_orig
 * [n_orig] (host or device) ordered like x for a batch: the original block
 * variables of every LP in block order, then every LP's original linking
 * variables; obj_offset (may be NULL) receives the constant the reduction
 * took out of the objective (summed over the LPs of a batch): the original
 * objective is c'x + obj_offset.  n_orig is returned by
 * arrowhead_lp_original_size.  LPs already in equality form map unchanged.
 */
int arrowhead_lp_recover(ahlp_problem *p, const double *x, double *x_orig, double *obj_offset);
int arrowhead_lp_original_size(const ahlp_problem *p, int64_t *n_orig);

/*
 * arrowhead_lp_autotune -- pick the trailing-update kernel of the FP32 and of
 * the float-float block factors for this handle's block sizes: each
 * candidate (FP32: tensor cores with one CTA per 128 x 64 output tile, the
 * persistent pipelined tensor-core kernel, or the FP32 pipe on 64 x 64
 * tiles; float-float: FP16 digit products on the tensor cores per tile or
 * persistent, or double-float arithmetic on the FP32 pipe) factors the
 * blocks at the point (x, z) (NULL: x = z = 1), timed with CUDA events on
 * the handle's stream (best of two after one warm-up), and the fastest is
 * written into the handle's options (fp32_update, ff_update).  Later calls
 * do not time anything, so results stay reproducible once the choice is
 * made.
 *   ms6 (may be NULL) : receives the six block-factor times [FP32 tensor
 *                       per tile, FP32 pipe, float-float tensor per tile,
 *                       float-float pipe, FP32 tensor persistent,
 *                       float-float tensor persistent]
 */
int arrowhead_lp_autotune(ahlp_problem *p, const double *x, const double *z, double *ms6);

/* Sizes of the global vectors. */
int arrowhead_lp_sizes(const ahlp_problem *p, int64_t *n_total, int64_t *m_total);

/* Stream used by all later calls on this handle (a cudaStream_t; NULL =
 * the legacy default stream). */
int arrowhead_lp_set_stream(ahlp_problem *p, void *stream);

/* Replace the options of an existing handle (same fields as at create). */
int arrowhead_lp_set_options(ahlp_problem *p, const ahlp_options *opt);

/*
 * arrowhead_lp_set_cb -- replace the objective c and/or the right-hand side b
 * of the problem (Sec. 3.2 statement) without touching its structure, e.g.
 * for parametric re-solves or for differentiating the optimum with respect to
 * (c, b).  c: [n] and b: [m] in the global orderings (x = [x_1..x_N, x_0],
 * y = [y_1..y_N, y_links, y_g]), host or device memory, copied; NULL keeps
 * the current vector.  NaN/Inf entries: AHLP_ERR_INVALID_ARG, nothing
 * replaced for that vector.
 */
int arrowhead_lp_set_cb(ahlp_problem *p, const double *c, const double *b);

/*
 * kkt_factor -- factor the Newton system at the interior point (x, z)
 * (Alg. 2 of Sec. 3.2 with the block systems in normal-equation form):
 *   (a) per block, M_i = A_i D_i A_i' + delta I with D_i = X_i Z_i^-1, stacked
 *       with G_i = [W_i | A_i D_i U_i' | A_i D_i Fg_i'] into the augmented
 *       matrix [M_i G_i; G_i' C_i] (C_i = [U_i;Fg_i] D_i [U_i;Fg_i]');
 *   (b) one batched partial Cholesky of all augmented matrices over their
 *       first m_i pivots, which leaves Y_i' = (L_i^-1 G_i)' below the factor
 *       and the Schur contribution C_i - G_i' M_i^-1 G_i in the corner
 *       (Alg. 1, and the block factorisation and Schur-contribution steps
 *       of Alg. 2; the partial-factorisation idea of Sec. 3.2);
 *   (c) fixed-order summation of the contributions into the block-
 *       tridiagonal-plus-border Schur complement of App. A, its block
 *       Cholesky along the link chain and the quasi-definite border factor
 *       (the Schur-complement assembly and factorisation of Alg. 2).
 *   x, z : [n_total], strictly positive (host or device)
 *   delta, rho : regularisation for this factor (negative = use options)
 * Returns AHLP_ERR_INVALID_ARG if some x or z is not > 0, AHLP_ERR_NOT_SPD if
 * a pivot is NaN.  Tiny pivots are replaced (their count is kept).
 */
int kkt_factor(ahlp_problem *p, const double *x, const double *z, double delta, double rho);

/*
 * kkt_solve -- solve the Newton system of Sec. 2.3 at the last factored
 * point,
 *     [0 A' I; A 0 0; Z 0 X] [dx; dy; dz] = [r_d; r_p; r_c],
 * by Alg. 3 (block forward solves, Schur right-hand side, Schur solve,
 * block back-substitution) followed by dx = D(A'dy - r_d + X^-1 r_c) and
 * dz = X^-1 (r_c - Z dx) (the elimination of Sec. 2.3).  When the relative
 * residual of the unregularised Newton system is still above refine_tol,
 * right-preconditioned FGMRES on that system (the block solve above as the
 * preconditioner) runs for at most refine_max iterations; when the true
 * residual after a cycle is still above refine_tol (the cycle's own estimate
 * can run ahead of it), the method restarts from it while each cycle at
 * least halves it.
 *   r_d [n_total], r_p [m_total], r_c [n_total] : right-hand side
 *   dx [n_total], dy [m_total], dz [n_total]    : output (caller-allocated)
 *   info : optional (NULL allowed)
 * Returns AHLP_ERR_INVALID_ARG if no factor exists.  Missing the refinement
 * target is reported in info, not as an error.
 */
int kkt_solve(ahlp_problem *p, const double *r_d, const double *r_p, const double *r_c,
              double *dx, double *dy, double *dz, ahlp_solve_info *info);

/*
 * kkt_adjoint_solve -- solve the transposed Newton system J' lam = g at the
 * last factored point, reusing the factors: J' reduces to the same
 * symmetric matrix [-D^-1 A'; A 0] with right-hand side
 * [g_x - Z X^-1 g_z; g_y], and lam_z = X^-1 (g_z - lam_x).  Used for
 * implicit differentiation of the optimum: with g = (c, 0, 0) at the
 * optimum, dObj/dc = x + lam_x and dObj/db = lam_y.
 *   g_x [n_total], g_y [m_total], g_z [n_total]; outputs likewise.
 */
int kkt_adjoint_solve(ahlp_problem *p, const double *g_x, const double *g_y, const double *g_z,
                      double *lam_x, double *lam_y, double *lam_z, ahlp_solve_info *info);

/*
 * ipm_solve -- infeasible primal-dual Mehrotra predictor-corrector IPM
 * (Sec. 2 and 2.3) with every linear-algebra step in this library's
 * kernels.  Starting point: Mehrotra's heuristic computed with two solves
 * at D = I, unless a warm start (x0, y0, z0 all non-NULL) is given.
 *   x0, y0, z0 : optional warm start (host or device, NULL = cold start)
 *   x, y, z    : final iterate (host or device, may be NULL)
 *   res        : optional result record
 * Returns AHLP_OK at convergence, AHLP_ERR_MAX_ITER, AHLP_ERR_INFEASIBLE,
 * AHLP_ERR_STOPPED (the option iter_cb returned nonzero) or an error from
 * the KKT calls.  The iterates are a deterministic function of the problem,
 * the options and the starting point: nothing depends on timings.
 */
int ipm_solve(ahlp_problem *p, const double *x0, const double *y0, const double *z0,
              double *x, double *y, double *z, ahlp_result *res);

/*
 * kkt_schur_dense -- diagnostic: copy the Schur complement assembled by the
 * last kkt_factor (before it was factored) into host memory as a dense
 * column-major matrix with leading dimension ld, ordered
 * [link rows (pair 1..N-1) | x_0 | global rows] (App. A, permuted).
 *   S  : host buffer of ld * dim doubles, dim = sum(l) + n0 + mg
 */
int kkt_schur_dense(ahlp_problem *p, double *S, int64_t ld);

/*
 * kkt_block_factor_dense -- diagnostic: copy block i's augmented matrix after
 * the last kkt_factor (its partial Cholesky over the first m_i pivots:
 * L_i on top, Y_i' below it, the Schur contribution C_i - G_i' M_i^-1 G_i in
 * the corner; the block steps of Alg. 2) into host memory as a dense column-major
 * a x a lower triangle, a = m_i + k_i (the upper triangle is zeroed).
 *   block : 0 <= block < N;  A : host buffer of ld * a doubles;  ld >= a
 *   order : receives a (may be NULL)
 * Values are widened to double in mixed precision.
 */
int kkt_block_factor_dense(ahlp_problem *p, int32_t block, double *A, int64_t ld,
                           int32_t *order);

/*
 * kkt_stage_times -- diagnostic: device times (ms) of the stages of the last
 * kkt_factor and kkt_solve: out[0] formation, out[1] block partial
 * Cholesky, out[2] Schur assembly + factor, out[3] last kkt_solve.
 */
int kkt_stage_times(ahlp_problem *p, double *out4);

/* Diagnostic: number of CUDA kernels this library has launched in this
 * process so far (all handles).  The difference of two readings is the
 * launch count of the calls made in between. */
int64_t ahlp_launch_count(void);

/* Diagnostic: device times (ms, CUDA events on the handle's stream) of the
 * block partial Cholesky of the last kkt_factor, by kernel class: ms3[0]
 * diagonal tiles, ms3[1] panels, ms3[2] trailing updates (the block
 * factorisation and Schur-contribution steps of Alg. 2); launches3 (may be
 * NULL) the number of launch groups of each class.  Zero unless the option
 * profile_kernels was set for that factor. */
int kkt_factor_kernel_times(const ahlp_problem *p, double *ms3, int64_t *launches3);

/* Diagnostic: the tile jobs one block partial Cholesky gives its tensor-core
 * trailing updates, summed over the pivot steps: *kept those it runs (fewer
 * than *dense when the option tile_sparse leaves out structurally zero tile
 * products), *dense every (block, row-tile pair, column tile) of the dense
 * enumeration.  Both 0 until the handle's first tensor-core factor.  Either
 * pointer may be NULL. */
int kkt_update_jobs(const ahlp_problem *p, int64_t *kept, int64_t *dense);

/*
 * ahlp_tile_sparse_jobs -- host only (no handle, no device): the tile jobs of
 * the tensor-core trailing updates that the option tile_sparse keeps, for
 * nblk blocks of the batched partial Cholesky (the block factorisation and
 * Schur-contribution steps of Alg. 2, on 64 x 64 tiles).  Step k of a block
 * with T tiles and Tp pivot tiles updates its trailing tiles I, J > k with
 * L_Ik L_Jk'; a job is (block, first row tile I0, column tile J, 1 if row
 * tile I0 + 1 belongs to it), rows I0 = k+1, k+3, ... in pairs, columns J =
 * k+1 .. min(I0+1, T-1).  A tile-level symbolic factorisation (right-looking
 * fill) of each block's pattern leaves out the jobs whose column tile J, or
 * both row tiles, are zero in pivot column k.
 *
 *   T, Tp      nblk tile counts (1 <= T[b] <= 32768, 0 <= Tp[b] <= T[b]).
 *   nz         per block a T[b] x T[b] row-major byte matrix, nonzero where
 *              the formed matrix has an entry in tile (I, J) (lower triangle
 *              read), blocks concatenated; NULL: every tile nonzero.
 *   jobs       out, 4 int32 per kept job, ordered by step, block, row pair,
 *              column (the dense enumeration's order); may be NULL.
 *   step_off   out, max(Tp) + 1 offsets: the jobs of step k are
 *              [step_off[k], step_off[k+1]); may be NULL.
 *   cap        capacity of jobs in jobs.
 *   njobs      out, the jobs kept; ndense (may be NULL) the dense count.
 * Returns AHLP_ERR_INVALID_ARG for bad sizes, a NULL njobs, or cap < *njobs
 * with jobs given (then *njobs is set and nothing is written to jobs).
 */
int ahlp_tile_sparse_jobs(int32_t nblk, const int32_t *T, const int32_t *Tp, const uint8_t *nz,
                          int32_t *jobs, int64_t *step_off, int64_t cap, int64_t *njobs,
                          int64_t *ndense);

/* Diagnostic: bytes this handle has copied host -> device and device -> host
 * since arrowhead_lp_create (the problem upload included; scalars read back
 * by the solvers included).  Either pointer may be NULL. */
int ahlp_transfer_bytes(const ahlp_problem *p, int64_t *h2d, int64_t *d2h);

/*
 * kkt_residual_noalloc -- ||J d - r||_2 / ||r||_2 for a direction
 * d = (dx, dy, dz) and right-hand side r = (r_d, r_p, r_c) at the point of
 * the last kkt_factor, J the Newton matrix of kkt_solve.  The paper has no
 * counterpart: this is a utility for callers that cannot allocate device
 * memory when they need the check (a memory budget that forbids new
 * allocations, an allocator owned by another component, or code that must
 * avoid the synchronisation an allocation can cause).  It allocates
 * nothing: besides the caller's vectors and the existing handle it uses one
 * fixed 192 KB device array compiled into the library (per GPU, held until
 * the process exits).
 *   all seven pointers : device memory of the handle's device, which must
 *                        also be the current device (else
 *                        AHLP_ERR_INVALID_ARG); rel_out receives one double,
 *                        written asynchronously on the handle's stream
 *   limits             : n_total and m_total at most 67,108,864, else
 *                        AHLP_ERR_UNSUPPORTED
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call reuses the same array, and each call overwrites every slot it
 * reads, so nothing carries over between calls -- but calls that run at the
 * same time on the GPU (other streams, other handles, other threads) race on
 * it and must be serialised by the caller.
 */
int kkt_residual_noalloc(ahlp_problem *p, const double *r_d, const double *r_p,
                         const double *r_c, const double *dx, const double *dy,
                         const double *dz, double *rel_out);

#ifdef __cplusplus
}
#endif

#endif /* AHLP_H */
