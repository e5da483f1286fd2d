// ipm_solve: infeasible primal-dual Mehrotra predictor-corrector method
// (Sec. 2 and 2.3).  The host only steers (a handful of scalars per
// iteration); residuals, KKT factor/solve, ratio tests and updates all run
// in this library's kernels on the problem's stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <utility>

#include "ahlp_internal.h"

using namespace ahlp;

namespace {

enum {
  V_X = 0, V_Y, V_Z, V_RP, V_RD, V_RC, V_DXA, V_DYA, V_DZA, V_DX, V_DY, V_DZ,
  V_RC2, V_DX2, V_DY2, V_DZ2, V_SD, V_SP, V_SC
};

// Gondzio's cap on the centrality correctors of one iteration: how many
// solves the factorisation is worth, from a fixed cost model of this GPU's
// kernels (sustained rates of the block factor per precision; the
// preconditioner application reads every block factor twice at the rate the
// wavefront triangular solves reach).  A model instead of measured times
// keeps the iterates independent of clocks, load and profilers.
int corrector_budget(const ahlp_problem *p, int last_krylov_steps) {
  constexpr double kRateFP32 = 25e12, kRateFF = 3e12, kRateFP64 = 1e12;   // flop/s
  constexpr double kApplyBW = 1.3e12;                                      // bytes/s
  const double rate = p->fac_prec == kPrecFP32 ? kRateFP32
                      : p->fac_prec == kPrecFF ? kRateFF
                                               : kRateFP64;
  const double fac_s = p->fac_flops / rate;
  const double word = p->fac_prec == kPrecFP32 ? 4.0 : 8.0;
  const double apply_s = 2.0 * p->tri_elems * word / kApplyBW;
  const double solve_s = (last_krylov_steps + 1) * apply_s;
  if (!(solve_s > 0.0)) return 0;
  const double r = fac_s / solve_s;
  return r >= 8.0 ? 8 : (int)r;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

extern "C" int ipm_solve(ahlp_problem *p, const double *x0, const double *y0, const double *z0,
                         double *x, double *y, double *z, ahlp_result *res) {
  if (!p) return AHLP_ERR_INVALID_ARG;
  const double t_start = now_ms();
  ahlp_result R{};
  int status = AHLP_OK;
  try {
    cudaStream_t s = p->stream;
    const long long n = p->n, m = p->m;
    double **v = p->ipmv;
    double *X = v[V_X], *Y = v[V_Y], *Z = v[V_Z];
    const double eta = p->opt.eta;
    const double rho = p->opt.rho;
    // Safeguards of the factor, all kept for the later iterations once raised:
    //  - the block factors start in FP32 in mixed precision and move to
    //    float-float once D spans more than fp32_cond_max (or an FP32 factor
    //    produces a NaN), and to FP64 when float-float fails in turn;
    //  - the pivot clamping threshold starts at pivot_tol;
    //  - the regularisation starts at delta.
    // A direction whose Newton residual stays above `stalled` after the Krylov
    // refinement (the degenerate end game, where the clamped factors stop
    // being a good preconditioner) moves the blocks one precision up, else makes
    // the threshold 100x coarser (up to kMaxPivotTol).  A NaN in the factor or
    // in the direction does the same, except that a float-float factor first
    // gets delta 100x larger (up to kFFMaxDelta); once those are exhausted it
    // raises the regularisation 100x (up to kMaxDelta) and then regularises D
    // itself, d = x / (z + rho_x x) with rho_x from kMinRhoX up to kMaxRhoX,
    // which bounds the factor's conditioning when complementarity products
    // collapse.  The Krylov refinement always solves the unregularised Newton
    // system, so all this only weakens the preconditioner.  A NaN pivot that
    // passed the threshold is one that lost nearly all its digits to
    // cancellation; its rounding noise is amplified through the later clamped
    // columns.
    constexpr double kEscalate = 1e-6, kMaxPivotTol = 1e-8, kMaxDelta = 1e-4;
    constexpr double kMinRhoX = 1e-10, kMaxRhoX = 1e-6;
    // a float-float factor that breaks down (its FP32 exponent range is
    // exceeded behind clamped pivots) first gets more regularisation, up to
    // kFFMaxDelta, before the blocks move to FP64 at ~6x its cost
    constexpr double kFFMaxDelta = 1e-4;
    constexpr double kStallAccept = 1e-1;
    // inexact Newton: the IPM's directions are solved to a relative residual
    // of ipm_refine_tol, not the refine_tol of kkt_solve
    const double ipm_tol = std::max(p->opt.refine_tol, p->opt.ipm_refine_tol);
    // a direction counts as stalled above this (well clear of the target, so
    // that the Krylov estimate and the recomputed residual cannot straddle it)
    const double stalled = std::max(kEscalate, 10.0 * ipm_tol);
    p->fac_rho_x = rho > 0 ? rho : 0.0;
    constexpr double kCorrectorBelow = 0.9;   // correctors only below this step length
    double ptol = p->opt.pivot_tol;
    double delta = p->opt.delta;
    double last_rel = 0.0;
    int last_steps = 0;
    int cur_iter = 0;
    p->fac_prec = p->opt.precision == AHLP_PREC_MIXED ? kPrecFP32 : kPrecFP64;
    R.fp64_switch_iter = p->fac_prec == kPrecFP32 ? -1 : 0;
    // batch: LPs that already meet the tolerances stop moving (see below)
    const int nlp = p->batch > 1 ? (int)p->lp_rng.size() : 0;
    std::vector<char> frozen(nlp, 0);
    // set the x ranges (or y ranges) of the frozen LPs of vec to val
    auto fill_frozen = [&](double *vec, double val, bool on_y) {
      for (int b = 0; b < nlp; ++b) {
        if (!frozen[b]) continue;
        const auto &r = p->lp_rng[b];
        if (on_y) {
          ck(launch_fill(vec + r.yb0, val, r.yb1 - r.yb0, s), "fill");
          ck(launch_fill(vec + r.yl0, val, r.yl1 - r.yl0, s), "fill");
          ck(launch_fill(vec + r.yg0, val, r.yg1 - r.yg0, s), "fill");
        } else {
          ck(launch_fill(vec + r.xb0, val, r.xb1 - r.xb0, s), "fill");
          ck(launch_fill(vec + r.x00, val, r.x01 - r.x00, s), "fill");
        }
      }
    };
    auto factor_at = [&](const double *xx, const double *zz) {
      ck(cudaMemcpyAsync(p->x, xx, n * 8, cudaMemcpyDeviceToDevice, s), "copy");
      ck(cudaMemcpyAsync(p->z, zz, n * 8, cudaMemcpyDeviceToDevice, s), "copy");
      // a frozen LP of a batch sits at its converged, extremely ill-conditioned
      // point; its direction is zero (its right-hand sides are zeroed), so its
      // blocks are factored at x = z = 1 instead -- the LPs share no rows or
      // columns, so nothing else changes
      fill_frozen(p->x, 1.0, false);
      fill_frozen(p->z, 1.0, false);
      const int before = p->fac_prec;
      int st = factor_impl(p, delta, rho, ptol, false);
      if (before == kPrecFP32 && p->fac_prec != kPrecFP32 && R.fp64_switch_iter < 0)
        R.fp64_switch_iter = cur_iter;
      R.ms_factor += p->stage_ms[0] + p->stage_ms[1] + p->stage_ms[2];
      R.tiny_pivots = p->tiny_pivots;
      if (st == AHLP_OK) {
        if (p->fac_prec == kPrecFP32) {
          ++R.factors_fp32;
          R.ms_block_fp32 += p->stage_ms[1];
        } else if (p->fac_prec == kPrecFF) {
          ++R.factors_ff;
          R.ms_block_ff += p->stage_ms[1];
        } else {
          ++R.factors_fp64;
          R.ms_block_fp64 += p->stage_ms[1];
        }
      }
      return st;
    };
    // Batch: the Newton matrix is the direct sum of the LPs' ones, so every
    // LP's slice of the right-hand side can be scaled by its own factor and its
    // slice of the solution scaled back.  Each LP's slice is brought to unit
    // norm before the Krylov solve, so that the relative residual it is
    // stopped on bounds every LP's own relative residual, not a total that an
    // LP with a large right-hand side dominates.
    std::vector<double> lp_scale;
    int n_active = 0;   // LPs whose slice was brought to unit norm
    auto balance = [&](const double *rd, const double *rp, const double *rc) {
      lp_scale.assign(nlp, 1.0);
      n_active = 0;
      std::vector<double> nd(nlp);   // squared norm of each LP's slice
      for (int c0 = 0; c0 < nlp; c0 += 6) {
        const int cn = std::min(6, nlp - c0);
        for (int k = 0; k < cn; ++k) {
          const auto &r = p->lp_rng[c0 + k];
          double *sc = p->scal + 20 + 5 * k;
          ck(launch_reduce(p, RED_DOT, rd + r.xb0, rd + r.xb0, r.xb1 - r.xb0, sc + 0), "reduce");
          ck(launch_reduce(p, RED_DOT, rd + r.x00, rd + r.x00, r.x01 - r.x00, sc + 1), "reduce");
          ck(launch_reduce(p, RED_DOT, rc + r.xb0, rc + r.xb0, r.xb1 - r.xb0, sc + 2), "reduce");
          ck(launch_reduce(p, RED_DOT, rc + r.x00, rc + r.x00, r.x01 - r.x00, sc + 3), "reduce");
          ck(launch_reduce(p, RED_DOT, rp + r.yb0, rp + r.yb0, r.yb1 - r.yb0, sc + 4), "reduce");
        }
        read_scalars(p, 20 + 5 * cn);
        for (int k = 0; k < cn; ++k) {
          const double *h = p->h_scal + 20 + 5 * k;
          nd[c0 + k] = h[0] + h[1] + h[2] + h[3] + h[4];
        }
        // the link and global rows of each LP
        for (int k = 0; k < cn; ++k) {
          const auto &r = p->lp_rng[c0 + k];
          double *sc = p->scal + 20 + 2 * k;
          ck(launch_reduce(p, RED_DOT, rp + r.yl0, rp + r.yl0, r.yl1 - r.yl0, sc + 0), "reduce");
          ck(launch_reduce(p, RED_DOT, rp + r.yg0, rp + r.yg0, r.yg1 - r.yg0, sc + 1), "reduce");
        }
        read_scalars(p, 20 + 2 * cn);
        for (int k = 0; k < cn; ++k) nd[c0 + k] += p->h_scal[20 + 2 * k] + p->h_scal[21 + 2 * k];
      }
      const long long n = p->n, m = p->m;
      ck(cudaMemcpyAsync(v[V_SD], rd, n * 8, cudaMemcpyDeviceToDevice, s), "copy");
      ck(cudaMemcpyAsync(v[V_SP], rp, m * 8, cudaMemcpyDeviceToDevice, s), "copy");
      ck(cudaMemcpyAsync(v[V_SC], rc, n * 8, cudaMemcpyDeviceToDevice, s), "copy");
      auto scale = [&](double *vec, long long lo, long long hi, double f) {
        if (hi > lo) ck(launch_axpby(vec + lo, vec + lo, f - 1.0, 1.0, hi - lo, s), "scale");
      };
      for (int b = 0; b < nlp; ++b) {
        const double nrm = std::sqrt(nd[b]);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) continue;   // a frozen LP: zero stays zero
        lp_scale[b] = nrm;
        ++n_active;
        const auto &r = p->lp_rng[b];
        const double f = 1.0 / nrm;
        scale(v[V_SD], r.xb0, r.xb1, f);
        scale(v[V_SD], r.x00, r.x01, f);
        scale(v[V_SC], r.xb0, r.xb1, f);
        scale(v[V_SC], r.x00, r.x01, f);
        scale(v[V_SP], r.yb0, r.yb1, f);
        scale(v[V_SP], r.yl0, r.yl1, f);
        scale(v[V_SP], r.yg0, r.yg1, f);
      }
    };
    auto unbalance = [&](double *dx, double *dy, double *dz) {
      auto scale = [&](double *vec, long long lo, long long hi, double f) {
        if (hi > lo && f != 1.0) ck(launch_axpby(vec + lo, vec + lo, f - 1.0, 1.0, hi - lo, s), "scale");
      };
      for (int b = 0; b < nlp; ++b) {
        const auto &r = p->lp_rng[b];
        const double f = lp_scale[b];
        scale(dx, r.xb0, r.xb1, f);
        scale(dx, r.x00, r.x01, f);
        scale(dz, r.xb0, r.xb1, f);
        scale(dz, r.x00, r.x01, f);
        scale(dy, r.yb0, r.yb1, f);
        scale(dy, r.yl0, r.yl1, f);
        scale(dy, r.yg0, r.yg1, f);
      }
    };
    auto solve = [&](const double *rd, const double *rp, const double *rc, double *dx, double *dy,
                     double *dz) {
      ahlp_solve_info info{};
      if (nlp > 0) {
        balance(rd, rp, rc);
        rd = v[V_SD];
        rp = v[V_SP];
        rc = v[V_SC];
      }
      int st = solve_impl(p, rd, rp, rc, dx, dy, dz, false, &info, ipm_tol);
      if (nlp > 0 && st == AHLP_OK) unbalance(dx, dy, dz);
      R.ms_solve += p->stage_ms[3];
      R.refine_steps += info.refine_steps;
      R.kkt_residual = std::max(R.kkt_residual, info.rel_residual);
      last_rel = info.rel_residual;
      last_steps = info.refine_steps;
      return st;
    };
    static const char *kPrecName[] = {"FP64", "FP32", "float-float"};
    // next safeguard; false when none is left (allow_delta: NaN recovery only)
    auto escalate = [&](bool allow_delta, const char *why) {
      // A stalled direction (Krylov budget spent above `stalled`) whose
      // residual is still at most kStallAccept is an acceptable inexact
      // Newton step once the remaining safeguards are an FP64 refactor or a
      // coarser pivot threshold: in the degenerate end game the factors of
      // every precision stop being good preconditioners (FP64 ones too), so
      // a refactor costs several float-float factors and buys no accuracy.
      // In a batch every active LP's slice of the right-hand side has unit
      // norm (balance), so the total relative residual times sqrt(active
      // LPs) bounds each LP's own relative residual, and that bound is what
      // is tested.
      const double per_lp =
          nlp > 0 ? last_rel * std::sqrt((double)std::max(n_active, 1)) : last_rel;
      if (!allow_delta && per_lp <= kStallAccept &&
          (p->fac_prec == kPrecFF || p->fac_prec == kPrecFP64)) {
        if (p->opt.verbose)
          printf("       %s accepted (%s factor, residual %.2e)\n", why,
                 kPrecName[p->fac_prec], last_rel);
        return false;
      }
      if (p->opt.verbose)
        printf("       safeguard after %s (%s factor, residual %.2e)\n", why,
               kPrecName[p->fac_prec], last_rel);
      if (allow_delta && p->fac_prec == kPrecFF && delta > 0 &&
          delta * 100.0 <= kFFMaxDelta * 1.0001) {
        delta *= 100.0;
      } else if (p->fac_prec != kPrecFP64) {   // FP32 -> float-float -> FP64
        if (p->fac_prec == kPrecFP32 && R.fp64_switch_iter < 0) R.fp64_switch_iter = cur_iter;
        p->fac_prec = p->fac_prec == kPrecFP32 ? kPrecFF : kPrecFP64;
      } else if (ptol * 100.0 <= kMaxPivotTol * 1.0001) {
        ptol *= 100.0;
      } else if (allow_delta && delta > 0 && delta * 100.0 <= kMaxDelta * 1.0001) {
        delta *= 100.0;
      } else if (allow_delta && p->fac_rho_x * 100.0 <= kMaxRhoX * 1.0001) {
        // primal regularisation of the preconditioner: d = x / (z + rho_x x)
        p->fac_rho_x = p->fac_rho_x > 0.0 ? p->fac_rho_x * 100.0 : kMinRhoX;
      } else {
        return false;
      }
      ++R.escalations;
      return true;
    };
    // Batch (a direct sum of independent LPs).  Each LP runs its own IPM on
    // the shared factorisations: its own mu, sigma and primal / dual step
    // lengths, computed over its index ranges, and it stops moving once it
    // meets the tolerances on its own (its D then stays fixed and well
    // conditioned while the others converge).  The reported measures are the
    // worst LP's.  Reductions over the LPs' ranges go through scalar slots
    // 20..51, sixteen LPs per host read.
    std::vector<double> lp_mu(nlp, 0.0), lp_ap(nlp, 0.0), lp_ad(nlp, 0.0), lp_smu(nlp, 0.0);
    auto lp_nx = [&](const ahlp_problem::LpRange &r) {
      return (double)((r.xb1 - r.xb0) + (r.x01 - r.x00));
    };
    // out[b] = op over LP b's x ranges (min for step lengths, sum for dots)
    auto lp_xreduce = [&](int op, const double *a, const double *bv, std::vector<double> &out) {
      for (int c0 = 0; c0 < nlp; c0 += 16) {
        const int cn = std::min(16, nlp - c0);
        for (int k = 0; k < cn; ++k) {
          const auto &r = p->lp_rng[c0 + k];
          ck(launch_reduce(p, op, a + r.xb0, bv ? bv + r.xb0 : nullptr, r.xb1 - r.xb0,
                           p->scal + 20 + 2 * k),
             "reduce");
          ck(launch_reduce(p, op, a + r.x00, bv ? bv + r.x00 : nullptr, r.x01 - r.x00,
                           p->scal + 21 + 2 * k),
             "reduce");
        }
        read_scalars(p, 20 + 2 * cn);
        for (int k = 0; k < cn; ++k) {
          const double u = p->h_scal[20 + 2 * k], w = p->h_scal[21 + 2 * k];
          out[c0 + k] = op == RED_MINSTEP ? std::min(u, w) : u + w;
        }
      }
    };
    // per-LP measures; freezes the LPs that meet the tolerances; true when all do
    auto batch_measures = [&]() {
      double wp = 0.0, wd = 0.0, wg = 0.0;
      for (int b = 0; b < nlp; ++b) {
        const auto &r = p->lp_rng[b];
        double *sc = p->scal + 20;
        ck(launch_reduce(p, RED_MAXABS, v[V_RP] + r.yb0, nullptr, r.yb1 - r.yb0, sc + 0), "reduce");
        ck(launch_reduce(p, RED_MAXABS, v[V_RP] + r.yl0, nullptr, r.yl1 - r.yl0, sc + 1), "reduce");
        ck(launch_reduce(p, RED_MAXABS, v[V_RP] + r.yg0, nullptr, r.yg1 - r.yg0, sc + 2), "reduce");
        ck(launch_reduce(p, RED_MAXABS, v[V_RD] + r.xb0, nullptr, r.xb1 - r.xb0, sc + 3), "reduce");
        ck(launch_reduce(p, RED_MAXABS, v[V_RD] + r.x00, nullptr, r.x01 - r.x00, sc + 4), "reduce");
        ck(launch_reduce(p, RED_DOT, p->c + r.xb0, X + r.xb0, r.xb1 - r.xb0, sc + 5), "reduce");
        ck(launch_reduce(p, RED_DOT, p->c + r.x00, X + r.x00, r.x01 - r.x00, sc + 6), "reduce");
        ck(launch_reduce(p, RED_DOT, p->b + r.yb0, Y + r.yb0, r.yb1 - r.yb0, sc + 7), "reduce");
        ck(launch_reduce(p, RED_DOT, p->b + r.yl0, Y + r.yl0, r.yl1 - r.yl0, sc + 8), "reduce");
        ck(launch_reduce(p, RED_DOT, p->b + r.yg0, Y + r.yg0, r.yg1 - r.yg0, sc + 9), "reduce");
        ck(launch_reduce(p, RED_DOT, X + r.xb0, Z + r.xb0, r.xb1 - r.xb0, sc + 10), "reduce");
        ck(launch_reduce(p, RED_DOT, X + r.x00, Z + r.x00, r.x01 - r.x00, sc + 11), "reduce");
        read_scalars(p, 32);
        const double *h = p->h_scal + 20;
        const double pinf = std::max({h[0], h[1], h[2]}) / (1.0 + r.bnorm);
        const double dinf = std::max(h[3], h[4]) / (1.0 + r.cnorm);
        const double pobj = h[5] + h[6], dobj = h[7] + h[8] + h[9];
        const double gap = std::fabs(pobj - dobj) / (1.0 + std::fabs(pobj));
        lp_mu[b] = (h[10] + h[11]) / std::max(lp_nx(r), 1.0);
        if (pinf <= p->opt.tol && dinf <= p->opt.tol && gap <= p->opt.tol) frozen[b] = 1;
        wp = std::max(wp, pinf);
        wd = std::max(wd, dinf);
        wg = std::max(wg, gap);
      }
      R.pinf = wp;
      R.dinf = wd;
      R.rel_gap = wg;
      for (int b = 0; b < nlp; ++b)
        if (!frozen[b]) return false;
      return true;
    };
    // LP-wise axpby over its x ranges (y ranges when on_y): y += a_b x
    auto lp_axpy = [&](double *yv, const double *xv, const std::vector<double> &a, bool on_y) {
      for (int b = 0; b < nlp; ++b) {
        const auto &r = p->lp_rng[b];
        if (a[b] == 0.0) continue;
        if (on_y) {
          ck(launch_axpby(yv + r.yb0, xv + r.yb0, a[b], 1.0, r.yb1 - r.yb0, s), "update");
          ck(launch_axpby(yv + r.yl0, xv + r.yl0, a[b], 1.0, r.yl1 - r.yl0, s), "update");
          ck(launch_axpby(yv + r.yg0, xv + r.yg0, a[b], 1.0, r.yg1 - r.yg0, s), "update");
        } else {
          ck(launch_axpby(yv + r.xb0, xv + r.xb0, a[b], 1.0, r.xb1 - r.xb0, s), "update");
          ck(launch_axpby(yv + r.x00, xv + r.x00, a[b], 1.0, r.x01 - r.x00, s), "update");
        }
      }
    };
    const bool warm = x0 && y0 && z0;
    if (warm) {
      const double *a = stage_in(p, x0, n, p->stg[0]);
      ck(cudaMemcpyAsync(X, a, n * 8, cudaMemcpyDeviceToDevice, s), "copy");
      const double *b = stage_in(p, y0, m, p->stg[1]);
      ck(cudaMemcpyAsync(Y, b, m * 8, cudaMemcpyDeviceToDevice, s), "copy");
      const double *c = stage_in(p, z0, n, p->stg[2]);
      ck(cudaMemcpyAsync(Z, c, n * 8, cudaMemcpyDeviceToDevice, s), "copy");
    } else {
      // Mehrotra's starting point from two solves at D = I
      double *ones = v[V_RC], *zero_n = v[V_RD], *zero_m = v[V_RP];
      ck(launch_fill(ones, 1.0, n, s), "fill");
      ck(launch_fill(zero_n, 0.0, n, s), "fill");
      ck(launch_fill(zero_m, 0.0, m, s), "fill");
      int st = factor_at(ones, ones);
      if (st != AHLP_OK) throw Fail{st, p->err};
      ck(launch_fill(ones, 0.0, n, s), "fill");   // r_c = 0 from here on
      // x~ = A'(AA')^-1 b
      st = solve(zero_n, p->b, ones, v[V_DX], v[V_DY], v[V_DZ]);
      if (st != AHLP_OK) throw Fail{st, p->err};
      // y~ = (AA')^-1 A c, z~ = c - A'y~ (= the dz of this solve)
      st = solve(p->c, zero_m, ones, v[V_DXA], Y, Z);
      if (st != AHLP_OK) throw Fail{st, p->err};
      ck(cudaMemcpyAsync(X, v[V_DX], n * 8, cudaMemcpyDeviceToDevice, s), "copy");
      ck(launch_reduce(p, RED_MIN, X, nullptr, n, p->scal + 0), "reduce");
      ck(launch_reduce(p, RED_MIN, Z, nullptr, n, p->scal + 1), "reduce");
      read_scalars(p, 2);
      ck(launch_add_scalar(X, X, std::max(-1.5 * p->h_scal[0], 0.0), n, s), "shift");
      ck(launch_add_scalar(Z, Z, std::max(-1.5 * p->h_scal[1], 0.0), n, s), "shift");
      ck(launch_reduce(p, RED_DOT, X, Z, n, p->scal + 0), "reduce");
      ck(launch_reduce(p, RED_SUM, X, nullptr, n, p->scal + 1), "reduce");
      ck(launch_reduce(p, RED_SUM, Z, nullptr, n, p->scal + 2), "reduce");
      read_scalars(p, 3);
      const double xz = p->h_scal[0], sx = p->h_scal[1], sz = p->h_scal[2];
      const double ax = sz > 0 ? 0.5 * xz / sz : 1.0, az = sx > 0 ? 0.5 * xz / sx : 1.0;
      ck(launch_add_scalar(X, X, ax > 0 ? ax : 1.0, n, s), "shift");
      ck(launch_add_scalar(Z, Z, az > 0 ? az : 1.0, n, s), "shift");
    }
    int it = 0;
    constexpr double kDiverge = 1e12;
    double xscale0 = 0.0, yscale0 = 0.0;
    status = AHLP_ERR_MAX_ITER;
    for (it = 0;; ++it) {
      // residuals r_p = b - Ax, r_d = c - A'y - z
      ck(launch_spmv(p->Amat, X, v[V_RP], -1.0, p->b, s), "spmv");
      ck(launch_spmv(p->ATmat, Y, v[V_RD], -1.0, p->c, s), "spmv");
      ck(launch_axpby(v[V_RD], Z, -1.0, 1.0, n, s), "axpby");
      ck(launch_reduce(p, RED_MAXABS, v[V_RP], nullptr, m, p->scal + 0), "reduce");
      ck(launch_reduce(p, RED_MAXABS, v[V_RD], nullptr, n, p->scal + 1), "reduce");
      ck(launch_reduce(p, RED_DOT, p->c, X, n, p->scal + 2), "reduce");
      ck(launch_reduce(p, RED_DOT, p->b, Y, m, p->scal + 3), "reduce");
      ck(launch_reduce(p, RED_DOT, X, Z, n, p->scal + 4), "reduce");
      ck(launch_reduce(p, RED_MAXABS, X, nullptr, n, p->scal + 5), "reduce");
      ck(launch_reduce(p, RED_MAXABS, Y, nullptr, m, p->scal + 6), "reduce");
      read_scalars(p, 7);
      const double *hs = p->h_scal;
      R.pinf = hs[0] / (1.0 + p->bnorm_inf);
      R.dinf = hs[1] / (1.0 + p->cnorm_inf);
      R.pobj = hs[2];
      R.dobj = hs[3];
      R.rel_gap = std::fabs(hs[2] - hs[3]) / (1.0 + std::fabs(hs[2]));
      R.mu = n > 0 ? hs[4] / n : 0.0;
      R.iterations = it;
      if (p->opt.verbose) {
        printf("ipm %3d  pobj %+.10e  dobj %+.10e  pinf %.2e  dinf %.2e  gap %.2e  mu %.2e", it,
               R.pobj, R.dobj, R.pinf, R.dinf, R.rel_gap, R.mu);
        if (nlp > 0) {
          int nf = 0;
          for (int b = 0; b < nlp; ++b) nf += frozen[b];
          printf("  frozen %d/%d", nf, nlp);
        }
        printf("\n");
      }
      if (p->opt.iter_cb && p->opt.iter_cb(p->opt.iter_cb_ctx, it, &R) != 0) {
        status = AHLP_ERR_STOPPED;
        p->err = "ipm_solve: stopped by the iteration callback";
        break;
      }
      if (!(R.pinf == R.pinf) || !(R.dinf == R.dinf)) {
        status = AHLP_ERR_NOT_SPD;
        p->err = "ipm_solve: NaN in the iterate";
        break;
      }
      if (nlp > 0) {
        if (batch_measures()) {
          status = AHLP_OK;
          break;
        }
        fill_frozen(v[V_RD], 0.0, false);
        fill_frozen(v[V_RP], 0.0, true);
      } else if (R.pinf <= p->opt.tol && R.dinf <= p->opt.tol && R.rel_gap <= p->opt.tol) {
        status = AHLP_OK;
        break;
      }
      // divergence: an infeasible LP drives y (a dual ray) and an unbounded
      // one drives x (a primal ray) to infinity, while a solvable LP's
      // iterates stay within a moderate factor of the starting point's scale
      if (it == 0) {
        xscale0 = hs[5];
        yscale0 = hs[6];
      }
      if (hs[5] > 1e30 || hs[6] > 1e30 || hs[5] > kDiverge * (1.0 + xscale0) ||
          hs[6] > kDiverge * (1.0 + yscale0)) {
        status = AHLP_ERR_INFEASIBLE;
        p->err = "ipm_solve: iterates diverge (LP infeasible or unbounded)";
        break;
      }
      if (it >= p->opt.max_iter) {
        status = AHLP_ERR_MAX_ITER;
        p->err = "ipm_solve: iteration limit reached";
        break;
      }
      const double mu = R.mu;
      cur_iter = it;
      double sigma = 0.0;
      for (;;) {
        int st = factor_at(X, Z);
        if (st == AHLP_ERR_NOT_SPD && p->opt.verbose) printf("       %s\n", p->err.c_str());
        if (st == AHLP_ERR_NOT_SPD && escalate(true, "a NaN pivot")) continue;
        if (st != AHLP_OK) throw Fail{st, p->err};
        // predictor: r_c = -XZe
        ck(launch_mul(v[V_RC], X, Z, -1.0, n, s), "mul");
        fill_frozen(v[V_RC], 0.0, false);
        st = solve(v[V_RD], v[V_RP], v[V_RC], v[V_DXA], v[V_DYA], v[V_DZA]);
        if (st == AHLP_ERR_NOT_SPD && escalate(true, "a NaN predictor")) continue;
        if (st != AHLP_OK) throw Fail{st, p->err};
        if (last_rel > stalled && escalate(false, "a stalled predictor")) continue;
        const int pred_steps = last_steps;
        const double pred_rel = last_rel;
        if (nlp > 0) {
          // each LP's affine step, mu_aff and sigma, and its corrector rhs
          lp_xreduce(RED_MINSTEP, X, v[V_DXA], lp_ap);
          lp_xreduce(RED_MINSTEP, Z, v[V_DZA], lp_ad);
          for (int c0 = 0; c0 < nlp; c0 += 16) {
            const int cn = std::min(16, nlp - c0);
            for (int k = 0; k < cn; ++k) {
              const auto &r = p->lp_rng[c0 + k];
              const double a1 = std::min(1.0, lp_ap[c0 + k]), a2 = std::min(1.0, lp_ad[c0 + k]);
              ck(launch_step_dot(X + r.xb0, v[V_DXA] + r.xb0, a1, Z + r.xb0, v[V_DZA] + r.xb0, a2,
                                 r.xb1 - r.xb0, p->red_part, p->scal + 20 + 2 * k, s),
                 "reduce");
              ck(launch_step_dot(X + r.x00, v[V_DXA] + r.x00, a1, Z + r.x00, v[V_DZA] + r.x00, a2,
                                 r.x01 - r.x00, p->red_part, p->scal + 21 + 2 * k, s),
                 "reduce");
            }
            read_scalars(p, 20 + 2 * cn);
            for (int k = 0; k < cn; ++k) {
              if (frozen[c0 + k]) continue;   // its r_c stays zero
              const auto &r = p->lp_rng[c0 + k];
              const double mua = (p->h_scal[20 + 2 * k] + p->h_scal[21 + 2 * k]) /
                                 std::max(lp_nx(r), 1.0);
              const double mub = lp_mu[c0 + k];
              const double sig = mub > 0.0 ? std::pow(mua / mub, 3.0) : 0.0;
              lp_smu[c0 + k] = sig * mub;
              ck(launch_ipm_rc(v[V_RC] + r.xb0, X + r.xb0, Z + r.xb0, v[V_DXA] + r.xb0,
                               v[V_DZA] + r.xb0, sig * mub, r.xb1 - r.xb0, s),
                 "rc");
              ck(launch_ipm_rc(v[V_RC] + r.x00, X + r.x00, Z + r.x00, v[V_DXA] + r.x00,
                               v[V_DZA] + r.x00, sig * mub, r.x01 - r.x00, s),
                 "rc");
            }
          }
        } else {
          ck(launch_reduce(p, RED_MINSTEP, X, v[V_DXA], n, p->scal + 0), "reduce");
          ck(launch_reduce(p, RED_MINSTEP, Z, v[V_DZA], n, p->scal + 1), "reduce");
          read_scalars(p, 2);
          const double apa = std::min(1.0, p->h_scal[0]), ada = std::min(1.0, p->h_scal[1]);
          ck(launch_step_dot(X, v[V_DXA], apa, Z, v[V_DZA], ada, n, p->red_part, p->scal + 0, s),
             "reduce");
          read_scalars(p, 1);
          const double mu_aff = p->h_scal[0] / n;
          sigma = std::pow(mu_aff / mu, 3.0);
          // corrector: r_c = sigma mu e - XZe - dXa dZa e
          ck(launch_ipm_rc(v[V_RC], X, Z, v[V_DXA], v[V_DZA], sigma * mu, n, s), "rc");
        }
        st = solve(v[V_RD], v[V_RP], v[V_RC], v[V_DX], v[V_DY], v[V_DZ]);
        if (st == AHLP_ERR_NOT_SPD && escalate(true, "a NaN corrector")) continue;
        if (st != AHLP_OK) throw Fail{st, p->err};
        if (last_rel > stalled && escalate(false, "a stalled corrector")) continue;
        if (p->opt.verbose)
          printf("       %s factor %.1f ms; predictor %d steps (%.1e), corrector %d steps (%.1e)\n",
                 kPrecName[p->fac_prec], p->stage_ms[0] + p->stage_ms[1] + p->stage_ms[2],
                 pred_steps, pred_rel, last_steps, last_rel);
        break;
      }
      // Multiple centrality correctors (Gondzio), reusing the factor: the
      // products (x + a dx)(z + a dz) at an enlarged trial step are pushed into
      // [0.1 sigma mu, 10 sigma mu]; a corrected direction is kept only while
      // it lengthens the step.  Tried only when the step is short, and at
      // most as many as the factorisation costs in solves (Gondzio's rule).
      // Both costs come from a fixed model of the work, not from timings, so
      // that the trajectory is reproducible: a block factor is its flops at
      // its precision's rate, a solve is its preconditioner applications (the
      // last direction's Krylov steps + 1), each reading every block factor
      // twice at the achieved bandwidth of the triangular solves.
      const int kmax = p->opt.correctors_by_cost
                           ? std::min(p->opt.max_correctors, corrector_budget(p, last_steps))
                           : p->opt.max_correctors;
      if (kmax > 0 && nlp == 0) {
        auto steps = [&](const double *dxv, const double *dzv, double &a_p, double &a_d) {
          ck(launch_reduce(p, RED_MINSTEP, X, dxv, n, p->scal + 0), "reduce");
          ck(launch_reduce(p, RED_MINSTEP, Z, dzv, n, p->scal + 1), "reduce");
          read_scalars(p, 2);
          a_p = std::min(1.0, p->h_scal[0]);
          a_d = std::min(1.0, p->h_scal[1]);
        };
        double a_p = 1.0, a_d = 1.0;
        steps(v[V_DX], v[V_DZ], a_p, a_d);
        for (int k = 0; k < kmax && std::min(a_p, a_d) < kCorrectorBelow; ++k) {
          const double tp = std::min(1.0, 1.5 * a_p + 0.1), td = std::min(1.0, 1.5 * a_d + 0.1);
          const double smu = sigma * mu;
          ck(launch_centrality_rc(v[V_RC2], v[V_RC], X, v[V_DX], tp, Z, v[V_DZ], td, 0.1 * smu,
                                  10.0 * smu, n, s),
             "corrector rhs");
          const int st = solve(v[V_RD], v[V_RP], v[V_RC2], v[V_DX2], v[V_DY2], v[V_DZ2]);
          if (st != AHLP_OK || last_rel > stalled) break;   // keep the previous direction
          double b_p = 0.0, b_d = 0.0;
          steps(v[V_DX2], v[V_DZ2], b_p, b_d);
          if (!(std::min(b_p, b_d) >= 1.01 * std::min(a_p, a_d))) break;
          std::swap(v[V_DX], v[V_DX2]);
          std::swap(v[V_DY], v[V_DY2]);
          std::swap(v[V_DZ], v[V_DZ2]);
          std::swap(v[V_RC], v[V_RC2]);
          a_p = b_p;
          a_d = b_d;
          ++R.correctors;
        }
      } else if (kmax > 0) {
        // batch: one shared solve per corrector round; every LP whose step is
        // still short gets its own centrality term (its own sigma mu and
        // trial steps) and keeps the corrected slice of the direction only if
        // its own step grows; an LP that stops improving drops out
        lp_xreduce(RED_MINSTEP, X, v[V_DX], lp_ap);
        lp_xreduce(RED_MINSTEP, Z, v[V_DZ], lp_ad);
        std::vector<char> active(nlp, 0);
        for (int k = 0; k < kmax; ++k) {
          int nact = 0;
          ck(cudaMemcpyAsync(v[V_RC2], v[V_RC], n * 8, cudaMemcpyDeviceToDevice, s), "copy");
          for (int b = 0; b < nlp; ++b) {
            const double ab = std::min(std::min(1.0, lp_ap[b]), std::min(1.0, lp_ad[b]));
            active[b] = (k == 0 || active[b]) && !frozen[b] && ab < kCorrectorBelow;
            if (!active[b]) continue;
            ++nact;
            const auto &r = p->lp_rng[b];
            const double tp = std::min(1.0, 1.5 * std::min(1.0, lp_ap[b]) + 0.1);
            const double td = std::min(1.0, 1.5 * std::min(1.0, lp_ad[b]) + 0.1);
            const double smu = lp_smu[b];
            ck(launch_centrality_rc(v[V_RC2] + r.xb0, v[V_RC] + r.xb0, X + r.xb0,
                                    v[V_DX] + r.xb0, tp, Z + r.xb0, v[V_DZ] + r.xb0, td,
                                    0.1 * smu, 10.0 * smu, r.xb1 - r.xb0, s),
               "corrector rhs");
            ck(launch_centrality_rc(v[V_RC2] + r.x00, v[V_RC] + r.x00, X + r.x00,
                                    v[V_DX] + r.x00, tp, Z + r.x00, v[V_DZ] + r.x00, td,
                                    0.1 * smu, 10.0 * smu, r.x01 - r.x00, s),
               "corrector rhs");
          }
          if (nact == 0) break;
          const int st = solve(v[V_RD], v[V_RP], v[V_RC2], v[V_DX2], v[V_DY2], v[V_DZ2]);
          if (st != AHLP_OK || last_rel > stalled) break;   // keep the previous direction
          std::vector<double> bp(nlp, 0.0), bd(nlp, 0.0);
          lp_xreduce(RED_MINSTEP, X, v[V_DX2], bp);
          lp_xreduce(RED_MINSTEP, Z, v[V_DZ2], bd);
          auto take = [&](double *dst, const double *src, long long lo, long long hi) {
            if (hi > lo)
              ck(cudaMemcpyAsync(dst + lo, src + lo, (hi - lo) * 8, cudaMemcpyDeviceToDevice, s),
                 "copy");
          };
          for (int b = 0; b < nlp; ++b) {
            if (!active[b]) continue;
            const double a0 = std::min(std::min(1.0, lp_ap[b]), std::min(1.0, lp_ad[b]));
            const double a1 = std::min(std::min(1.0, bp[b]), std::min(1.0, bd[b]));
            if (!(a1 >= 1.01 * a0)) {
              active[b] = 0;
              continue;
            }
            const auto &r = p->lp_rng[b];
            for (auto [dst, src] : {std::pair<double *, double *>{v[V_DX], v[V_DX2]},
                                   {v[V_DZ], v[V_DZ2]}, {v[V_RC], v[V_RC2]}}) {
              take(dst, src, r.xb0, r.xb1);
              take(dst, src, r.x00, r.x01);
            }
            take(v[V_DY], v[V_DY2], r.yb0, r.yb1);
            take(v[V_DY], v[V_DY2], r.yl0, r.yl1);
            take(v[V_DY], v[V_DY2], r.yg0, r.yg1);
            lp_ap[b] = bp[b];
            lp_ad[b] = bd[b];
            ++R.correctors;
          }
        }
      }
      if (nlp > 0) {
        lp_xreduce(RED_MINSTEP, X, v[V_DX], lp_ap);
        lp_xreduce(RED_MINSTEP, Z, v[V_DZ], lp_ad);
        for (int b = 0; b < nlp; ++b) {
          lp_ap[b] = frozen[b] ? 0.0 : std::min(1.0, eta * lp_ap[b]);
          lp_ad[b] = frozen[b] ? 0.0 : std::min(1.0, eta * lp_ad[b]);
        }
        lp_axpy(X, v[V_DX], lp_ap, false);
        lp_axpy(Y, v[V_DY], lp_ad, true);
        lp_axpy(Z, v[V_DZ], lp_ad, false);
        continue;
      }
      ck(launch_reduce(p, RED_MINSTEP, X, v[V_DX], n, p->scal + 0), "reduce");
      ck(launch_reduce(p, RED_MINSTEP, Z, v[V_DZ], n, p->scal + 1), "reduce");
      read_scalars(p, 2);
      const double ap = std::min(1.0, eta * p->h_scal[0]), ad = std::min(1.0, eta * p->h_scal[1]);
      ck(launch_axpby(X, v[V_DX], ap, 1.0, n, s), "update");
      ck(launch_axpby(Y, v[V_DY], ad, 1.0, m, s), "update");
      ck(launch_axpby(Z, v[V_DZ], ad, 1.0, n, s), "update");
    }
    // outputs
    auto put = [&](double *dst, const double *src, long long len) {
      if (!dst || len == 0) return;
      if (!is_device_ptr(dst)) p->bytes_d2h += len * 8;
      ck(cudaMemcpyAsync(dst, src, len * 8,
                         is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
         "copy out");
    };
    put(x, X, n);
    put(y, Y, m);
    put(z, Z, n);
    ck(cudaStreamSynchronize(s), "sync");
  } catch (const Fail &f) {
    status = f.code;
    p->err = f.msg;
  }
  R.status = status;
  R.ms_total = now_ms() - t_start;
  if (res) *res = R;
  return status;
}
