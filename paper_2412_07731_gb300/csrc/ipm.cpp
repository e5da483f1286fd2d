// ipm_solve: infeasible primal-dual Mehrotra predictor-corrector method
// (Sec. 2 and 2.3).  The host only steers (a handful of scalars per
// iteration); residuals, KKT factor/solve, ratio tests and updates all run
// in this library's kernels on the problem's stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>

#include "ahlp_internal.h"

using namespace ahlp;

namespace {

enum {
  V_X = 0, V_Y, V_Z, V_RP, V_RD, V_RC, V_DXA, V_DYA, V_DZA, V_DX, V_DY, V_DZ,
  V_RC2, V_DX2, V_DY2, V_DZ2
};

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
    // A direction whose Newton residual stays above kEscalate after the Krylov
    // refinement (the degenerate end game, where the clamped factors stop
    // being a good preconditioner) moves the blocks one precision up, else makes
    // the threshold 100x coarser (up to kMaxPivotTol).  A NaN in the factor or
    // in the direction does the same and, once those are exhausted, raises
    // the regularisation 100x (up to kMaxDelta): the Krylov refinement always
    // solves the unregularised Newton system, so this only weakens the
    // preconditioner.  A NaN pivot that passed the threshold is one that lost
    // nearly all its digits to cancellation; its rounding noise is amplified
    // through the later clamped columns.
    constexpr double kEscalate = 1e-6, kMaxPivotTol = 1e-8, kMaxDelta = 1e-4;
    constexpr double kCorrectorBelow = 0.9;   // correctors only below this step length
    double ptol = p->opt.pivot_tol;
    double delta = p->opt.delta;
    double last_rel = 0.0;
    int cur_iter = 0;
    p->fac_prec = p->opt.precision == AHLP_PREC_MIXED ? kPrecFP32 : kPrecFP64;
    R.fp64_switch_iter = p->fac_prec == kPrecFP32 ? -1 : 0;
    auto factor_at = [&](const double *xx, const double *zz) {
      ck(cudaMemcpyAsync(p->x, xx, n * 8, cudaMemcpyDeviceToDevice, s), "copy");
      ck(cudaMemcpyAsync(p->z, zz, n * 8, cudaMemcpyDeviceToDevice, s), "copy");
      const int before = p->fac_prec;
      int st = factor_impl(p, delta, rho, ptol);
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
    auto solve = [&](const double *rd, const double *rp, const double *rc, double *dx, double *dy,
                     double *dz) {
      ahlp_solve_info info{};
      int st = solve_impl(p, rd, rp, rc, dx, dy, dz, false, &info);
      R.ms_solve += p->stage_ms[3];
      R.refine_steps += info.refine_steps;
      R.kkt_residual = std::max(R.kkt_residual, info.rel_residual);
      last_rel = info.rel_residual;
      return st;
    };
    // next safeguard; false when none is left (allow_delta: NaN recovery only)
    auto escalate = [&](bool allow_delta) {
      if (p->fac_prec != kPrecFP64) {   // FP32 -> float-float -> FP64
        if (p->fac_prec == kPrecFP32 && R.fp64_switch_iter < 0) R.fp64_switch_iter = cur_iter;
        p->fac_prec = p->fac_prec == kPrecFP32 ? kPrecFF : kPrecFP64;
      } else if (ptol * 100.0 <= kMaxPivotTol * 1.0001) {
        ptol *= 100.0;
      } else if (allow_delta && delta > 0 && delta * 100.0 <= kMaxDelta * 1.0001) {
        delta *= 100.0;
      } else {
        return false;
      }
      ++R.escalations;
      return true;
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
      if (p->opt.verbose)
        printf("ipm %3d  pobj %+.10e  dobj %+.10e  pinf %.2e  dinf %.2e  gap %.2e  mu %.2e\n", it,
               R.pobj, R.dobj, R.pinf, R.dinf, R.rel_gap, R.mu);
      if (!(R.pinf == R.pinf) || !(R.dinf == R.dinf)) {
        status = AHLP_ERR_NOT_SPD;
        p->err = "ipm_solve: NaN in the iterate";
        break;
      }
      if (R.pinf <= p->opt.tol && R.dinf <= p->opt.tol && R.rel_gap <= p->opt.tol) {
        status = AHLP_OK;
        break;
      }
      if (hs[5] > 1e30 || hs[6] > 1e30) {
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
        if (st == AHLP_ERR_NOT_SPD && escalate(true)) continue;
        if (st != AHLP_OK) throw Fail{st, p->err};
        // predictor: r_c = -XZe
        ck(launch_mul(v[V_RC], X, Z, -1.0, n, s), "mul");
        st = solve(v[V_RD], v[V_RP], v[V_RC], v[V_DXA], v[V_DYA], v[V_DZA]);
        if (st == AHLP_ERR_NOT_SPD && escalate(true)) continue;
        if (st != AHLP_OK) throw Fail{st, p->err};
        if (last_rel > kEscalate && escalate(false)) continue;
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
        st = solve(v[V_RD], v[V_RP], v[V_RC], v[V_DX], v[V_DY], v[V_DZ]);
        if (st == AHLP_ERR_NOT_SPD && escalate(true)) continue;
        if (st != AHLP_OK) throw Fail{st, p->err};
        if (last_rel > kEscalate && escalate(false)) continue;
        break;
      }
      // Multiple centrality correctors (Gondzio), reusing the factor: the
      // products (x + a dx)(z + a dz) at an enlarged trial step are pushed into
      // [0.1 sigma mu, 10 sigma mu]; a corrected direction is kept only while
      // it lengthens the step.  Tried only when the step is short, and at
      // most as many as the factorisation costs in solves.
      if (p->opt.max_correctors > 0) {
        auto steps = [&](const double *dxv, const double *dzv, double &a_p, double &a_d) {
          ck(launch_reduce(p, RED_MINSTEP, X, dxv, n, p->scal + 0), "reduce");
          ck(launch_reduce(p, RED_MINSTEP, Z, dzv, n, p->scal + 1), "reduce");
          read_scalars(p, 2);
          a_p = std::min(1.0, p->h_scal[0]);
          a_d = std::min(1.0, p->h_scal[1]);
        };
        double a_p = 1.0, a_d = 1.0;
        steps(v[V_DX], v[V_DZ], a_p, a_d);
        // as many as the factorisation is worth in solves (Gondzio's rule)
        const double fac_ms = p->stage_ms[0] + p->stage_ms[1] + p->stage_ms[2];
        const double sol_ms = std::max((double)p->stage_ms[3], 1e-3);
        const int kmax = std::min(p->opt.max_correctors, (int)(fac_ms / sol_ms));
        for (int k = 0; k < kmax && std::min(a_p, a_d) < kCorrectorBelow; ++k) {
          const double tp = std::min(1.0, 1.5 * a_p + 0.1), td = std::min(1.0, 1.5 * a_d + 0.1);
          const double smu = sigma * mu;
          ck(launch_centrality_rc(v[V_RC2], v[V_RC], X, v[V_DX], tp, Z, v[V_DZ], td, 0.1 * smu,
                                  10.0 * smu, n, s),
             "corrector rhs");
          const int st = solve(v[V_RD], v[V_RP], v[V_RC2], v[V_DX2], v[V_DY2], v[V_DZ2]);
          if (st != AHLP_OK || last_rel > kEscalate) break;   // keep the previous direction
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
