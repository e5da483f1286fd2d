// The full LP statement of Sec. 3.2 -- equality rows, two-sided inequality
// rows d <= (row) x <= f, and bounds l <= x <= u -- reduced on the host, at
// create, to the equality form with x >= 0 that the solver factors, keeping
// the arrowhead block structure:
//
//  * an inequality row becomes an equality row (row) x - s = 0 with a new
//    variable s bounded by [d, f]; the slack of a block row joins its block,
//    the slack of a local link row of pair (j, j+1) joins block j, the slack
//    of a global row joins the last block;
//  * every variable v with bounds [lo, hi] (original or slack) becomes
//        lo finite, hi = +inf : v = lo + p                     (p >= 0)
//        lo = -inf, hi finite : v = hi - p                     (column negated)
//        both finite          : v = lo + p, p + w = hi - lo     (a new row in v's
//                               block -- a global row for a linking variable --
//                               and a new column w beside p)
//        both infinite        : v = p - q                      (a second column)
//    and the right-hand sides take the shifts.  A variable with lo = hi is a
//    box of width zero.
//
// The map back to the original variables (x = shift + sign p [- q]) and the
// constant c'(shift) of the objective are kept on the handle
// (arrowhead_lp_recover).
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "ahlp_internal.h"

namespace ahlp {

namespace {

[[noreturn]] void gfail(int code, const std::string &m) { throw Fail{code, m}; }

using Entry = StdCsc::Entry;
using Col = StdCsc::Col;

// column j of a CSC matrix (may be NULL: no entries), rows shifted by off
void col_of(const ahlp_csc *M, int m, int n, int j, int off, Col &out, double sign,
            const std::string &what) {
  if (!M || !M->colptr || n == 0) return;
  if (M->m != m || M->n != n) gfail(AHLP_ERR_DIM_MISMATCH, what + ": wrong shape");
  for (int q = M->colptr[j]; q < M->colptr[j + 1]; ++q) {
    const int r = M->rowidx[q];
    const double v = M->val[q];
    if (r < 0 || r >= m) gfail(AHLP_ERR_INVALID_ARG, what + ": row index out of range");
    if (!std::isfinite(v)) gfail(AHLP_ERR_INVALID_ARG, what + ": NaN or Inf entry");
    out.push_back({r + off, sign * v});
  }
}

// one variable before its bound transform: its entries in the block rows
// of its block (or, for a linking variable, of every block), the link rows
// and the global rows
struct VarCols {
  Col blk, prev, next, glob;   // block variable: block rows, pair i-1, pair i, global
  std::vector<Col> perblk, perpair;   // linking variable: per block, per pair
  double cost = 0, lo = 0, hi = INFINITY;
};

double bound_at(const double *const *arr, int i, int j, double dflt) {
  return (arr && arr[i]) ? arr[i][j] : dflt;
}

}  // namespace

bool desc_is_general(const ahlp_desc &d) {
  return d.lb || d.ub || d.lb0 || d.ub0 || d.mD || d.lG || d.mgG > 0;
}

void standardize(const ahlp_desc &d, StdDesc &S) {
  const int N = d.N, n0 = d.n0, mg = d.mg, mgG = d.mgG;
  if (N < 1 || n0 < 0 || mg < 0 || mgG < 0)
    gfail(AHLP_ERR_INVALID_ARG, "N >= 1, n0 >= 0, mg >= 0, mgG >= 0 required");
  if (!d.A || !d.W || !d.b || !d.c) gfail(AHLP_ERR_INVALID_ARG, "A, W, b, c must be given");
  if (N > 1 && !d.l) gfail(AHLP_ERR_INVALID_ARG, "l must be given when N > 1");
  const int P = N - 1;
  auto mD = [&](int i) { return d.mD ? d.mD[i] : 0; };
  auto lG = [&](int j) { return d.lG ? d.lG[j] : 0; };
  for (int i = 0; i < N; ++i)
    if (mD(i) < 0) gfail(AHLP_ERR_INVALID_ARG, "mD must be >= 0");
  for (int j = 0; j < P; ++j)
    if (lG(j) < 0 || d.l[j] < 0) gfail(AHLP_ERR_INVALID_ARG, "l and lG must be >= 0");
  for (int i = 0; i < N; ++i)
    if (mD(i) > 0 && (!d.D || !d.dlo || !d.dhi || !d.dlo[i] || !d.dhi[i]))
      gfail(AHLP_ERR_INVALID_ARG, "block " + std::to_string(i) +
                                      ": inequality rows need D, dlo and dhi");
  for (int j = 0; j < P; ++j)
    if (lG(j) > 0 && (!d.glo || !d.ghi || !d.glo[j] || !d.ghi[j]))
      gfail(AHLP_ERR_INVALID_ARG, "pair " + std::to_string(j) +
                                      ": link inequality rows need glo and ghi");
  if (mgG > 0 && (!d.gglo || !d.gghi))
    gfail(AHLP_ERR_INVALID_ARG, "global inequality rows need gglo and gghi");
  for (int i = 0; i < N; ++i)
    if (d.A[i].m < 0 || d.A[i].n < 0) gfail(AHLP_ERR_INVALID_ARG, "negative block size");
  auto check_lohi = [&](double lo, double hi, const std::string &what) {
    if (std::isnan(lo) || std::isnan(hi) || lo == INFINITY || hi == -INFINITY || lo > hi)
      gfail(AHLP_ERR_INVALID_ARG, what + ": bounds must satisfy -inf <= lo <= hi <= +inf");
  };
  // row counts of the standard form (box rows added below)
  std::vector<int> mrow(N), lrow(P);
  for (int i = 0; i < N; ++i) mrow[i] = d.A[i].m + mD(i);
  for (int j = 0; j < P; ++j) lrow[j] = d.l[j] + lG(j);
  const int grow0 = mg + mgG;   // global rows before the linking-variable boxes
  S.N = N;
  S.recov.clear();
  S.const_obj = 0.0;
  std::vector<std::vector<double>> rhs_blk(N), rhs_lnk(P);
  std::vector<double> rhs_g(grow0, 0.0);
  for (int i = 0; i < N; ++i) {
    rhs_blk[i].assign(mrow[i], 0.0);
    for (int r = 0; r < d.A[i].m; ++r) rhs_blk[i][r] = d.b[i][r];
  }
  for (int j = 0; j < P; ++j) {
    rhs_lnk[j].assign(lrow[j], 0.0);
    for (int r = 0; r < d.l[j]; ++r) rhs_lnk[j][r] = d.blink ? d.blink[j][r] : 0.0;
  }
  for (int r = 0; r < mg; ++r) rhs_g[r] = d.bg ? d.bg[r] : 0.0;
  // applies v's shift to every right-hand side its columns touch
  auto shift_rhs = [&](const VarCols &v, int blk, double s) {
    if (s == 0.0) return;
    if (blk >= 0) {
      for (auto &e : v.blk) rhs_blk[blk][e.first] -= e.second * s;
      if (blk > 0) for (auto &e : v.prev) rhs_lnk[blk - 1][e.first] -= e.second * s;
      if (blk < P) for (auto &e : v.next) rhs_lnk[blk][e.first] -= e.second * s;
    } else {
      for (int i = 0; i < N; ++i)
        for (auto &e : v.perblk[i]) rhs_blk[i][e.first] -= e.second * s;
      for (int j = 0; j < P; ++j)
        for (auto &e : v.perpair[j]) rhs_lnk[j][e.first] -= e.second * s;
    }
    for (auto &e : v.glob) rhs_g[e.first] -= e.second * s;
  };
  // ---- block variables ------------------------------------------------------
  std::vector<std::vector<Col>> fgcols(N);   // global-row parts of the final columns
  std::vector<std::vector<Col>> prevc(N), nextc(N), blkc(N);
  std::vector<std::vector<double>> costs(N);
  std::vector<std::vector<Entry>> boxrows(N);   // per block: (row, width) placeholders
  std::vector<int> nbox(N, 0);
  for (int i = 0; i < N; ++i) {
    const int mi = d.A[i].m, ni = d.A[i].n;
    const std::string tag = "block " + std::to_string(i);
    const int nvar = ni + mD(i) + (i < P ? lG(i) : 0) + (i == N - 1 ? mgG : 0);
    for (int t = 0; t < nvar; ++t) {
      VarCols v;
      int orig = -1;
      if (t < ni) {   // an original variable of the block
        orig = t;
        col_of(&d.A[i], mi, ni, t, 0, v.blk, 1.0, tag + " A");
        if (d.D && mD(i)) col_of(&d.D[i], mD(i), ni, t, mi, v.blk, 1.0, tag + " D");
        if (i > 0) {
          col_of(d.FR ? &d.FR[i - 1] : nullptr, d.l[i - 1], ni, t, 0, v.prev, 1.0, tag + " FR");
          if (lG(i - 1))
            col_of(d.GR ? &d.GR[i - 1] : nullptr, lG(i - 1), ni, t, d.l[i - 1], v.prev, 1.0,
                   tag + " GR");
        }
        if (i < P) {
          col_of(d.FL ? &d.FL[i] : nullptr, d.l[i], ni, t, 0, v.next, 1.0, tag + " FL");
          if (lG(i))
            col_of(d.GL ? &d.GL[i] : nullptr, lG(i), ni, t, d.l[i], v.next, 1.0, tag + " GL");
        }
        col_of(d.Fg ? &d.Fg[i] : nullptr, mg, ni, t, 0, v.glob, 1.0, tag + " Fg");
        if (mgG) col_of(d.Gg ? &d.Gg[i] : nullptr, mgG, ni, t, mg, v.glob, 1.0, tag + " Gg");
        v.cost = d.c[i][t];
        v.lo = bound_at(d.lb, i, t, 0.0);
        v.hi = bound_at(d.ub, i, t, INFINITY);
        if (!std::isfinite(v.cost)) gfail(AHLP_ERR_INVALID_ARG, tag + " c: NaN or Inf");
      } else {
        int r = t - ni;
        if (r < mD(i)) {   // slack of a block inequality row
          v.blk.push_back({mi + r, -1.0});
          v.lo = d.dlo[i][r];
          v.hi = d.dhi[i][r];
        } else if ((r -= mD(i)) < (i < P ? lG(i) : 0)) {   // of a link inequality row of pair i
          v.next.push_back({d.l[i] + r, -1.0});
          v.lo = d.glo[i][r];
          v.hi = d.ghi[i][r];
        } else {   // of a global inequality row (last block)
          r -= (i < P ? lG(i) : 0);
          v.glob.push_back({mg + r, -1.0});
          v.lo = d.gglo[r];
          v.hi = d.gghi[r];
        }
      }
      check_lohi(v.lo, v.hi, tag + " variable " + std::to_string(t));
      const int k = (int)blkc[i].size();   // index of the first final column
      auto add = [&](double sign, double cost) {
        Col b, pv, nx, g;
        for (auto &e : v.blk) b.push_back({e.first, sign * e.second});
        for (auto &e : v.prev) pv.push_back({e.first, sign * e.second});
        for (auto &e : v.next) nx.push_back({e.first, sign * e.second});
        for (auto &e : v.glob) g.push_back({e.first, sign * e.second});
        blkc[i].push_back(std::move(b));
        prevc[i].push_back(std::move(pv));
        nextc[i].push_back(std::move(nx));
        fgcols[i].push_back(std::move(g));
        costs[i].push_back(cost);
      };
      StdDesc::Recov rc{i, orig, 0.0, k, 1.0, -1};
      if (std::isfinite(v.lo)) {
        rc.shift = v.lo;
        add(1.0, v.cost);
        if (std::isfinite(v.hi)) {   // box: p + w = hi - lo, w a new column
          const int row = mrow[i] + nbox[i]++;
          blkc[i][k].push_back({row, 1.0});
          boxrows[i].push_back({row, v.hi - v.lo});
          add(1.0, 0.0);
          blkc[i].back() = Col{{row, 1.0}};
          prevc[i].back().clear();
          nextc[i].back().clear();
          fgcols[i].back().clear();
        }
      } else if (std::isfinite(v.hi)) {
        rc.shift = v.hi;
        rc.sign = -1.0;
        add(-1.0, -v.cost);
      } else {
        add(1.0, v.cost);
        add(-1.0, -v.cost);
        rc.k2 = k + 1;
      }
      shift_rhs(v, i, rc.shift);
      S.const_obj += v.cost * rc.shift;
      if (orig >= 0) S.recov.push_back(rc);
    }
  }
  // ---- linking variables -----------------------------------------------------
  std::vector<Col> x0g;                       // global-row parts
  std::vector<std::vector<Col>> x0b(N), x0p(P);   // per block / per pair parts
  std::vector<double> c0s;
  std::vector<Entry> x0box;   // (global row, width)
  for (int t = 0; t < n0; ++t) {
    VarCols v;
    v.perblk.assign(N, {});
    v.perpair.assign(P, {});
    for (int i = 0; i < N; ++i) {
      const std::string tag = "block " + std::to_string(i);
      col_of(&d.W[i], d.A[i].m, n0, t, 0, v.perblk[i], 1.0, tag + " W");
      if (mD(i)) col_of(d.C ? &d.C[i] : nullptr, mD(i), n0, t, d.A[i].m, v.perblk[i], 1.0,
                        tag + " C");
    }
    for (int j = 0; j < P; ++j) {
      const std::string tag = "pair " + std::to_string(j);
      col_of(d.F0 ? &d.F0[j] : nullptr, d.l[j], n0, t, 0, v.perpair[j], 1.0, tag + " F0");
      if (lG(j)) col_of(d.G0 ? &d.G0[j] : nullptr, lG(j), n0, t, d.l[j], v.perpair[j], 1.0,
                        tag + " G0");
    }
    col_of(d.Fg0, mg, n0, t, 0, v.glob, 1.0, "Fg0");
    if (mgG) col_of(d.Gg0, mgG, n0, t, mg, v.glob, 1.0, "Gg0");
    v.cost = d.c0 ? d.c0[t] : 0.0;
    v.lo = d.lb0 ? d.lb0[t] : 0.0;
    v.hi = d.ub0 ? d.ub0[t] : INFINITY;
    check_lohi(v.lo, v.hi, "linking variable " + std::to_string(t));
    const int k = (int)c0s.size();
    auto add = [&](double sign, double cost) {
      for (int i = 0; i < N; ++i) {
        Col c;
        for (auto &e : v.perblk[i]) c.push_back({e.first, sign * e.second});
        x0b[i].push_back(std::move(c));
      }
      for (int j = 0; j < P; ++j) {
        Col c;
        for (auto &e : v.perpair[j]) c.push_back({e.first, sign * e.second});
        x0p[j].push_back(std::move(c));
      }
      Col g;
      for (auto &e : v.glob) g.push_back({e.first, sign * e.second});
      x0g.push_back(std::move(g));
      c0s.push_back(cost);
    };
    StdDesc::Recov rc{-1, t, 0.0, k, 1.0, -1};
    if (std::isfinite(v.lo)) {
      rc.shift = v.lo;
      add(1.0, v.cost);
      if (std::isfinite(v.hi)) {   // box: a global row p + w = hi - lo
        const int row = grow0 + (int)x0box.size();
        x0g[k].push_back({row, 1.0});
        x0box.push_back({row, v.hi - v.lo});
        add(1.0, 0.0);
        for (int i = 0; i < N; ++i) x0b[i].back().clear();
        for (int j = 0; j < P; ++j) x0p[j].back().clear();
        x0g.back() = Col{{row, 1.0}};
      }
    } else if (std::isfinite(v.hi)) {
      rc.shift = v.hi;
      rc.sign = -1.0;
      add(-1.0, -v.cost);
    } else {
      add(1.0, v.cost);
      add(-1.0, -v.cost);
      rc.k2 = k + 1;
    }
    shift_rhs(v, -1, rc.shift);
    S.const_obj += v.cost * rc.shift;
    S.recov.push_back(rc);
  }
  // ---- assemble the standard-form description -------------------------------
  const int mgS = grow0 + (int)x0box.size();
  const int n0S = (int)c0s.size();
  S.A.assign(N, {});
  S.W.assign(N, {});
  S.Fg.assign(N, {});
  S.FL.assign(P, {});
  S.FR.assign(P, {});
  S.F0.assign(P, {});
  S.b.assign(N, {});
  S.c.assign(N, {});
  S.blink.assign(P, {});
  for (int i = 0; i < N; ++i) {
    const int mS = mrow[i] + nbox[i];
    S.A[i].m = mS;
    S.Fg[i].m = mgS;
    for (size_t k = 0; k < blkc[i].size(); ++k) {
      S.A[i].push(blkc[i][k]);
      S.Fg[i].push(fgcols[i][k]);
    }
    S.W[i].m = mS;
    for (int k = 0; k < n0S; ++k) S.W[i].push(x0b[i][k]);
    S.b[i] = rhs_blk[i];
    for (auto &e : boxrows[i]) S.b[i].push_back(e.second);
    S.c[i] = costs[i];
  }
  for (int j = 0; j < P; ++j) {
    S.FL[j].m = S.FR[j].m = S.F0[j].m = lrow[j];
    for (auto &c : nextc[j]) S.FL[j].push(c);
    for (auto &c : prevc[j + 1]) S.FR[j].push(c);
    for (int k = 0; k < n0S; ++k) S.F0[j].push(x0p[j][k]);
    S.blink[j] = rhs_lnk[j];
    S.l.push_back(lrow[j]);
  }
  S.Fg0.m = mgS;
  for (auto &c : x0g) S.Fg0.push(c);
  S.bg = rhs_g;
  for (auto &e : x0box) S.bg.push_back(e.second);
  S.c0 = c0s;
  S.n_orig.clear();
  for (int i = 0; i < N; ++i) S.n_orig.push_back(d.A[i].n);
  S.n0_orig = n0;
  // the description the solver reads
  S.Ac.clear();
  S.Wc.clear();
  S.Fgc.clear();
  S.FLc.clear();
  S.FRc.clear();
  S.F0c.clear();
  S.bp.clear();
  S.cp.clear();
  S.blp.clear();
  for (int i = 0; i < N; ++i) {
    S.Ac.push_back(S.A[i].csc());
    S.Wc.push_back(S.W[i].csc());
    S.Fgc.push_back(S.Fg[i].csc());
    S.bp.push_back(S.b[i].data());
    S.cp.push_back(S.c[i].data());
  }
  for (int j = 0; j < P; ++j) {
    S.FLc.push_back(S.FL[j].csc());
    S.FRc.push_back(S.FR[j].csc());
    S.F0c.push_back(S.F0[j].csc());
    S.blp.push_back(S.blink[j].data());
  }
  S.Fg0c = S.Fg0.csc();
  ahlp_desc &o = S.d;
  o = ahlp_desc{};
  o.N = N;
  o.n0 = n0S;
  o.mg = mgS;
  o.c0 = S.c0.data();
  o.A = S.Ac.data();
  o.W = S.Wc.data();
  o.b = S.bp.data();
  o.c = S.cp.data();
  o.l = S.l.data();
  o.FL = S.FLc.data();
  o.FR = S.FRc.data();
  o.F0 = S.F0c.data();
  o.blink = S.blp.data();
  o.Fg = S.Fgc.data();
  o.Fg0 = &S.Fg0c;
  o.bg = S.bg.data();
}

}  // namespace ahlp
