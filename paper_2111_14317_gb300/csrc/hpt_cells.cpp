// Fine mixed cells of lifted supports by a pruned depth-first search (the
// cell step that Section 2 leaves to the literature).  A fine mixed cell picks
// one pair (edge) e_k = {p0, p1} of every support S_k such that some inner
// normal alpha makes each pair the lowest points of its lifted support:
//   <a_p0, alpha> + w(p0) = <a_p1, alpha> + w(p1) <= <a, alpha> + w(a), a in S_k.
// The search fixes the pairs equation by equation and keeps a partial choice
// only while these conditions, for the equations fixed so far, have a
// solution alpha (a linear feasibility problem in FP64: the pair equations
// are eliminated, then a point test, an interval, a Fourier-Motzkin
// elimination for two free variables, or the Farkas alternative by a small
// two-phase simplex).
// Candidate pairs of each support are its lower edges alone (the same test
// with one equation), and a table of which edges of two supports can be
// lowest together (the test with two equations) discards most branches
// before any larger problem is solved.  Every complete choice is then
// confirmed exactly
// (integer arithmetic: alpha solves the pair equations and every other point
// of every support lies strictly above), and |det V| of the confirmed cells
// sums to the mixed volume.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hpt_internal.h"

namespace hpt {
namespace {

// Feasibility of {x : E x = f, G x >= h} (x free), Phase I of the simplex
// method on x = u - v, G x - s = h, u, v, s >= 0 with one artificial per row,
// Bland's rule.  Returns true when the artificial sum reaches (about) zero.
struct LpScratch {
  std::vector<double> T;
  std::vector<int> basis;
};

bool lp_feasible(int n, const std::vector<double>& E, const std::vector<double>& f, const std::vector<double>& G,
                 const std::vector<double>& h, LpScratch& W) {
  const int me = (int)f.size(), mg = (int)h.size(), m = me + mg;
  if (m == 0) return true;
  const int nv = 2 * n + mg;          // u, v, s
  const int cols = nv + m + 1;        // + artificials + rhs
  std::vector<double>& T = W.T;
  T.assign((size_t)(m + 1) * cols, 0.0);
  auto at = [&](int r, int c) -> double& { return T[(size_t)r * cols + c]; };
  double scale = 1.0;
  for (int r = 0; r < m; ++r) {
    const bool eq = r < me;
    const double* a = eq ? &E[(size_t)r * n] : &G[(size_t)(r - me) * n];
    double b = eq ? f[r] : h[r - me];
    for (int j = 0; j < n; ++j) {
      at(r, j) = a[j];
      at(r, n + j) = -a[j];
    }
    if (!eq) at(r, 2 * n + (r - me)) = -1.0;
    const double sg = b < 0 ? -1.0 : 1.0;
    if (sg < 0)
      for (int c = 0; c < nv; ++c) at(r, c) = -at(r, c);
    at(r, nv + r) = 1.0;
    at(r, cols - 1) = sg * b;
    scale = std::max(scale, fabs(b));
  }
  // objective row: minimise the sum of artificials (reduced costs in row m)
  for (int c = 0; c < cols; ++c) {
    double s = 0;
    for (int r = 0; r < m; ++r) s += at(r, c);
    at(m, c) = (c >= nv && c < nv + m) ? 0.0 : -s;
  }
  std::vector<int>& basis = W.basis;
  basis.resize(m);
  for (int r = 0; r < m; ++r) basis[r] = nv + r;
  const double eps = 1e-10;
  for (int it = 0; it < 50 * (m + nv); ++it) {
    int enter = -1;
    for (int c = 0; c < nv + m; ++c)
      if (at(m, c) < -eps) { enter = c; break; }   // Bland: lowest index
    if (enter < 0) break;
    int leave = -1;
    double best = 0;
    for (int r = 0; r < m; ++r) {
      const double a = at(r, enter);
      if (a > eps) {
        const double ratio = at(r, cols - 1) / a;
        if (leave < 0 || ratio < best - 1e-12 || (ratio <= best + 1e-12 && basis[r] < basis[leave])) {
          leave = r;
          best = ratio;
        }
      }
    }
    if (leave < 0) break;   // unbounded in Phase I cannot happen; stop
    const double pv = at(leave, enter);
    for (int c = 0; c < cols; ++c) at(leave, c) /= pv;
    for (int r = 0; r <= m; ++r) {
      if (r == leave) continue;
      const double fct = at(r, enter);
      if (fct == 0.0) continue;
      for (int c = 0; c < cols; ++c) at(r, c) -= fct * at(leave, c);
    }
    basis[leave] = enter;
  }
  return -at(m, cols - 1) <= 1e-7 * scale;
}

// Feasibility of {t in R^d : G t >= h} (mg rows of G) through the Farkas
// alternative: the system is infeasible exactly when some y >= 0 with
// G^T y = 0 and sum y = 1 has h^T y > 0.  Two-phase simplex on those d + 1
// equality rows (Bland's rule): if Phase I finds no such y the system is
// feasible (strictly, by Gordan's theorem); otherwise Phase II maximises
// h^T y.  The tableau has d + 1 rows where the primal Phase I of lp_feasible
// has mg, which is what makes it the cheaper test for many conditions in few
// variables.
bool farkas_feasible(int d, int mg, const std::vector<double>& G, const std::vector<double>& h, LpScratch& W) {
  if (mg == 0) return true;
  const int R = d + 1, C = mg + R + 1;   // y, artificials, rhs
  std::vector<double>& T = W.T;
  T.assign((size_t)(R + 2) * C, 0.0);    // + Phase I and Phase II objective rows
  auto at = [&](int r, int c) -> double& { return T[(size_t)r * C + c]; };
  double hmax = 0.0;
  for (int i = 0; i < mg; ++i) {
    for (int q = 0; q < d; ++q) at(q, i) = G[(size_t)i * d + q];
    at(d, i) = 1.0;
    hmax = std::max(hmax, fabs(h[i]));
  }
  at(d, C - 1) = 1.0;
  for (int r = 0; r < R; ++r) at(r, mg + r) = 1.0;
  // reduced costs with the artificials basic: Phase I (minimise their sum)
  // in row R, Phase II (minimise -h^T y) in row R + 1
  for (int i = 0; i < mg; ++i) {
    double s = 0.0;
    for (int r = 0; r < R; ++r) s += at(r, i);
    at(R, i) = -s;
    at(R + 1, i) = -h[i];
  }
  at(R, C - 1) = -1.0;
  std::vector<int>& basis = W.basis;
  basis.resize(R);
  for (int r = 0; r < R; ++r) basis[r] = mg + r;
  const double eps = 1e-10;
  auto pivot = [&](int pr, int pc) {
    const double pv = at(pr, pc);
    for (int c = 0; c < C; ++c) at(pr, c) /= pv;
    for (int r = 0; r < R + 2; ++r) {
      if (r == pr) continue;
      const double fct = at(r, pc);
      if (fct == 0.0) continue;
      for (int c = 0; c < C; ++c) at(r, c) -= fct * at(pr, c);
    }
    basis[pr] = pc;
  };
  // one simplex phase on objective row `obj`; only y columns enter
  auto run = [&](int obj) {
    for (int it = 0; it < 50 * (R + mg); ++it) {
      int enter = -1;
      for (int c = 0; c < mg; ++c)
        if (at(obj, c) < -eps) { enter = c; break; }   // Bland: lowest index
      if (enter < 0) return;
      int leave = -1;
      double best = 0.0;
      for (int r = 0; r < R; ++r) {
        const double a = at(r, enter);
        if (a > eps) {
          const double ratio = at(r, C - 1) / a;
          if (leave < 0 || ratio < best - 1e-12 || (ratio <= best + 1e-12 && basis[r] < basis[leave])) {
            leave = r;
            best = ratio;
          }
        }
      }
      if (leave < 0) return;   // unbounded: cannot happen with sum y = 1
      pivot(leave, enter);
    }
  };
  run(R);
  if (-at(R, C - 1) > 1e-9) return true;   // no y: the conditions hold strictly somewhere
  // artificials left in the basis (at zero) leave it on any y column; a row
  // with no y entry is redundant and stays out of the ratio tests
  for (int r = 0; r < R; ++r) {
    if (basis[r] < mg) continue;
    for (int c = 0; c < mg; ++c)
      if (fabs(at(r, c)) > eps) { pivot(r, c); break; }
  }
  run(R + 1);
  return !(at(R + 1, C - 1) > 1e-7 * std::max(1.0, hmax));   // max h^T y
}

struct Search {
  int n;
  std::vector<int32_t> msz, off;
  const int32_t* exps;
  const int64_t* lift;
  std::vector<std::vector<std::pair<int, int>>> edges;   // lower edges per support
  // rel[k * n + l][i * E_l + j]: edge i of support k and edge j of support l
  // can be lowest together (the two-equation conditions are feasible)
  std::vector<std::vector<uint8_t>> rel;
  std::vector<int> pick;                                    // chosen edge index per equation
  std::vector<int> order;                                   // equations in search order
  std::vector<std::pair<int, int>> chosen;                  // per equation
  int64_t cap, found = 0;
  i128 volume = 0;
  int32_t* out;
  hpt_status err = HPT_OK;
  int64_t ties = 0;   // complete choices the FP64 search kept that fail the exact test
  // level d of the search (the first d equations of `order` fixed): the
  // inner normals alpha = a0 + N t, t in R^nf, that satisfy their pair
  // equations, and their other conditions G2 t >= h2 (nf values per row)
  struct Level {
    int nf = 0;
    std::vector<double> a0, N, G2, h2;
  };
  std::vector<Level> lv;
  std::vector<double> u;
  mutable LpScratch lp;

  // the conditions of equation k with pair (p0, p1), appended to E/f, G/h
  void add(int k, int p0, int p1, std::vector<double>& E, std::vector<double>& f, std::vector<double>& G,
           std::vector<double>& h) const {
    const int32_t* a0 = exps + (size_t)(off[k] + p0) * n;
    const int32_t* a1 = exps + (size_t)(off[k] + p1) * n;
    for (int j = 0; j < n; ++j) E.push_back((double)a1[j] - a0[j]);
    f.push_back((double)(lift[off[k] + p0] - lift[off[k] + p1]));
    for (int l = 0; l < msz[k]; ++l) {
      if (l == p0 || l == p1) continue;
      const int32_t* al = exps + (size_t)(off[k] + l) * n;
      for (int j = 0; j < n; ++j) G.push_back((double)al[j] - a0[j]);
      h.push_back((double)(lift[off[k] + p0] - lift[off[k] + l]));
    }
  }

  // Whether {t in R^nf : G2 t >= h2} has a solution (rows of G2 hold nf
  // values): a point test (nf = 0), an interval (nf = 1), Fourier-Motzkin
  // (nf = 2), else the Farkas alternative.
  bool solve_t(int nf, const std::vector<double>& G2, const std::vector<double>& h2) const {
    const int mg = (int)h2.size();
    const double tol = 1e-7;
    if (nf == 0) {
      for (int i = 0; i < mg; ++i)
        if (h2[i] > tol * (1.0 + fabs(h2[i]))) return false;
      return true;
    }
    // one free variable: conditions g t >= c bound t from below or above
    double lo = -INFINITY, hi = INFINITY;
    auto bound = [&](double g, double c) -> bool {
      if (fabs(g) < 1e-12) return !(c > tol * (1.0 + fabs(c)));
      if (g > 0) lo = std::max(lo, c / g);
      else hi = std::min(hi, c / g);
      return true;
    };
    if (nf == 1) {
      for (int i = 0; i < mg; ++i)
        if (!bound(G2[i], h2[i])) return false;
      return lo <= hi + tol * (1.0 + fabs(lo) + fabs(hi));
    }
    if (nf == 2) {
      // Fourier-Motzkin: a condition with a positive t2 coefficient bounds
      // t2 from below by c_i - d_i t1, one with a negative coefficient from
      // above by c_j - d_j t1 (both rows divided by |g_2|); t2 exists
      // exactly when every lower bound is at most every upper bound, i.e.
      // (d_i - d_j) t1 >= c_i - c_j for each such pair, together with the
      // conditions that do not involve t2
      for (int i = 0; i < mg; ++i) {
        const double gi = G2[2 * i + 1];
        if (fabs(gi) < 1e-12) {
          if (!bound(G2[2 * i], h2[i])) return false;
        } else if (gi > 0) {
          const double di = G2[2 * i] / gi, ci = h2[i] / gi;
          for (int j = 0; j < mg; ++j) {
            const double gj = G2[2 * j + 1];
            if (!(gj < -1e-12)) continue;
            const double dj = G2[2 * j] / gj, cj = h2[j] / gj;
            if (!bound(di - dj, ci - cj)) return false;
          }
        }
      }
      return lo <= hi + tol * (1.0 + fabs(lo) + fabs(hi));
    }
    return farkas_feasible(nf, mg, G2, h2, lp);
  }


  // Level d + 1 of the search from level d: the pair equation of equation
  // order[d] in the current parameters t (u.t = c) removes one parameter,
  // pivoting on its largest coefficient so that N's entries never grow (a
  // dependent equation removes none, an inconsistent one ends the branch);
  // the inherited conditions are rewritten in the remaining parameters and
  // the conditions of the new support appended.  Returns false when the
  // equation contradicts the ones fixed before.
  bool descend(int depth) {
    const Level& P = lv[depth];
    Level& Q = lv[depth + 1];
    const int k = order[depth];
    const int p0 = chosen[k].first, p1 = chosen[k].second;
    const int32_t* ap0 = exps + (size_t)(off[k] + p0) * n;
    const int32_t* ap1 = exps + (size_t)(off[k] + p1) * n;
    const int nf = P.nf;
    u.assign(nf, 0.0);
    double c = (double)(lift[off[k] + p0] - lift[off[k] + p1]);
    for (int x = 0; x < n; ++x) {
      const double e = (double)ap1[x] - ap0[x];
      if (e == 0.0) continue;
      c -= e * P.a0[x];
      for (int q = 0; q < nf; ++q) u[q] += e * P.N[(size_t)x * nf + q];
    }
    int piv = -1;
    double best = 1e-9;
    for (int q = 0; q < nf; ++q)
      if (fabs(u[q]) > best) { best = fabs(u[q]); piv = q; }
    const int mg = (int)P.h2.size();
    if (piv < 0) {
      if (fabs(c) > 1e-7 * (1.0 + fabs(c))) return false;
      Q.nf = nf;
      Q.a0 = P.a0;
      Q.N = P.N;
      Q.G2 = P.G2;
      Q.h2 = P.h2;
    } else {
      // t_piv = (c - sum_{q != piv} u_q t_q) / u_piv
      const int nq = nf - 1;
      const double up = u[piv], tp = c / up;
      Q.nf = nq;
      Q.a0.resize(n);
      Q.N.resize((size_t)n * nq);
      for (int x = 0; x < n; ++x) {
        const double np = P.N[(size_t)x * nf + piv];
        Q.a0[x] = P.a0[x] + np * tp;
        for (int q = 0, j = 0; q < nf; ++q)
          if (q != piv) Q.N[(size_t)x * nq + j++] = P.N[(size_t)x * nf + q] - np * (u[q] / up);
      }
      Q.G2.resize((size_t)mg * nq);
      Q.h2.resize(mg);
      for (int i = 0; i < mg; ++i) {
        const double gp = P.G2[(size_t)i * nf + piv];
        Q.h2[i] = P.h2[i] - gp * tp;
        for (int q = 0, j = 0; q < nf; ++q)
          if (q != piv) Q.G2[(size_t)i * nq + j++] = P.G2[(size_t)i * nf + q] - gp * (u[q] / up);
      }
    }
    // the new support's conditions (a_l - a_p0).alpha >= w(p0) - w(l)
    const int nq = Q.nf;
    for (int l = 0; l < msz[k]; ++l) {
      if (l == p0 || l == p1) continue;
      const int32_t* al = exps + (size_t)(off[k] + l) * n;
      double hh = (double)(lift[off[k] + p0] - lift[off[k] + l]);
      const size_t base = Q.G2.size();
      Q.G2.resize(base + nq, 0.0);
      for (int x = 0; x < n; ++x) {
        const double g = (double)al[x] - ap0[x];
        if (g == 0.0) continue;
        hh -= g * Q.a0[x];
        for (int q = 0; q < nq; ++q) Q.G2[base + q] += g * Q.N[(size_t)x * nq + q];
      }
      Q.h2.push_back(hh);
    }
    return true;
  }

  void leaf() {
    std::vector<int32_t> pairs(2 * n);
    for (int k = 0; k < n; ++k) {
      pairs[2 * k] = chosen[k].first;
      pairs[2 * k + 1] = chosen[k].second;
    }
    hpt_cell cell;
    memset(&cell, 0, sizeof(cell));
    cell.kind = HPT_CELL_PAIRS;
    cell.pairs = pairs.data();
    int64_t D = 0;
    const hpt_status lrc = hpt_lift_exponents(n, msz.data(), exps, lift, &cell, nullptr, &D, nullptr, nullptr);
    if (lrc == HPT_ENOTCELL) {   // a tie with another point (or det V = 0): the lifting is not generic
      ++ties;
      return;
    }
    if (lrc != HPT_OK) {
      err = lrc;
      return;
    }
    // |det V| exactly (the pair matrix of a confirmed cell is nonsingular)
    std::vector<int64_t> V((size_t)n * n);
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        V[k * n + j] = (int64_t)exps[(size_t)(off[k] + pairs[2 * k + 1]) * n + j] -
                       exps[(size_t)(off[k] + pairs[2 * k]) * n + j];
    i128 det = 0;
    hpt_status rc = exact_det(n, V, det);
    if (rc) { err = rc; return; }
    volume += det < 0 ? -det : det;
    if (volume >= ((i128)1 << 62)) { set_error("mixed volume beyond 2^62"); err = HPT_ERANGE; return; }
    if (found < cap && out) memcpy(out + (size_t)found * 2 * n, pairs.data(), 2 * n * sizeof(int32_t));
    ++found;
  }

  bool compatible(int k, int i, int depth) const {
    for (int d = 0; d < depth; ++d) {
      const int l = order[d];
      if (!rel[(size_t)k * n + l][(size_t)i * edges[l].size() + pick[l]]) return false;
    }
    return true;
  }

  void dfs(int depth) {
    if (err) return;
    if (depth == n) { leaf(); return; }
    const int k = order[depth];
    for (int i = 0; i < (int)edges[k].size(); ++i) {
      if (!compatible(k, i, depth)) continue;   // a pair of edges that cannot be lowest together
      chosen[k] = edges[k][i];
      pick[k] = i;
      if (!descend(depth)) continue;
      // one equation with a lower edge is always feasible
      if (depth < 1 || solve_t(lv[depth + 1].nf, lv[depth + 1].G2, lv[depth + 1].h2)) dfs(depth + 1);
      if (err) return;
    }
  }
};

}  // namespace
}  // namespace hpt

using namespace hpt;

extern "C" hpt_status hpt_mixed_cells(int32_t n, const int32_t* msz, const int32_t* exps, const int64_t* lifting,
                                      int64_t cap, int32_t* pairs_out, int64_t* ncells, int64_t* mixed_volume) {
  if (n < 1 || n > kMaxN || !msz || !exps || !lifting || cap < 0 || (cap > 0 && !pairs_out)) {
    set_error("bad arguments");
    return HPT_EINVAL;
  }
  Search S;
  S.n = n;
  S.msz.assign(msz, msz + n);
  S.off.resize(n);
  int64_t M = 0;
  for (int k = 0; k < n; ++k) {
    if (msz[k] < 2 || msz[k] > 4096) { set_error("m_%d=%d outside [2,4096]", k, msz[k]); return HPT_EINVAL; }
    S.off[k] = (int32_t)M;
    M += msz[k];
  }
  for (int64_t i = 0; i < M * n; ++i)
    if (exps[i] < -(1 << 20) || exps[i] > (1 << 20)) { set_error("exponent too large"); return HPT_ERANGE; }
  // the exact confirmation's range (hpt_lift_exponents), checked before the
  // search so that no lifting difference below can overflow
  for (int64_t i = 0; i < M; ++i)
    if (lifting[i] < -(1LL << 40) || lifting[i] > (1LL << 40)) { set_error("lifting too large"); return HPT_ERANGE; }
  S.exps = exps;
  S.lift = lifting;
  S.cap = cap;
  S.out = pairs_out;
  S.chosen.assign(n, {0, 1});
  // lower edges of every lifted support alone
  S.edges.resize(n);
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < msz[k]; ++i)
      for (int j = i + 1; j < msz[k]; ++j) {
        std::vector<double> E, f, G, h;
        S.add(k, i, j, E, f, G, h);
        if (lp_feasible(n, E, f, G, h, S.lp)) S.edges[k].push_back({i, j});
      }
  // relation table of every two supports' lower edges
  S.rel.assign((size_t)n * n, {});
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      if (l == k) continue;
      auto& R = S.rel[(size_t)k * n + l];
      R.assign(S.edges[k].size() * S.edges[l].size(), 0);
      if (l < k) {   // symmetric: copy the transposed table
        const auto& T = S.rel[(size_t)l * n + k];
        for (size_t i = 0; i < S.edges[k].size(); ++i)
          for (size_t j = 0; j < S.edges[l].size(); ++j) R[i * S.edges[l].size() + j] = T[j * S.edges[k].size() + i];
        continue;
      }
      for (size_t i = 0; i < S.edges[k].size(); ++i)
        for (size_t j = 0; j < S.edges[l].size(); ++j) {
          std::vector<double> E, f, G, h;
          S.add(k, S.edges[k][i].first, S.edges[k][i].second, E, f, G, h);
          S.add(l, S.edges[l][j].first, S.edges[l][j].second, E, f, G, h);
          R[i * S.edges[l].size() + j] = lp_feasible(n, E, f, G, h, S.lp) ? 1 : 0;
        }
    }
  S.pick.assign(n, 0);
  S.lv.resize(n + 1);
  S.lv[0].nf = n;
  S.lv[0].a0.assign(n, 0.0);
  S.lv[0].N.assign((size_t)n * n, 0.0);
  for (int x = 0; x < n; ++x) S.lv[0].N[(size_t)x * n + x] = 1.0;
  // fewest candidate edges first
  S.order.resize(n);
  for (int k = 0; k < n; ++k) S.order[k] = k;
  std::stable_sort(S.order.begin(), S.order.end(),
                   [&](int a, int b) { return S.edges[a].size() < S.edges[b].size(); });
  S.dfs(0);
  if (S.err) return S.err;
  if (ncells) *ncells = S.found;
  if (mixed_volume) *mixed_volume = (int64_t)S.volume;
  if (S.ties) {
    set_error("the lifting is not generic: %lld choices tie with another point; draw a new lifting",
              (long long)S.ties);
    return HPT_ENOTCELL;
  }
  return HPT_OK;
}
