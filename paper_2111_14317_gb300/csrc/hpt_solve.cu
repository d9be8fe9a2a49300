// Consolidated Euler+Newton solve (Section 6, eq. (11), affine form) and the
// per-path step control, plus the small kernels around them (state init,
// active count, Newton polish at t = 1, implicit-function adjoint).
//
// The scratch holds D_z H = H_y diag(y) (z = log y).  H_y d = r is solved as
// D_z H w = r, d = diag(y) w: the diag(1/y) scaling of op. 3 of Algorithm 2
// costs n products per path here instead of n^2 in the evaluation.
//
// Solve mapping: a group of G lanes owns one path and every lane holds R rows
// of [D_z H | -H_tau | -H] in registers (rows lane, lane + G, ...), n <= G R.
// The rows are equilibrated by exact powers of two, then Gaussian elimination
// with partial pivoting runs over a run-time column loop.  Rows are "shifted":
// after column j is eliminated every live row moves one register to the left,
// so the current column is always register 0 and the loop body uses static
// register indices only.  The pivot (largest |.|^2; ties to the lowest row, as
// LAPACK's getrf) comes from one packed integer max per butterfly level; its
// owner writes the pivot row, relative to column j, into row j of the group's
// shared-memory factor U, from where every lane reads it.  Back substitution
// works column by column on U.  Two right-hand sides [-H_tau, -H] give the
// Euler direction dE and the Newton direction dN from one factorisation.
#include <math.h>

#include <algorithm>

#include "hpt_internal.h"
#include "hpt_cx.cuh"

namespace hpt {
namespace {

// Pivot key: |a|^2 rounded to float with the low five mantissa bits replaced
// by (31 - row), so that one integer max picks the largest magnitude, ties to
// the lowest row.  Rows already used as pivots get key 0.
template <typename T>
__device__ __forceinline__ unsigned pivot_key(T v, bool used, int row) {
  if (used) return 0u;
  float f = (float)v;
  if (!(f == f)) f = 0.f;   // NaN rows stay eligible; the pivot test flags them
  return (__float_as_uint(f) & ~31u) | (unsigned)(31 - row);
}

// Shared memory of one group: U (NC rows of LD complex; LD even keeps rows
// 16-byte aligned, LD - 1 odd keeps the column reads of the back substitution
// on distinct banks) then the column scales (NC reals), padded so that
// consecutive groups start 8 banks apart.
template <typename T, int NC>
struct GroupSmem {
  static constexpr int LD = NC + 4;
  static constexpr int raw_words = (NC * LD * 2 * (int)sizeof(T) + NC * (int)sizeof(T)) / 4;
  static constexpr int words = (raw_words + 31) / 32 * 32 + 8;
  static constexpr int bytes = words * 4;
};

constexpr int kSolveThreads = 128;

// Rows of one path for a group: lane l holds rows l + G s, s < R, as
// a[s][0..NC) plus the two right-hand sides.
template <typename T, int G, int R>
struct PathRows {
  static constexpr int NC = G * R;
  cx<T> a[R][NC];
  cx<T> bE[R], bN[R];
};


// Loads the rows of [D_z H | -H_tau | -H] (adjoint = false) or of
// [(D_z H)^H | g | 0] (adjoint = true, g from gx) for one path; returns
// whether every entry is finite (group-uniform).
template <typename T, typename S, int G, int R>
__device__ __forceinline__ bool load_rows(int n, int nmax, const void* ext, int64_t q, size_t vbase, bool valid,
                                          bool adjoint, const double2* gx, PathRows<T, G, R>& P) {
  constexpr int NC = G * R;
  const int lane = threadIdx.x & (G - 1);
  T chk = T(0);
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = lane + G * s;
    const bool have = valid && r < n;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      P.a[s][c] = mk<T>(0, 0);
      if (have && c < n) {
        cx<S> v = adjoint ? ld<S>(ext, ext_index(q, c, r, nmax)) : ld<S>(ext, ext_index(q, r, c, nmax));
        P.a[s][c] = adjoint ? mk<T>((T)v.x, -(T)v.y) : mk<T>((T)v.x, (T)v.y);
        chk += t_abs(P.a[s][c].x) + t_abs(P.a[s][c].y);
      }
    }
    P.bE[s] = mk<T>(0, 0);
    P.bN[s] = mk<T>(0, 0);
    if (have) {
      if (adjoint) {
        const double2 g = gx[vbase + r];
        P.bE[s] = mk<T>((T)g.x, (T)g.y);
      } else {
        const cx<S> ht = ld<S>(ext, ext_index(q, r, n, nmax));
        const cx<S> h = ld<S>(ext, ext_index(q, r, n + 1, nmax));
        P.bE[s] = mk<T>(-(T)ht.x, -(T)ht.y);
        P.bN[s] = mk<T>(-(T)h.x, -(T)h.y);
      }
      chk += t_abs(P.bE[s].x) + t_abs(P.bE[s].y) + t_abs(P.bN[s].x) + t_abs(P.bN[s].y);
    }
  }
  // a sum of magnitudes is finite iff every entry is
  const unsigned ball = __ballot_sync(0xffffffffu, isfinite(chk));
  const unsigned seg = group_mask<G>();
  return (ball & seg) == seg;
}

// 32-lane groups (one path per warp) would load every entry of the
// position-interleaved scratch from its own 32-byte sector.  Instead the
// block's four paths (consecutive positions q0..q0+3 of one tile, so one n)
// are staged cooperatively: four threads read the same entry of the four
// paths, one sector, and write it to the path's group region in shared memory
// as rows of kStageLD entries (odd, so the row reads below hit distinct
// banks).  Only paths with act set are read.  Call with every thread of the
// block between two block barriers.
constexpr int kStageLD = 35;
template <typename S>
__device__ __forceinline__ void stage_block_rows(int n, int nmax, const void* __restrict__ ext, int64_t q0, bool act,
                                                 unsigned char* smem, int region_bytes) {
  if (!act) return;   // act: path (threadIdx.x & 3) of the block is to be solved
  typedef typename cplx_t<S>::type V;
  const int i = threadIdx.x & 3;
  V* region = (V*)(smem + i * region_bytes);
  const int np2 = n + 2, total = n * np2;
  for (int e = threadIdx.x >> 2; e < total; e += 32) {
    const int k = e / np2, u = e - k * np2;
    region[k * kStageLD + u] = ((const V*)ext)[ext_index(q0 + i, k, u, nmax)];
  }
}

// load_rows for a 32-lane group from its staged region (lane r = row r).
template <typename T, typename S>
__device__ __forceinline__ bool load_rows_staged(int n, const unsigned char* region, bool valid,
                                                 PathRows<T, 32, 1>& P) {
  typedef typename cplx_t<S>::type V;
  const V* rg = (const V*)region;
  const int r = threadIdx.x & 31;
  const bool have = valid && r < n;
  T chk = T(0);
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    P.a[0][c] = mk<T>(0, 0);
    if (have && c < n) {
      const V v = rg[r * kStageLD + c];
      P.a[0][c] = mk<T>((T)v.x, (T)v.y);
      chk += t_abs(P.a[0][c].x) + t_abs(P.a[0][c].y);
    }
  }
  P.bE[0] = mk<T>(0, 0);
  P.bN[0] = mk<T>(0, 0);
  if (have) {
    const V ht = rg[r * kStageLD + n], h = rg[r * kStageLD + n + 1];
    P.bE[0] = mk<T>(-(T)ht.x, -(T)ht.y);
    P.bN[0] = mk<T>(-(T)h.x, -(T)h.y);
    chk += t_abs(P.bE[0].x) + t_abs(P.bE[0].y) + t_abs(P.bN[0].x) + t_abs(P.bN[0].y);
  }
  __syncwarp();   // every row is in registers before the solve writes U over the region
  return __all_sync(0xffffffffu, isfinite(chk));
}

// Solves the path held in P (n <= G R) with equilibration and partial
// pivoting.  Returns false (group-uniform) when a pivot is zero or not
// finite; cond receives max |u_jj| / min |u_jj|.  On return lane l holds
// solution components l + G s in xE[s], xN[s].  sm is the group's shared
// memory (GroupSmem).
template <typename T, int G, int R>
__device__ __forceinline__ bool group_solve(int n, PathRows<T, G, R>& P, cx<T> (&xE)[R], cx<T> (&xN)[R], T& cond,
                            unsigned char* sm) {
  constexpr int NC = G * R, LD = GroupSmem<T, NC>::LD;
  cx<T>* U = (cx<T>*)sm;
  T* dcol = (T*)(sm + NC * LD * sizeof(cx<T>));
  const int lane = threadIdx.x & (G - 1);

  // equilibration: rows, then columns, by exact powers of two
#pragma unroll
  for (int s = 0; s < R; ++s) {
    T m = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) m = t_max(m, cmag(P.a[s][c]));
    const T dr = pow2_inv(m);
#pragma unroll
    for (int c = 0; c < NC; ++c) P.a[s][c] = cscale(P.a[s][c], dr);
    P.bE[s] = cscale(P.bE[s], dr);
    P.bN[s] = cscale(P.bN[s], dr);
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (c < n) {
      T m = T(0);
#pragma unroll
      for (int s = 0; s < R; ++s) m = t_max(m, cmag(P.a[s][c]));
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) m = t_max(m, __shfl_xor_sync(0xffffffffu, m, o, G));
      const T d = pow2_inv(m);
#pragma unroll
      for (int s = 0; s < R; ++s) P.a[s][c] = cscale(P.a[s][c], d);
      if (lane == 0) dcol[c] = d;
    }
  }

  bool used[R];
#pragma unroll
  for (int s = 0; s < R; ++s) used[s] = lane + G * s >= n;
  bool ok = true;
  T pmax = 0, pmin = 0;   // extreme |u_jj|^2
#pragma unroll 1
  for (int j = 0; j < n; ++j) {
    unsigned key = 0u;
#pragma unroll
    for (int s = 0; s < R; ++s) key = max(key, pivot_key<T>(abs2(P.a[s][0]), used[s], lane + G * s));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o, G));
    const int br = 31 - (int)(key & 31u);
    if (lane == (br & (G - 1))) {
      // the owner's slot chosen entry by entry (a per-slot conditional store
      // would be turned into a dynamically indexed, local-memory row)
      const int bs = br / G;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        cx<T> v = P.a[0][c];
#pragma unroll
        for (int s = 1; s < R; ++s) v = (bs == s) ? P.a[s][c] : v;
        U[j * LD + c] = v;
      }
      cx<T> e = P.bE[0], f = P.bN[0];
#pragma unroll
      for (int s = 1; s < R; ++s) {
        e = (bs == s) ? P.bE[s] : e;
        f = (bs == s) ? P.bN[s] : f;
      }
      U[j * LD + NC] = e;
      U[j * LD + NC + 1] = f;
#pragma unroll
      for (int s = 0; s < R; ++s) used[s] = used[s] || (bs == s);
    }
    __syncwarp();
    const cx<T> pj = U[j * LD];
    const T p2 = abs2(pj);
    if (!(p2 > T(0)) || !isfinite(p2)) ok = false;
    pmax = j == 0 ? p2 : t_max(pmax, p2);
    pmin = j == 0 ? p2 : t_min(pmin, p2);
    const T rp = t_rcp(p2);   // one reciprocal per pivot, shared by all rows
    // multipliers; rows already used get 0, so the unpredicated update below
    // only shifts them (their values are no longer read)
    cx<T> l[R];
#pragma unroll
    for (int s = 0; s < R; ++s) l[s] = used[s] ? mk<T>(0, 0) : cmul_conj_scale(P.a[s][0], pj, rp);
    // shifted update: a[c-1] = a[c] - l u_{j, j+c} over the live width, in
    // chunks of four columns behind one warp-uniform branch each (the
    // columns of the last chunk beyond the live width are updated too; they
    // are never read again)
    const int lim = n - 1 - j;
#pragma unroll
    for (int c0 = 1; c0 < NC; c0 += 4) {
      if (c0 <= lim) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c) {
          if (c < NC) {
            const cx<T> u = U[j * LD + c];
#pragma unroll
            for (int s = 0; s < R; ++s) P.a[s][c - 1] = csub_mul(P.a[s][c], l[s], u);
          }
        }
      }
    }
    const cx<T> uE = U[j * LD + NC], uN = U[j * LD + NC + 1];
#pragma unroll
    for (int s = 0; s < R; ++s) {
      P.bE[s] = csub_mul(P.bE[s], l[s], uE);
      P.bN[s] = csub_mul(P.bN[s], l[s], uN);
    }
  }
  __syncwarp();
  // back substitution on U (row i holds u_{i, i+c} at c, then the two
  // right-hand sides); lane l carries the right-hand sides of rows l + G s
  cx<T> rE[R], rN[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int i = lane + G * s;
    rE[s] = i < n ? U[i * LD + NC] : mk<T>(0, 0);
    rN[s] = i < n ? U[i * LD + NC + 1] : mk<T>(0, 0);
    xE[s] = mk<T>(0, 0);
    xN[s] = mk<T>(0, 0);
  }
#pragma unroll 1
  for (int j = n - 1; j >= 0; --j) {
    const cx<T> ujj = U[j * LD];
    const int js = j / G;
    cx<T> vE = rE[0], vN = rN[0];
#pragma unroll
    for (int s = 1; s < R; ++s)
      if (s == js) { vE = rE[s]; vN = rN[s]; }
    vE = shfl<T, G>(vE, j & (G - 1));
    vN = shfl<T, G>(vN, j & (G - 1));
    const T ru = t_rcp(abs2(ujj));
    const cx<T> xe = cmul_conj_scale(vE, ujj, ru), xn = cmul_conj_scale(vN, ujj, ru);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const int i = lane + G * s;
      if (i == j) { xE[s] = xe; xN[s] = xn; }
      if (i < j) {
        const cx<T> u = U[i * LD + (j - i)];
        rE[s] = csub_mul(rE[s], u, xe);
        rN[s] = csub_mul(rN[s], u, xn);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int i = lane + G * s;
    if (i < n) {
      const T d = dcol[i];
      xE[s] = cscale(xE[s], d);
      xN[s] = cscale(xN[s], d);
    }
  }
  __syncwarp();   // the group's shared memory is reused by its next solve
  cond = pmin > T(0) ? t_sqrt(pmax / pmin) : T(INFINITY);
  return ok;
}

// Step control of one path (all lanes of its group), given the directions:
// accept/reject, then the next prediction (Euler, or with prm.predictor = 1
// and two accepted points the cubic Hermite interpolant through them; the
// point being replaced by an accept is kept in the state's *_prev arrays).
// TS is the state precision; lane l handles the variables l + G s.
// The state a step reads, loaded ahead of the solve so that its loads are in
// flight together with the Jacobian's (the Hermite predictor's extra fields
// are read only when used).
template <typename TS, int R>
struct StepState {
  cx<TS> y[R], yacc[R], dEacc[R];
  double tau, dtau, tauacc;
  int32_t steps, accepts, rejects, streak;
};

template <typename TS, int G, int R>
__device__ __forceinline__ void load_step_state(int n, int64_t path, size_t vbase, const hpt_paths& S,
                                                StepState<TS, R>& Q) {
  const int lane = threadIdx.x & (G - 1);
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    const bool mine = j < n;
    const size_t vi = vbase + j;
    Q.y[s] = mine ? ld<TS>(S.y, vi) : mk<TS>(0, 0);
    Q.yacc[s] = mine ? ld<TS>(S.y_acc, vi) : mk<TS>(0, 0);
    Q.dEacc[s] = mine ? ld<TS>(S.dE_acc, vi) : mk<TS>(0, 0);
  }
  Q.tau = S.tau[path];
  Q.dtau = S.dtau[path];
  Q.tauacc = S.tau_acc[path];
  Q.steps = S.steps[path];
  Q.accepts = S.accepts[path];
  Q.rejects = S.rejects[path];
  Q.streak = S.streak[path];
}

template <typename TS, int G, int R>
__device__ __forceinline__ void update_path(int n, int64_t path, size_t vbase, int32_t status, bool ok,
                                            const cx<TS> (&wE)[R], const cx<TS> (&wN)[R], const hpt_paths& S,
                                            const hpt_params& prm, const StepState<TS, R>& Q) {
  const int lane = threadIdx.x & (G - 1);
  const unsigned gmask = group_mask<G>();
  cx<TS> y[R], yacc[R], dEacc[R], xE[R], xN[R];
  bool solfin = true;
  TS ny = TS(0), nd = TS(0);
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    const bool mine = j < n;
    y[s] = Q.y[s];
    yacc[s] = Q.yacc[s];
    dEacc[s] = Q.dEacc[s];
    // the scratch holds D_z H = H_y diag(y): the solve gave diag(1/y) times
    // the directions
    xE[s] = cmul(y[s], wE[s]);
    xN[s] = cmul(y[s], wN[s]);
    if (mine) {
      solfin = solfin && finite(xE[s]) && finite(xN[s]);
      ny = t_max(ny, cabs_t(y[s]));
      nd = t_max(nd, cabs_t(xN[s]));
    }
  }
  solfin = (__ballot_sync(gmask, solfin) & gmask) == gmask;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    ny = t_max(ny, __shfl_xor_sync(gmask, ny, o, G));
    nd = t_max(nd, __shfl_xor_sync(gmask, nd, o, G));
  }
  const bool bad = !(ok && solfin);
  double tau = Q.tau, dtau = Q.dtau, tauacc = Q.tauacc;
  int32_t steps = Q.steps + 1, accepts = Q.accepts, rejects = Q.rejects, streak = Q.streak;
  const TS err = nd / t_max(TS(1), ny);
  const bool accept = !bad && err <= (TS)prm.tol_accept;
  const bool herm = prm.predictor == 1;
  bool predict = true, keep_prev = false, retry = false;
  cx<TS> yp[R], dp[R];   // the accepted point before the last one (Hermite predictor)
  double taup = 0.0;
  if (accept) {
    keep_prev = herm && accepts >= 1;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      yp[s] = yacc[s];
      dp[s] = dEacc[s];
      yacc[s] = mk<TS>(y[s].x + xN[s].x, y[s].y + xN[s].y);
      dEacc[s] = xE[s];
    }
    taup = tauacc;
    tauacc = tau;
    accepts += 1;
    streak += 1;
    if (tauacc == 0.0) {
      status = HPT_PATH_CONVERGED;
      predict = false;
    } else {
      bool div = false;
#pragma unroll
      for (int s = 0; s < R; ++s) {
        if (lane + G * s < n) {
          const TS m = cabs_t(yacc[s]);
          div = div || !(m < (TS)prm.div_bound) || !(m > (TS)(1.0 / prm.div_bound));
        }
      }
      div = (__ballot_sync(gmask, div) & gmask) != 0u;
      if (div) {
        status = HPT_PATH_DIVERGED;
        predict = false;
      } else if (streak >= prm.grow_after) {
        dtau = fmin(dtau * prm.grow, prm.dtau_max);
        streak = 0;
      }
    }
  } else {
    rejects += 1;
    streak = 0;
    if (accepts == 0) {
      predict = false;
      if (bad) {
        status = HPT_PATH_SINGULAR;
      } else {
#pragma unroll
        for (int s = 0; s < R; ++s) {
          y[s] = mk<TS>(y[s].x + xN[s].x, y[s].y + xN[s].y);
          yacc[s] = y[s];
        }
        if (steps >= prm.max_steps) status = HPT_PATH_MAX_STEPS;
      }
    } else {
      // a rejected cubic prediction is retried with Euler at the same step
      // size; a rejected Euler prediction shrinks the step
      retry = herm && S.hermite[path] != 0;
      if (!retry) {
        dtau *= prm.shrink;
        if (dtau < prm.dtau_min) {
          status = HPT_PATH_UNDERFLOW;
          predict = false;
        }
      }
    }
  }
  if (predict) {
    const double h = fmin(dtau, -tauacc);
    bool cubic = false;
    if (herm && !retry && accepts >= 2) {
      if (!keep_prev) {   // a rejected step: the previous point from the state
#pragma unroll
        for (int s = 0; s < R; ++s) {
          const bool mine = lane + G * s < n;
          yp[s] = mine ? ld<TS>(S.y_prev, vbase + lane + G * s) : mk<TS>(0, 0);
          dp[s] = mine ? ld<TS>(S.dE_prev, vbase + lane + G * s) : mk<TS>(0, 0);
        }
        taup = S.tau_prev[path];
      }
      cubic = tauacc - taup > 0.0;
    }
    if (cubic) {
      // cubic Hermite through (taup, yp, dp) and (tauacc, yacc, dEacc) at tauacc + h
      const double d = tauacc - taup, u = 1.0 + h / d, u2 = u * u, u3 = u2 * u;
      const TS h00 = (TS)(2 * u3 - 3 * u2 + 1), h10 = (TS)((u3 - 2 * u2 + u) * d);
      const TS h01 = (TS)(-2 * u3 + 3 * u2), h11 = (TS)((u3 - u2) * d);
#pragma unroll
      for (int s = 0; s < R; ++s)
        y[s] = mk<TS>(h00 * yp[s].x + h10 * dp[s].x + h01 * yacc[s].x + h11 * dEacc[s].x,
                      h00 * yp[s].y + h10 * dp[s].y + h01 * yacc[s].y + h11 * dEacc[s].y);
    } else {
#pragma unroll
      for (int s = 0; s < R; ++s) y[s] = mk<TS>(yacc[s].x + (TS)h * dEacc[s].x, yacc[s].y + (TS)h * dEacc[s].y);
    }
    tau = tauacc + h;
    if (steps >= prm.max_steps) status = HPT_PATH_MAX_STEPS;
    if (herm && lane == 0) S.hermite[path] = cubic ? 1 : 0;
  }
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    if (j < n) {
      const size_t vi = vbase + j;
      st<TS>(S.y, vi, y[s]);
      st<TS>(S.y_acc, vi, yacc[s]);
      st<TS>(S.dE_acc, vi, dEacc[s]);
      if (keep_prev) {
        st<TS>(S.y_prev, vi, yp[s]);
        st<TS>(S.dE_prev, vi, dp[s]);
      }
    }
  }
  if (keep_prev && lane == 0) S.tau_prev[path] = taup;
  if (lane == 0) {
    S.tau[path] = tau;
    S.dtau[path] = dtau;
    S.tau_acc[path] = tauacc;
    S.status[path] = status;
    S.steps[path] = steps;
    S.accepts[path] = accepts;
    S.rejects[path] = rejects;
    S.streak[path] = streak;
  }
}

template <typename TS, int G, int R>
__device__ __forceinline__ void update_path(int n, int64_t path, size_t vbase, int32_t status, bool ok,
                                            const cx<TS> (&wE)[R], const cx<TS> (&wN)[R], const hpt_paths& S,
                                            const hpt_params& prm) {
  StepState<TS, R> Q;
  load_step_state<TS, G, R>(n, path, vbase, S, Q);
  update_path<TS, G, R>(n, path, vbase, status, ok, wE, wN, S, prm, Q);
}

__device__ __forceinline__ int64_t pm_path(const PathMap& m, int64_t q) { return m.list ? m.list[q] : q; }
__device__ __forceinline__ int pm_n(const PathMap& m, int64_t q, int n) {
  return m.sys_n ? m.sys_n[m.tile_sys[q >> 7]] : n;
}
__device__ __forceinline__ size_t pm_vbase(const PathMap& m, int64_t path, int n) {
  return m.vofs ? (size_t)m.vofs[path] : (size_t)path * n;
}
__device__ __forceinline__ int64_t pm_count(const PathMap& m, int64_t p) { return m.npos ? (int64_t)*m.npos : p; }
__device__ __forceinline__ int64_t pm_begin(const PathMap& m) { return m.pos_begin ? (int64_t)*m.pos_begin : 0; }

// One Euler-Newton step per ACTIVE path: consolidated solve, then the step
// control.  T is the state and solve precision.  FP32 solves whose pivot
// ratio (after equilibration) exceeds prm.cond_max are not applied here: the
// position goes to redo_list and is solved again in FP64 by redo_fp64_kernel.
// One system: G threads per path, a grid that covers every path once.  The
// FP32 8-lane two-row form is register-capped for five resident blocks per
// SM (shared memory allows five): more warps to cover each warp's dependent
// chain of loads, shuffles and shared-memory round trips.
template <typename T, int G, int R>
__global__ void __launch_bounds__(kSolveThreads, (sizeof(T) == 4 && G == 8 && R == 2) ? 5 : 1)
solve_update_kernel(int n, int64_t p, const void* __restrict__ ext, hpt_paths S, hpt_params prm,
                    int32_t* __restrict__ redo_count, int64_t* __restrict__ redo_list) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & (G - 1);
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int32_t status = path < p ? S.status[path] : -1;
  const bool valid = status == HPT_PATH_ACTIVE;
  unsigned char* sm = smem + (threadIdx.x / G) * GroupSmem<T, G * R>::bytes;
  if (G == 32) {   // block-uniform: stage the block's four paths
    const int64_t q0 = (int64_t)blockIdx.x * (kSolveThreads / 32);
    const int64_t qi = q0 + (threadIdx.x & 3);
    stage_block_rows<T>(n, n, ext, q0, qi < p && S.status[qi] == HPT_PATH_ACTIVE, smem, GroupSmem<T, G * R>::bytes);
    __syncthreads();
  }
  if (!__any_sync(0xffffffffu, valid)) return;   // warp-uniform exit
  const size_t vbase = (size_t)path * n;
  PathRows<T, G, R> P;
  bool fin;
  if constexpr (G == 32) fin = load_rows_staged<T, T>(n, sm, valid, P);
  else fin = load_rows<T, T, G, R>(n, n, ext, path, vbase, valid, false, nullptr, P);
  cx<T> xE[R], xN[R];
  T cond;
  const bool ok = group_solve<T, G, R>(n, P, xE, xN, cond, sm) && fin;
  if (!valid) return;   // group-uniform; only group-masked shuffles below
  if (sizeof(T) == 4 && redo_list && ok && !(cond <= (T)prm.cond_max)) {
    if (lane == 0) redo_list[atomicAdd(redo_count, 1)] = path;
    return;
  }
  update_path<T, G, R>(n, path, vbase, status, ok, xE, xN, S, prm);
}

// FP32 step of one system with n <= G R by Gauss-Jordan elimination.  A
// G-lane group owns one path as in group_solve: lane l holds rows l + G s,
// s < R, of [D_z H | -H_tau | -H] in registers, here as packed FP32 pairs
// (rows >= n are zero).  After the exact power-of-two row and column
// equilibration of group_solve (the column magnitudes go through shared
// memory, one reduction per column instead of a butterfly per column), each
// column is eliminated from every other row, the rows already used as pivots
// included: group_solve updates those rows too, with zero multipliers, so
// the elimination costs the same and no back substitution follows.  At the
// end row i holds only its pivot u_i and its two right-hand sides, and the
// unknowns of the column it pivoted are b_i / u_i.  The pivot of a column is
// the one of group_solve (largest |.|^2 among the unused rows, ties to the
// lowest row), so the pivots, the condition proxy and the FP64 re-solve
// list are those of the LU form.  Each entry of the pivot row reaches the
// group by a shuffle from its owner (every lane selects the pivot's slot, the
// same in the whole group): no shared-memory round trip, and no per-entry
// packing by the owner alone, which cost 25 of 140 us.  A row's update
// a - l u is two paired FMAs with u and u swapped.  Rows are shifted as in
// group_solve (column j is always register 0).
template <int NC>
struct GjSmem {
  union {
    float cm[NC][NC + 4];       // the rows' entry magnitudes, read back by column
    struct {
      float4 x[NC];             // the solutions by column: (xE.re, xE.im, xN.re, xN.im)
    } e;
  } u;
  float dcol[NC];               // the column scales
};
// Per-group stride in words, = G (mod 32): the column reads of cm by the
// groups of a warp fall on distinct banks.
template <int G, int NC>
struct GjLayout {
  static constexpr int raw = (int)(sizeof(GjSmem<NC>) / 4);
  static constexpr int words = (raw - G + 31) / 32 * 32 + G;
  static constexpr int bytes = words * 4;
};

__device__ __forceinline__ float cmag2(uint64_t v) {
  const float2 f = upk2(v);
  return fmaxf(fabsf(f.x), fabsf(f.y));
}

// One path (position q of the scratch, laid out for nmax variables) for
// every lane of its group; call with the whole warp converged.  Returns with
// the state updated, or the position queued for the FP64 re-solve.
template <int G, int R>
__device__ __forceinline__ void gj_path(int n, int nmax, int64_t q, int64_t path, size_t vbase, int32_t status,
                                        const float2* __restrict__ ext, const hpt_paths& S, const hpt_params& prm,
                                        int32_t* __restrict__ redo_count, int64_t* __restrict__ redo_list,
                                        unsigned char* smem) {
  constexpr int NC = G * R;
  const int lane = threadIdx.x & (G - 1);
  const bool valid = status == HPT_PATH_ACTIVE;
  GjSmem<NC>& sh = *(GjSmem<NC>*)(smem + (threadIdx.x / G) * GjLayout<G, NC>::bytes);
  const unsigned gmask = group_mask<G>();

  // rows lane + G s and their right-hand sides
  uint64_t a[R][NC], bE[R], bN[R];
  float chk = 0.f;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = lane + G * s;
    const bool have = valid && r < n;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float2 v = make_float2(0.f, 0.f);
      if (have && c < n) v = ext[ext_index(q, r, c, nmax)];
      a[s][c] = pk2(v.x, v.y);
      chk += fabsf(v.x) + fabsf(v.y);
    }
    float2 ht = make_float2(0.f, 0.f), h = make_float2(0.f, 0.f);
    if (have) {
      ht = ext[ext_index(q, r, n, nmax)];
      h = ext[ext_index(q, r, n + 1, nmax)];
    }
    bE[s] = pk2(-ht.x, -ht.y);
    bN[s] = pk2(-h.x, -h.y);
    chk += fabsf(ht.x) + fabsf(ht.y) + fabsf(h.x) + fabsf(h.y);
  }
  // a sum of magnitudes is finite iff every entry is
  const bool fin = (__ballot_sync(0xffffffffu, isfinite(chk)) & gmask) == gmask;

  // equilibration: each row, then the columns, by exact powers of two
#pragma unroll
  for (int s = 0; s < R; ++s) {
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < NC; ++c) m = fmaxf(m, cmag2(a[s][c]));
    const float dr = pow2_inv(m);
    const uint64_t DR = pk2(dr, dr);
#pragma unroll
    for (int c = 0; c < NC; ++c) a[s][c] = mul_x2(a[s][c], DR);
    bE[s] = mul_x2(bE[s], DR);
    bN[s] = mul_x2(bN[s], DR);
#pragma unroll
    for (int c = 0; c < NC; c += 4)
      *(float4*)&sh.u.cm[lane + G * s][c] =
          make_float4(cmag2(a[s][c]), cmag2(a[s][c + 1]), cmag2(a[s][c + 2]), cmag2(a[s][c + 3]));
  }
  __syncwarp();
  float dc[R];   // the scales of columns lane + G s
#pragma unroll
  for (int s = 0; s < R; ++s) {
    float mc = 0.f;
#pragma unroll
    for (int r = 0; r < NC; ++r) mc = fmaxf(mc, sh.u.cm[r][lane + G * s]);
    dc[s] = pow2_inv(mc);   // 1 for a zero column
    sh.dcol[lane + G * s] = dc[s];
  }
  __syncwarp();   // every column magnitude read before the pivot rows reuse the space
#pragma unroll
  for (int c = 0; c < NC; c += 4) {
    const float4 d = *(const float4*)&sh.dcol[c];
    const uint64_t D0 = pk2(d.x, d.x), D1 = pk2(d.y, d.y), D2 = pk2(d.z, d.z), D3 = pk2(d.w, d.w);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      a[s][c] = mul_x2(a[s][c], D0);
      a[s][c + 1] = mul_x2(a[s][c + 1], D1);
      a[s][c + 2] = mul_x2(a[s][c + 2], D2);
      a[s][c + 3] = mul_x2(a[s][c + 3], D3);
    }
  }

  // elimination
  bool used[R];
  int step[R];
  uint64_t piv[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    used[s] = lane + G * s >= n;
    step[s] = 0;
    piv[s] = pk2(1.f, 0.f);
  }
  bool ok = true;
  float pmax = 0.f, pmin = 0.f;   // extreme |u_jj|^2
#pragma unroll 1
  for (int j = 0; j < n; ++j) {
    unsigned key = 0u;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const float2 v = upk2(a[s][0]);
      key = max(key, pivot_key<float>(v.x * v.x + v.y * v.y, used[s], lane + G * s));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o, G));
    const int br = 31 - (int)(key & 31u);
    const int bs = br / G;
    const bool owner = lane == (br & (G - 1));
    const int lim = n - 1 - j;   // live registers 1..lim
    // the pivot row by shuffles from its owner: every lane picks slot bs
    // (uniform in the group) and reads the owner's copy
    const int ol = br & (G - 1);
    auto pick_bcast = [&](const uint64_t* col) -> uint64_t {   // col[s] for s < R
      uint64_t v = col[0];
#pragma unroll
      for (int s = 1; s < R; ++s) v = bs == s ? col[s] : v;
      return __shfl_sync(0xffffffffu, v, ol, G);
    };
    if (owner) {
#pragma unroll
      for (int s = 0; s < R; ++s) {
        if (bs == s) {
          used[s] = true;
          step[s] = j;
          piv[s] = a[s][0];
        }
      }
    }
    uint64_t col0[R];
#pragma unroll
    for (int s = 0; s < R; ++s) col0[s] = a[s][0];
    const float2 pv = upk2(pick_bcast(col0));
    const float p2 = pv.x * pv.x + pv.y * pv.y;
    if (!(p2 > 0.f) || !isfinite(p2)) ok = false;
    pmax = j == 0 ? p2 : fmaxf(pmax, p2);
    pmin = j == 0 ? p2 : fminf(pmin, p2);
    const float rp = t_rcp(p2);   // one reciprocal per pivot, shared by all rows
    // multipliers a_s0 / pivot; the pivot row itself keeps its values
    uint64_t NL[R], LS[R];
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const float2 v = upk2(a[s][0]);
      float lr = (v.x * pv.x + v.y * pv.y) * rp, li = (v.y * pv.x - v.x * pv.y) * rp;
      if (owner && bs == s) {
        lr = 0.f;
        li = 0.f;
      }
      NL[s] = pk2(-lr, -lr);
      LS[s] = pk2(li, -li);
    }
    // shifted update a[c-1] = a[c] - l u over the live width, in chunks of
    // four columns behind one warp-uniform branch each (the columns of the
    // last chunk beyond the live width are never read again)
#pragma unroll
    for (int c0 = 1; c0 < NC; c0 += 4) {
      if (c0 <= lim) {
#pragma unroll
        for (int c = c0; c < c0 + 4 && c < NC; ++c) {
          uint64_t colc[R];
#pragma unroll
          for (int s = 0; s < R; ++s) colc[s] = a[s][c];
          const uint64_t U = pick_bcast(colc);
          const float2 uf = upk2(U);
          const uint64_t US = pk2(uf.y, uf.x);
#pragma unroll
          for (int s = 0; s < R; ++s) a[s][c - 1] = fma_x2(LS[s], US, fma_x2(NL[s], U, a[s][c]));
        }
      }
    }
    {
      const uint64_t U = pick_bcast(bE), V = pick_bcast(bN);
      const float2 uf = upk2(U), vf = upk2(V);
      const uint64_t US = pk2(uf.y, uf.x), VS = pk2(vf.y, vf.x);
#pragma unroll
      for (int s = 0; s < R; ++s) {
        bE[s] = fma_x2(LS[s], US, fma_x2(NL[s], U, bE[s]));
        bN[s] = fma_x2(LS[s], VS, fma_x2(NL[s], V, bN[s]));
      }
    }
  }
  // row i < n now holds its pivot and right-hand sides: the unknowns of the
  // column it pivoted, put in column order through shared memory
#pragma unroll
  for (int s = 0; s < R; ++s) {
    if (lane + G * s < n) {
      const float2 u = upk2(piv[s]), e = upk2(bE[s]), f = upk2(bN[s]);
      const float ru = t_rcp(u.x * u.x + u.y * u.y);
      sh.u.e.x[step[s]] = make_float4((e.x * u.x + e.y * u.y) * ru, (e.y * u.x - e.x * u.y) * ru,
                                      (f.x * u.x + f.y * u.y) * ru, (f.y * u.x - f.x * u.y) * ru);
    }
  }
  __syncwarp();
  cx<float> wE[R], wN[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    wE[s] = mk<float>(0.f, 0.f);
    wN[s] = mk<float>(0.f, 0.f);
    if (lane + G * s < n) {
      const float4 v = sh.u.e.x[lane + G * s];
      wE[s] = mk<float>(v.x * dc[s], v.y * dc[s]);
      wN[s] = mk<float>(v.z * dc[s], v.w * dc[s]);
    }
  }
  const float cond = pmin > 0.f ? sqrtf(pmax / pmin) : INFINITY;
  ok = ok && fin;
  __syncwarp();   // the group's shared memory is reused by its next path
  if (!valid) return;   // group-uniform; only group-masked shuffles below
  if (redo_list && ok && !(cond <= (float)prm.cond_max)) {
    if (lane == 0) redo_list[atomicAdd(redo_count, 1)] = q;
    return;
  }
  update_path<float, G, R>(n, path, vbase, status, ok, wE, wN, S, prm);
}

template <int G, int R>
__global__ void __launch_bounds__(kSolveThreads, R == 1 ? 6 : 4)
gj_update_kernel(int n, int64_t p, const float2* __restrict__ ext, hpt_paths S, hpt_params prm,
                 int32_t* __restrict__ redo_count, int64_t* __restrict__ redo_list) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int32_t status = path < p ? S.status[path] : -1;
  if (!__any_sync(0xffffffffu, status == HPT_PATH_ACTIVE)) return;   // warp-uniform exit
  gj_path<G, R>(n, n, path, path, (size_t)path * n, status, ext, S, prm, redo_count, redo_list, smem);
}

// The same over a position map (many systems), persistent as
// solve_update_map_kernel: a warp's 32/G consecutive positions lie in one
// 128-position tile, so n is warp-uniform.
template <int G, int R>
__global__ void __launch_bounds__(kSolveThreads, R == 1 ? 6 : 4)
gj_update_map_kernel(int n0, int64_t p, const float2* __restrict__ ext, hpt_paths S, hpt_params prm,
                     int32_t* __restrict__ redo_count, int64_t* __restrict__ redo_list, PathMap pm) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int per_warp = 32 / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  const int g = (threadIdx.x & 31) / G;
  const int64_t npos = pm_count(pm, p);
  for (int64_t base = pm_begin(pm) + warp_id * per_warp; base < npos; base += nwarps * per_warp) {
    const int64_t q = base + g;
    const int n = pm_n(pm, base, n0);
    const int64_t path = q < npos ? pm_path(pm, q) : -1;
    const int32_t status = path >= 0 ? S.status[path] : -1;
    if (!__any_sync(0xffffffffu, status == HPT_PATH_ACTIVE)) continue;   // warp-uniform skip
    const size_t vbase = status == HPT_PATH_ACTIVE ? pm_vbase(pm, path, n) : 0;
    gj_path<G, R>(n, pm.nmax, q, path, vbase, status, ext, S, prm, redo_count, redo_list, smem);
  }
}

// The same over a position map (many systems).  Persistent: the warps loop
// over the positions of [*pos_begin, *npos) (32/G consecutive positions per
// warp, always inside one 128-position tile, so n is warp-uniform).
template <typename T, int G, int R>
__global__ void __launch_bounds__(kSolveThreads)
solve_update_map_kernel(int n0, int64_t p, const void* __restrict__ ext, hpt_paths S, hpt_params prm,
                        int32_t* __restrict__ redo_count, int64_t* __restrict__ redo_list, PathMap pm) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int per_warp = 32 / G;
  const int lane = threadIdx.x & (G - 1);
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  const int g = (threadIdx.x & 31) / G;
  unsigned char* sm = smem + (threadIdx.x / G) * GroupSmem<T, G * R>::bytes;
  const int64_t npos = pm_count(pm, p);
  const int nmax = pm.nmax;
  // with 32-lane groups the block's four warps take consecutive positions of
  // one tile and run the same number of iterations (npos is a multiple of
  // 128), so the staging barriers below are reached by the whole block
  for (int64_t base = pm_begin(pm) + warp_id * per_warp; base < npos; base += nwarps * per_warp) {
    const int64_t q = base + g;
    const int n = pm_n(pm, base, n0);
    const int64_t path = q < npos ? pm_path(pm, q) : -1;
    const int32_t status = path >= 0 ? S.status[path] : -1;
    const bool valid = status == HPT_PATH_ACTIVE;
    if (G == 32) {
      const int64_t q0 = base - (threadIdx.x >> 5);
      const int64_t pi = pm_path(pm, q0 + (threadIdx.x & 3));
      __syncthreads();   // the previous iteration's solves are done with the regions
      stage_block_rows<T>(n, nmax, ext, q0, pi >= 0 && S.status[pi] == HPT_PATH_ACTIVE, smem,
                          GroupSmem<T, G * R>::bytes);
      __syncthreads();
    }
    if (!__any_sync(0xffffffffu, valid)) continue;   // warp-uniform skip
    const size_t vbase = valid ? pm_vbase(pm, path, n) : 0;
    PathRows<T, G, R> P;
    bool fin;
    if constexpr (G == 32) fin = load_rows_staged<T, T>(n, sm, valid, P);
    else fin = load_rows<T, T, G, R>(n, nmax, ext, q, vbase, valid, false, nullptr, P);
    cx<T> xE[R], xN[R];
    T cond;
    const bool ok = group_solve<T, G, R>(n, P, xE, xN, cond, sm) && fin;
    if (valid) {   // group-uniform; only group-masked shuffles below
      if (sizeof(T) == 4 && redo_list && ok && !(cond <= (T)prm.cond_max)) {
        if (lane == 0) redo_list[atomicAdd(redo_count, 1)] = q;
      } else {
        update_path<T, G, R>(n, path, vbase, status, ok, xE, xN, S, prm);
      }
    }
    __syncwarp();
  }
}

// FP64 re-solve of the positions listed by the FP32 kernel (same FP32
// Jacobian, FP64 factorisation), then their step control in the FP32 state.
// Entries of the list sit next to any other, so n may differ between the
// groups of a warp: the warp solves with the largest n of its groups and a
// smaller system gets identity rows for the unknowns it does not have.
template <int G, int R>
__global__ void __launch_bounds__(kSolveThreads)
redo_fp64_kernel(int n0, const void* __restrict__ ext, hpt_paths S, hpt_params prm,
                 const int32_t* __restrict__ redo_count, const int64_t* __restrict__ redo_list, PathMap pm) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int count = *redo_count;
  constexpr int per_warp = 32 / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  const int g = (threadIdx.x & 31) / G;
  unsigned char* sm = smem + (threadIdx.x / G) * GroupSmem<double, G * R>::bytes;
  for (int64_t base = warp_id * per_warp; base < count; base += nwarps * per_warp) {
    const int64_t i = base + g;
    const bool valid = i < count;
    const int64_t q = valid ? redo_list[i] : 0;
    const int64_t path = valid ? pm_path(pm, q) : 0;
    const int n = valid ? pm_n(pm, q, n0) : 0;
    int nw = n;   // the warp's largest n: group_solve needs a warp-uniform size
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nw = max(nw, __shfl_xor_sync(0xffffffffu, nw, o));
    const size_t vbase = valid ? pm_vbase(pm, path, n) : 0;
    PathRows<double, G, R> P;
    const bool fin = load_rows<double, float, G, R>(n, pm.nmax, ext, q, vbase, valid, false, nullptr, P);
    // rows n..nw-1 become identity rows (their unknowns solve to 0)
    const int lane = threadIdx.x & (G - 1);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const int r = lane + G * s;
      if (r >= n && r < nw) {
#pragma unroll
        for (int c = 0; c < G * R; ++c)
          if (c == r) P.a[s][c] = mk<double>(1.0, 0.0);
      }
    }
    cx<double> xE[R], xN[R];
    double cond;
    const bool ok = group_solve<double, G, R>(nw, P, xE, xN, cond, sm) && fin;
    if (valid) {
      cx<float> fE[R], fN[R];
#pragma unroll
      for (int s = 0; s < R; ++s) {
        fE[s] = mk<float>((float)xE[s].x, (float)xE[s].y);
        fN[s] = mk<float>((float)xN[s].x, (float)xN[s].y);
      }
      update_path<float, G, R>(n, path, vbase, S.status[path], ok, fE, fN, S, prm);
    }
    __syncwarp();
  }
}

// Newton polish update at t = 1 (FP64): x += dN until the error left is below
// tol: |dN|/max(1,|x|) <= tol, or, once the corrections shrink quadratically,
// the error after this update, about r_k^3 / r_{k-1}^2 for the relative
// corrections r of the last two iterations (last[] keeps r_{k-1}; 0: none).
// MAP: positions [*pm.pos_begin, *pm.npos) of a position map (a warp's
// positions lie in one tile, so n is warp-uniform); otherwise the p paths of
// one system.
template <int G, int R, bool MAP>
__global__ void __launch_bounds__(kSolveThreads)
newton_kernel(int n0, int64_t p, const void* __restrict__ ext, double2* __restrict__ x,
              int32_t* __restrict__ done, float* __restrict__ last, double tol, PathMap pm) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & (G - 1);
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G + (MAP ? (int64_t)*pm.pos_begin : 0);
  const int64_t end = MAP ? (int64_t)*pm.npos : p;
  const bool in = q < end;
  const int64_t path = in ? (MAP ? pm.list[q] : q) : -1;
  const bool valid = path >= 0 && done[path] == 0;
  unsigned char* sm = smem + (threadIdx.x / G) * GroupSmem<double, G * R>::bytes;
  if (G == 32) {   // block-uniform: stage the block's four positions
    const int64_t q0 = q - (threadIdx.x >> 5);
    if (q0 >= end) return;   // the whole block (end is a multiple of 4)
    const int n = MAP ? pm.sys_n[pm.tile_sys[q0 >> 7]] : n0;
    const int64_t qi = q0 + (threadIdx.x & 3);
    const int64_t pi = qi < end ? (MAP ? pm.list[qi] : qi) : -1;
    stage_block_rows<double>(n, MAP ? pm.nmax : n, ext, q0, pi >= 0 && done[pi] == 0, smem,
                             GroupSmem<double, G * R>::bytes);
    __syncthreads();
  }
  if (!__any_sync(0xffffffffu, valid)) return;
  const int n = MAP ? pm.sys_n[pm.tile_sys[q >> 7]] : n0;
  const size_t vbase = MAP ? (valid ? (size_t)pm.vofs[path] : 0) : (size_t)path * n;
  PathRows<double, G, R> P;
  bool fin;
  if constexpr (G == 32) fin = load_rows_staged<double, double>(n, sm, valid, P);
  else fin = load_rows<double, double, G, R>(n, MAP ? pm.nmax : n, ext, q, vbase, valid, false, nullptr, P);
  cx<double> xE[R], xN[R];
  double cond;
  const bool ok = group_solve<double, G, R>(n, P, xE, xN, cond, sm) && fin;
  if (!valid) return;
  const unsigned gmask = group_mask<G>();
  bool sfin = true;
  double ny = 0.0, nd = 0.0;
  cx<double> y[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    y[s] = j < n ? ld<double>(x, vbase + j) : mk<double>(0, 0);
    xN[s] = cmul(y[s], xN[s]);   // D_z H in the scratch: the correction is x * w
    if (j < n) {
      sfin = sfin && finite(xN[s]);
      y[s] = mk<double>(y[s].x + xN[s].x, y[s].y + xN[s].y);
      ny = fmax(ny, cabs_t(y[s]));
      nd = fmax(nd, cabs_t(xN[s]));
    }
  }
  sfin = (__ballot_sync(gmask, sfin) & gmask) == gmask;
  if (!(ok && sfin)) {
    if (lane == 0) done[path] = 2;
    return;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    ny = fmax(ny, __shfl_xor_sync(gmask, ny, o, G));
    nd = fmax(nd, __shfl_xor_sync(gmask, nd, o, G));
  }
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    if (j < n) st<double>(x, vbase + j, y[s]);
  }
  if (lane == 0) {
    const double r = nd / fmax(1.0, ny), rp = (double)last[path];
    const bool settled = rp > 0.0 && r <= 0.1 * rp && r * r * r <= tol * rp * rp;
    if (r <= tol || settled) done[path] = 1;
    last[path] = (float)r;
  }
}

// Adjoint, part 1: per solution, lambda from J^H lambda = gx (J from the
// extended Jacobian at t = 1), then contrib[q][i] = -lambda_k conj(x^{a_i})
// for every monomial i of equation k (monomials by exp of <a, log x>).
template <int G, int R>
__global__ void __launch_bounds__(kSolveThreads)
adjoint_kernel(int n, int64_t p, const int32_t* __restrict__ msz, const int32_t* __restrict__ off,
               const double* __restrict__ ahat, int M, const void* __restrict__ ext,
               const double2* __restrict__ x, const double2* __restrict__ gx,
               double2* __restrict__ contrib) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double2 zsh[kSolveThreads / G][G * R];
  const int lane = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G;
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const bool valid = path < p;
  PathRows<double, G, R> P;
  const bool fin = load_rows<double, double, G, R>(n, n, ext, path, (size_t)path * n, valid, true, gx, P);
  // D_z H = H_y diag(x) in the scratch: H_y^H lambda = g becomes
  // (D_z H)^H lambda = conj(x) g
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = lane + G * s;
    if (valid && r < n) {
      const double2 v = x[(size_t)path * n + r];
      P.bE[s] = cmul(mk<double>(v.x, -v.y), P.bE[s]);
    }
  }
  cx<double> lam[R], dummy[R];
  double cond;
  const bool ok =
      group_solve<double, G, R>(n, P, lam, dummy, cond, smem + grp * GroupSmem<double, G * R>::bytes) && fin;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    if (valid && j < n) {
      const double2 v = x[(size_t)path * n + j];
      zsh[grp][j] = make_double2(log(hypot(v.x, v.y)), atan2(v.y, v.x));
    }
  }
  __syncthreads();
  if (!valid) return;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int k = lane + G * s;
    if (k >= n) continue;
    for (int i = off[k]; i < off[k] + msz[k]; ++i) {
      const double* ai = ahat + (size_t)i * (n + 1);
      double wr = 0.0, wi = 0.0;
      for (int j = 0; j < n; ++j) {
        wr = fma(ai[j], zsh[grp][j].x, wr);
        wi = fma(ai[j], zsh[grp][j].y, wi);
      }
      double sn, cs;
      sincos(wi, &sn, &cs);
      const double m = exp(wr);
      // -lambda_k * conj(m (cs + i sn))
      const double mr = m * cs, mi = -m * sn;
      double2 v = make_double2(-(lam[s].x * mr - lam[s].y * mi), -(lam[s].x * mi + lam[s].y * mr));
      if (!ok) v = make_double2(NAN, NAN);
      contrib[(size_t)path * M + i] = v;
    }
  }
}

// Adjoint, part 2: gc[i] += sum over the chunk's solutions of contrib[q][i],
// in a fixed order (the same bits on every run).  First pass: block (cb, r)
// sums rows r, r + kAdjRowBlocks, ... of 32 consecutive columns, its 8 warps
// each a strided subset, the warps' sums added in warp order (a warp reads 32
// consecutive columns of one row: coalesced); second pass: every column's
// kAdjRowBlocks partial sums added in order.
constexpr int kAdjRowBlocks = 64;

__global__ void __launch_bounds__(256) sum_columns_part_kernel(int64_t p, int M, const double2* __restrict__ contrib,
                                                                double2* __restrict__ part) {
  __shared__ double2 red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + tx;
  double2 acc = make_double2(0.0, 0.0);
  if (i < M)
    for (int64_t q = (int64_t)blockIdx.y + (int64_t)kAdjRowBlocks * ty; q < p; q += (int64_t)kAdjRowBlocks * 8) {
      const double2 v = contrib[(size_t)q * M + i];
      acc.x += v.x;
      acc.y += v.y;
    }
  red[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && i < M) {
    for (int w = 1; w < 8; ++w) {
      acc.x += red[w][tx].x;
      acc.y += red[w][tx].y;
    }
    part[(size_t)blockIdx.y * M + i] = acc;
  }
}

__global__ void sum_columns_kernel(int M, const double2* __restrict__ part, double2* __restrict__ gc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int r = 0; r < kAdjRowBlocks; ++r) {
    const double2 v = part[(size_t)r * M + i];
    acc.x += v.x;
    acc.y += v.y;
  }
  gc[i].x += acc.x;   // chunks of solutions are added in order
  gc[i].y += acc.y;
}

template <typename T>
__global__ void paths_init_kernel(int n, int64_t p, const double2* __restrict__ y0, double tau0,
                                  double dtau0, hpt_paths S) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p * n) {
    const double2 v = y0[i];
    cx<T> c = mk<T>((T)v.x, (T)v.y);
    st<T>(S.y, i, c);
    st<T>(S.y_acc, i, c);
    st<T>(S.dE_acc, i, mk<T>(0, 0));
    if (S.y_prev) {
      st<T>(S.y_prev, i, mk<T>(0, 0));
      st<T>(S.dE_prev, i, mk<T>(0, 0));
    }
  }
  if (i < p) {
    if (S.tau_prev) S.tau_prev[i] = tau0;
    if (S.hermite) S.hermite[i] = 0;
    S.tau[i] = tau0;
    S.tau_acc[i] = tau0;
    S.dtau[i] = dtau0;
    S.status[i] = HPT_PATH_ACTIVE;
    S.steps[i] = 0;
    S.accepts[i] = 0;
    S.rejects[i] = 0;
    S.streak[i] = 0;
  }
}

__global__ void count_active_kernel(int64_t p, const int32_t* __restrict__ status, int32_t* count) {
  int c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p;
       i += (int64_t)gridDim.x * blockDim.x)
    c += status[i] == HPT_PATH_ACTIVE;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

template <typename T>
__global__ void finish_track_kernel(int n, int64_t p, hpt_paths S, double2* __restrict__ x,
                                    int32_t* __restrict__ status_out, int32_t* __restrict__ steps_out,
                                    int32_t* __restrict__ done) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p * n) {
    cx<T> v = ld<T>(S.y_acc, i);
    x[i] = make_double2((double)v.x, (double)v.y);
  }
  if (i < p) {
    const int32_t s = S.status[i];
    if (status_out) status_out[i] = s;
    if (steps_out) steps_out[i] = S.steps[i];
    done[i] = s == HPT_PATH_CONVERGED ? 0 : 3;
  }
}

__global__ void init_done_kernel(int64_t p, const int32_t* __restrict__ status, int32_t* done) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p) done[i] = (!status || status[i] == HPT_PATH_CONVERGED) ? 0 : 3;
}

inline unsigned blocks_for(int64_t threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

// Lane-group shape for n: (G, R) = (8, 1) for n <= 8, (8, 2) for n <= 16,
// (32, 1) for n <= 32.
inline int shape_of(int n) { return n <= 8 ? 0 : (n <= 16 ? 1 : 2); }

template <typename K>
cudaError_t set_smem(K kernel, int bytes) {
  return bytes > 48 * 1024 ? cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                           : cudaSuccess;
}

// Persistent grids: enough blocks to cover the positions once, capped at a
// few waves of resident blocks (the kernels loop over positions).
inline unsigned solve_grid(int64_t p, int G) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int64_t need = std::max<int64_t>(1, (p * G + kSolveThreads - 1) / kSolveThreads);
  return (unsigned)std::min<int64_t>(need, (int64_t)sms * 32);
}

template <typename T, int G, int R>
cudaError_t launch_solve_shape(const StepArgs& a, int32_t* rc, int64_t* rl, cudaStream_t st) {
  const int smem = (kSolveThreads / G) * GroupSmem<T, G * R>::bytes;
  if (!a.map.list) {
    cudaError_t e = set_smem(solve_update_kernel<T, G, R>, smem);
    if (e != cudaSuccess) return e;
    solve_update_kernel<T, G, R><<<blocks_for(a.p * G, kSolveThreads), kSolveThreads, smem, st>>>(
        a.n, a.p, a.ext, a.st, a.prm, rc, rl);
    return cudaGetLastError();
  }
  cudaError_t e = set_smem(solve_update_map_kernel<T, G, R>, smem);
  if (e != cudaSuccess) return e;
  PathMap pm = a.map;
  if (!pm.nmax) pm.nmax = a.n;
  solve_update_map_kernel<T, G, R><<<solve_grid(a.p, G), kSolveThreads, smem, st>>>(a.n, a.p, a.ext, a.st, a.prm,
                                                                                     rc, rl, pm);
  return cudaGetLastError();
}

// FP32 Gauss-Jordan solve + update (n <= 16: (G, R) = (8, 1) or (8, 2)), one
// system or a position map.
template <int G, int R>
cudaError_t launch_gj(const StepArgs& a, cudaStream_t st) {
  const int smem = (kSolveThreads / G) * GjLayout<G, G * R>::bytes;
  if (!a.map.list) {
    cudaError_t e = set_smem(gj_update_kernel<G, R>, smem);
    if (e != cudaSuccess) return e;
    gj_update_kernel<G, R><<<blocks_for(a.p * G, kSolveThreads), kSolveThreads, smem, st>>>(
        a.n, a.p, (const float2*)a.ext, a.st, a.prm, a.redo_count, a.redo_list);
    return cudaGetLastError();
  }
  cudaError_t e = set_smem(gj_update_map_kernel<G, R>, smem);
  if (e != cudaSuccess) return e;
  PathMap pm = a.map;
  if (!pm.nmax) pm.nmax = a.n;
  gj_update_map_kernel<G, R><<<solve_grid(a.p, G), kSolveThreads, smem, st>>>(
      a.n, a.p, (const float2*)a.ext, a.st, a.prm, a.redo_count, a.redo_list, pm);
  return cudaGetLastError();
}

template <int G, int R>
cudaError_t launch_redo_shape(const StepArgs& a, cudaStream_t st) {
  const int smem = (kSolveThreads / G) * GroupSmem<double, G * R>::bytes;
  cudaError_t e = set_smem(redo_fp64_kernel<G, R>, smem);
  if (e != cudaSuccess) return e;
  PathMap pm = a.map;
  if (!pm.nmax) pm.nmax = a.n;
  const unsigned nb = blocks_for(std::min<int64_t>(a.p, 8192) * G, kSolveThreads);
  redo_fp64_kernel<G, R><<<nb, kSolveThreads, smem, st>>>(a.n, a.ext, a.st, a.prm, a.redo_count, a.redo_list, pm);
  return cudaGetLastError();
}

template <int G, int R>
cudaError_t launch_newton_shape(int n, int64_t p, const void* ext, void* x, int32_t* done, float* last,
                                double tol, const PathMap* pm, cudaStream_t st) {
  const int smem = (kSolveThreads / G) * GroupSmem<double, G * R>::bytes;
  if (pm) {
    cudaError_t e = set_smem(newton_kernel<G, R, true>, smem);
    if (e != cudaSuccess) return e;
    newton_kernel<G, R, true><<<blocks_for(p * G, kSolveThreads), kSolveThreads, smem, st>>>(
        n, p, ext, (double2*)x, done, last, tol, *pm);
    return cudaGetLastError();
  }
  cudaError_t e = set_smem(newton_kernel<G, R, false>, smem);
  if (e != cudaSuccess) return e;
  newton_kernel<G, R, false><<<blocks_for(p * G, kSolveThreads), kSolveThreads, smem, st>>>(
      n, p, ext, (double2*)x, done, last, tol, PathMap());
  return cudaGetLastError();
}

template <int G, int R>
cudaError_t launch_adjoint_shape(hpt_system s, int64_t p, const void* ext, const void* x, const void* gx,
                                 void* contrib, cudaStream_t st) {
  const int smem = (kSolveThreads / G) * GroupSmem<double, G * R>::bytes;
  cudaError_t e = set_smem(adjoint_kernel<G, R>, smem);
  if (e != cudaSuccess) return e;
  adjoint_kernel<G, R><<<blocks_for(p * G, kSolveThreads), kSolveThreads, smem, st>>>(
      s->n, p, s->d_msz, s->d_off, s->d_ahat, s->M, ext, (const double2*)x, (const double2*)gx,
      (double2*)contrib);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_solve_update(hpt_system s, const StepArgs& a, cudaStream_t st) {
  if (a.p <= 0) return cudaSuccess;
  const int shape = shape_of(a.n);
  cudaError_t e;
  if (s->prec == HPT_FP64) {
    int pi = prof_begin(s, "solve_update_fp64", st);
    e = shape == 0 ? launch_solve_shape<double, 8, 1>(a, nullptr, nullptr, st)
      : shape == 1 ? launch_solve_shape<double, 8, 2>(a, nullptr, nullptr, st)
                   : launch_solve_shape<double, 32, 1>(a, nullptr, nullptr, st);
    prof_end(s, pi, st);
    return e;
  }
  e = cudaMemsetAsync(a.redo_count, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  int pi;
  if (!a.map.list && shape <= 1) {   // one system, n <= 16: Gauss-Jordan
    pi = prof_begin(s, "solve_gj_fp32", st);
    e = shape == 0 ? launch_gj<8, 1>(a, st) : launch_gj<8, 2>(a, st);
  } else {
    pi = prof_begin(s, "solve_update_fp32", st);
    e = shape == 0 ? launch_solve_shape<float, 8, 1>(a, a.redo_count, a.redo_list, st)
      : shape == 1 ? launch_solve_shape<float, 8, 2>(a, a.redo_count, a.redo_list, st)
                   : launch_solve_shape<float, 32, 1>(a, a.redo_count, a.redo_list, st);
  }
  prof_end(s, pi, st);
  if (e != cudaSuccess) return e;
  // FP64 re-solves: a fixed grid that loops over the device-side list
  pi = prof_begin(s, "redo_fp64", st);
  e = shape == 0 ? launch_redo_shape<8, 1>(a, st)
    : shape == 1 ? launch_redo_shape<8, 2>(a, st)
                 : launch_redo_shape<32, 1>(a, st);
  prof_end(s, pi, st);
  return e;
}

int solve_shape_of(int n) { return shape_of(n); }

cudaError_t launch_newton_map(int shape, int64_t cap, const void* ext, void* x, int32_t* done, float* last,
                              double tol, const PathMap& pm, cudaStream_t st) {
  if (cap <= 0) return cudaSuccess;
  if (!pm.list || !pm.tile_sys || !pm.sys_n || !pm.vofs || !pm.npos || !pm.pos_begin) return cudaErrorInvalidValue;
  return shape == 0 ? launch_newton_shape<8, 1>(0, cap, ext, x, done, last, tol, &pm, st)
       : shape == 1 ? launch_newton_shape<8, 2>(0, cap, ext, x, done, last, tol, &pm, st)
                    : launch_newton_shape<32, 1>(0, cap, ext, x, done, last, tol, &pm, st);
}

cudaError_t launch_solve_fp32_shape(int shape, const StepArgs& a, cudaStream_t st) {
  if (a.p <= 0) return cudaSuccess;
  return shape == 0 ? launch_gj<8, 1>(a, st)
       : shape == 1 ? launch_gj<8, 2>(a, st)
       : shape == kShape8x3 ? launch_solve_shape<float, 8, 3>(a, a.redo_count, a.redo_list, st)
                    : launch_solve_shape<float, 32, 1>(a, a.redo_count, a.redo_list, st);
}

cudaError_t launch_redo_fp64_shape(int shape, const StepArgs& a, cudaStream_t st) {
  if (a.p <= 0) return cudaSuccess;
  return shape == 0 ? launch_redo_shape<8, 1>(a, st)
       : shape == 1 ? launch_redo_shape<8, 2>(a, st)
                    : launch_redo_shape<32, 1>(a, st);
}

cudaError_t launch_newton_update(hpt_system s, int64_t p, const void* ext, void* x, int32_t* done,
                                 float* last, double tol, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const int shape = shape_of(s->n);
  int pi = prof_begin(s, "newton_fp64", st);
  cudaError_t e = shape == 0 ? launch_newton_shape<8, 1>(s->n, p, ext, x, done, last, tol, nullptr, st)
                : shape == 1 ? launch_newton_shape<8, 2>(s->n, p, ext, x, done, last, tol, nullptr, st)
                             : launch_newton_shape<32, 1>(s->n, p, ext, x, done, last, tol, nullptr, st);
  prof_end(s, pi, st);
  return e;
}

size_t adjoint_part_bytes(int M) { return (size_t)kAdjRowBlocks * M * 16; }

cudaError_t launch_adjoint(hpt_system s, int64_t p, const void* ext, const void* x, const void* gx,
                           void* partial, void* part, void* gc, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const int shape = shape_of(s->n);
  int pi = prof_begin(s, "adjoint_fp64", st);
  cudaError_t e = shape == 0 ? launch_adjoint_shape<8, 1>(s, p, ext, x, gx, partial, st)
                : shape == 1 ? launch_adjoint_shape<8, 2>(s, p, ext, x, gx, partial, st)
                             : launch_adjoint_shape<32, 1>(s, p, ext, x, gx, partial, st);
  prof_end(s, pi, st);
  if (e != cudaSuccess) return e;
  pi = prof_begin(s, "adjoint_sum", st);
  sum_columns_part_kernel<<<dim3((unsigned)((s->M + 31) / 32), kAdjRowBlocks), 256, 0, st>>>(
      p, s->M, (const double2*)partial, (double2*)part);
  sum_columns_kernel<<<blocks_for(s->M, 128), 128, 0, st>>>(s->M, (const double2*)part, (double2*)gc);
  prof_end(s, pi, st);
  return cudaGetLastError();
}

cudaError_t launch_paths_init(hpt_system s, int64_t p, const void* y0, double tau0,
                              const hpt_params& prm, const hpt_paths& S, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const unsigned nb = blocks_for(p * s->n, 256);
  if (s->prec == HPT_FP64)
    paths_init_kernel<double><<<nb, 256, 0, st>>>(s->n, p, (const double2*)y0, tau0, prm.dtau_init, S);
  else
    paths_init_kernel<float><<<nb, 256, 0, st>>>(s->n, p, (const double2*)y0, tau0, prm.dtau_init, S);
  return cudaGetLastError();
}

cudaError_t launch_count_active(int64_t p, const int32_t* status, int32_t* count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t), st);
  if (e != cudaSuccess || p <= 0) return e;
  unsigned nb = blocks_for(p, 256);
  if (nb > 1024) nb = 1024;
  count_active_kernel<<<nb, 256, 0, st>>>(p, status, count);
  return cudaGetLastError();
}

cudaError_t launch_finish_track(hpt_system s, int64_t p, const hpt_paths& S, void* x_out,
                                int32_t* status_out, int32_t* steps_out, int32_t* done,
                                cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const unsigned nb = blocks_for(p * s->n, 256);
  if (s->prec == HPT_FP64)
    finish_track_kernel<double><<<nb, 256, 0, st>>>(s->n, p, S, (double2*)x_out, status_out, steps_out, done);
  else
    finish_track_kernel<float><<<nb, 256, 0, st>>>(s->n, p, S, (double2*)x_out, status_out, steps_out, done);
  return cudaGetLastError();
}

cudaError_t launch_init_done(int64_t p, const int32_t* status, int32_t* done, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  init_done_kernel<<<blocks_for(p, 256), 256, 0, st>>>(p, status, done);
  return cudaGetLastError();
}

}  // namespace hpt
