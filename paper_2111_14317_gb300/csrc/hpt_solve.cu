// Consolidated Euler+Newton solve (Section 6, eq. (11), affine form) and the
// per-path step control, plus the small kernels around them (state init,
// active count, Newton polish at t = 1, implicit-function adjoint).
//
// Solve mapping: a group of G lanes owns one path; lane r holds row r of
// [H_y | H_tau | H] in registers.  Gaussian elimination with partial pivoting
// (pivot = largest |.|^2, ties to the lowest row, as LAPACK's getrf) selects a
// pivot lane per column with a butterfly arg-max, broadcasts the pivot row by
// shuffles and eliminates the remaining rows in place; rows are never moved,
// the column -> pivot-lane map is kept instead.  Back substitution runs
// column-wise: the owner of column j divides, broadcasts x_j, and every row
// pivoting an earlier column updates its right-hand side.  Two right-hand
// sides [-H_tau, -H] give the Euler direction dE and the Newton direction dN
// from one factorisation.
#include <math.h>

#include <algorithm>

#include "hpt_internal.h"

namespace hpt {
namespace {

template <typename T>
struct cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cx<T> csub_mul(cx<T> acc, cx<T> a, cx<T> b) {  // acc - a b
  return mk<T>(acc.x - (a.x * b.x - a.y * b.y), acc.y - (a.x * b.y + a.y * b.x));
}
template <typename T>
__device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
  const T d = b.x * b.x + b.y * b.y;
  return mk<T>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
template <typename T>
__device__ __forceinline__ T abs2(cx<T> a) {
  return a.x * a.x + a.y * a.y;
}
template <typename T>
__device__ __forceinline__ bool finite(cx<T> a) {
  return isfinite(a.x) && isfinite(a.y);
}
template <typename T, int G>
__device__ __forceinline__ cx<T> shfl(cx<T> v, int src) {
  return mk<T>(__shfl_sync(0xffffffffu, v.x, src, G), __shfl_sync(0xffffffffu, v.y, src, G));
}
template <int G>
__device__ __forceinline__ bool group_all(bool v) {
  unsigned m = __ballot_sync(0xffffffffu, v);
  const int lane = threadIdx.x & 31;
  const unsigned seg = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  return (m & seg) == seg;
}
template <typename T, int G>
__device__ __forceinline__ T group_max(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o, G));
  return v;
}

__device__ __forceinline__ float t_hypot(float a, float b) { return hypotf(a, b); }
__device__ __forceinline__ double t_hypot(double a, double b) { return hypot(a, b); }
__device__ __forceinline__ float t_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double t_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float t_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double t_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float t_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double t_sqrt(double a) { return sqrt(a); }
// 2^-e for m in [2^(e-1), 2^e): an exact power-of-two scale bringing m to [1/2, 1)
__device__ __forceinline__ float pow2_inv(float m) {
  int e;
  frexpf(m, &e);
  return (m > 0.f && isfinite(m)) ? ldexpf(1.f, -e) : 1.f;
}
__device__ __forceinline__ double pow2_inv(double m) {
  int e;
  frexp(m, &e);
  return (m > 0.0 && isfinite(m)) ? ldexp(1.0, -e) : 1.0;
}

template <typename T>
__device__ __forceinline__ T cabs_t(cx<T> a) {
  return t_hypot(a.x, a.y);
}
template <typename T>
__device__ __forceinline__ T cmag(cx<T> a) {   // max(|re|, |im|): a cheap magnitude for scaling
  return t_max(fabs(a.x), fabs(a.y));
}

// Entry j of a register row without dynamic indexing.
template <typename T, int G>
__device__ __forceinline__ cx<T> pick(const cx<T> (&a)[G], int j) {
  cx<T> r = a[0];
#pragma unroll
  for (int c = 1; c < G; ++c)
    if (c == j) r = a[c];
  return r;
}

template <typename T, int G>
__device__ __forceinline__ T pick_s(const T (&a)[G], int j) {
  T r = a[0];
#pragma unroll
  for (int c = 1; c < G; ++c)
    if (c == j) r = a[c];
  return r;
}

// Pivot key: the magnitude |a_jj|^2 rounded to float with the low five
// mantissa bits replaced by (31 - row), so that one integer max over the
// group picks the largest magnitude, ties to the lowest row.  Rows already
// used as pivots get key 0 and are never picked.
template <typename T>
__device__ __forceinline__ unsigned pivot_key(T v, bool used, int lane) {
  if (used) return 0u;
  float f = (float)v;
  if (!(f == f)) f = 0.f;   // NaN rows stay eligible; the pivot test flags them
  return (__float_as_uint(f) & ~31u) | (unsigned)(31 - lane);
}

// Two-sided equilibration by exact powers of two: every row, then every
// column of [a] is brought to magnitude [1/2, 1).  The solution of the scaled
// system is x = diag(dcol) x'; pivots then reflect the matrix's conditioning
// rather than the scales of y and t^s in its rows and columns.
template <typename T, int G>
__device__ __forceinline__ void equilibrate(cx<T> (&a)[G], cx<T>& rhsE, cx<T>& rhsN, T (&dcol)[G]) {
  T m = T(0);
#pragma unroll
  for (int c = 0; c < G; ++c) m = t_max(m, cmag(a[c]));
  const T dr = pow2_inv(m);
#pragma unroll
  for (int c = 0; c < G; ++c) a[c] = mk<T>(a[c].x * dr, a[c].y * dr);
  rhsE = mk<T>(rhsE.x * dr, rhsE.y * dr);
  rhsN = mk<T>(rhsN.x * dr, rhsN.y * dr);
#pragma unroll
  for (int c = 0; c < G; ++c) {
    T mc = cmag(a[c]);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) mc = t_max(mc, __shfl_xor_sync(0xffffffffu, mc, o, G));
    dcol[c] = pow2_inv(mc);
    a[c] = mk<T>(a[c].x * dcol[c], a[c].y * dcol[c]);
  }
}

// Solves rows [a | rhsE | rhsN] of an n x n system held one row per lane
// (n <= G) with partial pivoting.  prow is this group's shared-memory pivot
// row buffer (G + 2 entries, 16-byte aligned).  On return lane j (< n) holds
// xE, xN = solution component j.  Returns false (group-uniform) when a pivot
// is zero or not finite; cond receives max |u_jj| / min |u_jj|.
template <typename T, int G>
__device__ bool group_solve(int n, cx<T> (&a)[G], cx<T>& rhsE, cx<T>& rhsN, cx<T>& xE,
                            cx<T>& xN, T& cond, cx<T>* prow) {
  const int lane = threadIdx.x & (G - 1);
  const int gbase = (threadIdx.x & 31) & ~(G - 1);
  bool used = lane >= n;
  int my_col = G;
  bool ok = true;
  T pmax = 0, pmin = 0;
#pragma unroll 1
  for (int j = 0; j < n; ++j) {
    const cx<T> aj = pick<T, G>(a, j);
    unsigned key = pivot_key<T>(abs2(aj), used, lane);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o, G));
    const int bl = 31 - (int)(key & 31u);
    const bool was_used = used;
    if (lane == bl) {
#pragma unroll
      for (int c = 0; c < G; ++c) prow[c] = a[c];
      prow[G] = rhsE;
      prow[G + 1] = rhsN;
      used = true;
      my_col = j;
    }
    __syncwarp();
    const cx<T> pj = prow[j];
    const T p2 = abs2(pj);
    if (!(p2 > T(0)) || !isfinite(p2)) ok = false;
    const T pa = t_sqrt(p2);
    if (j == 0) { pmax = pa; pmin = pa; }
    else { pmax = t_max(pmax, pa); pmin = t_min(pmin, pa); }
    if (!was_used && lane != bl) {
      const cx<T> l = cdiv(aj, pj);
#pragma unroll
      for (int c = 1; c < G; ++c)
        if (c > j) a[c] = csub_mul(a[c], l, prow[c]);
      rhsE = csub_mul(rhsE, l, prow[G]);
      rhsN = csub_mul(rhsN, l, prow[G + 1]);
    }
    __syncwarp();
  }
  xE = mk<T>(0, 0);
  xN = mk<T>(0, 0);
#pragma unroll 1
  for (int j = n - 1; j >= 0; --j) {
    // the lane that pivoted column j
    const unsigned b = __ballot_sync(0xffffffffu, my_col == j);
    const unsigned seg = (G == 32) ? b : ((b >> gbase) & ((1u << G) - 1u));
    const int owner = seg ? (__ffs(seg) - 1) : 0;
    const cx<T> aj = pick<T, G>(a, j);
    cx<T> ve = mk<T>(0, 0), vn = mk<T>(0, 0);
    if (lane == owner) {
      ve = cdiv(rhsE, aj);
      vn = cdiv(rhsN, aj);
    }
    ve = shfl<T, G>(ve, owner);
    vn = shfl<T, G>(vn, owner);
    if (lane == j) { xE = ve; xN = vn; }
    if (my_col < j) {
      rhsE = csub_mul(rhsE, aj, ve);
      rhsN = csub_mul(rhsN, aj, vn);
    }
  }
  cond = pmin > T(0) ? pmax / pmin : T(INFINITY);
  return ok;
}

template <typename T>
struct cplx_t;
template <>
struct cplx_t<double> {
  typedef double2 type;
};
template <>
struct cplx_t<float> {
  typedef float2 type;
};

template <typename T>
__device__ __forceinline__ cx<T> ld(const void* base, size_t idx) {
  const typename cplx_t<T>::type v = ((const typename cplx_t<T>::type*)base)[idx];
  return mk<T>(v.x, v.y);
}
template <typename T>
__device__ __forceinline__ void st(void* base, size_t idx, cx<T> v) {
  typename cplx_t<T>::type w;
  w.x = v.x;
  w.y = v.y;
  ((typename cplx_t<T>::type*)base)[idx] = w;
}

// Loads row `lane` of path `path` from the extended Jacobian (T-precision
// storage S) into the solve registers.
template <typename T, typename S, int G>
__device__ __forceinline__ void load_row(int n, const void* ext, int64_t path, bool valid, cx<T> (&a)[G],
                                         cx<T>& rhsE, cx<T>& rhsN) {
  const int lane = threadIdx.x & (G - 1);
  const bool have = valid && lane < n;
  const size_t base = ((size_t)path * n + lane) * (n + 2);
#pragma unroll
  for (int c = 0; c < G; ++c) {
    a[c] = mk<T>(0, 0);
    if (have && c < n) {
      cx<S> v = ld<S>(ext, base + c);
      a[c] = mk<T>((T)v.x, (T)v.y);
    }
  }
  rhsE = mk<T>(0, 0);
  rhsN = mk<T>(0, 0);
  if (have) {
    cx<S> ht = ld<S>(ext, base + n), h = ld<S>(ext, base + n + 1);
    rhsE = mk<T>(-(T)ht.x, -(T)ht.y);
    rhsN = mk<T>(-(T)h.x, -(T)h.y);
  }
}

// Equilibrated solve of one path's [H_y | -H_tau | -H]; the solution is
// returned unscaled.  Precision T, extended Jacobian stored in precision S.
template <typename T, typename S, int G>
__device__ __forceinline__ bool path_solve(int n, const void* ext, int64_t path, bool valid, cx<T>* prow,
                                           cx<T>& xE, cx<T>& xN, T& cond) {
  const int lane = threadIdx.x & (G - 1);
  cx<T> a[G], rhsE, rhsN;
  load_row<T, S, G>(n, ext, path, valid, a, rhsE, rhsN);
  bool fin = true;
#pragma unroll
  for (int c = 0; c < G; ++c) fin = fin && finite(a[c]);
  fin = group_all<G>(fin && finite(rhsE) && finite(rhsN));
  T dcol[G];
  equilibrate<T, G>(a, rhsE, rhsN, dcol);
  const bool ok = group_solve<T, G>(n, a, rhsE, rhsN, xE, xN, cond, prow) && fin;
  const T dj = pick_s<T, G>(dcol, lane);
  xE = mk<T>(xE.x * dj, xE.y * dj);
  xN = mk<T>(xN.x * dj, xN.y * dj);
  return ok;
}

// Step control of one path (all lanes of its group), given the directions:
// accept/reject, then the next prediction.  TS is the state precision.
template <typename TS, int G>
__device__ __forceinline__ void update_path(int n, int64_t path, int32_t status, bool ok, cx<TS> xE,
                                            cx<TS> xN, const hpt_paths& S, const hpt_params& prm) {
  const int lane = threadIdx.x & (G - 1);
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const bool mine = lane < n;
  const size_t vi = (size_t)path * n + lane;
  cx<TS> y = mine ? ld<TS>(S.y, vi) : mk<TS>(0, 0);
  bool solfin = !mine || (finite(xE) && finite(xN));
  solfin = (__ballot_sync(gmask, solfin) & gmask) == gmask;
  TS ny = mine ? cabs_t(y) : TS(0), nd = mine ? cabs_t(xN) : TS(0);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    ny = t_max(ny, __shfl_xor_sync(gmask, ny, o, G));
    nd = t_max(nd, __shfl_xor_sync(gmask, nd, o, G));
  }
  const bool bad = !(ok && solfin);
  double tau = S.tau[path], dtau = S.dtau[path], tauacc = S.tau_acc[path];
  int32_t steps = S.steps[path] + 1, accepts = S.accepts[path], rejects = S.rejects[path],
          streak = S.streak[path];
  const TS err = nd / t_max(TS(1), ny);
  const bool accept = !bad && err <= (TS)prm.tol_accept;
  cx<TS> yacc = mine ? ld<TS>(S.y_acc, vi) : mk<TS>(0, 0);
  cx<TS> dEacc = mine ? ld<TS>(S.dE_acc, vi) : mk<TS>(0, 0);
  bool predict = true;
  if (accept) {
    yacc = mk<TS>(y.x + xN.x, y.y + xN.y);
    dEacc = xE;
    tauacc = tau;
    accepts += 1;
    streak += 1;
    if (tauacc == 0.0) {
      status = HPT_PATH_CONVERGED;
      predict = false;
    } else {
      const TS m = mine ? cabs_t(yacc) : TS(1);
      bool div = mine && (!(m < (TS)prm.div_bound) || !(m > (TS)(1.0 / prm.div_bound)));
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
        y = mk<TS>(y.x + xN.x, y.y + xN.y);
        yacc = y;
        if (steps >= prm.max_steps) status = HPT_PATH_MAX_STEPS;
      }
    } else {
      dtau *= prm.shrink;
      if (dtau < prm.dtau_min) {
        status = HPT_PATH_UNDERFLOW;
        predict = false;
      }
    }
  }
  if (predict) {
    const double h = fmin(dtau, -tauacc);
    y = mk<TS>(yacc.x + (TS)h * dEacc.x, yacc.y + (TS)h * dEacc.y);
    tau = tauacc + h;
    if (steps >= prm.max_steps) status = HPT_PATH_MAX_STEPS;
  }
  if (mine) {
    st<TS>(S.y, vi, y);
    st<TS>(S.y_acc, vi, yacc);
    st<TS>(S.dE_acc, vi, dEacc);
  }
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

// One Euler-Newton step per ACTIVE path: consolidated solve, then the step
// control.  T is the state and solve precision.  FP32 solves whose pivot
// ratio (after equilibration) exceeds prm.cond_max are not applied here: the
// path goes to redo_list and is solved again in FP64 by redo_fp64_kernel.
template <typename T, int G>
__global__ void __launch_bounds__(128)
solve_update_kernel(int n, int64_t p, const void* __restrict__ ext, hpt_paths S, hpt_params prm,
                    int32_t* __restrict__ redo_count, int64_t* __restrict__ redo_list) {
  const int lane = threadIdx.x & (G - 1);
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  bool valid = path < p;
  const int32_t status = valid ? S.status[path] : -1;
  valid = valid && status == HPT_PATH_ACTIVE;
  if (!__any_sync(0xffffffffu, valid)) return;   // warp-uniform exit
  __shared__ __align__(16) cx<T> prow_buf[128 / G][G + 2];
  cx<T> xE, xN;
  T cond;
  const bool ok = path_solve<T, T, G>(n, ext, path, valid, prow_buf[threadIdx.x / G], xE, xN, cond);
  if (!valid) return;   // group-uniform; only group-masked shuffles below
  if (sizeof(T) == 4 && redo_list && ok && !(cond <= (T)prm.cond_max)) {
    if (lane == 0) redo_list[atomicAdd(redo_count, 1)] = path;
    return;
  }
  update_path<T, G>(n, path, status, ok, xE, xN, S, prm);
}

// FP64 re-solve of the paths listed by the FP32 kernel (same FP32 Jacobian,
// FP64 factorisation), then their step control in the FP32 state.
template <int G>
__global__ void __launch_bounds__(128)
redo_fp64_kernel(int n, const void* __restrict__ ext, hpt_paths S, hpt_params prm,
                 const int32_t* __restrict__ redo_count, const int64_t* __restrict__ redo_list) {
  __shared__ __align__(16) cx<double> prow_buf[128 / G][G + 2];
  const int count = *redo_count;
  const int groups_per_warp = 32 / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  const int g = (threadIdx.x & 31) / G;
  for (int64_t base = warp_id * groups_per_warp; base < count; base += nwarps * groups_per_warp) {
    const int64_t i = base + g;
    const bool valid = i < count;
    const int64_t path = valid ? redo_list[i] : 0;
    cx<double> xE, xN;
    double cond;
    const bool ok = path_solve<double, float, G>(n, ext, path, valid, prow_buf[threadIdx.x / G], xE, xN, cond);
    if (valid)
      update_path<float, G>(n, path, S.status[path], ok, mk<float>((float)xE.x, (float)xE.y),
                            mk<float>((float)xN.x, (float)xN.y), S, prm);
    __syncwarp();
  }
}

// Newton polish update at t = 1 (FP64): x += dN until |dN|/max(1,|x|) <= tol.
template <int G>
__global__ void __launch_bounds__(128)
newton_kernel(int n, int64_t p, const void* __restrict__ ext, double2* __restrict__ x,
              int32_t* __restrict__ done, double tol) {
  const int lane = threadIdx.x & (G - 1);
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const bool valid = path < p && done[path] == 0;
  if (!__any_sync(0xffffffffu, valid)) return;
  __shared__ __align__(16) cx<double> prow_buf[128 / G][G + 2];
  cx<double> xE, xN;
  double cond;
  bool ok = path_solve<double, double, G>(n, ext, path, valid, prow_buf[threadIdx.x / G], xE, xN, cond);
  if (!valid) return;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const bool mine = lane < n;
  const size_t vi = (size_t)path * n + lane;
  cx<double> y = mine ? ld<double>(x, vi) : mk<double>(0, 0);
  bool fin = !mine || finite(xN);
  fin = (__ballot_sync(gmask, fin) & gmask) == gmask;
  if (!(ok && fin)) {
    if (lane == 0) done[path] = 2;
    return;
  }
  y = mk<double>(y.x + xN.x, y.y + xN.y);
  double ny = mine ? cabs_t(y) : 0.0, nd = mine ? cabs_t(xN) : 0.0;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    ny = fmax(ny, __shfl_xor_sync(gmask, ny, o, G));
    nd = fmax(nd, __shfl_xor_sync(gmask, nd, o, G));
  }
  if (mine) st<double>(x, vi, y);
  if (lane == 0 && nd / fmax(1.0, ny) <= tol) done[path] = 1;
}

// Adjoint, part 1: per solution, lambda from J^H lambda = gx (J from the
// extended Jacobian at t = 1), then contrib[q][i] = -lambda_k conj(x^{a_i})
// for every monomial i of equation k (monomials by exp of <a, log x>).
template <int G>
__global__ void __launch_bounds__(128)
adjoint_kernel(int n, int64_t p, const int32_t* __restrict__ msz, const int32_t* __restrict__ off,
               const double* __restrict__ ahat, int M, const void* __restrict__ ext,
               const double2* __restrict__ x, const double2* __restrict__ gx,
               double2* __restrict__ contrib) {
  __shared__ double2 zsh[128 / G][G];
  const int lane = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G;
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const bool valid = path < p;
  cx<double> a[G], rE, rN, lam, dummy;
  const bool have = valid && lane < n;
  // row `lane` of J^H = conj of column `lane` of J
#pragma unroll
  for (int c = 0; c < G; ++c) {
    a[c] = mk<double>(0, 0);
    if (have && c < n) {
      cx<double> v = ld<double>(ext, ((size_t)path * n + c) * (n + 2) + lane);
      a[c] = mk<double>(v.x, -v.y);
    }
  }
  rE = have ? ld<double>(gx, (size_t)path * n + lane) : mk<double>(0, 0);
  rN = mk<double>(0, 0);
  double cond;
  __shared__ __align__(16) cx<double> prow_buf[128 / G][G + 2];
  bool ok = group_solve<double, G>(n, a, rE, rN, lam, dummy, cond, prow_buf[threadIdx.x / G]);
  if (have) {
    const double2 v = x[(size_t)path * n + lane];
    zsh[grp][lane] = make_double2(log(hypot(v.x, v.y)), atan2(v.y, v.x));
  }
  __syncwarp();
  __syncthreads();
  if (!have) return;
  const int k = lane;
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
    double2 v = make_double2(-(lam.x * mr - lam.y * mi), -(lam.x * mi + lam.y * mr));
    if (!ok) v = make_double2(NAN, NAN);
    contrib[(size_t)path * M + i] = v;
  }
}

// Adjoint, part 2: gc[i] += sum over the chunk's solutions of contrib[q][i],
// in order.
__global__ void sum_columns_kernel(int64_t p, int M, const double2* __restrict__ contrib,
                                   double2* __restrict__ gc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t q = 0; q < p; ++q) {
    const double2 v = contrib[(size_t)q * M + i];
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
  }
  if (i < p) {
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

}  // namespace

cudaError_t launch_solve_update(hpt_system s, const StepArgs& a, cudaStream_t st) {
  if (a.p <= 0) return cudaSuccess;
  const bool dbl = s->prec == HPT_FP64;
  const int G = a.n <= 8 ? 8 : (a.n <= 16 ? 16 : 32);
  const unsigned nb = blocks_for(a.p * G, 128);
  if (dbl) {
    int pi = prof_begin(s, "solve_update_fp64", st);
    if (G == 8) solve_update_kernel<double, 8><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr, nullptr);
    else if (G == 16) solve_update_kernel<double, 16><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr, nullptr);
    else solve_update_kernel<double, 32><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr, nullptr);
    prof_end(s, pi, st);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(a.redo_count, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  int pi = prof_begin(s, "solve_update_fp32", st);
  if (G == 8) solve_update_kernel<float, 8><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, a.redo_count, a.redo_list);
  else if (G == 16) solve_update_kernel<float, 16><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, a.redo_count, a.redo_list);
  else solve_update_kernel<float, 32><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, a.redo_count, a.redo_list);
  prof_end(s, pi, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // FP64 re-solves: a fixed grid that loops over the device-side list
  unsigned rb = blocks_for(std::min<int64_t>(a.p, 8192) * G, 128);
  pi = prof_begin(s, "redo_fp64", st);
  if (G == 8) redo_fp64_kernel<8><<<rb, 128, 0, st>>>(a.n, a.ext, a.st, a.prm, a.redo_count, a.redo_list);
  else if (G == 16) redo_fp64_kernel<16><<<rb, 128, 0, st>>>(a.n, a.ext, a.st, a.prm, a.redo_count, a.redo_list);
  else redo_fp64_kernel<32><<<rb, 128, 0, st>>>(a.n, a.ext, a.st, a.prm, a.redo_count, a.redo_list);
  prof_end(s, pi, st);
  return cudaGetLastError();
}

cudaError_t launch_newton_update(hpt_system s, int64_t p, const void* ext, void* x, int32_t* done,
                                 double tol, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const int G = s->n <= 8 ? 8 : (s->n <= 16 ? 16 : 32);
  const unsigned nb = blocks_for(p * G, 128);
  int pi = prof_begin(s, "newton_fp64", st);
  if (G == 8) newton_kernel<8><<<nb, 128, 0, st>>>(s->n, p, ext, (double2*)x, done, tol);
  else if (G == 16) newton_kernel<16><<<nb, 128, 0, st>>>(s->n, p, ext, (double2*)x, done, tol);
  else newton_kernel<32><<<nb, 128, 0, st>>>(s->n, p, ext, (double2*)x, done, tol);
  prof_end(s, pi, st);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(hpt_system s, int64_t p, const void* ext, const void* x, const void* gx,
                           void* partial, int64_t nblk, void* gc, cudaStream_t st) {
  (void)nblk;
  if (p <= 0) return cudaSuccess;
  const int G = s->n <= 8 ? 8 : (s->n <= 16 ? 16 : 32);
  const unsigned nb = blocks_for(p * G, 128);
  int pi = prof_begin(s, "adjoint_fp64", st);
  if (G == 8)
    adjoint_kernel<8><<<nb, 128, 0, st>>>(s->n, p, s->d_msz, s->d_off, s->d_ahat, s->M, ext, (const double2*)x, (const double2*)gx, (double2*)partial);
  else if (G == 16)
    adjoint_kernel<16><<<nb, 128, 0, st>>>(s->n, p, s->d_msz, s->d_off, s->d_ahat, s->M, ext, (const double2*)x, (const double2*)gx, (double2*)partial);
  else
    adjoint_kernel<32><<<nb, 128, 0, st>>>(s->n, p, s->d_msz, s->d_off, s->d_ahat, s->M, ext, (const double2*)x, (const double2*)gx, (double2*)partial);
  prof_end(s, pi, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  pi = prof_begin(s, "adjoint_sum", st);
  sum_columns_kernel<<<blocks_for(s->M, 128), 128, 0, st>>>(p, s->M, (const double2*)partial, (double2*)gc);
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
