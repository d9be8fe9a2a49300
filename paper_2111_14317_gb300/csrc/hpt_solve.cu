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

template <typename T>
__device__ __forceinline__ T cabs_t(cx<T> a) {
  return hypot(a.x, a.y);
}

// Entry j of a register row without dynamic indexing (folds to a[j] when the
// caller's loop is unrolled).
template <typename T, int G>
__device__ __forceinline__ cx<T> pick(const cx<T> (&a)[G], int j) {
  cx<T> r = a[0];
#pragma unroll
  for (int c = 1; c < G; ++c)
    if (c == j) r = a[c];
  return r;
}

// Solves rows [a | rhsE | rhsN] of an n x n system held one row per lane
// (n <= G).  On return lane j (< n) holds xE, xN = solution component j.
// Returns false (group-uniform) when a pivot is zero or not finite.  cond
// receives max |u_jj| / min |u_jj| over the pivots.  Every loop has a
// constant trip count and rows are only indexed by unrolled constants, so the
// rows stay in registers.
template <typename T, int G>
__device__ bool group_solve(int n, cx<T> (&a)[G], cx<T>& rhsE, cx<T>& rhsN, cx<T>& xE,
                            cx<T>& xN, T& cond) {
  const int lane = threadIdx.x & (G - 1);
  const int gbase = (threadIdx.x & 31) & ~(G - 1);
  bool used = lane >= n;
  int my_col = G;
  bool ok = true;
  T pmax = 0, pmin = 0;
#pragma unroll
  for (int j = 0; j < G; ++j) {
    if (j < n) {
      const cx<T> aj = pick<T, G>(a, j);
      T bv = used ? T(-1) : abs2(aj);
      if (!used && !(bv == bv)) bv = T(0);   // NaN rows stay eligible, flagged below
      int bl = lane;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o, G);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, o, G);
        if (ov > bv || (ov == bv && ol < bl)) { bv = ov; bl = ol; }
      }
      if (!(bv > T(0)) || !isfinite(bv)) ok = false;
      const T pa = sqrt(bv > T(0) ? bv : T(0));
      if (j == 0) { pmax = pa; pmin = pa; }
      else { pmax = fmax(pmax, pa); pmin = fmin(pmin, pa); }
      // broadcast the pivot row one entry at a time and eliminate
      const cx<T> pj = shfl<T, G>(aj, bl);
      const bool elim = !used && lane != bl;
      const cx<T> l = elim ? cdiv(aj, pj) : mk<T>(0, 0);
#pragma unroll
      for (int c = 1; c < G; ++c) {
        if (c > j && c < n) {
          const cx<T> pc = shfl<T, G>(a[c], bl);
          if (elim) a[c] = csub_mul(a[c], l, pc);
        }
      }
      const cx<T> pE = shfl<T, G>(rhsE, bl), pN = shfl<T, G>(rhsN, bl);
      if (elim) {
        rhsE = csub_mul(rhsE, l, pE);
        rhsN = csub_mul(rhsN, l, pN);
      }
      if (lane == bl) {
        used = true;
        my_col = j;
      }
    }
  }
  xE = mk<T>(0, 0);
  xN = mk<T>(0, 0);
#pragma unroll
  for (int jj = 0; jj < G; ++jj) {
    const int j = G - 1 - jj;
    if (j < n) {
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

// One Euler-Newton step per ACTIVE path: solve, then accept/reject and the
// next prediction.  T is the state and solve precision; FP32 solves whose
// pivot ratio exceeds prm.cond_max are redone in FP64 from the same data.
template <typename T, int G>
__global__ void __launch_bounds__(128)
solve_update_kernel(int n, int64_t p, const void* __restrict__ ext, hpt_paths S, hpt_params prm,
                    int32_t* __restrict__ n_fp64) {
  const int lane = threadIdx.x & (G - 1);
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  bool valid = path < p;
  int32_t status = valid ? S.status[path] : -1;
  valid = valid && status == HPT_PATH_ACTIVE;
  if (!__any_sync(0xffffffffu, valid)) return;   // warp-uniform exit

  cx<T> a[G], rhsE, rhsN, xE, xN;
  load_row<T, T, G>(n, ext, path, valid, a, rhsE, rhsN);
  bool fin = true;
#pragma unroll
  for (int c = 0; c < G; ++c) fin = fin && finite(a[c]);
  fin = fin && finite(rhsE) && finite(rhsN);
  fin = group_all<G>(fin);
  T cond;
  bool ok = group_solve<T, G>(n, a, rhsE, rhsN, xE, xN, cond) && fin;
  if (sizeof(T) == 4) {
    // Ill-conditioned in FP32: redo the factorisation in FP64 from the same
    // (FP32) Jacobian.
    const bool redo = valid && ok && !(cond <= (T)prm.cond_max);
    if (__any_sync(0xffffffffu, redo)) {
      cx<double> a2[G], e2, n2, xe2, xn2;
      load_row<double, T, G>(n, ext, path, valid, a2, e2, n2);
      double c2;
      bool ok2 = group_solve<double, G>(n, a2, e2, n2, xe2, xn2, c2);
      if (redo) {
        xE = mk<T>((T)xe2.x, (T)xe2.y);
        xN = mk<T>((T)xn2.x, (T)xn2.y);
        ok = ok2;
        if (lane == 0 && n_fp64) atomicAdd(n_fp64, 1);
      }
    }
  }
  if (!valid) return;   // no shuffles below

  const bool mine = lane < n;
  const size_t vi = (size_t)path * n + lane;
  cx<T> y = mine ? ld<T>(S.y, vi) : mk<T>(0, 0);
  bool solfin = !mine || (finite(xE) && finite(xN));
  // group reductions (only the group's own lanes reach here: all lanes of an
  // active group are valid together)
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  solfin = (__ballot_sync(gmask, solfin) & gmask) == gmask;
  T ny = mine ? cabs_t(y) : T(0), nd = mine ? cabs_t(xN) : T(0);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    ny = fmax(ny, __shfl_xor_sync(gmask, ny, o, G));
    nd = fmax(nd, __shfl_xor_sync(gmask, nd, o, G));
  }
  const bool bad = !(ok && solfin);
  double tau = S.tau[path], dtau = S.dtau[path], tauacc = S.tau_acc[path];
  int32_t steps = S.steps[path] + 1, accepts = S.accepts[path], rejects = S.rejects[path],
          streak = S.streak[path];
  const T err = nd / fmax(T(1), ny);
  const bool accept = !bad && err <= (T)prm.tol_accept;
  cx<T> yacc = mine ? ld<T>(S.y_acc, vi) : mk<T>(0, 0);
  cx<T> dEacc = mine ? ld<T>(S.dE_acc, vi) : mk<T>(0, 0);
  bool predict = true;
  if (accept) {
    yacc = mk<T>(y.x + xN.x, y.y + xN.y);
    dEacc = xE;
    tauacc = tau;
    accepts += 1;
    streak += 1;
    if (tauacc == 0.0) {
      status = HPT_PATH_CONVERGED;
      predict = false;
    } else {
      const T m = mine ? cabs_t(yacc) : T(1);
      bool div = mine && (!(m < (T)prm.div_bound) || !(m > (T)(1.0 / prm.div_bound)));
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
        y = mk<T>(y.x + xN.x, y.y + xN.y);
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
    y = mk<T>(yacc.x + (T)h * dEacc.x, yacc.y + (T)h * dEacc.y);
    tau = tauacc + h;
    if (steps >= prm.max_steps) status = HPT_PATH_MAX_STEPS;
  }
  if (mine) {
    st<T>(S.y, vi, y);
    st<T>(S.y_acc, vi, yacc);
    st<T>(S.dE_acc, vi, dEacc);
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

// Newton polish update at t = 1 (FP64): x += dN until |dN|/max(1,|x|) <= tol.
template <int G>
__global__ void __launch_bounds__(128)
newton_kernel(int n, int64_t p, const void* __restrict__ ext, double2* __restrict__ x,
              int32_t* __restrict__ done, double tol) {
  const int lane = threadIdx.x & (G - 1);
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const bool valid = path < p && done[path] == 0;
  if (!__any_sync(0xffffffffu, valid)) return;
  cx<double> a[G], rE, rN, xE, xN;
  load_row<double, double, G>(n, ext, path, valid, a, rE, rN);
  double cond;
  bool ok = group_solve<double, G>(n, a, rE, rN, xE, xN, cond);
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
  bool ok = group_solve<double, G>(n, a, rE, rN, lam, dummy, cond);
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
  int pi = prof_begin(s, dbl ? "solve_update_fp64" : "solve_update_fp32", st);
  if (dbl) {
    if (G == 8) solve_update_kernel<double, 8><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr);
    else if (G == 16) solve_update_kernel<double, 16><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr);
    else solve_update_kernel<double, 32><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr);
  } else {
    if (G == 8) solve_update_kernel<float, 8><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr);
    else if (G == 16) solve_update_kernel<float, 16><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr);
    else solve_update_kernel<float, 32><<<nb, 128, 0, st>>>(a.n, a.p, a.ext, a.st, a.prm, nullptr);
  }
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
