// Algorithm 3 (EulerNewton, Section 6) in its QR null-space form, for the
// projective formulation (Section 2.2) and, without the y^* row, for the
// affine one; plus the step of the projective tracker.
//
// The consolidated matrix of one point is
//   J = [[dH/dy, dH/dtau, H], [y^*, 0, 0]]      (N x (N+2), N = nv)
// (projective: n equations and the y^* row, nv = n + 1; affine: the n
// equations alone, nv = n).  The paper factors J^T = Q [R; 0]; the rows of
// [e_{N+1}; e_{N+2}] Q^* span the null space of J, and the row reduction that
// makes their rightmost 2 x 2 block the identity leaves the Euler direction
// (eq. (4)) and the Newton direction (eq. (5)) in their first N columns.
//
// Here the same factorisation is computed on J itself: Householder
// reflections applied from the right, P_k = I - beta_k conj(g_k) g_k^T on
// columns k.., reduce J to [L 0] (L = R^T lower triangular); Qt = P_0 ..
// P_{N-1} equals conj(Q), so the null vectors conj(Q e_{N+1}), conj(Q e_{N+2})
// of the paper are Qt e_N, Qt e_{N+1}, formed by applying the reflectors to
// e_N and e_{N+1} in reverse order.  Reflector of row r (its live part
// r_0, r_1, ..): sigma = |r|, g = r + e^{i arg r_0} sigma e_0, beta =
// 1 / (sigma (sigma + |r_0|)); r P = -e^{i arg r_0} sigma e_0.
//
// Log coordinates: the scratch holds D_z H = (dH/dy) diag(y).  The null
// vectors of J diag(y, 1, 1) are those of J with their first nv entries
// divided by y, so the kernel factors [[D_z H, H_tau, H], [|y_j|^2, 0, 0]]
// and multiplies its directions by y at the end (n products, no divisions).
// Every row is first scaled by an exact power of two (its null space does
// not change).
//
// Mapping (as the LU solve): a group of G lanes owns one path, lane l holds
// rows l + G s (s < R) in registers, "shifted" so that register 0 is the
// current column; row k's owner writes g_k (live width, padded with zeros to
// a multiple of four) into the group's shared memory, packed row after row,
// from where all lanes read it for the dot products <row, g> and the
// updates.  In the reverse pass column c of both null vectors lives in lane
// c mod G, so lane l ends with the entries of its own variables l + G s.
#include <math.h>

#include "hpt_cx.cuh"
#include "hpt_internal.h"

namespace hpt {
namespace {

constexpr int kQrThreads = 128;

// Shared memory of one group: the reflectors g_k packed (row k holds
// round_up(C - k, 4) complex) and beta_k; padded so that consecutive groups
// start 8 banks apart.
template <typename T, int G, int R, int CM>
struct QrSmem {
  static constexpr int NR = G * R;
  static constexpr int entries = NR * CM + 4 * NR;   // >= sum_k round_up(C - k, 4) + CM slack
  static constexpr int raw_words = (entries * 2 * (int)sizeof(T) + NR * (int)sizeof(T)) / 4;
  static constexpr int words = (raw_words + 31) / 32 * 32 + 8;
  static constexpr int bytes = words * 4;
};

__device__ __forceinline__ int round4(int v) { return (v + 3) & ~3; }

// Loads the rows of one path (rows < n from the scratch, the y^* row in log
// coordinates if proj), scales each by a power of two; returns whether every
// entry is finite (group-uniform).
template <typename T, typename S, int G, int R, int CM>
__device__ __forceinline__ bool qr_load(int n, int nv, int proj, const void* __restrict__ ext, int64_t q,
                                        const void* __restrict__ y, size_t vbase, bool valid, cx<T> (&a)[R][CM]) {
  const int lane = threadIdx.x & (G - 1);
  const int C = nv + 2;
  T chk = T(0);
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = lane + G * s;
    const bool eq = valid && r < n;
    const bool ystar = valid && proj && r == n;
#pragma unroll
    for (int c = 0; c < CM; ++c) {
      a[s][c] = mk<T>(0, 0);
      if (c < C) {
        if (eq) {
          const cx<S> v = ld<S>(ext, ext_index(q, r, c, nv));
          a[s][c] = mk<T>((T)v.x, (T)v.y);
        } else if (ystar && c < nv) {
          const cx<S> v = ld<S>(y, vbase + c);
          a[s][c] = mk<T>((T)v.x * (T)v.x + (T)v.y * (T)v.y, T(0));
        }
      }
      chk += t_abs(a[s][c].x) + t_abs(a[s][c].y);
    }
    T m = T(0);
#pragma unroll
    for (int c = 0; c < CM; ++c) m = t_max(m, cmag(a[s][c]));
    const T d = pow2_inv(m);
#pragma unroll
    for (int c = 0; c < CM; ++c) a[s][c] = cscale(a[s][c], d);
  }
  const unsigned ball = __ballot_sync(0xffffffffu, isfinite(chk));
  const unsigned seg = group_mask<G>();
  return (ball & seg) == seg;
}

// The factorisation and the null space of one path (N = nv rows, C = nv + 2
// columns; every group of the warp has the same nv).  On return lane l holds
// the directions of variables j = l + G s in log coordinates (wE[s], wN[s],
// still to be multiplied by y_j); false (group-uniform) when a reflector
// norm is zero, the 2 x 2 block is singular or a value is not finite.
template <typename T, int G, int R, int CM>
__device__ __forceinline__ bool qr_null(int nv, cx<T> (&a)[R][CM], cx<T> (&wE)[R], cx<T> (&wN)[R],
                                        unsigned char* sm) {
  const int lane = threadIdx.x & (G - 1);
  const int N = nv, C = nv + 2;
  cx<T>* U = (cx<T>*)sm;
  T* beta = (T*)(sm + QrSmem<T, G, R, CM>::entries * sizeof(cx<T>));
  bool used[R];
#pragma unroll
  for (int s = 0; s < R; ++s) used[s] = false;
  bool ok = true;
  int off = 0;   // packed offset of row k's reflector
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    const int width = C - k, len = round4(width);
    const int ol = k & (G - 1), os = k / G;
    if (lane == ol) {
      // the owner's slot chosen entry by entry (static register indices)
      T s2 = T(0);
#pragma unroll
      for (int c = 0; c < CM; ++c) {
        cx<T> v = a[0][c];
#pragma unroll
        for (int s = 1; s < R; ++s) v = (os == s) ? a[s][c] : v;
        if (c < width) s2 += abs2(v);
      }
      const T sigma = t_sqrt(s2);
      cx<T> r0 = a[0][0];
#pragma unroll
      for (int s = 1; s < R; ++s) r0 = (os == s) ? a[s][0] : r0;
      const T m0 = cabs_t(r0);
      // e^{i arg r0} sigma (phase 1 when r0 = 0)
      const cx<T> ph = m0 > T(0) ? cscale(r0, sigma / m0) : mk<T>(sigma, T(0));
      const T b = sigma > T(0) ? T(1) / (sigma * (sigma + m0)) : T(0);
#pragma unroll
      for (int c = 0; c < CM; ++c) {
        cx<T> v = a[0][c];
#pragma unroll
        for (int s = 1; s < R; ++s) v = (os == s) ? a[s][c] : v;
        if (c == 0) v = mk<T>(v.x + ph.x, v.y + ph.y);
        if (c < len) U[off + c] = c < width ? v : mk<T>(0, 0);
      }
      beta[k] = b;
#pragma unroll
      for (int s = 0; s < R; ++s) used[s] = used[s] || (os == s);
    }
    __syncwarp();
    const T b = beta[k];
    if (!(b > T(0)) || !isfinite(b)) ok = false;
    // t_s = beta <row_s, g> over the live width (rows already used: 0)
    cx<T> t[R];
#pragma unroll
    for (int s = 0; s < R; ++s) t[s] = mk<T>(0, 0);
#pragma unroll
    for (int c0 = 0; c0 < CM; c0 += 4) {
      if (c0 < width) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c) {
          if (c < CM) {
            const cx<T> g = U[off + c];
#pragma unroll
            for (int s = 0; s < R; ++s) {   // t += row conj(g)
              t[s].x += a[s][c].x * g.x + a[s][c].y * g.y;
              t[s].y += a[s][c].y * g.x - a[s][c].x * g.y;
            }
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < R; ++s) t[s] = used[s] ? mk<T>(0, 0) : cscale(t[s], b);
    // shifted update: a[c-1] = a[c] - t g[c] (column k leaves the rows: it is L's)
#pragma unroll
    for (int c0 = 0; c0 < CM; c0 += 4) {
      if (c0 < width) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c) {
          if (c >= 1 && c < CM) {
            const cx<T> g = U[off + c];
#pragma unroll
            for (int s = 0; s < R; ++s) a[s][c - 1] = csub_mul(a[s][c], t[s], g);
          }
        }
      }
    }
    off += len;
  }
  // reverse pass: z1 = Qt e_N, z2 = Qt e_{N+1}, z <- P_k z for k = N-1 .. 0,
  // P_k z = z - beta_k conj(g_k) (g_k . z) on the absolute columns k .. C-1.
  // Column c of both vectors lives in lane c mod G, slot c / G; the dot
  // products are butterfly sums over the group.
  constexpr int RC = (CM + G - 1) / G;
  cx<T> z1[RC], z2[RC];
#pragma unroll
  for (int i = 0; i < RC; ++i) {
    const int c = lane + G * i;
    z1[i] = mk<T>(c == N ? T(1) : T(0), T(0));
    z2[i] = mk<T>(c == N + 1 ? T(1) : T(0), T(0));
  }
#pragma unroll 1
  for (int k = N - 1; k >= 0; --k) {
    off -= round4(C - k);
    const T b = beta[k];
    cx<T> g[RC];
    cx<T> s1 = mk<T>(0, 0), s2 = mk<T>(0, 0);
#pragma unroll
    for (int i = 0; i < RC; ++i) {
      const int c = lane + G * i;
      g[i] = (c >= k && c < C) ? U[off + c - k] : mk<T>(0, 0);
      s1 = mk<T>(s1.x + g[i].x * z1[i].x - g[i].y * z1[i].y, s1.y + g[i].x * z1[i].y + g[i].y * z1[i].x);
      s2 = mk<T>(s2.x + g[i].x * z2[i].x - g[i].y * z2[i].y, s2.y + g[i].x * z2[i].y + g[i].y * z2[i].x);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      s1.x += __shfl_xor_sync(0xffffffffu, s1.x, o, G);
      s1.y += __shfl_xor_sync(0xffffffffu, s1.y, o, G);
      s2.x += __shfl_xor_sync(0xffffffffu, s2.x, o, G);
      s2.y += __shfl_xor_sync(0xffffffffu, s2.y, o, G);
    }
    s1 = cscale(s1, b);
    s2 = cscale(s2, b);
#pragma unroll
    for (int i = 0; i < RC; ++i) {
      const cx<T> gc = mk<T>(g[i].x, -g[i].y);
      z1[i] = csub_mul(z1[i], s1, gc);
      z2[i] = csub_mul(z2[i], s2, gc);
    }
  }
  // 2 x 2 reduction: [[a, b], [c, d]] = rightmost block of [z1^T; z2^T]
  // (columns N and N + 1), passed through the group's shared memory by the
  // lanes that hold them (predicated stores keep the register indices static)
  __syncwarp();   // every lane is done with the reflectors
#pragma unroll
  for (int i = 0; i < RC; ++i) {
    const int c = lane + G * i;
    if (c == N) { U[0] = z1[i]; U[1] = z2[i]; }
    if (c == N + 1) { U[2] = z1[i]; U[3] = z2[i]; }
  }
  __syncwarp();
  const cx<T> ea = U[0], ec = U[1], eb = U[2], ed = U[3];
  __syncwarp();   // the group's shared memory is reused by its next path
  const cx<T> det = mk<T>(ea.x * ed.x - ea.y * ed.y - (eb.x * ec.x - eb.y * ec.y),
                          ea.x * ed.y + ea.y * ed.x - (eb.x * ec.y + eb.y * ec.x));
  const T d2 = abs2(det);
  if (!(d2 > T(0)) || !isfinite(d2)) ok = false;
  const cx<T> idet = mk<T>(det.x / d2, -det.y / d2);
  // variable j = lane + G s is column j: slot s of this lane
#pragma unroll
  for (int s = 0; s < R; ++s) {
    // row 0 of the reduced V: (d z1 - b z2) / det; row 1: (a z2 - c z1) / det
    wE[s] = cmul(csub_mul(cmul(ed, z1[s]), eb, z2[s]), idet);
    wN[s] = cmul(csub_mul(cmul(ea, z2[s]), ec, z1[s]), idet);
  }
  return ok;
}

// Step control of one projective path (all lanes of its group), given the
// directions in y coordinates: the affine rule with the point scaled back to
// unit norm after every correction and divergence judged on y_j / y_n.
template <typename T, int G, int R>
__device__ __forceinline__ void update_proj(int n, int nv, int64_t path, size_t vbase, int32_t status, bool ok,
                                            const cx<T> (&xE)[R], const cx<T> (&xN)[R], const hpt_paths& S,
                                            const hpt_params& prm) {
  const int lane = threadIdx.x & (G - 1);
  const unsigned gmask = group_mask<G>();
  cx<T> y[R], yacc[R], dEacc[R];
  bool solfin = true;
  T ny = T(0), nd = T(0);
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    const bool mine = j < nv;
    y[s] = mine ? ld<T>(S.y, vbase + j) : mk<T>(0, 0);
    yacc[s] = mine ? ld<T>(S.y_acc, vbase + j) : mk<T>(0, 0);
    dEacc[s] = mine ? ld<T>(S.dE_acc, vbase + j) : mk<T>(0, 0);
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
  double tau = S.tau[path], dtau = S.dtau[path], tauacc = S.tau_acc[path];
  int32_t steps = S.steps[path] + 1, accepts = S.accepts[path], rejects = S.rejects[path],
          streak = S.streak[path];
  const T err = nd / t_max(T(1), ny);
  const bool accept = !bad && err <= (T)prm.tol_accept;
  // |w|_2 of w = y + dN over the group
  auto unit = [&](cx<T>(&w)[R]) -> T {
    T s2 = T(0);
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (lane + G * s < nv) s2 += abs2(w[s]);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s2 += __shfl_xor_sync(gmask, s2, o, G);
    return T(1) / t_sqrt(s2);
  };
  bool predict = true;
  if (accept) {
    cx<T> w[R];
#pragma unroll
    for (int s = 0; s < R; ++s) w[s] = mk<T>(y[s].x + xN[s].x, y[s].y + xN[s].y);
    const T inv = unit(w);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      yacc[s] = cscale(w[s], inv);
      dEacc[s] = cscale(xE[s], inv);
    }
    tauacc = tau;
    accepts += 1;
    streak += 1;
    // |y_n| from its lane, then the dehomogenized magnitudes |y_j / y_n|
    cx<T> vh = yacc[0];
#pragma unroll
    for (int s = 1; s < R; ++s)
      if (s == n / G) vh = yacc[s];
    const T mh = __shfl_sync(gmask, cabs_t(vh), n & (G - 1), G);
    bool div = false;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      if (lane + G * s < n) {
        const T m = cabs_t(yacc[s]) / mh;
        div = div || !(m < (T)prm.div_bound) || !(m > (T)(1.0 / prm.div_bound));
      }
    }
    div = (__ballot_sync(gmask, div) & gmask) != 0u;
    if (div) {
      status = HPT_PATH_DIVERGED;
      predict = false;
    } else if (tauacc == 0.0) {
      status = HPT_PATH_CONVERGED;
      predict = false;
    } else if (streak >= prm.grow_after) {
      dtau = fmin(dtau * prm.grow, prm.dtau_max);
      streak = 0;
    }
  } else {
    rejects += 1;
    streak = 0;
    if (accepts == 0) {
      predict = false;
      if (bad) {
        status = HPT_PATH_SINGULAR;
      } else {
        cx<T> w[R];
#pragma unroll
        for (int s = 0; s < R; ++s) w[s] = mk<T>(y[s].x + xN[s].x, y[s].y + xN[s].y);
        const T inv = unit(w);
#pragma unroll
        for (int s = 0; s < R; ++s) {
          y[s] = cscale(w[s], inv);
          yacc[s] = y[s];
        }
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
#pragma unroll
    for (int s = 0; s < R; ++s) y[s] = mk<T>(yacc[s].x + (T)h * dEacc[s].x, yacc[s].y + (T)h * dEacc[s].y);
    tau = tauacc + h;
    if (steps >= prm.max_steps) status = HPT_PATH_MAX_STEPS;
  }
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    if (j < nv) {
      st<T>(S.y, vbase + j, y[s]);
      st<T>(S.y_acc, vbase + j, yacc[s]);
      st<T>(S.dE_acc, vbase + j, dEacc[s]);
    }
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

// One launch: G threads per position.  STEP = false: Algorithm 3 at the
// points y (p x nv), directions to dE, dN, regularity to ok.  STEP = true:
// one projective step of every ACTIVE path of the state.
template <typename T, int G, int R, int CM, bool STEP>
__global__ void __launch_bounds__(kQrThreads)
qr_kernel(int n, int nv, int proj, int64_t p, const void* __restrict__ ext, const void* __restrict__ yin,
          void* __restrict__ dE, void* __restrict__ dN, int32_t* __restrict__ okout, hpt_paths S, hpt_params prm) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & (G - 1);
  const int64_t path = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int32_t status = path < p ? (STEP ? S.status[path] : HPT_PATH_ACTIVE) : -1;
  const bool valid = status == HPT_PATH_ACTIVE;
  if (!__any_sync(0xffffffffu, valid)) return;   // warp-uniform exit
  unsigned char* sm = smem + (threadIdx.x / G) * QrSmem<T, G, R, CM>::bytes;
  const size_t vbase = valid ? (size_t)path * nv : 0;
  cx<T> a[R][CM];
  const bool fin = qr_load<T, T, G, R, CM>(n, nv, proj, ext, path, STEP ? S.y : yin, vbase, valid, a);
  cx<T> wE[R], wN[R];
  const bool ok = qr_null<T, G, R, CM>(nv, a, wE, wN, sm) && fin;
  if (!valid) return;   // group-uniform; only group-masked shuffles below
  cx<T> xE[R], xN[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    const cx<T> yj = j < nv ? ld<T>(STEP ? S.y : yin, vbase + j) : mk<T>(0, 0);
    xE[s] = cmul(yj, wE[s]);
    xN[s] = cmul(yj, wN[s]);
  }
  if constexpr (STEP) {
    update_proj<T, G, R>(n, nv, path, vbase, status, ok, xE, xN, S, prm);
  } else {
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const int j = lane + G * s;
      if (j < nv) {
        st<T>(dE, vbase + j, xE[s]);
        st<T>(dN, vbase + j, xN[s]);
      }
    }
    if (lane == 0) okout[path] = ok ? 1 : 0;
  }
}

template <typename T>
__global__ void paths_init_proj_kernel(int n, int64_t p, const double2* __restrict__ x0, double tau0, double dtau0,
                                       hpt_paths S) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  const int nv = n + 1;
  double s2 = 1.0;
  for (int j = 0; j < n; ++j) {
    const double2 v = x0[(size_t)i * n + j];
    s2 += v.x * v.x + v.y * v.y;
  }
  const double inv = 1.0 / sqrt(s2);
  for (int j = 0; j < nv; ++j) {
    const double2 v = j < n ? x0[(size_t)i * n + j] : make_double2(1.0, 0.0);
    const cx<T> c = mk<T>((T)(v.x * inv), (T)(v.y * inv));
    st<T>(S.y, (size_t)i * nv + j, c);
    st<T>(S.y_acc, (size_t)i * nv + j, c);
    st<T>(S.dE_acc, (size_t)i * nv + j, mk<T>(0, 0));
  }
  S.tau[i] = tau0;
  S.tau_acc[i] = tau0;
  S.dtau[i] = dtau0;
  S.status[i] = HPT_PATH_ACTIVE;
  S.steps[i] = 0;
  S.accepts[i] = 0;
  S.rejects[i] = 0;
  S.streak[i] = 0;
}

template <typename T>
__global__ void finish_proj_kernel(int n, int64_t p, hpt_paths S, double2* __restrict__ x, int32_t* __restrict__ status_out,
                                   int32_t* __restrict__ steps_out, int32_t* __restrict__ done) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  const int nv = n + 1;
  const cx<T> h = ld<T>(S.y_acc, (size_t)i * nv + n);
  const double hx = (double)h.x, hy = (double)h.y, d = hx * hx + hy * hy;
  for (int j = 0; j < n; ++j) {
    const cx<T> v = ld<T>(S.y_acc, (size_t)i * nv + j);
    const double vx = (double)v.x, vy = (double)v.y;
    x[(size_t)i * n + j] = make_double2((vx * hx + vy * hy) / d, (vy * hx - vx * hy) / d);
  }
  const int32_t s = S.status[i];
  if (status_out) status_out[i] = s;
  if (steps_out) steps_out[i] = S.steps[i];
  done[i] = s == HPT_PATH_CONVERGED ? 0 : 3;
}

template <typename K>
cudaError_t qr_smem_attr(K kernel, int bytes) {
  return bytes > 48 * 1024 ? cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                           : cudaSuccess;
}

template <typename T, int G, int R, int CM, bool STEP>
cudaError_t launch_qr_shape(hpt_system s, int64_t p, const void* ext, const void* y, void* dE, void* dN,
                            int32_t* ok, const hpt_paths& S, const hpt_params& prm, cudaStream_t st) {
  const int smem = (kQrThreads / G) * QrSmem<T, G, R, CM>::bytes;
  cudaError_t e = qr_smem_attr(qr_kernel<T, G, R, CM, STEP>, smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (p * G + kQrThreads - 1) / kQrThreads;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  int pi = prof_begin(s, STEP ? "qr_step" : "qr_directions", st);
  qr_kernel<T, G, R, CM, STEP><<<(unsigned)blocks, kQrThreads, smem, st>>>(s->n, s->nv, s->proj, p, ext, y, dE, dN,
                                                                          ok, S, prm);
  prof_end(s, pi, st);
  return cudaGetLastError();
}

// Shapes by N = nv: (G, R, CM) = (8, 1, 10) for N <= 8, (8, 2, 18) for
// N <= 16, (8, 3, 26) for N <= 24 (FP32), (32, 1, 34) otherwise.
template <bool STEP>
cudaError_t launch_qr_any(hpt_system s, int64_t p, const void* ext, const void* y, void* dE, void* dN, int32_t* ok,
                          const hpt_paths& S, const hpt_params& prm, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const int N = s->nv;
  if (s->prec == HPT_FP64) {
    if (N <= 8) return launch_qr_shape<double, 8, 1, 10, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
    if (N <= 16) return launch_qr_shape<double, 8, 2, 18, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
    return launch_qr_shape<double, 32, 1, 34, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
  }
  if (N <= 8) return launch_qr_shape<float, 8, 1, 10, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
  if (N <= 16) return launch_qr_shape<float, 8, 2, 18, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
  if (N <= 24) return launch_qr_shape<float, 8, 3, 26, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
  return launch_qr_shape<float, 32, 1, 34, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
}

inline unsigned nblocks(int64_t threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

}  // namespace

cudaError_t launch_qr_directions(hpt_system s, int64_t p, const void* ext, const void* y, void* dE, void* dN,
                                 int32_t* ok, cudaStream_t st) {
  const hpt_paths none{};
  hpt_params prm{};
  return launch_qr_any<false>(s, p, ext, y, dE, dN, ok, none, prm, st);
}

cudaError_t launch_qr_step(hpt_system s, int64_t p, const void* ext, const hpt_paths& S, const hpt_params& prm,
                           cudaStream_t st) {
  return launch_qr_any<true>(s, p, ext, nullptr, nullptr, nullptr, nullptr, S, prm, st);
}

cudaError_t launch_paths_init_proj(hpt_system s, int64_t p, const void* x0, double tau0, const hpt_params& prm,
                                   const hpt_paths& S, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  if (s->prec == HPT_FP64)
    paths_init_proj_kernel<double><<<nblocks(p, 256), 256, 0, st>>>(s->n, p, (const double2*)x0, tau0, prm.dtau_init, S);
  else
    paths_init_proj_kernel<float><<<nblocks(p, 256), 256, 0, st>>>(s->n, p, (const double2*)x0, tau0, prm.dtau_init, S);
  return cudaGetLastError();
}

cudaError_t launch_finish_track_proj(hpt_system s, int64_t p, const hpt_paths& S, void* x_out, int32_t* status_out,
                                     int32_t* steps_out, int32_t* done, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  if (s->prec == HPT_FP64)
    finish_proj_kernel<double><<<nblocks(p, 256), 256, 0, st>>>(s->n, p, S, (double2*)x_out, status_out, steps_out, done);
  else
    finish_proj_kernel<float><<<nblocks(p, 256), 256, 0, st>>>(s->n, p, S, (double2*)x_out, status_out, steps_out, done);
  return cudaGetLastError();
}

}  // namespace hpt
