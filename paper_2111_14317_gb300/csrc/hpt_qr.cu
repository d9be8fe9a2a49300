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
// R rows in registers (row_in_slot), "shifted" so that register 0 is the
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
// round_up(C - k, 4) complex, C = N + 2 <= CM) and beta_k; padded so that
// consecutive groups start 8 banks apart.
constexpr int packed_entries(int CM) {
  int e = 0;
  for (int w = 3; w <= CM; ++w) e += (w + 3) / 4 * 4;   // widths C - k for N = CM - 2 rows
  return e;
}
template <typename T, int G, int R, int CM>
struct QrSmem {
  static constexpr int NR = G * R;
  static constexpr int entries = packed_entries(CM);
  static constexpr int raw_words = (entries * 2 * (int)sizeof(T) + NR * (int)sizeof(T)) / 4;
  static constexpr int words = (raw_words + 31) / 32 * 32 + 8;
  static constexpr int bytes = words * 4;
};

__device__ __forceinline__ int round4(int v) { return (v + 3) & ~3; }

// Two consecutive complex entries of a group's reflector storage (an even
// index: 16-byte aligned for complex64, one 16-byte load).
__device__ __forceinline__ void ld_pair(const cx<float>* U, int i, cx<float>& g0, cx<float>& g1) {
  const float4 v = *(const float4*)(U + i);
  g0 = mk<float>(v.x, v.y);
  g1 = mk<float>(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const cx<double>* U, int i, cx<double>& g0, cx<double>& g1) {
  g0 = U[i];
  g1 = U[i + 1];
}

// Row order.  The rows are factored in index order, and slot s of every lane
// holds a block of consecutive rows, so that whole slots finish early and are
// skipped (a warp-uniform test): the first r0 = N - G (R - 1) rows sit in the
// last slot (lanes 0 .. r0-1; the rest of that slot is zero padding), the next
// G in slot 0, then slot 1, ..  Returns the row of (slot s, lane) or N (padding).
template <int G, int R>
__device__ __forceinline__ int row_in_slot(int N, int s, int lane) {
  const int r0 = N - G * (R - 1);
  return s == R - 1 ? (lane < r0 ? lane : N) : r0 + G * s + lane;
}
// The largest row index of slot s (the slot is done once k passes it).
template <int G, int R>
__device__ __forceinline__ int slot_last_row(int N, int s) {
  const int r0 = N - G * (R - 1);
  return s == R - 1 ? r0 - 1 : r0 + G * s + G - 1;
}

// Loads the rows of one path (rows < n from the scratch, the y^* row in log
// coordinates if proj), scales each by a power of two; returns whether every
// entry is finite (group-uniform).
template <typename T, typename S, int G, int R, int CM>
__device__ __forceinline__ bool qr_load(int n, int nv, int proj, const void* __restrict__ ext, int64_t q,
                                        const void* __restrict__ y, size_t vbase, bool valid, cx<T> (&a)[R][CM]) {
  typedef typename cplx_t<S>::type V;
  const int lane = threadIdx.x & (G - 1);
  const int C = nv + 2;
  // entry (q, r, c) of the scratch sits at tile base + (r C + c) 128 (ext_index)
  const V* tile = (const V*)ext + ((size_t)(q >> 7) * (size_t)(nv * C)) * 128 + (size_t)(q & 127);
  // all loads first (independent, so they overlap), then the checks
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = row_in_slot<G, R>(nv, s, lane);
    const bool eq = valid && r < n;
    const bool ystar = valid && proj && r == n;
    const V* row = tile + (size_t)(eq ? r : 0) * C * 128;
#pragma unroll
    for (int c = 0; c < CM; ++c) {
      V v = V{0, 0};
      if (c < C && eq) v = row[(size_t)c * 128];
      if (c < nv && ystar) {
        const V w = ((const V*)y)[vbase + c];
        v.x = w.x * w.x + w.y * w.y;
        v.y = 0;
      }
      a[s][c] = mk<T>((T)v.x, (T)v.y);
    }
  }
  T chk = T(0);
#pragma unroll
  for (int s = 0; s < R; ++s) {
    T m = T(0);
#pragma unroll
    for (int c = 0; c < CM; ++c) {
      chk += t_abs(a[s][c].x) + t_abs(a[s][c].y);
      m = t_max(m, cmag(a[s][c]));
    }
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
  int rowi[R];
#pragma unroll
  for (int s = 0; s < R; ++s) rowi[s] = row_in_slot<G, R>(N, s, lane);
  const int r0 = N - G * (R - 1);
  bool ok = true;
  int off = 0;   // packed offset of row k's reflector
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    const int width = C - k, len = round4(width);
    const int ol = k < r0 ? k : (k - r0) & (G - 1), os = k < r0 ? R - 1 : (k - r0) / G;
    // the owner forms the reflector of row k from its registers (os is
    // warp-uniform, so one copy runs): sigma = |live part|, g = r +
    // e^{i arg r_0} sigma e_0 (phase 1 when r_0 = 0), beta = 1 / (sigma (sigma
    // + |r_0|)); it stores g (zero-padded to len) and beta for the group
    if (lane == ol) {
#pragma unroll
      for (int s = 0; s < R; ++s) {
        if (s == os) {
          T s2 = T(0);
#pragma unroll
          for (int c = 0; c < CM; ++c)
            if (c < width) s2 += abs2(a[s][c]);
          const cx<T> r0v = a[s][0];
          const T sigma = t_sqrt(s2), m0 = t_sqrt(abs2(r0v));
          const T im0 = t_rcp(m0);   // m0 flushed to zero: any unit phase will do
          const cx<T> ph = (m0 > T(0) && isfinite(im0)) ? cscale(r0v, sigma * im0) : mk<T>(sigma, T(0));
          beta[k] = sigma > T(0) ? t_rcp(sigma * (sigma + m0)) : T(0);
          U[off] = mk<T>(r0v.x + ph.x, r0v.y + ph.y);
#pragma unroll
          for (int c = 1; c < CM; ++c)
            if (c < len) U[off + c] = c < width ? a[s][c] : mk<T>(0, 0);
        }
      }
    }
    __syncwarp();
    const T b = beta[k];
    if (!(b > T(0)) || !isfinite(b)) ok = false;
    // per slot whose rows are not all done (a warp-uniform test): t = beta
    // <row, g> over the live width (two partial sums, even and odd columns,
    // for independent chains; rows up to k get t = 0), then the shifted
    // update a[c-1] = a[c] - t g[c] (column k leaves the rows: it is L's)
#pragma unroll
    for (int s = 0; s < R; ++s) {
      if (slot_last_row<G, R>(N, s) > k) {
        cx<T> t0 = mk<T>(0, 0), t1 = mk<T>(0, 0);
#pragma unroll
        for (int c0 = 0; c0 < CM; c0 += 4) {
          if (c0 < width) {
#pragma unroll
            for (int c = c0; c < c0 + 4 && c < CM; c += 2) {
              cx<T> g0, g1;
              ld_pair(U, off + c, g0, g1);
              t0.x += a[s][c].x * g0.x + a[s][c].y * g0.y;
              t0.y += a[s][c].y * g0.x - a[s][c].x * g0.y;
              if (c + 1 < CM) {
                t1.x += a[s][c + 1].x * g1.x + a[s][c + 1].y * g1.y;
                t1.y += a[s][c + 1].y * g1.x - a[s][c + 1].x * g1.y;
              }
            }
          }
        }
        const cx<T> ts = rowi[s] <= k ? mk<T>(0, 0) : cscale(mk<T>(t0.x + t1.x, t0.y + t1.y), b);
#pragma unroll
        for (int c0 = 0; c0 < CM; c0 += 4) {
          if (c0 < width) {
#pragma unroll
            for (int c = c0; c < c0 + 4 && c < CM; c += 2) {
              cx<T> g0, g1;
              ld_pair(U, off + c, g0, g1);
              if (c >= 1) a[s][c - 1] = csub_mul(a[s][c], ts, g0);
              if (c + 1 < CM) a[s][c] = csub_mul(a[s][c + 1], ts, g1);
            }
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
// directions in y coordinates: the affine rule (and predictor choice) with
// the point scaled back to unit norm after every correction and divergence
// tested on y_j / y_n.
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
      ny = t_max(ny, t_sqrt(abs2(y[s])));   // unit-norm points, small corrections: no overflow
      nd = t_max(nd, t_sqrt(abs2(xN[s])));
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
  const bool herm = prm.predictor == 1;
  bool predict = true, keep_prev = false, retry = false;
  cx<T> yp[R], dp[R];   // the accepted point before the last one (Hermite predictor)
  double taup = 0.0;
  if (accept) {
    keep_prev = herm && accepts >= 1;
    cx<T> w[R];
#pragma unroll
    for (int s = 0; s < R; ++s) w[s] = mk<T>(y[s].x + xN[s].x, y[s].y + xN[s].y);
    const T inv = unit(w);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      yp[s] = yacc[s];
      dp[s] = dEacc[s];
      yacc[s] = cscale(w[s], inv);
      dEacc[s] = cscale(xE[s], inv);
    }
    taup = tauacc;
    tauacc = tau;
    accepts += 1;
    streak += 1;
    // |y_n| from its lane, then the dehomogenized magnitudes |y_j / y_n|
    cx<T> vh = yacc[0];
#pragma unroll
    for (int s = 1; s < R; ++s)
      if (s == n / G) vh = yacc[s];
    const T mh = __shfl_sync(gmask, t_sqrt(abs2(vh)), n & (G - 1), G);
    bool div = false;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      if (lane + G * s < n) {
        const T m = t_sqrt(abs2(yacc[s])) / mh;
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
          const bool mine = lane + G * s < nv;
          yp[s] = mine ? ld<T>(S.y_prev, vbase + lane + G * s) : mk<T>(0, 0);
          dp[s] = mine ? ld<T>(S.dE_prev, vbase + lane + G * s) : mk<T>(0, 0);
        }
        taup = S.tau_prev[path];
      }
      cubic = tauacc - taup > 0.0;
    }
    if (cubic) {
      // the previous point turned into the phase of the last (y_acc^* y_prev
      // real and positive): the corrector leaves a homogeneous point's phase
      // free, and the extrapolation would amplify phase differences
      cx<T> dot = mk<T>(0, 0);
#pragma unroll
      for (int s = 0; s < R; ++s) {
        dot.x += yacc[s].x * yp[s].x + yacc[s].y * yp[s].y;
        dot.y += yacc[s].x * yp[s].y - yacc[s].y * yp[s].x;
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        dot.x += __shfl_xor_sync(gmask, dot.x, o, G);
        dot.y += __shfl_xor_sync(gmask, dot.y, o, G);
      }
      const T md = t_sqrt(abs2(dot));
      const cx<T> ph = md > T(0) ? mk<T>(dot.x / md, -dot.y / md) : mk<T>(T(1), T(0));
      // cubic Hermite through (taup, yp, dp) and (tauacc, yacc, dEacc) at tauacc + h
      const double d = tauacc - taup, u = 1.0 + h / d, u2 = u * u, u3 = u2 * u;
      const T h00 = (T)(2 * u3 - 3 * u2 + 1), h10 = (T)((u3 - 2 * u2 + u) * d);
      const T h01 = (T)(-2 * u3 + 3 * u2), h11 = (T)((u3 - u2) * d);
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const cx<T> a0 = cmul(yp[s], ph), a1 = cmul(dp[s], ph);
        y[s] = mk<T>(h00 * a0.x + h10 * a1.x + h01 * yacc[s].x + h11 * dEacc[s].x,
                     h00 * a0.y + h10 * a1.y + h01 * yacc[s].y + h11 * dEacc[s].y);
      }
    } else {
#pragma unroll
      for (int s = 0; s < R; ++s) y[s] = mk<T>(yacc[s].x + (T)h * dEacc[s].x, yacc[s].y + (T)h * dEacc[s].y);
    }
    tau = tauacc + h;
    if (steps >= prm.max_steps) status = HPT_PATH_MAX_STEPS;
    if (herm && lane == 0) S.hermite[path] = cubic ? 1 : 0;
  }
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = lane + G * s;
    if (j < nv) {
      st<T>(S.y, vbase + j, y[s]);
      st<T>(S.y_acc, vbase + j, yacc[s]);
      st<T>(S.dE_acc, vbase + j, dEacc[s]);
      if (keep_prev) {
        st<T>(S.y_prev, vbase + j, yp[s]);
        st<T>(S.dE_prev, vbase + j, dp[s]);
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

// One launch: G threads per position.  STEP = false: Algorithm 3 at the
// points y (p x nv), directions to dE, dN, regularity to ok.  STEP = true:
// one projective step of every ACTIVE path of the state.
template <typename T, int G, int R, int CM, bool STEP>
__global__ void __launch_bounds__(kQrThreads, (sizeof(T) == 4 && R == 3 && CM == 20) ? 3 : 1)
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
    if (S.y_prev) {
      st<T>(S.y_prev, (size_t)i * nv + j, mk<T>(0, 0));
      st<T>(S.dE_prev, (size_t)i * nv + j, mk<T>(0, 0));
    }
  }
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

// Shapes by N = nv (CM >= N + 2 columns in registers): (G, R, CM) =
// (8, 1, 10) for N <= 8, (8, 2, 18) for N <= 16; FP32: (8, 3, 20) for N <= 18,
// (8, 3, 26) for N <= 24, (32, 1, 34) above; FP64 (whose rows take twice the
// registers): (16, 2, 20), (32, 1, 26), (32, 1, 34).
template <bool STEP>
cudaError_t launch_qr_any(hpt_system s, int64_t p, const void* ext, const void* y, void* dE, void* dN, int32_t* ok,
                          const hpt_paths& S, const hpt_params& prm, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const int N = s->nv;
  if (s->prec == HPT_FP64) {
    if (N <= 8) return launch_qr_shape<double, 8, 1, 10, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
    if (N <= 16) return launch_qr_shape<double, 8, 2, 18, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
    if (N <= 18) return launch_qr_shape<double, 16, 2, 20, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
    if (N <= 24) return launch_qr_shape<double, 32, 1, 26, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
    return launch_qr_shape<double, 32, 1, 34, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
  }
  if (N <= 8) return launch_qr_shape<float, 8, 1, 10, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
  if (N <= 16) return launch_qr_shape<float, 8, 2, 18, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
  if (N <= 18) return launch_qr_shape<float, 8, 3, 20, STEP>(s, p, ext, y, dE, dN, ok, S, prm, st);
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
