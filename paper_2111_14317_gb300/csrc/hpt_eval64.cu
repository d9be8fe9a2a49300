// FP64 evaluation of the homotopy and its extended Jacobian (Algorithm 2,
// Section 5) on the CUDA cores.
//
// For every point: z = log y (eq. (6)); for every monomial W = <z, a> +
// tau e/D (one row of Z A, eq. (7)); E = exp(W); the extended Jacobian row of
// equation k is sum_i E_i B_k[:, i] = [D_z h_k | D_tau h_k | h_k] (eq. (8) and
// the extended-Jacobian identity), and D_y h_k = D_z h_k diag(e^{-z}).
//
// The same kernel serves the projective form (Section 2.2): n equations in nv
// = n + 1 homogeneous coordinates, exponents (a, deg_k - 1^T a); the extended
// Jacobian row is then [D_z h_k (nv entries) | D_tau h_k | h_k].
//
// Mapping: a block owns 32 points (one per lane) and its four warps take the
// equations k = warp, warp + 4, ...; all lanes of a warp read the same
// monomial constants (broadcast), z is staged in shared memory transposed so
// that lane q reads column q without bank conflicts.
#include <math.h>

#include "hpt_internal.h"

namespace hpt {
namespace {

// MAP: 32 consecutive positions of a position map per block (inside one
// 128-position tile, so one system: S from the per-system table); otherwise
// positions are the paths of the single system S.  NMAX bounds the variables.
template <int NMAX, bool MAP>
__global__ void __launch_bounds__(128)
eval_fp64_kernel(Fp64Sys S, int64_t p, const double2* __restrict__ y, const double* __restrict__ tin,
                 int tau_is_t, double2* __restrict__ ext, double2* __restrict__ oH, double2* __restrict__ oHy,
                 double2* __restrict__ oHt, PathMap pm, const Fp64Sys* __restrict__ tab) {
  __shared__ double2 zs[NMAX][32];
  __shared__ double2 iys[NMAX][32];
  __shared__ double taus[32];
  __shared__ double tinv[32];
  __shared__ int64_t spath[32];
  int64_t base = (int64_t)blockIdx.x * 32;
  int nmax = S.nv;
  if (MAP) {
    base += *pm.pos_begin;
    if (base >= *pm.npos) return;
    S = tab[pm.tile_sys[base >> 7]];
    nmax = pm.nmax;
  }
  const int n = S.n, nv = S.nv;
  const int32_t* __restrict__ msz = S.msz;
  const int32_t* __restrict__ off = S.off;
  const double* __restrict__ ahat = S.ahat;
  const double2* __restrict__ bcol = S.b;
  if (threadIdx.x < 32) {
    const int64_t q = base + threadIdx.x;
    spath[threadIdx.x] = MAP ? pm.list[q] : (q < p ? q : -1);
  }
  __syncthreads();

  // op. 1 of Algorithm 2: Z <- log Y (principal branch), and 1/y for the
  // final diag(e^{-z}) scaling.
  for (int idx = threadIdx.x; idx < 32 * nv; idx += blockDim.x) {
    const int q = idx / nv, j = idx - q * nv;
    const int64_t path = spath[q];
    double2 v = make_double2(1.0, 0.0);
    if (path >= 0) v = y[(MAP ? (size_t)pm.vofs[path] : (size_t)path * nv) + j];
    const double r2 = v.x * v.x + v.y * v.y;
    zs[j][q] = make_double2(log(hypot(v.x, v.y)), atan2(v.y, v.x));
    iys[j][q] = make_double2(v.x / r2, -v.y / r2);
  }
  if (threadIdx.x < 32) {
    const int64_t path = spath[threadIdx.x];
    double tv = (path >= 0 && tin) ? tin[path] : (tau_is_t ? 1.0 : 0.0);   // no tin: t = 1
    double tau = tau_is_t ? log(tv) : tv;
    taus[threadIdx.x] = tau;
    tinv[threadIdx.x] = tau_is_t ? 1.0 / tv : exp(-tau);
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t path = spath[lane];
  const int64_t pos = base + lane;
  const double tau = taus[lane];
  const int np2 = nv + 2;
  for (int k = warp; k < n; k += 4) {
    double2 accJ[NMAX];
#pragma unroll
    for (int u = 0; u < NMAX; ++u) accJ[u] = make_double2(0.0, 0.0);
    double2 accT = make_double2(0.0, 0.0), accH = make_double2(0.0, 0.0);
    const int i0 = off[k], i1 = off[k] + msz[k];
    for (int i = i0; i < i1; ++i) {
      // op. 2 of Algorithm 2, one monomial: W = [z, tau] . A[:, i]
      const double* a = ahat + (size_t)i * (nv + 1);
      double wr = a[nv] * tau, wi = 0.0;
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        if (j < nv) {
          const double aj = a[j];
          const double2 z = zs[j][lane];
          wr = fma(aj, z.x, wr);
          wi = fma(aj, z.y, wi);
        }
      }
      double sn, cs;
      sincos(wi, &sn, &cs);
      const double mag = exp(wr);
      const double er = mag * cs, ei = mag * sn;
      // ... times B_k[:, i] (complex), accumulated over the equation's monomials
      const double2* bb = bcol + (size_t)i * np2;
#pragma unroll
      for (int u = 0; u < NMAX; ++u) {
        if (u < nv) {
          const double2 c = bb[u];
          accJ[u].x = fma(er, c.x, fma(-ei, c.y, accJ[u].x));
          accJ[u].y = fma(er, c.y, fma(ei, c.x, accJ[u].y));
        }
      }
      const double2 ct = bb[nv], ch = bb[nv + 1];
      accT.x = fma(er, ct.x, fma(-ei, ct.y, accT.x));
      accT.y = fma(er, ct.y, fma(ei, ct.x, accT.y));
      accH.x = fma(er, ch.x, fma(-ei, ch.y, accH.x));
      accH.y = fma(er, ch.y, fma(ei, ch.x, accH.y));
    }
    if (path < 0) continue;
    // the step scratch keeps D_z h_k: op. 3 of Algorithm 2 (the diag(e^{-z})
    // scaling) is applied by the solve to its n-vector solutions instead of
    // to the n x n block here
    if (ext) {
#pragma unroll
      for (int u = 0; u < NMAX; ++u)
        if (u < nv) ext[ext_index(pos, k, u, nmax)] = accJ[u];
      ext[ext_index(pos, k, nv, nmax)] = accT;
      ext[ext_index(pos, k, nv + 1, nmax)] = accH;
    }
    // op. 3 of Algorithm 2 for the caller's H_y: D_y h_k = D_z h_k diag(e^{-z})
    if (oHy) {
      double2* row = oHy + ((size_t)path * n + k) * nv;
#pragma unroll
      for (int u = 0; u < NMAX; ++u) {
        if (u < nv) {
          const double2 iy = iys[u][lane];
          row[u] = make_double2(accJ[u].x * iy.x - accJ[u].y * iy.y, accJ[u].x * iy.y + accJ[u].y * iy.x);
        }
      }
    }
    if (oH) oH[(size_t)path * n + k] = accH;
    if (oHt) {
      const double ti = tinv[lane];   // dH/dt = (dH/dtau) / t
      oHt[(size_t)path * n + k] = make_double2(accT.x * ti, accT.y * ti);
    }
  }
}

}  // namespace

Fp64Sys fp64_sys_of(const hpt_system s) {
  Fp64Sys f;
  f.n = s->n;
  f.nv = s->nv;
  f.msz = s->d_msz;
  f.off = s->d_off;
  f.ahat = s->d_ahat;
  f.b = (const double2*)s->d_b;
  return f;
}

cudaError_t launch_eval_fp64(hpt_system s, int64_t p, const void* y, const double* tau,
                             int tau_is_t, const EvalOut& out, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const int64_t blocks = (p + 31) / 32;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  int pi = prof_begin(s, "eval_fp64", st);
  const double2* yy = (const double2*)y;
  double2* ext = (double2*)out.ext;
  double2* H = (double2*)out.H;
  double2* Hy = (double2*)out.Hy;
  double2* Ht = (double2*)out.Ht;
  const Fp64Sys f = fp64_sys_of(s);
  const PathMap none;
  if (s->nv <= 8)
    eval_fp64_kernel<8, false><<<(unsigned)blocks, 128, 0, st>>>(f, p, yy, tau, tau_is_t, ext, H, Hy, Ht, none, nullptr);
  else if (s->nv <= 16)
    eval_fp64_kernel<16, false><<<(unsigned)blocks, 128, 0, st>>>(f, p, yy, tau, tau_is_t, ext, H, Hy, Ht, none, nullptr);
  else if (s->nv <= 24)
    eval_fp64_kernel<24, false><<<(unsigned)blocks, 128, 0, st>>>(f, p, yy, tau, tau_is_t, ext, H, Hy, Ht, none, nullptr);
  else
    eval_fp64_kernel<32, false><<<(unsigned)blocks, 128, 0, st>>>(f, p, yy, tau, tau_is_t, ext, H, Hy, Ht, none, nullptr);
  prof_end(s, pi, st);
  return cudaGetLastError();
}

cudaError_t launch_eval_fp64_map(int shape, const Fp64Sys* tab, int64_t cap, const void* y, const double* tau,
                                 const PathMap& pm, void* ext, cudaStream_t st) {
  if (cap <= 0) return cudaSuccess;
  if (!pm.list || !pm.tile_sys || !pm.vofs || !pm.npos || !pm.pos_begin || !tab) return cudaErrorInvalidValue;
  const int64_t blocks = (cap + 31) / 32;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  const Fp64Sys f{};
  const double2* yy = (const double2*)y;
  double2* e = (double2*)ext;
  if (shape == 0)
    eval_fp64_kernel<8, true><<<(unsigned)blocks, 128, 0, st>>>(f, cap, yy, tau, 0, e, nullptr, nullptr, nullptr, pm, tab);
  else if (shape == 1)
    eval_fp64_kernel<16, true><<<(unsigned)blocks, 128, 0, st>>>(f, cap, yy, tau, 0, e, nullptr, nullptr, nullptr, pm, tab);
  else if (shape == kEval24)
    eval_fp64_kernel<24, true><<<(unsigned)blocks, 128, 0, st>>>(f, cap, yy, tau, 0, e, nullptr, nullptr, nullptr, pm, tab);
  else
    eval_fp64_kernel<32, true><<<(unsigned)blocks, 128, 0, st>>>(f, cap, yy, tau, 0, e, nullptr, nullptr, nullptr, pm, tab);
  return cudaGetLastError();
}

}  // namespace hpt
