// Host side of libhpt: exact integer bookkeeping of the cell, constant images
// of Algorithm 1 (Initialize), handle lifetime, scratch, errors, profiling.
#include <cuda_bf16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hpt_internal.h"

namespace hpt {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// ------------------------------------------------------------ exact rationals
typedef __int128 i128;
static const i128 kLim = ((i128)1) << 62;   // every stored value stays below

static i128 iabs(i128 v) { return v < 0 ? -v : v; }
static i128 igcd(i128 a, i128 b) {
  a = iabs(a);
  b = iabs(b);
  while (b) { i128 t = a % b; a = b; b = t; }
  return a;
}

struct Rat {
  i128 num = 0, den = 1;
};

static bool norm(Rat& r) {
  if (r.den < 0) { r.num = -r.num; r.den = -r.den; }
  i128 g = igcd(r.num, r.den);
  if (g > 1) { r.num /= g; r.den /= g; }
  if (r.num == 0) r.den = 1;
  return iabs(r.num) < kLim && r.den < kLim;
}
static bool rmul(const Rat& a, const Rat& b, Rat& out) {
  // reduce crosswise first so the products stay small
  i128 g1 = igcd(a.num, b.den), g2 = igcd(b.num, a.den);
  if (g1 == 0) g1 = 1;
  if (g2 == 0) g2 = 1;
  out.num = (a.num / g1) * (b.num / g2);
  out.den = (a.den / g2) * (b.den / g1);
  return norm(out);
}
static bool rsub(const Rat& a, const Rat& b, Rat& out) {
  i128 g = igcd(a.den, b.den);
  i128 l = a.den / g * b.den;
  if (iabs(l) >= kLim) return false;
  out.num = a.num * (l / a.den) - b.num * (l / b.den);
  out.den = l;
  return norm(out);
}
static bool rdiv(const Rat& a, const Rat& b, Rat& out) {
  Rat inv;
  inv.num = b.den;
  inv.den = b.num;
  if (!norm(inv)) return false;
  return rmul(a, inv, out);
}

// ------------------------------------------------------------ modular determinant
// Exact nonsingularity test of an integer matrix: det V is computed modulo
// primes below 2^62 until their product exceeds Hadamard's bound prod_k
// |row_k|_2 >= |det V|; then det V = 0 exactly when every residue is 0.
typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1;
  for (a %= p; e; e >>= 1, a = mulmod(a, a, p))
    if (e & 1) r = mulmod(r, a, p);
  return r;
}
// Miller-Rabin with the first twelve primes as bases: exact below 3.3e24.
static bool is_prime64(uint64_t n) {
  static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (uint64_t b : bases)
    if (n % b == 0) return n == b;
  uint64_t d = n - 1;
  int r = 0;
  while (!(d & 1)) { d >>= 1; ++r; }
  for (uint64_t b : bases) {
    uint64_t x = powmod(b, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < r && comp; ++i) {
      x = mulmod(x, x, n);
      if (x == n - 1) comp = false;
    }
    if (comp) return false;
  }
  return true;
}
static uint64_t det_mod(int n, const std::vector<int64_t>& V, uint64_t p) {
  std::vector<uint64_t> A((size_t)n * n);
  for (int i = 0; i < n * n; ++i) {
    const int64_t v = V[i] % (int64_t)p;
    A[i] = (uint64_t)(v < 0 ? v + (int64_t)p : v);
  }
  uint64_t det = 1;
  for (int j = 0; j < n; ++j) {
    int piv = -1;
    for (int i = j; i < n && piv < 0; ++i)
      if (A[i * n + j]) piv = i;
    if (piv < 0) return 0;
    if (piv != j) {
      for (int c = 0; c < n; ++c) std::swap(A[piv * n + c], A[j * n + c]);
      det = (p - det) % p;
    }
    det = mulmod(det, A[j * n + j], p);
    const uint64_t inv = powmod(A[j * n + j], p - 2, p);
    for (int i = j + 1; i < n; ++i) {
      const uint64_t f = mulmod(A[i * n + j], inv, p);
      if (!f) continue;
      for (int c = j; c < n; ++c) A[i * n + c] = (A[i * n + c] + p - mulmod(f, A[j * n + c], p)) % p;
    }
  }
  return det;
}
// HPT_OK (nonsingular), HPT_ENOTCELL (singular).
static hpt_status nonsingular_exact(int n, const std::vector<int64_t>& V) {
  double log2_bound = 1.0;
  for (int k = 0; k < n; ++k) {
    double r2 = 0;
    for (int j = 0; j < n; ++j) r2 += (double)V[k * n + j] * (double)V[k * n + j];
    if (r2 == 0) return HPT_ENOTCELL;
    log2_bound += 0.5 * log2(r2);
  }
  double covered = 0;
  for (uint64_t cand = ((uint64_t)1 << 62) - 1; covered <= log2_bound; cand -= 2) {
    if (!is_prime64(cand)) continue;
    if (det_mod(n, V, cand) != 0) return HPT_OK;
    covered += log2((double)cand);
  }
  return HPT_ENOTCELL;
}

// Solves V x = rhs exactly (Gauss-Jordan over the rationals).  Returns
// HPT_OK, HPT_ENOTCELL (singular) or HPT_ERANGE.
static hpt_status solve_exact(int n, const std::vector<int64_t>& V, const std::vector<int64_t>& rhs,
                              std::vector<Rat>& x) {
  std::vector<Rat> A((size_t)n * (n + 1));
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) A[i * (n + 1) + j].num = V[i * n + j];
    A[i * (n + 1) + n].num = rhs[i];
  }
  for (int j = 0; j < n; ++j) {
    int piv = -1;
    for (int i = j; i < n; ++i)
      if (A[i * (n + 1) + j].num != 0) { piv = i; break; }
    if (piv < 0) return HPT_ENOTCELL;
    if (piv != j)
      for (int c = 0; c <= n; ++c) std::swap(A[j * (n + 1) + c], A[piv * (n + 1) + c]);
    for (int i = 0; i < n; ++i) {
      if (i == j || A[i * (n + 1) + j].num == 0) continue;
      Rat f;
      if (!rdiv(A[i * (n + 1) + j], A[j * (n + 1) + j], f)) return HPT_ERANGE;
      for (int c = j; c <= n; ++c) {
        Rat t;
        if (!rmul(f, A[j * (n + 1) + c], t)) return HPT_ERANGE;
        if (!rsub(A[i * (n + 1) + c], t, A[i * (n + 1) + c])) return HPT_ERANGE;
      }
    }
  }
  x.resize(n);
  for (int i = 0; i < n; ++i)
    if (!rdiv(A[i * (n + 1) + n], A[i * (n + 1) + i], x[i])) return HPT_ERANGE;
  return HPT_OK;
}

struct Lifted {
  std::vector<int64_t> e, alpha, beta;
  int64_t D = 1;
};

static hpt_status check_shape(int32_t n, const int32_t* msz, int32_t* M_out) {
  if (n < 1 || n > kMaxN) { set_error("n=%d outside [1,%d]", n, kMaxN); return HPT_EINVAL; }
  if (!msz) { set_error("support_sizes is NULL"); return HPT_EINVAL; }
  int64_t M = 0;
  for (int k = 0; k < n; ++k) {
    if (msz[k] < 1 || msz[k] > 4096) { set_error("m_%d=%d outside [1,4096]", k, msz[k]); return HPT_EINVAL; }
    M += msz[k];
  }
  if (M > (1 << 20)) { set_error("too many monomials"); return HPT_EINVAL; }
  *M_out = (int32_t)M;
  return HPT_OK;
}

static hpt_status lift(int32_t n, const int32_t* msz, const int32_t* exps, const int64_t* lifting,
                       const hpt_cell* cell, Lifted& L) {
  int32_t M;
  hpt_status rc = check_shape(n, msz, &M);
  if (rc) return rc;
  if (!exps || !lifting || !cell) { set_error("NULL exponents, lifting or cell"); return HPT_EINVAL; }
  std::vector<int32_t> off(n);
  for (int k = 0, acc = 0; k < n; ++k) { off[k] = acc; acc += msz[k]; }
  for (int64_t i = 0; i < (int64_t)M * n; ++i)
    if (exps[i] < -(1 << 20) || exps[i] > (1 << 20)) { set_error("exponent too large"); return HPT_ERANGE; }
  for (int i = 0; i < M; ++i)
    if (lifting[i] < -(1LL << 40) || lifting[i] > (1LL << 40)) { set_error("lifting too large"); return HPT_ERANGE; }
  L.alpha.assign(n, 0);
  L.beta.assign(n, 0);
  std::vector<int> p0(n, -1), p1(n, -1);
  if (cell->kind == HPT_CELL_PAIRS) {
    if (!cell->pairs) { set_error("cell.pairs is NULL"); return HPT_EINVAL; }
    std::vector<int64_t> V((size_t)n * n), rhs(n);
    for (int k = 0; k < n; ++k) {
      p0[k] = cell->pairs[2 * k];
      p1[k] = cell->pairs[2 * k + 1];
      if (p0[k] < 0 || p1[k] < 0 || p0[k] >= msz[k] || p1[k] >= msz[k] || p0[k] == p1[k]) {
        set_error("bad pair for equation %d", k);
        return HPT_EINVAL;
      }
      const int32_t* a0 = exps + (size_t)(off[k] + p0[k]) * n;
      const int32_t* a1 = exps + (size_t)(off[k] + p1[k]) * n;
      for (int j = 0; j < n; ++j) V[k * n + j] = (int64_t)a1[j] - a0[j];
      rhs[k] = lifting[off[k] + p0[k]] - lifting[off[k] + p1[k]];
    }
    std::vector<Rat> alpha;
    bool zero_rhs = true;
    for (int k = 0; k < n; ++k) zero_rhs = zero_rhs && rhs[k] == 0;
    if (zero_rhs) {
      // equal lifting values on every pair: the inner normal is 0 whatever
      // the size of V, and only its nonsingularity needs checking
      rc = nonsingular_exact(n, V);
      alpha.assign(n, Rat());
    } else {
      rc = solve_exact(n, V, rhs, alpha);
    }
    if (rc == HPT_ENOTCELL) { set_error("pair matrix is singular"); return rc; }
    if (rc) { set_error("overflow solving for alpha"); return rc; }
    i128 D = 1;
    for (int j = 0; j < n; ++j) {
      i128 g = igcd(D, alpha[j].den);
      D = D / g * alpha[j].den;
      if (D >= kLim) { set_error("denominator overflow"); return HPT_ERANGE; }
    }
    L.D = (int64_t)D;
    for (int j = 0; j < n; ++j) {
      i128 v = alpha[j].num * (D / alpha[j].den);
      if (iabs(v) >= kLim) { set_error("alpha overflow"); return HPT_ERANGE; }
      L.alpha[j] = (int64_t)v;
    }
    for (int k = 0; k < n; ++k) {
      const int32_t* a0 = exps + (size_t)(off[k] + p0[k]) * n;
      i128 b = (i128)L.D * lifting[off[k] + p0[k]];
      for (int j = 0; j < n; ++j) b += (i128)a0[j] * L.alpha[j];
      if (iabs(b) >= kLim) { set_error("beta overflow"); return HPT_ERANGE; }
      L.beta[k] = (int64_t)b;
    }
  } else if (cell->kind == HPT_CELL_EXPLICIT || cell->kind == HPT_CELL_LOWER) {
    if (!cell->alpha_num || (cell->kind == HPT_CELL_EXPLICIT && !cell->beta_num)) {
      set_error("cell.alpha_num / beta_num is NULL");
      return HPT_EINVAL;
    }
    if (cell->denom < 1 || cell->denom >= (int64_t)kLim) { set_error("cell.denom must be >= 1"); return HPT_EINVAL; }
    L.D = cell->denom;
    for (int j = 0; j < n; ++j) {
      if (cell->alpha_num[j] <= -(1LL << 40) || cell->alpha_num[j] >= (1LL << 40)) {
        set_error("alpha too large");
        return HPT_ERANGE;
      }
      L.alpha[j] = cell->alpha_num[j];
    }
    for (int k = 0; k < n; ++k) {
      if (cell->kind == HPT_CELL_EXPLICIT) {
        L.beta[k] = cell->beta_num[k];
        continue;
      }
      i128 best = 0;
      for (int i = 0; i < msz[k]; ++i) {
        const int32_t* a = exps + (size_t)(off[k] + i) * n;
        i128 v = (i128)L.D * lifting[off[k] + i];
        for (int j = 0; j < n; ++j) v += (i128)a[j] * L.alpha[j];
        if (i == 0 || v < best) best = v;
      }
      if (iabs(best) >= kLim) { set_error("beta overflow"); return HPT_ERANGE; }
      L.beta[k] = (int64_t)best;
    }
  } else {
    set_error("unknown cell kind %d", cell->kind);
    return HPT_EINVAL;
  }
  L.e.assign(M, 0);
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < msz[k]; ++i) {
      const int32_t* a = exps + (size_t)(off[k] + i) * n;
      i128 v = (i128)L.D * lifting[off[k] + i] - L.beta[k];
      for (int j = 0; j < n; ++j) v += (i128)a[j] * L.alpha[j];
      if (iabs(v) >= kLim) { set_error("t-exponent overflow"); return HPT_ERANGE; }
      L.e[off[k] + i] = (int64_t)v;
      const bool on_pair = (cell->kind == HPT_CELL_PAIRS) && (i == p0[k] || i == p1[k]);
      if (on_pair && v != 0) { set_error("internal: pair off its facet"); return HPT_ENOTCELL; }
      if (!on_pair && v < 0) { set_error("monomial %d of equation %d lies below the cell", i, k); return HPT_ENOTCELL; }
      if (cell->kind == HPT_CELL_PAIRS && !on_pair && v == 0) {
        set_error("lifting not generic: monomial %d of equation %d on the cell's facet", i, k);
        return HPT_ENOTCELL;
      }
    }
  }
  return HPT_OK;
}

// ------------------------------------------------------------ bf16 (host)
// Round-to-nearest-even of an IEEE binary32 to its upper 16 bits.
static uint16_t bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
static float bf16_value(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}
static void split2(double v, uint16_t& hi, uint16_t& lo) {
  hi = bf16_bits((float)v);
  lo = bf16_bits((float)(v - (double)bf16_value(hi)));
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

static MixedLayout mixed_layout(int n, int max_m, bool big, bool affine) {
  MixedLayout L;
  L.MP = round_up(max_m, 16);
  L.KX = round_up(3 * n, 16);
  L.NJ = round_up(2 * (n + 2), 16);
  L.KC = 2 * L.MP;
  // exponent part (operand, t-exponents, and for large exponents the mask
  // and int16 exponent vectors) first, coefficient part after, each starting
  // on a 128-byte boundary, so that the evaluation can copy them separately
  L.off_bexp = 0;
  L.off_texp = L.MP * L.KX * 2;
  int end = L.off_texp + L.MP * 4;
  if (big) {
    L.off_bigm = round_up(end, 16);
    L.off_aint = round_up(L.off_bigm + L.MP / 8, 16);   // MP / 32 words
    end = L.off_aint + L.MP * n * 2;
  }
  L.off_bhi = round_up(end, 128);
  L.off_blo = L.off_bhi + L.NJ * L.KC * 2;
  L.chunk_bytes = round_up(L.off_blo + L.NJ * L.KC * 2, 128);
  L.grouped = affine && j_grouped(L.MP, L.NJ);
  int cols = 4 * L.MP + (L.grouped ? 3 : 1) * L.NJ, t = 32;   // two exponent accumulators (Re, Im each) and J
  while (t < cols) t *= 2;
  L.tmem_cols = t;
  return L;
}

// Uploads the device constants of s: the FP64 form (A_hat columns (a; e/D)
// and B_k columns [c a; c e/D; c], eq. (8)) and, for HPT_MIXED, the
// split-BF16 operand images.  ex holds M exponent vectors of s->nv entries
// (the system's own, or the homogenized ones of the projective form); the
// n equations come from s->msz / s->off.
#define CUU(call)                                                             \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));              \
      return e_ == cudaErrorMemoryAllocation ? HPT_ENOMEM : HPT_ECUDA;        \
    }                                                                         \
  } while (0)
static hpt_status upload_constants(hpt_system s, const int32_t* ex) {
  const int n = s->n, nv = s->nv, M = s->M;
  const double* coeffs = s->coef.data();
  std::vector<double> ahat((size_t)M * (nv + 1)), b((size_t)M * (nv + 2) * 2);
  for (int i = 0; i < M; ++i) {
    const double sexp = (double)s->texp[i] / (double)s->D;
    const double cr = coeffs[2 * i], ci = coeffs[2 * i + 1];
    for (int j = 0; j < nv; ++j) {
      const double a = (double)ex[(size_t)i * nv + j];
      ahat[(size_t)i * (nv + 1) + j] = a;
      b[((size_t)i * (nv + 2) + j) * 2] = cr * a;
      b[((size_t)i * (nv + 2) + j) * 2 + 1] = ci * a;
    }
    ahat[(size_t)i * (nv + 1) + nv] = sexp;
    b[((size_t)i * (nv + 2) + nv) * 2] = cr * sexp;
    b[((size_t)i * (nv + 2) + nv) * 2 + 1] = ci * sexp;
    b[((size_t)i * (nv + 2) + nv + 1) * 2] = cr;
    b[((size_t)i * (nv + 2) + nv + 1) * 2 + 1] = ci;
  }
  CUU(cudaMalloc(&s->d_msz, n * sizeof(int32_t)));
  CUU(cudaMalloc(&s->d_off, n * sizeof(int32_t)));
  CUU(cudaMalloc(&s->d_ahat, ahat.size() * sizeof(double)));
  CUU(cudaMalloc(&s->d_b, b.size() * sizeof(double)));
  CUU(cudaMemcpy(s->d_msz, s->msz.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
  CUU(cudaMemcpy(s->d_off, s->off.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
  CUU(cudaMemcpy(s->d_ahat, ahat.data(), ahat.size() * sizeof(double), cudaMemcpyHostToDevice));
  CUU(cudaMemcpy(s->d_b, b.data(), b.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (s->prec != HPT_MIXED) return HPT_OK;

  MixedLayout& ml = s->ml;
  bool big = false;
  for (int i = 0; i < M; ++i) {
    int64_t s1 = 0;
    for (int j = 0; j < nv; ++j) s1 += std::abs(ex[(size_t)i * nv + j]);
    big = big || s1 > kBigPhase;
  }
  ml = mixed_layout(nv, s->max_m, big, nv == s->n);
  int max_smem = 0;
  CUU(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device));
  if (!eval_mixed_fits(nv, ml.MP, ml.KX, ml.NJ, ml.KC, ml.chunk_bytes, big, ml.grouped, max_smem)) {
    set_error("%d variables with m_k up to %d exceed the mixed form's on-chip memory", nv, s->max_m);
    return HPT_ENOTSUP;
  }
  std::vector<uint8_t> img((size_t)n * ml.chunk_bytes, 0);
  for (int k = 0; k < n; ++k) {
    uint8_t* ch = img.data() + (size_t)k * ml.chunk_bytes;
    uint16_t* bexp = (uint16_t*)(ch + ml.off_bexp);
    uint16_t* bhi = (uint16_t*)(ch + ml.off_bhi);
    uint16_t* blo = (uint16_t*)(ch + ml.off_blo);
    float* tf = (float*)(ch + ml.off_texp);
    uint32_t* bigm = ml.off_bigm ? (uint32_t*)(ch + ml.off_bigm) : nullptr;
    int16_t* aint = ml.off_aint ? (int16_t*)(ch + ml.off_aint) : nullptr;
    for (int i = 0; i < s->msz[k]; ++i) {
      const int idx = s->off[k] + i;
      if (aint) {
        int64_t s1 = 0;
        for (int j = 0; j < nv; ++j) {
          aint[(size_t)i * nv + j] = (int16_t)ex[(size_t)idx * nv + j];
          s1 += std::abs(ex[(size_t)idx * nv + j]);
        }
        if (s1 > kBigPhase) bigm[i / 32] |= 1u << (i % 32);
      }
      for (int sp = 0; sp < 3; ++sp)
        for (int j = 0; j < nv; ++j)
          bexp[canon_offset(i, sp * nv + j, ml.KX) / 2] = bf16_bits((float)ex[(size_t)idx * nv + j]);
      tf[i] = (float)s->texp[idx];
      // realified B_k^T: output column 2u = Re J_u, 2u+1 = Im J_u; K index
      // i = Re E_i, MP + i = Im E_i.
      for (int u = 0; u < nv + 2; ++u) {
        const double br = b[((size_t)idx * (nv + 2) + u) * 2], bi = b[((size_t)idx * (nv + 2) + u) * 2 + 1];
        uint16_t h, l;
        split2(br, h, l);
        bhi[canon_offset(2 * u, i, ml.KC) / 2] = h;
        blo[canon_offset(2 * u, i, ml.KC) / 2] = l;
        split2(-bi, h, l);
        bhi[canon_offset(2 * u, ml.MP + i, ml.KC) / 2] = h;
        blo[canon_offset(2 * u, ml.MP + i, ml.KC) / 2] = l;
        split2(bi, h, l);
        bhi[canon_offset(2 * u + 1, i, ml.KC) / 2] = h;
        blo[canon_offset(2 * u + 1, i, ml.KC) / 2] = l;
        split2(br, h, l);
        bhi[canon_offset(2 * u + 1, ml.MP + i, ml.KC) / 2] = h;
        blo[canon_offset(2 * u + 1, ml.MP + i, ml.KC) / 2] = l;
      }
    }
  }
  CUU(cudaMalloc(&s->d_chunks, img.size()));
  CUU(cudaMemcpy(s->d_chunks, img.data(), img.size(), cudaMemcpyHostToDevice));
  return HPT_OK;
}
#undef CUU

}  // namespace hpt

using namespace hpt;

extern "C" {

void hpt_default_params(hpt_params* o) {
  if (!o) return;
  o->tol_accept = 1e-3;
  o->dtau_init = 0.05;
  o->dtau_min = 1e-8;
  o->dtau_max = 0.5;
  o->grow = 2.0;
  o->shrink = 0.5;
  o->grow_after = 3;
  o->max_steps = 10000;
  o->div_bound = 1e8;
  o->polish_tol = 1e-13;
  o->polish_iters = 8;
  o->check_every = 32;
  o->cond_max = 3e4;
  o->eps0 = 1e-10;
  o->predictor = 0;
  o->pad_ = 0;
}

const char* hpt_status_string(hpt_status s) {
  switch (s) {
    case HPT_OK: return "ok";
    case HPT_EINVAL: return "invalid argument";
    case HPT_ENOMEM: return "out of memory";
    case HPT_ECUDA: return "CUDA error";
    case HPT_ERANGE: return "value out of range";
    case HPT_ENOTCELL: return "not a cell";
    case HPT_ETIMEOUT: return "device wait timed out";
    case HPT_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

const char* hpt_last_error(void) { return g_err; }

hpt_status hpt_lift_exponents(int32_t n, const int32_t* msz, const int32_t* exps,
                              const int64_t* lifting, const hpt_cell* cell, int64_t* texp,
                              int64_t* denom, int64_t* alpha_num, int64_t* beta_num) {
  Lifted L;
  hpt_status rc = lift(n, msz, exps, lifting, cell, L);
  if (rc) return rc;
  if (texp) memcpy(texp, L.e.data(), L.e.size() * sizeof(int64_t));
  if (denom) *denom = L.D;
  if (alpha_num) memcpy(alpha_num, L.alpha.data(), n * sizeof(int64_t));
  if (beta_num) memcpy(beta_num, L.beta.data(), n * sizeof(int64_t));
  return HPT_OK;
}

}  // extern "C"

namespace hpt {
// det V exactly (modular determinants over primes below 2^62, Chinese
// remainder theorem on two of them within Hadamard's bound): HPT_ERANGE when
// the bound exceeds the two primes' product / 4.
hpt_status exact_det(int n, const std::vector<int64_t>& V, i128& det) {
  double log2_h = 0.0;
  for (int k = 0; k < n; ++k) {
    double r2 = 0;
    for (int j = 0; j < n; ++j) r2 += (double)V[k * n + j] * (double)V[k * n + j];
    if (r2 == 0) { det = 0; return HPT_OK; }
    log2_h += 0.5 * log2(r2);
  }
  uint64_t p[2], d[2];
  uint64_t cand = ((uint64_t)1 << 62) - 1;
  for (int t = 0; t < 2; cand -= 2) {
    if (!is_prime64(cand)) continue;
    p[t] = cand;
    d[t] = det_mod(n, V, cand);
    ++t;
  }
  if (log2_h >= log2((double)p[0]) + log2((double)p[1]) - 2.0) {
    set_error("pair matrix entries too large for the exact determinant");
    return HPT_ERANGE;
  }
  const i128 P = (i128)p[0] * (i128)p[1];
  const uint64_t m1 = powmod(p[0] % p[1], p[1] - 2, p[1]);
  const uint64_t t = mulmod((d[1] + p[1] - d[0] % p[1]) % p[1], m1, p[1]);
  i128 x = (i128)d[0] + (i128)p[0] * (i128)t;
  if (x > P / 2) x -= P;
  det = x;
  return HPT_OK;
}

// The host part of the start points of a pairs cell: the integer diagonal
// form U V W = diag(d) (exact), z0 = V^{-1} log b (FP64) and the phase
// constants of every solution's 2 pi i W diag(1/d) m reduced modulo 1
// (StartConsts).  Validates first/count against |det V| (= *total).
hpt_status binomial_setup(int32_t n, const int32_t* msz, const int32_t* exps, const double* coeffs,
                          const int32_t* pairs, int64_t first, int64_t count, bool need_out, StartConsts& S,
                          int64_t* total) {
  int32_t M;
  hpt_status rc = check_shape(n, msz, &M);
  if (rc) return rc;
  if (!exps || !coeffs || !pairs || first < 0 || count < 0 || (count > 0 && !need_out)) {
    set_error("bad arguments");
    return HPT_EINVAL;
  }
  std::vector<int32_t> off(n);
  for (int k = 0, acc = 0; k < n; ++k) { off[k] = acc; acc += msz[k]; }
  // V_k = a_{k,p1} - a_{k,p0};  b_k = -c_{k,p0} / c_{k,p1}
  std::vector<int64_t> V((size_t)n * n);
  std::vector<double> br(n), bi(n);
  for (int k = 0; k < n; ++k) {
    const int p0 = pairs[2 * k], p1 = pairs[2 * k + 1];
    if (p0 < 0 || p1 < 0 || p0 >= msz[k] || p1 >= msz[k] || p0 == p1) { set_error("bad pair"); return HPT_EINVAL; }
    for (int j = 0; j < n; ++j)
      V[k * n + j] = (int64_t)exps[(size_t)(off[k] + p1) * n + j] - exps[(size_t)(off[k] + p0) * n + j];
    const double c0r = coeffs[2 * (off[k] + p0)], c0i = coeffs[2 * (off[k] + p0) + 1];
    const double c1r = coeffs[2 * (off[k] + p1)], c1i = coeffs[2 * (off[k] + p1) + 1];
    const double d = c1r * c1r + c1i * c1i;
    if (!(d > 0)) { set_error("zero coefficient in the cell"); return HPT_EINVAL; }
    br[k] = -(c0r * c1r + c0i * c1i) / d;
    bi[k] = -(c0i * c1r - c0r * c1i) / d;
  }
  // det V and adj V exactly, from V^{-1} modulo two primes below 2^62 and
  // the Chinese remainder theorem: exact while Hadamard's bound prod |row_k|
  // (which bounds |det V| and every (n-1)-minor) stays below p1 p2 / 2
  double log2_h = 0.0;
  for (int k = 0; k < n; ++k) {
    double r2 = 0;
    for (int j = 0; j < n; ++j) r2 += (double)V[k * n + j] * (double)V[k * n + j];
    if (r2 == 0) { set_error("the cell's pair matrix is singular"); return HPT_ENOTCELL; }
    log2_h += 0.5 * log2(r2);
  }
  uint64_t pr[2];
  std::vector<uint64_t> inv[2];
  uint64_t detp[2];
  uint64_t cand = ((uint64_t)1 << 62) - 1;
  // every prime tried exceeds 2^61, so k of them dividing det V means
  // |det V| >= 2^(61 k) or det V = 0; past Hadamard's bound it is 0
  int nsing = 0;
  for (int t = 0; t < 2; ++t) {
    for (;; cand -= 2) {
      if (!is_prime64(cand)) continue;
      const uint64_t p = cand;
      // Gauss-Jordan inverse modulo p (fails when p divides det V)
      std::vector<uint64_t> A((size_t)n * n), B((size_t)n * n, 0);
      for (int q = 0; q < n * n; ++q) {
        const int64_t v = V[q] % (int64_t)p;
        A[q] = (uint64_t)(v < 0 ? v + (int64_t)p : v);
      }
      for (int q = 0; q < n; ++q) B[q * n + q] = 1;
      uint64_t det = 1;
      bool sing = false;
      for (int c = 0; c < n && !sing; ++c) {
        int piv = -1;
        for (int r = c; r < n && piv < 0; ++r)
          if (A[r * n + c]) piv = r;
        if (piv < 0) { sing = true; break; }
        if (piv != c) {
          for (int x = 0; x < n; ++x) { std::swap(A[piv * n + x], A[c * n + x]); std::swap(B[piv * n + x], B[c * n + x]); }
          det = (p - det) % p;
        }
        det = mulmod(det, A[c * n + c], p);
        const uint64_t iv = powmod(A[c * n + c], p - 2, p);
        for (int x = 0; x < n; ++x) { A[c * n + x] = mulmod(A[c * n + x], iv, p); B[c * n + x] = mulmod(B[c * n + x], iv, p); }
        for (int r = 0; r < n; ++r) {
          if (r == c || !A[r * n + c]) continue;
          const uint64_t f = A[r * n + c];
          for (int x = 0; x < n; ++x) {
            A[r * n + x] = (A[r * n + x] + p - mulmod(f, A[c * n + x], p)) % p;
            B[r * n + x] = (B[r * n + x] + p - mulmod(f, B[c * n + x], p)) % p;
          }
        }
      }
      if (sing) {   // p divides det V: next prime, unless det V must be 0
        if (61.0 * ++nsing > log2_h + 1.0) {
          set_error("the cell's pair matrix is singular");
          return HPT_ENOTCELL;
        }
        continue;
      }
      pr[t] = p;
      detp[t] = det;
      inv[t].resize((size_t)n * n);
      for (int q = 0; q < n * n; ++q) inv[t][q] = mulmod(B[q], det, p);   // adj V mod p
      cand -= 2;
      break;
    }
  }
  if (log2_h >= log2((double)pr[0]) + log2((double)pr[1]) - 2.0) {
    set_error("the pair matrix's entries are too large for the exact enumeration");
    return HPT_ERANGE;
  }
  const i128 P = (i128)pr[0] * (i128)pr[1];
  const uint64_t m1 = powmod(pr[0] % pr[1], pr[1] - 2, pr[1]);   // p1^{-1} mod p2
  auto crt = [&](uint64_t a1, uint64_t a2) -> i128 {   // symmetric residue mod p1 p2
    const uint64_t t = mulmod((a2 + pr[1] - a1 % pr[1]) % pr[1], m1, pr[1]);
    i128 x = (i128)a1 + (i128)pr[0] * (i128)t;
    if (x > P / 2) x -= P;
    return x;
  };
  const i128 det = crt(detp[0], detp[1]);
  if (det == 0) { set_error("the cell's pair matrix is singular"); return HPT_ENOTCELL; }
  const i128 D = det < 0 ? -det : det;
  if (D >= kLim) { set_error("too many start solutions"); return HPT_ERANGE; }
  if (total) *total = (int64_t)D;
  if (first + count > (int64_t)D) {
    set_error("solutions %lld..%lld requested of %lld", (long long)first, (long long)(first + count), (long long)D);
    return HPT_ERANGE;
  }
  // coset representatives of Z^n / V Z^n: k_i in [0, h_i), h = the diagonal
  // of the Hermite normal form of the lattice V Z^n, computed modulo D (the
  // lattice contains D Z^n): column operations, rows from the last, the
  // modulus divided by each diagonal entry found
  std::vector<i128> H((size_t)n * n);
  i128 R = D;
  for (int q = 0; q < n * n; ++q) H[q] = ((i128)V[q] % R + R) % R;
  auto egcd = [](i128 a, i128 b, i128& u, i128& v) -> i128 {
    i128 r0 = a, r1 = b, u0 = 1, u1 = 0, v0 = 0, v1 = 1;
    while (r1 != 0) {
      const i128 qq = r0 / r1;
      i128 t = r0 - qq * r1; r0 = r1; r1 = t;
      t = u0 - qq * u1; u0 = u1; u1 = t;
      t = v0 - qq * v1; v0 = v1; v1 = t;
    }
    u = u0; v = v0;
    return r0;
  };
  std::vector<int64_t> h(n);
  i128 prod = 1;
  for (int i = n - 1; i >= 0; --i) {
    const int k = i;
    for (int jj = k - 1; jj >= 0; --jj) {
      if (H[i * n + jj] == 0) continue;
      i128 u, v;
      const i128 a = H[i * n + k], b = H[i * n + jj];
      const i128 g = egcd(a, b, u, v);
      const i128 ag = a / g, bg = b / g;
      u = (u % R + R) % R;
      v = (v % R + R) % R;
      for (int r = 0; r <= i; ++r) {
        const i128 xk = H[r * n + k], xj = H[r * n + jj];
        H[r * n + k] = ((u * xk) % R + (v * xj) % R) % R;
        H[r * n + jj] = (((ag % R + R) % R) * xj % R + R - ((bg % R + R) % R) * xk % R) % R;
      }
    }
    i128 u, v;
    const i128 g = egcd(H[i * n + k], R, u, v);
    const i128 gi = g < 0 ? -g : g;
    h[i] = (int64_t)gi;
    prod *= gi;
    R /= gi;
    if (R == 0) R = 1;
    for (int r = 0; r < i; ++r)
      for (int c = 0; c < i; ++c) H[r * n + c] %= R;
  }
  if (prod != D) { set_error("Hermite diagonal does not multiply to |det V|"); return HPT_ERANGE; }
  // log y = V^{-1} log b + 2 pi i V^{-1} k: the first term by Gaussian
  // elimination with partial pivoting in FP64; the second reduced modulo 1
  // exactly, V^{-1} k = adj(V) k / det V, numerators modulo D
  std::vector<double> Vd((size_t)n * n), zr0(n), zi0(n);
  for (int k = 0; k < n; ++k) {
    for (int j = 0; j < n; ++j) Vd[k * n + j] = (double)V[k * n + j];
    zr0[k] = 0.5 * log(br[k] * br[k] + bi[k] * bi[k]);
    zi0[k] = atan2(bi[k], br[k]);
  }
  for (int j = 0; j < n; ++j) {
    int piv = j;
    for (int i = j + 1; i < n; ++i)
      if (fabs(Vd[i * n + j]) > fabs(Vd[piv * n + j])) piv = i;
    if (piv != j) {
      for (int c = 0; c < n; ++c) std::swap(Vd[piv * n + c], Vd[j * n + c]);
      std::swap(zr0[piv], zr0[j]);
      std::swap(zi0[piv], zi0[j]);
    }
    for (int i = j + 1; i < n; ++i) {
      const double f = Vd[i * n + j] / Vd[j * n + j];
      for (int c = j; c < n; ++c) Vd[i * n + c] -= f * Vd[j * n + c];
      zr0[i] -= f * zr0[j];
      zi0[i] -= f * zi0[j];
    }
  }
  for (int j = n - 1; j >= 0; --j) {
    double sr = zr0[j], si = zi0[j];
    for (int c = j + 1; c < n; ++c) { sr -= Vd[j * n + c] * zr0[c]; si -= Vd[j * n + c] * zi0[c]; }
    zr0[j] = sr / Vd[j * n + j];
    zi0[j] = si / Vd[j * n + j];
  }
  S.n = n;
  S.D = (uint64_t)D;
  for (int j = 0; j < n; ++j) {
    S.h[j] = h[j];
    S.zr0[j] = zr0[j];
    S.zi0[j] = zi0[j];
  }
  for (int q = 0; q < n * n; ++q) {
    i128 a = crt(inv[0][q], inv[1][q]);   // adj V entry, exact
    if (det < 0) a = -a;                  // V^{-1} = sign(det) adj V / D
    S.adjm[q] = (uint64_t)((a % D + D) % D);
  }
  return HPT_OK;
}
}  // namespace hpt

extern "C" {

hpt_status hpt_binomial_start(int32_t n, const int32_t* msz, const int32_t* exps, const double* coeffs,
                               const int32_t* pairs, int64_t first, int64_t count, double* y0,
                               int64_t* total) {
  StartConsts S;
  hpt_status rc = binomial_setup(n, msz, exps, coeffs, pairs, first, count, y0 != nullptr, S, total);
  if (rc) return rc;
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<int64_t> k(n);
  for (int64_t q = 0; q < count; ++q) {
    int64_t idx = first + q;   // mixed radix over the Hermite diagonal, last coordinate fastest
    for (int j = n - 1; j >= 0; --j) { k[j] = idx % S.h[j]; idx /= S.h[j]; }
    for (int r = 0; r < n; ++r) {
      i128 num = 0;
      for (int j = 0; j < n; ++j)
        if (k[j]) num = (num + ((i128)S.adjm[r * n + j] * (i128)k[j]) % (i128)S.D) % (i128)S.D;
      const double frac = (double)num / (double)S.D;
      const double mag = exp(S.zr0[r]);
      const double ang = S.zi0[r] + two_pi * frac;
      y0[(q * n + r) * 2] = mag * cos(ang);
      y0[(q * n + r) * 2 + 1] = mag * sin(ang);
    }
  }
  return HPT_OK;
}

hpt_status hpt_binomial_points(int32_t n, const int32_t* msz, const int32_t* exps, const double* coeffs,
                                const int32_t* pairs, int64_t count, const int64_t* kvec, double* y0) {
  int32_t M;
  hpt_status rc = check_shape(n, msz, &M);
  if (rc) return rc;
  if (!exps || !coeffs || !pairs || count < 0 || (count > 0 && (!kvec || !y0))) {
    set_error("bad arguments");
    return HPT_EINVAL;
  }
  std::vector<int32_t> off(n);
  for (int k = 0, acc = 0; k < n; ++k) { off[k] = acc; acc += msz[k]; }
  // V_k = a_{k,p1} - a_{k,p0}, log b_k (principal) with b_k = -c_{k,p0}/c_{k,p1}
  std::vector<double> V((size_t)n * n), lr(n), li(n);
  double vmax = 0;
  for (int k = 0; k < n; ++k) {
    const int p0 = pairs[2 * k], p1 = pairs[2 * k + 1];
    if (p0 < 0 || p1 < 0 || p0 >= msz[k] || p1 >= msz[k] || p0 == p1) { set_error("bad pair"); return HPT_EINVAL; }
    for (int j = 0; j < n; ++j) {
      V[k * n + j] = (double)exps[(size_t)(off[k] + p1) * n + j] - (double)exps[(size_t)(off[k] + p0) * n + j];
      vmax = std::max(vmax, fabs(V[k * n + j]));
    }
    const double c0r = coeffs[2 * (off[k] + p0)], c0i = coeffs[2 * (off[k] + p0) + 1];
    const double c1r = coeffs[2 * (off[k] + p1)], c1i = coeffs[2 * (off[k] + p1) + 1];
    const double d = c1r * c1r + c1i * c1i;
    if (!(d > 0)) { set_error("zero coefficient in the cell"); return HPT_EINVAL; }
    const double br = -(c0r * c1r + c0i * c1i) / d, bi = -(c0i * c1r - c0r * c1i) / d;
    lr[k] = 0.5 * log(br * br + bi * bi);
    li[k] = atan2(bi, br);
  }
  // LU with partial pivoting of V (kept for every right-hand side)
  std::vector<int> perm(n);
  for (int j = 0; j < n; ++j) perm[j] = j;
  for (int j = 0; j < n; ++j) {
    int piv = j;
    for (int i = j + 1; i < n; ++i)
      if (fabs(V[i * n + j]) > fabs(V[piv * n + j])) piv = i;
    if (!(fabs(V[piv * n + j]) > 1e-9 * vmax)) { set_error("the cell's pair matrix is singular"); return HPT_ENOTCELL; }
    if (piv != j) {
      for (int c = 0; c < n; ++c) std::swap(V[piv * n + c], V[j * n + c]);
      std::swap(perm[piv], perm[j]);
    }
    for (int i = j + 1; i < n; ++i) {
      const double f = V[i * n + j] / V[j * n + j];
      V[i * n + j] = f;
      for (int c = j + 1; c < n; ++c) V[i * n + c] -= f * V[j * n + c];
    }
  }
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> zr(n), zi(n);
  for (int64_t q = 0; q < count; ++q) {
    const int64_t* kq = kvec + q * n;
    for (int j = 0; j < n; ++j) {
      zr[j] = lr[perm[j]];
      zi[j] = li[perm[j]] + two_pi * (double)kq[perm[j]];
    }
    for (int j = 0; j < n; ++j)
      for (int i = j + 1; i < n; ++i) {
        zr[i] -= V[i * n + j] * zr[j];
        zi[i] -= V[i * n + j] * zi[j];
      }
    for (int j = n - 1; j >= 0; --j) {
      double sr = zr[j], si = zi[j];
      for (int c = j + 1; c < n; ++c) { sr -= V[j * n + c] * zr[c]; si -= V[j * n + c] * zi[c]; }
      zr[j] = sr / V[j * n + j];
      zi[j] = si / V[j * n + j];
    }
    for (int r = 0; r < n; ++r) {
      const double mag = exp(zr[r]);
      y0[(q * n + r) * 2] = mag * cos(zi[r]);
      y0[(q * n + r) * 2 + 1] = mag * sin(zi[r]);
    }
  }
  return HPT_OK;
}

#define CU(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));              \
      hpt_destroy(s);                                                         \
      return e_ == cudaErrorMemoryAllocation ? HPT_ENOMEM : HPT_ECUDA;        \
    }                                                                         \
  } while (0)

hpt_status hpt_create_system(int32_t n, const int32_t* msz, const int32_t* exps,
                             const double* coeffs, const int64_t* lifting, const hpt_cell* cell,
                             hpt_precision prec, hpt_system* out) {
  if (!out) { set_error("out is NULL"); return HPT_EINVAL; }
  *out = nullptr;
  if (prec != HPT_FP64 && prec != HPT_MIXED) { set_error("bad precision"); return HPT_EINVAL; }
  if (!coeffs) { set_error("coeffs is NULL"); return HPT_EINVAL; }
  Lifted L;
  hpt_status rc = lift(n, msz, exps, lifting, cell, L);
  if (rc) return rc;
  int32_t M = (int32_t)L.e.size();
  for (int i = 0; i < 2 * M; ++i)
    if (!isfinite(coeffs[i])) { set_error("coefficient %d is not finite", i / 2); return HPT_EINVAL; }
  int max_m = 0;
  for (int k = 0; k < n; ++k) max_m = std::max(max_m, (int)msz[k]);
  if (prec == HPT_MIXED) {
    if (max_m > kMixedMaxM) { set_error("mixed form supports m_k <= %d", kMixedMaxM); return HPT_ENOTSUP; }
    // monomials with sum |a_j| > kBigPhase keep the tensor-core exponent GEMM
    // for |y^a| and take their phase in fixed point (upload_constants)
    for (int i = 0; i < M; ++i) {
      for (int j = 0; j < n; ++j) {
        int a = exps[(size_t)i * n + j];
        if (a > 256 || a < -256) { set_error("|a| > 256 is not exact in bf16"); return HPT_ERANGE; }
      }
      if (L.e[i] >= (1 << 24) || L.e[i] <= -(1 << 24)) { set_error("t-exponent not exact in fp32"); return HPT_ERANGE; }
    }
  }
  hpt_system s = new hpt_system_s();
  s->n = n;
  s->M = M;
  s->prec = prec;
  s->max_m = max_m;
  s->msz.assign(msz, msz + n);
  s->off.resize(n);
  for (int k = 0, acc = 0; k < n; ++k) { s->off[k] = acc; acc += msz[k]; }
  s->exps.assign(exps, exps + (size_t)M * n);
  s->coef.assign(coeffs, coeffs + 2 * (size_t)M);
  s->texp = L.e;
  s->D = L.D;
  s->alpha_num = L.alpha;
  s->beta_num = L.beta;
  s->nv = n;
  CU(cudaGetDevice(&s->device));
  CU(cudaMalloc(&s->d_err, sizeof(int32_t)));
  CU(cudaMemset(s->d_err, 0, sizeof(int32_t)));
  CU(cudaMallocHost(&s->h_count, sizeof(int32_t)));
  if ((rc = upload_constants(s, s->exps.data()))) {
    hpt_destroy(s);
    return rc;
  }
  *out = s;
  return HPT_OK;
}
#undef CU

static hpt_system clone_host_data(const hpt_system a, hpt_precision prec) {
  hpt_system s = new hpt_system_s();
  s->n = a->n;
  s->M = a->M;
  s->prec = prec;
  s->device = a->device;
  s->max_m = a->max_m;
  s->msz = a->msz;
  s->off = a->off;
  s->exps = a->exps;
  s->coef = a->coef;
  s->texp = a->texp;
  s->D = a->D;
  s->alpha_num = a->alpha_num;
  s->beta_num = a->beta_num;
  s->nv = a->n;
  return s;
}

hpt_status hpt_homogenize(hpt_system a, hpt_system* out) {
  if (!out) { set_error("out is NULL"); return HPT_EINVAL; }
  *out = nullptr;
  if (!a) { set_error("NULL handle"); return HPT_EINVAL; }
  if (a->proj) { set_error("the handle is already projective"); return HPT_EINVAL; }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != a->device) {
    set_error("the handle belongs to device %d, current device is %d", a->device, dev);
    return HPT_EINVAL;
  }
  const int n = a->n, nv = n + 1, M = a->M;
  if (nv > kMaxN) { set_error("the projective form supports n <= %d", kMaxN - 1); return HPT_ENOTSUP; }
  // deg_k = the largest 1^T a over S_k; a_hat = (a, deg_k - 1^T a) (Section 2.2)
  std::vector<int64_t> deg(n);
  std::vector<int32_t> ex((size_t)M * nv);
  for (int k = 0; k < n; ++k) {
    int64_t d = INT64_MIN;
    for (int i = a->off[k]; i < a->off[k] + a->msz[k]; ++i) {
      int64_t t = 0;
      for (int j = 0; j < n; ++j) t += a->exps[(size_t)i * n + j];
      d = std::max(d, t);
    }
    deg[k] = d;
    for (int i = a->off[k]; i < a->off[k] + a->msz[k]; ++i) {
      int64_t t = 0, s1 = 0;
      for (int j = 0; j < n; ++j) {
        const int32_t v = a->exps[(size_t)i * n + j];
        ex[(size_t)i * nv + j] = v;
        t += v;
        s1 += v < 0 ? -(int64_t)v : v;
      }
      const int64_t last = d - t;   // >= 0
      if (last > INT32_MAX) { set_error("homogenizing exponent overflows int32"); return HPT_ERANGE; }
      ex[(size_t)i * nv + n] = (int32_t)last;
      if (a->prec == HPT_MIXED && (last > 256 || s1 + last > 64)) {
        set_error("homogenized monomial %d: the mixed form needs |a_j| <= 256 and sum |a_j| <= 64", i);
        return HPT_ERANGE;
      }
    }
  }
  hpt_system s = clone_host_data(a, a->prec);
  s->nv = nv;
  s->proj = 1;
  s->deg = deg;
  hpt_system f = clone_host_data(a, HPT_FP64);
  s->affine = f;   // freed with s
  hpt_status rc = HPT_OK;
  cudaError_t e = cudaSuccess;
  for (hpt_system h : {s, f}) {
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_count, sizeof(int32_t));
  }
  if (e != cudaSuccess) {
    set_error("allocation failed: %s", cudaGetErrorString(e));
    rc = e == cudaErrorMemoryAllocation ? HPT_ENOMEM : HPT_ECUDA;
  }
  if (!rc) rc = upload_constants(s, ex.data());
  if (!rc) rc = upload_constants(f, f->exps.data());
  if (rc) {
    hpt_destroy(s);
    return rc;
  }
  *out = s;
  return HPT_OK;
}

hpt_status hpt_get_nvars(hpt_system s, int32_t* nv, int32_t* projective, int64_t* degrees) {
  if (!s) { set_error("NULL handle"); return HPT_EINVAL; }
  if (nv) *nv = s->nv;
  if (projective) *projective = s->proj;
  if (degrees && s->proj) memcpy(degrees, s->deg.data(), s->n * sizeof(int64_t));
  return HPT_OK;
}

hpt_status hpt_destroy(hpt_system s) {
  if (!s) return HPT_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  if (s->self_batch) hpt_batch_destroy(s->self_batch);
  if (s->affine) hpt_destroy(s->affine);
  cudaFree(s->d_msz);
  cudaFree(s->d_off);
  cudaFree(s->d_ahat);
  cudaFree(s->d_b);
  cudaFree(s->d_chunks);
  cudaFree(s->d_err);
  cudaFree(s->d_scratch);
  cudaFree(s->d_track);
  if (s->h_count) cudaFreeHost(s->h_count);
  for (auto& k : s->stats)
    for (auto& pr : k.pending) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (auto ev : s->event_pool) cudaEventDestroy(ev);
  cudaSetDevice(prev);
  delete s;
  return HPT_OK;
}

hpt_status hpt_get_info(hpt_system s, int32_t* n, int32_t* M, int32_t* prec, double eps0,
                        double* tau0) {
  if (!s) { set_error("NULL handle"); return HPT_EINVAL; }
  if (n) *n = s->n;
  if (M) *M = s->M;
  if (prec) *prec = (int32_t)s->prec;
  if (tau0) {
    if (!(eps0 > 0.0 && eps0 < 1.0)) eps0 = 1e-10;
    int64_t emin = 0;
    for (int64_t v : s->texp)
      if (v > 0 && (emin == 0 || v < emin)) emin = v;
    *tau0 = emin == 0 ? log(eps0) : log(eps0) / ((double)emin / (double)s->D);
  }
  return HPT_OK;
}

hpt_status hpt_get_texp(hpt_system s, int64_t* texp, int64_t* denom, int64_t* alpha_num,
                        int64_t* beta_num) {
  if (!s) { set_error("NULL handle"); return HPT_EINVAL; }
  if (texp) memcpy(texp, s->texp.data(), s->texp.size() * sizeof(int64_t));
  if (denom) *denom = s->D;
  if (alpha_num) memcpy(alpha_num, s->alpha_num.data(), s->n * sizeof(int64_t));
  if (beta_num) memcpy(beta_num, s->beta_num.data(), s->n * sizeof(int64_t));
  return HPT_OK;
}

hpt_status hpt_device_error(hpt_system s) {
  if (!s) { set_error("NULL handle"); return HPT_EINVAL; }
  int32_t v = 0;
  if (cudaMemcpy(&v, s->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("reading the device error flag failed");
    return HPT_ECUDA;
  }
  if (v) {
    cudaMemset(s->d_err, 0, sizeof(int32_t));
    set_error("a bounded device wait gave up (code %d)", v);
    return HPT_ETIMEOUT;
  }
  return HPT_OK;
}

hpt_status hpt_profile_enable(hpt_system s, int32_t enable) {
  if (!s) { set_error("NULL handle"); return HPT_EINVAL; }
  s->profiling = enable != 0;
  return HPT_OK;
}

hpt_status hpt_profile_read(hpt_system s, int32_t cap, const char** names, int64_t* launches,
                            double* ms, int32_t* count) {
  if (!s) { set_error("NULL handle"); return HPT_EINVAL; }
  for (auto& k : s->stats) {
    for (auto& pr : k.pending) {
      cudaEventSynchronize(pr.second);
      float t = 0.f;
      cudaEventElapsedTime(&t, pr.first, pr.second);
      k.ms += t;
      s->event_pool.push_back(pr.first);
      s->event_pool.push_back(pr.second);
    }
    k.pending.clear();
  }
  int i = 0;
  for (auto& k : s->stats) {
    if (i < cap) {
      if (names) names[i] = k.name.c_str();
      if (launches) launches[i] = k.launches;
      if (ms) ms[i] = k.ms;
    }
    ++i;
  }
  if (count) *count = (int32_t)s->stats.size();
  return HPT_OK;
}

}  // extern "C"

namespace hpt {

hpt_status ensure_scratch(hpt_system s, size_t bytes) {
  if (bytes <= s->scratch_bytes) return HPT_OK;
  cudaFree(s->d_scratch);
  s->d_scratch = nullptr;
  s->scratch_bytes = 0;
  if (cudaMalloc(&s->d_scratch, bytes) != cudaSuccess) {
    set_error("scratch allocation of %zu bytes failed", bytes);
    return HPT_ENOMEM;
  }
  s->scratch_bytes = bytes;
  return HPT_OK;
}

hpt_status ensure_track(hpt_system s, size_t bytes) {
  if (bytes <= s->track_bytes) return HPT_OK;
  cudaFree(s->d_track);
  s->d_track = nullptr;
  s->track_bytes = 0;
  if (cudaMalloc(&s->d_track, bytes) != cudaSuccess) {
    set_error("track state allocation of %zu bytes failed", bytes);
    return HPT_ENOMEM;
  }
  s->track_bytes = bytes;
  return HPT_OK;
}

static cudaEvent_t pool_event(hpt_system s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

int prof_begin(hpt_system s, const char* name, cudaStream_t st) {
  if (!s || !s->profiling) return -1;
  int idx = -1;
  for (size_t i = 0; i < s->stats.size(); ++i)
    if (s->stats[i].name == name) idx = (int)i;
  if (idx < 0) {
    s->stats.push_back(KernelStat());
    s->stats.back().name = name;
    idx = (int)s->stats.size() - 1;
  }
  cudaEvent_t a = pool_event(s), b = pool_event(s);
  cudaEventRecord(a, st);
  s->stats[idx].pending.push_back({a, b});
  return idx;
}

void prof_end(hpt_system s, int idx, cudaStream_t st) {
  if (idx < 0) return;
  KernelStat& k = s->stats[idx];
  cudaEventRecord(k.pending.back().second, st);
  k.launches += 1;
}

}  // namespace hpt
