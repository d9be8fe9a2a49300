/*
 * hpt.h -- C ABI of libhpt, a GB300 (sm_103a) implementation of the data-parallel
 * core of a polyhedral-homotopy path tracker (T. Chen, "GPU-accelerated path
 * tracker for polyhedral homotopy", arXiv:2111.14317).
 *
 * What the library computes, for a square Laurent system F = (f_1..f_n),
 * f_k(x) = sum_{a in S_k} c_{k,a} x^a (Section 2), an integer lifting w and a
 * cell (alpha, beta) of the lifted supports:
 *
 *   H_k(y, t) = sum_{a in S_k} c_{k,a} y^a t^{s_{k,a}},
 *   s_{k,a}   = <a, alpha> + w_k(a) - beta_k = e_{k,a} / D   (e integer, D >= 1),
 *
 * i.e. the polyhedral homotopy of eq. (1) after the change of variables
 * x = y t^alpha and division of h_k by t^{beta_k}; H(y, 1) = F(y).  The path
 * parameter is tau = ln t (Section 2.1, eq. (2)); tracking runs from tau0 < 0
 * to tau = 0.
 *
 * Evaluation follows Section 5: z = log y (eq. (6)), the monomials of every
 * point are exp of one row of Z A (eq. (7)), and [D_z h_k | D_tau h_k | h_k]
 * = e^{Z A} B_k^T with B_k = [A diag(c_k); c_k^T] (eq. (8) and the extended
 * Jacobian that follows), scaled by diag(e^{-z}, 1, 1) to y-coordinates.  The
 * Euler direction dE and the Newton direction dN (Section 2.3, affine form)
 * come from one factorisation of H_y with two right-hand sides, the affine
 * counterpart of the consolidated system eq. (11) of Section 6:
 *
 *   H_y [dE dN] = [-H_tau, -H].
 *
 * Conventions for every entry point:
 *   - Complex numbers are interleaved (re, im).  HPT_FP64 systems use
 *     complex128 (2 doubles) for y and every output; HPT_MIXED systems use
 *     complex64 (2 floats) for y, the step state and hpt_eval's outputs.
 *     Track outputs and the adjoint are always complex128.
 *   - Pointers named *_dev are device pointers owned by the caller; the
 *     library never frees them.  The library owns the handle's constants and
 *     its scratch (per-handle, grown on demand by cudaMalloc, released by
 *     hpt_destroy).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; only hpt_track and the host-side
 *     getters synchronise.
 *   - A handle may be used by one host thread at a time.
 *   - The library never aborts and has no CPU fallback.  Argument errors are
 *     returned as status codes; per-path numerical failures go to the per-path
 *     status arrays, never to the return code.  hpt_last_error() returns a
 *     message for the last failing call of the calling thread.
 *   - Device-side waits are bounded; a wait that gives up sets a flag that
 *     hpt_device_error() reports as HPT_ETIMEOUT.
 */
#ifndef HPT_H_
#define HPT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hpt_system_s* hpt_system;

typedef enum {
  HPT_OK = 0,
  HPT_EINVAL = 1,    /* bad argument (null pointer, size out of range, bad enum) */
  HPT_ENOMEM = 2,    /* device or host allocation failed */
  HPT_ECUDA = 3,     /* a CUDA runtime call failed */
  HPT_ERANGE = 4,    /* integer overflow, or a value not exactly representable in
                        the precision form that needs it */
  HPT_ENOTCELL = 5,  /* the cell is singular, not a lower facet, or the lifting is
                        not generic for it */
  HPT_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
  HPT_ENOTSUP = 7    /* shape not supported by the requested precision form */
} hpt_status;

typedef enum { HPT_FP64 = 0, HPT_MIXED = 1 } hpt_precision;

/* Per-path status codes written by hpt_step / hpt_track. */
typedef enum {
  HPT_PATH_ACTIVE = 0,
  HPT_PATH_CONVERGED = 1,   /* reached tau = 0 (then polished by hpt_track) */
  HPT_PATH_DIVERGED = 2,    /* |y_j| left [1/div_bound, div_bound] */
  HPT_PATH_UNDERFLOW = 3,   /* step size fell below dtau_min */
  HPT_PATH_SINGULAR = 4,    /* singular or non-finite system before any accept */
  HPT_PATH_MAX_STEPS = 5    /* step budget exhausted */
} hpt_path_status;

typedef enum { HPT_CELL_PAIRS = 0, HPT_CELL_EXPLICIT = 1, HPT_CELL_LOWER = 2 } hpt_cell_kind;

/* Cell of the lifted supports (Section 2 defers the cell step to Huber and
 * Sturmfels; these are its three standard descriptions).
 *   HPT_CELL_PAIRS:    pairs[2k], pairs[2k+1] are two local monomial indices of
 *                      S_k.  alpha solves V alpha = (w_{k,p0} - w_{k,p1})_k with
 *                      V_k = a_{k,p1} - a_{k,p0}; D is the least positive common
 *                      denominator of alpha; alpha_num = D alpha; beta_num_k =
 *                      <a_{k,p0}, alpha_num> + D w_{k,p0}.  Every other monomial
 *                      must get e > 0 (HPT_ENOTCELL otherwise).
 *   HPT_CELL_EXPLICIT: alpha_num (n), beta_num (n), denom = D > 0 as given;
 *                      every e must be >= 0.
 *   HPT_CELL_LOWER:    alpha_num (n), denom = D > 0; beta_num_k = min over S_k of
 *                      <a, alpha_num> + D w(a) (so min_i e_{k,i} = 0).
 * In all kinds e_{k,i} = <a_{k,i}, alpha_num> + D w_{k,i} - beta_num_k.      */
typedef struct {
  int32_t kind;
  const int32_t* pairs;      /* 2n, kind PAIRS */
  const int64_t* alpha_num;  /* n, kinds EXPLICIT and LOWER */
  const int64_t* beta_num;   /* n, kind EXPLICIT */
  int64_t denom;             /* kinds EXPLICIT and LOWER */
} hpt_cell;

/* Step-size control (the paper fixes one Euler prediction and one Newton
 * iteration per step, Section 8; the control rule is this library's).  A
 * step evaluates at the predicted point y(tau); it is accepted when
 * |dN|_inf / max(1, |y|_inf) <= tol_accept; then y_acc = y + dN, and after
 * grow_after accepts in a row dtau = min(grow * dtau, dtau_max).  On reject
 * dtau *= shrink (below dtau_min: HPT_PATH_UNDERFLOW).  The next prediction is
 * y = y_acc + h dE_acc, tau = tau_acc + h, h = min(dtau, -tau_acc).  Before the
 * first accept a rejected step keeps correcting at tau0 (y += dN).            */
typedef struct {
  double tol_accept;    /* default 1e-3 (FP64) -- use 3e-3 for HPT_MIXED */
  double dtau_init;     /* default 0.05 */
  double dtau_min;      /* default 1e-8 */
  double dtau_max;      /* default 0.5 */
  double grow;          /* default 2 */
  double shrink;        /* default 0.5 */
  int32_t grow_after;   /* default 3 */
  int32_t max_steps;    /* default 10000 */
  double div_bound;     /* default 1e8 */
  double polish_tol;    /* default 1e-13: the FP64 Newton polish at t = 1 stops when the
                           relative correction |dN|/max(1,|x|) is below it, or when the
                           error it leaves is: r_k^3 / r_{k-1}^2 <= polish_tol for the last
                           two corrections once they shrink at least tenfold (quadratic
                           convergence) */
  int32_t polish_iters; /* default 8 */
  int32_t check_every;  /* hpt_track: steps between host checks, default 32 */
  double cond_max;      /* HPT_MIXED: bound on the pivot ratio max|u_jj|/min|u_jj| of the
                           power-of-two equilibrated D_z H above which the FP32 solve is
                           redone in FP64, default 3e4: the ratio understates kappa_1 by a
                           median factor of about 33 (at most about 540 on 20,000 points of
                           the n = 16 throughput workload), so the default re-solves the
                           typical path whose kappa_1 exceeds about 1e6 (Section 6's remark
                           on ill-conditioned systems).  A lower bound costs time: each
                           launch that re-solves any path takes about 0.14 ms, the latency of
                           one FP64 solve on this part */
  double eps0;          /* tau0 = ln(eps0) / s_min (smallest positive e/D), default 1e-10 */
  int32_t predictor;    /* 0 (default): Euler, y = y_acc + h dE_acc.  1: cubic Hermite, once a
                           path has two accepted points (tau0, y0, d0), (tau1, y1, d1) (the state's
                           *_prev arrays and y_acc, dE_acc): the cubic with those values and
                           derivatives at tau0 and tau1, evaluated at tau1 + h (Section 2.3
                           names it among the predictors built on the Euler direction).  In the
                           projective form y0 and d0 are first multiplied by the unit phase that
                           makes y1^* y0 real and positive.  A rejected cubic prediction is
                           retried once with the Euler prediction at the same step size (the
                           step shrinks only when an Euler prediction is rejected).  Needs the
                           *_prev and hermite state arrays. */
  int32_t pad_;
} hpt_params;

/* Structure-of-arrays path state (caller-owned device buffers, p paths).
 * y, y_acc, dE_acc: p x n complex of the system's precision, row-major. */
typedef struct {
  void* y;            /* predicted point at tau */
  double* tau;
  double* dtau;
  void* y_acc;        /* last accepted (corrected) point */
  double* tau_acc;
  void* dE_acc;       /* Euler direction at the last accepted point */
  int32_t* status;    /* hpt_path_status */
  int32_t* steps;     /* step attempts */
  int32_t* accepts;
  int32_t* rejects;
  int32_t* streak;    /* accepts in a row since the last growth or reject */
  /* The accepted point before the last one (p x n complex, p doubles) and
   * whether the pending prediction is a cubic Hermite one (p int32): read and
   * written only with params->predictor == 1 (NULL otherwise). */
  void* y_prev;
  double* tau_prev;
  void* dE_prev;
  int32_t* hermite;
} hpt_paths;

/* Fills the defaults listed in hpt_params. */
void hpt_default_params(hpt_params* out);

const char* hpt_status_string(hpt_status s);
const char* hpt_last_error(void);

/* Host-only exact bookkeeping (no device work; usable without a GPU).
 * Inputs: n (1..32); support_sizes[n] = m_k >= 1 (pairs need m_k >= 2);
 * exponents[M*n] int32, row-major, grouped by equation (M = sum m_k);
 * lifting[M] int64; cell as above.  Outputs (any may be NULL): texp[M] the
 * numerators e, *denom D, alpha_num[n], beta_num[n].  Exact int64 arithmetic
 * with 128-bit intermediates; HPT_ERANGE on overflow, HPT_ENOTCELL as above. */
hpt_status hpt_lift_exponents(int32_t n, const int32_t* support_sizes, const int32_t* exponents,
                              const int64_t* lifting, const hpt_cell* cell, int64_t* texp,
                              int64_t* denom, int64_t* alpha_num, int64_t* beta_num);

/* Host-only fine mixed cells of the lifted supports (the cell step Section 2
 * leaves to Huber and Sturmfels): every choice of one pair {p0, p1} per
 * support S_k for which some inner normal alpha makes each pair the lowest
 * points of its lifted support, <a_p0, alpha> + w(p0) = <a_p1, alpha> +
 * w(p1) < <a, alpha> + w(a) for every other a in S_k.  A depth-first search
 * fixes the pairs equation by equation among each support's lower edges and
 * prunes a partial choice as soon as its conditions have no solution alpha
 * (FP64 linear feasibility: the pair equations eliminated, then an interval,
 * a Fourier-Motzkin step, or a small simplex on the Farkas alternative);
 * every complete choice is
 * confirmed exactly as hpt_lift_exponents does for a PAIRS cell.  For a
 * generic lifting these are the cells of the fine mixed subdivision and the
 * sum of their |det V| is the mixed volume (the root count of Section 2).
 * Inputs as hpt_lift_exponents (m_k >= 2).  Writes up to cap cells to
 * pairs_out[cap * 2n] (local indices, the hpt_cell PAIRS layout), the number
 * found to *ncells and sum |det V| to *mixed_volume (either may be NULL).
 * HPT_ERANGE when a lifting value lies outside [-2^40, 2^40], or when a
 * determinant, an exact cell test or the volume leaves the exact range.
 * HPT_ENOTCELL when the lifting is not generic: some complete choice passed
 * the FP64 search but failed the exact test (a tie with another point); the
 * cells and volume written are then incomplete, so draw a new lifting. */
hpt_status hpt_mixed_cells(int32_t n, const int32_t* support_sizes, const int32_t* exponents, const int64_t* lifting,
                           int64_t cap, int32_t* pairs_out, int64_t* ncells, int64_t* mixed_volume);

/* Host-only start points of a cell of kind PAIRS: the solutions in (C*)^n of
 * the binomial start system H(y, t=0) = 0, i.e. c_{k,p0} y^{a_{k,p0}} +
 * c_{k,p1} y^{a_{k,p1}} = 0 (Section 2 leaves this step to Huber and
 * Sturmfels).  With V_k = a_{k,p1} - a_{k,p0} and b_k = -c_{k,p0}/c_{k,p1},
 * the |det V| solutions are y = exp(V^{-1}(log b + 2 pi i k)) for k in the
 * coset representatives 0 <= k_j < h_j of Z^n / V Z^n, h the diagonal of the
 * Hermite normal form of the lattice V Z^n.  Exact integer work: det V and
 * adj V from V^{-1} modulo two primes below 2^62 (Chinese remainder theorem,
 * within Hadamard's bound), the Hermite diagonal modulo |det V|, and the phase
 * V^{-1} k = adj(V) k / det V reduced modulo 1 exactly; V^{-1} log b in FP64.
 * Writes solutions first..first+count-1 (mixed-radix order of k, last
 * coordinate fastest) to y0[count*n] complex128 (interleaved) and |det V| to
 * *total (may be NULL).  HPT_ENOTCELL for a singular pair matrix, HPT_ERANGE
 * for |det V| >= 2^62, entries beyond the exact range, or a range beyond
 * |det V|. */
hpt_status hpt_binomial_start(int32_t n, const int32_t* support_sizes, const int32_t* exponents,
                              const double* coeffs, const int32_t* pairs, int64_t first, int64_t count,
                              double* y0, int64_t* total);

/* The start points of hpt_binomial_start computed on the device: host inputs
 * as there (the exact diagonal form is formed on the host), solutions
 * first..first+count-1 written by a kernel to y0_dev[count*n] complex128 (a
 * device pointer owned by the caller), one thread per solution with exact
 * 64-bit modular phase arithmetic (the constants travel as one kernel
 * argument: no device allocation); asynchronous on `stream` (cudaStream_t as
 * void*, NULL = legacy default stream).  *total (may be NULL) receives
 * |det V|.  Same errors as hpt_binomial_start; HPT_ECUDA if the launch fails.
 * Agrees with hpt_binomial_start to rounding (device exp/sincos). */
hpt_status hpt_binomial_start_device(int32_t n, const int32_t* support_sizes, const int32_t* exponents,
                                     const double* coeffs, const int32_t* pairs, int64_t first, int64_t count,
                                     void* y0_dev, int64_t* total, void* stream);

/* Host-only start points of a PAIRS cell for chosen lattice vectors: for each
 * k (kvec[count*n] int64, row q = k of solution q) writes y = exp(z) with
 * V z = log b + 2 pi i k (log b principal, V and b as in hpt_binomial_start)
 * to y0[count*n] complex128.  Every solution of the start system is of this
 * form; k and k' give the same solution exactly when k - k' lies in V Z^n.
 * Floating-point (FP64 LU with partial pivoting), so it serves any |det V|,
 * where hpt_binomial_start's exact enumeration needs |det V| < 2^62.
 * HPT_ENOTCELL for a singular pair matrix. */
hpt_status hpt_binomial_points(int32_t n, const int32_t* support_sizes, const int32_t* exponents,
                               const double* coeffs, const int32_t* pairs, int64_t count, const int64_t* kvec,
                               double* y0);

/* Algorithm 1 (Initialize): exact bookkeeping as hpt_lift_exponents, then one
 * upload of the constants (A with the t-exponent row, B_k for every k, and for
 * HPT_MIXED their split-BF16 operand images) to the current device.
 * coeffs[2M] are c_{k,i} as (re, im) doubles.  HPT_MIXED needs |a_j| <= 256 and
 * sum_j |a_j| <= 64 for every monomial (HPT_ERANGE), n <= 32, m_k <= 128 and
 * operand shapes that fit the evaluation kernel's shared and tensor memory
 * (for example n = 24 with m_k <= 96, n = 8 with m_k <= 128; HPT_ENOTSUP
 * otherwise).  *out receives the handle. */
hpt_status hpt_create_system(int32_t n, const int32_t* support_sizes, const int32_t* exponents,
                             const double* coeffs, const int64_t* lifting, const hpt_cell* cell,
                             hpt_precision prec, hpt_system* out);

hpt_status hpt_destroy(hpt_system sys);

/* Projective formulation (Section 2.2, eq. (3)): a new handle of the same
 * precision and device for the homogenized homotopy of sys, n equations in
 * nv = n + 1 homogeneous coordinates y = (y_0 .. y_{n-1}, y_n), the
 * homogenizing coordinate last.  Every exponent a of equation k becomes
 * (a, deg_k - 1^T a) with deg_k = max over S_k of 1^T a (the total degree of
 * a polynomial f_k; for a Laurent support the least degree that keeps the
 * new exponent non-negative), so h_k(lambda y) = lambda^deg_k h_k(y) and
 * h_k((x, 1), t) = H_k(x, t).  sys is not referenced afterwards (the new
 * handle keeps its own copy of the affine constants for the polish and the
 * adjoint).  On the new handle:
 *   - hpt_eval takes y_dev[p*nv] and writes H[p*n], Hy[p*n*nv], Ht[p*n];
 *   - hpt_euler_newton gives the projective directions (below);
 *   - hpt_paths_init takes AFFINE start points y0_dev[p*n] complex128 and
 *     stores (x0, 1)/|(x0, 1)|; the state holds p*nv entries per array;
 *   - hpt_step runs the projective step: Algorithm 3 by QR, then the step
 *     control of hpt_params with two changes: after every Newton correction
 *     the point (and the stored Euler direction, by the same factor) is
 *     scaled to unit Euclidean norm, and a path is HPT_PATH_DIVERGED when a
 *     dehomogenized coordinate |y_j / y_n| leaves [1/div_bound, div_bound],
 *     tested before the end-of-path test (a path may reach t = 1 at
 *     infinity);
 *   - hpt_track takes affine start points, tracks in homogeneous coordinates
 *     (both precisions step through hpt_step's launches, not a batch) and
 *     writes dehomogenized end points x = y'/y_n, FP64-polished;
 *   - hpt_polish and hpt_adjoint work on affine points x[p*n];
 *   - hpt_step_static and hpt_batch_create return HPT_ENOTSUP.
 * HPT_ENOTSUP for n > 31; HPT_ERANGE when a homogenized monomial of an
 * HPT_MIXED system breaks its exponent limits (below); HPT_EINVAL when sys is
 * already projective. */
hpt_status hpt_homogenize(hpt_system sys, hpt_system* out);

/* Variables per point (nv = n, or n + 1 for a projective handle), whether the
 * handle is projective, and for a projective handle the degrees deg_k
 * (degrees[n] int64, may be NULL). */
hpt_status hpt_get_nvars(hpt_system sys, int32_t* nv, int32_t* projective, int64_t* degrees);

/* Host getters: sizes, form, tau0 for params->eps0 (NULL = default), and the
 * exact integer data the handle was built from (arrays may be NULL). */
hpt_status hpt_get_info(hpt_system sys, int32_t* n, int32_t* M, int32_t* prec, double eps0,
                        double* tau0);
hpt_status hpt_get_texp(hpt_system sys, int64_t* texp, int64_t* denom, int64_t* alpha_num,
                        int64_t* beta_num);

/* Algorithm 2 (Evaluate) for p points: y_dev[p*n] complex, t_dev[p] doubles
 * in (0, 1].  Writes H_dev[p*n] (H_k), Hy_dev[p*n*n] (dH_k/dy_j at [q][k][j])
 * and Ht_dev[p*n] (dH_k/dt = (dH_k/dtau) / t), complex of the system's
 * precision.  Any output pointer may be NULL.  p = 0 is a no-op. */
hpt_status hpt_eval(hpt_system sys, int64_t p, const void* y_dev, const double* t_dev,
                    void* H_dev, void* Hy_dev, void* Ht_dev, void* stream);

/* Algorithm 3 (EulerNewton, Section 6) for p points y_dev[p*nv] (complex of
 * the handle's precision) at tau_dev[p] (tau = ln t <= 0): the consolidated
 * matrix J = [[dH/dy, dH/dtau, H], [y^*, 0, 0]] (N = nv rows; an affine
 * handle has no y^* row, N = n) is factored as J^T = Q [R; 0] by Householder
 * reflections; the two rightmost columns of Q give the null space of J, and
 * the reduction that turns their last two entries into the 2 x 2 identity
 * gives the Euler direction dE (dH/dy dE + dH/dtau = 0, eq. (4)) and the
 * Newton direction dN (dH/dy dN + H = 0, eq. (5)), both with y^* d = 0 in the
 * projective form.  Writes dE_dev[p*nv], dN_dev[p*nv] (the handle's complex
 * type) and ok_dev[p] int32 (1 when every reflector norm is nonzero, the
 * 2 x 2 block is invertible and all values are finite).  HPT_MIXED: FP32
 * factorisation of the tensor-core evaluation.  Asynchronous on `stream`. */
hpt_status hpt_euler_newton(hpt_system sys, int64_t p, const void* y_dev, const double* tau_dev, void* dE_dev,
                            void* dN_dev, int32_t* ok_dev, void* stream);

/* Prepares a path state for tracking from start points y0_dev[p*n] complex128
 * at tau0 (from params->eps0): y = y_acc = y0, tau = tau_acc = tau0,
 * dtau = dtau_init, dE_acc = 0, counters 0, status ACTIVE. */
hpt_status hpt_paths_init(hpt_system sys, int64_t p, const void* y0_dev, const hpt_params* params,
                          const hpt_paths* state, void* stream);

/* nsteps Euler-Newton steps (Section 8: one Euler prediction, one Newton
 * iteration) for every ACTIVE path of the state (Algorithms 2 and 3 per step).
 * Paths that are not ACTIVE are left unchanged. */
hpt_status hpt_step(hpt_system sys, int64_t p, const hpt_paths* state, int32_t nsteps,
                    const hpt_params* params, void* stream);

/* The step of hpt_step with no device-memory allocation.  The paper has no
 * counterpart of this entry point.  Its scratch (the extended Jacobians of
 * the p paths and the FP64 re-solve list) comes from a 32 MiB array compiled
 * into the library (a file-scope __device__ array that every GPU loading the
 * library holds until the process exits) instead of from cudaMalloc.  It is
 * for callers that must not allocate device memory while they run:
 * applications that give all device memory to their own allocator or pool and
 * forbid libraries from allocating behind it, code with a fixed device-memory
 * budget, and loops that cannot afford the device synchronisation of
 * cudaMalloc/cudaFree.  The caller still owns the state buffers.
 * Limit: p <= (32 MiB - 511 - 127 n (n+2) c) / (n (n+2) c + 8) paths, c = 16
 * bytes (HPT_FP64) or 8 (HPT_MIXED); for n = 16 that is 7,142 (FP64) or 14,386
 * (mixed) paths.
 * Larger p returns HPT_ERANGE (split the batch).  The first call on a device
 * looks up the array's device address with cudaGetSymbolAddress (with that
 * device current) and caches it; make that first call before any stream
 * capture.  All calls on a device share the one array: calls whose GPU work
 * overlaps (other streams, other host threads) race and corrupt each other.
 * Like hpt_step it runs in rounds of at most 65,536 paths.
 * Same arguments, results and error behaviour as hpt_step otherwise. */
hpt_status hpt_step_static(hpt_system sys, int64_t p, const hpt_paths* state, int32_t nsteps,
                           const hpt_params* params, void* stream);

/* Whole tracks: start points y0_dev[p*n] complex128 at tau0 -> tau = 0, then an
 * FP64 Newton polish at t = 1 of the converged paths.  Section 2.1, eq. (2):
 * with t = e^tau the paths run over tau in (-inf, 0], starting from a tau0 < 0
 * of large magnitude (tau0 = ln(eps0) / s_min, s_min the smallest positive
 * t-exponent) and ending at tau = 0, where H(x, 1) = F(x) (Section 2, below
 * eq. (1)); each step is the Euler-Newton step of Section 8.  Writes x_out_dev[p*n]
 * complex128, status_dev[p], steps_dev[p].  Synchronises the stream.  The
 * HPT_MIXED form runs as a one-system hpt_batch_track (created on first use
 * and kept with the handle), which compacts finished paths out of the
 * launches; results are those of stepping all paths together. */
hpt_status hpt_track(hpt_system sys, int64_t p, const void* y0_dev, const hpt_params* params,
                     void* x_out_dev, int32_t* status_dev, int32_t* steps_dev, void* stream);

/* FP64 Newton polish at t = 1 of x_dev[p*n] complex128 in place, for paths
 * whose status_dev entry is HPT_PATH_CONVERGED (status_dev NULL: all paths).
 * Section 2.3: repeated affine Newton directions, dH/dx dN = -H, at tau = 0,
 * where H(x, 1) = F(x) is the target system (Section 2, below eq. (1));
 * stops when |dN|_inf / max(1, |x|_inf) <= polish_tol or after polish_iters
 * iterations. */
hpt_status hpt_polish(hpt_system sys, int64_t p, void* x_dev, const int32_t* status_dev,
                      const hpt_params* params, void* stream);

/* Implicit-function adjoint.  The paper has no counterpart of this entry
 * point; it reuses the Jacobian dH/dx of Section 2.3 at tau = 0 (J = F_x,
 * since H(x, 1) = F(x)).  At solutions x_dev[p*n] complex128 of F = H(., 1):
 * with J = F_x and gx_dev[p*n] = dL/dRe x + i dL/dIm x of a real loss L, solves
 * J^H lambda = gx per solution and writes gc_dev[M] complex128 =
 * -sum over solutions of lambda_k conj(x^{a_{k,i}}), the gradient of L with
 * respect to the coefficients in the same convention (FP64). */
hpt_status hpt_adjoint(hpt_system sys, int64_t p, const void* x_dev, const void* gx_dev,
                       void* gc_dev, void* stream);

/* Reads and clears the handle's device error flag (synchronises the device):
 * HPT_OK or HPT_ETIMEOUT. */
hpt_status hpt_device_error(hpt_system sys);

/* Diagnostic: enqueues on `stream` one CTA that waits, with the library's
 * bounded device-side wait, on an mbarrier that nothing completes; after about
 * 2 s the wait gives up and sets the handle's error flag, so that the next
 * hpt_device_error returns HPT_ETIMEOUT and the context stays usable.  For
 * testing the failure path without any device fault. */
hpt_status hpt_check_bounded_wait(hpt_system sys, void* stream);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every kernel the handle launches while enabled.  hpt_profile_read returns,
 * for up to cap kernels, the name, the number of launches and the summed
 * milliseconds (synchronises), and the number of distinct kernels. */
hpt_status hpt_profile_enable(hpt_system sys, int32_t enable);
hpt_status hpt_profile_read(hpt_system sys, int32_t cap, const char** names, int64_t* launches,
                            double* ms, int32_t* count);

/* ---- Batching form: many systems of different sizes in one tracker ----
 *
 * Problem (d) of Section 1 asks for parallelism at several levels; Section 5
 * batches the points of one system.  A batch goes one level up: the paths of
 * many HPT_MIXED systems (n may differ) advance together.  Every step is one
 * launch of the mixed evaluation kernel over all live paths of all systems
 * (each 128-path tile belongs to one system and reads that system's
 * constants), one FP32 solve launch per lane-group shape (n <= 8, <= 16,
 * <= 32) and one FP64 re-solve launch.  After every round of K steps the live
 * paths are compacted on the device (finished paths leave the launches) and
 * the position count comes back to the host, which stops when it is 0.  A
 * round (K steps + compaction + count read-back) is a captured CUDA graph,
 * replayed.  Converged paths get the FP64 polish of hpt_track per system.
 */
typedef struct hpt_batch_s* hpt_batch;

typedef struct {
  int32_t steps_per_round;    /* K: steps between compactions (1..256) */
  int32_t eval_ctas_per_sm;   /* resident evaluation CTAs per SM: 1 or 2 (capped by tensor memory) */
  int32_t solve_lanes_n17_24; /* FP32 solve of systems with 17 <= n <= 24: 8 lanes x 3 rows or
                                 32 lanes x 1 row per path (8 or 32) */
} hpt_batch_tuning;

/* Groups nsys (>= 1) HPT_MIXED system handles of the current device (their
 * constant images are copied; the handles must outlive the batch, whose
 * polish uses them).  Default tuning: K = 16, 2 CTAs/SM where they fit.
 * HPT_ENOTSUP if a handle is HPT_FP64. */
hpt_status hpt_batch_create(int32_t nsys, const hpt_system* systems, hpt_batch* out);
hpt_status hpt_batch_destroy(hpt_batch b);
hpt_status hpt_batch_get_tuning(hpt_batch b, hpt_batch_tuning* t);
hpt_status hpt_batch_set_tuning(hpt_batch b, const hpt_batch_tuning* t);

/* Tracks paths[s] (host array, >= 0) paths of every system s from t = 0 to
 * t = 1 and polishes the converged ones, as hpt_track does for one system.
 * y0: device complex128 start points, system 0's paths[0] x n_0 values, then
 * system 1's, ... (concatenated, path-major).  x_out: device complex128 in
 * the same layout; status_out, steps_out: device int32 per path in the same
 * order (either may be NULL).  The batch owns its state and scratch (grown
 * on demand, kept for the next call).  Work is ordered after earlier work on
 * `stream`; returns after it is done. */
hpt_status hpt_batch_track(hpt_batch b, const int64_t* paths, const void* y0, const hpt_params* prm,
                           void* x_out, int32_t* status_out, int32_t* steps_out, void* stream);

/* The project's autotuner: times whole hpt_batch_track calls on the given
 * problem, one knob at a time from the current tuning (coordinate descent):
 * the mid-size solve shape (8 or 32 lanes), then eval CTAs/SM (1, 2 where
 * tensor memory allows), then K in {2, 4, 8, 16, 32}; keeps the fastest as the
 * batch's tuning.  Writes the chosen tuning to *best, and, where not NULL,
 * each timed candidate's tuning and milliseconds to cand[] / ms[] (capacity
 * *ncand in, count out). */
hpt_status hpt_batch_autotune(hpt_batch b, const int64_t* paths, const void* y0, const hpt_params* prm,
                              void* x_out, void* stream, hpt_batch_tuning* best, hpt_batch_tuning* cand,
                              double* ms, int32_t* ncand);

/* Counters of the last hpt_batch_track: rounds (graph replays), positions
 * evaluated summed over steps (live paths + tile padding), and the number of
 * kernels one round launches. */
hpt_status hpt_batch_stats(hpt_batch b, int64_t* rounds, int64_t* position_steps, int32_t* kernels_per_round);

#ifdef __cplusplus
}
#endif

#endif /* HPT_H_ */
