/*
 * CPU oracle for the polyhedral-homotopy path tracker -- TEST INFRASTRUCTURE.
 *
 * This file is the plain, slow, obviously correct complex128 reference that
 * the CUDA library is checked against.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark load it; the library never does.
 * It shares no code with the library.
 *
 * What it computes (T. Chen, "GPU-accelerated path tracker for polyhedral
 * homotopy"):
 *
 *   H_k(y, tau) = sum_i c_{k,i} y^{a_{k,i}} t^{s_{k,i}},   t = e^tau,
 *   s_{k,i} = e_{k,i} / D  (integer numerator over a common denominator),
 *
 * the cell-transformed form of the polyhedral homotopy of Section 2, eq. (1)
 * with the logarithmic parameter of Section 2.1, eq. (2).  Monomials are formed
 * by repeated multiplication (no logarithms, unlike the GEMM formulation of
 * Section 5), derivatives by direct differentiation of every term:
 *
 *   dH_k/dy_j   = sum_i c a_j y^{a - e_j} t^s,
 *   dH_k/dtau   = sum_i c s y^a t^s,
 *
 * and t^s = exp(s * tau) (real).  The Euler and Newton directions are the
 * solutions of the two affine linear systems of Section 2.3, solved together
 * as in Section 6, eq. (11) (affine form: one LU factorisation of H_y, two
 * right-hand sides [-H_tau, -H]).
 *
 * The step and step-size control follow the simplified Euler-Newton step of
 * Section 8 (one Euler prediction, one Newton iteration); the paper gives no
 * step-size rule, so the rule here is a stated reading (accept on the size of
 * the Newton correction, halve on reject, double after a run of accepts).
 *
 * Parity status: every function here is pinned by the CPU tests (finite
 * differences, the log-coordinate identity of Section 5, H(y,1) = F(y),
 * numpy.polyval for one variable, numpy.linalg.solve, closed-form paths,
 * the BKK root count, finite differences of the adjoint; the tolerance
 * scales of ora_scale against the term magnitudes summed with numpy powers,
 * with planted mistakes that the pin must reject).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

#define ORA_NMAX 32

typedef struct {
    int32_t n;             /* variables = equations */
    int32_t M;             /* total number of monomials */
    const int32_t* msz;    /* n: support sizes m_k */
    const int32_t* off;    /* n: first monomial of equation k */
    const int32_t* exps;   /* M*n: exponent vectors a_{k,i}, row-major */
    const double* coef;    /* 2M: coefficients c_{k,i} (re, im) */
    const int64_t* texp;   /* M: t-exponent numerators e_{k,i} */
    int64_t D;             /* common denominator of the t-exponents */
} ora_sys;

typedef struct {
    double tol_accept;     /* accept if |dN|_inf / max(1, |y|_inf) <= tol */
    double dtau_init;
    double dtau_min;
    double dtau_max;
    double grow;           /* step growth factor after a run of accepts */
    double shrink;         /* step factor on reject */
    int32_t grow_after;    /* accepts in a row before growing */
    int32_t max_steps;
    double div_bound;      /* |y_j| > bound or |y_j| < 1/bound: diverged */
    double polish_tol;     /* final Newton stop: |dN|_inf/max(1,|y|_inf) */
    int32_t polish_iters;
    int32_t predictor;     /* 0: Euler; 1: cubic Hermite through the last two accepted points */
} ora_params;

enum { ORA_ACTIVE = 0, ORA_CONVERGED = 1, ORA_DIVERGED = 2, ORA_UNDERFLOW = 3,
       ORA_SINGULAR = 4, ORA_MAX_STEPS = 5 };

static inline cplx coef_at(const ora_sys* s, int idx) {
    return s->coef[2 * idx] + I * s->coef[2 * idx + 1];
}

/* prod_l y_l^{a_l - [l == jdec]} by repeated multiplication; negative powers
 * multiply the reciprocal. */
static cplx powprod(int n, const cplx* y, const cplx* yinv, const int32_t* a, int jdec) {
    cplx r = 1.0;
    for (int l = 0; l < n; ++l) {
        int e = a[l] - (l == jdec ? 1 : 0);
        if (e > 0) { for (int q = 0; q < e; ++q) r *= y[l]; }
        else if (e < 0) { for (int q = 0; q < -e; ++q) r *= yinv[l]; }
    }
    return r;
}

/* H, H_y (n x n row-major, [k][j]), H_tau at one point. */
static void eval_one(const ora_sys* s, const cplx* y, double tau,
                     cplx* H, cplx* Hy, cplx* Htau) {
    const int n = s->n;
    cplx yinv[ORA_NMAX];
    for (int j = 0; j < n; ++j) yinv[j] = 1.0 / y[j];
    for (int k = 0; k < n; ++k) {
        cplx h = 0.0, ht = 0.0;
        for (int j = 0; j < n; ++j) Hy[k * n + j] = 0.0;
        for (int i = 0; i < s->msz[k]; ++i) {
            const int idx = s->off[k] + i;
            const int32_t* a = s->exps + (size_t)idx * n;
            const double sexp = (double)s->texp[idx] / (double)s->D;
            const double ts = exp(sexp * tau);
            const cplx c = coef_at(s, idx);
            const cplx mono = powprod(n, y, yinv, a, -1);
            h += c * mono * ts;
            ht += c * sexp * mono * ts;
            for (int j = 0; j < n; ++j) {
                if (a[j] == 0) continue;
                Hy[k * n + j] += c * (double)a[j] * powprod(n, y, yinv, a, j) * ts;
            }
        }
        H[k] = h;
        Htau[k] = ht;
    }
}

/* Componentwise magnitude scales of the same sums (sum of |term|). */
static void scale_one(const ora_sys* s, const cplx* y, double tau,
                      double* SH, double* SHy, double* SHtau) {
    const int n = s->n;
    cplx yinv[ORA_NMAX];
    for (int j = 0; j < n; ++j) yinv[j] = 1.0 / y[j];
    for (int k = 0; k < n; ++k) {
        double h = 0.0, ht = 0.0;
        for (int j = 0; j < n; ++j) SHy[k * n + j] = 0.0;
        for (int i = 0; i < s->msz[k]; ++i) {
            const int idx = s->off[k] + i;
            const int32_t* a = s->exps + (size_t)idx * n;
            const double sexp = (double)s->texp[idx] / (double)s->D;
            const double ts = exp(sexp * tau);
            const double c = cabs(coef_at(s, idx));
            const double mono = cabs(powprod(n, y, yinv, a, -1));
            h += c * mono * ts;
            ht += c * fabs(sexp) * mono * ts;
            for (int j = 0; j < n; ++j) {
                if (a[j] == 0) continue;
                SHy[k * n + j] += c * fabs((double)a[j]) * cabs(powprod(n, y, yinv, a, j)) * ts;
            }
        }
        SH[k] = h;
        SHtau[k] = ht;
    }
}

static inline double abs2(cplx z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

/* Gaussian elimination with partial pivoting (pivot = largest |.|^2, ties to
 * the lowest row) on A (n x n, row-major, overwritten) with nrhs right-hand
 * sides B (n x nrhs, row-major, overwritten by the solution).
 * Returns 0, or 1 when a pivot is exactly zero. */
static int lu_solve(int n, cplx* A, cplx* B, int nrhs) {
    for (int j = 0; j < n; ++j) {
        int piv = j;
        double best = abs2(A[j * n + j]);
        for (int i = j + 1; i < n; ++i) {
            double v = abs2(A[i * n + j]);
            if (v > best) { best = v; piv = i; }
        }
        if (!(best > 0.0)) return 1;
        if (piv != j) {
            for (int c = 0; c < n; ++c) { cplx t = A[j * n + c]; A[j * n + c] = A[piv * n + c]; A[piv * n + c] = t; }
            for (int c = 0; c < nrhs; ++c) { cplx t = B[j * nrhs + c]; B[j * nrhs + c] = B[piv * nrhs + c]; B[piv * nrhs + c] = t; }
        }
        for (int i = j + 1; i < n; ++i) {
            cplx l = A[i * n + j] / A[j * n + j];
            A[i * n + j] = 0.0;
            for (int c = j + 1; c < n; ++c) A[i * n + c] -= l * A[j * n + c];
            for (int c = 0; c < nrhs; ++c) B[i * nrhs + c] -= l * B[j * nrhs + c];
        }
    }
    for (int j = n - 1; j >= 0; --j) {
        for (int c = 0; c < nrhs; ++c) {
            cplx acc = B[j * nrhs + c];
            for (int q = j + 1; q < n; ++q) acc -= A[j * n + q] * B[q * nrhs + c];
            B[j * nrhs + c] = acc / A[j * n + j];
        }
    }
    return 0;
}

static int all_finite(const cplx* v, int len) {
    for (int i = 0; i < len; ++i)
        if (!isfinite(creal(v[i])) || !isfinite(cimag(v[i]))) return 0;
    return 1;
}

static double inf_norm(const cplx* v, int n) {
    double m = 0.0;
    for (int j = 0; j < n; ++j) { double a = cabs(v[j]); if (a > m) m = a; }
    return m;
}

/* Euler and Newton directions at (y, tau): H_y [dE dN] = [-H_tau, -H].
 * Returns 0 on success, 1 when singular or not finite. */
static int directions(const ora_sys* s, const cplx* y, double tau, cplx* dE, cplx* dN) {
    const int n = s->n;
    cplx H[ORA_NMAX], Htau[ORA_NMAX], A[ORA_NMAX * ORA_NMAX], B[ORA_NMAX * 2];
    eval_one(s, y, tau, H, A, Htau);
    for (int k = 0; k < n; ++k) { B[2 * k] = -Htau[k]; B[2 * k + 1] = -H[k]; }
    if (!all_finite(A, n * n) || !all_finite(B, 2 * n)) return 1;
    if (lu_solve(n, A, B, 2)) return 1;
    for (int k = 0; k < n; ++k) { dE[k] = B[2 * k]; dN[k] = B[2 * k + 1]; }
    if (!all_finite(dE, n) || !all_finite(dN, n)) return 1;
    return 0;
}

/* Per-path tracker state (one path). */
typedef struct {
    cplx* y; double* tau; double* dtau; cplx* yacc; double* tauacc; cplx* dEacc;
    int32_t* status; int32_t* steps; int32_t* accepts; int32_t* rejects; int32_t* streak;
    cplx* yprev; double* tauprev; cplx* dEprev;   /* the accepted point before the last one */
    int32_t* hflag;   /* 1 while the pending prediction is a cubic Hermite one */
} ora_path;

/* The prediction at tau_acc + h.  Euler (Section 2.3): y_acc + h dE_acc.
 * Cubic Hermite (one of the predictors Section 2.3 names for the Euler
 * direction): the cubic p with p(tau0) = y0, p'(tau0) = d0, p(tau1) = y1,
 * p'(tau1) = d1 through the last two accepted points, evaluated at tau1 + h;
 * with s = (tau - tau0)/(tau1 - tau0) its basis is h00 = 2s^3 - 3s^2 + 1,
 * h10 = s^3 - 2s^2 + s, h01 = -2s^3 + 3s^2, h11 = s^3 - s^2 (the derivative
 * terms scaled by tau1 - tau0).  Used once two accepted points exist,
 * except for the Euler retry of a rejected cubic prediction (cubic = 0);
 * the flag records the choice. */
static void predict(int n, const ora_params* P, const ora_path* q, double h, int cubic, cplx* out) {
    const double d = *q->tauacc - (q->tauprev ? *q->tauprev : 0.0);
    if (q->hflag) *q->hflag = 0;
    if (cubic && P->predictor == 1 && *q->accepts >= 2 && d > 0.0) {
        *q->hflag = 1;
        const double s = 1.0 + h / d, s2 = s * s, s3 = s2 * s;
        const double h00 = 2 * s3 - 3 * s2 + 1, h10 = s3 - 2 * s2 + s, h01 = -2 * s3 + 3 * s2, h11 = s3 - s2;
        for (int j = 0; j < n; ++j)
            out[j] = h00 * q->yprev[j] + h10 * d * q->dEprev[j] + h01 * q->yacc[j] + h11 * d * q->dEacc[j];
        return;
    }
    for (int j = 0; j < n; ++j) out[j] = q->yacc[j] + h * q->dEacc[j];
}

/* One Euler-Newton step (Section 8: one Euler prediction, one Newton
 * iteration) with step-size control.  The state holds the predicted point y
 * at tau and the last accepted point.  One evaluation and one factorisation
 * at y give the Newton correction dN and the Euler direction dE together. */
static void step_one(const ora_sys* s, const ora_params* P, ora_path* q) {
    const int n = s->n;
    if (*q->status != ORA_ACTIVE) return;
    cplx dE[ORA_NMAX], dN[ORA_NMAX];
    int bad = directions(s, q->y, *q->tau, dE, dN);
    *q->steps += 1;
    int accept = 0, retry = 0;
    if (!bad) {
        double err = inf_norm(dN, n) / fmax(1.0, inf_norm(q->y, n));
        accept = err <= P->tol_accept;
    }
    if (accept) {
        if (P->predictor == 1 && *q->accepts >= 1) {   /* keep the accepted point being replaced */
            for (int j = 0; j < n; ++j) { q->yprev[j] = q->yacc[j]; q->dEprev[j] = q->dEacc[j]; }
            *q->tauprev = *q->tauacc;
        }
        for (int j = 0; j < n; ++j) { q->yacc[j] = q->y[j] + dN[j]; q->dEacc[j] = dE[j]; }
        *q->tauacc = *q->tau;
        *q->accepts += 1;
        *q->streak += 1;
        if (*q->tauacc == 0.0) { *q->status = ORA_CONVERGED; return; }
        for (int j = 0; j < n; ++j) {
            double a = cabs(q->yacc[j]);
            if (!(a < P->div_bound) || !(a > 1.0 / P->div_bound)) { *q->status = ORA_DIVERGED; return; }
        }
        if (*q->streak >= P->grow_after) {
            *q->dtau = fmin(*q->dtau * P->grow, P->dtau_max);
            *q->streak = 0;
        }
    } else {
        *q->rejects += 1;
        *q->streak = 0;
        if (*q->accepts == 0) {
            /* No accepted point yet: keep correcting at the start parameter. */
            if (bad) { *q->status = ORA_SINGULAR; return; }
            for (int j = 0; j < n; ++j) { q->y[j] += dN[j]; q->yacc[j] = q->y[j]; }
            if (*q->steps >= P->max_steps) *q->status = ORA_MAX_STEPS;
            return;
        }
        /* a rejected cubic prediction is retried with Euler at the same step
         * size; a rejected Euler prediction shrinks the step */
        retry = P->predictor == 1 && q->hflag && *q->hflag;
        if (!retry) {
            *q->dtau *= P->shrink;
            if (*q->dtau < P->dtau_min) { *q->status = ORA_UNDERFLOW; return; }
        }
    }
    double h = fmin(*q->dtau, -*q->tauacc);
    predict(n, P, q, h, !retry, q->y);
    *q->tau = *q->tauacc + h;
    if (*q->steps >= P->max_steps) *q->status = ORA_MAX_STEPS;
}

/* Newton's method at t = 1 (tau = 0) until the relative correction is below
 * polish_tol or polish_iters corrections were made.  Returns the last relative
 * correction size. */
static double polish_one(const ora_sys* s, const ora_params* P, cplx* y) {
    const int n = s->n;
    cplx dE[ORA_NMAX], dN[ORA_NMAX];
    double err = INFINITY;
    for (int it = 0; it < P->polish_iters; ++it) {
        if (directions(s, y, 0.0, dE, dN)) return INFINITY;
        for (int j = 0; j < n; ++j) y[j] += dN[j];
        err = inf_norm(dN, n) / fmax(1.0, inf_norm(y, n));
        if (err <= P->polish_tol) break;
    }
    return err;
}

/* ------------------------------------------------------------------ API -- */

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

int ora_eval(const ora_sys* s, int64_t p, const double* y, const double* tau,
             double* H, double* Hy, double* Htau) {
    if (s->n < 1 || s->n > ORA_NMAX) return 1;
    const int n = s->n;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t q = 0; q < p; ++q)
        eval_one(s, (const cplx*)y + q * n, tau[q], (cplx*)H + q * n,
                 (cplx*)Hy + q * n * n, (cplx*)Htau + q * n);
    return 0;
}

int ora_scale(const ora_sys* s, int64_t p, const double* y, const double* tau,
              double* SH, double* SHy, double* SHtau) {
    if (s->n < 1 || s->n > ORA_NMAX) return 1;
    const int n = s->n;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t q = 0; q < p; ++q)
        scale_one(s, (const cplx*)y + q * n, tau[q], SH + q * n, SHy + q * n * n, SHtau + q * n);
    return 0;
}

/* Solve A X = B for a batch of p independent n x n systems with nrhs columns.
 * Returns the number of singular systems (their X is left as zero). */
int64_t ora_solve(int n, int nrhs, int64_t p, const double* A, const double* B, double* X) {
    if (n < 1 || n > ORA_NMAX || nrhs < 1 || nrhs > 4) return -1;
    int64_t nsing = 0;
#pragma omp parallel for reduction(+ : nsing) schedule(static)
    for (int64_t q = 0; q < p; ++q) {
        cplx a[ORA_NMAX * ORA_NMAX], b[ORA_NMAX * 4];
        memcpy(a, (const cplx*)A + q * n * n, sizeof(cplx) * n * n);
        memcpy(b, (const cplx*)B + q * n * nrhs, sizeof(cplx) * n * nrhs);
        if (lu_solve(n, a, b, nrhs)) { memset(b, 0, sizeof(cplx) * n * nrhs); nsing++; }
        memcpy((cplx*)X + q * n * nrhs, b, sizeof(cplx) * n * nrhs);
    }
    return nsing;
}

/* Euler and Newton directions for p points; ok[q] = 1 when regular. */
int ora_directions(const ora_sys* s, int64_t p, const double* y, const double* tau,
                   double* dE, double* dN, int32_t* ok) {
    const int n = s->n;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t q = 0; q < p; ++q)
        ok[q] = !directions(s, (const cplx*)y + q * n, tau[q], (cplx*)dE + q * n, (cplx*)dN + q * n);
    return 0;
}

/* nsteps Euler-Newton steps for every path (structure-of-arrays state). */
int ora_step(const ora_sys* s, const ora_params* P, int64_t p, int32_t nsteps,
             double* y, double* tau, double* dtau, double* yacc, double* tauacc,
             double* dEacc, int32_t* status, int32_t* steps, int32_t* accepts,
             int32_t* rejects, int32_t* streak, double* yprev, double* tauprev, double* dEprev,
             int32_t* hflag) {
    const int n = s->n;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < p; ++q) {
        ora_path st = {(cplx*)y + q * n, tau + q, dtau + q, (cplx*)yacc + q * n, tauacc + q,
                       (cplx*)dEacc + q * n, status + q, steps + q, accepts + q, rejects + q,
                       streak + q, (cplx*)yprev + q * n, tauprev + q, (cplx*)dEprev + q * n, hflag + q};
        for (int r = 0; r < nsteps; ++r) step_one(s, P, &st);
    }
    return 0;
}

/* Track every path from y0 at tau0 to tau = 0, then polish converged paths.
 * Outputs x (p x n), status, steps, and the final polish correction size. */
int ora_track(const ora_sys* s, const ora_params* P, int64_t p, const double* y0,
              double tau0, double* x, int32_t* status_out, int32_t* steps_out,
              double* polish_err) {
    const int n = s->n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < p; ++q) {
        cplx y[ORA_NMAX], yacc[ORA_NMAX], dEacc[ORA_NMAX], yprev[ORA_NMAX], dEprev[ORA_NMAX];
        double tau = tau0, dtau = P->dtau_init, tauacc = tau0, tauprev = tau0;
        int32_t hflag = 0;
        int32_t st = ORA_ACTIVE, steps = 0, acc = 0, rej = 0, streak = 0;
        memcpy(y, (const cplx*)y0 + q * n, sizeof(cplx) * n);
        memcpy(yacc, y, sizeof(cplx) * n);
        for (int j = 0; j < n; ++j) dEacc[j] = 0.0;
        ora_path ps = {y, &tau, &dtau, yacc, &tauacc, dEacc, &st, &steps, &acc, &rej, &streak,
                       yprev, &tauprev, dEprev, &hflag};
        while (st == ORA_ACTIVE) step_one(s, P, &ps);
        double perr = NAN;
        if (st == ORA_CONVERGED) perr = polish_one(s, P, yacc);
        memcpy((cplx*)x + q * n, yacc, sizeof(cplx) * n);
        status_out[q] = st;
        steps_out[q] = steps;
        polish_err[q] = perr;
    }
    return 0;
}

/* Newton polish at t = 1 of p points in place. */
int ora_polish(const ora_sys* s, const ora_params* P, int64_t p, double* y, double* err) {
    const int n = s->n;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < p; ++q) err[q] = polish_one(s, P, (cplx*)y + q * n);
    return 0;
}

/* Adjoint (implicit-function) gradient of a real loss L(x) over p solutions
 * x of F(x; c) = 0 at t = 1, given gx = dL/dRe x + i dL/dIm x.  With J = F_x,
 * J^H lambda = gx and dF_k/dc_{k,i} = x^{a_{k,i}}, the gradient is
 * gc_{k,i} = -sum_paths lambda_k conj(x^{a_{k,i}}).  Paths are summed in
 * order.  Returns the number of singular Jacobians (skipped). */
int64_t ora_adjoint(const ora_sys* s, int64_t p, const double* x, const double* gx, double* gc) {
    const int n = s->n, M = s->M;
    cplx* contrib = (cplx*)calloc((size_t)p * M, sizeof(cplx));
    int32_t* sing = (int32_t*)calloc((size_t)p, sizeof(int32_t));
    if (!contrib || !sing) { free(contrib); free(sing); return -1; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < p; ++q) {
        const cplx* xq = (const cplx*)x + q * n;
        cplx H[ORA_NMAX], Htau[ORA_NMAX], J[ORA_NMAX * ORA_NMAX], JH[ORA_NMAX * ORA_NMAX], lam[ORA_NMAX], yinv[ORA_NMAX];
        eval_one(s, xq, 0.0, H, J, Htau);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) JH[a * n + b] = conj(J[b * n + a]);
        memcpy(lam, (const cplx*)gx + q * n, sizeof(cplx) * n);
        if (lu_solve(n, JH, lam, 1)) { sing[q] = 1; continue; }
        for (int j = 0; j < n; ++j) yinv[j] = 1.0 / xq[j];
        for (int k = 0; k < n; ++k)
            for (int i = 0; i < s->msz[k]; ++i) {
                int idx = s->off[k] + i;
                cplx mono = powprod(n, xq, yinv, s->exps + (size_t)idx * n, -1);
                contrib[(size_t)q * M + idx] = -lam[k] * conj(mono);
            }
    }
    int64_t nsing = 0;
    for (int i = 0; i < 2 * M; ++i) gc[i] = 0.0;
    for (int64_t q = 0; q < p; ++q) {
        nsing += sing[q];
        for (int i = 0; i < M; ++i) {
            gc[2 * i] += creal(contrib[(size_t)q * M + i]);
            gc[2 * i + 1] += cimag(contrib[(size_t)q * M + i]);
        }
    }
    free(contrib);
    free(sing);
    return nsing;
}
