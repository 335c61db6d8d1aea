/*
 * phc_oracle.c -- plain, slow, obviously-correct CPU path tracker.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the GPU library is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code with the GPU library.
 *
 * What it computes (paper: Verschelde, "A Blackbox Polynomial System Solver
 * on Parallel Shared Memory Computers"):
 *   - Section 2.1 / eq. (2): an embedded system E_D is solved by a homotopy;
 *     Section 5 names the Bezout bound, so the start system here is the
 *     total-degree one, g_i = x_i^{d_i} - 1, and the homotopy is
 *       H(x,t) = (1-t) * gamma * g(x) + t * f(x),  t from 0 to 1.
 *   - Section 3.1: a cascade stage k -> k-1 tracks the solutions of E_k with
 *     z_k != 0; hyperplane k keeps z_k and has the rest of its terms scaled
 *     by (1-t), so at t = 1 the slack z_k is zero and the system is E_{k-1}.
 *   - Section 1: paths are independent; the work crew model (threads popping
 *     jobs from a shared counter) runs them in parallel.
 *   - Section 1 / Section 5 (double double arithmetic): endpoints with a
 *     large condition number are refined by Newton's method in complex
 *     double double arithmetic.
 * The paper gives no predictor, corrector, step control or classification
 * rule; the readings used here (RK4 predictor, <= 3 Newton corrections,
 * halve/double step control, end Newton at t = 1, condition number and
 * residual tests) are stated next to each function and are the same
 * readings the GPU library implements, written independently.
 *
 * Style: complex double via C99 <complex.h>; every monomial and every
 * partial derivative is evaluated from scratch (no shared products); LU with
 * partial pivoting; compiled with -ffp-contract=off.
 *
 * Parity pins live in tests/ (Bezout counts, roots of unity, residuals,
 * companion-matrix and resultant roots, gamma invariance, cyclic symmetry,
 * Example 2.1 and Example 3.1 counts, double double against exact rationals).
 * The per-path step counts are pinned only where the step rules alone fix
 * them (a linear path, every step accepted, counted by hand); elsewhere they
 * and the path-to-root map are "parity unpinned": reported, never pinned.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- options */

/* Tracking options.  All values are readings (the paper fixes none). */
typedef struct {
    double h_init;          /* first step size in t                         */
    double h_max;           /* largest step size                            */
    double h_min;           /* a step below this stalls the path            */
    int32_t expand_after;   /* consecutive accepted steps before expanding  */
    double expand;          /* step multiplier after expand_after accepts   */
    double shrink;          /* step multiplier after a rejected step        */
    int32_t max_corr_iters; /* Newton corrections per step                  */
    double corr_tol;        /* converged: ||dx|| <= corr_tol (1 + ||x||)    */
    double corr_contract;   /* rejected: ||dx_j|| > corr_contract ||dx_j-1|| */
    int32_t max_steps;      /* accepted + rejected steps per path           */
    int32_t max_steps_decade; /* steps without crossing a decade of 1-t: stalled */
    double diverge_norm;    /* ||x|| above this during tracking: at infinity */
    double endpoint_inf_norm; /* endpoint with ||x|| above this: at infinity  */
    double end_zone;        /* stalled before this t: failed                 */
    double growth_inf;      /* stalled and ||x|| grew by more than growth_inf
                               per decade of 1-t: at infinity (a ratio)       */
    int32_t end_iters;      /* Newton iterations at t = 1                    */
    double end_tol;         /* end Newton stops at ||dx|| <= end_tol(1+||x||) */
    double cond_regular;    /* regular needs cond <= cond_regular (see end_measures) */
    double res_regular;     /* regular needs relative residual <= this        */
    double slack_tol;       /* slack zero: |z| <= slack_tol (1 + ||x||)       */
} orc_opts;

void orc_default_opts(orc_opts *o)
{
    o->h_init = 0.01;
    o->h_max = 0.1;
    o->h_min = 1e-14;
    o->expand_after = 3;
    o->expand = 2.0;
    o->shrink = 0.5;
    o->max_corr_iters = 3;
    o->corr_tol = 1e-9;
    o->corr_contract = 0.5;
    o->max_steps = 20000;
    o->max_steps_decade = 300;
    o->diverge_norm = 1e6;
    o->endpoint_inf_norm = 1e4;
    o->end_zone = 0.9;
    o->growth_inf = 1.1220184543019633; /* 10^0.05 */
    o->end_iters = 8;
    o->end_tol = 1e-13;
    o->cond_regular = 1e6;
    o->res_regular = 1e-12;
    o->slack_tol = 1e-8;
}

enum { ORC_REGULAR = 0, ORC_SINGULAR = 1, ORC_AT_INFINITY = 2, ORC_FAILED = 3 };

/* ---------------------------------------------------------------- homotopy */

/* A homotopy on n unknowns.  kind 0: total-degree homotopy with target f,
 * start g_i = x_i^{deg_i} - 1 and constant gamma.  kind 1: cascade stage on
 * the embedded system f = E_k; equation `row` is hyperplane k and variable
 * `slack` is z_k.  kind 2: coefficient-parameter homotopy
 * (1-t) gamma g(x) + t f(x) where g has the supports of f and the
 * coefficients coefs0 (Section 2.3: the solutions of a random coefficient
 * system start the paths to the target system).  kind 3: polyhedral
 * homotopy of one mixed cell (Section 2.2): the term c x^a of f carries
 * the factor t^{p}, p = powers[term] (0 on the cell's two terms per
 * equation, >= 1 elsewhere), so at t = 0 only the cell's binomial system
 * remains and at t = 1 the system is f. */
typedef struct {
    int32_t kind;
    int32_t n;
    int32_t n_terms;
    const int32_t *terms_per_eq; /* [n]                  */
    const uint8_t *exps;         /* [n_terms][n]         */
    const double *coefs;         /* [n_terms][2] re, im  */
    double gamma_re, gamma_im;   /* kinds 0 and 2        */
    int32_t row, slack;          /* kind 1               */
    const double *coefs0;        /* kind 2: [n_terms][2] coefficients of g */
    const double *powers;        /* kind 3: [n_terms] power of t per term  */
} orc_homotopy;

typedef struct {
    double t;             /* last t reached            */
    double h;             /* last step size            */
    double cond;          /* condition number of the endpoint (end_measures) */
    double relres;        /* relative residual at t=1  */
    double norm_x;        /* max-norm of the endpoint  */
    int32_t n_accept;     /* accepted steps            */
    int32_t n_reject;     /* rejected steps            */
    int32_t n_newton;     /* corrector + end Newton iterations */
    int32_t n_solve;      /* evaluate + factor + solve units   */
    int32_t cls;          /* class code                */
    int32_t stop;         /* 0 reached t=1, 1 diverged, 2 stalled (h), 3 budget, 4 non-finite */
    double growth;        /* log10 growth of ||x|| per decade of 1-t over the last checkpoints */
} orc_stats;

static cplx coef_of(const orc_homotopy *h, int k)
{
    return h->coefs[2 * k] + I * h->coefs[2 * k + 1];
}

/* |z|_1 = |Re z| + |Im z|; all norms of vectors use max_j max(|Re|,|Im|). */
static double abs1(cplx z) { return fabs(creal(z)) + fabs(cimag(z)); }
static double absinf(cplx z) { double a = fabs(creal(z)), b = fabs(cimag(z)); return a > b ? a : b; }

static double vnorm(int n, const cplx *v)
{
    double m = 0.0;
    for (int j = 0; j < n; j++) {
        double a = absinf(v[j]);
        if (!(a <= m)) m = a; /* NaN propagates */
    }
    return m;
}

static cplx ipow(cplx x, int e)
{
    cplx r = 1.0;
    for (int k = 0; k < e; k++) r = r * x;
    return r;
}

/* Monomial value x^a, from scratch. */
static cplx monomial(int n, const uint8_t *a, const cplx *x)
{
    cplx v = 1.0;
    for (int j = 0; j < n; j++) v = v * ipow(x[j], a[j]);
    return v;
}

/* d/dx_j of x^a, from scratch: a_j x_j^{a_j-1} prod_{i != j} x_i^{a_i}. */
static cplx monomial_dx(int n, const uint8_t *a, const cplx *x, int j)
{
    if (a[j] == 0) return 0.0;
    cplx v = (double)a[j] * ipow(x[j], a[j] - 1);
    for (int i = 0; i < n; i++)
        if (i != j) v = v * ipow(x[i], a[i]);
    return v;
}

/* Degree of equation i of the target system. */
static int eq_degree(const orc_homotopy *h, int i, int off)
{
    int d = 0;
    for (int k = 0; k < h->terms_per_eq[i]; k++) {
        int s = 0;
        for (int j = 0; j < h->n; j++) s += h->exps[(size_t)(off + k) * h->n + j];
        if (s > d) d = s;
    }
    return d;
}

static int is_unit(const uint8_t *a, int n, int j)
{
    for (int i = 0; i < n; i++)
        if (a[i] != (i == j ? 1 : 0)) return 0;
    return 1;
}

/* H(x,t), H_x(x,t) (row-major n x n, may be NULL), H_t(x,t) (may be NULL),
 * scale_i = sum over the terms of equation i of |c_i(t)|_1 |x^a|_1 (may be
 * NULL), where c_i(t) is the term's coefficient in H at this t. */
static void eval_homotopy(const orc_homotopy *h, const cplx *x, double t, cplx *H, cplx *Hx, cplx *Ht,
                          double *scale)
{
    const int n = h->n;
    const cplx gamma = h->gamma_re + I * h->gamma_im;
    int off = 0;
    for (int i = 0; i < n; i++) {
        cplx f = 0.0, ft = 0.0;
        double sc = 0.0;
        if (Hx)
            for (int j = 0; j < n; j++) Hx[i * n + j] = 0.0;
        for (int k = 0; k < h->terms_per_eq[i]; k++) {
            const uint8_t *a = h->exps + (size_t)(off + k) * n;
            cplx c = coef_of(h, off + k);
            cplx m = monomial(n, a, x);
            /* coefficient of this term in H at t, and its t-derivative */
            cplx ct, dct;
            if (h->kind == 0) {
                ct = t * c;
                dct = c;
            } else if (h->kind == 2) {
                const cplx c0 = h->coefs0[2 * (off + k)] + I * h->coefs0[2 * (off + k) + 1];
                ct = (1.0 - t) * gamma * c0 + t * c;
                dct = c - gamma * c0;
            } else if (h->kind == 3) {
                /* c t^p and d/dt = c p t^{p-1}, with 0^0 = 1; p >= 1 when p != 0 */
                const double p = h->powers[off + k];
                if (p == 0.0) {
                    ct = c;
                    dct = 0.0;
                } else if (t == 0.0) {
                    ct = 0.0;
                    dct = p == 1.0 ? c : 0.0;
                } else {
                    ct = c * pow(t, p);
                    dct = c * (p * pow(t, p - 1.0));
                }
            } else if (i == h->row && !is_unit(a, n, h->slack)) {
                ct = (1.0 - t) * c;
                dct = -c;
            } else {
                ct = c;
                dct = 0.0;
            }
            f += ct * m;
            ft += dct * m;
            sc += abs1(ct) * abs1(m);
            if (Hx)
                for (int j = 0; j < n; j++) Hx[i * n + j] += ct * monomial_dx(n, a, x, j);
        }
        if (h->kind == 0) {
            /* start system g_i = x_i^{d_i} - 1, weighted by (1-t) gamma */
            int d = eq_degree(h, i, off);
            cplx g = ipow(x[i], d) - 1.0;
            cplx w = (1.0 - t) * gamma;
            f += w * g;
            ft -= gamma * g;
            sc += abs1(w) * (abs1(ipow(x[i], d)) + 1.0);
            if (Hx) Hx[i * n + i] += w * (double)d * ipow(x[i], d - 1);
        }
        H[i] = f;
        if (Ht) Ht[i] = ft;
        if (scale) scale[i] = sc;
        off += h->terms_per_eq[i];
    }
}

/* ---------------------------------------------------------------- linear algebra */

/* LU with partial pivoting of the n x n row-major A (overwritten), pivot by
 * the largest |.|_1, the first row on ties.  Returns 0, or -1 when a pivot is
 * exactly zero. */
static int lu_factor(int n, cplx *A, int *piv)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = abs1(A[k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = abs1(A[i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(best > 0.0)) return -1;
        if (p != k)
            for (int j = 0; j < n; j++) { cplx s = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = s; }
        for (int i = k + 1; i < n; i++) {
            cplx l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (int j = k + 1; j < n; j++) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}

/* Solve with the factors of lu_factor: b is overwritten by the solution. */
static void lu_solve(int n, const cplx *LU, const int *piv, cplx *b)
{
    for (int k = 0; k < n; k++)
        if (piv[k] != k) { cplx s = b[k]; b[k] = b[piv[k]]; b[piv[k]] = s; }
    for (int i = 1; i < n; i++)
        for (int j = 0; j < i; j++) b[i] -= LU[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; i--) {
        for (int j = i + 1; j < n; j++) b[i] -= LU[i * n + j] * b[j];
        b[i] = b[i] / LU[i * n + i];
    }
}

/* Exported for tests: solve A x = b (A row-major, unchanged). Returns -1 if singular. */
int orc_lu_solve(int n, const double *A_ri, const double *b_ri, double *x_ri)
{
    cplx A[32 * 32], b[32];
    int piv[32];
    if (n < 1 || n > 32) return -2;
    for (int k = 0; k < n * n; k++) A[k] = A_ri[2 * k] + I * A_ri[2 * k + 1];
    for (int k = 0; k < n; k++) b[k] = b_ri[2 * k] + I * b_ri[2 * k + 1];
    if (lu_factor(n, A, piv)) return -1;
    lu_solve(n, A, piv, b);
    for (int k = 0; k < n; k++) { x_ri[2 * k] = creal(b[k]); x_ri[2 * k + 1] = cimag(b[k]); }
    return 0;
}

/* Exported for tests: H, H_x, H_t at (x, t); arrays as interleaved re,im. */
int orc_eval(const orc_homotopy *h, const double *x_ri, double t, double *H_ri, double *Hx_ri, double *Ht_ri)
{
    enum { NM = 32 };
    cplx x[NM], H[NM], Hx[NM * NM], Ht[NM];
    int n = h->n;
    if (n < 1 || n > NM) return -2;
    for (int j = 0; j < n; j++) x[j] = x_ri[2 * j] + I * x_ri[2 * j + 1];
    eval_homotopy(h, x, t, H, Hx, Ht, NULL);
    for (int j = 0; j < n; j++) {
        H_ri[2 * j] = creal(H[j]); H_ri[2 * j + 1] = cimag(H[j]);
        Ht_ri[2 * j] = creal(Ht[j]); Ht_ri[2 * j + 1] = cimag(Ht[j]);
    }
    for (int k = 0; k < n * n; k++) { Hx_ri[2 * k] = creal(Hx[k]); Hx_ri[2 * k + 1] = cimag(Hx[k]); }
    return 0;
}

/* ---------------------------------------------------------------- tracking */

#define NMAX 32

/* Davidenko field v(x,t) = -H_x(x,t)^{-1} H_t(x,t).  Returns -1 if singular. */
static int tangent(const orc_homotopy *h, const cplx *x, double t, cplx *v, orc_stats *st)
{
    cplx H[NMAX], Hx[NMAX * NMAX];
    int piv[NMAX];
    eval_homotopy(h, x, t, H, Hx, v, NULL);
    st->n_solve++;
    if (lu_factor(h->n, Hx, piv)) return -1;
    lu_solve(h->n, Hx, piv, v);
    for (int j = 0; j < h->n; j++) v[j] = -v[j];
    return 0;
}

/* One Newton step at fixed t: dx = -H_x^{-1} H, x += dx.  Returns ||dx||, or
 * NAN when H_x is singular. */
static double newton_step(const orc_homotopy *h, cplx *x, double t, orc_stats *st)
{
    cplx H[NMAX], Hx[NMAX * NMAX];
    int piv[NMAX];
    eval_homotopy(h, x, t, H, Hx, NULL, NULL);
    st->n_solve++;
    st->n_newton++;
    if (lu_factor(h->n, Hx, piv)) return NAN;
    lu_solve(h->n, Hx, piv, H);
    for (int j = 0; j < h->n; j++) x[j] -= H[j];
    return vnorm(h->n, H);
}

static int all_finite(int n, const cplx *x)
{
    for (int j = 0; j < n; j++)
        if (!isfinite(creal(x[j])) || !isfinite(cimag(x[j]))) return 0;
    return 1;
}

/* Condition number of the endpoint as a root of H(.,1), and its relative
 * residual.  With J = H_x(x,1) and s_i = 1 + scale_i,
 *   cond   = max_j sum_i |(J^{-1})_{ji}|_1 s_i / (1 + ||x||)
 * bounds the relative change of x under relative changes of the
 * coefficients (J^{-1} from the LU, one column per unit vector);
 *   relres = max_i |H_i(x,1)|_1 / s_i. */
static void end_measures(const orc_homotopy *h, const cplx *x, double *cond, double *relres)
{
    const int n = h->n;
    cplx H[NMAX], Hx[NMAX * NMAX], col[NMAX];
    double scale[NMAX], rowacc[NMAX];
    int piv[NMAX];
    eval_homotopy(h, x, 1.0, H, Hx, NULL, scale);
    double rr = 0.0;
    for (int i = 0; i < n; i++) {
        double r = abs1(H[i]) / (1.0 + scale[i]);
        if (!(r <= rr)) rr = r;
    }
    *relres = rr;
    if (lu_factor(n, Hx, piv)) { *cond = INFINITY; return; }
    for (int j = 0; j < n; j++) rowacc[j] = 0.0;
    for (int i = 0; i < n; i++) {
        for (int q = 0; q < n; q++) col[q] = (q == i) ? 1.0 : 0.0;
        lu_solve(n, Hx, piv, col);
        for (int j = 0; j < n; j++) rowacc[j] += abs1(col[j]) * (1.0 + scale[i]);
    }
    double m = 0.0;
    for (int j = 0; j < n; j++)
        if (!(rowacc[j] <= m)) m = rowacc[j];
    *cond = m / (1.0 + vnorm(n, x));
    if (!isfinite(*cond)) *cond = INFINITY;
}

/* Exported for tests: cond and relres of end_measures at the point x. */
int orc_end_measures(const orc_homotopy *h, const double *x_ri, double *cond, double *relres)
{
    cplx x[NMAX];
    if (h->n < 1 || h->n > NMAX) return -2;
    for (int j = 0; j < h->n; j++) x[j] = x_ri[2 * j] + I * x_ri[2 * j + 1];
    end_measures(h, x, cond, relres);
    return 0;
}

/* Track one path from (x, t=0) to t = 1 and classify its endpoint.
 *
 * Predictor: classical fourth-order Runge-Kutta on dx/dt = v(x,t).
 * Corrector: at most max_corr_iters Newton steps at t + h; converged when
 *   ||dx|| <= corr_tol (1 + ||x||), rejected when a correction fails to
 *   contract by corr_contract or none converges.
 * Step control: the step is clamped to land on t = 1; after expand_after
 *   consecutive accepts it grows by `expand` (at most h_max), a rejection
 *   multiplies it by `shrink`.
 * Stop: t = 1; ||x|| > diverge_norm (at infinity; for a polyhedral path
 *   diverge_norm * max(1, ||x(0)||)); h < h_min, max_steps, or
 *   max_steps_decade steps without 1-t crossing a power of ten (stalled);
 *   non-finite values (failed).
 * End (only for paths that reached t = 1): Newton at t = 1 (<= end_iters),
 *   then the condition number and the relative residual; REGULAR when both
 *   are small.
 * Every endpoint with ||x|| > endpoint_inf_norm is AT_INFINITY.
 * A stalled path is never REGULAR: it is AT_INFINITY when ||x|| > endpoint_inf_norm
 *   or when ||x|| grew by more than growth_inf per decade of 1-t over its last
 *   (at most four) decade checkpoints, FAILED when it stalled before end_zone,
 *   SINGULAR otherwise. */
static void track_one(const orc_homotopy *h, const orc_opts *o, cplx *x, orc_stats *st)
{
    const int n = h->n;
    cplx x0[NMAX], xs[NMAX], k1[NMAX], k2[NMAX], k3[NMAX], k4[NMAX];
    double t = 0.0, step = o->h_init;
    /* divergence bound; a polyhedral path starts at a solution of its cell's
       binomial system in the scaled coordinates, whose norm may already
       exceed diverge_norm: its bound is diverge_norm * max(1, ||x(0)||) */
    double div_bound = o->diverge_norm;
    if (h->kind == 3) {
        const double s0 = vnorm(n, x);
        div_bound = o->diverge_norm * (s0 > 1.0 ? s0 : 1.0);
    }
    int streak = 0, steps = 0;
    /* decade checkpoints: ||x|| at the first accepted t with 1-t <= 10^-k;
       the last five are kept (ring), nck counts all of them */
    double ck[5];
    int nck = 0;
    double next_s = 0.1;
    int since_ck = 0; /* steps since the last decade checkpoint (or the start) */
    memset(st, 0, sizeof *st);
    st->stop = 0;

    while (t < 1.0) {
        double he = step;
        double t1 = t + he;
        if (he >= 1.0 - t) { he = 1.0 - t; t1 = 1.0; }
        memcpy(x0, x, sizeof(cplx) * n);

        /* predictor: RK4 */
        int ok = 1;
        ok = ok && !tangent(h, x0, t, k1, st);
        for (int j = 0; j < n; j++) xs[j] = x0[j] + (0.5 * he) * k1[j];
        ok = ok && !tangent(h, xs, t + 0.5 * he, k2, st);
        for (int j = 0; j < n; j++) xs[j] = x0[j] + (0.5 * he) * k2[j];
        ok = ok && !tangent(h, xs, t + 0.5 * he, k3, st);
        for (int j = 0; j < n; j++) xs[j] = x0[j] + he * k3[j];
        ok = ok && !tangent(h, xs, t1, k4, st);
        if (ok)
            for (int j = 0; j < n; j++) x[j] = x0[j] + (he / 6.0) * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);

        /* corrector: Newton at t1 */
        int conv = 0;
        double prev = INFINITY;
        for (int it = 0; ok && it < o->max_corr_iters; it++) {
            double d = newton_step(h, x, t1, st);
            if (!(d == d) || !all_finite(n, x)) break;
            if (d <= o->corr_tol * (1.0 + vnorm(n, x))) { conv = 1; break; }
            if (it > 0 && d > o->corr_contract * prev) break;
            prev = d;
        }

        steps++;
        if (conv) {
            t = t1;
            st->n_accept++;
            while (1.0 - t <= next_s && next_s > 0.0) {
                ck[nck % 5] = vnorm(n, x);
                nck++;
                since_ck = 0;
                next_s *= 0.1;
                if (nck >= 40) next_s = 0.0;
            }
            if (vnorm(n, x) > div_bound) { st->stop = 1; break; }
            if (++streak >= o->expand_after) {
                streak = 0;
                step = step * o->expand;
                if (step > o->h_max) step = o->h_max;
            }
        } else {
            memcpy(x, x0, sizeof(cplx) * n);
            st->n_reject++;
            streak = 0;
            step = he * o->shrink;
            if (step < o->h_min) { st->stop = 2; break; }
        }
        if (steps >= o->max_steps) { st->stop = 3; break; }
        if (++since_ck >= o->max_steps_decade && t < 1.0) { st->stop = 3; break; }
    }
    st->t = t;
    st->h = step;

    /* growth over the last m <= 4 decades: ||x|| at checkpoint l against
       checkpoint l-m, compared with growth_inf^m */
    int grew = 0;
    st->growth = 0.0;
    if (nck >= 2) {
        int l = nck - 1, m = l < 4 ? l : 4;
        double a = ck[l % 5], b = ck[(l - m) % 5], g = 1.0;
        for (int k = 0; k < m; k++) g *= o->growth_inf;
        grew = a > b * g;
        st->growth = log10(a / b) / m;
    }

    /* classification at the end of the path */
    if (!all_finite(n, x)) { st->stop = 4; st->cls = ORC_FAILED; st->norm_x = NAN; st->cond = NAN; st->relres = NAN; return; }
    st->norm_x = vnorm(n, x);
    if (st->stop == 1) { st->cls = ORC_AT_INFINITY; st->cond = INFINITY; st->relres = NAN; return; }
    if (st->stop != 0) {
        /* stalled before t = 1: never regular */
        end_measures(h, x, &st->cond, &st->relres);
        if (st->norm_x > o->endpoint_inf_norm || (t >= o->end_zone && grew)) st->cls = ORC_AT_INFINITY;
        else if (t < o->end_zone) st->cls = ORC_FAILED;
        else st->cls = ORC_SINGULAR;
        return;
    }
    /* reached t = 1: end Newton */
    for (int it = 0; it < o->end_iters; it++) {
        double d = newton_step(h, x, 1.0, st);
        if (!(d == d) || !all_finite(n, x)) break;
        if (d <= o->end_tol * (1.0 + vnorm(n, x))) break;
    }
    if (!all_finite(n, x)) { st->stop = 4; st->cls = ORC_FAILED; st->norm_x = NAN; st->cond = NAN; st->relres = NAN; return; }
    st->norm_x = vnorm(n, x);
    end_measures(h, x, &st->cond, &st->relres);
    if (st->norm_x > o->endpoint_inf_norm) st->cls = ORC_AT_INFINITY;
    else if (st->cond <= o->cond_regular && st->relres <= o->res_regular) st->cls = ORC_REGULAR;
    else st->cls = ORC_SINGULAR;
}

/* Start solution of path p of the total-degree start system: the digits of
 * p in the mixed radix (d_1, ..., d_n), first variable fastest, select the
 * roots of unity x_i = exp(2 pi i k_i / d_i). */
static void start_solution(const orc_homotopy *h, int64_t p, cplx *x)
{
    int off = 0;
    for (int i = 0; i < h->n; i++) {
        int d = eq_degree(h, i, off);
        off += h->terms_per_eq[i];
        int k = (int)(p % d);
        p /= d;
        double a = 2.0 * M_PI * (double)k / (double)d;
        x[i] = cos(a) + I * sin(a);
    }
}

int64_t orc_num_paths(const orc_homotopy *h)
{
    int64_t P = 1;
    int off = 0;
    for (int i = 0; i < h->n; i++) {
        P *= eq_degree(h, i, off);
        off += h->terms_per_eq[i];
    }
    return P;
}

/* Work crew (Section 1): threads take the next path from a shared counter. */
typedef struct {
    const orc_homotopy *h;
    const orc_opts *o;
    const double *starts;  /* [n_paths][n][2] or NULL: total-degree starts */
    int64_t first, n_paths;
    double *x_out;         /* [n_paths][n][2] */
    int8_t *cls_out;
    orc_stats *stats_out;
    atomic_llong next;
} crew_t;

static void *crew_worker(void *arg)
{
    crew_t *c = (crew_t *)arg;
    const int n = c->h->n;
    cplx x[NMAX];
    orc_stats st;
    for (;;) {
        int64_t q = atomic_fetch_add(&c->next, 1);
        if (q >= c->n_paths) break;
        if (c->starts)
            for (int j = 0; j < n; j++) x[j] = c->starts[(q * n + j) * 2] + I * c->starts[(q * n + j) * 2 + 1];
        else
            start_solution(c->h, c->first + q, x);
        track_one(c->h, c->o, x, &st);
        for (int j = 0; j < n; j++) {
            c->x_out[(q * n + j) * 2] = creal(x[j]);
            c->x_out[(q * n + j) * 2 + 1] = cimag(x[j]);
        }
        if (c->cls_out) c->cls_out[q] = (int8_t)st.cls;
        if (c->stats_out) c->stats_out[q] = st;
    }
    return NULL;
}

/* Track n_paths paths with n_threads threads.  starts == NULL selects the
 * total-degree start solutions first .. first+n_paths-1 (kind 0 only). */
int orc_track(const orc_homotopy *h, const double *starts, int64_t first, int64_t n_paths, const orc_opts *o_in,
              int n_threads, double *x_out, int8_t *cls_out, orc_stats *stats_out)
{
    orc_opts o;
    if (o_in) o = *o_in; else orc_default_opts(&o);
    if (h->n < 1 || h->n > NMAX || n_paths < 0) return -1;
    if (!starts && h->kind != 0) return -1;
    crew_t c;
    c.h = h; c.o = &o; c.starts = starts; c.first = first; c.n_paths = n_paths;
    c.x_out = x_out; c.cls_out = cls_out; c.stats_out = stats_out;
    atomic_init(&c.next, 0);
    if (n_threads < 1) n_threads = 1;
    if (n_threads == 1) { crew_worker(&c); return 0; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    for (int k = 0; k < n_threads; k++) pthread_create(&th[k], NULL, crew_worker, &c);
    for (int k = 0; k < n_threads; k++) pthread_join(th[k], NULL);
    free(th);
    return 0;
}

/* Exported for tests: the total-degree start solution of path p. */
void orc_start_solution(const orc_homotopy *h, int64_t p, double *x_ri)
{
    cplx x[NMAX];
    start_solution(h, p, x);
    for (int j = 0; j < h->n; j++) { x_ri[2 * j] = creal(x[j]); x_ri[2 * j + 1] = cimag(x[j]); }
}

/* ================================================================ double double
 * Double double arithmetic after Hida, Li and Bailey (the paper's [HLB00]):
 * an unevaluated sum hi + lo with |lo| <= ulp(hi)/2.  Error-free transforms:
 * Knuth's TwoSum and Dekker's split/TwoProduct (no fused multiply-add). */

typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; } cdd;

static dd two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = { s, e };
    return r;
}

static dd quick_two_sum(double a, double b)
{
    double s = a + b;
    double e = b - (s - a);
    dd r = { s, e };
    return r;
}

static void split(double a, double *hi, double *lo)
{
    const double SPLITTER = 134217729.0; /* 2^27 + 1 */
    double t = SPLITTER * a;
    *hi = t - (t - a);
    *lo = a - *hi;
}

static dd two_prod(double a, double b)
{
    double p = a * b, ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    double e = ((ah * bh - p) + ah * bl + al * bh) + al * bl;
    dd r = { p, e };
    return r;
}

static dd dd_add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

static dd dd_neg(dd a) { dd r = { -a.hi, -a.lo }; return r; }
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

static dd dd_mul(dd a, dd b)
{
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}

static dd dd_div(dd a, dd b)
{
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul((dd){ q1, 0.0 }, b));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul((dd){ q2, 0.0 }, b));
    double q3 = r.hi / b.hi;
    dd q = quick_two_sum(q1, q2);
    return dd_add(q, (dd){ q3, 0.0 });
}

static dd dd_from(double a) { dd r = { a, 0.0 }; return r; }
static double dd_abs_approx(dd a) { return fabs(a.hi); }

/* exported for the exact-rational tests: out = {hi, lo} */
void orc_two_sum(double a, double b, double *out) { dd r = two_sum(a, b); out[0] = r.hi; out[1] = r.lo; }
void orc_two_prod(double a, double b, double *out) { dd r = two_prod(a, b); out[0] = r.hi; out[1] = r.lo; }
void orc_dd_add(const double *a, const double *b, double *out) { dd r = dd_add((dd){a[0], a[1]}, (dd){b[0], b[1]}); out[0] = r.hi; out[1] = r.lo; }
void orc_dd_mul(const double *a, const double *b, double *out) { dd r = dd_mul((dd){a[0], a[1]}, (dd){b[0], b[1]}); out[0] = r.hi; out[1] = r.lo; }
void orc_dd_div(const double *a, const double *b, double *out) { dd r = dd_div((dd){a[0], a[1]}, (dd){b[0], b[1]}); out[0] = r.hi; out[1] = r.lo; }

static cdd cdd_add(cdd a, cdd b) { cdd r = { dd_add(a.re, b.re), dd_add(a.im, b.im) }; return r; }
static cdd cdd_sub(cdd a, cdd b) { cdd r = { dd_sub(a.re, b.re), dd_sub(a.im, b.im) }; return r; }
static cdd cdd_mul(cdd a, cdd b)
{
    cdd r = { dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re)) };
    return r;
}
static cdd cdd_div(cdd a, cdd b)
{
    dd den = dd_add(dd_mul(b.re, b.re), dd_mul(b.im, b.im));
    cdd num = { dd_add(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_sub(dd_mul(a.im, b.re), dd_mul(a.re, b.im)) };
    cdd r = { dd_div(num.re, den), dd_div(num.im, den) };
    return r;
}
static cdd cdd_from(cplx z) { cdd r = { dd_from(creal(z)), dd_from(cimag(z)) }; return r; }
static double cdd_abs1(cdd a) { return dd_abs_approx(a.re) + dd_abs_approx(a.im); }
static double cdd_absinf(cdd a) { double x = fabs(a.re.hi), y = fabs(a.im.hi); return x > y ? x : y; }

static cdd cdd_ipow(cdd x, int e)
{
    cdd r = { dd_from(1.0), dd_from(0.0) };
    for (int k = 0; k < e; k++) r = cdd_mul(r, x);
    return r;
}

/* H(x,1) and H_x(x,1) in complex double double, from scratch per monomial. */
static void eval_end_dd(const orc_homotopy *h, const cdd *x, cdd *H, cdd *Hx)
{
    const int n = h->n;
    int off = 0;
    for (int i = 0; i < n; i++) {
        cdd f = cdd_from(0.0);
        for (int j = 0; j < n; j++) Hx[i * n + j] = cdd_from(0.0);
        for (int k = 0; k < h->terms_per_eq[i]; k++) {
            const uint8_t *a = h->exps + (size_t)(off + k) * n;
            cplx c = coef_of(h, off + k);
            /* coefficient at t = 1: kinds 0 and 2 keep c; kind 1 zeroes the scaled hyperplane terms */
            if (h->kind == 1 && i == h->row && !is_unit(a, n, h->slack)) continue;
            cdd cc = cdd_from(c);
            cdd m = cdd_from(1.0);
            for (int j = 0; j < n; j++) m = cdd_mul(m, cdd_ipow(x[j], a[j]));
            f = cdd_add(f, cdd_mul(cc, m));
            for (int j = 0; j < n; j++) {
                if (a[j] == 0) continue;
                cdd d = cdd_mul(cdd_from((double)a[j]), cdd_ipow(x[j], a[j] - 1));
                for (int q = 0; q < n; q++)
                    if (q != j) d = cdd_mul(d, cdd_ipow(x[q], a[q]));
                Hx[i * n + j] = cdd_add(Hx[i * n + j], cdd_mul(cc, d));
            }
        }
        H[i] = f;
        off += h->terms_per_eq[i];
    }
}

/* Solve A x = b in complex double double, partial pivoting by |.|_1. */
static int lu_solve_dd(int n, cdd *A, cdd *b)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = cdd_abs1(A[k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = cdd_abs1(A[i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        if (!(best > 0.0)) return -1;
        if (p != k) {
            for (int j = 0; j < n; j++) { cdd s = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = s; }
            cdd s = b[k]; b[k] = b[p]; b[p] = s;
        }
        for (int i = k + 1; i < n; i++) {
            cdd l = cdd_div(A[i * n + k], A[k * n + k]);
            for (int j = k + 1; j < n; j++) A[i * n + j] = cdd_sub(A[i * n + j], cdd_mul(l, A[k * n + j]));
            b[i] = cdd_sub(b[i], cdd_mul(l, b[k]));
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        for (int j = i + 1; j < n; j++) b[i] = cdd_sub(b[i], cdd_mul(A[i * n + j], b[j]));
        b[i] = cdd_div(b[i], A[i * n + i]);
    }
    return 0;
}

/* Refine one endpoint by Newton's method at t = 1 in complex double double.
 * x_hi (in/out) is the double part, x_lo (out) the low part.  Returns 1 when
 * a correction fell to ||dx|| <= 1e-20 (1 + ||x||) within max_iters. */
static int refine_one(const orc_homotopy *h, double *x_hi, double *x_lo, int max_iters)
{
    const int n = h->n;
    cdd x[NMAX], H[NMAX], Hx[NMAX * NMAX];
    for (int j = 0; j < n; j++) {
        x[j].re = dd_from(x_hi[2 * j]);
        x[j].im = dd_from(x_hi[2 * j + 1]);
    }
    int conv = 0;
    for (int it = 0; it < max_iters; it++) {
        eval_end_dd(h, x, H, Hx);
        if (lu_solve_dd(n, Hx, H)) break;
        double dn = 0.0, xn = 0.0;
        for (int j = 0; j < n; j++) {
            x[j] = cdd_sub(x[j], H[j]);
            double a = cdd_absinf(H[j]);
            if (!(a <= dn)) dn = a;
            double b = cdd_absinf(x[j]);
            if (b > xn) xn = b;
        }
        if (!(dn == dn)) break;
        if (dn <= 1e-20 * (1.0 + xn)) { conv = 1; break; }
    }
    for (int j = 0; j < n; j++) {
        x_hi[2 * j] = x[j].re.hi; x_lo[2 * j] = x[j].re.lo;
        x_hi[2 * j + 1] = x[j].im.hi; x_lo[2 * j + 1] = x[j].im.lo;
    }
    return conv;
}

/* Refine the endpoints that reached t = 1, whose class is SINGULAR or
 * REGULAR and whose cond is above cond_threshold: REGULAR when double double Newton converges and the
 * condition number at the refined point is at most cond_max, else SINGULAR.
 * x_hi [n_paths][n][2] in/out, x_lo out (zero for untouched endpoints),
 * cls in/out, cond in/out, reached[p] != 0 when path p reached t = 1. */
int orc_refine(const orc_homotopy *h, double *x_hi, double *x_lo, int64_t n_paths, double cond_threshold,
               double cond_max, int max_iters, int8_t *cls, double *cond, const int32_t *reached)
{
    const int n = h->n;
    for (int64_t p = 0; p < n_paths; p++) {
        double *xh = x_hi + (size_t)p * n * 2, *xl = x_lo + (size_t)p * n * 2;
        for (int j = 0; j < 2 * n; j++) xl[j] = 0.0;
        if (!(reached[p] && (cls[p] == ORC_SINGULAR || cls[p] == ORC_REGULAR) && cond[p] > cond_threshold)) continue;
        int conv = refine_one(h, xh, xl, max_iters);
        cplx x[NMAX];
        for (int j = 0; j < n; j++) x[j] = xh[2 * j] + I * xh[2 * j + 1];
        double c, r;
        end_measures(h, x, &c, &r);
        cond[p] = c;
        cls[p] = (conv && c <= cond_max) ? ORC_REGULAR : ORC_SINGULAR;
    }
    return 0;
}

/* ================================================================ Cauchy endgame
 * A path that converges to a singular endpoint x* of a total-degree
 * homotopy has near t = 1 an expansion x(s) = x* + sum_k a_k s^{k/c} in
 * s = 1 - t, c the cycle number.  The endgame tracks the path to
 * t0 = 1 - EG_RADIUS, then around the circle s = EG_RADIUS e^{i theta}
 * (complex t) until the path closes up after c loops, sampling x at
 * EG_SAMPLES equally spaced angles per loop; by Cauchy's integral formula
 * in the variable s^{1/c} the mean of the c * EG_SAMPLES samples is x*
 * (the trapezoidal rule, exact up to terms of order EG_RADIUS^EG_SAMPLES).
 * A path that runs to infinity closes up too (a pole in s), but the mean of
 * its samples is no root, so an estimate counts only when its relative
 * residual (end_measures) is at most EG_RES. */

#define EG_RADIUS 0.01
#define EG_SAMPLES 16
#define EG_MAX_CYCLES 8
#define EG_CLOSE_TOL 1e-8
#define EG_RES 1e-10

/* H, H_x, H_t of the total-degree homotopy at a complex t (as eval_homotopy). */
static void eval_homotopy_ct(const orc_homotopy *h, const cplx *x, cplx t, cplx *H, cplx *Hx, cplx *Ht)
{
    const int n = h->n;
    const cplx gamma = h->gamma_re + I * h->gamma_im;
    int off = 0;
    for (int i = 0; i < n; i++) {
        cplx f = 0.0, ft = 0.0;
        for (int j = 0; j < n; j++) Hx[i * n + j] = 0.0;
        for (int k = 0; k < h->terms_per_eq[i]; k++) {
            const uint8_t *a = h->exps + (size_t)(off + k) * n;
            cplx c = coef_of(h, off + k);
            cplx m = monomial(n, a, x);
            f += t * c * m;
            ft += c * m;
            for (int j = 0; j < n; j++) Hx[i * n + j] += t * c * monomial_dx(n, a, x, j);
        }
        int d = eq_degree(h, i, off);
        cplx g = ipow(x[i], d) - 1.0;
        cplx w = (1.0 - t) * gamma;
        f += w * g;
        ft -= gamma * g;
        Hx[i * n + i] += w * (double)d * ipow(x[i], d - 1);
        H[i] = f;
        Ht[i] = ft;
        off += h->terms_per_eq[i];
    }
}

/* dx/dtheta at (x, theta) on the circle t = 1 - r e^{i theta}:
 * -H_x^{-1} H_t dt/dtheta, dt/dtheta = -i r e^{i theta}. */
static int tangent_theta(const orc_homotopy *h, const cplx *x, double r, double th, cplx *v, orc_stats *st)
{
    cplx H[NMAX], Hx[NMAX * NMAX];
    int piv[NMAX];
    const cplx e = cos(th) + I * sin(th);
    eval_homotopy_ct(h, x, 1.0 - r * e, H, Hx, v);
    st->n_solve++;
    if (lu_factor(h->n, Hx, piv)) return -1;
    lu_solve(h->n, Hx, piv, v);
    const cplx dt = -I * r * e;
    for (int j = 0; j < h->n; j++) v[j] = -v[j] * dt;
    return 0;
}

static double newton_theta(const orc_homotopy *h, cplx *x, double r, double th, orc_stats *st)
{
    cplx H[NMAX], Hx[NMAX * NMAX], Ht[NMAX];
    int piv[NMAX];
    const cplx e = cos(th) + I * sin(th);
    eval_homotopy_ct(h, x, 1.0 - r * e, H, Hx, Ht);
    st->n_solve++;
    st->n_newton++;
    if (lu_factor(h->n, Hx, piv)) return NAN;
    lu_solve(h->n, Hx, piv, H);
    for (int j = 0; j < h->n; j++) x[j] -= H[j];
    return vnorm(h->n, H);
}

/* Tracks x from t = 0 to t0 = 1 - EG_RADIUS with the tracker's readings
 * (track_one, the step clamped to land on t0), then around the circle.
 * Returns the cycle number (0 when the path stopped before t0 or did not
 * close within EG_MAX_CYCLES loops); x holds the Cauchy estimate of the
 * endpoint (or the last point). */
static int endgame_one(const orc_homotopy *h, const orc_opts *o, cplx *x, orc_stats *st)
{
    const int n = h->n;
    const double t0 = 1.0 - EG_RADIUS;
    cplx x0[NMAX], xs[NMAX], k1[NMAX], k2[NMAX], k3[NMAX], k4[NMAX];
    double t = 0.0, step = o->h_init;
    int streak = 0, steps = 0;
    memset(st, 0, sizeof *st);
    /* ---- to t0 */
    while (t < t0) {
        double he = step;
        double t1 = t + he;
        if (he >= t0 - t) { he = t0 - t; t1 = t0; }
        memcpy(x0, x, sizeof(cplx) * n);
        int ok = 1;
        ok = ok && !tangent(h, x0, t, k1, st);
        for (int j = 0; j < n; j++) xs[j] = x0[j] + (0.5 * he) * k1[j];
        ok = ok && !tangent(h, xs, t + 0.5 * he, k2, st);
        for (int j = 0; j < n; j++) xs[j] = x0[j] + (0.5 * he) * k2[j];
        ok = ok && !tangent(h, xs, t + 0.5 * he, k3, st);
        for (int j = 0; j < n; j++) xs[j] = x0[j] + he * k3[j];
        ok = ok && !tangent(h, xs, t1, k4, st);
        if (ok)
            for (int j = 0; j < n; j++) x[j] = x0[j] + (he / 6.0) * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
        int conv = 0;
        double prev = INFINITY;
        for (int it = 0; ok && it < o->max_corr_iters; it++) {
            double d = newton_step(h, x, t1, st);
            if (!(d == d) || !all_finite(n, x)) break;
            if (d <= o->corr_tol * (1.0 + vnorm(n, x))) { conv = 1; break; }
            if (it > 0 && d > o->corr_contract * prev) break;
            prev = d;
        }
        steps++;
        if (conv) {
            t = t1;
            st->n_accept++;
            if (vnorm(n, x) > o->diverge_norm) { st->stop = 1; break; }
            if (++streak >= o->expand_after) {
                streak = 0;
                step = step * o->expand;
                if (step > o->h_max) step = o->h_max;
            }
        } else {
            memcpy(x, x0, sizeof(cplx) * n);
            st->n_reject++;
            streak = 0;
            step = he * o->shrink;
            if (step < o->h_min) { st->stop = 2; break; }
        }
        if (steps >= o->max_steps) { st->stop = 3; break; }
    }
    st->t = t;
    if (st->stop != 0 || t < t0) return 0;
    /* ---- around the circle s = r e^{i theta} */
    const double r = EG_RADIUS, dth = 2.0 * M_PI / EG_SAMPLES, hmin = dth * 9.5367431640625e-07; /* 2^-20 */
    cplx start[NMAX], sum[NMAX];
    memcpy(start, x, sizeof(cplx) * n);
    for (int j = 0; j < n; j++) sum[j] = 0.0;
    double th = 0.0, hth = dth;
    streak = 0;
    for (int sample = 1; sample <= EG_SAMPLES * EG_MAX_CYCLES; sample++) {
        for (int j = 0; j < n; j++) sum[j] += x[j];
        const double target = sample * dth;
        while (th < target) {
            double he = hth;
            double t1 = th + he;
            if (he >= target - th) { he = target - th; t1 = target; }
            memcpy(x0, x, sizeof(cplx) * n);
            int ok = 1;
            ok = ok && !tangent_theta(h, x0, r, th, k1, st);
            for (int j = 0; j < n; j++) xs[j] = x0[j] + (0.5 * he) * k1[j];
            ok = ok && !tangent_theta(h, xs, r, th + 0.5 * he, k2, st);
            for (int j = 0; j < n; j++) xs[j] = x0[j] + (0.5 * he) * k2[j];
            ok = ok && !tangent_theta(h, xs, r, th + 0.5 * he, k3, st);
            for (int j = 0; j < n; j++) xs[j] = x0[j] + he * k3[j];
            ok = ok && !tangent_theta(h, xs, r, t1, k4, st);
            if (ok)
                for (int j = 0; j < n; j++) x[j] = x0[j] + (he / 6.0) * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
            int conv = 0;
            double prev = INFINITY;
            for (int it = 0; ok && it < o->max_corr_iters; it++) {
                double d = newton_theta(h, x, r, t1, st);
                if (!(d == d) || !all_finite(n, x)) break;
                if (d <= o->corr_tol * (1.0 + vnorm(n, x))) { conv = 1; break; }
                if (it > 0 && d > o->corr_contract * prev) break;
                prev = d;
            }
            if (conv) {
                th = t1;
                st->n_accept++;
                if (++streak >= o->expand_after) {
                    streak = 0;
                    hth = hth * o->expand;
                    if (hth > dth) hth = dth;
                }
            } else {
                memcpy(x, x0, sizeof(cplx) * n);
                st->n_reject++;
                streak = 0;
                hth = he * o->shrink;
                if (hth < hmin) { st->stop = 2; return 0; }
            }
        }
        if (sample % EG_SAMPLES == 0) {
            cplx dx[NMAX];
            for (int j = 0; j < n; j++) dx[j] = x[j] - start[j];
            if (vnorm(n, dx) <= EG_CLOSE_TOL * (1.0 + vnorm(n, start))) {
                const int c = sample / EG_SAMPLES;
                for (int j = 0; j < n; j++) x[j] = sum[j] / (double)sample;
                st->t = 1.0;
                st->norm_x = vnorm(n, x);
                end_measures(h, x, &st->cond, &st->relres);
                return st->relres <= EG_RES ? c : 0;
            }
        }
    }
    return 0;
}

/* Exported: the Cauchy endgame of the total-degree paths first..first+n-1,
 * one thread (x_out [n][dim][2]; cycle_out [n], 0 = no estimate). */
int orc_endgame(const orc_homotopy *h, int64_t first, int64_t n_paths, const orc_opts *o_in, double *x_out,
                int32_t *cycle_out, orc_stats *stats_out)
{
    orc_opts o;
    if (o_in) o = *o_in; else orc_default_opts(&o);
    if (h->kind != 0 || h->n < 1 || h->n > NMAX) return -1;
    const int n = h->n;
    cplx x[NMAX];
    orc_stats st;
    for (int64_t q = 0; q < n_paths; q++) {
        start_solution(h, first + q, x);
        const int c = endgame_one(h, &o, x, &st);
        for (int j = 0; j < n; j++) { x_out[(q * n + j) * 2] = creal(x[j]); x_out[(q * n + j) * 2 + 1] = cimag(x[j]); }
        cycle_out[q] = c;
        if (stats_out) stats_out[q] = st;
    }
    return 0;
}

/* ================================================================ double double path tracking
 * Section 5 and Table 2 run the whole solver in double double arithmetic
 * ("quality up").  Here a path is tracked with the readings of track_one
 * (RK4 predictor, Newton corrector, the same step control, tolerances,
 * stall and divergence rules), but the point x, the predictor stages, H,
 * H_x, H_t, the LU and the solves are complex double double; t, the step
 * sizes and the norms (taken from the double parts) stay double.  The end
 * Newton at t = 1 stops at ||dx|| <= END_TOL_DD (1 + ||x||); the endpoint is
 * classified from its double part with end_measures, as a double endpoint. */

#define END_TOL_DD 1e-26

static cdd cdd_scale(double a, cdd z)
{
    cdd r = { dd_mul(dd_from(a), z.re), dd_mul(dd_from(a), z.im) };
    return r;
}

/* H(x,t), H_x(x,t), H_t(x,t) in complex double double, every monomial and
 * partial derivative from scratch (as eval_homotopy). */
static void eval_homotopy_dd(const orc_homotopy *h, const cdd *x, double t, cdd *H, cdd *Hx, cdd *Ht)
{
    const int n = h->n;
    const cdd gamma = cdd_from(h->gamma_re + I * h->gamma_im);
    const cdd one = cdd_from(1.0);
    const dd omt = dd_sub(dd_from(1.0), dd_from(t)); /* 1 - t, exact */
    const cdd w1 = { omt, dd_from(0.0) };
    const cdd tt = cdd_from(t);
    int off = 0;
    for (int i = 0; i < n; i++) {
        cdd f = cdd_from(0.0), ft = cdd_from(0.0);
        for (int j = 0; j < n; j++) Hx[i * n + j] = cdd_from(0.0);
        for (int k = 0; k < h->terms_per_eq[i]; k++) {
            const uint8_t *a = h->exps + (size_t)(off + k) * n;
            const cdd c = cdd_from(coef_of(h, off + k));
            cdd ct, dct;
            if (h->kind == 0) {
                ct = cdd_mul(tt, c);
                dct = c;
            } else if (h->kind == 2) {
                const cdd c0 = cdd_from(h->coefs0[2 * (off + k)] + I * h->coefs0[2 * (off + k) + 1]);
                const cdd gc0 = cdd_mul(gamma, c0);
                ct = cdd_add(cdd_mul(w1, gc0), cdd_mul(tt, c));
                dct = cdd_sub(c, gc0);
            } else if (i == h->row && !is_unit(a, n, h->slack)) {
                ct = cdd_mul(w1, c);
                dct = cdd_sub(cdd_from(0.0), c);
            } else {
                ct = c;
                dct = cdd_from(0.0);
            }
            cdd m = one;
            for (int j = 0; j < n; j++) m = cdd_mul(m, cdd_ipow(x[j], a[j]));
            f = cdd_add(f, cdd_mul(ct, m));
            ft = cdd_add(ft, cdd_mul(dct, m));
            for (int j = 0; j < n; j++) {
                if (a[j] == 0) continue;
                cdd d = cdd_scale((double)a[j], cdd_ipow(x[j], a[j] - 1));
                for (int q = 0; q < n; q++)
                    if (q != j) d = cdd_mul(d, cdd_ipow(x[q], a[q]));
                Hx[i * n + j] = cdd_add(Hx[i * n + j], cdd_mul(ct, d));
            }
        }
        if (h->kind == 0) {
            /* start system g_i = x_i^{d_i} - 1, weighted by (1-t) gamma */
            const int d = eq_degree(h, i, off);
            const cdd xd = cdd_ipow(x[i], d);
            const cdd g = cdd_sub(xd, one);
            const cdd w = cdd_mul(w1, gamma);
            f = cdd_add(f, cdd_mul(w, g));
            ft = cdd_sub(ft, cdd_mul(gamma, g));
            Hx[i * n + i] = cdd_add(Hx[i * n + i], cdd_mul(w, cdd_scale((double)d, cdd_ipow(x[i], d - 1))));
        }
        H[i] = f;
        Ht[i] = ft;
        off += h->terms_per_eq[i];
    }
}

static double vnorm_dd(int n, const cdd *v)
{
    double m = 0.0;
    for (int j = 0; j < n; j++) {
        double a = cdd_absinf(v[j]);
        if (!(a <= m)) m = a;
    }
    return m;
}

static int all_finite_dd(int n, const cdd *x)
{
    for (int j = 0; j < n; j++)
        if (!isfinite(x[j].re.hi) || !isfinite(x[j].im.hi) || !isfinite(x[j].re.lo) || !isfinite(x[j].im.lo)) return 0;
    return 1;
}

/* v = -H_x^{-1} H_t at (x, t).  Returns -1 if the LU meets a zero pivot. */
static int tangent_dd(const orc_homotopy *h, const cdd *x, double t, cdd *v, orc_stats *st)
{
    cdd H[NMAX], Hx[NMAX * NMAX];
    eval_homotopy_dd(h, x, t, H, Hx, v);
    st->n_solve++;
    if (lu_solve_dd(h->n, Hx, v)) return -1;
    for (int j = 0; j < h->n; j++) v[j] = cdd_sub(cdd_from(0.0), v[j]);
    return 0;
}

/* One Newton step at fixed t: x -= H_x^{-1} H.  Returns ||dx||, NAN when singular. */
static double newton_step_dd(const orc_homotopy *h, cdd *x, double t, orc_stats *st)
{
    cdd H[NMAX], Hx[NMAX * NMAX], Ht[NMAX];
    eval_homotopy_dd(h, x, t, H, Hx, Ht);
    st->n_solve++;
    st->n_newton++;
    if (lu_solve_dd(h->n, Hx, H)) return NAN;
    for (int j = 0; j < h->n; j++) x[j] = cdd_sub(x[j], H[j]);
    return vnorm_dd(h->n, H);
}

/* track_one in complex double double (the same readings, step for step). */
static void track_one_dd(const orc_homotopy *h, const orc_opts *o, cdd *x, orc_stats *st)
{
    const int n = h->n;
    cdd x0[NMAX], xs[NMAX], k1[NMAX], k2[NMAX], k3[NMAX], k4[NMAX];
    double t = 0.0, step = o->h_init;
    int streak = 0, steps = 0;
    double ck[5];
    int nck = 0;
    double next_s = 0.1;
    int since_ck = 0;
    memset(st, 0, sizeof *st);
    while (t < 1.0) {
        double he = step;
        double t1 = t + he;
        if (he >= 1.0 - t) { he = 1.0 - t; t1 = 1.0; }
        memcpy(x0, x, sizeof(cdd) * n);
        const cdd hh = cdd_from(0.5 * he), hf = cdd_from(he), h6 = cdd_from(he / 6.0), two = cdd_from(2.0);
        int ok = 1;
        ok = ok && !tangent_dd(h, x0, t, k1, st);
        for (int j = 0; j < n; j++) xs[j] = cdd_add(x0[j], cdd_mul(hh, k1[j]));
        ok = ok && !tangent_dd(h, xs, t + 0.5 * he, k2, st);
        for (int j = 0; j < n; j++) xs[j] = cdd_add(x0[j], cdd_mul(hh, k2[j]));
        ok = ok && !tangent_dd(h, xs, t + 0.5 * he, k3, st);
        for (int j = 0; j < n; j++) xs[j] = cdd_add(x0[j], cdd_mul(hf, k3[j]));
        ok = ok && !tangent_dd(h, xs, t1, k4, st);
        if (ok)
            for (int j = 0; j < n; j++) {
                cdd acc = cdd_add(cdd_add(k1[j], cdd_mul(two, k2[j])), cdd_add(cdd_mul(two, k3[j]), k4[j]));
                x[j] = cdd_add(x0[j], cdd_mul(h6, acc));
            }
        int conv = 0;
        double prev = INFINITY;
        for (int it = 0; ok && it < o->max_corr_iters; it++) {
            double d = newton_step_dd(h, x, t1, st);
            if (!(d == d) || !all_finite_dd(n, x)) break;
            if (d <= o->corr_tol * (1.0 + vnorm_dd(n, x))) { conv = 1; break; }
            if (it > 0 && d > o->corr_contract * prev) break;
            prev = d;
        }
        steps++;
        if (conv) {
            t = t1;
            st->n_accept++;
            while (1.0 - t <= next_s && next_s > 0.0) {
                ck[nck % 5] = vnorm_dd(n, x);
                nck++;
                since_ck = 0;
                next_s *= 0.1;
                if (nck >= 40) next_s = 0.0;
            }
            if (vnorm_dd(n, x) > o->diverge_norm) { st->stop = 1; break; }
            if (++streak >= o->expand_after) {
                streak = 0;
                step = step * o->expand;
                if (step > o->h_max) step = o->h_max;
            }
        } else {
            memcpy(x, x0, sizeof(cdd) * n);
            st->n_reject++;
            streak = 0;
            step = he * o->shrink;
            if (step < o->h_min) { st->stop = 2; break; }
        }
        if (steps >= o->max_steps) { st->stop = 3; break; }
        if (++since_ck >= o->max_steps_decade && t < 1.0) { st->stop = 3; break; }
    }
    st->t = t;
    st->h = step;
    int grew = 0;
    st->growth = 0.0;
    if (nck >= 2) {
        int l = nck - 1, m = l < 4 ? l : 4;
        double a = ck[l % 5], b = ck[(l - m) % 5], g = 1.0;
        for (int k = 0; k < m; k++) g *= o->growth_inf;
        grew = a > b * g;
        st->growth = log10(a / b) / m;
    }
    cplx xh[NMAX];
    if (!all_finite_dd(n, x)) { st->stop = 4; st->cls = ORC_FAILED; st->norm_x = NAN; st->cond = NAN; st->relres = NAN; return; }
    st->norm_x = vnorm_dd(n, x);
    if (st->stop == 1) { st->cls = ORC_AT_INFINITY; st->cond = INFINITY; st->relres = NAN; return; }
    if (st->stop != 0) {
        for (int j = 0; j < n; j++) xh[j] = x[j].re.hi + I * x[j].im.hi;
        end_measures(h, xh, &st->cond, &st->relres);
        if (st->norm_x > o->endpoint_inf_norm || (t >= o->end_zone && grew)) st->cls = ORC_AT_INFINITY;
        else if (t < o->end_zone) st->cls = ORC_FAILED;
        else st->cls = ORC_SINGULAR;
        return;
    }
    for (int it = 0; it < o->end_iters; it++) {
        double d = newton_step_dd(h, x, 1.0, st);
        if (!(d == d) || !all_finite_dd(n, x)) break;
        if (d <= END_TOL_DD * (1.0 + vnorm_dd(n, x))) break;
    }
    if (!all_finite_dd(n, x)) { st->stop = 4; st->cls = ORC_FAILED; st->norm_x = NAN; st->cond = NAN; st->relres = NAN; return; }
    st->norm_x = vnorm_dd(n, x);
    for (int j = 0; j < n; j++) xh[j] = x[j].re.hi + I * x[j].im.hi;
    end_measures(h, xh, &st->cond, &st->relres);
    if (st->norm_x > o->endpoint_inf_norm) st->cls = ORC_AT_INFINITY;
    else if (st->cond <= o->cond_regular && st->relres <= o->res_regular) st->cls = ORC_REGULAR;
    else st->cls = ORC_SINGULAR;
}

typedef struct {
    const orc_homotopy *h;
    const orc_opts *o;
    const double *starts; /* [n_paths][n][2] or NULL */
    int64_t first, n_paths;
    double *x_hi, *x_lo;  /* [n_paths][n][2] */
    int8_t *cls_out;
    orc_stats *stats_out;
    atomic_llong next;
} crew_dd_t;

static void *crew_dd_worker(void *arg)
{
    crew_dd_t *c = (crew_dd_t *)arg;
    const int n = c->h->n;
    cdd x[NMAX];
    cplx xs[NMAX];
    orc_stats st;
    for (;;) {
        int64_t q = atomic_fetch_add(&c->next, 1);
        if (q >= c->n_paths) break;
        if (c->starts)
            for (int j = 0; j < n; j++) xs[j] = c->starts[(q * n + j) * 2] + I * c->starts[(q * n + j) * 2 + 1];
        else
            start_solution(c->h, c->first + q, xs);
        for (int j = 0; j < n; j++) x[j] = cdd_from(xs[j]);
        track_one_dd(c->h, c->o, x, &st);
        for (int j = 0; j < n; j++) {
            c->x_hi[(q * n + j) * 2] = x[j].re.hi;
            c->x_hi[(q * n + j) * 2 + 1] = x[j].im.hi;
            c->x_lo[(q * n + j) * 2] = x[j].re.lo;
            c->x_lo[(q * n + j) * 2 + 1] = x[j].im.lo;
        }
        if (c->cls_out) c->cls_out[q] = (int8_t)st.cls;
        if (c->stats_out) c->stats_out[q] = st;
    }
    return NULL;
}

/* Track paths in complex double double (see track_one_dd); x_hi and x_lo
 * receive the two parts of every endpoint. */
int orc_track_dd(const orc_homotopy *h, const double *starts, int64_t first, int64_t n_paths, const orc_opts *o_in,
                 int n_threads, double *x_hi, double *x_lo, int8_t *cls_out, orc_stats *stats_out)
{
    orc_opts o;
    if (o_in) o = *o_in; else orc_default_opts(&o);
    if (h->n < 1 || h->n > NMAX || n_paths < 0) return -1;
    if (!starts && h->kind != 0) return -1;
    if (h->kind == 3) return -1; /* double double tracking covers kinds 0..2 */
    crew_dd_t c;
    c.h = h; c.o = &o; c.starts = starts; c.first = first; c.n_paths = n_paths;
    c.x_hi = x_hi; c.x_lo = x_lo; c.cls_out = cls_out; c.stats_out = stats_out;
    atomic_init(&c.next, 0);
    if (n_threads < 1) n_threads = 1;
    if (n_threads == 1) { crew_dd_worker(&c); return 0; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    for (int k = 0; k < n_threads; k++) pthread_create(&th[k], NULL, crew_dd_worker, &c);
    for (int k = 0; k < n_threads; k++) pthread_join(th[k], NULL);
    free(th);
    return 0;
}

/* ================================================================ quad double
 * Quad double arithmetic (the paper runs the solver in double double and in
 * quad double, Section 5 and Table 2, with the arithmetic of [HLB00]): a
 * value is an unevaluated sum of four doubles x0 + x1 + x2 + x3 of
 * decreasing magnitude.  Every operation here writes an expansion whose sum
 * is the exact result (TwoSum and TwoProduct pairs; the partial products of
 * order u^4 relative in plain double), and qd_from_expansion turns it into
 * four components: sort the terms by decreasing magnitude and run TwoSum
 * from the bottom up twice (the top term becomes the sum, rounded, and the
 * others hold the exact rest), keep the top term, repeat on the rest.  Every
 * step is error free, so the only error is the rest after the fourth term. */

typedef struct { double x[4]; } qd;
typedef struct { qd re, im; } cqd;

#define QD_MAXTERMS 40
#define END_TOL_QD 1e-58

static void sort_by_magnitude(double *e, int m)
{
    for (int i = 1; i < m; i++) {
        double v = e[i];
        int k = i - 1;
        while (k >= 0 && fabs(e[k]) < fabs(v)) { e[k + 1] = e[k]; k--; }
        e[k + 1] = v;
    }
}

static void sum_up(double *e, int m)
{
    for (int i = m - 1; i > 0; i--) {
        dd s = two_sum(e[i - 1], e[i]);
        e[i - 1] = s.hi;
        e[i] = s.lo;
    }
}

static qd qd_from_expansion(double *e, int m)
{
    qd r = {{0.0, 0.0, 0.0, 0.0}};
    int lo = 0;
    for (int k = 0; k < 4 && lo < m; k++) {
        for (int pass = 0; pass < 2; pass++) {
            sort_by_magnitude(e + lo, m - lo);
            sum_up(e + lo, m - lo);
        }
        r.x[k] = e[lo];
        lo++;
    }
    return r;
}

static qd qd_from(double a) { qd r = {{a, 0.0, 0.0, 0.0}}; return r; }
static qd qd_neg(qd a) { qd r = {{-a.x[0], -a.x[1], -a.x[2], -a.x[3]}}; return r; }

static qd qd_add(qd a, qd b)
{
    double e[8];
    for (int i = 0; i < 4; i++) { e[2 * i] = a.x[i]; e[2 * i + 1] = b.x[i]; }
    return qd_from_expansion(e, 8);
}

static qd qd_sub(qd a, qd b) { return qd_add(a, qd_neg(b)); }

static qd qd_mul(qd a, qd b)
{
    double e[QD_MAXTERMS];
    int m = 0;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            if (i + j <= 3) {
                dd p = two_prod(a.x[i], b.x[j]);
                e[m++] = p.hi;
                e[m++] = p.lo;
            } else if (i + j == 4) {
                e[m++] = a.x[i] * b.x[j];
            }
        }
    return qd_from_expansion(e, m);
}

static qd qd_mul_d(qd a, double b)
{
    double e[8];
    for (int i = 0; i < 4; i++) {
        dd p = two_prod(a.x[i], b);
        e[2 * i] = p.hi;
        e[2 * i + 1] = p.lo;
    }
    return qd_from_expansion(e, 8);
}

/* Long division: q_k = r_0 / b_0, r <- r - q_k b, five quotient digits. */
static qd qd_div(qd a, qd b)
{
    double q[5];
    qd r = a;
    for (int k = 0; k < 5; k++) {
        q[k] = r.x[0] / b.x[0];
        if (k < 4) r = qd_sub(r, qd_mul_d(b, q[k]));
    }
    return qd_from_expansion(q, 5);
}

void orc_qd_add(const double *a, const double *b, double *out)
{
    qd x, y;
    memcpy(x.x, a, sizeof x.x);
    memcpy(y.x, b, sizeof y.x);
    qd r = qd_add(x, y);
    memcpy(out, r.x, sizeof r.x);
}
void orc_qd_mul(const double *a, const double *b, double *out)
{
    qd x, y;
    memcpy(x.x, a, sizeof x.x);
    memcpy(y.x, b, sizeof y.x);
    qd r = qd_mul(x, y);
    memcpy(out, r.x, sizeof r.x);
}
void orc_qd_div(const double *a, const double *b, double *out)
{
    qd x, y;
    memcpy(x.x, a, sizeof x.x);
    memcpy(y.x, b, sizeof y.x);
    qd r = qd_div(x, y);
    memcpy(out, r.x, sizeof r.x);
}

static cqd cqd_from(cplx z) { cqd r = { qd_from(creal(z)), qd_from(cimag(z)) }; return r; }
static cqd cqd_add(cqd a, cqd b) { cqd r = { qd_add(a.re, b.re), qd_add(a.im, b.im) }; return r; }
static cqd cqd_sub(cqd a, cqd b) { cqd r = { qd_sub(a.re, b.re), qd_sub(a.im, b.im) }; return r; }
static cqd cqd_mul(cqd a, cqd b)
{
    cqd r = { qd_sub(qd_mul(a.re, b.re), qd_mul(a.im, b.im)), qd_add(qd_mul(a.re, b.im), qd_mul(a.im, b.re)) };
    return r;
}
static cqd cqd_div(cqd a, cqd b)
{
    qd d = qd_add(qd_mul(b.re, b.re), qd_mul(b.im, b.im));
    cqd num = { qd_add(qd_mul(a.re, b.re), qd_mul(a.im, b.im)), qd_sub(qd_mul(a.im, b.re), qd_mul(a.re, b.im)) };
    cqd r = { qd_div(num.re, d), qd_div(num.im, d) };
    return r;
}
static cqd cqd_scale(double a, cqd z) { cqd r = { qd_mul_d(z.re, a), qd_mul_d(z.im, a) }; return r; }
static cqd cqd_ipow(cqd x, int e)
{
    cqd r = cqd_from(1.0);
    for (int k = 0; k < e; k++) r = cqd_mul(r, x);
    return r;
}
static double cqd_abs1(cqd a) { return fabs(a.re.x[0]) + fabs(a.im.x[0]); }
static double cqd_absinf(cqd a) { double x = fabs(a.re.x[0]), y = fabs(a.im.x[0]); return x > y ? x : y; }

/* H(x,t), H_x(x,t), H_t(x,t) in complex quad double, every monomial and
 * partial derivative from scratch (as eval_homotopy); kinds 0..2. */
static void eval_homotopy_qd(const orc_homotopy *h, const cqd *x, double t, cqd *H, cqd *Hx, cqd *Ht)
{
    const int n = h->n;
    const cqd gamma = cqd_from(h->gamma_re + I * h->gamma_im);
    const cqd one = cqd_from(1.0), zero = cqd_from(0.0);
    const cqd w1 = { qd_sub(qd_from(1.0), qd_from(t)), qd_from(0.0) }; /* 1 - t, exact */
    const cqd tt = cqd_from(t);
    int off = 0;
    for (int i = 0; i < n; i++) {
        cqd f = zero, ft = zero;
        for (int j = 0; j < n; j++) Hx[i * n + j] = zero;
        for (int k = 0; k < h->terms_per_eq[i]; k++) {
            const uint8_t *a = h->exps + (size_t)(off + k) * n;
            const cqd c = cqd_from(coef_of(h, off + k));
            cqd ct, dct;
            if (h->kind == 0) {
                ct = cqd_mul(tt, c);
                dct = c;
            } else if (h->kind == 2) {
                const cqd c0 = cqd_from(h->coefs0[2 * (off + k)] + I * h->coefs0[2 * (off + k) + 1]);
                const cqd gc0 = cqd_mul(gamma, c0);
                ct = cqd_add(cqd_mul(w1, gc0), cqd_mul(tt, c));
                dct = cqd_sub(c, gc0);
            } else if (i == h->row && !is_unit(a, n, h->slack)) {
                ct = cqd_mul(w1, c);
                dct = cqd_sub(zero, c);
            } else {
                ct = c;
                dct = zero;
            }
            cqd m = one;
            for (int j = 0; j < n; j++) m = cqd_mul(m, cqd_ipow(x[j], a[j]));
            f = cqd_add(f, cqd_mul(ct, m));
            ft = cqd_add(ft, cqd_mul(dct, m));
            for (int j = 0; j < n; j++) {
                if (a[j] == 0) continue;
                cqd d = cqd_scale((double)a[j], cqd_ipow(x[j], a[j] - 1));
                for (int q = 0; q < n; q++)
                    if (q != j) d = cqd_mul(d, cqd_ipow(x[q], a[q]));
                Hx[i * n + j] = cqd_add(Hx[i * n + j], cqd_mul(ct, d));
            }
        }
        if (h->kind == 0) {
            /* start system g_i = x_i^{d_i} - 1, weighted by (1-t) gamma */
            const int d = eq_degree(h, i, off);
            const cqd g = cqd_sub(cqd_ipow(x[i], d), one);
            const cqd w = cqd_mul(w1, gamma);
            f = cqd_add(f, cqd_mul(w, g));
            ft = cqd_sub(ft, cqd_mul(gamma, g));
            Hx[i * n + i] = cqd_add(Hx[i * n + i], cqd_mul(w, cqd_scale((double)d, cqd_ipow(x[i], d - 1))));
        }
        H[i] = f;
        Ht[i] = ft;
        off += h->terms_per_eq[i];
    }
}

/* Solves A y = b in place (b := y) by LU with partial pivoting by the largest
 * |.|_1 of the leading parts (the first row on ties).  Returns -1 on a zero
 * pivot. */
static int lu_solve_qd(int n, cqd *A, cqd *b)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = cqd_abs1(A[k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double a = cqd_abs1(A[i * n + k]);
            if (a > best) { best = a; p = i; }
        }
        if (!(best > 0.0)) return -1;
        if (p != k) {
            for (int j = 0; j < n; j++) { cqd tmp = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = tmp; }
            cqd tmp = b[k]; b[k] = b[p]; b[p] = tmp;
        }
        for (int i = k + 1; i < n; i++) {
            cqd l = cqd_div(A[i * n + k], A[k * n + k]);
            for (int j = k + 1; j < n; j++) A[i * n + j] = cqd_sub(A[i * n + j], cqd_mul(l, A[k * n + j]));
            b[i] = cqd_sub(b[i], cqd_mul(l, b[k]));
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        cqd s = b[i];
        for (int j = i + 1; j < n; j++) s = cqd_sub(s, cqd_mul(A[i * n + j], b[j]));
        b[i] = cqd_div(s, A[i * n + i]);
    }
    return 0;
}

static double vnorm_qd(int n, const cqd *v)
{
    double m = 0.0;
    for (int j = 0; j < n; j++) {
        double a = cqd_absinf(v[j]);
        if (!(a <= m)) m = a;
    }
    return m;
}

static int all_finite_qd(int n, const cqd *x)
{
    for (int j = 0; j < n; j++)
        for (int k = 0; k < 4; k++)
            if (!isfinite(x[j].re.x[k]) || !isfinite(x[j].im.x[k])) return 0;
    return 1;
}

static int tangent_qd(const orc_homotopy *h, const cqd *x, double t, cqd *v, orc_stats *st)
{
    cqd H[NMAX], Hx[NMAX * NMAX];
    eval_homotopy_qd(h, x, t, H, Hx, v);
    st->n_solve++;
    if (lu_solve_qd(h->n, Hx, v)) return -1;
    for (int j = 0; j < h->n; j++) v[j] = cqd_sub(cqd_from(0.0), v[j]);
    return 0;
}

static double newton_step_qd(const orc_homotopy *h, cqd *x, double t, orc_stats *st)
{
    cqd H[NMAX], Hx[NMAX * NMAX], Ht[NMAX];
    eval_homotopy_qd(h, x, t, H, Hx, Ht);
    st->n_solve++;
    st->n_newton++;
    if (lu_solve_qd(h->n, Hx, H)) return NAN;
    for (int j = 0; j < h->n; j++) x[j] = cqd_sub(x[j], H[j]);
    return vnorm_qd(h->n, H);
}

/* track_one in complex quad double (the readings of track_one, step for
 * step); the end Newton at t = 1 stops at ||dx|| <= END_TOL_QD (1 + ||x||). */
static void track_one_qd(const orc_homotopy *h, const orc_opts *o, cqd *x, orc_stats *st)
{
    const int n = h->n;
    cqd x0[NMAX], xs[NMAX], k1[NMAX], k2[NMAX], k3[NMAX], k4[NMAX];
    double t = 0.0, step = o->h_init;
    int streak = 0, steps = 0;
    double ck[5];
    int nck = 0;
    double next_s = 0.1;
    int since_ck = 0;
    memset(st, 0, sizeof *st);
    while (t < 1.0) {
        double he = step;
        double t1 = t + he;
        if (he >= 1.0 - t) { he = 1.0 - t; t1 = 1.0; }
        memcpy(x0, x, sizeof(cqd) * n);
        const cqd hh = cqd_from(0.5 * he), hf = cqd_from(he), h6 = cqd_from(he / 6.0), two = cqd_from(2.0);
        int ok = 1;
        ok = ok && !tangent_qd(h, x0, t, k1, st);
        for (int j = 0; j < n; j++) xs[j] = cqd_add(x0[j], cqd_mul(hh, k1[j]));
        ok = ok && !tangent_qd(h, xs, t + 0.5 * he, k2, st);
        for (int j = 0; j < n; j++) xs[j] = cqd_add(x0[j], cqd_mul(hh, k2[j]));
        ok = ok && !tangent_qd(h, xs, t + 0.5 * he, k3, st);
        for (int j = 0; j < n; j++) xs[j] = cqd_add(x0[j], cqd_mul(hf, k3[j]));
        ok = ok && !tangent_qd(h, xs, t1, k4, st);
        if (ok)
            for (int j = 0; j < n; j++) {
                cqd acc = cqd_add(cqd_add(k1[j], cqd_mul(two, k2[j])), cqd_add(cqd_mul(two, k3[j]), k4[j]));
                x[j] = cqd_add(x0[j], cqd_mul(h6, acc));
            }
        int conv = 0;
        double prev = INFINITY;
        for (int it = 0; ok && it < o->max_corr_iters; it++) {
            double d = newton_step_qd(h, x, t1, st);
            if (!(d == d) || !all_finite_qd(n, x)) break;
            if (d <= o->corr_tol * (1.0 + vnorm_qd(n, x))) { conv = 1; break; }
            if (it > 0 && d > o->corr_contract * prev) break;
            prev = d;
        }
        steps++;
        if (conv) {
            t = t1;
            st->n_accept++;
            while (1.0 - t <= next_s && next_s > 0.0) {
                ck[nck % 5] = vnorm_qd(n, x);
                nck++;
                since_ck = 0;
                next_s *= 0.1;
                if (nck >= 40) next_s = 0.0;
            }
            if (vnorm_qd(n, x) > o->diverge_norm) { st->stop = 1; break; }
            if (++streak >= o->expand_after) {
                streak = 0;
                step = step * o->expand;
                if (step > o->h_max) step = o->h_max;
            }
        } else {
            memcpy(x, x0, sizeof(cqd) * n);
            st->n_reject++;
            streak = 0;
            step = he * o->shrink;
            if (step < o->h_min) { st->stop = 2; break; }
        }
        if (steps >= o->max_steps) { st->stop = 3; break; }
        if (++since_ck >= o->max_steps_decade && t < 1.0) { st->stop = 3; break; }
    }
    st->t = t;
    st->h = step;
    int grew = 0;
    st->growth = 0.0;
    if (nck >= 2) {
        int l = nck - 1, m = l < 4 ? l : 4;
        double a = ck[l % 5], b = ck[(l - m) % 5], g = 1.0;
        for (int k = 0; k < m; k++) g *= o->growth_inf;
        grew = a > b * g;
        st->growth = log10(a / b) / m;
    }
    cplx xh[NMAX];
    if (!all_finite_qd(n, x)) { st->stop = 4; st->cls = ORC_FAILED; st->norm_x = NAN; st->cond = NAN; st->relres = NAN; return; }
    st->norm_x = vnorm_qd(n, x);
    if (st->stop == 1) { st->cls = ORC_AT_INFINITY; st->cond = INFINITY; st->relres = NAN; return; }
    if (st->stop != 0) {
        for (int j = 0; j < n; j++) xh[j] = x[j].re.x[0] + I * x[j].im.x[0];
        end_measures(h, xh, &st->cond, &st->relres);
        if (st->norm_x > o->endpoint_inf_norm || (t >= o->end_zone && grew)) st->cls = ORC_AT_INFINITY;
        else if (t < o->end_zone) st->cls = ORC_FAILED;
        else st->cls = ORC_SINGULAR;
        return;
    }
    for (int it = 0; it < o->end_iters; it++) {
        double d = newton_step_qd(h, x, 1.0, st);
        if (!(d == d) || !all_finite_qd(n, x)) break;
        if (d <= END_TOL_QD * (1.0 + vnorm_qd(n, x))) break;
    }
    if (!all_finite_qd(n, x)) { st->stop = 4; st->cls = ORC_FAILED; st->norm_x = NAN; st->cond = NAN; st->relres = NAN; return; }
    st->norm_x = vnorm_qd(n, x);
    for (int j = 0; j < n; j++) xh[j] = x[j].re.x[0] + I * x[j].im.x[0];
    end_measures(h, xh, &st->cond, &st->relres);
    if (st->norm_x > o->endpoint_inf_norm) st->cls = ORC_AT_INFINITY;
    else if (st->cond <= o->cond_regular && st->relres <= o->res_regular) st->cls = ORC_REGULAR;
    else st->cls = ORC_SINGULAR;
}

typedef struct {
    const orc_homotopy *h;
    const orc_opts *o;
    const double *starts; /* [n_paths][n][2] or NULL */
    int64_t first, n_paths;
    double *x_out;        /* [n_paths][n][4][2] */
    int8_t *cls_out;
    orc_stats *stats_out;
    atomic_llong next;
} crew_qd_t;

static void *crew_qd_worker(void *arg)
{
    crew_qd_t *c = (crew_qd_t *)arg;
    const int n = c->h->n;
    cqd x[NMAX];
    cplx xs[NMAX];
    orc_stats st;
    for (;;) {
        int64_t q = atomic_fetch_add(&c->next, 1);
        if (q >= c->n_paths) break;
        if (c->starts)
            for (int j = 0; j < n; j++) xs[j] = c->starts[(q * n + j) * 2] + I * c->starts[(q * n + j) * 2 + 1];
        else
            start_solution(c->h, c->first + q, xs);
        for (int j = 0; j < n; j++) x[j] = cqd_from(xs[j]);
        track_one_qd(c->h, c->o, x, &st);
        for (int j = 0; j < n; j++)
            for (int k = 0; k < 4; k++) {
                c->x_out[((q * n + j) * 4 + k) * 2] = x[j].re.x[k];
                c->x_out[((q * n + j) * 4 + k) * 2 + 1] = x[j].im.x[k];
            }
        if (c->cls_out) c->cls_out[q] = (int8_t)st.cls;
        if (c->stats_out) c->stats_out[q] = st;
    }
    return NULL;
}

/* Track paths in complex quad double (see track_one_qd); x_out receives the
 * four parts of every endpoint coordinate, [n_paths][n][4] complex. */
int orc_track_qd(const orc_homotopy *h, const double *starts, int64_t first, int64_t n_paths, const orc_opts *o_in,
                 int n_threads, double *x_out, int8_t *cls_out, orc_stats *stats_out)
{
    orc_opts o;
    if (o_in) o = *o_in; else orc_default_opts(&o);
    if (h->n < 1 || h->n > NMAX || n_paths < 0) return -1;
    if (!starts && h->kind != 0) return -1;
    if (h->kind == 3) return -1; /* quad double tracking covers kinds 0..2 */
    crew_qd_t c;
    c.h = h; c.o = &o; c.starts = starts; c.first = first; c.n_paths = n_paths;
    c.x_out = x_out; c.cls_out = cls_out; c.stats_out = stats_out;
    atomic_init(&c.next, 0);
    if (n_threads < 1) n_threads = 1;
    if (n_threads == 1) { crew_qd_worker(&c); return 0; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    for (int k = 0; k < n_threads; k++) pthread_create(&th[k], NULL, crew_qd_worker, &c);
    for (int k = 0; k < n_threads; k++) pthread_join(th[k], NULL);
    free(th);
    return 0;
}

/* Size of the stats record, so the Python side can check its mirror. */
int orc_stats_size(void) { return (int)sizeof(orc_stats); }
int orc_opts_size(void) { return (int)sizeof(orc_opts); }
int orc_homotopy_size(void) { return (int)sizeof(orc_homotopy); }
