// track.cu -- the path tracker on sm_103a.
//
// One thread tracks one path (the paths of a homotopy are independent,
// Section 1 of the paper); a block stages the homotopy's tables into shared
// memory once and keeps every thread's evaluation point, residual, t-
// derivative and Jacobian there, laid out lane-fastest so a warp touches 32
// consecutive 16-byte slots per element (no bank conflicts).
//
// Every trip through the main loop is one "unit" for every live lane: evaluate
// H, H_x, H_t at (xe, te), factor H_x with partial pivoting and solve for one
// right-hand side.  What the unit is for depends on the lane's phase:
//   phase 0..3  the four stages of the Runge-Kutta predictor (rhs -H_t)
//   phase 4     a Newton correction at t + h (rhs -H)
//   phase 5     a Newton correction at t = 1 (rhs -H)
// so lanes at different points of their paths still execute the same
// arithmetic together.  A lane whose path ends writes its endpoint and takes
// the next path index from a global atomic counter (the GPU form of the work
// crew of Section 1).  Classification runs afterwards in classify_kernel.
//
// The step logic follows the readings documented in include/phc.h; the CPU
// oracle implements the same readings independently.
#include <cstdio>

#include "phc_internal.h"

namespace phc {

// ------------------------------------------------------------------ complex arithmetic

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c - a b
__device__ __forceinline__ double2 cfms(double2 c, double2 a, double2 b)
{
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
// a + s b
__device__ __forceinline__ double2 caxpy(double2 a, double s, double2 b)
{
    return make_double2(fma(s, b.x, a.x), fma(s, b.y, a.y));
}
__device__ __forceinline__ double abs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ double absinf(double2 a)
{
    double u = fabs(a.x), v = fabs(a.y);
    return u > v ? u : v;
}
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Strided per-thread slot i of a shared array (stride = threads per block).
#define SL(arr, i) (arr)[(i) * bt]

// ------------------------------------------------------------------ tables in shared memory

struct SmTab {
    int n_terms;
    const TermRec *terms;
    const uint8_t *vars;
    const uint8_t *exps;
    const double2 *c0;  // system 0; system s at + s * n_terms (shared or global memory)
    const double2 *c1;
};

__device__ SmTab stage_table(const DevTables &g, char *smem)
{
    SmTab s;
    TermRec *terms = reinterpret_cast<TermRec *>(smem);
    uint8_t *vars = reinterpret_cast<uint8_t *>(terms + g.n_terms);
    uint8_t *exps = vars + g.n_ve;
    size_t b = (size_t)g.n_terms * sizeof(TermRec) + 2 * (size_t)g.n_ve;
    b = (b + 15) & ~(size_t)15;
    for (int i = threadIdx.x; i < g.n_terms; i += blockDim.x) terms[i] = g.terms[i];
    for (int i = threadIdx.x; i < g.n_ve; i += blockDim.x) {
        vars[i] = g.vars[i];
        exps[i] = g.exps[i];
    }
    if (coefs_in_smem(g)) {
        const int nc = g.n_terms * g.n_sys;
        double2 *c0 = reinterpret_cast<double2 *>(smem + b);
        double2 *c1 = c0 + nc;
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
            c0[i] = g.c0[i];
            c1[i] = g.c1[i];
        }
        s.c0 = c0;
        s.c1 = c1;
    } else {
        s.c0 = g.c0;
        s.c1 = g.c1;
    }
    __syncthreads();
    s.n_terms = g.n_terms;
    s.terms = terms;
    s.vars = vars;
    s.exps = exps;
    return s;
}

// ------------------------------------------------------------------ evaluation

// H(xe,t), H_x (row-major N x N in J) and H_t at the thread's point xe.
// Each term c(t) x^a with support v_0..v_{k-1} is split as
//   x^a = cf * prod_j x_{v_j},  cf = prod_j x_{v_j}^{a_j - 1}   (common factor)
// and its partial derivatives come from prefix and suffix products of the
// x_{v_j} (Speelpenning's product rule):
//   d/dx_{v_j} c(t) x^a = a_j c(t) cf prod_{i<j} x_{v_i} prod_{i>j} x_{v_i}.
// With SCALE, S[i].x accumulates sum over the terms of equation i of
// |c(t)|_1 |x^a|_1 (for the relative residual and the condition number).
template <int N, bool SCALE>
__device__ __forceinline__ void evaluate(const SmTab &tb, int sys, double t, const double2 *xe, double2 *H,
                                         double2 *Ht, double2 *J, double2 *P, double2 *S, int bt)
{
    const double2 *C0 = tb.c0 + (size_t)sys * tb.n_terms;
    const double2 *C1 = tb.c1 + (size_t)sys * tb.n_terms;
    const double2 zero = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < N; i++) {
        SL(H, i) = zero;
        SL(Ht, i) = zero;
        if (SCALE) SL(S, i) = zero;
    }
#pragma unroll
    for (int i = 0; i < N * N; i++) SL(J, i) = zero;

    for (int q = 0; q < tb.n_terms; q++) {
        const TermRec r = tb.terms[q];
        const double2 c0 = C0[q], c1 = C1[q];
        const double2 ct = make_double2(fma(t, c1.x, c0.x), fma(t, c1.y, c0.y));
        const int k = r.k;
        if (k == 0) {
            SL(H, r.eq) = cadd(SL(H, r.eq), ct);
            SL(Ht, r.eq) = cadd(SL(Ht, r.eq), c1);
            if (SCALE) SL(S, r.eq).x += abs1(ct);
            continue;
        }
        const uint8_t *v = tb.vars + r.off;
        const uint8_t *e = tb.exps + r.off;
        double2 cf = make_double2(1.0, 0.0);
        const bool powers = (r.flags & TERM_POWERS) != 0;
        if (powers) {
            for (int j = 0; j < k; j++) {
                const int a = e[j];
                if (a > 1) {
                    const double2 xv = SL(xe, v[j]);
                    double2 pw = xv;
                    for (int m = 2; m < a; m++) pw = cmul(pw, xv);
                    cf = cmul(cf, pw);
                }
            }
        }
        // prefix products: P[j] = ct cf prod_{i<j} x_{v_i}
        double2 pre = powers ? cmul(ct, cf) : ct;
        SL(P, 0) = pre;
        for (int j = 1; j < k; j++) {
            pre = cmul(pre, SL(xe, v[j - 1]));
            SL(P, j) = pre;
        }
        // suffix products and the derivatives
        double2 suf = SL(xe, v[k - 1]);
        {
            double2 d = SL(P, k - 1);
            const int a = e[k - 1];
            if (a > 1) d = cscale((double)a, d);
            const int idx = r.eq * N + v[k - 1];
            SL(J, idx) = cadd(SL(J, idx), d);
        }
        for (int j = k - 2; j >= 0; j--) {
            double2 d = cmul(SL(P, j), suf);
            const int a = e[j];
            if (a > 1) d = cscale((double)a, d);
            const int idx = r.eq * N + v[j];
            SL(J, idx) = cadd(SL(J, idx), d);
            suf = cmul(suf, SL(xe, v[j]));
        }
        // suf = prod_j x_{v_j}; the monomial is cf * suf
        const double2 mono = powers ? cmul(cf, suf) : suf;
        SL(H, r.eq) = cadd(SL(H, r.eq), cmul(ct, mono));
        SL(Ht, r.eq) = cadd(SL(Ht, r.eq), cmul(c1, mono));
        if (SCALE) SL(S, r.eq).x += abs1(ct) * abs1(mono);
    }
}

// ------------------------------------------------------------------ linear algebra

// LU with partial pivoting of the thread's N x N matrix in J: the pivot of
// column k is the first row of largest |.|_1; rows are swapped whole (the
// multipliers move with them); the diagonal is replaced by its reciprocal.
// Returns false when a pivot is zero (or not a number).
template <int N>
__device__ __forceinline__ bool lu_factor(double2 *J, int (&perm)[N], int bt)
{
#pragma unroll
    for (int k = 0; k < N; k++) {
        int p = k;
        double best = abs1(SL(J, k * N + k));
#pragma unroll
        for (int i = k + 1; i < N; i++) {
            const double val = abs1(SL(J, i * N + k));
            if (val > best) {
                best = val;
                p = i;
            }
        }
        perm[k] = p;
        if (!(best > 0.0)) return false;
#pragma unroll
        for (int j = 0; j < N; j++) {
            const double2 a = SL(J, k * N + j), c = SL(J, p * N + j);
            SL(J, k * N + j) = c;
            SL(J, p * N + j) = a;
        }
        const double2 pv = SL(J, k * N + k);
        const double rd = 1.0 / fma(pv.x, pv.x, pv.y * pv.y);
        const double2 inv = make_double2(pv.x * rd, -pv.y * rd);
        SL(J, k * N + k) = inv;
#pragma unroll
        for (int i = k + 1; i < N; i++) {
            const double2 l = cmul(SL(J, i * N + k), inv);
            SL(J, i * N + k) = l;
#pragma unroll
            for (int j = k + 1; j < N; j++) SL(J, i * N + j) = cfms(SL(J, i * N + j), l, SL(J, k * N + j));
        }
    }
    return true;
}

// b := (LU)^{-1} P b in place (b strided in shared memory).
template <int N>
__device__ __forceinline__ void lu_solve(const double2 *J, const int (&perm)[N], double2 *b, int bt)
{
#pragma unroll
    for (int k = 0; k < N; k++) {
        const int p = perm[k];
        const double2 a = SL(b, k), c = SL(b, p);
        SL(b, k) = c;
        SL(b, p) = a;
    }
#pragma unroll
    for (int i = 1; i < N; i++) {
        double2 s = SL(b, i);
#pragma unroll
        for (int j = 0; j < i; j++) s = cfms(s, SL(J, i * N + j), SL(b, j));
        SL(b, i) = s;
    }
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
        double2 s = SL(b, i);
#pragma unroll
        for (int j = i + 1; j < N; j++) s = cfms(s, SL(J, i * N + j), SL(b, j));
        SL(b, i) = cmul(s, SL(J, i * N + i));
    }
}

// ------------------------------------------------------------------ tracker

struct ThreadArrays {
    double2 *xe, *H, *Ht, *P, *S, *J;
};

template <int N>
__device__ __forceinline__ ThreadArrays thread_arrays(char *smem, size_t table_bytes, int bt)
{
    ThreadArrays a;
    a.xe = reinterpret_cast<double2 *>(smem + table_bytes) + threadIdx.x;
    a.H = a.xe + N * bt;
    a.Ht = a.H + N * bt;
    a.P = a.Ht + N * bt;
    a.S = a.P + N * bt;
    a.J = a.S + N * bt;
    return a;
}

template <int N>
__global__ void __launch_bounds__(256) track_kernel(const TrackLaunch L, size_t table_bytes)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    const int bt = blockDim.x;
    const ThreadArrays A = thread_arrays<N>(smem, table_bytes, bt);
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths;

    double2 x0[N], acc[N];
    int perm[N];
    int64_t q = -1;
    int sys = 0;
    double t = 0.0, h = 0.0, he = 0.0, t1 = 0.0, te = 0.0, prev = 0.0, next_s = 0.0;
    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, r4 = 0.0;  // last five decade checkpoints, r4 newest
    int streak = 0, steps = 0, phase = 0, it = 0, nck = 0;
    int n_acc = 0, n_rej = 0, n_newt = 0, n_solve = 0;

    // start a new step from the accepted point x0
    auto begin_step = [&]() {
        he = h;
        t1 = t + he;
        if (he >= 1.0 - t) {
            he = 1.0 - t;
            t1 = 1.0;
        }
#pragma unroll
        for (int j = 0; j < N; j++) {
            SL(A.xe, j) = x0[j];
            acc[j] = make_double2(0.0, 0.0);
        }
        te = t;
        phase = 0;
    };

    auto finish = [&](int stop) {
        for (int j = 0; j < N; j++) L.x_out[(int64_t)j * np + q] = x0[j];
        int grew = 0;
        double growth = 0.0;
        if (nck >= 2) {
            const int l = nck - 1, m = l < 4 ? l : 4;
            const double a = r4, b = (m == 1) ? r3 : (m == 2) ? r2 : (m == 3) ? r1 : r0;
            double g = 1.0;
            for (int k = 0; k < m; k++) g *= o.growth_inf;
            grew = a > b * g;
            growth = log10(a / b) / m;
        }
        phc_path_stats s;
        s.t = t;
        s.h = h;
        s.cond = 0.0;
        s.relres = 0.0;
        s.norm_x = 0.0;
        s.growth = growth;
        s.n_accept = n_acc;
        s.n_reject = n_rej;
        s.n_newton = n_newt;
        s.n_solve = n_solve;
        s.stop = stop;
        s.n_fp32 = 0;
        s.grew = grew;
        s.system = sys;
        L.stats[q] = s;
        q = -1;
    };

    auto reject = [&]() {
        n_rej++;
        steps++;
        streak = 0;
        h = he * o.shrink;
        if (h < o.h_min) {
            finish(PHC_STOP_STEP_MIN);
            return;
        }
        if (steps >= o.max_steps) {
            finish(PHC_STOP_BUDGET);
            return;
        }
        begin_step();
    };

    auto accept = [&]() {
        t = t1;
        double nx = 0.0;
#pragma unroll
        for (int j = 0; j < N; j++) {
            x0[j] = SL(A.xe, j);
            const double a = absinf(x0[j]);
            if (!(a <= nx)) nx = a;
        }
        n_acc++;
        steps++;
        while (1.0 - t <= next_s && next_s > 0.0) {
            r0 = r1;
            r1 = r2;
            r2 = r3;
            r3 = r4;
            r4 = nx;
            nck++;
            next_s *= 0.1;
            if (nck >= 40) next_s = 0.0;
        }
        if (nx > o.diverge_norm) {
            finish(PHC_STOP_DIVERGED);
            return;
        }
        if (++streak >= o.expand_after) {
            streak = 0;
            h = h * o.expand;
            if (h > o.h_max) h = o.h_max;
        }
        if (steps >= o.max_steps) {
            finish(PHC_STOP_BUDGET);
            return;
        }
        if (t >= 1.0) {
            phase = 5;  // end Newton at t = 1 from x0 (already in xe)
            it = 0;
            te = 1.0;
        } else {
            begin_step();
        }
    };

    for (;;) {
        if (q < 0) {
            const unsigned long long c = atomicAdd(L.qhead, 1ull);
            if (c >= (unsigned long long)np) break;
            q = (int64_t)c;
            if (L.start_mode == 0) {
                const int64_t gid = L.first + q;
                sys = (int)(gid / L.paths_per_system);
                int64_t pid = gid - (int64_t)sys * L.paths_per_system;
#pragma unroll
                for (int i = 0; i < N; i++) {
                    const int d = L.deg[i];
                    const int k = (int)(pid % d);
                    pid /= d;
                    x0[i] = L.roots[L.root_off[i] + k];
                }
            } else {
#pragma unroll
                for (int i = 0; i < N; i++) x0[i] = L.starts[(int64_t)i * np + q];
            }
            t = 0.0;
            h = o.h_init;
            streak = steps = 0;
            nck = 0;
            next_s = 0.1;
            r0 = r1 = r2 = r3 = r4 = 0.0;
            n_acc = n_rej = n_newt = n_solve = 0;
            begin_step();
        }

        // one unit: evaluate, factor, solve
        evaluate<N, false>(tb, sys, te, A.xe, A.H, A.Ht, A.J, A.P, A.S, bt);
        double2 *b = (phase < 4) ? A.Ht : A.H;
        const bool ok = lu_factor<N>(A.J, perm, bt);
        if (ok) lu_solve<N>(A.J, perm, b, bt);
        n_solve++;

        if (phase < 4) {
            // Runge-Kutta stage: k = -J^{-1} H_t
            if (!ok) {
                reject();
                continue;
            }
            if (phase == 0) {
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double2 kj = make_double2(-SL(b, j).x, -SL(b, j).y);
                    acc[j] = kj;
                    SL(A.xe, j) = caxpy(x0[j], 0.5 * he, kj);
                }
                te = t + 0.5 * he;
                phase = 1;
            } else if (phase == 1) {
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double2 kj = make_double2(-SL(b, j).x, -SL(b, j).y);
                    acc[j] = caxpy(acc[j], 2.0, kj);
                    SL(A.xe, j) = caxpy(x0[j], 0.5 * he, kj);
                }
                te = t + 0.5 * he;
                phase = 2;
            } else if (phase == 2) {
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double2 kj = make_double2(-SL(b, j).x, -SL(b, j).y);
                    acc[j] = caxpy(acc[j], 2.0, kj);
                    SL(A.xe, j) = caxpy(x0[j], he, kj);
                }
                te = t1;
                phase = 3;
            } else {
                const double w = he / 6.0;
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double2 kj = make_double2(-SL(b, j).x, -SL(b, j).y);
                    acc[j] = cadd(acc[j], kj);
                    SL(A.xe, j) = caxpy(x0[j], w, acc[j]);
                }
                te = t1;
                phase = 4;
                it = 0;
                prev = 0.0;
            }
        } else if (phase == 4) {
            // Newton correction at t1
            n_newt++;
            if (!ok) {
                reject();
                continue;
            }
            double d = 0.0, nx = 0.0;
            bool fin = true;
#pragma unroll
            for (int j = 0; j < N; j++) {
                const double2 dj = SL(b, j);
                const double2 xj = make_double2(SL(A.xe, j).x - dj.x, SL(A.xe, j).y - dj.y);
                SL(A.xe, j) = xj;
                const double a = absinf(dj);
                if (!(a <= d)) d = a;
                const double c = absinf(xj);
                if (!(c <= nx)) nx = c;
                fin = fin && finite2(xj);
            }
            if (!(d == d) || !fin) {
                reject();
            } else if (d <= o.corr_tol * (1.0 + nx)) {
                accept();
            } else if (it > 0 && d > o.corr_contract * prev) {
                reject();
            } else {
                prev = d;
                if (++it >= o.max_corr_iters) reject();
            }
        } else {
            // Newton at t = 1
            n_newt++;
            if (!ok) {
                finish(PHC_STOP_REACHED);
                continue;
            }
            double d = 0.0, nx = 0.0;
            bool fin = true;
#pragma unroll
            for (int j = 0; j < N; j++) {
                const double2 dj = SL(b, j);
                const double2 xj = make_double2(SL(A.xe, j).x - dj.x, SL(A.xe, j).y - dj.y);
                SL(A.xe, j) = xj;
                x0[j] = xj;
                const double a = absinf(dj);
                if (!(a <= d)) d = a;
                const double c = absinf(xj);
                if (!(c <= nx)) nx = c;
                fin = fin && finite2(xj);
            }
            if (!(d == d) || !fin) {
                finish(fin ? PHC_STOP_REACHED : PHC_STOP_NONFINITE);
            } else if (d <= o.end_tol * (1.0 + nx) || ++it >= o.end_iters) {
                finish(PHC_STOP_REACHED);
            }
        }
    }
}

// ------------------------------------------------------------------ classification

// Condition number, relative residual and class of every endpoint (the
// readings in include/phc.h, identical to the oracle's).
template <int N>
__global__ void __launch_bounds__(256) classify_kernel(const ClassifyLaunch L, size_t table_bytes)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    const int bt = blockDim.x;
    const ThreadArrays A = thread_arrays<N>(smem, table_bytes, bt);
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths;
    int perm[N];

    for (int64_t q = (int64_t)blockIdx.x * bt + threadIdx.x; q < np; q += (int64_t)gridDim.x * bt) {
        const bool active = true;
        phc_path_stats s;
        bool fin = true;
        double nx = 0.0;
        if (active) {
            s = L.stats[q];
#pragma unroll
            for (int j = 0; j < N; j++) {
                const double2 xj = L.x[(int64_t)j * np + q];
                SL(A.xe, j) = xj;
                fin = fin && finite2(xj);
                const double a = absinf(xj);
                if (!(a <= nx)) nx = a;
            }
        }
        int8_t cls = PHC_FAILED;
        double cond = NAN, relres = NAN;
        const bool measure = active && fin && s.stop != PHC_STOP_DIVERGED;
        if (measure) {
            evaluate<N, true>(tb, s.system, 1.0, A.xe, A.H, A.Ht, A.J, A.P, A.S, bt);
            double rr = 0.0;
#pragma unroll
            for (int i = 0; i < N; i++) {
                const double r = abs1(SL(A.H, i)) / (1.0 + SL(A.S, i).x);
                if (!(r <= rr)) rr = r;
            }
            relres = rr;
            if (!lu_factor<N>(A.J, perm, bt)) {
                cond = INFINITY;
            } else {
                double rowacc[N];
#pragma unroll
                for (int j = 0; j < N; j++) rowacc[j] = 0.0;
#pragma unroll
                for (int i = 0; i < N; i++) {
#pragma unroll
                    for (int j = 0; j < N; j++) SL(A.H, j) = make_double2(i == j ? 1.0 : 0.0, 0.0);
                    lu_solve<N>(A.J, perm, A.H, bt);
                    const double si = 1.0 + SL(A.S, i).x;
#pragma unroll
                    for (int j = 0; j < N; j++) rowacc[j] += abs1(SL(A.H, j)) * si;
                }
                double m = 0.0;
#pragma unroll
                for (int j = 0; j < N; j++)
                    if (!(rowacc[j] <= m)) m = rowacc[j];
                cond = m / (1.0 + nx);
                if (!isfinite(cond)) cond = INFINITY;
            }
        }
        if (active) {
            if (!fin) {
                cls = PHC_FAILED;
                s.stop = PHC_STOP_NONFINITE;
                nx = NAN;
            } else if (s.stop == PHC_STOP_DIVERGED) {
                cls = PHC_AT_INFINITY;
                cond = INFINITY;
            } else if (s.stop != PHC_STOP_REACHED) {
                if (nx > o.stall_inf_norm || (s.t >= o.end_zone && s.grew)) cls = PHC_AT_INFINITY;
                else if (s.t < o.end_zone) cls = PHC_FAILED;
                else cls = PHC_SINGULAR;
            } else {
                if (nx > o.diverge_norm) cls = PHC_AT_INFINITY;
                else if (cond <= o.cond_regular && relres <= o.res_regular) cls = PHC_REGULAR;
                else cls = PHC_SINGULAR;
            }
            s.cond = cond;
            s.relres = relres;
            s.norm_x = nx;
            L.stats[q] = s;
            L.cls[q] = cls;
        }
    }
}

// ------------------------------------------------------------------ small kernels

__global__ void roots_kernel(const int32_t *deg, const int32_t *root_off, double2 *roots, int n)
{
    const int i = blockIdx.x;
    if (i >= n) return;
    const int d = deg[i];
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)d, &s, &c);
        roots[root_off[i] + k] = make_double2(c, s);
    }
}

__global__ void drop_last_kernel(const double2 *x_full, int n_full, int64_t np, double2 *x_out, uint8_t *slack_zero,
                                 int has_next_slack, double slack_tol)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        double nx = 0.0;
        for (int j = 0; j < n_full - 1; j++) {
            const double2 v = x_full[(int64_t)j * np + q];
            x_out[(int64_t)j * np + q] = v;
            const double a = absinf(v);
            if (!(a <= nx)) nx = a;
        }
        uint8_t z = 0;
        if (has_next_slack) z = absinf(x_full[(int64_t)(n_full - 2) * np + q]) <= slack_tol * (1.0 + nx);
        slack_zero[q] = z;
    }
}

// ------------------------------------------------------------------ launchers

static int g_num_sms = 0, g_smem_optin = 0;

static void device_limits()
{
    if (g_num_sms) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
}

int track_block_threads(int n, size_t table_bytes, int requested)
{
    device_limits();
    const size_t per = thread_smem_bytes(n);
    long fit = ((long)g_smem_optin - (long)table_bytes) / (long)per;
    int bt = (int)((fit / 32) * 32);
    if (bt > 256) bt = 256;
    if (requested > 0 && requested < bt) bt = (requested / 32) * 32;
    if (bt < 32) bt = 0;  // does not fit
    return bt;
}

template <int N>
static cudaError_t launch_track_n(const TrackLaunch &L, int bt, int max_blocks, cudaStream_t s)
{
    const size_t tb = table_smem_bytes(L.tab);
    const size_t smem = tb + (size_t)bt * thread_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(track_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_kernel<N>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t want = (L.n_paths + bt - 1) / bt;
    int64_t grid = (int64_t)g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    track_kernel<N><<<(unsigned)grid, bt, smem, s>>>(L, tb);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_classify_n(const ClassifyLaunch &L, cudaStream_t s)
{
    const size_t tb = table_smem_bytes(L.tab);
    const int bt = track_block_threads(N, tb, 128);
    if (bt == 0) return cudaErrorInvalidConfiguration;
    const size_t smem = tb + (size_t)bt * thread_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(classify_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (L.n_paths + bt - 1) / bt;
    if (grid > (int64_t)g_num_sms * 8) grid = (int64_t)g_num_sms * 8;
    if (grid < 1) grid = 1;
    classify_kernel<N><<<(unsigned)grid, bt, smem, s>>>(L, tb);
    return cudaGetLastError();
}

#define PHC_DISPATCH_N(n, CALL)                                                                                    \
    switch (n) {                                                                                                   \
    case 1: return CALL(1);                                                                                        \
    case 2: return CALL(2);                                                                                        \
    case 3: return CALL(3);                                                                                        \
    case 4: return CALL(4);                                                                                        \
    case 5: return CALL(5);                                                                                        \
    case 6: return CALL(6);                                                                                        \
    case 7: return CALL(7);                                                                                        \
    case 8: return CALL(8);                                                                                        \
    case 9: return CALL(9);                                                                                        \
    case 10: return CALL(10);                                                                                      \
    case 11: return CALL(11);                                                                                      \
    case 12: return CALL(12);                                                                                      \
    default: return cudaErrorInvalidValue;                                                                         \
    }

cudaError_t launch_track(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
    const size_t tb = table_smem_bytes(L.tab);
    const int bt = track_block_threads(L.tab.n, tb, block_threads);
    if (bt == 0) return cudaErrorInvalidConfiguration;
#define PHC_CALL_TRACK(NN) launch_track_n<NN>(L, bt, max_blocks, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_TRACK)
#undef PHC_CALL_TRACK
}

cudaError_t launch_classify(const ClassifyLaunch &L, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
#define PHC_CALL_CLS(NN) launch_classify_n<NN>(L, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_CLS)
#undef PHC_CALL_CLS
}

cudaError_t launch_roots(const int32_t *deg, const int32_t *root_off, double2 *roots, int n, int total, cudaStream_t s)
{
    (void)total;
    roots_kernel<<<n, 64, 0, s>>>(deg, root_off, roots, n);
    return cudaGetLastError();
}

cudaError_t launch_drop_last(const double2 *x_full, int n_full, int64_t n_paths, double2 *x_out, uint8_t *slack_zero,
                             int has_next_slack, double slack_tol, cudaStream_t s)
{
    device_limits();
    if (n_paths <= 0) return cudaSuccess;
    int64_t grid = (n_paths + 255) / 256;
    if (grid > (int64_t)g_num_sms * 16) grid = (int64_t)g_num_sms * 16;
    drop_last_kernel<<<(unsigned)grid, 256, 0, s>>>(x_full, n_full, n_paths, x_out, slack_zero, has_next_slack,
                                                    slack_tol);
    return cudaGetLastError();
}

}  // namespace phc
