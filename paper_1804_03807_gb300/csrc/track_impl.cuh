// track_impl.cuh -- the path tracker on sm_103a (device code shared by the
// translation units track.cu, track_pipe.cu and track_multi.cu, which
// instantiate its three modes in parallel compilations).
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
// crew of Section 1).  Classification runs afterwards in classify_kernel
// (mode 0) or inline (modes 1 and 2).  Once most lanes find the counter
// exhausted, paths that start a new step save their state and leave for the
// tail kernels of track_tail.cu, which finish them a warp per path with the
// same arithmetic (add_term, the LU's operation order, lu_solve's order).
//
// The step logic follows the readings documented in include/phc.h; the CPU
// oracle implements the same readings independently.
#pragma once
#include <cstdio>

#include "phc_internal.h"

namespace phc {

extern int g_num_sms, g_smem_optin;
void device_limits();

// ------------------------------------------------------------------ complex arithmetic

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// c - a b
__device__ __forceinline__ double2 cfms(double2 c, double2 a, double2 b)
{
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfms(float2 c, float2 a, float2 b)
{
    return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
// c + a b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c)
{
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
// __dmul_rn: the product is rounded on its own and never merged into a
// following addition, so a scaled derivative rounds the same whether it is
// added at once (one-thread tracker) or stored and added later (tail kernel).
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(__dmul_rn(s, a.x), __dmul_rn(s, a.y)); }
__device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
// a + s b
__device__ __forceinline__ double2 caxpy(double2 a, double s, double2 b)
{
    return make_double2(fma(s, b.x, a.x), fma(s, b.y, a.y));
}
__device__ __forceinline__ double abs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ float abs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__device__ __forceinline__ double absinf(double2 a)
{
    double u = fabs(a.x), v = fabs(a.y);
    return u > v ? u : v;
}
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ double2 recip(double2 p)
{
    const double rd = 1.0 / fma(p.x, p.x, p.y * p.y);
    return make_double2(p.x * rd, -p.y * rd);
}
__device__ __forceinline__ float2 recip(float2 p)
{
    const float rd = 1.0f / fmaf(p.x, p.x, p.y * p.y);
    return make_float2(p.x * rd, -p.y * rd);
}
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 to_f(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_d(float2 a) { return make_double2((double)a.x, (double)a.y); }

template <typename C> struct real_of;
template <> struct real_of<double2> { typedef double type; };
template <> struct real_of<float2> { typedef float type; };

// Strided per-thread slot i of a shared array (stride = threads per block).
// A slot holds a complex double; a complex float lives in its first half.
#define SL(arr, i) (arr)[(i) * bt]

template <typename C> __device__ __forceinline__ C ld(const double2 *a, int i, int bt);
template <> __device__ __forceinline__ double2 ld<double2>(const double2 *a, int i, int bt) { return a[i * bt]; }
template <> __device__ __forceinline__ float2 ld<float2>(const double2 *a, int i, int bt)
{
    return *reinterpret_cast<const float2 *>(a + i * bt);
}
__device__ __forceinline__ void st(double2 *a, int i, int bt, double2 v) { a[i * bt] = v; }
__device__ __forceinline__ void st(double2 *a, int i, int bt, float2 v) { *reinterpret_cast<float2 *>(a + i * bt) = v; }

// ------------------------------------------------------------------ tables in shared memory

struct SmTab {
    int n_terms;
    const TermRec *terms;
    const uint8_t *vars;
    const uint8_t *exps;
    const double2 *c0;  // system 0; system s at + s * n_terms (shared or global memory)
    const double2 *c1;
    const float2 *c0f;
    const float2 *c1f;
};

static __device__ SmTab stage_table(const DevTables &g, char *smem)
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
        s.c0f = g.c0f;
        s.c1f = g.c1f;
        if (g.f32) {
            float2 *c0f = reinterpret_cast<float2 *>(c1 + nc);
            float2 *c1f = c0f + nc;
            for (int i = threadIdx.x; i < nc; i += blockDim.x) {
                c0f[i] = g.c0f[i];
                c1f[i] = g.c1f[i];
            }
            s.c0f = c0f;
            s.c1f = c1f;
        }
    } else {
        s.c0 = g.c0;
        s.c1 = g.c1;
        s.c0f = g.c0f;
        s.c1f = g.c1f;
    }
    __syncthreads();
    s.n_terms = g.n_terms;
    s.terms = terms;
    s.vars = vars;
    s.exps = exps;
    return s;
}

// One warp stages one system's table into its own region (multi-system
// launches: the warps of a block may work on different systems).
static __device__ SmTab stage_table_warp(const DevTables &g, char *region)
{
    const int lane = threadIdx.x & 31;
    SmTab s;
    TermRec *terms = reinterpret_cast<TermRec *>(region);
    uint8_t *vars = reinterpret_cast<uint8_t *>(terms + g.n_terms);
    uint8_t *exps = vars + g.n_ve;
    size_t b = (size_t)g.n_terms * sizeof(TermRec) + 2 * (size_t)g.n_ve;
    b = (b + 15) & ~(size_t)15;
    double2 *c0 = reinterpret_cast<double2 *>(region + b);
    double2 *c1 = c0 + g.n_terms;
    float2 *c0f = reinterpret_cast<float2 *>(c1 + g.n_terms);
    float2 *c1f = c0f + g.n_terms;
    for (int i = lane; i < g.n_terms; i += 32) {
        terms[i] = g.terms[i];
        c0[i] = g.c0[i];
        c1[i] = g.c1[i];
        if (g.f32) {
            c0f[i] = g.c0f[i];
            c1f[i] = g.c1f[i];
        }
    }
    for (int i = lane; i < g.n_ve; i += 32) {
        vars[i] = g.vars[i];
        exps[i] = g.exps[i];
    }
    __syncwarp();
    s.n_terms = g.n_terms;
    s.terms = terms;
    s.vars = vars;
    s.exps = exps;
    s.c0 = c0;
    s.c1 = c1;
    s.c0f = c0f;
    s.c1f = c1f;
    return s;
}

// ------------------------------------------------------------------ evaluation

// One term (support size k >= 1) of an equation, c x^a with coefficient ct
// in the Jacobian and cr in the right-hand side.  Produces, in this order,
//   sink.last(v_{k-1}, d)           d = a_{k-1} P_{k-1}
//   sink.deriv(j, v_j, p_j, s_j)    p_j = a_j P_j, s_j = prod_{i>j} x_{v_i}, j = k-2..0
//   sink.rhs(cr, x^a)
// where P_j = ct cf prod_{i<j} x_{v_i} are the prefix products (kept through
// sink.put_prefix / get_prefix) and cf = prod_j x_{v_j}^{a_j - 1} the common
// factor; the partial derivative d/dx_{v_j} of ct x^a is p_j s_j.  Returns x^a.
// A term whose exponents are all 1 (the TERM_POWERS flag is clear; the flag
// is the same for every lane, so the branch does not diverge) takes a path
// with no common factor and no exponent scaling: written as selects, those
// would cost FP64 multiplications on every term.
// AccumSink adds every piece into the thread's row at once (J += p_j s_j as
// one complex fused multiply-add); the tail kernel's StoreSink keeps the
// pieces and adds them later with the same operations in the same order, so
// both round alike.
template <typename C, typename Sink>
__device__ __forceinline__ C add_term(const TermRec r, const uint8_t *v, const uint8_t *e, C ct, C cr,
                                      const double2 *X, int bt, Sink &sink)
{
    typedef typename real_of<C>::type Real;
    const int k = r.k;
    C mono;
    if (!(r.flags & TERM_POWERS)) {
        C pre = ct;
        if (k > 1) sink.put_prefix(0, pre);
        for (int j = 1; j < k; j++) {
            pre = cmul(pre, ld<C>(X, v[j - 1], bt));
            if (j < k - 1) sink.put_prefix(j, pre);
        }
        C suf = ld<C>(X, v[k - 1], bt);
        sink.last(v[k - 1], pre);
        for (int j = k - 2; j >= 0; j--) {
            sink.deriv(j, v[j], sink.get_prefix(j), suf);
            suf = cmul(suf, ld<C>(X, v[j], bt));
        }
        mono = suf;
    } else {
        C cf = {Real(1), Real(0)};
        for (int j = 0; j < k; j++) {
            const int a = e[j];
            if (a > 1) {
                const C xv = ld<C>(X, v[j], bt);
                C pw = xv;
                for (int m = 2; m < a; m++) pw = cmul(pw, xv);
                cf = cmul(cf, pw);
            }
        }
        C pre = cmul(ct, cf);
        if (k > 1) sink.put_prefix(0, pre);
        for (int j = 1; j < k; j++) {
            pre = cmul(pre, ld<C>(X, v[j - 1], bt));
            if (j < k - 1) sink.put_prefix(j, pre);
        }
        C suf = ld<C>(X, v[k - 1], bt);
        sink.last(v[k - 1], cscale((Real)e[k - 1], pre));
        for (int j = k - 2; j >= 0; j--) {
            sink.deriv(j, v[j], cscale((Real)e[j], sink.get_prefix(j)), suf);
            suf = cmul(suf, ld<C>(X, v[j], bt));
        }
        mono = cmul(cf, suf);
    }
    sink.rhs(cr, mono);
    return mono;
}

// Adds a term's pieces into row Jrow / Rrow of the thread (slot stride bt);
// prefix products in P (shared memory) or, with LP, in the thread's local
// memory (NP entries).
template <typename C, bool LP = false, int NP = 1>
struct AccumSink {
    double2 *Jrow, *Rrow, *P;
    int bt;
    bool want_rhs;
    C pl[LP ? NP : 1];
    __device__ __forceinline__ void put_prefix(int j, C p)
    {
        if constexpr (LP) pl[j] = p;
        else st(P, j, bt, p);
    }
    __device__ __forceinline__ C get_prefix(int j) const
    {
        if constexpr (LP) return pl[j];
        else return ld<C>(P, j, bt);
    }
    __device__ __forceinline__ void last(int col, C d) { st(Jrow, col, bt, cadd(ld<C>(Jrow, col, bt), d)); }
    __device__ __forceinline__ void deriv(int, int col, C pj, C suf)
    {
        st(Jrow, col, bt, cfma(pj, suf, ld<C>(Jrow, col, bt)));
    }
    __device__ __forceinline__ void rhs(C cr, C mono)
    {
        if (want_rhs) st(Rrow, 0, bt, cfma(cr, mono, ld<C>(Rrow, 0, bt)));
    }
};

// One pass over the terms at the thread's point X (slots of complex C):
// J = H_x (row-major N x N) and, when want_rhs, R = H_t (dt) or H (!dt), for
// the homotopy sum_q (c0_q + t c1_q) x^{a_q}.  Each term c(t) x^a with
// support v_0..v_{k-1} is split as
//   x^a = cf * prod_j x_{v_j},  cf = prod_j x_{v_j}^{a_j - 1}   (common factor)
// and its partial derivatives come from prefix and suffix products of the
// x_{v_j} (Speelpenning's product rule):
//   d/dx_{v_j} c(t) x^a = a_j c(t) cf prod_{i<j} x_{v_i} prod_{i>j} x_{v_i}.
// With SCALE, S[i].x accumulates sum over the terms of equation i of
// |c(t)|_1 |x^a|_1 (relative residual and condition number; double only).
template <int N, typename C, bool SCALE, bool LP = false>
__device__ __forceinline__ void evaluate(const C *C0, const C *C1, const SmTab &tb,
                                         typename real_of<C>::type t, bool dt, bool want_rhs, const double2 *X,
                                         double2 *R, double2 *J, double2 *P, double2 *S, int bt)
{
    typedef typename real_of<C>::type Real;
    const C zero = {Real(0), Real(0)};
#pragma unroll
    for (int i = 0; i < N; i++) {
        if (want_rhs) st(R, i, bt, zero);
        if (SCALE) SL(S, i) = make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int i = 0; i < N * N; i++) st(J, i, bt, zero);

    for (int q = 0; q < tb.n_terms; q++) {
        const TermRec r = tb.terms[q];
        const C c0 = C0[q], c1 = C1[q];
        const C ct = {fmar(t, c1.x, c0.x), fmar(t, c1.y, c0.y)};
        const C cr = dt ? c1 : ct;  // coefficient of the right-hand side
        if (r.k == 0) {
            if (want_rhs) st(R, r.eq, bt, cadd(ld<C>(R, r.eq, bt), cr));
            if (SCALE) SL(S, r.eq).x += abs1(ct);
            continue;
        }
        AccumSink<C, LP, N> sink{J + r.eq * N * bt, R + r.eq * bt, P, bt, want_rhs, {}};
        const C mono = add_term<C>(r, tb.vars + r.off, tb.exps + r.off, ct, cr, X, bt, sink);
        if (SCALE) SL(S, r.eq).x += abs1(ct) * abs1(mono);
    }
}

// R = H(X, t) in double, values only (the residual of a Newton correction
// whose Jacobian is factored in single precision).
template <int N>
__device__ __forceinline__ void residual64(const double2 *C0, const double2 *C1, const SmTab &tb, double t,
                                           const double2 *X, double2 *R, int bt)
{
#pragma unroll
    for (int i = 0; i < N; i++) SL(R, i) = make_double2(0.0, 0.0);
    for (int q = 0; q < tb.n_terms; q++) {
        const TermRec r = tb.terms[q];
        const double2 c0 = C0[q], c1 = C1[q];
        double2 m = make_double2(fma(t, c1.x, c0.x), fma(t, c1.y, c0.y));
        const uint8_t *v = tb.vars + r.off;
        const uint8_t *e = tb.exps + r.off;
        for (int j = 0; j < r.k; j++) {
            const double2 xv = SL(X, v[j]);
            for (int a = 0; a < e[j]; a++) m = cmul(m, xv);
        }
        SL(R, r.eq) = cadd(SL(R, r.eq), m);
    }
}

// ------------------------------------------------------------------ linear algebra

// LU with partial pivoting of the thread's N x N matrix in J: the pivot of
// column k is the first row of largest |.|_1; rows are swapped whole (the
// multipliers move with them); the diagonal is replaced by its reciprocal.
// Returns false when a pivot is zero (or not a number).
// A single precision factorization whose pivots spread by more than
// max_ratio counts as failed (the step is retried in double): the spread
// bounds the condition number from below, and a float Jacobian with a
// condition number of 1e4 keeps about three digits.
template <int N, typename C>
__device__ __forceinline__ bool lu_factor(double2 *J, int (&perm)[N], int bt, float max_ratio = 0.0f)
{
    typedef typename real_of<C>::type Real;
    const bool guard = sizeof(Real) == 4;
    Real pmin = Real(0), pmax = Real(0);
#pragma unroll
    for (int k = 0; k < N; k++) {
        int p = k;
        Real best = abs1(ld<C>(J, k * N + k, bt));
#pragma unroll
        for (int i = k + 1; i < N; i++) {
            const Real val = abs1(ld<C>(J, i * N + k, bt));
            if (val > best) {
                best = val;
                p = i;
            }
        }
        perm[k] = p;
        if (!(best > Real(0))) return false;
        if (guard) {
            pmin = (k == 0 || best < pmin) ? best : pmin;
            pmax = (k == 0 || best > pmax) ? best : pmax;
        }
#pragma unroll
        for (int j = 0; j < N; j++) {
            const C a = ld<C>(J, k * N + j, bt), c = ld<C>(J, p * N + j, bt);
            st(J, k * N + j, bt, c);
            st(J, p * N + j, bt, a);
        }
        const C inv = recip(ld<C>(J, k * N + k, bt));
        st(J, k * N + k, bt, inv);
#pragma unroll
        for (int i = k + 1; i < N; i++) {
            const C l = cmul(ld<C>(J, i * N + k, bt), inv);
            st(J, i * N + k, bt, l);
#pragma unroll
            for (int j = k + 1; j < N; j++)
                st(J, i * N + j, bt, cfms(ld<C>(J, i * N + j, bt), l, ld<C>(J, k * N + j, bt)));
        }
    }
    if (guard && pmax > Real(max_ratio) * pmin) return false;
    return true;
}

// b := (LU)^{-1} P b in place (b strided in shared memory).
template <int N, typename C>
__device__ __forceinline__ void lu_solve(const double2 *J, const int (&perm)[N], double2 *b, int bt)
{
#pragma unroll
    for (int k = 0; k < N; k++) {
        const int p = perm[k];
        const C a = ld<C>(b, k, bt), c = ld<C>(b, p, bt);
        st(b, k, bt, c);
        st(b, p, bt, a);
    }
#pragma unroll
    for (int i = 1; i < N; i++) {
        C s = ld<C>(b, i, bt);
#pragma unroll
        for (int j = 0; j < i; j++) s = cfms(s, ld<C>(J, i * N + j, bt), ld<C>(b, j, bt));
        st(b, i, bt, s);
    }
    // back substitution, columns from the last to the first (the order the
    // tail kernels use, so both produce the same rounding)
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
        C s = ld<C>(b, i, bt);
#pragma unroll
        for (int j = N - 1; j > i; j--) s = cfms(s, ld<C>(J, i * N + j, bt), ld<C>(b, j, bt));
        st(b, i, bt, cmul(s, ld<C>(J, i * N + i, bt)));
    }
}

// ------------------------------------------------------------------ tracker

struct ThreadArrays {
    double2 *xe, *R, *P, *X, *J, *S;
};

// The layout of thread_smem_bytes; without f32 there is no X (it aliases R
// or P and is never touched); with LP there is no P (prefix products in
// local memory).
template <int N, bool LP = false>
__device__ __forceinline__ ThreadArrays thread_arrays(char *smem, size_t table_bytes, int bt, bool f32)
{
    ThreadArrays a;
    a.xe = reinterpret_cast<double2 *>(smem + table_bytes) + threadIdx.x;
    a.R = a.xe + N * bt;
    a.P = LP ? nullptr : a.R + N * bt;
    double2 *after = LP ? a.R + N * bt : a.P + N * bt;
    a.X = f32 ? after : a.R;
    a.J = f32 ? after + N * bt : after;
    a.S = a.J + N * N * bt;  // classification only
    return a;
}

// ------------------------------------------------------------------ classification

// Condition number, relative residual and class of the endpoint in A.xe (the
// readings in include/phc.h, identical to the oracle's).  s carries stop, t,
// grew and system in; cond, relres and norm_x (and stop for a non-finite
// endpoint) out.
template <int N, bool LP = false>
__device__ __forceinline__ int8_t classify_one(const SmTab &tb, const ThreadArrays &A, phc_path_stats &s,
                                               const phc_opts &o, int bt)
{
    int perm[N];
    bool fin = true;
    double nx = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) {
        const double2 xj = SL(A.xe, j);
        fin = fin && finite2(xj);
        const double a = absinf(xj);
        if (!(a <= nx)) nx = a;
    }
    int8_t cls = PHC_FAILED;
    double cond = NAN, relres = NAN;
    if (s.stop == PHC_STOP_SKIPPED) return -1;
    if (fin && s.stop != PHC_STOP_DIVERGED) {
        const double2 *C0 = tb.c0 + (size_t)s.system * tb.n_terms, *C1 = tb.c1 + (size_t)s.system * tb.n_terms;
        evaluate<N, double2, true, LP>(C0, C1, tb, 1.0, false, true, A.xe, A.R, A.J, A.P, A.S, bt);
        double rr = 0.0;
#pragma unroll
        for (int i = 0; i < N; i++) {
            const double r = abs1(SL(A.R, i)) / (1.0 + SL(A.S, i).x);
            if (!(r <= rr)) rr = r;
        }
        relres = rr;
        if (!lu_factor<N, double2>(A.J, perm, bt)) {
            cond = INFINITY;
        } else {
            double rowacc[N];
#pragma unroll
            for (int j = 0; j < N; j++) rowacc[j] = 0.0;
#pragma unroll 1
            for (int i = 0; i < N; i++) {
#pragma unroll
                for (int j = 0; j < N; j++) SL(A.R, j) = make_double2(i == j ? 1.0 : 0.0, 0.0);
                lu_solve<N, double2>(A.J, perm, A.R, bt);
                const double si = 1.0 + SL(A.S, i).x;
#pragma unroll
                for (int j = 0; j < N; j++) rowacc[j] += abs1(SL(A.R, j)) * si;
            }
            double m = 0.0;
#pragma unroll
            for (int j = 0; j < N; j++)
                if (!(rowacc[j] <= m)) m = rowacc[j];
            cond = m / (1.0 + nx);
            if (!isfinite(cond)) cond = INFINITY;
        }
    }
    if (!fin) {
        cls = PHC_FAILED;
        s.stop = PHC_STOP_NONFINITE;
        nx = NAN;
    } else if (s.stop == PHC_STOP_DIVERGED) {
        cls = PHC_AT_INFINITY;
        cond = INFINITY;
    } else if (s.stop != PHC_STOP_REACHED) {
        if (nx > o.endpoint_inf_norm || (s.t >= o.end_zone && s.grew)) cls = PHC_AT_INFINITY;
        else if (s.t < o.end_zone) cls = PHC_FAILED;
        else cls = PHC_SINGULAR;
    } else {
        if (nx > o.endpoint_inf_norm) cls = PHC_AT_INFINITY;
        else if (cond <= o.cond_regular && relres <= o.res_regular) cls = PHC_REGULAR;
        else cls = PHC_SINGULAR;
    }
    s.cond = cond;
    s.relres = relres;
    s.norm_x = nx;
    return cls;
}

template <int N>
__global__ void __launch_bounds__(256) classify_kernel(const ClassifyLaunch L, size_t table_bytes)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    const int bt = blockDim.x;
    const ThreadArrays A = thread_arrays<N>(smem, table_bytes, bt, false);
    const int64_t np = L.n_paths, xld = L.x_ld ? L.x_ld : np;
    for (int64_t q = (int64_t)blockIdx.x * bt + threadIdx.x; q < np; q += (int64_t)gridDim.x * bt) {
        phc_path_stats s = L.stats[q];
#pragma unroll
        for (int j = 0; j < N; j++) SL(A.xe, j) = L.x[(int64_t)j * xld + q];
        const int8_t cls = classify_one<N>(tb, A, s, L.o, bt);
        L.stats[q] = s;
        L.cls[q] = cls;
    }
}

// Units between two compaction checks of the single-homotopy tracker (a power of two).
#define COMPACT_EVERY 8
// Shared memory of the compaction bookkeeping: 64 ints and one int16 per thread.
__host__ __device__ inline size_t compact_smem_bytes(int bt) { return 64 * sizeof(int) + (size_t)bt * sizeof(int16_t); }

// Largest ||x|| at which a step may run in single precision (x^d stays far
// from the float range for the degrees the library accepts).
#define FP32_NORM_LIMIT 1.0e4

// MODE 0: one homotopy (or a batch sharing supports); classification by
// classify_kernel.  MODE 1: pipeline (top stage + cascade stage in the same
// thread).  MODE 2: many systems of different structure, one per warp at a
// time.  Modes 1 and 2 classify inline.
enum { MODE_SINGLE = 0, MODE_PIPE = 1, MODE_MULTI = 2 };

// Whether the tracker of this mode and N keeps its prefix products in local memory.
template <int N, int MODE>
__host__ __device__ constexpr bool mode_localp()
{
    return (MODE == MODE_SINGLE && localp_of(N)) || (MODE == MODE_PIPE && localp_pipe_of(N));
}

template <int N, int MODE>
__global__ void __launch_bounds__(256) track_kernel(const TrackLaunch L, size_t table_bytes, size_t table2_bytes)
{
    constexpr bool PIPE = MODE == MODE_PIPE;
    constexpr bool MULTI = MODE == MODE_MULTI;
    // prefix products in local memory for the numbers of unknowns in PHC_LOCALP_MASK
    // (PHC_LOCALP_PIPE_MASK for the pipeline)
    constexpr bool LOCALP = mode_localp<N, MODE>();
    // compaction needs 3N + 11 free slots per thread between units (R, (P), J:
    // N^2 + 2N, with LOCALP N^2 + N)
    constexpr bool COMPACT = MODE == MODE_SINGLE && N >= (LOCALP ? 5 : 4);
    extern __shared__ __align__(16) char smem[];
    SmTab tb{}, tb2{};
    if constexpr (!MULTI) {
        tb = stage_table(L.tab, smem);
        tb2 = tb;
        if constexpr (PIPE) tb2 = stage_table(L.tab2, smem + table_bytes);
    }
    const int bt = blockDim.x;
    const bool f32 = L.o.precision == PHC_PREC_FP32_INTERIOR;
    const ThreadArrays A = thread_arrays<N, LOCALP>(smem, table_bytes + table2_bytes, bt, f32);
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths;
    const bool interior32 = o.precision == PHC_PREC_FP32_INTERIOR;
    int stage = 0;  // pipeline: 0 top homotopy, 1 cascade stage
    const SmTab *cur = &tb;
    // multi-system state (warp-uniform): the warp's system and its table
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    char *wregion = smem + (size_t)(threadIdx.x >> 5) * (size_t)L.warp_table_bytes;
    int ws = 0;
    bool exhausted = true;
    if constexpr (MULTI) {
        // start where this warp's share of all paths begins
        const int64_t nw = (int64_t)gridDim.x * (bt >> 5);
        const int64_t w = (int64_t)blockIdx.x * (bt >> 5) + (threadIdx.x >> 5);
        const int64_t target = w * L.multi_prefix[L.n_multi] / nw;
        int s0 = 0;
        while (s0 + 1 < L.n_multi && L.multi_prefix[s0 + 1] <= target) s0++;
        ws = s0;
        tb = stage_table_warp(L.multi[ws].tab, wregion);
        exhausted = false;
    }

    double2 x0[N], acc[N], sol[N];
    int perm[N];
    int64_t q = -1;
    int sys = 0;
    double t = 0.0, h = 0.0, he = 0.0, t1 = 0.0, te = 0.0, prev = 0.0, next_s = 0.0, nx0 = 0.0;
    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, r4 = 0.0;  // last five decade checkpoints, r4 newest
    int streak = 0, steps = 0, phase = 0, it = 0, nck = 0;
    int since_ck = 0;  // steps since the last decade checkpoint (or the start)
    int n_acc = 0, n_rej = 0, n_newt = 0, n_solve = 0, n_f32 = 0;
    bool use32 = false, fp32_off = false;  // fp32_off: the path fell back to double for good
    bool fresh = false;                    // x0 holds a new start point
    bool counted = false;                  // multi-system: this lane is in idle_n
    const unsigned long long multi_total = MULTI ? (unsigned long long)L.multi_prefix[L.n_multi] : 0ull;
    // multi-system: once every path of every system is claimed, an idle lane
    // stays idle; it counts itself once towards the tail hand-off
    auto count_idle = [&]() {
        if (MULTI && L.drain_at && !counted &&
            *reinterpret_cast<volatile unsigned long long *>(L.multi_claimed) >= multi_total) {
            atomicAdd(L.idle_n, 1ull);
            counted = true;
        }
    };

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
        use32 = interior32 && !fp32_off && t1 <= o.fp32_t_max && nx0 <= FP32_NORM_LIMIT;
    };

    enum { ACT_NONE = 0, ACT_ACCEPT, ACT_REJECT, ACT_END };

    // Compaction (single-homotopy mode).  Once the queue is empty, lanes go
    // idle one by one while the paths left run on; an idle lane still costs
    // its warp's FP64 instructions, so every COMPACT_EVERY units the block
    // moves its running paths to its lowest lanes (their state goes through
    // the owner's evaluation slots, which are free between units), and the
    // warps left without a path stop issuing.  No path's arithmetic changes.
    // Lanes then never leave the loop alone: the block leaves it together
    // once every lane is idle and has found the queue empty.  The checks
    // start once the queue is empty: before that no lane idles, and a block
    // barrier would hold the warps of less loaded SM partitions (a block of
    // 6 warps puts two on each of two partitions, each of which issues one
    // FP64 warp instruction per ~64 cycles) at the pace of the loaded ones.
    // Each thread passes one joining barrier when it first sees the queue
    // empty and counts its iterations from there, so every thread passes the
    // same sequence of barriers.
    const bool compact = COMPACT && L.compact;
    bool joined = false;
    bool done = false;  // (compaction) this lane is idle and counted in idle_n (it found the queue
                        // empty or handed its path off); lanes the compaction empties are counted
                        // too, and a counted lane that receives a path is taken off again, so
                        // idle_n stays the number of idle lanes
    int iter = 0;
    int *cinfo = nullptr;  // [32] warp counts, [32] warp offsets
    int16_t *cmap = nullptr;  // [bt] source lane of each destination
    if constexpr (COMPACT) {
        cinfo = reinterpret_cast<int *>(smem + table_bytes + table2_bytes +
                                        (size_t)bt * thread_smem_bytes(N, false, f32, LOCALP));
        cmap = reinterpret_cast<int16_t *>(cinfo + 64);
    }

    for (;;) {
        if constexpr (COMPACT) {
            if (compact && !joined && *reinterpret_cast<volatile unsigned long long *>(L.qhead) >= (unsigned long long)np) {
                __syncthreads();
                joined = true;
            }
            if (compact && joined && (iter++ & (COMPACT_EVERY - 1)) == 0) {
                // every thread of the block reaches these barriers at the same count of
                // iterations since its joining barrier
                if (__syncthreads_and(q < 0 && done)) break;
                const int live = __syncthreads_count(q >= 0);
                const bool warp_live = __any_sync(FULL, q >= 0);
                const int wl = __syncthreads_count(lane == 0 && warp_live);
                const int settled = __syncthreads_and(q >= 0 || done);
                if (settled && (live + 31) / 32 < wl) {
                    const unsigned bal = __ballot_sync(FULL, q >= 0);
                    const int w = threadIdx.x >> 5, nw = bt >> 5;
                    if (lane == 0) cinfo[w] = __popc(bal);
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        int o2 = 0;
                        for (int k = 0; k < nw; k++) {
                            cinfo[32 + k] = o2;
                            o2 += cinfo[k];
                        }
                    }
                    __syncthreads();
                    // [R, P, (X), J] of a thread are contiguous slots, free between units
                    double2 *base = A.R - threadIdx.x;
                    if (q >= 0) {
                        const int rank = cinfo[32 + w] + __popc(bal & ((1u << lane) - 1u));
                        cmap[rank] = (int16_t)threadIdx.x;
                        double2 *o = base + threadIdx.x;
#pragma unroll
                        for (int j = 0; j < N; j++) {
                            o[j * bt] = x0[j];
                            o[(N + j) * bt] = acc[j];
                            o[(2 * N + j) * bt] = SL(A.xe, j);
                        }
                        double2 *sc = o + 3 * N * bt;
                        sc[0] = make_double2(t, h);
                        sc[bt] = make_double2(he, t1);
                        sc[2 * bt] = make_double2(te, prev);
                        sc[3 * bt] = make_double2(next_s, nx0);
                        sc[4 * bt] = make_double2(r0, r1);
                        sc[5 * bt] = make_double2(r2, r3);
                        sc[6 * bt] = make_double2(r4, __longlong_as_double((long long)q));
                        reinterpret_cast<int4 *>(sc)[7 * bt] = make_int4(sys, phase, it, streak);
                        reinterpret_cast<int4 *>(sc)[8 * bt] = make_int4(steps, nck, since_ck, n_acc);
                        reinterpret_cast<int4 *>(sc)[9 * bt] = make_int4(n_rej, n_newt, n_solve, n_f32);
                        reinterpret_cast<int4 *>(sc)[10 * bt] = make_int4(use32 ? 1 : 0, fp32_off ? 1 : 0, 0, 0);
                    }
                    __syncthreads();
                    if ((int)threadIdx.x < live) {
                        const double2 *o = base + cmap[threadIdx.x];
                        double2 xs[N];
#pragma unroll
                        for (int j = 0; j < N; j++) {
                            x0[j] = o[j * bt];
                            acc[j] = o[(N + j) * bt];
                            xs[j] = o[(2 * N + j) * bt];
                        }
                        const double2 *sc = o + 3 * N * bt;
                        double2 v = sc[0];
                        t = v.x, h = v.y;
                        v = sc[bt];
                        he = v.x, t1 = v.y;
                        v = sc[2 * bt];
                        te = v.x, prev = v.y;
                        v = sc[3 * bt];
                        next_s = v.x, nx0 = v.y;
                        v = sc[4 * bt];
                        r0 = v.x, r1 = v.y;
                        v = sc[5 * bt];
                        r2 = v.x, r3 = v.y;
                        v = sc[6 * bt];
                        r4 = v.x;
                        const int64_t qn = (int64_t)__double_as_longlong(v.y);
                        int4 a = reinterpret_cast<const int4 *>(sc)[7 * bt];
                        sys = a.x, phase = a.y, it = a.z, streak = a.w;
                        a = reinterpret_cast<const int4 *>(sc)[8 * bt];
                        steps = a.x, nck = a.y, since_ck = a.z, n_acc = a.w;
                        a = reinterpret_cast<const int4 *>(sc)[9 * bt];
                        n_rej = a.x, n_newt = a.y, n_solve = a.z, n_f32 = a.w;
                        a = reinterpret_cast<const int4 *>(sc)[10 * bt];
                        use32 = a.x != 0, fp32_off = a.y != 0;
                        q = qn;
                        // a thread's xe slots are not part of the staging area
#pragma unroll
                        for (int j = 0; j < N; j++) SL(A.xe, j) = xs[j];
                        // idle_n counts the idle lanes: this one holds a path again
                        if (done) {
                            done = false;
                            if (L.drain_at) atomicAdd(L.idle_n, ~0ull);
                            __threadfence();
                        }
                    } else {
                        q = -1;
                    }
                    __syncthreads();  // every read done before the next unit writes the slots
                    // lanes emptied by the compaction count as idle, after the decrements
                    if ((int)threadIdx.x >= live && !done) {
                        done = true;
                        if (L.drain_at) atomicAdd(L.idle_n, 1ull);
                    }
                }
            }
        }
        // ---------------------------------------------------------- claim a path
        if constexpr (MULTI) {
            // claim from the warp's system; when every lane of the warp is
            // idle, the warp moves to the next system with unclaimed paths
            if (q < 0 && !exhausted) {
                const SysDesc &d = L.multi[ws];
                const unsigned long long c = atomicAdd(&L.multi_q[ws], 1ull);
                if (c < (unsigned long long)d.n_paths) {
                    if (L.drain_at) atomicAdd(L.multi_claimed, 1ull);
                    q = (int64_t)c;
                    int64_t pid = q;
#pragma unroll
                    for (int i = 0; i < N; i++) {
                        const int dg = d.deg[i];
                        const int k = (int)(pid % dg);
                        pid /= dg;
                        x0[i] = d.roots[d.root_off[i] + k];
                    }
                    sys = 0;
                    fresh = true;
                } else {
                    exhausted = true;
                }
            }
            if (q < 0) count_idle();
            if (__all_sync(FULL, q < 0)) {
                int next = -1;
                if (lane == 0) {
                    for (int k = 1; k <= L.n_multi; k++) {
                        const int cand = (ws + k) % L.n_multi;
                        const unsigned long long used = atomicAdd(&L.multi_q[cand], 0ull);
                        if (used < (unsigned long long)L.multi[cand].n_paths) {
                            next = cand;
                            break;
                        }
                    }
                }
                next = __shfl_sync(FULL, next, 0);
                if (next < 0) {
                    if (L.drain_at && !counted) atomicAdd(L.idle_n, 1ull);
                    break;
                }
                __syncwarp();
                ws = next;
                tb = stage_table_warp(L.multi[ws].tab, wregion);
                exhausted = false;
                continue;
            }
            if (q < 0) continue;
        } else if (q < 0) {
            if (compact && done) continue;  // idle until the block leaves the loop
            const unsigned long long c = atomicAdd(L.qhead, 1ull);
            if (c >= (unsigned long long)np) {
                if (L.drain_at) atomicAdd(L.idle_n, 1ull);
                if (compact) {
                    done = true;
                    continue;
                }
                break;
            }
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
                sys = L.starts_per_system > 0 ? (int)(q / L.starts_per_system) : 0;
                double nx = 0.0;
#pragma unroll
                for (int i = 0; i < N; i++) {
                    x0[i] = L.starts[(int64_t)i * np + q];
                    const double a = absinf(x0[i]);
                    if (!(a <= nx)) nx = a;
                }
                if (L.start_mode == 2) {
                    // a start of this stage: a regular endpoint with z_k != 0
                    bool sel = L.sel_cls[q] == PHC_REGULAR;
                    if (L.sel_sz) sel = sel && L.sel_sz[q] == 0;
                    else sel = sel && absinf(x0[N - 1]) > o.slack_tol * (1.0 + nx);
                    if (!sel) {
                        phc_path_stats rec = {};
                        rec.stop = PHC_STOP_SKIPPED;
                        L.stats[q] = rec;
                        for (int j = 0; j < N; j++) L.x_out[(int64_t)j * np + q] = make_double2(0.0, 0.0);
                        q = -1;
                        continue;
                    }
                }
            }
            if constexpr (PIPE) {
                stage = 0;
                cur = &tb;
            }
            fresh = true;
        }
        if (fresh) {
            // reset the per-path state and start tracking from x0 at t = 0
            fresh = false;
            double nx = 0.0;
#pragma unroll
            for (int i = 0; i < N; i++) {
                const double a = absinf(x0[i]);
                if (!(a <= nx)) nx = a;
            }
            nx0 = nx;
            t = 0.0;
            h = o.h_init;
            streak = steps = 0;
            nck = 0;
            since_ck = 0;
            next_s = 0.1;
            r0 = r1 = r2 = r3 = r4 = 0.0;
            n_acc = n_rej = n_newt = n_solve = n_f32 = 0;
            fp32_off = false;
            begin_step();
        }

        // ---------------------------------------------------------- one unit: evaluate, factor, solve
        const bool dt = phase < 4;
        bool ok;
        if (use32) {
            // single precision Jacobian and factorization; the right-hand side
            // of a Newton correction is the double precision residual
            const float2 *C0f = cur->c0f + (size_t)sys * cur->n_terms, *C1f = cur->c1f + (size_t)sys * cur->n_terms;
#pragma unroll
            for (int j = 0; j < N; j++) st(A.X, j, bt, to_f(SL(A.xe, j)));
            if (!dt) {
                const double2 *C0 = cur->c0 + (size_t)sys * cur->n_terms, *C1 = cur->c1 + (size_t)sys * cur->n_terms;
                residual64<N>(C0, C1, *cur, te, A.xe, A.R, bt);
#pragma unroll
                for (int j = 0; j < N; j++) st(A.R, j, bt, to_f(SL(A.R, j)));
            }
            evaluate<N, float2, false, LOCALP>(C0f, C1f, *cur, (float)te, true, dt, A.X, A.R, A.J, A.P, A.S, bt);
            ok = lu_factor<N, float2>(A.J, perm, bt, (float)o.fp32_pivot_ratio);
            if (ok) lu_solve<N, float2>(A.J, perm, A.R, bt);
#pragma unroll
            for (int j = 0; j < N; j++) sol[j] = to_d(ld<float2>(A.R, j, bt));
            n_f32++;
        } else {
            const double2 *C0 = cur->c0 + (size_t)sys * cur->n_terms, *C1 = cur->c1 + (size_t)sys * cur->n_terms;
            evaluate<N, double2, false, LOCALP>(C0, C1, *cur, te, dt, true, A.xe, A.R, A.J, A.P, A.S, bt);
            ok = lu_factor<N, double2>(A.J, perm, bt);
            if (ok) lu_solve<N, double2>(A.J, perm, A.R, bt);
#pragma unroll
            for (int j = 0; j < N; j++) sol[j] = SL(A.R, j);
        }
        n_solve++;

        // ---------------------------------------------------------- what the unit was for
        int act = ACT_NONE, stop = -1;
        if (phase < 4) {
            // Runge-Kutta stage: k = -J^{-1} H_t
            bool fin = ok;
#pragma unroll
            for (int j = 0; j < N; j++) fin = fin && finite2(sol[j]);
            if (!fin) {
                act = ACT_REJECT;
            } else {
                // stage weights 1, 2, 2, 1; next stage points at t + h/2, t + h/2, t + h
                const double wacc = (phase == 0 || phase == 3) ? 1.0 : 2.0;
                const double hs = (phase < 2) ? 0.5 * he : he;
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double2 kj = make_double2(-sol[j].x, -sol[j].y);
                    acc[j] = (phase == 0) ? kj : caxpy(acc[j], wacc, kj);
                    SL(A.xe, j) = (phase < 3) ? caxpy(x0[j], hs, kj) : caxpy(x0[j], he / 6.0, acc[j]);
                }
                te = (phase < 2) ? t + 0.5 * he : t1;
                if (phase == 3) {
                    it = 0;
                    prev = 0.0;
                }
                phase++;
            }
        } else {
            // Newton correction at t1 (phase 4) or at t = 1 (phase 5)
            n_newt++;
            double d = 0.0, nx = 0.0;
            bool fin = true;
            if (ok) {
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double2 dj = sol[j];
                    const double2 xj = make_double2(SL(A.xe, j).x - dj.x, SL(A.xe, j).y - dj.y);
                    SL(A.xe, j) = xj;
                    if (phase == 5) x0[j] = xj;
                    const double a = absinf(dj);
                    if (!(a <= d)) d = a;
                    const double c = absinf(xj);
                    if (!(c <= nx)) nx = c;
                    fin = fin && finite2(xj);
                }
            }
            if (phase == 4) {
                if (!ok || !(d == d) || !fin) act = ACT_REJECT;
                else if (d <= o.corr_tol * (1.0 + nx)) act = ACT_ACCEPT;
                else if (it > 0 && d > o.corr_contract * prev) act = ACT_REJECT;
                else {
                    prev = d;
                    if (++it >= o.max_corr_iters) act = ACT_REJECT;
                }
            } else {
                if (!ok) stop = PHC_STOP_REACHED;
                else if (!(d == d) || !fin) stop = fin ? PHC_STOP_REACHED : PHC_STOP_NONFINITE;
                else if (d <= o.end_tol * (1.0 + nx) || ++it >= o.end_iters) stop = PHC_STOP_REACHED;
            }
        }

        // ---------------------------------------------------------- step control
        if (act == ACT_ACCEPT) {
            t = t1;
            double nx = 0.0;
#pragma unroll
            for (int j = 0; j < N; j++) {
                x0[j] = SL(A.xe, j);
                const double a = absinf(x0[j]);
                if (!(a <= nx)) nx = a;
            }
            nx0 = nx;
            n_acc++;
            steps++;
            while (1.0 - t <= next_s && next_s > 0.0) {
                r0 = r1;
                r1 = r2;
                r2 = r3;
                r3 = r4;
                r4 = nx;
                nck++;
                since_ck = 0;
                next_s *= 0.1;
                if (nck >= 40) next_s = 0.0;
            }
            if (nx > o.diverge_norm) {
                stop = PHC_STOP_DIVERGED;
            } else {
                if (++streak >= o.expand_after) {
                    streak = 0;
                    h = h * o.expand;
                    if (h > o.h_max) h = o.h_max;
                }
                if (steps >= o.max_steps) stop = PHC_STOP_BUDGET;
                else if (++since_ck >= o.max_steps_decade && t < 1.0) stop = PHC_STOP_BUDGET;
                else if (t >= 1.0) {
                    phase = 5;  // end Newton at t = 1 from x0 (already in xe)
                    it = 0;
                    te = 1.0;
                    use32 = false;
                } else {
                    begin_step();
                }
            }
        } else if (act == ACT_REJECT) {
            n_rej++;
            steps++;
            streak = 0;
            if (use32) {
                // a single precision step that failed is retried in double,
                // and the rest of the path stays in double
                fp32_off = true;
            } else {
                h = he * o.shrink;
                if (h < o.h_min) stop = PHC_STOP_STEP_MIN;
            }
            if (stop < 0 && steps >= o.max_steps) stop = PHC_STOP_BUDGET;
            if (stop < 0 && ++since_ck >= o.max_steps_decade) stop = PHC_STOP_BUDGET;
            if (stop < 0) begin_step();
        }
        {
            // most lanes are idle: a path that starts a new step moves to
            // the tail kernel (which repeats this arithmetic exactly, so
            // where a path is finished does not change it)
            // (FP32 interior: only a path whose remaining steps are all double
            // precision -- t already at fp32_t_max, so every later step ends
            // beyond it even after rejections, or fallen back for good --
            // since the tail kernel computes in double only)
            if (stop < 0 && act != ACT_NONE && phase == 0 && L.drain_at &&
                (!interior32 || fp32_off || t >= o.fp32_t_max) &&
                *reinterpret_cast<volatile unsigned long long *>(L.idle_n) >= L.drain_at) {
                Handoff &hd = L.handoff[atomicAdd(L.handoff_n, 1ull)];
                for (int j = 0; j < N; j++) hd.x0[j] = x0[j];
                hd.t = t;
                hd.h = h;
                hd.next_s = next_s;
                hd.nx0 = nx0;
                hd.r0 = r0;
                hd.r1 = r1;
                hd.r2 = r2;
                hd.r3 = r3;
                hd.r4 = r4;
                hd.q = q;
                hd.sys = MULTI ? ws : sys;
                hd.streak = streak;
                hd.steps = steps;
                hd.since_ck = since_ck;
                hd.nck = nck;
                hd.n_acc = n_acc;
                hd.n_rej = n_rej;
                hd.n_newt = n_newt;
                hd.n_solve = n_solve;
                hd.n_f32 = n_f32;
                hd.stage = stage;
                if constexpr (MULTI) {
                    // the lane stays in the warp's claim loop, idle
                    q = -1;
                    if (!counted) {
                        atomicAdd(L.idle_n, 1ull);
                        counted = true;
                    }
                    continue;
                } else {
                    if (compact) {
                        q = -1;
                        done = true;
                        continue;
                    }
                    break;
                }
            }
        }
        if (stop < 0) continue;

        // ---------------------------------------------------------- the path ends
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
        phc_path_stats rec;
        rec.t = t;
        rec.h = h;
        rec.cond = 0.0;
        rec.relres = 0.0;
        rec.norm_x = 0.0;
        rec.growth = growth;
        rec.n_accept = n_acc;
        rec.n_reject = n_rej;
        rec.n_newton = n_newt;
        rec.n_solve = n_solve;
        rec.stop = stop;
        rec.n_fp32 = n_f32;
        rec.grew = grew;
        rec.system = sys;
        if constexpr (!PIPE && !MULTI) {
            for (int j = 0; j < N; j++) L.x_out[(int64_t)j * np + q] = x0[j];
            L.stats[q] = rec;
            q = -1;
            continue;
        } else {
        // modes 1 and 2 classify here
#pragma unroll
        for (int j = 0; j < N; j++) SL(A.xe, j) = x0[j];
        const int8_t c = classify_one<N, LOCALP>(*cur, A, rec, o, bt);
        if constexpr (MULTI) {
            const SysDesc &d = L.multi[ws];
            for (int j = 0; j < N; j++) d.x_out[(int64_t)j * d.n_paths + q] = x0[j];
            rec.system = ws;
            d.stats[q] = rec;
            d.cls_out[q] = c;
        } else if (stage == 0) {
            for (int j = 0; j < N; j++) L.x_out[(int64_t)j * np + q] = x0[j];
            L.stats[q] = rec;
            L.cls_out[q] = c;
            // continue regular endpoints with z_k != 0 on the cascade stage
            if (c == PHC_REGULAR && absinf(x0[N - 1]) > o.slack_tol * (1.0 + rec.norm_x)) {
                stage = 1;
                cur = &tb2;
                sys = 0;
                fresh = true;
                continue;
            }
            L.cls_out2[q] = -1;
        } else {
            double nx = 0.0;
            for (int j = 0; j < N - 1; j++) {
                L.x_out2[(int64_t)j * np + q] = x0[j];
                const double a = absinf(x0[j]);
                if (!(a <= nx)) nx = a;
            }
            L.stats2[q] = rec;
            L.cls_out2[q] = c;
            L.slack_zero2[q] = L.has_next_slack ? (absinf(x0[N - 2]) <= o.slack_tol * (1.0 + nx)) : 0;
        }
        q = -1;
        }
    }
}

// ------------------------------------------------------------------ launch helper

// Lanes (grid x block) launch_track_n launches in mode MODE for L (with
// block size bt): the same shared memory and grid arithmetic.
template <int N, int MODE>
static int64_t lanes_n(const TrackLaunch &L, int bt, int max_blocks)
{
    const bool f32 = L.o.precision == PHC_PREC_FP32_INTERIOR;
    const size_t tb = MODE == MODE_MULTI  ? (size_t)(bt / 32) * (size_t)L.warp_table_bytes
                      : MODE == MODE_PIPE ? table_smem_bytes(L.tab) + table_smem_bytes(L.tab2)
                                          : table_smem_bytes(L.tab);
    const size_t smem = tb + (size_t)bt * thread_smem_bytes(N, MODE != MODE_SINGLE, f32, mode_localp<N, MODE>()) +
                        (MODE == MODE_SINGLE ? compact_smem_bytes(bt) : 0);
    if (cudaFuncSetAttribute(track_kernel<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_kernel<N, MODE>, bt, smem) != cudaSuccess)
        return -1;
    int64_t want = (L.n_paths + bt - 1) / bt;
    int64_t grid = (int64_t)g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    return grid * bt;
}

template <int N, int MODE>
static cudaError_t launch_track_n(const TrackLaunch &L_in, int bt, int max_blocks, int64_t work, cudaStream_t s)
{
    TrackLaunch L = L_in;
    size_t tb, tb2 = 0;
    if (MODE == MODE_MULTI) {
        tb = (size_t)(bt / 32) * (size_t)L.warp_table_bytes;
    } else {
        tb = table_smem_bytes(L.tab);
        if (MODE == MODE_PIPE) tb2 = table_smem_bytes(L.tab2);
    }
    const size_t smem =
        tb + tb2 +
        (size_t)bt * thread_smem_bytes(N, MODE != MODE_SINGLE, L.o.precision == PHC_PREC_FP32_INTERIOR,
                                       mode_localp<N, MODE>()) +
        (MODE == MODE_SINGLE ? compact_smem_bytes(bt) : 0);
    cudaError_t e =
        cudaFuncSetAttribute(track_kernel<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_kernel<N, MODE>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t want = (work + bt - 1) / bt;
    int64_t grid = (int64_t)g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    L.drain_at = 0;
    if (L.drain_frac > 0.0 && L.handoff) {
        const int64_t lanes = grid * bt;
        unsigned long long at = (unsigned long long)(L.drain_frac * (double)lanes);
        // a lane that finds the queue empty stays idle, so when idle_n >= at at most
        // lanes - at lanes hold a path, and each writes at most one record
        if (L.handoff_cap > 0 && lanes - L.handoff_cap > (int64_t)at) at = (unsigned long long)(lanes - L.handoff_cap);
        L.drain_at = at < 1 ? 1 : at;
    }
    track_kernel<N, MODE><<<(unsigned)grid, bt, smem, s>>>(L, tb, tb2);
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

}  // namespace phc
