// refine.cu -- Newton's method at t = 1 in complex double double arithmetic.
//
// Double double numbers are unevaluated sums hi + lo with |lo| <= ulp(hi)/2
// (Hida, Li and Bailey, the paper's [HLB00]; the paper's "phc -B2" runs its
// whole solver in this arithmetic, Section 5).  Here only ill-conditioned
// endpoints are refined: a regular root converges quadratically to about
// 1e-30, a singular one only linearly, which separates the two.
//
// Error-free transforms: Knuth's TwoSum and the fused multiply-add form of
// TwoProduct (a*b - fl(a*b) is exact as fma(a, b, -fl(a*b))).
#include "dd.cuh"

namespace phc {

// Table reads go through the read-only path (few endpoints are refined).
template <int N>
__device__ void eval_dd(const DevTables &tab, int sys, const cdd *x, cdd *H, cdd *J)
{
    const size_t cof = (size_t)sys * tab.n_terms;
    const cdd zero = {{0.0, 0.0}, {0.0, 0.0}};
    for (int i = 0; i < N; i++) H[i] = zero;
    for (int i = 0; i < N * N; i++) J[i] = zero;
    for (int q = 0; q < tab.n_terms; q++) {
        const TermRec r = tab.terms[q];
        const double2 c0 = __ldg(&tab.c0[cof + q]), c1 = __ldg(&tab.c1[cof + q]);
        // coefficient at t = 1 (exact: the pairs are (0,c), (g,-g), (c,0), (c,-c))
        const double2 c = make_double2(c0.x + c1.x, c0.y + c1.y);
        if (c.x == 0.0 && c.y == 0.0) continue;
        const cdd cc = cdd_from(c);
        const int k = r.k;
        const uint8_t *v = tab.vars + r.off;
        const uint8_t *e = tab.exps + r.off;
        // value c x^a
        cdd m = cc;
        for (int j = 0; j < k; j++)
            for (int a = 0; a < e[j]; a++) m = cdd_mul(m, x[v[j]]);
        H[r.eq] = cdd_add(H[r.eq], m);
        // derivatives c a_j x_j^{a_j-1} prod_{i != j} x_i^{a_i}, from scratch
        for (int j = 0; j < k; j++) {
            cdd d = cdd_mul(cc, cdd_from(make_double2((double)e[j], 0.0)));
            for (int i = 0; i < k; i++) {
                const int a = (i == j) ? e[i] - 1 : e[i];
                for (int b = 0; b < a; b++) d = cdd_mul(d, x[v[i]]);
            }
            J[r.eq * N + v[j]] = cdd_add(J[r.eq * N + v[j]], d);
        }
    }
}

// Solve J d = H in place (H := d); partial pivoting on |hi|_1.
template <int N>
__device__ bool solve_dd(cdd *J, cdd *b)
{
    for (int k = 0; k < N; k++) {
        int p = k;
        double best = cdd_abs1(J[k * N + k]);
        for (int i = k + 1; i < N; i++) {
            const double val = cdd_abs1(J[i * N + k]);
            if (val > best) {
                best = val;
                p = i;
            }
        }
        if (!(best > 0.0)) return false;
        if (p != k) {
            for (int j = 0; j < N; j++) {
                const cdd s = J[k * N + j];
                J[k * N + j] = J[p * N + j];
                J[p * N + j] = s;
            }
            const cdd s = b[k];
            b[k] = b[p];
            b[p] = s;
        }
        for (int i = k + 1; i < N; i++) {
            const cdd l = cdd_div(J[i * N + k], J[k * N + k]);
            for (int j = k + 1; j < N; j++) J[i * N + j] = cdd_sub(J[i * N + j], cdd_mul(l, J[k * N + j]));
            b[i] = cdd_sub(b[i], cdd_mul(l, b[k]));
        }
    }
    for (int i = N - 1; i >= 0; i--) {
        for (int j = i + 1; j < N; j++) b[i] = cdd_sub(b[i], cdd_mul(J[i * N + j], b[j]));
        b[i] = cdd_div(b[i], J[i * N + i]);
    }
    return true;
}

// Root condition number at the double point x (same definition as the
// classification: max_j sum_i |(J^-1)_ji|_1 (1 + scale_i) / (1 + ||x||)),
// computed here in double double for simplicity.
template <int N>
__device__ double cond_at(const DevTables &tab, int sys, const double2 *x2)
{
    const size_t cof = (size_t)sys * tab.n_terms;
    cdd x[N], H[N], J[N * N], col[N];
    double scale[N];
    for (int j = 0; j < N; j++) x[j] = cdd_from(x2[j]);
    for (int i = 0; i < N; i++) scale[i] = 0.0;
    // scale_i from a plain double evaluation of the monomials
    for (int q = 0; q < tab.n_terms; q++) {
        const TermRec r = tab.terms[q];
        const double2 c0 = __ldg(&tab.c0[cof + q]), c1 = __ldg(&tab.c1[cof + q]);
        const double2 c = make_double2(c0.x + c1.x, c0.y + c1.y);
        double2 mono = make_double2(1.0, 0.0);
        for (int j = 0; j < r.k; j++) {
            const double2 xv = x2[tab.vars[r.off + j]];
            for (int a = 0; a < tab.exps[r.off + j]; a++)
                mono = make_double2(mono.x * xv.x - mono.y * xv.y, mono.x * xv.y + mono.y * xv.x);
        }
        scale[r.eq] += (fabs(c.x) + fabs(c.y)) * (fabs(mono.x) + fabs(mono.y));
    }
    eval_dd<N>(tab, sys, x, H, J);
    // one full solve per unit vector (N <= 12; only refined endpoints get here)
    double rowacc[N];
    for (int j = 0; j < N; j++) rowacc[j] = 0.0;
    cdd Jc[N * N];
    for (int i = 0; i < N; i++) {
        for (int a = 0; a < N * N; a++) Jc[a] = J[a];
        for (int j = 0; j < N; j++) col[j] = cdd_from(make_double2(i == j ? 1.0 : 0.0, 0.0));
        if (!solve_dd<N>(Jc, col)) return INFINITY;
        for (int j = 0; j < N; j++) rowacc[j] += cdd_abs1(col[j]) * (1.0 + scale[i]);
    }
    double m = 0.0, nx = 0.0;
    for (int j = 0; j < N; j++) {
        if (!(rowacc[j] <= m)) m = rowacc[j];
        const double u = fabs(x2[j].x), v = fabs(x2[j].y);
        const double a = u > v ? u : v;
        if (a > nx) nx = a;
    }
    const double c = m / (1.0 + nx);
    return isfinite(c) ? c : INFINITY;
}

template <int N>
__global__ void refine_kernel(const RefineLaunch L)
{
    const int64_t n = L.n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < N; j++) L.x_lo[(int64_t)j * n + q] = make_double2(0.0, 0.0);
        phc_path_stats s = L.stats[q];
        const int8_t c0 = L.cls[q];
        if (!(s.stop == PHC_STOP_REACHED && (c0 == PHC_SINGULAR || c0 == PHC_REGULAR) && s.cond > L.cond_threshold))
            continue;
        cdd x[N], H[N], J[N * N];
        for (int j = 0; j < N; j++) x[j] = cdd_from(L.x_hi[(int64_t)j * n + q]);
        bool conv = false;
        for (int it = 0; it < L.max_iters; it++) {
            eval_dd<N>(L.tab, s.system, x, H, J);
            if (!solve_dd<N>(J, H)) break;
            double dn = 0.0, xn = 0.0;
            for (int j = 0; j < N; j++) {
                x[j] = cdd_sub(x[j], H[j]);
                const double a = cdd_absinf(H[j]);
                if (!(a <= dn)) dn = a;
                const double b = cdd_absinf(x[j]);
                if (b > xn) xn = b;
            }
            if (!(dn == dn)) break;
            if (dn <= 1e-20 * (1.0 + xn)) {
                conv = true;
                break;
            }
        }
        double2 xh[N];
        for (int j = 0; j < N; j++) {
            xh[j] = make_double2(x[j].re.hi, x[j].im.hi);
            L.x_hi[(int64_t)j * n + q] = xh[j];
            L.x_lo[(int64_t)j * n + q] = make_double2(x[j].re.lo, x[j].im.lo);
        }
        const double c = cond_at<N>(L.tab, s.system, xh);
        s.cond = c;
        L.stats[q] = s;
        L.cls[q] = (conv && c <= L.cond_max) ? PHC_REGULAR : PHC_SINGULAR;
    }
}

template <int N>
static cudaError_t launch_refine_n(const RefineLaunch &L, cudaStream_t s)
{
    int64_t grid = (L.n + 127) / 128;
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    refine_kernel<N><<<(unsigned)grid, 128, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_refine(const RefineLaunch &L, cudaStream_t s)
{
    if (L.n <= 0) return cudaSuccess;
    switch (L.tab.n) {
    case 1: return launch_refine_n<1>(L, s);
    case 2: return launch_refine_n<2>(L, s);
    case 3: return launch_refine_n<3>(L, s);
    case 4: return launch_refine_n<4>(L, s);
    case 5: return launch_refine_n<5>(L, s);
    case 6: return launch_refine_n<6>(L, s);
    case 7: return launch_refine_n<7>(L, s);
    case 8: return launch_refine_n<8>(L, s);
    case 9: return launch_refine_n<9>(L, s);
    case 10: return launch_refine_n<10>(L, s);
    case 11: return launch_refine_n<11>(L, s);
    case 12: return launch_refine_n<12>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace phc
